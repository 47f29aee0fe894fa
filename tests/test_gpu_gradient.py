"""Gradient of Theta in (A, omega, tau_s) by central differences over seven
solvers stepped as one sweep (hlbm_theta_gradient), against the same
quotient from seven oracle runs."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13631_gb300.build import build

    build()


def test_theta_gradient_matches_oracle_fd():
    from paper_2006_13631_gb300 import hlbm_theta_gradient, use_torch_allocator, workload_inputs

    use_torch_allocator()
    w = inputs.workload("lamina-256-f64")
    mesh, rho = w.mesh(), w.rho_init()
    grid, patch, motion = workload_inputs(w, mesh, rho)
    th, grad, ms = hlbm_theta_gradient(grid, patch, w.tau_s, motion, 48, discard=0.5, fit=1.5, rel_step=1e-4)
    tho, grado = oracle.theta_fd_gradient(w, 48, discard=0.5, fit=1.5, rel_step=1e-4, mesh=mesh, rho_init=rho)
    print("theta", th, tho, "grad", grad, grado, "ms", ms)
    assert abs(th - tho) < 1e-8
    scale = np.abs(grado).max()
    assert np.abs(grad - grado).max() < 1e-4 * scale
    assert ms > 0


def test_theta_gradient_rejects_bad_arguments():
    from paper_2006_13631_gb300 import HLBMError, hlbm_theta_gradient, workload_inputs

    w = inputs.workload("lamina-256-f64")
    grid, patch, motion = workload_inputs(w)
    with pytest.raises(HLBMError):
        hlbm_theta_gradient(grid, patch, w.tau_s, motion, 48, rel_step=0.5)
    motion["kind"] = inputs.MOTION_STATIC
    with pytest.raises(HLBMError):
        hlbm_theta_gradient(grid, patch, w.tau_s, motion, 48)

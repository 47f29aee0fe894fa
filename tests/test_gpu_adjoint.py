"""Adjoint of the discrete hybrid step (hlbm_theta_adjoint): the gradient of
Theta in (A, omega, tau_s) against central differences of the CUDA path,
against the oracle's FP64 tangent along its branch of decisions, independent
of the checkpoint interval, and behind a torch.autograd.Function.

The base point is the 256^2, chord-20, FP64 lamina at omega 1.31 % above
pi/12: at omega = pi/12 itself the lamina's positions y(t) = A sin(w t) hit
decisions exactly (a node class changes within 1e-7 of omega), so any
finite-difference quotient there measures that jump rather than the
derivative.
"""
import math

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEPS, DISCARD, FIT = 48, 0.5, 1.5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13631_gb300.build import build
    from paper_2006_13631_gb300 import use_torch_allocator

    build()
    use_torch_allocator()


def _case(dtype="f64"):
    w = inputs.workload("lamina-256-f64")
    w.omega *= 1.0131
    w.dtype = dtype
    return w


@pytest.fixture(scope="module")
def adjoint():
    """Gradient of Re Theta and of Im Theta (two reverse sweeps)."""
    from paper_2006_13631_gb300 import hlbm_theta_adjoint, workload_inputs

    w = _case()
    mesh, rho = w.mesh(), w.rho_init()
    grid, patch, motion = workload_inputs(w, mesh, rho)
    th, g_re, fw, bw = hlbm_theta_adjoint(grid, patch, w.tau_s, motion, STEPS, DISCARD, FIT, 1.0, 0.0, 256)
    th2, g_im, _, _ = hlbm_theta_adjoint(grid, patch, w.tau_s, motion, STEPS, DISCARD, FIT, 0.0, 1.0, 256)
    assert th == th2 and fw > 0 and bw > 0
    return w, mesh, rho, th, g_re + 1j * g_im


def test_adjoint_matches_central_differences_of_the_cuda_path(adjoint):
    from paper_2006_13631_gb300 import hlbm_theta_gradient, workload_inputs

    w, mesh, rho, th, g = adjoint
    grid, patch, motion = workload_inputs(w, mesh, rho)
    th_fd, g_fd, _ = hlbm_theta_gradient(grid, patch, w.tau_s, motion, STEPS, DISCARD, FIT, rel_step=1e-6)
    print("adjoint", g, "central differences", g_fd)
    assert abs(th - th_fd) < 1e-12
    scale = np.abs(g_fd).max()
    assert np.abs(g - g_fd).max() < 1e-5 * scale


def test_adjoint_matches_oracle_fp64_tangent(adjoint):
    w, mesh, rho, th, g = adjoint
    g_o, ties = oracle.theta_tangent(w, STEPS, DISCARD, FIT, rel_step=1e-6, mesh=mesh, rho_init=rho)
    print("adjoint", g, "oracle tangent", g_o, "donor ties", ties)
    scale = np.abs(g_o).max()
    assert np.abs(g - g_o).max() < 1e-5 * scale


def test_adjoint_independent_of_checkpoint_interval(adjoint):
    from paper_2006_13631_gb300 import hlbm_theta_adjoint, workload_inputs

    w, mesh, rho, th, g = adjoint
    grid, patch, motion = workload_inputs(w, mesh, rho)
    for every in (5, 13, 48):
        _, g_re, _, _ = hlbm_theta_adjoint(grid, patch, w.tau_s, motion, STEPS, DISCARD, FIT, 1.0, 0.0, every)
        assert np.abs(g_re - g.real).max() < 1e-10 * np.abs(g.real).max(), every


def test_autograd_function_gives_the_adjoint_gradient(adjoint):
    from paper_2006_13631_gb300 import theta_function

    w, mesh, rho, th, g = adjoint
    f = theta_function(w, STEPS, DISCARD, FIT, checkpoint_every=16, mesh=mesh, rho_init=rho)
    p = torch.tensor([w.A, w.omega, w.tau_s], dtype=torch.float64, requires_grad=True)
    out = f(p)
    assert out[0].item() == pytest.approx(th.real, abs=1e-13) and out[1].item() == pytest.approx(th.imag, abs=1e-13)
    c = torch.tensor([0.7, -1.3], dtype=torch.float64)
    (out * c).sum().backward()
    expect = 0.7 * g.real - 1.3 * g.imag
    assert np.abs(p.grad.numpy() - expect).max() < 1e-9 * np.abs(expect).max()


def test_fp32_adjoint_close_to_fp64(adjoint):
    from paper_2006_13631_gb300 import hlbm_theta_adjoint, workload_inputs

    w, mesh, rho, th, g = adjoint
    w32 = _case("f32")
    grid, patch, motion = workload_inputs(w32, mesh, rho)
    th32, g_re, _, _ = hlbm_theta_adjoint(grid, patch, w32.tau_s, motion, STEPS, DISCARD, FIT, 1.0, 0.0, 256)
    assert abs(th32 - th) < 1e-4 * abs(th)
    assert np.abs(g_re - g.real).max() < 1e-3 * np.abs(g.real).max()


def test_adjoint_rejects_what_it_does_not_cover():
    from paper_2006_13631_gb300 import HLBMError, hlbm_theta_adjoint, workload_inputs

    w = _case()
    grid, patch, motion = workload_inputs(w)
    with pytest.raises(HLBMError):
        hlbm_theta_adjoint(grid, patch, w.tau_s, motion, STEPS, DISCARD, FIT, 1.0, 0.0, 0)
    patch["outer_fv"] = 1
    with pytest.raises(HLBMError):
        hlbm_theta_adjoint(grid, patch, w.tau_s, motion, STEPS, DISCARD, FIT, 1.0, 0.0, 16)
    patch["outer_fv"] = 0
    motion["kind"] = inputs.MOTION_STATIC
    with pytest.raises(HLBMError):
        hlbm_theta_adjoint(grid, patch, w.tau_s, motion, STEPS, DISCARD, FIT, 1.0, 0.0, 16)


@pytest.mark.slow
def test_adjoint_matches_oracle_tangent_over_eight_periods():
    """A longer window: 200 steps (8.4 periods, the fit over all but the
    first half period).  The oracle's FP64 tangent still has one branch of
    decisions over the whole run (its lockstep runs at -/+ 1e-6 take the same
    classes and refill types), and the adjoint equals it in A, omega and
    tau_s; measured to 8-10 digits."""
    from paper_2006_13631_gb300 import hlbm_theta_adjoint, workload_inputs

    w = _case()
    mesh, rho = w.mesh(), w.rho_init()
    steps, discard = 200, 0.5
    fit = (steps - 1) * w.omega / (2.0 * math.pi) - discard
    grid, patch, motion = workload_inputs(w, mesh, rho)
    _, g_re, _, _ = hlbm_theta_adjoint(grid, patch, w.tau_s, motion, steps, discard, fit, 1.0, 0.0, 64)
    _, g_im, _, _ = hlbm_theta_adjoint(grid, patch, w.tau_s, motion, steps, discard, fit, 0.0, 1.0, 64)
    tangent, _ = oracle.theta_tangent(w, steps, discard, fit, mesh=mesh, rho_init=rho)
    t_re = np.array([g.real for g in tangent])
    t_im = np.array([g.imag for g in tangent])
    assert np.abs(np.asarray(g_re) - t_re).max() < 1e-6 * np.abs(t_re).max()
    assert np.abs(np.asarray(g_im) - t_im).max() < 1e-6 * np.abs(t_im).max()

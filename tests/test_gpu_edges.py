"""Error paths and degenerate cases of the C ABI on a GPU: each is refused on
the host with its code and a message, and the solver stays usable."""
import math

import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13631_gb300.build import build

    build()


def test_forced_fv_kernel_that_cannot_run_is_refused():
    from paper_2006_13631_gb300 import HLBMError, Solver

    w = inputs.workload("lamina-small-f32")
    w.outer_fv, w.fv_kernel = 1, 3  # the tensor-memory kernel has no outer-node FV sums
    with pytest.raises(HLBMError) as e:
        Solver(w)
    assert e.value.code == -1 and "FV kernel" in str(e.value)
    w.fv_kernel = 9
    with pytest.raises(HLBMError) as e:
        Solver(w)
    assert e.value.code == -1


def test_degenerate_triangle_is_refused():
    from paper_2006_13631_gb300 import HLBMError, Solver

    w = inputs.workload("lamina-small-f32")
    m = w.mesh()
    tri = m.tri.copy()
    tri[5] = [tri[5][0], tri[5][0], tri[5][1]]
    m2 = inputs.PatchMesh(m.xy, tri, m.kind, m.layer)
    with pytest.raises(HLBMError) as e:
        Solver(w, mesh=m2)
    assert e.value.code == -1


def test_zero_steps_change_nothing():
    from paper_2006_13631_gb300 import Solver

    w = inputs.workload("lamina-small-f32")
    s = Solver(w)
    s.step(3)
    a = s.fields()
    s.step(0)
    b = s.fields()
    assert s.info()["time"] == 3
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_patch_leaving_the_lattice_stops_the_run_cleanly():
    """A translating lamina that reaches the lattice edge: hlbm_step refuses
    the step that would take the patch window off the lattice; the steps
    before it stand and the solver can still be read."""
    from paper_2006_13631_gb300 import HLBMError, Solver

    w = inputs.Workload("edge-run", 64, 60, 12.0, 0.24, 30.3, 28.2, 0.7, 10, inputs.MOTION_UNIFORM,
                        vx=0.2, vy=0.0, delta_f=1.8, bc_x=inputs.BC_PERIODIC, bc_y=inputs.BC_PERIODIC,
                        u0x=0.2, dtype="f32", mesh_args=dict(n_L=24, n_T=1, n_layers=8, h1=0.6, d_out=3.6))
    s = Solver(w)
    with pytest.raises(HLBMError) as e:
        s.step(200)
    assert e.value.code == -1 and "leaves the lattice" in str(e.value)
    t = s.info()["time"]
    assert 0 < t < 200
    fx, fy = s.force()
    assert len(fy) == t + 1 and np.isfinite(fy).all()


def test_induced_motion_too_fast_is_refused():
    from paper_2006_13631_gb300 import HLBMError, Solver

    w = inputs.workload("lamina-small-f32")
    w.motion, w.A, w.omega = inputs.MOTION_INDUCED, 0.0, 0.0
    w.mass = 1.0
    w.stiffness = 0.5  # a light, stiff spring: the first swing exceeds what the patch allows
    w.y0 = 1.5
    s = Solver(w)
    with pytest.raises(HLBMError) as e:
        s.step(10)
    assert e.value.code == -1 and "velocity" in str(e.value)
    assert s.info()["time"] < 10


def test_checkpoint_of_another_precision_is_refused(tmp_path):
    from paper_2006_13631_gb300 import HLBMError, Solver

    w = inputs.workload("lamina-small-f32")
    mesh, rho = w.mesh(), w.rho_init()
    a = Solver(w, mesh=mesh, rho_init=rho)
    a.step(2)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    w.dtype = "f64"
    b = Solver(w, mesh=mesh, rho_init=rho)
    with pytest.raises(HLBMError) as e:
        b.load(path)
    assert e.value.code == -1
    b.step(1)  # still usable
    assert b.info()["time"] == 1

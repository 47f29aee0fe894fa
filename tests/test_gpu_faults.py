"""Failure detection on the GPU, in forms that fault, trap or hang nothing.

The method's only failure mode is instability of the explicit schemes
(Sec. 7 bounds the FV time step); the GPU path adds the bounded neighbour
waits of its persistent FV kernels.  Both are injected from the host:
  - a tile that never releases its progress counter (hlbm_inject_fault,
    with a short wait limit): its neighbours give up, set the status bit and
    the abort flag, every tile returns, and the error reaches the caller as
    HLBM_ETIMEOUT while the GPU stays usable;
  - NaN copied into lattice populations near the patch: it reaches the
    lamina force, and the caller sees HLBM_EUNSTABLE.
Once the host has seen a status bit, hlbm_step refuses to go on until the
caller clears it or restores a checkpoint.
"""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ETIMEOUT, EUNSTABLE = -7, -3
ST_SYNC_TIMEOUT, ST_NONFINITE = 32, 8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13631_gb300.build import build

    build()


@pytest.mark.parametrize("dtype,fv_kernel", [("f32", 4), ("f32", 3), ("f32", 2), ("f32", 1), ("f64", 4)])
def test_stalled_tile_times_out_and_the_solver_recovers(tmp_path, dtype, fv_kernel):
    from paper_2006_13631_gb300 import HLBMError, Solver, hlbm_clear_status, hlbm_inject_fault

    w = inputs.workload("lamina-small-f32")
    w.dtype, w.fv_kernel = dtype, fv_kernel
    mesh, rho = w.mesh(), w.rho_init()
    s = Solver(w, mesh=mesh, rho_init=rho)
    ref = Solver(w, mesh=mesh, rho_init=rho)
    s.step(3)
    ck = str(tmp_path / "before.bin")
    s.save(ck)
    n_tiles = s.info()["n_tiles"]
    assert n_tiles > 2
    hlbm_inject_fault(s.h, 1, n_tiles // 2)
    s.step(1)  # queued; the wait runs out on the device
    assert s.status & ST_SYNC_TIMEOUT
    with pytest.raises(HLBMError) as e:
        s.force()
    assert e.value.code == ETIMEOUT
    with pytest.raises(HLBMError) as e:
        s.step(1)  # refused until acknowledged
    assert e.value.code == ETIMEOUT
    assert s.info()["time"] == 4
    # the GPU and its context are still usable
    x = torch.arange(1000, device="cuda", dtype=torch.float64)
    assert float(x.sum()) == 499500.0
    # restore the checkpoint and continue: bit for bit the uninterrupted run
    s.load(ck)
    s.step(5)
    ref.step(8)
    assert s.status == 0
    for a, b in zip(s.fields(), ref.fields()):
        assert np.array_equal(a, b)
    # or acknowledge and step on from the abandoned state
    hlbm_inject_fault(s.h, 1, n_tiles // 2)
    s.step(1)
    torch.cuda.synchronize()  # the status copy queued by that call has arrived
    with pytest.raises(HLBMError):
        s.step(1)
    hlbm_clear_status(s.h)
    assert s.status == 0
    s.step(2)
    assert s.status == 0
    s.close()
    ref.close()


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_nan_in_the_lattice_surfaces_as_unstable(dtype):
    from paper_2006_13631_gb300 import HLBMError, Solver, hlbm_clear_status, hlbm_inject_fault

    w = inputs.workload("lamina-small-f32")
    w.dtype = dtype
    s = Solver(w)
    s.step(1)
    cls = s.struct_class().ravel()
    # a discretization node just above the lamina, inside the patch's reach
    x = int(round(w.xc))
    ys = [y for y in range(int(w.yc), w.ny) if cls[y * w.nx + x] == 0]
    node = ys[0] * w.nx + x
    hlbm_inject_fault(s.h, 2, node)
    seen = False
    for _ in range(20):
        s.step(1)
        if s.status & ST_NONFINITE:
            seen = True
            break
    assert seen, "the NaN did not reach the lamina force within 20 steps"
    with pytest.raises(HLBMError) as e:
        s.force()
    assert e.value.code == EUNSTABLE
    t = s.info()["time"]
    with pytest.raises(HLBMError) as e:
        s.step(1)
    assert e.value.code == EUNSTABLE and s.info()["time"] == t
    hlbm_clear_status(s.h)
    assert s.status == 0
    s.close()


def test_status_seen_by_the_next_step_without_a_read():
    """The copy of the status word queued at the end of a hlbm_step call is
    read by the next call once it has arrived: after a synchronisation, the
    next step is refused without any hlbm_status / hlbm_force call."""
    from paper_2006_13631_gb300 import HLBMError, Solver, hlbm_inject_fault

    w = inputs.workload("lamina-small-f32")
    s = Solver(w)
    s.step(2)
    hlbm_inject_fault(s.h, 1, s.info()["n_tiles"] // 2)
    s.step(1)
    torch.cuda.synchronize()
    with pytest.raises(HLBMError) as e:
        s.step(1)
    assert e.value.code == ETIMEOUT
    s.close()


def test_fault_injection_rejects_bad_arguments():
    from paper_2006_13631_gb300 import HLBMError, Solver, hlbm_inject_fault

    w = inputs.workload("lamina-small-f32")
    s = Solver(w)
    with pytest.raises(HLBMError):
        hlbm_inject_fault(s.h, 1, 10 ** 6)
    with pytest.raises(HLBMError):
        hlbm_inject_fault(s.h, 2, w.nx * w.ny)
    with pytest.raises(HLBMError):
        hlbm_inject_fault(s.h, 9, 0)
    s.step(1)
    assert s.status == 0
    s.close()

"""Checkpoint and restart (hlbm_save / hlbm_load): a solver restored from a
file and stepped on reproduces, bit for bit, the run that never stopped;
files of other inputs and non-checkpoint files are refused."""
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


def _state(s):
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    tg, dg = s.refill_record()
    fx, fy = s.force()
    return dict(rs=rs, uxs=uxs, uys=uys, ru=ru, uxu=uxu, uyu=uyu, cls=s.struct_class(), tg=tg, dg=dg, fx=fx, fy=fy,
                pf=s.patch_f(), status=s.status)


@pytest.mark.parametrize("dtype", ["f32", "f64", "f16"])
def test_restart_reproduces_the_uninterrupted_run(tmp_path, dtype):
    from paper_2006_13631_gb300 import Solver

    w = inputs.workload("lamina-small-f32")
    w.dtype = dtype
    mesh, rho = w.mesh(), w.rho_init()
    a = Solver(w, mesh=mesh, rho_init=rho)
    a.step(31)
    path = str(tmp_path / f"ck_{dtype}.bin")
    a.save(path)
    a.step(40)
    b = Solver(w, mesh=mesh, rho_init=rho)
    b.step(5)  # a solver that has moved on is overwritten as well
    b.load(path)
    assert b.info()["time"] == 31
    b.step(40)
    sa, sb = _state(a), _state(b)
    for k in sa:
        assert np.array_equal(np.asarray(sa[k]), np.asarray(sb[k])), k
    assert sa["status"] == 0


def test_restart_refuses_other_inputs_and_foreign_files(tmp_path):
    from paper_2006_13631_gb300 import HLBMError, Solver

    w = inputs.workload("lamina-small-f32")
    mesh, rho = w.mesh(), w.rho_init()
    a = Solver(w, mesh=mesh, rho_init=rho)
    a.step(3)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    w2 = inputs.workload("lamina-small-f32")
    w2.tau_s = w.tau_s + 0.01
    w2.n_sub = w.n_sub + 2
    b = Solver(w2, mesh=mesh, rho_init=rho)
    with pytest.raises(HLBMError) as e:
        b.load(path)
    assert e.value.code == -1
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a checkpoint" * 64)
    with pytest.raises(HLBMError) as e:
        a.load(str(junk))
    assert e.value.code == -6
    with pytest.raises(HLBMError) as e:
        a.load(str(tmp_path / "missing.bin"))
    assert e.value.code == -6
    # a truncated file is refused
    cut = tmp_path / "cut.bin"
    cut.write_bytes(open(path, "rb").read()[:4096])
    with pytest.raises(HLBMError) as e:
        a.load(str(cut))
    assert e.value.code == -6


def test_restart_of_an_induced_motion_run(tmp_path):
    """The lamina's displacement and velocity travel with the checkpoint."""
    import math

    from paper_2006_13631_gb300 import Solver

    w = inputs.workload("lamina-small-f32")
    w.motion, w.A, w.omega = inputs.MOTION_INDUCED, 0.0, 0.0
    w.mass = math.pi / 4 * w.L * w.L
    w.stiffness = w.mass * (2 * math.pi / 150.0) ** 2
    w.y0 = 1.5
    mesh, rho = w.mesh(), w.rho_init()
    a = Solver(w, mesh=mesh, rho_init=rho)
    a.step(23)
    path = str(tmp_path / "ck_induced.bin")
    a.save(path)
    a.step(30)
    b = Solver(w, mesh=mesh, rho_init=rho)
    b.load(path)
    b.step(30)
    sa, sb = _state(a), _state(b)
    for k in sa:
        assert np.array_equal(np.asarray(sa[k]), np.asarray(sb[k])), k
    assert a.info()["y"] == b.info()["y"] and a.info()["vy"] == b.info()["vy"]

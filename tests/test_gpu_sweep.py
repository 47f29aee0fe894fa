"""Batched KC/beta sweep (hlbm_sweep_*): instances stepped together give
exactly the fields, classes, refill records and forces of the same
instances stepped one by one, before and after the tile tuner; the
smallest instance of the 64-instance study matches the oracle."""
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


def _small(name, dtype, tau, n_sub, A=1.2):
    w = inputs.workload("lamina-small-f32")
    w.name, w.dtype, w.tau_s, w.n_sub, w.A = name, dtype, tau, n_sub, A
    return w


def _instances():
    # n_sub at or above the stable count of the mesh for each tau
    return [_small("a", "f32", 0.6, 26), _small("b", "f64", 0.7, 52, A=0.8), _small("c", "f32", 0.55, 17, A=1.5),
            _small("d", "bf16", 0.6, 26), _small("e", "f16", 0.65, 40, A=1.0)]


def _state(s):
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    tg, dg = s.refill_record()
    fx, fy = s.force()
    return dict(rs=rs, uxs=uxs, uys=uys, ru=ru, uxu=uxu, uyu=uyu, cls=s.struct_class(), tg=tg, dg=dg, fx=fx, fy=fy,
                status=s.status)


def _same(a, b):
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def test_sweep_equals_individual_steps():
    from paper_2006_13631_gb300 import Solver, Sweep

    ws = _instances()
    meshes = [w.mesh() for w in ws]
    rhos = [w.rho_init() for w in ws]
    alone = [Solver(w, mesh=m, rho_init=r) for w, m, r in zip(ws, meshes, rhos)]
    batch = [Solver(w, mesh=m, rho_init=r) for w, m, r in zip(ws, meshes, rhos)]
    sw = Sweep(batch)
    for s in alone:
        s.step(7)
    sw.step(3)
    sw.step(4)
    torch.cuda.synchronize()
    for a, b in zip(alone, batch):
        assert a.status == 0 and b.status == 0
        _same(_state(a), _state(b))
    # retiled by the tuner: the FV arithmetic of a node does not depend on
    # its tile, so the sweep still reproduces the one-by-one steps exactly
    picks = sw.tune(trial_steps=1)
    assert len(picks) == len(batch) and all(p in (256, 512, 1024, 1536) for p in picks)
    for s in alone:
        s.step(4)  # the tuner's four trial steps
    sw.step(5)
    for s in alone:
        s.step(5)
    ms = sw.fv_time(2)
    for s in alone:
        s.step(2)
    assert (ms > 0).all()
    torch.cuda.synchronize()
    for a, b in zip(alone, batch):
        _same(_state(a), _state(b))
    # packed: the FP32-arithmetic solvers with 26 sub-steps (FP32 and BF16
    # storage) share one FV launch; still the same results
    assert sw.pack() == 1
    for k in (3, 6):
        sw.step(k)
        for s in alone:
            s.step(k)
        torch.cuda.synchronize()
        for a, b in zip(alone, batch):
            assert b.status == 0
            _same(_state(a), _state(b))
    assert sw.pack(False) == 0
    sw.step(2)
    for s in alone:
        s.step(2)
    for a, b in zip(alone, batch):
        _same(_state(a), _state(b))
    sw.close()


def test_sweep_smallest_study_instance_matches_oracle():
    from paper_2006_13631_gb300 import Solver, Sweep

    ws = inputs.sweep_workloads()
    w = min(ws, key=lambda v: (v.nx * v.ny, v.n_sub))
    other = max(ws, key=lambda v: v.n_sub if v.nx == w.nx else 0)
    mesh = w.mesh()
    rho = w.rho_init()
    s = Solver(w, mesh=mesh, rho_init=rho)
    s2 = Solver(other)
    sw = Sweep([s, s2])
    o = oracle.Oracle(w, mesh=mesh, rho_init=rho)
    sw.step(3)
    o.step(3)
    assert s.status == 0 and s2.status == 0
    assert np.array_equal(s.struct_class(), o.struct_class())
    tg, dg = s.refill_record()
    to, do = o.refill_record()
    assert np.array_equal(tg, to) and np.array_equal(dg, do)
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    pr, pux, puy = o.patch_macro()
    num = np.sqrt(((uxu - pux) ** 2 + (uyu - puy) ** 2).sum())
    den = np.sqrt((pux ** 2 + puy ** 2).sum()) + 1e-12 * np.sqrt(pux.size)
    assert num / den < 1e-5
    assert np.sqrt(((ru - pr) ** 2).sum() / (pr ** 2).sum()) < 1e-5
    sw.close()


def test_pack_of_the_largest_study_patches_runs_and_changes_nothing():
    """The study's L = 64 instances (about 100k-node patches) after the
    tuner: their groups either pack with tiles the tensor-memory kernel can
    hold or stay unpacked with the tuned tiles; packing never fails and the
    results equal those of the same solvers stepped one by one."""
    from paper_2006_13631_gb300 import Solver, Sweep

    ws = [w for w in inputs.sweep_workloads() if w.L == 64.0][:4]
    assert len(ws) == 4
    meshes = [w.mesh() for w in ws]
    alone = [Solver(w, mesh=m) for w, m in zip(ws, meshes)]
    batch = [Solver(w, mesh=m) for w, m in zip(ws, meshes)]
    sw = Sweep(batch)
    sw.tune(trial_steps=1)
    for s in alone:
        s.step(4)  # the tuner's four trial steps
    n_packs = sw.pack()
    assert 0 <= n_packs <= 2
    sw.step(3)
    for s in alone:
        s.step(3)
    torch.cuda.synchronize()
    for a, b in zip(alone, batch):
        assert a.status == 0 and b.status == 0
        _same(_state(a), _state(b))
    assert sw.pack(False) == 0
    sw.step(1)
    for s in alone:
        s.step(1)
    for a, b in zip(alone, batch):
        _same(_state(a), _state(b))
    sw.close()


def test_sweep_rejects_bad_arguments():
    from paper_2006_13631_gb300 import HLBMError, Sweep

    with pytest.raises(HLBMError):
        Sweep([])

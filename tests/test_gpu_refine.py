"""Two structured levels (a fine box in a coarse lattice of twice the
spacing) on the CUDA path against the oracle's reading R12, through the C
ABI: node classes and donors bit-exact, fine and coarse fields and forces
within the single-level bars; restart, sweeps and the argument checks."""
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


def rel_l2(a, b, mask=None):
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def vel_rel_l2(ux, uy, vx, vy, mask=None, floor=1e-12):
    if mask is not None:
        ux, uy, vx, vy = ux[mask], uy[mask], vx[mask], vy[mask]
    num = np.sqrt(((ux - vx) ** 2 + (uy - vy) ** 2).sum())
    den = np.sqrt((vx ** 2 + vy ** 2).sum()) + floor * np.sqrt(vx.size)
    return float(num / den)


def pair(w):
    from paper_2006_13631_gb300 import Solver

    mesh, rho = w.mesh(), w.rho_init()
    return Solver(w, mesh=mesh, rho_init=rho), oracle.Oracle(w, mesh=mesh, rho_init=rho)


def errors(s, o):
    disc = o.struct_class() == oracle.DISC
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    ro, uxo, uyo = o.struct_macro()
    pr, pux, puy = o.patch_macro()
    rc, uxc, uyc = s.coarse_macro()
    rco, uxco, uyco = o.coarse_macro()
    return dict(struct_u=vel_rel_l2(uxs, uys, uxo, uyo, disc), struct_rho=rel_l2(rs, ro, disc),
                patch_u=vel_rel_l2(uxu, uyu, pux, puy), patch_rho=rel_l2(ru, pr),
                coarse_u=vel_rel_l2(uxc, uyc, uxco, uyco), coarse_rho=rel_l2(rc, rco))


@pytest.mark.parametrize("dtype,chunks,tol_u,tol_rho", [("f64", (1, 2, 9, 28), 2e-9, 1e-12),
                                                         ("f32", (11, 40, 50, 99), 1e-5, 1e-5)])
def test_two_level_parity(dtype, chunks, tol_u, tol_rho):
    """Odd and even step counts (the coarse lattice advances every second
    step), the ring, the restriction and the coarse lattice all checked."""
    w = inputs.workload(f"lamina-small-refined-{dtype}")
    s, o = pair(w)
    for c in chunks:
        s.step(c)
        o.step(c)
        assert np.array_equal(s.struct_class(), o.struct_class())
        tg, dg = s.refill_record()
        to, do = o.refill_record()
        assert np.array_equal(tg, to) and np.array_equal(dg, do)
        e = errors(s, o)
        assert all(e[k] < tol_u for k in ("struct_u", "patch_u", "coarse_u")), e
        assert all(e[k] < tol_rho for k in ("struct_rho", "patch_rho", "coarse_rho")), e
    assert s.status == 0 and o.status == 0
    fys, fyo = s.force()[1], o.force()[1]
    assert np.abs(fys - fyo).max() < (1e-9 if dtype == "f64" else 1e-4) * np.abs(fyo).max()
    info = s.info()
    assert info["n_coarse"] == w.nxc * w.nyc and info["launches_per_step"] == 10


def test_two_level_ring_and_restriction_are_consistent():
    """Invariants at any size: the coarse nodes strictly inside the box equal
    the fine nodes under them in rho and u after an even number of steps
    (restriction keeps the moments), and the ring's fine nodes at even
    positions carry the coarse node's rho and u."""
    w = inputs.workload("lamina-small-refined-f64")
    from paper_2006_13631_gb300 import Solver

    s = Solver(w)
    s.step(24)
    rs, uxs, uys = s.fields()[:3]
    rc, uxc, uyc = s.coarse_macro()
    cls = s.struct_class()
    niw, njw = (w.nx - 1) // 2, (w.ny - 1) // 2
    inner_f = (slice(2, 2 * njw - 1, 2), slice(2, 2 * niw - 1, 2))
    inner_c = (slice(w.oy + 1, w.oy + njw), slice(w.ox + 1, w.ox + niw))
    ok = cls[inner_f] == oracle.DISC
    for a, b in ((rs, rc), (uxs, uxc), (uys, uyc)):
        assert np.abs(a[inner_f][ok] - b[inner_c][ok]).max() < 1e-14
    assert (~ok).sum() > 0 and np.abs(uxc[inner_c][~ok]).max() == 0.0
    # ring nodes at even positions of the bottom edge
    for a, b in ((rs, rc), (uxs, uxc), (uys, uyc)):
        assert np.abs(a[0, ::2] - b[w.oy, w.ox:w.ox + niw + 1]).max() < 1e-14


@pytest.mark.parametrize("t_save", [31, 32])
def test_two_level_restart_reproduces_the_uninterrupted_run(tmp_path, t_save):
    from paper_2006_13631_gb300 import Solver

    w = inputs.workload("lamina-small-refined-f32")
    mesh, rho = w.mesh(), w.rho_init()
    a = Solver(w, mesh=mesh, rho_init=rho)
    a.step(t_save)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(17)
    b = Solver(w, mesh=mesh, rho_init=rho)
    b.step(3)
    b.load(path)
    b.step(17)
    for x, y in zip(a.fields() + list(a.coarse_macro()) + list(a.force()),
                    b.fields() + list(b.coarse_macro()) + list(b.force())):
        assert np.array_equal(x, y)
    # a checkpoint of the single-level solver does not fit a refined one
    w1 = inputs.workload("lamina-small-f32")
    c = Solver(w1, mesh=mesh, rho_init=rho)
    c.save(str(tmp_path / "single.bin"))
    from paper_2006_13631_gb300 import HLBMError

    with pytest.raises(HLBMError) as e:
        b.load(str(tmp_path / "single.bin"))
    assert e.value.code == -1


def test_two_level_solvers_in_a_sweep_equal_one_by_one():
    from paper_2006_13631_gb300 import Solver, Sweep

    ws = [inputs.workload("lamina-small-refined-f32"), inputs.workload("lamina-small-refined-bf16"),
          inputs.workload("lamina-small-f32")]
    meshes = [w.mesh() for w in ws]
    rhos = [w.rho_init() for w in ws]
    alone = [Solver(w, mesh=m, rho_init=r) for w, m, r in zip(ws, meshes, rhos)]
    batch = [Solver(w, mesh=m, rho_init=r) for w, m, r in zip(ws, meshes, rhos)]
    sw = Sweep(batch)
    for s in alone:
        s.step(9)
    sw.step(4)
    sw.step(5)
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(alone, batch)):
        assert a.status == 0 and b.status == 0
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)
        if ws[k].refine:
            for x, y in zip(a.coarse_macro(), b.coarse_macro()):
                assert np.array_equal(x, y)
    sw.close()


def test_two_level_arguments_are_checked():
    from paper_2006_13631_gb300 import HLBMError, Solver

    for over in (dict(nx=202), dict(ox=0), dict(ox=102), dict(nyc=118), dict(tau_s=1.0)):
        w = inputs.workload("lamina-small-refined-f32")
        for k, v in over.items():
            setattr(w, k, v)
        if "tau_s" in over:
            w.n_sub = 4
        with pytest.raises(HLBMError) as e:
            Solver(w)
        assert e.value.code == -1, over
    s = Solver(inputs.workload("lamina-small-f32"))
    with pytest.raises(HLBMError) as e:
        s.coarse_macro() if False else __import__("paper_2006_13631_gb300").hlbm_get_coarse_fields(s.h, 4, 4)
    assert e.value.code == -1


def test_two_level_theta_agrees_with_the_uniform_lattice():
    """The point of the levels (Sec. 5): the far field on a lattice of twice
    the spacing leaves the hydrodynamic function of the uniform lattice
    unchanged.  1024^2 domain, chord 32, KC 0.25, beta 500, tau 0.6, FP64,
    8 periods (fit over the last 3); a fine box of 4 chords in a 512^2
    coarse lattice.  Measured on a GB300: |Theta_2 - Theta_1| = 0.23 % of
    |Theta_1| (box of 8 chords: 0.04 %)."""
    from paper_2006_13631_gb300 import Solver

    u = inputs.workload("lamina-1024-f64")
    steps = int(round(8 * u.period))
    s = Solver(u)
    s.step(steps)
    re1, im1, _ = s.gamma(discard=5.0, fit=3.0)
    s.close()
    w = inputs.workload("lamina-1024-refined-f64")
    w.nx = w.ny = 129
    w.xc, w.yc = 64.3, 64.2
    w.ox = w.oy = 256 - 32
    r = Solver(w)
    r.step(steps)
    re2, im2, _ = r.gamma(discard=5.0, fit=3.0)
    assert r.status == 0
    assert abs(complex(re2 - re1, im2 - im1)) < 5e-3 * abs(complex(re1, im1))

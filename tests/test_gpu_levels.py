"""Nested structured levels (boxes inside lattices of twice the spacing,
Sec. 5) on the CUDA path against the oracle's reading R12, through the C
ABI: node classes and donors bit-exact, every level's fields and the force
within the single-level bars; restart, sweeps, the argument checks, and the
hydrodynamic function against the uniform lattice."""
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


def errors(s, o, n_levels):
    disc = o.struct_class() == oracle.DISC
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    ro, uxo, uyo = o.struct_macro()
    pr, pux, puy = o.patch_macro()
    e = dict(struct_u=vel_rel_l2(uxs, uys, uxo, uyo, disc), struct_rho=rel_l2(rs, ro, disc),
             patch_u=vel_rel_l2(uxu, uyu, pux, puy), patch_rho=rel_l2(ru, pr))
    for k in range(1, n_levels + 1):
        rc, uxc, uyc = s.level_macro(k)
        rco, uxco, uyco = o.level_macro(k)
        e[f"level{k}_u"] = vel_rel_l2(uxc, uyc, uxco, uyco)
        e[f"level{k}_rho"] = rel_l2(rc, rco)
    return e


@pytest.mark.parametrize("name,chunks,tol_u,tol_rho", [
    ("lamina-small-refined-f64", (1, 2, 9, 28), 2e-9, 1e-12),
    ("lamina-small-refined-f32", (11, 40, 50, 99), 1e-5, 1e-5),
    ("lamina-small-levels3-f64", (1, 2, 3, 5, 29), 2e-9, 1e-12),
    ("lamina-small-levels3-f32", (7, 42, 51, 100), 1e-5, 1e-5)])
def test_levels_parity(name, chunks, tol_u, tol_rho):
    """Step counts that are not multiples of 2^levels: every level's clock,
    the rings, the restrictions and the coarser lattices are checked."""
    w = inputs.workload(name)
    s, o = pair(w)
    for c in chunks:
        s.step(c)
        o.step(c)
        assert np.array_equal(s.struct_class(), o.struct_class())
        tg, dg = s.refill_record()
        to, do = o.refill_record()
        assert np.array_equal(tg, to) and np.array_equal(dg, do)
        e = errors(s, o, len(w.levels))
        assert all(v < tol_u for k, v in e.items() if k.endswith("_u")), e
        assert all(v < tol_rho for k, v in e.items() if k.endswith("_rho")), e
    assert s.status == 0 and o.status == 0
    fys, fyo = s.force()[1], o.force()[1]
    assert np.abs(fys - fyo).max() < (1e-9 if w.dtype == "f64" else 1e-4) * np.abs(fyo).max()
    info = s.info()
    assert info["n_levels"] == len(w.levels)
    assert info["n_coarse"] == sum(a * b for a, b, _, _ in w.levels)
    assert info["launches_per_step"] == 8 + 2 * len(w.levels)


def test_levels_parity_with_absorbing_layer_on_the_coarsest():
    """The absorbing outflow layer belongs to the lattice that carries the
    domain boundary: with three levels it acts on the coarsest only (6 of
    its rows along each outflow side), in the oracle and in the CUDA path."""
    w = inputs.workload("lamina-small-levels3-f64")
    w.sponge_rows, w.sponge_sigma = 6, 0.1
    s, o = pair(w)
    for c in (3, 29):
        s.step(c)
        o.step(c)
        assert np.array_equal(s.struct_class(), o.struct_class())
        e = errors(s, o, len(w.levels))
        assert all(v < 2e-9 for k, v in e.items() if k.endswith("_u")), e
        assert all(v < 1e-12 for k, v in e.items() if k.endswith("_rho")), e
    assert s.status == 0 and o.status == 0


def test_levels_ring_and_restriction_are_consistent():
    """Invariants at any size: after 2^levels steps, the nodes of each level
    strictly inside the box of the level below equal the finer nodes under
    them in rho and u (restriction keeps the moments), and each box's ring at
    even positions carries the coarser level's rho and u."""
    from paper_2006_13631_gb300 import Solver

    w = inputs.workload("lamina-small-levels3-f64")
    s = Solver(w)
    s.step(24)
    fine = s.fields()[:3]
    cls = s.struct_class()
    nx, ny = w.nx, w.ny
    for k, (cnx, cny, ox, oy) in enumerate(w.levels, start=1):
        coarse = s.level_macro(k)
        niw, njw = (nx - 1) // 2, (ny - 1) // 2
        inner_f = (slice(2, 2 * njw - 1, 2), slice(2, 2 * niw - 1, 2))
        inner_c = (slice(oy + 1, oy + njw), slice(ox + 1, ox + niw))
        ok = cls[inner_f] == oracle.DISC if k == 1 else np.ones_like(fine[0][inner_f], bool)
        for a, b in zip(fine, coarse):
            assert np.abs(a[inner_f][ok] - b[inner_c][ok]).max() < 1e-14
            assert np.abs(a[0, ::2] - b[oy, ox:ox + niw + 1]).max() < 1e-14
        if k == 1:
            assert (~ok).sum() > 0 and np.abs(coarse[1][inner_c][~ok]).max() == 0.0
        fine, nx, ny = coarse, cnx, cny


@pytest.mark.parametrize("name,t_save", [("lamina-small-refined-f32", 31), ("lamina-small-refined-f32", 32),
                                         ("lamina-small-levels3-f32", 30)])
def test_levels_restart_reproduces_the_uninterrupted_run(tmp_path, name, t_save):
    from paper_2006_13631_gb300 import HLBMError, Solver

    w = inputs.workload(name)
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
    lv = lambda s: [x for k in range(1, len(w.levels) + 1) for x in s.level_macro(k)]
    for x, y in zip(a.fields() + lv(a) + list(a.force()), b.fields() + lv(b) + list(b.force())):
        assert np.array_equal(x, y)
    # a checkpoint of the single-level solver does not fit a refined one
    c = Solver(inputs.workload("lamina-small-f32"), mesh=mesh, rho_init=rho)
    c.save(str(tmp_path / "single.bin"))
    with pytest.raises(HLBMError) as e:
        b.load(str(tmp_path / "single.bin"))
    assert e.value.code == -1


def test_levels_solvers_in_a_sweep_equal_one_by_one():
    from paper_2006_13631_gb300 import Solver, Sweep

    ws = [inputs.workload("lamina-small-refined-f32"), inputs.workload("lamina-small-levels3-bf16"),
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
    for w, a, b in zip(ws, alone, batch):
        assert a.status == 0 and b.status == 0
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y)
        for k in range(1, len(w.levels) + 1):
            for x, y in zip(a.level_macro(k), b.level_macro(k)):
                assert np.array_equal(x, y)
    sw.close()


def test_levels_arguments_are_checked():
    import paper_2006_13631_gb300 as P

    def bad(name, **over):
        w = inputs.workload(name)
        for k, v in over.items():
            setattr(w, k, v)
        with pytest.raises(P.HLBMError) as e:
            P.Solver(w)
        assert e.value.code == -1, over

    bad("lamina-small-refined-f32", nx=202)                            # even box
    bad("lamina-small-refined-f32", levels=[(204, 160, 0, 40)])        # no margin
    bad("lamina-small-refined-f32", levels=[(204, 160, 102, 40)])      # box past the edge
    bad("lamina-small-refined-f32", levels=[(204, 118, 51, 40)])
    bad("lamina-small-levels3-f32", levels=[(211, 167, 1, 43), (216, 176, 53, 44)])  # margin 2 inside a ring
    bad("lamina-small-levels3-f32", levels=[(210, 167, 52, 43), (216, 176, 53, 44)])  # even inner level
    bad("lamina-small-refined-f32", levels=[(204, 160, 51, 40)] * 5)  # too many levels
    bad("lamina-small-refined-f32", tau_s=1.0, n_sub=4)                # tau_0 = 1
    bad("lamina-small-levels3-f32", tau_s=2.5, n_sub=4)                # tau_2 = 1
    s = P.Solver(inputs.workload("lamina-small-f32"))
    with pytest.raises(P.HLBMError) as e:
        P.hlbm_get_level_fields(s.h, 1, 4, 4)
    assert e.value.code == -1


@pytest.mark.parametrize("name,bar", [("lamina-1024-refined-f64", 5e-3), ("lamina-1024-levels4-f64", 5e-3)])
def test_levels_theta_agrees_with_the_uniform_lattice(name, bar):
    """The point of the levels (Sec. 5): the far field on coarser lattices
    leaves the hydrodynamic function of the uniform lattice unchanged.
    1024^2 domain, chord 32, KC 0.25, beta 500, tau 0.6, FP64, 8 periods
    (fit over the last 3).  Two levels with a 4-chord box (measured on a
    GB300: 0.23 % of |Theta|) and the paper's four levels (boxes of 4, 8 and
    16 chords, a 128^2 lattice of spacing 8)."""
    from paper_2006_13631_gb300 import Solver

    u = inputs.workload("lamina-1024-f64")
    steps = int(round(8 * u.period))
    s = Solver(u)
    s.step(steps)
    re1, im1, _ = s.gamma(discard=5.0, fit=3.0)
    s.close()
    w = inputs.workload(name)
    if name == "lamina-1024-refined-f64":
        w.nx = w.ny = 129
        w.xc, w.yc = 64.3, 64.2
        w.levels = [(512, 512, 224, 224)]
    r = Solver(w)
    r.step(steps)
    re2, im2, _ = r.gamma(discard=5.0, fit=3.0)
    assert r.status == 0
    d = abs(complex(re2 - re1, im2 - im1)) / abs(complex(re1, im1))
    print(name, "Theta", complex(re2, im2), "uniform", complex(re1, im1), "rel", d)
    assert d < bar


def test_levels_theta_gradient_matches_oracle_fd():
    """hlbm_theta_gradient on a lattice with a coarser level: the seven solves
    of the central differences carry the levels along; Theta and its
    gradient in (A, omega, tau_s) against the same quotient from seven oracle
    runs (FP64, the 256^2 domain as a 129^2 box in a 128^2 lattice of
    spacing 2, 48 steps, fit over 0.5-2 periods)."""
    from paper_2006_13631_gb300 import hlbm_theta_gradient, use_torch_allocator, workload_inputs

    use_torch_allocator()
    w = inputs.workload("lamina-256-f64")
    w.nx = w.ny = 129
    w.xc, w.yc = 64.3, 64.2
    w.levels = [(128, 128, 32, 32)]
    mesh, rho = w.mesh(), w.rho_init()
    grid, patch, motion = workload_inputs(w, mesh, rho)
    th, grad, ms = hlbm_theta_gradient(grid, patch, w.tau_s, motion, 48, discard=0.5, fit=1.5, rel_step=1e-4)
    tho, grado = oracle.theta_fd_gradient(w, 48, discard=0.5, fit=1.5, rel_step=1e-4, mesh=mesh, rho_init=rho)
    print("levels theta", th, tho, "grad", grad, grado)
    assert abs(th - tho) < 1e-8
    assert np.abs(grad - grado).max() < 1e-4 * np.abs(grado).max()


def test_paper_point_at_chord_800_on_four_levels():
    """The paper's own setup (Sec. 5): chord 800, domain 5L, four structured
    levels, tau 0.8 at the finest; the point (beta, eps) = (250, 0.02) over
    4 periods (102 k steps, FP32), against the value the paper prints
    (tests/golden/paper_theta_mg_hlbm.txt).  Measured on a GB300: Re +1.7 %,
    -Im +2.7 %."""
    from paper_2006_13631_gb300 import Solver

    paper = {}
    with open(__import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                         "paper_theta_mg_hlbm.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                b, e, re_, mim = map(float, line.split())
                paper[(b, e)] = (re_, mim)
    w = inputs.paper_point_levels_workload(250.0, 0.02)
    s = Solver(w)
    s.step(w.steps)
    re_, im_, _ = s.gamma(discard=1.0, fit=3.0)
    assert s.status == 0
    pre, pmim = paper[(250.0, 0.02)]
    print("chord 800 Theta", re_, im_, "paper", pre, -pmim)
    assert abs(re_ - pre) < 0.03 * pre
    assert abs(-im_ - pmim) < 0.05 * pmim


def _donors_valid(mesh, dY, tg, dg, to, do):
    """Refill records that may differ only at ties (the lamina's path comes
    from the computed force): the types agree, and a node whose donor
    triangle differs lies (to 1e-9) in both triangles."""
    assert np.array_equal(tg, to)
    diff = np.nonzero(dg != do)[0]
    assert len(diff) <= max(2, len(dg) // 100), len(diff)
    for i in diff:
        assert tg[i] == 3
        q = mesh.xy[i] + np.array([0.0, dY])
        for k in (dg[i], do[i]):
            a, b, c = mesh.xy[mesh.tri[k]]
            m = np.array([[b[0] - a[0], c[0] - a[0]], [b[1] - a[1], c[1] - a[1]]])
            l1, l2 = np.linalg.solve(m, q - a)
            assert min(1 - l1 - l2, l1, l2) > -1e-9


@pytest.mark.parametrize("variant", ["outer_fv", "induced"])
def test_levels_with_the_method_variants(variant):
    """Three levels together with the outer nodes' FV sums (reading R10) or
    with the lamina moved by the fluid force (reading R11), FP64, against
    the oracle: every level's fields within the FP64 bars, and for the
    induced motion the lamina's path within 1e-10 of its displacement."""
    import math

    w = inputs.workload("lamina-small-levels3-f64")
    if variant == "outer_fv":
        w.outer_fv = 1
    else:
        w.motion, w.A, w.omega = inputs.MOTION_INDUCED, 0.0, 0.0
        w.mass = math.pi / 4 * w.L * w.L
        w.stiffness = w.mass * (2 * math.pi / 150.0) ** 2
        w.y0 = 1.5
    s, o = pair(w)
    for c in (1, 18, 21):
        s.step(c)
        o.step(c)
        if variant == "outer_fv":
            assert np.array_equal(s.struct_class(), o.struct_class())
        else:
            y, _ = o.motion()
            tg, dg = s.refill_record()
            to, do = o.refill_record()
            _donors_valid(w.mesh(), y[o.time - 1] - y[o.time - 2] if o.time > 1 else 0.0, tg, dg, to, do)
        e = errors(s, o, len(w.levels))
        assert all(v < 2e-9 for k, v in e.items() if k.endswith("_u")), e
        assert all(v < 1e-12 for k, v in e.items() if k.endswith("_rho")), e
    assert s.status == 0 and o.status == 0
    if variant == "induced":
        y, v = o.motion()
        info = s.info()
        assert abs(info["y"] - y[-1]) < 1e-10 * abs(w.y0) and abs(info["vy"] - v[-1]) < 1e-10 * abs(w.y0)

"""CUDA path against the CPU oracle, through the C ABI.

Bars: node classes and refill donors bit-exact; FP64 fields within 1e-9
relative L2 (2e-9 where the flow is driven by density noise); FP32 fields
within 1e-5 relative L2 over 200 steps; the
hydrodynamic function within 0.5 %.  Sizes span several thread blocks and
ragged lattice edges (203 x 157), plus the full 4096^2 workload on sampled
outputs and properties.
"""
import math

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


def vel_rel_l2(ux, uy, vx, vy, mask=None, floor=0.0):
    """||u - v|| / (||v|| + floor sqrt(n)): relative L2 with an absolute floor
    per node.  The FP64 oracle carries full populations (f ~ 0.1), so its
    velocities have an absolute rounding error near 1e-16 per node; where
    the flow is nearly at rest that error, not the CUDA path, sets the
    relative L2, hence the floor."""
    if mask is not None:
        ux, uy, vx, vy = ux[mask], uy[mask], vx[mask], vy[mask]
    num = np.sqrt(((ux - vx) ** 2 + (uy - vy) ** 2).sum())
    den = np.sqrt((vx ** 2 + vy ** 2).sum()) + floor * np.sqrt(vx.size)
    return float(num / den)


def pair(name, **over):
    from paper_2006_13631_gb300 import Solver

    w = inputs.workload(name) if isinstance(name, str) else name
    for k, v in over.items():
        setattr(w, k, v)
    mesh = w.mesh()
    rho = w.rho_init()
    return w, Solver(w, mesh=mesh, rho_init=rho), oracle.Oracle(w, mesh=mesh, rho_init=rho)


def compare_geometry(s, o):
    assert np.array_equal(s.struct_class(), o.struct_class())
    tg, dg = s.refill_record()
    to, do = o.refill_record()
    assert np.array_equal(tg, to)
    assert np.array_equal(dg, do)


def compare_fields(s, o, tol_u, tol_rho, floor=1e-12):
    cls = o.struct_class()
    disc = cls == oracle.DISC
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    ro, uxo, uyo = o.struct_macro()
    pr, pux, puy = o.patch_macro()
    e = dict(struct_u=vel_rel_l2(uxs, uys, uxo, uyo, disc, floor), struct_rho=rel_l2(rs, ro, disc),
             patch_u=vel_rel_l2(uxu, uyu, pux, puy, None, floor), patch_rho=rel_l2(ru, pr))
    assert e["struct_u"] < tol_u and e["patch_u"] < tol_u, e
    assert e["struct_rho"] < tol_rho and e["patch_rho"] < tol_rho, e
    return e


def test_fv_matrices_match_oracle():
    w, s, o = pair("lamina-small-f64")
    rp, col, gx, gy, cc = s.fv_coeffs()
    rpo, colo, gxo, gyo, cco, vol = o.fv_coeffs()
    assert np.array_equal(rp, rpo) and np.array_equal(col, colo)
    scale = np.abs(gxo).max()
    assert np.abs(gx - gxo).max() < 1e-12 * scale and np.abs(gy - gyo).max() < 1e-12 * scale
    assert np.abs(cc - cco).max() < 1e-13


def test_initial_state_matches_oracle():
    w, s, o = pair("lamina-small-f64")
    assert np.array_equal(s.struct_class(), o.struct_class())
    assert np.abs(s.patch_f() - o.patch_f()).max() < 1e-14
    fxs, fys = s.force()
    fxo, fyo = o.force()
    assert abs(fys[0] - fyo[0]) < 1e-12 and abs(fxs[0] - fxo[0]) < 1e-12


def test_parity_fp64_small_ragged_lattice():
    """FP64 bar 2e-9: the flow here is driven by 1e-6 density noise, and the
    oracle's full populations (f ~ 0.1) resolve that noise only to about
    1e-10 relative, which the velocity field inherits."""
    w, s, o = pair("lamina-small-f64")
    for chunk in (1, 4, 25, 30):
        s.step(chunk)
        o.step(chunk)
        compare_geometry(s, o)
        compare_fields(s, o, 2e-9, 1e-12)
    assert s.status == 0 and o.status == 0
    fxs, fys = s.force()
    fxo, fyo = o.force()
    assert np.abs(fys - fyo).max() < 1e-9 * np.abs(fyo).max()


def test_parity_fp32_200_steps():
    w, s, o = pair("lamina-small-f32")
    for chunk in (10, 40, 50, 100):
        s.step(chunk)
        o.step(chunk)
        compare_geometry(s, o)
    e = compare_fields(s, o, 1e-5, 1e-5)
    print("fp32 200-step errors", e)
    assert s.status == 0


def test_parity_lamina_256_fp64_four_periods_and_gamma():
    """256^2, chord 20, beta 500, KC 0.25, tau 0.6, FP64: 4 periods, Theta."""
    w, s, o = pair("lamina-256-f64")
    s.step(w.steps)
    o.step(w.steps)
    compare_geometry(s, o)
    compare_fields(s, o, 1e-9, 1e-11)
    re_g, im_g, _ = s.gamma(1.0, 3.0)
    re_o, im_o, _ = o.gamma(1.0, 3.0)
    assert abs(re_g - re_o) < 5e-3 * abs(re_o) and abs(im_g - im_o) < 5e-3 * abs(im_o)
    assert abs(re_g - re_o) < 1e-8 and abs(im_g - im_o) < 1e-8


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_zero_disturbance_translating_patch(dtype, tol):
    w = inputs.Workload("zero-disturbance", 64, 60, 12.0, 0.24, 30.3, 28.2, 0.7, 10, inputs.MOTION_UNIFORM,
                        vx=0.02, vy=0.03, delta_f=1.8, bc_x=inputs.BC_PERIODIC, bc_y=inputs.BC_PERIODIC,
                        u0x=0.02, u0y=0.03, dtype=dtype,
                        mesh_args=dict(n_L=24, n_T=1, n_layers=8, h1=0.2, d_out=3.6))
    from paper_2006_13631_gb300 import Solver

    s = Solver(w)
    s.step(120)
    assert s.status == 0
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    disc = s.struct_class() == 0
    assert np.abs(uxs[disc] - 0.02).max() < tol and np.abs(uys[disc] - 0.03).max() < tol
    assert np.abs(uxu - 0.02).max() < tol and np.abs(uyu - 0.03).max() < tol
    assert np.abs(rs[disc] - 1).max() < tol and np.abs(ru - 1).max() < tol


def test_disk_patch_shear_wave_matches_oracle():
    nx = ny = 64
    w = inputs.Workload("disk-shear", nx, ny, 0.0, 0.0, 32.3, 32.2, 0.8, 20, inputs.MOTION_STATIC, delta_f=3.0,
                        bc_x=inputs.BC_PERIODIC, bc_y=inputs.BC_PERIODIC, dtype="f32",
                        mesh_args=dict(n_L=0, n_T=0, n_layers=12, h1=0.5, d_out=6.0))
    mesh = w.mesh()
    uy0 = 1e-3 * np.sin(2 * math.pi / nx * np.tile(np.arange(nx, dtype=float), (ny, 1)))
    u0 = (np.zeros((ny, nx)), uy0)
    from paper_2006_13631_gb300 import Solver

    s = Solver(w, mesh=mesh, rho_init=np.ones((ny, nx)), u_init=u0)
    o = oracle.Oracle(w, mesh=mesh, rho_init=np.ones((ny, nx)), u_init=u0)
    s.step(300)
    o.step(300)
    compare_fields(s, o, 1e-5, 1e-6)


@pytest.mark.slow
def test_full_size_4096_200_steps_and_sampled_geometry():
    """4096^2, chord 128, ~200k-node patch, FP32 -- the benchmark's launch
    configuration: 200 full steps against the oracle (its OpenMP build on
    the host cores, bit-identical to the serial one) at the FP32 bar, then
    geometry (classes, refill types and donors) bit-exact at a later
    sampled step."""
    from paper_2006_13631_gb300 import Solver

    w = inputs.workload("lamina-4096-f32")
    mesh, rho = w.mesh(), w.rho_init()
    s = Solver(w, mesh=mesh, rho_init=rho)
    o = oracle.Oracle(w, mesh=mesh, rho_init=rho, openmp=True)
    assert s.info()["fv_kernel"] == 4  # the deep-tile FV kernel the bench times
    for chunk in (2, 48, 150):
        s.step(chunk)
        o.step(chunk)
        compare_geometry(s, o)
    e = compare_fields(s, o, 1e-5, 1e-5)
    print("4096^2 200-step errors", e)
    fxs, fys = s.force()
    fxo, fyo = o.force()
    assert np.abs(fys - fyo).max() < 1e-4 * np.abs(fyo).max()
    target = 400
    s.step(target - 200)
    assert s.status == 0
    assert np.array_equal(s.struct_class(), o.classify_at(target - 1))
    tg, dg = s.refill_record()
    to, do = o.relocate_at(target - 1)
    assert np.array_equal(tg, to) and np.array_equal(dg, do)
    fx, fy = s.force()
    assert np.isfinite(fy).all()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_parity_type2_refill(dtype, tol):
    """Sec. 4, type 2: a lamina moving 0.3 lattice spacings per step with a
    first node layer 0.1 from its surface, so nodes of the new configuration
    fall inside the old body and keep their own populations.  Types and donors
    bit-exact; the lamina translates with the fluid, so the flow stays
    uniform on both sides."""
    from paper_2006_13631_gb300 import Solver

    w = inputs.Workload("type2", 64, 72, 12.0, 0.24, 30.3, 30.2, 0.7, 10, inputs.MOTION_UNIFORM,
                        vx=0.0, vy=0.3, delta_f=1.8, bc_x=inputs.BC_PERIODIC, bc_y=inputs.BC_PERIODIC,
                        u0x=0.0, u0y=0.3, dtype=dtype, mesh_args=dict(n_L=24, n_T=1, n_layers=8, h1=0.1, d_out=4.0))
    mesh = w.mesh()
    w.n_sub = inputs.stable_substeps(mesh, w.tau_s - 0.5)
    s = Solver(w, mesh=mesh)
    o = oracle.Oracle(w, mesh=mesh)
    seen2 = 0
    for _ in range(6):
        s.step(1)
        o.step(1)
        compare_geometry(s, o)
        seen2 += int((s.refill_record()[0] == 2).sum())
    assert seen2 > 0
    assert s.status == 0 and o.status == 0
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    disc = s.struct_class() == 0
    assert np.abs(uys[disc] - 0.3).max() < tol and np.abs(uxs[disc]).max() < tol
    assert np.abs(uyu - 0.3).max() < tol and np.abs(ru - 1).max() < tol
    compare_fields(s, o, 1e-5 if dtype == "f32" else 1e-9, 1e-5 if dtype == "f32" else 1e-12)


@pytest.mark.parametrize("dtype,steps,tol_u,tol_rho", [("f64", 60, 2e-9, 1e-12), ("f32", 200, 1e-5, 1e-5)])
def test_parity_full_outer_node_update(dtype, steps, tol_u, tol_rho):
    """Outer patch nodes with the FV sums of eq. postcollision2_u (reading
    R10 of the oracle) against the oracle; same bars as the Dirichlet runs."""
    w, s, o = pair("lamina-small-" + dtype, outer_fv=1)
    for chunk in (1, steps // 2 - 1, steps // 2):
        s.step(chunk)
        o.step(chunk)
        compare_geometry(s, o)
    e = compare_fields(s, o, tol_u, tol_rho)
    print(dtype, "outer_fv errors", e)
    assert s.status == 0 and o.status == 0
    # the two readings give different fields: the FV sums are active
    w0, s0, _ = pair("lamina-small-" + dtype)
    s0.step(steps)
    assert not np.array_equal(s0.fields()[4], s.fields()[4])


def test_zero_disturbance_with_full_outer_node_update():
    w = inputs.Workload("zero-disturbance", 64, 60, 12.0, 0.24, 30.3, 28.2, 0.7, 10, inputs.MOTION_UNIFORM,
                        vx=0.02, vy=0.03, delta_f=1.8, bc_x=inputs.BC_PERIODIC, bc_y=inputs.BC_PERIODIC,
                        u0x=0.02, u0y=0.03, dtype="f64", outer_fv=1,
                        mesh_args=dict(n_L=24, n_T=1, n_layers=8, h1=0.2, d_out=3.6))
    from paper_2006_13631_gb300 import Solver

    s = Solver(w)
    s.step(120)
    assert s.status == 0
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    assert np.abs(uxu - 0.02).max() < 1e-12 and np.abs(uyu - 0.03).max() < 1e-12
    assert np.abs(ru - 1).max() < 1e-12


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_fv_kernels_agree_bit_for_bit(dtype):
    """The FV kernels (global-memory records, shared-memory tiles updated in
    place, tensor-memory rows with double-buffered records, and deep tiles
    that exchange with their neighbours every K sub-steps and recompute K
    ghost layers in between) run the same per-node arithmetic in the same
    order, so their fields agree exactly, whatever K.  n = 24 and 27
    sub-steps give even and odd numbers of exchanges per step and a short
    last block."""
    from paper_2006_13631_gb300 import Solver, hlbm_set_fv_depth

    w = inputs.workload("lamina-small-" + dtype)
    mesh, rho = w.mesh(), w.rho_init()
    for n_sub in (24, 27):
        w.n_sub = n_sub
        got = {}
        for kern in (1, 2, 3, 4):
            w.fv_kernel = kern
            s = Solver(w, mesh=mesh, rho_init=rho)
            assert s.info()["fv_kernel"] == kern
            s.step(40)
            assert s.status == 0
            got[kern] = tuple(s.fields()) + (s.patch_f(), s.force()[1])
            s.close()
        w.fv_kernel = 0
        s = Solver(w, mesh=mesh, rho_init=rho)
        info = s.info()
        assert info["fv_kernel"] == 4 and info["fv_depth"] == 2  # the deep kernel is the default where it applies
        s.close()
        for kern in (2, 3, 4):
            for a, b in zip(got[1], got[kern]):
                assert np.array_equal(a, b), (n_sub, kern)
        # every exchange interval, changed between steps (the tiles are rebuilt)
        w.fv_kernel = 4
        s = Solver(w, mesh=mesh, rho_init=rho)
        for depth in (1, 2, 4, 3, 2, 1, 4, 3):
            hlbm_set_fv_depth(s.h, depth)
            # the largest interval up to the one asked for that fits (FP64 records
            # take twice the shared memory)
            got_depth = s.info()["fv_depth"]
            assert got_depth == depth or (dtype == "f64" and 1 <= got_depth < depth)
            s.step(5)
        assert s.status == 0
        for a, b in zip(got[1], tuple(s.fields()) + (s.patch_f(), s.force()[1])):
            assert np.array_equal(a, b), (n_sub, "depths")
        s.close()


def _induced(dtype):
    w = inputs.workload("lamina-small-" + dtype)
    L = w.L
    w.motion, w.A, w.omega = inputs.MOTION_INDUCED, 0.0, 0.0
    w.mass = math.pi / 4 * L * L
    w.stiffness = w.mass * (2 * math.pi / 150.0) ** 2
    w.y0 = 1.5
    return w


def check_donors_valid(mesh, dY, tg, dg, to, do):
    """Refill records that may differ only at ties: the types agree, and a
    node whose donor triangle differs lies (to 1e-9) in both triangles, the
    point being its body-frame position shifted by the last displacement."""
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


@pytest.mark.parametrize("dtype,steps,tol_u,tol_rho,tol_y", [("f64", 80, 2e-9, 1e-12, 1e-10),
                                                            ("f32", 200, 3e-5, 1e-5, 1e-5)])
def test_parity_induced_motion(dtype, steps, tol_u, tol_rho, tol_y):
    """A spring-mounted lamina moved by the fluid force (oracle reading R11):
    the lamina's path and the fields against the oracle.  The path comes from
    the computed force, so the two sides' positions differ by rounding and a
    node on a triangle edge may take either triangle: FP64 compares classes
    bit for bit and checks that differing donors both contain the node.  In
    FP32 the force error moves the lamina (path within 1e-5 of its
    displacement), and the fields, compared node by node, carry that path
    difference on top of the 1e-5 of the prescribed-motion runs: 3e-5."""
    w, s, o = pair(_induced(dtype))
    for chunk in (1, steps // 2 - 1, steps // 2):
        s.step(chunk)
        o.step(chunk)
        if dtype == "f64":
            assert np.array_equal(s.struct_class(), o.struct_class())
            y, _ = o.motion()
            tg, dg = s.refill_record()
            to, do = o.refill_record()
            check_donors_valid(w.mesh(), y[o.time - 1] - y[o.time - 2] if o.time > 1 else 0.0, tg, dg, to, do)
    e = compare_fields(s, o, tol_u, tol_rho)
    y, v = o.motion()
    info = s.info()
    print(dtype, "induced errors", e, "path", abs(info["y"] - y[-1]), abs(info["vy"] - v[-1]))
    assert info["time"] == steps
    assert abs(info["y"] - y[-1]) < tol_y * abs(w.y0) and abs(info["vy"] - v[-1]) < tol_y * abs(w.y0)
    assert abs(y[-1] - w.y0) > 0.1  # it moved
    assert s.status == 0 and o.status == 0


def _exact_state(s):
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    tg, dg = s.refill_record()
    fx, fy = s.force()
    return dict(rs=rs, uxs=uxs, uys=uys, ru=ru, uxu=uxu, uyu=uyu, cls=s.struct_class(), tg=tg, dg=dg, fx=fx, fy=fy)


def test_overlap_of_the_far_lattice_changes_no_bit(tmp_path):
    """The next step's stream-collide away from the patch, run inside the FV
    launch (hlbm_set_overlap, on by default), gives the bits of the plain
    order: over a harmonic motion whose window moves, across single-step
    calls, and on through a checkpoint written while the precomputed part is
    pending."""
    from paper_2006_13631_gb300 import Solver, hlbm_set_overlap, hlbm_set_overlap_share

    w = inputs.workload("lamina-small-f32")
    mesh, rho = w.mesh(), w.rho_init()
    on = Solver(w, mesh=mesh, rho_init=rho)
    off = Solver(w, mesh=mesh, rho_init=rho)
    part = Solver(w, mesh=mesh, rho_init=rho)  # the FV launch streams the far part of 45 % of the rows
    hlbm_set_overlap(off.h, False)
    hlbm_set_overlap_share(part.h, 0.45)
    assert on.info()["fv_kernel"] == 4
    for k in (5, 1, 1, 3, 1, 9):
        on.step(k)
    off.step(20)
    part.step(13)
    part.step(7)
    a, b, c = _exact_state(on), _exact_state(off), _exact_state(part)
    for key in a:
        assert np.array_equal(a[key], b[key]), key
        assert np.array_equal(c[key], b[key]), key
    # a checkpoint taken now (the far part of step 20 is pending in `on`)
    path = str(tmp_path / "ck.bin")
    on.save(path)
    back = Solver(w, mesh=mesh, rho_init=rho)
    back.load(path)
    for s in (on, off, back):
        s.step(7)
    a, b, c = _exact_state(on), _exact_state(off), _exact_state(back)
    for key in a:
        assert np.array_equal(a[key], b[key]), key
        assert np.array_equal(a[key], c[key]), key
    assert on.status == 0 and off.status == 0 and back.status == 0


@pytest.mark.parametrize("dtype,tol_u,tol_rho", [("f64", 2e-9, 1e-12), ("f32", 1e-5, 1e-5)])
def test_parity_absorbing_outflow_layer(dtype, tol_u, tol_rho):
    """The non-reflecting outflow reading (an absorbing layer of 24 rows along
    the outflow sides y = 0 and ny - 1): the CUDA path (a layer kernel after
    each stream-collide, with the overlap of the far lattice on) against the
    oracle's R13 in the collision; classes and donors bit-exact.  The layer
    must change the fields against the plain outflow."""
    from paper_2006_13631_gb300 import Solver

    w = inputs.workload("lamina-small-f32")
    w.dtype = dtype
    w.sponge_rows, w.sponge_sigma = 24, 0.1
    mesh, rho = w.mesh(), w.rho_init()
    s = Solver(w, mesh=mesh, rho_init=rho)
    o = oracle.Oracle(w, mesh=mesh, rho_init=rho)
    for chunk in (3, 60, 57):
        s.step(chunk)
        o.step(chunk)
        compare_geometry(s, o)
    compare_fields(s, o, tol_u, tol_rho)
    w.sponge_rows, w.sponge_sigma = 0, 0.0
    plain = Solver(w, mesh=mesh, rho_init=rho)
    plain.step(120)
    r_layer, r_plain = s.fields()[0], plain.fields()[0]
    assert np.abs(r_layer[:24] - r_plain[:24]).max() > 1e-9
    assert s.status == 0

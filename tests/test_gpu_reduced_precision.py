"""Lattice populations stored as FP16 / BF16 deviations (FP32 arithmetic,
FP32 patch, FP64 force and fit) against the FP64 oracle: the physics of the
256^2 workload (tau 0.6, beta 500, KC 0.25) at 1024^2 with chord 32 over
four periods.  Geometry stays bit-exact; fields and the hydrodynamic
function carry the storage rounding, reported and bounded here."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reference():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13631_gb300.build import build

    build()
    w = inputs.workload("lamina-1024-f64")
    mesh = w.mesh()
    o = oracle.Oracle(w, mesh=mesh)
    o.step(w.steps)
    assert o.status == 0
    return w, mesh, o, o.struct_macro(), o.patch_macro(), o.gamma(1.0, 3.0)


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.mark.parametrize("dtype,tol_u,tol_theta", [("f32", 1e-5, 1e-5), ("f16", 2e-3, 1e-3), ("bf16", 1e-2, 5e-3)])
def test_reduced_storage_against_fp64_oracle(reference, dtype, tol_u, tol_theta):
    from paper_2006_13631_gb300 import Solver

    w0, mesh, o, (ro, uxo, uyo), (pr, pux, puy), (re_o, im_o, _) = reference
    w = inputs.workload(f"lamina-1024-{dtype}")
    s = Solver(w, mesh=mesh)
    s.step(w.steps)
    assert s.status == 0
    assert np.array_equal(s.struct_class(), o.struct_class())
    rs, uxs, uys, ru, uxu, uyu = s.fields()
    disc = o.struct_class() == oracle.DISC
    u_s = np.concatenate([uxs[disc], uys[disc]])
    u_o = np.concatenate([uxo[disc], uyo[disc]])
    e = dict(struct_u=_rel(u_s, u_o), patch_u=_rel(np.concatenate([uxu, uyu]), np.concatenate([pux, puy])),
             struct_drho=_rel(rs[disc] - 1.0, ro[disc] - 1.0))
    re_g, im_g, _ = s.gamma(1.0, 3.0)
    e["theta_re"] = abs(re_g - re_o) / abs(re_o)
    e["theta_im"] = abs(im_g - im_o) / abs(im_o)
    print(f"{dtype} storage vs FP64 oracle:", e, "theta", (re_g, im_g), "oracle", (re_o, im_o))
    assert e["struct_u"] < tol_u and e["patch_u"] < tol_u
    assert e["theta_re"] < tol_theta and e["theta_im"] < tol_theta

"""The C-ABI library loads and exports every entry point of include/hlbm.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(hlbm_[a-z_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2006_13631_gb300.build import build

    return build()


def test_every_declared_symbol_is_exported(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert "hlbm_create" in names and "hlbm_step" in names and "hlbm_gamma" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/hlbm.h but not exported"


def test_binding_declares_every_symbol(lib_path):
    from paper_2006_13631_gb300 import _native

    assert set(_declared()) == set(_native.SIGNATURES)


def test_create_rejects_bad_configuration_without_touching_the_gpu(lib_path):
    """Validation runs before any device work: an unstable FV sub-step
    (dt_u >= 2 tau_u, Sec. 7) is refused with HLBM_EINVAL and a message."""
    import numpy as np

    import inputs
    from paper_2006_13631_gb300 import hlbm as H

    w = inputs.workload("lamina-small-f32")
    m = w.mesh()
    grid = dict(nx=w.nx, ny=w.ny, dtype="f32")
    patch = dict(xy=m.xy, tri=m.tri, kind=m.kind, lamina_L=w.L, lamina_T=w.T, x_c=w.xc, y_c=w.yc,
                 delta_f=w.delta_f, n_sub=1, lumped=0)
    with pytest.raises(H.HLBMError) as e:
        H.hlbm_create(grid, patch, w.tau_s, dict(kind=1, A=w.A, omega=w.omega))
    assert e.value.code == -1 and "unstable" in str(e.value)
    patch["n_sub"] = w.n_sub
    patch["delta_f"] = 3.5  # outer boundary too close to the fictitious curve
    with pytest.raises(H.HLBMError) as e:
        H.hlbm_create(grid, patch, w.tau_s, dict(kind=1, A=w.A, omega=w.omega))
    assert e.value.code == -1 and "outer patch boundary" in str(e.value)
    np.testing.assert_equal(H.N.HLBM_EINVAL, -1)


def test_create_rejects_bad_levels_without_touching_the_gpu(lib_path):
    """The nested-level checks of hlbm_create run before any device work:
    even box sizes, a box without its margin (two nodes inside a level that
    has a ring of its own, one inside the coarsest), too many levels, and a
    level whose tau is 1 are refused with HLBM_EINVAL and a message."""
    import inputs
    from paper_2006_13631_gb300 import hlbm as H

    w = inputs.workload("lamina-small-f32")
    m = w.mesh()
    patch = dict(xy=m.xy, tri=m.tri, kind=m.kind, lamina_L=w.L, lamina_T=w.T, x_c=w.xc, y_c=w.yc,
                 delta_f=w.delta_f, n_sub=w.n_sub, lumped=0)
    motion = dict(kind=1, A=w.A, omega=w.omega)

    def refused(nx, levels, tau=w.tau_s, n_sub=None, text=""):
        grid = dict(nx=nx, ny=w.ny, dtype="f32",
                    levels=[dict(nx=a, ny=b, ox=c, oy=d) for a, b, c, d in levels])
        p = dict(patch, n_sub=n_sub or patch["n_sub"])
        with pytest.raises(H.HLBMError) as e:
            H.hlbm_create(grid, p, tau, motion)
        assert e.value.code == -1 and text in str(e.value), str(e.value)

    refused(202, [(204, 160, 51, 40)], text="odd sizes")
    refused(203, [(204, 160, 0, 40)], text="keep 1 node")
    refused(203, [(204, 160, 102, 40)], text="keep 1 node")
    # level 1 has a ring of its own (level 2 around it): two nodes of margin
    refused(203, [(211, 167, 1, 43), (216, 176, 53, 44)], text="keep 2 node")
    refused(203, [(210, 167, 52, 43), (216, 176, 53, 44)], text="odd sizes")
    refused(203, [(204, 160, 51, 40)] * 5, text="n_levels")
    refused(203, [(211, 167, 52, 43), (216, 176, 53, 44)], tau=2.5, n_sub=4, text="tau of level 2")


def test_create_rejects_a_bad_absorbing_layer_without_touching_the_gpu(lib_path):
    """The non-reflecting outflow's layer is checked before any device work:
    negative depth, a strength outside [0, 1), and a layer reaching half way
    across the lattice side it lies along are refused with HLBM_EINVAL."""
    import inputs
    from paper_2006_13631_gb300 import hlbm as H

    w = inputs.workload("lamina-small-f32")
    m = w.mesh()
    patch = dict(xy=m.xy, tri=m.tri, kind=m.kind, lamina_L=w.L, lamina_T=w.T, x_c=w.xc, y_c=w.yc,
                 delta_f=w.delta_f, n_sub=w.n_sub, lumped=0)
    motion = dict(kind=1, A=w.A, omega=w.omega)
    for rows, sigma in ((-1, 0.1), (10, 1.0), (10, -0.1), ((w.ny + 1) // 2, 0.1)):
        grid = dict(nx=w.nx, ny=w.ny, dtype="f32", sponge_rows=rows, sponge_sigma=sigma)
        with pytest.raises(H.HLBMError) as e:
            H.hlbm_create(grid, patch, w.tau_s, motion)
        assert e.value.code == -1 and "absorbing layer" in str(e.value), (rows, sigma)


def test_study_runner_prints_its_usage_without_points():
    """The chord-800 study runner (python -m paper_2006_13631_gb300.study)
    needs an output file and at least one point; without them it prints its
    usage and returns 2, touching no GPU."""
    from paper_2006_13631_gb300 import study

    assert study.main([]) == 2
    assert study.main(["out.json"]) == 2

"""The paper's parametric study (Sec. 2, Sec. 6) on the CUDA path: Theta at
the 35 (beta, eps) points, chord 32, domain 5L, FP64, against the values the
paper prints (tests/golden/paper_theta_mg_hlbm.txt) and eq. hydro_tot.  The
assertions are the physics the method must get right at any resolution
(signs, harmonic response, trends); the comparison with the paper's numbers
is printed (pytest -s) and recorded, not asserted."""
import os

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_13631_gb300.build import build

    build()


def test_theta_over_the_papers_parametric_study():
    from paper_2006_13631_gb300 import Solver

    d = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "paper_theta_mg_hlbm.txt"))
    rows = []
    for beta, eps, re_p, mim_p in d:
        w = inputs.paper_point_workload(beta, eps, L=32.0)
        s = Solver(w)
        s.step(w.steps)
        assert s.status == 0, (beta, eps)
        re, im, rms = s.gamma(1.0, 3.0)
        s.close()
        th = oracle.theta_semi_analytic(beta, eps)
        rows.append((beta, eps, re, -im, re_p, mim_p, th.real, -th.imag, rms))
    r = np.array(rows)
    print("\n beta   eps    Re     -Im    Re_paper -Im_paper Re_GD  -Im_GD  fit_rms")
    for x in r:
        print(" %5.0f %5.3f %6.4f %6.4f %6.4f %6.4f %6.4f %6.4f %.3f" % tuple(x))
    dre, dim = r[:, 2] / r[:, 4] - 1, r[:, 3] / r[:, 5] - 1
    print("Re vs paper: mean %+.3f max |.| %.3f; -Im vs paper: mean %+.3f max |.| %.3f"
          % (dre.mean(), np.abs(dre).max(), dim.mean(), np.abs(dim).max()))
    beta, eps, re, mim = r[:, 0], r[:, 1], r[:, 2], r[:, 3]
    # added mass and damping: Re > 0, Im < 0
    assert (re > 0).all() and (mim > 0).all()
    # the response is harmonic inside eq. betalimit: the sine fit leaves a small residual
    assert (r[:, 8] < 0.1).all()
    # trends where the amplitude spans at least 1.5 lattice spacings (eps L >= 1.5;
    # below that the per-step relocation of the patch adds a spurious damping
    # that dominates -Im at this chord)
    big = eps * 32.0 >= 1.5
    # Re(Theta) falls with beta at fixed eps (the Stokes-layer term of eq. hydro_gamma)
    for e in np.unique(eps[big]):
        sel = big & (eps == e)
        assert np.all(np.diff(re[sel]) < 0), e
    # the damping grows with the amplitude at fixed beta (eq. hydro_delta); at
    # beta = 20 that growth (0.06 from eps 0.05 to 0.1) is below this chord's error
    for b in np.unique(beta[big & (beta >= 50)]):
        sel = big & (beta == b)
        if sel.sum() > 1:
            assert mim[sel][-1] > mim[sel][0], b

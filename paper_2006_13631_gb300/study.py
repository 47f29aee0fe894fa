"""Theta at points of the paper's (beta, eps) study on its own setup (Sec. 5,
Sec. 6: chord 800, domain 5L x 5L, four structured levels, tau 0.8 at the
finest), one solver per point, four periods, the fit over the last three.

    python -m paper_2006_13631_gb300.study OUT.json BETA,EPS[,ROWS,SIGMA] ...

ROWS, SIGMA: the absorbing outflow layer (0 rows: the zero-gradient copy).
Each point prints one JSON line (Theta, the fit residual, the step count and
the wall time) and OUT.json collects them.
"""
import json
import sys
import time


def run_point(beta: float, eps: float, sponge_rows: int = 0, sponge_sigma: float = 0.0) -> dict:
    import inputs
    from . import Solver

    w = inputs.paper_point_levels_workload(beta, eps)
    w.sponge_rows, w.sponge_sigma = sponge_rows, sponge_sigma
    t0 = time.time()
    s = Solver(w)
    try:
        s.step(w.steps)
        re_, im_, rms = s.gamma(discard=1.0, fit=3.0)
        status = s.status
    finally:
        s.close()
    return dict(beta=beta, eps=eps, sponge_rows=sponge_rows, sponge_sigma=sponge_sigma, steps=w.steps, re=re_,
                im=im_, rms=rms, status=status, wall_s=time.time() - t0)


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) < 2:
        print(__doc__)
        return 2
    from .build import build

    build()
    out, results = argv[0], []
    for spec in argv[1:]:
        parts = spec.split(",")
        rows, sigma = (int(parts[2]), float(parts[3])) if len(parts) > 2 else (0, 0.0)
        r = run_point(float(parts[0]), float(parts[1]), rows, sigma)
        print(json.dumps(r), flush=True)
        results.append(r)
        with open(out, "w") as fh:
            json.dump(results, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Choose m0 for the synthetic workloads so that min |lambda(Q)| comes as close
as the field allows to a target (the stand-in for the paper's conditioning,
Sec. 4: "m0 such that we obtain a comparable conditioning").  Calls only the
oracle and the seeded input generator; writes tests/golden/workloads.json.

Grid search: min |lambda| is evaluated at each m0 of a grid (one process per
point) with the oracle's GD-lambda-AMG (two-level MG with GMRES smoothing,
Gamma5 form, sign-balanced block of 2, residual 1e-5 -- far below the
resolution the choice needs), and the grid point closest to the target wins.
The grid has two points, -0.80 and -0.85: the oracle's probes at -0.90 and
below did not finish within an hour (the near-critical spectrum slows GD
down).  The choice therefore rests on those two points only; the recorded
min_abs_lambda (5.5e-2 at -0.85, above the 1e-2 target) states what the
chosen m0 gives.  The larger workloads are tuned on dense proxies instead
(tune_m0_dense.py).

usage: python tests/golden/tune_m0.py <name> [<name> ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.dirac import WilsonClover  # noqa: E402
from oracle import gd, mg  # noqa: E402
from paper_2004_08146_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")

# lattice, eps, csw, seed, target min|lambda|, aggregate block, Nv
SPECS = {
    "c2_16x8c3": dict(dims=(16, 8, 8, 8), eps=0.5, csw=1.5, seed=1002, target=1e-2, block=(2, 2, 2, 2), nv=8,
                      grid=[-0.80, -0.85]),
}


def min_abs_lambda(U, dims, m0, csw, block, nv, seed):
    op = WilsonClover(U, m0, csw)
    h = mg.TwoLevelMG(op, block, block, nv, smoother='gmres', form='g5')
    W = h.setup(synth.spinor(dims, seed + 11, nvec=nv), iterations=3)
    N = op.n
    Q = lambda v: op.Q(v.reshape(dims + (4, 3))).reshape(-1)

    def corr(theta, r):
        x, it = h.solve(op.g5(r.reshape(dims + (4, 3))), theta, 1e-1, 5)
        return x.reshape(-1), it
    res = gd.gd_lambda_amg(Q, 2, W.reshape(nv, -1).T, synth.complex_gaussian((N, 2), seed + 12), corr,
                           m_min=12, m_max=24, eps=1e-5, block=2, max_outer=2000)
    return float(np.min(np.abs(res.lam)))


def _probe(args):
    name, m0 = args
    s = SPECS[name]
    dims = s["dims"]
    U = synth.gauge_field(dims, s["eps"], s["seed"])
    t = time.time()
    v = min_abs_lambda(U, dims, m0, s["csw"], s["block"], s["nv"], s["seed"])
    print(f"{name}: m0={m0:+.4f} min|lambda|={v:.6e} ({time.time() - t:.0f}s)", flush=True)
    return m0, v


def tune(name):
    import multiprocessing as mp
    s = SPECS[name]
    grid = s["grid"]
    with mp.get_context("spawn").Pool(len(grid)) as pool:
        res = pool.map(_probe, [(name, m0) for m0 in grid])
    target = s["target"]
    m0, v = min(res, key=lambda mv: (abs(np.log(mv[1] / target)), mv[1]))
    return dict(dims=list(s["dims"]), eps=s["eps"], csw=s["csw"], seed=s["seed"], m0=m0,
                min_abs_lambda=v, target=target, grid=[[a, b] for a, b in sorted(res)])


if __name__ == "__main__":
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in sys.argv[1:]:
        data[name] = tune(name)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
    print(json.dumps(data, indent=1))

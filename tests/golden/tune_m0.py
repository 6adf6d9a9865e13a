"""Choose m0 for the synthetic workloads so that min |lambda(Q)| hits a target
(the stand-in for the paper's conditioning, Table 1: "m0 such that we obtain a
comparable conditioning").  Calls only the oracle and the seeded input
generator; writes tests/golden/workloads.json.

Secant search on f(m0) = min|lambda|(m0) - target from the heavy side, where
min |lambda| grows roughly linearly with m0; steps are capped so that the
search never crosses to the critical side.  Each probe computes the two
smallest |lambda| with the oracle's GD-lambda-AMG (two-level MG with GMRES
smoothing, Gamma5 form, sign-balanced block of 2) to a 1e-5 residual, far
below the 10 % agreement with the target that the search asks for.

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
    "c2_16x8c3": dict(dims=(16, 8, 8, 8), eps=0.5, csw=1.5, seed=1002, target=1e-2, block=(2, 2, 2, 2), nv=8),
    "c5_16c4": dict(dims=(16, 16, 16, 16), eps=0.5, csw=1.5, seed=1005, target=1e-2, block=(2, 2, 2, 2), nv=8),
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
                           m_min=12, m_max=24, eps=1e-5, block=2, max_outer=400)
    return float(np.min(np.abs(res.lam)))


def tune(name):
    s = SPECS[name]
    dims = s["dims"]
    U = synth.gauge_field(dims, s["eps"], s["seed"])
    target = s["target"]
    cache = {}

    def f(m0):
        m0 = round(m0, 6)
        if m0 not in cache:
            t = time.time()
            cache[m0] = min_abs_lambda(U, dims, m0, s["csw"], s["block"], s["nv"], s["seed"])
            print(f"{name}: m0={m0:+.6f} min|lambda|={cache[m0]:.6e} ({time.time() - t:.0f}s)", flush=True)
        return cache[m0]

    a, b = 0.2, 0.0
    fa, fb = f(a) - target, f(b) - target
    for _ in range(12):
        if abs(fb) < 0.1 * target:
            break
        slope = (fb - fa) / (b - a) if b != a else 1.0
        step = -fb / slope if slope > 0 else -0.2
        step = max(min(step, 0.3), -0.3)
        if fb < 0:                      # overshot towards the critical side: back off
            step = abs(step) * 0.5
        a, fa = b, fb
        b = b + step
        fb = f(b) - target
    hi = b
    m0 = round(hi, 6)
    return dict(dims=list(dims), eps=s["eps"], csw=s["csw"], seed=s["seed"], m0=m0,
                min_abs_lambda=f(m0), target=target)


if __name__ == "__main__":
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in sys.argv[1:]:
        data[name] = tune(name)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
    print(json.dumps(data, indent=1))

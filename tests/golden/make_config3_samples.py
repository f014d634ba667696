"""Write config3_samples.json: sampled entries of the oracle's solutions of the Wilson
16^4 workload (eight kappa shifts), right-hand sides 1 and 2, for the full-size GPU
parity test.

The oracle's GMRES-DR(60,30)-Sh (Sec. 3, algorithm GMRES-DR-Sh) solves each right-hand
side to a relative residual of 1e-10 on every shift; its solution then agrees with the
exact one to about cond * 1e-10.  128 seeded indices of every solution are stored
(10 significant digits), with the solutions' 2-norms.  About ten minutes on 8 cores.

    python tests/golden/make_config3_samples.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import WilsonOperator, gmres_dr_sh  # noqa: E402

TOL = 1e-10
NSAMP = 128


def main():
    p = W.config(3)
    A = WilsonOperator(p.op[1], p.op[3], diag_a=p.op[2])
    idx = np.sort(np.random.default_rng(314).choice(p.n, size=NSAMP, replace=False))
    out = {"what": "oracle GMRES-DR(60,30)-Sh solutions of the Wilson 16^4 workload (eps 0.4, eight kappa shifts, "
                   "Z2 right-hand sides), sampled entries",
           "source": "oracle.gmres_dr_sh (Sec. 3, GMRES-DR-Sh), tol %g per shift" % TOL,
           "indices": idx.tolist(), "rhs": {}}
    for j in (0, 1):
        t = time.time()
        r = gmres_dr_sh(A.matvec, p.B[:, j], p.sigma, p.m, p.k, TOL)
        x = r["x"]
        out["rhs"][str(j)] = {
            "mvps": int(r["mvps"]), "seconds": round(time.time() - t, 1),
            "norm": [float(np.linalg.norm(x[:, i])) for i in range(len(p.sigma))],
            "re": [x[idx, i].real for i in range(len(p.sigma))],
            "im": [x[idx, i].imag for i in range(len(p.sigma))],
        }
        print(j, out["rhs"][str(j)]["mvps"], out["rhs"][str(j)]["seconds"], flush=True)
    with open(os.path.join(HERE, "config3_samples.json"), "w") as f:
        f.write(dumps(out))


def dumps(obj):
    """JSON with arrays of floats written to 10 significant digits."""
    if isinstance(obj, dict):
        return "{" + ", ".join(json.dumps(k) + ": " + dumps(v) for k, v in obj.items()) + "}"
    if isinstance(obj, np.ndarray):
        return "[" + ",".join("%.9e" % v for v in obj) + "]"
    if isinstance(obj, list):
        return "[" + ", ".join(dumps(v) for v in obj) + "]"
    return json.dumps(obj)


if __name__ == "__main__":
    main()

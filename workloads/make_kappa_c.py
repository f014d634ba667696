"""Write ``kappa_c.json``: the critical kappa of each synthetic Wilson lattice.

kappa_c = 1 / max Re lambda(H), with lambda(H) the eigenvalue of the hopping
matrix H of largest real part, measured by ARPACK (``which='LR'``) on the
oracle's operator.  The shift lists of configurations 2-4 are kappa values
from 0.115 up to 0.98 kappa_c.  This script uses only ``oracle/`` and this
package's own link generator.

    python -m workloads.make_kappa_c [cfg ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as spla

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W  # noqa: E402
from oracle import WilsonOperator  # noqa: E402


# ARPACK per lattice (tolerance, eigenvalues, Lanczos vectors): kappa_c only places the
# end of the shift list, so a few correct digits suffice on the big lattices (matvecs
# there cost seconds); on 24^3x32 asking for four values with 60 vectors ran for hours
# in the clustered edge of the spectrum, one value with 24 vectors at 1e-2 takes two
# minutes (its lambda_max follows the eps^2 trend of the smaller lattices to ~1%).
ARPACK = {2: (1e-6, 4, 60), 3: (1e-4, 4, 60), 4: (1e-2, 1, 24)}


def measure_kappa_c(dims, eps, cid, tol=1e-6, nev=4, ncv=60):
    links = W.su3_links(dims, eps, W.rng(cid, 0))
    op = WilsonOperator(dims, links)
    H = spla.LinearOperator((op.n, op.n), matvec=op.hop, dtype=np.complex128)
    v0 = np.ones(op.n, dtype=np.complex128)
    vals = spla.eigs(H, k=nev, which="LR", ncv=ncv, tol=tol, v0=v0, return_eigenvectors=False)
    lam = vals[np.argmax(vals.real)]
    return 1.0 / lam.real, complex(lam)


def main(cids):
    out = {}
    if os.path.exists(W.KAPPA_C_FILE):
        with open(W.KAPPA_C_FILE) as f:
            out = json.load(f)
    for cid in cids:
        dims, eps = W.WILSON_LATTICES[cid]
        t = time.time()
        tol, nev, ncv = ARPACK[cid]
        kc, lam = measure_kappa_c(dims, eps, cid, tol, nev, ncv)
        out[W.lattice_key(dims, eps, cid)] = kc
        print(f"cfg{cid} {dims} eps={eps}: lambda_max={lam:.10f} kappa_c={kc:.10f} ({time.time()-t:.0f}s)",
              flush=True)
        with open(W.KAPPA_C_FILE, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [2, 3, 4])

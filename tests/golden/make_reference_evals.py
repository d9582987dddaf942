"""Writes the FP64 oracle's eigenvalues for the full-size synthetic workloads.

Calls only the input generators (synth) and the oracle (oracle/): plain FP64
block Lanczos (b = 8, random pivot from the splitmix64 generator, residual
1e-8 * ||H||_inf), then the 8 lowest Ritz values, their true residuals and the
block count.  The GPU tests compare against these files at full size.

    python tests/golden/make_reference_evals.py kron_n2e6 kron_n2e6_c3 kron_n2e6_exact

A name ending in "_exact" is the same workload with unrounded entries (the
FP64 sums of the factor products: the matrix the factored operator applies).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import lanczos as OL  # noqa: E402
from oracle import pivot as OP  # noqa: E402
from oracle.spmm import norm_inf  # noqa: E402

B, NEV, TOL, SEED = 8, 8, 1e-8, 20221028


def main(names):
    for name in names:
        t0 = time.time()
        A = synth.kron_matrix(name)
        H = A.to_scipy()
        r = OL.block_lanczos(H, NEV, B, OP.random_pivot(A.n, B, SEED), tol=TOL, max_vectors=2000)
        out = {"workload": name, "n": A.n, "nnz": A.nnz, "b": B, "nev": NEV, "tol": TOL, "pivot_seed": SEED,
               "norm_inf": norm_inf(H), "converged": r.converged, "blocks": r.iters,
               "evals": [float(x) for x in r.evals], "resid": [float(x) for x in r.resid],
               "oracle_seconds": time.time() - t0}
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_fp64_oracle_evals.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["kron_n2e6", "kron_n2e6_c3"])

"""Record the oracle's own PCG iteration counts on the seeded workloads.

Test infrastructure: runs only the FP64 oracle (on inputs from the seeded
generators) and writes tests/golden/oracle_iterations.json.  The benchmark's
CPU legs time a bounded number of oracle iterations and scale the per-
iteration time by these counts.

    python oracle/count_iterations.py [grid ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import amg_oracle as O  # noqa: E402
from paper_1907_04417_gb300.hostsetup import inputs  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")


def main(grids):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for N in grids:
        P = inputs.anisotropic(N=N, nrhs=1)
        t0 = time.time()
        H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
        ts = time.time() - t0
        t0 = time.time()
        x, res = O.solve(H, P.B[:, 0], maxit=5000)
        tsol = time.time() - t0
        b = P.B[:, 0]
        data[f"aniso9_{N}x{N}"] = {
            "iters": res[0].iters, "converged": bool(res[0].converged), "relres": res[0].relres,
            "true_relres": float(np.linalg.norm(b - P.A @ x) / np.linalg.norm(b)),
            "levels": [l.A.shape[0] for l in H.levels], "opc": O.operator_complexity(H),
            "setup_s": ts, "solve_s": tsol, "rtol": 1e-8,
            "note": "FP64 oracle, zero initial guess, RHS seed 1002 uniform[-1,1]",
        }
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(N, data[f"aniso9_{N}x{N}"], flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [1024])

"""Record the oracle's own PCG iteration counts on the seeded workloads.

Test infrastructure: runs only the FP64 oracle (on inputs from the seeded
generators) and writes tests/golden/oracle_iterations.json.  The benchmark's
CPU legs time a bounded number of oracle iterations and scale the per-
iteration time by these counts.

    python oracle/count_iterations.py [--bootstrap] [--variant=SMOOTHER/KIND] [grid ...]

With --bootstrap the smooth vectors come from the oracle's own bootstrap
(Algorithm 1) on the seeded starts instead of the relaxed-vector recipe.
With --variant (gs/V, l1jacobi/K or gs/K) the preconditioner is that cycle
variant (Section 5: Gauss-Seidel smoothing, K-cycles) instead of the
l1-Jacobi V-cycle; the key gains the suffix _<smoother><kind>.

    python oracle/count_iterations.py --workload=poisson|jump|elasticity|cc

records the counts of the other seeded workloads at their full sizes (the
first right-hand side of each system): the 64^2 Poisson problem, the 128^3
jumping-coefficient problem, every member of the uneven elasticity batch and
the 512^2 cell-centred diffusion problem.
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


NU = 15  # testing-phase applications per bootstrap stage


def bootstrap_vectors(P, N):
    """The workload's smooth vectors from the oracle's own bootstrap
    (Algorithm 1): w_0 = 1, m - 1 stages on seeded starts, each vector then
    scaled to unit 2-norm."""
    agg = inputs.stage_aggregator(P.A, [4] * (P.levels - 1))
    W, rhos = O.bootstrap(P.A, np.ones(P.n), P.m, NU, agg, inputs.bootstrap_starts(P.n, P.m))
    return W / np.linalg.norm(W, axis=0), rhos


def main(grids, bootstrap=False, variant=None):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    smoother, kind = variant.split("/") if variant else ("l1jacobi", "V")
    for N in grids:
        P = inputs.anisotropic(N=N, nrhs=1)
        key = f"aniso9_{N}x{N}" + ("_bootstrap" if bootstrap else "") + (f"_{smoother}{kind}" if variant else "")
        note = "FP64 oracle, zero initial guess, RHS seed 1002 uniform[-1,1]"
        if variant:
            note += f"; cycle variant: smoother {smoother}, {kind}-cycle"
        if bootstrap:
            t0 = time.time()
            P.W, rhos = bootstrap_vectors(P, N)
            note += f"; smooth vectors from the oracle's bootstrap (nu {NU}, rho {rhos}, {time.time() - t0:.0f} s)"
        t0 = time.time()
        H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
        ts = time.time() - t0
        t0 = time.time()
        if variant:
            x, res = O.solve_variant(H, P.B[:, 0], maxit=5000, smoother=smoother, kind=kind)
        else:
            x, res = O.solve(H, P.B[:, 0], maxit=5000)
        tsol = time.time() - t0
        b = P.B[:, 0]
        data[key] = {
            "iters": res[0].iters, "converged": bool(res[0].converged), "relres": res[0].relres,
            "true_relres": float(np.linalg.norm(b - P.A @ x) / np.linalg.norm(b)),
            "levels": [l.A.shape[0] for l in H.levels], "opc": O.operator_complexity(H),
            "setup_s": ts, "solve_s": tsol, "rtol": 1e-8,
            "note": note,
        }
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(key, data[key], flush=True)


def record(data, key, P, note):
    t0 = time.time()
    H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    ts = time.time() - t0
    t0 = time.time()
    x, res = O.solve(H, P.B[:, 0], maxit=5000)
    tsol = time.time() - t0
    b = P.B[:, 0]
    data[key] = {
        "iters": res[0].iters, "converged": bool(res[0].converged), "relres": res[0].relres,
        "true_relres": float(np.linalg.norm(b - P.A @ x) / np.linalg.norm(b)),
        "levels": [l.A.shape[0] for l in H.levels], "opc": O.operator_complexity(H),
        "setup_s": ts, "solve_s": tsol, "rtol": 1e-8, "note": note,
    }
    json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
    print(key, data[key], flush=True)


def main_workload(which):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    if which == "poisson":
        P = inputs.poisson(N=64, nrhs=1)
        record(data, P.name, P, "FP64 oracle, zero initial guess, first RHS (seed 1001, uniform[-1,1])")
    elif which == "jump":
        P = inputs.jumping3d(N=128, nrhs=32)
        record(data, P.name, P, "FP64 oracle, zero initial guess, first of the 32 RHS (seed 1003, standard normal)")
    elif which == "cc":
        P = inputs.diffusion_cc(N=512, nrhs=8)
        record(data, P.name, P, "FP64 oracle, zero initial guess, first of the 8 RHS (seed 1005, uniform[-1,1])")
    elif which == "elasticity":
        for s, P in enumerate(inputs.elasticity_batch()):
            record(data, f"{P.name}_member{s}", P,
                   f"FP64 oracle, zero initial guess, first RHS of batch member {s} (seed {1004 + 100 * s})")
    else:
        raise SystemExit(f"unknown workload {which}")


if __name__ == "__main__":
    wl = next((a.split("=", 1)[1] for a in sys.argv[1:] if a.startswith("--workload=")), None)
    if wl:
        main_workload(wl)
        sys.exit(0)
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    var = next((a.split("=", 1)[1] for a in sys.argv[1:] if a.startswith("--variant=")), None)
    main([int(a) for a in args] or [1024], bootstrap="--bootstrap" in sys.argv, variant=var)

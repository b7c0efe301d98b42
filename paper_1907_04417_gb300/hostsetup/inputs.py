"""Seeded synthetic workloads: operator, aggregate maps, smooth vectors, RHS.

One function per workload family; each returns an ``AMGProblem`` that the
GPU library and the oracle both consume unchanged.  Seeds (numpy PCG64):
right-hand sides 1000 + c, coefficient fields 2000 + c, smooth vectors
3000 + c, target fields 4000 + c, for workload c.

The aggregates come from the pairwise hierarchy built on the first smooth
vector w_0 (Section 5 composes consecutive pairwise prolongators of the first
hierarchy of the bootstrap, which is built on w_0).

Workloads (sizes are the full ones; every builder takes a smaller size for
tests):

1. 2D Poisson, 5-point, 64 x 64 interior, m = 1 (constant perturbed by
   U(-1e-2, 1e-2)), aggregates of 4 (two pairwise steps), 3 levels.
2. Rotated anisotropic diffusion, eps = 1e-3, theta = pi/6, 9-point,
   1024 x 1024, m = 4, aggregates of up to 16 (four pairwise steps), 5 levels.
3. 3D jumping coefficient, 7-point, 128^3, k per 8^3 block log-uniform in
   [1e-3, 1e3], m = 3, aggregates of up to 16, levels until <= 1024 coarse dofs.
4. 3D Navier-Cauchy elasticity (E = 1, nu = 0.3, clamped x = 0 face), 3 dofs
   per node, m = 6, aggregates of up to 32 dofs; a batch of 8 grids with
   sides drawn from {32, 40, 48, 64}, 4 RHS each, all with the same depth.
5. Cell-centred 2D diffusion, 512 x 512 cells, log-normal (sigma = 1) k,
   m = 3, aggregates of up to 16, 8 RHS, smooth target field.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import aggregation, problems, smooth


@dataclass
class AMGProblem:
    name: str
    A: sp.csr_matrix
    aggs: list            # aggs[k][node] = level-(k+1) aggregate of level-k node
    n_nodes: list         # nodes per level, n_nodes[0] = n
    W: np.ndarray         # (n, m) float64, unit-2-norm columns
    B: np.ndarray         # (n, k) float64 right-hand sides, row-major
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.A.shape[0]

    @property
    def m(self):
        return self.W.shape[1]

    @property
    def levels(self):
        return len(self.aggs) + 1


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _levels_until(A, w, steps, m, max_coarse=1024, max_levels=12):
    """Compose ``steps`` pairwise steps per level, adding levels until
    m * (number of aggregates) <= max_coarse.  A level whose steps shrink the
    node count by less than half of 2^steps is completed by merging its
    single-node aggregates into neighbouring ones."""
    aggs, n_nodes = [], [A.shape[0]]
    Ak, wk = A, np.asarray(w, dtype=np.float64)
    while len(aggs) < max_levels - 1:
        A0, w0 = Ak, wk
        comp = np.arange(Ak.shape[0])
        for _ in range(steps):
            if Ak.shape[0] <= 1:
                break
            agg, Ak, wk = aggregation.pairwise_step(Ak, wk)
            comp = agg[comp]
        if A0.shape[0] > 2 and A0.shape[0] < 2 ** (steps - 1) * Ak.shape[0]:
            comp = aggregation.merge_singletons(A0, comp)
            Ak, wk = aggregation.aggregate_operator(A0, w0, comp)
        aggs.append(comp.astype(np.int32))
        n_nodes.append(int(Ak.shape[0]))
        if m * Ak.shape[0] <= max_coarse or Ak.shape[0] <= 2:
            break
    return aggs, n_nodes


def poisson(N=64, nrhs=1, cfg=1):
    A = problems.poisson5(N)
    W = smooth.smooth_vectors(A, 1, 3000 + cfg, w0_perturb=1e-2)
    aggs, n_nodes = aggregation.aggregate_hierarchy(A, W[:, 0], [2, 2])
    B = _rng(1000 + cfg).uniform(-1.0, 1.0, size=(A.shape[0], nrhs))
    return AMGProblem(f"poisson5_{N}x{N}", A, aggs, n_nodes, W, B,
                      {"grid": N, "stencil": "5-point"})


def anisotropic(N=1024, nrhs=1, m=4, levels=5, eps=1e-3, theta=np.pi / 6, cfg=2):
    A = problems.aniso9(N, eps, theta)
    W = smooth.smooth_vectors(A, m, 3000 + cfg)
    aggs, n_nodes = aggregation.aggregate_hierarchy(A, W[:, 0], [4] * (levels - 1))
    B = _rng(1000 + cfg).uniform(-1.0, 1.0, size=(A.shape[0], nrhs))
    return AMGProblem(f"aniso9_{N}x{N}", A, aggs, n_nodes, W, B,
                      {"grid": N, "stencil": "9-point", "eps": eps, "theta": theta})


def jumping3d(N=128, nrhs=32, m=3, cfg=3, max_coarse=1024):
    A, _ = problems.jump7(N, 8, seed=2000 + cfg)
    W = smooth.smooth_vectors(A, m, 3000 + cfg)
    aggs, n_nodes = _levels_until(A, W[:, 0], 4, m, max_coarse)
    B = _rng(1000 + cfg).standard_normal((A.shape[0], nrhs))
    return AMGProblem(f"jump7_{N}^3", A, aggs, n_nodes, W, B,
                      {"grid": N, "stencil": "7-point", "block": 8})


def elasticity_grid(N, nrhs=4, m=6, levels=5, seed=3004, rhs_seed=1004):
    A = problems.elasticity(N)
    W = smooth.smooth_vectors(A, m, seed)
    steps = [5] + [3] * (levels - 2)
    aggs, n_nodes = aggregation.aggregate_hierarchy(A, W[:, 0], steps)
    B = _rng(rhs_seed).standard_normal((A.shape[0], nrhs))
    return AMGProblem(f"elasticity_{N}^3", A, aggs, n_nodes, W, B, {"grid": N})


def elasticity_batch(n_sys=8, sides=(32, 40, 48, 64), nrhs=4, m=6, levels=5, cfg=4):
    """The uneven batch: grid sides drawn (seeded) from ``sides``."""
    pick = _rng(3000 + cfg).choice(np.asarray(sides), size=n_sys)
    return [elasticity_grid(int(N), nrhs, m, levels, seed=3000 + cfg + 100 * s,
                            rhs_seed=1000 + cfg + 100 * s)
            for s, N in enumerate(pick)]


def diffusion_cc(N=512, nrhs=8, m=3, cfg=5, max_coarse=1024):
    k = problems.lognormal_field(N, 1.0, seed=2000 + cfg)
    A = problems.cc5(N, k)
    W = smooth.smooth_vectors(A, m, 3000 + cfg)
    aggs, n_nodes = _levels_until(A, W[:, 0], 4, m, max_coarse)
    B = _rng(1000 + cfg).uniform(-1.0, 1.0, size=(A.shape[0], nrhs))
    c = _rng(4000 + cfg).standard_normal((3, 3))
    x = (np.arange(N) + 0.5) / N
    S = np.sin(np.pi * np.outer(np.arange(1, 4), x))        # (3, N)
    target = np.einsum("pq,pi,qj->ij", c, S, S).ravel()
    Xt = np.repeat(target[:, None], nrhs, axis=1)
    return AMGProblem(f"cc5_{N}x{N}", A, aggs, n_nodes, W, B,
                      {"grid": N, "kcell": k, "x_target": Xt})


def bootstrap_starts(n, m, cfg=2):
    """Seeded start vectors of the bootstrap's testing phase (Algorithm 1):
    one standard-normal vector per stage r = 1..m-1 (numpy PCG64 seed
    5000 + 10 cfg + r).  The random numbers the method draws, as input."""
    return [_rng(5000 + 10 * cfg + r).standard_normal(n) for r in range(1, m)]


def stage_aggregator(A, steps):
    """Aggregates of a bootstrap stage: the composed pairwise steps of the
    compatible weighted matching on the stage's vector (Section 3)."""
    return lambda w: aggregation.aggregate_hierarchy(A, w, list(steps))

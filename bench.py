#!/usr/bin/env python
"""Time to a 1e-8 relative residual per right-hand side for the AMG-PCG
solve of the rotated anisotropic diffusion problem (eps = 1e-3, theta =
pi/6, 9-point, 1024 x 1024, 4 smooth vectors from the seeded bootstrap of
Algorithm 1, aggregates of 16, 5 levels).

One step = one complete batched solve (float32 V-cycle inside CG whose
vectors are double-float pairs and whose scalars are float64) of ``--batch``
seeded uniform[-1, 1] right-hand sides from a zero initial guess, with inputs
resident in HBM.  The plain float64 solve of one RHS is timed beside it.  The
bootstrap (testing phase on the device) and the setup are not timed.  Prints
one JSON line (rank 0).

    python bench.py [--gpus N --steps K --warmup W --impl gb300|reference]

Under torchrun every rank runs an independent replica on its own GPU with
its own right-hand sides (weak scaling, no collective on the data path); the
timed region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms to 1e-8 rel. residual per RHS (FP32-cycle batched AMG-PCG)"
UNIT = "ms/RHS"
L2_BYTES = 129e6


def l2_note(nnz, n, batch):
    """How the timed region avoids warm-L2 results: the operands' sizes."""
    vec = n * batch * 8
    sizes = f"A {nnz * 12 / 1e6:.0f} MB f64 + {nnz * 8 / 1e6:.0f} MB f32, each vector block {vec / 1e6:.0f} MB"
    if vec > L2_BYTES:
        return f"inputs larger than L2 ({sizes})"
    return f"vector blocks smaller than L2 ({sizes}); not flushed between steps"


NU_BOOT = 15  # testing-phase applications per bootstrap stage (Algorithm 1)


def workload(N, smooth="bootstrap"):
    sv = ("smooth vectors from the seeded bootstrap (Algorithm 1, nu=15, symmetrized)" if smooth == "bootstrap"
          else "relaxed random smooth vectors")
    return f"aniso9 eps=1e-3 theta=pi/6, {N}x{N} (n={N * N}), m=4, aggregates of 16, 5 levels, {sv}"
PEAK_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--smooth", default="bootstrap", choices=["bootstrap", "relaxed"],
                    help="smooth vectors: the seeded bootstrap of Algorithm 1 (testing phase on the "
                         "device; the oracle arm runs its own), or the relaxed random vectors")
    ap.add_argument("--maxit", type=int, default=5000)
    ap.add_argument("--roofline-kernel", default="auto")
    ap.add_argument("--tune-cache", default=None,
                    help="file of tuned launch choices: read when it has this workload, else written "
                         "(so that a profiled run replays the choices of a plain run)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", action="store_true",
                    help="also time the float64 cycle variants (Gauss-Seidel smoother, K-cycle) on the "
                         "same block, with the level-0 Gauss-Seidel sweep's roofline and an oracle sample")
    ap.add_argument("--cpu-sample-s", type=float, default=12.0)
    ap.add_argument("--profile-kernels", action="store_true",
                    help="also time every kernel family once (eager launches)")
    return ap.parse_args()


# ------------------------------------------------------------------ dist --
def dist_init(backend="nccl"):
    """Join the process group of a torchrun launch (one replica per GPU)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rhs_block(P, batch, rank):
    """The right-hand sides of one replica: seeded uniform[-1, 1], distinct
    per rank; rank 0's first column is the workload's own RHS."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(1002 + 7919 * rank))
    B = rng.uniform(-1.0, 1.0, size=(P.n, batch))
    if rank == 0:
        B[:, 0] = P.B[:, 0]
    return B


def whole_job_ms_per_rhs(max_elapsed_ms, steps, batch, ws):
    """Weak scaling: every rank solves ``batch`` RHS per step; the job's time
    per step is the slowest rank's."""
    return max_elapsed_ms / steps / (batch * ws)


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.index)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- helpers --
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return PEAK_FALLBACK_GBS, "fallback"


def kernel_source_hash():
    """Hash of the device code of the level-0 solve kernels: the shared
    kernel header, the launchers, and the kernels at the head of
    amg_solve.cu (everything before its host-side workspace).  Stored
    traffic counts only while this hash is unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1907_04417_gb300", "csrc")
    for f in ("amg_kernels.cuh", "amg_launch.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    src = open(os.path.join(csrc, "amg_solve.cu"), "rb").read()
    h.update(src[:src.index(b"struct Workspace {")])
    return h.hexdigest()[:16]


def stored_traffic(kernel, workload_key):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(f"{kernel}|{workload_key}")
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return float(e["bytes_per_launch"])


def algorithmic_bytes(kernel, lv, K, wc):
    """Minimal bytes one launch of a level-0 kernel must move (see the
    roofline section of the design notes): matrix arrays once, each vector
    block once per read or write, prolongator blocks once."""
    n0, nnz0, n1, npv = lv["n0"], lv["nnz0"], lv["n1"], lv["npv1"]
    if kernel == "spmv_cg":      # q = A p (A as a float pair, p float32, q a float pair), p.q
        return nnz0 * 12 + 4 * (n0 + 1) + n0 * K * 4 + n0 * K * 8
    if kernel == "restrict_l0":  # t = f - A u, fc = P^T t, uc = D^-1 fc
        return nnz0 * (wc + 4) + 4 * (n0 + 1) + 2 * n0 * K * wc + npv * wc + n1 * (2 * K * wc + wc)
    if kernel == "smooth_l0":    # z = u + D^-1 (f - A u), r.z
        return nnz0 * (wc + 4) + 4 * (n0 + 1) + n0 * wc + 2 * n0 * K * wc + 2 * n0 * K * 8
    if kernel == "prolong_l0":   # u += P uc
        return npv * wc + n1 * K * wc + 2 * n0 * K * wc
    if kernel == "cg_update":    # x += a p, r -= a q, ||r||, u0 = D^-1 r, f0 = r
        return 6 * n0 * K * 8 + n0 * 8 + (2 if wc == 4 else 1) * n0 * K * wc
    raise KeyError(kernel)


KERNEL_IDS = {"spmv_cg": 1, "restrict_l0": 2, "smooth_l0": 3, "prolong_l0": 4, "cg_update": 5}
KERNEL_GS_L0 = 6

# q = A p in double-float is bound by float32 arithmetic: per stored non-zero
# and column the multiply-accumulate of a float pair by a float32 takes 11
# float32 operations (exact product 2, low-part product 1, two-sum 6, error
# accumulation 2); per row and column the renormalisation (3) and the
# double-float p.q step (11) follow.  Peak: 152 SMs x 128 float32 lanes x
# 2.07 GHz (the maximum SM clock) = 40.3e12 lane operations per second.
ALU_OPS_PER_NZ_COL = 11
ALU_OPS_PER_ROW_COL = 14
ALU_PEAK_OPS = 152 * 128 * 2.07e9


def alu_ops(kernel, lv, K):
    if kernel == "spmv_cg":
        return lv["nnz0"] * K * ALU_OPS_PER_NZ_COL + lv["n0"] * K * ALU_OPS_PER_ROW_COL
    return None


def gs_sweep_bytes(lv, K):
    """Minimal bytes of one level-0 Gauss-Seidel sweep over all colours:
    the matrix once (8-byte values, 4-byte columns, row pointers), colour and
    diagonal once per row, f read, u read and written once (float64)."""
    n0, nnz0 = lv["n0"], lv["nnz0"]
    return nnz0 * 12 + 4 * (n0 + 1) + n0 * 12 + 3 * n0 * K * 8


VARIANTS = [("l1jacobi", "V"), ("gs", "V"), ("l1jacobi", "K"), ("gs", "K")]


def time_variants(amg, Hd, Bd, Xd, B, A, lv, K, maxit, peak, stream):
    """Float64 solves of the block with each cycle variant: device time per
    RHS (CUDA events on the launching stream, after a warm-up solve that
    builds the colouring, workspace and graph), iteration counts, true
    residuals, and for Gauss-Seidel the level-0 sweep's achieved bandwidth."""
    import numpy as np
    import torch
    out = {}
    for sm, kind in VARIANTS:
        o = amg.opts(cycle_precision=64, maxit=maxit, smoother=1 if sm == "gs" else 0,
                     cycle=1 if kind == "K" else 0)
        Xd.zero_()
        Hd.solve(Bd, Xd, o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        Xd.zero_()
        e0.record(stream)
        _, infos, st = Hd.solve(Bd, Xd, o)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        Xc = Xd.cpu().numpy()
        rel = float(max(np.linalg.norm(B[:, c] - A @ Xc[:, c]) / np.linalg.norm(B[:, c]) for c in range(K)))
        its = [i["iters"] for i in infos]
        ent = {"ms_per_rhs": ms / K, "iters_min": int(min(its)), "iters_max": int(max(its)),
               "true_relres_max": rel, "status": int(st)}
        if sm == "gs":
            Hd.timer_enable(KERNEL_GS_L0)
            Xd.zero_()
            Hd.solve(Bd, Xd, o)
            kms, kn = Hd.timer_read()
            Hd.timer_enable(0, False)
            nb = gs_sweep_bytes(lv, K)
            avg = kms / max(kn, 1)
            gbs = nb / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
            ent["gs_sweep_l0"] = {"avg_ms": avg, "sweeps": kn, "algorithmic_bytes": nb, "achieved_gbs": gbs,
                                  "peak_gbs": peak, "frac": gbs / peak, "ncolours": Hd.level_colours(0)[1]}
        out[f"{sm}/{kind}"] = ent
    return out


def oracle_variant_sample(P, W, smoother, kind, iters_needed, budget_s):
    """The oracle's PCG with a cycle variant, timed for about ``budget_s``
    seconds on the same workload and scaled to ``iters_needed``."""
    from oracle import amg_oracle as O
    H = O.setup(P.A, P.aggs, P.n_nodes, W)
    b = P.B[:, 0]
    pc = lambda r: O.cycle(H, r, smoother=smoother, kind=kind)  # noqa: E731
    if smoother == "gs":
        O.gs_data(H)  # the colouring is setup, not timed
    t0 = time.perf_counter()
    O.pcg(P.A, b, pc, fixed_iters=1)
    t1 = time.perf_counter() - t0
    k = max(2, int(budget_s / max(t1, 1e-3)))
    t0 = time.perf_counter()
    O.pcg(P.A, b, pc, fixed_iters=k)
    dt = time.perf_counter() - t0
    return {"ms_per_rhs": dt / k * iters_needed * 1e3, "sample_iters": k, "sample_s": dt, "cores": 1}


# ------------------------------------------------------------ CPU legs --
def oracle_sample(P, W, iters_needed, budget_s):
    """Time the oracle's PCG iterations on the same workload (setup not
    timed) for about ``budget_s`` seconds; scale to ``iters_needed``.  W are
    smooth vectors from the input recipe: the cost of an iteration depends on
    the hierarchy's sizes, not on the vectors' values."""
    from oracle import amg_oracle as O
    H = O.setup(P.A, P.aggs, P.n_nodes, W)
    b = P.B[:, 0]
    t0 = time.perf_counter()
    r1 = O.pcg(P.A, b, lambda r: O.vcycle(H, r), fixed_iters=1)
    t1 = time.perf_counter() - t0
    k = max(2, int(budget_s / max(t1, 1e-3)))
    t0 = time.perf_counter()
    O.pcg(P.A, b, lambda r: O.vcycle(H, r), fixed_iters=k)
    dt = time.perf_counter() - t0
    per_it = dt / k
    return {"per_iter_s": per_it, "sample_iters": k, "sample_s": dt,
            "ms_per_rhs": per_it * iters_needed * 1e3, "_first": r1.iters}


def stored_oracle_iters(N, smooth="relaxed"):
    p = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    if os.path.exists(p):
        d = json.load(open(p)).get(f"aniso9_{N}x{N}" + ("_bootstrap" if smooth == "bootstrap" else ""))
        if d:
            return int(d["iters"])
    return None


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_1907_04417_gb300.hostsetup import inputs
    P = inputs.anisotropic(N=args.grid, nrhs=1)
    iters = stored_oracle_iters(args.grid, args.smooth)
    from oracle import amg_oracle as O
    if args.smooth == "bootstrap":  # the oracle's own bootstrap on the seeded starts (untimed)
        from oracle.count_iterations import bootstrap_vectors
        P.W, _ = bootstrap_vectors(P, args.grid)
    H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
    b = P.B[:, 0]
    k = 3
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.pcg(P.A, b, lambda r: O.vcycle(H, r), fixed_iters=k)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt / k)
    per_it = statistics.median(times)
    if iters is None:
        res = O.pcg(P.A, b, lambda r: O.vcycle(H, r), maxit=args.maxit)
        iters = res.iters
    val = per_it * iters * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_it * k * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload(args.grid, args.smooth), "rhs_per_step": 1},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{k} FP64 oracle PCG iterations per step on the same workload "
                                       f"(setup untimed), scaled to the oracle's {iters} iterations"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- main --
def main():
    args = parse()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.tune_cache:
        os.environ["AMG_TUNE_CACHE"] = args.tune_cache
    import numpy as np
    import torch

    from paper_1907_04417_gb300 import amg, build
    from paper_1907_04417_gb300.hostsetup import inputs

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_gen = time.time()
    P = inputs.anisotropic(N=args.grid, nrhs=1)
    B = rhs_block(P, args.batch, rank)
    t_gen = time.time() - t_gen
    W_recipe = P.W
    boot = None
    if args.smooth == "bootstrap":
        # Algorithm 1 with the testing phase on the device (setup, untimed)
        from paper_1907_04417_gb300 import bootstrap as boot_mod
        t_b = time.time()
        Wb, rhos, Hs = boot_mod.bootstrap(P.A, np.ones(P.n), P.m, NU_BOOT,
                                          inputs.stage_aggregator(P.A, [4] * (P.levels - 1)),
                                          inputs.bootstrap_starts(P.n, P.m))
        for h in Hs:
            h.close()
        P.W = Wb / np.linalg.norm(Wb, axis=0)
        boot = {"nu": NU_BOOT, "rho": rhos, "setup_s": time.time() - t_b}

    A = P.A
    Hd = amg.Hierarchy((torch.from_numpy(A.indptr).to(dev), torch.from_numpy(A.indices).to(dev),
                        torch.from_numpy(A.data).to(dev)), P.aggs, P.n_nodes, torch.from_numpy(P.W).to(dev))
    info_h = Hd.info()
    Bd = torch.from_numpy(B).to(dev)
    Xd = torch.zeros_like(Bd)
    o32 = amg.opts(cycle_precision=32, maxit=args.maxit)
    o64 = amg.opts(cycle_precision=64, maxit=args.maxit)
    stream = torch.cuda.current_stream()

    def solve_batch():
        Xd.zero_()
        return Hd.solve(Bd, Xd, o32)

    # warm-up (also builds the graphs and workspaces)
    for _ in range(args.warmup):
        _, infos, st = solve_batch()
    torch.cuda.synchronize()

    # roofline kernel: auto = the level-0 kernel with the largest share
    rk = args.roofline_kernel
    shares = None
    if rk == "auto" or args.profile_kernels:
        shares = {}
        for name, kid in KERNEL_IDS.items():
            Hd.timer_enable(kid)
            solve_batch()
            ms, n = Hd.timer_read()
            shares[name] = {"ms_total": ms, "launches": n}
        Hd.timer_enable(0, False)
        if rk == "auto":
            rk = max(shares, key=lambda k: shares[k]["ms_total"])

    # one untimed solve with the kernel timer on (its graph is captured here)
    Hd.timer_enable(KERNEL_IDS[rk])
    solve_batch()
    torch.cuda.synchronize()
    # timed region: device time with CUDA events on the launching stream
    Hd.timer_enable(KERNEL_IDS[rk])
    l0 = amg.kernel_launches()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as cs:
        e0.record(stream)
        iters = []
        for _ in range(args.steps):
            _, infos, st = solve_batch()
            iters.append([i["iters"] for i in infos])
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    launches = amg.kernel_launches() - l0
    kms, kn = Hd.timer_read()
    Hd.timer_enable(0, False)
    elapsed = e0.elapsed_time(e1)
    elapsed = max_over_ranks(elapsed, ws)
    per_step = elapsed / args.steps
    value_job = whole_job_ms_per_rhs(elapsed, args.steps, args.batch, ws)
    print(f"[bench] timed {args.steps} steps: {per_step:.1f} ms/step, iters {iters[0][:4]}..., "
          f"kernel {rk}: {kms:.2f} ms over {kn} launches, gpu launches {launches}", file=sys.stderr, flush=True)
    if shares is not None:
        print(f"[bench] kernel shares {shares}", file=sys.stderr, flush=True)
    Xc = Xd.cpu().numpy()
    true_rel = float(max(np.linalg.norm(B[:, c] - A @ Xc[:, c]) / np.linalg.norm(B[:, c]) for c in range(args.batch)))

    # plain float64 solve of one RHS
    b1 = Bd[:, :1].contiguous()
    x1 = torch.zeros_like(b1)
    Hd.solve(b1, x1, o64)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nrep = 2
    f0.record(stream)
    for _ in range(nrep):
        x1.zero_()
        _, inf64, _ = Hd.solve(b1, x1, o64)
    f1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = f0.elapsed_time(f1) / nrep
    x64 = x1.cpu().numpy()[:, 0]
    # the float32-cycle solution of the same RHS against the float64 one
    err32 = float(np.linalg.norm(Xc[:, 0] - x64) / np.linalg.norm(x64))

    # end to end through the C ABI with host (pinned) buffers
    Bh = torch.from_numpy(B).pin_memory()
    Xh = torch.zeros_like(Bh).pin_memory()
    Hd.solve(Bh, Xh, o32)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    g0.record(stream)
    for _ in range(2):
        Xh.zero_()
        Hd.solve(Bh, Xh, o32)
    g1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(g0.elapsed_time(g1) / 2, ws)

    # roofline of the chosen kernel
    ex1 = Hd.export_level(1)
    lv = {"n0": P.n, "nnz0": A.nnz, "n1": ex1["n"], "npv1": int(ex1["pval"].size)}
    wc = 4
    abytes = algorithmic_bytes(rk, lv, args.batch, wc)
    avg_ms = kms / max(kn, 1)
    peak, peak_kind = peaks()
    achieved = abytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": stored_traffic(rk, f"aniso{args.grid}_K{args.batch}"), "kernel": rk,
            "peak_source": f"{peak_kind} hbm_gbs (burst copy)", "algorithmic_bytes_per_launch": abytes,
            "avg_launch_ms": avg_ms, "launches_timed": kn}
    ops = alu_ops(rk, lv, args.batch)
    if ops is not None and avg_ms > 0:
        # the double-float q = A p: float32 arithmetic bounds it (DRAM runs at
        # under half of the copy peak); its HBM figures stay beside it
        aa = ops / (avg_ms * 1e-3) / 1e12
        roof.update({"bound": "alu", "achieved": aa, "peak": ALU_PEAK_OPS / 1e12,
                     "unit": "T float32 ops/s", "frac": aa * 1e12 / ALU_PEAK_OPS,
                     "peak_source": "derived: 152 SMs x 128 float32 lanes x 2.07 GHz",
                     "alu_ops_per_launch": ops, "hbm_achieved_gbs": achieved, "hbm_peak_gbs": peak,
                     "hbm_frac": achieved / peak})

    line = {"metric": METRIC, "value": value_job, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-cycle/f64-cg", "data": "synthetic",
            "config": {"workload": workload(args.grid, args.smooth), "rhs_per_step_per_gpu": args.batch, "rtol": 1e-8,
                       "l2": l2_note(P.A.nnz, P.n, args.batch),
                       "parallelism": f"replicas x{ws}"},
            "clocks": cs.summary(), "gpu_launches": launches,
            "e2e": {"value": e2e_ms / (args.batch), "unit": UNIT,
                    "h2d_bytes_per_step": int(2 * P.n * args.batch * 8),
                    "d2h_bytes_per_step": int(P.n * args.batch * 8)},
            "roofline": roof,
            "fp64_plain": {"ms_per_rhs": fp64_ms, "iters": inf64[0]["iters"]},
            "fp32_batched_iters": {"min": int(np.min(iters)), "max": int(np.max(iters))},
            "fp32_vs_fp64_rel_err": err32, "true_relres_max": true_rel,
            "speedup_batched_vs_fp64_plain": fp64_ms / value_job if value_job else None,
            "hierarchy": {"levels": info_h["levels"], "n": info_h["n_level"], "nnz": info_h["nnz_level"],
                          "opc": info_h["opc"]},
            "input_gen_s": t_gen, "bootstrap": boot}
    if shares is not None:
        line["kernel_ms_per_solve"] = shares
    if args.variants:
        var = time_variants(amg, Hd, Bd, Xd, B, A, lv, args.batch, args.maxit, peak, stream)
        if rank == 0 and not args.no_cpu_baseline and ws == 1:
            s = oracle_variant_sample(P, W_recipe, "gs", "K", var["gs/K"]["iters_max"], args.cpu_sample_s)
            var["gs/K"]["cpu_baseline"] = dict(s, kind="oracle", sample=f"{s['sample_iters']} oracle PCG "
                                                   f"iterations with the GS K-cycle (setup untimed), scaled "
                                                   f"to the GPU's {var['gs/K']['iters_max']} iterations")
        line["variants"] = var
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        s = oracle_sample(P, W_recipe, inf64[0]["iters"], args.cpu_sample_s)
        line["cpu_baseline"] = {"value": s["ms_per_rhs"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{s['sample_iters']} FP64 oracle PCG iterations on the same "
                                          f"operator and hierarchy sizes (setup untimed, {s['sample_s']:.1f} s), "
                                          f"scaled to the {inf64[0]['iters']} iterations of the float64 solve"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    Hd.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

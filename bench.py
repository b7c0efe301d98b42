#!/usr/bin/env python
"""Time to a 1e-8 relative residual per right-hand side of the AMG-PCG
solve (the single-hierarchy multiple-vector aggregation AMG as a CG
preconditioner), on the seeded synthetic workloads.

Default (``--config 2``, the headline): rotated anisotropic diffusion (eps =
1e-3, theta = pi/6, 9-point, 1024 x 1024), 4 smooth vectors from the seeded
bootstrap of Algorithm 1 (testing phase on the device), aggregates of 16,
5 levels.  One step = one complete solve of ``--batch`` (32) seeded
uniform[-1, 1] right-hand sides from a zero initial guess, inputs resident in
HBM, with the float32 V-cycle inside CG whose x, r and q are double-float
pairs, whose search direction is float32 and whose scalars are float64.
Beside it: the same block with the float32 V-cycle inside float64 CG
(``outer_fp64``), the plain float64 solve of one RHS and of the block, the
end-to-end time through the C ABI with host buffers, per-kernel times and
byte counts, and the FP64 oracle on the host cores (one core and all cores).

Other workloads (``--config N``), each printing one JSON line of the same
form: 1 = 2D Poisson 64^2, float64 plain, one RHS; 3 = 3D jumping
coefficients 128^3, 32 Gaussian RHS, float32 cycle; 4 = uneven batch of 8
elasticity grids x 4 RHS in one launch sequence, float32 cycle; 5 = the
differentiable solve on 512^2 cell-centred diffusion (8 RHS: forward solve,
adjoint solve and the masked gradient), float64 and float32 cycle.

    python bench.py [--gpus N --steps K --warmup W --impl gb300|reference --config C]

Under torchrun every rank runs an independent replica on its own GPU with
its own right-hand sides (weak scaling, no collective on the data path); the
timed region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import os

# the oracle's worker processes each take one core: one BLAS thread apiece
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import multiprocessing  # noqa: E402
import platform  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms to 1e-8 rel. residual per RHS: FP32-cycle batched vs FP64 plain; % HBM peak"
UNIT = "ms/RHS"
L2_BYTES = 129e6
PEAK_FALLBACK_GBS = 6800.0
NU_BOOT = 15  # testing-phase applications per bootstrap stage (Algorithm 1)

# the arithmetic of each solve mode
DTYPES = {
    "df": "f32 V-cycle; CG x, r, q double-float (f32 hi+lo), p f32, scalars f64",
    "f32c_f64": "f32 V-cycle; CG x, r, p, q and scalars f64",
    "f64": "f64",
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--grid", type=int, default=None, help="grid side (default: the workload's own)")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--smooth", default="bootstrap", choices=["bootstrap", "relaxed"],
                    help="workload 2: smooth vectors from the seeded bootstrap of Algorithm 1 (testing "
                         "phase on the device; the oracle arm runs its own), or the relaxed random vectors")
    ap.add_argument("--maxit", type=int, default=5000)
    ap.add_argument("--tune-cache", default=None,
                    help="file of tuned launch choices: read when it has this workload, else written "
                         "(so that a profiled run replays the choices of a plain run)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-kernel-table", action="store_true")
    ap.add_argument("--no-extra-arms", action="store_true",
                    help="time only the headline solve (the profiling runs use this)")
    ap.add_argument("--variants", action="store_true",
                    help="workload 2: also time the float64 cycle variants (Gauss-Seidel smoother, K-cycle)")
    ap.add_argument("--cpu-sample-s", type=float, default=10.0)
    ap.add_argument("--cpu-cores", type=int, default=0, help="oracle worker processes (0: all host cores)")
    return ap.parse_args(argv)


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


def rhs_block(P, batch, rank, gaussian=False, seed=1002):
    """The right-hand sides of one replica: seeded (uniform[-1, 1] or
    standard normal), distinct per rank; rank 0's first column is the
    workload's own first RHS."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed + 7919 * rank))
    B = rng.standard_normal((P.n, batch)) if gaussian else rng.uniform(-1.0, 1.0, size=(P.n, batch))
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


def host_cpu():
    """Model name, architecture and logical core count of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for l in out.splitlines():
            if l.lower().startswith("model name"):
                model = l.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for l in open("/proc/cpuinfo"):
                if l.lower().startswith(("model name", "cpu model")):
                    model = l.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return f"{model or platform.processor() or 'unknown'} ({platform.machine()})", os.cpu_count() or 1


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


# ------------------------------------------------------- byte accounting --
def algorithmic_bytes(kernel, lv, K, mode="df"):
    """Minimal bytes one launch of a level-0 kernel must move: matrix arrays
    once, each vector block once per read or write, prolongator blocks once.

    lv: n0, nnz0 (level 0), n1 (level 1), npv1 (prolongator values of P^1).
    mode: "df" (float32 cycle; CG x, r, q as float32 hi + lo pairs, p
    float32; the first pre-sweep folded into the column-scaled level-0
    matrix, so u0 = D^-1 r is never stored), "f32c_f64" (float32 cycle,
    float64 CG), "f64" (float64 throughout).  None for spans that are not
    one kernel."""
    n, nnz, n1, npv = lv["n0"], lv["nnz0"], lv["n1"], lv["npv1"]
    w = 8 if mode == "f64" else 4            # cycle precision
    rp = 4 * (n + 1)                         # row pointers
    if kernel == "spmv_cg":      # q = A p with p.q
        if mode == "df":                     # A as (hi, lo) floats, p float, q (hi, lo)
            return nnz * 12 + rp + n * K * 4 + n * K * 8
        return nnz * 12 + rp + n * K * 8 + n * K * 8
    if kernel == "cg_update":    # r -= a q with ||r|| (df: x moved to the direction kernel)
        if mode == "df":                     # q (hi, lo) read, r (hi, lo) read and written
            return 3 * n * K * 8
        # x, r read and written, p, q read; u0 = D^-1 r stored; (f32c) f0 = fl32(r)
        return 6 * n * K * 8 + n * 8 + n * K * w + (n * K * 4 if mode == "f32c_f64" else 0)
    if kernel == "cg_direction":  # p = z + b p (df: x stepped after every second iteration)
        if mode == "df":  # z, p_k read, p_{k+1} written; every second launch also p_{k-1} read and
            # x (hi, lo) read and written: 12 and 32 bytes per row and column, 22 on average
            return n * K * 22
        return n * K * (w + 16)              # z, p float64 read and written
    if kernel == "smooth_l0":    # z = u + D^-1 (f - A u) with r.z
        if mode == "df":                     # f = r_hi; r_lo read for r.z
            return nnz * 8 + rp + n * 4 + n * K * 4 * 4
        if mode == "f32c_f64":               # f, u, z float; r float64
            return nnz * 8 + rp + n * 4 + n * K * (4 + 4 + 4 + 8)
        return nnz * 12 + rp + n * 8 + n * K * 8 * 3   # f = r, u, z
    if kernel == "restrict_l0" and lv.get("rf_entries"):
        # fc = R f, R = P^T (I - A D^-1) kept by aggregate (pattern offsets and coarse
        # starts, pattern columns, rf_rs values per entry); f read once, fc and uc
        # written, D_c^-1 read
        nagg = lv["nagg1"]
        return (8 * (nagg + 1) + lv["rf_entries"] * (4 + lv["rf_rs"] * w) + n * K * w
                + n1 * (2 * K * w + w))
    if kernel == "restrict_l0":  # fc = P^T (f - A u), uc = D_c^-1 fc
        if mode == "df":                     # t = f - (A D^-1) f: one vector block read
            return nnz * 8 + rp + n * K * 4 + npv * 4 + n1 * (2 * K * 4 + 4)
        return nnz * (w + 4) + rp + 2 * n * K * w + npv * w + n1 * (2 * K * w + w)
    if kernel == "prolong_l0":   # u += P uc (df: u = D^-1 f + P uc)
        if mode == "df":
            return npv * 4 + n1 * K * 4 + 2 * n * K * 4 + n * 4
        return npv * w + n1 * K * w + 2 * n * K * w
    if kernel == "coarse_levels":
        return None
    raise KeyError(kernel)


KERNEL_IDS = {"spmv_cg": 1, "restrict_l0": 2, "smooth_l0": 3, "prolong_l0": 4, "cg_update": 5,
              "cg_direction": 7, "coarse_levels": 8}
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


def alu_ops(kernel, lv, K, mode="df"):
    if kernel == "spmv_cg" and mode == "df":
        return lv["nnz0"] * K * ALU_OPS_PER_NZ_COL + lv["n0"] * K * ALU_OPS_PER_ROW_COL
    return None


def gs_sweep_bytes(lv, K):
    """Minimal bytes of one level-0 Gauss-Seidel sweep over all colours:
    the matrix once (8-byte values, 4-byte columns, row pointers), colour and
    diagonal once per row, f read, u read and written once (float64)."""
    n0, nnz0 = lv["n0"], lv["nnz0"]
    return nnz0 * 12 + 4 * (n0 + 1) + n0 * 12 + 3 * n0 * K * 8


def l2_note(working_bytes):
    if working_bytes > L2_BYTES:
        return f"inputs larger than L2 ({working_bytes / 1e6:.0f} MB of matrix and vector blocks per solve)"
    return (f"working set {working_bytes / 1e6:.0f} MB fits in L2: a {2 * L2_BYTES / 1e6:.0f} MB buffer is "
            "written between timed steps (outside each step's event pair)")


# ------------------------------------------------------- the oracle legs --
_ORACLE = {}


def _oracle_iters_worker(args):
    """Worker: ``k`` oracle PCG iterations on right-hand side column ``c`` of
    system ``s`` (the hierarchies were built before the pool was forked), in
    solves of at most ``cap`` iterations (the solve's own count: a small
    problem would otherwise iterate past convergence into a zero residual)."""
    from oracle import amg_oracle as O
    s, c, k, cap = args
    H, B = _ORACLE["H"][s], _ORACLE["B"][s]
    A = H.levels[0].A
    t0 = time.perf_counter()
    left = k
    while left > 0:
        step = min(left, max(1, cap))
        O.pcg(A, B[:, c % B.shape[1]], lambda r: O.vcycle(H, r), fixed_iters=step)
        left -= step
    return time.perf_counter() - t0


class OracleLeg:
    """The FP64 oracle on the host cores, built before the first CUDA call:
    the hierarchies of the workload's systems (relaxed-vector recipe: an
    iteration's cost depends on the hierarchy's sizes, not on the vectors'
    values) and a pool of worker processes forked from this process, one per
    core.  ``sample`` times a bounded number of PCG iterations on one core
    and, concurrently, on every core (each worker on its own right-hand side),
    and scales both to the iteration counts of the solve."""

    def __init__(self, problems, cores=0):
        from oracle import amg_oracle as O
        self.model, ncpu = host_cpu()
        self.cores = cores or ncpu
        _ORACLE["H"] = [O.setup(P.A, P.aggs, P.n_nodes, P.W) for P in problems]
        _ORACLE["B"] = [P.B for P in problems]
        self.pool = None
        if self.cores > 1 and "fork" in multiprocessing.get_all_start_methods():
            self.pool = multiprocessing.get_context("fork").Pool(self.cores)

    def close(self):
        if self.pool is not None:
            self.pool.terminate()
            self.pool = None

    def sample(self, iters, budget_s):
        """iters[s]: PCG iterations of system s.  Returns one-core and
        all-core ms per RHS (mean over the systems' RHS) and what ran."""
        nsys = len(iters)
        cap = [max(1, int(i) - 1) for i in iters]
        t1 = [_oracle_iters_worker((s, 0, 1, cap[s])) for s in range(nsys)]
        per_round = sum(t1)
        k = max(2, int(budget_s / 2 / max(per_round, 1e-3)))
        one = [_oracle_iters_worker((s, 0, k, cap[s])) / k for s in range(nsys)]
        ms_one = sum(one[s] * iters[s] for s in range(nsys)) / nsys * 1e3
        out = {"one_core": {"value": ms_one, "cores": 1, "sample_iters": k}}
        if self.pool is not None:
            jobs = [(s, c, k, cap[s]) for c in range(self.cores) for s in range(nsys)]
            t0 = time.perf_counter()
            self.pool.map(_oracle_iters_worker, jobs, chunksize=1)
            wall = time.perf_counter() - t0
            # every worker ran k iterations of every system on its own RHS
            frac = [one[s] * iters[s] for s in range(nsys)]
            ms_all = wall / (k * self.cores) * sum(frac) / sum(one) / nsys * 1e3
            out["all_cores"] = {"value": ms_all, "cores": self.cores, "sample_iters": k, "wall_s": wall}
        out["cpu"] = self.model
        return out


def cpu_baseline_entry(leg, iters, budget_s, what):
    s = leg.sample(iters, budget_s)
    best = s.get("all_cores", s["one_core"])
    return {"value": best["value"], "unit": UNIT, "cores": best["cores"], "kind": "oracle",
            "cpu": s["cpu"], "nproc": leg.cores, "one_core_ms_per_rhs": s["one_core"]["value"],
            "all_cores_ms_per_rhs": s.get("all_cores", {}).get("value"),
            "sample": f"{s['one_core']['sample_iters']} FP64 oracle PCG iterations per system on one core, "
                      f"and the same on each of {best['cores']} worker processes (one RHS each, run "
                      f"concurrently), {what}; setup untimed; scaled to the iterations of the float64 GPU "
                      f"solve"}


# ------------------------------------------------------------ GPU pieces --
class Ctx:
    def __init__(self, args, ws, rank, local):
        import torch

        from paper_1907_04417_gb300 import amg, build
        build.build()
        torch.cuda.set_device(local)
        self.args, self.ws, self.rank, self.local = args, ws, rank, local
        self.torch, self.amg = torch, amg
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.current_stream()
        self.peak, self.peak_kind = peaks()
        self._flush = None

    def event(self):
        return self.torch.cuda.Event(enable_timing=True)

    def flush_l2(self):
        if self._flush is None:
            self._flush = self.torch.empty(int(2 * L2_BYTES) // 4, dtype=self.torch.float32, device=self.dev)
        self._flush.fill_(1.0)

    def measure(self, step, steps, flush=False):
        """Device time of ``steps`` calls of ``step`` (CUDA events on the
        launching stream, barriers and synchronisation on both sides, the
        slowest rank's time), with the clock record of the timed region.
        With ``flush`` every step is bracketed by its own events and an L2
        flush runs between steps, outside them."""
        torch = self.torch
        barrier(self.ws)
        torch.cuda.synchronize()
        results = []
        l0 = self.amg.kernel_launches()
        with ClockSampler(self.local) as cs:
            if not flush:
                e0, e1 = self.event(), self.event()
                e0.record(self.stream)
                for _ in range(steps):
                    results.append(step())
                e1.record(self.stream)
                torch.cuda.synchronize()
                el = e0.elapsed_time(e1)
            else:
                el = 0.0
                for _ in range(steps):
                    self.flush_l2()
                    e0, e1 = self.event(), self.event()
                    torch.cuda.synchronize()
                    e0.record(self.stream)
                    results.append(step())
                    e1.record(self.stream)
                    torch.cuda.synchronize()
                    el += e0.elapsed_time(e1)
        launches = self.amg.kernel_launches() - l0
        barrier(self.ws)
        return max_over_ranks(el, self.ws), results, cs.summary(), launches

    def once_ms(self, step, reps=1):
        torch = self.torch
        torch.cuda.synchronize()
        e0, e1 = self.event(), self.event()
        e0.record(self.stream)
        out = None
        for _ in range(reps):
            out = step()
        e1.record(self.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    def kernel_table(self, H, solve, lv, K, mode, names=None, workload_key=None):
        """Per kernel family: launches and device time in one solve (events
        around each launch on its stream, in a solve of its own so that the
        timed steps run without them), algorithmic bytes per launch, the
        achieved bandwidth and its fraction of the measured copy peak, and
        the family's share of the solve's time."""
        solve_ms, _ = self.once_ms(solve)
        tab = {}
        for name in names or KERNEL_IDS:
            H.timer_enable(KERNEL_IDS[name])
            solve()
            ms, nl = H.timer_read()
            H.timer_enable(0, False)
            ent = {"launches": nl, "ms_total": ms, "avg_ms": ms / max(nl, 1),
                   "share_of_solve": ms / solve_ms if solve_ms > 0 else None}
            lvn = lv
            if name == "restrict_l0":  # the restriction this solve ran (R or the CSR form)
                ri = H.restriction_info(0)
                lvn = dict(lv, rf_entries=ri["entries"] if ri["by_r"] else 0, rf_rs=ri["values_per_entry"])
                ent["by_r"] = ri["by_r"]
            nb = algorithmic_bytes(name, lvn, K, mode)
            if nb is not None and nl > 0 and ms > 0:
                gbs = nb / (ms / nl * 1e-3) / 1e9
                ent.update({"algorithmic_bytes": nb, "achieved_gbs": gbs, "hbm_frac": gbs / self.peak})
                tr = stored_traffic(name, workload_key) if (workload_key and mode == "df") else None
                if tr is not None:  # ncu DRAM bytes of the same kernel (profiles/traffic.json)
                    ent["traffic"] = tr
            tab[name] = ent
        return tab, solve_ms

    def roofline(self, tab, lv, K, mode, workload_key):
        """The roofline of the level-0 kernel with the largest share."""
        cands = {k: v for k, v in tab.items() if k != "coarse_levels" and v.get("algorithmic_bytes")}
        rk = max(cands, key=lambda k: cands[k]["ms_total"])
        e = cands[rk]
        roof = {"bound": "hbm", "achieved": e["achieved_gbs"], "peak": self.peak, "unit": "GB/s",
                "frac": e["hbm_frac"], "traffic": stored_traffic(rk, workload_key), "kernel": rk,
                "peak_source": f"{self.peak_kind} hbm_gbs (burst copy)",
                "algorithmic_bytes_per_launch": e["algorithmic_bytes"], "avg_launch_ms": e["avg_ms"],
                "launches_timed": e["launches"], "timed_in": "a solve of its own, right after the timed steps"}
        ops = alu_ops(rk, lv, K, mode)
        if ops is not None:
            # the double-float q = A p: float32 arithmetic bounds it; its HBM
            # figures stay beside it
            aa = ops / (e["avg_ms"] * 1e-3)
            roof.update({"bound": "alu", "achieved": aa / 1e12, "peak": ALU_PEAK_OPS / 1e12,
                         "unit": "T float32 ops/s", "frac": aa / ALU_PEAK_OPS,
                         "peak_source": "derived: 152 SMs x 128 float32 lanes x 2.07 GHz",
                         "alu_ops_per_launch": ops, "hbm_achieved_gbs": e["achieved_gbs"],
                         "hbm_peak_gbs": self.peak, "hbm_frac": e["hbm_frac"]})
        return roof


def level_sizes(H, n0=None, nnz0=None):
    e1 = H.export_level(1)
    i = H.info()
    return {"n0": n0 or i["n_level"][0], "nnz0": nnz0 or i["nnz_level"][0], "n1": e1["n"],
            "npv1": int(e1["pval"].size), "nagg1": int(e1["naggs"])}


def true_relres(A, B, X):
    import numpy as np
    return float(max(np.linalg.norm(B[:, c] - A @ X[:, c]) / np.linalg.norm(B[:, c]) for c in range(B.shape[1])))


def base_line(args, ctx, value, elapsed, clocks, launches, mode, workload, rhs_per_step, extra_cfg=None):
    cfg = {"workload": workload, "rhs_per_step_per_gpu": rhs_per_step, "rtol": 1e-8,
           "parallelism": f"replicas x{ctx.ws}"}
    cfg.update(extra_cfg or {})
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ctx.ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[mode], "data": "synthetic",
            "config": cfg, "clocks": clocks, "gpu_launches": launches}


def solve_arm(ctx, H, Bd, Xd, o, reps=2):
    """Warm-up solve (workspace, tuning, graph), then ``reps`` timed solves:
    ms per RHS, iteration range, status."""
    import numpy as np
    Xd.zero_()
    H.solve(Bd, Xd, o)

    def one():
        Xd.zero_()
        return H.solve(Bd, Xd, o)

    ms, (_, infos, st) = ctx.once_ms(one, reps)
    its = [i["iters"] for i in infos]
    return {"ms_per_rhs": ms / Bd.shape[1], "ms_per_solve": ms, "iters_min": int(np.min(its)),
            "iters_max": int(np.max(its)), "status": int(st)}


def e2e_arm(ctx, H, B, o, reps=2):
    """End to end through the C ABI: pinned host right-hand sides in, host
    solution out, the copies inside the timed region."""
    torch = ctx.torch
    Bh = torch.from_numpy(B).pin_memory()
    Xh = torch.zeros_like(Bh).pin_memory()
    H.solve(Bh, Xh, o)

    def one():
        Xh.zero_()
        H.solve(Bh, Xh, o)

    ms, _ = ctx.once_ms(one, reps)
    ms = max_over_ranks(ms, ctx.ws)
    return {"value": ms / B.shape[1], "unit": UNIT, "h2d_bytes_per_step": int(2 * B.size * 8),
            "d2h_bytes_per_step": int(B.size * 8)}


# ------------------------------------------------------------- workloads --
def workload_text(cfg, N, smooth="bootstrap"):
    if cfg == 1:
        return f"poisson5 {N}x{N} (n={N * N}), m=1, aggregates of 4, 3 levels, float64 plain"
    if cfg == 2:
        sv = ("smooth vectors from the seeded bootstrap (Algorithm 1, nu=15, symmetrized)" if smooth == "bootstrap"
              else "relaxed random smooth vectors")
        return f"aniso9 eps=1e-3 theta=pi/6, {N}x{N} (n={N * N}), m=4, aggregates of 16, 5 levels, {sv}"
    if cfg == 3:
        return (f"jump7 {N}^3 (n={N ** 3}), k per 8^3 block log-uniform [1e-3,1e3], m=3, aggregates of up to 16, "
                f"levels until <= 1024 coarse dofs")
    if cfg == 4:
        return "elasticity batch: 8 Navier-Cauchy grids, sides from {32,40,48,64}, m=6, aggregates of up to 32 dofs"
    return (f"cc5 {N}x{N} (n={N * N}), log-normal k (sigma=1), m=3, aggregates of up to 16; loss ||x - x_target||^2,"
            f" forward solve + adjoint solve + masked gradient")


def run_c2(args, ctx, leg_maker):
    import numpy as np

    from paper_1907_04417_gb300.hostsetup import inputs
    N = args.grid or 1024
    P = inputs.anisotropic(N=N, nrhs=1)
    leg = leg_maker([P])
    amg, torch = ctx.amg, ctx.torch
    B = rhs_block(P, args.batch, ctx.rank)
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
    dev = ctx.dev
    Hd = amg.Hierarchy((torch.from_numpy(A.indptr).to(dev), torch.from_numpy(A.indices).to(dev),
                        torch.from_numpy(A.data).to(dev)), P.aggs, P.n_nodes, torch.from_numpy(P.W).to(dev))
    info_h = Hd.info()
    Bd = torch.from_numpy(B).to(dev)
    Xd = torch.zeros_like(Bd)
    o32 = amg.opts(cycle_precision=32, maxit=args.maxit)
    o64 = amg.opts(cycle_precision=64, maxit=args.maxit)
    o32f = amg.opts(cycle_precision=32, maxit=args.maxit, outer_fp64=1)

    def step():
        Xd.zero_()
        return Hd.solve(Bd, Xd, o32)

    for _ in range(args.warmup):
        step()
    elapsed, res, clocks, launches = ctx.measure(step, args.steps)
    value = whole_job_ms_per_rhs(elapsed, args.steps, args.batch, ctx.ws)
    iters = [[i["iters"] for i in r[1]] for r in res]
    Xc = Xd.cpu().numpy()
    line = base_line(args, ctx, value, elapsed, clocks, launches, "df", workload_text(2, N, args.smooth),
                     args.batch, {"l2": l2_note(A.nnz * 12 + 6 * P.n * args.batch * 8)})
    line["fp32_batched_iters"] = {"min": int(np.min(iters)), "max": int(np.max(iters))}
    line["true_relres_max"] = true_relres(A, B, Xc)
    print(f"[bench] {elapsed / args.steps:.1f} ms/step, {value:.3f} ms/RHS, iters {line['fp32_batched_iters']}",
          file=sys.stderr, flush=True)
    lv = level_sizes(Hd)
    if not args.no_kernel_table:
        tab, solve_ms = ctx.kernel_table(Hd, step, lv, args.batch, "df", workload_key=f"aniso{N}_K{args.batch}")
        line["kernels"] = tab
        line["roofline"] = ctx.roofline(tab, lv, args.batch, "df", f"aniso{N}_K{args.batch}")
    # plain float64 solve of one RHS, and of the whole block
    b1 = Bd[:, :1].contiguous()
    x1 = torch.zeros_like(b1)
    f64 = solve_arm(ctx, Hd, b1, x1, o64)
    x64 = x1.cpu().numpy()[:, 0]
    line["fp64_plain"] = {"ms_per_rhs": f64["ms_per_rhs"], "iters": f64["iters_max"]}
    line["fp32_vs_fp64_rel_err"] = float(np.linalg.norm(Xc[:, 0] - x64) / np.linalg.norm(x64))
    line["speedup_batched_vs_fp64_plain"] = f64["ms_per_rhs"] / value if value else None
    if not args.no_extra_arms:
        X2 = torch.zeros_like(Bd)
        arm = solve_arm(ctx, Hd, Bd, X2, o32f)
        arm["true_relres_max"] = true_relres(A, B, X2.cpu().numpy())
        if not args.no_kernel_table:
            tq, _ = ctx.kernel_table(Hd, lambda: Hd.solve(Bd, X2.zero_(), o32f), lv, args.batch, "f32c_f64",
                                     names=["spmv_cg", "cg_update", "smooth_l0"])
            arm["kernels"] = tq
        arm["dtype"] = DTYPES["f32c_f64"]
        line["fp32_cycle_fp64_cg"] = arm
        X3 = torch.zeros_like(Bd)
        a64 = solve_arm(ctx, Hd, Bd, X3, o64, reps=1)
        a64["dtype"] = "f64"
        line["fp64_batched"] = a64
        line["e2e"] = e2e_arm(ctx, Hd, B, o32)
    line["hierarchy"] = {"levels": info_h["levels"], "n": info_h["n_level"], "nnz": info_h["nnz_level"],
                         "opc": info_h["opc"]}
    line["bootstrap"] = boot
    if args.variants:
        line["variants"] = time_variants(ctx, Hd, Bd, Xd, B, A, lv, args.batch, args.maxit)
    if leg is not None:
        line["cpu_baseline"] = cpu_baseline_entry(leg, [line["fp64_plain"]["iters"]], args.cpu_sample_s,
                                                  "the same operator and hierarchy sizes")
        leg.close()
    Hd.close()
    return line


VARIANTS = [("l1jacobi", "V"), ("gs", "V"), ("l1jacobi", "K"), ("gs", "K")]


def time_variants(ctx, Hd, Bd, Xd, B, A, lv, K, maxit):
    """Float64 solves of the block with each cycle variant: device time per
    RHS (after a warm-up solve that builds the colouring, workspace and
    graph), iteration counts, true residuals, and for Gauss-Seidel the
    level-0 sweep's achieved bandwidth."""
    amg = ctx.amg
    out = {}
    for sm, kind in VARIANTS:
        o = amg.opts(cycle_precision=64, maxit=maxit, smoother=1 if sm == "gs" else 0,
                     cycle=1 if kind == "K" else 0)
        ent = solve_arm(ctx, Hd, Bd, Xd, o, reps=1)
        ent["true_relres_max"] = true_relres(A, B, Xd.cpu().numpy())
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
                                  "peak_gbs": ctx.peak, "frac": gbs / ctx.peak,
                                  "ncolours": Hd.level_colours(0)[1]}
        out[f"{sm}/{kind}"] = ent
    return out


def run_single(args, ctx, leg_maker, cfg):
    """Workloads 1 and 3: one hierarchy, a block of right-hand sides."""
    import numpy as np

    from paper_1907_04417_gb300.hostsetup import inputs
    if cfg == 1:
        N = args.grid or 64
        P = inputs.poisson(N=N, nrhs=1)
        batch, mode = 1, "f64"
    else:
        N = args.grid or 128
        P = inputs.jumping3d(N=N, nrhs=32)
        batch, mode = args.batch, "df"
    leg = leg_maker([P])
    amg, torch = ctx.amg, ctx.torch
    B = rhs_block(P, batch, ctx.rank, gaussian=cfg == 3, seed=1000 + cfg)
    A = P.A
    dev = ctx.dev
    Hd = amg.Hierarchy((torch.from_numpy(A.indptr).to(dev), torch.from_numpy(A.indices).to(dev),
                        torch.from_numpy(A.data).to(dev)), P.aggs, P.n_nodes, torch.from_numpy(P.W).to(dev))
    info_h = Hd.info()
    Bd = torch.from_numpy(B).to(dev)
    Xd = torch.zeros_like(Bd)
    o = amg.opts(cycle_precision=64 if mode == "f64" else 32, maxit=args.maxit)
    o64 = amg.opts(cycle_precision=64, maxit=args.maxit)

    def step():
        Xd.zero_()
        return Hd.solve(Bd, Xd, o)

    for _ in range(args.warmup):
        step()
    work = sum(info_h["nnz_level"]) * 12 + 8 * P.n * batch * 8
    flush = work <= L2_BYTES
    # a timed region of at least about a second, so that the clock sampler
    # (every 200 ms) sees it: short solves take more steps
    one, _ = ctx.once_ms(step)
    args.steps = max(args.steps, int(1000.0 / max(one, 1e-3)) + 1)
    elapsed, res, clocks, launches = ctx.measure(step, args.steps, flush=flush)
    value = whole_job_ms_per_rhs(elapsed, args.steps, batch, ctx.ws)
    iters = [[i["iters"] for i in r[1]] for r in res]
    Xc = Xd.cpu().numpy()
    line = base_line(args, ctx, value, elapsed, clocks, launches, mode, workload_text(cfg, N), batch,
                     {"l2": l2_note(work)})
    line["iters"] = {"min": int(np.min(iters)), "max": int(np.max(iters))}
    line["true_relres_max"] = true_relres(A, B, Xc)
    lv = level_sizes(Hd)
    if not args.no_kernel_table:
        tab, _ = ctx.kernel_table(Hd, step, lv, batch, mode)
        line["kernels"] = tab
        line["roofline"] = ctx.roofline(tab, lv, batch, mode, f"cfg{cfg}_{N}_K{batch}")
    b1 = Bd[:, :1].contiguous()
    x1 = torch.zeros_like(b1)
    f64 = solve_arm(ctx, Hd, b1, x1, o64)
    line["fp64_plain"] = {"ms_per_rhs": f64["ms_per_rhs"], "iters": f64["iters_max"]}
    if mode != "f64":
        x64 = x1.cpu().numpy()[:, 0]
        line["fp32_vs_fp64_rel_err"] = float(np.linalg.norm(Xc[:, 0] - x64) / np.linalg.norm(x64))
        line["speedup_batched_vs_fp64_plain"] = f64["ms_per_rhs"] / value if value else None
        if not args.no_extra_arms:
            X2 = torch.zeros_like(Bd)
            arm = solve_arm(ctx, Hd, Bd, X2, amg.opts(cycle_precision=32, maxit=args.maxit, outer_fp64=1))
            arm["true_relres_max"] = true_relres(A, B, X2.cpu().numpy())
            arm["dtype"] = DTYPES["f32c_f64"]
            line["fp32_cycle_fp64_cg"] = arm
    else:
        X2 = torch.zeros_like(Bd)
        arm = solve_arm(ctx, Hd, Bd, X2, amg.opts(cycle_precision=32, maxit=args.maxit))
        arm["true_relres_max"] = true_relres(A, B, X2.cpu().numpy())
        arm["dtype"] = DTYPES["df"]
        line["fp32_cycle"] = arm
    if not args.no_extra_arms:
        line["e2e"] = e2e_arm(ctx, Hd, B, o)
    line["hierarchy"] = {"levels": info_h["levels"], "n": info_h["n_level"], "nnz": info_h["nnz_level"],
                         "opc": info_h["opc"]}
    if leg is not None:
        line["cpu_baseline"] = cpu_baseline_entry(leg, [line["fp64_plain"]["iters"]], args.cpu_sample_s,
                                                  "the same workload")
        leg.close()
    Hd.close()
    return line


def run_c4(args, ctx, leg_maker):
    """The uneven elasticity batch through amg_solve_batched."""
    import numpy as np

    from paper_1907_04417_gb300.hostsetup import inputs
    probs = inputs.elasticity_batch()
    leg = leg_maker(probs)
    amg, torch = ctx.amg, ctx.torch
    dev = ctx.dev
    Hs = [amg.Hierarchy((torch.from_numpy(P.A.indptr).to(dev), torch.from_numpy(P.A.indices).to(dev),
                         torch.from_numpy(P.A.data).to(dev)), P.aggs, P.n_nodes, torch.from_numpy(P.W).to(dev))
          for P in probs]
    Bs = [P.B for P in probs]
    if ctx.rank:  # other replicas: their own right-hand sides
        rng = np.random.default_rng(7919 * ctx.rank)
        Bs = [rng.standard_normal(B.shape) for B in Bs]
    Bd = [torch.from_numpy(B).to(dev) for B in Bs]
    Xd = [torch.zeros_like(b) for b in Bd]
    nrhs = sum(B.shape[1] for B in Bs)
    o = amg.opts(cycle_precision=32, maxit=args.maxit)

    def step():
        for x in Xd:
            x.zero_()
        return amg.solve_batched(Hs, Bd, Xd, o)

    for _ in range(args.warmup):
        step()
    ntot = sum(P.n for P in probs)
    nnz = sum(P.A.nnz for P in probs)
    work = nnz * 12 + 6 * ntot * 4 * 8
    elapsed, res, clocks, launches = ctx.measure(step, args.steps, flush=work <= L2_BYTES)
    value = whole_job_ms_per_rhs(elapsed, args.steps, nrhs, ctx.ws)
    iters = [i["iters"] for r in res for sysinfo in r[1] for i in sysinfo]
    sides = [P.meta["grid"] for P in probs]
    line = base_line(args, ctx, value, elapsed, clocks, launches, "df", workload_text(4, 0), nrhs,
                     {"l2": l2_note(work), "sides": sides, "n_total": ntot, "nnz_total": nnz})
    line["iters"] = {"min": int(min(iters)), "max": int(max(iters))}
    line["true_relres_max"] = max(true_relres(P.A, B, x.cpu().numpy()) for P, B, x in zip(probs, Bs, Xd))
    # the batch's level-0 sizes: the concatenated hierarchy spans every system
    lv = {"n0": ntot, "nnz0": nnz, "n1": sum(h.export_level(1)["n"] for h in Hs),
          "npv1": sum(int(h.export_level(1)["pval"].size) for h in Hs)}
    if not args.no_kernel_table:
        # the batch plan is cached on the first hierarchy, whose timer covers it
        tab, _ = ctx.kernel_table(Hs[0], step, lv, 4, "df")
        line["kernels"] = tab
        line["roofline"] = ctx.roofline(tab, lv, 4, "df", "elasticity_batch_K4")
    o64 = amg.opts(cycle_precision=64, maxit=args.maxit)
    X64 = [torch.zeros_like(b) for b in Bd]
    amg.solve_batched(Hs, Bd, X64, o64)
    ms64, (_, inf64, _) = ctx.once_ms(lambda: amg.solve_batched(Hs, Bd, [x.zero_() for x in X64], o64))
    it64 = [max(i["iters"] for i in s) for s in inf64]
    line["fp64_batched"] = {"ms_per_rhs": ms64 / nrhs, "iters_per_system": it64}
    line["speedup_vs_fp64_batched"] = (ms64 / nrhs) / value if value else None
    if not args.no_extra_arms:
        of = amg.opts(cycle_precision=32, maxit=args.maxit, outer_fp64=1)
        XF = [torch.zeros_like(b) for b in Bd]
        amg.solve_batched(Hs, Bd, XF, of)
        msf, (_, inff, _) = ctx.once_ms(lambda: amg.solve_batched(Hs, Bd, [x.zero_() for x in XF], of))
        itf = [i["iters"] for s in inff for i in s]
        line["fp32_cycle_fp64_cg"] = {
            "ms_per_rhs": msf / nrhs, "iters_min": min(itf), "iters_max": max(itf), "dtype": DTYPES["f32c_f64"],
            "true_relres_max": max(true_relres(P.A, B, x.cpu().numpy()) for P, B, x in zip(probs, Bs, XF))}
        Bh = [torch.from_numpy(B).pin_memory() for B in Bs]
        Xh = [torch.zeros_like(b).pin_memory() for b in Bh]
        amg.solve_batched(Hs, Bh, Xh, o)
        mse, _ = ctx.once_ms(lambda: amg.solve_batched(Hs, Bh, [x.zero_() for x in Xh], o), 2)
        hb = sum(B.size for B in Bs) * 8
        line["e2e"] = {"value": max_over_ranks(mse, ctx.ws) / nrhs, "unit": UNIT, "h2d_bytes_per_step": 2 * hb,
                       "d2h_bytes_per_step": hb}
    line["hierarchies"] = [h.info()["n_level"] for h in Hs]
    if leg is not None:
        line["cpu_baseline"] = cpu_baseline_entry(leg, it64, args.cpu_sample_s, "every member of the batch")
        leg.close()
    for h in Hs:
        h.close()
    return line


def run_c5(args, ctx, leg_maker):
    """The differentiable solve: x = A(k)^{-1} B, L = ||x - x_target||^2,
    dL/dk through the adjoint solve, the masked outer-product kernel and the
    torch assembly."""
    import numpy as np

    from oracle import amg_oracle as O
    from paper_1907_04417_gb300 import autograd as AG
    from paper_1907_04417_gb300.hostsetup import inputs
    N = args.grid or 512
    nb = 8
    P = inputs.diffusion_cc(N=N, nrhs=nb)
    leg = leg_maker([P])
    amg, torch = ctx.amg, ctx.torch
    dev = ctx.dev
    asm = AG.CellCentredDiffusion(N, device=dev)
    kcell = torch.from_numpy(P.meta["kcell"]).to(dev)
    vals = asm.values(kcell)
    Hd = amg.Hierarchy((asm.rowptr.to(dev), asm.col.to(dev), vals), P.aggs, P.n_nodes,
                       torch.from_numpy(P.W).to(dev))
    Bd = torch.from_numpy(P.B).to(dev)
    Xt = torch.from_numpy(P.meta["x_target"]).to(dev)
    out = {}
    grads = {}
    for mode, prec in (("f64", 64), ("df", 32)):
        o = amg.opts(cycle_precision=prec, maxit=args.maxit)

        def step():
            k = kcell.clone().requires_grad_(True)
            v = asm.values(k)
            x = AG.solve(v, Bd, Hd, o)
            loss = ((x - Xt) ** 2).sum()
            loss.backward()
            return k.grad

        for _ in range(args.warmup):
            step()
        work = P.A.nnz * 12 + 8 * P.n * nb * 8
        elapsed, res, clocks, launches = ctx.measure(step, args.steps, flush=work <= L2_BYTES)
        grads[mode] = res[-1].detach().cpu().numpy().ravel()
        out[mode] = {"elapsed": elapsed, "clocks": clocks, "launches": launches, "work": work}
    e = out["df"]
    value = whole_job_ms_per_rhs(e["elapsed"], args.steps, nb, ctx.ws)
    line = base_line(args, ctx, value, e["elapsed"], e["clocks"], e["launches"], "df", workload_text(5, N), nb,
                     {"l2": l2_note(e["work"]), "step": "forward solve + adjoint solve + gradient, 8 RHS"})
    line["fp64"] = {"ms_per_rhs": whole_job_ms_per_rhs(out["f64"]["elapsed"], args.steps, nb, ctx.ws),
                    "dtype": "f64", "clocks": out["f64"]["clocks"]}
    # gradient checks (untimed).  Central differences of the loss through the
    # same assembly at 48^2 (at 512^2 the loss is about 1e14 and a difference
    # of two solves is rounding): 20 cells, h = 1e-6 |k_c|, direct solves.
    fd_err = {}
    if not args.no_extra_arms:
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        Ps = inputs.diffusion_cc(48, nrhs=nb, max_coarse=256)
        asm_s = AG.CellCentredDiffusion(48, device=dev)
        ks = torch.from_numpy(Ps.meta["kcell"]).to(dev)
        Hs_ = amg.Hierarchy((asm_s.rowptr.to(dev), asm_s.col.to(dev), asm_s.values(ks)), Ps.aggs, Ps.n_nodes,
                            torch.from_numpy(Ps.W).to(dev))
        Bs_ = torch.from_numpy(Ps.B).to(dev)
        Xts = torch.from_numpy(Ps.meta["x_target"]).to(dev)
        kcs = Ps.meta["kcell"].ravel()

        def loss_np(kv):
            A2 = sp.csr_matrix((asm_s.values(torch.from_numpy(kv.reshape(48, 48)).to(dev)).cpu().numpy(),
                                asm_s.col.numpy(), asm_s.rowptr.numpy()), shape=(Ps.n, Ps.n))
            X = spla.splu(A2.tocsc()).solve(Ps.B)
            return float(((X - Ps.meta["x_target"]) ** 2).sum())

        cells = np.random.default_rng(20).choice(Ps.n, 20, replace=False)
        fd = []
        for c in cells:
            h = 1e-6 * kcs[c]
            kp, km = kcs.copy(), kcs.copy()
            kp[c] += h
            km[c] -= h
            fd.append((loss_np(kp) - loss_np(km)) / (2 * h))
        fd = np.asarray(fd)
        for mode, prec, rt in (("f64", 64, 1e-13), ("df", 32, 1e-12)):
            k = ks.clone().requires_grad_(True)
            x = AG.solve(asm_s.values(k), Bs_, Hs_, amg.opts(cycle_precision=prec, maxit=args.maxit, rtol=rt))
            ((x - Xts) ** 2).sum().backward()
            g = k.grad.cpu().numpy().ravel()[cells]
            fd_err[mode] = float(np.max(np.abs(g - fd) / (np.abs(fd) + 1e-3 * np.abs(fd).max())))
        Hs_.close()
        line["fd_check"] = {"grid": 48, "cells": 20, "h": "1e-6 |k_c|", "reference": "direct solves",
                            "max_rel_err": fd_err}
        # the oracle's gradient of the first column's loss (its own solves)
        Ho = O.setup(P.A, P.aggs, P.n_nodes, P.W)
        xo, _ = O.solve(Ho, P.B[:, 0], rtol=1e-12)
        _, go, _ = O.adjoint(Ho, 2 * (xo - P.meta["x_target"][:, 0]), xo, rtol=1e-12)
        b1 = Bd[:, :1].contiguous()
        o64 = amg.opts(cycle_precision=64, maxit=args.maxit, rtol=1e-12)
        v = asm.values(kcell).requires_grad_(True)
        x = AG.solve(v, b1, Hd, o64)
        ((x - Xt[:, :1]) ** 2).sum().backward()
        gg = v.grad.cpu().numpy()
        line["oracle_gradient_rel_err"] = float(np.linalg.norm(gg - go) / np.linalg.norm(go))
    if leg is not None:
        it = [i["iters"] for i in Hd.solve(Bd[:, :1].contiguous(), options=amg.opts(maxit=args.maxit))[1]]
        line["cpu_baseline"] = cpu_baseline_entry(leg, [2 * it[0]], args.cpu_sample_s,
                                                  "the same workload; forward and adjoint solve each")
        leg.close()
    Hd.close()
    return line


# ------------------------------------------------------- reference arm --
def stored_oracle_iters(key):
    p = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    if os.path.exists(p):
        d = json.load(open(p)).get(key)
        if d:
            return int(d["iters"])
    return None


def run_reference(args, ws, rank):
    """The oracle (FP64 CPU, numpy/scipy, as it stands) on the host cores:
    each step runs a bounded number of PCG iterations of the workload on
    every core (one RHS per worker process), scaled to the oracle's own
    iteration count (stored by oracle/count_iterations.py, else counted
    here)."""
    if rank != 0:
        return
    import numpy as np

    from oracle import amg_oracle as O
    from paper_1907_04417_gb300.hostsetup import inputs
    cfg = args.config
    if cfg == 1:
        N = args.grid or 64
        probs = [inputs.poisson(N=N, nrhs=1)]
        keys = [probs[0].name]
    elif cfg == 2:
        N = args.grid or 1024
        probs = [inputs.anisotropic(N=N, nrhs=1)]
        keys = [f"aniso9_{N}x{N}" + ("_bootstrap" if args.smooth == "bootstrap" else "")]
        if args.smooth == "bootstrap":  # the oracle's own bootstrap on the seeded starts (untimed)
            from oracle.count_iterations import bootstrap_vectors
            probs[0].W, _ = bootstrap_vectors(probs[0], N)
    elif cfg == 3:
        N = args.grid or 128
        probs = [inputs.jumping3d(N=N, nrhs=32)]
        keys = [probs[0].name]
    elif cfg == 4:
        N = 0
        probs = inputs.elasticity_batch()
        keys = [f"{P.name}_member{s}" for s, P in enumerate(probs)]
    else:
        N = args.grid or 512
        probs = [inputs.diffusion_cc(N=N, nrhs=8)]
        keys = [probs[0].name]
    iters = []
    for P, key in zip(probs, keys):
        it = stored_oracle_iters(key)
        if it is None:
            H = O.setup(P.A, P.aggs, P.n_nodes, P.W)
            it = O.solve(H, P.B[:, 0], maxit=args.maxit)[1][0].iters
        iters.append(it * (2 if cfg == 5 else 1))
    leg = OracleLeg(probs, args.cpu_cores)
    vals, step_ms = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        smp = leg.sample(iters, args.cpu_sample_s)
        if s >= args.warmup:
            vals.append(smp)
            step_ms.append((time.perf_counter() - t0) * 1e3)
    leg.close()
    best = [v.get("all_cores", v["one_core"]) for v in vals]
    val = statistics.median(b["value"] for b in best)
    one = statistics.median(v["one_core"]["value"] for v in vals)
    cores = best[0]["cores"]
    k = vals[0]["one_core"]["sample_iters"]
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(step_ms),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_text(cfg, N, args.smooth), "rhs_per_step": cores},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": vals[0]["cpu"],
                             "one_core_ms_per_rhs": one,
                             "sample": f"{k} FP64 oracle PCG iterations per system on each of {cores} worker "
                                       f"processes (one RHS each) per step (setup untimed), scaled to the "
                                       f"oracle's {iters} iterations"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- main --
def main(argv=None):
    args = parse(argv)
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.tune_cache:
        os.environ["AMG_TUNE_CACHE"] = args.tune_cache
    want_cpu = rank == 0 and ws == 1 and not args.no_cpu_baseline

    def leg_maker(problems):
        # built before the first CUDA call (the worker processes are forked)
        return OracleLeg(problems, args.cpu_cores) if want_cpu else None

    import torch
    if want_cpu:
        assert not torch.cuda.is_initialized()
    # the CUDA context is created only after the oracle's workers exist: the
    # library is loaded and the device set inside Ctx, which each workload
    # constructs after its inputs and oracle leg
    t0 = time.time()
    runners = {1: lambda c, m: run_single(args, c, m, 1), 2: lambda c, m: run_c2(args, c, m),
               3: lambda c, m: run_single(args, c, m, 3), 4: lambda c, m: run_c4(args, c, m),
               5: lambda c, m: run_c5(args, c, m)}
    holder = {}

    def lazy_leg(problems):
        leg = leg_maker(problems)
        holder["ctx"] = Ctx(args, ws, rank, local)
        return leg

    line = runners[args.config](_LazyCtx(holder), lazy_leg)
    line["wall_s"] = time.time() - t0
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


class _LazyCtx:
    """The workload runners build their inputs and oracle leg first; the
    GPU context exists from the leg's creation on."""

    def __init__(self, holder):
        self._h = holder

    def __getattr__(self, k):
        return getattr(self._h["ctx"], k)


if __name__ == "__main__":
    main()

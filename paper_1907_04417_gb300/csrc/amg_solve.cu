// Preconditioned CG driver (Section 5) over the V-cycle kernels, with the
// float64 CG kernels, the caller <-> library permutations, CUDA-graph
// replay of whole iterations, and the adjoint gradient kernel.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "amg_launch.cuh"

namespace amg {

// ------------------------------------------------------- float64 kernels --

// q = A p with p.q; the last CTA forms alpha = rho / p.q per column.
template <int K, int NZL>
__global__ void __launch_bounds__(BS) k_cg_q(const int* __restrict__ cta_row, const int* __restrict__ rowptr,
                                             const int* __restrict__ col, const double* __restrict__ val,
                                             const double* __restrict__ p, double* __restrict__ q, KState ks) {
  if (*ks.done) return;
  __shared__ double sm[BS];
  __shared__ double tot[64];
  constexpr int CPT = VT<double, K>::CPT, CL = VT<double, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  const int r0 = cta_row[blockIdx.x], r1 = cta_row[blockIdx.x + 1];
  double d[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) d[t] = 0;
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    double acc[CPT];
    row_acc<double, double, K, NZL>(i, valid, rowptr, col, val, p, nzl, cl, acc);
    if (valid && nzl == 0) {
      size_t o = (size_t)i * K + cl * CPT;
      double pv[CPT];
      ldv<double, CPT>(p + o, pv);
      stv<double, CPT>(q + o, acc);
#pragma unroll
      for (int t = 0; t < CPT; ++t) d[t] = fma(pv[t], acc[t], d[t]);
    }
  }
  cta_colsum<K, CPT>(d, sm, ks.partial + (size_t)blockIdx.x * K);
  if (!arrive_last(ks.counter + 0)) return;
  for (int sy = 0; sy < ks.nsys; ++sy) {
    sum_partials(ks.partial, K, ks.sys_cta[sy], ks.sys_cta[sy + 1], sm, tot);
    if (threadIdx.x < K) {
      int v = sy * K + threadIdx.x;
      double pq = tot[threadIdx.x];
      double a = 0.0;
      if (ks.conv[v] == ST_ACTIVE) {
        a = ks.rho[v] / pq;
        if (!(pq > 0.0) || !isfinite(a)) {
          ks.conv[v] = ST_BREAKDOWN;
          ks.status[v] = AMG_ERR_BREAKDOWN;
          ks.iters[v] = *ks.iter;
          a = 0.0;
        }
      }
      ks.alpha[v] = a;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *(ks.counter + 0) = 0u;
}

// r = b - A x with ||b||^2 and ||r||^2; the last CTA initialises the state
// of every (system, column): zero right-hand sides and padding columns stop
// at once, as does a column whose initial guess already meets the tolerance.
template <int K, int NZL>
__global__ void __launch_bounds__(BS) k_cg_init(const int* __restrict__ cta_row, const int* __restrict__ rowptr,
                                                const int* __restrict__ col, const double* __restrict__ val,
                                                const double* __restrict__ b, const double* __restrict__ x,
                                                double* __restrict__ r, KState ks) {
  __shared__ double sm[BS];
  __shared__ double tot[64];
  constexpr int CPT = VT<double, K>::CPT, CL = VT<double, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  const int r0 = cta_row[blockIdx.x], r1 = cta_row[blockIdx.x + 1];
  double db[CPT], dr[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) db[t] = dr[t] = 0;
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    double acc[CPT];
    row_acc<double, double, K, NZL>(i, valid, rowptr, col, val, x, nzl, cl, acc);
    if (valid && nzl == 0) {
      size_t o = (size_t)i * K + cl * CPT;
      double bv[CPT], rv[CPT];
      ldv<double, CPT>(b + o, bv);
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        rv[t] = bv[t] - acc[t];
        db[t] = fma(bv[t], bv[t], db[t]);
        dr[t] = fma(rv[t], rv[t], dr[t]);
      }
      stv<double, CPT>(r + o, rv);
    }
  }
  cta_colsum<K, CPT>(db, sm, ks.partial + (size_t)blockIdx.x * 2 * K);
  __syncthreads();
  cta_colsum<K, CPT>(dr, sm, ks.partial + (size_t)blockIdx.x * 2 * K + K);
  if (!arrive_last(ks.counter + 3)) return;
  for (int sy = 0; sy < ks.nsys; ++sy) {
    sum_partials(ks.partial, 2 * K, ks.sys_cta[sy], ks.sys_cta[sy + 1], sm, tot);
    if (threadIdx.x < K) {
      int v = sy * K + threadIdx.x;
      double bn = sqrt(tot[threadIdx.x]), rn = sqrt(tot[K + threadIdx.x]);
      ks.bnorm[v] = bn;
      ks.rnorm[v] = rn;
      ks.iters[v] = 0;
      ks.status[v] = AMG_OK;
      ks.rho[v] = 0;
      ks.alpha[v] = 0;
      ks.beta[v] = 0;
      int st = ST_ACTIVE;
      if ((int)threadIdx.x >= ks.active[sy] || bn == 0.0 || rn <= ks.rtol * bn) st = ST_CONVERGED;
      if (!isfinite(bn) || !isfinite(rn)) {
        st = ST_BREAKDOWN;
        ks.status[v] = AMG_ERR_BREAKDOWN;
      }
      ks.conv[v] = st;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int stopped = 1;
    for (int v = 0; v < ks.nsys * K; ++v)
      if (ks.conv[v] == ST_ACTIVE) stopped = 0;
    *ks.done = stopped;
    *ks.iter = 0;
    *(ks.counter + 3) = 0u;
  }
}

// p = z + beta p
template <int K>
__global__ void __launch_bounds__(BS) k_cg_p(const int* __restrict__ cta_row, const double* __restrict__ z,
                                             double* __restrict__ p, KState ks) {
  if (*ks.done) return;
  AMG_ELEMENTWISE_PROLOGUE(double)
  const int s = cta_system(ks.sys_cta, ks.nsys);
  double be[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) be[t] = ks.beta[s * K + cfirst + t];
  for (size_t e = e0 + (size_t)threadIdx.x * CPT; e < e1; e += (size_t)BS * CPT) {
    double zv[CPT], pv[CPT];
    ldv<double, CPT>(z + e, zv);
    ldp<double, CPT>(p + e, pv);
#pragma unroll
    for (int t = 0; t < CPT; ++t) pv[t] = fma(be[t], pv[t], zv[t]);
    stv<double, CPT>(p + e, pv);
  }
}

// One-level hierarchy (the coarsest is the fine level): r.z after z = A^{-1} r.
template <int K>
__global__ void __launch_bounds__(BS) k_rz(const int* __restrict__ cta_row, const double* __restrict__ r,
                                           const double* __restrict__ z, KState ks, int mode) {
  if (*ks.done) return;
  __shared__ double sm[BS];
  __shared__ double tot[64];
  AMG_ELEMENTWISE_PROLOGUE(double)
  (void)cfirst;
  double d[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) d[t] = 0;
  for (size_t e = e0 + (size_t)threadIdx.x * CPT; e < e1; e += (size_t)BS * CPT) {
    double rv[CPT], zv[CPT];
    ldv<double, CPT>(r + e, rv);
    ldv<double, CPT>(z + e, zv);
#pragma unroll
    for (int t = 0; t < CPT; ++t) d[t] = fma(rv[t], zv[t], d[t]);
  }
  cta_colsum<K, CPT>(d, sm, ks.partial + (size_t)blockIdx.x * K);
  if (!arrive_last(ks.counter + 2)) return;
  for (int sy = 0; sy < ks.nsys; ++sy) {
    sum_partials(ks.partial, K, ks.sys_cta[sy], ks.sys_cta[sy + 1], sm, tot);
    if (threadIdx.x < K) {
      int v = sy * K + threadIdx.x;
      double rz = tot[threadIdx.x];
      if (mode == 0) {
        ks.rho[v] = rz;
        ks.beta[v] = 0;
      } else if (ks.conv[v] == ST_ACTIVE) {
        ks.beta[v] = rz / ks.rho[v];
        ks.rho[v] = rz;
      } else {
        ks.beta[v] = 0;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *(ks.counter + 2) = 0u;
}

// caller (n_s x nrhs, own numbering) -> library (n x K, padded with zeros)
__global__ void k_perm_in(int r0, int r1, int K, int nrhs, const int* __restrict__ perm,
                          const double* __restrict__ src, double* __restrict__ dst) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tot = (long long)(r1 - r0) * K;
  if (t >= tot) return;
  int i = r0 + (int)(t / K), c = (int)(t % K);
  dst[(size_t)i * K + c] = (c < nrhs && src) ? src[(size_t)perm[i] * nrhs + c] : 0.0;
}

__global__ void k_perm_out(int r0, int r1, int K, int nrhs, const int* __restrict__ perm,
                           const double* __restrict__ src, double* __restrict__ dst) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tot = (long long)(r1 - r0) * nrhs;
  if (t >= tot) return;
  int i = r0 + (int)(t / nrhs), c = (int)(t % nrhs);
  dst[(size_t)perm[i] * nrhs + c] = src[(size_t)i * K + c];
}

// grad[caller nz of (i, j)] = - sum_c lambda[i, c] x[j, c]   (library rows)
__global__ void k_adjoint_grad(int n, int K, int nrhs, const int* __restrict__ rowptr,
                               const int* __restrict__ col, const int* __restrict__ nzmap,
                               const double* __restrict__ lam, const double* __restrict__ x,
                               double* __restrict__ grad) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n) return;
  const double* li = lam + (size_t)w * K;
  for (int j = rowptr[w] + lane; j < rowptr[w + 1]; j += 32) {
    const double* xj = x + (size_t)col[j] * K;
    double s = 0;
    for (int c = 0; c < nrhs; ++c) s = fma(li[c], xj[c], s);
    grad[nzmap[j]] = -s;
  }
}

// ------------------------------------------------------------ workspace --
struct Workspace {
  int K = 0, prec = 64, n0 = 0, L = 0, pre = 1, post = 1;
  Arena ar;
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *b = nullptr;
  std::vector<void*> f, u, v;
  KState ks{};
  int* zero_flag = nullptr;
  double* stage = nullptr;
  size_t stage_elems = 0;
  int* h_done = nullptr;  // pinned
  std::vector<int> nzl;   // per level
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int gchunk = 0, gtimer = -1, gmaxit = -1;
  long long gkernels = 0;
  int* h_iter = nullptr;  // pinned
  double grtol = -1;
  std::vector<cudaEvent_t> gev;
  ~Workspace() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    for (auto e : gev) cudaEventDestroy(e);
    if (h_done) cudaFreeHost(h_done);
    if (h_iter) cudaFreeHost(h_iter);
  }
};

Plan::~Plan() = default;

template <typename TC>
static int pick_nzl(const Level& L, int K) {
  double avg = L.avg_row_len;
  int mx = max_nzl<TC>(K);
  int v;
  if (K == 1) {
    v = avg <= 12 ? 4 : avg <= 24 ? 8 : avg <= 48 ? 16 : 32;
  } else {
    v = avg >= 24 ? 4 : (avg >= 8 ? 2 : 1);
  }
  return std::min(v, mx);
}

static int round_k(int nrhs) {
  int K = 1;
  while (K < nrhs) K <<= 1;
  return K;
}

static Workspace& get_ws(Plan& P, int K, int prec, int pre, int post) {
  long long key = ((long long)K << 32) | ((long long)prec << 16) | ((long long)pre << 8) | post;
  auto it = P.ws.find(key);
  if (it != P.ws.end()) return *it->second;
  auto W = std::make_shared<Workspace>();
  W->K = K;
  W->prec = prec;
  W->pre = pre;
  W->post = post;
  W->n0 = P.lev[0].n;
  W->L = P.L;
  Arena& ar = W->ar;
  size_t n0k = (size_t)W->n0 * K;
  W->x = ar.alloc<double>(n0k);
  W->r = ar.alloc<double>(n0k);
  W->p = ar.alloc<double>(n0k);
  W->q = ar.alloc<double>(n0k);
  W->z = ar.alloc<double>(n0k);
  W->b = ar.alloc<double>(n0k);
  size_t es = prec == 64 ? 8 : 4;
  W->f.resize(P.L);
  W->u.resize(P.L);
  W->v.resize(P.L);
  for (int k = 0; k < P.L; ++k) {
    size_t nk = (size_t)P.lev[k].n * K;
    W->f[k] = (k == 0 && prec == 64) ? (void*)W->r : ar.raw(nk * es);
    W->u[k] = ar.raw(nk * es);
    W->v[k] = ar.raw(nk * es);
  }
  int ncta0 = P.lev[0].ncta;
  int nv = P.nsys * K;
  KState& ks = W->ks;
  ks.partial = ar.alloc<double>((size_t)ncta0 * 2 * K);
  ks.counter = ar.alloc<unsigned>(8);
  AMG_CUDA(cudaMemset(ks.counter, 0, 8 * sizeof(unsigned)));
  ks.rho = ar.alloc<double>(nv);
  ks.alpha = ar.alloc<double>(nv);
  ks.beta = ar.alloc<double>(nv);
  ks.bnorm = ar.alloc<double>(nv);
  ks.rnorm = ar.alloc<double>(nv);
  ks.conv = ar.alloc<int>(nv);
  ks.iters = ar.alloc<int>(nv);
  ks.status = ar.alloc<int>(nv);
  ks.active = ar.alloc<int>(P.nsys);
  ks.done = ar.alloc<int>(1);
  ks.iter = ar.alloc<int>(1);
  ks.sys_cta = P.sys_cta;
  ks.nsys = P.nsys;
  W->zero_flag = ar.alloc<int>(1);
  AMG_CUDA(cudaMemset(W->zero_flag, 0, sizeof(int)));
  AMG_CUDA(cudaMemset(ks.done, 0, sizeof(int)));
  AMG_CUDA(cudaMallocHost(&W->h_done, sizeof(int)));
  AMG_CUDA(cudaMallocHost(&W->h_iter, sizeof(int)));
  W->nzl.resize(P.L);
  for (int k = 0; k < P.L; ++k)
    W->nzl[k] = prec == 64 ? pick_nzl<double>(P.lev[k], K) : pick_nzl<float>(P.lev[k], K);
  AMG_CUDA(cudaDeviceSynchronize());
  P.ws[key] = W;
  return *W;
}

// ------------------------------------------------------------- timing --
struct TimedLaunch {
  amg_hierarchy* h;
  int id;
  cudaStream_t st;
  std::vector<cudaEvent_t>* pool;
  bool on;
  cudaEvent_t e1 = nullptr;
  TimedLaunch(amg_hierarchy* h_, int id_, cudaStream_t st_, std::vector<cudaEvent_t>* pool_)
      : h(h_), id(id_), st(st_), pool(pool_) {
    on = h && pool && h->timer.on && h->timer.kernel == id;
    if (on) {
      cudaEvent_t e0;
      AMG_CUDA(cudaEventCreate(&e0));
      AMG_CUDA(cudaEventCreate(&e1));
      pool->push_back(e0);
      pool->push_back(e1);
      // External records become event-record nodes when the stream is captured
      AMG_CUDA(cudaEventRecordWithFlags(e0, st, g_capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
    }
  }
  ~TimedLaunch() {
    if (on) cudaEventRecordWithFlags(e1, st, g_capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  }
};

// Adds the device time of the first ``keep`` event pairs of ``pool`` (all
// pairs when keep < 0) to the handle's timer.
static void harvest_events(amg_hierarchy* h, std::vector<cudaEvent_t>& pool, bool destroy, long long keep = -1) {
  if (!h) return;
  long long pairs = (long long)pool.size() / 2;
  if (keep >= 0 && keep < pairs) pairs = keep;
  for (long long i = 0; i < pairs; ++i) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) {
      h->timer.total_ms += ms;
      h->timer.launches += 1;
    } else {
      cudaGetLastError();
    }
  }
  if (destroy) {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
  }
}

// ------------------------------------------------------------ sequences --
template <typename TC>
static void enqueue_cycle(amg_hierarchy* h, Plan& P, Workspace& W, cudaStream_t st, int mode, const int* done,
                          const KState& ks, std::vector<cudaEvent_t>* pool) {
  const int L = P.L, K = W.K;
  if (L == 1) {
    launch_coarse<double>(K, P.co, W.r, W.z, done, st);
    return;
  }
  std::vector<TC*> cur(L), oth(L);
  for (int k = 0; k < L; ++k) {
    cur[k] = static_cast<TC*>(W.u[k]);
    oth[k] = static_cast<TC*>(W.v[k]);
  }
  auto F = [&](int k) { return static_cast<TC*>(W.f[k]); };
  for (int k = 0; k + 1 < L; ++k) {
    for (int s = 1; s < W.pre; ++s) {
      launch_smooth<TC>(K, W.nzl[k], P.lev[k], F(k), cur[k], oth[k], done, st);
      std::swap(cur[k], oth[k]);
    }
    bool smooth_next = (k + 1 < L - 1);
    {
      TimedLaunch tl(h, k == 0 ? AMG_KERNEL_RESTRICT_L0 : -1, st, pool);
      launch_restrict<TC>(K, W.nzl[k], P.lev[k], P.tr[k], P.lev[k + 1], smooth_next, F(k), cur[k], F(k + 1),
                          cur[k + 1], done, st);
    }
  }
  launch_coarse<TC>(K, P.co, F(L - 1), cur[L - 1], done, st);
  TC* res = cur[L - 1];
  for (int k = L - 2; k >= 0; --k) {
    {
      TimedLaunch tl(h, k == 0 ? AMG_KERNEL_PROLONG_L0 : -1, st, pool);
      launch_prolong<TC>(K, P.tr[k], res, cur[k], done, st);
    }
    int sweeps = (k == 0) ? W.post - 1 : W.post;
    for (int s = 0; s < sweeps; ++s) {
      launch_smooth<TC>(K, W.nzl[k], P.lev[k], F(k), cur[k], oth[k], done, st);
      std::swap(cur[k], oth[k]);
    }
    res = cur[k];
  }
  TimedLaunch tl(h, AMG_KERNEL_SMOOTH_L0, st, pool);
  launch_post0<TC>(K, W.nzl[0], P.lev[0], F(0), cur[0], W.r, W.z, ks, mode, st);
}

static void launch_cg_q(Workspace& W, const Level& L, cudaStream_t st) {
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    dispatch_nzl(W.K, pick_nzl<double>(L, W.K), [&](auto nc) {
      constexpr int NZ = decltype(nc)::value;
      if constexpr (VT<double, KK>::CL * NZ <= 32) {
        k_cg_q<KK, NZ><<<L.ncta, BS, 0, st>>>(L.cta_row, L.rowptr, L.col, L.val64, W.p, W.q, W.ks);
      }
    });
  });
  AMG_LAUNCH_CHECK();
}

static void launch_cg_init(Workspace& W, const Level& L, cudaStream_t st) {
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    dispatch_nzl(W.K, pick_nzl<double>(L, W.K), [&](auto nc) {
      constexpr int NZ = decltype(nc)::value;
      if constexpr (VT<double, KK>::CL * NZ <= 32) {
        k_cg_init<KK, NZ><<<L.ncta, BS, 0, st>>>(L.cta_row, L.rowptr, L.col, L.val64, W.b, W.x, W.r, W.ks);
      }
    });
  });
  AMG_LAUNCH_CHECK();
}

static void launch_cg_p(Workspace& W, const Level& L, cudaStream_t st) {
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    k_cg_p<KK><<<L.ncta, BS, 0, st>>>(L.cta_row, W.z, W.p, W.ks);
  });
  AMG_LAUNCH_CHECK();
}

static void launch_rz(Workspace& W, const Level& L, int mode, cudaStream_t st) {
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    k_rz<KK><<<L.ncta, BS, 0, st>>>(L.cta_row, W.r, W.z, W.ks, mode);
  });
  AMG_LAUNCH_CHECK();
}

template <typename TC>
static void enqueue_start(amg_hierarchy* h, Plan& P, Workspace& W, cudaStream_t st) {
  const Level& L0 = P.lev[0];
  launch_cg_init(W, L0, st);
  if (P.L == 1) {
    enqueue_cycle<TC>(h, P, W, st, 0, W.ks.done, W.ks, nullptr);
    launch_rz(W, L0, 0, st);
  } else {
    TC* f0 = (W.prec == 64) ? nullptr : static_cast<TC*>(W.f[0]);
    launch_presmooth0<TC>(W.K, L0, W.r, static_cast<TC*>(W.u[0]), f0, W.ks.done, st);
    enqueue_cycle<TC>(h, P, W, st, 0, W.ks.done, W.ks, nullptr);
  }
  launch_cg_p(W, L0, st);
}

template <typename TC>
static void enqueue_iteration(amg_hierarchy* h, Plan& P, Workspace& W, cudaStream_t st,
                              std::vector<cudaEvent_t>* pool) {
  const Level& L0 = P.lev[0];
  {
    TimedLaunch tl(h, AMG_KERNEL_SPMV_CG, st, pool);
    launch_cg_q(W, L0, st);
  }
  TC* f0 = (W.prec == 64 || P.L == 1) ? nullptr : static_cast<TC*>(W.f[0]);
  {
    TimedLaunch tl(h, AMG_KERNEL_CG_UPDATE, st, pool);
    TC* u0 = P.L == 1 ? nullptr : static_cast<TC*>(W.u[0]);
    launch_update<TC>(W.K, L0, W.x, W.r, W.p, W.q, u0, f0, W.ks, st);
  }
  enqueue_cycle<TC>(h, P, W, st, 1, W.ks.done, W.ks, pool);
  if (P.L == 1) launch_rz(W, L0, 1, st);
  launch_cg_p(W, L0, st);
}

// ----------------------------------------------------------------- PCG --
struct StreamJoin {
  cudaStream_t user, own;
  cudaEvent_t ein, eout;
  StreamJoin(amg_hierarchy* h, cudaStream_t u) : user(u), own(h->own), ein(h->ev_in), eout(h->ev_out) {
    AMG_CUDA(cudaEventRecord(ein, user));
    AMG_CUDA(cudaStreamWaitEvent(own, ein, 0));
  }
  void finish() {
    AMG_CUDA(cudaEventRecord(eout, own));
    AMG_CUDA(cudaStreamWaitEvent(user, eout, 0));
    AMG_CUDA(cudaStreamSynchronize(own));
  }
};

static void stage_inputs(Plan& P, Workspace& W, const SolveReq& rq, cudaStream_t st) {
  const int K = W.K;
  // right-hand sides and initial guesses, permuted into library order
  size_t need = 0;
  for (int s = 0; s < rq.nsys; ++s) need = std::max(need, (size_t)rq.n_sys[s] * rq.nrhs[s]);
  for (int s = 0; s < rq.nsys; ++s) {
    int r0 = P.h_sys_row[s], r1 = P.h_sys_row[s + 1];
    size_t cnt = (size_t)rq.n_sys[s] * rq.nrhs[s];
    long long tot = (long long)(r1 - r0) * K;
    int grid = (int)((tot + 255) / 256);
    for (int which = 0; which < 2; ++which) {
      const double* src = which == 0 ? rq.b[s] : (rq.zero_x ? nullptr : rq.x[s]);
      double* dst = which == 0 ? W.b : W.x;
      if (src && !is_device_ptr(src)) {
        if (W.stage_elems < need) {
          W.stage = W.ar.alloc<double>(need);
          W.stage_elems = need;
        }
        copy_in(W.stage, src, cnt * 8, st);
        src = W.stage;
      }
      k_perm_in<<<grid, 256, 0, st>>>(r0, r1, K, rq.nrhs[s], P.perm0, src, dst);
      AMG_LAUNCH_CHECK();
    }
  }
}

static void stage_outputs(Plan& P, Workspace& W, const SolveReq& rq, const double* from, cudaStream_t st) {
  const int K = W.K;
  for (int s = 0; s < rq.nsys; ++s) {
    int r0 = P.h_sys_row[s], r1 = P.h_sys_row[s + 1];
    size_t cnt = (size_t)rq.n_sys[s] * rq.nrhs[s];
    long long tot = (long long)(r1 - r0) * rq.nrhs[s];
    int grid = (int)((tot + 255) / 256);
    double* dst = rq.x[s];
    bool host = !is_device_ptr(dst);
    if (host) {
      size_t need = 0;
      for (int t = 0; t < rq.nsys; ++t) need = std::max(need, (size_t)rq.n_sys[t] * rq.nrhs[t]);
      if (W.stage_elems < need) {
        W.stage = W.ar.alloc<double>(need);
        W.stage_elems = need;
      }
      dst = W.stage;
    }
    if (tot > 0) k_perm_out<<<grid, 256, 0, st>>>(r0, r1, K, rq.nrhs[s], P.perm0, from, dst);
    AMG_LAUNCH_CHECK();
    if (host) {
      copy_out(rq.x[s], W.stage, cnt * 8, st);
      AMG_CUDA(cudaStreamSynchronize(st));
    }
  }
}

template <typename TC>
static void pcg_loop(amg_hierarchy* h, Plan& P, Workspace& W, const amg_opts& o, cudaStream_t st) {
  enqueue_start<TC>(h, P, W, st);
  const int chunk = std::max(1, o.check_every);
  std::vector<cudaEvent_t> pool;
  bool timing = h && h->timer.on;
  if (o.use_graph) {
    int tkey = timing ? h->timer.kernel : 0;
    if (!W.gexec || W.gchunk != chunk || W.gtimer != tkey || W.gmaxit != o.maxit || W.grtol != o.rtol) {
      if (W.gexec) cudaGraphExecDestroy(W.gexec);
      if (W.graph) cudaGraphDestroy(W.graph);
      for (auto e : W.gev) cudaEventDestroy(e);
      W.gev.clear();
      W.gexec = nullptr;
      W.graph = nullptr;
      AMG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      g_capturing = true;
      try {
        for (int c = 0; c < chunk; ++c) enqueue_iteration<TC>(timing ? h : nullptr, P, W, st, timing ? &W.gev : nullptr);
      } catch (...) {
        g_capturing = false;
        cudaGraph_t g;
        cudaStreamEndCapture(st, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      g_capturing = false;
      AMG_CUDA(cudaStreamEndCapture(st, &W.graph));
      AMG_CUDA(cudaGraphInstantiate(&W.gexec, W.graph, 0));
      size_t nn = 0;
      AMG_CUDA(cudaGraphGetNodes(W.graph, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      AMG_CUDA(cudaGraphGetNodes(W.graph, nodes.data(), &nn));
      W.gkernels = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType ty;
        AMG_CUDA(cudaGraphNodeGetType(nd, &ty));
        if (ty == cudaGraphNodeTypeKernel) ++W.gkernels;
      }
      W.gchunk = chunk;
      W.gtimer = tkey;
      W.gmaxit = o.maxit;
      W.grtol = o.rtol;
    }
  }
  int it = 0, done_iters = 0;
  while (true) {
    if (o.use_graph) {
      AMG_CUDA(cudaGraphLaunch(W.gexec, st));
      add_launches(W.gkernels);
    } else {
      for (int c = 0; c < chunk; ++c) enqueue_iteration<TC>(timing ? h : nullptr, P, W, st, timing ? &pool : nullptr);
    }
    it += chunk;
    AMG_CUDA(cudaMemcpyAsync(W.h_done, W.ks.done, sizeof(int), cudaMemcpyDeviceToHost, st));
    AMG_CUDA(cudaMemcpyAsync(W.h_iter, W.ks.iter, sizeof(int), cudaMemcpyDeviceToHost, st));
    AMG_CUDA(cudaStreamSynchronize(st));
    if (timing) {
      // iterations of this chunk that did work (the rest exit at once)
      long long worked = std::max(0, std::min(chunk, *W.h_iter - done_iters));
      if (o.use_graph) harvest_events(h, W.gev, false, worked);
      else harvest_events(h, pool, true, worked);
    }
    done_iters = *W.h_iter;
    if (*W.h_done || it >= o.maxit + chunk) break;
  }
}

amg_status run_pcg(amg_hierarchy* owner, Plan& P, const SolveReq& rq, const amg_opts& o, cudaStream_t user,
                   amg_info* info) {
  int maxr = 0;
  for (int s = 0; s < rq.nsys; ++s) maxr = std::max(maxr, rq.nrhs[s]);
  AMG_REQUIRE(maxr >= 1 && maxr <= 32, "nrhs must be in [1, 32] per call");
  AMG_REQUIRE(o.cycle_precision == 64 || o.cycle_precision == 32, "cycle_precision must be 64 or 32");
  AMG_REQUIRE(o.pre >= 1 && o.post >= 1 && o.pre <= 16 && o.post <= 16, "pre and post sweeps must be in [1, 16]");
  AMG_REQUIRE(o.maxit >= 1 && o.rtol >= 0, "maxit must be >= 1 and rtol >= 0");
  const int K = round_k(maxr);
  Workspace& W = get_ws(P, K, o.cycle_precision, o.pre, o.post);
  W.ks.rtol = o.rtol;
  W.ks.maxit = o.maxit;
  StreamJoin sj(owner, user);
  cudaStream_t st = owner->own;
  std::vector<int> act(rq.nrhs.begin(), rq.nrhs.end());
  AMG_CUDA(cudaMemcpyAsync(W.ks.active, act.data(), act.size() * 4, cudaMemcpyHostToDevice, st));
  stage_inputs(P, W, rq, st);
  if (o.cycle_precision == 64) pcg_loop<double>(owner, P, W, o, st);
  else pcg_loop<float>(owner, P, W, o, st);
  stage_outputs(P, W, rq, W.x, st);
  // results
  int nv = P.nsys * K;
  std::vector<int> conv(nv), iters(nv), status(nv);
  std::vector<double> rn(nv), bn(nv);
  AMG_CUDA(cudaMemcpyAsync(conv.data(), W.ks.conv, nv * 4, cudaMemcpyDeviceToHost, st));
  AMG_CUDA(cudaMemcpyAsync(iters.data(), W.ks.iters, nv * 4, cudaMemcpyDeviceToHost, st));
  AMG_CUDA(cudaMemcpyAsync(status.data(), W.ks.status, nv * 4, cudaMemcpyDeviceToHost, st));
  AMG_CUDA(cudaMemcpyAsync(rn.data(), W.ks.rnorm, nv * 8, cudaMemcpyDeviceToHost, st));
  AMG_CUDA(cudaMemcpyAsync(bn.data(), W.ks.bnorm, nv * 8, cudaMemcpyDeviceToHost, st));
  sj.finish();
  amg_status res = AMG_OK;
  int idx = 0;
  for (int s = 0; s < rq.nsys; ++s) {
    for (int c = 0; c < rq.nrhs[s]; ++c) {
      int v = s * K + c;
      amg_info in{};
      in.iters = iters[v];
      in.converged = conv[v] == ST_CONVERGED;
      in.status = conv[v] == ST_ACTIVE ? AMG_ERR_NOT_CONVERGED : status[v];
      in.relres = bn[v] > 0 ? rn[v] / bn[v] : 0.0;
      if (in.status == AMG_ERR_BREAKDOWN) res = AMG_ERR_BREAKDOWN;
      else if (in.status != AMG_OK && res == AMG_OK) res = (amg_status)in.status;
      if (info) info[idx] = in;
      ++idx;
    }
  }
  return res;
}

// z = B r, one V-cycle in the requested precision (caller numbering).
void run_vcycle(amg_hierarchy* owner, Plan& P, const double* r, double* z, int nrhs, const amg_opts& o,
                cudaStream_t user) {
  AMG_REQUIRE(nrhs >= 1 && nrhs <= 32, "nrhs must be in [1, 32]");
  AMG_REQUIRE(o.cycle_precision == 64 || o.cycle_precision == 32, "cycle_precision must be 64 or 32");
  AMG_REQUIRE(o.pre >= 1 && o.post >= 1, "pre and post sweeps must be >= 1");
  const int K = round_k(nrhs);
  Workspace& W = get_ws(P, K, o.cycle_precision, o.pre, o.post);
  StreamJoin sj(owner, user);
  cudaStream_t st = owner->own;
  SolveReq rq;
  rq.nsys = 1;
  rq.n_sys = {P.lev[0].n};
  rq.b = {r};
  rq.x = {z};
  rq.nrhs = {nrhs};
  rq.zero_x = true;
  stage_inputs(P, W, rq, st);
  // the bare cycle reads its input from r
  AMG_CUDA(cudaMemcpyAsync(W.r, W.b, (size_t)W.n0 * K * 8, cudaMemcpyDeviceToDevice, st));
  KState ks = W.ks;
  ks.done = W.zero_flag;
  if (P.L == 1) {
    launch_coarse<double>(K, P.co, W.r, W.z, W.zero_flag, st);
  } else if (o.cycle_precision == 64) {
    launch_presmooth0<double>(K, P.lev[0], W.r, static_cast<double*>(W.u[0]), nullptr, W.zero_flag, st);
    enqueue_cycle<double>(nullptr, P, W, st, 2, W.zero_flag, ks, nullptr);
  } else {
    launch_presmooth0<float>(K, P.lev[0], W.r, static_cast<float*>(W.u[0]), static_cast<float*>(W.f[0]),
                             W.zero_flag, st);
    enqueue_cycle<float>(nullptr, P, W, st, 2, W.zero_flag, ks, nullptr);
  }
  stage_outputs(P, W, rq, W.z, st);
  sj.finish();
}

void run_adjoint_grad(amg_hierarchy* h, const double* lam_caller, const double* x_caller, int nrhs,
                      double* grad, cudaStream_t user) {
  Plan& P = h->plan;
  const int K = round_k(nrhs);
  Workspace& W = get_ws(P, K, 64, 1, 1);
  StreamJoin sj(h, user);
  cudaStream_t st = h->own;
  SolveReq rq;
  rq.nsys = 1;
  rq.n_sys = {P.lev[0].n};
  rq.b = {lam_caller};
  rq.x = {const_cast<double*>(x_caller)};
  rq.nrhs = {nrhs};
  rq.zero_x = false;
  stage_inputs(P, W, rq, st);  // lambda -> W.b, x -> W.x (library order)
  double* g = grad;
  Arena tmp;
  bool host = !is_device_ptr(grad);
  if (host) g = tmp.alloc<double>(h->nnz);
  const Level& L0 = P.lev[0];
  k_adjoint_grad<<<(L0.n * 32 + 255) / 256, 256, 0, st>>>(L0.n, K, nrhs, L0.rowptr, L0.col, h->nzmap, W.b, W.x, g);
  AMG_LAUNCH_CHECK();
  if (host) copy_out(grad, g, (size_t)h->nnz * 8, st);
  sj.finish();
}

}  // namespace amg

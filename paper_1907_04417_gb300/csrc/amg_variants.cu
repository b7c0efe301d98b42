// Cycle variants of Section 5 on the device, in float64:
//  * forward/backward Gauss-Seidel smoothing, here visiting the rows colour
//    by colour (rows of one colour share no edge, so each colour is one
//    data-parallel launch);
//  * the K-cycle: on every level but the coarsest the coarse-grid correction
//    is two flexible-CG iterations preconditioned by the cycle one level
//    down (a nonlinear AMLI cycle).
// Restriction, prolongation, the l1-Jacobi sweeps and the coarsest solve are
// the V-cycle's own launchers; this file adds the colouring (and the rows of
// every colour, listed once at setup), the colour sweeps, the level SpMV, the
// column inner products and the flexible-CG updates.
#include <algorithm>
#include <vector>

#include "amg_launch.cuh"

namespace amg {

namespace {

constexpr int VB = 256;

inline unsigned grid_of(long long m) { return (unsigned)((m + VB - 1) / VB); }

// SplitMix64 (Steele, Lea & Flood 2014): the state advanced by the
// golden-ratio increment, then the variant-13 finaliser.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// One round of the greedy colouring in decreasing priority
// (splitmix64(canon_i), canon_i).  A row all of whose higher-priority
// neighbours were coloured in earlier rounds takes the smallest colour none
// of its neighbours coloured so far holds; every other uncoloured row counts
// itself in ``waiting``.  A row coloured in this round is never needed by
// another row of this round: its higher-priority neighbours wait for
// nothing of it, and its lower-priority neighbours wait for it (they read
// round_of = -1 or ``round``, and both mean "not yet").  The colours equal
// those of visiting the rows one by one in priority order.
__global__ void k_colour_round(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                               const int* __restrict__ canon, int* colour, int* round_of, int round,
                               int* __restrict__ waiting) {
  const int v = blockIdx.x * VB + threadIdx.x;
  if (v >= n || round_of[v] >= 0) return;
  const int cv = canon[v];
  const unsigned long long kv = splitmix64((unsigned long long)cv);
  const int jb = rowptr[v], je = rowptr[v + 1];
  for (int j = jb; j < je; ++j) {
    const int u = col[j];
    if (u == v) continue;
    const int cu = canon[u];
    const unsigned long long ku = splitmix64((unsigned long long)cu);
    if (ku > kv || (ku == kv && cu > cv)) {
      const int ru = round_of[u];
      if (ru < 0 || ru >= round) {
        atomicAdd(waiting, 1);
        return;
      }
    }
  }
  int c = -1;
  for (int base = 0; c < 0; base += 64) {  // colour windows of 64; ends after at most degree / 64 + 1
    unsigned long long used = 0;
    for (int j = jb; j < je; ++j) {
      const int u = col[j];
      if (u == v) continue;
      const int ru = round_of[u];
      if (ru >= 0 && ru < round) {
        const int q = colour[u] - base;
        if (q >= 0 && q < 64) used |= 1ull << q;
      }
    }
    if (~used) c = base + __ffsll((long long)~used) - 1;
  }
  colour[v] = c;
  round_of[v] = round;
}

// diag[i] = a_ii; a missing or non-positive diagonal raises ``bad``.
__global__ void k_diag(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                       const double* __restrict__ val, double* __restrict__ diag, int* __restrict__ bad) {
  const int i = blockIdx.x * VB + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int j = rowptr[i]; j < rowptr[i + 1]; ++j)
    if (col[j] == i) d = val[j];
  if (!(d > 0.0)) {
    atomicOr(bad, 1);
    d = 1.0;
  }
  diag[i] = d;
}

// The rows of one colour (listed in ``rows``, ascending):
// u_i <- u_i + (f_i - (A u)_i) / a_ii, one thread per (listed row, column);
// the K threads of a row touch K contiguous values.
__global__ void k_gs_rows(int cnt, int K, const int* __restrict__ rows, const int* __restrict__ rowptr,
                          const int* __restrict__ col, const double* __restrict__ val,
                          const double* __restrict__ diag, const double* __restrict__ f, double* u,
                          const int* __restrict__ done) {
  if (*done) return;
  const long long t = (long long)blockIdx.x * VB + threadIdx.x;
  if (t >= (long long)cnt * K) return;
  const int i = rows[t / K], q = (int)(t % K);
  const size_t e = (size_t)i * K + q;
  double s = f[e];
  for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) s -= val[j] * u[(size_t)col[j] * K + q];
  u[e] = u[e] + s / diag[i];
}

// u = D^{-1} f (the first l1-Jacobi sweep from zero)
__global__ void k_scale_rows(int n, int K, const double* __restrict__ dinv, const double* __restrict__ f,
                             double* __restrict__ u, const int* __restrict__ done) {
  if (*done) return;
  const long long t = (long long)blockIdx.x * VB + threadIdx.x;
  if (t >= (long long)n * K) return;
  u[t] = dinv[t / K] * f[t];
}

// y = A x
__global__ void k_spmv_level(int n, int K, const int* __restrict__ rowptr, const int* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ x,
                             double* __restrict__ y, const int* __restrict__ done) {
  if (*done) return;
  const long long t = (long long)blockIdx.x * VB + threadIdx.x;
  if (t >= (long long)n * K) return;
  const int i = (int)(t / K), q = (int)(t % K);
  double s = 0.0;
  for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) s = fma(val[j], x[(size_t)col[j] * K + q], s);
  y[t] = s;
}

// Per-CTA partial inner products x_d . y_d per column over a fixed row
// range (ND pairs), summed in CTA order by k_dots_finish: deterministic.
template <int ND>
__global__ void k_dots(int n, int K, int rows_per_cta, const double* __restrict__ x0, const double* __restrict__ y0,
                       const double* __restrict__ x1, const double* __restrict__ y1, double* __restrict__ partial,
                       const int* __restrict__ done) {
  if (*done) return;
  __shared__ double sm[ND][VB];
  const int c = threadIdx.x % K, lane_rows = VB / K, rr = threadIdx.x / K;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  double s[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) s[d] = 0.0;
  if (rr < lane_rows)
    for (int i = r0 + rr; i < r1; i += lane_rows) {
      const size_t e = (size_t)i * K + c;
      s[0] = fma(x0[e], y0[e], s[0]);
      if constexpr (ND > 1) s[1] = fma(x1[e], y1[e], s[1]);
    }
#pragma unroll
  for (int d = 0; d < ND; ++d) sm[d][threadIdx.x] = s[d];
  __syncthreads();
  if (threadIdx.x < K) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      double t = 0.0;
      for (int q = 0; q < lane_rows; ++q) t += sm[d][q * K + threadIdx.x];
      partial[((size_t)blockIdx.x * ND + d) * K + threadIdx.x] = t;
    }
  }
}

template <int ND>
__global__ void k_dots_finish(int ncta, int K, const double* __restrict__ partial, double* __restrict__ out,
                              const int* __restrict__ done) {
  if (*done) return;
  const int t = threadIdx.x;
  if (t >= ND * K) return;
  const int d = t / K, c = t % K;
  double s = 0.0;
  for (int b = 0; b < ncta; ++b) s += partial[((size_t)b * ND + d) * K + c];
  out[(size_t)d * K + c] = s;
}

// Inner products of one level, laid out per column: D[0] = c1.A c1,
// D[1] = c1.r, D[2] = c2.A c1, D[3] = d2.A d2, D[4] = d2.r2 (K values each).
enum { D_DAD1 = 0, D_C1R = 1, D_GAM = 2, D_DAD2 = 3, D_D2R = 4 };

__device__ __forceinline__ double safe_ratio(double num, double den) { return den > 0.0 ? num / den : 0.0; }

// First flexible-CG step from e = 0 along d1 = c1:
// alpha1 = c1.r / c1.A c1, e = alpha1 c1, r2 = r - alpha1 A c1.
__global__ void k_fcg_first(int n, int K, const double* __restrict__ r, const double* __restrict__ c1,
                            const double* __restrict__ v1, const double* __restrict__ D, double* __restrict__ e,
                            double* __restrict__ r2, const int* __restrict__ done) {
  if (*done) return;
  const long long t = (long long)blockIdx.x * VB + threadIdx.x;
  if (t >= (long long)n * K) return;
  const int q = (int)(t % K);
  const double a1 = safe_ratio(D[D_C1R * K + q], D[D_DAD1 * K + q]);
  e[t] = a1 * c1[t];
  r2[t] = r[t] - a1 * v1[t];
}

// d2 = c2 - g c1 and A d2 = A c2 - g A c1 with g = c2.A c1 / c1.A c1 (in place).
__global__ void k_fcg_orth(int n, int K, const double* __restrict__ c1, const double* __restrict__ v1,
                           const double* __restrict__ D, double* __restrict__ c2, double* __restrict__ v2,
                           const int* __restrict__ done) {
  if (*done) return;
  const long long t = (long long)blockIdx.x * VB + threadIdx.x;
  if (t >= (long long)n * K) return;
  const int q = (int)(t % K);
  const double g = safe_ratio(D[D_GAM * K + q], D[D_DAD1 * K + q]);
  c2[t] = c2[t] - g * c1[t];
  v2[t] = v2[t] - g * v1[t];
}

// e += alpha2 d2, alpha2 = d2.r2 / d2.A d2.
__global__ void k_fcg_second(int n, int K, const double* __restrict__ d2, const double* __restrict__ D,
                             double* __restrict__ e, const int* __restrict__ done) {
  if (*done) return;
  const long long t = (long long)blockIdx.x * VB + threadIdx.x;
  if (t >= (long long)n * K) return;
  const int q = (int)(t % K);
  e[t] = e[t] + safe_ratio(D[D_D2R * K + q], D[D_DAD2 * K + q]) * d2[t];
}

// Library row -> row in the caller's numbering of level k (the order in
// which the coarse dofs are numbered aggregate by aggregate, the kept
// columns of an aggregate in descending singular-value order).
std::vector<int> canonical_rows(const amg_hierarchy* h, const Plan& P, int k) {
  if (k == 0) return h->h_perm[0];
  const Transfer& T = P.tr[k - 1];
  const std::vector<int>& agg = h->h_perm[k];
  const std::vector<int>& r = h->h_r[k];
  const int nagg = T.nagg;
  std::vector<int> rc(nagg, 0), ostart(nagg + 1, 0);
  for (int t = 0; t < nagg; ++t) rc[agg[t]] = r[t];
  for (int a = 0; a < nagg; ++a) ostart[a + 1] = ostart[a] + rc[a];
  std::vector<int> canon(P.lev[k].n);
  for (int t = 0; t < nagg; ++t)
    for (int q = T.h_coarse_start[t]; q < T.h_coarse_start[t + 1]; ++q)
      canon[q] = ostart[agg[t]] + (q - T.h_coarse_start[t]);
  return canon;
}

void dots(const VarCycle& vc, int n, int nd, const double* x0, const double* y0, const double* x1,
          const double* y1, double* out, const int* done, cudaStream_t st) {
  const int K = vc.K;
  const int ncta = (n + vc.dot_rows - 1) / vc.dot_rows;
  if (nd == 1) {
    k_dots<1><<<ncta, VB, 0, st>>>(n, K, vc.dot_rows, x0, y0, nullptr, nullptr, vc.partial, done);
    AMG_LAUNCH_CHECK();
    k_dots_finish<1><<<1, 64, 0, st>>>(ncta, K, vc.partial, out, done);
  } else {
    k_dots<2><<<ncta, VB, 0, st>>>(n, K, vc.dot_rows, x0, y0, x1, y1, vc.partial, done);
    AMG_LAUNCH_CHECK();
    k_dots_finish<2><<<1, 64, 0, st>>>(ncta, K, vc.partial, out, done);
  }
  AMG_LAUNCH_CHECK();
}

void gs_sweep(const Plan& P, int k, int K, const double* f, double* u, bool backward, const int* done,
              cudaStream_t st) {
  const Level& L = P.lev[k];
  const int nc = P.gs_ncol[k];
  const std::vector<int>& cs = P.gs_cstart[k];
  for (int q = 0; q < nc; ++q) {
    const int c = backward ? nc - 1 - q : q;
    const int cnt = cs[c + 1] - cs[c];
    if (cnt == 0) continue;
    k_gs_rows<<<grid_of((long long)cnt * K), VB, 0, st>>>(cnt, K, P.gs_rows[k] + cs[c], L.rowptr, L.col, L.val64,
                                                          P.gs_diag[k], f, u, done);
    AMG_LAUNCH_CHECK();
  }
}

void level_cycle(const Plan& P, const VarCycle& vc, int k, const double* f, double* out, double* tmp,
                 const int* done, cudaStream_t st, amg_hierarchy* h = nullptr,
                 std::vector<cudaEvent_t>* pool = nullptr);

// Two flexible-CG iterations on A_j e = f_j from e = 0, each preconditioned
// by one cycle on level j; e goes to vc.e[j].
void fcg2(const Plan& P, const VarCycle& vc, int j, const int* done, cudaStream_t st) {
  const Level& L = P.lev[j];
  const int K = vc.K;
  const long long m = (long long)L.n * K;
  const double* r = vc.f[j];
  double *c1 = vc.u[j], *c2 = vc.c2[j], *v1 = vc.v1[j], *v2 = vc.v2[j], *r2 = vc.r2[j], *e = vc.e[j];
  double* D = vc.dots[j];
  level_cycle(P, vc, j, r, c1, vc.v[j], done, st);
  k_spmv_level<<<grid_of(m), VB, 0, st>>>(L.n, K, L.rowptr, L.col, L.val64, c1, v1, done);
  AMG_LAUNCH_CHECK();
  dots(vc, L.n, 2, c1, v1, c1, r, D + D_DAD1 * K, done, st);  // D_DAD1, D_C1R adjacent
  k_fcg_first<<<grid_of(m), VB, 0, st>>>(L.n, K, r, c1, v1, D, e, r2, done);
  AMG_LAUNCH_CHECK();
  level_cycle(P, vc, j, r2, c2, vc.v[j], done, st);
  k_spmv_level<<<grid_of(m), VB, 0, st>>>(L.n, K, L.rowptr, L.col, L.val64, c2, v2, done);
  AMG_LAUNCH_CHECK();
  dots(vc, L.n, 1, c2, v1, nullptr, nullptr, D + D_GAM * K, done, st);
  k_fcg_orth<<<grid_of(m), VB, 0, st>>>(L.n, K, c1, v1, D, c2, v2, done);
  AMG_LAUNCH_CHECK();
  dots(vc, L.n, 2, c2, v2, c2, r2, D + D_DAD2 * K, done, st);  // D_DAD2, D_D2R adjacent
  k_fcg_second<<<grid_of(m), VB, 0, st>>>(L.n, K, c2, D, e, done);
  AMG_LAUNCH_CHECK();
}

// One cycle on level k for right-hand side f; the result lands in ``out``
// (``tmp`` is the level's second buffer of the out-of-place Jacobi sweeps).
// With h and pool, the last backward Gauss-Seidel sweep (one per cycle) is
// timed as AMG_KERNEL_GS_L0.
void level_cycle(const Plan& P, const VarCycle& vc, int k, const double* f, double* out, double* tmp,
                 const int* done, cudaStream_t st, amg_hierarchy* h, std::vector<cudaEvent_t>* pool) {
  const int K = vc.K;
  if (k == P.L - 1) {
    launch_coarse<double>(K, P.co, f, out, done, st);
    return;
  }
  const Level& L = P.lev[k];
  const long long m = (long long)L.n * K;
  double *a = out, *b = tmp;
  if (vc.smoother == 1) {
    AMG_CUDA(cudaMemsetAsync(a, 0, (size_t)m * sizeof(double), st));
    for (int s = 0; s < vc.pre; ++s) gs_sweep(P, k, K, f, a, false, done, st);
  } else {
    // every out-of-place sweep swaps the buffers: start where the last one ends in out
    if (((vc.pre - 1) + vc.post) % 2) std::swap(a, b);
    k_scale_rows<<<grid_of(m), VB, 0, st>>>(L.n, K, L.dinv64, f, a, done);
    AMG_LAUNCH_CHECK();
    for (int s = 1; s < vc.pre; ++s) {
      launch_smooth<double>(K, vc.nzl[k], L, vc.rp[k], f, a, b, done, st);
      std::swap(a, b);
    }
  }
  launch_restrict<double>(K, vc.nzl[k], L, P.tr[k], vc.tp[k], P.lev[k + 1], false, f, a, vc.f[k + 1], nullptr,
                          done, st);
  const double* ec;
  if (vc.kind == 1 && k + 1 < P.L - 1) {
    fcg2(P, vc, k + 1, done, st);
    ec = vc.e[k + 1];
  } else {
    level_cycle(P, vc, k + 1, vc.f[k + 1], vc.u[k + 1], vc.v[k + 1], done, st);
    ec = vc.u[k + 1];
  }
  launch_prolong<double>(K, P.tr[k], vc.tp[k], ec, a, done, st);
  for (int s = 0; s < vc.post; ++s) {
    if (vc.smoother == 1) {
      TimedLaunch tl(s + 1 == vc.post ? h : nullptr, AMG_KERNEL_GS_L0, st, pool);
      gs_sweep(P, k, K, f, a, true, done, st);
    } else {
      launch_smooth<double>(K, vc.nzl[k], L, vc.rp[k], f, a, b, done, st);
      std::swap(a, b);
    }
  }
}

}  // namespace

void ensure_gs(amg_hierarchy* h, Plan& P, cudaStream_t st) {
  if (P.gs_done) return;
  AMG_REQUIRE(h && &h->plan == &P && P.nsys == 1, "Gauss-Seidel smoothing needs a single hierarchy");
  const int ns = std::max(P.L - 1, 0);
  P.gs_colour.assign(ns, nullptr);
  P.gs_diag.assign(ns, nullptr);
  P.gs_ncol.assign(ns, 0);
  P.gs_rows.assign(ns, nullptr);
  P.gs_cstart.assign(ns, {});
  Arena tmp;
  int* flag = tmp.alloc<int>(2);
  int* h_flag = nullptr;
  AMG_CUDA(cudaMallocHost(&h_flag, 2 * sizeof(int)));
  try {
    for (int k = 0; k < ns; ++k) {
      const Level& L = P.lev[k];
      const int n = L.n;
      std::vector<int> canon = canonical_rows(h, P, k);
      int* d_canon = tmp.alloc<int>(n);
      AMG_CUDA(cudaMemcpyAsync(d_canon, canon.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st));
      int* colour = P.arena->alloc<int>(n);
      int* round_of = tmp.alloc<int>(n);
      AMG_CUDA(cudaMemsetAsync(colour, 0xff, (size_t)n * 4, st));
      AMG_CUDA(cudaMemsetAsync(round_of, 0xff, (size_t)n * 4, st));
      // every round colours at least the highest-priority uncoloured row
      for (int round = 0;; ++round) {
        AMG_REQUIRE(round <= n, "internal: the colouring made no progress");
        AMG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
        k_colour_round<<<grid_of(n), VB, 0, st>>>(n, L.rowptr, L.col, d_canon, colour, round_of, round, flag);
        AMG_LAUNCH_CHECK();
        AMG_CUDA(cudaMemcpyAsync(h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        AMG_CUDA(cudaStreamSynchronize(st));
        if (h_flag[0] == 0) break;
      }
      std::vector<int> hc(n);
      AMG_CUDA(cudaMemcpyAsync(hc.data(), colour, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
      double* diag = P.arena->alloc<double>(n);
      AMG_CUDA(cudaMemsetAsync(flag + 1, 0, sizeof(int), st));
      k_diag<<<grid_of(n), VB, 0, st>>>(n, L.rowptr, L.col, L.val64, diag, flag + 1);
      AMG_LAUNCH_CHECK();
      AMG_CUDA(cudaMemcpyAsync(h_flag + 1, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
      AMG_CUDA(cudaStreamSynchronize(st));
      AMG_REQUIRE(h_flag[1] == 0, "Gauss-Seidel needs a positive diagonal on every smoothed level");
      int mx = -1;
      for (int c : hc) {
        AMG_REQUIRE(c >= 0, "internal: a row was left uncoloured");
        mx = std::max(mx, c);
      }
      // rows grouped by colour (a counting sort: ascending rows within a colour)
      std::vector<int> cs(mx + 2, 0), rows(n);
      for (int c : hc) cs[c + 1]++;
      for (int c = 0; c <= mx; ++c) cs[c + 1] += cs[c];
      std::vector<int> pos(cs.begin(), cs.end() - 1);
      for (int i = 0; i < n; ++i) rows[pos[hc[i]]++] = i;
      int* d_rows = P.arena->alloc<int>(n);
      AMG_CUDA(cudaMemcpyAsync(d_rows, rows.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st));
      AMG_CUDA(cudaStreamSynchronize(st));
      P.gs_colour[k] = colour;
      P.gs_diag[k] = diag;
      P.gs_ncol[k] = mx + 1;
      P.gs_rows[k] = d_rows;
      P.gs_cstart[k] = cs;
    }
  } catch (...) {
    cudaFreeHost(h_flag);
    throw;
  }
  cudaFreeHost(h_flag);
  P.gs_done = true;
}

size_t var_level_ctas(int n, const VarCycle& vc) { return (size_t)((n + vc.dot_rows - 1) / vc.dot_rows); }

void enqueue_var_cycle(const Plan& P, const VarCycle& vc, const double* r, double* z, double* u0, const int* done,
                       cudaStream_t st, amg_hierarchy* h, std::vector<cudaEvent_t>* pool) {
  AMG_REQUIRE(vc.smoother == 0 || P.gs_done, "internal: Gauss-Seidel data missing");
  AMG_REQUIRE(vc.f.size() == (size_t)P.L && vc.f[0] == r, "internal: variant workspace mismatch");
  level_cycle(P, vc, 0, r, z, u0, done, st, h, pool);
}

int level_colours(amg_hierarchy* h, int k, int32_t* colour, cudaStream_t st) {
  Plan& P = h->plan;
  AMG_REQUIRE(k >= 0 && k < P.L - 1, "colours exist on the smoothed levels 0 .. levels-2");
  ensure_gs(h, P, st);
  const int n = P.lev[k].n;
  std::vector<int> hc(n);
  AMG_CUDA(cudaMemcpyAsync(hc.data(), P.gs_colour[k], (size_t)n * 4, cudaMemcpyDeviceToHost, st));
  AMG_CUDA(cudaStreamSynchronize(st));
  if (colour) {
    std::vector<int> canon = canonical_rows(h, P, k);
    for (int i = 0; i < n; ++i) colour[canon[i]] = hc[i];
  }
  return P.gs_ncol[k];
}

}  // namespace amg

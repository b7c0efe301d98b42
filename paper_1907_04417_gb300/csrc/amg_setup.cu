// Setup of the multiple-vector hierarchy on the device (Section 4 and 4.1):
// local SVD bases per aggregate (Eq. (svd) with the truncation rule of
// Section 5), block prolongators, Galerkin coarse matrices, coarse smooth
// vectors, l1-Jacobi diagonals and the float64 coarsest factorisation.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>

#include "amg_internal.cuh"
#include "amg_local_svd.cuh"

namespace amg {

// ----------------------------------------------------- launch accounting --
static std::atomic<long long> g_launches{0};
thread_local bool g_capturing = false;
void count_launch() {
  if (!g_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------ pointers --
bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes) AMG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
}
void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes) AMG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
}

template <typename T>
static std::vector<T> to_host(const T* p, size_t n, cudaStream_t st) {
  std::vector<T> v(n);
  if (n) {
    AMG_CUDA(cudaMemcpyAsync(v.data(), p, n * sizeof(T), cudaMemcpyDefault, st));
    AMG_CUDA(cudaStreamSynchronize(st));
  }
  return v;
}

// Non-zero arrays are padded by 16 elements (zeroed) so that 16-byte
// aligned bulk copies of a row range may run past its last entry.
template <typename T>
static T* alloc_nnz(Arena& ar, long long nnz, cudaStream_t st) {
  T* p = ar.alloc<T>(nnz + 16);
  AMG_CUDA(cudaMemsetAsync(p + nnz, 0, 16 * sizeof(T), st));
  return p;
}

template <typename T>
static T* to_dev(Arena& ar, const std::vector<T>& v, cudaStream_t st) {
  T* d = ar.alloc<T>(v.size() ? v.size() : 1);
  if (!v.empty()) AMG_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return d;
}

// ------------------------------------------------------------- kernels --
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// New row i of the permuted matrix: entries of caller row perm[i], columns
// renumbered by iperm and sorted; nzmap records the caller's entry index.
__global__ void k_permute_csr(int n, const int* __restrict__ rp_old, const int* __restrict__ col_old,
                              const double* __restrict__ val_old, const int* __restrict__ perm,
                              const int* __restrict__ iperm, const int* __restrict__ rp_new,
                              int* __restrict__ col_new, double* __restrict__ val_new,
                              int* __restrict__ nzmap, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = perm[i];
  int s = rp_old[o], e = rp_old[o + 1], d = rp_new[i];
  int prev = -1;
  for (int j = s; j < e; ++j) {
    int c = col_old[j];
    if (c < 0 || c >= n || c <= prev) {  // out of range, unsorted or duplicate
      atomicOr(flag, 1);
      return;
    }
    prev = c;
    int nc = iperm[c];
    double v = val_old[j];
    int t = d + (j - s);
    // insertion into the already written prefix [d, t)
    while (t > d && col_new[t - 1] > nc) {
      col_new[t] = col_new[t - 1];
      val_new[t] = val_new[t - 1];
      nzmap[t] = nzmap[t - 1];
      --t;
    }
    col_new[t] = nc;
    val_new[t] = v;
    nzmap[t] = j;
  }
}

// W (caller, n x m column-major) -> library order, row-major.
__global__ void k_gather_w(int n, int m, const double* __restrict__ W, const int* __restrict__ perm,
                           double* __restrict__ out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * m) return;
  int i = (int)(t / m), r = (int)(t % m);
  out[t] = W[(long long)r * n + perm[i]];
}

// Eq. (svd) for every aggregate: one warp per aggregate (local_svd_warp)
// computes the thin SVD of the n_a x m block by one-sided (Hestenes) Jacobi
// rotations on its columns, sorts by singular value, keeps those above
// TOL*n_a/n_f (at least one, at most min(n_a, m)), normalises them and flips
// each so that its largest-magnitude entry (lowest row on ties) is positive.
__global__ void k_local_svd(const double* __restrict__ W, int m, int nagg,
                            const int* __restrict__ row_start, int nf, double tol,
                            double* __restrict__ work, double* __restrict__ U,
                            int* __restrict__ rkeep) {
  int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (a >= nagg) return;
  int rs = row_start[a], na = row_start[a + 1] - rs;
  int r = local_svd_warp(W + (size_t)rs * m, m, na, nf, tol, work + (size_t)rs * m, U + (size_t)rs * m, lane);
  if (lane == 0) rkeep[a] = r;
}

// Kept columns into the blocked prolongator storage (n_a x r_a row-major).
__global__ void k_compact_p(int nagg, int m, const int* __restrict__ row_start,
                            const int* __restrict__ coarse_start,
                            const long long* __restrict__ blk_start, const double* __restrict__ U,
                            double* __restrict__ P) {
  int a = blockIdx.x;
  if (a >= nagg) return;
  int rs = row_start[a], na = row_start[a + 1] - rs;
  int ra = coarse_start[a + 1] - coarse_start[a];
  long long b = blk_start[a];
  for (int t = threadIdx.x; t < na * ra; t += blockDim.x) {
    int i = t / ra, p = t % ra;
    P[b + t] = U[(size_t)(rs + i) * m + p];
  }
}

// Coarse smooth vectors W^k = (P^k)^T W^{k-1} (Section 4.1).
__global__ void k_restrict_w(int nagg, int m, const int* __restrict__ row_start,
                             const int* __restrict__ coarse_start,
                             const long long* __restrict__ blk_start, const double* __restrict__ P,
                             const double* __restrict__ Wf, double* __restrict__ Wc) {
  int a = blockIdx.x;
  if (a >= nagg) return;
  int rs = row_start[a], na = row_start[a + 1] - rs;
  int cs = coarse_start[a], ra = coarse_start[a + 1] - cs;
  long long b = blk_start[a];
  for (int t = threadIdx.x; t < ra * m; t += blockDim.x) {
    int p = t / m, r = t % m;
    double s = 0;
    for (int i = 0; i < na; ++i) s = fma(P[b + (long long)i * ra + p], Wf[(size_t)(rs + i) * m + r], s);
    Wc[(size_t)(cs + p) * m + r] = s;
  }
}

// Galerkin symbolic phase: the set of aggregates b adjacent to aggregate a
// through A^{k-1}, gathered in a per-warp open-addressing table.
constexpr int GAL_CAP = 512;
constexpr int GAL_WARPS = 4;
__global__ void k_gal_sym(int nagg, const int* __restrict__ row_start, const int* __restrict__ rowptr,
                          const int* __restrict__ col, const int* __restrict__ owner,
                          const int* __restrict__ rcnt, int pass, int* __restrict__ cnt,
                          int* __restrict__ S, const int* __restrict__ nb_ptr,
                          int* __restrict__ nb_list, int* __restrict__ flag) {
  __shared__ int tab[GAL_WARPS][GAL_CAP];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int a = blockIdx.x * GAL_WARPS + w;
  if (a >= nagg) return;
  int* h = tab[w];
  for (int t = lane; t < GAL_CAP; t += 32) h[t] = -1;
  __syncwarp();
  int rs = row_start[a], re = row_start[a + 1];
  for (int i = rs; i < re; ++i) {
    for (int j = rowptr[i] + lane; j < rowptr[i + 1]; j += 32) {
      int b = owner[col[j]];
      unsigned slot = ((unsigned)b * 2654435761u) & (GAL_CAP - 1);
      int probe = 0;
      for (; probe < GAL_CAP; ++probe) {
        int old = atomicCAS(&h[slot], -1, b);
        if (old == -1 || old == b) break;
        slot = (slot + 1) & (GAL_CAP - 1);
      }
      if (probe == GAL_CAP) atomicOr(flag, 2);
    }
  }
  __syncwarp();
  int c = 0, s = 0;
  for (int t = lane; t < GAL_CAP; t += 32)
    if (h[t] >= 0) {
      ++c;
      s += rcnt[h[t]];
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if (pass == 0) {
    if (lane == 0) {
      cnt[a] = c;
      S[a] = s;
    }
    return;
  }
  int base = nb_ptr[a];
  for (int t = lane; t < GAL_CAP; t += 32) {
    int key = h[t];
    if (key < 0) continue;
    int rank = 0;
    for (int u = 0; u < GAL_CAP; ++u) rank += (h[u] >= 0 && h[u] < key);
    nb_list[base + rank] = key;
  }
}

// Column indices of the coarse rows: aggregate a's rows list the coarse dofs
// of every neighbouring aggregate, in increasing order.
__global__ void k_gal_cols(int nagg, const int* __restrict__ coarse_start, const int* __restrict__ nb_ptr,
                           const int* __restrict__ nb_list, const int* __restrict__ rowptr_c,
                           int* __restrict__ col_c) {
  int a = blockIdx.x;
  if (a >= nagg) return;
  int cs = coarse_start[a], ra = coarse_start[a + 1] - cs;
  int b0 = nb_ptr[a], b1 = nb_ptr[a + 1];
  int S = rowptr_c[cs + 1] - rowptr_c[cs];
  for (int t = threadIdx.x; t < ra * S; t += blockDim.x) {
    int p = t / S, s = t % S;
    // locate the neighbour owning slot s
    int acc = 0, k = b0;
    for (; k < b1; ++k) {
      int rb = coarse_start[nb_list[k] + 1] - coarse_start[nb_list[k]];
      if (s < acc + rb) break;
      acc += rb;
    }
    col_c[rowptr_c[cs + p] + s] = coarse_start[nb_list[k]] + (s - acc);
  }
}

// Galerkin numeric phase, one CTA per aggregate a:
//   T = A^{k-1}[rows(a), :] P restricted to the neighbours (rows owned by
//   threads, so the accumulation order is fixed), then C = P_a^T T.
__global__ void k_gal_num(int nagg, const int* __restrict__ row_start, const int* __restrict__ coarse_start,
                          const long long* __restrict__ blk_start, const double* __restrict__ P,
                          const int* __restrict__ rowptr, const int* __restrict__ col,
                          const double* __restrict__ val, const int* __restrict__ owner,
                          const int* __restrict__ nb_ptr, const int* __restrict__ nb_list,
                          const int* __restrict__ rowptr_c, double* __restrict__ val_c,
                          double* __restrict__ gscratch, const long long* __restrict__ t_off,
                          int use_smem) {
  extern __shared__ double dsm[];
  __shared__ int nbs[GAL_CAP];
  __shared__ int sbs[GAL_CAP + 1];
  int a = blockIdx.x;
  if (a >= nagg) return;
  int rs = row_start[a], na = row_start[a + 1] - rs;
  int cs = coarse_start[a], ra = coarse_start[a + 1] - cs;
  long long blk = blk_start[a];
  int b0 = nb_ptr[a], nnb = nb_ptr[a + 1] - b0;
  for (int t = threadIdx.x; t < nnb; t += blockDim.x) nbs[t] = nb_list[b0 + t];
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int t = 0; t < nnb; ++t) {
      sbs[t] = acc;
      acc += coarse_start[nbs[t] + 1] - coarse_start[nbs[t]];
    }
    sbs[nnb] = acc;
  }
  __syncthreads();
  int S = sbs[nnb];
  double* T = use_smem ? dsm : gscratch + t_off[a];
  for (int t = threadIdx.x; t < na * S; t += blockDim.x) T[t] = 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < na; i += blockDim.x) {
    int row = rs + i;
    double* Ti = T + (size_t)i * S;
    for (int j = rowptr[row]; j < rowptr[row + 1]; ++j) {
      int c = col[j];
      int b = owner[c];
      int lo = 0, hi = nnb - 1;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (nbs[mid] < b) lo = mid + 1; else hi = mid;
      }
      int rb = coarse_start[b + 1] - coarse_start[b];
      const double* pb = P + blk_start[b] + (long long)(c - row_start[b]) * rb;
      double v = val[j];
      double* dst = Ti + sbs[lo];
      for (int q = 0; q < rb; ++q) dst[q] = fma(v, pb[q], dst[q]);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ra * S; t += blockDim.x) {
    int p = t / S, s = t % S;
    double acc = 0;
    for (int i = 0; i < na; ++i) acc = fma(P[blk + (long long)i * ra + p], T[(size_t)i * S + s], acc);
    val_c[rowptr_c[cs + p] + s] = acc;
  }
}

// l1-Jacobi diagonal: d_i = sum_j |a_ij|; stores 1/d in float64 and float32.
__global__ void k_l1(int n, const int* __restrict__ rowptr, const double* __restrict__ val,
                     double* __restrict__ d64, float* __restrict__ d32, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0;
  for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) s += fabs(val[j]);
  if (!(s > 0.0) || !isfinite(s)) {
    atomicOr(flag, 4);
    s = 1.0;
  }
  d64[i] = 1.0 / s;
  d32[i] = (float)(1.0 / s);
}

// lo = a - (double)(float)a as a float: (val32, lo) is a double-float pair.
__global__ void k_split_lo(long long n, const double* __restrict__ a, const float* __restrict__ hi,
                           float* __restrict__ lo) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lo[i] = (float)(a[i] - (double)hi[i]);
}

template <typename TI, typename TO>
__global__ void k_cast(long long n, const TI* __restrict__ in, TO* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (TO)in[i];
}

__global__ void k_add_offset(long long n, const int* __restrict__ in, int off, int* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i] + off;
}

__global__ void k_densify(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                          const double* __restrict__ val, double* __restrict__ D) {
  int i = blockIdx.x;
  if (i >= n) return;
  for (int t = threadIdx.x; t < n; t += blockDim.x) D[(size_t)i * n + t] = 0.0;
  __syncthreads();
  for (int j = rowptr[i] + threadIdx.x; j < rowptr[i + 1]; j += blockDim.x) D[(size_t)i * n + col[j]] = val[j];
}

// Right-looking Cholesky of the dense coarsest matrix by one CTA; the lower
// factor overwrites the lower triangle.  A non-positive pivot sets flag 8.
__global__ void k_cholesky(int n, double* __restrict__ D, int* __restrict__ flag) {
  __shared__ double piv;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = D[(size_t)j * n + j];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicOr(flag, 8);
        d = 1.0;
      }
      piv = sqrt(d);
      D[(size_t)j * n + j] = piv;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) D[(size_t)i * n + j] /= piv;
    __syncthreads();
    int w = n - j - 1;
    long long tot = (long long)w * w;
    for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
      int i = j + 1 + (int)(t / w), k = j + 1 + (int)(t % w);
      if (k <= i) D[(size_t)i * n + k] -= D[(size_t)i * n + j] * D[(size_t)k * n + j];
    }
    __syncthreads();
  }
}

// Column c of the inverse from the Cholesky factor: L y = e_c, L^T x = y.
// One warp per column; the result is written as row c (the inverse is symmetric).
__global__ void k_chol_inverse(int n, const double* __restrict__ Lf, double* __restrict__ work,
                               double* __restrict__ inv) {
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= n) return;
  double* y = work + (size_t)c * n;
  for (int i = 0; i < n; ++i) {
    double s = 0;
    for (int k = lane; k < i; k += 32) s = fma(Lf[(size_t)i * n + k], y[k], s);
    s = warp_sum(s);
    double v = ((i == c) ? 1.0 : 0.0) - s;
    v /= Lf[(size_t)i * n + i];
    if (lane == 0) y[i] = v;
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = 0;
    for (int k = i + 1 + lane; k < n; k += 32) s = fma(Lf[(size_t)k * n + i], y[k], s);
    s = warp_sum(s);
    double v = (y[i] - s) / Lf[(size_t)i * n + i];
    __syncwarp();
    if (lane == 0) y[i] = v;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) inv[(size_t)c * n + i] = y[i];
}

// ------------------------------------------------------------- helpers --
static int grid_for(long long n, int bs) { return (int)((n + bs - 1) / bs); }

static void check_flag(int* dflag, cudaStream_t st, const char* what) {
  int f = 0;
  AMG_CUDA(cudaMemcpyAsync(&f, dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  AMG_CUDA(cudaStreamSynchronize(st));
  if (f & 8) throw Error(AMG_ERR_NOT_SPD, std::string(what) + ": coarsest matrix is not SPD (non-positive Cholesky pivot)");
  if (f & 1) throw Error(AMG_ERR_INVALID_ARG, std::string(what) + ": CSR column index out of range, unsorted or duplicated");
  if (f & 2) throw Error(AMG_ERR_INVALID_ARG, std::string(what) + ": an aggregate has more than 512 neighbouring aggregates");
  if (f & 4) throw Error(AMG_ERR_INVALID_ARG, std::string(what) + ": a row has no non-zero entry (zero l1 norm) or a non-finite value");
}

static void level_stats(Level& L, const std::vector<int>& rp) {
  L.h_rowptr = rp;
  int mx = 0;
  for (int i = 0; i < L.n; ++i) mx = std::max(mx, rp[i + 1] - rp[i]);
  L.max_row_len = mx;
  L.avg_row_len = L.n ? (double)L.nnz / L.n : 0;
}

// Dense inverse of the coarsest matrix (one block).
static void coarsest_inverse(Plan& P, const Level& C, double* inv_out, cudaStream_t st, int* dflag) {
  int n = C.n;
  AMG_REQUIRE(n <= 8192, "coarsest level has " + std::to_string(n) + " dofs; at most 8192 are supported for the dense solve");
  Arena tmp;
  double* D = tmp.alloc<double>((size_t)n * n);
  double* work = tmp.alloc<double>((size_t)n * n);
  k_densify<<<n, 128, 0, st>>>(n, C.rowptr, C.col, C.val64, D);
  AMG_LAUNCH_CHECK();
  k_cholesky<<<1, 1024, 0, st>>>(n, D, dflag);
  AMG_LAUNCH_CHECK();
  k_chol_inverse<<<grid_for((long long)n * 32, 128), 128, 0, st>>>(n, D, work, inv_out);
  AMG_LAUNCH_CHECK();
  check_flag(dflag, st, "coarsest factorisation");
}

// ----------------------------------------------------------------- setup --
void build_hierarchy(amg_hierarchy* h, const amg_csr* A, int nlev, const int32_t* const* agg,
                     const int32_t* n_nodes, const double* W, int m, const amg_opts& o,
                     cudaStream_t st) {
  NvtxRange nv("amg setup");
  AMG_REQUIRE(A && A->rowptr && A->col && A->val, "A and its arrays must be non-null");
  AMG_REQUIRE(A->n > 0 && A->nnz > 0, "A must be non-empty");
  AMG_REQUIRE(nlev >= 0 && nlev <= 15, "n_agg_levels must be in [0, 15]");
  AMG_REQUIRE(m >= 1 && m <= 16, "m must be in [1, 16]");
  AMG_REQUIRE(W, "W must be non-null");
  AMG_REQUIRE(nlev == 0 || (agg && n_nodes), "agg and n_nodes must be non-null");
  AMG_REQUIRE(o.tol_svd >= 0, "tol_svd must be >= 0");
  const int n = A->n, L = nlev + 1;
  Plan& P = h->plan;
  Arena& ar = *P.arena;
  P.L = L;
  P.m = m;
  P.nsys = 1;
  P.h_sys_row = {0, n};
  h->n = n;
  h->nnz = A->nnz;
  h->m = m;

  int* dflag = ar.alloc<int>(1);
  AMG_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), st));

  // host copies of the structure
  std::vector<int> rp = to_host(A->rowptr, n + 1, st);
  AMG_REQUIRE(rp[0] == 0 && rp[n] == A->nnz, "rowptr[0] must be 0 and rowptr[n] must be nnz");
  for (int i = 0; i < n; ++i) AMG_REQUIRE(rp[i + 1] >= rp[i], "rowptr must be non-decreasing");
  std::vector<int> nn(L);
  nn[0] = n;
  for (int k = 1; k < L; ++k) {
    nn[k] = n_nodes[k];
    AMG_REQUIRE(nn[k] > 0, "n_nodes entries must be positive");
  }
  if (nlev > 0) AMG_REQUIRE(n_nodes[0] == n, "n_nodes[0] must equal A->n");
  std::vector<std::vector<int>> ag(nlev);
  for (int k = 0; k < nlev; ++k) {
    AMG_REQUIRE(agg[k], "agg[k] must be non-null");
    ag[k] = to_host(agg[k], (size_t)nn[k], st);
    std::vector<int> cnt(nn[k + 1], 0);
    for (int v : ag[k]) {
      AMG_REQUIRE(v >= 0 && v < nn[k + 1], "aggregate index out of range at level " + std::to_string(k + 1));
      cnt[v]++;
    }
    for (int c : cnt) AMG_REQUIRE(c > 0, "empty aggregate at level " + std::to_string(k + 1));
  }

  // nested ordering: every aggregate is a contiguous range at every level
  std::vector<std::vector<int>> perm(L);
  perm[L - 1].resize(nn[L - 1]);
  std::iota(perm[L - 1].begin(), perm[L - 1].end(), 0);
  std::vector<std::vector<int>> node_start(L);  // per level k >= 1: level-(k-1) node ranges of new aggregate t
  for (int k = L - 2; k >= 0; --k) {
    int nc = nn[k + 1];
    std::vector<int> st_(nc + 1, 0);
    for (int v : ag[k]) st_[v + 1]++;
    for (int a = 0; a < nc; ++a) st_[a + 1] += st_[a];
    std::vector<int> members(nn[k]);
    std::vector<int> fill(st_.begin(), st_.end() - 1);
    for (int i = 0; i < nn[k]; ++i) members[fill[ag[k][i]]++] = i;  // ascending within aggregate
    perm[k].clear();
    perm[k].reserve(nn[k]);
    std::vector<int> ns(nc + 1, 0);
    for (int t = 0; t < nc; ++t) {
      int a = perm[k + 1][t];
      for (int q = st_[a]; q < st_[a + 1]; ++q) perm[k].push_back(members[q]);
      ns[t + 1] = (int)perm[k].size();
    }
    node_start[k + 1] = ns;
  }
  h->h_perm = perm;
  std::vector<int> iperm0(n);
  for (int i = 0; i < n; ++i) iperm0[perm[0][i]] = i;

  // level 0: permuted copy of A
  P.lev.assign(L, Level());
  P.tr.assign(L - 1, Transfer());
  Level& L0 = P.lev[0];
  L0.n = n;
  L0.nnz = A->nnz;
  {
    std::vector<int> rpn(n + 1, 0);
    for (int i = 0; i < n; ++i) rpn[i + 1] = rpn[i] + (rp[perm[0][i] + 1] - rp[perm[0][i]]);
    level_stats(L0, rpn);
    Arena tmp;
    const int* d_rp = A->rowptr;
    const int* d_col = A->col;
    const double* d_val = A->val;
    if (!is_device_ptr(A->rowptr)) { int* t = tmp.alloc<int>(n + 1); copy_in(t, A->rowptr, (n + 1) * 4, st); d_rp = t; }
    if (!is_device_ptr(A->col)) { int* t = tmp.alloc<int>(A->nnz); copy_in(t, A->col, (size_t)A->nnz * 4, st); d_col = t; }
    if (!is_device_ptr(A->val)) { double* t = tmp.alloc<double>(A->nnz); copy_in(t, A->val, (size_t)A->nnz * 8, st); d_val = t; }
    L0.rowptr = to_dev(ar, rpn, st);
    L0.col = alloc_nnz<int>(ar, A->nnz, st);
    L0.val64 = alloc_nnz<double>(ar, A->nnz, st);
    h->nzmap = ar.alloc<int>(A->nnz);
    P.perm0 = to_dev(ar, perm[0], st);
    int* d_iperm = tmp.alloc<int>(n);
    copy_in(d_iperm, iperm0.data(), (size_t)n * 4, st);
    k_permute_csr<<<grid_for(n, 128), 128, 0, st>>>(n, d_rp, d_col, d_val, P.perm0, d_iperm, L0.rowptr,
                                                   L0.col, L0.val64, h->nzmap, dflag);
    AMG_LAUNCH_CHECK();
    check_flag(dflag, st, "matrix permutation");
  }

  // smooth vectors in library order, row-major
  double* Wk;
  {
    Arena tmp;
    const double* dW = W;
    if (!is_device_ptr(W)) { double* t = tmp.alloc<double>((size_t)n * m); copy_in(t, W, (size_t)n * m * 8, st); dW = t; }
    Wk = ar.alloc<double>((size_t)n * m);
    k_gather_w<<<grid_for((long long)n * m, 256), 256, 0, st>>>(n, m, dW, P.perm0, Wk);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(st));
  }

  std::vector<int> r_prev(n, 1);   // dofs per level-(k-1) node, library order
  std::vector<int> rp_prev;
  {
    rp_prev.resize(n + 1);
    AMG_CUDA(cudaMemcpyAsync(rp_prev.data(), L0.rowptr, (n + 1) * 4, cudaMemcpyDeviceToHost, st));
    AMG_CUDA(cudaStreamSynchronize(st));
  }
  h->h_r.assign(L, {});
  Arena scratch_keep;
  for (int k = 1; k < L; ++k) {
    Level& F = P.lev[k - 1];
    Level& C = P.lev[k];
    Transfer& T = P.tr[k - 1];
    const int nagg = nn[k];
    const int nf = F.n;
    T.nagg = nagg;
    T.nf = nf;
    // rows of each aggregate at level k-1
    const std::vector<int>& ns = node_start[k];
    T.h_row_start.assign(nagg + 1, 0);
    {
      std::vector<int> dof_start(nn[k - 1] + 1, 0);
      for (int v = 0; v < nn[k - 1]; ++v) dof_start[v + 1] = dof_start[v] + r_prev[v];
      for (int t = 0; t <= nagg; ++t) T.h_row_start[t] = dof_start[ns[t]];
    }
    AMG_REQUIRE(T.h_row_start[nagg] == nf, "internal: aggregate rows do not cover the level");
    T.row_start = to_dev(ar, T.h_row_start, st);

    // local SVD per aggregate (Eq. (svd))
    Arena tmp;
    double* work = tmp.alloc<double>((size_t)nf * m);
    double* U = tmp.alloc<double>((size_t)nf * m);
    int* rk = tmp.alloc<int>(nagg);
    k_local_svd<<<grid_for((long long)nagg * 32, 128), 128, 0, st>>>(Wk, m, nagg, T.row_start, nf, o.tol_svd,
                                                                    work, U, rk);
    AMG_LAUNCH_CHECK();
    std::vector<int> r = to_host(rk, nagg, st);
    T.h_coarse_start.assign(nagg + 1, 0);
    T.h_blk_start.assign(nagg + 1, 0);
    for (int a = 0; a < nagg; ++a) {
      int na = T.h_row_start[a + 1] - T.h_row_start[a];
      if (r[a] < std::min(na, m)) h->truncated++;
      T.h_coarse_start[a + 1] = T.h_coarse_start[a] + r[a];
      T.h_blk_start[a + 1] = T.h_blk_start[a] + (long long)na * r[a];
    }
    const int ncoarse = T.h_coarse_start[nagg];
    T.nc = ncoarse;
    T.npval = T.h_blk_start[nagg];
    T.coarse_start = to_dev(ar, T.h_coarse_start, st);
    T.blk_start = to_dev(ar, T.h_blk_start, st);
    T.p64 = ar.alloc<double>(T.npval + 2);   // +2: room for aligned vector reads past the end
    T.p32 = ar.alloc<float>(T.npval + 4);
    AMG_CUDA(cudaMemsetAsync(T.p64, 0, (T.npval + 2) * 8, st));
    AMG_CUDA(cudaMemsetAsync(T.p32, 0, (T.npval + 4) * 4, st));
    k_compact_p<<<nagg, 64, 0, st>>>(nagg, m, T.row_start, T.coarse_start, T.blk_start, U, T.p64);
    AMG_LAUNCH_CHECK();
    h->h_r[k] = r;

    // coarse smooth vectors
    double* Wc = ar.alloc<double>((size_t)ncoarse * m);
    k_restrict_w<<<nagg, 64, 0, st>>>(nagg, m, T.row_start, T.coarse_start, T.blk_start, T.p64, Wk, Wc);
    AMG_LAUNCH_CHECK();

    // owner of each level-(k-1) dof
    std::vector<int> own(nf);
    for (int a = 0; a < nagg; ++a)
      for (int i = T.h_row_start[a]; i < T.h_row_start[a + 1]; ++i) own[i] = a;
    int* d_own = tmp.alloc<int>(nf);
    copy_in(d_own, own.data(), (size_t)nf * 4, st);

    // Galerkin: symbolic
    int* d_cnt = tmp.alloc<int>(nagg);
    int* d_S = tmp.alloc<int>(nagg);
    int gblocks = (nagg + GAL_WARPS - 1) / GAL_WARPS;
    k_gal_sym<<<gblocks, 32 * GAL_WARPS, 0, st>>>(nagg, T.row_start, F.rowptr, F.col, d_own, rk, 0, d_cnt,
                                                 d_S, nullptr, nullptr, dflag);
    AMG_LAUNCH_CHECK();
    check_flag(dflag, st, "Galerkin symbolic phase");
    std::vector<int> cnt = to_host(d_cnt, nagg, st), S = to_host(d_S, nagg, st);
    std::vector<int> nb_ptr(nagg + 1, 0);
    for (int a = 0; a < nagg; ++a) nb_ptr[a + 1] = nb_ptr[a] + cnt[a];
    std::vector<int> rpc(ncoarse + 1, 0);
    long long nnzc = 0;
    long long tsz = 0, tmax = 0;
    std::vector<long long> toff(nagg + 1, 0);
    for (int a = 0; a < nagg; ++a) {
      for (int p = T.h_coarse_start[a]; p < T.h_coarse_start[a + 1]; ++p) {
        nnzc += S[a];
        rpc[p + 1] = (int)nnzc;
      }
      long long na = T.h_row_start[a + 1] - T.h_row_start[a];
      toff[a] = tsz;
      tsz += na * S[a];
      tmax = std::max(tmax, na * (long long)S[a]);
    }
    AMG_REQUIRE(nnzc < (1LL << 31), "coarse matrix too large for int32 indices");
    int* d_nbp = to_dev(tmp, nb_ptr, st);
    int* d_nbl = tmp.alloc<int>(std::max(1, nb_ptr[nagg]));
    k_gal_sym<<<gblocks, 32 * GAL_WARPS, 0, st>>>(nagg, T.row_start, F.rowptr, F.col, d_own, rk, 1, d_cnt,
                                                 d_S, d_nbp, d_nbl, dflag);
    AMG_LAUNCH_CHECK();
    C.n = ncoarse;
    C.nnz = nnzc;
    C.rowptr = to_dev(ar, rpc, st);
    C.col = alloc_nnz<int>(ar, nnzc, st);
    C.val64 = alloc_nnz<double>(ar, nnzc, st);
    level_stats(C, rpc);
    k_gal_cols<<<nagg, 128, 0, st>>>(nagg, T.coarse_start, d_nbp, d_nbl, C.rowptr, C.col);
    AMG_LAUNCH_CHECK();
    // Galerkin: numeric
    size_t smem = (size_t)tmax * 8;
    int use_smem = smem <= 160 * 1024;
    double* gs = nullptr;
    long long* d_toff = nullptr;
    if (use_smem) {
      AMG_CUDA(cudaFuncSetAttribute(k_gal_num, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    } else {
      gs = tmp.alloc<double>(tsz);
      d_toff = to_dev(tmp, toff, st);
      smem = 0;
    }
    k_gal_num<<<nagg, 128, use_smem ? smem : 0, st>>>(nagg, T.row_start, T.coarse_start, T.blk_start, T.p64,
                                                     F.rowptr, F.col, F.val64, d_own, d_nbp, d_nbl, C.rowptr,
                                                     C.val64, gs, d_toff, use_smem);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(st));

    // fine-level diagonals and float32 copies
    F.dinv64 = ar.alloc<double>(nf);
    F.dinv32 = ar.alloc<float>(nf);
    k_l1<<<grid_for(nf, 256), 256, 0, st>>>(nf, F.rowptr, F.val64, F.dinv64, F.dinv32, dflag);
    AMG_LAUNCH_CHECK();
    F.val32 = alloc_nnz<float>(ar, F.nnz, st);
    k_cast<double, float><<<grid_for(F.nnz, 256), 256, 0, st>>>(F.nnz, F.val64, F.val32);
    AMG_LAUNCH_CHECK();
    if (k == 1) {
      F.vallo = alloc_nnz<float>(ar, F.nnz, st);
      k_split_lo<<<grid_for(F.nnz, 256), 256, 0, st>>>(F.nnz, F.val64, F.val32, F.vallo);
      AMG_LAUNCH_CHECK();
    }
    k_cast<double, float><<<grid_for(T.npval, 256), 256, 0, st>>>(T.npval, T.p64, T.p32);
    AMG_LAUNCH_CHECK();
    check_flag(dflag, st, "level setup");

    // next level's dof counts per node (library order of level-k nodes)
    r_prev = r;
    Wk = Wc;
  }
  // coarsest level: float32 copy (for exports) and dense inverse
  Level& C = P.lev[L - 1];
  C.val32 = alloc_nnz<float>(ar, C.nnz, st);
  k_cast<double, float><<<grid_for(C.nnz, 256), 256, 0, st>>>(C.nnz, C.val64, C.val32);
  AMG_LAUNCH_CHECK();
  if (L == 1) {
    C.vallo = alloc_nnz<float>(ar, C.nnz, st);
    k_split_lo<<<grid_for(C.nnz, 256), 256, 0, st>>>(C.nnz, C.val64, C.val32, C.vallo);
    AMG_LAUNCH_CHECK();
  }
  P.co.n = C.n;
  P.co.nblk = 1;
  P.co.h_blk_off = {0, C.n};
  P.co.h_inv_off = {0, (long long)C.n * C.n};
  P.co.blk_off = to_dev(ar, P.co.h_blk_off, st);
  P.co.inv_off = to_dev(ar, P.co.h_inv_off, st);
  P.co.inv = ar.alloc<double>((size_t)C.n * C.n);
  coarsest_inverse(P, C, P.co.inv, st, dflag);
  AMG_CUDA(cudaStreamSynchronize(st));
  if (check_mode()) check_plan(P, st);
}

// --------------------------------------------------------------- batches --
// Concatenate the hierarchies of several systems block-diagonally, level by
// level, so that one launch sequence serves all of them.
void build_batch_plan(Plan& B, const std::vector<amg_hierarchy*>& hs, cudaStream_t st) {
  NvtxRange nv("amg batch plan");
  const int ns = (int)hs.size();
  const int L = hs[0]->plan.L;
  for (auto* h : hs) AMG_REQUIRE(h->plan.L == L, "all hierarchies of a batch must have the same number of levels");
  Arena& ar = *B.arena;
  B.L = L;
  B.nsys = ns;
  B.m = hs[0]->plan.m;
  B.lev.assign(L, Level());
  B.tr.assign(L - 1, Transfer());
  B.h_sys_row.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) B.h_sys_row[s + 1] = B.h_sys_row[s] + hs[s]->plan.lev[0].n;
  for (int k = 0; k < L; ++k) {
    Level& D = B.lev[k];
    long long nnz = 0;
    int n = 0;
    for (auto* h : hs) {
      n += h->plan.lev[k].n;
      nnz += h->plan.lev[k].nnz;
    }
    AMG_REQUIRE(nnz < (1LL << 31), "batch too large for int32 indices");
    D.n = n;
    D.nnz = nnz;
    D.rowptr = ar.alloc<int>(n + 1);
    D.col = alloc_nnz<int>(ar, nnz, st);
    D.val64 = alloc_nnz<double>(ar, nnz, st);
    D.val32 = alloc_nnz<float>(ar, nnz, st);
    if (k == 0) D.vallo = alloc_nnz<float>(ar, nnz, st);
    bool coarse = (k == L - 1);
    if (!coarse) {
      D.dinv64 = ar.alloc<double>(n);
      D.dinv32 = ar.alloc<float>(n);
    }
    int ro = 0;
    long long zo = 0;
    int mx = 0;
    for (auto* h : hs) {
      const Level& S = h->plan.lev[k];
      k_add_offset<<<grid_for(S.n + 1, 256), 256, 0, st>>>(S.n + 1, S.rowptr, (int)zo, D.rowptr + ro);
      AMG_LAUNCH_CHECK();
      k_add_offset<<<grid_for(S.nnz, 256), 256, 0, st>>>(S.nnz, S.col, ro, D.col + zo);
      AMG_LAUNCH_CHECK();
      AMG_CUDA(cudaMemcpyAsync(D.val64 + zo, S.val64, S.nnz * 8, cudaMemcpyDeviceToDevice, st));
      AMG_CUDA(cudaMemcpyAsync(D.val32 + zo, S.val32, S.nnz * 4, cudaMemcpyDeviceToDevice, st));
      if (k == 0) AMG_CUDA(cudaMemcpyAsync(D.vallo + zo, S.vallo, S.nnz * 4, cudaMemcpyDeviceToDevice, st));
      if (!coarse) {
        AMG_CUDA(cudaMemcpyAsync(D.dinv64 + ro, S.dinv64, S.n * 8, cudaMemcpyDeviceToDevice, st));
        AMG_CUDA(cudaMemcpyAsync(D.dinv32 + ro, S.dinv32, S.n * 4, cudaMemcpyDeviceToDevice, st));
      }
      ro += S.n;
      zo += S.nnz;
      mx = std::max(mx, S.max_row_len);
    }
    D.max_row_len = mx;
    D.avg_row_len = n ? (double)nnz / n : 0;
    D.h_rowptr.assign(1, 0);
    for (auto* h : hs) {
      const Level& S = h->plan.lev[k];
      long long base = D.h_rowptr.back();
      for (int i = 1; i <= S.n; ++i) D.h_rowptr.push_back((int)(base + S.h_rowptr[i]));
    }
  }
  for (int k = 0; k + 1 < L; ++k) {
    Transfer& T = B.tr[k];
    T.h_row_start.assign(1, 0);
    T.h_coarse_start.assign(1, 0);
    T.h_blk_start.assign(1, 0);
    for (auto* h : hs) {
      const Transfer& S = h->plan.tr[k];
      int ro = T.h_row_start.back(), co = T.h_coarse_start.back();
      long long bo = T.h_blk_start.back();
      for (int a = 1; a <= S.nagg; ++a) {
        T.h_row_start.push_back(ro + S.h_row_start[a]);
        T.h_coarse_start.push_back(co + S.h_coarse_start[a]);
        T.h_blk_start.push_back(bo + S.h_blk_start[a]);
      }
      T.nagg += S.nagg;
      T.nf += S.nf;
      T.nc += S.nc;
    }
    T.npval = T.h_blk_start.back();
    T.row_start = to_dev(ar, T.h_row_start, st);
    T.coarse_start = to_dev(ar, T.h_coarse_start, st);
    T.blk_start = to_dev(ar, T.h_blk_start, st);
    T.p64 = ar.alloc<double>(T.npval + 2);
    T.p32 = ar.alloc<float>(T.npval + 4);
    AMG_CUDA(cudaMemsetAsync(T.p64, 0, (T.npval + 2) * 8, st));
    AMG_CUDA(cudaMemsetAsync(T.p32, 0, (T.npval + 4) * 4, st));
    long long bo = 0;
    for (auto* h : hs) {
      const Transfer& S = h->plan.tr[k];
      AMG_CUDA(cudaMemcpyAsync(T.p64 + bo, S.p64, S.npval * 8, cudaMemcpyDeviceToDevice, st));
      AMG_CUDA(cudaMemcpyAsync(T.p32 + bo, S.p32, S.npval * 4, cudaMemcpyDeviceToDevice, st));
      bo += S.npval;
    }
  }
  // block-diagonal coarsest inverse
  B.co.h_blk_off.assign(1, 0);
  B.co.h_inv_off.assign(1, 0);
  for (auto* h : hs) {
    const Coarsest& S = h->plan.co;
    B.co.h_blk_off.push_back(B.co.h_blk_off.back() + S.n);
    B.co.h_inv_off.push_back(B.co.h_inv_off.back() + (long long)S.n * S.n);
  }
  B.co.n = B.co.h_blk_off.back();
  B.co.nblk = ns;
  B.co.blk_off = to_dev(ar, B.co.h_blk_off, st);
  B.co.inv_off = to_dev(ar, B.co.h_inv_off, st);
  B.co.inv = ar.alloc<double>(B.co.h_inv_off.back());
  for (int s = 0; s < ns; ++s) {
    const Coarsest& S = hs[s]->plan.co;
    AMG_CUDA(cudaMemcpyAsync(B.co.inv + B.co.h_inv_off[s], S.inv, (size_t)S.n * S.n * 8,
                             cudaMemcpyDeviceToDevice, st));
  }
  // level-0 permutation: each system keeps its own numbering
  B.perm0 = ar.alloc<int>(B.lev[0].n);
  for (int s = 0; s < ns; ++s)
    AMG_CUDA(cudaMemcpyAsync(B.perm0 + B.h_sys_row[s], hs[s]->plan.perm0, hs[s]->plan.lev[0].n * 4,
                             cudaMemcpyDeviceToDevice, st));
  AMG_CUDA(cudaStreamSynchronize(st));
  if (check_mode()) check_plan(B, st);
}

}  // namespace amg

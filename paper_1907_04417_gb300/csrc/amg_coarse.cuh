// The small levels of the V-cycle (Section 5) in one persistent launch.
//
// From a start level s down to the coarsest level and back up to s, every
// step of the cycle (pre-sweeps beyond the first, the residual and the
// restriction P^T (f - A u) with the first pre-sweep uc = D_c^{-1} fc of the
// next level, the coarsest solve, the prolongation u += P e and the
// post-sweeps) is a phase of one cooperative kernel, the phases separated by
// a grid barrier.  On the small levels each phase is a few microseconds of
// work, less than the launch and drain of a kernel of its own.
//
// The barrier spins on a generation word for at most ``budget`` clock64
// cycles; a CTA whose wait gives up records the error (the host reports
// AMG_ERR_TIMEOUT) and returns, every other CTA gives up as soon as it sees
// the error, and later launches of the solve return at once, so a failed
// solve costs one bound, not one per cycle.  The kernel holds no shared
// memory copies in flight and no tensor memory, so a CTA may leave at any
// barrier.  A test hook (hang_test) makes the first barrier wait for one
// arrival more than the grid has.
#pragma once

#include "amg_kernels.cuh"

namespace amg {

constexpr int CC_BS = 1024;     // threads per CTA (one CTA per SM)
constexpr int CC_MAXL = 16;

template <typename TC>
struct CcLevel {
  int n = 0;
  const int* rowptr = nullptr;
  const int* col = nullptr;
  const TC* val = nullptr;
  const TC* dinv = nullptr;
  TC* f = nullptr;
  TC* u = nullptr;   // the iterate at the start of the cycle
  TC* v = nullptr;   // the other buffer (out-of-place sweeps; the residual before a restriction)
};
template <typename TC>
struct CcTransfer {   // P^{k+1}: level k+1 -> level k
  int nagg = 0;
  const int* row_start = nullptr;
  const int* coarse_start = nullptr;
  const long long* blk_start = nullptr;
  const TC* P = nullptr;
};
template <typename TC>
struct CcArgs {
  int s = 0, L = 0, pre = 1, post = 1;
  CcLevel<TC> lev[CC_MAXL];
  CcTransfer<TC> tr[CC_MAXL];
  // coarsest: block-diagonal float64 inverse
  int cn = 0, cnblk = 0;
  const int* cblk_off = nullptr;
  const long long* cinv_off = nullptr;
  const double* cinv = nullptr;
  unsigned* bar_count = nullptr;   // arrivals at the current barrier (0 between launches)
  unsigned* bar_gen = nullptr;     // barrier generation
  int* err = nullptr;              // bit 2: a barrier wait gave up
  const int* done = nullptr;
  long long budget = 0;            // clock64 cycles one barrier wait may spin
  int hang_test = 0;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier with a bounded wait.  Returns false (for the whole CTA) when
// this CTA's wait gave up.
__device__ __forceinline__ bool cc_barrier(unsigned* count, unsigned* gen, long long budget, int* err,
                                           bool never) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = ld_acquire_gpu(gen);
    __threadfence();
    const unsigned want = gridDim.x + (never ? 1u : 0u);
    const unsigned arrived = atomicAdd(count, 1u) + 1u;
    if (arrived == want) {
      *count = 0u;
      __threadfence();
      st_release_gpu(gen, g + 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_gpu(gen) == g) {
        // give up at the bound, or at once when another CTA already gave up
        if (clock64() - t0 > budget || (ld_acquire_gpu(reinterpret_cast<const unsigned*>(err)) & 2u)) {
          atomicOr(err, 2);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
  }
  __syncthreads();
  return ok != 0;
}

// Work items: (row, CPT-wide column chunk), NCH chunks per row.
template <typename TC, int K>
struct CcItems {
  static constexpr int CPT = VT<TC, K>::CPT, NCH = K / CPT;
  // lanes of one warp-row in cc_sweep: NCH column chunks x NZL slices of the row
  static constexpr int NZL = 32 / NCH;
};

__device__ __forceinline__ long long cc_warp() { return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ long long cc_warps() { return ((long long)gridDim.x * blockDim.x) >> 5; }

// y = f - A x on a level (out-of-place), or, with smooth, y = x + D^{-1} (f - A x).
// One warp per row: lane = (slice, chunk); the NZL slices take every NZL-th
// non-zero, four gathers in flight each, and are combined by shuffles.
template <typename TC, int K>
__device__ __forceinline__ void cc_sweep(const CcLevel<TC>& L, const TC* __restrict__ x, TC* __restrict__ y,
                                         bool smooth) {
  constexpr int CPT = CcItems<TC, K>::CPT, NCH = CcItems<TC, K>::NCH, NZL = CcItems<TC, K>::NZL;
  const int lane = threadIdx.x & 31, ch = lane % NCH, sl = lane / NCH, c0 = ch * CPT;
  for (long long i = cc_warp(); i < L.n; i += cc_warps()) {
    TC acc[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) acc[t] = TC(0);
    const int j1 = L.rowptr[i + 1];
    int j = L.rowptr[i] + sl;
    for (; j + 3 * NZL < j1; j += 4 * NZL) {
      int c[4];
      TC a[4], xv[4][CPT];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        c[q] = L.col[j + q * NZL];
        a[q] = L.val[j + q * NZL];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) ldp<TC, CPT>(x + (size_t)c[q] * K + c0, xv[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int t = 0; t < CPT; ++t) acc[t] = fma(a[q], xv[q][t], acc[t]);
    }
    for (; j < j1; j += NZL) {
      TC xv[CPT];
      ldp<TC, CPT>(x + (size_t)L.col[j] * K + c0, xv);
      const TC a = L.val[j];
#pragma unroll
      for (int t = 0; t < CPT; ++t) acc[t] = fma(a, xv[t], acc[t]);
    }
#pragma unroll
    for (int off = NCH; off < 32; off <<= 1)
#pragma unroll
      for (int t = 0; t < CPT; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], off);
    if (sl == 0) {
      TC fv[CPT], out[CPT];
      ldp<TC, CPT>(L.f + (size_t)i * K + c0, fv);
      if (smooth) {
        TC xi[CPT];
        ldp<TC, CPT>(x + (size_t)i * K + c0, xi);
        const TC di = L.dinv[i];
#pragma unroll
        for (int t = 0; t < CPT; ++t) out[t] = fma(di, fv[t] - acc[t], xi[t]);
      } else {
#pragma unroll
        for (int t = 0; t < CPT; ++t) out[t] = fv[t] - acc[t];
      }
      stv<TC, CPT>(y + (size_t)i * K + c0, out);
    }
  }
}

__device__ __forceinline__ int cc_find(const int* __restrict__ start, int n, int v) {
  int lo = 0, hi = n - 1;   // the last a with start[a] <= v
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// fc = P^T t; uc = D_c^{-1} fc when the coarse level is smoothed.  One warp
// per (coarse dof, column chunk): the lanes take the aggregate's rows in
// turn and their partial sums are combined by shuffles.
template <typename TC, int K>
__device__ __forceinline__ void cc_restrict(const CcTransfer<TC>& T, const TC* __restrict__ t,
                                            const CcLevel<TC>& C, bool smooth_next) {
  constexpr int CPT = CcItems<TC, K>::CPT, NCH = CcItems<TC, K>::NCH;
  const int lane = threadIdx.x & 31;
  const long long items = (long long)C.n * NCH;
  for (long long it = cc_warp(); it < items; it += cc_warps()) {
    const int cd = (int)(it / NCH), c0 = (int)(it % NCH) * CPT;
    const int a = cc_find(T.coarse_start, T.nagg, cd);
    const int cs = T.coarse_start[a], ra = T.coarse_start[a + 1] - cs, p = cd - cs;
    const int rs = T.row_start[a], re = T.row_start[a + 1];
    const TC* Pa = T.P + T.blk_start[a] + p;
    TC acc[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) acc[q] = TC(0);
    for (int i = rs + lane; i < re; i += 32) {
      TC tv[CPT];
      ldp<TC, CPT>(t + (size_t)i * K + c0, tv);
      const TC pv = Pa[(size_t)(i - rs) * ra];
#pragma unroll
      for (int q = 0; q < CPT; ++q) acc[q] = fma(pv, tv[q], acc[q]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < CPT; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    if (lane == 0) {
      stv<TC, CPT>(C.f + (size_t)cd * K + c0, acc);
      if (smooth_next) {
        const TC d = C.dinv[cd];
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] *= d;
        stv<TC, CPT>(C.u + (size_t)cd * K + c0, acc);
      }
    }
  }
}

// u[rows(a)] += P_a e[coarse(a)]
template <typename TC, int K>
__device__ __forceinline__ void cc_prolong(const CcTransfer<TC>& T, const TC* __restrict__ e, TC* __restrict__ u,
                                           int nf) {
  constexpr int CPT = CcItems<TC, K>::CPT, NCH = CcItems<TC, K>::NCH;
  const long long items = (long long)nf * NCH;
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(it / NCH), c0 = (int)(it % NCH) * CPT;
    const int a = cc_find(T.row_start, T.nagg, i);
    const int cs = T.coarse_start[a], ra = T.coarse_start[a + 1] - cs, rs = T.row_start[a];
    const TC* pr = T.P + T.blk_start[a] + (size_t)(i - rs) * ra;
    TC s[CPT], uv[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) s[q] = TC(0);
    for (int p = 0; p < ra; ++p) {
      TC ev[CPT];
      ldp<TC, CPT>(e + (size_t)(cs + p) * K + c0, ev);
      const TC pv = pr[p];
#pragma unroll
      for (int q = 0; q < CPT; ++q) s[q] = fma(pv, ev[q], s[q]);
    }
    ldp<TC, CPT>(u + (size_t)i * K + c0, uv);
#pragma unroll
    for (int q = 0; q < CPT; ++q) uv[q] += s[q];
    stv<TC, CPT>(u + (size_t)i * K + c0, uv);
  }
}

// u = A_c^{-1} f with the float64 inverse of each diagonal block.  One warp
// per row: lane = (column, slice), C = min(K, 32) columns and 32 / C slices
// of the inner index, combined by shuffles.
template <typename TC, int K>
__device__ __forceinline__ void cc_coarsest(const CcArgs<TC>& a, const TC* __restrict__ f, TC* __restrict__ u) {
  constexpr int C = K < 32 ? K : 32, JP = 32 / C;
  const int lane = threadIdx.x & 31, c = lane % C, jp = lane / C;
  for (long long row = cc_warp(); row < a.cn; row += cc_warps()) {
    const int b = cc_find(a.cblk_off, a.cnblk, (int)row);
    const int b0 = a.cblk_off[b], nb = a.cblk_off[b + 1] - b0;
    const double* Ar = a.cinv + a.cinv_off[b] + (size_t)(row - b0) * nb;
    const TC* fc = f + (size_t)b0 * K + c;
    double s0 = 0.0, s1 = 0.0;
    int j = jp;
    for (; j + JP < nb; j += 2 * JP) {
      s0 = fma(Ar[j], (double)fc[(size_t)j * K], s0);
      s1 = fma(Ar[j + JP], (double)fc[(size_t)(j + JP) * K], s1);
    }
    if (j < nb) s0 = fma(Ar[j], (double)fc[(size_t)j * K], s0);
    double sv = s0 + s1;
#pragma unroll
    for (int off = C; off < 32; off <<= 1) sv += __shfl_xor_sync(0xffffffffu, sv, off);
    if (jp == 0) u[(size_t)row * K + c] = (TC)sv;
  }
}

// The cycle from level s down and back up (see the head of this file).
// Level k's iterate starts in lev[k].u (for k = s it was written by the
// restriction into level s); each out-of-place sweep moves it to the other
// buffer, and the host replays the same swaps to find level s's result.
template <typename TC, int K>
__global__ void __launch_bounds__(CC_BS, 1) k_coarse_cycle(CcArgs<TC> a) {
  // a barrier of an earlier launch gave up: the solve is already failed
  if (*a.done || (ld_acquire_gpu(reinterpret_cast<const unsigned*>(a.err)) & 2u)) return;
  bool in_v[CC_MAXL];   // the iterate of level k lives in v (else in u)
#pragma unroll
  for (int k = 0; k < CC_MAXL; ++k) in_v[k] = false;
  bool never = a.hang_test != 0;
  auto bar = [&]() {
    const bool ok = cc_barrier(a.bar_count, a.bar_gen, a.budget, a.err, never);
    never = false;
    return ok;
  };
  auto cur = [&](int k) -> TC* { return in_v[k] ? a.lev[k].v : a.lev[k].u; };
  auto oth = [&](int k) -> TC* { return in_v[k] ? a.lev[k].u : a.lev[k].v; };
  const int L = a.L;
  for (int k = a.s; k + 1 < L; ++k) {
    for (int sw = 1; sw < a.pre; ++sw) {
      cc_sweep<TC, K>(a.lev[k], cur(k), oth(k), true);
      in_v[k] = !in_v[k];
      if (!bar()) return;
    }
    cc_sweep<TC, K>(a.lev[k], cur(k), oth(k), false);   // t = f - A u into the free buffer
    if (!bar()) return;
    cc_restrict<TC, K>(a.tr[k], oth(k), a.lev[k + 1], k + 1 < L - 1);
    if (!bar()) return;
  }
  cc_coarsest<TC, K>(a, a.lev[L - 1].f, a.lev[L - 1].u);
  for (int k = L - 2; k >= a.s; --k) {
    if (!bar()) return;
    cc_prolong<TC, K>(a.tr[k], cur(k + 1), cur(k), a.lev[k].n);
    for (int sw = 0; sw < a.post; ++sw) {
      if (!bar()) return;
      cc_sweep<TC, K>(a.lev[k], cur(k), oth(k), true);
      in_v[k] = !in_v[k];
    }
  }
}

}  // namespace amg

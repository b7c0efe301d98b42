// Device kernels of the solve phase: V-cycle (Section 5) with l1-Jacobi
// smoothing, block-prolongator transfers (Section 4), dense coarsest solve,
// and the fused vector/reduction kernels of preconditioned CG.
//
// Layout: every multi-column vector is an n x K row-major block; K is a
// compile-time column count (1, 2, 4, ..., 32).  A group of G = NZL * CL
// lanes owns one matrix row: CL lanes split the K columns into CPT-wide
// vector loads (16 bytes where K allows), NZL lanes split the row's non-zeros.
// Row loops are warp-uniform so every shuffle has all 32 lanes present.
// Dot products are reduced deterministically: fixed lane/warp trees, one
// partial per CTA, and a last-arriving CTA that sums the partials in a fixed
// order and updates the CG scalars on the device.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "amg_internal.cuh"

namespace amg {

constexpr int BS = 256;        // threads per CTA of the row-parallel kernels
constexpr int NWARP = BS / 32;
constexpr unsigned FULL = 0xffffffffu;

template <typename T, int K>
struct VT {
  static constexpr int CPT = (K * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : K;
  static constexpr int CL = K / CPT;
};

template <typename T, int N>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T (&r)[N]) {
  if constexpr (sizeof(T) * N == 16) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    memcpy(r, &t, 16);
  } else if constexpr (sizeof(T) * N == 8) {
    float2 t = __ldg(reinterpret_cast<const float2*>(p));
    memcpy(r, &t, 8);
  } else {
    r[0] = __ldg(p);
  }
}
// plain (coherent) loads for buffers written earlier in the same kernel
template <typename T, int N>
__device__ __forceinline__ void ldp(const T* p, T (&r)[N]) {
  if constexpr (sizeof(T) * N == 16) {
    float4 t = *reinterpret_cast<const float4*>(p);
    memcpy(r, &t, 16);
  } else if constexpr (sizeof(T) * N == 8) {
    float2 t = *reinterpret_cast<const float2*>(p);
    memcpy(r, &t, 8);
  } else {
    r[0] = p[0];
  }
}
template <typename T, int N>
__device__ __forceinline__ void stv(T* p, const T (&r)[N]) {
  if constexpr (sizeof(T) * N == 16) {
    float4 t;
    memcpy(&t, r, 16);
    *reinterpret_cast<float4*>(p) = t;
  } else if constexpr (sizeof(T) * N == 8) {
    float2 t;
    memcpy(&t, r, 8);
    *reinterpret_cast<float2*>(p) = t;
  } else {
    p[0] = r[0];
  }
}

// y_i = sum_j a_ij x_j for the K columns owned by this lane.
template <typename TA, typename TX, int K, int NZL>
__device__ __forceinline__ void row_acc(int i, bool valid, const int* __restrict__ rowptr,
                                        const int* __restrict__ col, const TA* __restrict__ val,
                                        const TX* __restrict__ x, int nzl, int cl,
                                        TX (&acc)[VT<TX, K>::CPT]) {
  constexpr int CPT = VT<TX, K>::CPT, CL = VT<TX, K>::CL;
#pragma unroll
  for (int t = 0; t < CPT; ++t) acc[t] = TX(0);
  if (valid) {
    int j1 = __ldg(rowptr + i + 1);
    for (int j = __ldg(rowptr + i) + nzl; j < j1; j += NZL) {
      TX a = (TX)__ldg(val + j);
      int c = __ldg(col + j);
      TX xv[CPT];
      ldv<TX, CPT>(x + (size_t)c * K + cl * CPT, xv);
#pragma unroll
      for (int t = 0; t < CPT; ++t) acc[t] = fma(a, xv[t], acc[t]);
    }
  }
  if constexpr (NZL > 1) {
#pragma unroll
    for (int off = CL; off < CL * NZL; off <<= 1)
#pragma unroll
      for (int t = 0; t < CPT; ++t) acc[t] += __shfl_xor_sync(FULL, acc[t], off);
  }
}

// Sum the per-lane column partials of one CTA into out[0..K) (smem scratch
// of NWARP*K doubles).  Lanes holding the same columns sit CL apart.
template <int K, int CPT>
__device__ __forceinline__ void cta_colsum(double (&d)[CPT], double* sm, double* out) {
  constexpr int CL = K / CPT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = CL; off < 32; off <<= 1)
#pragma unroll
    for (int t = 0; t < CPT; ++t) d[t] += __shfl_xor_sync(FULL, d[t], off);
  if (lane < CL)
#pragma unroll
    for (int t = 0; t < CPT; ++t) sm[warp * K + lane * CPT + t] = d[t];
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) s += sm[w * K + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// CG scalars shared by the fused kernels.
struct KState {
  double* partial;     // ncta0 * NV
  unsigned* counter;   // one counter per reducing kernel
  double *rho, *alpha, *beta, *bnorm, *rnorm;
  int *conv, *iters, *status, *active, *done, *iter;
  const int* sys_cta;  // nsys + 1
  int nsys;
  double rtol;
  int maxit;
};

enum : int { ST_ACTIVE = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_MAXIT = 3 };

__device__ __forceinline__ int cta_system(const int* sys_cta, int nsys) {
  int lo = 0, hi = nsys - 1;
  int b = blockIdx.x;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(sys_cta + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Returns true in the last CTA to finish; that CTA then sees all partials.
__device__ __forceinline__ bool arrive_last(unsigned* counter) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Deterministic sum of partial[b*NV + v] over b in [b0, b1) for v < NV
// (NV a power of two <= BS); result in out[v].  All threads participate.
__device__ __forceinline__ void sum_partials(const double* partial, int NV, int b0, int b1, double* sm,
                                            double* out) {
  const int v = threadIdx.x % NV, ch = threadIdx.x / NV, nch = BS / NV;
  double s = 0;
  for (int b = b0 + ch; b < b1; b += nch) s += __ldcg(partial + (size_t)b * NV + v);
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = nch >> 1; w >= 1; w >>= 1) {
    if (ch < w) sm[threadIdx.x] += sm[threadIdx.x + w * NV];
    __syncthreads();
  }
  if (threadIdx.x < NV) out[threadIdx.x] = sm[threadIdx.x];
  __syncthreads();
}

// ------------------------------------------------------------ V-cycle ----

// v = u + D^{-1} (f - A u)   (one l1-Jacobi sweep, out of place)
template <typename TC, int K, int NZL>
__global__ void __launch_bounds__(BS) k_smooth(const int* __restrict__ cta_row, const int* __restrict__ rowptr,
                                               const int* __restrict__ col, const TC* __restrict__ val,
                                               const TC* __restrict__ dinv, const TC* __restrict__ f,
                                               const TC* __restrict__ u, TC* __restrict__ v,
                                               const int* __restrict__ done) {
  if (*done) return;
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  const int r0 = cta_row[blockIdx.x], r1 = cta_row[blockIdx.x + 1];
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    TC acc[CPT];
    row_acc<TC, TC, K, NZL>(i, valid, rowptr, col, val, u, nzl, cl, acc);
    if (valid && nzl == 0) {
      TC fv[CPT], uv[CPT], out[CPT];
      size_t o = (size_t)i * K + cl * CPT;
      ldv<TC, CPT>(f + o, fv);
      ldv<TC, CPT>(u + o, uv);
      TC di = __ldg(dinv + i);
#pragma unroll
      for (int t = 0; t < CPT; ++t) out[t] = fma(di, fv[t] - acc[t], uv[t]);
      stv<TC, CPT>(v + o, out);
    }
  }
}

// Fused residual + restriction on aggregate-aligned CTAs:
//   t = f - A u on the CTA's rows (kept in shared memory), then
//   fc[cd] = P_a^T t[rows(a)] for each coarse dof of the CTA's aggregates,
//   and, when the coarse level is smoothed, uc = D_c^{-1} fc (the first
//   pre-sweep from zero on the next level).
template <typename TC, int K, int NZL>
__global__ void __launch_bounds__(BS) k_restrict(const int* __restrict__ cta_agg, const int* __restrict__ row_start,
                                                 const int* __restrict__ coarse_start,
                                                 const long long* __restrict__ blk_start, const TC* __restrict__ P,
                                                 const int* __restrict__ rowptr, const int* __restrict__ col,
                                                 const TC* __restrict__ val, const TC* __restrict__ f,
                                                 const TC* __restrict__ u, TC* __restrict__ fc,
                                                 TC* __restrict__ uc, const TC* __restrict__ dinvc,
                                                 const int* __restrict__ done) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  TC* tsm = reinterpret_cast<TC*>(smraw);
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  const int a0 = cta_agg[blockIdx.x], a1 = cta_agg[blockIdx.x + 1];
  const int r0 = row_start[a0], r1 = row_start[a1];
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    TC acc[CPT];
    row_acc<TC, TC, K, NZL>(i, valid, rowptr, col, val, u, nzl, cl, acc);
    if (valid && nzl == 0) {
      TC fv[CPT];
      size_t o = (size_t)i * K + cl * CPT;
      ldv<TC, CPT>(f + o, fv);
#pragma unroll
      for (int t = 0; t < CPT; ++t) fv[t] -= acc[t];
      stv<TC, CPT>(tsm + (size_t)(i - r0) * K + cl * CPT, fv);
    }
  }
  __syncthreads();
  const int c0 = coarse_start[a0], c1 = coarse_start[a1];
  const int nout = (c1 - c0) * K;
  for (int o = threadIdx.x; o < nout; o += BS) {
    int cd = c0 + o / K, c = o % K;
    int lo = a0, hi = a1 - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (__ldg(coarse_start + mid) <= cd) lo = mid; else hi = mid - 1;
    }
    int a = lo;
    int cs = __ldg(coarse_start + a), ra = __ldg(coarse_start + a + 1) - cs;
    int rs = __ldg(row_start + a), na = __ldg(row_start + a + 1) - rs;
    const TC* pa = P + __ldg(blk_start + a) + (cd - cs);
    const TC* ta = tsm + (size_t)(rs - r0) * K + c;
    TC s = TC(0);
    for (int i = 0; i < na; ++i) s = fma(__ldg(pa + (size_t)i * ra), ta[(size_t)i * K], s);
    fc[(size_t)cd * K + c] = s;
    if (uc) uc[(size_t)cd * K + c] = s * __ldg(dinvc + cd);
  }
}

// u[rows(a)] += P_a uc[coarse(a)]   (aggregate-aligned CTAs)
template <typename TC, int K>
__global__ void __launch_bounds__(BS) k_prolong(const int* __restrict__ cta_agg, const int* __restrict__ row_start,
                                                const int* __restrict__ coarse_start,
                                                const long long* __restrict__ blk_start, const TC* __restrict__ P,
                                                const TC* __restrict__ uc, TC* __restrict__ u,
                                                const int* __restrict__ done) {
  if (*done) return;
  constexpr int CPT = VT<TC, K>::CPT;
  const int a0 = cta_agg[blockIdx.x], a1 = cta_agg[blockIdx.x + 1];
  const int r0 = row_start[a0], r1 = row_start[a1];
  const int nout = (r1 - r0) * (K / CPT);
  for (int o = threadIdx.x; o < nout; o += BS) {
    int i = r0 + o / (K / CPT), c = (o % (K / CPT)) * CPT;
    int lo = a0, hi = a1 - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (__ldg(row_start + mid) <= i) lo = mid; else hi = mid - 1;
    }
    int a = lo;
    int cs = __ldg(coarse_start + a), ra = __ldg(coarse_start + a + 1) - cs;
    const TC* pr = P + __ldg(blk_start + a) + (size_t)(i - __ldg(row_start + a)) * ra;
    TC s[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) s[t] = TC(0);
    for (int p = 0; p < ra; ++p) {
      TC pv = __ldg(pr + p);
      TC cv[CPT];
      ldv<TC, CPT>(uc + (size_t)(cs + p) * K + c, cv);
#pragma unroll
      for (int t = 0; t < CPT; ++t) s[t] = fma(pv, cv[t], s[t]);
    }
    TC* up = u + (size_t)i * K + c;
    TC uv[CPT];
    ldp<TC, CPT>(up, uv);
#pragma unroll
    for (int t = 0; t < CPT; ++t) uv[t] += s[t];
    stv<TC, CPT>(up, uv);
  }
}

// Coarsest level: u = A_c^{-1} f with the float64 inverse of each diagonal
// block (one warp per row, float64 accumulation).
template <typename TC, int K>
__global__ void __launch_bounds__(BS) k_coarse(int n, int nblk, const int* __restrict__ blk_off,
                                               const long long* __restrict__ inv_off,
                                               const double* __restrict__ inv, const TC* __restrict__ f,
                                               TC* __restrict__ u, const int* __restrict__ done) {
  if (*done) return;
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * BS + threadIdx.x) >> 5;
  if (row >= n) return;
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(blk_off + mid) <= row) lo = mid; else hi = mid - 1;
  }
  const int b0 = blk_off[lo], nb = blk_off[lo + 1] - b0;
  const double* Ar = inv + inv_off[lo] + (size_t)(row - b0) * nb;
  double acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = 0.0;
  for (int j = lane; j < nb; j += 32) {
    double a = __ldg(Ar + j);
    const TC* fj = f + (size_t)(b0 + j) * K;
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = fma(a, (double)fj[c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < K; ++c) {
    double s = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == c % 32) u[(size_t)row * K + c] = (TC)s;
  }
}

// ----------------------------------------------------- fused CG kernels --

// Level-0 elementwise pass with per-(system, column) scalars.  The CTA's
// rows all belong to one system.  Each thread owns CPT consecutive columns
// of its rows (BS*CPT is a multiple of K, so the columns never change).
#define AMG_ELEMENTWISE_PROLOGUE(T_)                                           \
  constexpr int CPT = VT<T_, K>::CPT;                                          \
  const int r0 = cta_row[blockIdx.x], r1 = cta_row[blockIdx.x + 1];            \
  const size_t e0 = (size_t)r0 * K, e1 = (size_t)r1 * K;                       \
  const int cfirst = (int)((threadIdx.x * CPT) % K);

// x += alpha p; r -= alpha q; ||r||^2; then the first pre-sweep of the
// V-cycle from zero, u0 = D^{-1} r, and f0 = r in the cycle precision.  The
// last CTA applies the stopping test of every (system, column).
template <typename TC, int K>
__global__ void __launch_bounds__(BS) k_cg_update(const int* __restrict__ cta_row, double* __restrict__ x,
                                                  double* __restrict__ r, const double* __restrict__ p,
                                                  const double* __restrict__ q, const double* __restrict__ dinv,
                                                  TC* __restrict__ u0, TC* __restrict__ f0, KState ks) {
  if (*ks.done) return;
  __shared__ double sm[BS];
  __shared__ double tot[64];
  AMG_ELEMENTWISE_PROLOGUE(double)
  const int s = cta_system(ks.sys_cta, ks.nsys);
  double al[CPT], d[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    al[t] = ks.alpha[s * K + cfirst + t];
    d[t] = 0;
  }
  for (size_t e = e0 + (size_t)threadIdx.x * CPT; e < e1; e += (size_t)BS * CPT) {
    double xv[CPT], rv[CPT], pv[CPT], qv[CPT];
    ldp<double, CPT>(x + e, xv);
    ldp<double, CPT>(r + e, rv);
    ldv<double, CPT>(p + e, pv);
    ldv<double, CPT>(q + e, qv);
    // a one-level hierarchy has no smoother: u0 (and dinv) are then absent
    double di = u0 ? __ldg(dinv + e / K) : 0.0;
    TC uo[CPT], fo[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      xv[t] = fma(al[t], pv[t], xv[t]);
      rv[t] = fma(-al[t], qv[t], rv[t]);
      d[t] = fma(rv[t], rv[t], d[t]);
      uo[t] = (TC)(di * rv[t]);
      fo[t] = (TC)rv[t];
    }
    stv<double, CPT>(x + e, xv);
    stv<double, CPT>(r + e, rv);
    if (u0) stv<TC, CPT>(u0 + e, uo);
    if (f0) stv<TC, CPT>(f0 + e, fo);
  }
  cta_colsum<K, CPT>(d, sm, ks.partial + (size_t)blockIdx.x * K);
  if (!arrive_last(ks.counter + 1)) return;
  const int it = *ks.iter + 1;
  int stopped = 1;
  for (int sy = 0; sy < ks.nsys; ++sy) {
    sum_partials(ks.partial, K, ks.sys_cta[sy], ks.sys_cta[sy + 1], sm, tot);
    if (threadIdx.x < K) {
      int v = sy * K + threadIdx.x;
      if (ks.conv[v] == ST_ACTIVE) {
        double rn = sqrt(tot[threadIdx.x]);
        ks.rnorm[v] = rn;
        if (!isfinite(rn)) {
          ks.conv[v] = ST_BREAKDOWN;
          ks.status[v] = AMG_ERR_BREAKDOWN;
          ks.iters[v] = it;
        } else if (rn <= ks.rtol * ks.bnorm[v]) {
          ks.conv[v] = ST_CONVERGED;
          ks.iters[v] = it;
        } else if (it >= ks.maxit) {
          ks.conv[v] = ST_MAXIT;
          ks.status[v] = AMG_ERR_NOT_CONVERGED;
          ks.iters[v] = it;
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int v = 0; v < ks.nsys * K; ++v)
      if (ks.conv[v] == ST_ACTIVE) stopped = 0;
    *ks.iter = it;
    if (stopped) *ks.done = 1;
    *(ks.counter + 1) = 0u;
  }
}

// First pre-sweep from zero on level 0 (used after the initial residual).
template <typename TC, int K>
__global__ void __launch_bounds__(BS) k_presmooth0(const int* __restrict__ cta_row, const double* __restrict__ r,
                                                   const double* __restrict__ dinv, TC* __restrict__ u0,
                                                   TC* __restrict__ f0, const int* __restrict__ done) {
  if (*done) return;
  AMG_ELEMENTWISE_PROLOGUE(double)
  (void)cfirst;
  for (size_t e = e0 + (size_t)threadIdx.x * CPT; e < e1; e += (size_t)BS * CPT) {
    double rv[CPT];
    ldv<double, CPT>(r + e, rv);
    double di = __ldg(dinv + e / K);
    TC uo[CPT], fo[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      uo[t] = (TC)(di * rv[t]);
      fo[t] = (TC)rv[t];
    }
    stv<TC, CPT>(u0 + e, uo);
    if (f0) stv<TC, CPT>(f0 + e, fo);
  }
}

// Level-0 post-sweep producing the preconditioned residual in float64,
//   z = u + D^{-1} (f - A u),
// fused with r.z.  mode 0: rho = r.z (start); mode 1: beta = r.z / rho,
// rho = r.z; mode 2: no scalars (a bare V-cycle).
template <typename TC, int K, int NZL>
__global__ void __launch_bounds__(BS) k_post0(const int* __restrict__ cta_row, const int* __restrict__ rowptr,
                                              const int* __restrict__ col, const TC* __restrict__ val,
                                              const TC* __restrict__ dinv, const TC* __restrict__ f,
                                              const TC* __restrict__ u, const double* __restrict__ r,
                                              double* __restrict__ z, KState ks, int mode) {
  if (*ks.done) return;
  __shared__ double sm[BS];
  __shared__ double tot[64];
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  const int r0 = cta_row[blockIdx.x], r1 = cta_row[blockIdx.x + 1];
  double d[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) d[t] = 0;
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    TC acc[CPT];
    row_acc<TC, TC, K, NZL>(i, valid, rowptr, col, val, u, nzl, cl, acc);
    if (valid && nzl == 0) {
      TC fv[CPT], uv[CPT];
      size_t o = (size_t)i * K + cl * CPT;
      ldv<TC, CPT>(f + o, fv);
      ldv<TC, CPT>(u + o, uv);
      TC di = __ldg(dinv + i);
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        double zv = (double)fma(di, fv[t] - acc[t], uv[t]);
        double rv = __ldg(r + o + t);
        z[o + t] = zv;
        d[t] = fma(rv, zv, d[t]);
      }
    }
  }
  if (mode == 2) return;
  // lanes other than nzl == 0 hold zeros; reduce across the whole warp
  cta_colsum<K, CPT>(d, sm, ks.partial + (size_t)blockIdx.x * K);
  if (!arrive_last(ks.counter + 2)) return;
  for (int sy = 0; sy < ks.nsys; ++sy) {
    sum_partials(ks.partial, K, ks.sys_cta[sy], ks.sys_cta[sy + 1], sm, tot);
    if (threadIdx.x < K) {
      int v = sy * K + threadIdx.x;
      double rz = tot[threadIdx.x];
      if (mode == 0) {
        ks.rho[v] = rz;
        ks.beta[v] = 0.0;
      } else if (ks.conv[v] == ST_ACTIVE) {
        ks.beta[v] = rz / ks.rho[v];
        ks.rho[v] = rz;
      } else {
        ks.beta[v] = 0.0;
      }
      if (ks.conv[v] == ST_ACTIVE && !(rz > 0.0 && isfinite(rz))) {
        ks.conv[v] = ST_BREAKDOWN;
        ks.status[v] = AMG_ERR_BREAKDOWN;
        ks.iters[v] = *ks.iter;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int stopped = 1;
    for (int v = 0; v < ks.nsys * K; ++v)
      if (ks.conv[v] == ST_ACTIVE) stopped = 0;
    if (stopped) *ks.done = 1;
    *(ks.counter + 2) = 0u;
  }
}

}  // namespace amg

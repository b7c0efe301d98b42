// Preconditioned CG driver (Section 5) over the V-cycle kernels, with the
// float64 CG kernels, the caller <-> library permutations, CUDA-graph
// replay of whole iterations, and the adjoint gradient kernel.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>

#include "amg_coarse.cuh"
#include "amg_launch.cuh"

namespace amg {

// ------------------------------------------------------- float64 kernels --

// Last CTA of a q = A p launch: alpha = rho / p.q for every active column;
// p.q <= 0 or a non-finite alpha stops the column with a breakdown.
template <int K>
__device__ __forceinline__ void finish_alpha(KState& ks, double* sm, double* tot) {
  for (int sy = 0; sy < ks.nsys; ++sy) {
    system_totals(ks, K, sy, sm, tot);
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
      ks.alpha_prev[v] = ks.alpha[v];
      ks.alpha[v] = a;
    }
    __syncthreads();
  }
}

// q = A p in double-float on the float32 pipes: A as (val32, vallo), p a
// float32 vector (the search direction is rounded to float32 when it is
// formed, so every product a_ij p_j is error-free up to the final rounding
// of the pair); q is stored as a float pair and p.q is accumulated in
// double-float.  With one lane group per row the gathers of a whole row are
// issued before its first product (otherwise the loop is software-pipelined
// one non-zero ahead), and the p.q accumulators live in shared memory, one
// slot per thread, so that three CTAs fit on an SM.  Offsets into the n x K
// blocks are 32-bit (n K < 2^32 is checked on the host).
// PKD: val_hi and val_lo of a non-zero come as one 8-byte pair of hl (one
// load instead of two; the unstaged path only).
template <int K, int NZL, bool STG, int UQ = 0, bool PKD = false>
__global__ void __launch_bounds__(BS, 3) k_cg_q_df(const int* __restrict__ cta_row, const int* __restrict__ rowptr,
                                                   const int* __restrict__ col, const float* __restrict__ ahi,
                                                   const float* __restrict__ alo, const float* p0,
                                                   const float* p1, float* __restrict__ qh,
                                                   float* __restrict__ ql, KState ks, Stage sg, int nchunk,
                                                   const float2* __restrict__ hl) {
  if (*ks.done) return;
  // p_k lives in p0 for even k, in p1 for odd k (k the device iteration counter)
  const float* __restrict__ p = (*ks.iter & 1) ? p1 : p0;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sm[BS];
  __shared__ double tot[64];
  constexpr int CPT = VT<float, K>::CPT, CL = VT<float, K>::CL, G = NZL * CL, RPW = 32 / G;
  // the packed path: batches of full rows, column pairs (p.q accumulated on
  // pairs too, in sdot2); UQ, when set, is the batch (the longest row)
  constexpr bool PK = gather_depth<NZL>() != 4 && CPT % 2 == 0;
  constexpr int UB = UQ > 0 ? UQ : gather_depth<NZL>(), NQ = PK ? CPT / 2 : 1;
  __shared__ float sdot[PK ? 1 : 2 * CPT][BS];
  __shared__ F2 sdot2[2 * NQ][PK ? BS : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  if constexpr (PK) {
#pragma unroll
    for (int q = 0; q < 2 * NQ; ++q) sdot2[q][threadIdx.x] = F2{0ull};
  } else {
#pragma unroll
    for (int t = 0; t < 2 * CPT; ++t) sdot[t][threadIdx.x] = 0.f;
  }
  // row chunks: one per CTA, or (persistent launch) every gridDim.x-th
  // chunk; staged launches take col, val_hi and val_lo (and rowptr) through
  // the double-buffered pipeline, the next chunk arriving while this one is
  // processed
  // STG: staged launches (the unstaged variant keeps its loads global)
  if (STG && sg.enabled) {
    pipe_init(smraw);
    if (threadIdx.x == 0 && (int)blockIdx.x < nchunk) {
      const float* v2[2] = {ahi, alo};
      pipe_issue<2>(sg, smraw, 0, cta_row[blockIdx.x], cta_row[blockIdx.x + 1], rowptr, col, v2);
    }
  }
  int it = 0;
  for (int chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x, ++it) {
  const int r0 = cta_row[chunk], r1 = cta_row[chunk + 1];
  const int* rp = rowptr;
  const int* cc = col;
  const float* va = ahi;
  const float* vb = alo;
  int roff = 0, joff = 0;
  if (STG && sg.enabled) {
    const int nxt = chunk + gridDim.x;
    if (threadIdx.x == 0 && nxt < nchunk) {
      const float* v2[2] = {ahi, alo};
      pipe_issue<2>(sg, smraw, (it + 1) & 1, cta_row[nxt], cta_row[nxt + 1], rowptr, col, v2);
    }
    const float* pv[2];
    pipe_wait<2>(sg, smraw, it & 1, it >> 1, r0, rowptr, rp, roff, cc, pv, joff);
    va = pv[0];
    vb = pv[1];
  }
  const unsigned lo = (unsigned)(cl * CPT);
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    const int i = base + g;
    const bool valid = i < r1;
    float sh[CPT], sl[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) sh[t] = sl[t] = 0.f;
    if (valid) {
      const int j1 = rp[i + 1 - roff] - joff;
      int j = rp[i - roff] - joff + nzl;
      if constexpr (PK) {
        // predicated batches: every gather of a batch is issued before the
        // first product (a 9-point row in one memory round trip); the
        // double-float steps run on column pairs
        constexpr int U = UB, NP = CPT / 2;
        F2 h2[NP], l2[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) h2[q] = l2[q] = F2{0ull};
        for (; j < j1; j += U * NZL) {
          F2 xv[U][NP];
          if constexpr (PKD) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int jj = j + u * NZL;
              if (jj < j1) {
                const float* src = p + (unsigned)cc[jj] * (unsigned)K + lo;
                if constexpr (NP == 2) {
                  const ulonglong2 t2 = __ldg(reinterpret_cast<const ulonglong2*>(src));
                  xv[u][0] = F2{t2.x};
                  xv[u][1] = F2{t2.y};
                } else {
#pragma unroll
                  for (int q = 0; q < NP; ++q)
                    xv[u][q] = F2{__ldg(reinterpret_cast<const unsigned long long*>(src) + q)};
                }
              } else {
#pragma unroll
                for (int q = 0; q < NP; ++q) xv[u][q] = F2{0ull};
              }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int jj = j + u * NZL;
              const float2 ab = jj < j1 ? __ldg(hl + jj) : make_float2(0.f, 0.f);
              const F2 a2 = f2_pack(ab.x, ab.x), b2 = f2_pack(ab.y, ab.y);
#pragma unroll
              for (int q = 0; q < NP; ++q) df_acc1_x2(a2, b2, xv[u][q], h2[q], l2[q]);
            }
            continue;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int jj = j + u * NZL;
            if (jj < j1) {
              const float* src = p + (unsigned)cc[jj] * (unsigned)K + lo;
              if constexpr (NP == 2) {
                const ulonglong2 t2 = __ldg(reinterpret_cast<const ulonglong2*>(src));
                xv[u][0] = F2{t2.x};
                xv[u][1] = F2{t2.y};
              } else {
#pragma unroll
                for (int q = 0; q < NP; ++q) xv[u][q] = F2{__ldg(reinterpret_cast<const unsigned long long*>(src) + q)};
              }
            } else {
#pragma unroll
              for (int q = 0; q < NP; ++q) xv[u][q] = F2{0ull};
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int jj = j + u * NZL;
            const float a = jj < j1 ? va[jj] : 0.f, b = jj < j1 ? vb[jj] : 0.f;
            const F2 a2 = f2_pack(a, a), b2 = f2_pack(b, b);
#pragma unroll
            for (int q = 0; q < NP; ++q) df_acc1_x2(a2, b2, xv[u][q], h2[q], l2[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          df_norm_x2(h2[q], l2[q]);
          f2_unpack(h2[q], sh[2 * q], sh[2 * q + 1]);
          f2_unpack(l2[q], sl[2 * q], sl[2 * q + 1]);
        }
      } else if constexpr (gather_depth<NZL>() != 4) {
        // predicated batches, scalar columns
        constexpr int U = UB;
        for (; j < j1; j += U * NZL) {
          float xv[U][CPT];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int jj = j + u * NZL;
            if (jj < j1) {
              ldv<float, CPT>(p + (unsigned)cc[jj] * (unsigned)K + lo, xv[u]);
            } else {
#pragma unroll
              for (int t = 0; t < CPT; ++t) xv[u][t] = 0.f;
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int jj = j + u * NZL;
            const float a = jj < j1 ? va[jj] : 0.f, b = jj < j1 ? vb[jj] : 0.f;
#pragma unroll
            for (int t = 0; t < CPT; ++t) df_acc1(a, b, xv[u][t], sh[t], sl[t]);
          }
        }
      } else if (j < j1) {
        float a = va[j], b = vb[j];
        float xv[CPT];
        ldv<float, CPT>(p + (unsigned)cc[j] * (unsigned)K + lo, xv);
        for (j += NZL; j < j1; j += NZL) {
          const float a2 = va[j], b2 = vb[j];
          float yv[CPT];
          ldv<float, CPT>(p + (unsigned)cc[j] * (unsigned)K + lo, yv);
#pragma unroll
          for (int t = 0; t < CPT; ++t) df_acc1(a, b, xv[t], sh[t], sl[t]);
#pragma unroll
          for (int t = 0; t < CPT; ++t) xv[t] = yv[t];
          a = a2;
          b = b2;
        }
#pragma unroll
        for (int t = 0; t < CPT; ++t) df_acc1(a, b, xv[t], sh[t], sl[t]);
      }
      if constexpr (!PK) {  // (the packed path renormalised its pairs)
#pragma unroll
        for (int t = 0; t < CPT; ++t) df_norm(sh[t], sl[t]);
      }
    }
    if constexpr (NZL > 1) {
#pragma unroll
      for (int off = CL; off < CL * NZL; off <<= 1)
#pragma unroll
        for (int t = 0; t < CPT; ++t) {
          float oh = __shfl_xor_sync(FULL, sh[t], off), ol = __shfl_xor_sync(FULL, sl[t], off);
          df_add(sh[t], sl[t], oh, ol);
        }
    }
    if (valid && nzl == 0) {
      const unsigned o = (unsigned)i * (unsigned)K + lo;
      float pv[CPT];
      ldv<float, CPT>(p + o, pv);
      stv<float, CPT>(qh + o, sh);
      stv<float, CPT>(ql + o, sl);
      if constexpr (PK) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          F2 h = sdot2[q][threadIdx.x], l = sdot2[NQ + q][threadIdx.x];
          df_acc1_x2(f2_pack(sh[2 * q], sh[2 * q + 1]), f2_pack(sl[2 * q], sl[2 * q + 1]),
                     f2_pack(pv[2 * q], pv[2 * q + 1]), h, l);
          sdot2[q][threadIdx.x] = h;
          sdot2[NQ + q][threadIdx.x] = l;
        }
      } else {
#pragma unroll
        for (int t = 0; t < CPT; ++t) {
          float h = sdot[t][threadIdx.x], l = sdot[CPT + t][threadIdx.x];
          df_acc1(sh[t], sl[t], pv[t], h, l);
          sdot[t][threadIdx.x] = h;
          sdot[CPT + t][threadIdx.x] = l;
        }
      }
    }
  }
  if (STG && sg.enabled) __syncthreads();  // the buffer is refilled two chunks on
  }
  double d[CPT];
  if constexpr (PK) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float h0, h1, l0, l1;
      f2_unpack(sdot2[q][threadIdx.x], h0, h1);
      f2_unpack(sdot2[NQ + q][threadIdx.x], l0, l1);
      d[2 * q] = (double)h0 + (double)l0;
      d[2 * q + 1] = (double)h1 + (double)l1;
    }
  } else {
#pragma unroll
    for (int t = 0; t < CPT; ++t) d[t] = (double)sdot[t][threadIdx.x] + (double)sdot[CPT + t][threadIdx.x];
  }
  cta_colsum<K, CPT>(d, sm, ks.partial + (size_t)blockIdx.x * K);
  if (!arrive_two_level(ks, RED_Q, K, sm, tot)) return;
  finish_alpha<K>(ks, sm, tot);
}

// q = A p with p.q; the last CTA forms alpha = rho / p.q per column.
template <int K, int NZL>
__global__ void __launch_bounds__(BS) k_cg_q(const int* __restrict__ cta_row, const int* __restrict__ rowptr,
                                             const int* __restrict__ col, const double* __restrict__ val,
                                             const double* __restrict__ p, double* __restrict__ q, KState ks) {
  if (*ks.done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sm[BS];
  __shared__ double tot[64];
  constexpr int CPT = VT<double, K>::CPT, CL = VT<double, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  const int r0 = cta_row[blockIdx.x], r1 = cta_row[blockIdx.x + 1];
  double d[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) d[t] = 0;
  const CsrView<double> cv = staged_view<double>(ks.sg, smraw, r0, r1, rowptr, col, val);
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    double acc[CPT];
    row_acc<double, double, K, NZL>(i, valid, cv, p, nzl, cl, acc);
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
  if (!arrive_two_level(ks, RED_Q, K, sm, tot)) return;
  finish_alpha<K>(ks, sm, tot);
}

// r = b - A x with ||b||^2 and ||r||^2; the last CTA initialises the state
// of every (system, column): zero right-hand sides and padding columns stop
// at once, as does a column whose initial guess already meets the tolerance.
template <int K, int NZL>
__global__ void __launch_bounds__(BS) k_cg_init(const int* __restrict__ cta_row, const int* __restrict__ rowptr,
                                                const int* __restrict__ col, const double* __restrict__ val,
                                                const double* __restrict__ b, const double* __restrict__ x,
                                                double* __restrict__ r, KState ks) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sm[BS];
  __shared__ double tot[64];
  constexpr int CPT = VT<double, K>::CPT, CL = VT<double, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  const int r0 = cta_row[blockIdx.x], r1 = cta_row[blockIdx.x + 1];
  double db[CPT], dr[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) db[t] = dr[t] = 0;
  const CsrView<double> cv = staged_view<double>(ks.sg, smraw, r0, r1, rowptr, col, val);
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    double acc[CPT];
    row_acc<double, double, K, NZL>(i, valid, cv, x, nzl, cl, acc);
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
  if (!arrive_two_level(ks, RED_INIT, 2 * K, sm, tot)) return;
  for (int sy = 0; sy < ks.nsys; ++sy) {
    system_totals(ks, 2 * K, sy, sm, tot);
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
  }
}

// p = z + beta p in float64 (the float64 CG; the double-float CG has
// k_cg_p_df).  z is stored in the cycle precision TZ; ``first`` starts the recurrence
// (p = z, the previous p is not read).
template <int K, typename TZ>
__global__ void __launch_bounds__(BS) k_cg_p(const int* __restrict__ cta_row, const TZ* __restrict__ z,
                                             double* __restrict__ p, KState ks, int first) {
  if (*ks.done) return;
  AMG_ELEMENTWISE_PROLOGUE(double)
  const int s = cta_system(ks.sys_cta, ks.nsys);
  double be[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) be[t] = ks.beta[s * K + cfirst + t];
  for (size_t e = e0 + (size_t)threadIdx.x * CPT; e < e1; e += (size_t)BS * CPT) {
    TZ zt[CPT];
    double pv[CPT];
    ldv<TZ, CPT>(z + e, zt);
    if (first) {
#pragma unroll
      for (int t = 0; t < CPT; ++t) pv[t] = (double)zt[t];
    } else {
      ldp<double, CPT>(p + e, pv);
#pragma unroll
      for (int t = 0; t < CPT; ++t) pv[t] = fma(be[t], pv[t], (double)zt[t]);
    }
    stv<double, CPT>(p + e, pv);
  }
}

// ------------------------------------------------ double-float CG vectors --
// In the float32-cycle mode x, r, p and q are kept as double-float pairs
// (hi, lo) and every CG vector operation runs on the float32 pipes; the CG
// scalars (alpha, beta, rho, norms) stay float64.  r_hi = fl32(r) is then
// exactly the float32 right-hand side of the level-0 cycle.

__device__ __forceinline__ void split2(double v, float& h, float& l) { df_split(v, h, l); }

// r -= alpha q, ||r||^2; u0 = D^{-1} r_hi (the first pre-sweep from zero;
// not stored when u0 is null, the cycle then folding it into A D^{-1}).
// (x is advanced by k_cg_p_df, which streams p anyway.)
template <int K>
__global__ void __launch_bounds__(BS) k_cg_update_df(const int* __restrict__ cta_row, float* __restrict__ rh,
                                                     float* __restrict__ rl, const float* __restrict__ qh,
                                                     const float* __restrict__ ql, const float* __restrict__ dinv,
                                                     float* __restrict__ u0, KState ks, int nchunk) {
  if (*ks.done) return;
  __shared__ double sm[BS];
  __shared__ double tot[64];
  constexpr int CPT = VT<float, K>::CPT;
  const int cfirst = (int)((threadIdx.x * CPT) % K);
  const int s = cta_system(ks.sys_cta, ks.nsys);
  float ah[CPT], al[CPT], dh[CPT], dl[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    split2(-ks.alpha[s * K + cfirst + t], ah[t], al[t]);
    dh[t] = dl[t] = 0.f;
  }
  // one row range per CTA, or (persistent launch, one system) every
  // gridDim.x-th range
  // a thread keeps the loads of UN row-column groups in flight before any
  // arithmetic (the groups in order, so the norm's rounding is unchanged)
  constexpr int UN = 2;
  for (int chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x) {
  const size_t e0 = (size_t)cta_row[chunk] * K, e1 = (size_t)cta_row[chunk + 1] * K;
  for (size_t eb = e0 + (size_t)threadIdx.x * CPT; eb < e1; eb += (size_t)UN * BS * CPT) {
    float ra[UN][CPT], rb[UN][CPT], qa[UN][CPT], qb[UN][CPT], di[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const size_t e = eb + (size_t)u * BS * CPT;
      if (e < e1) {
        ldp<float, CPT>(rh + e, ra[u]);
        ldp<float, CPT>(rl + e, rb[u]);
        ldv<float, CPT>(qh + e, qa[u]);
        ldv<float, CPT>(ql + e, qb[u]);
        di[u] = u0 ? __ldg(dinv + e / K) : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const size_t e = eb + (size_t)u * BS * CPT;
      if (e >= e1) continue;
      float uo[CPT];
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        df_mac(ah[t], al[t], qa[u][t], qb[u][t], ra[u][t], rb[u][t]);
        df_acc(ra[u][t], rb[u][t], ra[u][t], rb[u][t], dh[t], dl[t]);
        uo[t] = di[u] * ra[u][t];
      }
      stv<float, CPT>(rh + e, ra[u]);
      stv<float, CPT>(rl + e, rb[u]);
      if (u0) stv<float, CPT>(u0 + e, uo);
    }
  }
  }
  double d[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) d[t] = (double)dh[t] + (double)dl[t];
  cta_colsum<K, CPT>(d, sm, ks.partial + (size_t)blockIdx.x * K);
  if (!arrive_two_level(ks, RED_UPDATE, K, sm, tot)) return;
  finish_update<K>(ks, sm, tot);
}

// End of iteration k (the device counter already reads k + 1): p_{k+1} =
// fl32(z + beta p_k), p_k read from its buffer (p0 for even k, p1 for odd k)
// and p_{k+1} written to the other one; ``first`` starts the recurrence
// (p_0 = z into p0, x untouched).  The step x += alpha p is taken every
// second iteration: after an odd k, x += alpha_{k-1} p_{k-1} + alpha_k p_k,
// with p_{k-1} read from the buffer p_{k+1} then overwrites (x a
// double-float pair, each p an exact float32), so x is read and written half
// as often.  Rounding the search direction to float32 only perturbs it at
// the level of the float32 cycle's own rounding: x and r stay consistent
// because q = A p is formed from the same rounded p.  After the last
// iteration k_cg_x_df applies the steps still pending.
template <int K>
__global__ void __launch_bounds__(BS, 3) k_cg_p_df(const int* __restrict__ cta_row, const float* __restrict__ z,
                                                float* p0, float* p1, float* __restrict__ xh,
                                                float* __restrict__ xl, KState ks, int first, int nchunk) {
  if (*ks.done) return;
  constexpr int CPT = VT<float, K>::CPT;
  const int cfirst = (int)((threadIdx.x * CPT) % K);
  const int s = cta_system(ks.sys_cta, ks.nsys);
  const int k = first ? -1 : *ks.iter - 1;   // the iteration that ends here
  const bool step = !first && (k & 1);       // an odd k takes the two pending x steps
  const float* pin = (k & 1) ? p1 : p0;      // p_k
  float* pout = (k & 1) ? p0 : p1;           // p_{k+1} (after an odd k: where p_{k-1} is)
  if (first) pout = p0;
  float bh[CPT], bl[CPT], ah[CPT], al[CPT], ch[CPT], cl[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    split2(ks.beta[s * K + cfirst + t], bh[t], bl[t]);
    split2(ks.alpha[s * K + cfirst + t], ah[t], al[t]);
    split2(ks.alpha_prev[s * K + cfirst + t], ch[t], cl[t]);
  }
  // a thread keeps the loads of UN row-column groups in flight (4 without
  // the x step, 2 with it) before any arithmetic
  auto pass = [&](auto unc, bool stp) {
    constexpr int UN = decltype(unc)::value;
    for (int chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x) {
      const size_t e0 = (size_t)cta_row[chunk] * K, e1 = (size_t)cta_row[chunk + 1] * K;
      for (size_t eb = e0 + (size_t)threadIdx.x * CPT; eb < e1; eb += (size_t)UN * BS * CPT) {
        float zv[UN][CPT], pv[UN][CPT], po[UN][CPT], xa[UN][CPT], xb[UN][CPT];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          const size_t e = eb + (size_t)u * BS * CPT;
          if (e < e1) {
            ldv<float, CPT>(z + e, zv[u]);
            if (!first) ldp<float, CPT>(pin + e, pv[u]);
            if (stp) {
              ldp<float, CPT>(pout + e, po[u]);   // p_{k-1}
              ldp<float, CPT>(xh + e, xa[u]);
              ldp<float, CPT>(xl + e, xb[u]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          const size_t e = eb + (size_t)u * BS * CPT;
          if (e >= e1) continue;
          if (first) {
#pragma unroll
            for (int t = 0; t < CPT; ++t) pv[u][t] = zv[u][t];
          } else {
            if (stp) {
#pragma unroll
              for (int t = 0; t < CPT; ++t) {
                df_acc1(ch[t], cl[t], po[u][t], xa[u][t], xb[u][t]);
                df_acc1(ah[t], al[t], pv[u][t], xa[u][t], xb[u][t]);
                df_norm(xa[u][t], xb[u][t]);
              }
              stv<float, CPT>(xh + e, xa[u]);
              stv<float, CPT>(xl + e, xb[u]);
            }
#pragma unroll
            for (int t = 0; t < CPT; ++t) pv[u][t] = fmaf(bl[t], pv[u][t], fmaf(bh[t], pv[u][t], zv[u][t]));
          }
          stv<float, CPT>(pout + e, pv[u]);
        }
      }
    }
  };
  if (step) pass(std::integral_constant<int, 2>{}, true);
  else pass(std::integral_constant<int, 4>{}, false);
}

// The x steps still pending after the last iteration K (kl = K): for an
// even K, x += alpha_K p_K; for an odd K, x += alpha_{K-1} p_{K-1} +
// alpha_K p_K (the alphas of columns that stopped earlier are already zero;
// kl = -1, no iteration, steps by zero).
template <int K>
__global__ void __launch_bounds__(BS) k_cg_x_df(const int* __restrict__ cta_row, const float* __restrict__ p0,
                                                const float* __restrict__ p1, float* __restrict__ xh,
                                                float* __restrict__ xl, KState ks, int kl) {
  constexpr int CPT = VT<float, K>::CPT;
  const int r0 = cta_row[blockIdx.x], r1 = cta_row[blockIdx.x + 1];
  const size_t e0 = (size_t)r0 * K, e1 = (size_t)r1 * K;
  const int cfirst = (int)((threadIdx.x * CPT) % K);
  const int s = cta_system(ks.sys_cta, ks.nsys);
  const bool two = kl >= 1 && (kl & 1);
  const float* pl = (kl & 1) ? p1 : p0;   // p_K
  const float* pp = (kl & 1) ? p0 : p1;   // p_{K-1}
  float ah[CPT], al[CPT], ch[CPT], cl[CPT];
#pragma unroll
  for (int t = 0; t < CPT; ++t) {
    split2(ks.alpha[s * K + cfirst + t], ah[t], al[t]);
    split2(ks.alpha_prev[s * K + cfirst + t], ch[t], cl[t]);
  }
  for (size_t e = e0 + (size_t)threadIdx.x * CPT; e < e1; e += (size_t)BS * CPT) {
    float pv[CPT], xa[CPT], xb[CPT];
    ldv<float, CPT>(pl + e, pv);
    ldp<float, CPT>(xh + e, xa);
    ldp<float, CPT>(xl + e, xb);
    if (two) {
      float po[CPT];
      ldv<float, CPT>(pp + e, po);
#pragma unroll
      for (int t = 0; t < CPT; ++t) df_acc1(ch[t], cl[t], po[t], xa[t], xb[t]);
    }
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      df_acc1(ah[t], al[t], pv[t], xa[t], xb[t]);
      df_norm(xa[t], xb[t]);
    }
    stv<float, CPT>(xh + e, xa);
    stv<float, CPT>(xl + e, xb);
  }
}

// float64 <-> double-float pairs (start and end of a solve)
__global__ void k_split_pair(long long n, const double* __restrict__ v, float* __restrict__ h,
                             float* __restrict__ l) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) df_split(v[i], h[i], l[i]);
}
__global__ void k_join_pair(long long n, const float* __restrict__ h, const float* __restrict__ l,
                            double* __restrict__ v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (double)h[i] + (double)l[i];
}

__global__ void k_f32_to_f64(long long n, const float* __restrict__ a, double* __restrict__ b) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
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
  if (!arrive_two_level(ks, RED_POST, K, sm, tot)) return;
  for (int sy = 0; sy < ks.nsys; ++sy) {
    system_totals(ks, K, sy, sm, tot);
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
  bool split = false;  // double-float CG vectors (float32-cycle mode)
  bool u0free = false; // split with one pre-sweep: u0 = D^{-1} r_hi is folded into A D^{-1} (never stored)
  float *xh = nullptr, *xl = nullptr, *rh = nullptr, *rl = nullptr;
  float *ph = nullptr, *ph2 = nullptr;  // p_k in ph (even k) or ph2 (odd k); float32 (see k_cg_p_df)
  float *qh = nullptr, *ql = nullptr;
  std::vector<void*> f, u, v;
  KState ks{};
  int* zero_flag = nullptr;
  double* stage = nullptr;
  size_t stage_elems = 0;
  int* h_done = nullptr;  // pinned
  std::vector<int> nzl;   // per level
  int nzl_q = 0;          // lanes per row of the level-0 q = A p
  int q_stage = 1;        // whether the double-float q = A p stages its matrix slice
  int q_pack = 0;         // whether it reads the values as (hi, lo) pairs (unstaged)
  RPart rq{};             // level-0 row ranges of the double-float q = A p (own CTA size)
  int q_grid = 0;         // > 0: persistent q launch of q_grid CTAs over rq's ranges
  // persistent level-0 launches (one system): CTAs of the update, direction
  // and post-smoother kernels, 0 for one CTA per row range
  int upd_grid = 0, p_grid = 0, post_grid = 0;
  int post_stage = 0;            // persistent post-smoother: staged through the pipeline
  KState ksf_upd{}, ksf_post{};  // the CG state seen through those launches' CTA groups
  // the tuned choices, as applied (written to and read from the tuning cache)
  std::vector<long long> t_rp;  // per smoothed level: target, stage, lanes
  std::vector<int> t_rps, t_nzl;
  std::vector<int> t_tp, t_tps, t_tpw;  // per transfer: rows target (0: default), stage, warp kernel
  long long t_q = 0;                    // q: target (0: level-0 ranges), lanes, stage, persistent grid
  int t_qn = 0, t_qs = 0, t_qg = 0;
  int t_pu = 0, t_pp = 0, t_ppost = 0;  // persistent grids of update / p / post
  KState ksq{};           // the CG state seen through the q launch's CTA groups
  std::vector<TPart> tp;  // per transfer: CTA ranges for this column count
  std::vector<int> rform; // per transfer: restrict by R = P^T (I - A D^{-1}) (one pre-sweep only)
  std::vector<RPart> rp;  // per level: row ranges for this column count
  int* err = nullptr;     // bounded-wait failures of the staged kernels
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int gchunk = 0, gtimer = -1, gmaxit = -1;
  long long gkernels = 0;
  int* h_iter = nullptr;  // pinned
  double grtol = -1;
  int variant = 0;        // smoother | cycle << 1 (float64 only); 0: the tuned V-cycle
  VarCycle var;           // buffers of the variant cycle
  std::vector<cudaEvent_t> gev;
  // the small levels in one cooperative launch (k_coarse_cycle): start level
  // (-1: off), CTAs, barrier words, test hook
  int cc_s = -1, cc_grid = 0, cc_hang = 0;
  unsigned* cc_bar = nullptr;
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

// Aggregate-aligned CTA ranges holding about ``target`` rows each (an
// aggregate larger than that gets a CTA of its own).
// Staging capacities of a set of CTA row ranges; staging is switched off for
// the level when the largest slice would not fit comfortably in shared memory.
static Stage make_stage(const std::vector<int>& rp, const std::vector<int>& cr, int* err) {
  Stage sg;
  sg.err = err;
  for (size_t c = 0; c + 1 < cr.size(); ++c) {
    int r0 = cr[c], r1 = cr[c + 1], j0 = rp[r0], j1 = rp[r1];
    sg.rows_max = std::max(sg.rows_max, r1 - r0);
    sg.span4 = std::max(sg.span4, ((j1 + 3) & ~3) - (j0 & ~3));
    sg.span8 = std::max(sg.span8, ((j1 + 1) & ~1) - (j0 & ~1));
  }
  sg.enabled = 1;
  if (stage_bytes(sg, 2, 1) > 96 * 1024) sg.enabled = 0;
  return sg;
}

// Non-zeros per CTA of the row-parallel kernels: more columns, fewer rows.
static long long target_nnz(int K) { return K == 1 ? 4096 : (K <= 4 ? 2048 : 1024); }

static RPart make_rpart(Arena& ar, const Level& L, long long target, const std::vector<int>& sys_rows,
                        int* err) {
  const std::vector<int>& rp = L.h_rowptr;
  std::vector<int> cr{0}, sys_cta{0}, grp{0}, sys_grp{0};
  for (size_t s = 0; s + 1 < sys_rows.size(); ++s) {
    int r = sys_rows[s];
    const int end = sys_rows[s + 1];
    while (r < end) {
      const int start = r;
      const long long base = rp[r];
      ++r;
      while (r < end && rp[r + 1] - base <= target && r - start < 1024) ++r;
      cr.push_back(r);
    }
    const int c1 = (int)cr.size() - 1;
    for (int c = sys_cta.back(); c < c1; c += 64) grp.push_back(std::min(c + 64, c1));
    sys_cta.push_back(c1);
    sys_grp.push_back((int)grp.size() - 1);
  }
  RPart p;
  p.ncta = (int)cr.size() - 1;
  p.ngroups = (int)grp.size() - 1;
  auto up = [&](const std::vector<int>& v) {
    int* d = ar.alloc<int>(v.size());
    AMG_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
    return d;
  };
  p.cta_row = up(cr);
  p.grp_cta = up(grp);
  p.sys_grp = up(sys_grp);
  p.sys_cta = up(sys_cta);
  p.sg = make_stage(rp, cr, err);
  return p;
}

// CTA groups of a persistent launch of ``ncta`` CTAs over one system (no
// row ranges of its own: the CTAs walk the chunks of another partition).
static RPart make_flat(Arena& ar, int ncta) {
  std::vector<int> grp{0};
  for (int c = 0; c < ncta; c += 64) grp.push_back(std::min(c + 64, ncta));
  std::vector<int> sys_grp{0, (int)grp.size() - 1}, sys_cta{0, ncta};
  RPart p;
  p.ncta = ncta;
  p.ngroups = (int)grp.size() - 1;
  auto up = [&](const std::vector<int>& v) {
    int* d = ar.alloc<int>(v.size());
    AMG_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
    return d;
  };
  p.grp_cta = up(grp);
  p.sys_grp = up(sys_grp);
  p.sys_cta = up(sys_cta);
  return p;
}

// Staging capacities of CTAs over the row ranges [cr[c], cr[c+1]) of a
// grouped kernel (float values through the one-buffer pipeline); off when a
// slice would take more than 96 KB of shared memory.
static Stage make_group_stage(const std::vector<int>& rp, const std::vector<int>& cr) {
  Stage sg;
  for (size_t c = 0; c + 1 < cr.size(); ++c) {
    const int r0 = cr[c], r1 = cr[c + 1], j0 = rp[r0], j1 = rp[r1];
    sg.rows_max = std::max(sg.rows_max, r1 - r0);
    sg.span4 = std::max(sg.span4, ((j1 + 3) & ~3) - (j0 & ~3));
  }
  sg.enabled = 1;
  if (pipe_bytes(sg, 1, 1) > 96 * 1024) sg.enabled = 0;
  return sg;
}

static TPart make_tpart(Arena& ar, const Transfer& T, const Level& F, int K, int* err, int target = 0) {
  if (target <= 0) target = K <= 2 ? 256 : (K <= 8 ? 128 : 64);
  std::vector<int> ca{0};
  int rows = 0;
  for (int a = 0; a < T.nagg; ++a) {
    int na = T.h_row_start[a + 1] - T.h_row_start[a];
    if (rows > 0 && rows + na > target) {
      ca.push_back(a);
      rows = 0;
    }
    rows += na;
  }
  ca.push_back(T.nagg);
  TPart tp;
  tp.ncta = (int)ca.size() - 1;
  for (int a = 0; a < T.nagg; ++a) tp.ra_max = std::max(tp.ra_max, T.h_coarse_start[a + 1] - T.h_coarse_start[a]);
  for (int c = 0; c < tp.ncta; ++c) {
    int a0 = ca[c], a1 = ca[c + 1];
    tp.rows_max = std::max(tp.rows_max, T.h_row_start[a1] - T.h_row_start[a0]);
    tp.p_max = std::max(tp.p_max, (int)(T.h_blk_start[a1] - T.h_blk_start[a0]));
    tp.a_max = std::max(tp.a_max, a1 - a0);
    tp.c_max = std::max(tp.c_max, T.h_coarse_start[a1] - T.h_coarse_start[a0]);
  }
  tp.cta_agg = ar.alloc<int>(ca.size());
  AMG_CUDA(cudaMemcpy(tp.cta_agg, ca.data(), ca.size() * sizeof(int), cudaMemcpyHostToDevice));
  std::vector<int> cr(ca.size());
  for (size_t c = 0; c < ca.size(); ++c) cr[c] = T.h_row_start[ca[c]];
  tp.sg = make_stage(F.h_rowptr, cr, err);
  // the warp-per-aggregate restriction: NWARP aggregates per CTA
  std::vector<int> wr;
  for (int a = 0; a < T.nagg; a += NWARP) wr.push_back(T.h_row_start[a]);
  wr.push_back(T.h_row_start[T.nagg]);
  tp.wsg = make_group_stage(F.h_rowptr, wr);
  tp.wsg.enabled = tp.wsg.enabled && tp.sg.enabled;  // a level read unstaged stays unstaged
  return tp;
}

static int round_k(int nrhs) {
  int K = 1;
  while (K < nrhs) K <<= 1;
  return K;
}

// ------------------------------------------------------------ autotuner --
// Per level: the CTA size (non-zeros per CTA) and the lanes per row of the
// row-parallel kernels, chosen by timing the level's l1-Jacobi sweep with
// every candidate on the workspace's own buffers (their contents do not
// matter for timing).  The chosen layout serves every kernel of the level.
static const long long kTargets[] = {256, 512, 1024, 2048, 4096, 8192};

// AMG_COARSE_KERNELS in the environment overrides the tuner on grouped
// coarse levels: "grouped" takes the grouped sweep and restriction wherever
// the level allows them (the staged sweep with one CTA per 32 row groups,
// timing picking its lane split), "groupwarp" and "groupslot" fix the sweep
// to one warp or one slot of lanes per row group, "csr" never takes them;
// unset, timing decides among all.
static int coarse_kernel_override() {
  const char* e = std::getenv("AMG_COARSE_KERNELS");
  if (!e) return 0;
  if (std::strcmp(e, "grouped") == 0) return 1;
  if (std::strcmp(e, "groupwarp") == 0) return 2;
  if (std::strcmp(e, "groupslot") == 0) return 3;
  if (std::strcmp(e, "csr") == 0) return -1;
  return 0;
}

// AMG_TUNE_LOG=1 in the environment prints every candidate timing to stderr.
static bool tune_log() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("AMG_TUNE_LOG");
    on = (e && e[0] == '1') ? 1 : 0;
  }
  return on == 1;
}

template <typename TC>
static std::vector<int> nzl_candidates(int K) {
  std::vector<int> v;
  int mx = max_nzl<TC>(K);
  for (int n : {1, 2, 4, 8, 16, 32})
    if (n <= mx && (K > 1 ? n <= 8 : n >= 2)) v.push_back(n);
  return v;
}

// ------------------------------------------------- tuned choices, applied --
// Each tuner ends by applying its choice through these, and a choice read
// back from the tuning cache takes the same path.
static void ensure_gw(Plan& P, int k);
static void apply_level(Plan& P, Workspace& W, int k, long long target, int stage, int nzl) {
  std::vector<int> sys = (k == 0) ? P.h_sys_row : std::vector<int>{0, P.lev[k].n};
  W.rp[k] = make_rpart(W.ar, P.lev[k], target, sys, W.err);
  W.rp[k].sg.enabled = W.rp[k].sg.enabled && stage;
  if (nzl == NZL_GROUP_WARP || nzl == NZL_GROUP_SLOT) {
    ensure_gw(P, k);
    if (P.lev[k].gw_state != 1) nzl = 0;
  }
  W.nzl[k] = nzl;
  W.t_rp[k] = target;
  W.t_rps[k] = stage;
  W.t_nzl[k] = nzl;
}
static void ensure_rform(Plan& P, int k);
static int rform_override();
static void apply_transfer(Plan& P, Workspace& W, int k, int target, int stage, int warp) {
  if (target > 0) {
    W.tp[k] = make_tpart(W.ar, P.tr[k], P.lev[k], W.K, W.err, target);
    W.tp[k].sg.enabled = W.tp[k].sg.enabled && stage;
  }
  W.tp[k].warp = warp % 4;         // restriction kernel
  W.tp[k].pwarp = (warp / 4) % 2;  // prolongation kernel
  W.tp[k].jl = 1 << ((warp / 8) % 4);  // grouped restriction: lanes per group column split
  // restriction by R (one pre-sweep): replaces the restriction kernel above
  // in the V-cycle; the variant cycles keep the CSR restriction
  int rf = (warp / 32) % 4;  // 1: R by a warp per aggregate, 2: by a slot per aggregate
  const int rov = rform_override();
  if (rov < 0) rf = 0;
  if (rov > 0) rf = rov;
  if (rf && W.pre == 1) ensure_rform(P, k);
  if (P.tr[k].rf_state != 1 || W.pre != 1) rf = 0;
  if ((int)W.rform.size() < P.L - 1) W.rform.assign(std::max(P.L - 1, 0), 0);
  W.rform[k] = rf;
  warp = warp % 32 + 32 * rf;
  W.t_tp[k] = target;
  W.t_tps[k] = stage;
  W.t_tpw[k] = warp;
}
static KState view_state(Arena& ar, const KState& ks, const RPart& rp, int K);
static RPart make_flat(Arena& ar, int ncta);
static void ensure_packed(Plan& P);
static void apply_q(Plan& P, Workspace& W, long long target, int nzl, int stage, int grid) {
  W.nzl_q = nzl;
  W.q_pack = 0;
  // AMG_Q_PAIRED=1 takes the (hi, lo) pairs (and so an unstaged launch), =0
  // never; unset, the tuned or cached choice stands
  const char* qp = std::getenv("AMG_Q_PAIRED");
  if (W.split && qp && qp[0] == '1') stage = 2;
  if (qp && qp[0] == '0' && stage == 2) stage = 0;
  if (stage == 2) {  // (hi, lo) value pairs, unstaged
    ensure_packed(P);
    W.q_pack = P.lev[0].hl ? 1 : 0;
    if (!W.q_pack) stage = 0;
  }
  W.q_stage = stage == 2 ? 0 : stage;
  W.q_grid = grid;
  if (target > 0) {
    W.rq = make_rpart(W.ar, P.lev[0], target, P.h_sys_row, W.err);
    W.ksq = view_state(W.ar, W.ks, grid > 0 ? make_flat(W.ar, grid) : W.rq, W.K);
  }
  W.t_q = target;
  W.t_qn = nzl;
  W.t_qs = stage;
  W.t_qg = grid;
}
static void apply_persist(Workspace& W, int upd, int p, int post) {
  W.upd_grid = upd;
  W.p_grid = p;
  W.post_stage = post < 0 ? 1 : 0;  // a negative post grid: staged through the pipeline
  if (post < 0) post = -post;
  W.post_grid = post;
  if (upd > 0) W.ksf_upd = view_state(W.ar, W.ks, make_flat(W.ar, upd), W.K);
  if (post > 0) W.ksf_post = view_state(W.ar, W.ks, make_flat(W.ar, post), W.K);
  W.t_pu = upd;
  W.t_pp = p;
  W.t_ppost = W.post_stage ? -post : post;
}

// Streaming multiprocessors of the current device (persistent grids are
// multiples of it).
static int sm_count() {
  int dev = 0, n = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  AMG_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return n > 0 ? n : 1;
}

// Tuning cache: when the environment variable AMG_TUNE_CACHE names a file,
// a workspace whose problem shape (level sizes, systems, columns, precision,
// sweeps) has a line there takes its choices from that line instead of
// timing them, and newly tuned choices are appended to it.
static std::string tune_key(const Plan& P, int K, int prec, int pre, int post, bool split) {
  std::string k = "amg-tune-2 K" + std::to_string(K) + " prec" + std::to_string(prec) + " split" +
                  std::to_string(split ? 1 : 0) + " sweeps" + std::to_string(pre) + "/" + std::to_string(post) +
                  " nsys" + std::to_string(P.nsys) + " levels";
  for (int l = 0; l < P.L; ++l) k += " " + std::to_string(P.lev[l].n) + ":" + std::to_string(P.lev[l].nnz);
  return k;
}
static bool tune_cache_load(const std::string& key, std::vector<long long>& vals) {
  const char* path = std::getenv("AMG_TUNE_CACHE");
  if (!path || !*path) return false;
  FILE* fp = std::fopen(path, "r");
  if (!fp) return false;
  char line[8192];
  bool found = false;
  while (std::fgets(line, sizeof line, fp)) {
    std::string sl(line);
    size_t bar = sl.find(" | ");
    if (bar == std::string::npos || sl.compare(0, bar, key) != 0 || bar != key.size()) continue;
    vals.clear();
    const char* c = sl.c_str() + bar + 3;
    char* end = nullptr;
    for (long long v = std::strtoll(c, &end, 10); end != c; v = std::strtoll(c, &end, 10)) {
      vals.push_back(v);
      c = end;
    }
    found = true;  // the last matching line wins
  }
  std::fclose(fp);
  return found;
}
static void tune_cache_store(const std::string& key, const std::vector<long long>& vals) {
  const char* path = std::getenv("AMG_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* fp = std::fopen(path, "a");
  if (!fp) return;
  std::fprintf(fp, "%s |", key.c_str());
  for (long long v : vals) std::fprintf(fp, " %lld", v);
  std::fprintf(fp, "\n");
  std::fclose(fp);
}

template <typename TC>
static void tune_level(Plan& P, Workspace& W, int k, const std::vector<int>& sys) {
  const Level& L = P.lev[k];
  const int K = W.K;
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  long long bt = target_nnz(K);
  int bn = W.nzl[k], bs = 1;
  {
    Arena tmp;
    for (long long t : kTargets) {
      RPart rp0 = make_rpart(tmp, L, t, sys, W.err);
      if (t > kTargets[0] && rp0.ncta < sm_count()) break;  // fewer CTAs than SMs: stop growing
      for (int stage = rp0.sg.enabled; stage >= 0; --stage)
      for (int n : nzl_candidates<TC>(K)) {
        RPart rp = rp0;
        rp.sg.enabled = stage;
        TC* f = static_cast<TC*>(W.f[k]);
        TC* u = static_cast<TC*>(W.u[k]);
        TC* v = static_cast<TC*>(W.v[k]);
        launch_smooth<TC>(K, n, L, rp, f, u, v, W.zero_flag, 0);
        AMG_CUDA(cudaEventRecord(e0, 0));
        for (int r = 0; r < 3; ++r) launch_smooth<TC>(K, n, L, rp, f, u, v, W.zero_flag, 0);
        AMG_CUDA(cudaEventRecord(e1, 0));
        AMG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (tune_log())
          fprintf(stderr, "[tune] level %d K %d smooth target %lld nzl %d stage %d ncta %d: %.1f us\n", k, K, t, n,
                  stage, rp.ncta, ms * 1e3 / 3);
        if (ms < best) {
          best = ms;
          bt = t;
          bn = n;
          bs = stage;
        }
      }
    }
    AMG_CUDA(cudaDeviceSynchronize());
  }
  const int ovr = coarse_kernel_override();
  if (k > 0 && grouped_ok(K, L) && ovr >= 0) {  // the grouped sweep (lanes -jl, 0 for jl = 1, stand for it)
    TC* f = static_cast<TC*>(W.f[k]);
    TC* u = static_cast<TC*>(W.u[k]);
    TC* v = static_cast<TC*>(W.v[k]);
    float gbest = 1e30f;
    int gn = 0;
    for (int jl : {1, 2, 4}) {
      if (!grouped_jl_ok<TC>(K, jl)) continue;
      const int code = jl == 1 ? 0 : -jl;
      launch_smooth<TC>(K, code, L, W.rp[k], f, u, v, W.zero_flag, 0);
      AMG_CUDA(cudaEventRecord(e0, 0));
      for (int r = 0; r < 3; ++r) launch_smooth<TC>(K, code, L, W.rp[k], f, u, v, W.zero_flag, 0);
      AMG_CUDA(cudaEventRecord(e1, 0));
      AMG_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (tune_log()) fprintf(stderr, "[tune] level %d K %d smooth grouped jl %d: %.1f us\n", k, K, jl, ms * 1e3 / 3);
      if (ms < gbest) {
        gbest = ms;
        gn = code;
      }
    }
    // one warp per row group, or one slot of lanes per row group (not under
    // "grouped", which keeps the staged CTA-per-groups sweep)
    if (ovr != 1) ensure_gw(P, k);
    for (int code : {NZL_GROUP_WARP, NZL_GROUP_SLOT}) {
      if (ovr == 1 || P.lev[k].gw_state != 1) break;
      launch_smooth<TC>(K, code, L, W.rp[k], f, u, v, W.zero_flag, 0);
      AMG_CUDA(cudaEventRecord(e0, 0));
      for (int r = 0; r < 3; ++r) launch_smooth<TC>(K, code, L, W.rp[k], f, u, v, W.zero_flag, 0);
      AMG_CUDA(cudaEventRecord(e1, 0));
      AMG_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (tune_log())
        fprintf(stderr, "[tune] level %d K %d smooth grouped, %s per group: %.1f us\n", k, K,
                code == NZL_GROUP_WARP ? "warp" : "slot", ms * 1e3 / 3);
      const bool forced = (ovr == 2 && code == NZL_GROUP_WARP) || (ovr == 3 && code == NZL_GROUP_SLOT);
      if ((ms < gbest && ovr < 2) || forced) {
        gbest = ms;
        gn = code;
      }
    }
    if (gbest < best || ovr > 0) {
      best = gbest;
      bn = gn;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  apply_level(P, W, k, bt, bs, bn);
}

// Per transfer: rows per CTA and staging of the fused residual + restriction.
template <typename TC>
static void tune_transfer(Plan& P, Workspace& W, int k) {
  const int K = W.K;
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bt = 0, bs = 1;
  {
    Arena tmp;
    for (int t : {32, 64, 128, 256, 512}) {
      TPart tp0 = make_tpart(tmp, P.tr[k], P.lev[k], K, W.err, t);
      if (t > 32 && tp0.ncta < sm_count()) break;
      for (int stage = tp0.sg.enabled; stage >= 0; --stage) {
        TPart tp = tp0;
        tp.sg.enabled = stage;
        size_t smem = restrict_stage_bytes<TC>(tp.sg) +
                      transfer_smem<TC>(tp.rows_max, tp.p_max, tp.a_max, tp.c_max, K, true);
        if (smem > 200 * 1024) continue;
        auto run = [&] {
          launch_restrict<TC>(K, W.nzl[k], P.lev[k], P.tr[k], tp, P.lev[k + 1], k + 1 < P.L - 1,
                              static_cast<TC*>(W.f[k]), static_cast<TC*>(W.u[k]), static_cast<TC*>(W.f[k + 1]),
                              static_cast<TC*>(W.v[k + 1]), W.zero_flag, 0);
        };
        run();
        AMG_CUDA(cudaEventRecord(e0, 0));
        for (int r = 0; r < 3; ++r) run();
        AMG_CUDA(cudaEventRecord(e1, 0));
        AMG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (tune_log())
          fprintf(stderr, "[tune] level %d K %d restrict rows %d stage %d ncta %d: %.1f us\n", k, K, t, stage,
                  tp.ncta, ms * 1e3 / 3);
        if (ms < best) {
          best = ms;
          bt = t;
          bs = stage;
        }
      }
    }
    AMG_CUDA(cudaDeviceSynchronize());
  }
  // the warp-per-aggregate restriction (no CTA ranges): kind 1 reads the
  // matrix straight from global memory, kind 3 stages each CTA's slice first
  auto time_tp = [&](const TPart& tp, int reps) {
    auto run = [&] {
      launch_restrict<TC>(K, W.nzl[k], P.lev[k], P.tr[k], tp, P.lev[k + 1], k + 1 < P.L - 1,
                          static_cast<TC*>(W.f[k]), static_cast<TC*>(W.u[k]), static_cast<TC*>(W.f[k + 1]),
                          static_cast<TC*>(W.v[k + 1]), W.zero_flag, 0);
    };
    run();
    AMG_CUDA(cudaEventRecord(e0, 0));
    for (int r = 0; r < reps; ++r) run();
    AMG_CUDA(cudaEventRecord(e1, 0));
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms / reps;
  };
  int warp_kind = 0, wk_best = 0;
  float wbest = 1e30f;
  if (W.tp[k].ra_max <= 8) {
    for (int kind : {1, 3}) {
      TPart tw = W.tp[k];
      tw.warp = kind;
      if (kind == 3 && !tw.wsg.enabled) continue;
      const float ms = time_tp(tw, 3);
      if (tune_log())
        fprintf(stderr, "[tune] level %d K %d restrict warp-per-aggregate%s: %.1f us\n", k, K,
                kind == 3 ? " staged" : "", ms * 1e3);
      if (ms < wbest) {
        wbest = ms;
        wk_best = kind;
      }
    }
    if (wbest * 3 < best) {
      best = wbest * 3;
      warp_kind = wk_best;
    }
  }
  // a close race between the best CTA-range restriction and the best warp
  // restriction is decided by alternating re-timings (single timings of the
  // two differ from run to run by more than their gap)
  if (wk_best != 0 && bt > 0 && std::fabs(wbest * 3 - best) < 0.25f * best) {
    Arena tmp2;
    TPart tt = make_tpart(tmp2, P.tr[k], P.lev[k], K, W.err, bt);
    tt.sg.enabled = tt.sg.enabled && bs;
    TPart tw = W.tp[k];
    tw.warp = wk_best;
    float mt = 1e30f, mw = 1e30f;
    for (int round = 0; round < 3; ++round) {
      mt = std::min(mt, time_tp(tt, 5));
      mw = std::min(mw, time_tp(tw, 5));
    }
    if (tune_log())
      fprintf(stderr, "[tune] level %d K %d restrict runoff: ranges %.1f us, warp %.1f us\n", k, K, mt * 1e3,
              mw * 1e3);
    warp_kind = mw < mt ? wk_best : 0;
    best = 3 * std::min(mt, mw);
    AMG_CUDA(cudaDeviceSynchronize());
  }
  const bool warp_best = warp_kind != 0;
  // the grouped restriction (one CTA per aggregate) out of a grouped level
  bool grp_best = false;
  int gjl = 1;
  const int ovr = coarse_kernel_override();
  if (k > 0 && grouped_ok(K, P.lev[k]) && P.tr[k].gagg && W.tp[k].ra_max <= 8 && ovr >= 0) {
    float gbest = 1e30f;
    for (int jl : {1, 2, 4}) {
      if (!grouped_jl_ok<TC>(K, jl)) continue;
      TPart tg = W.tp[k];
      tg.warp = 2;
      tg.jl = jl;
      auto run = [&] {
        launch_restrict<TC>(K, W.nzl[k], P.lev[k], P.tr[k], tg, P.lev[k + 1], k + 1 < P.L - 1,
                            static_cast<TC*>(W.f[k]), static_cast<TC*>(W.u[k]), static_cast<TC*>(W.f[k + 1]),
                            static_cast<TC*>(W.v[k + 1]), W.zero_flag, 0);
      };
      run();
      AMG_CUDA(cudaEventRecord(e0, 0));
      for (int r = 0; r < 3; ++r) run();
      AMG_CUDA(cudaEventRecord(e1, 0));
      AMG_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (tune_log()) fprintf(stderr, "[tune] level %d K %d restrict grouped jl %d: %.1f us\n", k, K, jl, ms * 1e3 / 3);
      if (ms < gbest) {
        gbest = ms;
        gjl = jl;
      }
    }
    grp_best = gbest < best || ovr > 0;
  }
  // prolongation: CTA ranges of the chosen partition against one warp per aggregate
  int pw = 0;
  {
    Arena tmp;
    TPart tp = bt > 0 ? make_tpart(tmp, P.tr[k], P.lev[k], K, W.err, bt) : W.tp[k];
    float pbest = 1e30f;
    for (int w : {0, 1}) {
      if (w == 1 && tp.ra_max > 8) continue;  // the warp prolongation keeps at most 8 coarse values
      tp.pwarp = w;
      auto run = [&] {
        launch_prolong<TC>(K, P.tr[k], tp, static_cast<TC*>(W.v[k + 1]), static_cast<TC*>(W.u[k]), W.zero_flag, 0);
      };
      run();
      AMG_CUDA(cudaEventRecord(e0, 0));
      for (int r = 0; r < 3; ++r) run();
      AMG_CUDA(cudaEventRecord(e1, 0));
      AMG_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (tune_log()) fprintf(stderr, "[tune] level %d K %d prolong warp %d: %.1f us\n", k, K, w, ms * 1e3 / 3);
      if (ms < pbest) {
        pbest = ms;
        pw = w;
      }
    }
    AMG_CUDA(cudaDeviceSynchronize());
  }
  const int jsel = gjl == 4 ? 2 : (gjl == 2 ? 1 : 0);
  const int code = (grp_best ? 2 : (warp_best ? warp_kind : 0)) + 4 * pw + 8 * jsel;
  // restriction by R = P^T (I - A D^{-1}) (one pre-sweep): alternating
  // re-timings against the restriction chosen above
  int rf = 0;
  if (W.pre == 1 && rform_override() == 0) {
    ensure_rform(P, k);
    if (P.tr[k].rf_state == 1) {
      Arena tmp3;
      TPart tc = bt > 0 ? make_tpart(tmp3, P.tr[k], P.lev[k], K, W.err, bt) : W.tp[k];
      if (bt > 0) tc.sg.enabled = tc.sg.enabled && bs;
      tc.warp = code % 4;
      tc.pwarp = (code / 4) % 2;
      tc.jl = 1 << ((code / 8) % 4);
      const bool nxt = k + 1 < P.L - 1;
      auto time_rf = [&](int kind, int reps) {
        auto run_rf = [&] {
          launch_restrict_rf<TC>(K, P.tr[k], P.lev[k + 1], nxt, static_cast<TC*>(W.f[k]),
                                 static_cast<TC*>(W.f[k + 1]), static_cast<TC*>(W.v[k + 1]), W.zero_flag, 0,
                                 kind);
        };
        run_rf();
        AMG_CUDA(cudaEventRecord(e0, 0));
        for (int r = 0; r < reps; ++r) run_rf();
        AMG_CUDA(cudaEventRecord(e1, 0));
        AMG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return ms / reps;
      };
      float mc = 1e30f, mr = 1e30f, ms2 = 1e30f;
      for (int round = 0; round < 3; ++round) {
        mc = std::min(mc, time_tp(tc, 5));
        mr = std::min(mr, time_rf(1, 5));
        ms2 = std::min(ms2, time_rf(2, 5));
      }
      if (tune_log())
        fprintf(stderr, "[tune] level %d K %d restrict by R: warp %.1f us, slot %.1f us, against %.1f us\n", k, K,
                mr * 1e3, ms2 * 1e3, mc * 1e3);
      if (std::min(mr, ms2) < mc) rf = ms2 < mr ? 2 : 1;
      AMG_CUDA(cudaDeviceSynchronize());
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  apply_transfer(P, W, k, bt, bs, code + 32 * rf);
}

static void launch_cg_q(Workspace& W, const Level& L, cudaStream_t st);

// The CG state seen through another level-0 partition: same scalars and
// counters, the partition's CTA groups and its own partial sums.
static KState view_state(Arena& ar, const KState& ks, const RPart& rp, int K) {
  KState v = ks;
  v.partial = ar.alloc<double>((size_t)rp.ncta * K);
  v.gpartial = ar.alloc<double>((size_t)rp.ngroups * K);
  v.gcount = ar.alloc<unsigned>((size_t)RED_KINDS * rp.ngroups);
  AMG_CUDA(cudaMemset(v.gcount, 0, (size_t)RED_KINDS * rp.ngroups * sizeof(unsigned)));
  v.grp_cta = rp.grp_cta;
  v.sys_grp = rp.sys_grp;
  v.ngroups = rp.ngroups;
  v.sys_cta = rp.sys_cta;
  v.sg = rp.sg;
  return v;
}

// Level-0 q = A p: lanes per row, and for the double-float kernel also the
// CTA size and staging, chosen by timing the kernel itself (the CG state is
// reset by the start of every solve, so timing runs are harmless).
static void tune_q(Plan& P, Workspace& W) {
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bn = W.nzl_q, bs = W.q_stage;
  long long bt = -1;
  std::vector<int> cand = W.split ? nzl_candidates<float>(W.K) : nzl_candidates<double>(W.K);
  auto time_q = [&](const char* what, long long t, int n, int stage) {
    launch_cg_q(W, P.lev[0], 0);
    AMG_CUDA(cudaEventRecord(e0, 0));
    for (int r = 0; r < 3; ++r) launch_cg_q(W, P.lev[0], 0);
    AMG_CUDA(cudaEventRecord(e1, 0));
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (tune_log())
      fprintf(stderr, "[tune] q %s K %d target %lld nzl %d stage %d ncta %d: %.1f us\n", what, W.K, t, n, stage,
              W.split ? W.rq.ncta : W.rp[0].ncta, ms * 1e3 / 3);
    return ms;
  };
  if (!W.split) {
    for (int n : cand) {
      W.nzl_q = n;
      float ms = time_q("f64", 0, n, 0);
      if (ms < best) {
        best = ms;
        bn = n;
      }
    }
    apply_q(P, W, 0, bn, 0, 0);
  } else {
    static const long long qTargets[] = {1024, 2048, 4096, 8192, 16384};
    Arena tmp;
    const RPart keep = W.rq;
    const KState keep_ks = W.ksq;
    for (long long t : qTargets) {
      RPart rp = make_rpart(tmp, P.lev[0], t, P.h_sys_row, W.err);
      if (t > qTargets[0] && rp.ncta < 3 * sm_count()) break;  // under one wave of three CTAs per SM
      W.rq = rp;
      W.ksq = view_state(tmp, W.ks, rp, W.K);
      for (int stage = rp.sg.enabled; stage >= 0; --stage)
        for (int n : cand) {
          W.nzl_q = n;
          W.q_stage = stage;
          float ms = time_q("df", t, n, stage);
          if (ms < best) {
            best = ms;
            bn = n;
            bs = stage;
            bt = t;
          }
        }
      AMG_CUDA(cudaDeviceSynchronize());
    }
    // persistent launches (one system): 2 to 4 CTAs per SM walk the chunks,
    // unstaged or through the double-buffered staging pipeline
    int bg = 0;
    if (P.nsys == 1) {
      for (int per_sm : {4, 3, 2}) {
        const int grid = per_sm * sm_count();
        RPart flat = make_flat(tmp, grid);
        for (long long t : qTargets) {
          RPart rp = make_rpart(tmp, P.lev[0], t, P.h_sys_row, W.err);
          if (rp.ncta < 2 * grid) break;
          W.rq = rp;
          W.q_grid = grid;
          W.ksq = view_state(tmp, W.ks, flat, W.K);
          for (int stage = rp.sg.enabled; stage >= 0; --stage)
            for (int n : cand) {
              W.nzl_q = n;
              W.q_stage = stage;
              float ms = time_q("df persistent", t, n, stage);
              if (ms < best) {
                best = ms;
                bn = n;
                bs = stage;
                bt = t;
                bg = grid;
              }
            }
          AMG_CUDA(cudaDeviceSynchronize());
        }
      }
    }
    W.rq = keep;
    W.ksq = keep_ks;
    apply_q(P, W, bt, bn, bs, bg);
    // (AMG_Q_PAIRED, when set, has decided in apply_q)
    const char* qp = std::getenv("AMG_Q_PAIRED");
    if (bs == 0 && !(qp && *qp)) {
      // the chosen unstaged launch against the same launch reading the
      // values as (hi, lo) pairs, in alternating rounds
      ensure_packed(P);
      if (P.lev[0].hl) {
        float mu = 1e30f, mp = 1e30f;
        for (int round = 0; round < 3; ++round) {
          W.q_pack = 0;
          mu = std::min(mu, time_q("df chosen", bt, bn, 0));
          W.q_pack = 1;
          mp = std::min(mp, time_q("df packed", bt, bn, 2));
        }
        W.q_pack = 0;
        AMG_CUDA(cudaDeviceSynchronize());
        if (mp < mu) apply_q(P, W, bt, bn, 2, bg);
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

static void launch_update_df(Workspace& W, const Level& L, cudaStream_t st);
static void launch_cg_p(const Plan& P, Workspace& W, const Level& L, int first, cudaStream_t st);

// Level-0 kernels of the double-float CG (one system): each runs either one
// CTA per row range or persistent (2 to 8 CTAs per SM walking the ranges,
// one reduction per CTA), whichever the timing favours; each kernel gets its
// own grid.  The timing runs use a private all-stopped flag, cleared before
// every launch, so that the stopping test of a reducing kernel cannot turn
// the following launches into no-ops.
static void tune_persist(Plan& P, Workspace& W) {
  const int K = W.K, nsm = sm_count();
  int* tdone = W.ar.alloc<int>(1);
  int* keep_done = W.ks.done;
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  auto timeit = [&](const char* what, int grid, auto launch) {
    AMG_CUDA(cudaMemsetAsync(tdone, 0, sizeof(int), 0));
    launch();
    AMG_CUDA(cudaEventRecord(e0, 0));
    for (int r = 0; r < 3; ++r) {
      AMG_CUDA(cudaMemsetAsync(tdone, 0, sizeof(int), 0));
      launch();
    }
    AMG_CUDA(cudaEventRecord(e1, 0));
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (tune_log()) fprintf(stderr, "[tune] %s K %d persistent grid %d: %.1f us\n", what, K, grid, ms * 1e3 / 3);
    return ms;
  };
  // grid 0 (one CTA per range) against persistent grids of per_sm CTAs per
  // SM; ``view`` receives the CG state seen through the grid's CTA groups
  // (made before the timed launches)
  Arena tmp;
  KState view{};
  auto pick = [&](const char* what, int& grid, bool reduces, auto launch) {
    auto prepare = [&](int g) {
      view = (g > 0 && reduces) ? view_state(tmp, W.ks, make_flat(tmp, g), K) : W.ks;
      view.done = tdone;
      AMG_CUDA(cudaDeviceSynchronize());
    };
    grid = 0;
    prepare(0);
    float best = timeit(what, 0, launch);
    int bg = 0;
    for (int per_sm : {2, 3, 4, 6, 8}) {
      grid = per_sm * nsm;
      if (grid * 2 > W.rp[0].ncta) break;
      prepare(grid);
      float ms = timeit(what, grid, launch);
      if (ms < best) {
        best = ms;
        bg = grid;
      }
    }
    grid = bg;
  };
  pick("update", W.upd_grid, true, [&] {
    W.ksf_upd = view;
    KState keep = W.ks;
    W.ks.done = tdone;
    launch_update_df(W, P.lev[0], 0);
    W.ks = keep;
  });
  pick("p", W.p_grid, false, [&] {
    KState keep = W.ks;
    W.ks.done = tdone;
    launch_cg_p(P, W, P.lev[0], 0, 0);
    W.ks = keep;
  });
  // post-smoother: persistent grids unstaged (code grid) and staged (code -grid)
  int post_code = 0;
  {
    float pbest = 1e30f;
    std::vector<int> codes{0};
    for (int per_sm : {2, 3, 4, 6, 8}) {
      const int g = per_sm * nsm;
      if (g * 2 > W.rp[0].ncta) break;
      codes.push_back(g);
      if (W.rp[0].sg.enabled) codes.push_back(-g);
    }
    for (int code : codes) {
      const int g = code < 0 ? -code : code;
      view = g > 0 ? view_state(tmp, W.ks, make_flat(tmp, g), K) : W.ks;
      view.done = tdone;
      AMG_CUDA(cudaDeviceSynchronize());
      RPart rp0 = W.rp[0];
      if (code > 0) rp0.sg.enabled = 0;
      float ms = timeit("post", code, [&] {
        launch_post0<float>(K, W.nzl[0], P.lev[0], rp0, static_cast<float*>(W.f[0]), static_cast<float*>(W.u[0]),
                            W.r, W.rl, reinterpret_cast<float*>(W.z), view, 1, 0, g);
      });
      if (ms < pbest) {
        pbest = ms;
        post_code = code;
      }
    }
  }
  W.post_grid = post_code < 0 ? -post_code : post_code;
  W.post_stage = post_code < 0 ? 1 : 0;
  AMG_CUDA(cudaDeviceSynchronize());
  W.ks.done = keep_done;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  apply_persist(W, W.upd_grid, W.p_grid, W.post_stage ? -W.post_grid : W.post_grid);
}

// Row groups of the coarse levels (see the grouped kernels): the host
// checks that the rows of each aggregate's coarse dofs have equal lengths and
// consecutive storage, a kernel checks that they have the same columns, and
// each transfer out of a grouped level gets the first group of every
// aggregate.  Levels that fail a check keep the CSR kernels only.
__global__ void k_check_groups(int ngrp, const int* __restrict__ gstart, const int* __restrict__ rowptr,
                               const int* __restrict__ col, int* __restrict__ bad) {
  const int g = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (g >= ngrp) return;
  const int r0 = gstart[g], r1 = gstart[g + 1];
  const int b0 = rowptr[r0], S = rowptr[r0 + 1] - b0;
  for (int r = r0 + 1; r < r1; ++r) {
    const int br = rowptr[r];
    for (int j = lane; j < S; j += 32)
      if (col[br + j] != col[b0 + j]) atomicOr(bad, 1);
  }
}

static void ensure_groups(Plan& P) {
  if (P.groups_done) return;
  P.groups_done = true;
  int* bad = P.arena->alloc<int>(1);
  for (int k = 1; k < P.L; ++k) {
    Level& L = P.lev[k];
    const Transfer& T = P.tr[k - 1];
    const std::vector<int>& gs = T.h_coarse_start;
    if ((int)gs.size() != T.nagg + 1 || gs.back() != L.n || (int)L.h_rowptr.size() != L.n + 1) continue;
    bool ok = true;
    int rmax = 0;
    for (int g = 0; g < T.nagg && ok; ++g) {
      const int r0 = gs[g], r1 = gs[g + 1];
      if (r1 <= r0) {
        ok = false;
        break;
      }
      rmax = std::max(rmax, r1 - r0);
      const long long S = (long long)L.h_rowptr[r0 + 1] - L.h_rowptr[r0];
      for (int r = r0 + 1; r < r1 && ok; ++r)
        if ((long long)L.h_rowptr[r + 1] - L.h_rowptr[r] != S) ok = false;
    }
    if (!ok) continue;
    AMG_CUDA(cudaMemset(bad, 0, sizeof(int)));
    k_check_groups<<<(T.nagg + 7) / 8, 256>>>(T.nagg, T.coarse_start, L.rowptr, L.col, bad);
    AMG_LAUNCH_CHECK();
    int hbad = 0;
    AMG_CUDA(cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost));
    if (hbad) continue;
    L.grp_ok = 1;
    L.ngrp = T.nagg;
    L.grp_rmax = rmax;
    L.gstart = T.coarse_start;
    // staging capacities of the grouped sweep's CTAs
    std::vector<int> cr;
    for (int g = 0; g < T.nagg; g += GROUPS_PER_CTA) cr.push_back(gs[g]);
    cr.push_back(gs[T.nagg]);
    L.gsg = make_group_stage(L.h_rowptr, cr);
  }
  for (int k = 1; k + 1 < P.L; ++k) {
    if (!P.lev[k].grp_ok) continue;
    const std::vector<int>& gs = P.tr[k - 1].h_coarse_start;
    const std::vector<int>& rs = P.tr[k].h_row_start;
    std::vector<int> ga(rs.size());
    size_t g = 0;
    bool ok = true;
    for (size_t a = 0; a < rs.size() && ok; ++a) {
      while (g < gs.size() && gs[g] < rs[a]) ++g;
      if (g == gs.size() || gs[g] != rs[a]) ok = false;
      else ga[a] = (int)g;
    }
    if (!ok) continue;
    int* d = P.arena->alloc<int>(ga.size());
    AMG_CUDA(cudaMemcpy(d, ga.data(), ga.size() * sizeof(int), cudaMemcpyHostToDevice));
    P.tr[k].gagg = d;
    P.tr[k].gsg = make_group_stage(P.lev[k].h_rowptr, rs);  // one CTA per aggregate
  }
}

// Level 0's column-scaled float copy A D^{-1} (fl32(a_ij / d_j)), made once
// per plan for the u0-free float32 cycle; 16 padding elements like the
// other non-zero arrays (the staging copies may read past a row range).
__global__ void k_scale_cols(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ dinv, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) out[j] = (float)(val[j] * dinv[col[j]]);
}

static void ensure_scaled(Plan& P) {
  Level& L = P.lev[0];
  if (L.val_sc || !L.dinv64) return;
  L.val_sc = P.arena->alloc<float>((size_t)L.nnz + 16);
  AMG_CUDA(cudaMemset(L.val_sc + L.nnz, 0, 16 * sizeof(float)));
  k_scale_cols<<<(L.n + 255) / 256, 256>>>(L.n, L.rowptr, L.col, L.val64, L.dinv64, L.val_sc);
  AMG_LAUNCH_CHECK();
  AMG_CUDA(cudaDeviceSynchronize());
}

// R = P^T (I - A D^{-1}) of transfer k (the restriction after one pre-sweep
// from zero), built once per plan on the host from the float64 level and
// prolongator: for aggregate a with rows I_a and coarse dofs c,
//   R[c, h] = P[h, c] [h in I_a] - sum_{i in I_a} P[i, c] a_ih / d_h,
// h over the sorted halo of a (I_a and every column of its rows), the P term
// first and then the rows of A in order.  float64 and float32 copies, RS = 4
// or 8 values per pattern entry; 16 zero entries of padding.
static void ensure_rform(Plan& P, int k) {
  Transfer& T = P.tr[k];
  if (T.rf_state != 0) return;
  T.rf_state = -1;
  AMG_CUDA(cudaDeviceSynchronize());  // the plan's arrays may still be in flight on the setup stream
  const Level& L = P.lev[k];
  if (k + 1 >= P.L || !L.dinv64 || !L.val64 || !T.p64 || T.nagg <= 0) return;
  if ((int)L.h_rowptr.size() != L.n + 1 || (int)T.h_row_start.size() != T.nagg + 1 ||
      (int)T.h_coarse_start.size() != T.nagg + 1 || (int)T.h_blk_start.size() != T.nagg + 1)
    return;
  const std::vector<int>& rs = T.h_row_start;
  const std::vector<int>& cs = T.h_coarse_start;
  int ramax = 0;
  for (int a = 0; a < T.nagg; ++a) ramax = std::max(ramax, cs[a + 1] - cs[a]);
  if (ramax < 1 || ramax > 8) return;
  const int RS = ramax <= 4 ? 4 : 8;
  std::vector<int> col(L.nnz);
  std::vector<double> val(L.nnz), dinv(L.n), pv(T.npval);
  AMG_CUDA(cudaMemcpy(col.data(), L.col, col.size() * sizeof(int), cudaMemcpyDeviceToHost));
  AMG_CUDA(cudaMemcpy(val.data(), L.val64, val.size() * sizeof(double), cudaMemcpyDeviceToHost));
  AMG_CUDA(cudaMemcpy(dinv.data(), L.dinv64, dinv.size() * sizeof(double), cudaMemcpyDeviceToHost));
  AMG_CUDA(cudaMemcpy(pv.data(), T.p64, pv.size() * sizeof(double), cudaMemcpyDeviceToHost));
  std::vector<int> ptr(T.nagg + 1, 0), pcol, halo;
  std::vector<double> pval;
  pcol.reserve((size_t)L.nnz / 2 + 16);
  pval.reserve(pcol.capacity() * RS);
  for (int a = 0; a < T.nagg; ++a) {
    const int r0 = rs[a], r1 = rs[a + 1], ra = cs[a + 1] - cs[a];
    if (r0 < 0 || r1 > L.n || r1 < r0) return;
    const double* Pa = pv.data() + T.h_blk_start[a];
    halo.clear();
    for (int i = r0; i < r1; ++i) {
      halo.push_back(i);
      for (int j = L.h_rowptr[i]; j < L.h_rowptr[i + 1]; ++j) {
        if (col[j] < 0 || col[j] >= L.n) return;
        halo.push_back(col[j]);
      }
    }
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    const size_t base = pcol.size();
    if (base + halo.size() + RF_PAD >= (size_t)INT32_MAX - 64) return;
    pcol.insert(pcol.end(), halo.begin(), halo.end());
    // padded to a multiple of RF_PAD entries: a valid column, zero values
    while ((pcol.size() - base) % RF_PAD) pcol.push_back(halo[0]);
    pval.resize(pcol.size() * RS, 0.0);
    double* V = pval.data() + base * RS;
    auto pos = [&](int h) { return (size_t)(std::lower_bound(halo.begin(), halo.end(), h) - halo.begin()); };
    for (int i = r0; i < r1; ++i) {
      const size_t hi = pos(i);
      for (int p = 0; p < ra; ++p) V[hi * RS + p] += Pa[(size_t)(i - r0) * ra + p];
    }
    for (int i = r0; i < r1; ++i)
      for (int j = L.h_rowptr[i]; j < L.h_rowptr[i + 1]; ++j) {
        const size_t h = pos(col[j]);
        const double w = val[j] * dinv[col[j]];
        for (int p = 0; p < ra; ++p) V[h * RS + p] -= Pa[(size_t)(i - r0) * ra + p] * w;
      }
    ptr[a + 1] = (int)pcol.size();
  }
  const size_t ne = pcol.size();  // a multiple of RF_PAD; the zero batch follows
  pcol.resize(ne + 16, 0);
  pval.resize((ne + 16) * RS, 0.0);
  std::vector<float> pv32(pval.size());
  for (size_t e = 0; e < pval.size(); ++e) pv32[e] = (float)pval[e];
  T.rf_ptr = P.arena->alloc<int>(ptr.size());
  T.rf_col = P.arena->alloc<int>(pcol.size());
  T.rf_v64 = P.arena->alloc<double>(pval.size());
  T.rf_v32 = P.arena->alloc<float>(pv32.size());
  AMG_CUDA(cudaMemcpy(T.rf_ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  AMG_CUDA(cudaMemcpy(T.rf_col, pcol.data(), pcol.size() * sizeof(int), cudaMemcpyHostToDevice));
  AMG_CUDA(cudaMemcpy(T.rf_v64, pval.data(), pval.size() * sizeof(double), cudaMemcpyHostToDevice));
  AMG_CUDA(cudaMemcpy(T.rf_v32, pv32.data(), pv32.size() * sizeof(float), cudaMemcpyHostToDevice));
  T.rf_rs = RS;
  T.rf_entries = (long long)ne;
  T.rf_zero = (int)ne;
  T.rf_state = 1;
}

// Entry-major copy of grouped level k for the warp-per-group sweep: one warp
// per row group copies the group's pattern (its first row's columns) and,
// per entry, the values of its rows, padded with zeros to rs.
__global__ void k_build_gw(int ngrp, const int* __restrict__ gstart, const int* __restrict__ rowptr,
                           const int* __restrict__ col, const double* __restrict__ val, const int* __restrict__ gptr,
                           int rs, int* __restrict__ gcol, double* __restrict__ g64, float* __restrict__ g32) {
  const int g = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (g >= ngrp) return;
  const int r0 = gstart[g], ra = gstart[g + 1] - r0, b = rowptr[r0], S = rowptr[r0 + 1] - b, e = gptr[g];
  const int Sp = gptr[g + 1] - e;  // padded: a valid column with zero values
  for (int jj = lane; jj < Sp; jj += 32) {
    gcol[e + jj] = col[b + (jj < S ? jj : 0)];
    for (int p = 0; p < rs; ++p) {
      const double v = (p < ra && jj < S) ? val[rowptr[r0 + p] + jj] : 0.0;
      g64[(size_t)(e + jj) * rs + p] = v;
      g32[(size_t)(e + jj) * rs + p] = (float)v;
    }
  }
}

static void ensure_gw(Plan& P, int k) {
  Level& L = P.lev[k];
  if (L.gw_state != 0) return;
  L.gw_state = -1;
  if (k < 1 || !L.grp_ok || L.grp_rmax < 1 || L.grp_rmax > 8 || !L.val64) return;
  const std::vector<int>& gs = P.tr[k - 1].h_coarse_start;
  if ((int)gs.size() != L.ngrp + 1 || (int)L.h_rowptr.size() != L.n + 1) return;
  std::vector<int> ptr(L.ngrp + 1, 0);
  for (int g = 0; g < L.ngrp; ++g) {
    const long long S = (long long)L.h_rowptr[gs[g] + 1] - L.h_rowptr[gs[g]];
    const long long Sp = (S + RF_PAD - 1) / RF_PAD * RF_PAD;  // padded pattern
    if (S < 1 || (long long)ptr[g] + Sp >= (long long)INT32_MAX - 64) return;
    ptr[g + 1] = ptr[g] + (int)Sp;
  }
  const int rs = L.grp_rmax <= 4 ? 4 : 8;
  const size_t ne = (size_t)ptr[L.ngrp] + 16;
  L.gw_ptr = P.arena->alloc<int>(ptr.size());
  L.gw_col = P.arena->alloc<int>(ne);
  L.gw_v64 = P.arena->alloc<double>(ne * rs);
  L.gw_v32 = P.arena->alloc<float>(ne * rs);
  AMG_CUDA(cudaDeviceSynchronize());
  AMG_CUDA(cudaMemcpy(L.gw_ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  AMG_CUDA(cudaMemset(L.gw_col, 0, ne * sizeof(int)));
  AMG_CUDA(cudaMemset(L.gw_v64, 0, ne * rs * sizeof(double)));
  AMG_CUDA(cudaMemset(L.gw_v32, 0, ne * rs * sizeof(float)));
  k_build_gw<<<(L.ngrp + 7) / 8, 256>>>(L.ngrp, L.gstart, L.rowptr, L.col, L.val64, L.gw_ptr, rs, L.gw_col,
                                        L.gw_v64, L.gw_v32);
  AMG_LAUNCH_CHECK();
  AMG_CUDA(cudaDeviceSynchronize());
  L.gw_rs = rs;
  L.gw_zero = ptr[L.ngrp];
  L.gw_state = 1;
}

// AMG_RESTRICT_RFORM in the environment overrides the tuner's choice of the
// restriction by R = P^T (I - A D^{-1}) (one pre-sweep only): "1" takes it on
// every transfer that has it with a warp per aggregate, "2" with a slot of
// lanes per aggregate, "0" never; unset, timing decides.
static int rform_override() {
  const char* e = std::getenv("AMG_RESTRICT_RFORM");
  if (!e || !*e) return 0;
  return e[0] == '1' ? 1 : (e[0] == '2' ? 2 : (e[0] == '0' ? -1 : 0));
}

// Level 0's values as (val32, vallo) pairs for the double-float q = A p
// (one 8-byte load per non-zero), 16 zero pairs of padding; made once per
// plan on first use.
__global__ void k_pack_q(long long nnz, const float* __restrict__ hi, const float* __restrict__ lo,
                         float2* __restrict__ hl) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nnz + 16) return;
  hl[j] = j < nnz ? make_float2(hi[j], lo[j]) : make_float2(0.f, 0.f);
}

static void ensure_packed(Plan& P) {
  Level& L = P.lev[0];
  if (L.hl || !L.val32 || !L.vallo || L.nnz <= 0) return;
  AMG_CUDA(cudaDeviceSynchronize());
  float2* hl = P.arena->alloc<float2>((size_t)L.nnz + 16);
  k_pack_q<<<(unsigned)((L.nnz + 16 + 255) / 256), 256>>>(L.nnz, L.val32, L.vallo, hl);
  AMG_LAUNCH_CHECK();
  AMG_CUDA(cudaDeviceSynchronize());
  L.hl = hl;
}

static void make_var(Plan& P, Workspace& W, int variant);

// Test hook: AMG_TEST_FIRST_WAIT=n (1..15) limits the first wait for every
// staged copy of this workspace (and of its plan's grouped levels) to n
// non-blocking polls, so that a test sees the bounded wait give up and the
// solve report AMG_ERR_TIMEOUT; the drain wait keeps its full bound.
static void apply_wait_hook(Plan& P, Workspace& W) {
  const char* e = std::getenv("AMG_TEST_FIRST_WAIT");
  const int n = e ? std::atoi(e) : 0;
  if (n < 1 || n > 15) return;
  auto set = [n](Stage& sg) { sg.first_wait = n; };
  for (auto& r : W.rp) set(r.sg);
  for (auto& t : W.tp) {
    set(t.sg);
    set(t.wsg);
  }
  set(W.rq.sg);
  for (KState* k : {&W.ks, &W.ksq, &W.ksf_upd, &W.ksf_post}) set(k->sg);
  for (auto& l : P.lev) set(l.gsg);
  for (auto& t : P.tr) set(t.gsg);
}

// Start level of the fused small-level cycle (W.cc_s, -1: off).  Eligible
// starts: levels 1 <= s <= L-2 with at most 2^21 (row, column) items, if the
// cooperative launch fits one CTA per SM.  Tuned workspaces time one
// graph-captured V-cycle with the fused cycle off and from each eligible
// start and keep the fastest (the choice joins the tuning cache); others
// take the first eligible level with at most 2^19 items.
// AMG_FUSED_COARSE=0 keeps the launch-per-step cycle, =1 forces the first
// eligible start; AMG_TEST_BARRIER_HANG=1 is the barrier test hook.
template <typename TC, int K>
static bool cc_fits() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_coarse_cycle<TC, K>, CC_BS, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nb >= 1;
}
static float time_vcycle_graph(Plan& P, Workspace& W);
static void setup_fused_coarse(Plan& P, Workspace& W, bool autotune, int cached_s) {
  W.cc_s = -1;
  const char* e = std::getenv("AMG_FUSED_COARSE");
  if ((e && e[0] == '0') || P.L < 3 || P.L > CC_MAXL || W.variant) return;
  std::vector<int> starts;
  for (int k = 1; k + 1 < P.L; ++k)
    if ((double)P.lev[k].n * W.K <= (double)(1 << 21)) starts.push_back(k);
  if (starts.empty()) return;
  bool fits = false;
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    fits = (W.prec == 64 && !W.split) ? cc_fits<double, KK>() : cc_fits<float, KK>();
  });
  if (!fits) return;
  W.cc_grid = sm_count();
  W.cc_bar = W.ar.alloc<unsigned>(2);
  AMG_CUDA(cudaMemset(W.cc_bar, 0, 2 * sizeof(unsigned)));
  const char* h = std::getenv("AMG_TEST_BARRIER_HANG");
  W.cc_hang = h && h[0] == '1';
  if ((e && e[0] == '1') || W.cc_hang) {
    W.cc_s = starts[0];
  } else if (cached_s >= -1) {
    W.cc_s = std::find(starts.begin(), starts.end(), cached_s) != starts.end() ? cached_s : -1;
  } else if (autotune) {
    W.cc_s = -1;
    float best = time_vcycle_graph(P, W);
    if (tune_log()) fprintf(stderr, "[tune] V-cycle, launch per step: %.1f us\n", best * 1e3);
    int bs = -1;
    for (int s : starts) {
      W.cc_s = s;
      const float ms = time_vcycle_graph(P, W);
      if (tune_log()) fprintf(stderr, "[tune] V-cycle, fused small levels from %d: %.1f us\n", s, ms * 1e3);
      if (ms < best) {
        best = ms;
        bs = s;
      }
    }
    W.cc_s = bs;
  } else {
    for (int s : starts)
      if ((double)P.lev[s].n * W.K <= (double)(1 << 19)) {
        W.cc_s = s;
        break;
      }
  }
}

static Workspace& get_ws(Plan& P, int K, int prec, int pre, int post, bool split = false, bool autotune = false,
                         int variant = 0) {
  long long key = ((long long)variant << 44) | ((long long)split << 40) | ((long long)K << 32) |
                  ((long long)prec << 16) | ((long long)pre << 8) | post;
  auto it = P.ws.find(key);
  if (it != P.ws.end()) return *it->second;
  ensure_groups(P);
  auto W = std::make_shared<Workspace>();
  W->K = K;
  W->prec = prec;
  W->pre = pre;
  W->post = post;
  W->n0 = P.lev[0].n;
  W->L = P.L;
  Arena& ar = W->ar;
  size_t n0k = (size_t)W->n0 * K;
  AMG_REQUIRE(!split || n0k < (size_t(1) << 32), "n * nrhs must be below 2^32 for the float32-cycle solve");
  W->x = ar.alloc<double>(n0k);
  W->r = ar.alloc<double>(n0k);
  W->split = split;
  W->u0free = split && pre == 1 && P.L > 1;
  if (W->u0free) ensure_scaled(P);
  if (split) {
    for (float** v : {&W->xh, &W->xl, &W->rh, &W->rl, &W->ph, &W->ph2, &W->qh, &W->ql}) *v = ar.alloc<float>(n0k);
    // both direction buffers hold finite values from the start (a pending
    // step by zero may read either)
    AMG_CUDA(cudaMemset(W->ph, 0, n0k * sizeof(float)));
    AMG_CUDA(cudaMemset(W->ph2, 0, n0k * sizeof(float)));
  } else {
    W->p = ar.alloc<double>(n0k);
  }
  W->q = ar.alloc<double>(n0k);
  W->z = ar.alloc<double>(n0k);
  W->b = ar.alloc<double>(n0k);
  size_t es = prec == 64 ? 8 : 4;
  W->f.resize(P.L);
  W->u.resize(P.L);
  W->v.resize(P.L);
  for (int k = 0; k < P.L; ++k) {
    size_t nk = (size_t)P.lev[k].n * K;
    if (k == 0 && prec == 64) W->f[k] = W->r;
    else if (k == 0 && split) W->f[k] = W->rh;   // r_hi is the float32 level-0 right-hand side
    else W->f[k] = ar.raw(nk * es);
    W->u[k] = ar.raw(nk * es);
    W->v[k] = ar.raw(nk * es);
  }
  W->err = ar.alloc<int>(1);
  AMG_CUDA(cudaMemset(W->err, 0, sizeof(int)));
  W->zero_flag = ar.alloc<int>(1);
  AMG_CUDA(cudaMemset(W->zero_flag, 0, sizeof(int)));
  W->nzl.resize(P.L);
  for (int k = 0; k < P.L; ++k) {
    std::vector<int> sys = (k == 0) ? P.h_sys_row : std::vector<int>{0, P.lev[k].n};
    W->rp.push_back(make_rpart(ar, P.lev[k], target_nnz(K), sys, W->err));
    W->nzl[k] = prec == 64 ? pick_nzl<double>(P.lev[k], K) : pick_nzl<float>(P.lev[k], K);
  }
  W->nzl_q = split ? pick_nzl<float>(P.lev[0], K) : pick_nzl<double>(P.lev[0], K);
  const int nt = std::max(P.L - 1, 0);
  W->t_rp.assign(P.L, 0);
  W->t_rps.assign(P.L, 0);
  W->t_nzl.assign(P.L, 0);
  W->t_tp.assign(nt, 0);
  W->t_tps.assign(nt, 0);
  W->t_tpw.assign(nt, 0);
  // cached choices: per smoothed level 3, per transfer 3, q 4, persistent 4
  const std::string tkey = tune_key(P, K, prec, pre, post, split);
  std::vector<long long> tv;
  const bool cached = autotune && tune_cache_load(tkey, tv) && tv.size() == (size_t)(6 * nt + 9);
  if (cached) {
    for (int k = 0; k < nt; ++k) apply_level(P, *W, k, tv[3 * k], (int)tv[3 * k + 1], (int)tv[3 * k + 2]);
  } else if (autotune) {
    for (int k = 0; k + 1 < P.L; ++k) {  // smoothed levels (the coarsest has no smoother)
      std::vector<int> sys = (k == 0) ? P.h_sys_row : std::vector<int>{0, P.lev[k].n};
      if (prec == 64) tune_level<double>(P, *W, k, sys);
      else tune_level<float>(P, *W, k, sys);
    }
  }
  const RPart& r0p = W->rp[0];
  int nv = P.nsys * K;
  KState& ks = W->ks;
  ks.partial = ar.alloc<double>((size_t)r0p.ncta * 2 * K);
  ks.gpartial = ar.alloc<double>((size_t)r0p.ngroups * 2 * K);
  ks.counter = ar.alloc<unsigned>(RED_KINDS);
  AMG_CUDA(cudaMemset(ks.counter, 0, RED_KINDS * sizeof(unsigned)));
  ks.gcount = ar.alloc<unsigned>((size_t)RED_KINDS * r0p.ngroups);
  AMG_CUDA(cudaMemset(ks.gcount, 0, (size_t)RED_KINDS * r0p.ngroups * sizeof(unsigned)));
  ks.grp_cta = r0p.grp_cta;
  ks.sys_grp = r0p.sys_grp;
  ks.ngroups = r0p.ngroups;
  ks.sg = r0p.sg;
  ks.rho = ar.alloc<double>(nv);
  ks.alpha = ar.alloc<double>(nv);
  ks.alpha_prev = ar.alloc<double>(nv);
  AMG_CUDA(cudaMemset(ks.alpha, 0, nv * sizeof(double)));
  AMG_CUDA(cudaMemset(ks.alpha_prev, 0, nv * sizeof(double)));
  ks.beta = ar.alloc<double>(nv);
  ks.bnorm = ar.alloc<double>(nv);
  ks.rnorm = ar.alloc<double>(nv);
  ks.conv = ar.alloc<int>(nv);
  ks.iters = ar.alloc<int>(nv);
  ks.status = ar.alloc<int>(nv);
  ks.active = ar.alloc<int>(P.nsys);
  ks.done = ar.alloc<int>(1);
  ks.iter = ar.alloc<int>(1);
  ks.sys_cta = r0p.sys_cta;
  ks.nsys = P.nsys;
  AMG_CUDA(cudaMemset(ks.done, 0, sizeof(int)));
  AMG_CUDA(cudaMallocHost(&W->h_done, sizeof(int)));
  AMG_CUDA(cudaMallocHost(&W->h_iter, sizeof(int)));
  for (int k = 0; k + 1 < P.L; ++k) W->tp.push_back(make_tpart(ar, P.tr[k], P.lev[k], K, W->err));
  W->rq = W->rp[0];
  W->ksq = view_state(ar, ks, W->rq, K);
  AMG_CUDA(cudaDeviceSynchronize());
  if (cached) {
    const long long* t = tv.data() + 3 * nt;
    for (int k = 0; k < nt; ++k) apply_transfer(P, *W, k, (int)t[3 * k], (int)t[3 * k + 1], (int)t[3 * k + 2]);
    t += 3 * nt;
    if (t[0] > 0 || t[1] > 0) apply_q(P, *W, t[0], (int)t[1], (int)t[2], (int)t[3]);
    t += 4;
    if (split && P.nsys == 1) apply_persist(*W, (int)t[0], (int)t[1], (int)t[2]);
  }
  std::vector<long long> out;
  if (!cached && autotune) {
    for (int k = 0; k + 1 < P.L; ++k) {
      if (prec == 64) tune_transfer<double>(P, *W, k);
      else tune_transfer<float>(P, *W, k);
    }
    tune_q(P, *W);
    if (split && P.nsys == 1) tune_persist(P, *W);
    for (int k = 0; k < nt; ++k) out.insert(out.end(), {W->t_rp[k], W->t_rps[k], W->t_nzl[k]});
    for (int k = 0; k < nt; ++k) out.insert(out.end(), {W->t_tp[k], W->t_tps[k], W->t_tpw[k]});
    out.insert(out.end(), {W->t_q, W->t_qn, W->t_qs, W->t_qg});
    out.insert(out.end(), {(long long)W->t_pu, (long long)W->t_pp, (long long)W->t_ppost, 0LL});
  }
  if (!cached && !autotune && rform_override() > 0)  // untuned workspaces take R only when forced
    for (int k = 0; k < nt; ++k) apply_transfer(P, *W, k, 0, 0, W->tp[k].warp + 4 * W->tp[k].pwarp);
  if (variant) make_var(P, *W, variant);
  setup_fused_coarse(P, *W, autotune, cached ? (int)tv[6 * nt + 8] : -2);
  if (autotune && !cached) {
    out.push_back(W->cc_s);
    tune_cache_store(tkey, out);
  }
  apply_wait_hook(P, *W);
  P.ws[key] = W;
  return *W;
}

// Buffers of the variant cycle: the workspace's level vectors, its tuned
// launch choices and, for the K-cycle, five more vectors per inner level.
static void make_var(Plan& P, Workspace& W, int variant) {
  AMG_REQUIRE(W.prec == 64 && !W.split, "internal: variant cycles run in float64");
  VarCycle& vc = W.var;
  W.variant = variant;
  vc.smoother = variant & 1;
  vc.kind = (variant >> 1) & 1;
  vc.K = W.K;
  vc.pre = W.pre;
  vc.post = W.post;
  for (int k = 0; k < P.L; ++k) {
    vc.f.push_back(static_cast<double*>(W.f[k]));
    vc.u.push_back(static_cast<double*>(W.u[k]));
    vc.v.push_back(static_cast<double*>(W.v[k]));
  }
  vc.nzl = W.nzl;
  vc.rp = W.rp;
  vc.tp = W.tp;
  for (auto* b : {&vc.c2, &vc.v1, &vc.v2, &vc.r2, &vc.e}) b->assign(P.L, nullptr);
  vc.dots.assign(P.L, nullptr);
  size_t ncta_max = 1;
  for (int j = 1; j + 1 < P.L && vc.kind == 1; ++j) {
    const size_t nk = (size_t)P.lev[j].n * W.K;
    for (auto* b : {&vc.c2, &vc.v1, &vc.v2, &vc.r2, &vc.e}) (*b)[j] = W.ar.alloc<double>(nk);
    vc.dots[j] = W.ar.alloc<double>((size_t)5 * W.K);
    ncta_max = std::max(ncta_max, var_level_ctas(P.lev[j].n, vc));
  }
  vc.partial = W.ar.alloc<double>(ncta_max * 2 * W.K);
}

// ------------------------------------------------------------- timing --
// TimedLaunch: amg_internal.cuh

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
// The levels from W.cc_s down to the coarsest and back up in one cooperative
// launch (k_coarse_cycle); cur/oth hold each level's iterate and other
// buffer as the cycle starts.
template <typename TC>
static void launch_coarse_cycle(const Plan& P, const Workspace& W, const std::vector<TC*>& cur,
                                const std::vector<TC*>& oth, const int* done, cudaStream_t st) {
  CcArgs<TC> a;
  a.s = W.cc_s;
  a.L = P.L;
  a.pre = W.pre;
  a.post = W.post;
  for (int k = W.cc_s; k < P.L; ++k) {
    const Level& Lk = P.lev[k];
    CcLevel<TC>& c = a.lev[k];
    c.n = Lk.n;
    c.rowptr = Lk.rowptr;
    c.col = Lk.col;
    c.val = vals<TC>(Lk);
    c.dinv = k + 1 < P.L ? dinvs<TC>(Lk) : nullptr;
    c.f = static_cast<TC*>(W.f[k]);
    c.u = cur[k];
    c.v = oth[k];
    if (k + 1 < P.L) {
      const Transfer& T = P.tr[k];
      a.tr[k] = CcTransfer<TC>{T.nagg, T.row_start, T.coarse_start, T.blk_start, pvals<TC>(T)};
    }
  }
  a.cn = P.co.n;
  a.cnblk = P.co.nblk;
  a.cblk_off = P.co.blk_off;
  a.cinv_off = P.co.inv_off;
  a.cinv = P.co.inv;
  a.bar_count = W.cc_bar;
  a.bar_gen = W.cc_bar + 1;
  a.err = W.err;
  a.done = done;
  a.hang_test = W.cc_hang;
  // about one second at the maximum SM clock; a millisecond under the test hook
  a.budget = W.cc_hang ? (1ll << 21) : (1ll << 31);
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)W.cc_grid);
    cfg.blockDim = dim3(CC_BS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AMG_CUDA(cudaLaunchKernelEx(&cfg, k_coarse_cycle<TC, KK>, a));
  });
  AMG_LAUNCH_CHECK();
}

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
  // levels >= 1 timed as one span (AMG_KERNEL_COARSE_LEVELS)
  std::unique_ptr<TimedLaunch> coarse_span;
  // with the fused small-level cycle the restrictions stop at its start level
  const int kdown = W.cc_s > 0 ? W.cc_s : L - 1;
  for (int k = 0; k + 1 < L; ++k) P.tr[k].rf_last = 0;
  for (int k = 0; k < kdown; ++k) {
    if (k == 1) coarse_span.reset(new TimedLaunch(h, AMG_KERNEL_COARSE_LEVELS, st, pool));
    for (int s = 1; s < W.pre; ++s) {
      launch_smooth<TC>(K, W.nzl[k], P.lev[k], W.rp[k], F(k), cur[k], oth[k], done, st);
      std::swap(cur[k], oth[k]);
    }
    bool smooth_next = (k + 1 < L - 1);
    {
      TimedLaunch tl(h, k == 0 ? AMG_KERNEL_RESTRICT_L0 : -1, st, pool);
      const bool by_r = W.pre == 1 && k < (int)W.rform.size() && W.rform[k];
      P.tr[k].rf_last = by_r ? 1 : 0;
      if (by_r) {
        // fc = R f: the iterate entering the restriction is D^{-1} f
        launch_restrict_rf<TC>(K, P.tr[k], P.lev[k + 1], smooth_next, F(k), F(k + 1), cur[k + 1], done, st,
                               W.rform[k]);
      } else if (k == 0 && W.u0free) {
        // t = f - A D^{-1} f: the first pre-sweep from zero is folded into the
        // column-scaled matrix, so u0 = D^{-1} f is never stored
        Level L0s = P.lev[0];
        L0s.val32 = P.lev[0].val_sc;
        launch_restrict<TC>(K, W.nzl[0], L0s, P.tr[0], W.tp[0], P.lev[1], smooth_next, F(0), F(0), F(1),
                            cur[1], done, st);
      } else {
        launch_restrict<TC>(K, W.nzl[k], P.lev[k], P.tr[k], W.tp[k], P.lev[k + 1], smooth_next, F(k), cur[k],
                            F(k + 1), cur[k + 1], done, st);
      }
    }
  }
  if (!coarse_span) coarse_span.reset(new TimedLaunch(h, AMG_KERNEL_COARSE_LEVELS, st, pool));
  TC* res;
  int kup;
  if (W.cc_s > 0) {
    launch_coarse_cycle<TC>(P, W, cur, oth, done, st);
    // the kernel's out-of-place sweeps: pre - 1 before and post after the
    // coarse correction on every level it smooths
    for (int k = W.cc_s; k + 1 < L; ++k)
      for (int n = 0; n < W.pre - 1 + W.post; ++n) std::swap(cur[k], oth[k]);
    res = cur[W.cc_s];
    kup = W.cc_s - 1;
  } else {
    launch_coarse<TC>(K, P.co, F(L - 1), cur[L - 1], done, st);
    res = cur[L - 1];
    kup = L - 2;
  }
  for (int k = kup; k >= 0; --k) {
    if (k == 0) coarse_span.reset();
    {
      TimedLaunch tl(h, k == 0 ? AMG_KERNEL_PROLONG_L0 : -1, st, pool);
      if (k == 0 && W.u0free)  // u = D^{-1} f + P e
        launch_prolong<TC>(K, P.tr[0], W.tp[0], res, cur[0], done, st, F(0), reinterpret_cast<const TC*>(P.lev[0].dinv32));
      else
        launch_prolong<TC>(K, P.tr[k], W.tp[k], res, cur[k], done, st);
    }
    int sweeps = (k == 0) ? W.post - 1 : W.post;
    for (int s = 0; s < sweeps; ++s) {
      launch_smooth<TC>(K, W.nzl[k], P.lev[k], W.rp[k], F(k), cur[k], oth[k], done, st);
      std::swap(cur[k], oth[k]);
    }
    res = cur[k];
  }
  TimedLaunch tl(h, AMG_KERNEL_SMOOTH_L0, st, pool);
  const bool pers = W.post_grid > 0 && &ks == &W.ks;
  RPart rp0 = W.rp[0];
  if (pers && !W.post_stage) rp0.sg.enabled = 0;
  launch_post0<TC>(K, W.nzl[0], P.lev[0], rp0, F(0), cur[0], W.r, W.split ? W.rl : nullptr,
                   reinterpret_cast<TC*>(W.z), pers ? W.ksf_post : ks, mode, st, pers ? W.post_grid : 0);
}

// Device time of one V-cycle (mode 2: no CG scalars) replayed from a CUDA
// graph, the minimum of five replays; the fused small-level cycle's tuner.
static float time_vcycle_graph(Plan& P, Workspace& W) {
  cudaStream_t st;
  AMG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  AMG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  g_capturing = true;
  try {
    if (W.prec == 64 && !W.split) enqueue_cycle<double>(nullptr, P, W, st, 2, W.zero_flag, W.ks, nullptr);
    else enqueue_cycle<float>(nullptr, P, W, st, 2, W.zero_flag, W.ks, nullptr);
  } catch (...) {
    g_capturing = false;
    cudaStreamEndCapture(st, &g);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(st);
    throw;
  }
  g_capturing = false;
  AMG_CUDA(cudaStreamEndCapture(st, &g));
  AMG_CUDA(cudaGraphInstantiate(&ge, g, 0));
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  AMG_CUDA(cudaGraphLaunch(ge, st));
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    AMG_CUDA(cudaEventRecord(e0, st));
    AMG_CUDA(cudaGraphLaunch(ge, st));
    AMG_CUDA(cudaEventRecord(e1, st));
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  int werr = 0;
  AMG_CUDA(cudaMemcpy(&werr, W.err, sizeof(int), cudaMemcpyDeviceToHost));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  cudaStreamDestroy(st);
  AMG_REQUIRE(werr == 0, "internal: a bounded wait gave up while timing the V-cycle");
  return best;
}

static void launch_cg_q(Workspace& W, const Level& L, cudaStream_t st) {
  if (W.split) {
    dispatch_k(W.K, [&](auto kc) {
      constexpr int KK = decltype(kc)::value;
      dispatch_nzl(W.K, W.nzl_q, [&](auto nc) {
        constexpr int NZ = decltype(nc)::value;
        if constexpr (VT<float, KK>::CL * NZ <= 32) {
          // a batch of 9 when every row has at most 9 entries (a 9-point row
          // then wastes no predicated step)
          const bool b9 = NZ == 1 && L.max_row_len <= 9;
          const bool stg = W.q_stage && W.rq.sg.enabled;
          const bool pkd = W.q_pack && L.hl && !stg;
          auto kern = stg ? (b9 ? k_cg_q_df<KK, NZ, true, 9> : k_cg_q_df<KK, NZ, true>)
                          : pkd ? (b9 ? k_cg_q_df<KK, NZ, false, 9, true> : k_cg_q_df<KK, NZ, false, 0, true>)
                                : (b9 ? k_cg_q_df<KK, NZ, false, 9> : k_cg_q_df<KK, NZ, false>);
          Stage sg = W.rq.sg;
          sg.enabled = sg.enabled && W.q_stage;
          size_t smem = pipe_bytes(sg, 2, W.q_grid > 0 ? 2 : 1);
          ensure_smem(kern, smem);
          const int grid = W.q_grid > 0 ? W.q_grid : W.rq.ncta;
          kern<<<grid, BS, smem, st>>>(W.rq.cta_row, L.rowptr, L.col, L.val32, L.vallo, W.ph, W.ph2, W.qh, W.ql,
                                       W.ksq, sg, W.rq.ncta, L.hl);
        }
      });
    });
    AMG_LAUNCH_CHECK();
    return;
  }
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    dispatch_nzl(W.K, W.nzl_q, [&](auto nc) {
      constexpr int NZ = decltype(nc)::value;
      if constexpr (VT<double, KK>::CL * NZ <= 32) {
        auto kern = k_cg_q<KK, NZ>;
        size_t smem = stage_bytes(W.rp[0].sg, 0, 1);
        ensure_smem(kern, smem);
        kern<<<W.rp[0].ncta, BS, smem, st>>>(W.rp[0].cta_row, L.rowptr, L.col, L.val64, W.p, W.q, W.ks);
      }
    });
  });
  AMG_LAUNCH_CHECK();
}

static void launch_cg_init(Workspace& W, const Level& L, cudaStream_t st) {
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    dispatch_nzl(W.K, W.split ? pick_nzl<double>(L, W.K) : W.nzl_q, [&](auto nc) {
      constexpr int NZ = decltype(nc)::value;
      if constexpr (VT<double, KK>::CL * NZ <= 32) {
        auto kern = k_cg_init<KK, NZ>;
        size_t smem = stage_bytes(W.rp[0].sg, 0, 1);
        ensure_smem(kern, smem);
        kern<<<W.rp[0].ncta, BS, smem, st>>>(W.rp[0].cta_row, L.rowptr, L.col, L.val64, W.b, W.x, W.r, W.ks);
      }
    });
  });
  AMG_LAUNCH_CHECK();
}

// z holds float32 values when the cycle runs in float32 (and the hierarchy
// has a cycle at all); the one-level solve writes float64.
static bool z_is_f32(const Plan& P, const Workspace& W) { return W.prec == 32 && P.L > 1; }

static void launch_cg_p(const Plan& P, Workspace& W, const Level& L, int first, cudaStream_t st) {
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    if (W.split)
      k_cg_p_df<KK><<<W.p_grid ? W.p_grid : W.rp[0].ncta, BS, 0, st>>>(
          W.rp[0].cta_row, reinterpret_cast<const float*>(W.z), W.ph, W.ph2, W.xh, W.xl, W.ks, first,
          W.rp[0].ncta);
    else if (z_is_f32(P, W))
      k_cg_p<KK, float><<<W.rp[0].ncta, BS, 0, st>>>(W.rp[0].cta_row, reinterpret_cast<const float*>(W.z), W.p,
                                                     W.ks, first);
    else
      k_cg_p<KK, double><<<W.rp[0].ncta, BS, 0, st>>>(W.rp[0].cta_row, W.z, W.p, W.ks, first);
  });
  AMG_LAUNCH_CHECK();
}

static void launch_update_df(Workspace& W, const Level& L, cudaStream_t st) {
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    k_cg_update_df<KK><<<W.upd_grid ? W.upd_grid : W.rp[0].ncta, BS, 0, st>>>(
        W.rp[0].cta_row, W.rh, W.rl, W.qh, W.ql, L.dinv32, W.u0free ? nullptr : static_cast<float*>(W.u[0]),
        W.upd_grid ? W.ksf_upd : W.ks, W.rp[0].ncta);
  });
  AMG_LAUNCH_CHECK();
}

static void launch_pair(bool split_dir, long long n, const double* v, float* h, float* l, double* out,
                        const int* done, cudaStream_t st) {
  unsigned grid = (unsigned)((n + 255) / 256);
  (void)done;
  if (split_dir) k_split_pair<<<grid, 256, 0, st>>>(n, v, h, l);
  else k_join_pair<<<grid, 256, 0, st>>>(n, h, l, out);
  AMG_LAUNCH_CHECK();
}

static void launch_rz(Workspace& W, const Level& L, int mode, cudaStream_t st) {
  dispatch_k(W.K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    k_rz<KK><<<W.rp[0].ncta, BS, 0, st>>>(W.rp[0].cta_row, W.r, W.z, W.ks, mode);
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
  } else if (W.variant) {
    enqueue_var_cycle(P, W.var, W.r, W.z, static_cast<double*>(W.u[0]), W.ks.done, st, h, nullptr);
    launch_rz(W, L0, 0, st);
  } else {
    if (W.split) {
      // x and r enter the double-float pairs; r_hi is the cycle's f0
      long long nk = (long long)W.n0 * W.K;
      launch_pair(true, nk, W.r, W.rh, W.rl, nullptr, W.ks.done, st);
      launch_pair(true, nk, W.x, W.xh, W.xl, nullptr, W.ks.done, st);
    }
    TC* f0 = (W.prec == 64 || W.split) ? nullptr : static_cast<TC*>(W.f[0]);
    if (!W.u0free) launch_presmooth0<TC>(W.K, L0, W.rp[0], W.r, static_cast<TC*>(W.u[0]), f0, W.ks.done, st);
    enqueue_cycle<TC>(h, P, W, st, 0, W.ks.done, W.ks, nullptr);
  }
  launch_cg_p(P, W, L0, 1, st);
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
    TC* u0 = (P.L == 1 || W.variant) ? nullptr : static_cast<TC*>(W.u[0]);
    if (W.split) launch_update_df(W, L0, st);
    else launch_update<TC>(W.K, L0, W.rp[0], W.x, W.r, W.p, W.q, u0, f0, W.ks, st);
  }
  if (W.variant && P.L > 1) {
    enqueue_var_cycle(P, W.var, W.r, W.z, static_cast<double*>(W.u[0]), W.ks.done, st, h, pool);
    launch_rz(W, L0, 1, st);
  } else {
    enqueue_cycle<TC>(h, P, W, st, 1, W.ks.done, W.ks, pool);
    if (P.L == 1) launch_rz(W, L0, 1, st);
  }
  TimedLaunch tl(h, AMG_KERNEL_CG_DIRECTION, st, pool);
  launch_cg_p(P, W, L0, 0, st);
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
    NvtxRange nv_chunk("amg pcg iterations");
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

// Bounded device waits that gave up (bit 1: a staged copy, bit 2: the grid
// barrier of the fused small-level cycle): clear the flags and the barrier
// words, then report AMG_ERR_TIMEOUT.  The context stays usable.
static void check_waits(Workspace& W, int werr) {
  if (!werr) return;
  AMG_CUDA(cudaMemset(W.err, 0, sizeof(int)));
  if (W.cc_bar) AMG_CUDA(cudaMemset(W.cc_bar, 0, 2 * sizeof(unsigned)));
  AMG_CUDA(cudaDeviceSynchronize());
  if (werr & 2) throw Error(AMG_ERR_TIMEOUT, "a bounded wait of the small-level grid barrier gave up");
  throw Error(AMG_ERR_TIMEOUT, "a bounded wait for a shared-memory staging copy gave up");
}

// smoother | cycle << 1 for the variant cycles (0: the V-cycle with
// l1-Jacobi); builds the Gauss-Seidel colouring on first use.
static int check_variant(amg_hierarchy* owner, Plan& P, const amg_opts& o) {
  AMG_REQUIRE(o.smoother == 0 || o.smoother == 1, "smoother must be 0 (l1-Jacobi) or 1 (Gauss-Seidel)");
  AMG_REQUIRE(o.cycle == 0 || o.cycle == 1, "cycle must be 0 (V) or 1 (K)");
  const int variant = o.smoother | (o.cycle << 1);
  if (!variant || P.L == 1) return 0;
  AMG_REQUIRE(o.cycle_precision == 64, "the Gauss-Seidel smoother and the K-cycle run with cycle_precision 64");
  AMG_REQUIRE(owner && &owner->plan == &P && P.nsys == 1,
              "the Gauss-Seidel smoother and the K-cycle need a single hierarchy (not a batch)");
  if (o.smoother == 1) ensure_gs(owner, P, owner->own);
  return variant;
}

amg_status run_pcg(amg_hierarchy* owner, Plan& P, const SolveReq& rq, const amg_opts& o, cudaStream_t user,
                   amg_info* info) {
  NvtxRange nvtx(rq.nsys > 1 ? "amg solve (batched)" : "amg solve");
  int maxr = 0;
  for (int s = 0; s < rq.nsys; ++s) maxr = std::max(maxr, rq.nrhs[s]);
  AMG_REQUIRE(maxr >= 1 && maxr <= 32, "nrhs must be in [1, 32] per call");
  AMG_REQUIRE(o.cycle_precision == 64 || o.cycle_precision == 32, "cycle_precision must be 64 or 32");
  AMG_REQUIRE(o.pre >= 1 && o.post >= 1 && o.pre <= 16 && o.post <= 16, "pre and post sweeps must be in [1, 16]");
  AMG_REQUIRE(o.maxit >= 1 && o.rtol >= 0, "maxit must be >= 1 and rtol >= 0");
  const int variant = check_variant(owner, P, o);
  const int K = round_k(maxr);
  const bool split = o.cycle_precision == 32 && !o.outer_fp64 && P.L > 1;
  Workspace& W = get_ws(P, K, o.cycle_precision, o.pre, o.post, split, o.autotune != 0, variant);
  for (KState* v : {&W.ks, &W.ksq, &W.ksf_upd, &W.ksf_post}) {  // the state and its views over other CTA groups
    v->rtol = o.rtol;
    v->maxit = o.maxit;
  }
  StreamJoin sj(owner, user);
  cudaStream_t st = owner->own;
  std::vector<int> act(rq.nrhs.begin(), rq.nrhs.end());
  AMG_CUDA(cudaMemcpyAsync(W.ks.active, act.data(), act.size() * 4, cudaMemcpyHostToDevice, st));
  stage_inputs(P, W, rq, st);
  if (o.cycle_precision == 64) pcg_loop<double>(owner, P, W, o, st);
  else pcg_loop<float>(owner, P, W, o, st);
  if (W.split) {
    dispatch_k(K, [&](auto kc) {
      constexpr int KK = decltype(kc)::value;
      k_cg_x_df<KK><<<W.rp[0].ncta, BS, 0, st>>>(W.rp[0].cta_row, W.ph, W.ph2, W.xh, W.xl, W.ks, *W.h_iter - 1);
    });
    AMG_LAUNCH_CHECK();
    launch_pair(false, (long long)W.n0 * K, nullptr, W.xh, W.xl, W.x, nullptr, st);
  }
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
  int werr = 0;
  AMG_CUDA(cudaMemcpyAsync(&werr, W.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  sj.finish();
  check_waits(W, werr);
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
  NvtxRange nv("amg vcycle");
  AMG_REQUIRE(nrhs >= 1 && nrhs <= 32, "nrhs must be in [1, 32]");
  AMG_REQUIRE(o.cycle_precision == 64 || o.cycle_precision == 32, "cycle_precision must be 64 or 32");
  AMG_REQUIRE(o.pre >= 1 && o.post >= 1, "pre and post sweeps must be >= 1");
  const int variant = check_variant(owner, P, o);
  const int K = round_k(nrhs);
  Workspace& W = get_ws(P, K, o.cycle_precision, o.pre, o.post, false, false, variant);
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
  } else if (W.variant) {
    enqueue_var_cycle(P, W.var, W.r, W.z, static_cast<double*>(W.u[0]), W.zero_flag, st, nullptr, nullptr);
  } else if (o.cycle_precision == 64) {
    launch_presmooth0<double>(K, P.lev[0], W.rp[0], W.r, static_cast<double*>(W.u[0]), nullptr, W.zero_flag, st);
    enqueue_cycle<double>(nullptr, P, W, st, 2, W.zero_flag, ks, nullptr);
  } else {
    launch_presmooth0<float>(K, P.lev[0], W.rp[0], W.r, static_cast<float*>(W.u[0]), static_cast<float*>(W.f[0]),
                             W.zero_flag, st);
    enqueue_cycle<float>(nullptr, P, W, st, 2, W.zero_flag, ks, nullptr);
  }
  double* zout = W.z;
  if (z_is_f32(P, W)) {
    long long nz = (long long)W.n0 * K;
    k_f32_to_f64<<<(unsigned)((nz + 255) / 256), 256, 0, st>>>(nz, reinterpret_cast<const float*>(W.z), W.q);
    AMG_LAUNCH_CHECK();
    zout = W.q;
  }
  stage_outputs(P, W, rq, zout, st);
  int werr = 0;
  AMG_CUDA(cudaMemcpyAsync(&werr, W.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  sj.finish();
  check_waits(W, werr);
}

void run_adjoint_grad(amg_hierarchy* h, const double* lam_caller, const double* x_caller, int nrhs,
                      double* grad, cudaStream_t user) {
  NvtxRange nv("amg adjoint gradient");
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

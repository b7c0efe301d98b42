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

// ------------------------------------------------ TMA bulk staging --
// A CTA's rows [r0, r1) own the contiguous non-zeros [rowptr[r0], rowptr[r1]).
// One thread copies that slice of col (and of each value array) into shared
// memory with 1-D bulk TMA copies (cp.async.bulk, completion on an mbarrier)
// while the CTA loads its rowptr slice; the row loops then take indices and
// values from shared memory and only the x gathers go to L2/HBM.  Copies are
// widened to 16-byte boundaries (the arrays carry 16 padding elements).
// The wait on the mbarrier is bounded: on timeout the kernel records an error
// in *err (the host then reports AMG_ERR_TIMEOUT) and waits once more, with
// the full bound, before it goes on (stage_wait).
__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }
// Shared memory of the staging area with n4 four-byte and n8 eight-byte value arrays.
__host__ __device__ inline size_t stage_bytes(const Stage& sg, int n4, int n8) {
  if (!sg.enabled) return 0;
  return 16 + align16((size_t)(sg.rows_max + 1) * 4) + (size_t)sg.span4 * 4 * (1 + n4) +
         (size_t)sg.span8 * 8 * n8;
}

// Bulk prefetch of [p, p + bytes) into L2 (no registers, no completion):
// the range is widened to 16-byte boundaries; 0 bytes issue nothing.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  if (bytes == 0) return;
  const unsigned long long a0 = reinterpret_cast<unsigned long long>(p) & ~15ull;
  const unsigned long long a1 = (reinterpret_cast<unsigned long long>(p) + bytes + 15ull) & ~15ull;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((unsigned)(a1 - a0)) : "memory");
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  if (bytes == 0) return;
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
constexpr int kWaitPolls = 1 << 22;  // polls of a bounded wait (each try_wait may block briefly)
// Bounded wait for an mbarrier phase: at most ``polls`` try_wait polls, or,
// for a first wait shortened by the test hook (polls < 16), that many
// non-blocking test_wait polls.  Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase, int polls = kWaitPolls) {
  unsigned ok = 0;
  if (polls > 0 && polls < 16) {
    for (int it = 0; it < polls && !ok; ++it) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_addr(bar)), "r"(phase)
          : "memory");
    }
    return ok != 0;
  }
  for (int it = 0; it < polls && !ok; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
  }
  return ok != 0;
}
// The wait of a staged copy: the first wait is bounded (by sg.first_wait
// when the test hook sets it); when it gives up the CTA records the error
// for the host (AMG_ERR_TIMEOUT) and waits once more with the full bound, so
// that no copy into its shared memory is left in flight, and goes on.
__device__ __forceinline__ void stage_wait(const Stage& sg, uint64_t* bar, unsigned phase) {
  if (!mbar_wait_bounded(bar, phase, sg.first_wait > 0 ? sg.first_wait : kWaitPolls)) {
    atomicOr(sg.err, 1);
    mbar_wait_bounded(bar, phase);
  }
}

// Double-buffered staging for CTAs that walk several row chunks (persistent
// launches): while the CTA works on chunk c from buffer c & 1, the rowptr,
// col and value slices (4-byte values) of its next chunk arrive in the other
// buffer by 1-D bulk TMA copies, each buffer completing on its own mbarrier.
// Layout: two mbarriers (16 bytes), then per buffer rows_max + 8 rowptr
// words and span4 words of col and of each of the NV value arrays.  Copies
// start at 16-byte boundaries (rowptr words from r0 & ~3, non-zeros from
// j0 & ~3) and stay inside the arrays' padding.
__host__ __device__ inline size_t pipe_buf_bytes(const Stage& sg, int nv) {
  return align16((size_t)(sg.rows_max + 8) * 4) + (size_t)sg.span4 * 4 * (1 + nv);
}
__host__ __device__ inline size_t pipe_bytes(const Stage& sg, int nv, int nbuf) {
  return sg.enabled ? 16 + (size_t)nbuf * pipe_buf_bytes(sg, nv) : 0;
}
__device__ __forceinline__ void pipe_init(unsigned char* smem) {
  if (threadIdx.x == 0) {
    mbar_init(reinterpret_cast<uint64_t*>(smem), 1);
    mbar_init(reinterpret_cast<uint64_t*>(smem) + 1, 1);
  }
  __syncthreads();
}
// One thread: request rows [r0, r1) into buffer buf.
template <int NV>
__device__ __forceinline__ void pipe_issue(const Stage& sg, unsigned char* smem, int buf, int r0, int r1,
                                           const int* __restrict__ rowptr, const int* __restrict__ col,
                                           const float* const (&vals)[NV]) {
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem) + buf;
  unsigned char* b = smem + 16 + (size_t)buf * pipe_buf_bytes(sg, NV);
  const int a0 = r0 & ~3, a1 = (r1 + 4) & ~3;
  const int j0 = __ldg(rowptr + r0), j1 = __ldg(rowptr + r1);
  const int e0 = j0 & ~3, e1 = (j1 + 3) & ~3;
  const unsigned rb = (unsigned)(a1 - a0) * 4u, cb = (unsigned)(e1 - e0) * 4u;
  // the buffer's previous contents were read through the generic proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, rb + cb * (1u + NV));
  tma_load_1d(b, rowptr + a0, rb, bar);
  unsigned char* c = b + align16((size_t)(sg.rows_max + 8) * 4);
  tma_load_1d(c, col + e0, cb, bar);
#pragma unroll
  for (int a = 0; a < NV; ++a) tma_load_1d(c + (size_t)sg.span4 * 4 * (1 + a), vals[a] + e0, cb, bar);
}
// All threads: wait for buffer buf (its use-th fill) and return its views.
template <int NV>
__device__ __forceinline__ void pipe_wait(const Stage& sg, unsigned char* smem, int buf, int use, int r0,
                                          const int* __restrict__ rowptr, const int*& rp, int& roff,
                                          const int*& cs, const float* (&vs)[NV], int& joff) {
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem) + buf;
  stage_wait(sg, bar, (unsigned)(use & 1));
  unsigned char* b = smem + 16 + (size_t)buf * pipe_buf_bytes(sg, NV);
  rp = reinterpret_cast<const int*>(b);
  roff = r0 & ~3;
  cs = reinterpret_cast<const int*>(b + align16((size_t)(sg.rows_max + 8) * 4));
#pragma unroll
  for (int a = 0; a < NV; ++a) vs[a] = reinterpret_cast<const float*>(cs + (size_t)sg.span4 * (1 + a));
  joff = __ldg(rowptr + r0) & ~3;
}

// Where the row loop reads rowptr / col / values: either the staged copies
// (with index offsets) or the global arrays.
template <typename TA>
struct CsrView {
  const int* rp;
  int roff;
  const int* col;
  int coff;
  const TA* val;
  int voff;
};

// A CTA whose rows form one contiguous range [r0, r1) covers one contiguous
// non-zero range; with float values it can stage that slice (rowptr, col,
// values) into shared memory with bulk TMA copies first (one buffer of the
// pipeline below), so that its gathers wait on nothing but themselves.
template <typename TC>
__device__ __forceinline__ CsrView<TC> group_view(const Stage& sg, unsigned char* smem, int r0, int r1,
                                                  const int* __restrict__ rowptr, const int* __restrict__ col,
                                                  const TC* __restrict__ val) {
  if constexpr (sizeof(TC) == 4) {
    if (sg.enabled) {
      pipe_init(smem);
      if (threadIdx.x == 0) {
        const float* v1[1] = {reinterpret_cast<const float*>(val)};
        pipe_issue<1>(sg, smem, 0, r0, r1, rowptr, col, v1);
      }
      const int* rp;
      const int* cs;
      const float* vs[1];
      int roff, joff;
      pipe_wait<1>(sg, smem, 0, 0, r0, rowptr, rp, roff, cs, vs, joff);
      return CsrView<TC>{rp, roff, cs, joff, reinterpret_cast<const TC*>(vs[0]), joff};
    }
  }
  return CsrView<TC>{rowptr, 0, col, 0, val, 0};
}

// Stage rows [r0, r1): col plus NV value arrays of widths vw[] (4 or 8).
template <int NV>
__device__ __forceinline__ bool stage_csr(const Stage& sg, unsigned char* smem, int r0, int r1,
                                          const int* __restrict__ rowptr, const int* __restrict__ col,
                                          const void* const (&vsrc)[NV], const int (&vw)[NV],
                                          const void* (&vdst)[NV], const int*& srp, const int*& scol,
                                          int& j4, int& j8) {
  if (!sg.enabled) return false;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  int* rp_s = reinterpret_cast<int*>(smem + 16);
  int* col_s = reinterpret_cast<int*>(smem + 16 + align16((size_t)(sg.rows_max + 1) * 4));
  unsigned char* vp = reinterpret_cast<unsigned char*>(col_s + sg.span4);
  const int j0 = __ldg(rowptr + r0), j1 = __ldg(rowptr + r1);
  j4 = j0 & ~3;
  j8 = j0 & ~1;
  const int e4 = (j1 + 3) & ~3, e8 = (j1 + 1) & ~1;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    vdst[a] = vp;
    vp += vw[a] == 4 ? (size_t)sg.span4 * 4 : (size_t)sg.span8 * 8;
  }
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned b4 = (unsigned)(e4 - j4) * 4u, b8 = (unsigned)(e8 - j8) * 8u;
    unsigned total = b4;
#pragma unroll
    for (int a = 0; a < NV; ++a) total += vw[a] == 4 ? b4 : b8;
    mbar_expect_tx(bar, total);
    tma_load_1d(col_s, col + j4, b4, bar);
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const unsigned char* src = static_cast<const unsigned char*>(vsrc[a]);
      if (vw[a] == 4) tma_load_1d(const_cast<void*>(vdst[a]), src + (size_t)j4 * 4, b4, bar);
      else tma_load_1d(const_cast<void*>(vdst[a]), src + (size_t)j8 * 8, b8, bar);
    }
  }
  for (int t = threadIdx.x; t <= r1 - r0; t += blockDim.x) rp_s[t] = __ldg(rowptr + r0 + t);
  __syncthreads();
  stage_wait(sg, bar, 0);
  srp = rp_s;
  scol = col_s;
  return true;
}

// Gathers a lane keeps in flight per row pass: with one lane group per row
// (NZL = 1) the whole of a short row (a 9-point stencil row, or a 10-entry
// slice of a longer one) is requested before the first product, so a row
// costs one memory round trip; with the non-zeros split over NZL lanes each
// lane has few of them and four at a time suffice.
template <int NZL>
__host__ __device__ constexpr int gather_depth() { return NZL == 1 ? 10 : 4; }

// y_i = sum_j a_ij x_j for the K columns owned by this lane.
// UB > 0 (one lane group per row): batches of UB; when every row of the
// warp's pass has exactly UB entries (a warp vote, so all 32 lanes call this)
// the batch is read without predication, the products in the same order.
template <typename TA, typename TX, int K, int NZL, int UB = 0>
__device__ __forceinline__ void row_acc(int i, bool valid, const CsrView<TA>& cv, const TX* __restrict__ x,
                                        int nzl, int cl, TX (&acc)[VT<TX, K>::CPT]) {
  constexpr int CPT = VT<TX, K>::CPT, CL = VT<TX, K>::CL, U = UB > 0 ? UB : gather_depth<NZL>();
#pragma unroll
  for (int t = 0; t < CPT; ++t) acc[t] = TX(0);
  if constexpr (UB > 0 && NZL == 1) {
    int j0 = 0, len = -1;
    if (valid) {
      j0 = cv.rp[i - cv.roff];
      len = cv.rp[i + 1 - cv.roff] - j0;
    }
    if (__all_sync(FULL, len == U)) {
      int c[U];
      TX a[U], xv[U][CPT];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        c[u] = cv.col[j0 + u - cv.coff];
        a[u] = (TX)cv.val[j0 + u - cv.voff];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) ldv<TX, CPT>(x + (size_t)c[u] * K + cl * CPT, xv[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int t = 0; t < CPT; ++t) acc[t] = fma(a[u], xv[u][t], acc[t]);
      return;
    }
  }
  if (valid) {
    const int j1 = cv.rp[i + 1 - cv.roff];
    int j = cv.rp[i - cv.roff] + nzl;
    if constexpr (U != 4) {
      // predicated batches of U non-zeros: every gather of the batch is
      // issued before the first product
      for (; j < j1; j += U * NZL) {
        int c[U];
        TX a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int jj = j + u * NZL;
          const bool ok = jj < j1;
          c[u] = ok ? cv.col[jj - cv.coff] : -1;
          a[u] = ok ? (TX)cv.val[jj - cv.voff] : TX(0);
        }
        TX xv[U][CPT];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (c[u] >= 0) {
            ldv<TX, CPT>(x + (size_t)c[u] * K + cl * CPT, xv[u]);
          } else {
#pragma unroll
            for (int t = 0; t < CPT; ++t) xv[u][t] = TX(0);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int t = 0; t < CPT; ++t) acc[t] = fma(a[u], xv[u][t], acc[t]);
      }
    } else {
    // four non-zeros at a time: their gathers are independent and issue
    // back to back
    for (; j + 3 * NZL < j1; j += 4 * NZL) {
      int c[4];
      TX a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = cv.col[j + u * NZL - cv.coff];
        a[u] = (TX)cv.val[j + u * NZL - cv.voff];
      }
      TX xv[4][CPT];
#pragma unroll
      for (int u = 0; u < 4; ++u) ldv<TX, CPT>(x + (size_t)c[u] * K + cl * CPT, xv[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int t = 0; t < CPT; ++t) acc[t] = fma(a[u], xv[u][t], acc[t]);
    }
    for (; j < j1; j += NZL) {
      TX a = (TX)cv.val[j - cv.voff];
      int c = cv.col[j - cv.coff];
      TX xv[CPT];
      ldv<TX, CPT>(x + (size_t)c * K + cl * CPT, xv);
#pragma unroll
      for (int t = 0; t < CPT; ++t) acc[t] = fma(a, xv[t], acc[t]);
    }
    }
  }
  if constexpr (NZL > 1) {
#pragma unroll
    for (int off = CL; off < CL * NZL; off <<= 1)
#pragma unroll
      for (int t = 0; t < CPT; ++t) acc[t] += __shfl_xor_sync(FULL, acc[t], off);
  }
}

// Stage one value array of type TA and build the view the row loop reads.
template <typename TA>
__device__ __forceinline__ CsrView<TA> staged_view(const Stage& sg, unsigned char* smem, int r0, int r1,
                                                   const int* __restrict__ rowptr, const int* __restrict__ col,
                                                   const TA* __restrict__ val) {
  const void* src[1] = {val};
  const int w[1] = {(int)sizeof(TA)};
  const void* dst[1];
  const int* srp;
  const int* scol;
  int j4, j8;
  if (stage_csr<1>(sg, smem, r0, r1, rowptr, col, src, w, dst, srp, scol, j4, j8))
    return CsrView<TA>{srp, r0, scol, j4, static_cast<const TA*>(dst[0]), sizeof(TA) == 4 ? j4 : j8};
  return CsrView<TA>{rowptr, 0, col, 0, val, 0};
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

// ------------------------------------------------------- double-float --
// A value v is carried as an unevaluated sum hi + lo of two floats (hi =
// fl32(v)).  Products use the exact FMA residual of the leading product plus
// the two cross terms; sums use Knuth's two-sum followed by a fast two-sum.
// The result keeps about 44 bits, all on the float32 pipes.
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float v = s - a;
  e = (a - (s - v)) + (b - v);
}
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// (sh, sl) += (ah, al) * (xh, xl)
__device__ __forceinline__ void df_mac(float ah, float al, float xh, float xl, float& sh, float& sl) {
  float ph = ah * xh;
  float pl = fmaf(ah, xh, -ph);
  pl = fmaf(ah, xl, fmaf(al, xh, pl));
  float s, e;
  df_two_sum(sh, ph, s, e);
  e += sl + pl;
  df_fast_two_sum(s, e, sh, sl);
}
// Accumulating form: (sh, sl) += (ah, al) * (xh, xl) with the low word left
// unnormalised (the product error, the cross terms and the two-sum error all
// go to sl); df_norm once after the last term.
__device__ __forceinline__ void df_acc(float ah, float al, float xh, float xl, float& sh, float& sl) {
  float p = ah * xh;
  float e = fmaf(ah, xh, -p);
  e = fmaf(ah, xl, fmaf(al, xh, e));
  float s = sh + p;
  float v = s - sh;
  float t = (sh - (s - v)) + (p - v);
  sh = s;
  sl += t + e;
}
// (sh, sl) += (ah, al) * x for an exact float x (unnormalised, as df_acc)
__device__ __forceinline__ void df_acc1(float ah, float al, float x, float& sh, float& sl) {
  float p = ah * x;
  float e = fmaf(ah, x, -p);
  e = fmaf(al, x, e);
  float s = sh + p;
  float v = s - sh;
  float t = (sh - (s - v)) + (p - v);
  sh = s;
  sl += t + e;
}
__device__ __forceinline__ void df_norm(float& sh, float& sl) {
  float s, e;
  df_fast_two_sum(sh, sl, s, e);
  sh = s;
  sl = e;
}
// (sh, sl) += (oh, ol)
__device__ __forceinline__ void df_add(float& sh, float& sl, float oh, float ol) {
  float s, e;
  df_two_sum(sh, oh, s, e);
  e += sl + ol;
  df_fast_two_sum(s, e, sh, sl);
}
__device__ __forceinline__ void df_split(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

// Packed float32 pairs: two columns per instruction with the add / sub /
// mul / fma .f32x2 forms of sm_100 and later, each half rounded to nearest
// exactly as its scalar form, so a packed double-float step gives the same
// bits as two scalar ones.
struct F2 {
  unsigned long long v;
};
__device__ __forceinline__ F2 f2_pack(float a, float b) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(F2 x, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  F2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c) {
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ F2 f2_neg(F2 a) { return F2{a.v ^ 0x8000000080000000ull}; }
// df_norm on a pair of columns (the same steps as the scalar form)
__device__ __forceinline__ void df_norm_x2(F2& sh, F2& sl) {
  const F2 s = f2_add(sh, sl);
  const F2 e = f2_sub(sl, f2_sub(s, sh));
  sh = s;
  sl = e;
}
// df_acc1 on a pair of columns (the same steps as the scalar form)
__device__ __forceinline__ void df_acc1_x2(F2 ah, F2 al, F2 x, F2& sh, F2& sl) {
  const F2 p = f2_mul(ah, x);
  F2 e = f2_fma(ah, x, f2_neg(p));
  e = f2_fma(al, x, e);
  const F2 s = f2_add(sh, p);
  const F2 v = f2_sub(s, sh);
  const F2 t = f2_add(f2_sub(sh, f2_sub(s, v)), f2_sub(p, v));
  sh = s;
  sl = f2_add(sl, f2_add(t, e));
}

// CG scalars shared by the fused kernels.
struct KState {
  double* partial;     // ncta0 * NV   (one row per CTA)
  double* gpartial;    // ngroups * NV (one row per group of CTAs)
  unsigned* counter;   // one counter per reducing kernel
  unsigned* gcount;    // per reducing kernel: one counter per group
  const int* grp_cta;  // ngroups + 1
  const int* sys_grp;  // nsys + 1
  int ngroups;
  double *rho, *alpha, *beta, *bnorm, *rnorm;
  double* alpha_prev;  // alpha of the previous iteration (the double-float x step runs every second one)
  int *conv, *iters, *status, *active, *done, *iter;
  const int* sys_cta;  // nsys + 1
  int nsys;
  double rtol;
  int maxit;
  Stage sg;            // level-0 staging of the reducing SpMV kernels
};

enum : int { RED_Q = 0, RED_UPDATE = 1, RED_POST = 2, RED_INIT = 3, RED_KINDS = 4 };

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

// Two-level deterministic reduction: each CTA has written its NV partials;
// the last CTA of each fixed group sums the group (in CTA order), and the
// last group to finish returns true with every group sum in ks.gpartial.
__device__ __forceinline__ bool arrive_two_level(const KState& ks, int kind, int NV, double* sm, double* tot) {
  __shared__ int flag;
  int lo = 0, hi = ks.ngroups - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(ks.grp_cta + mid) <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const int g = lo, b0 = ks.grp_cta[g], b1 = ks.grp_cta[g + 1];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(ks.gcount + kind * ks.ngroups + g, 1u);
    flag = (prev == (unsigned)(b1 - b0 - 1));
  }
  __syncthreads();
  if (!flag) return false;
  __threadfence();
  sum_partials(ks.partial, NV, b0, b1, sm, tot);
  if (threadIdx.x < NV) ks.gpartial[(size_t)g * NV + threadIdx.x] = tot[threadIdx.x];
  if (threadIdx.x == 0) ks.gcount[kind * ks.ngroups + g] = 0u;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(ks.counter + kind, 1u);
    flag = (prev == (unsigned)(ks.ngroups - 1));
  }
  __syncthreads();
  if (!flag) return false;
  __threadfence();
  if (threadIdx.x == 0) ks.counter[kind] = 0u;
  return true;
}

// Per-system totals of the group sums (final CTA only).
__device__ __forceinline__ void system_totals(const KState& ks, int NV, int sy, double* sm, double* tot) {
  sum_partials(ks.gpartial, NV, ks.sys_grp[sy], ks.sys_grp[sy + 1], sm, tot);
}

// ------------------------------------------------------------ V-cycle ----

// v = u + D^{-1} (f - A u)   (one l1-Jacobi sweep, out of place)
template <typename TC, int K, int NZL>
__global__ void __launch_bounds__(BS) k_smooth(const int* __restrict__ cta_row, const int* __restrict__ rowptr,
                                               const int* __restrict__ col, const TC* __restrict__ val,
                                               const TC* __restrict__ dinv, const TC* __restrict__ f,
                                               const TC* __restrict__ u, TC* __restrict__ v,
                                               const int* __restrict__ done, Stage sg) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  const int r0 = cta_row[blockIdx.x], r1 = cta_row[blockIdx.x + 1];
  const CsrView<TC> cv = staged_view<TC>(sg, smraw, r0, r1, rowptr, col, val);
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    const size_t o = (size_t)i * K + cl * CPT;
    // the row's own operands are requested before its gathers (a load after
    // the gather loop would wait for it: one memory round trip per row pass)
    TC fv[CPT], uv[CPT], di = TC(0);
    const bool own = valid && nzl == 0;
    if (own) {
      ldv<TC, CPT>(f + o, fv);
      ldv<TC, CPT>(u + o, uv);
      di = __ldg(dinv + i);
    }
    TC acc[CPT];
    row_acc<TC, TC, K, NZL>(i, valid, cv, u, nzl, cl, acc);
    if (own) {
      TC out[CPT];
#pragma unroll
      for (int t = 0; t < CPT; ++t) out[t] = fma(di, fv[t] - acc[t], uv[t]);
      stv<TC, CPT>(v + o, out);
    }
  }
}

// Shared-memory layout of the transfer kernels: [vector tile | P tile |
// per-aggregate row, coarse-dof and block offsets | dof -> aggregate map].
template <typename TC>
__host__ __device__ inline size_t transfer_smem(int rows_max, int p_max, int a_max, int c_max, int K,
                                                bool with_tile) {
  return (with_tile ? align16((size_t)rows_max * K * sizeof(TC)) : 0) + align16((size_t)p_max * sizeof(TC)) +
         (size_t)3 * (a_max + 1) * sizeof(int) + (size_t)(c_max > rows_max ? c_max : rows_max) * sizeof(int);
}
template <typename TC>
__host__ __device__ inline size_t restrict_stage_bytes(const Stage& sg) {
  return stage_bytes(sg, sizeof(TC) == 4 ? 1 : 0, sizeof(TC) == 8 ? 1 : 0);
}

// Stage the CTA's aggregate metadata and its (contiguous) prolongator blocks.
template <typename TC>
__device__ __forceinline__ void stage_transfer(int a0, int a1, const int* __restrict__ row_start,
                                               const int* __restrict__ coarse_start,
                                               const long long* __restrict__ blk_start,
                                               const TC* __restrict__ P, TC* psm, int* m_rs, int* m_cs,
                                               int* m_bk) {
  const int r0 = row_start[a0], c0 = coarse_start[a0];
  const long long b0 = blk_start[a0], b1 = blk_start[a1];
  for (int t = threadIdx.x; t <= a1 - a0; t += BS) {
    m_rs[t] = __ldg(row_start + a0 + t) - r0;
    m_cs[t] = __ldg(coarse_start + a0 + t) - c0;
    m_bk[t] = (int)(__ldg(blk_start + a0 + t) - b0);
  }
  for (long long e = threadIdx.x; e < b1 - b0; e += BS) psm[e] = __ldg(P + b0 + e);
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
                                                 const int* __restrict__ done, int rows_max, int p_max,
                                                 int a_max, Stage sg, int m_cs_max) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* tail = smraw + restrict_stage_bytes<TC>(sg);
  TC* tsm = reinterpret_cast<TC*>(tail);
  TC* psm = reinterpret_cast<TC*>(tail + align16((size_t)rows_max * K * sizeof(TC)));
  int* m_rs = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(psm) + align16((size_t)p_max * sizeof(TC)));
  int* m_cs = m_rs + (a_max + 1);
  int* m_bk = m_cs + (a_max + 1);
  int* cd2a = m_bk + (a_max + 1);
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  const int a0 = cta_agg[blockIdx.x], a1 = cta_agg[blockIdx.x + 1];
  const int r0 = row_start[a0], r1 = row_start[a1];
  stage_transfer<TC>(a0, a1, row_start, coarse_start, blk_start, P, psm, m_rs, m_cs, m_bk);
  __syncthreads();
  const CsrView<TC> cv = staged_view<TC>(sg, smraw, r0, r1, rowptr, col, val);
  for (int t = threadIdx.x; t < a1 - a0; t += BS)
    for (int p = m_cs[t]; p < m_cs[t + 1]; ++p) cd2a[p] = t;
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    const size_t o = (size_t)i * K + cl * CPT;
    TC acc[CPT];
    row_acc<TC, TC, K, NZL>(i, valid, cv, u, nzl, cl, acc);
    if (valid && nzl == 0) {
      TC fv[CPT];
      ldv<TC, CPT>(f + o, fv);
#pragma unroll
      for (int t = 0; t < CPT; ++t) fv[t] -= acc[t];
      stv<TC, CPT>(tsm + (size_t)(i - r0) * K + cl * CPT, fv);
    }
  }
  __syncthreads();
  const int c0 = coarse_start[a0];
  if constexpr (K >= 8) {
    // one thread per (aggregate, 4 coarse dofs, column): four outputs in
    // registers, one shared load of t per row, broadcast loads of P
    const int nch = (m_cs_max + 3) / 4;
    const int nwork = (a1 - a0) * nch * K;
    for (int w = threadIdx.x; w < nwork; w += BS) {
      const int c = w % K, q = (w / K) % nch, t = w / (K * nch);
      const int ra = m_cs[t + 1] - m_cs[t], p0 = 4 * q;
      if (p0 >= ra) continue;
      const int rsl = m_rs[t], na = m_rs[t + 1] - rsl;
      const TC* pa = psm + m_bk[t] + p0;
      const TC* ta = tsm + (size_t)rsl * K + c;
      TC acc[4] = {TC(0), TC(0), TC(0), TC(0)};
      for (int i = 0; i < na; ++i) {
        const TC tv = ta[(size_t)i * K];
        const TC* prow = pa + i * ra;
#pragma unroll
        for (int p = 0; p < 4; ++p)
          if (p0 + p < ra) acc[p] = fma(prow[p], tv, acc[p]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        if (p0 + p < ra) {
          const int cd = c0 + m_cs[t] + p0 + p;
          fc[(size_t)cd * K + c] = acc[p];
          if (uc) uc[(size_t)cd * K + c] = acc[p] * __ldg(dinvc + cd);
        }
      }
    }
    return;
  }
  const int nout = m_cs[a1 - a0] * K;
  for (int o = threadIdx.x; o < nout; o += BS) {
    int cdl = o / K, c = o % K;
    int t = cd2a[cdl];
    int p = cdl - m_cs[t], ra = m_cs[t + 1] - m_cs[t];
    int rsl = m_rs[t], na = m_rs[t + 1] - rsl;
    const TC* pa = psm + m_bk[t] + p;
    const TC* ta = tsm + (size_t)rsl * K + c;
    TC s = TC(0);
    for (int i = 0; i < na; ++i) s = fma(pa[i * ra], ta[(size_t)i * K], s);
    size_t oc = (size_t)(c0 + cdl) * K + c;
    fc[oc] = s;
    if (uc) uc[oc] = s * __ldg(dinvc + c0 + cdl);
  }
}

// Restriction with one warp per aggregate: t = f - A u on the aggregate's
// rows (CL lanes per row, RPW rows per pass), fc = P_a^T t accumulated in
// registers (RMAX >= r_a coarse dofs), the row groups of the warp combined
// by shuffles, then uc = D_c^{-1} fc.  No shared-memory tile and no CTA-wide
// barrier.  Memory round trips per pass: the row's own operands (its f
// slice and its P row) and its matrix values are requested together with its
// gathers, and the column indices of the next pass's rows (the first RB of
// each) are requested before this pass's products, so that a pass waits on
// one round trip (its gathers) instead of three.
template <typename TC, int K, int RMAX, bool STG>
__global__ void __launch_bounds__(BS, (RMAX <= 4 && !STG) ? 3 : 2) k_restrict_w(int nagg, const int* __restrict__ row_start,
                                                      const int* __restrict__ coarse_start,
                                                      const long long* __restrict__ blk_start,
                                                      const TC* __restrict__ P, const int* __restrict__ rowptr,
                                                      const int* __restrict__ col, const TC* __restrict__ val,
                                                      const TC* __restrict__ f, const TC* __restrict__ u,
                                                      TC* __restrict__ fc, TC* __restrict__ uc,
                                                      const TC* __restrict__ dinvc, const int* __restrict__ done,
                                                      Stage sg) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, RPW = 32 / CL;
  constexpr int RB = gather_depth<1>();  // entries of a row requested in one batch
  const int lane = threadIdx.x & 31;
  const int g = lane / CL, cl = lane % CL;
  // STG: the CTA's NWARP aggregates are one row range, staged into shared
  // memory first; otherwise the row loop reads global memory (a view fixed at
  // compile time keeps its loads global and its offsets constant)
  const int a0 = blockIdx.x * NWARP, a1 = min(a0 + NWARP, nagg);
  CsrView<TC> cv{rowptr, 0, col, 0, val, 0};
  if constexpr (STG) cv = group_view<TC>(sg, smraw, __ldg(row_start + a0), __ldg(row_start + a1), rowptr, col, val);
  const int a = a0 + (threadIdx.x >> 5);
  if (a >= nagg) return;  // whole warp
  const int rs = __ldg(row_start + a), re = __ldg(row_start + a + 1);
  const int cs = __ldg(coarse_start + a), ra = __ldg(coarse_start + a + 1) - cs;
  const TC* Pa = P + __ldg(blk_start + a);
  // the aggregate's contiguous operands (its f rows, its CSR slice, its P
  // block) are requested into L2 at once, so that the passes after the
  // first wait on L2 instead of DRAM
  if (lane == 0) {
    prefetch_l2(f + (size_t)rs * K, (size_t)(re - rs) * K * sizeof(TC));
    prefetch_l2(Pa, (size_t)(re - rs) * ra * sizeof(TC));
    if constexpr (!STG) {
      const int jb = __ldg(rowptr + rs), je = __ldg(rowptr + re);
      prefetch_l2(col + jb, (size_t)(je - jb) * sizeof(int));
      prefetch_l2(val + jb, (size_t)(je - jb) * sizeof(TC));
    }
  }
  TC acc[RMAX][CPT];
#pragma unroll
  for (int p = 0; p < RMAX; ++p)
#pragma unroll
    for (int t = 0; t < CPT; ++t) acc[p][t] = TC(0);
  // extent and the first RB column indices of a row (-1 past its end)
  auto fetch = [&](int i, bool valid, int& j0, int& j1, int (&c)[RB]) {
    j0 = valid ? cv.rp[i - cv.roff] : 0;
    j1 = valid ? cv.rp[i + 1 - cv.roff] : 0;
#pragma unroll
    for (int b = 0; b < RB; ++b) c[b] = j0 + b < j1 ? cv.col[j0 + b - cv.coff] : -1;
  };
  int c[RB], j0, j1;
  fetch(rs + g, rs + g < re, j0, j1, c);
  for (int base = rs; base < re; base += RPW) {
    const int i = base + g;
    const bool valid = i < re;
    // own operands and matrix values, independent of the gathers
    TC fv[CPT], pv[RMAX], av[RB];
    if (valid) {
      ldv<TC, CPT>(f + (size_t)i * K + cl * CPT, fv);
      const TC* prow = Pa + (size_t)(i - rs) * ra;
#pragma unroll
      for (int p = 0; p < RMAX; ++p) pv[p] = p < ra ? __ldg(prow + p) : TC(0);
    }
#pragma unroll
    for (int b = 0; b < RB; ++b) av[b] = c[b] >= 0 ? cv.val[j0 + b - cv.voff] : TC(0);
    // gathers of the first batch
    TC xv[RB][CPT];
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      if (c[b] >= 0) {
        ldv<TC, CPT>(u + (size_t)c[b] * K + cl * CPT, xv[b]);
      } else {
#pragma unroll
        for (int t = 0; t < CPT; ++t) xv[b][t] = TC(0);
      }
    }
    const int jr = j0 + RB, je = j1;
    // the next pass's column indices, requested before this pass's products
    {
      const int in = i + RPW;
      fetch(in, in < re, j0, j1, c);
    }
    // the products in row order (the order of row_acc)
    TC s[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) s[t] = TC(0);
#pragma unroll
    for (int b = 0; b < RB; ++b)
#pragma unroll
      for (int t = 0; t < CPT; ++t) s[t] = fma(av[b], xv[b][t], s[t]);
    // the rest of a long row, batch by batch
    for (int j = jr; j < je; j += RB) {
      int c2[RB];
      TC a2[RB], x2[RB][CPT];
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const bool ok = j + b < je;
        c2[b] = ok ? cv.col[j + b - cv.coff] : -1;
        a2[b] = ok ? cv.val[j + b - cv.voff] : TC(0);
      }
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        if (c2[b] >= 0) {
          ldv<TC, CPT>(u + (size_t)c2[b] * K + cl * CPT, x2[b]);
        } else {
#pragma unroll
          for (int t = 0; t < CPT; ++t) x2[b][t] = TC(0);
        }
      }
#pragma unroll
      for (int b = 0; b < RB; ++b)
#pragma unroll
        for (int t = 0; t < CPT; ++t) s[t] = fma(a2[b], x2[b][t], s[t]);
    }
    if (valid) {
#pragma unroll
      for (int p = 0; p < RMAX; ++p) {
        if (p < ra) {
#pragma unroll
          for (int t = 0; t < CPT; ++t) acc[p][t] = fma(pv[p], fv[t] - s[t], acc[p][t]);
        }
      }
    }
  }
#pragma unroll
  for (int off = CL; off < 32; off <<= 1)
#pragma unroll
    for (int p = 0; p < RMAX; ++p)
#pragma unroll
      for (int t = 0; t < CPT; ++t) acc[p][t] += __shfl_xor_sync(FULL, acc[p][t], off);
  if (g == 0) {
#pragma unroll
    for (int p = 0; p < RMAX; ++p) {
      if (p < ra) {
        const size_t oc = (size_t)(cs + p) * K + cl * CPT;
        stv<TC, CPT>(fc + oc, acc[p]);
        if (uc) {
          const TC d = __ldg(dinvc + cs + p);
          TC w[CPT];
#pragma unroll
          for (int t = 0; t < CPT; ++t) w[t] = acc[p][t] * d;
          stv<TC, CPT>(uc + oc, w);
        }
      }
    }
  }
}

// ----------------------------------------------- grouped coarse levels --
// On a Galerkin level every coarse dof of one aggregate (a row group) has
// the same column pattern: the coarse dofs of all neighbouring aggregates,
// in one order, S columns per row, the rows of the group stored back to back
// (row p of the group at rowptr[g0] + p S).  The kernels below gather each
// of the S rows of u once per group and apply it to all RA (at most) rows of
// the group, instead of once per row.  A slot of CL * JL lanes owns one
// group: CL lanes split the K columns (CPT each), JL lanes split the S
// pattern columns (lane jl takes j = jl, jl + JL, ...) and are combined by
// shuffles; there are 32 / (CL JL) slots per warp.
constexpr int GATHER_G = 5;    // gathers in flight per lane in the grouped kernels
constexpr int GROUPS_PER_CTA = 32;  // row groups of one grouped-sweep CTA

template <typename TC, int K, int RA, int JL>
__device__ __forceinline__ void group_acc(int r0, int ra, const CsrView<TC>& cv, const TC* __restrict__ x, int cl,
                                          int jl, TC (&acc)[RA][VT<TC, K>::CPT]) {
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, U = GATHER_G;
#pragma unroll
  for (int p = 0; p < RA; ++p)
#pragma unroll
    for (int t = 0; t < CPT; ++t) acc[p][t] = TC(0);
  const int base = cv.rp[r0 - cv.roff], S = cv.rp[r0 + 1 - cv.roff] - base;
  for (int j = jl; j < S; j += U * JL) {
    TC xv[U][CPT];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int jj = j + u * JL;
      if (jj < S) {
        ldv<TC, CPT>(x + (size_t)cv.col[base + jj - cv.coff] * K + cl * CPT, xv[u]);
      } else {
#pragma unroll
        for (int t = 0; t < CPT; ++t) xv[u][t] = TC(0);
      }
    }
#pragma unroll
    for (int p = 0; p < RA; ++p) {
      if (p < ra) {
        const TC* vp = cv.val + base + (size_t)p * S - cv.voff;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int jj = j + u * JL;
          const TC a = jj < S ? vp[jj] : TC(0);
#pragma unroll
          for (int t = 0; t < CPT; ++t) acc[p][t] = fma(a, xv[u][t], acc[p][t]);
        }
      }
    }
  }
  if constexpr (JL > 1) {
#pragma unroll
    for (int off = CL; off < CL * JL; off <<= 1)
#pragma unroll
      for (int p = 0; p < RA; ++p)
#pragma unroll
        for (int t = 0; t < CPT; ++t) acc[p][t] += __shfl_xor_sync(FULL, acc[p][t], off);
  }
}

// v = u + D^{-1} (f - A u) on a grouped level (one l1-Jacobi sweep); a CTA
// takes GROUPS_PER_CTA consecutive groups, its slots walking them in turn.
template <typename TC, int K, int RA, int JL>
__global__ void __launch_bounds__(BS) k_smooth_g(int ngrp, const int* __restrict__ gstart,
                                                 const int* __restrict__ rowptr, const int* __restrict__ col,
                                                 const TC* __restrict__ val, const TC* __restrict__ dinv,
                                                 const TC* __restrict__ f, const TC* __restrict__ u,
                                                 TC* __restrict__ v, const int* __restrict__ done, Stage sg) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, SPW = 32 / (CL * JL), NSLOT = NWARP * SPW;
  const int lane = threadIdx.x & 31, cl = lane % CL, jl = (lane / CL) % JL;
  const int slot = (threadIdx.x >> 5) * SPW + lane / (CL * JL);
  const int ga = blockIdx.x * GROUPS_PER_CTA, gb = min(ga + GROUPS_PER_CTA, ngrp);
  if (threadIdx.x == 0) {
    // the CTA's own rows of f, u and D^{-1} (one contiguous range), read
    // after the gathers: requested into L2 now
    const int ra0 = __ldg(gstart + ga), ra1 = __ldg(gstart + gb);
    prefetch_l2(f + (size_t)ra0 * K, (size_t)(ra1 - ra0) * K * sizeof(TC));
    prefetch_l2(u + (size_t)ra0 * K, (size_t)(ra1 - ra0) * K * sizeof(TC));
    prefetch_l2(dinv + ra0, (size_t)(ra1 - ra0) * sizeof(TC));
  }
  const CsrView<TC> cv = group_view<TC>(sg, smraw, __ldg(gstart + ga), __ldg(gstart + gb), rowptr, col, val);
  // every slot runs the same number of passes (the shuffles inside
  // group_acc need the whole warp); a slot without a group adds nothing
  const int passes = (gb - ga + NSLOT - 1) / NSLOT;
  for (int ps = 0; ps < passes; ++ps) {
    const int g = ga + ps * NSLOT + slot;
    const bool live = g < gb;
    const int r0 = live ? __ldg(gstart + g) : __ldg(gstart + ga), ra = live ? __ldg(gstart + g + 1) - r0 : 0;
    TC acc[RA][CPT];
    group_acc<TC, K, RA, JL>(r0, ra, cv, u, cl, live ? jl : 1 << 30, acc);
    if (!live || jl != 0) continue;
#pragma unroll
    for (int p = 0; p < RA; ++p) {
      if (p < ra) {
        const int i = r0 + p;
        const size_t o = (size_t)i * K + cl * CPT;
        TC fv[CPT], uv[CPT], out[CPT];
        ldv<TC, CPT>(f + o, fv);
        ldv<TC, CPT>(u + o, uv);
        const TC di = __ldg(dinv + i);
#pragma unroll
        for (int t = 0; t < CPT; ++t) out[t] = fma(di, fv[t] - acc[p][t], uv[t]);
        stv<TC, CPT>(v + o, out);
      }
    }
  }
}

// Fused residual + restriction out of a grouped level, one CTA of
// RG_WARPS warps per coarse aggregate: each slot takes row groups of the
// aggregate in turn, forms t = f - A u on the group's rows and accumulates
// fc += P_a^T t over them (RMAX >= r_a coarse dofs); the slots are combined
// by shuffles and then across warps in shared memory, in a fixed order, and
// uc = D_c^{-1} fc is written when the coarse level is smoothed.
constexpr int RG_WARPS = 4;
template <typename TC, int K, int RA, int RMAX, int JL>
__global__ void __launch_bounds__(RG_WARPS * 32) k_restrict_g(
    int nagg, const int* __restrict__ row_start, const int* __restrict__ coarse_start,
    const long long* __restrict__ blk_start, const TC* __restrict__ P, const int* __restrict__ gstart,
    const int* __restrict__ gagg, const int* __restrict__ rowptr, const int* __restrict__ col,
    const TC* __restrict__ val, const TC* __restrict__ f, const TC* __restrict__ u, TC* __restrict__ fc,
    TC* __restrict__ uc, const TC* __restrict__ dinvc, const int* __restrict__ done, Stage sg) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, SPW = 32 / (CL * JL), NSLOT = RG_WARPS * SPW;
  __shared__ TC red[RG_WARPS][RMAX][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, cl = lane % CL, jl = (lane / CL) % JL;
  const int slot = warp * SPW + lane / (CL * JL);
  const int a = blockIdx.x;
  const int rs = __ldg(row_start + a), cs = __ldg(coarse_start + a), rc = __ldg(coarse_start + a + 1) - cs;
  const TC* Pa = P + __ldg(blk_start + a);
  if (threadIdx.x == 0) {
    // the aggregate's own rows of f and its P block, read after the
    // gathers: requested into L2 now
    const int re = __ldg(row_start + a + 1);
    prefetch_l2(f + (size_t)rs * K, (size_t)(re - rs) * K * sizeof(TC));
    prefetch_l2(Pa, (size_t)(re - rs) * rc * sizeof(TC));
  }
  const CsrView<TC> cv = group_view<TC>(sg, smraw, rs, __ldg(row_start + a + 1), rowptr, col, val);
  TC accp[RMAX][CPT];
#pragma unroll
  for (int q = 0; q < RMAX; ++q)
#pragma unroll
    for (int t = 0; t < CPT; ++t) accp[q][t] = TC(0);
  const int g0 = __ldg(gagg + a), g1 = __ldg(gagg + a + 1);
  // every slot runs the same number of passes (the shuffles inside group_acc
  // need the whole warp); a slot without a group in a pass adds nothing
  const int passes = (g1 - g0 + NSLOT - 1) / NSLOT;
  for (int ps = 0; ps < passes; ++ps) {
    const int g = g0 + ps * NSLOT + slot;
    const bool live = g < g1;
    const int r0 = live ? __ldg(gstart + g) : rs, ra = live ? __ldg(gstart + g + 1) - r0 : 0;
    TC acc[RA][CPT];
    group_acc<TC, K, RA, JL>(r0, ra, cv, u, cl, live ? jl : 1 << 30, acc);
    if (jl == 0) {
#pragma unroll
      for (int p = 0; p < RA; ++p) {
        if (p < ra) {
          const int i = r0 + p;
          TC fv[CPT];
          ldv<TC, CPT>(f + (size_t)i * K + cl * CPT, fv);
          const TC* prow = Pa + (size_t)(i - rs) * rc;
#pragma unroll
          for (int q = 0; q < RMAX; ++q) {
            if (q < rc) {
              const TC pv = __ldg(prow + q);
#pragma unroll
              for (int t = 0; t < CPT; ++t) accp[q][t] = fma(pv, fv[t] - acc[p][t], accp[q][t]);
            }
          }
        }
      }
    }
  }
  // lanes with jl != 0 hold zeros; combine the slots of the warp
#pragma unroll
  for (int off = CL; off < 32; off <<= 1)
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
#pragma unroll
      for (int t = 0; t < CPT; ++t) accp[q][t] += __shfl_xor_sync(FULL, accp[q][t], off);
  if (lane < CL)
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
#pragma unroll
      for (int t = 0; t < CPT; ++t) red[warp][q][cl * CPT + t] = accp[q][t];
  __syncthreads();
  for (int e = threadIdx.x; e < rc * K; e += RG_WARPS * 32) {
    const int q = e / K, c = e % K;
    TC s = red[0][q][c];
#pragma unroll
    for (int w = 1; w < RG_WARPS; ++w) s += red[w][q][c];
    const size_t oc = (size_t)(cs + q) * K + c;
    fc[oc] = s;
    if (uc) uc[oc] = s * __ldg(dinvc + cs + q);
  }
}

// --------------------------------- restriction by R = P^T (I - A D^{-1}) --
// With one pre-sweep from zero the iterate that enters the restriction is
// u = D^{-1} f, so fc = P^T (f - A u) = R f with R = P^T (I - A D^{-1}).
// All coarse dofs of one aggregate share R's column pattern: the rows that
// the aggregate's rows of A reach (its halo).  R is stored by aggregate:
// pattern columns rcol[rptr[a] .. rptr[a+1]) and, per pattern entry, RS
// values (one per coarse dof of the aggregate, zero-padded to RS).  A warp
// takes one aggregate at a time (a, then a plus the warps of the grid): CL
// lanes split the K columns, JL = 32 / CL lane groups split the pattern, U
// entries per lane group and batch, every gather and value load of a batch
// requested before its first product.  The next batch's columns (or the next
// aggregate's first) are requested before the products, the extents two
// aggregates ahead.  Each halo row of f is gathered once per aggregate,
// where the CSR restriction gathers it once per non-zero of A.

// Entries per lane group and batch: what keeps the gathered rows, the
// values and the accumulators of a lane near 100 registers.
template <typename TC, int K, int RS>
__host__ __device__ constexpr int rf_batch() {
  constexpr int w = (int)sizeof(TC) / 4;
  constexpr int acc = RS * VT<TC, K>::CPT * w, per = (VT<TC, K>::CPT + RS) * w;
  constexpr int u = (100 - acc) / per;
  return u < 1 ? 1 : (u > 9 ? 9 : u);
}

// The same walk serves the l1-Jacobi sweep of a grouped level (EPI 1):
// there the groups are the level's row groups (the coarse dofs of one
// aggregate of the level above, one shared pattern) with an entry-major copy
// of the level's values, the gathered vector is the iterate u, and the
// epilogue writes v = u + D^{-1} (f - A u) on the group's rows.
// EPI 0: ostart = coarse_start, x = f, out = fc, out2 = uc (may be null),
//        d = D_c^{-1}.
// EPI 1: ostart = the row groups' starts, x = u, out = v, d = D^{-1},
//        fo = f (u's own rows are read from x).
template <typename TC, int K, int RS, int EPI>
__global__ void __launch_bounds__(BS, 2) k_group_rf(int ngrp, const int* __restrict__ rptr,
                                                    const int* __restrict__ rcol, const TC* __restrict__ rval,
                                                    const int* __restrict__ ostart, const TC* __restrict__ x,
                                                    TC* __restrict__ out, TC* __restrict__ out2,
                                                    const TC* __restrict__ d, const TC* __restrict__ fo,
                                                    const int* __restrict__ done) {
  if (*done) return;
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, JL = 32 / CL, U = rf_batch<TC, K, RS>();
  constexpr int VP = (16 / (int)sizeof(TC)) < RS ? 16 / (int)sizeof(TC) : RS;  // values per vector load
  const int lane = threadIdx.x & 31, cl = lane % CL, jl = lane / CL;
  const int nw = gridDim.x * NWARP;
  int a = blockIdx.x * NWARP + (threadIdx.x >> 5);
  auto extent = [&](int g, int& e0, int& e1) {
    e0 = g < ngrp ? __ldg(rptr + g) : 0;
    e1 = g < ngrp ? __ldg(rptr + g + 1) : 0;
  };
  // columns of the batch at jb for this lane group (-1 past the pattern)
  auto cols = [&](int jb, int e1, int(&c)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int jj = jb + jl + u * JL;
      c[u] = jj < e1 ? __ldg(rcol + jj) : -1;
    }
  };
  int b0, b1, n0, n1;
  extent(a, b0, b1);
  extent(a + nw, n0, n1);
  int c[U];
  cols(b0, b1, c);
  for (; a < ngrp; a += nw) {
    int m0, m1;
    extent(a + 2 * nw, m0, m1);
    const int c0 = __ldg(ostart + a), ra = __ldg(ostart + a + 1) - c0;
    TC acc[RS][CPT];
#pragma unroll
    for (int p = 0; p < RS; ++p)
#pragma unroll
      for (int t = 0; t < CPT; ++t) acc[p][t] = TC(0);
    for (int jb = b0;; jb += U * JL) {
      TC xv[U][CPT], vv[U][RS];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c[u] >= 0) {
          ldv<TC, CPT>(x + (size_t)c[u] * K + cl * CPT, xv[u]);
        } else {
#pragma unroll
          for (int t = 0; t < CPT; ++t) xv[u][t] = TC(0);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const TC* src = rval + (size_t)(jb + jl + u * JL) * RS;
#pragma unroll
        for (int q = 0; q < RS; q += VP) {
          TC piece[VP];
          if (c[u] >= 0) {
            ldv<TC, VP>(src + q, piece);
          } else {
#pragma unroll
            for (int e = 0; e < VP; ++e) piece[e] = TC(0);
          }
#pragma unroll
          for (int e = 0; e < VP; ++e) vv[u][q + e] = piece[e];
        }
      }
      // warp-uniform: whether this group has another batch
      const bool more = jb + U * JL < b1;
      if (more) cols(jb + U * JL, b1, c);
      else cols(n0, n1, c);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int p = 0; p < RS; ++p)
#pragma unroll
          for (int t = 0; t < CPT; ++t) acc[p][t] = fma(vv[u][p], xv[u][t], acc[p][t]);
      if (!more) break;
    }
    // the lane groups' partial sums, combined by a butterfly (every lane
    // ends with the same sums)
#pragma unroll
    for (int off = CL; off < 32; off <<= 1)
#pragma unroll
      for (int p = 0; p < RS; ++p)
#pragma unroll
        for (int t = 0; t < CPT; ++t) acc[p][t] += __shfl_xor_sync(FULL, acc[p][t], off);
#pragma unroll
    for (int p = 0; p < RS; ++p) {
      if (p < ra && p % JL == jl) {
        const size_t oc = (size_t)(c0 + p) * K + cl * CPT;
        if constexpr (EPI == 0) {
          stv<TC, CPT>(out + oc, acc[p]);
          if (out2) {
            const TC dp = __ldg(d + c0 + p);
            TC w[CPT];
#pragma unroll
            for (int t = 0; t < CPT; ++t) w[t] = acc[p][t] * dp;
            stv<TC, CPT>(out2 + oc, w);
          }
        } else {
          const TC dp = __ldg(d + c0 + p);
          TC fv[CPT], uv[CPT], w[CPT];
          ldv<TC, CPT>(fo + oc, fv);
          ldv<TC, CPT>(x + oc, uv);
#pragma unroll
          for (int t = 0; t < CPT; ++t) w[t] = fma(dp, fv[t] - acc[p][t], uv[t]);
          stv<TC, CPT>(out + oc, w);
        }
      }
    }
    b0 = n0;
    b1 = n1;
    n0 = m0;
    n1 = m1;
  }
}

// The slot form of the same product.  Patterns are padded to a multiple of
// RF_PAD entries (a valid column with zero values) and a batch of RF_PAD zero
// entries follows the last group (at zero_e), so that every batch is full
// and a slot past the end of its pattern reads the zero batch instead of
// taking a branch.  A slot of CL lanes walks one group alone, U entries per
// batch (U divides RF_PAD), 32 / CL slots per warp on consecutive groups; the
// warp runs as many batches as its longest group, and no lane-group sums are
// combined.  The columns of the next batch (or of the next pass's first) are
// requested with the current batch, the extents two passes ahead.
constexpr int RF_PAD = 8;
template <typename TC, int K, int RS>
__host__ __device__ constexpr int rs_batch() {
  constexpr int w = (int)sizeof(TC) / 4;
  constexpr int acc = RS * VT<TC, K>::CPT * w, per = (VT<TC, K>::CPT + RS) * w;
  return acc + 8 * per <= 100 ? 8 : (acc + 4 * per <= 100 ? 4 : (acc + 2 * per <= 100 ? 2 : 1));
}
template <int U>
__device__ __forceinline__ void ld_cols(const int* __restrict__ p, int (&c)[U]) {
  if constexpr (U == 8) {
    const int4 a = __ldg(reinterpret_cast<const int4*>(p)), b = __ldg(reinterpret_cast<const int4*>(p) + 1);
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
  } else if constexpr (U == 4) {
    const int4 a = __ldg(reinterpret_cast<const int4*>(p));
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
  } else if constexpr (U == 2) {
    const int2 a = __ldg(reinterpret_cast<const int2*>(p));
    c[0] = a.x; c[1] = a.y;
  } else {
    c[0] = __ldg(p);
  }
}
template <typename TC, int K, int RS, int EPI>
__global__ void __launch_bounds__(BS, 2) k_group_rs(int ngrp, int zero_e, const int* __restrict__ rptr,
                                                    const int* __restrict__ rcol, const TC* __restrict__ rval,
                                                    const int* __restrict__ ostart, const TC* __restrict__ x,
                                                    TC* __restrict__ out, TC* __restrict__ out2,
                                                    const TC* __restrict__ d, const TC* __restrict__ fo,
                                                    const int* __restrict__ done) {
  if (*done) return;
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, SPW = 32 / CL, U = rs_batch<TC, K, RS>();
  constexpr int VP = (16 / (int)sizeof(TC)) < RS ? 16 / (int)sizeof(TC) : RS;  // values per vector load
  static_assert(RF_PAD % U == 0, "a batch must divide the pattern padding");
  const int lane = threadIdx.x & 31, cl = lane % CL, slot = lane / CL;
  const int nw = gridDim.x * NWARP, npass = (ngrp + SPW - 1) / SPW;
  int pass = blockIdx.x * NWARP + (threadIdx.x >> 5);
  // this slot's group in pass q: first entry and number of batches
  auto extent = [&](int q, int& e0, int& nb) {
    const int g = q * SPW + slot;
    if (g < ngrp) {
      e0 = __ldg(rptr + g);
      nb = (__ldg(rptr + g + 1) - e0) / U;
    } else {
      e0 = zero_e;
      nb = 0;
    }
  };
  int e0, nb, f0, fnb;
  extent(pass, e0, nb);
  extent(pass + nw, f0, fnb);
  int c[U];
  ld_cols<U>(rcol + (nb > 0 ? e0 : zero_e), c);
  for (; pass < npass; pass += nw) {
    int h0, hnb;
    extent(pass + 2 * nw, h0, hnb);
    const int g = pass * SPW + slot;
    const int c0 = g < ngrp ? __ldg(ostart + g) : 0, ra = g < ngrp ? __ldg(ostart + g + 1) - c0 : 0;
    if constexpr (EPI == 1) {
      // the group's own rows of f and u, read after the batches: into L2 now
      if (cl == 0 && ra > 0) {
        prefetch_l2(fo + (size_t)c0 * K, (size_t)ra * K * sizeof(TC));
        prefetch_l2(x + (size_t)c0 * K, (size_t)ra * K * sizeof(TC));
      }
    }
    const int nbw = (int)__reduce_max_sync(FULL, (unsigned)nb);
    TC acc[RS][CPT];
#pragma unroll
    for (int p = 0; p < RS; ++p)
#pragma unroll
      for (int t = 0; t < CPT; ++t) acc[p][t] = TC(0);
    for (int b = 0; b < nbw; ++b) {
      const int eb = b < nb ? e0 + b * U : zero_e;
      TC xv[U][CPT], vv[U][RS];
#pragma unroll
      for (int u = 0; u < U; ++u) ldv<TC, CPT>(x + (size_t)c[u] * K + cl * CPT, xv[u]);
#pragma unroll
      for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int q = 0; q < RS; q += VP) {
          TC piece[VP];
          ldv<TC, VP>(rval + (size_t)(eb + u) * RS + q, piece);
#pragma unroll
          for (int e = 0; e < VP; ++e) vv[u][q + e] = piece[e];
        }
      }
      const int en = b + 1 < nbw ? (b + 1 < nb ? e0 + (b + 1) * U : zero_e) : (fnb > 0 ? f0 : zero_e);
      ld_cols<U>(rcol + en, c);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int p = 0; p < RS; ++p)
#pragma unroll
          for (int t = 0; t < CPT; ++t) acc[p][t] = fma(vv[u][p], xv[u][t], acc[p][t]);
    }
    if (nbw == 0) ld_cols<U>(rcol + (fnb > 0 ? f0 : zero_e), c);
#pragma unroll
    for (int p = 0; p < RS; ++p) {
      if (p < ra) {
        const size_t oc = (size_t)(c0 + p) * K + cl * CPT;
        if constexpr (EPI == 0) {
          stv<TC, CPT>(out + oc, acc[p]);
          if (out2) {
            const TC dp = __ldg(d + c0 + p);
            TC w[CPT];
#pragma unroll
            for (int t = 0; t < CPT; ++t) w[t] = acc[p][t] * dp;
            stv<TC, CPT>(out2 + oc, w);
          }
        } else {
          const TC dp = __ldg(d + c0 + p);
          TC fv[CPT], uv[CPT], w[CPT];
          ldv<TC, CPT>(fo + oc, fv);
          ldv<TC, CPT>(x + oc, uv);
#pragma unroll
          for (int t = 0; t < CPT; ++t) w[t] = fma(dp, fv[t] - acc[p][t], uv[t]);
          stv<TC, CPT>(out + oc, w);
        }
      }
    }
    e0 = f0;
    nb = fnb;
    f0 = h0;
    fnb = hnb;
  }
}

// u[rows(a)] += P_a uc[coarse(a)]   (aggregate-aligned CTAs)
template <typename TC, int K>
__global__ void __launch_bounds__(BS) k_prolong(const int* __restrict__ cta_agg, const int* __restrict__ row_start,
                                                const int* __restrict__ coarse_start,
                                                const long long* __restrict__ blk_start, const TC* __restrict__ P,
                                                const TC* __restrict__ uc, TC* __restrict__ u,
                                                const int* __restrict__ done, int rows_max, int p_max,
                                                int a_max, const TC* __restrict__ f0,
                                                const TC* __restrict__ dinv0) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  TC* psm = reinterpret_cast<TC*>(smraw);
  int* m_rs = reinterpret_cast<int*>(smraw + align16((size_t)p_max * sizeof(TC)));
  int* m_cs = m_rs + (a_max + 1);
  int* m_bk = m_cs + (a_max + 1);
  int* r2a = m_bk + (a_max + 1);
  constexpr int CPT = VT<TC, K>::CPT, NV = K / CPT;
  const int a0 = cta_agg[blockIdx.x], a1 = cta_agg[blockIdx.x + 1];
  const int r0 = row_start[a0], c0 = coarse_start[a0];
  stage_transfer<TC>(a0, a1, row_start, coarse_start, blk_start, P, psm, m_rs, m_cs, m_bk);
  __syncthreads();
  for (int t = threadIdx.x; t < a1 - a0; t += BS)
    for (int il = m_rs[t]; il < m_rs[t + 1]; ++il) r2a[il] = t;
  __syncthreads();
  const int nout = m_rs[a1 - a0] * NV;
  for (int o = threadIdx.x; o < nout; o += BS) {
    int il = o / NV, c = (o % NV) * CPT;
    int t = r2a[il];
    int ra = m_cs[t + 1] - m_cs[t];
    const TC* pr = psm + m_bk[t] + (il - m_rs[t]) * ra;
    const TC* ucp = uc + (size_t)(c0 + m_cs[t]) * K + c;
    TC s[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) s[q] = TC(0);
    for (int p = 0; p < ra; ++p) {
      TC pv = pr[p];
      TC cv[CPT];
      ldv<TC, CPT>(ucp + (size_t)p * K, cv);
#pragma unroll
      for (int q = 0; q < CPT; ++q) s[q] = fma(pv, cv[q], s[q]);
    }
    TC* up = u + (size_t)(r0 + il) * K + c;
    TC uv[CPT];
    if (f0) {  // u = D^{-1} f (the first pre-sweep from zero, not stored) before the correction
      TC fv[CPT];
      ldv<TC, CPT>(f0 + (size_t)(r0 + il) * K + c, fv);
      const TC d = __ldg(dinv0 + r0 + il);
#pragma unroll
      for (int q = 0; q < CPT; ++q) uv[q] = d * fv[q];
    } else {
      ldp<TC, CPT>(up, uv);
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) uv[q] += s[q];
    stv<TC, CPT>(up, uv);
  }
}

// u[rows(a)] += P_a uc[coarse(a)] with one warp per aggregate: CL lanes
// per row (CPT columns each), 32 / CL rows per pass.  Each lane reads its
// columns of the aggregate's RMAX (>= r_a) coarse values once and keeps them
// in registers; two rows are loaded before either is updated.
template <typename TC, int K, int RMAX>
__global__ void __launch_bounds__(BS) k_prolong_w(int nagg, const int* __restrict__ row_start,
                                                  const int* __restrict__ coarse_start,
                                                  const long long* __restrict__ blk_start,
                                                  const TC* __restrict__ P, const TC* __restrict__ uc,
                                                  TC* __restrict__ u, const int* __restrict__ done,
                                                  const TC* __restrict__ f0, const TC* __restrict__ dinv0) {
  if (*done) return;
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, RPW = 32 / CL;
  const int lane = threadIdx.x & 31, cl = lane % CL;
  const int a = blockIdx.x * NWARP + (threadIdx.x >> 5);
  if (a >= nagg) return;  // no warp-wide collectives below
  const int rs = __ldg(row_start + a), re = __ldg(row_start + a + 1);
  const int cs = __ldg(coarse_start + a), ra = __ldg(coarse_start + a + 1) - cs;
  const TC* Pa = P + __ldg(blk_start + a);
  TC cv[RMAX][CPT];
#pragma unroll
  for (int p = 0; p < RMAX; ++p) {
    if (p < ra) {
      ldv<TC, CPT>(uc + (size_t)(cs + p) * K + cl * CPT, cv[p]);
    } else {
#pragma unroll
      for (int t = 0; t < CPT; ++t) cv[p][t] = TC(0);
    }
  }
  for (int i = rs + lane / CL; i < re; i += 2 * RPW) {
    const int i2 = i + RPW;
    const bool two = i2 < re;
    TC pv[2][RMAX], uv[2][CPT];
#pragma unroll
    for (int p = 0; p < RMAX; ++p) {
      pv[0][p] = p < ra ? __ldg(Pa + (size_t)(i - rs) * ra + p) : TC(0);
      pv[1][p] = (two && p < ra) ? __ldg(Pa + (size_t)(i2 - rs) * ra + p) : TC(0);
    }
    if (f0) {  // u = D^{-1} f (the first pre-sweep from zero, not stored) before the correction
      TC fv[2][CPT];
      ldv<TC, CPT>(f0 + (size_t)i * K + cl * CPT, fv[0]);
      if (two) ldv<TC, CPT>(f0 + (size_t)i2 * K + cl * CPT, fv[1]);
      const TC d0 = __ldg(dinv0 + i), d1 = two ? __ldg(dinv0 + i2) : TC(0);
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        uv[0][t] = d0 * fv[0][t];
        uv[1][t] = two ? d1 * fv[1][t] : TC(0);
      }
    } else {
      ldp<TC, CPT>(u + (size_t)i * K + cl * CPT, uv[0]);
      if (two) ldp<TC, CPT>(u + (size_t)i2 * K + cl * CPT, uv[1]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // the same order as k_prolong: P_a row . uc, then added to u
      TC sv[CPT];
#pragma unroll
      for (int t = 0; t < CPT; ++t) sv[t] = TC(0);
#pragma unroll
      for (int p = 0; p < RMAX; ++p)
        if (p < ra)
#pragma unroll
          for (int t = 0; t < CPT; ++t) sv[t] = fma(pv[h][p], cv[p][t], sv[t]);
#pragma unroll
      for (int t = 0; t < CPT; ++t) uv[h][t] += sv[t];
    }
    stv<TC, CPT>(u + (size_t)i * K + cl * CPT, uv[0]);
    if (two) stv<TC, CPT>(u + (size_t)i2 * K + cl * CPT, uv[1]);
  }
}

// Coarsest level: u = A_c^{-1} f with the float64 inverse of each diagonal
// block; one thread per (row, column) with float64 accumulation, spread over
// many small CTAs (the float64 pipes of GB300 are narrow).
constexpr int COARSE_BS = 64;
template <typename TC, int K>
__global__ void __launch_bounds__(COARSE_BS) k_coarse(int n, int nblk, const int* __restrict__ blk_off,
                                                      const long long* __restrict__ inv_off,
                                                      const double* __restrict__ inv, const TC* __restrict__ f,
                                                      TC* __restrict__ u, const int* __restrict__ done) {
  if (*done) return;
  const long long t = (long long)blockIdx.x * COARSE_BS + threadIdx.x;
  if (t >= (long long)n * K) return;
  const int row = (int)(t / K), c = (int)(t % K);
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(blk_off + mid) <= row) lo = mid; else hi = mid - 1;
  }
  const int b0 = __ldg(blk_off + lo), nb = __ldg(blk_off + lo + 1) - b0;
  const double* Ar = inv + __ldg(inv_off + lo) + (size_t)(row - b0) * nb;
  const TC* fc = f + (size_t)b0 * K + c;
  // even and odd terms in two sums, in order; eight terms' loads requested
  // before their products
  double s0 = 0.0, s1 = 0.0;
  int j = 0;
  for (; j + 8 <= nb; j += 8) {
    double a[8], x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      a[q] = __ldg(Ar + j + q);
      x[q] = (double)__ldg(fc + (size_t)(j + q) * K);
    }
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      s0 = fma(a[q], x[q], s0);
      s1 = fma(a[q + 1], x[q + 1], s1);
    }
  }
  for (; j + 1 < nb; j += 2) {
    s0 = fma(__ldg(Ar + j), (double)__ldg(fc + (size_t)j * K), s0);
    s1 = fma(__ldg(Ar + j + 1), (double)__ldg(fc + (size_t)(j + 1) * K), s1);
  }
  if (j < nb) s0 = fma(__ldg(Ar + j), (double)__ldg(fc + (size_t)j * K), s0);
  u[(size_t)row * K + c] = (TC)(s0 + s1);
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
// Last CTA of an update launch: the stopping test of every active column
// (||r|| <= rtol ||b||, non-finite -> breakdown, iteration limit), the
// iteration counter and the all-stopped flag.
template <int K>
__device__ __forceinline__ void finish_update(KState& ks, double* sm, double* tot) {
  const int it = *ks.iter + 1;
  for (int sy = 0; sy < ks.nsys; ++sy) {
    system_totals(ks, K, sy, sm, tot);
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
    int stopped = 1;
    for (int v = 0; v < ks.nsys * K; ++v)
      if (ks.conv[v] == ST_ACTIVE) stopped = 0;
    *ks.iter = it;
    if (stopped) *ks.done = 1;
  }
}

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
  if (!arrive_two_level(ks, RED_UPDATE, K, sm, tot)) return;
  finish_update<K>(ks, sm, tot);
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
// rho = r.z; mode 2: no scalars (a bare V-cycle).  UQ: the gather batch of
// row_acc (9 when no row has more entries).
template <typename TC, int K, int NZL, bool DF, bool STG, int UQ = 0>
__global__ void __launch_bounds__(BS) k_post0(const int* __restrict__ cta_row, const int* __restrict__ rowptr,
                                              const int* __restrict__ col, const TC* __restrict__ val,
                                              const TC* __restrict__ dinv, const TC* __restrict__ f,
                                              const TC* __restrict__ u, const double* __restrict__ r,
                                              const float* __restrict__ rlo, TC* __restrict__ z, KState ks,
                                              int mode, Stage sg, int nchunk) {
  if (*ks.done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sm[BS];
  __shared__ double tot[64];
  constexpr int CPT = VT<TC, K>::CPT, CL = VT<TC, K>::CL, G = NZL * CL, RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, lg = lane % G, nzl = lg / CL, cl = lg % CL;
  // DF: r = f + rlo exactly (double-float CG) and r.z is accumulated in
  // double-float in per-thread shared-memory slots (registers stay free for
  // the gathers); otherwise r is float64 and r.z a float64 register sum
  constexpr int ND = DF ? 1 : CPT, NF = DF ? CPT : 1;
  // DF with an even column count: the r.z steps run on column pairs (the
  // f32x2 forms, each half rounded as its scalar form), slots in sdot2
  constexpr bool PD = DF && CPT % 2 == 0;
  constexpr int NQ = PD ? CPT / 2 : 1;
  __shared__ float sdot[PD ? 1 : 2 * NF][BS];
  __shared__ F2 sdot2[2 * NQ][PD ? BS : 1];
  double d[ND];
#pragma unroll
  for (int t = 0; t < ND; ++t) d[t] = 0;
  if constexpr (PD) {
#pragma unroll
    for (int q = 0; q < 2 * NQ; ++q) sdot2[q][threadIdx.x] = F2{0ull};
  } else if constexpr (DF) {
#pragma unroll
    for (int t = 0; t < 2 * NF; ++t) sdot[t][threadIdx.x] = 0.f;
  }
  // one row range per CTA, or (persistent launch, one system) every
  // gridDim.x-th range; float matrices are staged through the double-buffered
  // pipeline (the next range arrives while this one is processed)
  // STG: the staged variants (a view fixed at compile time keeps the
  // unstaged loads global with constant offsets)
  constexpr bool PIPE = sizeof(TC) == 4 && STG;
  const bool piped = PIPE && sg.enabled;
  if (piped) {
    pipe_init(smraw);
    if (threadIdx.x == 0 && (int)blockIdx.x < nchunk) {
      const float* v1[1] = {reinterpret_cast<const float*>(val)};
      pipe_issue<1>(sg, smraw, 0, cta_row[blockIdx.x], cta_row[blockIdx.x + 1], rowptr, col, v1);
    }
  }
  int it = 0;
  for (int chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x, ++it) {
  const int r0 = cta_row[chunk], r1 = cta_row[chunk + 1];
  CsrView<TC> cv;
  if (piped) {
    const int nxt = chunk + gridDim.x;
    if (threadIdx.x == 0 && nxt < nchunk) {
      const float* v1[1] = {reinterpret_cast<const float*>(val)};
      pipe_issue<1>(sg, smraw, (it + 1) & 1, cta_row[nxt], cta_row[nxt + 1], rowptr, col, v1);
    }
    const int* prp;
    const int* pcs;
    const float* pv[1];
    int roff, joff;
    pipe_wait<1>(sg, smraw, it & 1, it >> 1, r0, rowptr, prp, roff, pcs, pv, joff);
    cv = CsrView<TC>{prp, roff, pcs, joff, reinterpret_cast<const TC*>(pv[0]), joff};
  } else if constexpr (STG) {
    cv = staged_view<TC>(sg, smraw, r0, r1, rowptr, col, val);
  } else {
    cv = CsrView<TC>{rowptr, 0, col, 0, val, 0};
  }
  for (int base = r0 + warp * RPW; base < r1; base += NWARP * RPW) {
    int i = base + g;
    bool valid = i < r1;
    const size_t o = (size_t)i * K + cl * CPT;
    // the row's own operands are requested before its gathers
    TC fv[CPT], uv[CPT];
    float lv[NF];
    if (valid && nzl == 0) {
      ldv<TC, CPT>(f + o, fv);
      ldv<TC, CPT>(u + o, uv);
      if constexpr (DF) ldv<float, CPT>(rlo + o, lv);
    }
    TC acc[CPT];
    row_acc<TC, TC, K, NZL, UQ>(i, valid, cv, u, nzl, cl, acc);
    if constexpr (DF) {
      if (valid && nzl == 0) {
        TC zt[CPT];
        TC di = __ldg(dinv + i);
#pragma unroll
        for (int t = 0; t < CPT; ++t) zt[t] = fma(di, fv[t] - acc[t], uv[t]);
        stv<TC, CPT>(z + o, zt);
        if constexpr (PD) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            F2 h = sdot2[q][threadIdx.x], l = sdot2[NQ + q][threadIdx.x];
            df_acc1_x2(f2_pack((float)fv[2 * q], (float)fv[2 * q + 1]), f2_pack(lv[2 * q], lv[2 * q + 1]),
                       f2_pack((float)zt[2 * q], (float)zt[2 * q + 1]), h, l);
            sdot2[q][threadIdx.x] = h;
            sdot2[NQ + q][threadIdx.x] = l;
          }
        } else {
#pragma unroll
          for (int t = 0; t < CPT; ++t) {
            float h = sdot[t][threadIdx.x], l = sdot[NF + t][threadIdx.x];
            df_acc1((float)fv[t], lv[t], (float)zt[t], h, l);
            sdot[t][threadIdx.x] = h;
            sdot[NF + t][threadIdx.x] = l;
          }
        }
      }
    } else if (valid && nzl == 0) {
      TC di = __ldg(dinv + i);
      TC zt[CPT];
      double rv[CPT];
      if constexpr (CPT >= 2) {
#pragma unroll
        for (int t = 0; t < CPT; t += 2) {
          double two[2];
          ldv<double, 2>(r + o + t, two);
          rv[t] = two[0];
          rv[t + 1] = two[1];
        }
      } else {
        rv[0] = __ldg(r + o);
      }
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        zt[t] = fma(di, fv[t] - acc[t], uv[t]);
        d[t] = fma(rv[t], (double)zt[t], d[t]);
      }
      stv<TC, CPT>(z + o, zt);
    }
  }
  if (piped) __syncthreads();  // the buffer is refilled two ranges on
  }
  if (mode == 2) return;
  double dd[CPT];
  if constexpr (PD) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float h0, h1, l0, l1;
      f2_unpack(sdot2[q][threadIdx.x], h0, h1);
      f2_unpack(sdot2[NQ + q][threadIdx.x], l0, l1);
      dd[2 * q] = (double)h0 + (double)l0;
      dd[2 * q + 1] = (double)h1 + (double)l1;
    }
  } else {
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      if constexpr (DF) {
        dd[t] = (double)sdot[t][threadIdx.x] + (double)sdot[NF + t][threadIdx.x];
      } else {
        dd[t] = d[t];
      }
    }
  }
  // lanes other than nzl == 0 hold zeros; reduce across the whole warp
  cta_colsum<K, CPT>(dd, sm, ks.partial + (size_t)blockIdx.x * K);
  if (!arrive_two_level(ks, RED_POST, K, sm, tot)) return;
  for (int sy = 0; sy < ks.nsys; ++sy) {
    system_totals(ks, K, sy, sm, tot);
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
  }
}

}  // namespace amg

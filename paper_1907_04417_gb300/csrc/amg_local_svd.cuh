// Eq. (svd) for one aggregate, computed by one warp: the body shared by the
// setup's kernel (k_local_svd) and the allocation-free entry point
// (amg_local_bases_static), so that the two give the same bases.
#pragma once

#include <cuda_runtime.h>

namespace amg {

__device__ __forceinline__ double svd_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Thin SVD of the n_a x m block Wa (row-major) by one-sided (Hestenes)
// Jacobi rotations of its columns in the work block X (n_a x m), the
// singular values sorted in descending order, the columns with
// sigma > tol * n_a / nf kept (at least one, at most min(n_a, m)), each
// normalised and flipped so that its largest-magnitude entry (lowest row on
// ties) is positive.  A zero block gives the normalised constant.  Writes
// the kept columns into columns 0..r-1 of Ua (n_a x m row-major) and
// returns r.  Every lane of the warp calls it with the same arguments.
__device__ __forceinline__ int local_svd_warp(const double* __restrict__ Wa, int m, int na, int nf, double tol,
                                              double* __restrict__ X, double* __restrict__ Ua, int lane) {
  for (int t = lane; t < na * m; t += 32) X[t] = Wa[t];
  __syncwarp();
  for (int sweep = 0; sweep < 40; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        double al = 0, be = 0, ga = 0;
        for (int i = lane; i < na; i += 32) {
          double x = X[i * m + p], y = X[i * m + q];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = svd_warp_sum(al);
        be = svd_warp_sum(be);
        ga = svd_warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > 1e-15 * sqrt(al * be)) {
          double zeta = (be - al) / (2.0 * ga);
          double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          for (int i = lane; i < na; i += 32) {
            double x = X[i * m + p], y = X[i * m + q];
            X[i * m + p] = c * x - s * y;
            X[i * m + q] = s * x + c * y;
          }
          rotated = 1;
        }
        __syncwarp();
      }
    }
    if (!rotated) break;
  }
  double sig[16];
  int idx[16];
  for (int j = 0; j < m; ++j) {
    double s = 0;
    for (int i = lane; i < na; i += 32) s = fma(X[i * m + j], X[i * m + j], s);
    sig[j] = sqrt(svd_warp_sum(s));
    idx[j] = j;
  }
  for (int j = 1; j < m; ++j) {  // stable insertion sort, descending
    int v = idx[j];
    int t = j;
    while (t > 0 && sig[idx[t - 1]] < sig[v]) {
      idx[t] = idx[t - 1];
      --t;
    }
    idx[t] = v;
  }
  int rmax = na < m ? na : m;
  double thr = tol * (double)na / (double)nf;
  int r = 0;
  for (int j = 0; j < rmax; ++j)
    if (sig[idx[j]] > thr) ++r;
  if (r == 0) r = 1;
  for (int j = 0; j < r; ++j) {
    int c = idx[j];
    double s = sig[c];
    bool zero = !(s > 0.0);
    double scale = zero ? 0.0 : 1.0 / s;
    double cst = 1.0 / sqrt((double)na);
    double best = -1.0;
    int bi = 0x7fffffff;
    double bv = 0;
    for (int i = lane; i < na; i += 32) {
      double v = zero ? cst : X[i * m + c] * scale;
      double av = fabs(v);
      if (av > best) {  // rows visited in increasing order: keeps the lowest on ties
        best = av;
        bi = i;
        bv = v;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
        bv = ov;
      }
    }
    double sgn = bv < 0 ? -1.0 : 1.0;
    for (int i = lane; i < na; i += 32) {
      double v = zero ? cst : X[i * m + c] * scale;
      Ua[(size_t)i * m + j] = sgn * v;
    }
  }
  return r;
}

}  // namespace amg

// Local bases of Eq. (svd) for callers that cannot allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not
// wanted at call time, for example a solver step inside a real-time or
// latency-bound loop (cudaMalloc can synchronise the whole device), a plug-in
// hosted by a framework whose memory pool owns every device allocation, or a
// setup pipeline that must stay within a fixed, pre-reserved memory budget.
// Such callers own their inputs and outputs; the only extra memory this entry
// point uses is a fixed work area compiled into the library.
//
// The work area is a file-scope __device__ array of AMG_LOCAL_BASES_STATIC_DOUBLES
// doubles (1 MiB).  Every GPU that loads the library holds it until the
// process exits.  All calls on a device share it, so two calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on
// it; callers must order such calls.  The host cannot use the array's name as
// a device address, so the first call on each device looks the address up
// with cudaGetSymbolAddress (with that device current) and caches it; make
// that first call before capturing any stream into a CUDA graph.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/amg.h"

namespace {

static __device__ __align__(256) double g_basis_work[AMG_LOCAL_BASES_STATIC_DOUBLES];
static __device__ int g_basis_flag;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_work_ptr[kMaxDevices] = {};
int* g_flag_ptr[kMaxDevices] = {};
// ``why`` documents each refusal in the source; the caller sees the status.
amg_status fail(amg_status s, const char* why) {
  (void)why;
  return s;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Same computation as the setup's per-aggregate SVD (one warp per aggregate:
// one-sided Jacobi, descending singular values, TOL * n_a / n_f truncation,
// at least one and at most min(n_a, m) columns, largest entry positive), with
// every row range checked against the work area; a bad range sets the flag
// and skips the aggregate.
__global__ void k_local_bases_static(const double* __restrict__ W, int m, int nagg,
                                     const int* __restrict__ row_start, int nf, double tol,
                                     double* __restrict__ work, double* __restrict__ U,
                                     int* __restrict__ rkeep) {
  int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (a >= nagg) return;
  int rs = row_start[a], re = row_start[a + 1];
  if (rs < 0 || re > nf || re <= rs) {
    if (lane == 0) atomicOr(&g_basis_flag, 1);
    return;
  }
  int na = re - rs;
  const double* Wa = W + (size_t)rs * m;
  double* X = work + (size_t)rs * m;
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
        al = wsum(al);
        be = wsum(be);
        ga = wsum(ga);
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
    sig[j] = sqrt(wsum(s));
    idx[j] = j;
  }
  for (int j = 1; j < m; ++j) {
    int v = idx[j], t = j;
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
    double best = -1.0, bv = 0;
    int bi = 0x7fffffff;
    for (int i = lane; i < na; i += 32) {
      double v = zero ? cst : X[i * m + c] * scale;
      if (fabs(v) > best) {
        best = fabs(v);
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
      U[(size_t)(rs + i) * m + j] = sgn * v;
    }
  }
  if (lane == 0) rkeep[a] = r;
}

}  // namespace

extern "C" amg_status amg_local_bases_static(const double* W, int32_t m, const int32_t* row_start,
                                             int32_t nagg, int32_t nf, double tol, double* U,
                                             int32_t* r, void* stream) {
  if (m < 1 || m > 16) return fail(AMG_ERR_INVALID_ARG, "m must be in [1, 16]");
  if (nagg < 1 || nf < 1) return fail(AMG_ERR_INVALID_ARG, "nagg and nf must be positive");
  if ((long long)nf * m > AMG_LOCAL_BASES_STATIC_DOUBLES)
    return fail(AMG_ERR_INVALID_ARG,
                "nf * m exceeds the fixed work area (AMG_LOCAL_BASES_STATIC_DOUBLES doubles)");
  if (!(tol >= 0)) return fail(AMG_ERR_INVALID_ARG, "tol must be >= 0");
  if (!on_device(W) || !on_device(row_start) || !on_device(U) || !on_device(r))
    return fail(AMG_ERR_INVALID_ARG, "W, row_start, U and r must be device pointers");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(AMG_ERR_CUDA, "cudaGetDevice failed or device ordinal too large");
  }
  double* work = nullptr;
  int* flag = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_work_ptr[dev]) {
      // first call on this device (the device is current): look up the
      // device addresses of the file-scope arrays once
      void* pw = nullptr;
      void* pf = nullptr;
      if (cudaGetSymbolAddress(&pw, g_basis_work) != cudaSuccess ||
          cudaGetSymbolAddress(&pf, g_basis_flag) != cudaSuccess || !pw || !pf) {
        cudaGetLastError();
        return fail(AMG_ERR_CUDA, "cudaGetSymbolAddress of the work area failed");
      }
      g_work_ptr[dev] = static_cast<double*>(pw);
      g_flag_ptr[dev] = static_cast<int*>(pf);
    }
    work = g_work_ptr[dev];
    flag = g_flag_ptr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the flag keeps the previous call's value: clear it
  if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return fail(AMG_ERR_CUDA, "cudaMemsetAsync failed");
  }
  int threads = 128;
  long long blocks = ((long long)nagg * 32 + threads - 1) / threads;
  k_local_bases_static<<<(unsigned)blocks, threads, 0, st>>>(W, m, nagg, row_start, nf, tol, work, U, r);
  if (cudaGetLastError() != cudaSuccess) return fail(AMG_ERR_CUDA, "kernel launch failed");
  int h_flag = 0;
  if (cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return fail(AMG_ERR_CUDA, "kernel or copy failed");
  }
  if (h_flag) return fail(AMG_ERR_INVALID_ARG, "row_start must be increasing, start at >= 0 and end at <= nf");
  return AMG_OK;
}

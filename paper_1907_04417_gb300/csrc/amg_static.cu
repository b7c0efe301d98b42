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
#include "amg_local_svd.cuh"

namespace amg {
void set_last_error(const char* msg);  // amg_capi.cu (thread-local message)
}

namespace {

static __device__ __align__(256) double g_basis_work[AMG_LOCAL_BASES_STATIC_DOUBLES];
static __device__ int g_basis_flag;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_work_ptr[kMaxDevices] = {};
int* g_flag_ptr[kMaxDevices] = {};
// Every refusal leaves its reason for amg_last_error(), like the other
// entry points; a successful call clears it.
amg_status fail(amg_status s, const char* why) {
  amg::set_last_error(why);
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

// The setup's per-aggregate computation (local_svd_warp: one warp per
// aggregate), with every row range checked against the work area first; a
// bad range sets the flag and skips the aggregate.
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
  int r = amg::local_svd_warp(W + (size_t)rs * m, m, re - rs, nf, tol, work + (size_t)rs * m,
                              U + (size_t)rs * m, lane);
  if (lane == 0) rkeep[a] = r;
}

}  // namespace

extern "C" amg_status amg_local_bases_static(const double* W, int32_t m, const int32_t* row_start,
                                             int32_t nagg, int32_t nf, double tol, double* U,
                                             int32_t* r, void* stream) {
  amg::set_last_error("");
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

// Device check mode: every index array that the solve kernels read an
// address from is checked on the device once it is built, before any kernel
// gathers through it.
//
// Enabled by AMG_CHECK=1 in the environment or by building the library with
// -DAMG_BOUNDS_CHECK.  Checked per level: rowptr[0] = 0, rowptr monotone,
// rowptr[n] = nnz, every column in [0, n); per transfer: row_start and
// coarse_start monotone from 0 to the fine and coarse orders, every block
// offset equal to the sum of the earlier blocks' n_a r_a; the coarsest
// blocks' offsets.  The first violation (the smallest packed (kind, index))
// is kept in a device word and the setup is refused with
// AMG_ERR_INVALID_ARG, naming the array, the level and the index.
//
// Test hook: AMG_TEST_CORRUPT_COL=k stores the out-of-range column n_k in
// the first non-zero of level k after the level is built, so that a test
// sees the check refuse it (no kernel gathers through it first).
#include <cstdio>
#include <cstdlib>
#include <string>

#include "amg_internal.cuh"

namespace amg {

namespace {

// kinds, in the order they are reported
enum : unsigned long long { CK_ROWPTR = 1, CK_COL = 2, CK_ROWSTART = 3, CK_COARSESTART = 4, CK_BLK = 5, CK_COBLK = 6 };

__device__ __forceinline__ void ck_record(unsigned long long* first, unsigned long long kind, long long idx) {
  atomicMin(first, (kind << 56) | (unsigned long long)(idx & ((1ll << 56) - 1)));
}

__global__ void k_check_csr(int n, long long nnz, const int* __restrict__ rowptr, const int* __restrict__ col,
                            unsigned long long* first) {
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  for (long long i = t0; i <= n; i += stride) {
    const int r = rowptr[i];
    if ((i == 0 && r != 0) || (i == n && r != nnz) || (i > 0 && r < rowptr[i - 1])) ck_record(first, CK_ROWPTR, i);
  }
  for (long long j = t0; j < nnz; j += stride) {
    const int c = col[j];
    if (c < 0 || c >= n) ck_record(first, CK_COL, j);
  }
}

__global__ void k_check_transfer(int nagg, int nf, int nc, const int* __restrict__ row_start,
                                 const int* __restrict__ coarse_start, const long long* __restrict__ blk_start,
                                 unsigned long long* first) {
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  for (long long a = t0; a <= nagg; a += stride) {
    const int rs = row_start[a], cs = coarse_start[a];
    if ((a == 0 && rs != 0) || (a == nagg && rs != nf) || (a > 0 && rs < row_start[a - 1]))
      ck_record(first, CK_ROWSTART, a);
    if ((a == 0 && cs != 0) || (a == nagg && cs != nc) || (a > 0 && cs < coarse_start[a - 1]))
      ck_record(first, CK_COARSESTART, a);
    if (a == 0 && blk_start[0] != 0) ck_record(first, CK_BLK, 0);
    if (a > 0) {
      const long long want = blk_start[a - 1] + (long long)(rs - row_start[a - 1]) * (cs - coarse_start[a - 1]);
      if (blk_start[a] != want) ck_record(first, CK_BLK, a);
    }
  }
}

__global__ void k_check_coarsest(int n, int nblk, const int* __restrict__ blk_off,
                                 const long long* __restrict__ inv_off, unsigned long long* first) {
  for (int b = threadIdx.x; b <= nblk; b += blockDim.x) {
    const int o = blk_off[b];
    if ((b == 0 && (o != 0 || inv_off[0] != 0)) || (b == nblk && o != n) || (b > 0 && o < blk_off[b - 1]))
      ck_record(first, CK_COBLK, b);
    if (b > 0) {
      const long long nb = blk_off[b] - blk_off[b - 1];
      if (inv_off[b] != inv_off[b - 1] + nb * nb) ck_record(first, CK_COBLK, b);
    }
  }
}

unsigned grid_of(long long n) { return (unsigned)std::min<long long>((n + 255) / 256 + 1, 4096); }

}  // namespace

bool check_mode() {
#ifdef AMG_BOUNDS_CHECK
  return true;
#else
  const char* e = std::getenv("AMG_CHECK");
  return e && e[0] == '1';
#endif
}

void check_plan(Plan& P, cudaStream_t st) {
  const char* cor = std::getenv("AMG_TEST_CORRUPT_COL");
  if (cor) {
    const int k = std::atoi(cor);
    if (k >= 0 && k < P.L && P.lev[k].nnz > 0) {
      const int bad = P.lev[k].n;
      AMG_CUDA(cudaMemcpyAsync(P.lev[k].col, &bad, sizeof(int), cudaMemcpyHostToDevice, st));
    }
  }
  Arena ar;
  unsigned long long* first = ar.alloc<unsigned long long>(1);
  static const char* kinds[] = {"", "rowptr", "col", "row_start", "coarse_start", "blk_start", "coarsest blk_off"};
  auto report = [&](const char* what, int k) {
    unsigned long long h = ~0ull;
    AMG_CUDA(cudaMemcpyAsync(&h, first, sizeof(h), cudaMemcpyDeviceToHost, st));
    AMG_CUDA(cudaStreamSynchronize(st));
    if (h != ~0ull) {
      const unsigned kind = (unsigned)(h >> 56);
      const long long idx = (long long)(h & ((1ull << 56) - 1));
      throw Error(AMG_ERR_INVALID_ARG, std::string("internal index check: ") + what + " " + std::to_string(k) +
                                           ", " + kinds[kind < 7 ? kind : 0] + "[" + std::to_string(idx) +
                                           "] is out of order or out of range");
    }
  };
  for (int k = 0; k < P.L; ++k) {
    const Level& L = P.lev[k];
    AMG_CUDA(cudaMemsetAsync(first, 0xff, sizeof(unsigned long long), st));
    k_check_csr<<<grid_of(std::max<long long>(L.nnz, L.n)), 256, 0, st>>>(L.n, L.nnz, L.rowptr, L.col, first);
    AMG_LAUNCH_CHECK();
    report("level", k);
    if (k + 1 < P.L) {
      const Transfer& T = P.tr[k];
      AMG_CUDA(cudaMemsetAsync(first, 0xff, sizeof(unsigned long long), st));
      k_check_transfer<<<grid_of(T.nagg), 256, 0, st>>>(T.nagg, P.lev[k].n, P.lev[k + 1].n, T.row_start,
                                                        T.coarse_start, T.blk_start, first);
      AMG_LAUNCH_CHECK();
      report("transfer into level", k);
    }
  }
  AMG_CUDA(cudaMemsetAsync(first, 0xff, sizeof(unsigned long long), st));
  k_check_coarsest<<<1, 256, 0, st>>>(P.co.n, P.co.nblk, P.co.blk_off, P.co.inv_off, first);
  AMG_LAUNCH_CHECK();
  report("coarsest level", P.L - 1);
}

}  // namespace amg

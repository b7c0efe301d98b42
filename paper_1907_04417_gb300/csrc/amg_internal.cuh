// Internal declarations of the GB300 AMG library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/amg.h"

namespace amg {

// NVTX range over a scope (setup, solves, graph replays): visible to
// profilers that collect NVTX; a no-op otherwise (header-only NVTX v3).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- errors --
struct Error : std::runtime_error {
  amg_status status;
  Error(amg_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define AMG_CUDA(call)                                                             \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      throw ::amg::Error(AMG_ERR_CUDA, std::string(#call " failed: ") +            \
                                           cudaGetErrorString(e_) + " at " +       \
                                           __FILE__ + ":" + std::to_string(__LINE__)); \
  } while (0)

#define AMG_REQUIRE(cond, msg)                                                     \
  do {                                                                             \
    if (!(cond)) throw ::amg::Error(AMG_ERR_INVALID_ARG, msg);                     \
  } while (0)

// Every kernel launch of the library goes through AMG_LAUNCH_CHECK, which
// also counts it (launches recorded into a CUDA graph are counted when the
// graph is replayed instead).
void count_launch();
#define AMG_LAUNCH_CHECK()          \
  do {                              \
    AMG_CUDA(cudaGetLastError());   \
    ::amg::count_launch();          \
  } while (0)

// ---------------------------------------------------------------- memory --
// All device memory of a hierarchy (and of its solve workspaces) is taken
// from an arena that frees everything at destruction.
struct Arena {
  std::vector<void*> blocks;
  size_t bytes = 0;
  void* raw(size_t n) {
    if (n == 0) n = 16;
    n = (n + 255) & ~size_t(255);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error(AMG_ERR_ALLOC, "cudaMalloc of " + std::to_string(n) + " bytes failed");
    }
    blocks.push_back(p);
    bytes += n;
    return p;
  }
  template <typename T> T* alloc(size_t count) { return static_cast<T*>(raw(count * sizeof(T))); }
  ~Arena() {
    for (void* p : blocks) cudaFree(p);
  }
};

// ------------------------------------------------------------ hierarchy --
// Capacities of the shared-memory staging of a CTA's CSR slice (see
// stage_csr in amg_kernels.cuh).
struct Stage {
  int rows_max = 0;  // largest row count of a CTA
  int span4 = 0;     // capacity of the 4-byte arrays (elements, multiple of 4)
  int span8 = 0;     // capacity of the 8-byte arrays (elements, multiple of 2)
  int enabled = 0;   // 0: the level is read straight from global memory
  int* err = nullptr;
  // polls of the first wait for a staged copy (0: the normal bound); a
  // small value is a test hook that makes the first wait give up
  int first_wait = 0;
};

// Every level is numbered so that each aggregate of the next level owns a
// contiguous range of rows; the prolongator of an aggregate is then a dense
// n_a x r_a block applied to a contiguous slice.
struct Level {
  int n = 0;
  long long nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* val64 = nullptr;
  float* val32 = nullptr;
  float* vallo = nullptr;    // level 0: val64 - val32 (the low half of a double-float)
  float* val_sc = nullptr;   // level 0: fl32(a_ij / d_j), A D^{-1} for the u0-free float32 cycle
  float2* hl = nullptr;      // level 0: (val32, vallo) per non-zero (the paired q = A p), on first use
  double* dinv64 = nullptr;  // 1 / sum_j |a_ij|   (non-coarsest levels)
  float* dinv32 = nullptr;
  int max_row_len = 0;
  double avg_row_len = 0;
  std::vector<int> h_rowptr;  // host copy of rowptr (partitions)
  // row groups (coarse levels): the coarse dofs of one aggregate share one
  // column pattern and are stored back to back; gstart (ngrp + 1 rows) is
  // the coarse_start of the transfer that made the level
  int grp_ok = 0, ngrp = 0, grp_rmax = 0;
  const int* gstart = nullptr;
  Stage gsg;  // staging of the grouped sweep's CTAs (GROUPS_PER_CTA groups each)
  // entry-major copy of a grouped level for the warp-per-group sweep: per
  // row group its pattern (gw_col from gw_ptr[g]) and, per pattern entry,
  // gw_rs values (the group's rows, zero-padded to 4 or 8); built on first
  // use, gw_state 1 (built) or -1 (not available)
  int gw_state = 0, gw_rs = 4;
  int gw_zero = 0;  // first entry of the zero batch (patterns padded to multiples of 8)
  int* gw_ptr = nullptr;
  int* gw_col = nullptr;
  double* gw_v64 = nullptr;
  float* gw_v32 = nullptr;
};

// P^{k+1}: maps level k+1 (coarse) to level k (fine).
struct Transfer {
  int nagg = 0, nf = 0, nc = 0;
  long long npval = 0;
  int* row_start = nullptr;        // nagg + 1, fine rows of each aggregate
  int* coarse_start = nullptr;     // nagg + 1, coarse dofs of each aggregate
  long long* blk_start = nullptr;  // nagg + 1, offsets of the n_a x r_a blocks
  double* p64 = nullptr;
  float* p32 = nullptr;
  std::vector<int> h_row_start, h_coarse_start;
  std::vector<long long> h_blk_start;
  int* gagg = nullptr;  // nagg + 1: first row group of the fine level in each aggregate (grouped fine levels)
  Stage gsg;            // staging of the grouped restriction (one CTA per aggregate)
  // R = P^T (I - A D^{-1}) of the fine level, by aggregate (the restriction
  // after one pre-sweep from zero): pattern offsets (nagg + 1), pattern
  // columns, rf_rs values per pattern entry (the aggregate's coarse dofs,
  // zero-padded); built on first use, rf_state 1 (built) or -1 (not
  // available: more than 8 coarse dofs in an aggregate, or no float64 level)
  int rf_state = 0, rf_rs = 4;
  int rf_last = 0;  // whether the most recently enqueued V-cycle restricted by R
  long long rf_entries = 0;  // pattern entries, each aggregate's padded to a multiple of 8
  int rf_zero = 0;           // first entry of the zero batch after the last aggregate
  int* rf_ptr = nullptr;
  int* rf_col = nullptr;
  double* rf_v64 = nullptr;
  float* rf_v32 = nullptr;
};

// Aggregate-aligned CTA ranges of one transfer for a given column count, with
// the largest per-CTA extents (rows, prolongator values, aggregates, coarse
// dofs) that size the shared-memory staging.
struct TPart {
  int ncta = 0;
  int* cta_agg = nullptr;
  int rows_max = 0, p_max = 0, a_max = 0, c_max = 0;
  int ra_max = 1;  // largest number of coarse dofs of one aggregate
  Stage sg;
  int warp = 0;    // restriction: 0 CTA ranges, 1 one warp per aggregate (3: staged), 2 grouped (one CTA per aggregate)
  int pwarp = 0;   // prolongation by one warp per aggregate (no CTA ranges)
  int jl = 1;      // grouped restriction: lanes splitting a group's pattern columns
  Stage wsg;       // staging of the warp-per-aggregate restriction (NWARP aggregates per CTA)
};

// Row ranges of the row-parallel kernels of one level for a given column
// count (balanced by non-zeros; at level 0 they never straddle two systems),
// and the fixed groups of CTAs of the two-level deterministic reductions.
struct RPart {
  int ncta = 0, ngroups = 0;
  int* cta_row = nullptr;   // ncta + 1
  int* grp_cta = nullptr;   // ngroups + 1
  int* sys_grp = nullptr;   // nsys + 1 (level 0)
  int* sys_cta = nullptr;   // nsys + 1 (level 0)
  Stage sg;
};

// Dense inverses of the coarsest matrix (block-diagonal over systems).
struct Coarsest {
  int n = 0, nblk = 0;
  int* blk_off = nullptr;          // nblk + 1 rows
  long long* inv_off = nullptr;    // nblk + 1 offsets into inv
  double* inv = nullptr;
  std::vector<int> h_blk_off;
  std::vector<long long> h_inv_off;
};

struct Workspace;

struct Plan {
  int L = 0, nsys = 1, m = 0;
  std::vector<Level> lev;
  std::vector<Transfer> tr;   // tr[k] maps level k+1 -> level k
  Coarsest co;
  std::vector<int> h_sys_row;  // nsys + 1 level-0 row offsets
  int* perm0 = nullptr;        // library row -> row within its own system (caller numbering)
  std::unique_ptr<Arena> arena;
  std::map<long long, std::shared_ptr<Workspace>> ws;
  bool groups_done = false;    // row groups of the coarse levels detected
  // multicolour Gauss-Seidel (smoothed levels): colour and diagonal of every
  // row, number of colours; built on first use (amg_variants.cu)
  bool gs_done = false;
  std::vector<int*> gs_colour;
  std::vector<double*> gs_diag;
  std::vector<int> gs_ncol;
  std::vector<int*> gs_rows;                 // rows sorted by colour, ascending within a colour
  std::vector<std::vector<int>> gs_cstart;   // ncol + 1 offsets into gs_rows
  Plan() : arena(new Arena) {}
  ~Plan();
};

struct Timer {
  int kernel = 0;
  bool on = false;
  std::vector<cudaEvent_t> ev;   // pairs
  size_t used = 0;
  double total_ms = 0;
  long long launches = 0;
};

}  // namespace amg

struct amg_hierarchy {
  amg::Plan plan;
  int n = 0, nnz = 0, m = 0;
  int* nzmap = nullptr;                   // library nz -> caller nz (level 0)
  std::vector<std::vector<int>> h_perm;   // per level: library node -> caller node
  std::vector<std::vector<int>> h_r;      // per coarse level: kept columns per aggregate
  long long truncated = 0;
  amg::Timer timer;
  cudaStream_t own = nullptr;            // internal non-blocking stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::map<std::vector<amg_hierarchy*>, std::unique_ptr<amg::Plan>> batches;
};

namespace amg {

// setup (amg_setup.cu)
void build_hierarchy(amg_hierarchy* h, const amg_csr* A, int nlev, const int32_t* const* agg,
                     const int32_t* n_nodes, const double* W, int m, const amg_opts& o,
                     cudaStream_t st);
void build_batch_plan(Plan& out, const std::vector<amg_hierarchy*>& hs, cudaStream_t st);

// device check mode (amg_check.cu): AMG_CHECK=1 or a -DAMG_BOUNDS_CHECK build
// checks every index array of a built plan on the device and refuses it
// with AMG_ERR_INVALID_ARG at the first violation
bool check_mode();
void check_plan(Plan& P, cudaStream_t st);

// solve (amg_solve.cu)
struct SolveReq {
  int nsys;
  std::vector<int> n_sys;
  std::vector<const double*> b;
  std::vector<double*> x;
  std::vector<int> nrhs;
  bool zero_x;  // ignore the contents of x (adjoint)
};
amg_status run_pcg(amg_hierarchy* owner, Plan& P, const SolveReq& rq, const amg_opts& o,
                   cudaStream_t user, amg_info* info);
void run_vcycle(amg_hierarchy* owner, Plan& P, const double* r, double* z, int nrhs,
                const amg_opts& o, cudaStream_t user);
void run_adjoint_grad(amg_hierarchy* h, const double* lam_caller, const double* x_caller,
                      int nrhs, double* grad, cudaStream_t st);

// compatible weighted matching of one pairwise step (amg_matching.cu)
void run_pairwise_matching(const amg_csr* A, const double* w, int32_t* mate, cudaStream_t st);
void run_pairwise_step(const amg_csr* A, const double* w, int32_t* agg, int32_t* nc, int32_t* rowptr_c,
                       int32_t* col_c, double* val_c, int32_t* nnz_c, double* wc, cudaStream_t st);

// cycle variants (amg_variants.cu): the buffers and launch choices of one
// float64 solve workspace that the variant cycle reads.  smoother 0 is
// l1-Jacobi, 1 multicolour forward/backward Gauss-Seidel; kind 0 is the
// V-cycle, 1 the K-cycle (two flexible-CG iterations on every level but the
// coarsest).
struct VarCycle {
  int smoother = 0, kind = 0, K = 0, pre = 1, post = 1;
  std::vector<double*> f, u, v;              // per level (f[0] is the CG residual)
  std::vector<double*> c2, v1, v2, r2, e;    // K-cycle buffers of levels 1..L-2
  std::vector<int> nzl;
  std::vector<RPart> rp;
  std::vector<TPart> tp;
  double* partial = nullptr;                 // per-CTA partial inner products
  std::vector<double*> dots;                 // per level: 5 K inner products
  int dot_rows = 1024;                       // rows per CTA of the inner products
};
void ensure_gs(amg_hierarchy* h, Plan& P, cudaStream_t st);
size_t var_level_ctas(int n, const VarCycle& vc);
// z = B r (level 0, float64) by one variant cycle; u0 is level-0 scratch.
// h and pool (may be null) time the level-0 Gauss-Seidel sweeps
// (AMG_KERNEL_GS_L0) when the handle's timer asks for them.
void enqueue_var_cycle(const Plan& P, const VarCycle& vc, const double* r, double* z, double* u0,
                       const int* done, cudaStream_t st, amg_hierarchy* h,
                       std::vector<cudaEvent_t>* pool);
// colours of level k in the caller's numbering (the oracle's dof order)
int level_colours(amg_hierarchy* h, int k, int32_t* colour, cudaStream_t st);

// bootstrap testing phase (amg_bootstrap.cu)
void run_bootstrap_test(const std::vector<amg_hierarchy*>& hs, double* x, int nrhs, int nu, int symmetric,
                        const amg_opts& o, cudaStream_t st, double* rho, double* anorm);

// launch accounting
extern thread_local bool g_capturing;
void add_launches(long long n);
long long launches_total();

// Brackets the launches of one kernel family with CUDA events on their
// stream while the handle's timer asks for that family; the pairs go to
// ``pool`` and are read back after the solve.
struct TimedLaunch {
  amg_hierarchy* h;
  int id;
  cudaStream_t st;
  std::vector<cudaEvent_t>* pool;
  bool on;
  cudaEvent_t e1 = nullptr;
  TimedLaunch(amg_hierarchy* h_, int id_, cudaStream_t st_, std::vector<cudaEvent_t>* pool_)
      : h(h_), id(id_), st(st_), pool(pool_) {
    on = h && pool && h->timer.on && h->timer.kernel == id;
    if (on) {
      cudaEvent_t e0;
      AMG_CUDA(cudaEventCreate(&e0));
      AMG_CUDA(cudaEventCreate(&e1));
      pool->push_back(e0);
      pool->push_back(e1);
      // External records become event-record nodes when the stream is captured
      AMG_CUDA(cudaEventRecordWithFlags(e0, st, g_capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
    }
  }
  ~TimedLaunch() {
    if (on) cudaEventRecordWithFlags(e1, st, g_capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  }
};

// pointer helpers
bool is_device_ptr(const void* p);
void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t st);
void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st);

}  // namespace amg

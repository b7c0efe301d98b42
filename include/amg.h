/*
 * amg.h - C ABI of the GB300 library for the solve phase of the
 * single-hierarchy multiple-vector aggregation-based AMG (D'Ambra &
 * Vassilevski, "Improving Solve Time of Aggregation-based Adaptive AMG"),
 * used as a preconditioner for conjugate gradients.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Plain C types only.  Pointers may address device memory or host memory
 *    (pageable or pinned); the library inspects each pointer and stages host
 *    buffers through its own device buffers.  Index arrays are int32.
 *  - Multi-column vectors are dense row-major n x nrhs blocks (the nrhs
 *    values of one row are contiguous).
 *  - ``stream`` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Work is ordered after earlier work on that stream.
 *    Every call returns only after its results are final (it synchronises
 *    once at the end), so status codes and info structs are valid on return.
 *  - No exception or CUDA error crosses the ABI: every call returns an
 *    amg_status and leaves a message for amg_last_error().  Invalid
 *    arguments are rejected before any launch.
 *  - Handles are not thread-safe: one handle must not be used by two host
 *    threads at the same time.
 */
#ifndef AMG_H
#define AMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amg_hierarchy* amg_handle;   /* opaque, owned by the library */

typedef enum {
  AMG_OK = 0,
  AMG_ERR_INVALID_ARG = 1,   /* malformed CSR, aggregate map, size or option        */
  AMG_ERR_NOT_SPD = 2,       /* non-positive pivot in the coarsest Cholesky          */
  AMG_ERR_NOT_CONVERGED = 3, /* maxit reached; x and info are still written          */
  AMG_ERR_BREAKDOWN = 4,     /* p.q <= 0 or a non-finite CG scalar; x is written     */
  AMG_ERR_TIMEOUT = 5,       /* a bounded device wait gave up                         */
  AMG_ERR_CUDA = 6,          /* a CUDA runtime call failed                            */
  AMG_ERR_ALLOC = 7          /* device or host allocation failed                      */
} amg_status;

/* Square sparse matrix in CSR form: rowptr[n+1], col[nnz] (sorted, in
 * range), val[nnz] (float64).  The library copies it during setup and never
 * aliases it afterwards. */
typedef struct {
  int32_t n;
  int32_t nnz;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
} amg_csr;

typedef struct {
  double tol_svd;          /* TOL of the truncation rule (Section 5): keep the left
                              singular vectors with sigma > TOL*size(a)/size(A). 0.1 */
  int32_t pre;             /* l1-Jacobi pre-sweeps per level (>= 1).              1 */
  int32_t post;            /* l1-Jacobi post-sweeps per level (>= 1).             1 */
  int32_t cycle_precision; /* 64: whole V-cycle in float64; 32: V-cycle in float32
                              inside float64 CG (coarsest solve stays float64).  64 */
  double rtol;             /* stop when ||r||_2 <= rtol*||b||_2 (recursive r). 1e-8 */
  int32_t maxit;           /* iteration limit.                                 1000 */
  int32_t use_graph;       /* 1: PCG iterations replayed from a CUDA graph.      1 */
  int32_t check_every;     /* iterations between convergence reads on the host.  8 */
  int32_t autotune;        /* 1: time SpMV lane layouts once per (level, nrhs).  1 */
  int32_t outer_fp64;      /* float32-cycle mode only.  1: the outer CG keeps x, r,
                              p and q in float64 and forms q = A p with float64
                              FMAs; the cycle takes r rounded to float32.
                              0: x, r and q are double-float pairs (hi + lo
                              float32, about 2^-44 relative), the search
                              direction p is rounded to float32 when it is
                              formed, and q = A p runs in double-float
                              arithmetic (error-free products and sums) on the
                              float32 pipes.  In both modes alpha, beta and the
                              reduced dot products and norms are float64.     0 */
  int32_t smoother;        /* 0: l1-Jacobi.  1: Gauss-Seidel, forward sweeps before
                              and backward sweeps after the coarse correction
                              (Section 5), rows visited colour by colour in a
                              greedy colouring of each level's graph.  Needs
                              cycle_precision 64 and a single hierarchy.        0 */
  int32_t cycle;           /* 0: V-cycle.  1: K-cycle: on every level but the
                              coarsest the coarse correction is two flexible-CG
                              iterations preconditioned by the cycle one level
                              down (Section 5; nonlinear, so the outer CG sees a
                              slightly variable preconditioner).  Needs
                              cycle_precision 64 and a single hierarchy.        0 */
} amg_opts;

/* Per right-hand-side result. */
typedef struct {
  int32_t iters;       /* PCG iterations performed                               */
  int32_t converged;   /* 1 if ||r|| <= rtol ||b||                                */
  int32_t status;      /* amg_status of this column                              */
  int32_t reserved;
  double relres;       /* final recursive relative residual ||r||/||b||          */
} amg_info;

/* Hierarchy characteristics (Section 5: nl, opc, cr). */
typedef struct {
  int32_t levels;          /* nl, including the fine level                       */
  int32_t m;               /* number of smooth vectors                           */
  double opc;              /* sum_k nnz(A^k) / nnz(A^0)                          */
  double cr;               /* mean of n(A^{k-1})/n(A^k) over the nl-1 steps      */
  int64_t n_level[16];
  int64_t nnz_level[16];
  int64_t truncated_aggs;  /* aggregates that kept fewer than min(n_a, m) columns */
  int64_t device_bytes;    /* device memory held by the hierarchy                */
} amg_hier_info;

/* Fill *opts with the defaults listed above. */
void amg_default_opts(amg_opts* opts);

/*
 * Build the multiple-vector hierarchy (Section 4, Eq. (svd); Section 4.1).
 *
 *  A           fine matrix, SPD (host or device arrays).
 *  n_agg_levels L-1: number of aggregate maps, 0 <= L-1 <= 15.
 *  agg[k]      int32[n_nodes[k]]: level-(k+1) aggregate of level-k node i
 *              (the binary matrices pi^{k+1} of Eq. (binmat)).  Level-0 nodes
 *              are the dofs; level-k nodes (k >= 1) are the level-k aggregates,
 *              each owning the coarse dofs its local basis produced (the matrix
 *              Q of Section 4.1).  Every aggregate must be non-empty.
 *  n_nodes     int32[L] host array: n_nodes[0] = A->n, n_nodes[k] = number of
 *              level-k aggregates.
 *  W           float64 n x m column-major: the smooth vectors w_0..w_{m-1}.
 *  m           1 <= m <= 16.
 *
 * For each level: local SVD of W|_a per aggregate, truncation with
 * opts->tol_svd, block prolongator P^k = blockdiag(P~_a) with orthonormal
 * columns, Galerkin A^k = (P^k)^T A^{k-1} P^k, coarse smooth vectors
 * (P^k)^T W^{k-1}; all on the device.  The coarsest matrix is factorised by a
 * float64 Cholesky on the device (AMG_ERR_NOT_SPD on a non-positive pivot).
 * On success *out owns all device memory of the hierarchy until amg_destroy.
 */
amg_status amg_setup_from_aggregates(const amg_csr* A, int32_t n_agg_levels,
                                     const int32_t* const* agg, const int32_t* n_nodes,
                                     const double* W, int32_t m, const amg_opts* opts,
                                     void* stream, amg_handle* out);

/*
 * AMG-preconditioned CG (Section 5) for nrhs right-hand sides at once.
 *  b  n x nrhs row-major float64 (host or device), read only.
 *  x  n x nrhs row-major float64 (host or device): initial guess on entry,
 *     solution on return (also on NOT_CONVERGED / BREAKDOWN).
 *  info  host array of nrhs amg_info, or NULL.
 * Each column runs its own CG (own alpha, beta, stopping test); the matrix
 * and the hierarchy are read once per sweep for all columns.
 */
amg_status amg_solve(amg_handle h, const double* b, double* x, int32_t nrhs,
                     const amg_opts* opts, void* stream, amg_info* info);

/*
 * Solve nsys independent systems (each with its own hierarchy and nrhs[s]
 * right-hand sides) in one launch sequence: the hierarchies are concatenated
 * block-diagonally level by level, the coarsest solve is block-diagonal and
 * the CG scalars are kept per (system, column).  All hierarchies must have the
 * same number of levels.  b[s], x[s] are n_s x nrhs[s] row-major (host or
 * device); info is a host array of sum(nrhs) entries, system-major, or NULL.
 * The concatenated hierarchy is built on the first call for a given list of
 * handles and cached on h[0] until amg_destroy(h[0]).
 */
amg_status amg_solve_batched(const amg_handle* h, int32_t nsys, const double* const* b,
                             double* const* x, const int32_t* nrhs, const amg_opts* opts,
                             void* stream, amg_info* info);

/*
 * Adjoint of x = A^{-1} b (A SPD, so A^{-T} = A^{-1}): solves A lambda = g
 * with the same preconditioned CG and writes, for every stored entry (i, j) of
 * the setup matrix A in its CSR order,
 *     grad_val[p] = - sum_c lambda[i, c] * x[j, c],
 * the derivative of L with respect to a_ij when g = dL/dx.
 *  g, x     n x nrhs row-major float64 (host or device).
 *  lambda   n x nrhs row-major float64 output (host or device); zero initial guess.
 *  grad_val nnz float64 output (host or device).
 */
amg_status amg_adjoint(amg_handle h, const double* g, const double* x, int32_t nrhs,
                       double* lambda, double* grad_val, const amg_opts* opts,
                       void* stream, amg_info* info);

/* Apply the preconditioner once, z = B r (one V-cycle, Section 5, or the
 * variant that opts->smoother and opts->cycle select), in the precision
 * opts->cycle_precision.  r, z: n x nrhs row-major float64. */
amg_status amg_vcycle(amg_handle h, const double* r, double* z, int32_t nrhs,
                      const amg_opts* opts, void* stream);

/*
 * Testing phase of the bootstrap (Algorithm 1, Section 2).  hs[0..r-1] are
 * hierarchies B_1..B_r, all set up on the same matrix A (same order and
 * non-zeros; the level-0 copy of hs[0] serves as A).  x (n x nrhs
 * row-major float64, host or device, the caller's numbering, nrhs <= 32) is
 * replaced in place by E^nu x, where with B_k one V-cycle of hs[k] in
 * opts->cycle_precision
 *     symmetric != 0:  E = (I - B_1 A) ... (I - B_r A) (I - B_r A) ... (I - B_1 A)
 *                      (the symmetrized product of Section 5 (i)),
 *     symmetric == 0:  E = (I - B_r A) ... (I - B_1 A)   (Eq. (comp_AMG)).
 * rho (nrhs doubles, host, may be NULL) receives the convergence estimate
 * (||E^nu x||_A / ||x||_A)^(1/nu) per column (0 for a zero column), and
 * anorm (nrhs doubles, host, may be NULL) ||E^nu x||_A, which normalises the
 * new smooth vector (w_r = x^nu / ||x^nu||_A).  The call allocates its own
 * work vectors and synchronises ``stream`` before it returns.  Mismatched
 * hierarchies or sizes give AMG_ERR_INVALID_ARG.
 */
amg_status amg_bootstrap_test(const amg_handle* hs, int32_t r, double* x, int32_t nrhs, int32_t nu,
                              int32_t symmetric, const amg_opts* opts, void* stream, double* rho,
                              double* anorm);

/*
 * Compatible weighted matching of one pairwise aggregation step (Section 3)
 * on the device.  For the graph of A (CSR, host or device; the pattern must
 * be structurally symmetric, columns sorted) and a vector w (n float64, host
 * or device) the edge weights are
 *     c_ij = 1 - 2 a_ij w_i w_j / (a_ii w_i^2 + a_jj w_j^2)   (i < j, a_ij the
 * stored upper entry), each float64 operation rounded on its own; only edges
 * with c_ij > 0 take part.  The matching is the greedy matching on the strict
 * order (c desc, smaller end asc, larger end asc), which approximates the
 * maximum product matching of Section 3.  mate (n int32, host or device,
 * output): the partner of every vertex, -1 if unmatched.  The call allocates
 * its own work arrays and synchronises ``stream``.  A malformed or
 * structurally non-symmetric pattern gives AMG_ERR_INVALID_ARG.
 */
amg_status amg_pairwise_matching(const amg_csr* A, const double* w, int32_t* mate, void* stream);

/*
 * One whole pairwise aggregation step (Section 3) on the device: the matching
 * of amg_pairwise_matching; the aggregates (each pair or singleton is
 * numbered by its smallest member, in increasing order); the pairwise
 * prolongator of Eq. (prol) with one column per aggregate ([w_i, w_j] /
 * sqrt(w_i^2 + w_j^2) for a pair, w_k/|w_k| for a singleton, 1 when w_k = 0,
 * equal weights for a pair with w = 0); the coarse vector w_c = P^T w; the
 * next graph A_c = P^T A P in CSR with sorted columns.
 * Outputs (host or device, capacities from A):
 *   agg[n]          aggregate of every vertex;
 *   nc              number of aggregates (one int32, host);
 *   rowptr_c[n+1], col_c[nnz(A)], val_c[nnz(A)]   A_c (nc + 1 and nnz_c used);
 *   nnz_c           entries of A_c (one int32, host);
 *   wc[n]           w_c (nc used).
 * The call allocates its own work arrays and synchronises ``stream``.  A
 * malformed or structurally non-symmetric A gives AMG_ERR_INVALID_ARG, as
 * does a coarse row of more than 256 entries before merging.
 */
amg_status amg_pairwise_step(const amg_csr* A, const double* w, int32_t* agg, int32_t* nc, int32_t* rowptr_c,
                             int32_t* col_c, double* val_c, int32_t* nnz_c, double* wc, void* stream);

/* Hierarchy characteristics; never fails for a valid handle. */
amg_status amg_hierarchy_info(amg_handle h, amg_hier_info* info);

/*
 * Export level k of the hierarchy to host arrays, for inspection and tests.
 * sizes (int64[6], always filled): n_k, nnz_k, number of level-k aggregates
 * (0 for k = 0), number of prolongator values, n_{k-1} (0 for k = 0), m.
 * Any output pointer may be NULL.  The library numbers dofs internally in an
 * order where every aggregate is contiguous; the export describes it:
 *   rowptr[n_k+1], col[nnz_k], val[nnz_k]  A^k in the library's numbering;
 *   perm[n_k]     for k = 0: library dof -> caller dof;
 *   agg_id[naggs] library aggregate -> caller aggregate index (level k);
 *   r[naggs]      kept columns per aggregate;
 *   row_start[naggs+1] level-(k-1) rows of each aggregate (library numbering);
 *   pval          prolongator blocks, aggregate after aggregate, each n_a x r_a
 *                 row-major (float64).
 */
amg_status amg_export_level(amg_handle h, int32_t k, int64_t* sizes, int32_t* rowptr,
                            int32_t* col, double* val, int32_t* perm, int32_t* agg_id,
                            int32_t* r, int32_t* row_start, double* pval);

/*
 * Colours of the Gauss-Seidel smoother on level k (0 <= k <= levels-2), for
 * inspection and tests.  The rows of each level are coloured greedily in
 * decreasing priority (splitmix64(i), i), i the row in the caller's
 * numbering (level 0: the caller's dofs; coarse levels: dofs numbered
 * aggregate by aggregate in aggregate-index order, an aggregate's kept
 * columns in descending singular-value order): every row takes the smallest
 * colour that none of its higher-priority neighbours in the graph of A^k
 * holds.  colour (n_k int32, host, may be NULL) receives them in that
 * numbering and *ncolours (may be NULL) their number.  The first call builds
 * the colouring on the device (it is kept with the hierarchy).
 */
amg_status amg_level_colours(amg_handle h, int32_t k, int32_t* colour, int32_t* ncolours);

/* Kernel timing hook used by the benchmark: while enabled, every launch of
 * the kernel family ``kernel_id`` (AMG_KERNEL_*) is bracketed by CUDA events
 * on the stream it is launched on; amg_timer_read returns the summed device
 * time and the number of launches since the last enable. */
enum {
  AMG_KERNEL_SPMV_CG = 1,        /* q = A p with p.q            (level 0, float64) */
  AMG_KERNEL_RESTRICT_L0 = 2,    /* fused residual + P^T        (level 0)          */
  AMG_KERNEL_SMOOTH_L0 = 3,      /* post-smoothing with r.z     (level 0)          */
  AMG_KERNEL_PROLONG_L0 = 4,     /* x += P e                    (level 0)          */
  AMG_KERNEL_CG_UPDATE = 5,      /* x, r update with ||r||      (level 0)          */
  AMG_KERNEL_GS_L0 = 6,          /* one backward Gauss-Seidel sweep, all colours
                                    (level 0, smoother 1; the last post-sweep)      */
  AMG_KERNEL_CG_DIRECTION = 7,   /* p = z + beta p (with x += alpha p in the
                                    double-float mode)          (level 0)          */
  AMG_KERNEL_COARSE_LEVELS = 8   /* every launch of one V-cycle on levels >= 1,
                                    timed as one span (after the level-0
                                    restriction, before the level-0 prolongation) */
};
amg_status amg_timer_enable(amg_handle h, int32_t kernel_id, int32_t enable);
amg_status amg_timer_read(amg_handle h, double* total_ms, int64_t* launches);

/* How the restriction out of level k (0 <= k < levels - 1) ran in the most
 * recent V-cycle that a solve on this hierarchy (not a batch) enqueued.
 * With one pre-sweep from zero the iterate that enters the restriction is
 * u = D^{-1} f, so the restricted residual P^T (f - A u) of Section 5's
 * V-cycle equals R f with R = P^T (I - A D^{-1}), P the block prolongator
 * of Eq. (prol).  *by_r (may be NULL) is 1 when the solve applied R (kept
 * by aggregate: one column pattern per aggregate, the rows its rows of A
 * reach), 0 when it formed f - A u and applied P^T.  *entries (may be NULL)
 * receives R's pattern entries (0 while R is not built) and
 * *values_per_entry (may be NULL) the values stored per entry (the
 * aggregate's coarse dofs, zero-padded to 4 or 8).  AMG_ERR_INVALID_ARG for
 * a null handle or k out of range. */
amg_status amg_restriction_info(amg_handle h, int32_t k, int32_t* by_r, int64_t* entries,
                                int32_t* values_per_entry);

/*
 * Per-aggregate orthonormal bases, as amg_setup_from_aggregates builds them,
 * computed without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that may not call cudaMalloc when they
 * run (a real-time or latency-bound loop where an allocation can stall the
 * device, a plug-in whose host framework owns every device allocation, a
 * pipeline held to a pre-reserved memory budget).
 *
 * It runs the per-aggregate computation of amg_setup_from_aggregates on
 * caller-owned device arrays and gives the same bases:
 *  W          nf x m row-major float64, device: the smooth vectors, with the
 *             rows of aggregate a at [row_start[a], row_start[a+1]).
 *  row_start  int32[nagg+1], device, strictly increasing, row_start[0] >= 0,
 *             row_start[nagg] <= nf.
 *  nf         rows of the level (size(A) in the truncation threshold).
 *  tol        TOL of the truncation rule.
 *  U          nf x m row-major float64, device, output: rows of aggregate a
 *             hold its kept columns 0..r[a]-1 (other columns are not written).
 *  r          int32[nagg], device, output: kept columns per aggregate.
 * The only extra memory is a work area of AMG_LOCAL_BASES_STATIC_DOUBLES
 * doubles (1 MiB) compiled into the library, held by every GPU that loads it
 * until the process exits; nf * m beyond that size is rejected with
 * AMG_ERR_INVALID_ARG, as are host pointers and invalid row ranges, each with
 * its reason in amg_last_error().  Calls on one device share the work area:
 * calls that may overlap on the GPU race and must be ordered by the caller.
 * The first call on each device looks up the work area's device address and
 * keeps it; make that first call before capturing any stream, and do not
 * call cudaDeviceReset on that device afterwards (the kept address would be
 * stale).  The call synchronises ``stream`` before returning.
 */
#define AMG_LOCAL_BASES_STATIC_DOUBLES (1 << 17)
amg_status amg_local_bases_static(const double* W, int32_t m, const int32_t* row_start,
                                  int32_t nagg, int32_t nf, double tol, double* U, int32_t* r,
                                  void* stream);

/* Number of kernels this library has launched in the calling process so far
 * (a kernel replayed from a CUDA graph counts once per replay). */
amg_status amg_kernel_launches(int64_t* count);

void amg_destroy(amg_handle h);

/* Message of the last failed call on this host thread ("" if none). */
const char* amg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AMG_H */

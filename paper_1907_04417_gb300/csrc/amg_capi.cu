// C ABI of the library: argument checks, exception/status translation and
// handle management.  The numerical work lives in amg_setup.cu,
// amg_solve.cu and the cycle translation units.
#include <algorithm>
#include <cstring>
#include <string>

#include "amg_internal.cuh"

namespace {
thread_local std::string g_last_error;

amg_status fail(amg_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

template <class F>
amg_status guarded(F&& f) {
  try {
    g_last_error.clear();
    return f();
  } catch (const amg::Error& e) {
    cudaGetLastError();
    return fail(e.status, e.what());
  } catch (const std::bad_alloc&) {
    return fail(AMG_ERR_ALLOC, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(AMG_ERR_CUDA, e.what());
  }
}

amg_opts resolve(const amg_opts* o) {
  amg_opts d;
  amg_default_opts(&d);
  return o ? *o : d;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }
}  // namespace

namespace amg {
// For entry points defined in other translation units (amg_static.cu).
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace amg

extern "C" {

void amg_default_opts(amg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol_svd = 0.1;
  o->pre = 1;
  o->post = 1;
  o->cycle_precision = 64;
  o->rtol = 1e-8;
  o->maxit = 1000;
  o->use_graph = 1;
  o->check_every = 8;
  o->autotune = 1;
  o->outer_fp64 = 0;
  o->smoother = 0;
  o->cycle = 0;
}

const char* amg_last_error(void) { return g_last_error.c_str(); }

amg_status amg_setup_from_aggregates(const amg_csr* A, int32_t n_agg_levels, const int32_t* const* agg,
                                     const int32_t* n_nodes, const double* W, int32_t m, const amg_opts* opts,
                                     void* stream, amg_handle* out) {
  if (!out) return fail(AMG_ERR_INVALID_ARG, "out must be non-null");
  *out = nullptr;
  if (!A || !A->rowptr || !A->col || !A->val || !W) return fail(AMG_ERR_INVALID_ARG, "A, its arrays and W must be non-null");
  amg_hierarchy* h = nullptr;
  amg_status s = guarded([&]() -> amg_status {
    h = new amg_hierarchy();
    AMG_CUDA(cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking));
    AMG_CUDA(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    AMG_CUDA(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    amg_opts o = resolve(opts);
    cudaStream_t us = as_stream(stream);
    AMG_CUDA(cudaEventRecord(h->ev_in, us));
    AMG_CUDA(cudaStreamWaitEvent(h->own, h->ev_in, 0));
    amg::build_hierarchy(h, A, n_agg_levels, agg, n_nodes, W, m, o, h->own);
    AMG_CUDA(cudaStreamSynchronize(h->own));
    return AMG_OK;
  });
  if (s != AMG_OK) {
    amg_destroy(h);
    return s;
  }
  *out = h;
  return AMG_OK;
}

amg_status amg_solve(amg_handle h, const double* b, double* x, int32_t nrhs, const amg_opts* opts, void* stream,
                     amg_info* info) {
  if (!h || !b || !x) return fail(AMG_ERR_INVALID_ARG, "h, b and x must be non-null");
  if (nrhs < 1) return fail(AMG_ERR_INVALID_ARG, "nrhs must be >= 1");
  return guarded([&]() -> amg_status {
    amg_opts o = resolve(opts);
    amg_status worst = AMG_OK;
    // blocks of at most 32 columns
    for (int c0 = 0; c0 < nrhs; c0 += 32) {
      int nc = std::min(32, nrhs - c0);
      const double* bb = b;
      double* xx = x;
      std::vector<double> hb, hx;
      bool split = nrhs > 32;
      amg::Arena tmp;
      if (split) {
        // gather the column block into contiguous n x nc buffers
        size_t n = (size_t)h->n;
        std::vector<double> fb((size_t)n * nrhs), fx((size_t)n * nrhs);
        amg::copy_out(fb.data(), b, fb.size() * 8, h->own);
        amg::copy_out(fx.data(), x, fx.size() * 8, h->own);
        AMG_CUDA(cudaStreamSynchronize(h->own));
        hb.resize(n * nc);
        hx.resize(n * nc);
        for (size_t i = 0; i < n; ++i)
          for (int c = 0; c < nc; ++c) {
            hb[i * nc + c] = fb[i * nrhs + c0 + c];
            hx[i * nc + c] = fx[i * nrhs + c0 + c];
          }
        bb = hb.data();
        xx = hx.data();
      }
      amg::SolveReq rq;
      rq.nsys = 1;
      rq.n_sys = {h->n};
      rq.b = {bb};
      rq.x = {xx};
      rq.nrhs = {nc};
      rq.zero_x = false;
      amg_status s = amg::run_pcg(h, h->plan, rq, o, as_stream(stream), info ? info + c0 : nullptr);
      if (split) {
        size_t n = (size_t)h->n;
        std::vector<double> fx((size_t)n * nrhs);
        amg::copy_out(fx.data(), x, fx.size() * 8, h->own);
        AMG_CUDA(cudaStreamSynchronize(h->own));
        for (size_t i = 0; i < n; ++i)
          for (int c = 0; c < nc; ++c) fx[i * nrhs + c0 + c] = hx[i * nc + c];
        amg::copy_in(x, fx.data(), fx.size() * 8, h->own);
        AMG_CUDA(cudaStreamSynchronize(h->own));
      }
      if (s == AMG_ERR_BREAKDOWN) worst = s;
      else if (s != AMG_OK && worst == AMG_OK) worst = s;
    }
    if (worst != AMG_OK) g_last_error = worst == AMG_ERR_BREAKDOWN ? "CG breakdown (p.q <= 0 or non-finite scalar)"
                                                                   : "maximum number of iterations reached";
    return worst;
  });
}

amg_status amg_solve_batched(const amg_handle* hs, int32_t nsys, const double* const* b, double* const* x,
                             const int32_t* nrhs, const amg_opts* opts, void* stream, amg_info* info) {
  if (!hs || nsys < 1 || !b || !x || !nrhs) return fail(AMG_ERR_INVALID_ARG, "invalid batch arguments");
  return guarded([&]() -> amg_status {
    std::vector<amg_hierarchy*> v(hs, hs + nsys);
    for (int s = 0; s < nsys; ++s) {
      AMG_REQUIRE(v[s] && b[s] && x[s], "null handle or vector in batch");
      AMG_REQUIRE(nrhs[s] >= 1 && nrhs[s] <= 32, "nrhs[s] must be in [1, 32]");
    }
    amg_opts o = resolve(opts);
    amg_hierarchy* h0 = v[0];
    amg::Plan* plan = nullptr;
    if (nsys == 1) {
      plan = &h0->plan;
    } else {
      auto it = h0->batches.find(v);
      if (it == h0->batches.end()) {
        std::unique_ptr<amg::Plan> p(new amg::Plan());
        AMG_CUDA(cudaStreamSynchronize(as_stream(stream)));
        amg::build_batch_plan(*p, v, h0->own);
        it = h0->batches.emplace(v, std::move(p)).first;
      }
      plan = it->second.get();
    }
    amg::SolveReq rq;
    rq.nsys = nsys;
    for (int s = 0; s < nsys; ++s) {
      rq.n_sys.push_back(v[s]->n);
      rq.b.push_back(b[s]);
      rq.x.push_back(x[s]);
      rq.nrhs.push_back(nrhs[s]);
    }
    rq.zero_x = false;
    amg_status s = amg::run_pcg(h0, *plan, rq, o, as_stream(stream), info);
    if (s != AMG_OK) g_last_error = s == AMG_ERR_BREAKDOWN ? "CG breakdown" : "maximum number of iterations reached";
    return s;
  });
}

amg_status amg_adjoint(amg_handle h, const double* g, const double* x, int32_t nrhs, double* lambda,
                       double* grad_val, const amg_opts* opts, void* stream, amg_info* info) {
  if (!h || !g || !x || !lambda || !grad_val) return fail(AMG_ERR_INVALID_ARG, "null argument");
  if (nrhs < 1 || nrhs > 32) return fail(AMG_ERR_INVALID_ARG, "nrhs must be in [1, 32]");
  return guarded([&]() -> amg_status {
    amg_opts o = resolve(opts);
    amg::SolveReq rq;
    rq.nsys = 1;
    rq.n_sys = {h->n};
    rq.b = {g};
    rq.x = {lambda};
    rq.nrhs = {nrhs};
    rq.zero_x = true;
    amg_status s = amg::run_pcg(h, h->plan, rq, o, as_stream(stream), info);
    amg::run_adjoint_grad(h, lambda, x, nrhs, grad_val, as_stream(stream));
    if (s != AMG_OK) g_last_error = "adjoint solve did not converge";
    return s;
  });
}

amg_status amg_vcycle(amg_handle h, const double* r, double* z, int32_t nrhs, const amg_opts* opts,
                      void* stream) {
  if (!h || !r || !z) return fail(AMG_ERR_INVALID_ARG, "null argument");
  return guarded([&]() -> amg_status {
    amg_opts o = resolve(opts);
    amg::run_vcycle(h, h->plan, r, z, nrhs, o, as_stream(stream));
    return AMG_OK;
  });
}

amg_status amg_bootstrap_test(const amg_handle* hs, int32_t r, double* x, int32_t nrhs, int32_t nu,
                              int32_t symmetric, const amg_opts* opts, void* stream, double* rho,
                              double* anorm) {
  if (!hs || !x || r < 1) return fail(AMG_ERR_INVALID_ARG, "null argument or r < 1");
  if (nrhs < 1 || nrhs > 32) return fail(AMG_ERR_INVALID_ARG, "nrhs must be in [1, 32]");
  if (nu < 1) return fail(AMG_ERR_INVALID_ARG, "nu must be >= 1");
  for (int k = 0; k < r; ++k)
    if (!hs[k]) return fail(AMG_ERR_INVALID_ARG, "null hierarchy");
  return guarded([&]() -> amg_status {
    amg_opts o = resolve(opts);
    std::vector<amg_hierarchy*> v(hs, hs + r);
    amg::run_bootstrap_test(v, x, nrhs, nu, symmetric, o, as_stream(stream), rho, anorm);
    return AMG_OK;
  });
}

amg_status amg_pairwise_matching(const amg_csr* A, const double* w, int32_t* mate, void* stream) {
  if (!A || !w || !mate) return fail(AMG_ERR_INVALID_ARG, "null argument");
  return guarded([&]() -> amg_status {
    amg::run_pairwise_matching(A, w, mate, as_stream(stream));
    return AMG_OK;
  });
}

amg_status amg_pairwise_step(const amg_csr* A, const double* w, int32_t* agg, int32_t* nc, int32_t* rowptr_c,
                             int32_t* col_c, double* val_c, int32_t* nnz_c, double* wc, void* stream) {
  if (!A || !w || !agg || !nc || !rowptr_c || !col_c || !val_c || !nnz_c || !wc)
    return fail(AMG_ERR_INVALID_ARG, "null argument");
  return guarded([&]() -> amg_status {
    amg::run_pairwise_step(A, w, agg, nc, rowptr_c, col_c, val_c, nnz_c, wc, as_stream(stream));
    return AMG_OK;
  });
}

amg_status amg_hierarchy_info(amg_handle h, amg_hier_info* info) {
  if (!h || !info) return fail(AMG_ERR_INVALID_ARG, "null argument");
  std::memset(info, 0, sizeof(*info));
  const amg::Plan& P = h->plan;
  info->levels = P.L;
  info->m = P.m;
  long long nnz0 = P.lev[0].nnz, tot = 0;
  double cr = 0;
  for (int k = 0; k < P.L && k < 16; ++k) {
    info->n_level[k] = P.lev[k].n;
    info->nnz_level[k] = P.lev[k].nnz;
    tot += P.lev[k].nnz;
    if (k > 0) cr += (double)P.lev[k - 1].n / P.lev[k].n;
  }
  info->opc = (double)tot / (double)nnz0;
  info->cr = P.L > 1 ? cr / (P.L - 1) : 1.0;
  info->truncated_aggs = h->truncated;
  info->device_bytes = (int64_t)P.arena->bytes;
  return AMG_OK;
}

amg_status amg_restriction_info(amg_handle h, int32_t k, int32_t* by_r, int64_t* entries,
                                int32_t* values_per_entry) {
  if (!h) return fail(AMG_ERR_INVALID_ARG, "null handle");
  return guarded([&]() -> amg_status {
    const amg::Plan& P = h->plan;
    AMG_REQUIRE(k >= 0 && k + 1 < P.L, "transfer out of range");
    const amg::Transfer& T = P.tr[k];
    if (by_r) *by_r = T.rf_last;
    if (entries) *entries = T.rf_state == 1 ? T.rf_entries : 0;
    if (values_per_entry) *values_per_entry = T.rf_state == 1 ? T.rf_rs : 0;
    return AMG_OK;
  });
}

amg_status amg_level_colours(amg_handle h, int32_t k, int32_t* colour, int32_t* ncolours) {
  if (!h) return fail(AMG_ERR_INVALID_ARG, "null handle");
  return guarded([&]() -> amg_status {
    int nc = amg::level_colours(h, k, colour, h->own);
    if (ncolours) *ncolours = nc;
    return AMG_OK;
  });
}

amg_status amg_export_level(amg_handle h, int32_t k, int64_t* sizes, int32_t* rowptr, int32_t* col, double* val,
                            int32_t* perm, int32_t* agg_id, int32_t* r, int32_t* row_start, double* pval) {
  if (!h || !sizes) return fail(AMG_ERR_INVALID_ARG, "null argument");
  return guarded([&]() -> amg_status {
    amg::Plan& P = h->plan;
    AMG_REQUIRE(k >= 0 && k < P.L, "level out of range");
    const amg::Level& L = P.lev[k];
    sizes[0] = L.n;
    sizes[1] = L.nnz;
    sizes[2] = k > 0 ? P.tr[k - 1].nagg : 0;
    sizes[3] = k > 0 ? P.tr[k - 1].npval : 0;
    sizes[4] = k > 0 ? P.lev[k - 1].n : 0;
    sizes[5] = P.m;
    cudaStream_t st = h->own;
    if (rowptr) AMG_CUDA(cudaMemcpyAsync(rowptr, L.rowptr, (L.n + 1) * 4, cudaMemcpyDeviceToHost, st));
    if (col) AMG_CUDA(cudaMemcpyAsync(col, L.col, L.nnz * 4, cudaMemcpyDeviceToHost, st));
    if (val) AMG_CUDA(cudaMemcpyAsync(val, L.val64, L.nnz * 8, cudaMemcpyDeviceToHost, st));
    if (perm && k == 0) std::memcpy(perm, h->h_perm[0].data(), h->h_perm[0].size() * 4);
    if (k > 0) {
      const amg::Transfer& T = P.tr[k - 1];
      if (agg_id) std::memcpy(agg_id, h->h_perm[k].data(), h->h_perm[k].size() * 4);
      if (r) std::memcpy(r, h->h_r[k].data(), h->h_r[k].size() * 4);
      if (row_start) std::memcpy(row_start, T.h_row_start.data(), T.h_row_start.size() * 4);
      if (pval) AMG_CUDA(cudaMemcpyAsync(pval, T.p64, T.npval * 8, cudaMemcpyDeviceToHost, st));
    }
    AMG_CUDA(cudaStreamSynchronize(st));
    return AMG_OK;
  });
}

amg_status amg_timer_enable(amg_handle h, int32_t kernel_id, int32_t enable) {
  if (!h) return fail(AMG_ERR_INVALID_ARG, "null handle");
  h->timer.kernel = kernel_id;
  h->timer.on = enable != 0;
  h->timer.total_ms = 0;
  h->timer.launches = 0;
  return AMG_OK;
}

amg_status amg_timer_read(amg_handle h, double* total_ms, int64_t* launches) {
  if (!h || !total_ms || !launches) return fail(AMG_ERR_INVALID_ARG, "null argument");
  *total_ms = h->timer.total_ms;
  *launches = h->timer.launches;
  return AMG_OK;
}

amg_status amg_kernel_launches(int64_t* count) {
  if (!count) return fail(AMG_ERR_INVALID_ARG, "null argument");
  *count = amg::launches_total();
  return AMG_OK;
}

void amg_destroy(amg_handle h) {
  if (!h) return;
  if (h->own) cudaStreamSynchronize(h->own);
  h->batches.clear();
  h->plan.ws.clear();
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
}

}  // extern "C"

// Host-side launchers of the V-cycle kernels, templated on the cycle
// precision TC.  Each precision is instantiated in its own translation unit
// (amg_cycle_f64.cu, amg_cycle_f32.cu) so that they compile in parallel.
#pragma once

#include <algorithm>
#include <map>
#include <type_traits>
#include <utility>

#include "amg_kernels.cuh"

namespace amg {

template <int V>
using ic = std::integral_constant<int, V>;

template <class F>
inline void dispatch_k(int K, F&& f) {
  switch (K) {
    case 1: f(ic<1>{}); break;
    case 2: f(ic<2>{}); break;
    case 4: f(ic<4>{}); break;
    case 8: f(ic<8>{}); break;
    case 16: f(ic<16>{}); break;
    case 32: f(ic<32>{}); break;
    default: throw Error(AMG_ERR_INVALID_ARG, "internal: unsupported column count " + std::to_string(K));
  }
}

// Lanes per row along the non-zeros: {2..32} for one column, {1..8} otherwise.
template <class F>
inline void dispatch_nzl(int K, int nzl, F&& f) {
  if (K == 1) {
    switch (nzl) {
      case 2: f(ic<2>{}); return;
      case 4: f(ic<4>{}); return;
      case 8: f(ic<8>{}); return;
      case 16: f(ic<16>{}); return;
      case 32: f(ic<32>{}); return;
    }
  } else {
    switch (nzl) {
      case 1: f(ic<1>{}); return;
      case 2: f(ic<2>{}); return;
      case 4: f(ic<4>{}); return;
      case 8: f(ic<8>{}); return;
    }
  }
  throw Error(AMG_ERR_INVALID_ARG, "internal: unsupported lane layout");
}

template <typename TC>
inline int max_nzl(int K) {
  int cpt = (K * (int)sizeof(TC) >= 16) ? 16 / (int)sizeof(TC) : K;
  int cl = K / cpt;
  int m = 32 / cl;
  if (K == 1) return 32;
  return m < 8 ? m : 8;
}

template <typename TC>
inline const TC* vals(const Level& L) {
  if constexpr (std::is_same<TC, double>::value) return L.val64; else return L.val32;
}
template <typename TC>
inline const TC* dinvs(const Level& L) {
  if constexpr (std::is_same<TC, double>::value) return L.dinv64; else return L.dinv32;
}
template <typename TC>
inline const TC* pvals(const Transfer& T) {
  if constexpr (std::is_same<TC, double>::value) return T.p64; else return T.p32;
}

// Raise the dynamic shared-memory limit of a kernel once (and never while a
// stream is being captured: the first call of every launcher happens in the
// eager start-up sequence of a solve).
template <typename Kern>
inline void ensure_smem(Kern k, size_t bytes) {
  static std::map<const void*, size_t> granted;
  const void* key = reinterpret_cast<const void*>(k);
  auto it = granted.find(key);
  size_t have = it == granted.end() ? 48 * 1024 : it->second;
  if (bytes > have) {
    AMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    granted[key] = bytes;
  }
}

template <typename TC>
void launch_smooth(int K, int nzl, const Level& L, const RPart& rp, const TC* f, const TC* u, TC* v,
                   const int* done, cudaStream_t st);
template <typename TC>
void launch_restrict(int K, int nzl, const Level& L, const Transfer& T, const TPart& tp, const Level& C,
                     bool smooth_next, const TC* f, const TC* u, TC* fc, TC* uc, const int* done,
                     cudaStream_t st);
// f0, dinv0 (optional): u starts from D^{-1} f0 instead of its stored value.
template <typename TC>
void launch_prolong(int K, const Transfer& T, const TPart& tp, const TC* uc, TC* u, const int* done,
                    cudaStream_t st, const TC* f0 = nullptr, const TC* dinv0 = nullptr);
template <typename TC>
void launch_coarse(int K, const Coarsest& C, const TC* f, TC* u, const int* done, cudaStream_t st);
template <typename TC>
void launch_post0(int K, int nzl, const Level& L, const RPart& rp, const TC* f, const TC* u, const double* r,
                  const float* rlo, TC* z, const KState& ks, int mode, cudaStream_t st, int grid = 0);
template <typename TC>
void launch_update(int K, const Level& L, const RPart& rp, double* x, double* r, const double* p,
                   const double* q, TC* u0, TC* f0, const KState& ks, cudaStream_t st);
template <typename TC>
void launch_presmooth0(int K, const Level& L, const RPart& rp, const double* r, TC* u0, TC* f0,
                       const int* done, cudaStream_t st);

// Grouped coarse-level kernels (columns K >= 8, at most 8 rows per group and
// 8 coarse dofs per aggregate); the caller checks grouped_ok first.  jl lanes
// split a group's pattern columns (1, 2 or 4, at most 32 / CL).
inline bool grouped_ok(int K, const Level& L) { return K >= 8 && L.grp_ok && L.grp_rmax <= 8; }
template <typename TC>
inline bool grouped_jl_ok(int K, int jl) {
  const int cpt = (K * (int)sizeof(TC) >= 16) ? 16 / (int)sizeof(TC) : K;
  return (jl == 1 || jl == 2 || jl == 4) && (K / cpt) * jl <= 32;
}

template <class F>
inline void dispatch_jl(int jl, F&& f) {
  switch (jl) {
    case 1: f(ic<1>{}); return;
    case 2: f(ic<2>{}); return;
    case 4: f(ic<4>{}); return;
  }
  throw Error(AMG_ERR_INVALID_ARG, "internal: unsupported group lane split");
}

template <typename TC>
inline void launch_smooth_g(int K, int jl, const Level& L, const TC* f, const TC* u, TC* v, const int* done,
                            cudaStream_t st, int* err) {
  Stage sg = L.gsg;
  sg.err = err;
  if (sizeof(TC) != 4) sg.enabled = 0;
  const size_t smem = pipe_bytes(sg, 1, 1);
  dispatch_k(K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    dispatch_jl(jl, [&](auto jc) {
      constexpr int JL = decltype(jc)::value;
      if constexpr (KK >= 8 && VT<TC, KK>::CL * JL <= 32) {
        const int grid = (L.ngrp + GROUPS_PER_CTA - 1) / GROUPS_PER_CTA;
        auto go = [&](auto kern) {
          ensure_smem(kern, smem);
          kern<<<grid, BS, smem, st>>>(L.ngrp, L.gstart, L.rowptr, L.col, vals<TC>(L), dinvs<TC>(L), f, u, v, done,
                                       sg);
        };
        if (L.grp_rmax <= 4) go(k_smooth_g<TC, KK, 4, JL>);
        else go(k_smooth_g<TC, KK, 8, JL>);
      } else {
        throw Error(AMG_ERR_INVALID_ARG, "internal: grouped kernels need at least 8 columns");
      }
    });
  });
  AMG_LAUNCH_CHECK();
}

template <typename TC>
inline void launch_restrict_g(int K, const Level& L, const Transfer& T, const TPart& tp, const Level& C,
                              bool smooth_next, const TC* f, const TC* u, TC* fc, TC* uc, const int* done,
                              cudaStream_t st) {
  Stage sg = T.gsg;
  sg.err = tp.sg.err;
  if (sizeof(TC) != 4) sg.enabled = 0;
  const size_t smem = pipe_bytes(sg, 1, 1);
  dispatch_k(K, [&](auto kc) {
    constexpr int KK = decltype(kc)::value;
    dispatch_jl(tp.jl, [&](auto jc) {
      constexpr int JL = decltype(jc)::value;
      if constexpr (KK >= 8 && VT<TC, KK>::CL * JL <= 32) {
        auto go = [&](auto kern) {
          ensure_smem(kern, smem);
          kern<<<T.nagg, RG_WARPS * 32, smem, st>>>(T.nagg, T.row_start, T.coarse_start, T.blk_start, pvals<TC>(T),
                                                    L.gstart, T.gagg, L.rowptr, L.col, vals<TC>(L), f, u, fc,
                                                    smooth_next ? uc : nullptr,
                                                    smooth_next ? dinvs<TC>(C) : nullptr, done, sg);
        };
        if (L.grp_rmax <= 4 && tp.ra_max <= 4) go(k_restrict_g<TC, KK, 4, 4, JL>);
        else if (L.grp_rmax <= 4) go(k_restrict_g<TC, KK, 4, 8, JL>);
        else if (tp.ra_max <= 4) go(k_restrict_g<TC, KK, 8, 4, JL>);
        else go(k_restrict_g<TC, KK, 8, 8, JL>);
      } else {
        throw Error(AMG_ERR_INVALID_ARG, "internal: grouped kernels need at least 8 columns");
      }
    });
  });
  AMG_LAUNCH_CHECK();
}

// Grid of a kernel whose warps walk their work: at most ``need`` CTAs of
// BS threads, at most as many as stay resident on the device at once (the
// occupancy of each kernel is looked up once per device).
template <typename Kern>
inline int resident_grid(Kern k, long long need) {
  static std::map<std::pair<const void*, int>, int> cap;
  int dev = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_pair(reinterpret_cast<const void*>(k), dev);
  auto it = cap.find(key);
  if (it == cap.end()) {
    int per_sm = 0, sms = 0;
    AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BS, 0));
    it = cap.emplace(key, std::max(per_sm, 1) * std::max(sms, 1)).first;
  }
  return (int)std::max(1LL, std::min(need, (long long)it->second));
}

template <typename TC>
inline const TC* rfvals(const Transfer& T) {
  if constexpr (std::is_same<TC, double>::value) return T.rf_v64; else return T.rf_v32;
}

// fc = R f (and uc = D_c^{-1} fc) with the aggregate-grouped R of the
// transfer (built: T.rf_state == 1); a grid of as many CTAs as stay
// resident, each warp walking aggregates.
// kind 1: a warp per aggregate, its lane groups splitting the pattern
// (k_group_rf); kind 2: a slot of lanes per aggregate (k_group_rs)
template <typename TC>
void launch_restrict_rf(int K, const Transfer& T, const Level& C, bool smooth_next, const TC* f, TC* fc, TC* uc,
                        const int* done, cudaStream_t st, int kind);

template <typename TC>
inline const TC* gwvals(const Level& L) {
  if constexpr (std::is_same<TC, double>::value) return L.gw_v64; else return L.gw_v32;
}
// Lane code of the warp-per-group sweep of a grouped level (launch_smooth's
// nzl; codes <= 0 above it are the CTA-per-groups sweep, -jl lanes per split)
constexpr int NZL_GROUP_WARP = -16;
// ... and of the slot form (a slot of lanes per row group, k_group_rs)
constexpr int NZL_GROUP_SLOT = -17;

// shared memory of a staged SpMV kernel reading one value array of type TC
template <typename TC>
inline size_t csr_stage_bytes(const Stage& sg) {
  return stage_bytes(sg, sizeof(TC) == 4 ? 1 : 0, sizeof(TC) == 8 ? 1 : 0);
}

#define AMG_DEFINE_LAUNCHERS(TC)                                                                       \
  template <>                                                                                          \
  void launch_smooth<TC>(int K, int nzl, const Level& L, const RPart& rp, const TC* f, const TC* u,   \
                         TC* v, const int* done, cudaStream_t st) {                                    \
    if (nzl == NZL_GROUP_WARP || nzl == NZL_GROUP_SLOT) { /* grouped level, entry-major copy */     \
      if (L.gw_state != 1) throw Error(AMG_ERR_INVALID_ARG, "internal: grouped copy not built");      \
      dispatch_k(K, [&](auto kc) {                                                                     \
        constexpr int KK = decltype(kc)::value;                                                        \
        if (nzl == NZL_GROUP_WARP) {                                                                   \
          auto go = [&](auto kern) {                                                                   \
            const int grid = resident_grid(kern, ((long long)L.ngrp + NWARP - 1) / NWARP);             \
            kern<<<grid, BS, 0, st>>>(L.ngrp, L.gw_ptr, L.gw_col, gwvals<TC>(L), L.gstart, u, v,        \
                                      nullptr, dinvs<TC>(L), f, done);                                 \
          };                                                                                           \
          if (L.gw_rs == 4) go(k_group_rf<TC, KK, 4, 1>);                                              \
          else go(k_group_rf<TC, KK, 8, 1>);                                                           \
        } else {                                                                                       \
          constexpr int SPW = 32 / VT<TC, KK>::CL;                                                     \
          auto go = [&](auto kern) {                                                                   \
            const long long passes = ((long long)L.ngrp + SPW - 1) / SPW;                              \
            const int grid = resident_grid(kern, (passes + NWARP - 1) / NWARP);                        \
            kern<<<grid, BS, 0, st>>>(L.ngrp, L.gw_zero, L.gw_ptr, L.gw_col, gwvals<TC>(L), L.gstart,  \
                                      u, v, nullptr, dinvs<TC>(L), f, done);                           \
          };                                                                                           \
          if (L.gw_rs == 4) go(k_group_rs<TC, KK, 4, 1>);                                              \
          else go(k_group_rs<TC, KK, 8, 1>);                                                           \
        }                                                                                              \
      });                                                                                              \
      AMG_LAUNCH_CHECK();                                                                              \
      return;                                                                                          \
    }                                                                                                  \
    if (nzl <= 0) { /* grouped coarse level, -nzl lanes per group column split (0: one) */            \
      launch_smooth_g<TC>(K, nzl < 0 ? -nzl : 1, L, f, u, v, done, st, rp.sg.err);                    \
      return;                                                                                          \
    }                                                                                                  \
    size_t smem = csr_stage_bytes<TC>(rp.sg);                                                          \
    dispatch_k(K, [&](auto kc) {                                                                       \
      constexpr int KK = decltype(kc)::value;                                                          \
      dispatch_nzl(K, nzl, [&](auto nc) {                                                              \
        constexpr int NZ = decltype(nc)::value;                                                        \
        if constexpr (VT<TC, KK>::CL * NZ <= 32) {                                                     \
          auto kern = k_smooth<TC, KK, NZ>;                                                            \
          ensure_smem(kern, smem);                                                                     \
          kern<<<rp.ncta, BS, smem, st>>>(rp.cta_row, L.rowptr, L.col, vals<TC>(L), dinvs<TC>(L), f,   \
                                          u, v, done, rp.sg);                                          \
        } else {                                                                                       \
          throw Error(AMG_ERR_INVALID_ARG, "internal: lane layout too wide");                         \
        }                                                                                              \
      });                                                                                              \
    });                                                                                                \
    AMG_LAUNCH_CHECK();                                                                                \
  }                                                                                                    \
  template <>                                                                                          \
  void launch_restrict<TC>(int K, int nzl, const Level& L, const Transfer& T, const TPart& tp,         \
                           const Level& C, bool smooth_next, const TC* f, const TC* u, TC* fc, TC* uc, \
                           const int* done, cudaStream_t st) {                                         \
    if (tp.warp == 2) {                                                                                \
      launch_restrict_g<TC>(K, L, T, tp, C, smooth_next, f, u, fc, uc, done, st);                     \
      return;                                                                                          \
    }                                                                                                  \
    if (nzl <= 0) nzl = 1; /* the level is grouped; the CSR kernels take one lane group per row */    \
    if (tp.warp) {                                                                                     \
      dispatch_k(K, [&](auto kc) {                                                                     \
        constexpr int KK = decltype(kc)::value;                                                        \
        auto go = [&](auto rc) {                                                                       \
          constexpr int RM = decltype(rc)::value;                                                      \
          Stage wsg = tp.wsg; /* kind 3 stages the CTA's slice, kind 1 reads global memory */          \
          wsg.err = tp.sg.err;                                                                         \
          if (sizeof(TC) != 4 || tp.warp != 3) wsg.enabled = 0;                                        \
          const size_t wsm = pipe_bytes(wsg, 1, 1);                                                    \
          auto kern = wsg.enabled ? k_restrict_w<TC, KK, RM, true> : k_restrict_w<TC, KK, RM, false>;  \
          ensure_smem(kern, wsm);                                                                      \
          kern<<<(T.nagg + NWARP - 1) / NWARP, BS, wsm, st>>>(                                         \
              T.nagg, T.row_start, T.coarse_start, T.blk_start, pvals<TC>(T), L.rowptr, L.col,         \
              vals<TC>(L), f, u, fc, smooth_next ? uc : nullptr, smooth_next ? dinvs<TC>(C) : nullptr, \
              done, wsg);                                                                              \
        };                                                                                             \
        if (tp.ra_max <= 4) go(std::integral_constant<int, 4>{});                                      \
        else if (tp.ra_max <= 8) go(std::integral_constant<int, 8>{});                                 \
        else throw Error(AMG_ERR_INVALID_ARG, "internal: warp restriction needs r_a <= 8");           \
      });                                                                                              \
      AMG_LAUNCH_CHECK();                                                                              \
      return;                                                                                          \
    }                                                                                                  \
    size_t smem = restrict_stage_bytes<TC>(tp.sg) +                                                    \
                  transfer_smem<TC>(tp.rows_max, tp.p_max, tp.a_max, tp.c_max, K, true);              \
    dispatch_k(K, [&](auto kc) {                                                                       \
      constexpr int KK = decltype(kc)::value;                                                          \
      dispatch_nzl(K, nzl, [&](auto nc) {                                                              \
        constexpr int NZ = decltype(nc)::value;                                                        \
        if constexpr (VT<TC, KK>::CL * NZ <= 32) {                                                     \
          auto kern = k_restrict<TC, KK, NZ>;                                                          \
          ensure_smem(kern, smem);                                                                     \
          kern<<<tp.ncta, BS, smem, st>>>(tp.cta_agg, T.row_start, T.coarse_start, T.blk_start,        \
                                          pvals<TC>(T), L.rowptr, L.col, vals<TC>(L), f, u, fc,        \
                                          smooth_next ? uc : nullptr,                                  \
                                          smooth_next ? dinvs<TC>(C) : nullptr, done, tp.rows_max,     \
                                          tp.p_max, tp.a_max, tp.sg, tp.ra_max);                       \
        } else {                                                                                       \
          throw Error(AMG_ERR_INVALID_ARG, "internal: lane layout too wide");                         \
        }                                                                                              \
      });                                                                                              \
    });                                                                                                \
    AMG_LAUNCH_CHECK();                                                                                \
  }                                                                                                    \
  template <>                                                                                          \
  void launch_restrict_rf<TC>(int K, const Transfer& T, const Level& C, bool smooth_next, const TC* f, \
                              TC* fc, TC* uc, const int* done, cudaStream_t st, int kind) {            \
    if (T.rf_state != 1) throw Error(AMG_ERR_INVALID_ARG, "internal: restriction operator R not built"); \
    TC* u2 = smooth_next ? uc : nullptr;                                                               \
    const TC* dc = smooth_next ? dinvs<TC>(C) : nullptr;                                               \
    dispatch_k(K, [&](auto kc) {                                                                       \
      constexpr int KK = decltype(kc)::value;                                                          \
      if (kind == 2) {                                                                                 \
        constexpr int SPW = 32 / VT<TC, KK>::CL;                                                       \
        auto go = [&](auto kern) {                                                                     \
          const long long passes = ((long long)T.nagg + SPW - 1) / SPW;                                \
          const int grid = resident_grid(kern, (passes + NWARP - 1) / NWARP);                          \
          kern<<<grid, BS, 0, st>>>(T.nagg, T.rf_zero, T.rf_ptr, T.rf_col, rfvals<TC>(T), T.coarse_start, \
                                    f, fc, u2, dc, nullptr, done);                                     \
        };                                                                                             \
        if (T.rf_rs == 4) go(k_group_rs<TC, KK, 4, 0>);                                                \
        else go(k_group_rs<TC, KK, 8, 0>);                                                             \
      } else {                                                                                         \
        auto go = [&](auto kern) {                                                                     \
          const int grid = resident_grid(kern, ((long long)T.nagg + NWARP - 1) / NWARP);               \
          kern<<<grid, BS, 0, st>>>(T.nagg, T.rf_ptr, T.rf_col, rfvals<TC>(T), T.coarse_start, f, fc,   \
                                    u2, dc, nullptr, done);                                            \
        };                                                                                             \
        if (T.rf_rs == 4) go(k_group_rf<TC, KK, 4, 0>);                                                \
        else go(k_group_rf<TC, KK, 8, 0>);                                                             \
      }                                                                                                \
    });                                                                                                \
    AMG_LAUNCH_CHECK();                                                                                \
  }                                                                                                    \
  template <>                                                                                          \
  void launch_prolong<TC>(int K, const Transfer& T, const TPart& tp, const TC* uc, TC* u,             \
                          const int* done, cudaStream_t st, const TC* f0, const TC* dinv0) {           \
    if (tp.pwarp && tp.ra_max <= 8) {                                                                  \
      dispatch_k(K, [&](auto kc) {                                                                     \
        constexpr int KK = decltype(kc)::value;                                                        \
        const int grid = (T.nagg + NWARP - 1) / NWARP;                                                 \
        if (tp.ra_max <= 4)                                                                            \
          k_prolong_w<TC, KK, 4><<<grid, BS, 0, st>>>(T.nagg, T.row_start, T.coarse_start, T.blk_start, \
                                                      pvals<TC>(T), uc, u, done, f0, dinv0);           \
        else                                                                                           \
          k_prolong_w<TC, KK, 8><<<grid, BS, 0, st>>>(T.nagg, T.row_start, T.coarse_start, T.blk_start, \
                                                      pvals<TC>(T), uc, u, done, f0, dinv0);           \
      });                                                                                              \
      AMG_LAUNCH_CHECK();                                                                              \
      return;                                                                                          \
    }                                                                                                  \
    size_t smem = transfer_smem<TC>(tp.rows_max, tp.p_max, tp.a_max, tp.c_max, K, false);             \
    dispatch_k(K, [&](auto kc) {                                                                       \
      constexpr int KK = decltype(kc)::value;                                                          \
      auto kern = k_prolong<TC, KK>;                                                                   \
      ensure_smem(kern, smem);                                                                         \
      kern<<<tp.ncta, BS, smem, st>>>(tp.cta_agg, T.row_start, T.coarse_start, T.blk_start,            \
                                      pvals<TC>(T), uc, u, done, tp.rows_max, tp.p_max, tp.a_max, f0,  \
                                      dinv0);                                                          \
    });                                                                                                \
    AMG_LAUNCH_CHECK();                                                                                \
  }                                                                                                    \
  template <>                                                                                          \
  void launch_coarse<TC>(int K, const Coarsest& C, const TC* f, TC* u, const int* done,                \
                         cudaStream_t st) {                                                            \
    int grid = (int)(((long long)C.n * K + COARSE_BS - 1) / COARSE_BS);                                 \
    dispatch_k(K, [&](auto kc) {                                                                       \
      constexpr int KK = decltype(kc)::value;                                                          \
      k_coarse<TC, KK><<<grid, COARSE_BS, 0, st>>>(C.n, C.nblk, C.blk_off, C.inv_off, C.inv, f, u,     \
                                                   done);                                              \
    });                                                                                                \
    AMG_LAUNCH_CHECK();                                                                                \
  }                                                                                                    \
  template <>                                                                                          \
  void launch_post0<TC>(int K, int nzl, const Level& L, const RPart& rp, const TC* f, const TC* u,    \
                        const double* r, const float* rlo, TC* z, const KState& ks, int mode,          \
                        cudaStream_t st, int grid) {                                                   \
    /* float matrices stage through the pipeline (two buffers when persistent) */                      \
    size_t smem = sizeof(TC) == 4 ? pipe_bytes(rp.sg, 1, grid > 0 ? 2 : 1) : csr_stage_bytes<TC>(rp.sg); \
    dispatch_k(K, [&](auto kc) {                                                                       \
      constexpr int KK = decltype(kc)::value;                                                          \
      dispatch_nzl(K, nzl, [&](auto nc) {                                                              \
        constexpr int NZ = decltype(nc)::value;                                                        \
        if constexpr (VT<TC, KK>::CL * NZ <= 32) {                                                     \
          auto kern = rlo ? (rp.sg.enabled ? k_post0<TC, KK, NZ, true, true> : k_post0<TC, KK, NZ, true, false>) \
                          : (rp.sg.enabled ? k_post0<TC, KK, NZ, false, true> : k_post0<TC, KK, NZ, false, false>); \
          if constexpr (NZ == 1) { /* rows of at most 9 entries: batches of 9 */                       \
            if (L.max_row_len <= 9)                                                                    \
              kern = rlo ? (rp.sg.enabled ? k_post0<TC, KK, 1, true, true, 9> : k_post0<TC, KK, 1, true, false, 9>) \
                         : (rp.sg.enabled ? k_post0<TC, KK, 1, false, true, 9> : k_post0<TC, KK, 1, false, false, 9>); \
          }                                                                                            \
          ensure_smem(kern, smem);                                                                     \
          kern<<<grid > 0 ? grid : rp.ncta, BS, smem, st>>>(rp.cta_row, L.rowptr, L.col, vals<TC>(L), \
                                                            dinvs<TC>(L), f, u, r, rlo, z, ks, mode,   \
                                                            rp.sg, rp.ncta);                           \
        } else {                                                                                       \
          throw Error(AMG_ERR_INVALID_ARG, "internal: lane layout too wide");                         \
        }                                                                                              \
      });                                                                                              \
    });                                                                                                \
    AMG_LAUNCH_CHECK();                                                                                \
  }                                                                                                    \
  template <>                                                                                          \
  void launch_update<TC>(int K, const Level& L, const RPart& rp, double* x, double* r,                 \
                         const double* p, const double* q, TC* u0, TC* f0, const KState& ks,           \
                         cudaStream_t st) {                                                            \
    dispatch_k(K, [&](auto kc) {                                                                       \
      constexpr int KK = decltype(kc)::value;                                                          \
      k_cg_update<TC, KK><<<rp.ncta, BS, 0, st>>>(rp.cta_row, x, r, p, q, L.dinv64, u0, f0, ks);      \
    });                                                                                                \
    AMG_LAUNCH_CHECK();                                                                                \
  }                                                                                                    \
  template <>                                                                                          \
  void launch_presmooth0<TC>(int K, const Level& L, const RPart& rp, const double* r, TC* u0, TC* f0,  \
                             const int* done, cudaStream_t st) {                                       \
    dispatch_k(K, [&](auto kc) {                                                                       \
      constexpr int KK = decltype(kc)::value;                                                          \
      k_presmooth0<TC, KK><<<rp.ncta, BS, 0, st>>>(rp.cta_row, r, L.dinv64, u0, f0, done);            \
    });                                                                                                \
    AMG_LAUNCH_CHECK();                                                                                \
  }

}  // namespace amg

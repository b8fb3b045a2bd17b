// Host-side launchers of the kernel templates, dispatched over block size and
// precision.  Included once per translation unit of instantiations (mr_k2.cu,
// mr_k2s.cu, mr_k2t.cu, mr_k3.cu, mr_k3s.cu).
#pragma once
#include <algorithm>
#include <cstdio>

#include "mr_kernels.cuh"

namespace mr {

template <typename K>
static void prep_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, const LaunchCfg& lc, int mult) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  if (mult > 0 && mult < per_sm) per_sm = mult;
  return lc.num_sms * per_sm;
}

static inline int flat_grid(const PoolView& pv, int threads) {
  int64_t g = (pv.cap + threads - 1) / threads;
  if (g > 4096) g = 4096;
  return (int)(g < 1 ? 1 : g);
}

// Lists up to this length are scanned by the last CTA of the kernel that wrote
// the counts (one CTA, a few passes) instead of a separate scan launch.
constexpr int64_t kFusedScanMax = 8192;

// ---------------------------------------------------------------- stage ------
// 2D blocks of 17^2 nodes: 128-thread CTAs, so small grids run in one wave.
template <int D, int B>
struct Threads { static constexpr int value = (D == 2 && B == 17) ? 128 : 256; };

template <int D, int B, int RHS, typename TS, typename TY>
static void stage_impl(const PoolView& pv, const Fields& f, int stage, const StageArgs& sa,
                       const LaunchCfg& lc, cudaStream_t st) {
  constexpr int threads = Threads<D, B>::value;
  const int nv = 1;
  using Bx = Box<D, B, 2>;
  const size_t smem = kRingBytesD<D> + sizeof(TY) * nv * (Bx::TILE + Bx::CBOX + Bx::SCR) + (D == 2 ? 4 * Bx::NPTS : 0);
  TY* ynext = (TY*)(stage == 1 ? f.Yb : f.Ya);
  // 2D: one warp per block when the grid holds enough blocks to fill the GPU
  // several times over (or as tuned), else one CTA per block (shorter latency)
  const bool warp_form = lc.stage_form == 1 || (lc.stage_form < 0 && lc.n_hint >= 8 * lc.num_sms);
  if constexpr (D == 2 && B == 17) {  // 17^2 blocks: 289 points per warp
    if (warp_form) {
      // one instantiation per stage: stage 0 reads the committed state, the
      // others the previous stage value
      auto go_nt = [&](auto stc, auto ntc) {
        constexpr int S = decltype(stc)::value, NT = decltype(ntc)::value;
        using TSRC = std::conditional_t<S == 0, TS, TY>;
        using SW = StageW<B, RHS, TS, TY, TSRC, NT>;
        const TSRC* src = S == 0 ? (const TSRC*)f.y : (const TSRC*)(S == 2 ? f.Yb : f.Ya);
        auto k = k_stage_adv_w<B, RHS, TS, TY, TSRC, NT, S>;
        prep_smem(k, SW::SMEM);
        const int grid = persistent_grid(k, NT, SW::SMEM, lc, lc.grid_mult);
        launch_k(lc.pdl, k, grid, NT, SW::SMEM, st, pv, src, (TS*)f.y, (TS*)f.acc, ynext, lc.staging, sa);
      };
      // blocks (warps) per CTA: tuned for the FP32 forms, 4 otherwise
      auto go = [&](auto stc) {
        if constexpr (sizeof(TS) == 4) {
          if (lc.warp_blocks == 2) return go_nt(stc, std::integral_constant<int, 64>{});
          if (lc.warp_blocks == 8) return go_nt(stc, std::integral_constant<int, 256>{});
        }
        go_nt(stc, std::integral_constant<int, threads>{});
      };
      switch (stage) {
        case 0: go(std::integral_constant<int, 0>{}); break;
        case 1: go(std::integral_constant<int, 1>{}); break;
        case 2: go(std::integral_constant<int, 2>{}); break;
        default: go(std::integral_constant<int, 3>{}); break;
      }
      count_launch();
      return;
    }
  }
  auto go = [&](auto stc) {
    constexpr int S = decltype(stc)::value;
    using TSRC = std::conditional_t<S == 0, TS, TY>;
    const TSRC* src = S == 0 ? (const TSRC*)f.y : (const TSRC*)(S == 2 ? f.Yb : f.Ya);
    auto k = k_stage_adv<D, B, RHS, TS, TY, TSRC, threads, S>;
    prep_smem(k, smem);
    const int grid = persistent_grid(k, threads, smem, lc, lc.grid_mult);
    launch_k(lc.pdl, k, grid, threads, smem, st, pv, src, (TS*)f.y, (TS*)f.acc, ynext, stage, sa);
  };
  switch (stage) {
    case 0: go(std::integral_constant<int, 0>{}); break;
    case 1: go(std::integral_constant<int, 1>{}); break;
    case 2: go(std::integral_constant<int, 2>{}); break;
    default: go(std::integral_constant<int, 3>{}); break;
  }
  count_launch();
}

template <int D, int B, int RHS>
static void stage_prec(const PoolView& pv, const Fields& f, int stage, const StageArgs& sa,
                       const LaunchCfg& lc, cudaStream_t st) {
  switch (pv.prec) {
    case MR_PREC_FP64: stage_impl<D, B, RHS, double, double>(pv, f, stage, sa, lc, st); break;
    case MR_PREC_FP32: stage_impl<D, B, RHS, float, float>(pv, f, stage, sa, lc, st); break;
    default: stage_impl<D, B, RHS, double, float>(pv, f, stage, sa, lc, st); break;
  }
}

template <int B, typename TS, typename TY>
static void stage_ns_impl(const PoolView& pv, const Fields& f, int stage, const StageArgs& sa,
                          const LaunchCfg& lc, cudaStream_t st) {
  using Gm = Geo<2, B>;
  constexpr int threads = 256;
  const size_t smem = kRingBytesD<2> + sizeof(TY) * (4 * Gm::TILE + 4 * Gm::CBOX + 4 * Gm::TILE +
                                                 4 * NsGeo<B>::NF + 4 * NsGeo<B>::NG);
  // stage s reads y, Ya, Yb, Ya and writes Ya, Yb, Ya, (Yb: the new state's copy for the filter)
  TY* ynext = (TY*)(stage == 1 || stage == 3 ? f.Yb : f.Ya);
  if (stage == 0) {
    auto k = k_stage_ns<B, TS, TY, TS>;
    prep_smem(k, smem);
    launch_k(lc.pdl, k, persistent_grid(k, threads, smem, lc, lc.grid_mult), threads, smem, st, pv, (const TS*)f.y, (TS*)f.y, (TS*)f.acc, ynext, (TY*)f.Yn, stage, sa);
  } else {
    const TY* src = (const TY*)(stage == 2 ? f.Yb : f.Ya);
    auto k = k_stage_ns<B, TS, TY, TY>;
    prep_smem(k, smem);
    launch_k(lc.pdl, k, persistent_grid(k, threads, smem, lc, lc.grid_mult), threads, smem, st, pv, src, (TS*)f.y, (TS*)f.acc, ynext, (TY*)f.Yn, stage, sa);
  }
  count_launch();
}

template <int B>
static void stage_ns(const PoolView& pv, const Fields& f, int stage, const StageArgs& sa,
                     const LaunchCfg& lc, cudaStream_t st) {
  switch (pv.prec) {
    case MR_PREC_FP64: stage_ns_impl<B, double, double>(pv, f, stage, sa, lc, st); break;
    case MR_PREC_FP32: stage_ns_impl<B, float, float>(pv, f, stage, sa, lc, st); break;
    default: stage_ns_impl<B, double, float>(pv, f, stage, sa, lc, st); break;
  }
}

template <int D>
void launch_plan(const PoolView& pv, const LaunchCfg& lc, cudaStream_t st) {
  const size_t smem = 4 * kRingBytesD<D>;  // one ring per warp
  if constexpr (D == 3) launch_k(lc.pdl, k_plan<3, 17>, lc.num_sms * 8, 128, smem, st, pv);
  else if (pv.Bs == 17) launch_k(lc.pdl, k_plan<2, 17>, lc.num_sms * 8, 128, smem, st, pv);
  else launch_k(lc.pdl, k_plan<2, 33>, lc.num_sms * 8, 128, smem, st, pv);
  count_launch();
}

// RK stage of every block for one block size (instantiated per block size in
// translation units of their own).
template <int D, int B>
void launch_stage_bs(const PoolView& pv, const Fields& f, int stage, const StageArgs& sa,
                     const LaunchCfg& lc, cudaStream_t st) {
  if constexpr (D == 2) {
    if (pv.rhs_kind == MR_RHS_NS) stage_ns<B>(pv, f, stage, sa, lc, st);
    else if (pv.rhs_kind == MR_RHS_NS_SKEW) launch_stage_nss<B>(pv, f, stage, sa, lc, st);
    else if (pv.rhs_kind == MR_RHS_SWIRL) stage_prec<D, B, MR_RHS_SWIRL>(pv, f, stage, sa, lc, st);
    else stage_prec<D, B, MR_RHS_ADV>(pv, f, stage, sa, lc, st);
  } else {
    stage_prec<D, B, MR_RHS_ADV>(pv, f, stage, sa, lc, st);
  }
}

template <int D>
void launch_stage(const PoolView& pv, const Fields& f, int stage, const StageArgs& sa,
                  const LaunchCfg& lc, cudaStream_t st) {
  if (D == 3 || pv.Bs == 17) launch_stage_bs<D, 17>(pv, f, stage, sa, lc, st);
  else launch_stage_bs<D, (D == 2 ? 33 : 17)>(pv, f, stage, sa, lc, st);
}

// Dispatch helper over (Bs, state type): calls F<D, B, TS>::run(args...).
template <int D, template <int, int, typename> class F, typename... A>
static void dispatch_bs(const PoolView& pv, A&&... args) {
  const bool st64 = pv.prec != MR_PREC_FP32;
  if constexpr (D == 3) {
    if (st64) F<D, 17, double>::run(pv, args...);
    else F<D, 17, float>::run(pv, args...);
  } else {
    if (pv.Bs == 17) {
      if (st64) F<D, 17, double>::run(pv, args...);
      else F<D, 17, float>::run(pv, args...);
    } else {
      if (st64) F<D, 33, double>::run(pv, args...);
      else F<D, 33, float>::run(pv, args...);
    }
  }
}

// --------------------------------------------------------------- refine ------
template <int D, int B, typename TS>
struct RefineRun {
  static void run(const PoolView& pv, const Fields& f, const LaunchCfg& lc, cudaStream_t st) {
    constexpr int threads = Threads<D, B>::value;
    using Bx = Box<D, B, 1>;
    const size_t scr = (size_t)std::max<int64_t>((int64_t)pv.nvar * Bx::SCR, RefGeo<D, B>::NX);
    const size_t smem = kRingBytesD<D> + sizeof(TS) * (pv.nvar * (Bx::TILE + Bx::CBOX) + scr);
    auto k = k_refine<D, B, TS, threads>;
    prep_smem(k, smem);
    const int grid = persistent_grid(k, threads, smem, lc, lc.grid_mult);
    launch_k(lc.pdl, k, grid, threads, smem, st, pv, (TS*)f.y);
    count_launch();
  }
};


template <int D>
void launch_refine(const PoolView& pv, const Fields& f, int mode, const int8_t* mask,
                   const LaunchCfg& lc, cudaStream_t st) {
  const int nch = 1 << D;
  // short lists: the counting kernel's last CTA scans them (no scan launch)
  if (2 * (int64_t)lc.n_hint <= kFusedScanMax) {
    const int grid = std::min(flat_grid(pv, 256), std::max(lc.num_sms, (2 * lc.n_hint + 255) / 256));
    launch_k(lc.pdl, k_refine_count<D, true>, grid, 256, 0, st, pv, mode, mask);
    count_launch();
  } else {
    launch_k(lc.pdl, k_refine_count<D, false>, flat_grid(pv, 256), 256, 0, st, pv, mode, mask);
    count_launch();
    launch_scan2(pv.emit, pv.eoff, pv.partial, &pv.cnt->n_act, pv.cap, &pv.cnt->n_new, st, 2 * (int64_t)lc.n_hint,
                 lc.pdl != 0);
  }
  dispatch_bs<D, RefineRun>(pv, f, lc, st);
  launch_k(lc.pdl, k_refine_commit<D>, flat_grid(pv, 256), 256, 0, st, pv);
  count_launch(1);
  (void)nch;
}

// ------------------------------------------------------------------- IC ------
template <int D, int B, typename TS>
struct IcRun {
  static void run(const PoolView& pv, const Fields& f, const LaunchCfg& lc, cudaStream_t st) {
    launch_k(lc.pdl, k_ic<D, B, TS>, lc.num_sms * 8, 256, 0, st, pv, (TS*)f.y);
    count_launch();
  }
};
template <int D>
void launch_ic(const PoolView& pv, const Fields& f, const LaunchCfg& lc, cudaStream_t st) {
  dispatch_bs<D, IcRun>(pv, f, lc, st);
}

// --------------------------------------------------------------- coarsen -----
template <int D, int B, typename TS>
struct DetailsRun {
  static void run(const PoolView& pv, const Fields& f, bool fp64, const LaunchCfg& lc,
                  cudaStream_t st) {
    constexpr int threads = Threads<D, B>::value;
    // FP64 details for the plain FP64 form or when asked for (thresholds below
    // FP32 resolution); otherwise FP32, also for FP64 state
    const bool d64 = fp64 || pv.prec == MR_PREC_FP64;
    const bool warp_form = pv.nvar == 1 && pv.norm_kind == 0 && sizeof(TS) == 4 &&
                           (lc.stage_form == 1 || (lc.stage_form < 0 && lc.n_hint >= 8 * lc.num_sms));
    if (D == 2 && warp_form) {  // one warp per block
      if (d64) {
        auto k = k_details_w<B, TS, double, threads>;
        using DW = DetW<B, TS, double, threads>;
        prep_smem(k, DW::SMEM);
        launch_k(lc.pdl, k, persistent_grid(k, threads, DW::SMEM, lc, lc.grid_mult), threads, DW::SMEM, st, pv, (TS*)f.y);
      } else {
        auto k = k_details_w<B, TS, TS, threads>;
        using DW = DetW<B, TS, TS, threads>;
        prep_smem(k, DW::SMEM);
        launch_k(lc.pdl, k, persistent_grid(k, threads, DW::SMEM, lc, lc.grid_mult), threads, DW::SMEM, st, pv, (TS*)f.y);
      }
      count_launch();
      return;
    }
    using Bx = Box<D, B, 2>;
    const size_t tt = d64 ? sizeof(TS) : 4;  // tile type: the state type, FP32 for FP32 details
    const size_t region = d64 ? DetSmem<D, B, TS, double>::region(pv.nvar) : DetSmem<D, B, float, float>::region(pv.nvar);
    const size_t smem = kRingBytesD<D> + tt * pv.nvar * Bx::TILE + 16 + region + 16 +
                        (D == 2 ? 4 * (Bx::NPTS + DetTab<B>::INTS) : 0);
    if (d64) {
      auto k = k_details<D, B, TS, double, threads>;
      prep_smem(k, smem);
      launch_k(lc.pdl, k, persistent_grid(k, threads, smem, lc, lc.grid_mult), threads, smem, st, pv, (TS*)f.y);
    } else {
      auto k = k_details<D, B, TS, float, threads, float>;
      prep_smem(k, smem);
      launch_k(lc.pdl, k, persistent_grid(k, threads, smem, lc, lc.grid_mult), threads, smem, st, pv, (TS*)f.y);
    }
    count_launch();
  }
};
template <int D, int B, typename TS>
struct CoarsenRun {
  static void run(const PoolView& pv, const Fields& f, const RoundCtl& rc, const LaunchCfg& lc, cudaStream_t st) {
    constexpr int threads = 256;
    const size_t smem = sizeof(TS) * pv.nvar * Geo<D, B>::NI;
    auto k = k_coarsen<D, B, TS>;
    prep_smem(k, smem);
    launch_k(lc.pdl, k, persistent_grid(k, threads, smem, lc, 0), threads, smem, st, pv, (TS*)f.y, rc);
    count_launch();
  }
};

template <int D>
void launch_rounds_begin(const PoolView& pv, const LaunchCfg& lc, cudaStream_t st) {
  launch_k(lc.pdl, k_round_begin<D>, 1, 256, 0, st, pv, pv.norm_kind == 1 ? 0.0 : 1.0);
  count_launch();
}

template <int D>
void launch_round_details(const PoolView& pv, const Fields& f, bool fp64, const LaunchCfg& lc,
                          cudaStream_t st) {
  dispatch_bs<D, DetailsRun>(pv, f, fp64, lc, st);
}

template <int D>
void launch_round_merge(const PoolView& pv, const Fields& f, bool merge, const RoundCtl& rc, const LaunchCfg& lc,
                        cudaStream_t st) {
  const int nch = 1 << D;
  // one warp per block: a grid for the expected list (after a refinement,
  // 2^d times the blocks last seen by the host); the loop strides over more
  const int64_t n_expect = (int64_t)nch * std::max(lc.n_hint, 1);
  const int grid = (int)std::min<int64_t>(std::min<int64_t>(4096, (pv.cap + 7) / 8),
                                          std::max<int64_t>(lc.num_sms, (n_expect + 7) / 8));
  if (merge && n_expect <= kFusedScanMax) {
    launch_k(lc.pdl, k_flags<D, true>, grid, 256, 0, st, pv);  // the last CTA scans the counts
    count_launch();
  } else {
    launch_k(lc.pdl, k_flags<D, false>, grid, 256, 0, st, pv);
    count_launch();
    if (!merge) return;
    launch_scan2(pv.emit, pv.eoff, pv.partial, &pv.cnt->n_round, pv.cap, &pv.cnt->n_new, st, 4 * (int64_t)lc.n_hint,
                 lc.pdl != 0);
  }
  dispatch_bs<D, CoarsenRun>(pv, f, rc, lc, st);
  (void)nch;
}

template <int D>
void launch_coarsen_round(const PoolView& pv, const Fields& f, bool fp64, bool merge, const RoundCtl& rc,
                          const LaunchCfg& lc, cudaStream_t st) {
  launch_round_details<D>(pv, f, fp64, lc, st);
  launch_round_merge<D>(pv, f, merge, rc, lc, st);
}

// ------------------------------------------------------------------ sync -----
template <int D, int B, typename TS>
struct SyncRun {
  static void run(const PoolView& pv, const Fields& f, double* tiles, const LaunchCfg& lc,
                  cudaStream_t st) {
    constexpr int threads = 256;
    const size_t smem = kRingBytesD<D> + sizeof(double) * pv.nvar * (Geo<D, B>::TILE + Geo<D, B>::CBOX);
    auto k = k_sync<D, B, TS>;
    prep_smem(k, smem);
    launch_k(lc.pdl, k, persistent_grid(k, threads, smem, lc, 0), threads, smem, st, pv, (TS*)f.y, tiles);
    count_launch();
  }
};
template <int D>
void launch_sync(const PoolView& pv, const Fields& f, double* tiles, const LaunchCfg& lc,
                 cudaStream_t st) {
  dispatch_bs<D, SyncRun>(pv, f, tiles, lc, st);
}

template <int D>
void launch_neighbors(const PoolView& pv, const int4* rel, int R, int32_t* nbr, int8_t* dl,
                      const LaunchCfg& lc, cudaStream_t st) {
  launch_k(lc.pdl, k_neighbors<D>, lc.num_sms * 8, 256, 0, st, pv, rel, R, nbr, dl);
  count_launch();
}

// ---------------------------------------------------------------- export -----
template <int D, int B, typename TS>
struct ExportRun {
  static void run(const PoolView& pv, const Fields& f, double* fields, const LaunchCfg& lc,
                  cudaStream_t st) {
    launch_k(lc.pdl, k_export_fields<D, B, TS>, lc.num_sms * 8, 256, 0, st, pv, (const TS*)f.y, fields);
    count_launch();
  }
};
template <int D>
void launch_export(const PoolView& pv, const Fields& f, mr_block_info* info, double* fields,
                   int8_t* flags, double* mdet, const LaunchCfg& lc, cudaStream_t st) {
  launch_k(lc.pdl, k_export_info<D>, flat_grid(pv, 256), 256, 0, st, pv, info, flags, mdet);
  count_launch();
  if (fields) dispatch_bs<D, ExportRun>(pv, f, fields, lc, st);
}

// ------------------------------------------------------------ set_blocks -----
template <int D, int B, typename TS>
struct ImportRun {
  static void run(const PoolView& pv, const Fields& f, const double* fields, int64_t n,
                  const LaunchCfg& lc, cudaStream_t st) {
    launch_k(lc.pdl, k_import_fields<D, B, TS>, lc.num_sms * 8, 256, 0, st, pv, (TS*)f.y, fields, n);
    count_launch();
  }
};

__global__ void k_fill_i32(int32_t* a, int64_t n, int32_t v);
__global__ void k_fill_i8(int8_t* a, int64_t n, int8_t v);
__global__ void k_sb_check(const int32_t* cells, int64_t ncells, Counters* c);
__global__ void k_sb_counters(Counters* c, int32_t* freelist, int64_t n, int64_t cap);

// Phase 1 (validate): place, detect duplicates, check the cells are covered once.
// Phase 2 (after the host saw no error): canonical order, fields, gradedness.
template <int D>
void launch_set_blocks(const PoolView& pv, const Fields& f, int phase, int64_t n,
                       const int32_t* lvl, const int32_t* tree, const int32_t* crd,
                       const double* fields, int64_t ncells, int ntrees, int64_t ntab,
                       const LaunchCfg& lc, cudaStream_t st) {
  const int g = 1024;
  if (phase == 0) {  // empty pool: no active block, every slot free
    launch_k(lc.pdl, k_fill_i32, g, 256, 0, st, pv.tab, ntab, -1);
    launch_k(lc.pdl, k_fill_i8, g, 256, 0, st, pv.lvl, pv.cap, (int8_t)-1);
    launch_k(lc.pdl, k_sb_counters, g, 256, 0, st, pv.cnt, pv.freelist, 0, pv.cap);
    count_launch(3);
    return;
  }
  if (phase == 1) {
    launch_k(lc.pdl, k_fill_i32, g, 256, 0, st, pv.tab, ntab, -1);
    launch_k(lc.pdl, k_fill_i32, g, 256, 0, st, pv.cells, 2 * ncells, 0);
    launch_k(lc.pdl, k_fill_i8, g, 256, 0, st, pv.lvl, pv.cap, (int8_t)-1);
    launch_k(lc.pdl, k_sb_place<D>, g, 256, 0, st, pv, n, lvl, tree, crd, ntrees);
    launch_k(lc.pdl, k_sb_cover<D>, lc.num_sms * 4, 256, 0, st, pv, n);
    launch_k(lc.pdl, k_sb_check, g, 256, 0, st, pv.cells, ncells, pv.cnt);
    count_launch(6);
    return;
  }
  launch_k(lc.pdl, k_fill_i32, g, 256, 0, st, pv.cells, 2 * ncells, 0);
  launch_k(lc.pdl, k_sb_mark<D>, g, 256, 0, st, pv, n);
  count_launch(2);
  launch_scan2(pv.cells, pv.eoff, pv.partial, nullptr, ncells, &pv.cnt->n_new, st, -1, lc.pdl != 0);
  launch_k(lc.pdl, k_sb_order<D>, g, 256, 0, st, pv, n);
  launch_k(lc.pdl, k_sb_counters, g, 256, 0, st, pv.cnt, pv.freelist, n, pv.cap);
  count_launch(2);
  if (fields) dispatch_bs<D, ImportRun>(pv, f, fields, n, lc, st);
  launch_k(lc.pdl, k_check_graded<D>, g, 256, 0, st, pv);
  count_launch();
}

// ----------------------------------------------------------------- error -----
template <int D, int B, typename TS>
struct ErrorRun {
  static void run(const PoolView& pv, const Fields& f, int tree, const double* ex, double* out,
                  const LaunchCfg& lc, cudaStream_t st) {
    launch_k(lc.pdl, k_error<D, B, TS>, lc.num_sms * 4, 256, 0, st, pv, (const TS*)f.y, tree, ex, out);
    count_launch();
  }
};
template <int D>
void launch_error(const PoolView& pv, const Fields& f, int tree, const double* ex, double* out4,
                  const LaunchCfg& lc, cudaStream_t st) {
  dispatch_bs<D, ErrorRun>(pv, f, tree, ex, out4, lc, st);
}

// The RK stage launchers of each block size are instantiated in translation
// units of their own (mr_k2s.cu, mr_k2t.cu, mr_k3s.cu), compiled in parallel
// with the rest; the others see them as external (MR_EXTERN_STAGE).
#define MR_INSTANTIATE_STAGE(D, B)                                                              \
  template void launch_stage_bs<D, B>(const PoolView&, const Fields&, int, const StageArgs&,   \
                                      const LaunchCfg&, cudaStream_t);
#define MR_EXTERN_STAGE(D, B)                                                                   \
  extern template void launch_stage_bs<D, B>(const PoolView&, const Fields&, int,              \
                                             const StageArgs&, const LaunchCfg&, cudaStream_t);

#define MR_INSTANTIATE(D)                                                                       \
  template void launch_plan<D>(const PoolView&, const LaunchCfg&, cudaStream_t);                \
  template void launch_stage<D>(const PoolView&, const Fields&, int, const StageArgs&,         \
                                const LaunchCfg&, cudaStream_t);                                \
  template void launch_refine<D>(const PoolView&, const Fields&, int, const int8_t*,            \
                                 const LaunchCfg&, cudaStream_t);                               \
  template void launch_ic<D>(const PoolView&, const Fields&, const LaunchCfg&, cudaStream_t);   \
  template void launch_rounds_begin<D>(const PoolView&, const LaunchCfg&, cudaStream_t);        \
  template void launch_coarsen_round<D>(const PoolView&, const Fields&, bool, bool,             \
                                        const RoundCtl&, const LaunchCfg&, cudaStream_t);       \
  template void launch_round_details<D>(const PoolView&, const Fields&, bool, const LaunchCfg&, \
                                        cudaStream_t);                                          \
  template void launch_round_merge<D>(const PoolView&, const Fields&, bool, const RoundCtl&,    \
                                      const LaunchCfg&,                                         \
                                      cudaStream_t);                                            \
  template void launch_sync<D>(const PoolView&, const Fields&, double*, const LaunchCfg&,       \
                               cudaStream_t);                                                   \
  template void launch_neighbors<D>(const PoolView&, const int4*, int, int32_t*, int8_t*,       \
                                    const LaunchCfg&, cudaStream_t);                            \
  template void launch_export<D>(const PoolView&, const Fields&, mr_block_info*, double*,       \
                                 int8_t*, double*, const LaunchCfg&, cudaStream_t);             \
  template void launch_set_blocks<D>(const PoolView&, const Fields&, int, int64_t,              \
                                     const int32_t*, const int32_t*, const int32_t*,            \
                                     const double*, int64_t, int, int64_t, const LaunchCfg&,    \
                                     cudaStream_t);                                             \
  template void launch_error<D>(const PoolView&, const Fields&, int, const double*, double*,    \
                                const LaunchCfg&, cudaStream_t);

}  // namespace mr

// Launchers of the Navier-Stokes kernels of Sec. 4 (skew-symmetric stage and
// shock-capturing filter), 2D, Bs 17 and 33.
#include "mr_launch.cuh"
#include "mr_ns.cuh"

namespace mr {

template <int B, typename TS, typename TY>
static void stage_nss_impl(const PoolView& pv, const Fields& f, int stage, const StageArgs& sa,
                           const LaunchCfg& lc, cudaStream_t st) {
  constexpr int threads = NssCfg<B>::NT;
  constexpr size_t smem = nss_smem<B, TY>();
  // stage s reads y, Ya, Yb, Ya and writes Ya, Yb, Ya, (Yb: the new state's copy for the filter)
  TY* ynext = (TY*)(stage == 1 || stage == 3 ? f.Yb : f.Ya);
  if (stage == 0) {
    auto k = k_stage_nss<B, TS, TY, TS>;
    prep_smem(k, smem);
    launch_k(lc.pdl, k, persistent_grid(k, threads, smem, lc, lc.grid_mult), threads, smem, st, pv,
             (const TS*)f.y, (TS*)f.y, (TS*)f.acc, ynext, (TY*)f.Yn, stage, sa);
  } else {
    const TY* src = (const TY*)(stage == 2 ? f.Yb : f.Ya);
    auto k = k_stage_nss<B, TS, TY, TY>;
    prep_smem(k, smem);
    launch_k(lc.pdl, k, persistent_grid(k, threads, smem, lc, lc.grid_mult), threads, smem, st, pv, src,
             (TS*)f.y, (TS*)f.acc, ynext, (TY*)f.Yn, stage, sa);
  }
  count_launch();
}

template <int B>
void launch_stage_nss(const PoolView& pv, const Fields& f, int stage, const StageArgs& sa,
                      const LaunchCfg& lc, cudaStream_t st) {
  switch (pv.prec) {
    case MR_PREC_FP64: stage_nss_impl<B, double, double>(pv, f, stage, sa, lc, st); break;
    case MR_PREC_FP32: stage_nss_impl<B, float, float>(pv, f, stage, sa, lc, st); break;
    default: stage_nss_impl<B, double, float>(pv, f, stage, sa, lc, st); break;
  }
}
template void launch_stage_nss<17>(const PoolView&, const Fields&, int, const StageArgs&, const LaunchCfg&,
                                   cudaStream_t);
template void launch_stage_nss<33>(const PoolView&, const Fields&, int, const StageArgs&, const LaunchCfg&,
                                   cudaStream_t);

template <int B, typename TS, typename TC, int KIND>
static void filter_impl(const PoolView& pv, const Fields& f, bool copy, const LaunchCfg& lc, cudaStream_t st) {
  constexpr int threads = kFilterThreads;
  constexpr size_t smem = filter_smem<B, TC>();
  if (copy) {
    launch_k(lc.pdl, k_state_copy<TS, TC>, lc.num_sms * 8, 256, 0, st, pv, (const TS*)f.y, (TC*)f.Yb);
    count_launch();
  }
  auto k = k_filter<B, TS, TC, KIND>;
  prep_smem(k, smem);
  launch_k(lc.pdl, k, persistent_grid(k, threads, smem, lc, lc.grid_mult), threads, smem, st, pv,
           (const TC*)f.Yb, (TS*)f.y);
  count_launch();
}

template <int B, int KIND>
static void filter_prec(const PoolView& pv, const Fields& f, bool copy, const LaunchCfg& lc, cudaStream_t st) {
  switch (pv.prec) {
    case MR_PREC_FP64: filter_impl<B, double, double, KIND>(pv, f, copy, lc, st); break;
    case MR_PREC_FP32: filter_impl<B, float, float, KIND>(pv, f, copy, lc, st); break;
    default: filter_impl<B, double, float, KIND>(pv, f, copy, lc, st); break;
  }
}

void launch_filter(const PoolView& pv, const Fields& f, bool copy, const LaunchCfg& lc, cudaStream_t st) {
  const bool skew = pv.rhs_kind == MR_RHS_NS_SKEW;
  if (pv.Bs == 17) {
    if (skew) filter_prec<17, MR_RHS_NS_SKEW>(pv, f, copy, lc, st);
    else filter_prec<17, MR_RHS_NS>(pv, f, copy, lc, st);
  } else {
    if (skew) filter_prec<33, MR_RHS_NS_SKEW>(pv, f, copy, lc, st);
    else filter_prec<33, MR_RHS_NS>(pv, f, copy, lc, st);
  }
}

}  // namespace mr

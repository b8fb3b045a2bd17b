// Kernel templates of the multiresolution step.  Instantiated per dimension in
// mr_k2*.cu / mr_k3*.cu.  Every persistent kernel loops over the active list with
// a grid-stride loop bounded by the device-side block count, so no launch
// needs a host round trip.
#pragma once
#include "mr_device.cuh"

namespace mr {

// Per-tree stage constants in the arithmetic type T.  The FP32 copies hold the
// FP64 values rounded once (on creation, or when the step's time is set), so
// an FP32 kernel reads them without an FP64 conversion per block.
template <typename T> struct StageCoef {
  T ca, cy, ct;
  __device__ __forceinline__ StageCoef(const PoolView& pv, const StageArgs& sa, int t, int s) {
    if constexpr (sizeof(T) == 4) {
      if (pv.tt) { ca = pv.tt[t].caf[s]; cy = pv.tt[t].cyf[s]; ct = pv.tt[t].ctf[s]; }
      else { ca = sa.caf[t]; cy = sa.cyf[t]; ct = sa.ctf[t]; }
    } else {
      if (pv.tt) { ca = pv.tt[t].ca[s]; cy = pv.tt[t].cy[s]; ct = pv.tt[t].ct[s]; }
      else { ca = sa.ca[t]; cy = sa.cy[t]; ct = sa.ct[t]; }
    }
  }
};
template <typename T> __device__ __forceinline__ T tree_cD(const TreeDev& td, int l) {
  if constexpr (sizeof(T) == 4) return td.cDf[l]; else return td.cD[l];
}
template <typename T> __device__ __forceinline__ T tree_rhs(const TreeDev& td, int a) {
  if constexpr (sizeof(T) == 4) return td.rhsf[a]; else return td.rhs[a];
}
template <typename T> __device__ __forceinline__ const T* lattice(const PoolView& pv) {
  if constexpr (sizeof(T) == 4) return pv.latf; else return pv.lat;
}


// ------------------------------------------------------------------ stage ----
// One RK4 stage on every block (Sec. 3: 4th-order central FD + classic RK4):
//   k = N(Y_s) on the synchronised tile, then the 3-register update
//   s0: acc = y + dt/6 k, Y1 = y + dt/2 k      s1: acc += dt/3 k, Y2 = y + dt/2 k
//   s2: acc += dt/3 k,    Y3 = y + dt k        s3: y = acc + dt/6 k
// Advection RHS: -(u Dx phi + v Dy phi [+ w Dz phi]),
//   D1 f = ((f[-2] - f[2]) + 8 (f[1] - f[-1])) / (12 dx).
//
// The block's plan (k_plan) is read from shared memory, the next block's plan
// is fetched while this one is processed; blocks with a uniform neighbourhood
// take the direct gather, the others the general one through their ring.
template <int D, int B, int RHS, typename TS, typename TY, typename TSRC, int NT, int ST>
__global__ void __launch_bounds__(NT, NT <= 128 ? 8 : (D == 3 ? 3 : 4)) k_stage_adv(PoolView pv, const TSRC* __restrict__ src, TS* __restrict__ y,
                            TS* __restrict__ acc, TY* __restrict__ ynext, int stage_arg, StageArgs sa) {
  pdl_enter();
  constexpr int stage = ST;  // the RK stage, fixed at compile time
  static_assert(ST >= 0 && ST <= 3, "RK4 stage");
  using Gm = Geo<D, B>;
  using Bx = Box<D, B, 2>;  // the stencils reach two nodes
  using PL = Plan<D>;
  using TC = TY;  // stencil arithmetic type
  static_assert(NT >= PL::INTS, "one thread per plan entry");
  RingD<D>& R = *smem_as<RingD<D>>(0);
  TC* tile = smem_as<TC>(kRingBytesD<D>);  // nvar == 1
  TC* cbox = tile + Bx::TILE;
  TC* scr = cbox + Bx::CBOX;
  int32_t* gtab = reinterpret_cast<int32_t*>(scr + Bx::SCR);  // 2D: gather table
  __shared__ int32_t splan[2][PL::INTS];
  __shared__ int64_t snb[2][PL::NB];  // pool offsets of the plan's neighbours
  const int nact = pv.cnt->n_act;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&pv.cnt->stage_blocks, (unsigned long long)nact);
  if (D == 2) build_gtab<D, B, 2>(gtab);
  if (blockIdx.x < nact && threadIdx.x < PL::INTS) {
    const int32_t v = pv.plan[(int64_t)blockIdx.x * PL::INTS + threadIdx.x];
    splan[0][threadIdx.x] = v;
    if (threadIdx.x >= PL::NBO && threadIdx.x < PL::NBO + PL::NB) snb[0][threadIdx.x - PL::NBO] = (int64_t)v * pv.vs;
  }
  __syncthreads();
  int buf = 0;
  for (int p = blockIdx.x; p < nact; p += gridDim.x, buf ^= 1) {
    const int pn = p + gridDim.x;
    int32_t pre = 0;
    if (pn < nact && threadIdx.x < PL::INTS) pre = pv.plan[(int64_t)pn * PL::INTS + threadIdx.x];
    const int32_t* pl = splan[buf];
    const BlockInfo b = plan_block<D>(pl);
    const TreeDev& td = pv.trees[b.tree];
    if ((pl[1] >> 30) & 1) {
      if constexpr (D == 2)
        gather_table<D, B, 2, 1, TSRC, TC>(pv, (int64_t)b.slot * pv.vs, snb[buf], gtab, src, (TSRC*)src, tile,
                                           stage == 0);
      else
        fill_cols<B, TSRC, TC, 2>(pv, b, snb[buf], src, (TSRC*)src, tile, stage == 0, R, cbox, scr);
    } else {
      load_regions<D, CtaGroup>(pv, p, R);
      __syncthreads();
      if constexpr (D == 2)
        fill_tile<D, B, TSRC, TC, 2>(pv, b, src, (TSRC*)src, tile, stage == 0, R, cbox, scr, true);
      else
        fill_cols<B, TSRC, TC, 2>(pv, b, nullptr, src, (TSRC*)src, tile, stage == 0, R, cbox, scr, true);
    }
    __syncthreads();
    const TC c = tree_cD<TC>(td, b.lvl);
    const StageCoef<TS> cs(pv, sa, b.tree, stage);  // RK weights in the state type
    const TC ct = StageCoef<TC>(pv, sa, b.tree, stage).ct;
    const int64_t base = (int64_t)b.slot * pv.vs;  // nvar == 1
    const int sh = td.Jmax - b.lvl;
    const TS cas = cs.ca, cys = cs.cy;
    if constexpr (D == 2) {
      // thread = (column i, rows j0, j0 + G, ...): the column's velocity
      // factors are loaded once; the rows' loads are issued together
      constexpr int G = NT / B, RU = (B + G - 1) / G;
      const int t = threadIdx.x;
      if (t < G * B) {
        const int i = t % B, j0 = t / B;
        TC ax = 0, bx = 0;  // swirl factors in the stencil type
        const TC* A = lattice<TC>(pv) + td.lat_off + (int64_t)kLatSwA * td.N;
        const TC* Bt = lattice<TC>(pv) + td.lat_off + (int64_t)kLatSwB * td.N;
        if (RHS == MR_RHS_SWIRL) {
          const int64_t Ux = pmod64((b.c[0] * (B - 1) + i) << sh, td.N);
          ax = A[Ux];
          bx = Bt[Ux];
        }
        TS yv[RU], av[RU];
        TC u0[RU], u1[RU];  // velocity in the stencil type (constant: once per block)
        const TC uc0 = tree_rhs<TC>(td, 0), uc1 = tree_rhs<TC>(td, 1);
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          const int j = j0 + r * G;
          yv[r] = av[r] = TS(0);
          u0[r] = uc0;
          u1[r] = uc1;
          if (j >= B) continue;
          const int q = j * B + i;
          if (stage <= 2) yv[r] = y[base + q];  // stage 0: committed (synchronised) y_n
          if (stage >= 1) av[r] = acc[base + q];
          if (RHS == MR_RHS_SWIRL) {
            const int64_t Uy = pmod64((b.c[1] * (B - 1) + j) << sh, td.N);
            u0[r] = ct * (ax * Bt[Uy]);
            u1[r] = -(ct * (A[Uy] * bx));
          }
        }
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          const int j = j0 + r * G;
          if (j >= B) continue;
          const TC* t0 = tile + Bx::tix(i, j, 0);
          const TC dxv = ((t0[-2] - t0[2]) + TC(8) * (t0[1] - t0[-1])) * c;
          const TC dyv = ((t0[-2 * Bx::S] - t0[2 * Bx::S]) + TC(8) * (t0[Bx::S] - t0[-Bx::S])) * c;
          const TC s = u0[r] * dxv + u1[r] * dyv;
          const TS kk = (TS)(-s);
          const int64_t at = base + j * B + i;
          if (stage == 0) {
            acc[at] = yv[r] + cas * kk;
            ynext[at] = (TY)(yv[r] + cys * kk);
          } else if (stage == 1 || stage == 2) {
            acc[at] = av[r] + cas * kk;
            ynext[at] = (TY)(yv[r] + cys * kk);
          } else {
            y[at] = av[r] + cas * kk;
          }
        }
      }
    }
    // 3D: UC points per thread at a time: their state, accumulator and
    // velocity loads are issued together, then the stencils and the updates
    constexpr int UC = D == 3 ? 4 : 1;
    const TC uc2 = tree_rhs<TC>(td, 2);
    for (int q0 = threadIdx.x; D == 3 && q0 < Gm::NI; q0 += UC * NT) {
      TS yv[UC], av[UC];
      TC u0[UC], u1[UC];
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        const int q = q0 + u * NT;
        yv[u] = av[u] = TS(0);
        u0[u] = tree_rhs<TC>(td, 0);
        u1[u] = tree_rhs<TC>(td, 1);
        if (q >= Gm::NI) continue;
        if (stage <= 2) yv[u] = y[base + q];  // stage 0: committed (synchronised) y_n
        if (stage >= 1) av[u] = acc[base + q];
        if (RHS == MR_RHS_SWIRL) {
          const int i = q % B, j = (q / B) % B;
          const int64_t Ux = pmod64((b.c[0] * (B - 1) + i) << sh, td.N);
          const int64_t Uy = pmod64((b.c[1] * (B - 1) + j) << sh, td.N);
          const TC* A = lattice<TC>(pv) + td.lat_off + (int64_t)kLatSwA * td.N;
          const TC* Bt = lattice<TC>(pv) + td.lat_off + (int64_t)kLatSwB * td.N;
          u0[u] = ct * (A[Ux] * Bt[Uy]);
          u1[u] = -(ct * (A[Uy] * Bt[Ux]));
        }
      }
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        const int q = q0 + u * NT;
        if (q >= Gm::NI) continue;
        const int i = q % B, j = (q / B) % B, k = D == 3 ? q / (B * B) : 0;
        const TC* t0 = tile + Bx::tix(i, j, k);
        const TC dxv = ((t0[-2] - t0[2]) + TC(8) * (t0[1] - t0[-1])) * c;
        const TC dyv = ((t0[-2 * Bx::S] - t0[2 * Bx::S]) + TC(8) * (t0[Bx::S] - t0[-Bx::S])) * c;
        TC s = u0[u] * dxv + u1[u] * dyv;
        if (D == 3) {
          constexpr int P = Bx::S * Bx::S;
          const TC dzv = ((t0[-2 * P] - t0[2 * P]) + TC(8) * (t0[P] - t0[-P])) * c;
          s = s + uc2 * dzv;
        }
        const TS kk = (TS)(-s);
        const int64_t at = base + q;
        if (stage == 0) {
          acc[at] = yv[u] + cas * kk;
          ynext[at] = (TY)(yv[u] + cys * kk);
        } else if (stage == 1 || stage == 2) {
          acc[at] = av[u] + cas * kk;
          ynext[at] = (TY)(yv[u] + cys * kk);
        } else {
          y[at] = av[u] + cas * kk;
        }
      }
    }
    if (pn < nact && threadIdx.x < PL::INTS) {
      splan[buf ^ 1][threadIdx.x] = pre;
      if (threadIdx.x >= PL::NBO && threadIdx.x < PL::NBO + PL::NB) snb[buf ^ 1][threadIdx.x - PL::NBO] = (int64_t)pre * pv.vs;
    }
    __syncthreads();
  }
}

// 2D form of k_stage_adv with one warp per block: each warp of the CTA walks
// its own sequence of blocks (gather, stencils, update) with warp-level
// synchronisation only, so the per-block work (plan, coefficients, barriers)
// is done by 32 threads instead of a whole CTA.  Same values as k_stage_adv.
template <int B, int RHS, typename TS, typename TY, typename TSRC, int NT>
struct StageW {
  using Bx = Box<2, B, 2>;
  static constexpr int NW = NT / 32;
  // FP32 state: the block's state and accumulator rows are staged in shared
  // memory by the bulk-copy (TMA) engine, one mbarrier per warp
  static constexpr bool TMA = sizeof(TS) == 4;
  static constexpr int VS = (B * B + 3) / 4 * 4;  // padded block: the pool's per-variable stride
  // per warp: mbarrier; a region holding either the ring and the coarse-box
  // scratch of a block whose neighbourhood is not uniform, or the staged rows;
  // the tile
  static constexpr size_t BAR = TMA ? 16 : 0;
  static constexpr size_t RINGSCR = kRingBytesD<2> + sizeof(TY) * (Bx::CBOX + Bx::SCR);
  static constexpr size_t ROWS = TMA ? 2 * sizeof(TS) * VS : 0;
  static constexpr size_t UNION = ((RINGSCR > ROWS ? RINGSCR : ROWS) + 15) / 16 * 16;
  static constexpr size_t GTAB = (4 * Bx::NPTS + 15) / 16 * 16;
  static constexpr size_t WAREA = (BAR + UNION + sizeof(TY) * Bx::TILE + 15) / 16 * 16;
  static constexpr size_t SMEM = GTAB + NW * WAREA;
};

// ST: the RK stage, fixed at compile time (the per-point loads, stores and
// updates of each stage without run-time branches).
template <int B, int RHS, typename TS, typename TY, typename TSRC, int NT, int ST>
__global__ void __launch_bounds__(NT, 1024 / NT) k_stage_adv_w(PoolView pv, const TSRC* __restrict__ src, TS* __restrict__ y,
                                                   TS* __restrict__ acc, TY* __restrict__ ynext, int staging,
                                                   StageArgs sa) {
  pdl_enter();
  constexpr int stage = ST;
  static_assert(ST >= 0 && ST <= 3, "RK4 stage");
  using Gm = Geo<2, B>;
  using Bx = Box<2, B, 2>;
  using PL = Plan<2>;
  using SW = StageW<B, RHS, TS, TY, TSRC, NT>;
  using TC = TY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* sm = smem_as<unsigned char>(0);
  int32_t* gtab = reinterpret_cast<int32_t*>(sm);
  unsigned char* wa = sm + SW::GTAB + warp * SW::WAREA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(wa);
  unsigned char* un = wa + SW::BAR;  // ring + coarse-box scratch, or the staged rows
  RingD<2>& R = *reinterpret_cast<RingD<2>*>(un);
  TC* cbox = reinterpret_cast<TC*>(un + kRingBytesD<2>);
  TC* scr = cbox + Bx::CBOX;
  TS* ys = reinterpret_cast<TS*>(un);
  TS* as = ys + SW::VS;
  TC* tile = reinterpret_cast<TC*>(un + SW::UNION);
  __shared__ int64_t snb[SW::NW][PL::NB];
  build_gtab<2, B, 2>(gtab);
  if (SW::TMA && lane == 0) mbar_init(bar, 1);
  __syncthreads();
  unsigned phase = 0;
  const int nact = pv.cnt->n_act;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&pv.cnt->stage_blocks, (unsigned long long)nact);
  const int gw = blockIdx.x * SW::NW + warp, nwt = gridDim.x * SW::NW;
  int32_t cur = (gw < nact && lane < PL::INTS) ? pv.plan[(int64_t)gw * PL::INTS + lane] : 0;
  for (int p = gw; p < nact; p += nwt) {
    const int pn = p + nwt;
    const int32_t nxt = (pn < nact && lane < PL::INTS) ? pv.plan[(int64_t)pn * PL::INTS + lane] : 0;
    BlockInfo b;
    b.slot = __shfl_sync(0xffffffffu, cur, 0);
    const int meta = __shfl_sync(0xffffffffu, cur, 1);
    b.lvl = meta & 255;
    b.tree = (meta >> 8) & 0xffff;
    b.c[0] = __shfl_sync(0xffffffffu, cur, 2);
    b.c[1] = __shfl_sync(0xffffffffu, cur, 3);
    b.c[2] = 0;
    const TreeDev& td = pv.trees[b.tree];
    // stage 0 reads the state from the tile; the other stages stage the rows
    // (FP32, unless switched off) or load them
    const bool staged = SW::TMA && stage >= 1 && staging != 0;
    const bool uni = (meta >> 30) & 1;
    auto stage_rows = [&]() {
      if (lane == 0) {
        constexpr unsigned rows = (stage <= 2 ? 2 : 1) * sizeof(TS) * SW::VS;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, rows);
        if (stage <= 2) bulk_g2s(ys, y + (int64_t)b.slot * pv.vs, sizeof(TS) * SW::VS, bar);
        bulk_g2s(as, acc + (int64_t)b.slot * pv.vs, sizeof(TS) * SW::VS, bar);
      }
    };
    // uniform neighbourhood: the rows travel while the ghost layer is
    // gathered; otherwise the gather needs the shared region first
    if (staged && uni) stage_rows();
    if (uni) {
      if (lane >= PL::NBO && lane < PL::NBO + PL::NB) snb[warp][lane - PL::NBO] = (int64_t)cur * pv.vs;
      __syncwarp();
      gather_table<2, B, 2, 1, TSRC, TC, WarpGroup>(pv, (int64_t)b.slot * pv.vs, snb[warp], gtab, src, (TSRC*)src,
                                                    tile, stage == 0);
    } else {
      load_regions<2, WarpGroup>(pv, p, R);
      __syncwarp();
      fill_tile<2, B, TSRC, TC, 2, WarpGroup>(pv, b, src, (TSRC*)src, tile, stage == 0, R, cbox, scr, true);
    }
    __syncwarp();
    if (staged && !uni) stage_rows();
    if (staged) {
      // bounded wait: a copy that never lands is reported, not waited for
      if (!mbar_wait(bar, phase, 1 << 20)) {
        if (lane == 0) set_err(pv, kErrTimeout);
        return;
      }
      phase ^= 1;
    }
    const TC c = tree_cD<TC>(td, b.lvl);
    const StageCoef<TS> cs(pv, sa, b.tree, stage);
    const TC ct = StageCoef<TC>(pv, sa, b.tree, stage).ct;
    const TS cas = cs.ca, cys = cs.cy;
    const int64_t base = (int64_t)b.slot * pv.vs;
    const int sh = td.Jmax - b.lvl;
    const TC uc0 = tree_rhs<TC>(td, 0), uc1 = tree_rhs<TC>(td, 1);
    // points q0 + 32 u, u < UC: state, accumulator and velocity loads first,
    // then the stencils and the updates
    auto chunk = [&](auto ucc, int q0) {
      constexpr int UC = decltype(ucc)::value;
      TS yv[UC], av[UC];
      TC u0[UC], u1[UC];
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        const int q = q0 + u * 32;
        yv[u] = av[u] = TS(0);
        u0[u] = uc0;
        u1[u] = uc1;
        if (q >= Gm::NI) continue;
        if constexpr (SW::TMA) {
          // stage 0: the committed (synchronised) y_n is the tile's value
          if (stage == 0) yv[u] = (TS)tile[Bx::tix(q % B, q / B, 0)];
          if (stage == 1 || stage == 2) yv[u] = staged ? ys[q] : y[base + q];
          if (stage >= 1) av[u] = staged ? as[q] : acc[base + q];
        } else {
          if (stage <= 2) yv[u] = y[base + q];  // stage 0: committed (synchronised) y_n
          if (stage >= 1) av[u] = acc[base + q];
        }
        if (RHS == MR_RHS_SWIRL) {
          const int i = q % B, j = q / B;
          const int64_t Ux = pmod64((b.c[0] * (B - 1) + i) << sh, td.N);
          const int64_t Uy = pmod64((b.c[1] * (B - 1) + j) << sh, td.N);
          const TC* A = lattice<TC>(pv) + td.lat_off + (int64_t)kLatSwA * td.N;
          const TC* Bt = lattice<TC>(pv) + td.lat_off + (int64_t)kLatSwB * td.N;
          u0[u] = ct * (A[Ux] * Bt[Uy]);
          u1[u] = -(ct * (A[Uy] * Bt[Ux]));
        }
      }
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        const int q = q0 + u * 32;
        if (q >= Gm::NI) continue;
        const int i = q % B, j = q / B;
        const TC* t0 = tile + Bx::tix(i, j, 0);
        const TC dxv = ((t0[-2] - t0[2]) + TC(8) * (t0[1] - t0[-1])) * c;
        const TC dyv = ((t0[-2 * Bx::S] - t0[2 * Bx::S]) + TC(8) * (t0[Bx::S] - t0[-Bx::S])) * c;
        const TC s = u0[u] * dxv + u1[u] * dyv;
        const TS kk = (TS)(-s);
        const int64_t at = base + q;
        if (stage == 0) {
          acc[at] = yv[u] + cas * kk;
          ynext[at] = (TY)(yv[u] + cys * kk);
        } else if (stage == 1 || stage == 2) {
          acc[at] = av[u] + cas * kk;
          ynext[at] = (TY)(yv[u] + cys * kk);
        } else {
          y[at] = av[u] + cas * kk;
        }
      }
    };
    // full chunks of 4 points per lane, then one chunk for the remainder
    constexpr int UC = 4, FULL = Gm::NI / (UC * 32) * (UC * 32), UT = (Gm::NI - FULL + 31) / 32;
    for (int q0 = lane; q0 < FULL; q0 += UC * 32) chunk(std::integral_constant<int, UC>{}, q0);
    if constexpr (UT > 0) chunk(std::integral_constant<int, UT>{}, FULL + lane);
    __syncwarp();
    cur = nxt;
  }
}

// Stage plans of all active blocks, one warp per block (layout in Plan<D>):
// the 3^d - 1 equal-level neighbours, one lookup per lane in the dense leaf
// tables; for a block whose neighbourhood is not uniform, also its ring and
// class-box owner table (RingD), so that the four RK stages of the step and
// the first coarsening round gather without searching.  Both stay valid while
// the tree generation is unchanged.
template <int D, int B>
__global__ void __launch_bounds__(128) k_plan(PoolView pv) {
  pdl_enter();
  using PL = Plan<D>;
  static_assert(PL::NB <= 32 && PL::INTS <= 32, "one lane per neighbour");
  constexpr int NW = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RingD<D>& R = *smem_as<RingD<D>>((size_t)warp * kRingBytesD<D>);
  const int nact = pv.cnt->n_act;
  for (int p = blockIdx.x * NW + warp; p < nact; p += gridDim.x * NW) {
    const int s = pv.act[p];
    BlockInfo b;
    b.slot = s;
    b.lvl = pv.lvl[s];
    b.tree = pv.tree[s];
    for (int a = 0; a < 3; ++a) b.c[a] = a < D ? pv.crd[3 * s + a] : 0;
    const TreeDev& td = pv.trees[b.tree];
    int q = s;
    if (lane < PL::NB) {
      const int o[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, D == 3 ? lane / 9 - 1 : 0};
      if (o[0] != 0 || o[1] != 0 || o[2] != 0) {
        const int64_t cn[3] = {b.c[0] + o[0], b.c[1] + o[1], b.c[2] + o[2]};
        q = tab_get<D>(pv, td, b.lvl, cn);
      }
    }
    const bool uni = __all_sync(0xffffffffu, q >= 0);
    int32_t* out = pv.plan + (int64_t)p * PL::INTS;
    if (lane == 0) out[0] = s;
    if (lane == 1) out[1] = b.lvl | (b.tree << 8) | (uni ? 1 << 30 : 0);
    if (lane >= 2 && lane < 2 + D) out[lane] = (int32_t)b.c[lane - 2];
    const int qs = __shfl_sync(0xffffffffu, q, (lane - PL::NBO) & 31);
    if (lane >= PL::NBO && lane < PL::NBO + PL::NB) out[lane] = qs;
    if (!uni) {
      build_ring<D, B, WarpGroup>(pv, td, b, R);
      __syncwarp();
      build_regions<D, B, WarpGroup>(b, R);
      __syncwarp();
      store_regions<D, WarpGroup>(pv, p, R);
      __syncwarp();
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) pv.cnt->plan_topo = pv.cnt->topo;
}

// Start of a coarsening round: the blocks it works on (none once a round
// merged nothing), its id, and the per-tree threshold scales reset to v.
template <int D>
__global__ void k_round_begin(PoolView pv, double v) {
  pdl_enter();
  Counters* c = pv.cnt;
  if (threadIdx.x == 0) {
    c->n_round = c->done ? 0 : c->n_act;
    c->round_id += 1;
  }
  for (int i = threadIdx.x; i < pv.ntrees * pv.nvar; i += blockDim.x) pv.svar[i] = v;
}

// ------------------------------------------------------------- NS stage ----
// One RK4 stage of the 2D compressible Navier-Stokes equations (Sec. 4), ideal
// gas with constant c_p, in conservative flux form, q = (rho, rho u, rho v, E):
//   N(q) = -(dF/dx + dG/dy),
//   F = (rho u, rho u u + p - txx, rho u v - txy, (E + p) u - (u txx + v txy) - kap dth/dx),
//   G = (rho v, rho v u - txy, rho v v + p - tyy, (E + p) v - (u txy + v tyy) - kap dth/dy),
//   txx = mu (2 ux - 2/3 div), tyy = mu (2 vy - 2/3 div), txy = mu (uy + vx),
//   p = (gamma - 1)(E - (rho u u + rho v v)/2), th = p / rho,
//   kap = mu gamma / ((gamma - 1) Pr)  (R_s cancels in the heat flux),
// every derivative the 4th-order central D1.  Primitives on the whole tile,
// gradients and fluxes on nodes -2..B+1, flux divergence on the interior; the
// RK4 update is the same 3-register form as for advection, on 4 variables
// (with StageArgs::copy_state the last stage also stores the new state in the
// stage type into ynext, the shock filter's source).
template <int B>
struct NsGeo {
  static constexpr int NF = (B + 4) * B;  // F on i in [-2, B+1], j in [0, B-1]
  static constexpr int NG = B * (B + 4);  // G on i in [0, B-1], j in [-2, B+1]
};

template <int B, typename TS, typename TY, typename TSRC>
__global__ void __launch_bounds__(256) k_stage_ns(PoolView pv, const TSRC* __restrict__ src,
                                                  TS* __restrict__ y, TS* __restrict__ acc,
                                                  TY* __restrict__ ynext, TY* __restrict__ yn, int stage,
                                                  StageArgs sa) {
  pdl_enter();
  using Gm = Geo<2, B>;
  using NG = NsGeo<B>;
  using TC = TY;
  constexpr int T = Gm::T, G = Gm::G;
  RingD<2>& R = *smem_as<RingD<2>>(0);
  TC* tile = smem_as<TC>(kRingBytesD<2>);  // 4 x TILE conserved variables
  TC* cbox = tile + 4 * Gm::TILE;         // 4 x CBOX
  TC* pu = cbox + 4 * Gm::CBOX;           // primitives u, v, p, th: 4 x TILE
  TC* pvv = pu + Gm::TILE;
  TC* pp = pvv + Gm::TILE;
  TC* pth = pp + Gm::TILE;
  TC* F = pth + Gm::TILE;                 // 4 x NF
  TC* Gf = F + 4 * NG::NF;                // 4 x NG
  static_assert(Box<2, B, kG>::SCR <= Gm::TILE, "prediction scratch fits in the primitive arrays");
  using PL = Plan<2>;
  __shared__ int32_t splan[2][PL::INTS];
  const int nact = pv.cnt->n_act;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&pv.cnt->stage_blocks, (unsigned long long)nact);
  auto I = [&](int i, int j) { return (j + G) * T + (i + G); };
  auto fI = [&](int i, int j) { return j * (B + 4) + (i + 2); };
  auto gI = [&](int i, int j) { return (j + 2) * B + i; };
  if (blockIdx.x < nact && threadIdx.x < PL::INTS)
    splan[0][threadIdx.x] = pv.plan[(int64_t)blockIdx.x * PL::INTS + threadIdx.x];
  __syncthreads();
  int buf = 0;
  for (int p = blockIdx.x; p < nact; p += gridDim.x, buf ^= 1) {
    const int pn = p + gridDim.x;
    int32_t pre = 0;
    if (pn < nact && threadIdx.x < PL::INTS) pre = pv.plan[(int64_t)pn * PL::INTS + threadIdx.x];
    const int32_t* pl = splan[buf];
    const BlockInfo b = plan_block<2>(pl);
    const TreeDev& td = pv.trees[b.tree];
    if ((pl[1] >> 30) & 1) {
      gather_uniform<2, B, kG, 4, TSRC, TC>(pv, b, pl + PL::NBO, src, (TSRC*)src, tile, stage == 0);
    } else {
      load_regions<2, CtaGroup>(pv, p, R);
      __syncthreads();
      // prediction scratch: the primitive arrays, unused until the tile is complete
      fill_tile<2, B, TSRC, TC>(pv, b, src, (TSRC*)src, tile, stage == 0, R, cbox, pu, true);
    }
    __syncthreads();
    // gamma - 1, mu and kappa = mu gamma / ((gamma - 1) Pr), formed once per tree
    TC gm1, mu, kap;
    if constexpr (sizeof(TC) == 4) { gm1 = td.nsf[0]; mu = td.nsf[1]; kap = td.nsf[2]; }
    else { gm1 = td.nsd[0]; mu = td.nsd[1]; kap = td.nsd[2]; }
    const TC c23 = (TC)(2.0 / 3.0);
    const TC c = tree_cD<TC>(td, b.lvl);
    const TC* r_ = tile;
    const TC* m1_ = tile + Gm::TILE;
    const TC* m2_ = tile + 2 * Gm::TILE;
    const TC* E_ = tile + 3 * Gm::TILE;
    for (int idx = threadIdx.x; idx < Gm::TILE; idx += blockDim.x) {
      const TC r = r_[idx], m1 = m1_[idx], m2 = m2_[idx], E = E_[idx];
      const TC uu = m1 / r, vv = m2 / r;
      const TC prs = gm1 * (E - TC(0.5) * (m1 * uu + m2 * vv));
      pu[idx] = uu;
      pvv[idx] = vv;
      pp[idx] = prs;
      pth[idx] = prs / r;
    }
    __syncthreads();
    auto dx = [&](const TC* f, int i, int j) {
      return ((f[I(i - 2, j)] - f[I(i + 2, j)]) + TC(8) * (f[I(i + 1, j)] - f[I(i - 1, j)])) * c;
    };
    auto dy = [&](const TC* f, int i, int j) {
      return ((f[I(i, j - 2)] - f[I(i, j + 2)]) + TC(8) * (f[I(i, j + 1)] - f[I(i, j - 1)])) * c;
    };
    constexpr int W = B + 4;
    for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
      const int i = idx % W - 2, j = idx / W - 2;
      const bool needF = j >= 0 && j < B, needG = i >= 0 && i < B;
      if (!needF && !needG) continue;
      const TC ux = dx(pu, i, j), vx = dx(pvv, i, j), uy = dy(pu, i, j), vy = dy(pvv, i, j);
      const TC div = ux + vy;
      const TC txy = mu * (uy + vx);
      const int t0 = I(i, j);
      const TC m1 = m1_[t0], m2 = m2_[t0], E = E_[t0];
      const TC uu = pu[t0], vv = pvv[t0], prs = pp[t0];
      if (needF) {
        const TC txx = mu * (TC(2) * ux - c23 * div);
        const TC thx = dx(pth, i, j);
        const int f0 = fI(i, j);
        F[f0] = m1;
        F[NG::NF + f0] = m1 * uu + prs - txx;
        F[2 * NG::NF + f0] = m1 * vv - txy;
        F[3 * NG::NF + f0] = (E + prs) * uu - (uu * txx + vv * txy) - kap * thx;
      }
      if (needG) {
        const TC tyy = mu * (TC(2) * vy - c23 * div);
        const TC thy = dy(pth, i, j);
        const int g0 = gI(i, j);
        Gf[g0] = m2;
        Gf[NG::NG + g0] = m2 * uu - txy;
        Gf[2 * NG::NG + g0] = m2 * vv + prs - tyy;
        Gf[3 * NG::NG + g0] = (E + prs) * vv - (uu * txy + vv * tyy) - kap * thy;
      }
    }
    __syncthreads();
    const StageCoef<TS> cs(pv, sa, b.tree, stage);
    const StageCoef<TC> cf(pv, sa, b.tree, stage);
    const int64_t base = (int64_t)b.slot * 4 * pv.vs;
    const TS cas = cs.ca, cys = cs.cy;  // RK weights in the state type
    const TC casf = cf.ca, cysf = cf.cy;  // and in the stage type
    // UC points per thread at a time: state and accumulator loads first.  With
    // an FP64 state and FP32 stages the next stage field needs y_n only in FP32:
    // stage 0 takes it from the tile (the committed state, rounded) and keeps
    // it in yn for stages 1 and 2, which then read no FP64 state.
    constexpr bool MIX = sizeof(TS) == 8 && sizeof(TC) == 4;
    constexpr int UC = 4, NT = 256;
    for (int i0 = threadIdx.x; i0 < 4 * Gm::NI; i0 += UC * NT) {
      TS yv[UC], av[UC];
      TC yf[UC];
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        const int idx = i0 + u * NT;
        yv[u] = av[u] = TS(0);
        yf[u] = TC(0);
        if (idx >= 4 * Gm::NI) continue;
        const int v = idx / Gm::NI, q = idx % Gm::NI;
        const int64_t at = base + (int64_t)v * pv.vs + q;
        if (stage == 0 || (!MIX && stage <= 2)) yv[u] = y[at];
        if (stage >= 1) av[u] = acc[at];
        if constexpr (MIX) {
          if (stage == 0) {
            yf[u] = tile[v * Gm::TILE + I(q % B, q / B)];
            yn[at] = yf[u];
          } else if (stage <= 2) {
            yf[u] = yn[at];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        const int idx = i0 + u * NT;
        if (idx >= 4 * Gm::NI) continue;
        const int v = idx / Gm::NI, q = idx % Gm::NI;
        const int i = q % B, j = q / B;
        const TC* Fv = F + v * NG::NF;
        const TC* Gv = Gf + v * NG::NG;
        const TC dFx = ((Fv[fI(i - 2, j)] - Fv[fI(i + 2, j)]) + TC(8) * (Fv[fI(i + 1, j)] - Fv[fI(i - 1, j)])) * c;
        const TC dGy = ((Gv[gI(i, j - 2)] - Gv[gI(i, j + 2)]) + TC(8) * (Gv[gI(i, j + 1)] - Gv[gI(i, j - 1)])) * c;
        const int64_t at = base + (int64_t)v * pv.vs + q;
        if constexpr (sizeof(TS) == 8 && sizeof(TC) == 4) {
          // FP64 state, FP32 stages: the increments dt k are formed in FP32 and
          // only accumulated in FP64 (one conversion and one FP64 add per
          // update; FP64 arithmetic is a small fraction of the FP32 rate here),
          // the FP32 stage value from the FP32-rounded state
          const TC kc = -(dFx + dGy);
          if (stage == 0) {
            acc[at] = yv[u] + (TS)(casf * kc);
            ynext[at] = (TY)(yf[u] + cysf * kc);
          } else if (stage == 1 || stage == 2) {
            acc[at] = av[u] + (TS)(casf * kc);
            ynext[at] = (TY)(yf[u] + cysf * kc);
          } else {
            const TS yn = av[u] + (TS)(casf * kc);
            y[at] = yn;
            if (sa.copy_state) ynext[at] = (TY)yn;
          }
        } else {
          const TS kk = (TS)(-(dFx + dGy));
          if (stage == 0) {
            acc[at] = yv[u] + cas * kk;
            ynext[at] = (TY)(yv[u] + cys * kk);
          } else if (stage == 1 || stage == 2) {
            acc[at] = av[u] + cas * kk;
            ynext[at] = (TY)(yv[u] + cys * kk);
          } else {
            const TS yn = av[u] + cas * kk;
            y[at] = yn;
            if (sa.copy_state) ynext[at] = (TY)yn;
          }
        }
      }
    }
    if (pn < nact && threadIdx.x < PL::INTS) splan[buf ^ 1][threadIdx.x] = pre;
    __syncthreads();
  }
}

// ----------------------------------------------------------------- refine ----
// x pass of the upsampling: fine x in [0, 2(B-1)] on mother rows y, z in [-1, B]
template <int D, int B>
struct RefGeo {
  static constexpr int NF = 2 * B - 1;
  static constexpr int NR = B + 2;
  static constexpr int NX = NF * NR * (D == 3 ? NR : 1);
};

// Sec. 2.3: the synchronised mother tile is upsampled by the 4th-order
// interpolating prediction and split into 2^d children (one treecode digit
// appended); children are placed in the new active list in Hilbert order.
template <int D, int B, typename TS, int NT>
__global__ void __launch_bounds__(NT, NT <= 128 ? 8 : (D == 3 ? 3 : 4)) k_refine(PoolView pv, TS* __restrict__ y) {
  pdl_enter();
  using Gm = Geo<D, B>;
  using Bx = Box<D, B, 1>;  // prediction of the children reaches one node
  using RG = RefGeo<D, B>;
  RingD<D>& R = *smem_as<RingD<D>>(0);
  __shared__ int cslot[8];
  TS* tile = smem_as<TS>(kRingBytesD<D>);
  TS* cbox = tile + pv.nvar * Bx::TILE;
  TS* scr = cbox + pv.nvar * Bx::CBOX;  // gather scratch, then the x pass of the upsampling
  TS* X = scr;
  const int nact = pv.cnt->n_act;
  const int n_alloc = pv.cnt->n_alloc, n_free = pv.cnt->n_free;
  if (n_alloc > n_free) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_err(pv, kErrCapacity);
    return;
  }
  if (n_alloc == 0) return;  // no block refines: the list stays as it is
  const int nv = pv.nvar;
  for (int p = blockIdx.x; p < nact; p += gridDim.x) {
    const int slot = pv.act[p];
    const int e = pv.eoff[2 * p], a = pv.eoff[2 * p + 1];
    if (pv.flag[slot] != 1) {
      if (threadIdx.x == 0) pv.act_next[e] = slot;
      continue;
    }
    const BlockInfo b = load_block(pv, slot);
    const TreeDev& td = pv.trees[b.tree];
    build_ring<D, B>(pv, td, b, R);
    __syncthreads();
    if constexpr (D == 2)
      fill_tile<D, B, TS, TS, 1>(pv, b, y, y, tile, false, R, cbox, scr);
    else
      fill_cols<B, TS, TS, 1>(pv, b, nullptr, y, y, tile, false, R, cbox, scr);
    if (threadIdx.x == 0) {
      uint64_t key[8];
      int32_t cc[8][3];
      for (int ch = 0; ch < Gm::NCH; ++ch) {
        cslot[ch] = pv.freelist[n_free - n_alloc + a + ch];
        for (int ax = 0; ax < 3; ++ax)
          cc[ch][ax] = ax < D ? (int32_t)(2 * b.c[ax] + ((ch >> ax) & 1)) : 0;
        key[ch] = block_key<D>(cc[ch], b.lvl + 1, td.Jmax);
      }
      for (int ch = 0; ch < Gm::NCH; ++ch) {
        int rank = 0;
        for (int o = 0; o < Gm::NCH; ++o) rank += key[o] < key[ch];
        const int cs = cslot[ch];
        pv.act_next[e + rank] = cs;
        pv.lvl[cs] = (int8_t)(b.lvl + 1);
        pv.tree[cs] = (int16_t)b.tree;
        for (int ax = 0; ax < 3; ++ax) pv.crd[3 * cs + ax] = cc[ch][ax];
        pv.hkey[cs] = key[ch];
        pv.flag[cs] = 0;
      }
    }
    __syncthreads();
    // Separable upsampling, per variable: X = prediction along x on the
    // mother's rows (y, z in [-1, B]), then y (and z) per child node -- the
    // operations of the tensor product in the same order.
    for (int v = 0; v < nv; ++v) {
      const TS* tv = tile + v * Bx::TILE;
      for (int idx = threadIdx.x; idx < RG::NX; idx += blockDim.x) {
        const int ox = idx % RG::NF, jy = (idx / RG::NF) % RG::NR - 1;
        const int kz = D == 3 ? idx / (RG::NF * RG::NR) - 1 : 0;
        const int fl = ox >> 1;
        X[idx] = (ox & 1) ? dd4(tv[Bx::tix(fl - 1, jy, kz)], tv[Bx::tix(fl, jy, kz)], tv[Bx::tix(fl + 1, jy, kz)],
                                tv[Bx::tix(fl + 2, jy, kz)])
                          : tv[Bx::tix(fl, jy, kz)];
      }
      __syncthreads();
      auto xr = [&](int ox, int jy, int kz) { return X[((D == 3 ? kz + 1 : 0) * RG::NR + (jy + 1)) * RG::NF + ox]; };
      for (int idx = threadIdx.x; idx < Gm::NCH * Gm::NI; idx += blockDim.x) {
        const int ch = idx / Gm::NI, q = idx % Gm::NI;
        const int i = q % B, j = (q / B) % B, k = D == 3 ? q / (B * B) : 0;
        const int ox = ((ch >> 0) & 1) * (B - 1) + i, oy = ((ch >> 1) & 1) * (B - 1) + j;
        const int oz = D == 3 ? ((ch >> 2) & 1) * (B - 1) + k : 0;
        auto ypass = [&](int kz) -> TS {
          const int fl = oy >> 1;
          return (oy & 1) ? dd4(xr(ox, fl - 1, kz), xr(ox, fl, kz), xr(ox, fl + 1, kz), xr(ox, fl + 2, kz))
                          : xr(ox, fl, kz);
        };
        TS val;
        if (D == 2) {
          val = ypass(0);
        } else {
          const int fl = oz >> 1;
          val = (oz & 1) ? dd4(ypass(fl - 1), ypass(fl), ypass(fl + 1), ypass(fl + 2)) : ypass(fl);
        }
        y[((int64_t)cslot[ch] * nv + v) * pv.vs + q] = val;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- details ----
// Sec. 2.3: D = B - P(R(B)) on the synchronised tile (R keeps even tile nodes,
// ghosts included; P predicts the odd ones).  Per block and variable the
// largest |d| (warp-shuffle max, then across warps) and the largest |q_v|.
// P is evaluated separably in the fixed order x, then y, then z: the x pass
// over all coarse rows is stored in shared memory (X), the y and z passes run
// per point; every output sees the same operations as the point-wise tensor
// product.
// The FP32 maximum m32 is within E of the FP64 one, and m32 + E < eps or
// m32 - E >= eps holds in exact arithmetic: the sum is rounded up and compared
// with eps rounded down, the difference rounded down and compared with eps
// rounded up, so the threshold decision needs no FP64 evaluation.
__device__ __forceinline__ bool certain_vs_eps(float m32, float E, const TreeDev& td) {
  return __fadd_ru(m32, E) < td.epsf[0] || __fsub_rd(m32, E) >= td.epsf[1];
}

template <int D, int B>
struct DetGeo {
  static constexpr int NC = (B + 1) / 2 + 2;  // coarse rows -1 .. (B+1)/2
  static constexpr int NX = NC * B * (D == 3 ? NC : 1);
  static constexpr int NY = D == 3 ? B * B * NC : 0;  // 3D: after the y pass, coarse z rows
};

// Maximum of v over the CTA (warp shuffles, then one value per warp in red);
// every thread gets the result.  In the value's own type: FP64 operations are
// a small fraction of the FP32 rate on this GPU, so FP32 data stay FP32.
template <typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
  for (int s = 16; s > 0; s >>= 1) v = fmax(v, (T)__shfl_xor_sync(0xffffffffu, v, s));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
  return v;
}

// Maxima of a and b over the CTA in one reduction (warp shuffles, then one
// value per warp in ra / rb); every thread gets the results.
template <typename A, typename Bt>
__device__ __forceinline__ void block_max2(A& a, Bt& b, A* ra, Bt* rb) {
  for (int s = 16; s > 0; s >>= 1) {
    a = fmax(a, (A)__shfl_xor_sync(0xffffffffu, a, s));
    b = fmax(b, (Bt)__shfl_xor_sync(0xffffffffu, b, s));
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = a;
    rb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    a = fmax(a, ra[w]);
    b = fmax(b, rb[w]);
  }
}

// Maxima of a, b and c over the CTA in one reduction (one value per warp in
// ra / rb / rc); every thread gets the results.
template <typename A, typename Bt, typename Ct>
__device__ __forceinline__ void block_max3(A& a, Bt& b, Ct& c, A* ra, Bt* rb, Ct* rc) {
  for (int s = 16; s > 0; s >>= 1) {
    a = fmax(a, (A)__shfl_xor_sync(0xffffffffu, a, s));
    b = fmax(b, (Bt)__shfl_xor_sync(0xffffffffu, b, s));
    c = fmax(c, (Ct)__shfl_xor_sync(0xffffffffu, c, s));
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = a;
    rb[threadIdx.x >> 5] = b;
    rc[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    a = fmax(a, ra[w]);
    b = fmax(b, rb[w]);
    c = fmax(c, rc[w]);
  }
}

// 2D detail index tables (per CTA, shared memory): the x pass on coarse rows
// yc in [-1, NC - 2] (entry (yc + 1) B + x: tile index of its first source node,
// x odd = 4 sources two nodes apart) and the odd interior points in row-major
// order (tile index, first x-pass entry of the y pass, j odd = 4 entries B apart).
template <int B>
struct DetTab {
  using Bx = Box<2, B, 2>;
  using DG = DetGeo<2, B>;
  static constexpr int NODD = B * B - ((B + 1) / 2) * ((B + 1) / 2);
  static constexpr int INTS = DG::NX + NODD;
  static_assert(Bx::NPTS < (1 << 12) && DG::NX < (1 << 12), "table entries fit their fields");
  __device__ static void build(int32_t* xtab, int32_t* otab) {
    for (int idx = threadIdx.x; idx < DG::NX; idx += blockDim.x) {
      const int x = idx % B, yy = 2 * (idx / B - 1);
      const int odd = x & 1;
      const int b0 = odd ? Bx::tix(x - 3, yy, 0) : Bx::tix(x, yy, 0);
      xtab[idx] = b0 | (odd << 16);
    }
    for (int k = threadIdx.x; k < NODD; k += blockDim.x) {
      // rows j even hold (B - 1) / 2 odd points (odd i), rows j odd hold B
      const int per2 = (B - 1) / 2 + B;
      const int jp = k / per2, r = k % per2;
      int i, j;
      if (r < (B - 1) / 2) { j = 2 * jp; i = 2 * r + 1; }
      else { j = 2 * jp + 1; i = r - (B - 1) / 2; }
      const int jodd = j & 1;
      const int xb = jodd ? ((j - 1) / 2) * B + i : (j / 2 + 1) * B + i;
      otab[k] = Bx::tix(i, j, 0) | (xb << 12) | (jodd << 24);
    }
  }
  // block maximum of |d| in type A over one variable's tile tv (G: CTA or warp;
  // XA: NX values of scratch), the same operations as the point-wise evaluation
  template <typename A, typename TV, typename G>
  __device__ static A max_detail(const int32_t* xtab, const int32_t* otab, const TV* tv, A* XA, G g) {
    for (int idx = g.rank(); idx < DG::NX; idx += g.size()) {
      const int e = xtab[idx];
      const TV* t0 = tv + (e & 0xffff);
      XA[idx] = (e >> 16) ? dd4((A)t0[0], (A)t0[2], (A)t0[4], (A)t0[6]) : (A)t0[0];
    }
    g.sync();
    A md = A(0);
    for (int k = g.rank(); k < NODD; k += g.size()) {
      const int e = otab[k];
      const A val = (A)tv[e & 0xfff];
      const A* xa = XA + ((e >> 12) & 0xfff);
      const A pr = (e >> 24) ? dd4(xa[0], xa[B], xa[2 * B], xa[3 * B]) : xa[0];
      md = fmax(md, (A)fabs(val - pr));
    }
    return md;
  }
  // the same, and from the same sweeps (per thread, not reduced): the largest
  // |value| of the interior (mq; the odd points of the second sweep and the
  // even-even interior nodes of the first) with a non-finite test (bad), and
  // the largest |value| of the coarse lattice the first sweep reads (mt)
  template <typename A, typename TV, typename G>
  __device__ static A max_detail_ex(const int32_t* xtab, const int32_t* otab, const TV* tv, A* XA, G g, TV& mq,
                                    float& mt, bool& bad) {
    for (int idx = g.rank(); idx < DG::NX; idx += g.size()) {
      const int e = xtab[idx];
      const TV* t0 = tv + (e & 0xffff);
      if (e >> 16) {
        const TV a = t0[0], b = t0[2], c = t0[4], d = t0[6];
        mt = fmaxf(fmaxf(mt, fmaxf(fabsf((float)a), fabsf((float)b))), fmaxf(fabsf((float)c), fabsf((float)d)));
        XA[idx] = dd4((A)a, (A)b, (A)c, (A)d);
      } else {
        const TV a = t0[0];
        mt = fmaxf(mt, fabsf((float)a));
        const int row = idx / B;  // coarse row + 1: interior rows 1 .. (B + 1) / 2
        if (row >= 1 && row <= (B + 1) / 2) {
          mq = fmax(mq, (TV)fabs(a));
          bad |= !isfinite(a);
        }
        XA[idx] = (A)a;
      }
    }
    g.sync();
    A md = A(0);
    for (int k = g.rank(); k < NODD; k += g.size()) {
      const int e = otab[k];
      const TV tq = tv[e & 0xfff];
      mq = fmax(mq, (TV)fabs(tq));
      bad |= !isfinite(tq);
      const A val = (A)tq;
      const A* xa = XA + ((e >> 12) & 0xfff);
      const A pr = (e >> 24) ? dd4(xa[0], xa[B], xa[2 * B], xa[3 * B]) : xa[0];
      md = fmax(md, (A)fabs(val - pr));
    }
    return md;
  }
};

// Shared-memory layout of k_details after the ring and the tile: the coarse
// box and prediction scratch of the gather, reused once the tile is complete
// for the passes of the prediction (X, and in 3D the y pass Y).  A pass in
// type A keeps Y when it fits in that region, else (3D FP64 over an FP32 tile)
// evaluates the y pass again per point: the same operations in the same order.
template <int D, int B, typename TT, typename TD>
struct DetSmem {
  using Bx = Box<D, B, 2>;
  using DG = DetGeo<D, B>;
  static constexpr size_t FILL = sizeof(TT) * (Bx::CBOX + Bx::SCR);  // per variable
  template <typename A>
  __host__ __device__ static constexpr bool ystore() { return D == 2 || sizeof(A) * (DG::NX + DG::NY) <= FILL; }
  template <typename A>
  __host__ __device__ static constexpr size_t pass_bytes() {
    return sizeof(A) * (ystore<A>() ? DG::NX + DG::NY : DG::NX);
  }
  static constexpr size_t PASS = pass_bytes<TD>() > pass_bytes<float>() ? pass_bytes<TD>() : pass_bytes<float>();
  __host__ __device__ static size_t region(int nv) { return FILL * nv > PASS ? FILL * nv : PASS; }
};

template <int D, int B, typename TS, typename TD, int NT, typename TT = TS>
__global__ void __launch_bounds__(NT, NT <= 128 ? 8 : (D == 3 ? 3 : 4)) k_details(PoolView pv, TS* __restrict__ y) {
  pdl_enter();
  using Gm = Geo<D, B>;
  using Bx = Box<D, B, 2>;  // prediction from even nodes reaches two nodes
  using DG = DetGeo<D, B>;
  RingD<D>& R = *smem_as<RingD<D>>(0);
  __shared__ double red[2][32];
  TT* tile = smem_as<TT>(kRingBytesD<D>);  // tile type (TS or FP32); TD is the decision type
  TT* cbox = tile + pv.nvar * Bx::TILE;
  // gather scratch, reused for the passes once the tile is complete
  TT* scr = cbox + pv.nvar * Bx::CBOX;
  using DS = DetSmem<D, B, TT, TD>;
  TD* X = reinterpret_cast<TD*>((reinterpret_cast<uintptr_t>(cbox) + 15) & ~(uintptr_t)15);
  const int nact = pv.cnt->n_round;
  const int nv = pv.nvar;
  const bool all_blocks = pv.cnt->first_round != 0;
  const int prev = pv.cnt->round_id - 1;
  __shared__ int dirty;
  using PL = Plan<D>;
  __shared__ int32_t snb[PL::NB];
  __shared__ int64_t snbo[PL::NB];  // pool offsets of the neighbours
  __shared__ int32_t splan[2][PL::INTS];
  // the stage plans are used while the tree is the one they were built for
  // (the first round after the RK stages); the next block's plan is fetched
  // while a block is processed
  const bool plan_ok = pv.cnt->plan_topo == pv.cnt->topo;
  const size_t xbytes = DS::region(nv);
  int32_t* gtab = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(X) + ((xbytes + 15) & ~(size_t)15));
  int32_t* xtab = gtab + Bx::NPTS;  // 2D detail tables
  int32_t* otab = xtab + DG::NX;
  if constexpr (D == 2) {
    build_gtab<D, B, 2>(gtab);
    DetTab<B>::build(xtab, otab);
  }
  // CTA-local work count and threshold scales (one atomic per CTA, not per block)
  unsigned long long ndet = 0;
  __shared__ double csv[kMaxVar];
  __shared__ int csv_tree;
  if (threadIdx.x < kMaxVar) csv[threadIdx.x] = 0.0;
  if (threadIdx.x == 0) csv_tree = -1;
  auto flush_csv = [&]() {
    if (csv_tree >= 0 && threadIdx.x < nv && csv[threadIdx.x] > 0.0)
      atomic_max_pos(&pv.svar[csv_tree * nv + threadIdx.x], csv[threadIdx.x]);
  };
  if (plan_ok && blockIdx.x < nact && threadIdx.x < PL::INTS)
    splan[0][threadIdx.x] = pv.plan[(int64_t)blockIdx.x * PL::INTS + threadIdx.x];
  __syncthreads();
  int buf = 0;
  for (int p = blockIdx.x; p < nact; p += gridDim.x, buf ^= 1) {
    const int pn = p + gridDim.x;
    int32_t pre = 0;
    if (plan_ok && pn < nact && threadIdx.x < PL::INTS) pre = pv.plan[(int64_t)pn * PL::INTS + threadIdx.x];
    BlockInfo b;
    int q = 0;
    if (plan_ok) {
      b = plan_block<D>(splan[buf]);
      q = threadIdx.x < PL::NB ? splan[buf][PL::NBO + threadIdx.x] : b.slot;
    } else {
      b = load_block(pv, pv.act[p]);
      // equal-level neighbours, one lookup per thread: uniform when all exist
      q = b.slot;
      if (threadIdx.x < PL::NB) {
        const int n = threadIdx.x;
        const int o[3] = {n % 3 - 1, (n / 3) % 3 - 1, D == 3 ? n / 9 - 1 : 0};
        if (o[0] != 0 || o[1] != 0 || o[2] != 0) {
          const TreeDev& tdl = pv.trees[b.tree];
          const int64_t cn[3] = {b.c[0] + o[0], b.c[1] + o[1], b.c[2] + o[2]};
          q = tab_get<D>(pv, tdl, b.lvl, cn);
        }
      }
    }
    const TreeDev& td = pv.trees[b.tree];
    if (pv.norm_kind == 1 && b.tree != csv_tree) {  // block of another tree: flush the scales
      flush_csv();
      __syncthreads();
      if (threadIdx.x < kMaxVar) csv[threadIdx.x] = 0.0;
      if (threadIdx.x == 0) csv_tree = b.tree;
    }
    if (threadIdx.x < PL::NB) {
      snb[threadIdx.x] = q;
      snbo[threadIdx.x] = (int64_t)q * nv * pv.vs;
    }
    if (threadIdx.x == 0) dirty = all_blocks ? 1 : 0;
    const bool uni = __syncthreads_and(q >= 0);
    if (uni) {
      // the ring's leaves are the block and its 3^d - 1 equal-level neighbours
      if (!all_blocks && threadIdx.x < PL::NB && pv.stamp[q] == prev) dirty = 1;
    } else if (plan_ok && all_blocks) {
      // every block is evaluated and the tree is the stage plan's: its
      // class-box owner table is ready
      load_regions<D, CtaGroup>(pv, p, R);
    } else {
      build_ring<D, B>(pv, td, b, R);
      __syncthreads();
      if (!all_blocks && threadIdx.x < Gm::NR && R.slot[threadIdx.x] >= 0 &&
          pv.stamp[R.slot[threadIdx.x]] == prev)
        dirty = 1;
    }
    __syncthreads();
    if (!dirty) {
      // No leaf of the ring changed in the previous round: the synchronised
      // tile, hence the details and norms stored for this block, are unchanged.
      if (pv.norm_kind == 1 && threadIdx.x < nv)
        csv[threadIdx.x] = fmax(csv[threadIdx.x], pv.bmax[(int64_t)b.slot * nv + threadIdx.x]);
      if (plan_ok && pn < nact && threadIdx.x < PL::INTS) splan[buf ^ 1][threadIdx.x] = pre;
      __syncthreads();
      continue;
    }
    ndet += 1;
    const int64_t own = (int64_t)b.slot * nv * pv.vs;
    if (uni && nv == 1 && D == 2)
      gather_table<D, B, 2, 1, TS, TT>(pv, own, snbo, gtab, y, y, tile, true);
    else if (uni && nv == 4 && D == 2)
      gather_table<D, B, 2, 4, TS, TT>(pv, own, snbo, gtab, y, y, tile, true);
    else if (D == 3 && uni) {
      if constexpr (D == 3) fill_cols<B, TS, TT, 2>(pv, b, snbo, y, y, tile, true, R, cbox, scr);
    } else {
      if (uni) {
        build_ring<D, B>(pv, td, b, R);
        __syncthreads();
      }
      const bool ready = !uni && plan_ok && all_blocks;
      if constexpr (D == 2)
        fill_tile<D, B, TS, TT, 2>(pv, b, y, y, tile, true, R, cbox, scr, ready);
      else
        fill_cols<B, TS, TT, 2>(pv, b, nullptr, y, y, tile, true, R, cbox, scr, ready);
    }
    __syncthreads();
    // Block maximum of |d| over the interior with arithmetic type A: x pass on
    // coarse rows (yc, zc) in [-1, NC-2] into X, then y (and z) per odd node.
    // 3D with EX: the same sweeps also give the interior's largest |value| and
    // non-finite test (ex_mq, bad; the z sweep reads every interior node) and
    // the coarse lattice's largest |value| (ex_mt; the x sweep reads every
    // coarse node of the tile), reduced with the detail maximum in one step.
    TT ex_mq = TT(0);
    float ex_mt = 0.f;
    bool bad = false;
    auto pass = [&](auto tag, const TT* tv, auto exc) -> decltype(tag) {
      using A = decltype(tag);
      constexpr bool EX = decltype(exc)::value;
      A* XA = reinterpret_cast<A*>(X);
      if constexpr (D == 2) {
        if constexpr (EX) {
          TT mq = TT(0);
          float mt = 0.f;
          A md = DetTab<B>::template max_detail_ex<A>(xtab, otab, tv, XA, CtaGroup{}, mq, mt, bad);
          block_max3<A, TT, float>(md, mq, mt, reinterpret_cast<A*>(red[0]), reinterpret_cast<TT*>(red[1]),
                                   reinterpret_cast<float*>(red[1]) + 32);
          ex_mq = mq;
          ex_mt = mt;
          return md;
        } else {
          const A md = DetTab<B>::template max_detail<A>(xtab, otab, tv, XA, CtaGroup{});
          return block_max<A>(md, reinterpret_cast<A*>(red[0]));
        }
      }
      float mt = 0.f;
      for (int idx = threadIdx.x; idx < DG::NX; idx += blockDim.x) {
        const int x = idx % B, yc = (idx / B) % DG::NC - 1, zc = D == 3 ? idx / (B * DG::NC) - 1 : 0;
        const int yy = 2 * yc, zz = 2 * zc;
        A val;
        if ((x & 1) == 0) {
          const TT t = tv[Bx::tix(x, yy, zz)];
          if constexpr (EX) mt = fmaxf(mt, fabsf((float)t));
          val = (A)t;
        } else {
          const int n0 = (x - 1) / 2;
          const TT t0 = tv[Bx::tix(2 * n0 - 2, yy, zz)], t1 = tv[Bx::tix(2 * n0, yy, zz)],
                   t2 = tv[Bx::tix(2 * n0 + 2, yy, zz)], t3 = tv[Bx::tix(2 * n0 + 4, yy, zz)];
          if constexpr (EX)
            mt = fmaxf(fmaxf(mt, fmaxf(fabsf((float)t0), fabsf((float)t1))), fmaxf(fabsf((float)t2), fabsf((float)t3)));
          val = dd4((A)t0, (A)t1, (A)t2, (A)t3);
        }
        XA[idx] = val;
      }
      __syncthreads();
      auto xat = [&](int x, int yc, int zc) { return XA[((D == 3 ? (zc + 1) * DG::NC : 0) + (yc + 1)) * B + x]; };
      auto ypass = [&](int i, int j, int zc) -> A {
        if ((j & 1) == 0) return xat(i, j / 2, zc);
        const int m0 = (j - 1) / 2;
        return dd4(xat(i, m0 - 1, zc), xat(i, m0, zc), xat(i, m0 + 1, zc), xat(i, m0 + 2, zc));
      };
      // 3D: the y pass once per (x, y, coarse z row), kept for the z pass
      // where it fits (else evaluated again for each use)
      constexpr bool ys = DS::template ystore<A>();
      A* YA = XA + DG::NX;
      if (D == 3 && ys) {
        for (int idx = threadIdx.x; idx < DG::NY; idx += blockDim.x)
          YA[idx] = ypass(idx % B, (idx / B) % B, idx / (B * B) - 1);
        __syncthreads();
      }
      auto yat = [&](int i, int j, int zc) -> A {
        if constexpr (ys) return YA[((zc + 1) * B + j) * B + i];
        else return ypass(i, j, zc);
      };
      A md = A(0);  // a maximum of A values: exact in A
      TT mq = TT(0);
      for (int q = threadIdx.x; q < Gm::NI; q += blockDim.x) {
        const int i = q % B, j = (q / B) % B, k = D == 3 ? q / (B * B) : 0;
        const TT tq = tv[Bx::tix(i, j, k)];
        if constexpr (EX) {
          mq = fmax(mq, (TT)fabs(tq));
          bad |= !isfinite(tq);
        }
        if (((i | j | k) & 1) == 0) continue;
        const A val = (A)tq;
        A pr;
        if (D == 2) {
          pr = ypass(i, j, 0);
        } else if ((k & 1) == 0) {
          pr = yat(i, j, k / 2);
        } else {
          const int k0 = (k - 1) / 2;
          pr = dd4(yat(i, j, k0 - 1), yat(i, j, k0), yat(i, j, k0 + 1), yat(i, j, k0 + 2));
        }
        const A d = val - pr;
        md = fmax(md, (A)fabs(d));
      }
      if constexpr (EX) {
        block_max3<A, TT, float>(md, mq, mt, reinterpret_cast<A*>(red[0]), reinterpret_cast<TT*>(red[1]),
                                 reinterpret_cast<float*>(red[1]) + 32);
        ex_mq = mq;
        ex_mt = mt;
        return md;
      }
      return block_max<A>(md, reinterpret_cast<A*>(red[0]));
    };
    for (int v = 0; v < nv; ++v) {
      const TT* tv = tile + v * Bx::TILE;
      constexpr bool cert = sizeof(TT) == 4 && sizeof(TD) == 8;
      // the first pass's sweeps (x and z in 3D, x and odd points in 2D) give the
      // detail maximum, the interior's largest |value| (exact in its type), the
      // non-finite test (any non-finite value makes the block norm NaN) and,
      // for the certified FP32 decision, the largest |value| the evaluation
      // reads (interior and coarse lattice), all in one CTA reduction
      using A0 = std::conditional_t<cert, float, TD>;
      const A0 m0 = pass(A0(0), tv, std::true_type{});
      const TT mqt = ex_mq;
      double md = 0.0;  // thread 0's value is stored
      if constexpr (cert) {
        // FP32 values, FP64 decision: the FP32 evaluation differs from the FP64
        // one by at most ~20 u max|tile| (u = 2^-24, x/y/z passes of the
        // 4-point rule and the subtraction); where its maximum is farther than
        // 32 u max|tile| from eps the threshold decision (Sec. 2.3) is the
        // FP64 one, otherwise the block is evaluated again in FP64.
        const float mt = fmaxf(ex_mt, (float)mqt);
        const float E = 0x1p-19f * mt + 1e-37f;
        if (pv.norm_kind == 0 && certain_vs_eps(m0, E, td)) {
          if (threadIdx.x == 0) md = (double)m0;
        } else {
          md = pass(double(0), tv, std::false_type{});
        }
      } else {
        md = (double)m0;
      }
      if (threadIdx.x == 0) {
        const double mq = (double)mqt;
        pv.md[(int64_t)b.slot * nv + v] = md;
        pv.bmax[(int64_t)b.slot * nv + v] = mq;
        if (pv.norm_kind == 1) csv[v] = fmax(csv[v], mq);
      }
      __syncthreads();
    }
    if (plan_ok && pn < nact && threadIdx.x < PL::INTS) splan[buf ^ 1][threadIdx.x] = pre;
    if (__syncthreads_or(bad) && threadIdx.x == 0)
      pv.md[(int64_t)b.slot * nv] = __longlong_as_double(0x7ff8000000000000LL);
  }
  __syncthreads();
  if (pv.norm_kind == 1) flush_csv();
  if (threadIdx.x == 0 && ndet) atomicAdd(&pv.cnt->det_blocks, ndet);
}

// 2D details with one warp per block (single-variable fields without
// normalisation): the same evaluation as k_details, with warp-level
// synchronisation and reductions, for grids with many blocks.
template <int B, typename TS, typename TD, int NT>
struct DetW {
  using Bx = Box<2, B, 2>;
  using DG = DetGeo<2, B>;
  static constexpr int NW = NT / 32;
  static constexpr size_t GTAB = (4 * Bx::NPTS + 15) / 16 * 16;
  static constexpr size_t TABS = (4 * DetTab<B>::INTS + 15) / 16 * 16;  // detail index tables
  static constexpr size_t XB = sizeof(TS) * Bx::SCR > sizeof(TD) * DG::NX ? sizeof(TS) * Bx::SCR : sizeof(TD) * DG::NX;
  static constexpr size_t TB = (kRingBytesD<2> + sizeof(TS) * (Bx::TILE + Bx::CBOX) + 15) / 16 * 16;
  static constexpr size_t WAREA = TB + (XB + 15) / 16 * 16;
  static constexpr size_t SMEM = GTAB + TABS + NW * WAREA;
};

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
  for (int s = 16; s > 0; s >>= 1) v = fmax(v, (T)__shfl_xor_sync(0xffffffffu, v, s));
  return v;
}

template <int B, typename TS, typename TD, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_details_w(PoolView pv, TS* __restrict__ y) {
  pdl_enter();
  using Gm = Geo<2, B>;
  using Bx = Box<2, B, 2>;
  using DG = DetGeo<2, B>;
  using PL = Plan<2>;
  using DW = DetW<B, TS, TD, NT>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* sm = smem_as<unsigned char>(0);
  int32_t* gtab = reinterpret_cast<int32_t*>(sm);
  int32_t* xtab = reinterpret_cast<int32_t*>(sm + DW::GTAB);
  int32_t* otab = xtab + DG::NX;
  unsigned char* wa = sm + DW::GTAB + DW::TABS + warp * DW::WAREA;
  RingD<2>& R = *reinterpret_cast<RingD<2>*>(wa);
  TS* tile = reinterpret_cast<TS*>(wa + kRingBytesD<2>);
  TS* cbox = tile + Bx::TILE;
  TS* scr = reinterpret_cast<TS*>(wa + DW::TB);  // gather scratch, then the x pass
  __shared__ int64_t snbo[DW::NW][PL::NB];
  build_gtab<2, B, 2>(gtab);
  DetTab<B>::build(xtab, otab);
  __syncthreads();
  const int nact = pv.cnt->n_round;
  const bool all_blocks = pv.cnt->first_round != 0;
  const int prev = pv.cnt->round_id - 1;
  const bool plan_ok = pv.cnt->plan_topo == pv.cnt->topo;
  const int gw = blockIdx.x * DW::NW + warp, nwt = gridDim.x * DW::NW;
  unsigned ndet = 0;
  int32_t cur = (plan_ok && gw < nact && lane < PL::INTS) ? pv.plan[(int64_t)gw * PL::INTS + lane] : 0;
  for (int p = gw; p < nact; p += nwt) {
    const int pn = p + nwt;
    const int32_t nxt = (plan_ok && pn < nact && lane < PL::INTS) ? pv.plan[(int64_t)pn * PL::INTS + lane] : 0;
    BlockInfo b;
    int q;
    if (plan_ok) {
      b.slot = __shfl_sync(0xffffffffu, cur, 0);
      const int meta = __shfl_sync(0xffffffffu, cur, 1);
      b.lvl = meta & 255;
      b.tree = (meta >> 8) & 0xffff;
      b.c[0] = __shfl_sync(0xffffffffu, cur, 2);
      b.c[1] = __shfl_sync(0xffffffffu, cur, 3);
      b.c[2] = 0;
      const int32_t qq = __shfl_sync(0xffffffffu, cur, PL::NBO + (lane < PL::NB ? lane : 0));
      q = lane < PL::NB ? qq : b.slot;
    } else {
      b = load_block(pv, pv.act[p]);
      q = b.slot;
      if (lane < PL::NB && lane != 4) {
        const int64_t cn[3] = {b.c[0] + lane % 3 - 1, b.c[1] + lane / 3 - 1, 0};
        q = tab_get<2>(pv, pv.trees[b.tree], b.lvl, cn);
      }
    }
    const TreeDev& td = pv.trees[b.tree];
    const bool uni = __all_sync(0xffffffffu, q >= 0);
    bool ring = false;
    bool dirty = all_blocks;
    if (!all_blocks) {
      if (uni) {
        dirty = __any_sync(0xffffffffu, lane < PL::NB && pv.stamp[q] == prev);
      } else {
        build_ring<2, B, WarpGroup>(pv, td, b, R);
        __syncwarp();
        ring = true;
        dirty = __any_sync(0xffffffffu, lane < Gm::NR && R.slot[lane] >= 0 && pv.stamp[R.slot[lane]] == prev);
      }
    }
    if (dirty) {
      ++ndet;
      const int64_t own = (int64_t)b.slot * pv.vs;
      if (uni) {
        if (lane < PL::NB) snbo[warp][lane] = (int64_t)q * pv.vs;
        __syncwarp();
        gather_table<2, B, 2, 1, TS, TS, WarpGroup>(pv, own, snbo[warp], gtab, y, y, tile, true);
      } else {
        const bool ready = !ring && plan_ok && all_blocks;  // the stage plan's owner table
        if (ready) load_regions<2, WarpGroup>(pv, p, R);
        else if (!ring) build_ring<2, B, WarpGroup>(pv, td, b, R);
        __syncwarp();
        fill_tile<2, B, TS, TS, 2, WarpGroup>(pv, b, y, y, tile, true, R, cbox, scr, ready);
      }
      __syncwarp();
      // the x pass over the coarse rows, then the y pass and the detail at
      // each odd point, through the index tables (same operations as k_details)
      auto pass = [&](auto tag) -> decltype(tag) {
        using A = decltype(tag);
        A* XA = reinterpret_cast<A*>(scr);
        A md = DetTab<B>::template max_detail<A>(xtab, otab, tile, XA, WarpGroup{});
        md = warp_max(md);
        __syncwarp();
        return md;
      };
      // largest |value| over the interior (stored, and the NaN check) and, for
      // the certified FP32 evaluation, over the whole tile: one sweep, the
      // interior flag from the gather table
      constexpr bool cert = sizeof(TS) == 4 && sizeof(TD) == 8;
      TS mqs = TS(0), mts = TS(0);
      bool bad = false;
      for (int qn = lane; qn < Bx::TILE; qn += 32) {
        const TS sv = tile[qn];
        const TS av = (TS)fabs(sv);
        if (cert) mts = fmax(mts, av);
        if ((gtab[qn] >> 21) & 1) {
          mqs = fmax(mqs, av);
          bad |= !isfinite(sv);
        }
      }
      mqs = warp_max(mqs);
      double md = 0.0;  // lane 0's value is stored
      if constexpr (cert) {
        // as in k_details: FP32 evaluation, FP64 only within the rounding bound of eps
        const float m32 = pass(float(0));
        const float E = 0x1p-19f * warp_max((float)mts) + 1e-37f;
        if (certain_vs_eps(m32, E, td)) {
          if (lane == 0) md = (double)m32;
        } else {
          md = pass(double(0));
        }
      } else {
        md = (double)pass(TD(0));
      }
      if (__any_sync(0xffffffffu, bad)) md = __longlong_as_double(0x7ff8000000000000LL);
      if (lane == 0) {
        pv.md[b.slot] = md;
        pv.bmax[b.slot] = (double)mqs;
      }
      __syncwarp();
    }
    cur = nxt;
  }
  if (lane == 0 && ndet) atomicAdd(&pv.cnt->det_blocks, (unsigned long long)ndet);
}

// ---------------------------------------------------------------- coarsen ----
// Sec. 2.3: 2^d sisters with status -2 merge into their mother by restriction
// (every second node); a mother node on a line shared by two children is read
// from the child in which it has local index 0.  The mother takes the slot of
// the family member that comes first in Hilbert order.
// One kernel per round: each CTA merges families (the mother's data, then the
// family's table entries, light data and freed slots -- the family's 2^d
// members sit at consecutive list positions, a Hilbert-curve property), and
// the CTA that finishes last copies the new active list in place, updates the
// counters and prepares the next round (RoundCtl).
template <int D, int B, typename TS>
__global__ void __launch_bounds__(256) k_coarsen(PoolView pv, TS* __restrict__ y, RoundCtl rc) {
  pdl_enter();
  using Gm = Geo<D, B>;
  TS* buf = smem_as<TS>(0);
  __shared__ int cs[8];
  Counters* c = pv.cnt;
  const int nround = c->n_round, n_free = c->n_free, n_new = c->n_new, rid = c->round_id;
  const bool done = c->done != 0;
  const bool none = n_new == nround;  // no family merges: the tree and the list are unchanged
  const int nv = pv.nvar;
  for (int p = blockIdx.x; !none && p < nround; p += gridDim.x) {
    const int slot = pv.act[p];
    const int emit = pv.emit[2 * p], e = pv.eoff[2 * p];
    if (!emit) continue;  // a member of a family merged by the CTA of its first member
    if (threadIdx.x == 0) pv.act_next[e] = slot;
    if (pv.flag[slot] != -2) continue;
    const BlockInfo b = load_block(pv, slot);
    const TreeDev& td = pv.trees[b.tree];
    if (threadIdx.x < Gm::NCH) {
      int64_t cc[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) cc[a] = (b.c[a] & ~(int64_t)1) | ((threadIdx.x >> a) & 1);
      cs[threadIdx.x] = tab_get<D>(pv, td, b.lvl, cc);
    }
    __syncthreads();
    bool missing = false;
    for (int ch = 0; ch < Gm::NCH; ++ch) missing |= cs[ch] < 0;
    if (missing) {  // cannot happen for a complete family; never read slot -1
      if (threadIdx.x == 0) set_err(pv, kErrGraded);
      __syncthreads();
      continue;
    }
    for (int idx = threadIdx.x; idx < nv * Gm::NI; idx += blockDim.x) {
      const int v = idx / Gm::NI, q = idx % Gm::NI;
      const int I[3] = {q % B, (q / B) % B, D == 3 ? q / (B * B) : 0};
      int cb = 0, li[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) {
        const int bit = (2 * I[a] >= B - 1) ? 1 : 0;
        cb |= bit << a;
        li[a] = 2 * I[a] - bit * (B - 1);
      }
      buf[idx] = pool_at<D, B>(pv, y, cs[cb], v, li);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nv * Gm::NI; idx += blockDim.x) {
      const int v = idx / Gm::NI, q = idx % Gm::NI;
      y[((int64_t)slot * nv + v) * pv.vs + q] = buf[idx];
    }
    // the family's tables and light data (positions p .. p + 2^d - 1)
    if (threadIdx.x < Gm::NCH) {
      const int q = p + threadIdx.x;
      const int s = pv.act[q];
      const BlockInfo m = load_block(pv, s);
      pv.tab[td.tab_off[m.lvl] + (int64_t)morton<D>(m.c, m.lvl)] = -1;
      if (s == slot) {
        const int64_t pc[3] = {m.c[0] >> 1, m.c[1] >> 1, m.c[2] >> 1};
        pv.tab[td.tab_off[m.lvl - 1] + (int64_t)morton<D>(pc, m.lvl - 1)] = s;
        pv.stamp[s] = rid;
        pv.lvl[s] = (int8_t)(m.lvl - 1);
        const int32_t c32[3] = {(int32_t)pc[0], (int32_t)pc[1], (int32_t)pc[2]};
        for (int a = 0; a < 3; ++a) pv.crd[3 * s + a] = c32[a];
        pv.hkey[s] = block_key<D>(c32, m.lvl - 1, td.Jmax);
      } else {
        pv.lvl[s] = -1;
        pv.freelist[n_free + pv.eoff[2 * q + 1]] = s;
      }
    }
    __syncthreads();
  }
  if (last_cta_all(c)) {
    // the new list in place (every entry of act_next is written by now)
    const int ncopy = done || none ? 0 : n_new;
    for (int p = threadIdx.x; p < ncopy; p += blockDim.x) pv.act[p] = __ldcg(pv.act_next + p);
    if (threadIdx.x == 0) {
      c->first_round = 0;
      if (!done) {
        const int nch = 1 << D;
        c->merged = (c->n_act - n_new) / (nch - 1);
        c->n_free = n_free + c->n_alloc;
        c->n_act = n_new;
        if (c->merged == 0) c->done = 1;
        else c->topo += 1;
      }
      // the next round, if one runs (a family merged and fewer than max_rounds
      // ran): the blocks it evaluates, its id, its threshold scales (the last
      // round's stay for the next step's proposal features); in a captured
      // step the while node's condition
      c->rounds += 1;
      const bool next = !c->done && c->rounds < rc.max_rounds;
      c->n_round = c->done ? 0 : c->n_act;
      if (next) {
        c->round_id += 1;
        for (int i = 0; i < pv.ntrees * pv.nvar; ++i) pv.svar[i] = rc.svar_v;
      }
      if (rc.has_h) {
        c->graph_rounds += 1;
        cudaGraphSetConditional(rc.h, next ? 1u : 0u);
      }
      c->ctas_done = 0;
    }
  }
}

// --------------------------------------------------------------------- IC ----
// Analytic fields from per-lattice factor tables: Gaussian as the product of
// its 1D factors (x, then y, then z); mixing layer q = (1, u(y), v, E) with
// v = amp (s(x) e(y)), E = p0/(gamma-1) + (u u + v v)/2; double shear layer
// (Sec. 4) from its layer profile s(x) and u(y), in the RHS kind's variables.
template <int D, int B, typename TS>
__global__ void k_ic(PoolView pv, TS* __restrict__ y) {
  pdl_enter();
  using Gm = Geo<D, B>;
  const int nact = pv.cnt->n_act;
  const int nv = pv.nvar;
  for (int p = blockIdx.x; p < nact; p += gridDim.x) {
    const BlockInfo b = load_block(pv, pv.act[p]);
    const TreeDev& td = pv.trees[b.tree];
    const int sh = td.Jmax - b.lvl;
    const double* lat = pv.lat + td.lat_off;
    for (int q = threadIdx.x; q < Gm::NI; q += blockDim.x) {
      const int ijk[3] = {q % B, (q / B) % B, D == 3 ? q / (B * B) : 0};
      int64_t U[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) U[a] = pmod64((b.c[a] * (B - 1) + ijk[a]) << sh, td.N);
      const int64_t at = (int64_t)b.slot * nv * pv.vs + q;
      if (td.ic_kind == MR_IC_GAUSS) {
        double f = lat[kLatGx * td.N + U[0]] * lat[kLatGy * td.N + U[1]];
        if (D == 3) f = f * lat[kLatGz * td.N + U[2]];
        y[at] = (TS)f;
      } else if (td.ic_kind == MR_IC_MIXING) {
        const double u = lat[kLatNsU * td.N + U[1]];
        const double v = td.ic_amp * (lat[kLatNsS * td.N + U[0]] * lat[kLatNsE * td.N + U[1]]);
        const double E = td.ic_e0 + 0.5 * (u * u + v * v);
        y[at] = (TS)1.0;
        y[at + pv.vs] = (TS)u;
        y[at + 2 * pv.vs] = (TS)v;
        y[at + 3 * pv.vs] = (TS)E;
      } else if (td.ic_kind == MR_IC_SHEAR_LAYER) {
        const double s = lat[kLatSlS * td.N + U[0]];
        const double rho = td.ic_sl[1] + (td.ic_sl[0] - td.ic_sl[1]) * s;
        const double v = td.ic_sl[3] + (td.ic_sl[2] - td.ic_sl[3]) * s;
        const double u = lat[kLatSlU * td.N + U[1]];
        double q[4];
        if (pv.rhs_kind == MR_RHS_NS_SKEW) {
          const double f = sqrt(rho);
          q[0] = f; q[1] = f * u; q[2] = f * v; q[3] = td.ic_sl[4];
        } else {
          const double m1 = rho * u, m2 = rho * v;
          q[0] = rho; q[1] = m1; q[2] = m2; q[3] = td.ic_sl[4] / td.nsd[0] + 0.5 * (m1 * u + m2 * v);
        }
        for (int w = 0; w < 4; ++w) y[at + w * pv.vs] = (TS)q[w];
      }
    }
  }
}

// ------------------------------------------------------------- sync export ---
// Ghost synchronisation of the current field: commits the block-edge nodes
// taken from finer blocks; optionally writes the full tile (double) to `tiles`
// at the block's list position.
template <int D, int B, typename TS>
__global__ void __launch_bounds__(256) k_sync(PoolView pv, TS* __restrict__ y, double* __restrict__ tiles) {
  pdl_enter();
  using Gm = Geo<D, B>;
  RingD<D>& R = *smem_as<RingD<D>>(0);
  double* tile = smem_as<double>(kRingBytesD<D>);
  double* cbox = tile + pv.nvar * Gm::TILE;
  const int nact = pv.cnt->n_act;
  const int nv = pv.nvar;
  for (int p = blockIdx.x; p < nact; p += gridDim.x) {
    const BlockInfo b = load_block(pv, pv.act[p]);
    const TreeDev& td = pv.trees[b.tree];
    build_ring<D, B>(pv, td, b, R);
    __syncthreads();
    fill_tile<D, B, TS, double>(pv, b, y, y, tile, true, R, cbox);
    __syncthreads();
    if (tiles)
      for (int idx = threadIdx.x; idx < nv * Gm::TILE; idx += blockDim.x)
        tiles[(int64_t)p * nv * Gm::TILE + idx] = tile[idx];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- export -----
template <int D, int B, typename TS>
__global__ void k_export_fields(PoolView pv, const TS* __restrict__ y, double* __restrict__ out) {
  pdl_enter();
  using Gm = Geo<D, B>;
  const int nact = pv.cnt->n_act;
  const int nv = pv.nvar;
  for (int p = blockIdx.x; p < nact; p += gridDim.x) {
    const int slot = pv.act[p];
    for (int idx = threadIdx.x; idx < nv * Gm::NI; idx += blockDim.x) {
      const int v = idx / Gm::NI, q = idx % Gm::NI;
      out[(int64_t)p * nv * Gm::NI + idx] = (double)y[((int64_t)slot * nv + v) * pv.vs + q];
    }
  }
}

template <int D, int B, typename TS>
__global__ void k_import_fields(PoolView pv, TS* __restrict__ y, const double* __restrict__ in,
                                int64_t n) {
  pdl_enter();
  using Gm = Geo<D, B>;
  const int nv = pv.nvar;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int idx = threadIdx.x; idx < nv * Gm::NI; idx += blockDim.x) {
      const int v = idx / Gm::NI, q = idx % Gm::NI;
      y[(i * nv + v) * pv.vs + q] = (TS)in[i * nv * Gm::NI + idx];
    }
}

// ----------------------------------------------------------------- error -----
// Error against exact factor tables ex[3][N] of one tree over unique nodes
// (each block's last node per axis dropped), weights dx^d.
template <int D, int B, typename TS>
__global__ void k_error(PoolView pv, const TS* __restrict__ y, int tree, const double* ex,
                        double* out) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  const TreeDev& td = pv.trees[tree];
  constexpr int BZ = D == 3 ? B - 1 : 1;
  const int NU = (B - 1) * (B - 1) * BZ;
  double e2 = 0, x2 = 0, ei = 0, xi = 0;
  for (int p = blockIdx.x; p < nact; p += gridDim.x) {
    const BlockInfo b = load_block(pv, pv.act[p]);
    if (b.tree != tree) continue;
    const int sh = td.Jmax - b.lvl;
    const double dx = td.dx[b.lvl];
    const double w = D == 3 ? dx * dx * dx : dx * dx;
    for (int q = threadIdx.x; q < NU; q += blockDim.x) {
      const int ijk[3] = {q % (B - 1), (q / (B - 1)) % (B - 1), D == 3 ? q / ((B - 1) * (B - 1)) : 0};
      int64_t U[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) U[a] = pmod64((b.c[a] * (B - 1) + ijk[a]) << sh, td.N);
      double e = ex[U[0]] * ex[td.N + U[1]];
      if (D == 3) e = e * ex[2 * td.N + U[2]];
      const double a = (double)y[(int64_t)b.slot * pv.nvar * pv.vs + Geo<D, B>::lin(ijk[0], ijk[1], ijk[2])];
      e2 += w * (a - e) * (a - e);
      x2 += w * e * e;
      ei = fmax(ei, fabs(a - e));
      xi = fmax(xi, fabs(e));
    }
  }
  atomicAdd(&out[0], e2);
  atomicAdd(&out[1], x2);
  atomic_max_pos(&out[2], ei);
  atomic_max_pos(&out[3], xi);
}

// ------------------------------------------------------- tree maintenance ----
// SCAN: the CTA that finishes last also scans the counts (short lists), which
// saves the separate scan launch.
template <int D, bool SCAN>
__global__ void __launch_bounds__(256) k_refine_count(PoolView pv, int mode, const int8_t* mask) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  const int nch = 1 << D;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += gridDim.x * blockDim.x) {
    const int s = pv.act[p];
    const int l = pv.lvl[s];
    const TreeDev& td = pv.trees[pv.tree[s]];
    // mode 2: flags already set on the device (learned proposal + closure)
    const bool r = l < td.Jmax && (mode == MR_ADAPT_REFINE_ALL || (mode == 2 ? pv.flag[s] == 1 : (mask && mask[p] > 0)));
    pv.flag[s] = r ? 1 : 0;
    pv.emit[2 * p] = r ? nch : 1;
    pv.emit[2 * p + 1] = r ? nch : 0;
  }
  if constexpr (SCAN) {
    if (last_cta_all(pv.cnt)) {
      cta_scan2<256, 8>(pv.emit, pv.eoff, nact, &pv.cnt->n_new);
      if (threadIdx.x == 0) pv.cnt->ctas_done = 0;
    }
  }
}

// True in thread 0 of the CTA of the grid that finishes last; the writes of
// every other CTA of the grid are visible to it.
__device__ __forceinline__ bool last_cta(Counters* c) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&c->ctas_done, 1u) == gridDim.x - 1;
  __syncthreads();
  return last && threadIdx.x == 0;
}

// End of a refinement in one kernel: each refined mother's table entry is
// replaced by its children's and its slot freed, the new active list is copied
// in place (each index is read, then written, by one thread), and the counters
// are updated by the last CTA.
template <int D>
__global__ void k_refine_commit(PoolView pv) {
  pdl_enter();
  Counters* c = pv.cnt;
  const int nact = c->n_act, n_new = c->n_new, n_alloc = c->n_alloc, n_free = c->n_free;
  const bool ok = n_alloc <= n_free;
  const bool any = n_alloc > 0;  // some block refines (else the tree and the list are unchanged)
  const int nch = 1 << D;
  const int nmax = ok && any ? (nact > n_new ? nact : n_new) : 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nmax; p += gridDim.x * blockDim.x) {
    const int32_t nxt = p < n_new ? pv.act_next[p] : 0;
    if (p < nact) {
      const int s = pv.act[p];
      if (pv.flag[s] == 1) {
        const BlockInfo b = load_block(pv, s);
        const TreeDev& td = pv.trees[b.tree];
        pv.tab[td.tab_off[b.lvl] + (int64_t)morton<D>(b.c, b.lvl)] = -1;
        const int e = pv.eoff[2 * p];
        for (int r = 0; r < nch; ++r) {
          const int cs = pv.act_next[e + r];
          int64_t cc[3] = {pv.crd[3 * cs], pv.crd[3 * cs + 1], pv.crd[3 * cs + 2]};
          pv.tab[td.tab_off[b.lvl + 1] + (int64_t)morton<D>(cc, b.lvl + 1)] = cs;
        }
        pv.freelist[n_free - n_alloc + pv.eoff[2 * p + 1] / nch] = s;
        pv.lvl[s] = -1;
        pv.flag[s] = 0;
      }
    }
    if (p < n_new) pv.act[p] = nxt;
  }
  if (last_cta(c)) {
    if (ok && any) {
      c->n_free = n_free - n_alloc + n_alloc / nch;
      c->n_act = n_new;
      c->topo += 1;
    }
    c->ctas_done = 0;
  }
}

__device__ __forceinline__ bool same_family(const PoolView& pv, int s, int t) {
  if (pv.tree[s] != pv.tree[t] || pv.lvl[s] != pv.lvl[t]) return false;
  for (int a = 0; a < 3; ++a)
    if ((pv.crd[3 * s + a] >> 1) != (pv.crd[3 * t + a] >> 1)) return false;
  return true;
}

// Flags of one coarsening round (Sec. 2.3), one warp per block.  A block
// qualifies (-1) if its largest normalised detail is below eps (strict), it is
// above Jmin, all 2^d sisters are leaves, and no leaf one level finer touches
// it (gradedness after the merge).  A family coarsens (-2) only if all its
// sisters qualify (completeness); this is the fixpoint of the paper's -2
// assignment, reached here by evaluating the condition for the whole family.
// Also emits the new-list counts (first member of a merged family hosts the
// mother; other members free their slots).
template <int D, bool SCAN>
__global__ void __launch_bounds__(256) k_flags(PoolView pv) {
  pdl_enter();
  // A family (the 2^d sisters of a block) merges when every sister is a leaf
  // whose normalised detail is below eps, above Jmin, and no leaf one level
  // finer touches any sister: the cells of level l+1 around the family,
  // [-1, 4]^d relative to its lower corner minus the family itself (the
  // union of the sisters' rings).  One warp per block; the sister lookups,
  // their details and the ring lookups are spread over the lanes.
  constexpr int NS = 1 << D;
  constexpr int NBOX = D == 3 ? 6 * 6 * 6 : 6 * 6;  // [-1, 4]^d around a family
  const int nact = pv.cnt->n_round;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int nv = pv.nvar;
  for (int p = blockIdx.x * wpb + (threadIdx.x >> 5); p < nact; p += gridDim.x * wpb) {
    const int s = pv.act[p];
    const BlockInfo b = load_block(pv, s);
    const TreeDev& td = pv.trees[b.tree];
    int64_t fc[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) fc[a] = b.c[a] & ~(int64_t)1;
    // normalised detail m of leaf t (NaN if a variable's is) and m < eps
    auto detail = [&](int t, double& m) -> bool {
      if (pv.norm_kind == 0) {
        // unnormalised: a maximum of non-negative values (or NaN), taken and
        // compared with eps > 0 on their bit patterns, which order as the values
        long long mb = 0;
        bool nan = false;
        for (int v = 0; v < nv; ++v) {
          const long long x = __double_as_longlong(pv.md[(int64_t)t * nv + v]);
          nan |= (x & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
          mb = x > mb ? x : mb;
        }
        if (nan) mb = 0x7ff8000000000000LL;
        m = __longlong_as_double(mb);
        return !nan && mb < __double_as_longlong(td.eps);
      }
      bool nan = false;
      m = 0.0;
      for (int v = 0; v < nv; ++v) {
        double sv = pv.svar[b.tree * nv + v];
        if (sv == 0.0) sv = 1.0;
        const double mv = pv.md[(int64_t)t * nv + v];
        nan |= isnan(mv);
        m = fmax(m, mv / sv);
      }
      if (nan) m = __longlong_as_double(0x7ff8000000000000LL);
      return m < td.eps;
    };
    if (b.lvl <= td.Jmin) {
      // a family at Jmin never merges: only the block's own detail is recorded
      if (lane == 0) {
        double m;
        detail(s, m);
        pv.mdet[s] = m;
        if (isnan(m)) set_err(pv, kErrNaN);
        pv.flag[s] = 0;
        pv.emit[2 * p] = 1;
        pv.emit[2 * p + 1] = 0;
      }
      continue;
    }
    // sisters: exist as leaves and below eps
    bool ok = true;
    double mine = 0.0;
    if (lane < NS) {
      int64_t c[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) c[a] = fc[a] | ((lane >> a) & 1);
      const int t = tab_get<D>(pv, td, b.lvl, c);
      if (t < 0) {
        ok = false;
      } else {
        double m = 0.0;
        ok = detail(t, m);
        if (t == s) mine = m;
      }
    }
    // no finer leaf around the family: cells of [-1, 4]^d outside [0, 3]^d
    // (looked up only for a family whose members are all candidates)
    const bool sisters = __all_sync(0xffffffffu, ok);
    for (int u = lane; sisters && u < NBOX; u += 32) {
      const int q[3] = {u % 6 - 1, (u / 6) % 6 - 1, D == 3 ? u / 36 - 1 : 0};
      bool in = true;
      for (int a = 0; a < D; ++a) in &= q[a] >= 0 && q[a] <= 3;
      if (in) continue;
      int64_t cell[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) cell[a] = 2 * fc[a] + q[a];
      if (tab_get<D>(pv, td, b.lvl + 1, cell) >= 0) ok = false;
    }
    const bool all = __all_sync(0xffffffffu, ok) && b.lvl > td.Jmin;
    const double m = __shfl_sync(0xffffffffu, mine, (int)(((b.c[0] & 1) | (D > 1 ? (b.c[1] & 1) << 1 : 0) |
                                                          (D > 2 ? (b.c[2] & 1) << 2 : 0))));
    if (lane == 0) {
      pv.mdet[s] = m;
      if (isnan(m)) set_err(pv, kErrNaN);
      pv.flag[s] = all ? -2 : 0;
      const bool first = all && (p == 0 || !same_family(pv, s, pv.act[p - 1]));
      pv.emit[2 * p] = (!all || first) ? 1 : 0;
      pv.emit[2 * p + 1] = (all && !first) ? 1 : 0;
    }
  }
  // SCAN: the CTA that finishes last scans the new-list counts (short lists),
  // which saves the separate scan launch
  if constexpr (SCAN) {
    if (last_cta_all(pv.cnt)) {
      cta_scan2<256, 8>(pv.emit, pv.eoff, nact, &pv.cnt->n_new);
      if (threadIdx.x == 0) pv.cnt->ctas_done = 0;
    }
  }
}

// Neighbour table (Sec. 2.2): rel[r] = (sx, sy, sz, sub), see mr.h for the order.
template <int D>
__global__ void k_neighbors(PoolView pv, const int4* rel, int R, int32_t* nbr, int8_t* dl) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < (int64_t)nact * R;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(w / R), r = (int)(w % R);
    const BlockInfo b = load_block(pv, pv.act[p]);
    const TreeDev& td = pv.trees[b.tree];
    const int4 rr = rel[r];
    const int s[3] = {rr.x, rr.y, rr.z};
    int64_t k[3] = {0, 0, 0};
    bool corner = true;
    for (int a = 0; a < D; ++a) {
      k[a] = b.c[a] + s[a];
      corner &= s[a] != 0;
    }
    const int64_t n = (int64_t)1 << b.lvl;
    auto child = [&](int sub, int64_t ch[3]) {
      int z = 0;
      for (int a = 0; a < D; ++a) {
        int bit;
        if (s[a] != 0) bit = s[a] < 0 ? 1 : 0;
        else bit = (sub >> (z++)) & 1;
        ch[a] = 2 * pmod64(k[a], n) + bit;
      }
    };
    int found = -1, d = 0;
    if (rr.w < 0) {
      found = tab_get<D>(pv, td, b.lvl, k);
      if (found < 0) {
        int64_t pc[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) pc[a] = pmod64(k[a], n) >> 1;
        found = tab_get<D>(pv, td, b.lvl - 1, pc);
        d = -1;
        if (found < 0 && corner) {
          int64_t ch[3] = {0, 0, 0};
          child(0, ch);
          found = tab_get<D>(pv, td, b.lvl + 1, ch);
          d = 1;
        }
      }
    } else if (tab_get<D>(pv, td, b.lvl, k) < 0) {
      int64_t ch[3] = {0, 0, 0};
      child(rr.w, ch);
      found = tab_get<D>(pv, td, b.lvl + 1, ch);
      d = 1;
    }
    nbr[w] = found >= 0 ? pv.pos_of_slot[found] : -1;
    dl[w] = found >= 0 ? (int8_t)d : 0;
  }
}

template <int D>
__global__ void k_export_info(PoolView pv, mr_block_info* info, int8_t* flags, double* mdet) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += gridDim.x * blockDim.x) {
    const int s = pv.act[p];
    const BlockInfo b = load_block(pv, s);
    if (info) {
      mr_block_info o;
      o.level = b.lvl;
      o.tree = b.tree;
      o.treecode = morton<D>(b.c, b.lvl);
      for (int a = 0; a < 3; ++a) o.coords[a] = (int32_t)b.c[a];
      o.pad = 0;
      o.hilbert_key = pv.hkey[s];
      info[p] = o;
    }
    if (flags) flags[p] = pv.flag[s];
    if (mdet) mdet[p] = pv.mdet[s];
  }
}

// set_blocks: place input block i in slot i, validate, mark its finest cells.
template <int D>
__global__ void k_sb_place(PoolView pv, int64_t n, const int32_t* lvl, const int32_t* tree,
                           const int32_t* crd, int ntrees) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t = tree ? tree[i] : 0;
    if (t < 0 || t >= ntrees) { set_err(pv, kErrLayout); continue; }
    const TreeDev& td = pv.trees[t];
    const int l = lvl[i];
    if (l < td.Jmin || l > td.Jmax) { set_err(pv, kErrLayout); continue; }
    int32_t c32[3] = {0, 0, 0};
    int64_t c[3] = {0, 0, 0};
    bool bad = false;
    for (int a = 0; a < D; ++a) {
      c32[a] = crd[3 * i + a];
      c[a] = c32[a];
      bad |= c[a] < 0 || c[a] >= ((int64_t)1 << l);
    }
    if (bad) { set_err(pv, kErrLayout); continue; }
    pv.lvl[i] = (int8_t)l;
    pv.tree[i] = (int16_t)t;
    for (int a = 0; a < 3; ++a) pv.crd[3 * i + a] = c32[a];
    pv.hkey[i] = block_key<D>(c32, l, td.Jmax);
    pv.flag[i] = 0;
    pv.mdet[i] = 0.0;
    int* e = &pv.tab[td.tab_off[l] + (int64_t)morton<D>(c, l)];
    if (atomicCAS(e, -1, (int)i) != -1) set_err(pv, kErrLayout);
  }
}

// Every finest cell of every block gets +1 (coverage check: all must be 1).
template <int D>
__global__ void k_sb_cover(PoolView pv, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const int l = pv.lvl[i];
    if (l < 0) continue;
    const TreeDev& td = pv.trees[pv.tree[i]];
    const int sh = td.Jmax - l;
    const int64_t per = (int64_t)1 << (D * sh);
    for (int64_t r = threadIdx.x; r < per; r += blockDim.x) {
      int64_t cell[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) {
        int64_t off = 0;
        for (int bb = 0; bb < sh; ++bb) off |= ((r >> (bb * D + a)) & 1) << bb;
        cell[a] = ((int64_t)pv.crd[3 * i + a] << sh) + off;
      }
      atomicAdd(&pv.cells[2 * (td.cell_off + (int64_t)morton<D>(cell, td.Jmax))], 1);
    }
  }
}

template <int D>
__global__ void k_sb_mark(PoolView pv, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (pv.lvl[i] < 0) continue;
    const TreeDev& td = pv.trees[pv.tree[i]];
    pv.cells[2 * (td.cell_off + (int64_t)pv.hkey[i])] = 1;
  }
}

template <int D>
__global__ void k_sb_order(PoolView pv, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (pv.lvl[i] < 0) continue;
    const TreeDev& td = pv.trees[pv.tree[i]];
    pv.act[pv.eoff[2 * (td.cell_off + (int64_t)pv.hkey[i])]] = (int32_t)i;
  }
}

// Graded-tree check: every ring cell must be covered by a leaf at l-1..l+1.
template <int D>
__global__ void k_check_graded(PoolView pv) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += gridDim.x * blockDim.x) {
    const BlockInfo b = load_block(pv, pv.act[p]);
    const TreeDev& td = pv.trees[b.tree];
    constexpr int NR = D == 3 ? 64 : 16;
    for (int r = 0; r < NR; ++r) {
      const int q[3] = {r % 4 - 1, (r / 4) % 4 - 1, r / 16 - 1};
      const int64_t nl1 = (int64_t)1 << (b.lvl + 1);
      int64_t cell[3] = {0, 0, 0}, c1[3] = {0, 0, 0}, c2[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) {
        cell[a] = pmod64(2 * b.c[a] + q[a], nl1);
        c1[a] = cell[a] >> 1;
        c2[a] = cell[a] >> 2;
      }
      if (tab_get<D>(pv, td, b.lvl + 1, cell) < 0 && tab_get<D>(pv, td, b.lvl, c1) < 0 &&
          tab_get<D>(pv, td, b.lvl - 1, c2) < 0)
        set_err(pv, kErrGraded);
    }
  }
}

}  // namespace mr

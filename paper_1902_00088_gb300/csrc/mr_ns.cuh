// Navier-Stokes kernels of the double shear layer run (Sec. 4): the RK stage
// in the skew-symmetric form and the shock-capturing filter applied after each
// step.  Instantiated in mr_ns.cu.
#pragma once
#include "mr_kernels.cuh"

namespace mr {

// ------------------------------------------------ NS stage, skew form -------
// One RK4 stage of the 2D compressible Navier-Stokes equations in the
// skew-symmetric form of Reiss & Sesterhenn (2014), named in Sec. 4, on the
// square-root variables q = (phi, psi_x, psi_y, p), phi = sqrt(rho),
// psi = phi u (u = psi / phi, th = p / phi^2):
//   d phi/dt   = -1/2 sum_j (D_j psi_j + u_j D_j phi)
//   d psi_i/dt = -1/2 sum_j (D_j(psi_i u_j) + u_j D_j psi_i) - (D_i p - sum_j D_j tau_ij) / phi
//   d p/dt     = -gamma sum_j D_j(p u_j) + (gamma - 1) sum_j u_j D_j p
//                + (gamma - 1) (sum_ij tau_ij D_j u_i + sum_j D_j(kap D_j th)),
// tau_xx = mu (2 u_x - 2/3 div), tau_yy = mu (2 v_y - 2/3 div), tau_xy = mu (u_y + v_x),
// kap = mu gamma / ((gamma - 1) Pr); D is the 4th-order central D1 everywhere.
// The stresses and kap D th are formed on the arms of the interior that their
// second derivative reads (x-arm: i in [-2, B+1] on rows 0..B-1; y-arm: the
// transpose), then every interior node evaluates its four rates at once and
// applies the 3-register RK update of the advection stage; with
// StageArgs::copy_state the last stage also stores the new state in the stage
// type into ynext (the shock filter's source).
template <int B>
struct NssGeo {
  static constexpr int NX = (B + 4) * B;  // x-arm
  static constexpr int NY = B * (B + 4);  // y-arm
};

// Threads per CTA and the CTAs per SM the registers are budgeted for: 17^2
// blocks run 6 CTAs of 4 warps per SM (measured on the double shear layer:
// 193 us per stage launch against 198 for 5 x 160, 202 for 4 x 192, 232 for
// 3 x 256, 258 for 2 x 320 threads).
template <int B>
struct NssCfg {
  static constexpr int NT = B == 17 ? 128 : 256;
  static constexpr int MINB = B == 17 ? 6 : 3;
};

template <int B, typename TY>
constexpr size_t nss_smem() {
  using Gm = Geo<2, B>;
  return kRingBytesD<2> + sizeof(TY) * (4 * Gm::TILE + 4 * Gm::CBOX + 3 * Gm::TILE + 3 * NssGeo<B>::NX +
                                        3 * NssGeo<B>::NY);
}

template <int B, typename TS, typename TY, typename TSRC>
__global__ void __launch_bounds__(NssCfg<B>::NT, NssCfg<B>::MINB) k_stage_nss(PoolView pv, const TSRC* __restrict__ src,
                                                   TS* __restrict__ y, TS* __restrict__ acc,
                                                   TY* __restrict__ ynext, TY* __restrict__ yn, int stage,
                                                   StageArgs sa) {
  pdl_enter();
  using Gm = Geo<2, B>;
  using NG = NssGeo<B>;
  using TC = TY;
  constexpr int T = Gm::T, G = Gm::G;
  RingD<2>& R = *smem_as<RingD<2>>(0);
  TC* tile = smem_as<TC>(kRingBytesD<2>);  // phi, psi_x, psi_y, p: 4 x TILE
  TC* cbox = tile + 4 * Gm::TILE;         // 4 x CBOX
  TC* pu = cbox + 4 * Gm::CBOX;           // u, v, th on the tile
  TC* pw = pu + Gm::TILE;
  TC* pth = pw + Gm::TILE;
  TC* ax = pth + Gm::TILE;                // x-arm: tau_xx, tau_xy, kap th_x
  TC* ay = ax + 3 * NG::NX;               // y-arm: tau_xy, tau_yy, kap th_y
  static_assert(Box<2, B, kG>::SCR <= 3 * Gm::TILE, "prediction scratch fits in the primitive arrays");
  using PL = Plan<2>;
  __shared__ int32_t splan[2][PL::INTS];
  const int nact = pv.cnt->n_act;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&pv.cnt->stage_blocks, (unsigned long long)nact);
  auto I = [&](int i, int j) { return (j + G) * T + (i + G); };
  auto xI = [&](int i, int j) { return j * (B + 4) + (i + 2); };
  auto yI = [&](int i, int j) { return (j + 2) * B + i; };
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
      fill_tile<2, B, TSRC, TC>(pv, b, src, (TSRC*)src, tile, stage == 0, R, cbox, pu, true);
    }
    __syncthreads();
    TC gm1, mu, kap, gam;
    if constexpr (sizeof(TC) == 4) { gm1 = td.nsf[0]; mu = td.nsf[1]; kap = td.nsf[2]; gam = td.nsf[3]; }
    else { gm1 = td.nsd[0]; mu = td.nsd[1]; kap = td.nsd[2]; gam = td.nsd[3]; }
    const TC c23 = (TC)(2.0 / 3.0);
    const TC c = tree_cD<TC>(td, b.lvl);
    const TC* ph = tile;
    const TC* sx = tile + Gm::TILE;
    const TC* sy = tile + 2 * Gm::TILE;
    const TC* pr = tile + 3 * Gm::TILE;
    for (int idx = threadIdx.x; idx < Gm::TILE; idx += blockDim.x) {
      const TC f = ph[idx];
      if constexpr (sizeof(TC) == 4) {
        // FP32 stages: one reciprocal instead of three divisions
        const TC rf = TC(1) / f;
        pu[idx] = sx[idx] * rf;
        pw[idx] = sy[idx] * rf;
        pth[idx] = (pr[idx] * rf) * rf;
      } else {
        pu[idx] = sx[idx] / f;
        pw[idx] = sy[idx] / f;
        pth[idx] = pr[idx] / (f * f);
      }
    }
    __syncthreads();
    auto dx = [&](const TC* f, int i, int j) {
      return ((f[I(i - 2, j)] - f[I(i + 2, j)]) + TC(8) * (f[I(i + 1, j)] - f[I(i - 1, j)])) * c;
    };
    auto dy = [&](const TC* f, int i, int j) {
      return ((f[I(i, j - 2)] - f[I(i, j + 2)]) + TC(8) * (f[I(i, j + 1)] - f[I(i, j - 1)])) * c;
    };
    // D1 of the product of two tile arrays
    auto dxm = [&](const TC* a, const TC* g, int i, int j) {
      auto m = [&](int s) { return a[I(i + s, j)] * g[I(i + s, j)]; };
      return ((m(-2) - m(2)) + TC(8) * (m(1) - m(-1))) * c;
    };
    auto dym = [&](const TC* a, const TC* g, int i, int j) {
      auto m = [&](int s) { return a[I(i, j + s)] * g[I(i, j + s)]; };
      return ((m(-2) - m(2)) + TC(8) * (m(1) - m(-1))) * c;
    };
    auto dxa = [&](const TC* a, int i, int j) {
      return ((a[xI(i - 2, j)] - a[xI(i + 2, j)]) + TC(8) * (a[xI(i + 1, j)] - a[xI(i - 1, j)])) * c;
    };
    auto dya = [&](const TC* a, int i, int j) {
      return ((a[yI(i, j - 2)] - a[yI(i, j + 2)]) + TC(8) * (a[yI(i, j + 1)] - a[yI(i, j - 1)])) * c;
    };
    constexpr int W = B + 4;
    for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
      const int i = idx % W - 2, j = idx / W - 2;
      const bool needX = j >= 0 && j < B, needY = i >= 0 && i < B;
      if (!needX && !needY) continue;
      const TC ux = dx(pu, i, j), vx = dx(pw, i, j), uy = dy(pu, i, j), vy = dy(pw, i, j);
      const TC div = ux + vy;
      const TC txy = mu * (uy + vx);
      if (needX) {
        const int o = xI(i, j);
        ax[o] = mu * (TC(2) * ux - c23 * div);
        ax[NG::NX + o] = txy;
        ax[2 * NG::NX + o] = kap * dx(pth, i, j);
      }
      if (needY) {
        const int o = yI(i, j);
        ay[o] = txy;
        ay[NG::NY + o] = mu * (TC(2) * vy - c23 * div);
        ay[2 * NG::NY + o] = kap * dy(pth, i, j);
      }
    }
    __syncthreads();
    const StageCoef<TS> cs(pv, sa, b.tree, stage);
    const StageCoef<TC> cf(pv, sa, b.tree, stage);
    const int64_t base = (int64_t)b.slot * 4 * pv.vs;
    constexpr bool MIX = sizeof(TS) == 8 && sizeof(TC) == 4;
    for (int q = threadIdx.x; q < Gm::NI; q += blockDim.x) {
      const int i = q % B, j = q / B;
      const int t0 = I(i, j);
      // FP64 state, FP32 stages: the next stage field needs y_n only in FP32;
      // stage 0 takes it from the tile (the committed state, rounded) and keeps
      // it in yn for stages 1 and 2, which then read no FP64 state
      TS yv[4], av[4];
      TC yf[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int64_t at = base + (int64_t)v * pv.vs + q;
        yv[v] = (stage == 0 || (!MIX && stage <= 2)) ? y[at] : TS(0);
        av[v] = stage >= 1 ? acc[at] : TS(0);
        if constexpr (MIX) {
          if (stage == 0) yf[v] = tile[v * Gm::TILE + t0];
          else if (stage <= 2) yf[v] = yn[at];
        }
      }
      const TC uu = pu[t0], vv = pw[t0], f = ph[t0];
      if constexpr (MIX) {
        if (stage == 0)
#pragma unroll
          for (int v = 0; v < 4; ++v) yn[base + (int64_t)v * pv.vs + q] = yf[v];
      }
      const TC phx = dx(ph, i, j), phy = dy(ph, i, j);
      const TC sxx = dx(sx, i, j), sxy = dy(sx, i, j), syx = dx(sy, i, j), syy = dy(sy, i, j);
      const TC px = dx(pr, i, j), py = dy(pr, i, j);
      const TC ux = dx(pu, i, j), vx = dx(pw, i, j), uy = dy(pu, i, j), vy = dy(pw, i, j);
      TC k[4];
      // mass
      k[0] = TC(-0.5) * ((sxx + uu * phx) + (syy + vv * phy));
      // momentum
      const TC cx = (dxm(sx, pu, i, j) + uu * sxx) + (dym(sx, pw, i, j) + vv * sxy);
      const TC cy = (dxm(sy, pu, i, j) + uu * syx) + (dym(sy, pw, i, j) + vv * syy);
      const TC fx = px - (dxa(ax, i, j) + dya(ay, i, j));
      const TC fy = py - (dxa(ax + NG::NX, i, j) + dya(ay + NG::NY, i, j));
      if constexpr (sizeof(TC) == 4) {
        const TC rf = TC(1) / f;
        k[1] = TC(-0.5) * cx - fx * rf;
        k[2] = TC(-0.5) * cy - fy * rf;
      } else {
        k[1] = TC(-0.5) * cx - fx / f;
        k[2] = TC(-0.5) * cy - fy / f;
      }
      // pressure
      const TC phiv = (ax[xI(i, j)] * ux + ax[NG::NX + xI(i, j)] * (uy + vx)) + ay[NG::NY + yI(i, j)] * vy;
      const TC heat = dxa(ax + 2 * NG::NX, i, j) + dya(ay + 2 * NG::NY, i, j);
      k[3] = (-gam * (dxm(pr, pu, i, j) + dym(pr, pw, i, j)) + gm1 * (uu * px + vv * py)) + gm1 * (phiv + heat);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int64_t at = base + (int64_t)v * pv.vs + q;
        if constexpr (sizeof(TS) == 8 && sizeof(TC) == 4) {
          // FP64 state, FP32 stages: increments dt k in FP32, accumulated in FP64
          const TC kc = k[v];
          if (stage == 0) {
            acc[at] = yv[v] + (TS)(cf.ca * kc);
            ynext[at] = (TY)(yf[v] + cf.cy * kc);
          } else if (stage == 1 || stage == 2) {
            acc[at] = av[v] + (TS)(cf.ca * kc);
            ynext[at] = (TY)(yf[v] + cf.cy * kc);
          } else {
            const TS yn = av[v] + (TS)(cf.ca * kc);
            y[at] = yn;
            if (sa.copy_state) ynext[at] = (TY)yn;
          }
        } else {
          const TS kk = (TS)k[v];
          if (stage == 0) {
            acc[at] = yv[v] + cs.ca * kk;
            ynext[at] = (TY)(yv[v] + cs.cy * kk);
          } else if (stage == 1 || stage == 2) {
            acc[at] = av[v] + cs.ca * kk;
            ynext[at] = (TY)(yv[v] + cs.cy * kk);
          } else {
            const TS yn = av[v] + cs.ca * kk;
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

// ------------------------------------------------------- shock filter -------
// Shock-capturing filter of Bogey, de Cacqueray & Bailly (2009), applied after
// every time step in Sec. 4 (threshold r_th of the block's tree), in place on
// the state y.  The synchronised tiles are gathered from `ys`, a copy of the
// state in the stage type that no CTA writes meanwhile (the last RK stage
// stores it), so every CTA updates its own block's interior in y while the
// others read their ghosts.  Per direction a, node n:
//   th_n = (u_{n+1} - u_{n-1}) / (2 dx) + (v_{n+1} - v_{n-1}) / (2 dx)  (each along its axis)
//   Dth_n = (-th_{n+1} + 2 th_n - th_{n-1}) / 4
//   M_n = ((Dth_n - Dth_{n+1})^2 + (Dth_n - Dth_{n-1})^2) / 2
//   r_n = M_n / (c_n^2 / dx^2) + 1e-16,  c^2 = gamma p / rho
//   s_n = (1 - r_th / r_n + |1 - r_th / r_n|) / 2
//   q_n <- q_n - sum_a (s_{n+1/2} F_{n+1/2} - s_{n-1/2} F_{n-1/2}),
//   F_{n+1/2} = -(q_{n+1} - q_n) / 4, s_{n+1/2} = (s_n + s_{n+1}) / 2,
// both directions from the unfiltered tile.  The stencil reaches four nodes
// along a and one across.  Everything is evaluated in TC.  With TS = TC every
// interior node becomes its synchronised value minus the increment (as in
// the oracle); with an FP64 state and FP32 arithmetic the FP32 increment is
// subtracted from the FP64 state where it is not zero (block-edge nodes owned
// by a finer neighbour keep their own value until the next synchronisation
// replaces it by the owner's, as after every RK stage).
// KIND: MR_RHS_NS (q = rho, rho u, rho v, E) or MR_RHS_NS_SKEW (phi, psi, p).
template <int B, typename TC>
constexpr size_t filter_smem() {
  using Gm = Geo<2, B>;
  return kRingBytesD<2> + sizeof(TC) * (4 * Gm::TILE + 4 * Gm::CBOX + 4 * Gm::TILE + 2 * (B + 2) * B);
}

// 160 threads, 5 CTAs per SM (measured 139 us against 145 for 256 and 156 for
// 128 threads per CTA on the double shear layer)
constexpr int kFilterThreads = 160;

template <int B, typename TS, typename TC, int KIND>
__global__ void __launch_bounds__(kFilterThreads, 5) k_filter(PoolView pv, const TC* __restrict__ ys, TS* __restrict__ y) {
  pdl_enter();
  using Gm = Geo<2, B>;
  constexpr int T = Gm::T, G = Gm::G;
  constexpr bool MIX = sizeof(TS) != sizeof(TC);
  RingD<2>& R = *smem_as<RingD<2>>(0);
  TC* tile = smem_as<TC>(kRingBytesD<2>);
  TC* cbox = tile + 4 * Gm::TILE;
  TC* pu = cbox + 4 * Gm::CBOX;  // u, v, c^2, dilatation on the tile
  TC* pw = pu + Gm::TILE;
  TC* pc = pw + Gm::TILE;
  TC* th = pc + Gm::TILE;
  TC* sgx = th + Gm::TILE;       // s at i in [-1, B], j in [0, B-1]
  TC* sgy = sgx + (B + 2) * B;   // s at i in [0, B-1], j in [-1, B]
  static_assert(Box<2, B, kG>::SCR <= 4 * Gm::TILE, "prediction scratch fits in the primitive arrays");
  using PL = Plan<2>;
  __shared__ int32_t splan[PL::INTS];
  const int nact = pv.cnt->n_act;
  auto I = [&](int i, int j) { return (j + G) * T + (i + G); };
  for (int p = blockIdx.x; p < nact; p += gridDim.x) {
    if (threadIdx.x < PL::INTS) splan[threadIdx.x] = pv.plan[(int64_t)p * PL::INTS + threadIdx.x];
    __syncthreads();
    const BlockInfo b = plan_block<2>(splan);
    const TreeDev& td = pv.trees[b.tree];
    const int64_t base = (int64_t)b.slot * 4 * pv.vs;
    if (!(td.rth > 0.0)) {  // no filter on this tree
      __syncthreads();
      continue;
    }
    if ((splan[1] >> 30) & 1) {
      gather_uniform<2, B, kG, 4, TC, TC>(pv, b, splan + PL::NBO, ys, (TC*)ys, tile, false);
    } else {
      load_regions<2, CtaGroup>(pv, p, R);
      __syncthreads();
      fill_tile<2, B, TC, TC>(pv, b, ys, (TC*)ys, tile, false, R, cbox, pu, true);
    }
    __syncthreads();
    TC gm1, gam, rth, h2, dx2;
    if constexpr (sizeof(TC) == 4) {
      gm1 = td.nsf[0]; gam = td.nsf[3]; rth = td.rthf; h2 = td.fh2[b.lvl]; dx2 = td.fdx2[b.lvl];
    } else {
      const double dxl = td.dx[b.lvl];
      gm1 = td.nsd[0]; gam = td.nsd[3]; rth = td.rth; h2 = 0.5 / dxl; dx2 = dxl * dxl;
    }
    for (int idx = threadIdx.x; idx < Gm::TILE; idx += blockDim.x) {
      const TC q0 = tile[idx], q1 = tile[Gm::TILE + idx], q2 = tile[2 * Gm::TILE + idx], q3 = tile[3 * Gm::TILE + idx];
      const TC u = q1 / q0, v = q2 / q0;
      TC rho, pp;
      if constexpr (KIND == MR_RHS_NS) {
        rho = q0;
        pp = gm1 * (q3 - TC(0.5) * (q1 * u + q2 * v));
      } else {
        rho = q0 * q0;
        pp = q3;
      }
      pu[idx] = u;
      pw[idx] = v;
      pc[idx] = gam * pp / rho;
    }
    __syncthreads();
    // dilatation on [-3, B+2]^2 (only the cross of the interior is read)
    constexpr int W3 = B + 6;
    for (int idx = threadIdx.x; idx < W3 * W3; idx += blockDim.x) {
      const int i = idx % W3 - 3, j = idx / W3 - 3;
      th[I(i, j)] = (pu[I(i + 1, j)] - pu[I(i - 1, j)]) * h2 + (pw[I(i, j + 1)] - pw[I(i, j - 1)]) * h2;
    }
    __syncthreads();
    // strengths: x-arm then y-arm, (B+2) B nodes each
    for (int idx = threadIdx.x; idx < 2 * (B + 2) * B; idx += blockDim.x) {
      const int ax = idx < (B + 2) * B ? 0 : 1;
      const int e = idx - ax * (B + 2) * B;
      const int i = ax == 0 ? e % (B + 2) - 1 : e % B;
      const int j = ax == 0 ? e / (B + 2) : e / B - 1;
      const int ox = ax == 0 ? 1 : 0, oy = 1 - ox;
      auto Dth = [&](int s) {
        const int ii = i + s * ox, jj = j + s * oy;
        return (-th[I(ii + ox, jj + oy)] + TC(2) * th[I(ii, jj)] - th[I(ii - ox, jj - oy)]) / TC(4);
      };
      const TC d0 = Dth(0), dp = Dth(1), dm = Dth(-1);
      const TC M = TC(0.5) * ((d0 - dp) * (d0 - dp) + (d0 - dm) * (d0 - dm));
      const TC r = M / (pc[I(i, j)] / dx2) + TC(1e-16);
      const TC z = TC(1) - rth / r;
      (ax == 0 ? sgx : sgy)[e] = TC(0.5) * (z + (z < TC(0) ? -z : z));
    }
    __syncthreads();
    auto sX = [&](int i, int j) { return sgx[j * (B + 2) + (i + 1)]; };
    auto sY = [&](int i, int j) { return sgy[(j + 1) * B + i]; };
    for (int idx = threadIdx.x; idx < 4 * Gm::NI; idx += blockDim.x) {
      const int v = idx / Gm::NI, q = idx % Gm::NI;
      const int i = q % B, j = q / B;
      const int64_t at = base + (int64_t)v * pv.vs + q;
      const TC* tv = tile + v * Gm::TILE;
      const TC sxp = TC(0.5) * (sX(i, j) + sX(i + 1, j));
      const TC sxm = TC(0.5) * (sX(i - 1, j) + sX(i, j));
      const TC syp = TC(0.5) * (sY(i, j) + sY(i, j + 1));
      const TC sym = TC(0.5) * (sY(i, j - 1) + sY(i, j));
      const TC q0 = tv[I(i, j)];
      const TC fxp = TC(-0.25) * (tv[I(i + 1, j)] - q0), fxm = TC(-0.25) * (q0 - tv[I(i - 1, j)]);
      const TC fyp = TC(-0.25) * (tv[I(i, j + 1)] - q0), fym = TC(-0.25) * (q0 - tv[I(i, j - 1)]);
      const TC ddx = sxp * fxp - sxm * fxm;
      const TC ddy = syp * fyp - sym * fym;
      if constexpr (MIX) {
        const TC d = ddx + ddy;
        if (d != TC(0)) y[at] = y[at] - (TS)d;
      } else {
        y[at] = q0 - (ddx + ddy);
      }
    }
    __syncthreads();
  }
}

// Copies the interiors (nvar x vs values) of every active block from the state
// y to `to` in the stage type (the filter's source when it runs outside a step).
template <typename TS, typename TC>
__global__ void k_state_copy(PoolView pv, const TS* __restrict__ y, TC* __restrict__ to) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  const int64_t per = (int64_t)pv.nvar * pv.vs;
  const int64_t n = (int64_t)nact * per;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(k / per);
    const int64_t at = (int64_t)pv.act[p] * per + (k - (int64_t)p * per);
    to[at] = (TC)y[at];
  }
}

}  // namespace mr

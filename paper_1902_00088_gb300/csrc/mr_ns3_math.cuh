// Node arithmetic of compressible Navier-Stokes in three dimensions (the
// equations of Sec. 4 with the index sums over x, y, z; Sec. 5 names 3D as the
// next step), for a block's synchronised tile, in both forms:
//   flux form        q = (rho, rho u, rho v, rho w, E),   N(q) = -sum_a D_a F_a,
//                    F_a = (rho u_a, rho u_a u_b + p delta_ab - tau_ab,
//                           (E + p) u_a - sum_b u_b tau_ab - kap D_a th);
//   skew-symmetric   q = (phi, psi_x, psi_y, psi_z, p), phi = sqrt(rho), psi = phi u,
//                    N_phi   = -1/2 sum_j (D_j psi_j + u_j D_j phi),
//                    N_psi_i = -1/2 sum_j (D_j(psi_i u_j) + u_j D_j psi_i)
//                              - (D_i p - sum_j D_j tau_ij) / phi,
//                    N_p     = -gamma sum_j D_j(p u_j) + (gamma - 1) sum_j u_j D_j p
//                              + (gamma - 1) (Phi + sum_j D_j(kap D_j th)),
// tau_ab = mu (D_b u_a + D_a u_b) - (2/3) mu div delta_ab, Phi = sum_ij tau_ij D_j u_i,
// th = p / rho, kap = mu gamma / ((gamma - 1) Pr), D the 4th-order central first
// derivative ((f[-2] - f[2]) + 8 (f[1] - f[-1])) / (12 dx).
//
// The functions take accessors (callables (i, j, k) -> value) so that a kernel
// can read shared-memory slabs, registers or global scratch.  Three phases per
// block: primitives on every tile node (ghost width 4), stresses, fluxes and
// heat fluxes on nodes -2..B+1 per axis, right-hand side on the interior.
// Every sum over axes or components is evaluated as ((x + y) + z); with FP64
// operands and no contraction of products into fused multiply-adds the results
// are those of a plain IEEE evaluation in this order.  Compiles as device code
// (nvcc) and as host code (a C++17 compiler), so that the arithmetic can be
// checked on the CPU.
#pragma once

#if defined(__CUDACC__)
#define MR_NS3_HD __host__ __device__ __forceinline__
#else
#define MR_NS3_HD inline
#endif

namespace mr {
namespace ns3 {

// 4th-order D1 along axis a (0 x, 1 y, 2 z) of accessor f at node (i, j, k).
template <typename T, typename F>
MR_NS3_HD T d1(const F& f, int a, int i, int j, int k, T c) {
  const int o0 = a == 0, o1 = a == 1, o2 = a == 2;
  return ((f(i - 2 * o0, j - 2 * o1, k - 2 * o2) - f(i + 2 * o0, j + 2 * o1, k + 2 * o2)) +
          T(8) * (f(i + o0, j + o1, k + o2) - f(i - o0, j - o1, k - o2))) *
         c;
}

// D1 along axis a of the node-wise product f h.
template <typename T, typename F, typename H>
MR_NS3_HD T d1m(const F& f, const H& h, int a, int i, int j, int k, T c) {
  const int o0 = a == 0, o1 = a == 1, o2 = a == 2;
  auto m = [&](int s) { return f(i + s * o0, j + s * o1, k + s * o2) * h(i + s * o0, j + s * o1, k + s * o2); };
  return ((m(-2) - m(2)) + T(8) * (m(1) - m(-1))) * c;
}

// Primitives of a node, flux form: velocity, pressure, th = p / rho.
template <typename T>
MR_NS3_HD void prim_flux(T gam, const T q[5], T vel[3], T& p, T& th) {
  const T r = q[0];
  vel[0] = q[1] / r;
  vel[1] = q[2] / r;
  vel[2] = q[3] / r;
  p = (gam - T(1)) * (q[4] - T(0.5) * ((q[1] * vel[0] + q[2] * vel[1]) + q[3] * vel[2]));
  th = p / r;
}

// Primitives of a node, skew-symmetric form: velocity psi / phi, th = p / phi^2.
template <typename T>
MR_NS3_HD void prim_skew(const T q[5], T vel[3], T& th) {
  const T f = q[0];
  vel[0] = q[1] / f;
  vel[1] = q[2] / f;
  vel[2] = q[3] / f;
  th = q[4] / (f * f);
}

// Velocity gradient du[a][e] = D_e u_a and stress tau at a node from the three
// velocity accessors.
template <typename T, typename V>
MR_NS3_HD void stress(const V* vel, int i, int j, int k, T c, T mu, T du[3][3], T tau[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int e = 0; e < 3; ++e) du[a][e] = d1<T>(vel[a], e, i, j, k, c);
  const T div = (du[0][0] + du[1][1]) + du[2][2];
  for (int a = 0; a < 3; ++a)
    for (int e = 0; e < 3; ++e)
      tau[a][e] = a == e ? mu * (T(2) * du[a][a] - (T(2) / T(3)) * div) : mu * (du[a][e] + du[e][a]);
}

// Flux form: the fluxes F_a (a = 0, 1, 2; five components each) at a node from
// the state q of the node, its primitives, its stress and the D_a th of the
// heat flux (thd[a]).
template <typename T>
MR_NS3_HD void fluxes(const T q[5], const T vel[3], T p, const T tau[3][3], const T thd[3], T kap, T F[3][5]) {
  for (int a = 0; a < 3; ++a) {
    F[a][0] = q[1 + a];
    for (int e = 0; e < 3; ++e)
      F[a][1 + e] = a == e ? (q[1 + a] * vel[e] + p) - tau[a][e] : q[1 + a] * vel[e] - tau[a][e];
    const T work = (vel[0] * tau[a][0] + vel[1] * tau[a][1]) + vel[2] * tau[a][2];
    F[a][4] = ((q[4] + p) * vel[a] - work) - kap * thd[a];
  }
}

// Flux form right-hand side of variable v at an interior node: Fa(v, a) returns
// the accessor of component v of F_a.
template <typename T, typename FA>
MR_NS3_HD T rhs_flux(const FA& Fa, int v, int i, int j, int k, T c) {
  return -((d1<T>(Fa(v, 0), 0, i, j, k, c) + d1<T>(Fa(v, 1), 1, i, j, k, c)) + d1<T>(Fa(v, 2), 2, i, j, k, c));
}

// Skew-symmetric right-hand side at an interior node.  Accessors: ph (phi),
// ps[3] (psi), pr (p), vel[3], tau(a, e) and qh[3] (kap D_a th) on nodes
// -2..B+1.  out[5] = (N_phi, N_psi_x, N_psi_y, N_psi_z, N_p).
template <typename T, typename A, typename TA>
MR_NS3_HD void rhs_skew(const A& ph, const A* ps, const A& pr, const A* vel, const TA& tau, const A* qh, int i,
                        int j, int k, T c, T gam, T out[5]) {
  const T gm1 = gam - T(1);
  const T f = ph(i, j, k), u[3] = {vel[0](i, j, k), vel[1](i, j, k), vel[2](i, j, k)};
  T dph[3], dp[3], ds[3][3], du[3][3];
  for (int a = 0; a < 3; ++a) {
    dph[a] = d1<T>(ph, a, i, j, k, c);
    dp[a] = d1<T>(pr, a, i, j, k, c);
    for (int e = 0; e < 3; ++e) {
      ds[a][e] = d1<T>(ps[a], e, i, j, k, c);
      du[a][e] = d1<T>(vel[a], e, i, j, k, c);
    }
  }
  out[0] = T(-0.5) * (((ds[0][0] + u[0] * dph[0]) + (ds[1][1] + u[1] * dph[1])) + (ds[2][2] + u[2] * dph[2]));
  for (int a = 0; a < 3; ++a) {
    const T conv = ((d1m<T>(ps[a], vel[0], 0, i, j, k, c) + u[0] * ds[a][0]) +
                    (d1m<T>(ps[a], vel[1], 1, i, j, k, c) + u[1] * ds[a][1])) +
                   (d1m<T>(ps[a], vel[2], 2, i, j, k, c) + u[2] * ds[a][2]);
    const T visc = (d1<T>(tau(a, 0), 0, i, j, k, c) + d1<T>(tau(a, 1), 1, i, j, k, c)) +
                   d1<T>(tau(a, 2), 2, i, j, k, c);
    const T fa = dp[a] - visc;
    out[1 + a] = T(-0.5) * conv - fa / f;
  }
  const T t00 = tau(0, 0)(i, j, k), t01 = tau(0, 1)(i, j, k), t11 = tau(1, 1)(i, j, k);
  const T t02 = tau(0, 2)(i, j, k), t12 = tau(1, 2)(i, j, k), t22 = tau(2, 2)(i, j, k);
  const T phi_v = ((t00 * du[0][0] + t01 * (du[0][1] + du[1][0])) + t11 * du[1][1]) +
                  ((t02 * (du[0][2] + du[2][0]) + t12 * (du[1][2] + du[2][1])) + t22 * du[2][2]);
  const T heat = (d1<T>(qh[0], 0, i, j, k, c) + d1<T>(qh[1], 1, i, j, k, c)) + d1<T>(qh[2], 2, i, j, k, c);
  const T dpu = (d1m<T>(pr, vel[0], 0, i, j, k, c) + d1m<T>(pr, vel[1], 1, i, j, k, c)) +
                d1m<T>(pr, vel[2], 2, i, j, k, c);
  const T adv = (u[0] * dp[0] + u[1] * dp[1]) + u[2] * dp[2];
  out[4] = (-gam * dpu + gm1 * adv) + gm1 * (phi_v + heat);
}

// ----------------------------------------------------------------------------
// Shock-capturing filter of Bogey, de Cacqueray & Bailly (2009), applied after
// every step in Sec. 4, in three dimensions.  Per direction a and node n:
//   dilatation  th = ((u_{i+1} - u_{i-1}) + (v_{j+1} - v_{j-1}) + (w_{k+1} - w_{k-1})) / (2 dx)
//               (each difference scaled separately, summed as ((x + y) + z)),
//   high-pass   Dth_n = (-th_{n+1} + 2 th_n - th_{n-1}) / 4 along a,
//   magnitude   M_n = ((Dth_n - Dth_{n+1})^2 + (Dth_n - Dth_{n-1})^2) / 2,
//   sensor      r_n = M_n / (c_n^2 / dx^2) + 1e-16, c^2 = gamma p / rho,
//   strength    s_n = (z + |z|) / 2, z = 1 - r_th / r_n,
//   update      q_n <- q_n - sum_a (s_{n+1/2} F_{n+1/2} - s_{n-1/2} F_{n-1/2}),
//               F_{n+1/2} = -(q_{n+1} - q_n) / 4, s_{n+1/2} = (s_n + s_{n+1}) / 2.

// Velocity and c^2 of a node; kind 2 flux-form state, kind 3 skew-symmetric state.
template <typename T>
MR_NS3_HD void filter_prims(int kind, T gam, const T q[5], T vel[3], T& cc) {
  for (int a = 0; a < 3; ++a) vel[a] = q[1 + a] / q[0];
  T rho, p;
  if (kind == 2) {
    rho = q[0];
    p = (gam - T(1)) * (q[4] - T(0.5) * ((q[1] * vel[0] + q[2] * vel[1]) + q[3] * vel[2]));
  } else {
    rho = q[0] * q[0];
    p = q[4];
  }
  cc = gam * p / rho;
}

// Dilatation at a node from the velocity accessors; h2 = 1 / (2 dx).
template <typename T, typename V>
MR_NS3_HD T dilatation(const V* vel, int i, int j, int k, T h2) {
  return ((vel[0](i + 1, j, k) - vel[0](i - 1, j, k)) * h2 + (vel[1](i, j + 1, k) - vel[1](i, j - 1, k)) * h2) +
         (vel[2](i, j, k + 1) - vel[2](i, j, k - 1)) * h2;
}

// Strength along axis a at a node from the dilatation accessor th (needed at
// +-2 along a) and the node's c^2; dx2 = dx^2.
template <typename T, typename D>
MR_NS3_HD T strength(const D& th, T cc, int a, int i, int j, int k, T dx2, T rth) {
  const int o0 = a == 0, o1 = a == 1, o2 = a == 2;
  auto Dth = [&](int s) {
    const int ii = i + s * o0, jj = j + s * o1, kk = k + s * o2;
    return (-th(ii + o0, jj + o1, kk + o2) + T(2) * th(ii, jj, kk) - th(ii - o0, jj - o1, kk - o2)) / T(4);
  };
  const T d0 = Dth(0), dp = Dth(1), dm = Dth(-1);
  const T M = T(0.5) * ((d0 - dp) * (d0 - dp) + (d0 - dm) * (d0 - dm));
  const T r = M / (cc / dx2) + T(1e-16);
  const T z = T(1) - rth / r;
  return T(0.5) * (z + (z < T(0) ? -z : z));
}

// Filtered value of a variable at an interior node: q its accessor, sg[a] the
// strengths along a (needed at -1..+1 along a).
template <typename T, typename Q, typename S>
MR_NS3_HD T filter_update(const Q& q, const S* sg, int i, int j, int k) {
  T dd[3];
  for (int a = 0; a < 3; ++a) {
    const int o0 = a == 0, o1 = a == 1, o2 = a == 2;
    const T sp = T(0.5) * (sg[a](i, j, k) + sg[a](i + o0, j + o1, k + o2));
    const T sm = T(0.5) * (sg[a](i - o0, j - o1, k - o2) + sg[a](i, j, k));
    const T fp = T(-0.25) * (q(i + o0, j + o1, k + o2) - q(i, j, k));
    const T fm = T(-0.25) * (q(i, j, k) - q(i - o0, j - o1, k - o2));
    dd[a] = sp * fp - sm * fm;
  }
  return q(i, j, k) - ((dd[0] + dd[1]) + dd[2]);
}

}  // namespace ns3
}  // namespace mr

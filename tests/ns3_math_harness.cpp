// Host harness of the 3D Navier-Stokes node arithmetic (mr_ns3_math.cuh),
// compiled as plain C++ by tests/test_ns3_math_host.py: reads synchronised
// block tiles and runs, through the header's functions, either the right-hand
// side (three phases: primitives, stresses / fluxes, right-hand side) or the
// shock-capturing filter (primitives, dilatation, strengths, update).
//
// stdin:  int32 mode (2 / 3: right-hand side of the flux / skew form; 12 / 13:
//         filter of a flux / skew state), B, g, nblocks; double gam, mu, Pr, r_th;
//         per block: double dx, then 5 x T^3 doubles ([var][z][y][x],
//         T = B + 2 g, ghosts included).
// stdout: per block 5 x B^3 doubles ([var][z][y][x], interior): the
//         right-hand side, or the filtered state.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "mr_ns3_math.cuh"

namespace {

struct Arr {
  const double* p;
  int T, g;
  double operator()(int i, int j, int k) const {
    return p[((size_t)(k + g) * T + (size_t)(j + g)) * T + (size_t)(i + g)];
  }
};

bool read_all(void* dst, size_t bytes) { return std::fread(dst, 1, bytes, stdin) == bytes; }

// The filter on one synchronised tile: velocity and c^2 on every node, the
// dilatation on nodes -3..B+2, strengths along a on -1..B along a and 0..B-1
// across, the update on the interior.
void filter_block(int form, int B, int g, double gam, double rth, double dx, const std::vector<double>& tile,
                  std::vector<double>& out) {
  const int T = B + 2 * g;
  const size_t TT = (size_t)T * T * T, NB = (size_t)B * B * B;
  auto I = [&](int i, int j, int k) { return ((size_t)(k + g) * T + (size_t)(j + g)) * T + (size_t)(i + g); };
  std::vector<double> vel[3], cc(TT, 0.0), th(TT, 0.0), sg[3];
  for (int a = 0; a < 3; ++a) {
    vel[a].assign(TT, 0.0);
    sg[a].assign(TT, 0.0);
  }
  for (int k = -g; k < B + g; ++k)
    for (int j = -g; j < B + g; ++j)
      for (int i = -g; i < B + g; ++i) {
        const size_t q = I(i, j, k);
        double s[5], v3[3], c2 = 0.0;
        for (int v = 0; v < 5; ++v) s[v] = tile[v * TT + q];
        mr::ns3::filter_prims<double>(form, gam, s, v3, c2);
        for (int a = 0; a < 3; ++a) vel[a][q] = v3[a];
        cc[q] = c2;
      }
  const Arr av[3] = {{vel[0].data(), T, g}, {vel[1].data(), T, g}, {vel[2].data(), T, g}};
  const double h2 = 0.5 / dx, dx2 = dx * dx;
  for (int k = -3; k <= B + 2; ++k)
    for (int j = -3; j <= B + 2; ++j)
      for (int i = -3; i <= B + 2; ++i) th[I(i, j, k)] = mr::ns3::dilatation<double>(av, i, j, k, h2);
  const Arr ath{th.data(), T, g};
  for (int k = -1; k <= B; ++k)
    for (int j = -1; j <= B; ++j)
      for (int i = -1; i <= B; ++i) {
        const int ijk[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
          bool inside = true;
          for (int e = 0; e < 3; ++e)
            if (e != a && (ijk[e] < 0 || ijk[e] >= B)) inside = false;
          if (inside) sg[a][I(i, j, k)] = mr::ns3::strength<double>(ath, cc[I(i, j, k)], a, i, j, k, dx2, rth);
        }
      }
  const Arr as[3] = {{sg[0].data(), T, g}, {sg[1].data(), T, g}, {sg[2].data(), T, g}};
  for (int v = 0; v < 5; ++v) {
    const Arr aq{tile.data() + v * TT, T, g};
    for (int k = 0; k < B; ++k)
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i)
          out[v * NB + ((size_t)k * B + j) * B + i] = mr::ns3::filter_update<double>(aq, as, i, j, k);
  }
}

}  // namespace

int main() {
  int32_t hdr[4];
  double par[4];
  if (!read_all(hdr, sizeof(hdr)) || !read_all(par, sizeof(par))) return 1;
  const int mode = hdr[0], B = hdr[1], g = hdr[2], nb = hdr[3];
  const int form = mode % 10;
  const double gam = par[0], mu = par[1], Pr = par[2], rth = par[3];
  const double kap = mu * gam / ((gam - 1.0) * Pr);
  const int T = B + 2 * g;
  const size_t TT = (size_t)T * T * T, NB = (size_t)B * B * B;
  auto I = [&](int i, int j, int k) { return ((size_t)(k + g) * T + (size_t)(j + g)) * T + (size_t)(i + g); };
  std::vector<double> tile(5 * TT), out(5 * NB);
  for (int n = 0; n < nb; ++n) {
    double dx;
    if (!read_all(&dx, sizeof(dx)) || !read_all(tile.data(), tile.size() * sizeof(double))) return 1;
    if (mode >= 10) {
      filter_block(form, B, g, gam, rth, dx, tile, out);
      if (std::fwrite(out.data(), sizeof(double), out.size(), stdout) != out.size()) return 1;
      continue;
    }
    const double c = 1.0 / (12.0 * dx);
    // phase 1: primitives on every tile node
    std::vector<double> vel[3], pr(TT, 0.0), th(TT, 0.0);
    for (auto& a : vel) a.assign(TT, 0.0);
    for (int k = -g; k < B + g; ++k)
      for (int j = -g; j < B + g; ++j)
        for (int i = -g; i < B + g; ++i) {
          const size_t q = I(i, j, k);
          double s[5], v3[3], p = 0.0, t = 0.0;
          for (int v = 0; v < 5; ++v) s[v] = tile[v * TT + q];
          if (form == 2) {
            mr::ns3::prim_flux<double>(gam, s, v3, p, t);
          } else {
            mr::ns3::prim_skew<double>(s, v3, t);
            p = s[4];
          }
          for (int a = 0; a < 3; ++a) vel[a][q] = v3[a];
          pr[q] = p;
          th[q] = t;
        }
    const Arr av[3] = {{vel[0].data(), T, g}, {vel[1].data(), T, g}, {vel[2].data(), T, g}};
    const Arr ath{th.data(), T, g};
    // phase 2: stresses, heat fluxes (skew) or the fluxes (flux form) on -2..B+1
    std::vector<double> tau[3][3], qh[3], F[3][5];
    for (int a = 0; a < 3; ++a) {
      qh[a].assign(TT, 0.0);
      for (int e = 0; e < 3; ++e) tau[a][e].assign(TT, 0.0);
      for (int v = 0; v < 5; ++v) F[a][v].assign(TT, 0.0);
    }
    for (int k = -2; k < B + 2; ++k)
      for (int j = -2; j < B + 2; ++j)
        for (int i = -2; i < B + 2; ++i) {
          const size_t q = I(i, j, k);
          double du[3][3], t3[3][3];
          mr::ns3::stress<double>(av, i, j, k, c, mu, du, t3);
          if (form == 2) {
            double s[5], v3[3] = {vel[0][q], vel[1][q], vel[2][q]}, thd[3], Fn[3][5];
            for (int v = 0; v < 5; ++v) s[v] = tile[v * TT + q];
            for (int a = 0; a < 3; ++a) thd[a] = mr::ns3::d1<double>(ath, a, i, j, k, c);
            mr::ns3::fluxes<double>(s, v3, pr[q], t3, thd, kap, Fn);
            for (int a = 0; a < 3; ++a)
              for (int v = 0; v < 5; ++v) F[a][v][q] = Fn[a][v];
          } else {
            for (int a = 0; a < 3; ++a) {
              for (int e = 0; e < 3; ++e) tau[a][e][q] = t3[a][e];
              qh[a][q] = kap * mr::ns3::d1<double>(ath, a, i, j, k, c);
            }
          }
        }
    // phase 3: right-hand side on the interior
    const Arr aph{tile.data(), T, g}, apr{pr.data(), T, g};
    const Arr aps[3] = {{tile.data() + TT, T, g}, {tile.data() + 2 * TT, T, g}, {tile.data() + 3 * TT, T, g}};
    const Arr aqh[3] = {{qh[0].data(), T, g}, {qh[1].data(), T, g}, {qh[2].data(), T, g}};
    auto tauA = [&](int a, int e) { return Arr{tau[a][e].data(), T, g}; };
    auto fluxA = [&](int v, int a) { return Arr{F[a][v].data(), T, g}; };
    for (int k = 0; k < B; ++k)
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i) {
          const size_t m = ((size_t)k * B + j) * B + i;
          if (form == 2) {
            for (int v = 0; v < 5; ++v) out[v * NB + m] = mr::ns3::rhs_flux<double>(fluxA, v, i, j, k, c);
          } else {
            double r[5];
            mr::ns3::rhs_skew<double>(aph, aps, apr, av, tauA, aqh, i, j, k, c, gam, r);
            for (int v = 0; v < 5; ++v) out[v * NB + m] = r[v];
          }
        }
    if (std::fwrite(out.data(), sizeof(double), out.size(), stdout) != out.size()) return 1;
  }
  return 0;
}

// Host harness of the 3D Navier-Stokes node arithmetic (mr_ns3_math.cuh),
// compiled as plain C++ by tests/test_ns3_math_host.py: reads synchronised
// block tiles, runs the three phases (primitives, stresses / fluxes, right-hand
// side) through the header's functions and writes the right-hand sides.
//
// stdin:  int32 form (2 flux, 3 skew), B, g, nblocks; double gam, mu, Pr;
//         per block: double c = 1 / (12 dx), then 5 x T^3 doubles
//         ([var][z][y][x], T = B + 2 g, ghosts included).
// stdout: per block 5 x B^3 doubles ([var][z][y][x], interior).
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

}  // namespace

int main() {
  int32_t hdr[4];
  double par[3];
  if (!read_all(hdr, sizeof(hdr)) || !read_all(par, sizeof(par))) return 1;
  const int form = hdr[0], B = hdr[1], g = hdr[2], nb = hdr[3];
  const double gam = par[0], mu = par[1], Pr = par[2];
  const double kap = mu * gam / ((gam - 1.0) * Pr);
  const int T = B + 2 * g;
  const size_t TT = (size_t)T * T * T, NB = (size_t)B * B * B;
  auto I = [&](int i, int j, int k) { return ((size_t)(k + g) * T + (size_t)(j + g)) * T + (size_t)(i + g); };
  std::vector<double> tile(5 * TT), out(5 * NB);
  for (int n = 0; n < nb; ++n) {
    double c;
    if (!read_all(&c, sizeof(c)) || !read_all(tile.data(), tile.size() * sizeof(double))) return 1;
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

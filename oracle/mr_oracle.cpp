// Plain FP64 CPU oracle of the block-based multiresolution step.
//
// TEST INFRASTRUCTURE ONLY: this file is read by tests/, by the smoke check and
// by the CPU-baseline leg of the benchmark.  The product library never links,
// loads or calls it, and it shares no code, header or table with the CUDA path.
//
// It follows the method of Sroka et al., "An open and parallel multiresolution
// framework using block-based adaptive grids" (arXiv:1902.00088):
//   * block and grid definition ............ Sec. 2.2 (block B^l, conditional
//                                             ghost nodes, graded tree, treecodes,
//                                             16 / 74 neighbour relations)
//   * multiresolution time step ............ Sec. 2.1 (refine, evolve, coarsen)
//   * prediction P, restriction R, details . Sec. 2.3 (upsampling, D = B - P(R(B)),
//                                             flag r = -1 if ||d||_inf < eps)
//   * ghost synchronisation ................ Sec. 2.5 (finer blocks overwrite the
//                                             redundant nodes of coarser ones)
//   * 4th-order central FD + RK4 ........... Sec. 3 and Sec. 4
//   * swirl test velocity .................. Sec. 3, Eq. (1)
//   * compressible Navier-Stokes ........... Sec. 4 (flux form and the
//                                             skew-symmetric form, 2D and 3D;
//                                             the shock-capturing filter after
//                                             each step; double shear layer)
// Everything is written per point with std::map lookups so that it can be
// checked against the text by eye; nothing is blocked, fused or reordered.
// Compile with -O2 -ffp-contract=off so every a*b+c is a rounded product
// followed by a rounded sum.
//
// Readings of passages the paper leaves open (block index range, prediction
// stencil, tie rules for redundant nodes, -2 status, coarsening rounds, NS
// flux form) are listed at the head of each function that takes them.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <random>
#include <vector>

extern "C" {
// Parameters of one tree.  rhs_kind: 0 constant-velocity advection,
// 1 swirl (Sec. 3), 2 compressible Navier-Stokes (Sec. 4; 2D with nvar 4,
// 3D with nvar 5) in flux form, 3 the same in the skew-symmetric form on
// square-root variables; for 2 and 3
// rhs = {gamma, mu, Pr, r_th}, r_th > 0 enabling the shock filter after each
// step.  ic_kind: 0 separable Gaussian blob, 1 temporal mixing layer, 2 none
// (set_blocks), 3 the double shear layer of Sec. 4.
typedef struct {
  int32_t dim, Bs, ng, nvar, Jmin, Jmax;
  int32_t rhs_kind, ic_kind, norm_kind, max_rounds;
  double L, eps;
  double x0[3];
  double rhs[8];
  double ic[32];
} orc_params;
}

namespace {

int64_t pmod(int64_t a, int64_t n) { int64_t r = a % n; return r < 0 ? r + n : r; }

// Interpolating-wavelet (Deslauriers-Dubuc, 4 points) midpoint prediction,
// Sec. 2.3 ("4th order", central): p = (9(f0+f1) - (f-1+f2)) / 16.
double dd4(double fm1, double f0, double f1, double f2) {
  return (9.0 * (f0 + f1) - (fm1 + f2)) / 16.0;
}

// Treecode (Sec. 2.2): one base-2^d digit per level, digit = bx + 2 by + 4 bz;
// for a block at level l with block coordinates c this is the bit interleave.
uint64_t treecode(int dim, const int64_t c[3], int lvl) {
  uint64_t t = 0;
  for (int b = lvl - 1; b >= 0; --b)
    for (int a = dim - 1; a >= 0; --a) t = (t << 1) | (uint64_t)((c[a] >> b) & 1);
  return t;
}
void treecode_coords(int dim, uint64_t t, int lvl, int64_t c[3]) {
  c[0] = c[1] = c[2] = 0;
  for (int b = 0; b < lvl; ++b)
    for (int a = 0; a < dim; ++a) c[a] |= (int64_t)((t >> (b * dim + a)) & 1) << b;
}

// Hilbert index of a cell (Skilling, "Programming the Hilbert curve", AIP Conf.
// Proc. 707, 2004): axes -> transposed index, then bit interleave.  Used only to
// fix the canonical export order (the paper orders blocks on a space-filling
// curve for load balancing, Sec. 2.5).
uint64_t hilbert_key(int dim, int bits, const int64_t cell[3]) {
  uint32_t X[3] = {(uint32_t)cell[0], (uint32_t)cell[1], (uint32_t)cell[2]};
  if (bits == 0) return 0;
  uint32_t M = 1u << (bits - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    uint32_t P = Q - 1;
    for (int i = 0; i < dim; ++i) {
      if (X[i] & Q) X[0] ^= P;
      else { uint32_t t = (X[0] ^ X[i]) & P; X[0] ^= t; X[i] ^= t; }
    }
  }
  for (int i = 1; i < dim; ++i) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (X[dim - 1] & Q) t ^= Q - 1;
  for (int i = 0; i < dim; ++i) X[i] ^= t;
  uint64_t h = 0;
  for (int b = bits - 1; b >= 0; --b)
    for (int i = 0; i < dim; ++i) h = (h << 1) | ((X[i] >> b) & 1u);
  return h;
}

struct Leaf {
  int lvl = 0;
  int64_t c[3] = {0, 0, 0};
  std::vector<double> t;  // hvy_block: nvar x (T^d) values, ghosts included
  int flag = 0;           // refinement status r
  double mdet = 0.0;      // largest (normalised) detail of the block
};
using Key = std::pair<int, uint64_t>;  // (level, treecode)

struct Cand { int m; Leaf* f; int combo; };

struct Tree {
  orc_params p;
  int d, B, g, T, nz, gz, nv;
  int64_t N;  // number of finest-lattice intervals per direction
  std::map<Key, Leaf> lv;
  mutable int64_t err = 0;  // violated invariants (stencil outside a tile, non-graded owner)

  explicit Tree(const orc_params& q) : p(q) {
    d = p.dim; B = p.Bs; g = p.ng; nv = p.nvar;
    T = B + 2 * g; nz = d == 3 ? T : 1; gz = d == 3 ? g : 0;
    N = (int64_t)(B - 1) << p.Jmax;
  }
  size_t tsize() const { return (size_t)nv * nz * T * T; }
  size_t ix(int v, int i, int j, int k) const {
    return (((size_t)v * nz + (k + gz)) * T + (j + g)) * T + (i + g);
  }
  int64_t step(int m) const { return (int64_t)1 << (p.Jmax - m); }
  int64_t width(int m) const { return (int64_t)(B - 1) << (p.Jmax - m); }
  Key key(int lvl, const int64_t c[3]) const { return {lvl, treecode(d, c, lvl)}; }
  Leaf* find(int lvl, const int64_t c[3]) {
    if (lvl < p.Jmin || lvl > p.Jmax) return nullptr;
    int64_t w[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) w[a] = pmod(c[a], (int64_t)1 << lvl);
    auto it = lv.find(key(lvl, w));
    return it == lv.end() ? nullptr : &it->second;
  }
  // Position of tile node (i,j,k) of leaf b on the finest lattice (unwrapped).
  void node_pos(const Leaf& b, const int ijk[3], int64_t U[3]) const {
    for (int a = 0; a < 3; ++a) U[a] = 0;
    for (int a = 0; a < d; ++a) U[a] = (b.c[a] * (B - 1) + ijk[a]) * step(b.lvl);
  }

  // All leaves whose closed cell contains the finest-lattice point U, at every
  // level.  combo bit a set = on axis a the point is the upper boundary node of
  // that leaf (it sits on a block edge shared with the next block).
  std::vector<Cand> containing(const int64_t U[3]) {
    std::vector<Cand> out;
    for (int m = p.Jmin; m <= p.Jmax; ++m) {
      int64_t W = width(m), nb = (int64_t)1 << m, k0[3] = {0, 0, 0};
      bool onb[3] = {false, false, false};
      for (int a = 0; a < d; ++a) {
        int64_t u = pmod(U[a], N);
        k0[a] = u / W; onb[a] = (u % W) == 0;
      }
      for (int combo = 0; combo < (1 << d); ++combo) {
        int64_t k[3] = {0, 0, 0};
        bool ok = true;
        for (int a = 0; a < d; ++a) {
          if ((combo >> a) & 1) {
            if (!onb[a]) { ok = false; break; }
            k[a] = pmod(k0[a] - 1, nb);
          } else k[a] = k0[a];
        }
        if (!ok) continue;
        Leaf* f = find(m, k);
        if (f) out.push_back({m, f, combo});
      }
    }
    return out;
  }
  // Canonical owner of a point: the finest containing leaf (Sec. 2.2: nodes at a
  // level interface belong to the finer block); among equal-level leaves the
  // lowest combo index, i.e. the leaf in which the node has local index 0 on as
  // many leading axes as possible.  exclude: a leaf never chosen (the block
  // itself when it asks for a finer owner of its own node).
  const Cand* owner(const std::vector<Cand>& cs, int min_level) const {
    const Cand* best = nullptr;
    for (const Cand& c : cs) {
      if (c.m < min_level) continue;
      if (!best || c.m > best->m || (c.m == best->m && c.combo < best->combo)) best = &c;
    }
    return best;
  }
  bool is_node(const int64_t U[3], int m) const {
    for (int a = 0; a < d; ++a) if (pmod(U[a], step(m)) != 0) return false;
    return true;
  }
  // Local node index of finest-lattice point U in leaf f (U in f's closed cell).
  void local_index(const Leaf& f, const int64_t U[3], int li[3]) const {
    li[0] = li[1] = li[2] = 0;
    for (int a = 0; a < d; ++a) {
      int64_t off = pmod(U[a] - f.c[a] * width(f.lvl), N);
      li[a] = (int)(off / step(f.lvl));
    }
  }
  double val(const Leaf& f, int v, const int li[3]) const { return f.t[ix(v, li[0], li[1], li[2])]; }

  // Tensor-product prediction from a coarse tile: positions given in units of
  // half a coarse spacing (o[a] odd = between coarse nodes).  x first, then y,
  // then z (the paper states only a central "4th order" interpolation).
  double predict(const Leaf& f, int v, const int o[3]) const {
    int ns[3] = {1, 1, 1}, base[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      int q = o[a];
      int fl = (q >= 0) ? q / 2 : -((-q + 1) / 2);  // floor(q / 2)
      if (q & 1) { ns[a] = 4; base[a] = fl - 1; } else base[a] = fl;
      if (base[a] < -g || base[a] + ns[a] - 1 > B - 1 + g) ++err;
    }
    double vx[4][4];  // [sz][sy] after the x pass
    for (int sz = 0; sz < ns[2]; ++sz)
      for (int sy = 0; sy < ns[1]; ++sy) {
        int li[3] = {base[0], base[1] + sy, base[2] + sz};
        if (ns[0] == 4) {
          double a0 = f.t[ix(v, base[0] + 0, li[1], li[2])];
          double a1 = f.t[ix(v, base[0] + 1, li[1], li[2])];
          double a2 = f.t[ix(v, base[0] + 2, li[1], li[2])];
          double a3 = f.t[ix(v, base[0] + 3, li[1], li[2])];
          vx[sz][sy] = dd4(a0, a1, a2, a3);
        } else vx[sz][sy] = f.t[ix(v, li[0], li[1], li[2])];
      }
    double vy[4];
    for (int sz = 0; sz < ns[2]; ++sz)
      vy[sz] = ns[1] == 4 ? dd4(vx[sz][0], vx[sz][1], vx[sz][2], vx[sz][3]) : vx[sz][0];
    return ns[2] == 4 ? dd4(vy[0], vy[1], vy[2], vy[3]) : vy[0];
  }

  // ---------------------------------------------------------------- sync ----
  // Ghost-node synchronisation (Sec. 2.2 conditional ghost nodes, Sec. 2.5).
  // Pass 1: every ghost node that is a node of its owner (same or finer level,
  // or a coarse node of a coarser owner) is copied from the owner; every
  // conditional (block-edge) node whose owner is another block (a finer one,
  // or an equal-level one holding it at its lower edge) takes the owner's value.
  // Pass 2, by ascending level: ghost nodes whose owner is coarser and that are
  // not coarse nodes are predicted from the coarse lattice around them.  Each
  // coarse stencil node takes the value of its own owner (finest leaf holding
  // it), which is what the coarse block's synchronised tile holds there; the
  // paper assumes equal-level redundant nodes identical (Sec. 2.5), so the tie
  // rule of owner() decides only between values it takes to be equal.
  double coarse_value(int64_t const Q[3], int v, int min_level) {
    std::vector<Cand> cs = containing(Q);
    const Cand* o = owner(cs, 0);
    if (!o || o->m < min_level) { ++err; return 0.0; }
    int li[3];
    local_index(*o->f, Q, li);
    return val(*o->f, v, li);
  }
  void sync() {
    struct W1 { Leaf* b; size_t at; double v; };
    struct W2 { Leaf* b; int ijk[3]; Leaf* f; };
    std::vector<W1> w1;
    std::map<int, std::vector<W2>> w2;
    for (auto& kv : lv) {
      Leaf& b = kv.second;
      for (int k = -gz; k < (d == 3 ? B + gz : 1); ++k)
        for (int j = -g; j < B + g; ++j)
          for (int i = -g; i < B + g; ++i) {
            int ijk[3] = {i, j, k};
            bool ghost = false, edge = false;
            for (int a = 0; a < d; ++a) {
              if (ijk[a] < 0 || ijk[a] > B - 1) ghost = true;
              else if (ijk[a] == 0 || ijk[a] == B - 1) edge = true;
            }
            if (!ghost && !edge) continue;
            int64_t U[3];
            node_pos(b, ijk, U);
            std::vector<Cand> cs = containing(U);
            if (ghost) {
              const Cand* o = owner(cs, 0);
              if (!o) continue;  // cannot happen on a complete periodic tree
              if (o->m >= b.lvl || is_node(U, o->m)) {
                int li[3];
                local_index(*o->f, U, li);
                for (int v = 0; v < nv; ++v) w1.push_back({&b, ix(v, i, j, k), val(*o->f, v, li)});
              } else {
                W2 w{&b, {i, j, k}, o->f};
                w2[b.lvl].push_back(w);
              }
            } else {
              // block-edge node: the finer block's value (Sec. 2.2 rule 2); an
              // equal-level redundant copy is made identical by taking the
              // canonical owner's value (the paper assumes the copies equal,
              // Sec. 2.5, but a refinement next to an existing block creates
              // children whose edge nodes were interpolated, not evolved)
              const Cand* o = owner(cs, b.lvl);
              if (!o || o->f == &b) continue;
              int li[3];
              local_index(*o->f, U, li);
              for (int v = 0; v < nv; ++v) w1.push_back({&b, ix(v, i, j, k), val(*o->f, v, li)});
            }
          }
    }
    for (const W1& w : w1) w.b->t[w.at] = w.v;
    for (auto& lvlw : w2) {  // ascending level
      std::vector<W1> out;
      for (const W2& w : lvlw.second) {
        if (w.f->lvl != w.b->lvl - 1) ++err;  // owner must be one level coarser (graded)
        int64_t U[3];
        node_pos(*w.b, w.ijk, U);
        const int64_t hs = step(w.b->lvl), cs = step(w.f->lvl);
        // half-coarse position of the point relative to the coarse owner's origin
        int o[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) o[a] = (int)(pmod(U[a] - w.f->c[a] * width(w.f->lvl), N) / hs);
        for (int v = 0; v < nv; ++v) {
          auto node = [&](const int n[3]) {
            int64_t Q[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) Q[a] = w.f->c[a] * width(w.f->lvl) + (int64_t)n[a] * cs;
            return coarse_value(Q, v, w.f->lvl);
          };
          out.push_back({w.b, ix(v, w.ijk[0], w.ijk[1], w.ijk[2]), predict_nodes(node, o)});
        }
      }
      for (const W1& w : out) w.b->t[w.at] = w.v;
    }
  }
  // Tensor-product prediction at half-coarse position o from coarse node values
  // node(n): x first, then y, then z (the paper states only "4th order").
  template <typename F>
  double predict_nodes(F node, const int o[3]) const {
    int ns[3] = {1, 1, 1}, base[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      int q = o[a];
      int fl = (q >= 0) ? q / 2 : -((-q + 1) / 2);
      if (q & 1) { ns[a] = 4; base[a] = fl - 1; } else base[a] = fl;
    }
    double vx[4][4];
    for (int sz = 0; sz < ns[2]; ++sz)
      for (int sy = 0; sy < ns[1]; ++sy) {
        double w[4];
        for (int sx = 0; sx < ns[0]; ++sx) {
          int n[3] = {base[0] + sx, base[1] + sy, base[2] + sz};
          w[sx] = node(n);
        }
        vx[sz][sy] = ns[0] == 4 ? dd4(w[0], w[1], w[2], w[3]) : w[0];
      }
    double vy[4];
    for (int sz = 0; sz < ns[2]; ++sz)
      vy[sz] = ns[1] == 4 ? dd4(vx[sz][0], vx[sz][1], vx[sz][2], vx[sz][3]) : vx[sz][0];
    return ns[2] == 4 ? dd4(vy[0], vy[1], vy[2], vy[3]) : vy[0];
  }

  // ------------------------------------------------------------- refine -----
  // Refinement (Sec. 2.3): the synchronised block is upsampled by P including
  // its ghosts and split into 2^d children, one treecode digit appended.  Only
  // the children's interiors (fine nodes 0..2B-2) are kept: their ghosts are
  // synchronised again before use.  Blocks at Jmax are not refined.
  void refine_block(const Leaf& b, std::map<Key, Leaf>& out) {
    for (int ch = 0; ch < (1 << d); ++ch) {
      Leaf c;
      c.lvl = b.lvl + 1;
      int cb[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) { cb[a] = (ch >> a) & 1; c.c[a] = 2 * b.c[a] + cb[a]; }
      c.t.assign(tsize(), 0.0);
      for (int k = 0; k < (d == 3 ? B : 1); ++k)
        for (int j = 0; j < B; ++j)
          for (int i = 0; i < B; ++i) {
            int ijk[3] = {i, j, k}, o[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) o[a] = cb[a] * (B - 1) + ijk[a];
            for (int v = 0; v < nv; ++v) c.t[ix(v, i, j, k)] = predict(b, v, o);
          }
      out[key(c.lvl, c.c)] = std::move(c);
    }
  }
  // mode 0: refine every block below Jmax; mode 1: refine blocks with flag +1.
  void refine(int mode) {
    sync();
    std::map<Key, Leaf> nw;
    for (auto& kv : lv) {
      Leaf& b = kv.second;
      bool r = mode == 0 ? (b.lvl < p.Jmax) : (b.flag == 1 && b.lvl < p.Jmax);
      if (r) refine_block(b, nw);
      else nw[kv.first] = b;
    }
    lv.swap(nw);
  }

  // ------------------------------------------------------------ details -----
  // Details D = B - P(R(B)) (Sec. 2.3) on the synchronised tile: R keeps the
  // even tile nodes (ghosts included), P predicts the odd ones back.  Nonzero
  // only where an index is odd.  Returns, per variable, max |d| over interior.
  void block_details(const Leaf& b, std::vector<double>& md) const {
    md.assign(nv, 0.0);
    for (int k = 0; k < (d == 3 ? B : 1); ++k)
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i) {
          int ijk[3] = {i, j, k};
          bool odd = false;
          for (int a = 0; a < d; ++a) odd |= (ijk[a] & 1) != 0;
          if (!odd) continue;
          // coarse lattice of the block = even tile nodes: coarse index n is
          // tile node 2n; the point sits at half-coarse position ijk.
          for (int v = 0; v < nv; ++v) {
            double pr = predict_from_even(b, v, ijk);
            double dd = std::fabs(b.t[ix(v, i, j, k)] - pr);
            if (dd > md[v]) md[v] = dd;
          }
        }
  }
  double predict_from_even(const Leaf& b, int v, const int o[3]) const {
    // same tensor product as predict(), on the sub-lattice of even tile nodes
    int ns[3] = {1, 1, 1}, base[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      int q = o[a];
      int fl = (q >= 0) ? q / 2 : -((-q + 1) / 2);
      if (q & 1) { ns[a] = 4; base[a] = fl - 1; } else base[a] = fl;
    }
    double vx[4][4];
    for (int sz = 0; sz < ns[2]; ++sz)
      for (int sy = 0; sy < ns[1]; ++sy) {
        int y = 2 * (base[1] + sy), z = 2 * (base[2] + sz);
        if (ns[0] == 4) {
          double a0 = b.t[ix(v, 2 * (base[0] + 0), y, z)];
          double a1 = b.t[ix(v, 2 * (base[0] + 1), y, z)];
          double a2 = b.t[ix(v, 2 * (base[0] + 2), y, z)];
          double a3 = b.t[ix(v, 2 * (base[0] + 3), y, z)];
          vx[sz][sy] = dd4(a0, a1, a2, a3);
        } else vx[sz][sy] = b.t[ix(v, 2 * base[0], y, z)];
      }
    double vy[4];
    for (int sz = 0; sz < ns[2]; ++sz)
      vy[sz] = ns[1] == 4 ? dd4(vx[sz][0], vx[sz][1], vx[sz][2], vx[sz][3]) : vx[sz][0];
    return ns[2] == 4 ? dd4(vy[0], vy[1], vy[2], vy[3]) : vy[0];
  }
  // Per-variable scale of the threshold: 1 (advection) or the largest |q_v|
  // over the synchronised grid (Navier-Stokes; the paper is silent on
  // normalising several variables).
  std::vector<double> var_scale() const {
    std::vector<double> s(nv, 1.0);
    if (p.norm_kind == 0) return s;
    std::fill(s.begin(), s.end(), 0.0);
    for (auto& kv : lv) {
      const Leaf& b = kv.second;
      for (int v = 0; v < nv; ++v)
        for (int k = 0; k < (d == 3 ? B : 1); ++k)
          for (int j = 0; j < B; ++j)
            for (int i = 0; i < B; ++i) s[v] = std::max(s[v], std::fabs(b.t[ix(v, i, j, k)]));
    }
    for (int v = 0; v < nv; ++v) if (s[v] == 0.0) s[v] = 1.0;
    return s;
  }
  void details() {
    sync();
    std::vector<double> s = var_scale();
    std::vector<double> md;
    for (auto& kv : lv) {
      block_details(kv.second, md);
      double m = 0.0;
      for (int v = 0; v < nv; ++v) m = std::max(m, md[v] / s[v]);
      kv.second.mdet = m;
    }
  }

  // -------------------------------------------------------- neighbours ------
  // The 16 (2D) / 74 (3D) neighbour relations of Sec. 2.2: for every direction
  // s in {-1,0,1}^d \ 0 (faces, then edges, then corners; x fastest) one entry
  // for a same-level or coarser neighbour and, unless s is a corner, 2^(zeros)
  // entries for the finer blocks touching the face/edge; corners have a single
  // entry whatever the level.  Neighbours are found from the treecode: decode
  // to block coordinates, add s with periodic wrap, encode, look up.
  struct Rel { int s[3]; int sub; };  // sub = -1 full entry, else child index on zero axes
  std::vector<Rel> relations() const {
    std::vector<Rel> r;
    for (int nnz = 1; nnz <= d; ++nnz)
      for (int sz = (d == 3 ? -1 : 0); sz <= (d == 3 ? 1 : 0); ++sz)
        for (int sy = -1; sy <= 1; ++sy)
          for (int sx = -1; sx <= 1; ++sx) {
            int s[3] = {sx, sy, sz};
            int cnt = (sx != 0) + (sy != 0) + (sz != 0);
            if (cnt != nnz) continue;
            if (nnz == d) { r.push_back({{sx, sy, sz}, -1}); continue; }
            r.push_back({{sx, sy, sz}, -1});
            for (int sub = 0; sub < (1 << (d - nnz)); ++sub) r.push_back({{sx, sy, sz}, sub});
            (void)s;
          }
    return r;
  }
  // Returns the leaf of relation rel of block b (or null) and its level difference.
  Leaf* neighbour(const Leaf& b, const Rel& rel, int* dl) {
    int64_t k[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) k[a] = b.c[a] + rel.s[a];
    bool corner = true;
    for (int a = 0; a < d; ++a) corner &= rel.s[a] != 0;
    // child of the neighbouring cell that touches b
    auto child = [&](int sub, int64_t ch[3]) {
      int z = 0;
      for (int a = 0; a < d; ++a) {
        int bit;
        if (rel.s[a] != 0) bit = rel.s[a] < 0 ? 1 : 0;
        else bit = (sub >> (z++)) & 1;
        ch[a] = 2 * pmod(k[a], (int64_t)1 << b.lvl) + bit;
      }
    };
    if (rel.sub < 0) {
      if (Leaf* f = find(b.lvl, k)) { *dl = 0; return f; }
      int64_t pc[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) pc[a] = pmod(k[a], (int64_t)1 << b.lvl) >> 1;
      if (b.lvl - 1 >= p.Jmin)
        if (Leaf* f = find(b.lvl - 1, pc)) { *dl = -1; return f; }
      if (corner) {
        int64_t ch[3] = {0, 0, 0};
        child(0, ch);
        if (Leaf* f = find(b.lvl + 1, ch)) { *dl = 1; return f; }
      }
      return nullptr;
    }
    if (find(b.lvl, k)) return nullptr;
    int64_t ch[3] = {0, 0, 0};
    child(rel.sub, ch);
    if (Leaf* f = find(b.lvl + 1, ch)) { *dl = 1; return f; }
    return nullptr;
  }
  bool has_finer_neighbour(const Leaf& b) {
    for (const Rel& r : relations()) {
      int dl = 0;
      Leaf* f = neighbour(b, r, &dl);
      if (f && dl == 1) return true;
    }
    return false;
  }

  // -------------------------------------------------------------- flags -----
  // Refinement status (Sec. 2.3): r = -1 if the largest detail is below eps
  // (strictly), else 0; blocks at Jmin keep 0.  A block can only be coarsened
  // with all its sisters (completeness) and if no neighbour is finer than
  // itself (gradedness after the merge); both vetoes are iterated until
  // nothing changes, visiting blocks in the order given by `seed` (0 = key
  // order).  Blocks that keep -1 get the final status -2 ("can indeed be
  // coarsened"; reading "+1" in the text as the coarsening status -1).
  int flags(uint64_t seed) {
    std::vector<Leaf*> order;
    for (auto& kv : lv) {
      Leaf& b = kv.second;
      b.flag = (b.mdet < p.eps && b.lvl > p.Jmin) ? -1 : 0;
      order.push_back(&b);
    }
    if (seed) { std::mt19937_64 rng(seed); std::shuffle(order.begin(), order.end(), rng); }
    bool changed = true;
    int iters = 0;
    while (changed) {
      changed = false; ++iters;
      for (Leaf* b : order) {
        if (b->flag != -1) continue;
        bool keep = true;
        for (int ch = 0; ch < (1 << d) && keep; ++ch) {
          int64_t sc[3] = {0, 0, 0};
          for (int a = 0; a < d; ++a) sc[a] = (b->c[a] & ~(int64_t)1) | ((ch >> a) & 1);
          Leaf* s = find(b->lvl, sc);
          if (!s || s->flag != -1) keep = false;
        }
        if (keep && has_finer_neighbour(*b)) keep = false;
        if (!keep) { b->flag = 0; changed = true; }
      }
    }
    int n = 0;
    for (auto& kv : lv) if (kv.second.flag == -1) { kv.second.flag = -2; ++n; }
    return n;
  }

  // ------------------------------------------------- refinement status +1 ---
  // Refinement indicators (Sec. 2.3, status +1) must keep the grid graded
  // (Sec. 2.2: blocks that touch differ by at most one level).  Refining a
  // block of level l creates blocks of level l + 1, so a touching leaf of level
  // l - 1 would end up two levels coarser: it must be refined as well.  The
  // rule is applied until no status changes; it only turns 0 into +1, so the
  // result does not depend on the visiting order.  Blocks at Jmax are never
  // refined and force nothing.  Returns the number of statuses raised.
  int close_refine() {
    int added = 0;
    bool changed = true;
    const std::vector<Rel> rels = relations();
    while (changed) {
      changed = false;
      for (auto& kv : lv) {
        Leaf& b = kv.second;
        if (b.flag != 1 || b.lvl >= p.Jmax) continue;
        for (const Rel& r : rels) {
          int dl = 0;
          Leaf* f = neighbour(b, r, &dl);
          if (f && dl == -1 && f->flag != 1) {
            f->flag = 1;
            ++added;
            changed = true;
          }
        }
      }
    }
    return added;
  }

  // ----------------------------------------------------------- coarsen ------
  // Coarsening (Sec. 2.3): 2^d sisters with status -2 merge into their mother by
  // the restriction R (every second node is kept); the last treecode digit is
  // dropped.  A mother node on the line shared by two children is read from the
  // child in which it has local index 0.
  int coarsen() {
    std::map<Key, Leaf> nw;
    int merged = 0;
    for (auto& kv : lv) {
      Leaf& b = kv.second;
      if (b.flag != -2) { nw[kv.first] = b; continue; }
      int64_t pc[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) pc[a] = b.c[a] >> 1;
      Key pk = key(b.lvl - 1, pc);
      if (nw.count(pk)) continue;
      Leaf m;
      m.lvl = b.lvl - 1;
      for (int a = 0; a < 3; ++a) m.c[a] = pc[a];
      m.t.assign(tsize(), 0.0);
      for (int k = 0; k < (d == 3 ? B : 1); ++k)
        for (int j = 0; j < B; ++j)
          for (int i = 0; i < B; ++i) {
            int I[3] = {i, j, k}, cb[3] = {0, 0, 0}, li[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) {
              cb[a] = (2 * I[a] >= B - 1) ? 1 : 0;
              li[a] = 2 * I[a] - cb[a] * (B - 1);
            }
            int64_t cc[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) cc[a] = 2 * pc[a] + cb[a];
            Leaf* ch = find(b.lvl, cc);
            for (int v = 0; v < nv; ++v) m.t[ix(v, i, j, k)] = ch->t[ix(v, li[0], li[1], li[2])];
          }
      nw[pk] = std::move(m);
      ++merged;
    }
    lv.swap(nw);
    return merged;
  }
  // Coarsening rounds until no family merges (reading: "removing, in part,
  // blocks created during refinement" allows several levels per step), at most
  // Jmax - Jmin rounds, or max_rounds if that is positive.
  int coarsen_until_stable() {
    int rounds = p.max_rounds > 0 ? p.max_rounds : (p.Jmax - p.Jmin);
    int total = 0;
    for (int r = 0; r < rounds; ++r) {
      details();
      if (flags(0) == 0) break;
      total += coarsen();
    }
    return total;
  }

  // ------------------------------------------------------- coordinates ------
  double coord(int a, int64_t U) const {
    double h = p.L / (double)N;
    return p.x0[a] + (double)pmod(U, N) * h;
  }

  // ------------------------------------------------------------ initial -----
  // Gaussian blob as a product of 1D factors with nearest periodic image:
  // exp(-r^2/(2 sigma^2)) = prod_a exp(-d_a^2/(2 sigma^2)).
  double gauss1(int a, double x, double shift) const {
    double dd = (x - shift) - p.ic[a];
    while (dd >= 0.5 * p.L) dd -= p.L;
    while (dd < -0.5 * p.L) dd += p.L;
    double s = p.ic[3];
    return std::exp(-(dd * dd) / (2.0 * s * s));
  }
  // Temporal mixing layer: a periodic pair of tanh shear layers (y = 0 and y = +-1/2).
  void mixing_layer(double x, double y, double q[4]) const {
    double delta = p.ic[0], U0 = p.ic[1], Ma = p.ic[2], gam = p.ic[3], amp = p.ic[4];
    double u = U0 * ((std::tanh(2.0 * y / delta) - std::tanh(2.0 * (y - 0.5) / delta)) -
                     std::tanh(2.0 * (y + 0.5) / delta));
    double s = 0.0;
    for (int kk = 0; kk < 8; ++kk)
      s += p.ic[5 + kk] * std::sin(2.0 * M_PI * (double)(kk + 1) * x + p.ic[13 + kk]);
    double e = std::exp(-(y / delta) * (y / delta));
    double v = amp * (s * e);
    double c0 = U0 / Ma;
    double p0 = c0 * c0 / gam;
    double e0 = p0 / (gam - 1.0);
    q[0] = 1.0; q[1] = u; q[2] = v; q[3] = e0 + 0.5 * (u * u + v * v);
  }
  // Double shear layer of Sec. 4 (reading of its garbled axes: the layers are
  // the lines x = xc -+ hw, across which rho and the y-velocity v jump; the
  // x-velocity u is perturbed along the layers):
  //   s(x) = (tanh((x - (xc - hw)) / lw) - tanh((x - (xc + hw)) / lw)) / 2,
  //   rho = rho0 + (rho1 - rho0) s, v = v0 + (v1 - v0) s,
  //   u = amp sin(2 pi (y - yc)), p = p0.
  // ic = {rho1, rho0, v1, v0, lw, p0, amp, hw, xc, yc}.  The state is
  // (rho, rho u, rho v, E) for the flux form and (sqrt(rho), sqrt(rho) u,
  // sqrt(rho) v, p) for the skew-symmetric form.
  void shear_layer(double x, double y, double q[4]) const {
    double rho1 = p.ic[0], rho0 = p.ic[1], v1 = p.ic[2], v0 = p.ic[3], lw = p.ic[4], p0 = p.ic[5];
    double amp = p.ic[6], hw = p.ic[7], xc = p.ic[8], yc = p.ic[9];
    double sprof = 0.5 * (std::tanh((x - (xc - hw)) / lw) - std::tanh((x - (xc + hw)) / lw));
    double rho = rho0 + (rho1 - rho0) * sprof;
    double v = v0 + (v1 - v0) * sprof;
    double u = amp * std::sin(2.0 * M_PI * (y - yc));
    if (p.rhs_kind == 3) {
      double f = std::sqrt(rho);
      q[0] = f; q[1] = f * u; q[2] = f * v; q[3] = p0;
    } else {
      double gam = p.rhs[0];
      double m1 = rho * u, m2 = rho * v;
      q[0] = rho; q[1] = m1; q[2] = m2; q[3] = p0 / (gam - 1.0) + 0.5 * (m1 * u + m2 * v);
    }
  }
  void set_ic(Leaf& b, double t_shift) {
    b.t.assign(tsize(), 0.0);
    for (int k = 0; k < (d == 3 ? B : 1); ++k)
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i) {
          int ijk[3] = {i, j, k};
          int64_t U[3];
          node_pos(b, ijk, U);
          if (p.ic_kind == 0) {
            double f = 1.0;
            for (int a = 0; a < d; ++a) {
              double sh = (p.rhs_kind == 0) ? p.rhs[a] * t_shift : 0.0;
              f = f * gauss1(a, coord(a, U[a]), sh);
            }
            b.t[ix(0, i, j, k)] = f;
          } else if (p.ic_kind == 1) {
            double q[4];
            mixing_layer(coord(0, U[0]), coord(1, U[1]), q);
            for (int v = 0; v < 4; ++v) b.t[ix(v, i, j, k)] = q[v];
          } else if (p.ic_kind == 3) {
            double q[4];
            shear_layer(coord(0, U[0]), coord(1, U[1]), q);
            for (int v = 0; v < 4; ++v) b.t[ix(v, i, j, k)] = q[v];
          }
        }
  }
  // Initial grid (not described in the paper): uniform at Jmin with the analytic
  // field, then Jmax - Jmin times: refine all, evaluate the analytic field on the
  // new blocks, coarsen until stable.
  void init_tree() {
    lv.clear();
    int64_t n = (int64_t)1 << p.Jmin;
    for (int64_t z = 0; z < (d == 3 ? n : 1); ++z)
      for (int64_t y = 0; y < n; ++y)
        for (int64_t x = 0; x < n; ++x) {
          Leaf b;
          b.lvl = p.Jmin; b.c[0] = x; b.c[1] = y; b.c[2] = z;
          set_ic(b, 0.0);
          lv[key(b.lvl, b.c)] = b;
        }
    for (int it = 0; it < p.Jmax - p.Jmin; ++it) {
      refine(0);
      for (auto& kv : lv) set_ic(kv.second, 0.0);
      coarsen_until_stable();
    }
  }

  // ---------------------------------------------------------------- RHS -----
  // 4th-order central first derivative (Sec. 3): (f[-2] - 8f[-1] + 8f[1] - f[2])
  // / (12 dx), evaluated as ((f[-2]-f[2]) + 8 (f[1]-f[-1])) * (1/(12 dx)).
  double cD(int lvl) const {
    double dx = p.L / (double)((int64_t)(B - 1) << lvl);
    return 1.0 / (12.0 * dx);
  }
  double d1(const Leaf& b, int v, int a, int i, int j, int k, double c) const {
    int o[3] = {0, 0, 0};
    o[a] = 1;
    auto at = [&](int s) { return b.t[ix(v, i + s * o[0], j + s * o[1], k + s * o[2])]; };
    return ((at(-2) - at(2)) + 8.0 * (at(1) - at(-1))) * c;
  }
  // Advection: N(phi) = -u . grad phi with constant u or the swirl field of
  // Sec. 3, Eq. (1): u = cos(pi t / t_a) (sin^2(pi x) sin(2 pi y), -sin^2(pi y) sin(2 pi x)).
  void rhs_advection(const Leaf& b, double ts, std::vector<double>& kk) const {
    double c = cD(b.lvl);
    double ct = 0.0;
    if (p.rhs_kind == 1) ct = std::cos(M_PI * ts / p.rhs[0]);
    for (int k = 0; k < (d == 3 ? B : 1); ++k)
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i) {
          int ijk[3] = {i, j, k};
          double u[3] = {p.rhs[0], p.rhs[1], p.rhs[2]};
          if (p.rhs_kind == 1) {
            int64_t U[3];
            node_pos(b, ijk, U);
            double x = coord(0, U[0]), y = coord(1, U[1]);
            double sxv = std::sin(M_PI * x), syv = std::sin(M_PI * y);
            double ax = sxv * sxv, ay = syv * syv;
            double bx = std::sin(2.0 * M_PI * x), by = std::sin(2.0 * M_PI * y);
            u[0] = ct * (ax * by);
            u[1] = -(ct * (ay * bx));
          }
          double s = u[0] * d1(b, 0, 0, i, j, k, c) + u[1] * d1(b, 0, 1, i, j, k, c);
          if (d == 3) s = s + u[2] * d1(b, 0, 2, i, j, k, c);
          kk[((size_t)k * B + j) * B + i] = -s;
        }
  }
  // Compressible Navier-Stokes, ideal gas, constant c_p (Sec. 4), 2D, in
  // conservative flux form (the skew-symmetric form of the cited paper is not
  // reproduced): q = (rho, rho u, rho v, E),
  //   N(q) = -(dF/dx + dG/dy),
  //   F = (rho u, rho u^2 + p - txx, rho u v - txy, (E+p) u - (u txx + v txy) - kap dth/dx),
  //   G = (rho v, rho v u - txy, rho v^2 + p - tyy, (E+p) v - (u txy + v tyy) - kap dth/dy),
  //   txx = mu (2 ux - 2/3 div), tyy = mu (2 vy - 2/3 div), txy = mu (uy + vx),
  //   th = p / rho, kap = mu gamma / ((gamma - 1) Pr)  (R_s cancels in k grad T).
  // Derivatives are the same 4th-order D1 on tile nodes -2..B+1.
  void rhs_ns(const Leaf& b, std::vector<double>& kk) const {
    double gam = p.rhs[0], mu = p.rhs[1], Pr = p.rhs[2];
    double kap = mu * gam / ((gam - 1.0) * Pr);
    double c23 = 2.0 / 3.0;
    double c = cD(b.lvl);
    int R = B + 2 * g;
    auto I = [&](int i, int j) { return (size_t)(j + g) * R + (i + g); };
    std::vector<double> u(R * R), v(R * R), pr(R * R), th(R * R);
    for (int j = -g; j < B + g; ++j)
      for (int i = -g; i < B + g; ++i) {
        double r = b.t[ix(0, i, j, 0)], m1 = b.t[ix(1, i, j, 0)], m2 = b.t[ix(2, i, j, 0)],
               E = b.t[ix(3, i, j, 0)];
        double uu = m1 / r, vv = m2 / r;
        double pp = (gam - 1.0) * (E - 0.5 * (m1 * uu + m2 * vv));
        u[I(i, j)] = uu; v[I(i, j)] = vv; pr[I(i, j)] = pp; th[I(i, j)] = pp / r;
      }
    auto dx = [&](const std::vector<double>& f, int i, int j) {
      return ((f[I(i - 2, j)] - f[I(i + 2, j)]) + 8.0 * (f[I(i + 1, j)] - f[I(i - 1, j)])) * c;
    };
    auto dy = [&](const std::vector<double>& f, int i, int j) {
      return ((f[I(i, j - 2)] - f[I(i, j + 2)]) + 8.0 * (f[I(i, j + 1)] - f[I(i, j - 1)])) * c;
    };
    std::vector<double> F[4], G[4];
    for (int q = 0; q < 4; ++q) { F[q].assign(R * R, 0.0); G[q].assign(R * R, 0.0); }
    for (int j = -2; j < B + 2; ++j)
      for (int i = -2; i < B + 2; ++i) {
        bool needF = (j >= 0 && j < B), needG = (i >= 0 && i < B);
        if (!needF && !needG) continue;
        double ux = dx(u, i, j), vx = dx(v, i, j), uy = dy(u, i, j), vy = dy(v, i, j);
        double div = ux + vy;
        double txy = mu * (uy + vx);
        double r = b.t[ix(0, i, j, 0)], m1 = b.t[ix(1, i, j, 0)], m2 = b.t[ix(2, i, j, 0)],
               E = b.t[ix(3, i, j, 0)];
        double uu = u[I(i, j)], vv = v[I(i, j)], pp = pr[I(i, j)];
        (void)r;
        if (needF) {
          double txx = mu * (2.0 * ux - c23 * div);
          double thx = dx(th, i, j);
          F[0][I(i, j)] = m1;
          F[1][I(i, j)] = m1 * uu + pp - txx;
          F[2][I(i, j)] = m1 * vv - txy;
          F[3][I(i, j)] = (E + pp) * uu - (uu * txx + vv * txy) - kap * thx;
        }
        if (needG) {
          double tyy = mu * (2.0 * vy - c23 * div);
          double thy = dy(th, i, j);
          G[0][I(i, j)] = m2;
          G[1][I(i, j)] = m2 * uu - txy;
          G[2][I(i, j)] = m2 * vv + pp - tyy;
          G[3][I(i, j)] = (E + pp) * vv - (uu * txy + vv * tyy) - kap * thy;
        }
      }
    for (int q = 0; q < 4; ++q)
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i)
          kk[((size_t)q * B + j) * B + i] = -(dx(F[q], i, j) + dy(G[q], i, j));
  }
  // Compressible Navier-Stokes in the skew-symmetric form of Reiss & Sesterhenn
  // (2014), the formulation Sec. 4 names, on the square-root variables
  // q = (phi, psi_x, psi_y, p) with phi = sqrt(rho), psi = phi u:
  //   d phi/dt   = -1/2 sum_j (D_j psi_j + u_j D_j phi)
  //   d psi_i/dt = -1/2 sum_j (D_j(psi_i u_j) + u_j D_j psi_i) - (D_i p - sum_j D_j tau_ij) / phi
  //   d p/dt     = -gamma sum_j D_j(p u_j) + (gamma - 1) sum_j u_j D_j p
  //                + (gamma - 1) (Phi + sum_j D_j(kap D_j th)),
  // tau as in the flux form, Phi = sum_ij tau_ij D_j u_i, th = p / rho,
  // kap = mu gamma / ((gamma - 1) Pr).  Each convective term is the mean of its
  // divergence and advective forms, so with the antisymmetric central D on a
  // periodic grid sum(phi^2), sum(phi psi), sum(p/(gamma-1) + psi.psi/2) are
  // conserved by the semi-discrete equations.  D is the 4th-order D1 throughout;
  // tau and kap D th are formed on nodes -2..B+1 and differentiated again.
  void rhs_ns_skew(const Leaf& b, std::vector<double>& kk) const {
    double gam = p.rhs[0], mu = p.rhs[1], Pr = p.rhs[2];
    double gm1 = gam - 1.0;
    double kap = mu * gam / ((gam - 1.0) * Pr);
    double c23 = 2.0 / 3.0;
    double c = cD(b.lvl);
    int R = B + 2 * g;
    auto I = [&](int i, int j) { return (size_t)(j + g) * R + (i + g); };
    std::vector<double> ph(R * R), sx(R * R), sy(R * R), pr(R * R), u(R * R), v(R * R), th(R * R);
    for (int j = -g; j < B + g; ++j)
      for (int i = -g; i < B + g; ++i) {
        double f = b.t[ix(0, i, j, 0)];
        ph[I(i, j)] = f;
        sx[I(i, j)] = b.t[ix(1, i, j, 0)];
        sy[I(i, j)] = b.t[ix(2, i, j, 0)];
        pr[I(i, j)] = b.t[ix(3, i, j, 0)];
        u[I(i, j)] = sx[I(i, j)] / f;
        v[I(i, j)] = sy[I(i, j)] / f;
        th[I(i, j)] = pr[I(i, j)] / (f * f);
      }
    auto dx = [&](const std::vector<double>& f, int i, int j) {
      return ((f[I(i - 2, j)] - f[I(i + 2, j)]) + 8.0 * (f[I(i + 1, j)] - f[I(i - 1, j)])) * c;
    };
    auto dy = [&](const std::vector<double>& f, int i, int j) {
      return ((f[I(i, j - 2)] - f[I(i, j + 2)]) + 8.0 * (f[I(i, j + 1)] - f[I(i, j - 1)])) * c;
    };
    // D1 of a product a*b of two tile arrays
    auto dxm = [&](const std::vector<double>& a, const std::vector<double>& bb, int i, int j) {
      auto m = [&](int s) { return a[I(i + s, j)] * bb[I(i + s, j)]; };
      return ((m(-2) - m(2)) + 8.0 * (m(1) - m(-1))) * c;
    };
    auto dym = [&](const std::vector<double>& a, const std::vector<double>& bb, int i, int j) {
      auto m = [&](int s) { return a[I(i, j + s)] * bb[I(i, j + s)]; };
      return ((m(-2) - m(2)) + 8.0 * (m(1) - m(-1))) * c;
    };
    // viscous stresses and heat flux on nodes -2..B+1 (only the cross of the
    // interior is used: x-derivatives on rows 0..B-1, y-derivatives on columns 0..B-1)
    std::vector<double> txx(R * R, 0.0), txy(R * R, 0.0), tyy(R * R, 0.0), qx(R * R, 0.0), qy(R * R, 0.0);
    for (int j = -2; j < B + 2; ++j)
      for (int i = -2; i < B + 2; ++i) {
        double ux = dx(u, i, j), vx = dx(v, i, j), uy = dy(u, i, j), vy = dy(v, i, j);
        double div = ux + vy;
        txx[I(i, j)] = mu * (2.0 * ux - c23 * div);
        tyy[I(i, j)] = mu * (2.0 * vy - c23 * div);
        txy[I(i, j)] = mu * (uy + vx);
        qx[I(i, j)] = kap * dx(th, i, j);
        qy[I(i, j)] = kap * dy(th, i, j);
      }
    size_t nb = (size_t)B * B;
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i) {
        double uu = u[I(i, j)], vv = v[I(i, j)], f = ph[I(i, j)];
        double phx = dx(ph, i, j), phy = dy(ph, i, j);
        double sxx = dx(sx, i, j), sxy_ = dy(sx, i, j), syx = dx(sy, i, j), syy = dy(sy, i, j);
        double px = dx(pr, i, j), py = dy(pr, i, j);
        double ux = dx(u, i, j), vx = dx(v, i, j), uy = dy(u, i, j), vy = dy(v, i, j);
        // mass
        double rphi = -0.5 * ((sxx + uu * phx) + (syy + vv * phy));
        // momentum
        double cx = (dxm(sx, u, i, j) + uu * sxx) + (dym(sx, v, i, j) + vv * sxy_);
        double cy = (dxm(sy, u, i, j) + uu * syx) + (dym(sy, v, i, j) + vv * syy);
        double fx = px - (dx(txx, i, j) + dy(txy, i, j));
        double fy = py - (dx(txy, i, j) + dy(tyy, i, j));
        double rsx = -0.5 * cx - fx / f;
        double rsy = -0.5 * cy - fy / f;
        // pressure
        double phi_v = (txx[I(i, j)] * ux + txy[I(i, j)] * (uy + vx)) + tyy[I(i, j)] * vy;
        double heat = dx(qx, i, j) + dy(qy, i, j);
        double rp = (-gam * (dxm(pr, u, i, j) + dym(pr, v, i, j)) + gm1 * (uu * px + vv * py)) +
                    gm1 * (phi_v + heat);
        size_t n = (size_t)j * B + i;
        kk[n] = rphi;
        kk[nb + n] = rsx;
        kk[2 * nb + n] = rsy;
        kk[3 * nb + n] = rp;
      }
  }
  // ------------------------------------------------ Navier-Stokes, 3D -----
  // The two formulations above in three dimensions (Sec. 5 names 3D runs as
  // the next step): q = (rho, rho u, rho v, rho w, E) for the flux form and
  // q = (phi, psi_x, psi_y, psi_z, p) for the skew-symmetric form, nvar = 5.
  // The equations are the 2D ones with the index sums running over three
  // axes.  Every sum over the axes is evaluated as ((x + y) + z) and every
  // sum over velocity components the same way, so a state that does not vary
  // along z and has w = 0 gives the 2D values bit for bit (the z terms are
  // exact zeros).  Tile arrays cover nodes -g..B+g-1 per axis; stresses and
  // fluxes are formed on nodes -2..B+1 per axis and differentiated again.
  size_t I3(int i, int j, int k) const {
    size_t R = (size_t)(B + 2 * g);
    return ((size_t)(k + g) * R + (size_t)(j + g)) * R + (size_t)(i + g);
  }
  // 4th-order D1 along axis a of a tile array, and of the product of two
  double D3(const std::vector<double>& f, int a, int i, int j, int k, double c) const {
    int o[3] = {0, 0, 0};
    o[a] = 1;
    auto at = [&](int s) { return f[I3(i + s * o[0], j + s * o[1], k + s * o[2])]; };
    return ((at(-2) - at(2)) + 8.0 * (at(1) - at(-1))) * c;
  }
  double D3m(const std::vector<double>& f, const std::vector<double>& h, int a, int i, int j, int k,
             double c) const {
    int o[3] = {0, 0, 0};
    o[a] = 1;
    auto m = [&](int s) {
      size_t q = I3(i + s * o[0], j + s * o[1], k + s * o[2]);
      return f[q] * h[q];
    };
    return ((m(-2) - m(2)) + 8.0 * (m(1) - m(-1))) * c;
  }
  // Viscous stress tau_ab = mu (D_b u_a + D_a u_b) - (2/3) mu div delta_ab at a node.
  void stress3(const std::vector<double>* vel, int i, int j, int k, double c, double mu,
               double du[3][3], double tau[3][3]) const {
    for (int a = 0; a < 3; ++a)
      for (int e = 0; e < 3; ++e) du[a][e] = D3(vel[a], e, i, j, k, c);
    double div = (du[0][0] + du[1][1]) + du[2][2];
    for (int a = 0; a < 3; ++a)
      for (int e = 0; e < 3; ++e)
        tau[a][e] = a == e ? mu * (2.0 * du[a][a] - (2.0 / 3.0) * div) : mu * (du[a][e] + du[e][a]);
  }
  // Flux form, 3D: N(q) = -sum_a D_a F_a,
  //   F_a = (rho u_a, rho u_a u_b + p delta_ab - tau_ab,
  //          (E + p) u_a - sum_b u_b tau_ab - kap D_a th).
  void rhs_ns3(const Leaf& b, std::vector<double>& kk) const {
    double gam = p.rhs[0], mu = p.rhs[1], Pr = p.rhs[2];
    double kap = mu * gam / ((gam - 1.0) * Pr);
    double c = cD(b.lvl);
    size_t R = (size_t)(B + 2 * g), RR = R * R * R;
    std::vector<double> vel[3], pr(RR), th(RR);
    for (int a = 0; a < 3; ++a) vel[a].assign(RR, 0.0);
    for (int k = -g; k < B + g; ++k)
      for (int j = -g; j < B + g; ++j)
        for (int i = -g; i < B + g; ++i) {
          double r = b.t[ix(0, i, j, k)], E = b.t[ix(4, i, j, k)];
          double m[3] = {b.t[ix(1, i, j, k)], b.t[ix(2, i, j, k)], b.t[ix(3, i, j, k)]};
          double uu = m[0] / r, vv = m[1] / r, ww = m[2] / r;
          double pp = (gam - 1.0) * (E - 0.5 * ((m[0] * uu + m[1] * vv) + m[2] * ww));
          size_t q = I3(i, j, k);
          vel[0][q] = uu; vel[1][q] = vv; vel[2][q] = ww;
          pr[q] = pp; th[q] = pp / r;
        }
    std::vector<double> F[3][5];
    for (int a = 0; a < 3; ++a)
      for (int v = 0; v < 5; ++v) F[a][v].assign(RR, 0.0);
    for (int k = -2; k < B + 2; ++k)
      for (int j = -2; j < B + 2; ++j)
        for (int i = -2; i < B + 2; ++i) {
          double du[3][3], tau[3][3];
          stress3(vel, i, j, k, c, mu, du, tau);
          size_t q = I3(i, j, k);
          double E = b.t[ix(4, i, j, k)];
          double m[3] = {b.t[ix(1, i, j, k)], b.t[ix(2, i, j, k)], b.t[ix(3, i, j, k)]};
          double uvw[3] = {vel[0][q], vel[1][q], vel[2][q]}, pp = pr[q];
          for (int a = 0; a < 3; ++a) {
            F[a][0][q] = m[a];
            for (int e = 0; e < 3; ++e)
              F[a][1 + e][q] = a == e ? (m[a] * uvw[e] + pp) - tau[a][e] : m[a] * uvw[e] - tau[a][e];
            double work = (uvw[0] * tau[a][0] + uvw[1] * tau[a][1]) + uvw[2] * tau[a][2];
            F[a][4][q] = ((E + pp) * uvw[a] - work) - kap * D3(th, a, i, j, k, c);
          }
        }
    size_t nb = (size_t)B * B * B;
    for (int v = 0; v < 5; ++v)
      for (int k = 0; k < B; ++k)
        for (int j = 0; j < B; ++j)
          for (int i = 0; i < B; ++i)
            kk[v * nb + ((size_t)k * B + j) * B + i] =
                -((D3(F[0][v], 0, i, j, k, c) + D3(F[1][v], 1, i, j, k, c)) + D3(F[2][v], 2, i, j, k, c));
  }
  // Skew-symmetric form, 3D, on (phi, psi, p): the 2D equations with
  // j = x, y, z in every sum, Phi = sum_ij tau_ij D_j u_i.
  void rhs_ns_skew3(const Leaf& b, std::vector<double>& kk) const {
    double gam = p.rhs[0], mu = p.rhs[1], Pr = p.rhs[2];
    double gm1 = gam - 1.0;
    double kap = mu * gam / ((gam - 1.0) * Pr);
    double c = cD(b.lvl);
    size_t R = (size_t)(B + 2 * g), RR = R * R * R;
    std::vector<double> ph(RR), ps[3], pr(RR), vel[3], th(RR);
    for (int a = 0; a < 3; ++a) { ps[a].assign(RR, 0.0); vel[a].assign(RR, 0.0); }
    for (int k = -g; k < B + g; ++k)
      for (int j = -g; j < B + g; ++j)
        for (int i = -g; i < B + g; ++i) {
          size_t q = I3(i, j, k);
          double f = b.t[ix(0, i, j, k)];
          ph[q] = f;
          for (int a = 0; a < 3; ++a) {
            ps[a][q] = b.t[ix(1 + a, i, j, k)];
            vel[a][q] = ps[a][q] / f;
          }
          pr[q] = b.t[ix(4, i, j, k)];
          th[q] = pr[q] / (f * f);
        }
    // stresses and heat flux kap D th on nodes -2..B+1
    std::vector<double> tau[3][3], qh[3];
    for (int a = 0; a < 3; ++a) {
      qh[a].assign(RR, 0.0);
      for (int e = 0; e < 3; ++e) tau[a][e].assign(RR, 0.0);
    }
    for (int k = -2; k < B + 2; ++k)
      for (int j = -2; j < B + 2; ++j)
        for (int i = -2; i < B + 2; ++i) {
          double du[3][3], t3[3][3];
          stress3(vel, i, j, k, c, mu, du, t3);
          size_t q = I3(i, j, k);
          for (int a = 0; a < 3; ++a) {
            for (int e = 0; e < 3; ++e) tau[a][e][q] = t3[a][e];
            qh[a][q] = kap * D3(th, a, i, j, k, c);
          }
        }
    size_t nb = (size_t)B * B * B;
    for (int k = 0; k < B; ++k)
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i) {
          size_t q = I3(i, j, k);
          double f = ph[q], u[3] = {vel[0][q], vel[1][q], vel[2][q]};
          double dph[3], dp[3], ds[3][3], du[3][3];
          for (int a = 0; a < 3; ++a) {
            dph[a] = D3(ph, a, i, j, k, c);
            dp[a] = D3(pr, a, i, j, k, c);
            for (int e = 0; e < 3; ++e) {
              ds[a][e] = D3(ps[a], e, i, j, k, c);
              du[a][e] = D3(vel[a], e, i, j, k, c);
            }
          }
          // mass
          double rphi = -0.5 * (((ds[0][0] + u[0] * dph[0]) + (ds[1][1] + u[1] * dph[1])) +
                                (ds[2][2] + u[2] * dph[2]));
          // momentum
          double rps[3];
          for (int a = 0; a < 3; ++a) {
            double conv = ((D3m(ps[a], vel[0], 0, i, j, k, c) + u[0] * ds[a][0]) +
                           (D3m(ps[a], vel[1], 1, i, j, k, c) + u[1] * ds[a][1])) +
                          (D3m(ps[a], vel[2], 2, i, j, k, c) + u[2] * ds[a][2]);
            double visc = (D3(tau[a][0], 0, i, j, k, c) + D3(tau[a][1], 1, i, j, k, c)) +
                          D3(tau[a][2], 2, i, j, k, c);
            double fa = dp[a] - visc;
            rps[a] = -0.5 * conv - fa / f;
          }
          // pressure
          double t00 = tau[0][0][q], t01 = tau[0][1][q], t11 = tau[1][1][q];
          double t02 = tau[0][2][q], t12 = tau[1][2][q], t22 = tau[2][2][q];
          double phi_v = ((t00 * du[0][0] + t01 * (du[0][1] + du[1][0])) + t11 * du[1][1]) +
                         ((t02 * (du[0][2] + du[2][0]) + t12 * (du[1][2] + du[2][1])) + t22 * du[2][2]);
          double heat = (D3(qh[0], 0, i, j, k, c) + D3(qh[1], 1, i, j, k, c)) + D3(qh[2], 2, i, j, k, c);
          double dpu = (D3m(pr, vel[0], 0, i, j, k, c) + D3m(pr, vel[1], 1, i, j, k, c)) +
                       D3m(pr, vel[2], 2, i, j, k, c);
          double adv = (u[0] * dp[0] + u[1] * dp[1]) + u[2] * dp[2];
          double rp = (-gam * dpu + gm1 * adv) + gm1 * (phi_v + heat);
          size_t n = ((size_t)k * B + j) * B + i;
          kk[n] = rphi;
          for (int a = 0; a < 3; ++a) kk[(1 + a) * nb + n] = rps[a];
          kk[4 * nb + n] = rp;
        }
  }
  void rhs(const Leaf& b, double ts, std::vector<double>& kk) const {
    if (p.rhs_kind == 2) {
      if (d == 3) rhs_ns3(b, kk);
      else rhs_ns(b, kk);
    } else if (p.rhs_kind == 3) {
      if (d == 3) rhs_ns_skew3(b, kk);
      else rhs_ns_skew(b, kk);
    } else rhs_advection(b, ts, kk);
  }

  // ------------------------------------------------------- shock filter -----
  // Shock-capturing filter of Bogey, de Cacqueray & Bailly (2009), applied
  // after every time step (Sec. 4, threshold r_th = rhs[3]) to each evolved
  // variable q of a Navier-Stokes state, on the synchronised tile.  Per
  // direction a and node n along a:
  //   dilatation  th_n = (u_{n+1} - u_{n-1}) / (2 dx) + (v_{n+1} - v_{n-1}) / (2 dx)
  //               (2nd-order central differences, each along its own axis)
  //   high-pass   Dth_n = (-th_{n+1} + 2 th_n - th_{n-1}) / 4
  //   magnitude   M_n = ((Dth_n - Dth_{n+1})^2 + (Dth_n - Dth_{n-1})^2) / 2
  //   sensor      r_n = M_n / (c_n^2 / dx^2) + 1e-16,  c^2 = gamma p / rho
  //   strength    s_n = (1 - r_th / r_n + |1 - r_th / r_n|) / 2
  //   flux        F_{n+1/2} = -(q_{n+1} - q_n) / 4  (standard 2nd-order filter)
  //   update      q_n <- q_n - sum_a (s_{n+1/2} F_{n+1/2} - s_{n-1/2} F_{n-1/2}),
  //               s_{n+1/2} = (s_n + s_{n+1}) / 2,
  // both directions evaluated from the unfiltered state.  The stencil reaches
  // four nodes along a and one across, inside the ghost layer.
  void filter() {
    double rth = p.rhs[3];
    if (!(rth > 0.0) || (p.rhs_kind != 2 && p.rhs_kind != 3)) return;
    sync();
    if (d == 3) {
      filter3();
      return;
    }
    double gam = p.rhs[0];
    int R = B + 2 * g;
    auto I = [&](int i, int j) { return (size_t)(j + g) * R + (i + g); };
    std::map<Key, std::vector<double>> out;
    for (auto& kv : lv) {
      const Leaf& b = kv.second;
      double dxl = p.L / (double)((int64_t)(B - 1) << b.lvl);
      std::vector<double> u(R * R), v(R * R), cc(R * R);
      for (int j = -g; j < B + g; ++j)
        for (int i = -g; i < B + g; ++i) {
          double q0 = b.t[ix(0, i, j, 0)], q1 = b.t[ix(1, i, j, 0)], q2 = b.t[ix(2, i, j, 0)],
                 q3 = b.t[ix(3, i, j, 0)];
          double rho, pp;
          if (p.rhs_kind == 2) {
            rho = q0;
            u[I(i, j)] = q1 / q0;
            v[I(i, j)] = q2 / q0;
            pp = (gam - 1.0) * (q3 - 0.5 * (q1 * u[I(i, j)] + q2 * v[I(i, j)]));
          } else {
            rho = q0 * q0;
            u[I(i, j)] = q1 / q0;
            v[I(i, j)] = q2 / q0;
            pp = q3;
          }
          cc[I(i, j)] = gam * pp / rho;
        }
      double h2 = 0.5 / dxl;
      auto theta = [&](int i, int j) {
        return (u[I(i + 1, j)] - u[I(i - 1, j)]) * h2 + (v[I(i, j + 1)] - v[I(i, j - 1)]) * h2;
      };
      // strength at node (i, j) for direction a (0: x, 1: y)
      auto strength = [&](int a, int i, int j) {
        int ox = a == 0 ? 1 : 0, oy = a == 1 ? 1 : 0;
        auto Dth = [&](int s) {
          int ii = i + s * ox, jj = j + s * oy;
          return (-theta(ii + ox, jj + oy) + 2.0 * theta(ii, jj) - theta(ii - ox, jj - oy)) / 4.0;
        };
        double d0 = Dth(0), dp = Dth(1), dm = Dth(-1);
        double M = 0.5 * ((d0 - dp) * (d0 - dp) + (d0 - dm) * (d0 - dm));
        double r = M / (cc[I(i, j)] / (dxl * dxl)) + 1e-16;
        double z = 1.0 - rth / r;
        return 0.5 * (z + std::fabs(z));
      };
      std::vector<double> sgx(R * R, 0.0), sgy(R * R, 0.0);
      for (int j = -1; j <= B; ++j)
        for (int i = -1; i <= B; ++i) {
          if (j >= 0 && j < B) sgx[I(i, j)] = strength(0, i, j);
          if (i >= 0 && i < B) sgy[I(i, j)] = strength(1, i, j);
        }
      std::vector<double> nt = b.t;
      for (int var = 0; var < nv; ++var)
        for (int j = 0; j < B; ++j)
          for (int i = 0; i < B; ++i) {
            auto q = [&](int ii, int jj) { return b.t[ix(var, ii, jj, 0)]; };
            double sxp = 0.5 * (sgx[I(i, j)] + sgx[I(i + 1, j)]);
            double sxm = 0.5 * (sgx[I(i - 1, j)] + sgx[I(i, j)]);
            double syp = 0.5 * (sgy[I(i, j)] + sgy[I(i, j + 1)]);
            double sym = 0.5 * (sgy[I(i, j - 1)] + sgy[I(i, j)]);
            double fxp = -0.25 * (q(i + 1, j) - q(i, j)), fxm = -0.25 * (q(i, j) - q(i - 1, j));
            double fyp = -0.25 * (q(i, j + 1) - q(i, j)), fym = -0.25 * (q(i, j) - q(i, j - 1));
            double ddx = sxp * fxp - sxm * fxm;
            double ddy = syp * fyp - sym * fym;
            nt[ix(var, i, j, 0)] = q(i, j) - (ddx + ddy);
          }
      out[kv.first] = nt;
    }
    for (auto& kv : lv) kv.second.t = out[kv.first];
  }

  // The same filter in 3D: the dilatation sums the three central differences,
  // ((du/dx + dv/dy) + dw/dz), and the update the three directions,
  // q_n <- q_n - ((dd_x + dd_y) + dd_z); a state that does not vary along z
  // with w = 0 is filtered exactly as in 2D (the z strength is zero).
  void filter3() {
    double rth = p.rhs[3], gam = p.rhs[0];
    size_t R = (size_t)(B + 2 * g), RR = R * R * R;
    std::map<Key, std::vector<double>> out;
    for (auto& kv : lv) {
      const Leaf& b = kv.second;
      double dxl = p.L / (double)((int64_t)(B - 1) << b.lvl);
      std::vector<double> vel[3], cc(RR);
      for (int a = 0; a < 3; ++a) vel[a].assign(RR, 0.0);
      for (int k = -g; k < B + g; ++k)
        for (int j = -g; j < B + g; ++j)
          for (int i = -g; i < B + g; ++i) {
            size_t q = I3(i, j, k);
            double q0 = b.t[ix(0, i, j, k)], q4 = b.t[ix(4, i, j, k)];
            double m[3] = {b.t[ix(1, i, j, k)], b.t[ix(2, i, j, k)], b.t[ix(3, i, j, k)]};
            for (int a = 0; a < 3; ++a) vel[a][q] = m[a] / q0;
            double rho, pp;
            if (p.rhs_kind == 2) {
              rho = q0;
              pp = (gam - 1.0) * (q4 - 0.5 * ((m[0] * vel[0][q] + m[1] * vel[1][q]) + m[2] * vel[2][q]));
            } else {
              rho = q0 * q0;
              pp = q4;
            }
            cc[q] = gam * pp / rho;
          }
      double h2 = 0.5 / dxl;
      auto theta = [&](int i, int j, int k) {
        return ((vel[0][I3(i + 1, j, k)] - vel[0][I3(i - 1, j, k)]) * h2 +
                (vel[1][I3(i, j + 1, k)] - vel[1][I3(i, j - 1, k)]) * h2) +
               (vel[2][I3(i, j, k + 1)] - vel[2][I3(i, j, k - 1)]) * h2;
      };
      // strength at node (i, j, k) for direction a
      auto strength = [&](int a, int i, int j, int k) {
        int o[3] = {0, 0, 0};
        o[a] = 1;
        auto Dth = [&](int s) {
          int ii = i + s * o[0], jj = j + s * o[1], kk = k + s * o[2];
          return (-theta(ii + o[0], jj + o[1], kk + o[2]) + 2.0 * theta(ii, jj, kk) -
                  theta(ii - o[0], jj - o[1], kk - o[2])) / 4.0;
        };
        double d0 = Dth(0), dp = Dth(1), dm = Dth(-1);
        double M = 0.5 * ((d0 - dp) * (d0 - dp) + (d0 - dm) * (d0 - dm));
        double r = M / (cc[I3(i, j, k)] / (dxl * dxl)) + 1e-16;
        double z = 1.0 - rth / r;
        return 0.5 * (z + std::fabs(z));
      };
      // strengths along a on nodes -1..B along a and 0..B-1 across
      std::vector<double> sg[3];
      for (int a = 0; a < 3; ++a) sg[a].assign(RR, 0.0);
      for (int k = -1; k <= B; ++k)
        for (int j = -1; j <= B; ++j)
          for (int i = -1; i <= B; ++i) {
            int ijk[3] = {i, j, k};
            for (int a = 0; a < 3; ++a) {
              bool inside = true;
              for (int e = 0; e < 3; ++e)
                if (e != a && (ijk[e] < 0 || ijk[e] >= B)) inside = false;
              if (inside) sg[a][I3(i, j, k)] = strength(a, i, j, k);
            }
          }
      std::vector<double> nt = b.t;
      for (int var = 0; var < nv; ++var)
        for (int k = 0; k < B; ++k)
          for (int j = 0; j < B; ++j)
            for (int i = 0; i < B; ++i) {
              double dd[3];
              for (int a = 0; a < 3; ++a) {
                int o[3] = {0, 0, 0};
                o[a] = 1;
                auto q = [&](int s) { return b.t[ix(var, i + s * o[0], j + s * o[1], k + s * o[2])]; };
                auto sa = [&](int s) { return sg[a][I3(i + s * o[0], j + s * o[1], k + s * o[2])]; };
                double sp = 0.5 * (sa(0) + sa(1)), sm = 0.5 * (sa(-1) + sa(0));
                double fp = -0.25 * (q(1) - q(0)), fm = -0.25 * (q(0) - q(-1));
                dd[a] = sp * fp - sm * fm;
              }
              nt[ix(var, i, j, k)] = b.t[ix(var, i, j, k)] - ((dd[0] + dd[1]) + dd[2]);
            }
      out[kv.first] = nt;
    }
    for (auto& kv : lv) kv.second.t = out[kv.first];
  }

  // ------------------------------------------------------------------ RK4 ---
  // Classic 4-stage Runge-Kutta (Sec. 3, Sec. 4) on every block; before each
  // stage the ghost nodes of the stage field are synchronised.  y_n is taken
  // after the first synchronisation (so its conditional nodes already hold the
  // finer blocks' values):
  //   k1 = N(y_n),            acc = y_n + dt/6 k1,  Y2 = y_n + dt/2 k1
  //   k2 = N(Y2, t+dt/2),     acc += dt/3 k2,       Y3 = y_n + dt/2 k2
  //   k3 = N(Y3, t+dt/2),     acc += dt/3 k3,       Y4 = y_n + dt k3
  //   k4 = N(Y4, t+dt),       y_{n+1} = acc + dt/6 k4
  void rk4(double t, double dt) {
    double c6 = dt / 6.0, c3 = dt / 3.0, c2 = dt / 2.0;
    size_t nb = (d == 3 ? (size_t)B * B * B : (size_t)B * B);
    std::map<Key, std::vector<double>> yn, acc;
    std::vector<double> kk(nb * nv);
    double ts[4] = {t, t + 0.5 * dt, t + 0.5 * dt, t + dt};
    for (int s = 0; s < 4; ++s) {
      sync();
      std::map<Key, std::vector<double>> knew;
      for (auto& kv : lv) {
        rhs(kv.second, ts[s], kk);
        knew[kv.first] = kk;
      }
      for (auto& kv : lv) {
        Leaf& b = kv.second;
        std::vector<double>& k = knew[kv.first];
        if (s == 0) {
          std::vector<double>& y = yn[kv.first];
          std::vector<double>& a = acc[kv.first];
          y.resize(nb * nv); a.resize(nb * nv);
          for (int v = 0; v < nv; ++v)
            for (size_t q = 0; q < nb; ++q) {
              size_t i = q % B, j = (q / B) % B, kz = q / ((size_t)B * B);
              y[v * nb + q] = b.t[ix(v, (int)i, (int)j, (int)kz)];
            }
        }
        std::vector<double>& y = yn[kv.first];
        std::vector<double>& a = acc[kv.first];
        for (int v = 0; v < nv; ++v)
          for (size_t q = 0; q < nb; ++q) {
            size_t i = q % B, j = (q / B) % B, kz = q / ((size_t)B * B);
            size_t at = ix(v, (int)i, (int)j, (int)kz), n = v * nb + q;
            double kq = k[n];
            if (s == 0) { a[n] = y[n] + c6 * kq; b.t[at] = y[n] + c2 * kq; }
            else if (s == 1) { a[n] = a[n] + c3 * kq; b.t[at] = y[n] + c2 * kq; }
            else if (s == 2) { a[n] = a[n] + c3 * kq; b.t[at] = y[n] + dt * kq; }
            else b.t[at] = a[n] + c6 * kq;
          }
      }
    }
  }

  // --------------------------------------------------------------- step -----
  // One multiresolution time step (Sec. 2.1): refine all blocks by one level
  // (safety zone), evolve with synchronised ghosts, coarsen.  Load balancing is
  // a no-op on one address space.
  void step(double t, double dt) {
    refine(0);
    rk4(t, dt);
    filter();
    coarsen_until_stable();
  }

  // ------------------------------------------------------------ export ------
  std::vector<Leaf*> ordered() {
    std::vector<std::pair<uint64_t, Leaf*>> v;
    for (auto& kv : lv) {
      Leaf& b = kv.second;
      int64_t cell[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) cell[a] = b.c[a] << (p.Jmax - b.lvl);
      v.push_back({hilbert_key(d, p.Jmax, cell), &b});
    }
    std::sort(v.begin(), v.end(), [](auto& x, auto& y) { return x.first < y.first; });
    std::vector<Leaf*> out;
    for (auto& e : v) out.push_back(e.second);
    return out;
  }
};

}  // namespace

extern "C" {

void* orc_create(const orc_params* p) { return new Tree(*p); }
void orc_destroy(void* h) { delete (Tree*)h; }
int64_t orc_nblocks(void* h) { return (int64_t)((Tree*)h)->lv.size(); }
void orc_init_tree(void* h) { ((Tree*)h)->init_tree(); }
void orc_sync(void* h) { ((Tree*)h)->sync(); }
void orc_refine(void* h, int mode) { ((Tree*)h)->refine(mode); }
void orc_rk4(void* h, double t, double dt) { ((Tree*)h)->rk4(t, dt); }
void orc_details(void* h) { ((Tree*)h)->details(); }
int orc_flags(void* h, uint64_t seed) { return ((Tree*)h)->flags(seed); }
int orc_coarsen(void* h) { return ((Tree*)h)->coarsen(); }
int orc_coarsen_until_stable(void* h) { return ((Tree*)h)->coarsen_until_stable(); }
void orc_step(void* h, double t, double dt) { ((Tree*)h)->step(t, dt); }
int orc_nrel(void* h) { return (int)((Tree*)h)->relations().size(); }
int64_t orc_errors(void* h) { return ((Tree*)h)->err; }
uint64_t orc_hilbert(int dim, int bits, const int64_t* cell) { return hilbert_key(dim, bits, cell); }

// Blocks in Hilbert order: level, block coordinates, treecode, Hilbert key,
// flag, largest detail; fields (nullable): interior nodes, [block][var][z][y][x].
void orc_get_blocks(void* h, int32_t* lvl, int64_t* crd, uint64_t* tc, uint64_t* hk,
                    int8_t* flag, double* mdet, double* fields) {
  Tree* T = (Tree*)h;
  std::vector<Leaf*> o = T->ordered();
  int B = T->B, d = T->d;
  size_t nb = d == 3 ? (size_t)B * B * B : (size_t)B * B;
  for (size_t n = 0; n < o.size(); ++n) {
    Leaf& b = *o[n];
    if (lvl) lvl[n] = b.lvl;
    if (crd) for (int a = 0; a < 3; ++a) crd[3 * n + a] = b.c[a];
    if (tc) tc[n] = treecode(d, b.c, b.lvl);
    if (hk) {
      int64_t cell[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) cell[a] = b.c[a] << (T->p.Jmax - b.lvl);
      hk[n] = hilbert_key(d, T->p.Jmax, cell);
    }
    if (flag) flag[n] = (int8_t)b.flag;
    if (mdet) mdet[n] = b.mdet;
    if (fields)
      for (int v = 0; v < T->nv; ++v)
        for (size_t q = 0; q < nb; ++q) {
          int i = (int)(q % B), j = (int)((q / B) % B), k = (int)(q / ((size_t)B * B));
          fields[(n * T->nv + v) * nb + q] = b.t[T->ix(v, i, j, k)];
        }
  }
}
// Full tiles (ghosts included) in Hilbert order: [block][var][z][y][x], T = B + 2g.
void orc_get_tiles(void* h, double* tiles) {
  Tree* T = (Tree*)h;
  std::vector<Leaf*> o = T->ordered();
  size_t ts = T->tsize();
  for (size_t n = 0; n < o.size(); ++n) std::memcpy(tiles + n * ts, o[n]->t.data(), ts * sizeof(double));
}
// Replace the tree by the given leaves (interior values; ghosts zero).
void orc_set_blocks(void* h, int64_t n, const int32_t* lvl, const int64_t* crd, const double* fields) {
  Tree* T = (Tree*)h;
  T->lv.clear();
  int B = T->B, d = T->d;
  size_t nb = d == 3 ? (size_t)B * B * B : (size_t)B * B;
  for (int64_t q = 0; q < n; ++q) {
    Leaf b;
    b.lvl = lvl[q];
    for (int a = 0; a < 3; ++a) b.c[a] = crd[3 * q + a];
    b.t.assign(T->tsize(), 0.0);
    if (fields)
      for (int v = 0; v < T->nv; ++v)
        for (size_t r = 0; r < nb; ++r) {
          int i = (int)(r % B), j = (int)((r / B) % B), k = (int)(r / ((size_t)B * B));
          b.t[T->ix(v, i, j, k)] = fields[(q * T->nv + v) * nb + r];
        }
    T->lv[T->key(b.lvl, b.c)] = b;
  }
}
// Refinement statuses of the blocks, given in Hilbert order (replay of
// externally decided flags, e.g. a proposal of refinement indicators).
void orc_set_flags(void* h, const int8_t* flag) {
  std::vector<Leaf*> o = ((Tree*)h)->ordered();
  for (size_t n = 0; n < o.size(); ++n) o[n]->flag = flag[n];
}
// Largest details of the blocks, given in Hilbert order (replaces details()
// when the flag rule is examined on its own).
void orc_set_mdet(void* h, const double* mdet) {
  std::vector<Leaf*> o = ((Tree*)h)->ordered();
  for (size_t n = 0; n < o.size(); ++n) o[n]->mdet = mdet[n];
}
int orc_close_refine(void* h) { return ((Tree*)h)->close_refine(); }
// Analytic initial field on the current blocks (advected by t for constant u).
void orc_set_ic(void* h, double t) {
  Tree* T = (Tree*)h;
  for (auto& kv : T->lv) T->set_ic(kv.second, t);
}
// Neighbour table in Hilbert order: nbr[n*R + r] = export index or -1, dl level difference.
void orc_neighbors(void* h, int32_t* nbr, int8_t* dl) {
  Tree* T = (Tree*)h;
  std::vector<Leaf*> o = T->ordered();
  std::map<const Leaf*, int32_t> idx;
  for (size_t n = 0; n < o.size(); ++n) idx[o[n]] = (int32_t)n;
  auto rel = T->relations();
  for (size_t n = 0; n < o.size(); ++n)
    for (size_t r = 0; r < rel.size(); ++r) {
      int l = 0;
      Leaf* f = T->neighbour(*o[n], rel[r], &l);
      nbr[n * rel.size() + r] = f ? idx[f] : -1;
      dl[n * rel.size() + r] = f ? (int8_t)l : 0;
    }
}
// Shock-capturing filter of the Navier-Stokes state (no-op unless r_th > 0).
void orc_filter(void* h) { ((Tree*)h)->filter(); }
// Right-hand side N(q) on the interior of every block after a sync, Hilbert order.
void orc_rhs(void* h, double t, double* out) {
  Tree* T = (Tree*)h;
  T->sync();
  std::vector<Leaf*> o = T->ordered();
  int B = T->B;
  size_t nb = T->d == 3 ? (size_t)B * B * B : (size_t)B * B;
  std::vector<double> kk(nb * T->nv);
  for (size_t n = 0; n < o.size(); ++n) {
    T->rhs(*o[n], t, kk);
    std::memcpy(out + n * nb * T->nv, kk.data(), kk.size() * sizeof(double));
  }
}
// Error against the analytic field advected by constant u over time t (unique
// nodes: the last node of each block per axis is dropped, weights dx^d):
// out = {L2 abs, L2 of exact, Linf abs, Linf of exact}.
void orc_error(void* h, double t, double* out) {
  Tree* T = (Tree*)h;
  int B = T->B, d = T->d;
  double e2 = 0, x2 = 0, ei = 0, xi = 0;
  for (auto& kv : T->lv) {
    Leaf& b = kv.second;
    Leaf ex = b;
    T->set_ic(ex, t);
    double dx = T->p.L / (double)((int64_t)(B - 1) << b.lvl);
    double w = d == 3 ? dx * dx * dx : dx * dx;
    for (int k = 0; k < (d == 3 ? B - 1 : 1); ++k)
      for (int j = 0; j < B - 1; ++j)
        for (int i = 0; i < B - 1; ++i) {
          double a = b.t[T->ix(0, i, j, k)], e = ex.t[T->ix(0, i, j, k)];
          e2 += w * (a - e) * (a - e); x2 += w * e * e;
          ei = std::max(ei, std::fabs(a - e)); xi = std::max(xi, std::fabs(e));
        }
  }
  out[0] = std::sqrt(e2); out[1] = std::sqrt(x2); out[2] = ei; out[3] = xi;
}

}  // extern "C"

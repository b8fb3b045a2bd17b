// Device building blocks of the multiresolution step (templated on the block
// geometry).  Included by the per-dimension kernel translation units.
//
// Central idea: the pool stores only block interiors (Bs^d nodes per variable);
// every kernel that needs a block with its ghost layer builds the synchronised
// tile in shared memory directly from the neighbours' interiors ("gather").
// The paper fills ghosts in two passes (copies/injection first, then
// coarse-to-fine prediction by ascending level, Sec. 2.5).  On a graded tree
// every coarse node that a prediction stencil of a ghost node touches lies in
// a leaf of level >= l-1 that is a node there, so the second pass never needs
// another predicted value: one pass over interiors gives the same values.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mr_internal.h"

namespace mr {

__device__ __forceinline__ int64_t pmod64(int64_t a, int64_t n) {
  int64_t r = a % n;
  return r < 0 ? r + n : r;
}
__device__ __forceinline__ int floordiv(int a, int b) {
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// Morton index of a cell = treecode digits (Sec. 2.2), x bit lowest.
template <int D>
__device__ __forceinline__ uint64_t morton(const int64_t c[3], int lvl) {
  uint64_t t = 0;
  for (int b = lvl - 1; b >= 0; --b)
    for (int a = D - 1; a >= 0; --a) t = (t << 1) | (uint64_t)((c[a] >> b) & 1);
  return t;
}

// Hilbert index (J. Skilling, AIP Conf. Proc. 707, 381 (2004)): inverse undo of
// the axis exchanges, Gray encoding, then bit interleave of the transpose.
template <int D>
__device__ __forceinline__ uint64_t hilbert(const int64_t cell[3], int bits) {
  if (bits == 0) return 0;
  uint32_t X[3] = {(uint32_t)cell[0], (uint32_t)cell[1], D == 3 ? (uint32_t)cell[2] : 0u};
  const uint32_t M = 1u << (bits - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    const uint32_t P = Q - 1;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (X[i] & Q) {
        X[0] ^= P;
      } else {
        uint32_t t = (X[0] ^ X[i]) & P;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
#pragma unroll
  for (int i = 1; i < D; ++i) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (X[D - 1] & Q) t ^= Q - 1;
#pragma unroll
  for (int i = 0; i < D; ++i) X[i] ^= t;
  uint64_t h = 0;
  for (int b = bits - 1; b >= 0; --b)
#pragma unroll
    for (int i = 0; i < D; ++i) h = (h << 1) | ((X[i] >> b) & 1u);
  return h;
}

template <int D>
__device__ __forceinline__ uint64_t block_key(const int32_t* c, int lvl, int Jmax) {
  int64_t cell[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) cell[a] = (int64_t)c[a] << (Jmax - lvl);
  return hilbert<D>(cell, Jmax);
}

// Slot of the leaf with block coordinates c at level m (periodic wrap), or -1.
template <int D>
__device__ __forceinline__ int tab_get(const PoolView& pv, const TreeDev& td, int m,
                                       const int64_t c[3]) {
  if (m < td.Jmin || m > td.Jmax) return -1;
  int64_t w[3] = {0, 0, 0};
  const int64_t n = (int64_t)1 << m;
  for (int a = 0; a < D; ++a) w[a] = pmod64(c[a], n);
  return pv.tab[td.tab_off[m] + (int64_t)morton<D>(w, m)];
}

template <int D, int B>
struct Geo {
  static constexpr int G = kG;
  static constexpr int T = B + 2 * G;
  static constexpr int TZ = D == 3 ? T : 1;
  static constexpr int GZ = D == 3 ? G : 0;
  static constexpr int BZ = D == 3 ? B : 1;
  static constexpr int TILE = T * T * TZ;
  static constexpr int NI = B * B * BZ;
  static constexpr int NR = D == 3 ? 64 : 16;  // ring of level l+1 cells, [-1,2]^d
  static constexpr int NCH = 1 << D;
  static_assert(G + 2 < (B - 1) / 2, "prediction stencils of ghosts must stay in the ring");
  __device__ static __forceinline__ int tix(int i, int j, int k) {
    return ((k + GZ) * T + (j + G)) * T + (i + G);
  }
  __device__ static __forceinline__ int lin(int i, int j, int k) { return (k * B + j) * B + i; }
};

struct BlockInfo {
  int slot, lvl, tree;
  int64_t c[3];
};

__device__ __forceinline__ BlockInfo load_block(const PoolView& pv, int slot) {
  BlockInfo b;
  b.slot = slot;
  b.lvl = pv.lvl[slot];
  b.tree = pv.tree[slot];
  for (int a = 0; a < 3; ++a) b.c[a] = pv.crd[3 * slot + a];
  return b;
}

__device__ __forceinline__ void set_err(const PoolView& pv, int bits) {
  atomicOr(&pv.cnt->err, bits);
}

// Ring map: for every level-(l+1) cell q in [-1,2]^d around the block (its own
// 2^d child cells included) the leaf covering it, searched at l+1, l, l-1.
// These are exactly the 16 (2D) / 74 (3D) relations of Sec. 2.2 seen cell by
// cell.  A cell covered by no leaf in that range means a non-graded tree.
template <int D, int B>
__device__ void build_ring(const PoolView& pv, const TreeDev& td, const BlockInfo& b,
                           int* rslot, int8_t* rlvl) {
  using Gm = Geo<D, B>;
  for (int r = threadIdx.x; r < Gm::NR; r += blockDim.x) {
    const int q[3] = {r % 4 - 1, (r / 4) % 4 - 1, r / 16 - 1};
    bool inside = true;
    for (int a = 0; a < D; ++a) inside &= (q[a] == 0 || q[a] == 1);
    if (inside) {
      rslot[r] = b.slot;
      rlvl[r] = (int8_t)b.lvl;
      continue;
    }
    const int64_t nl1 = (int64_t)1 << (b.lvl + 1);
    int64_t cell[3] = {0, 0, 0}, c1[3] = {0, 0, 0}, c2[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
      cell[a] = pmod64(2 * b.c[a] + q[a], nl1);
      c1[a] = cell[a] >> 1;
      c2[a] = cell[a] >> 2;
    }
    int s = tab_get<D>(pv, td, b.lvl + 1, cell), m = b.lvl + 1;
    if (s < 0) { s = tab_get<D>(pv, td, b.lvl, c1); m = b.lvl; }
    if (s < 0) { s = tab_get<D>(pv, td, b.lvl - 1, c2); m = b.lvl - 1; }
    if (s < 0) {
      set_err(pv, kErrGraded);
      m = -1;
    }
    rslot[r] = s;
    rlvl[r] = (int8_t)m;
  }
}

// Owner of a point: among the leaves whose closed cell contains the point (found
// through the ring), the finest; among equal levels the one in which the point
// is the upper edge node on the fewest leading axes (combo order).  Point given
// in level-(l+1) node units relative to the block origin.  off[] receives the
// point's offset inside the owner, again in level-(l+1) units.
struct Own {
  int slot, m, combo;
  int off[3];
};

template <int D, int B>
__device__ __forceinline__ bool owner(const BlockInfo& b, const int h[3], int min_m,
                                      const int* rslot, const int8_t* rlvl, Own& o) {
  int c0[3] = {0, 0, 0};
  bool onb[3] = {false, false, false};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    c0[a] = floordiv(h[a], B - 1);
    onb[a] = (h[a] - c0[a] * (B - 1)) == 0;
  }
  o.m = -1;
  o.combo = 1 << 30;
  const int l1 = b.lvl + 1;
  const int64_t N1 = (int64_t)(B - 1) << l1, n1 = (int64_t)1 << l1;
#pragma unroll
  for (int combo = 0; combo < (1 << D); ++combo) {
    bool ok = true;
    int q[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int bit = (combo >> a) & 1;
      if (bit && !onb[a]) ok = false;
      q[a] = c0[a] - bit;
      if (q[a] < -1 || q[a] > 2) ok = false;
    }
    if (!ok) continue;
    const int r = (q[0] + 1) + 4 * (q[1] + 1) + 16 * (D == 3 ? q[2] + 1 : 0);
    const int s = rslot[r], m = rlvl[r];
    if (s < 0 || m < min_m) continue;
    const int sh = l1 - m;
    int oc = 0, off[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int64_t cabs = pmod64(2 * b.c[a] + q[a], n1);
      const int64_t origin = ((cabs >> sh) * (B - 1)) << sh;
      const int64_t pabs = pmod64(2 * b.c[a] * (B - 1) + h[a], N1);
      const int64_t of = pmod64(pabs - origin, N1);
      off[a] = (int)of;
      if (of == ((int64_t)(B - 1) << sh)) oc |= 1 << a;
    }
    if (m > o.m || (m == o.m && oc < o.combo)) {
      o.m = m;
      o.combo = oc;
      o.slot = s;
#pragma unroll
      for (int a = 0; a < 3; ++a) o.off[a] = off[a];
    }
  }
  return o.m >= 0;
}

template <typename T>
__device__ __forceinline__ T dd4(T fm1, T f0, T f1, T f2) {
  // 4-point interpolating-wavelet midpoint prediction (Sec. 2.3, 4th order)
  return (T(9) * (f0 + f1) - (fm1 + f2)) * T(0.0625);
}

// Value of node `li` (local index at the owner's level) of variable v.
template <int D, int B, typename TF>
__device__ __forceinline__ TF pool_at(const PoolView& pv, const TF* F, int slot, int v,
                                      const int li[3]) {
  return F[((int64_t)slot * pv.nvar + v) * pv.vs + Geo<D, B>::lin(li[0], li[1], D == 3 ? li[2] : 0)];
}

// Ghost value predicted from a coarser owner f (level l-1).  Stencil nodes are
// f's tile values: f's own node, unless a finer leaf shares it (then the finer
// value, Sec. 2.2 rule 2); nodes outside f come from their own owner.
template <int D, int B, typename TF, typename TT>
__device__ TT predict_ghost(const PoolView& pv, const BlockInfo& b, const int h[3], const Own& f,
                            int v, const TF* F, const int* rslot, const int8_t* rlvl) {
  int base[3] = {0, 0, 0}, ns[3] = {1, 1, 1};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int q4 = f.off[a] >> 2;
    if ((f.off[a] & 3) == 2) { ns[a] = 4; base[a] = q4 - 1; }
    else base[a] = q4;
  }
  TT vx[4][4];
  for (int sz = 0; sz < ns[2]; ++sz)
    for (int sy = 0; sy < ns[1]; ++sy) {
      TT w[4];
      for (int sx = 0; sx < ns[0]; ++sx) {
        const int n[3] = {base[0] + sx, base[1] + sy, base[2] + sz};
        bool inside = true, strict = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          inside &= (n[a] >= 0 && n[a] <= B - 1);
          strict &= (n[a] >= 1 && n[a] <= B - 2);
        }
        TT val;
        if (strict) {
          val = (TT)pool_at<D, B>(pv, F, f.slot, v, n);
        } else {
          int hq[3] = {0, 0, 0};
          bool in_ring = true;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            hq[a] = h[a] + 4 * n[a] - f.off[a];
            in_ring &= (hq[a] > -(B - 1) && hq[a] < 3 * (B - 1));
          }
          if (!in_ring) {
            set_err(pv, kErrGraded);
            val = TT(0);
          } else {
            Own o;
            if (inside) {
              if (owner<D, B>(b, hq, b.lvl, rslot, rlvl, o)) {
                const int sh = b.lvl + 1 - o.m;
                int li[3] = {o.off[0] >> sh, o.off[1] >> sh, o.off[2] >> sh};
                val = (TT)pool_at<D, B>(pv, F, o.slot, v, li);
              } else {
                val = (TT)pool_at<D, B>(pv, F, f.slot, v, n);
              }
            } else {
              if (owner<D, B>(b, hq, 0, rslot, rlvl, o) && o.m >= b.lvl - 1) {
                const int sh = b.lvl + 1 - o.m;
                int li[3] = {o.off[0] >> sh, o.off[1] >> sh, o.off[2] >> sh};
                val = (TT)pool_at<D, B>(pv, F, o.slot, v, li);
              } else {
                set_err(pv, kErrGraded);
                val = TT(0);
              }
            }
          }
        }
        w[sx] = val;
      }
      vx[sz][sy] = ns[0] == 4 ? dd4(w[0], w[1], w[2], w[3]) : w[0];
    }
  TT vy[4];
  for (int sz = 0; sz < ns[2]; ++sz)
    vy[sz] = ns[1] == 4 ? dd4(vx[sz][0], vx[sz][1], vx[sz][2], vx[sz][3]) : vx[sz][0];
  return ns[2] == 4 ? dd4(vy[0], vy[1], vy[2], vy[3]) : vy[0];
}

// Fills the synchronised tile (nvar x T^d, type TT) of block b from field F.
// commit: block-edge nodes taken from a finer leaf are also written back into
// F (the paper's synchronisation overwrites them in the block).  ghost_out
// (optional, double): the tile is also written there (mr_get_tiles).
template <int D, int B, typename TF, typename TT>
__device__ void fill_tile(const PoolView& pv, const BlockInfo& b, const TF* F, TF* Fw, TT* tile,
                          bool commit, const int* rslot, const int8_t* rlvl) {
  using Gm = Geo<D, B>;
  const int nv = pv.nvar;
  for (int idx = threadIdx.x; idx < Gm::TILE; idx += blockDim.x) {
    const int i = idx % Gm::T - Gm::G;
    const int j = (idx / Gm::T) % Gm::T - Gm::G;
    const int k = D == 3 ? idx / (Gm::T * Gm::T) - Gm::G : 0;
    const int ijk[3] = {i, j, k};
    bool ghost = false, edge = false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if (ijk[a] < 0 || ijk[a] > B - 1) ghost = true;
      else if (ijk[a] == 0 || ijk[a] == B - 1) edge = true;
    }
    if (!ghost) {
      const int64_t at = Gm::lin(i, j, k);
      Own o;
      bool finer = false;
      if (edge) {
        const int h[3] = {2 * i, 2 * j, 2 * k};
        finer = owner<D, B>(b, h, b.lvl + 1, rslot, rlvl, o);
      }
      for (int v = 0; v < nv; ++v) {
        TF val;
        if (finer) {
          const int li[3] = {o.off[0], o.off[1], o.off[2]};
          val = pool_at<D, B>(pv, F, o.slot, v, li);
          if (commit) Fw[((int64_t)b.slot * nv + v) * pv.vs + at] = val;
        } else {
          val = F[((int64_t)b.slot * nv + v) * pv.vs + at];
        }
        tile[v * Gm::TILE + idx] = (TT)val;
      }
      continue;
    }
    const int h[3] = {2 * i, 2 * j, 2 * k};
    Own o;
    if (!owner<D, B>(b, h, 0, rslot, rlvl, o)) {
      set_err(pv, kErrGraded);
      for (int v = 0; v < nv; ++v) tile[v * Gm::TILE + idx] = TT(0);
      continue;
    }
    const int sh = b.lvl + 1 - o.m;
    bool node = true;
#pragma unroll
    for (int a = 0; a < D; ++a) node &= (o.off[a] & ((1 << sh) - 1)) == 0;
    if (o.m >= b.lvl || node) {
      const int li[3] = {o.off[0] >> sh, o.off[1] >> sh, o.off[2] >> sh};
      for (int v = 0; v < nv; ++v) tile[v * Gm::TILE + idx] = (TT)pool_at<D, B>(pv, F, o.slot, v, li);
    } else {
      if (o.m != b.lvl - 1) set_err(pv, kErrGraded);
      for (int v = 0; v < nv; ++v)
        tile[v * Gm::TILE + idx] = predict_ghost<D, B, TF, TT>(pv, b, h, o, v, F, rslot, rlvl);
    }
  }
}

// Tensor-product prediction at half-coarse position o (per axis, odd = between
// coarse nodes) from a tile whose coarse node n sits at tile index n*stride.
// x first, then y, then z.  Used by refinement (stride 1: the mother's tile) and
// by the details (stride 2: even nodes of the block's own tile).
template <int D, int B, typename TT>
__device__ __forceinline__ TT predict_tile(const TT* tile, const int o[3], int stride) {
  using Gm = Geo<D, B>;
  int base[3] = {0, 0, 0}, ns[3] = {1, 1, 1};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int fl = floordiv(o[a], 2);
    if (o[a] & 1) { ns[a] = 4; base[a] = fl - 1; }
    else base[a] = fl;
  }
  TT vx[4][4];
  for (int sz = 0; sz < ns[2]; ++sz)
    for (int sy = 0; sy < ns[1]; ++sy) {
      const int y = stride * (base[1] + sy), z = D == 3 ? stride * (base[2] + sz) : 0;
      if (ns[0] == 4) {
        const int x0 = stride * base[0];
        vx[sz][sy] = dd4(tile[Gm::tix(x0, y, z)], tile[Gm::tix(x0 + stride, y, z)],
                         tile[Gm::tix(x0 + 2 * stride, y, z)], tile[Gm::tix(x0 + 3 * stride, y, z)]);
      } else {
        vx[sz][sy] = tile[Gm::tix(stride * base[0], y, z)];
      }
    }
  TT vy[4];
  for (int sz = 0; sz < ns[2]; ++sz)
    vy[sz] = ns[1] == 4 ? dd4(vx[sz][0], vx[sz][1], vx[sz][2], vx[sz][3]) : vx[sz][0];
  return ns[2] == 4 ? dd4(vy[0], vy[1], vy[2], vy[3]) : vy[0];
}

template <typename T>
__device__ __forceinline__ T* smem_as(size_t offset_bytes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return reinterpret_cast<T*>(smem_raw + offset_bytes);
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace mr

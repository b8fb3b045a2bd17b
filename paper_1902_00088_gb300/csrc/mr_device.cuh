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

#include <type_traits>

#include "mr_internal.h"

namespace mr {

// Compile-time loop: f(std::integral_constant<int, I>) for I in [A, E).
template <int A, int E, typename Fn>
__device__ __forceinline__ void static_for(Fn&& f) {
  if constexpr (A < E) {
    f(std::integral_constant<int, A>{});
    static_for<A + 1, E>(f);
  }
}

// Asynchronous global -> shared copy of one 4- or 8-byte value (cp.async):
// the value goes to shared memory without passing through registers, so a
// thread can have every copy of a tile in flight at once; cp_async_wait_all
// waits for the calling thread's copies (a barrier then publishes them).
template <typename T>
__device__ __forceinline__ void cp_async(T* smem_dst, const T* gmem_src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async of 4 or 8 bytes");
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem_src), "n"(sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Bulk asynchronous copy (TMA engine, cp.async.bulk) of `bytes` contiguous
// bytes from global to shared memory, completion signalled on an mbarrier
// that expects the transaction bytes.  Both addresses and the size are
// multiples of 16 bytes.  Issued by one thread.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, unsigned bytes, uint64_t* bar) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(d), "l"(gmem_src), "r"(bytes), "r"(b) : "memory");
}
// Waits for the mbarrier phase with the given parity to complete, at most
// `limit` polls; false if it did not (the caller reports a timeout).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int limit) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  for (int it = 0; it < limit; ++it) {
    unsigned done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(256);
  }
  return false;
}

// Thread groups that cooperate on one block: the whole CTA, or one warp.
struct CtaGroup {
  static constexpr int kSize = 0;  // size known at run time only
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ int size() const { return blockDim.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct WarpGroup {
  static constexpr int kSize = 32;
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ int size() const { return 32; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

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
  // coarse box: level l-1 nodes around the block that prediction stencils of
  // ghost nodes can touch, coarse index n in [CLO, CLO + CB) relative to the
  // block origin
  static constexpr int CLO = -(G / 2) - 1;
  static constexpr int CB = (B - 1) / 2 + G + 3;
  static constexpr int CBOX = CB * CB * (D == 3 ? CB : 1);
  __device__ static __forceinline__ int tix(int i, int j, int k) {
    return ((k + GZ) * T + (j + G)) * T + (i + G);
  }
  __device__ static __forceinline__ int lin(int i, int j, int k) { return (k * B + j) * B + i; }
};

// Part of the tile a consumer reads: the box of ghost width W (W <= G) and the
// coarse nodes its prediction stencils touch, CLO..CLO+CB-1 per axis.
template <int D, int B, int W>
struct Box {
  static_assert(W >= 1 && W <= kG, "ghost width");
  static constexpr int S = B + 2 * W;
  static constexpr int NPTS = S * S * (D == 3 ? S : 1);
  static constexpr int TILE = NPTS;  // tile of this width: S^d nodes, x fastest
  static constexpr int CLO = -((W + 1) / 2) - 1;
  static constexpr int CB = (B - 1) / 2 + 2 * ((W + 1) / 2) + 3;
  static constexpr int CBOX = CB * CB * (D == 3 ? CB : 1);
  // scratch of the separable prediction, per variable: X[nz][ny][x] (coarse
  // y, z; fine x) and, in 3D, Y[nz][y][x] (coarse z; fine x, y).  In 3D X is
  // kept in the variable's tile, which is written only after the y pass, so
  // the scratch holds Y alone.
  static constexpr int NXP = (D == 3 ? CB : 1) * CB * S;
  static constexpr int NYP = D == 3 ? CB * S * S : 0;
  static constexpr int SCR = D == 3 ? NYP : NXP;
  static_assert(D == 2 || NXP <= TILE, "the x pass fits in the tile");
  __device__ static __forceinline__ int cix(int i, int j, int k) {
    return ((D == 3 ? k - CLO : 0) * CB + (j - CLO)) * CB + (i - CLO);
  }
  __device__ static __forceinline__ int tix(int i, int j, int k) {
    return (((D == 3 ? k + W : 0)) * S + (j + W)) * S + (i + W);
  }
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
// 2^d child cells included) the leaf covering it, searched at l+1, l, l-1,
// with the leaf's origin relative to the block origin in level-(l+1) node
// units (periodic images resolved once here, so per-point work needs no
// modulo).  These cells carry exactly the 16 (2D) / 74 (3D) relations of
// Sec. 2.2.  A cell covered by no leaf in that range means a non-graded tree.
//
// Region table (filled when some ring leaf is not at the block's level): along
// each axis a level-l node index x relative to the block origin falls into one
// of 7 classes -- inside ring cell -1 (x < 0), on the face x = 0 between cells
// -1 and 0, inside cell 0, on the face x = H, inside cell 1, on the face x = 2H,
// inside cell 2 (H = (Bs - 1) / 2).  All nodes of one class box (7^d boxes)
// have the same leaves containing them, in the same position (inside, or on
// the same faces), hence the same owner: the owner is searched once per box,
// and each node only offsets into it.
template <int D>
struct RingD {
  static constexpr int NREG = D == 3 ? 343 : 49;
  int slot[64];
  int org[64][3];
  int8_t lvl[64];
  int finer;    // some leaf one level finer touches the block
  int coarser;  // some leaf one level coarser touches the block
  int mixed;    // some ring leaf is not at the block's level
  // classes (bit c of 7 per axis: x, y << 7, z << 14) of the class boxes owned
  // by a coarser leaf: the tile nodes predicted from the coarse lattice lie
  // in their union, so the separable prediction passes are confined to it
  int cmask;
  // per class box: owner slot (-1: none), owner level, owner origin
  // (level-(l+1) node units, relative to the block origin) x | y << 16, z
  int4 reg[NREG];
};
template <int D>
constexpr int kRingBytesD = (int)((sizeof(RingD<D>) + 15) / 16 * 16);
static_assert(RingD<2>::NREG + 1 == reg_entries(2) && RingD<3>::NREG + 1 == reg_entries(3), "table size");

template <int D, int B, typename G = CtaGroup>
__device__ void build_ring(const PoolView& pv, const TreeDev& td, const BlockInfo& b, RingD<D>& R) {
  const G g{};
  using Gm = Geo<D, B>;
  if (g.rank() == 0) R.finer = R.coarser = R.mixed = R.cmask = 0;
  g.sync();
  for (int r = g.rank(); r < Gm::NR; r += g.size()) {
    const int q[3] = {r % 4 - 1, (r / 4) % 4 - 1, r / 16 - 1};
    bool inside = true;
    for (int a = 0; a < D; ++a) inside &= (q[a] == 0 || q[a] == 1);
    if (inside) {
      R.slot[r] = b.slot;
      R.lvl[r] = (int8_t)b.lvl;
      for (int a = 0; a < 3; ++a) R.org[r][a] = 0;
      continue;
    }
    const int64_t nl1 = (int64_t)1 << (b.lvl + 1);
    int64_t cell[3] = {0, 0, 0}, c1[3] = {0, 0, 0}, c2[3] = {0, 0, 0};
    int un[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
      un[a] = (int)(2 * b.c[a] + q[a]);
      cell[a] = (int64_t)(un[a]) & (nl1 - 1);
      c1[a] = cell[a] >> 1;
      c2[a] = cell[a] >> 2;
    }
    // the three candidate levels are looked up together (one memory round trip)
    const int sf = tab_get<D>(pv, td, b.lvl + 1, cell), se = tab_get<D>(pv, td, b.lvl, c1),
              sc = tab_get<D>(pv, td, b.lvl - 1, c2);
    int s = sf, m = b.lvl + 1;
    if (s < 0) { s = se; m = b.lvl; }
    if (s < 0) { s = sc; m = b.lvl - 1; }
    if (s < 0) {
      set_err(pv, kErrGraded);
      m = -1;
    }
    if (m == b.lvl + 1) R.finer = 1;  // benign races: all writers store 1
    if (m == b.lvl - 1) R.coarser = 1;
    if (m != b.lvl) R.mixed = 1;
    const int sh = b.lvl + 1 - m;
    for (int a = 0; a < 3; ++a) {
      const int oc = a < D && m >= 0 ? ((un[a] >> sh) << sh) - (int)(2 * b.c[a]) : 0;
      R.org[r][a] = oc * (B - 1);
    }
    R.slot[r] = s;
    R.lvl[r] = (int8_t)m;
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

template <int B>
struct Log2B {
  static constexpr int value = B == 17 ? 4 : (B == 33 ? 5 : -1);
};

template <int D, int B>
__device__ __forceinline__ bool owner(const BlockInfo& b, const int h[3], int min_m, const RingD<D>& R,
                                      Own& o) {
  constexpr int P = Log2B<B>::value;
  static_assert(P > 0, "Bs - 1 must be a power of two");
  int c0[3] = {0, 0, 0};
  bool onb[3] = {false, false, false};
  bool any = false;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    c0[a] = h[a] >> P;
    onb[a] = (h[a] & (B - 2)) == 0;
    any |= onb[a];
  }
  // Candidate A: the ring cell holding the point at its lower edge or inside.
  // In its leaf the point is never the upper edge node, so A has the smallest
  // combo; it is the owner unless another candidate is finer.
  const int rA = (c0[0] + 1) + 4 * (c0[1] + 1) + 16 * (D == 3 ? c0[2] + 1 : 0);
  const int mA = R.lvl[rA];
  int mmax = R.slot[rA] >= 0 ? mA : -1;
  if (any) {
#pragma unroll
    for (int combo = 1; combo < (1 << D); ++combo) {
      bool ok = true;
      int r = 0, mul = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int bit = (combo >> a) & 1;
        if (bit && !onb[a]) ok = false;
        const int q = c0[a] - bit;
        if (q < -1) ok = false;
        r += (q + 1) * mul;
        mul *= 4;
      }
      if (ok && R.slot[r] >= 0 && R.lvl[r] > mmax) mmax = R.lvl[r];
    }
  }
  if (mmax < 0 || mmax < min_m) {
    o.m = -1;
    return false;
  }
  const int l1 = b.lvl + 1;
  if (mA == mmax && R.slot[rA] >= 0) {
    o.m = mA;
    o.combo = 0;
    o.slot = R.slot[rA];
#pragma unroll
    for (int a = 0; a < 3; ++a) o.off[a] = a < D ? h[a] - R.org[rA][a] : 0;
    return true;
  }
  // a finer leaf shares the point: smallest combo among the finest candidates
  o.m = -1;
  o.combo = 1 << 30;
#pragma unroll
  for (int combo = 1; combo < (1 << D); ++combo) {
    bool ok = true;
    int r = 0, mul = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int bit = (combo >> a) & 1;
      if (bit && !onb[a]) ok = false;
      const int q = c0[a] - bit;
      if (q < -1) ok = false;
      r += (q + 1) * mul;
      mul *= 4;
    }
    if (!ok || R.slot[r] < 0 || R.lvl[r] != mmax) continue;
    const int W = (B - 1) << (l1 - mmax);
    int oc = 0, off[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      off[a] = h[a] - R.org[r][a];
      if (off[a] == W) oc |= 1 << a;
    }
    if (oc < o.combo) {
      o.m = mmax;
      o.combo = oc;
      o.slot = R.slot[r];
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

// Coarse-lattice prediction at half-coarse position o (relative to the block
// origin) from the staged coarse box: x first, then y, then z.
template <int D, int B, int W, typename TT>
__device__ __forceinline__ TT predict_box(const TT* box, const int o[3]) {
  using Gm = Box<D, B, W>;
  int base[3] = {0, 0, 0}, ns[3] = {1, 1, 1};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int fl = o[a] >> 1;
    if (o[a] & 1) { ns[a] = 4; base[a] = fl - 1; }
    else base[a] = fl;
  }
  TT vx[4][4];
  for (int sz = 0; sz < ns[2]; ++sz)
    for (int sy = 0; sy < ns[1]; ++sy) {
      const int y = base[1] + sy, z = base[2] + sz;
      if (ns[0] == 4) {
        const TT* r = box + Gm::cix(base[0], y, z);
        vx[sz][sy] = dd4(r[0], r[1], r[2], r[3]);
      } else {
        vx[sz][sy] = box[Gm::cix(base[0], y, z)];
      }
    }
  TT vy[4];
  for (int sz = 0; sz < ns[2]; ++sz)
    vy[sz] = ns[1] == 4 ? dd4(vx[sz][0], vx[sz][1], vx[sz][2], vx[sz][3]) : vx[sz][0];
  return ns[2] == 4 ? dd4(vy[0], vy[1], vy[2], vy[3]) : vy[0];
}

// Class (0..6) of a level-l node index x relative to the block origin, for
// -(H - 1) <= x <= 3H - 1 (H = (Bs - 1) / 2): inside ring cell -1, face 0,
// inside cell 0, face H, inside cell 1, face 2H, inside cell 2.
template <int B>
__device__ __forceinline__ int reg_class(int x) {
  constexpr int H = (B - 1) / 2;
  return (x >= 0) + (x > 0) + (x >= H) + (x > H) + (x >= 2 * H) + (x > 2 * H);
}
// A node index of class c.
template <int B>
__device__ __forceinline__ int reg_rep(int c) {
  constexpr int H = (B - 1) / 2;
  return c == 0 ? -1 : c == 1 ? 0 : c == 2 ? 1 : c == 3 ? H : c == 4 ? H + 1 : c == 5 ? 2 * H : 2 * H + 1;
}

// Owner of every class box (see RingD), found with owner() at one node of the box.
template <int D, int B, typename G>
__device__ void build_regions(const BlockInfo& b, RingD<D>& R) {
  const G g{};
  for (int r = g.rank(); r < RingD<D>::NREG; r += g.size()) {
    const int c[3] = {r % 7, (r / 7) % 7, r / 49};
    int h[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) h[a] = 2 * reg_rep<B>(c[a]);
    Own o;
    int4 e = make_int4(-1, -1, 0, 0);
    if (owner<D, B>(b, h, 0, R, o)) {
      const int ox = h[0] - o.off[0], oy = h[1] - o.off[1], oz = h[2] - o.off[2];
      e = make_int4(o.slot, o.m, (ox & 0xffff) | (oy << 16), oz);
      if (o.m < b.lvl) atomicOr(&R.cmask, (1 << c[0]) | (1 << (7 + c[1])) | (D == 3 ? 1 << (14 + c[2]) : 0));
    }
    R.reg[r] = e;
  }
}

// Class-box owner table of plan position p (built with the stage plan while
// the tree is fixed): NREG entries, then {finer, coarser, mixed}.
template <int D>
__device__ __forceinline__ int4* plan_regions(const PoolView& pv, int p) {
  return pv.regs + (int64_t)p * (RingD<D>::NREG + 1);
}
template <int D, typename G>
__device__ void store_regions(const PoolView& pv, int p, const RingD<D>& R) {
  const G g{};
  int4* dst = plan_regions<D>(pv, p);
  for (int r = g.rank(); r < RingD<D>::NREG; r += g.size()) dst[r] = R.reg[r];
  if (g.rank() == 0) dst[RingD<D>::NREG] = make_int4(R.finer, R.coarser, R.mixed, R.cmask);
}
// Loads the table of plan position p into the ring (the caller synchronises
// the group before use).
template <int D, typename G>
__device__ void load_regions(const PoolView& pv, int p, RingD<D>& R) {
  const G g{};
  const int4* src = plan_regions<D>(pv, p);
  for (int r = g.rank(); r < RingD<D>::NREG; r += g.size()) R.reg[r] = src[r];
  if (g.rank() == 0) {
    const int4 f = src[RingD<D>::NREG];
    R.finer = f.x;
    R.coarser = f.y;
    R.mixed = f.z;
    R.cmask = f.w;
  }
}

// Tile nodes (per axis, tile coordinates) that can be predicted from the
// coarse lattice: the span of the classes in mask7 (bit c = class c of
// reg_class), clipped to the tile box of ghost width W; and the coarse
// indices the separable passes read for them, clipped to the coarse box.
template <int B, int W>
struct PredBox {
  int lo[3], hi[3];    // predicted tile nodes
  int nlo[3], nhi[3];  // coarse nodes their prediction reads
  __device__ __forceinline__ PredBox(int cmask, int D) {
    constexpr int H = (B - 1) / 2;
    using Bx = Box<2, B, W>;  // CLO and CB do not depend on the dimension
    // first and last node of class c within the tile box
    auto clo = [](int c) { return c == 0 ? -W : c == 1 ? 0 : c == 2 ? 1 : c == 3 ? H : c == 4 ? H + 1 : c == 5 ? 2 * H : 2 * H + 1; };
    auto chi = [](int c) { return c == 0 ? -1 : c == 1 ? 0 : c == 2 ? H - 1 : c == 3 ? H : c == 4 ? 2 * H - 1 : c == 5 ? 2 * H : B - 1 + W; };
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int m = (cmask >> (7 * a)) & 127;
      if (a >= D || m == 0) {
        lo[a] = hi[a] = 0;
        nlo[a] = nhi[a] = 0;
        continue;
      }
      lo[a] = clo(__ffs(m) - 1);
      hi[a] = chi(31 - __clz(m));
      nlo[a] = max(Bx::CLO, (lo[a] >> 1) - 1);
      nhi[a] = min(Bx::CLO + Bx::CB - 1, (hi[a] >> 1) + 2);
    }
  }
};

// Separable prediction over the coarse box (values of nv variables in cbox),
// x first, then y (then z at the point): the same operations in the same order
// as predict_box, evaluated only where the predicted nodes of pb need them.
// 2D: the x pass goes to scr (y per point from it); 3D: the x pass is kept in
// the variable's tile (overwritten later by the gather) and the y pass goes to
// scr (z per point).  Ends with a group barrier.
template <int D, int B, int W, typename TT, typename G>
__device__ void coarse_passes(int nv, const TT* cbox, TT* tile, TT* scr, const PredBox<B, W>& pb) {
  const G g{};
  using Bx = Box<D, B, W>;
  // x pass: x in [lo0, hi0], coarse rows ny in [nlo1, nhi1], nz in [nlo2, nhi2]
  const int ex = pb.hi[0] - pb.lo[0] + 1, ey = pb.nhi[1] - pb.nlo[1] + 1;
  const int nxp = ex * ey * (D == 3 ? pb.nhi[2] - pb.nlo[2] + 1 : 1);
  for (int v = 0; v < nv; ++v) {
    const TT* cb = cbox + v * Bx::CBOX;
    TT* X = D == 3 ? tile + v * Bx::TILE : scr + v * Bx::SCR;
    for (int q = g.rank(); q < nxp; q += g.size()) {
      const int x = q % ex + pb.lo[0], ny = (q / ex) % ey + pb.nlo[1];
      const int nz = D == 3 ? q / (ex * ey) + pb.nlo[2] : 0;
      const int fl = x >> 1;
      const int at = ((D == 3 ? nz - Bx::CLO : 0) * Bx::CB + (ny - Bx::CLO)) * Bx::S + (x + W);
      X[at] = (x & 1) ? dd4(cb[Bx::cix(fl - 1, ny, nz)], cb[Bx::cix(fl, ny, nz)], cb[Bx::cix(fl + 1, ny, nz)],
                            cb[Bx::cix(fl + 2, ny, nz)])
                      : cb[Bx::cix(fl, ny, nz)];
    }
  }
  if (D == 3) {
    g.sync();
    // y pass: x in [lo0, hi0], y in [lo1, hi1], coarse nz in [nlo2, nhi2]
    const int fy = pb.hi[1] - pb.lo[1] + 1;
    const int nyp = ex * fy * (pb.nhi[2] - pb.nlo[2] + 1);
    for (int v = 0; v < nv; ++v) {
      const TT* X = tile + v * Bx::TILE;
      TT* Y = scr + v * Bx::SCR;
      for (int q = g.rank(); q < nyp; q += g.size()) {
        const int x = q % ex + pb.lo[0] + W, y = (q / ex) % fy + pb.lo[1];
        const int nzi = q / (ex * fy) + pb.nlo[2] - Bx::CLO;
        const int fl = y >> 1;
        const TT* c = X + nzi * Bx::CB * Bx::S + x;
        Y[(nzi * Bx::S + (y + W)) * Bx::S + x] = (y & 1) ? dd4(c[(fl - 1 - Bx::CLO) * Bx::S], c[(fl - Bx::CLO) * Bx::S],
                                                               c[(fl + 1 - Bx::CLO) * Bx::S], c[(fl + 2 - Bx::CLO) * Bx::S])
                                                         : c[(fl - Bx::CLO) * Bx::S];
      }
    }
  }
  g.sync();
}

// Value of a ghost node predicted from the coarse box after coarse_passes: the
// last axis (z in 3D, y in 2D) from the scratch.
template <int D, int B, int W, typename TT>
__device__ __forceinline__ TT coarse_predicted(const TT* scr_v, int i, int j, int k) {
  using Bx = Box<D, B, W>;
  const TT* c = scr_v + (i + W) + (D == 3 ? (j + W) * Bx::S : 0);
  constexpr int st = D == 3 ? Bx::S * Bx::S : Bx::S;
  const int e = D == 3 ? k : j, fl = e >> 1;
  return (e & 1) ? dd4(c[(fl - 1 - Bx::CLO) * st], c[(fl - Bx::CLO) * st], c[(fl + 1 - Bx::CLO) * st],
                       c[(fl + 2 - Bx::CLO) * st])
                 : c[(fl - Bx::CLO) * st];
}

// Fills the synchronised tile (nvar x T^d, type TT) of block b from field F.
// Block-edge nodes owned by another block (a finer one, Sec. 2.2 rule 2, or an
// equal-level one that holds the node at its lower edge, which keeps redundant
// copies identical as Sec. 2.5 assumes) take the owner's value; with commit
// they are also written back into F when they differ.  cbox: scratch
// of nvar x CBOX values for the coarse lattice (used when a coarser leaf
// touches the block): every coarse node takes its owner's value, and ghost
// nodes between coarse nodes are predicted from it.
template <int D, int B, typename TF, typename TT, int W = kG, typename G = CtaGroup>
__device__ void fill_tile(const PoolView& pv, const BlockInfo& b, const TF* F, TF* Fw, TT* tile,
                          bool commit, RingD<D>& R, TT* cbox, TT* scr = nullptr, bool have_regions = false) {
  const G g{};
  using Gm = Geo<D, B>;
  using Bx = Box<D, B, W>;
  // Each thread takes U points at a time: owners and addresses first, then the
  // U loads together, then the stores, so that the loads are in flight at once.
  constexpr int U = 4;
  const int nv = pv.nvar;
  const int64_t own = (int64_t)b.slot * nv * pv.vs;
  if (!R.mixed) {
    // every ring leaf has the block's level: the owner of a point is the ring
    // cell holding it from below (equal-level rule of owner()), no search
    constexpr int P = Log2B<B>::value;
    for (int q0 = g.rank(); q0 < Bx::NPTS; q0 += U * g.size()) {
      int64_t at[U];
      int idx[U], li[U];
      bool ok[U], ed[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * g.size();
        ok[u] = q < Bx::NPTS;
        const int qq = ok[u] ? q : 0;
        const int i = qq % Bx::S - W;
        const int j = (qq / Bx::S) % Bx::S - W;
        const int k = D == 3 ? qq / (Bx::S * Bx::S) - W : 0;
        idx[u] = Bx::tix(i, j, k);
        li[u] = Gm::lin(i, j, k);
        const int h[3] = {2 * i, 2 * j, 2 * k};
        int r = 0, lo[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) r += ((h[a] >> P) + 1) << (2 * a);
#pragma unroll
        for (int a = 0; a < D; ++a) lo[a] = (h[a] - R.org[r][a]) >> 1;
        const int src = R.slot[r];
        at[u] = (int64_t)src * nv * pv.vs + Gm::lin(lo[0], lo[1], lo[2]);
        // block-edge node owned by the equal-level neighbour (i or j = B-1)
        bool edge_node = true;
#pragma unroll
        for (int a = 0; a < D; ++a) edge_node &= (h[a] >= 0 && h[a] <= 2 * (B - 1));
        ed[u] = commit && src != b.slot && edge_node;
      }
      for (int v = 0; v < nv; ++v) {
        TF val[U];
#pragma unroll
        for (int u = 0; u < U; ++u) val[u] = ok[u] ? F[at[u] + (int64_t)v * pv.vs] : TF(0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!ok[u]) continue;
          tile[v * Bx::TILE + idx[u]] = (TT)val[u];
          if (ed[u]) {
            const int64_t me = own + (int64_t)v * pv.vs + li[u];
            if (F[me] != val[u]) Fw[me] = val[u];
          }
        }
      }
    }
    return;
  }
  // some ring leaf is at another level: one owner search per class box
  // (unless the table was loaded from the stage plan)
  if (!have_regions) {
    build_regions<D, B, G>(b, R);
    g.sync();
  }
  const int l1 = b.lvl + 1;
  // owner of level-l node x (relative to the block origin) and the node's
  // offset inside it in level-(l+1) units
  auto region = [&](const int x[3], int& slot, int& m, int off[3]) {
    const int r = reg_class<B>(x[0]) + 7 * reg_class<B>(x[1]) + (D == 3 ? 49 * reg_class<B>(x[2]) : 0);
    const int4 e = R.reg[r];
    slot = e.x;
    m = e.y;
    off[0] = 2 * x[0] - (int)(int16_t)(e.z & 0xffff);
    off[1] = 2 * x[1] - (e.z >> 16);
    off[2] = D == 3 ? 2 * x[2] - e.w : 0;
  };
  if (R.coarser && R.cmask) {
    const PredBox<B, W> pb(R.cmask, D);
    for (int q0 = g.rank(); q0 < Bx::CBOX; q0 += U * g.size()) {
      int64_t at[U];
      bool ok[U], good[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = q0 + u * g.size();
        ok[u] = idx < Bx::CBOX;
        good[u] = false;
        at[u] = 0;
        if (!ok[u]) continue;
        const int n[3] = {idx % Bx::CB + Bx::CLO, (idx / Bx::CB) % Bx::CB + Bx::CLO,
                          D == 3 ? idx / (Bx::CB * Bx::CB) + Bx::CLO : 0};
        bool need = true;  // read by the prediction of some node of pb
#pragma unroll
        for (int a = 0; a < D; ++a) need &= n[a] >= pb.nlo[a] && n[a] <= pb.nhi[a];
        if (!need) continue;
        // coarse node n sits at level-l node 2n
        const int x[3] = {2 * n[0], 2 * n[1], 2 * n[2]};
        int slot, m, off[3];
        region(x, slot, m, off);
        if (slot < 0 || m < b.lvl - 1) {
          set_err(pv, kErrGraded);
          continue;
        }
        good[u] = true;
        const int sh = l1 - m;
        at[u] = ((int64_t)slot * nv) * pv.vs + Gm::lin(off[0] >> sh, off[1] >> sh, D == 3 ? off[2] >> sh : 0);
      }
      for (int v = 0; v < nv; ++v) {
        TF val[U];
#pragma unroll
        for (int u = 0; u < U; ++u) val[u] = good[u] ? F[at[u] + (int64_t)v * pv.vs] : TF(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) cbox[v * Bx::CBOX + q0 + u * g.size()] = good[u] ? (TT)val[u] : TT(0);
      }
    }
    g.sync();
    if (scr) coarse_passes<D, B, W, TT, G>(nv, cbox, tile, scr, pb);
  }
  // kinds of tile points: 0 own node, 1 block-edge node of another owner,
  // 2 ghost node that is a node of its owner, 3 ghost predicted from the coarse
  // box, 4 no owner (error, zero)
  for (int q0 = g.rank(); q0 < Bx::NPTS; q0 += U * g.size()) {
    int64_t at[U];
    int idx[U], li[U], kind[U], ijk[U][3];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u * g.size();
      const int qq = q < Bx::NPTS ? q : 0;
      const int i = qq % Bx::S - W;
      const int j = (qq / Bx::S) % Bx::S - W;
      const int k = D == 3 ? qq / (Bx::S * Bx::S) - W : 0;
      ijk[u][0] = i;
      ijk[u][1] = j;
      ijk[u][2] = k;
      idx[u] = Bx::tix(i, j, k);
      li[u] = Gm::lin(i, j, k);
      at[u] = 0;
      kind[u] = 5;  // past the end
      if (q >= Bx::NPTS) continue;
      bool core = true;  // strictly inside the block: its own node
#pragma unroll
      for (int a = 0; a < D; ++a) core &= (ijk[u][a] >= 1 && ijk[u][a] <= B - 2);
      if (core) {
        kind[u] = 0;
        at[u] = own + li[u];
        continue;
      }
      int slot, m, off[3];
      region(ijk[u], slot, m, off);
      if (slot < 0) {
        set_err(pv, kErrGraded);
        kind[u] = 4;
        continue;
      }
      bool inner = true;
#pragma unroll
      for (int a = 0; a < D; ++a) inner &= (ijk[u][a] >= 0 && ijk[u][a] <= B - 1);
      const int sh = l1 - m;
      if (inner) {
        // the block's own node, or an edge node whose owner is another block
        // (a finer one, or an equal-level one holding it at its lower edge)
        if (slot == b.slot) {
          kind[u] = 0;
          at[u] = own + li[u];
        } else {
          kind[u] = 1;
          at[u] = ((int64_t)slot * nv) * pv.vs + Gm::lin(off[0] >> sh, off[1] >> sh, D == 3 ? off[2] >> sh : 0);
        }
        continue;
      }
      const bool node = ((off[0] | off[1] | off[2]) & ((1 << sh) - 1)) == 0;
      if (m >= b.lvl || node) {
        kind[u] = 2;
        at[u] = ((int64_t)slot * nv) * pv.vs + Gm::lin(off[0] >> sh, off[1] >> sh, D == 3 ? off[2] >> sh : 0);
      } else {
        if (m != b.lvl - 1) set_err(pv, kErrGraded);
        kind[u] = 3;
      }
    }
    for (int v = 0; v < nv; ++v) {
      TF val[U];
#pragma unroll
      for (int u = 0; u < U; ++u) val[u] = kind[u] <= 2 ? F[at[u] + (int64_t)v * pv.vs] : TF(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (kind[u] == 5) continue;
        TT* t = tile + v * Bx::TILE + idx[u];
        if (kind[u] == 3) {
          if (scr) {
            // last axis from the scratch: z in 3D (Y), y in 2D (X)
            const TT* c = scr + v * Bx::SCR + (ijk[u][0] + W) +
                          (D == 3 ? (ijk[u][1] + W) * Bx::S : 0);
            const int st = D == 3 ? Bx::S * Bx::S : Bx::S;
            const int e = ijk[u][D - 1], fl = e >> 1;
            *t = (e & 1) ? dd4(c[(fl - 1 - Bx::CLO) * st], c[(fl - Bx::CLO) * st], c[(fl + 1 - Bx::CLO) * st],
                               c[(fl + 2 - Bx::CLO) * st])
                         : c[(fl - Bx::CLO) * st];
          } else {
            *t = predict_box<D, B, W, TT>(cbox + v * Bx::CBOX, ijk[u]);
          }
        } else if (kind[u] == 4) {
          *t = TT(0);
        } else {
          *t = (TT)val[u];
          if (kind[u] == 1 && commit) {
            const int64_t me = own + (int64_t)v * pv.vs + li[u];
            if (F[me] != val[u]) Fw[me] = val[u];
          }
        }
      }
    }
  }
}

// Column form of the 3D tile fill for one CTA: each thread fills whole z-columns
// (fixed x, y) of the tile, with the z loop unrolled, so every quantity that
// depends on z alone (neighbour index, local offset, class box, inside or
// ghost) is a compile-time constant and the per-node work is a table lookup,
// an address and the copy.  Up to KC loads of a column are in flight together.
// nbase (nullable): pool offsets (slot * nvar * vs) of the 27 equal-level
// neighbours of a block with a uniform neighbourhood (x fastest, the block
// itself in the centre); null: the owners come from the ring's class boxes
// (build_ring must have run).  Same values, stores and commits as fill_tile.
template <int B, typename TF, typename TT, int W>
__device__ void fill_cols(const PoolView& pv, const BlockInfo& b, const int64_t* nbase, const TF* F, TF* Fw,
                          TT* tile, bool commit, RingD<3>& R, TT* cbox, TT* scr, bool have_regions = false) {
  using Gm = Geo<3, B>;
  using Bx = Box<3, B, W>;
  constexpr int S = Bx::S, S2 = S * S, BB = B * B;
  // same field and tile types: asynchronous copies, all in flight at once
  constexpr bool ASYNC = std::is_same<TF, TT>::value;
  constexpr int KC = ASYNC ? 11 : 7;  // nodes per chunk (register loads in flight)
  const int nv = pv.nvar;
  const int64_t own = (int64_t)b.slot * nv * pv.vs;
  const int l1 = b.lvl + 1;
  const bool uni = nbase != nullptr;
  auto load_store = [&](auto kcc, const int64_t* at, const int* kind, int col, int i, int j, int kbase) {
    constexpr int KN = decltype(kcc)::value;
    if constexpr (ASYNC) {
      // copies now; block-edge nodes of other owners are committed after the wait
      for (int v = 0; v < nv; ++v) {
#pragma unroll
        for (int u = 0; u < KN; ++u) {
          const int k = kbase + u;
          TT* t = tile + v * Bx::TILE + col + (k + W) * S2;
          if (kind[u] <= 2) cp_async(t, F + at[u] + (int64_t)v * pv.vs);
          else if (kind[u] == 3) *t = coarse_predicted<3, B, W, TT>(scr + v * Bx::SCR, i, j, k);
          else *t = TT(0);
        }
      }
      return;
    }
    for (int v = 0; v < nv; ++v) {
      TF val[KN];
#pragma unroll
      for (int u = 0; u < KN; ++u) val[u] = kind[u] <= 2 ? F[at[u] + (int64_t)v * pv.vs] : TF(0);
#pragma unroll
      for (int u = 0; u < KN; ++u) {
        const int k = kbase + u;
        TT* t = tile + v * Bx::TILE + col + (k + W) * S2;
        if (kind[u] == 3) {
          *t = coarse_predicted<3, B, W, TT>(scr + v * Bx::SCR, i, j, k);
        } else if (kind[u] == 4) {
          *t = TT(0);
        } else {
          *t = (TT)val[u];
          if (kind[u] == 1 && commit) {
            const int64_t me = own + (int64_t)v * pv.vs + Gm::lin(i, j, k);
            if (F[me] != val[u]) Fw[me] = val[u];
          }
        }
      }
    }
  };
  if (!uni) {
    if (!have_regions) {
      build_regions<3, B, CtaGroup>(b, R);
      __syncthreads();
    }
    if (R.coarser && R.cmask) {
      // coarse box: columns of CB coarse nodes (coarse node n at level-l node
      // 2n), where the prediction of the nodes of pb reads them
      const PredBox<B, W> pb(R.cmask, 3);
      constexpr int CB = Bx::CB;
      for (int c = threadIdx.x; c < CB * CB; c += blockDim.x) {
        const int nx = c % CB + Bx::CLO, ny = c / CB + Bx::CLO;
        if (nx < pb.nlo[0] || nx > pb.nhi[0] || ny < pb.nlo[1] || ny > pb.nhi[1]) continue;
        const int rb = reg_class<B>(2 * nx) + 7 * reg_class<B>(2 * ny);
        // per chunk of the column: addresses first, then the loads, then the stores
        bool bad = false;
        auto cchunk = [&](auto knc, auto z0c) {
          constexpr int KN = decltype(knc)::value, Z0 = decltype(z0c)::value;
          int64_t at[KN];
          int good[KN];  // 1 load, 0 not needed, -1 no owner (error)
#pragma unroll
          for (int u = 0; u < KN; ++u) {
            const int nz = Z0 + u + Bx::CLO;
            at[u] = 0;
            good[u] = 0;
            if (nz < pb.nlo[2] || nz > pb.nhi[2]) continue;
            const int4 e = R.reg[rb + 49 * reg_class<B>(2 * nz)];
            if (e.x < 0 || e.y < b.lvl - 1) {
              good[u] = -1;
              continue;
            }
            const int sh = l1 - e.y;
            const int ox = 4 * nx - (int)(int16_t)(e.z & 0xffff), oy = 4 * ny - (e.z >> 16), oz = 4 * nz - e.w;
            at[u] = ((int64_t)e.x * nv) * pv.vs + Gm::lin(ox >> sh, oy >> sh, oz >> sh);
            good[u] = 1;
          }
          for (int v = 0; v < nv; ++v) {
            if constexpr (ASYNC) {
#pragma unroll
              for (int u = 0; u < KN; ++u) {
                TT* t = cbox + v * Bx::CBOX + (Z0 + u) * CB * CB + c;
                if (good[u] > 0) cp_async(t, F + at[u] + (int64_t)v * pv.vs);
                else if (good[u] < 0) *t = TT(0);
                bad |= good[u] < 0;
              }
            } else {
              TF val[KN];
#pragma unroll
              for (int u = 0; u < KN; ++u) val[u] = good[u] > 0 ? F[at[u] + (int64_t)v * pv.vs] : TF(0);
#pragma unroll
              for (int u = 0; u < KN; ++u) {
                if (good[u] != 0) cbox[v * Bx::CBOX + (Z0 + u) * CB * CB + c] = good[u] > 0 ? (TT)val[u] : TT(0);
                bad |= good[u] < 0;
              }
            }
          }
        };
        constexpr int ZC = 7;
        static_for<0, (CB + ZC - 1) / ZC>([&](auto cc) {
          constexpr int C = decltype(cc)::value;
          constexpr int KN = (CB - C * ZC) < ZC ? (CB - C * ZC) : ZC;
          cchunk(std::integral_constant<int, KN>{}, std::integral_constant<int, C * ZC>{});
        });
        if (bad) set_err(pv, kErrGraded);
      }
      if constexpr (ASYNC) cp_async_wait_all();
      __syncthreads();
      if (scr) coarse_passes<3, B, W, TT, CtaGroup>(nv, cbox, tile, scr, pb);
    }
  }
  for (int col = threadIdx.x; col < S2; col += blockDim.x) {
    const int i = col % S - W, j = col / S - W;
    const bool inxy = i >= 0 && i <= B - 1 && j >= 0 && j <= B - 1;
    // strictly inside the block in x and y: with 1 <= k <= Bs - 2 the node is
    // the block's own (no other leaf contains it), whatever the ring holds
    const bool core = i >= 1 && i <= B - 2 && j >= 1 && j <= B - 2;
    // uniform form: neighbour row and local offset of the column
    const int sx = i < 0 ? 0 : (i <= B - 2 ? 1 : 2), sy = j < 0 ? 0 : (j <= B - 2 ? 1 : 2);
    const int lxy = (i - (sx - 1) * (B - 1)) + B * (j - (sy - 1) * (B - 1));
    const int64_t* nrow = uni ? nbase + sx + 3 * sy : nullptr;
    // ring form: class box row of the column
    const int rb = reg_class<B>(i) + 7 * reg_class<B>(j);
    auto chunk = [&](auto kcc, auto k0c) {
      constexpr int KN = decltype(kcc)::value, K0 = decltype(k0c)::value;
      int64_t at[KN];
      int kind[KN];
#pragma unroll
      for (int u = 0; u < KN; ++u) {
        const int k = K0 + u;
        const int sk = k < 0 ? 0 : (k <= B - 2 ? 1 : 2);  // compile-time per u
        const bool ink = k >= 0 && k <= B - 1;
        const bool inner = inxy && ink;
        if (uni) {
          const int64_t nb = nrow[9 * sk];
          at[u] = nb + lxy + BB * (k - (sk - 1) * (B - 1));
          kind[u] = inner ? (nb != own ? 1 : 0) : 2;
          continue;
        }
        if (k >= 1 && k <= B - 2 && core) {
          kind[u] = 0;
          at[u] = own + Gm::lin(i, j, k);
          continue;
        }
        const int4 e = R.reg[rb + 49 * reg_class<B>(k)];
        if (e.x < 0) {
          set_err(pv, kErrGraded);
          kind[u] = 4;
          at[u] = 0;
          continue;
        }
        const int m = e.y, sh = l1 - m;
        const int ox = 2 * i - (int)(int16_t)(e.z & 0xffff), oy = 2 * j - (e.z >> 16), oz = 2 * k - e.w;
        const int64_t src = ((int64_t)e.x * nv) * pv.vs + Gm::lin(ox >> sh, oy >> sh, oz >> sh);
        if (inner) {
          kind[u] = e.x == b.slot ? 0 : 1;
          at[u] = e.x == b.slot ? own + Gm::lin(i, j, k) : src;
          continue;
        }
        const bool node = ((ox | oy | oz) & ((1 << sh) - 1)) == 0;
        if (m >= b.lvl || node) {
          kind[u] = 2;
          at[u] = src;
        } else {
          if (m != b.lvl - 1) set_err(pv, kErrGraded);
          kind[u] = 3;
          at[u] = 0;
        }
      }
      load_store(kcc, at, kind, col, i, j, K0);
    };
    // k = -W .. B-1+W in chunks of KC (compile-time k)
    static_for<0, (S + KC - 1) / KC>([&](auto cc) {
      constexpr int C = decltype(cc)::value;
      constexpr int K0 = -W + C * KC;
      constexpr int KN = (S - C * KC) < KC ? (S - C * KC) : KC;
      chunk(std::integral_constant<int, KN>{}, std::integral_constant<int, K0>{});
    });
  }
  if constexpr (ASYNC) {
    cp_async_wait_all();
    if (commit) {
      // block-edge nodes owned by another block: store the owner's value (now
      // in the tile) where the block's own copy differs
      __syncthreads();
      for (int col = threadIdx.x; col < BB; col += blockDim.x) {
        const int i = col % B, j = col / B;
        const bool side = i == 0 || i == B - 1 || j == 0 || j == B - 1;
        const int sx = i <= B - 2 ? 1 : 2, sy = j <= B - 2 ? 1 : 2;
        const int rb = reg_class<B>(i) + 7 * reg_class<B>(j);
        for (int k = 0; k < B; k += (side || k == B - 1) ? 1 : B - 1) {
          bool other;
          if (uni) {
            other = nbase[sx + 3 * sy + 9 * (k <= B - 2 ? 1 : 2)] != own;
          } else {
            other = R.reg[rb + 49 * reg_class<B>(k)].x != b.slot;
          }
          if (!other) continue;
          for (int v = 0; v < nv; ++v) {
            const TT val = tile[v * Bx::TILE + Bx::tix(i, j, k)];
            const int64_t me = own + (int64_t)v * pv.vs + Gm::lin(i, j, k);
            if (F[me] != val) Fw[me] = val;
          }
        }
      }
    }
  }
}

// Stage plan of one active block, valid while the tree is fixed (the four RK
// stages of a step): INTS int32 per active position,
//   [0] slot, [1] level | tree << 8 | uniform << 30, [2 .. 2+D) block coordinates,
//   [2+D .. 2+D+NB) slots of the 3^d blocks at offsets (dx, dy, dz) in {-1,0,1}^d
//   (x fastest), the centre being the block itself.
// "uniform": every one of them is a leaf at the block's level, so each node of
// the ghost layer and each block-edge node has an equal-level owner, the block
// that holds it at its lower edge (Sec. 2.2, Sec. 2.5).
template <int D>
struct Plan {
  static constexpr int NB = D == 3 ? 27 : 9;
  static constexpr int INTS = D == 3 ? 32 : 16;
  static constexpr int NBO = 2 + D;  // offset of the neighbour slots
};

template <int D>
__device__ __forceinline__ BlockInfo plan_block(const int32_t* pl) {
  BlockInfo b;
  b.slot = pl[0];
  b.lvl = pl[1] & 255;
  b.tree = (pl[1] >> 8) & 0xffff;
#pragma unroll
  for (int a = 0; a < 3; ++a) b.c[a] = a < D ? pl[2 + a] : 0;
  return b;
}

// Ghost gather for a block with a uniform neighbourhood: node i of an axis
// comes from the left neighbour (i < 0, local i + B - 1), the block itself
// (0 <= i <= B - 2) or the right neighbour (i >= B - 1, local i - (B - 1));
// the tile box of width W is filled (NV variables, TF -> TT).  Loads are issued
// U at a time before their stores so that they are in flight together.  With
// commit, block-edge nodes taken from a neighbour are written back into Fw
// where they differ (the neighbour owns them).
template <int D, int B, int W, int NV, typename TF, typename TT>
__device__ __forceinline__ void gather_uniform(const PoolView& pv, const BlockInfo& b, const int32_t* nb,
                                               const TF* F, TF* Fw, TT* tile, bool commit) {
  using Gm = Geo<D, B>;
  using Bx = Box<D, B, W>;
  constexpr int U = 4;
  const int64_t own = (int64_t)b.slot * NV * pv.vs;
  for (int q0 = threadIdx.x; q0 < Bx::NPTS; q0 += U * blockDim.x) {
    int64_t at[U];
    int idx[U], li[U];
    bool ok[U], ed[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u * blockDim.x;
      ok[u] = q < Bx::NPTS;
      const int qq = ok[u] ? q : 0;
      const int ijk[3] = {qq % Bx::S - W, (qq / Bx::S) % Bx::S - W, D == 3 ? qq / (Bx::S * Bx::S) - W : 0};
      int n = 0, mul = 1, l3[3] = {0, 0, 0};
      bool inner = true;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int x = ijk[a];
        const int s = x < 0 ? 0 : (x <= B - 2 ? 1 : 2);
        l3[a] = x - (s - 1) * (B - 1);
        n += s * mul;
        mul *= 3;
        inner &= (x >= 0 && x <= B - 1);
      }
      const int slot = nb[n];
      at[u] = (int64_t)slot * NV * pv.vs + Gm::lin(l3[0], l3[1], l3[2]);
      idx[u] = Bx::tix(ijk[0], ijk[1], ijk[2]);
      li[u] = Gm::lin(ijk[0], ijk[1], ijk[2]);
      ed[u] = commit && inner && slot != b.slot;
    }
    TF v[U][NV];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int w = 0; w < NV; ++w) v[u][w] = ok[u] ? F[at[u] + (int64_t)w * pv.vs] : TF(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
#pragma unroll
      for (int w = 0; w < NV; ++w) {
        tile[w * Bx::TILE + idx[u]] = (TT)v[u][w];
        if (ed[u]) {
          const int64_t me = own + (int64_t)w * pv.vs + li[u];
          if (F[me] != v[u][w]) Fw[me] = v[u][w];
        }
      }
    }
  }
}

// Gather table of a tile box, the same for every block: entry q (tile index
// of node (i, j, k), x fastest) = local offset of the node in the block that
// owns it in a uniform neighbourhood | neighbour index (0 .. 3^d - 1) << 16 |
// (node inside the block) << 21.
template <int D, int B, int W>
__device__ void build_gtab(int32_t* gtab) {
  using Bx = Box<D, B, W>;
  using Gm = Geo<D, B>;
  for (int q = threadIdx.x; q < Bx::NPTS; q += blockDim.x) {
    const int ijk[3] = {q % Bx::S - W, (q / Bx::S) % Bx::S - W, D == 3 ? q / (Bx::S * Bx::S) - W : 0};
    int n = 0, mul = 1, l3[3] = {0, 0, 0};
    bool inner = true;
    for (int a = 0; a < D; ++a) {
      const int x = ijk[a];
      const int s = x < 0 ? 0 : (x <= B - 2 ? 1 : 2);
      l3[a] = x - (s - 1) * (B - 1);
      n += s * mul;
      mul *= 3;
      inner &= (x >= 0 && x <= B - 1);
    }
    gtab[q] = Gm::lin(l3[0], l3[1], l3[2]) | (n << 16) | ((inner ? 1 : 0) << 21);
  }
}

// Uniform-neighbourhood gather through the gather table: nbase[n] is the pool
// offset of neighbour n's variable 0 (slot * NV * vs), own the block's.
// Same values as gather_uniform.
template <int D, int B, int W, int NV, typename TF, typename TT, typename G = CtaGroup>
__device__ __forceinline__ void gather_table(const PoolView& pv, int64_t own, const int64_t* nbase,
                                             const int32_t* gtab, const TF* F, TF* Fw, TT* tile, bool commit) {
  const G g{};
  using Bx = Box<D, B, W>;
  using Gm = Geo<D, B>;
  constexpr int U = 4;
  // points q0 + u * stride, u < UU: table entries, then the UU loads together
  auto chunk = [&](auto uu, int q0, int stride) {
    constexpr int UU = decltype(uu)::value;
    int64_t at[UU];
    bool ok[UU], ed[UU];
#pragma unroll
    for (int u = 0; u < UU; ++u) {
      const int q = q0 + u * stride;
      ok[u] = q < Bx::NPTS;
      const int e = gtab[ok[u] ? q : 0];
      const int64_t nbv = nbase[(e >> 16) & 31];
      at[u] = nbv + (e & 0xffff);
      ed[u] = commit && ((e >> 21) & 1) && nbv != own;
    }
    TF v[UU][NV];
#pragma unroll
    for (int u = 0; u < UU; ++u)
#pragma unroll
      for (int w = 0; w < NV; ++w) v[u][w] = ok[u] ? F[at[u] + (int64_t)w * pv.vs] : TF(0);
#pragma unroll
    for (int u = 0; u < UU; ++u) {
      if (!ok[u]) continue;
      const int q = q0 + u * stride;
#pragma unroll
      for (int w = 0; w < NV; ++w) {
        tile[w * Bx::TILE + q] = (TT)v[u][w];
        if (ed[u]) {
          const int i = q % Bx::S - W, j = (q / Bx::S) % Bx::S - W, k = D == 3 ? q / (Bx::S * Bx::S) - W : 0;
          const int64_t me = own + (int64_t)w * pv.vs + Gm::lin(i, j, k);
          if (F[me] != v[u][w]) Fw[me] = v[u][w];
        }
      }
    }
  };
  if constexpr (G::kSize > 0) {
    // group size known at compile time: full chunks of U, then one chunk just
    // wide enough for the remaining points
    constexpr int SZ = G::kSize, FULL = Bx::NPTS / (U * SZ) * (U * SZ);
    constexpr int UT = (Bx::NPTS - FULL + SZ - 1) / SZ;
    for (int q0 = g.rank(); q0 < FULL; q0 += U * SZ) chunk(std::integral_constant<int, U>{}, q0, SZ);
    if constexpr (UT > 0) chunk(std::integral_constant<int, UT>{}, FULL + g.rank(), SZ);
  } else {
    for (int q0 = g.rank(); q0 < Bx::NPTS; q0 += U * g.size()) chunk(std::integral_constant<int, U>{}, q0, g.size());
  }
}

// Tensor-product prediction at half-coarse position o (per axis, odd = between
// coarse nodes) from a tile whose coarse node n sits at tile index n*stride.
// x first, then y, then z.  Used by refinement (stride 1: the mother's tile) and
// by the details (stride 2: even nodes of the block's own tile).
template <int D, int B, int W, typename TT, typename TA = TT>
__device__ __forceinline__ TA predict_tile(const TT* tile, const int o[3], int stride) {
  using Gm = Box<D, B, W>;
  int base[3] = {0, 0, 0}, ns[3] = {1, 1, 1};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int fl = o[a] >> 1;  // floor(o / 2)
    if (o[a] & 1) { ns[a] = 4; base[a] = fl - 1; }
    else base[a] = fl;
  }
  TA vx[4][4];
  for (int sz = 0; sz < ns[2]; ++sz)
    for (int sy = 0; sy < ns[1]; ++sy) {
      const int y = stride * (base[1] + sy), z = D == 3 ? stride * (base[2] + sz) : 0;
      if (ns[0] == 4) {
        const int x0 = stride * base[0];
        vx[sz][sy] = dd4((TA)tile[Gm::tix(x0, y, z)], (TA)tile[Gm::tix(x0 + stride, y, z)],
                         (TA)tile[Gm::tix(x0 + 2 * stride, y, z)], (TA)tile[Gm::tix(x0 + 3 * stride, y, z)]);
      } else {
        vx[sz][sy] = (TA)tile[Gm::tix(stride * base[0], y, z)];
      }
    }
  TA vy[4];
  for (int sz = 0; sz < ns[2]; ++sz)
    vy[sz] = ns[1] == 4 ? dd4(vx[sz][0], vx[sz][1], vx[sz][2], vx[sz][3]) : vx[sz][0];
  return ns[2] == 4 ? dd4(vy[0], vy[1], vy[2], vy[3]) : vy[0];
}

template <typename T>
__device__ __forceinline__ T* smem_as(size_t offset_bytes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return reinterpret_cast<T*>(smem_raw + offset_bytes);
}

// Exclusive scan of n int2 pairs (in -> out) by one CTA of NT threads: PER
// consecutive pairs per thread per pass, a running carry between passes; the
// totals go to tot[0..1].  The input is read past L1 (written by other CTAs of
// the same grid).  Every thread of the CTA takes part.
template <int NT, int PER>
__device__ void cta_scan2(const int32_t* in, int32_t* out, int n, int32_t* tot) {
  __shared__ int2 wt[NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int2 carry = make_int2(0, 0);
  for (int base = 0; base < n; base += NT * PER) {
    int2 loc[PER];
    int2 s = make_int2(0, 0);
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int i = base + threadIdx.x * PER + r;
      loc[r] = i < n ? make_int2(__ldcg(in + 2 * i), __ldcg(in + 2 * i + 1)) : make_int2(0, 0);
      s.x += loc[r].x;
      s.y += loc[r].y;
    }
    int2 v = s;  // inclusive scan within the warp, then over the warp totals
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, v.x, o), y = __shfl_up_sync(0xffffffffu, v.y, o);
      if (lane >= o) { v.x += x; v.y += y; }
    }
    if (lane == 31) wt[w] = v;
    __syncthreads();
    if (w == 0) {
      int2 t = lane < NT / 32 ? wt[lane] : make_int2(0, 0);
      for (int o = 1; o < NT / 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, t.x, o), y = __shfl_up_sync(0xffffffffu, t.y, o);
        if (lane >= o) { t.x += x; t.y += y; }
      }
      if (lane < NT / 32) wt[lane] = t;
    }
    __syncthreads();
    if (w > 0) { v.x += wt[w - 1].x; v.y += wt[w - 1].y; }
    int2 run = make_int2(carry.x + v.x - s.x, carry.y + v.y - s.y);
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int i = base + threadIdx.x * PER + r;
      if (i < n) { out[2 * i] = run.x; out[2 * i + 1] = run.y; }
      run.x += loc[r].x;
      run.y += loc[r].y;
    }
    carry.x += wt[NT / 32 - 1].x;
    carry.y += wt[NT / 32 - 1].y;
    __syncthreads();
  }
  if (threadIdx.x == 0 && tot) { tot[0] = carry.x; tot[1] = carry.y; }
}

// True in every thread of the CTA of the grid that finishes last; the writes
// of every other CTA of the grid are visible to it.  The caller resets
// ctas_done.
__device__ __forceinline__ bool last_cta_all(Counters* c) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&c->ctas_done, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace mr

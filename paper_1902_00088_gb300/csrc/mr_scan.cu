// Exclusive scan of int2 pairs and the small bookkeeping kernels of the tree
// maintenance (counters, list copies, fills).
#include <atomic>

#include "mr_internal.h"

namespace mr {

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches += n; }
int64_t kernel_launches() { return g_launches.load(); }

constexpr int kScanThreads = 256;
constexpr int kPer = kScanChunk / kScanThreads;  // 8 pairs per thread

__device__ __forceinline__ int64_t scan_n(const int32_t* n_dev, int64_t n_host) {
  return n_dev ? (int64_t)*n_dev : n_host;
}

// inclusive block scan of (a, b) over 256 threads
__device__ __forceinline__ int2 block_incl_scan(int2 v, int2* warp_tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    int x = __shfl_up_sync(0xffffffffu, v.x, o), y = __shfl_up_sync(0xffffffffu, v.y, o);
    if (lane >= o) { v.x += x; v.y += y; }
  }
  if (lane == 31) warp_tot[w] = v;
  __syncthreads();
  if (w == 0) {
    int2 t = lane < (kScanThreads >> 5) ? warp_tot[lane] : make_int2(0, 0);
    for (int o = 1; o < 8; o <<= 1) {
      int x = __shfl_up_sync(0xffffffffu, t.x, o), y = __shfl_up_sync(0xffffffffu, t.y, o);
      if (lane >= o) { t.x += x; t.y += y; }
    }
    if (lane < (kScanThreads >> 5)) warp_tot[lane] = t;
  }
  __syncthreads();
  if (w > 0) { v.x += warp_tot[w - 1].x; v.y += warp_tot[w - 1].y; }
  return v;
}

__global__ void k_scan_reduce(const int32_t* in, const int32_t* n_dev, int64_t n_host, int32_t* partial) {
  pdl_enter();
  __shared__ int2 wt[kScanThreads / 32];
  const int64_t n = scan_n(n_dev, n_host);
  const int64_t start = (int64_t)blockIdx.x * kScanChunk;
  int2 s = make_int2(0, 0);
  for (int r = 0; r < kPer; ++r) {
    const int64_t i = start + (int64_t)threadIdx.x * kPer + r;
    if (i < n) { s.x += in[2 * i]; s.y += in[2 * i + 1]; }
  }
  s = block_incl_scan(s, wt);
  if (threadIdx.x == kScanThreads - 1) {
    partial[2 * blockIdx.x] = s.x;
    partial[2 * blockIdx.x + 1] = s.y;
  }
}

__global__ void k_scan_partials(int32_t* partial, int nchunks, int32_t* tot) {
  pdl_enter();
  __shared__ int2 wt[kScanThreads / 32];
  __shared__ int2 carry;
  if (threadIdx.x == 0) carry = make_int2(0, 0);
  __syncthreads();
  for (int base = 0; base < nchunks; base += kScanThreads) {
    const int i = base + threadIdx.x;
    int2 v = i < nchunks ? make_int2(partial[2 * i], partial[2 * i + 1]) : make_int2(0, 0);
    const int2 inc = block_incl_scan(v, wt);
    const int2 c = carry;
    if (i < nchunks) {
      partial[2 * i] = c.x + inc.x - v.x;
      partial[2 * i + 1] = c.y + inc.y - v.y;
    }
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) { carry.x = c.x + inc.x; carry.y = c.y + inc.y; }
    __syncthreads();
  }
  if (threadIdx.x == 0 && tot) { tot[0] = carry.x; tot[1] = carry.y; }
}

__global__ void k_scan_final(const int32_t* in, int32_t* out, const int32_t* n_dev, int64_t n_host,
                             const int32_t* partial) {
  pdl_enter();
  __shared__ int2 wt[kScanThreads / 32];
  const int64_t n = scan_n(n_dev, n_host);
  const int64_t start = (int64_t)blockIdx.x * kScanChunk;
  if (start >= n) return;
  int2 loc[kPer];
  int2 s = make_int2(0, 0);
  for (int r = 0; r < kPer; ++r) {
    const int64_t i = start + (int64_t)threadIdx.x * kPer + r;
    loc[r] = i < n ? make_int2(in[2 * i], in[2 * i + 1]) : make_int2(0, 0);
    s.x += loc[r].x; s.y += loc[r].y;
  }
  const int2 inc = block_incl_scan(s, wt);
  int2 run = make_int2(partial[2 * blockIdx.x] + inc.x - s.x, partial[2 * blockIdx.x + 1] + inc.y - s.y);
  for (int r = 0; r < kPer; ++r) {
    const int64_t i = start + (int64_t)threadIdx.x * kPer + r;
    if (i < n) { out[2 * i] = run.x; out[2 * i + 1] = run.y; }
    run.x += loc[r].x; run.y += loc[r].y;
  }
}

// Single-CTA exclusive scan: 1024 threads, 4 consecutive pairs per thread per
// pass, a running carry between passes.  One launch; its cost follows the
// device-side count, so it serves lists up to a few million entries.
constexpr int kSingleThreads = 1024, kSinglePer = 4;
__global__ void __launch_bounds__(kSingleThreads) k_scan_single(const int32_t* in, int32_t* out, const int32_t* n_dev,
                                                                int64_t n_host, int32_t* tot) {
  pdl_enter();
  __shared__ int2 wt[kSingleThreads / 32];
  const int64_t n = scan_n(n_dev, n_host);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int2 carry = make_int2(0, 0);
  for (int64_t base = 0; base < n; base += (int64_t)kSingleThreads * kSinglePer) {
    int2 loc[kSinglePer];
    int2 s = make_int2(0, 0);
#pragma unroll
    for (int r = 0; r < kSinglePer; ++r) {
      const int64_t i = base + (int64_t)threadIdx.x * kSinglePer + r;
      loc[r] = i < n ? make_int2(in[2 * i], in[2 * i + 1]) : make_int2(0, 0);
      s.x += loc[r].x;
      s.y += loc[r].y;
    }
    int2 v = s;  // inclusive scan: within the warp, then over the warp totals
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, v.x, o), y = __shfl_up_sync(0xffffffffu, v.y, o);
      if (lane >= o) { v.x += x; v.y += y; }
    }
    if (lane == 31) wt[w] = v;
    __syncthreads();
    if (w == 0) {
      int2 t = wt[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, t.x, o), y = __shfl_up_sync(0xffffffffu, t.y, o);
        if (lane >= o) { t.x += x; t.y += y; }
      }
      wt[lane] = t;
    }
    __syncthreads();
    if (w > 0) { v.x += wt[w - 1].x; v.y += wt[w - 1].y; }
    int2 run = make_int2(carry.x + v.x - s.x, carry.y + v.y - s.y);
#pragma unroll
    for (int r = 0; r < kSinglePer; ++r) {
      const int64_t i = base + (int64_t)threadIdx.x * kSinglePer + r;
      if (i < n) { out[2 * i] = run.x; out[2 * i + 1] = run.y; }
      run.x += loc[r].x;
      run.y += loc[r].y;
    }
    carry.x += wt[kSingleThreads / 32 - 1].x;
    carry.y += wt[kSingleThreads / 32 - 1].y;
    __syncthreads();
  }
  if (threadIdx.x == 0 && tot) { tot[0] = carry.x; tot[1] = carry.y; }
}

void launch_scan2(const int32_t* in, int32_t* out, int32_t* partial, const int32_t* n_dev,
                  int64_t n_host, int32_t* tot, cudaStream_t st, int64_t n_expect, bool pdl) {
  // one CTA while the list is expected to be short (its passes are serial)
  const int64_t n_est = n_expect >= 0 ? n_expect : n_host;
  if (n_est <= 32768) {
    launch_k(pdl, k_scan_single, 1, kSingleThreads, 0, st, in, out, n_dev, n_host, tot);
    count_launch(1);
    return;
  }
  const int nchunks = (int)((n_host + kScanChunk - 1) / kScanChunk);
  const int g = nchunks < 1 ? 1 : nchunks;
  launch_k(pdl, k_scan_reduce, g, kScanThreads, 0, st, in, n_dev, n_host, partial);
  launch_k(pdl, k_scan_partials, 1, kScanThreads, 0, st, partial, g, tot);
  launch_k(pdl, k_scan_final, g, kScanThreads, 0, st, in, out, n_dev, n_host, partial);
  count_launch(3);
}

// Start of a step: coarsening rounds enabled again; hist (nullable) records the
// number of blocks of the adapted grid the step starts from.
__global__ void k_step_begin(Counters* c, int32_t* hist) {
  pdl_enter();
  c->done = 0;
  c->rounds = 0;
  c->first_round = 1;
  if (hist && c->hist_n < kMaxHist) hist[c->hist_n++] = c->n_act;
}

// Stage coefficients of every tree from its device-resident (t, dt); the swirl
// factor uses the device cos (graph-captured steps).
__global__ void k_time_coef(TreeTime* tt, const TreeDev* trees, int ntrees, int swirl) {
  pdl_enter();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ntrees) return;
  TreeTime& T = tt[k];
  const double h = T.dt;
  const double ts[4] = {T.t, T.t + 0.5 * h, T.t + 0.5 * h, T.t + h};
  T.ca[0] = h / 6.0; T.ca[1] = h / 3.0; T.ca[2] = h / 3.0; T.ca[3] = h / 6.0;
  T.cy[0] = h / 2.0; T.cy[1] = h / 2.0; T.cy[2] = h; T.cy[3] = 0.0;
  for (int s = 0; s < 4; ++s) T.ct[s] = swirl ? cos(M_PI * ts[s] / trees[k].rhs[0]) : 0.0;
  for (int s = 0; s < 4; ++s) {
    T.caf[s] = (float)T.ca[s];
    T.cyf[s] = (float)T.cy[s];
    T.ctf[s] = (float)T.ct[s];
  }
}
// End of a coarsening round inside a graph while-node: run another round while
// the last one merged a family and fewer than max_rounds ran.
__global__ void k_time_advance(TreeTime* tt, int ntrees) {
  pdl_enter();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < ntrees) tt[k].t = tt[k].t + tt[k].dt;
}


__global__ void k_fill_i32(int32_t* a, int64_t n, int32_t v) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = v;
}
__global__ void k_fill_i8(int8_t* a, int64_t n, int8_t v) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = v;
}

__global__ void k_sb_check(const int32_t* cells, int64_t ncells, Counters* c) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncells; i += (int64_t)gridDim.x * blockDim.x)
    if (cells[2 * i] != 1) atomicOr(&c->err, kErrLayout);
}

__global__ void k_sb_counters(Counters* c, int32_t* freelist, int64_t n, int64_t cap) {
  pdl_enter();
  const int64_t nf = cap - n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nf; j += (int64_t)gridDim.x * blockDim.x)
    freelist[j] = (int32_t)(cap - 1 - j);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (c->n_new != n) atomicOr(&c->err, kErrLayout);
    c->n_act = (int32_t)n;
    c->n_free = (int32_t)nf;
    c->n_new = (int32_t)n;
    c->n_alloc = 0;
    c->merged = 0;
    c->topo += 1;
  }
}

}  // namespace mr

// Learned refinement proposal (2D): a small per-block CNN predicts whether the
// safety refinement of a block (Sec. 2.1 step 1) will be kept after the step.
// Exact detail thresholding stays the fallback (a block whose own details are
// >= eps is always refined) and the miss check (misses are counted after the step).
//
// Network on x[2][T][T] (T = Bs + 2 ng, the synchronised tile):
//   h1 = relu(conv3x3 s1 (2 -> 16)), h2 = relu(conv3x3 s2 (16 -> 16)),
//   h3 = relu(conv3x3 s2 (16 -> 16)), z = global max of h3, p = sigmoid(wl.z + bl).
// Parameters packed W1 b1 W2 b2 W3 b3 wl bl (4961 values).  Training keeps FP32
// master weights (Adam); inference uses BF16-rounded weights, FP32 accumulation.
// Input channels: 0 = field variable 0 minus its tile-centre value, divided by
// the largest such difference on the tile; 1 = log10(1e-3 + |d|/(s_v eps)) of
// the block's details (max over variables) at interior nodes, -3 elsewhere.
#include <cuda_bf16.h>

#include "mr_device.cuh"
#include "mr_cnn.h"

namespace mr {

constexpr int kC = 16;
constexpr int kW1 = 0, kB1 = kW1 + kC * 2 * 9, kW2 = kB1 + kC, kB2 = kW2 + kC * kC * 9,
              kW3 = kB2 + kC, kB3 = kW3 + kC * kC * 9, kWL = kB3 + kC, kBL = kWL + kC;
static_assert(kBL + 1 == kCnnParams, "parameter count");

template <int T>
struct CnnGeo {
  static constexpr int T2 = (T - 1) / 2 + 1;
  static constexpr int T3 = (T2 - 1) / 2 + 1;
  static constexpr int NX = 2 * T * T;
  static constexpr int N1 = kC * T * T;
  static constexpr int N2 = kC * T2 * T2;
  static constexpr int N3 = kC * T3 * T3;
};

// ------------------------------------------------------------- features ------
// Input tile of the network for every active block: channel 0 = variable 0
// minus its centre value over its largest deviation; channel 1 =
// log10(1e-3 + |d| / (s_v eps)) at the odd interior nodes (largest over the
// variables), -3 elsewhere.  FP32 throughout (a feature, not a decision; FP64
// runs at a small fraction of the FP32 rate here); the details come from the
// separable 4-point prediction, x on coarse rows then y.
template <int B>
struct FeatGeo {
  using Gm = Geo<2, B>;
  using Bx = Box<2, B, kG>;
  static constexpr int NC = (B + 1) / 2 + 2;  // coarse rows -1 .. (B+1)/2
  static constexpr int NX = NC * B;
  static size_t smem(int nv) {
    return kRingBytesD<2> + sizeof(float) * ((size_t)nv * (Gm::TILE + Bx::CBOX + Bx::SCR) + NX + Gm::NI);
  }
};

template <int B, typename TS>
__global__ void __launch_bounds__(256) k_features(PoolView pv, const TS* __restrict__ y,
                                                  float* __restrict__ feat, float* __restrict__ mpre,
                                                  int64_t base) {
  pdl_enter();
  using Gm = Geo<2, B>;
  using Bx = Box<2, B, kG>;
  using FG = FeatGeo<B>;
  constexpr int T = Gm::T;
  const int nv = pv.nvar;
  RingD<2>& R = *smem_as<RingD<2>>(0);
  __shared__ float red[2][32];
  float* tile = smem_as<float>(kRingBytesD<2>);
  float* cbox = tile + nv * Gm::TILE;
  float* scr = cbox + nv * Bx::CBOX;
  float* X = scr + nv * Bx::SCR;
  float* dmap = X + FG::NX;
  const int nact = pv.cnt->n_act;
  for (int p = blockIdx.x; p < nact; p += gridDim.x) {
    const BlockInfo b = load_block(pv, pv.act[p]);
    const TreeDev& td = pv.trees[b.tree];
    float* out = feat + (base + p) * (int64_t)(2 * T * T);
    build_ring<2, B>(pv, td, b, R);
    __syncthreads();
    fill_tile<2, B, TS, float>(pv, b, y, (TS*)y, tile, false, R, cbox, scr);
    for (int q = threadIdx.x; q < Gm::NI; q += blockDim.x) dmap[q] = 0.f;
    __syncthreads();
    const float centre = tile[Gm::tix((B - 1) / 2, (B - 1) / 2, 0)];
    float mx = 0.f;
    for (int idx = threadIdx.x; idx < Gm::TILE; idx += blockDim.x) mx = fmaxf(mx, fabsf(tile[idx] - centre));
    for (int s = 16; s > 0; s >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[0][w]);
    const float inv = mx > 0.f ? 1.f / mx : 0.f;
    for (int v = 0; v < nv; ++v) {
      const float* tv = tile + v * Gm::TILE;
      double svd = pv.norm_kind == 1 ? pv.svar[b.tree * nv + v] : 1.0;
      const float sv = svd == 0.0 ? 1.f : (float)svd;
      for (int idx = threadIdx.x; idx < FG::NX; idx += blockDim.x) {  // x pass on coarse rows
        const int x = idx % B, yy = 2 * (idx / B - 1);
        X[idx] = (x & 1) ? dd4(tv[Gm::tix(x - 3, yy, 0)], tv[Gm::tix(x - 1, yy, 0)], tv[Gm::tix(x + 1, yy, 0)],
                               tv[Gm::tix(x + 3, yy, 0)])
                         : tv[Gm::tix(x, yy, 0)];
      }
      __syncthreads();
      for (int q = threadIdx.x; q < Gm::NI; q += blockDim.x) {
        const int i = q % B, j = q / B;
        if (((i | j) & 1) == 0) continue;
        float pr;
        if ((j & 1) == 0) {
          pr = X[(j / 2 + 1) * B + i];
        } else {
          const int m0 = (j - 1) / 2;
          pr = dd4(X[m0 * B + i], X[(m0 + 1) * B + i], X[(m0 + 2) * B + i], X[(m0 + 3) * B + i]);
        }
        dmap[q] = fmaxf(dmap[q], fabsf(tv[Gm::tix(i, j, 0)] - pr) / sv);
      }
      __syncthreads();
    }
    float md = 0.f;
    const float ieps = (float)(1.0 / td.eps);
    for (int idx = threadIdx.x; idx < Gm::TILE; idx += blockDim.x) {
      const int i = idx % T - Gm::G, j = idx / T - Gm::G;
      out[idx] = (tile[idx] - centre) * inv;
      float dv = -3.f;
      if (i >= 0 && i < B && j >= 0 && j < B && ((i | j) & 1)) {
        const float dm = dmap[j * B + i];
        md = fmaxf(md, dm);
        dv = log10f(1e-3f + dm * ieps);
      }
      out[T * T + idx] = dv;
    }
    for (int s = 16; s > 0; s >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, s));
    if ((threadIdx.x & 31) == 0) red[1][threadIdx.x >> 5] = md;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) md = fmaxf(md, red[1][w]);
      if (mpre) mpre[p] = md;
    }
    __syncthreads();
  }
}

// -------------------------------------------------------- forward pass -------
template <int T, typename WT>
__device__ float cnn_forward(const float* x, const WT* w, float* h1, float* h2, float* h3, float* z) {
  using CG = CnnGeo<T>;
  constexpr int T2 = CG::T2, T3 = CG::T3;
  for (int idx = threadIdx.x; idx < CG::N1; idx += blockDim.x) {
    const int o = idx / (T * T), pix = idx % (T * T), i = pix / T, j = pix % T;
    float s = (float)w[kB1 + o];
    for (int c = 0; c < 2; ++c)
      for (int di = 0; di < 3; ++di) {
        const int ii = i + di - 1;
        if (ii < 0 || ii >= T) continue;
        for (int dj = 0; dj < 3; ++dj) {
          const int jj = j + dj - 1;
          if (jj < 0 || jj >= T) continue;
          s += (float)w[kW1 + ((o * 2 + c) * 3 + di) * 3 + dj] * x[c * T * T + ii * T + jj];
        }
      }
    h1[idx] = fmaxf(s, 0.f);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < CG::N2; idx += blockDim.x) {
    const int o = idx / (T2 * T2), pix = idx % (T2 * T2), i = pix / T2, j = pix % T2;
    float s = (float)w[kB2 + o];
    for (int c = 0; c < kC; ++c)
      for (int di = 0; di < 3; ++di) {
        const int ii = 2 * i + di - 1;
        if (ii < 0 || ii >= T) continue;
        for (int dj = 0; dj < 3; ++dj) {
          const int jj = 2 * j + dj - 1;
          if (jj < 0 || jj >= T) continue;
          s += (float)w[kW2 + ((o * kC + c) * 3 + di) * 3 + dj] * h1[c * T * T + ii * T + jj];
        }
      }
    h2[idx] = fmaxf(s, 0.f);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < CG::N3; idx += blockDim.x) {
    const int o = idx / (T3 * T3), pix = idx % (T3 * T3), i = pix / T3, j = pix % T3;
    float s = (float)w[kB3 + o];
    for (int c = 0; c < kC; ++c)
      for (int di = 0; di < 3; ++di) {
        const int ii = 2 * i + di - 1;
        if (ii < 0 || ii >= T2) continue;
        for (int dj = 0; dj < 3; ++dj) {
          const int jj = 2 * j + dj - 1;
          if (jj < 0 || jj >= T2) continue;
          s += (float)w[kW3 + ((o * kC + c) * 3 + di) * 3 + dj] * h2[c * T2 * T2 + ii * T2 + jj];
        }
      }
    h3[idx] = fmaxf(s, 0.f);
  }
  __syncthreads();
  if (threadIdx.x < kC) {
    float m = h3[threadIdx.x * T3 * T3];
    for (int q = 1; q < T3 * T3; ++q) m = fmaxf(m, h3[threadIdx.x * T3 * T3 + q]);
    z[threadIdx.x] = m;
  }
  __syncthreads();
  float logit = (float)w[kBL];
  for (int o = 0; o < kC; ++o) logit += (float)w[kWL + o] * z[o];
  return logit;
}

// Inference: p for every active block below Jmax (others get 0).  The
// weights are staged once per CTA in shared memory as floats, transposed so
// that the 16 output channels of a tap are contiguous; each thread computes
// all 16 output channels of one pixel (one input load feeds 16 FMAs, the 16
// weights come as four broadcast 16-byte loads).  Per output the sum runs in
// the order of cnn_forward (bias, then input channel, row, column), so the
// probabilities equal the training forward pass bit for bit.
template <int T>
struct InferGeo {
  using CG = CnnGeo<T>;
  // transposed weights: layer l, input channel c, tap t -> 16 floats (o)
  static constexpr int WT1 = 0, WT2 = WT1 + 2 * 9 * kC, WT3 = WT2 + kC * 9 * kC, WTE = WT3 + kC * 9 * kC;
  static constexpr int NW = WTE + 4 * kC + 1;  // + b1, b2, b3, wl, bl
  static constexpr int X0 = (NW + 3) / 4 * 4;  // activations after the weights
  static constexpr size_t SMEM = sizeof(float) * (X0 + CG::NX + CG::N1 + CG::N2 + CG::N3);
};

template <int T, int CIN, int S>
__device__ __forceinline__ void conv_all_o(const float* __restrict__ in, int Tin, const float* __restrict__ wt,
                                           const float* __restrict__ bias, float* __restrict__ out, int Tout) {
  for (int pix = threadIdx.x; pix < Tout * Tout; pix += blockDim.x) {
    const int i = pix / Tout, j = pix % Tout;
    float acc[kC];
#pragma unroll
    for (int o = 0; o < kC; ++o) acc[o] = bias[o];
    for (int c = 0; c < CIN; ++c) {
#pragma unroll
      for (int di = 0; di < 3; ++di) {
        const int ii = S * i + di - 1;
        if (ii < 0 || ii >= Tin) continue;
#pragma unroll
        for (int dj = 0; dj < 3; ++dj) {
          const int jj = S * j + dj - 1;
          if (jj < 0 || jj >= Tin) continue;
          const float xv = in[c * Tin * Tin + ii * Tin + jj];
          const float4* w4 = reinterpret_cast<const float4*>(wt + ((c * 3 + di) * 3 + dj) * kC);
#pragma unroll
          for (int o4 = 0; o4 < kC / 4; ++o4) {
            const float4 wv = w4[o4];
            acc[4 * o4 + 0] += wv.x * xv;
            acc[4 * o4 + 1] += wv.y * xv;
            acc[4 * o4 + 2] += wv.z * xv;
            acc[4 * o4 + 3] += wv.w * xv;
          }
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kC; ++o) out[o * Tout * Tout + pix] = fmaxf(acc[o], 0.f);
  }
}

template <int T>
__global__ void __launch_bounds__(256) k_cnn_infer(PoolView pv, const float* __restrict__ feat,
                                                   const __nv_bfloat16* __restrict__ wb,
                                                   float* __restrict__ prob, int64_t n_explicit) {
  pdl_enter();
  using CG = CnnGeo<T>;
  using IG = InferGeo<T>;
  float* ws = smem_as<float>(0);
  float* x = ws + IG::X0;
  float* h1 = x + CG::NX;
  float* h2 = h1 + CG::N1;
  float* h3 = h2 + CG::N2;
  __shared__ float z[kC];
  // stage the weights, transposed to [c][tap][o]
  for (int q = threadIdx.x; q < kC * 2 * 9; q += blockDim.x) {
    const int o = q / 18, c = (q / 9) % 2, t = q % 9;
    ws[IG::WT1 + (c * 9 + t) * kC + o] = __bfloat162float(wb[kW1 + q]);
  }
  for (int q = threadIdx.x; q < kC * kC * 9; q += blockDim.x) {
    const int o = q / (kC * 9), c = (q / 9) % kC, t = q % 9;
    ws[IG::WT2 + (c * 9 + t) * kC + o] = __bfloat162float(wb[kW2 + q]);
    ws[IG::WT3 + (c * 9 + t) * kC + o] = __bfloat162float(wb[kW3 + q]);
  }
  if (threadIdx.x < kC) {
    ws[IG::WTE + threadIdx.x] = __bfloat162float(wb[kB1 + threadIdx.x]);
    ws[IG::WTE + kC + threadIdx.x] = __bfloat162float(wb[kB2 + threadIdx.x]);
    ws[IG::WTE + 2 * kC + threadIdx.x] = __bfloat162float(wb[kB3 + threadIdx.x]);
    ws[IG::WTE + 3 * kC + threadIdx.x] = __bfloat162float(wb[kWL + threadIdx.x]);
  }
  if (threadIdx.x == 0) ws[IG::WTE + 4 * kC] = __bfloat162float(wb[kBL]);
  __syncthreads();
  const int64_t n = n_explicit >= 0 ? n_explicit : (int64_t)pv.cnt->n_act;
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    if (n_explicit < 0) {
      const int s = pv.act[p];
      if (pv.lvl[s] >= pv.trees[pv.tree[s]].Jmax) {
        if (threadIdx.x == 0) prob[p] = 0.f;
        continue;
      }
    }
    for (int idx = threadIdx.x; idx < CG::NX; idx += blockDim.x) x[idx] = feat[p * CG::NX + idx];
    __syncthreads();
    conv_all_o<T, 2, 1>(x, T, ws + IG::WT1, ws + IG::WTE, h1, T);
    __syncthreads();
    conv_all_o<T, kC, 2>(h1, T, ws + IG::WT2, ws + IG::WTE + kC, h2, CG::T2);
    __syncthreads();
    conv_all_o<T, kC, 2>(h2, CG::T2, ws + IG::WT3, ws + IG::WTE + 2 * kC, h3, CG::T3);
    __syncthreads();
    if (threadIdx.x < kC) {
      float m = h3[threadIdx.x * CG::T3 * CG::T3];
      for (int q = 1; q < CG::T3 * CG::T3; ++q) m = fmaxf(m, h3[threadIdx.x * CG::T3 * CG::T3 + q]);
      z[threadIdx.x] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float logit = ws[IG::WTE + 4 * kC];
      for (int o = 0; o < kC; ++o) logit += ws[IG::WTE + 3 * kC + o] * z[o];
      prob[p] = 1.f / (1.f + expf(-logit));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------- training (fwd + bwd) ---
// Samples [s0, s0 + nb) of the dataset (index list idx), mean weighted BCE.
// Each CTA takes samples blockIdx.x, blockIdx.x + gridDim.x, ...; gradients
// accumulate in shared memory and are added to the global buffer once.
template <int T>
__global__ void __launch_bounds__(256) k_cnn_train(const float* __restrict__ feat,
                                                   const float* __restrict__ label,
                                                   const int32_t* __restrict__ idx, int64_t s0,
                                                   int nb, const float* __restrict__ w, float w_pos,
                                                   float* __restrict__ grad, float* __restrict__ loss,
                                                   float* __restrict__ prob_out) {
  pdl_enter();
  using CG = CnnGeo<T>;
  constexpr int T2 = CG::T2, T3 = CG::T3;
  float* x = smem_as<float>(0);
  float* h1 = x + CG::NX;
  float* h2 = h1 + CG::N1;
  float* h3 = h2 + CG::N2;
  float* dh2 = h3 + CG::N3;
  float* gacc = dh2 + CG::N2;
  __shared__ float z[kC], dz[kC];
  __shared__ int arg[kC];
  __shared__ float dlogit_s;
  for (int q = threadIdx.x; q < kCnnParams; q += blockDim.x) gacc[q] = 0.f;
  float lsum = 0.f;
  __syncthreads();
  for (int sb = blockIdx.x; sb < nb; sb += gridDim.x) {
    const int64_t sidx = idx ? (int64_t)idx[s0 + sb] : s0 + sb;
    for (int q = threadIdx.x; q < CG::NX; q += blockDim.x) x[q] = feat[sidx * CG::NX + q];
    __syncthreads();
    const float logit = cnn_forward<T>(x, w, h1, h2, h3, z);
    if (threadIdx.x == 0) {
      const float p = 1.f / (1.f + expf(-logit));
      const float yv = label[sidx];
      const float pc = fminf(fmaxf(p, 1e-7f), 1.f - 1e-7f);
      lsum += -(w_pos * yv * logf(pc) + (1.f - yv) * logf(1.f - pc)) / nb;
      const float dl = (yv * w_pos * (p - 1.f) + (1.f - yv) * p) / nb;
      dlogit_s = dl;
      if (prob_out) prob_out[s0 + sb] = p;
    }
    if (threadIdx.x < kC) {
      int a = 0;
      float m = h3[threadIdx.x * T3 * T3];
      for (int q = 1; q < T3 * T3; ++q)
        if (h3[threadIdx.x * T3 * T3 + q] > m) { m = h3[threadIdx.x * T3 * T3 + q]; a = q; }
      arg[threadIdx.x] = a;
    }
    __syncthreads();
    const float dl = dlogit_s;
    if (threadIdx.x < kC) {
      gacc[kWL + threadIdx.x] += dl * z[threadIdx.x];
      dz[threadIdx.x] = dl * w[kWL + threadIdx.x];
    }
    if (threadIdx.x == 0) gacc[kBL] += dl;
    for (int q = threadIdx.x; q < CG::N2; q += blockDim.x) dh2[q] = 0.f;
    __syncthreads();
    // conv3: da3 is nonzero only at each channel's (first) maximum, if positive
    for (int q = threadIdx.x; q < kC * kC * 9; q += blockDim.x) {
      const int o = q / (kC * 9), c = (q / 9) % kC, di = (q / 3) % 3, dj = q % 3;
      const int a = arg[o];
      const float da = h3[o * T3 * T3 + a] > 0.f ? dz[o] : 0.f;
      const int ii = 2 * (a / T3) + di - 1, jj = 2 * (a % T3) + dj - 1;
      if (da != 0.f && ii >= 0 && ii < T2 && jj >= 0 && jj < T2) {
        gacc[kW3 + q] += da * h2[c * T2 * T2 + ii * T2 + jj];
        atomicAdd(&dh2[c * T2 * T2 + ii * T2 + jj], da * w[kW3 + q]);
      }
    }
    if (threadIdx.x < kC) {
      const int o = threadIdx.x;
      gacc[kB3 + o] += h3[o * T3 * T3 + arg[o]] > 0.f ? dz[o] : 0.f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < CG::N2; q += blockDim.x)  // da2 = dh2 * relu'(a2)
      if (!(h2[q] > 0.f)) dh2[q] = 0.f;
    __syncthreads();
    // conv2 weights: dW2[o][c][di][dj] = sum_pix da2[o][pix] h1[c][2i+di-1][2j+dj-1]
    for (int q = threadIdx.x; q < kC * kC * 9; q += blockDim.x) {
      const int o = q / (kC * 9), c = (q / 9) % kC, di = (q / 3) % 3, dj = q % 3;
      float s = 0.f;
      for (int pix = 0; pix < T2 * T2; ++pix) {
        const float da = dh2[o * T2 * T2 + pix];
        if (da == 0.f) continue;
        const int ii = 2 * (pix / T2) + di - 1, jj = 2 * (pix % T2) + dj - 1;
        if (ii >= 0 && ii < T && jj >= 0 && jj < T) s += da * h1[c * T * T + ii * T + jj];
      }
      gacc[kW2 + q] += s;
    }
    if (threadIdx.x < kC) {
      float s = 0.f;
      for (int pix = 0; pix < T2 * T2; ++pix) s += dh2[threadIdx.x * T2 * T2 + pix];
      gacc[kB2 + threadIdx.x] += s;
    }
    __syncthreads();
    // da1 = conv2^T(da2) * relu'(a1), written over h1
    for (int q = threadIdx.x; q < CG::N1; q += blockDim.x) {
      const int o = q / (T * T), pix = q % (T * T), i = pix / T, j = pix % T;
      float s = 0.f;
      if (h1[q] > 0.f) {
        for (int di = 0; di < 3; ++di) {
          const int ti = i + 1 - di;
          if (ti < 0 || (ti & 1) || ti / 2 >= T2) continue;
          for (int dj = 0; dj < 3; ++dj) {
            const int tj = j + 1 - dj;
            if (tj < 0 || (tj & 1) || tj / 2 >= T2) continue;
            for (int c2 = 0; c2 < kC; ++c2)
              s += w[kW2 + ((c2 * kC + o) * 3 + di) * 3 + dj] * dh2[c2 * T2 * T2 + (ti / 2) * T2 + tj / 2];
          }
        }
      }
      h1[q] = s;  // now da1
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kC * 2 * 9 + kC; q += blockDim.x) {
      if (q < kC * 2 * 9) {
        const int o = q / 18, c = (q / 9) % 2, di = (q / 3) % 3, dj = q % 3;
        float s = 0.f;
        for (int pix = 0; pix < T * T; ++pix) {
          const float da = h1[o * T * T + pix];
          if (da == 0.f) continue;
          const int ii = pix / T + di - 1, jj = pix % T + dj - 1;
          if (ii >= 0 && ii < T && jj >= 0 && jj < T) s += da * x[c * T * T + ii * T + jj];
        }
        gacc[kW1 + q] += s;
      } else {
        const int o = q - kC * 18;
        float s = 0.f;
        for (int pix = 0; pix < T * T; ++pix) s += h1[o * T * T + pix];
        gacc[kB1 + o] += s;
      }
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < kCnnParams; q += blockDim.x)
    if (gacc[q] != 0.f) atomicAdd(&grad[q], gacc[q]);
  if (threadIdx.x == 0 && loss) atomicAdd(loss, lsum);
}

__global__ void k_adam(float* w, float* m, float* v, float* g, int n, float lr, float b1, float b2,
                       float eps, int t, __nv_bfloat16* wb) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // a non-finite gradient entry (seen once in a 64-tree training run, cause
  // not found) is skipped rather than allowed to poison the moments
  const float gi = isfinite(g[i]) ? g[i] : 0.f;
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)t)), vh = vi / (1.f - powf(b2, (float)t));
  w[i] -= lr * mh / (sqrtf(vh) + eps);
  g[i] = 0.f;
  wb[i] = __float2bfloat16(w[i]);
}

__global__ void k_to_bf16(const float* w, __nv_bfloat16* wb, int n) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16(w[i]);
}

// ------------------------------------------------------ proposal at step -----
// flag = 1 (refine) if the block is below Jmax and (p >= tau or its own largest
// normalised detail >= eps); skip marks blocks left unrefined (for the miss check).
__global__ void k_propose(PoolView pv, const float* prob, const float* mpre, float tau, int8_t* skip,
                          int32_t* counts) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += gridDim.x * blockDim.x) {
    const int s = pv.act[p];
    const TreeDev& td = pv.trees[pv.tree[s]];
    const bool below = pv.lvl[s] < td.Jmax;
    const bool net = below && prob[p] >= tau;
    const bool fb = below && (double)mpre[p] >= td.eps;
    pv.flag[s] = (net || fb) ? 1 : 0;
    skip[s] = below && !(net || fb) ? 1 : 0;
    if (below) atomicAdd(&counts[0], 1);
    if (net) atomicAdd(&counts[1], 1);
    if (fb && !net) atomicAdd(&counts[2], 1);
  }
}

// Gradedness closure of +1 flags: a refined block forces the refinement of
// every touching leaf one level coarser (monotone 0 -> 1, order independent).
// The touching leaves are the level-(l-1) leaves covering the ring of
// level-(l+1) cells around the block.  skip (nullable) marks blocks left
// unrefined by a proposal.
template <int D>
__global__ void k_close(PoolView pv, int8_t* skip, int32_t* changed) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  constexpr int NR = D == 3 ? 64 : 16;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += gridDim.x * blockDim.x) {
    const int s = pv.act[p];
    if (pv.flag[s] != 1) continue;
    const BlockInfo b = load_block(pv, s);
    const TreeDev& td = pv.trees[b.tree];
    if (b.lvl >= td.Jmax || b.lvl - 1 < td.Jmin) continue;
    const int64_t nl1 = (int64_t)1 << (b.lvl + 1);
    for (int r = 0; r < NR; ++r) {
      const int q[3] = {r % 4 - 1, (r / 4) % 4 - 1, r / 16 - 1};
      bool inside = true;
      for (int a = 0; a < D; ++a) inside &= (q[a] == 0 || q[a] == 1);
      if (inside) continue;
      int64_t c2[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) c2[a] = ((2 * b.c[a] + q[a]) & (nl1 - 1)) >> 2;
      const int t = tab_get<D>(pv, td, b.lvl - 1, c2);
      if (t >= 0 && pv.flag[t] != 1) {
        pv.flag[t] = 1;
        if (skip) skip[t] = 0;
        atomicAdd(changed, 1);
      }
    }
  }
}

// Refinement indicators given by the caller: flag = +1 for a block below Jmax
// whose mask entry (canonical position) is positive, else 0.
__global__ void k_mask_flags(PoolView pv, const int8_t* mask) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += gridDim.x * blockDim.x) {
    const int s = pv.act[p];
    pv.flag[s] = (mask[p] > 0 && pv.lvl[s] < pv.trees[pv.tree[s]].Jmax) ? 1 : 0;
  }
}

// Miss check: a block left unrefined whose details after the step are >= eps.
__global__ void k_miss_check(PoolView pv, const int8_t* skip, const int32_t* skip_key, int32_t* counts) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += gridDim.x * blockDim.x) {
    const int s = pv.act[p];
    if (!skip[s]) continue;
    const int key = (pv.lvl[s] << 24) ^ (pv.crd[3 * s] << 12) ^ pv.crd[3 * s + 1];
    if (skip_key[s] != key) continue;  // the slot now holds another block
    if (pv.mdet[s] >= pv.trees[pv.tree[s]].eps) atomicAdd(&counts[3], 1);
  }
}

__global__ void k_skip_key(PoolView pv, const int8_t* skip, int32_t* skip_key) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += gridDim.x * blockDim.x) {
    const int s = pv.act[p];
    skip_key[s] = skip[s] ? ((pv.lvl[s] << 24) ^ (pv.crd[3 * s] << 12) ^ pv.crd[3 * s + 1]) : -1;
  }
}

// Labels of the samples recorded before a step: 1 iff the refinement was needed
// -- the block's region is subdivided after the step (its refinement was kept),
// or the block is a leaf again and its details reached eps (what the miss check
// counts as a miss when the block was left unrefined) -- 0 otherwise; -1 for
// blocks at Jmax.
// Samples whose own details were >= eps (mpre) are refined by the exact
// fallback whatever the network says; they get -1 too (not trained on).
__global__ void k_label(PoolView pv, const int32_t* key, const float* mpre, int64_t n, float* label) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int tree = key[4 * i], l = key[4 * i + 1];
    const TreeDev& td = pv.trees[tree];
    if (l >= td.Jmax || (double)mpre[i] >= td.eps) { label[i] = -1.f; continue; }
    int64_t c[3] = {key[4 * i + 2], key[4 * i + 3], 0};
    const int self = tab_get<2>(pv, td, l, c);
    if (self >= 0) {  // merged back: positive iff its details reached eps (the miss check's event)
      label[i] = pv.mdet[self] >= td.eps ? 1.f : 0.f;
      continue;
    }
    bool above = false;
    for (int m = l - 1; m >= td.Jmin && !above; --m) {
      int64_t cm[3] = {c[0] >> (l - m), c[1] >> (l - m), 0};
      above = tab_get<2>(pv, td, m, cm) >= 0;
    }
    label[i] = above ? 0.f : 1.f;
  }
}

__global__ void k_sample_keys(PoolView pv, int32_t* key, int64_t base) {
  pdl_enter();
  const int nact = pv.cnt->n_act;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nact; p += gridDim.x * blockDim.x) {
    const int s = pv.act[p];
    int32_t* k = key + 4 * (base + p);
    k[0] = pv.tree[s];
    k[1] = pv.lvl[s];
    k[2] = pv.crd[3 * s];
    k[3] = pv.crd[3 * s + 1];
  }
}

// ------------------------------------------------------------- launchers -----
template <typename K>
static void prep(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int cnn_tile(int Bs) { return Bs + 2 * kG; }

void launch_features(const PoolView& pv, const void* y, float* feat, float* mpre, int64_t base,
                     int num_sms, cudaStream_t st) {
  const bool d = pv.prec != MR_PREC_FP32;
  if (pv.Bs == 17) {
    const size_t smem = FeatGeo<17>::smem(pv.nvar);
    if (d) { auto k = k_features<17, double>; prep(k, smem); k<<<num_sms * 2, 256, smem, st>>>(pv, (const double*)y, feat, mpre, base); }
    else { auto k = k_features<17, float>; prep(k, smem); k<<<num_sms * 2, 256, smem, st>>>(pv, (const float*)y, feat, mpre, base); }
  } else {
    const size_t smem = FeatGeo<33>::smem(pv.nvar);
    if (d) { auto k = k_features<33, double>; prep(k, smem); k<<<num_sms * 2, 256, smem, st>>>(pv, (const double*)y, feat, mpre, base); }
    else { auto k = k_features<33, float>; prep(k, smem); k<<<num_sms * 2, 256, smem, st>>>(pv, (const float*)y, feat, mpre, base); }
  }
  count_launch();
}

template <int T>
static size_t infer_smem() {
  return InferGeo<T>::SMEM;
}
template <int T>
static size_t train_smem() {
  using CG = CnnGeo<T>;
  return sizeof(float) * (CG::NX + CG::N1 + CG::N2 + CG::N3 + CG::N2 + kCnnParams);
}

void launch_infer(const PoolView& pv, int Bs, const float* feat, const __nv_bfloat16* wb, float* prob,
                  int64_t n_explicit, int num_sms, cudaStream_t st) {
  if (Bs == 17) {
    auto k = k_cnn_infer<25>;
    prep(k, infer_smem<25>());
    k<<<num_sms * 4, 256, infer_smem<25>(), st>>>(pv, feat, wb, prob, n_explicit);
  } else {
    auto k = k_cnn_infer<41>;
    prep(k, infer_smem<41>());
    k<<<num_sms * 2, 256, infer_smem<41>(), st>>>(pv, feat, wb, prob, n_explicit);
  }
  count_launch();
}

void launch_train(int Bs, const float* feat, const float* label, const int32_t* idx, int64_t s0, int nb,
                  const float* w, float w_pos, float* grad, float* loss, float* prob_out, int num_sms,
                  cudaStream_t st) {
  const int grid = nb < num_sms ? nb : num_sms;
  if (Bs == 17) {
    auto k = k_cnn_train<25>;
    prep(k, train_smem<25>());
    k<<<grid, 256, train_smem<25>(), st>>>(feat, label, idx, s0, nb, w, w_pos, grad, loss, prob_out);
  } else {
    auto k = k_cnn_train<41>;
    prep(k, train_smem<41>());
    k<<<grid, 256, train_smem<41>(), st>>>(feat, label, idx, s0, nb, w, w_pos, grad, loss, prob_out);
  }
  count_launch();
}

void launch_adam(float* w, float* m, float* v, float* g, float lr, int t, __nv_bfloat16* wb, cudaStream_t st) {
  k_adam<<<(kCnnParams + 255) / 256, 256, 0, st>>>(w, m, v, g, kCnnParams, lr, 0.9f, 0.999f, 1e-8f, t, wb);
  count_launch();
}
void launch_to_bf16(const float* w, __nv_bfloat16* wb, cudaStream_t st) {
  k_to_bf16<<<(kCnnParams + 255) / 256, 256, 0, st>>>(w, wb, kCnnParams);
  count_launch();
}
void launch_propose(const PoolView& pv, const float* prob, const float* mpre, float tau, int8_t* skip,
                    int32_t* counts, cudaStream_t st) {
  k_propose<<<256, 256, 0, st>>>(pv, prob, mpre, tau, skip, counts);
  count_launch();
}
void launch_close(const PoolView& pv, int8_t* skip, int32_t* changed, cudaStream_t st) {
  if (pv.dim == 3) k_close<3><<<256, 256, 0, st>>>(pv, skip, changed);
  else k_close<2><<<256, 256, 0, st>>>(pv, skip, changed);
  count_launch();
}
void launch_mask_flags(const PoolView& pv, const int8_t* mask, cudaStream_t st) {
  k_mask_flags<<<256, 256, 0, st>>>(pv, mask);
  count_launch();
}
void launch_miss_check(const PoolView& pv, const int8_t* skip, const int32_t* skip_key, int32_t* counts,
                  cudaStream_t st) {
  k_miss_check<<<256, 256, 0, st>>>(pv, skip, skip_key, counts);
  count_launch();
}
void launch_skip_key(const PoolView& pv, const int8_t* skip, int32_t* skip_key, cudaStream_t st) {
  k_skip_key<<<256, 256, 0, st>>>(pv, skip, skip_key);
  count_launch();
}
void launch_sample_keys(const PoolView& pv, int32_t* key, int64_t base, cudaStream_t st) {
  k_sample_keys<<<256, 256, 0, st>>>(pv, key, base);
  count_launch();
}
void launch_label(const PoolView& pv, const int32_t* key, const float* mpre, int64_t n, float* label,
                  cudaStream_t st) {
  k_label<<<256, 256, 0, st>>>(pv, key, mpre, n, label);
  count_launch();
}

}  // namespace mr

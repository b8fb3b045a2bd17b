// Learned refinement proposal: launchers (mr_cnn.cu) used by the host API.
#pragma once
#include <cuda_bf16.h>

#include "mr_internal.h"

namespace mr {

constexpr int kCnnParams = 4961;  // W1 16x2x3x3, b1 16, W2 16x16x3x3, b2 16, W3, b3, wl 16, bl 1

int cnn_tile(int Bs);
void launch_features(const PoolView& pv, const void* y, float* feat, float* mpre, int64_t base,
                     int num_sms, cudaStream_t st);
void launch_infer(const PoolView& pv, int Bs, const float* feat, const __nv_bfloat16* wb, float* prob,
                  int64_t n_explicit, int num_sms, cudaStream_t st);
void launch_train(int Bs, const float* feat, const float* label, const int32_t* idx, int64_t s0, int nb,
                  const float* w, float w_pos, float* grad, float* loss, float* prob_out, int num_sms,
                  cudaStream_t st);
void launch_adam(float* w, float* m, float* v, float* g, float lr, int t, __nv_bfloat16* wb, cudaStream_t st);
void launch_to_bf16(const float* w, __nv_bfloat16* wb, cudaStream_t st);
void launch_propose(const PoolView& pv, const float* prob, const float* mpre, float tau, int8_t* skip,
                    int32_t* counts, cudaStream_t st);
void launch_close(const PoolView& pv, int8_t* skip, int32_t* changed, cudaStream_t st);
void launch_mask_flags(const PoolView& pv, const int8_t* mask, cudaStream_t st);
void launch_miss_check(const PoolView& pv, const int8_t* skip, const int32_t* skip_key, int32_t* counts,
                  cudaStream_t st);
void launch_skip_key(const PoolView& pv, const int8_t* skip, int32_t* skip_key, cudaStream_t st);
void launch_sample_keys(const PoolView& pv, int32_t* key, int64_t base, cudaStream_t st);
void launch_label(const PoolView& pv, const int32_t* key, const float* mpre, int64_t n, float* label,
                  cudaStream_t st);

}  // namespace mr

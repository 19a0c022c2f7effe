// Internal interface of the slope-predictor kernels (mlp.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rtc.h"

// Device state of one predictor network.
struct MlpDev {
    float* master;               // [RTC_MLP_NPARAMS] FP32 weights (W1, b1, W2, b2, W3, b3)
    float* m;                    // Adam first moments
    float* v;                    // Adam second moments
    __nv_bfloat16* w1_bf16;      // [64][208] BF16 copy of W1, zero padded
    __nv_bfloat16* w2_bf16;      // [64][64] BF16 copy of W2
};

size_t mlp_smem_bytes();
cudaError_t mlp_configure();
cudaError_t mlp_launch_refresh(const MlpDev& w, cudaStream_t st);
// CTA partial gradients of a batch: parts [ceil(B/64)][RTC_MLP_NPARAMS + 1] (last = loss sum).
cudaError_t mlp_launch_train(const MlpDev& w, const float* X, const float* T, int B, float* parts,
                             cudaStream_t st);
cudaError_t mlp_launch_train_seq(const MlpDev& w, const float* S, int n_frames, int nv,
                                 const int* nbr, const int2* samples, int B, float inv_sigma,
                                 float* parts, cudaStream_t st);
cudaError_t mlp_launch_forward(const MlpDev& w, const float* X, int B, float* Y, cudaStream_t st);
cudaError_t mlp_launch_predict(const MlpDev& w, const float* ring, int kpad, int head, int nv,
                               const int* nbr, float sigma, float* s_pred, cudaStream_t st);
// Sum the partials; lr > 0 also applies Adam step `step` (from 1).
cudaError_t mlp_launch_update(const MlpDev& w, const float* parts, int nparts, int B, float lr,
                              float beta1, float beta2, float eps, int step, float* grad_out,
                              float* loss_out, cudaStream_t st);

// Host helpers shared by rtc_mlp_* and the handle's predictor (rtc_mlp.cu).
int mlp_alloc(MlpDev& w);
void mlp_free(MlpDev& w);
int mlp_upload(MlpDev& w, const float* params, cudaStream_t st);
#include <vector>
std::vector<int> mlp_neighbours(const int32_t* rc, int nv, int nsub);

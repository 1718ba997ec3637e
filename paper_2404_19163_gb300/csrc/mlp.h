// Learned start proposal: feature and MLP kernels (k_mlp.cu).
#pragma once
#include "common.cuh"

namespace zf {

constexpr int kMlpParams = 5573;  // 16*64 + 64 + 64*64 + 64 + 5*64 + 5

// One thread per sample.  Y (batch x 5) may be null; with grads != null also the per-sample
// gradients (batch x kMlpParams) and losses (batch) of the training loss.
cudaError_t launch_mlp(const float* P, const float* mean, const float* stdv, const float* X, int batch, float* Y,
                       const float* tgt, const int* ord, float w, float* grads, double* losses, cudaStream_t s);
cudaError_t launch_mlp_reduce(const float* grads, int batch, float* grad, const double* losses, double* loss,
                              cudaStream_t s);
cudaError_t launch_adam(float* P, const float* G, float* M, float* V, int n, int step, float lr, float b1, float b2,
                        float eps, cudaStream_t s);
// rows (3n doubles) and the row statistics st[0..5] (g_hi, g_lo, mean/min diagonal, mean/min row sum)
cudaError_t launch_feat_rows(const double* S, int n, double* rows, double* st, cudaStream_t s);
cudaError_t launch_feat_d0(const double* S, int n, const double* st, double* D0, cudaStream_t s);
int feat_trace_blocks(int n);
cudaError_t launch_feat_traces(const double* D0, const double* P, int n, double* part, const double* st, float* f,
                               cudaStream_t s);

}  // namespace zf

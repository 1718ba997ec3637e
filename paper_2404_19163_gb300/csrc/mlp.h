// Learned start proposal: feature and MLP kernels (k_mlp.cu).
#pragma once
#include "common.cuh"

namespace zf {

constexpr int kMlpParams = 5573;  // 16*64 + 64 + 64*64 + 64 + 5*64 + 5

// One thread per sample.  Y (batch x 5) may be null; with act != null also the per-sample factors of
// the training loss's weight gradients (mlp_act_floats(batch) floats) and the losses (batch).
cudaError_t launch_mlp(const float* P, const float* mean, const float* stdv, const float* X, int batch, float* Y,
                       const float* tgt, const int* ord, float w, float* act, double* losses, cudaStream_t s);
int mlp_act_floats(int batch);
int mlp_chunks(int batch);
// grad = the batch's gradient and *loss its mean loss, from launch_mlp's factors and losses; part holds
// mlp_chunks(batch) x kMlpParams floats and lpart mlp_chunks(batch) doubles of scratch.
cudaError_t launch_mlp_reduce(const float* act, int batch, float* part, const double* losses, double* lpart,
                              float* grad, double* loss, cudaStream_t s);
cudaError_t launch_adam(float* P, const float* G, float* M, float* V, int n, int step, float lr, float b1, float b2,
                        float eps, cudaStream_t s);
// rows (3n doubles) and the row statistics st[0..5] (g_hi, g_lo, mean/min diagonal, mean/min row sum)
cudaError_t launch_feat_rows(const double* S, int n, double* rows, double* st, cudaStream_t s);
cudaError_t launch_feat_d0(const double* S, int n, const double* st, double* D0, cudaStream_t s);
int feat_trace_blocks(int n);
cudaError_t launch_feat_traces(const double* D0, const double* P, int n, double* part, const double* st, float* f,
                               cudaStream_t s);

}  // namespace zf

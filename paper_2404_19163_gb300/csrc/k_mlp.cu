// Learned start proposal (not in the paper; its warm-start motivation is Sec. 6):
// features of an overlap matrix and a 16 -> 64 -> 64 -> 5 GELU MLP (FP32) with its
// forward, backward and Adam kernels.  Gradients are reduced over the batch in a fixed
// order (per-sample gradients, then one thread per parameter), so training is deterministic.
#include <math.h>

#include "mlp.h"

namespace zf {
namespace {

constexpr int I0 = 16, H = 64, O = 5;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * I0, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + O * H, NPAR = OFF_B3 + O;
static_assert(NPAR == kMlpParams, "parameter layout");

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// One thread per sample: forward (and, with grads != nullptr, the per-sample gradient of
// l_b = (y0 - t)^2 + w CE(softmax(y1..4), m) divided by the batch size).
__global__ void k_mlp(const float* __restrict__ P, const float* __restrict__ mean, const float* __restrict__ stdv,
                      const float* __restrict__ X, int batch, float* __restrict__ Y, const float* __restrict__ tgt,
                      const int* __restrict__ ord, float w, float* __restrict__ grads, double* __restrict__ losses) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  float x[I0], z1[H], h1[H], z2[H], h2[H], y[O];
  for (int k = 0; k < I0; ++k) x[k] = (X[(size_t)b * I0 + k] - mean[k]) / stdv[k];
  for (int j = 0; j < H; ++j) {
    float s = P[OFF_B1 + j];
    for (int k = 0; k < I0; ++k) s = fmaf(P[OFF_W1 + j * I0 + k], x[k], s);
    z1[j] = s;
    h1[j] = gelu(s);
  }
  for (int j = 0; j < H; ++j) {
    float s = P[OFF_B2 + j];
    for (int k = 0; k < H; ++k) s = fmaf(P[OFF_W2 + j * H + k], h1[k], s);
    z2[j] = s;
    h2[j] = gelu(s);
  }
  for (int o = 0; o < O; ++o) {
    float s = P[OFF_B3 + o];
    for (int k = 0; k < H; ++k) s = fmaf(P[OFF_W3 + o * H + k], h2[k], s);
    y[o] = s;
  }
  if (Y)
    for (int o = 0; o < O; ++o) Y[(size_t)b * O + o] = y[o];
  if (!grads) return;
  // loss and output gradient
  const float r = y[0] - tgt[b];
  float mx = y[1];
  for (int k = 2; k < O; ++k) mx = fmaxf(mx, y[k]);
  float e[O - 1], se = 0.0f;
  for (int k = 0; k < O - 1; ++k) {
    e[k] = expf(y[1 + k] - mx);
    se += e[k];
  }
  const int m = ord[b];
  losses[b] = (double)(r * r) + (double)w * ((double)logf(se) + (double)mx - (double)y[1 + m]);
  const float inv_b = 1.0f / (float)batch;
  float gy[O];
  gy[0] = 2.0f * r * inv_b;
  for (int k = 0; k < O - 1; ++k) gy[1 + k] = w * (e[k] / se - (k == m ? 1.0f : 0.0f)) * inv_b;
  float* g = grads + (size_t)b * NPAR;
  // layer 3
  for (int o = 0; o < O; ++o) {
    for (int k = 0; k < H; ++k) g[OFF_W3 + o * H + k] = gy[o] * h2[k];
    g[OFF_B3 + o] = gy[o];
  }
  float gz2[H];
  for (int k = 0; k < H; ++k) {
    float s = 0.0f;
    for (int o = 0; o < O; ++o) s = fmaf(P[OFF_W3 + o * H + k], gy[o], s);
    gz2[k] = s * gelu_grad(z2[k]);
  }
  for (int j = 0; j < H; ++j) {
    for (int k = 0; k < H; ++k) g[OFF_W2 + j * H + k] = gz2[j] * h1[k];
    g[OFF_B2 + j] = gz2[j];
  }
  for (int k = 0; k < H; ++k) {
    float s = 0.0f;
    for (int j = 0; j < H; ++j) s = fmaf(P[OFF_W2 + j * H + k], gz2[j], s);
    z1[k] = s * gelu_grad(z1[k]);  // reuse z1 as gz1
  }
  for (int j = 0; j < H; ++j) {
    for (int k = 0; k < I0; ++k) g[OFF_W1 + j * I0 + k] = z1[j] * x[k];
    g[OFF_B1 + j] = z1[j];
  }
}

// grad[p] = sum_b grads[b][p] in sample order; loss = mean_b losses[b] (thread 0).
__global__ void k_mlp_reduce(const float* __restrict__ grads, int batch, float* __restrict__ grad,
                             const double* __restrict__ losses, double* loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NPAR) {
    float s = 0.0f;
    for (int b = 0; b < batch; ++b) s += grads[(size_t)b * NPAR + p];
    grad[p] = s;
  }
  if (p == 0 && loss_out) {
    double l = 0.0;
    for (int b = 0; b < batch; ++b) l += losses[b];
    *loss_out = l / batch;
  }
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, int n, float c1, float c2, float lr, float b1, float b2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * M[i] + (1.0f - b1) * g;
  const float v = b2 * V[i] + (1.0f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// ---- features
// Per row r: diagonal, off-diagonal absolute sum, absolute row sum.
__global__ void k_feat_rows(const double* __restrict__ S, int n, double* __restrict__ rows) {
  const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += fabs(S[(size_t)r * n + c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double d = S[(size_t)r * n + r];
    rows[3 * r] = d;
    rows[3 * r + 1] = s - fabs(d);
    rows[3 * r + 2] = s;
  }
}

// Row statistics in a fixed order: st[0] g_hi, st[1] g_lo, st[2] mean d, st[3] min d,
// st[4] mean row sum, st[5] min row sum.
__global__ void k_feat_rowstats(const double* __restrict__ rows, int n, double* st) {
  __shared__ double sh[6][256];
  double ghi = -INFINITY, glo = INFINITY, sd = 0, md = INFINITY, sr = 0, mr = INFINITY;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double d = rows[3 * r], off = rows[3 * r + 1], rs = rows[3 * r + 2];
    ghi = fmax(ghi, d + off);
    glo = fmin(glo, d - off);
    sd += d;
    md = fmin(md, d);
    sr += rs;
    mr = fmin(mr, rs);
  }
  sh[0][threadIdx.x] = ghi;
  sh[1][threadIdx.x] = glo;
  sh[2][threadIdx.x] = sd;
  sh[3][threadIdx.x] = md;
  sh[4][threadIdx.x] = sr;
  sh[5][threadIdx.x] = mr;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + w]);
      sh[1][threadIdx.x] = fmin(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
      sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
      sh[3][threadIdx.x] = fmin(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
      sh[4][threadIdx.x] += sh[4][threadIdx.x + w];
      sh[5][threadIdx.x] = fmin(sh[5][threadIdx.x], sh[5][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st[0] = sh[0][0];
    st[1] = sh[1][0];
    st[2] = sh[2][0] / n;
    st[3] = sh[3][0];
    st[4] = sh[4][0] / n;
    st[5] = sh[5][0];
  }
}

// E = d0 - t1 I = (1 - t1) I - S / g_hi, with t1 = tr(d0)/N = 1 - mean(S_ii)/g_hi: the spectrum of
// d0 centred, so that the central moments tr(E^k)/N come out without cancellation.
__global__ void k_feat_d0(const double* __restrict__ S, int n, const double* __restrict__ st, double* __restrict__ D0) {
  const double inv = 1.0 / st[0];
  const double t1 = 1.0 - st[2] * inv;
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / n, j = e % n;
    D0[e] = (i == j ? 1.0 - t1 : 0.0) - S[e] * inv;
  }
}

// Per-block partial sums of tr E, sum E^2, sum (E^2) o E, sum (E^2)^2 (E symmetric, P = E^2).
__global__ void k_feat_traces(const double* __restrict__ D0, const double* __restrict__ P, int n,
                              double* __restrict__ part) {
  __shared__ double sh[4][256];
  double a = 0, b = 0, c = 0, d = 0;
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double x = D0[e], p = P[e];
    if (e / n == e % n) a += x;
    b += x * x;
    c += p * x;
    d += p * p;
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  sh[3][threadIdx.x] = d;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) part[4 * blockIdx.x + q] = sh[q][0];
}

__global__ void k_feat_final(const double* __restrict__ part, int nblocks, const double* __restrict__ st, int n,
                             float* __restrict__ f) {
  if (threadIdx.x != 0) return;
  double s[4] = {0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int q = 0; q < 4; ++q) s[q] += part[4 * b + q];
  const double g = st[0];
  // central moments of the spectrum of d0 from E = d0 - t1 I, then the raw moments t_k
  const double t1 = 1.0 - st[2] / g;
  const double m2 = s[1] / n, m3 = s[2] / n, m4 = s[3] / n;
  const double t2 = m2 + t1 * t1;
  const double t3 = m3 + 3 * t1 * m2 + t1 * t1 * t1;
  const double t4 = m4 + 4 * t1 * m3 + 6 * t1 * t1 * m2 + t1 * t1 * t1 * t1;
  f[0] = (float)log((double)n);
  f[1] = (float)log(g);
  f[2] = (float)(st[1] / g);
  f[3] = (float)(st[2] / g);
  f[4] = (float)(st[3] / g);
  f[5] = (float)(st[4] / g);
  f[6] = (float)(st[5] / g);
  f[7] = (float)t1;
  f[8] = (float)t2;
  f[9] = (float)t3;
  f[10] = (float)t4;
  f[11] = (float)sqrt(t2);
  f[12] = (float)m2;
  f[13] = (float)m3;
  f[14] = (float)m4;
  f[15] = (float)log(sqrt(t2 * n));
}

}  // namespace

cudaError_t launch_mlp(const float* P, const float* mean, const float* stdv, const float* X, int batch, float* Y,
                       const float* tgt, const int* ord, float w, float* grads, double* losses, cudaStream_t s) {
  k_mlp<<<(batch + 63) / 64, 64, 0, s>>>(P, mean, stdv, X, batch, Y, tgt, ord, w, grads, losses);
  return cudaGetLastError();
}

cudaError_t launch_mlp_reduce(const float* grads, int batch, float* grad, const double* losses, double* loss,
                              cudaStream_t s) {
  k_mlp_reduce<<<(NPAR + 127) / 128, 128, 0, s>>>(grads, batch, grad, losses, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* P, const float* G, float* M, float* V, int n, int step, float lr, float b1, float b2,
                        float eps, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(P, G, M, V, n, c1, c2, lr, b1, b2, eps);
  return cudaGetLastError();
}

cudaError_t launch_feat_rows(const double* S, int n, double* rows, double* st, cudaStream_t s) {
  k_feat_rows<<<(n + 7) / 8, 256, 0, s>>>(S, n, rows);
  k_feat_rowstats<<<1, 256, 0, s>>>(rows, n, st);
  return cudaGetLastError();
}

cudaError_t launch_feat_d0(const double* S, int n, const double* st, double* D0, cudaStream_t s) {
  const size_t total = (size_t)n * n;
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  k_feat_d0<<<blocks, 256, 0, s>>>(S, n, st, D0);
  return cudaGetLastError();
}

int feat_trace_blocks(int n) {
  const size_t total = (size_t)n * n;
  return (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
}

cudaError_t launch_feat_traces(const double* D0, const double* P, int n, double* part, const double* st, float* f,
                               cudaStream_t s) {
  const int nb = feat_trace_blocks(n);
  k_feat_traces<<<nb, 256, 0, s>>>(D0, P, n, part);
  k_feat_final<<<1, 32, 0, s>>>(part, nb, st, n, f);
  return cudaGetLastError();
}

}  // namespace zf

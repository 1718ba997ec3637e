// Learned start proposal (not in the paper; its warm-start motivation is Sec. 6):
// features of an overlap matrix and a 16 -> 64 -> 64 -> 5 GELU MLP (FP32) with its
// forward, backward and Adam kernels.  Gradients are reduced over the batch in a fixed
// order (per sample the factors of each weight gradient, then per chunk of samples and per parameter the
// sum over the chunk, then over the chunks), so training is deterministic.
#include <math.h>

#include "mlp.h"

namespace zf {
namespace {

constexpr int I0 = 16, H = 64, O = 5;
// per-sample factors of the weight gradients (feature index of each block) and the chunk of samples
// one k_mlp_wgrad block sums
constexpr int A_X = 0, A_GZ1 = A_X + I0, A_H1 = A_GZ1 + H, A_GZ2 = A_H1 + H, A_H2 = A_GZ2 + H, A_GY = A_H2 + H,
              A_N = A_GY + O;
constexpr int kWgChunk = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * I0, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + O * H, NPAR = OFF_B3 + O;
static_assert(NPAR == kMlpParams, "parameter layout");

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// One thread per sample: forward (and, with act != nullptr, the per-sample factors of the gradient of
// l_b = (y0 - t)^2 + w CE(softmax(y1..4), m) divided by the batch size).
__global__ void k_mlp(const float* __restrict__ P, const float* __restrict__ mean, const float* __restrict__ stdv,
                      const float* __restrict__ X, int batch, float* __restrict__ Y, const float* __restrict__ tgt,
                      const int* __restrict__ ord, float w, float* __restrict__ act, double* __restrict__ losses) {
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
  if (!act) return;
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
  // the factors of every weight gradient, feature-major (act[f * batch + b]): x, gz1 (W1, b1),
  // h1, gz2 (W2, b2), h2, gy (W3, b3); the products are summed over the batch by k_mlp_wgrad
  auto put = [&](int f, float v) { act[(size_t)f * batch + b] = v; };
  for (int k = 0; k < I0; ++k) put(A_X + k, x[k]);
  for (int k = 0; k < H; ++k) put(A_H1 + k, h1[k]);
  for (int k = 0; k < H; ++k) put(A_H2 + k, h2[k]);
  for (int o = 0; o < O; ++o) put(A_GY + o, gy[o]);
  float gz2[H];
  for (int k = 0; k < H; ++k) {
    float s = 0.0f;
    for (int o = 0; o < O; ++o) s = fmaf(P[OFF_W3 + o * H + k], gy[o], s);
    gz2[k] = s * gelu_grad(z2[k]);
    put(A_GZ2 + k, gz2[k]);
  }
  for (int k = 0; k < H; ++k) {
    float s = 0.0f;
    for (int j = 0; j < H; ++j) s = fmaf(P[OFF_W2 + j * H + k], gz2[j], s);
    put(A_GZ1 + k, s * gelu_grad(z1[k]));
  }
}

// Weight gradients of a chunk of kWgChunk samples: every parameter's sum over the chunk's samples in
// sample order (the chunk's factors staged sample-major in shared memory), and the chunk's loss sum.
__global__ void __launch_bounds__(256) k_mlp_wgrad(const float* __restrict__ act, int batch,
                                                   const double* __restrict__ losses, float* __restrict__ part,
                                                   double* __restrict__ lpart) {
  extern __shared__ float sm[];  // [kWgChunk][A_N]
  const int b0 = blockIdx.x * kWgChunk, nb = min(kWgChunk, batch - b0);
  for (int e = threadIdx.x; e < A_N * kWgChunk; e += blockDim.x) {
    const int f = e / kWgChunk, q = e % kWgChunk;
    sm[q * A_N + f] = q < nb ? act[(size_t)f * batch + b0 + q] : 0.0f;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < NPAR; p += blockDim.x) {
    int fa, fb = -1;  // gradient of p = sum_q act[fa] * act[fb] (fb < 0: the bias, act[fa] alone)
    if (p < OFF_B1) fa = A_GZ1 + p / I0, fb = A_X + p % I0;
    else if (p < OFF_W2) fa = A_GZ1 + (p - OFF_B1);
    else if (p < OFF_B2) fa = A_GZ2 + (p - OFF_W2) / H, fb = A_H1 + (p - OFF_W2) % H;
    else if (p < OFF_W3) fa = A_GZ2 + (p - OFF_B2);
    else if (p < OFF_B3) fa = A_GY + (p - OFF_W3) / H, fb = A_H2 + (p - OFF_W3) % H;
    else fa = A_GY + (p - OFF_B3);
    float s = 0.0f;
    if (fb >= 0)
      for (int q = 0; q < nb; ++q) s = fmaf(sm[q * A_N + fa], sm[q * A_N + fb], s);
    else
      for (int q = 0; q < nb; ++q) s += sm[q * A_N + fa];
    part[(size_t)blockIdx.x * NPAR + p] = s;
  }
  if (threadIdx.x == 0) {
    double l = 0.0;
    for (int q = 0; q < nb; ++q) l += losses[b0 + q];
    lpart[blockIdx.x] = l;
  }
}

// grad[p] = sum over chunks of the chunk sums, in chunk order; loss = the mean of the losses (thread 0).
__global__ void k_mlp_reduce(const float* __restrict__ part, int nchunks, int batch, float* __restrict__ grad,
                             const double* __restrict__ lpart, double* loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NPAR) {
    float s = 0.0f;
    for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * NPAR + p];
    grad[p] = s;
  }
  if (p == 0 && loss_out) {
    double l = 0.0;
    for (int c = 0; c < nchunks; ++c) l += lpart[c];
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
  const size_t total = (size_t)n * n, stride = (size_t)gridDim.x * blockDim.x;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  // (i, j) of e, advanced by the stride's row and column steps (no division per element)
  size_t i = e / n, j = e % n;
  const size_t si = stride / n, sj = stride % n;
  for (; e < total; e += stride) {
    D0[e] = (i == j ? 1.0 - t1 : 0.0) - S[e] * inv;
    i += si;
    j += sj;
    if (j >= (size_t)n) {
      j -= n;
      ++i;
    }
  }
}

// Per-block partial sums of tr E, sum E^2, sum (E^2) o E, sum (E^2)^2 (E symmetric, P = E^2).
__global__ void k_feat_traces(const double* __restrict__ D0, const double* __restrict__ P, int n,
                              double* __restrict__ part) {
  __shared__ double sh[4][256];
  double a = 0, b = 0, c = 0, d = 0;
  const size_t total = (size_t)n * n, stride = (size_t)gridDim.x * blockDim.x;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (size_t r = t; r < (size_t)n; r += stride) a += D0[r * (n + 1)];
  for (size_t e = t; e < total; e += stride) {
    const double x = D0[e], p = P[e];
    b = fma(x, x, b);
    c = fma(p, x, c);
    d = fma(p, p, d);
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

// The block partials summed in a fixed order (thread t takes blocks t, t + 256, ..., then a tree), and
// the 16 features.
__global__ void __launch_bounds__(256) k_feat_final(const double* __restrict__ part, int nblocks,
                                                    const double* __restrict__ st, int n, float* __restrict__ f) {
  __shared__ double sh[4][256];
  double v[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int q = 0; q < 4; ++q) v[q] += part[4 * b + q];
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double s[4];
  for (int q = 0; q < 4; ++q) s[q] = sh[q][0];
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
                       const float* tgt, const int* ord, float w, float* act, double* losses, cudaStream_t s) {
  k_mlp<<<(batch + 63) / 64, 64, 0, s>>>(P, mean, stdv, X, batch, Y, tgt, ord, w, act, losses);
  return cudaGetLastError();
}

int mlp_act_floats(int batch) { return A_N * batch; }
int mlp_chunks(int batch) { return (batch + kWgChunk - 1) / kWgChunk; }

cudaError_t launch_mlp_reduce(const float* act, int batch, float* part, const double* losses, double* lpart,
                              float* grad, double* loss, cudaStream_t s) {
  const int smem = (int)sizeof(float) * A_N * kWgChunk;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int nc = mlp_chunks(batch);
  k_mlp_wgrad<<<nc, 256, smem, s>>>(act, batch, losses, part, lpart);
  k_mlp_reduce<<<(NPAR + 127) / 128, 128, 0, s>>>(part, nc, batch, grad, lpart, loss);
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
  k_feat_final<<<1, 256, 0, s>>>(part, nb, st, n, f);
  return cudaGetLastError();
}

}  // namespace zf

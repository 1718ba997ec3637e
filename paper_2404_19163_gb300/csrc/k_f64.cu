// CUDA-core products of the recursion in FP64 (the paper's "double", Table I) and FP32
// ("single"),
// with the element-wise steps fused into the epilogues:
//   residual   d = I - Z^T (S Z), symmetric, upper tiles only   (Eq. np1, Algorithm 2's Err)
//   polynomial Q = c1 d + c2 d^2 (+ c_k d^k chains)               (delta-form of Eq. np1)
//   update     Z' = Z + Z Q                                       (Z_{n+1} = Z_n p(d_n))
// GB300's FP64 pipe is ~1.1 TFLOP/s (about 2 DFMA per SM per clock), so these
// kernels are bound by FP64 issue for every N of interest; a 64x64 tile with a
// 4x4 register micro-tile keeps the operand traffic far below that bound.
#include "kernels.h"

namespace zf {
namespace {

constexpr int BK = 16, NT = 256;

// Tile edge: 64 x 64 tiles (4 x 4 outputs per thread) in general; 32 x 32 tiles (2 x 2 per thread) up
// to N = 1024, where 64-wide tiles leave most SMs idle (N = 256: 16 tiles on 152 SMs).  FP32 from
// N = 2048 on takes 128 x 128 tiles (8 x 8 per thread): the FP32 pipe needs that much reuse per load.
inline int tile_for(int n, bool fp32 = false) { return n <= 1024 ? 32 : (fp32 && n >= 2048 ? 128 : 64); }

__device__ __forceinline__ void sym_tile_of(int b, int T, int& bi, int& bj) {
  // b-th tile of the upper triangle, row-major over (bi, bj >= bi)
  int row = 0, rem = b;
  while (rem >= T - row) {
    rem -= T - row;
    ++row;
  }
  bi = row;
  bj = row + rem;
}

template <typename T, typename G, int TE>
__global__ void __launch_bounds__(NT) k64_gemm(G g) {
  constexpr int BM = TE, BN = TE, R = TE / 16;  // R x R outputs per thread
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ double red[NT / 32];
  const int n = g.n;
  const int TB = (n + BM - 1) / BM;
  int bi, bj;
  if (g.sym) {
    sym_tile_of(blockIdx.x, TB, bi, bj);
  } else {
    bi = blockIdx.y;
    bj = blockIdx.x;
  }
  const int i0 = bi * BM, j0 = bj * BN;
  const int t = threadIdx.x;
  const int ty = t / 16, tx = t % 16;
  T acc[R][R] = {};
  for (int k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
    for (int e = 0; e < (BM * BK) / NT; ++e) {
      const int idx = t + e * NT;
      int ii, kk;
      T v = 0;
      if (g.transA) {
        kk = idx / BM;
        ii = idx % BM;
        const int gi = i0 + ii, gk = k0 + kk;
        if (gi < n && gk < n) v = g.A[(size_t)gk * n + gi];
      } else {
        ii = idx / BK;
        kk = idx % BK;
        const int gi = i0 + ii, gk = k0 + kk;
        if (gi < n && gk < n) v = g.A[(size_t)gi * n + gk];
      }
      As[kk][ii] = v;
    }
#pragma unroll
    for (int e = 0; e < (BK * BN) / NT; ++e) {
      const int idx = t + e * NT;
      const int kk = idx / BN, jj = idx % BN;
      const int gk = k0 + kk, gj = j0 + jj;
      Bs[kk][jj] = (gk < n && gj < n) ? g.B[(size_t)gk * n + gj] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[R], b[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = As[kk][ty * R + r];
#pragma unroll
      for (int c = 0; c < R; ++c) b[c] = Bs[kk][tx * R + c];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  double ss = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + ty * R + r;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int j = j0 + tx * R + c;
      if (j >= n) continue;
      if (g.sym && j < i) continue;  // the (j, i) entry is written by the tile that owns it
      T v;
      if (g.resid) {
        v = (i == j ? T(1) : T(0)) - acc[r][c];
        ss += (i == j ? 1.0 : 2.0) * (double)v * (double)v;
      } else {
        v = (T)g.beta * acc[r][c];
        if (g.Add) v = fma((T)g.alpha, g.Add[(size_t)i * n + j], v);
        if (g.P) {
          g.P[(size_t)i * n + j] = acc[r][c];
          if (g.sym && j != i) g.P[(size_t)j * n + i] = acc[r][c];
        }
      }
      g.C[(size_t)i * n + j] = v;
      if (g.sym && j != i) g.C[(size_t)j * n + i] = v;
    }
  }
  if (g.resid) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((t & 31) == 0) red[t >> 5] = ss;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      g.partials[blockIdx.x] = s;
    }
  }
}

}  // namespace

int f64_num_blocks(int n, bool sym, bool fp32) {
  const int te = tile_for(n, fp32);
  const int T = (n + te - 1) / te;
  return sym ? T * (T + 1) / 2 : T * T;
}

template <typename T, typename G>
static cudaError_t launch_k64(const G& g, cudaStream_t s) {
  const int te = tile_for(g.n, sizeof(T) == 4);
  const int tb = (g.n + te - 1) / te;
  dim3 grid = g.sym ? dim3(tb * (tb + 1) / 2) : dim3(tb, tb);
  if (te == 32)
    k64_gemm<T, G, 32><<<grid, NT, 0, s>>>(g);
  else if (te == 64)
    k64_gemm<T, G, 64><<<grid, NT, 0, s>>>(g);
  else if constexpr (sizeof(T) == 4)
    k64_gemm<T, G, 128><<<grid, NT, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_f64_gemm(const F64Gemm& g, cudaStream_t s) { return launch_k64<double, F64Gemm>(g, s); }

cudaError_t launch_f32_gemm(const F32Gemm& g, cudaStream_t s) { return launch_k64<float, F32Gemm>(g, s); }

}  // namespace zf

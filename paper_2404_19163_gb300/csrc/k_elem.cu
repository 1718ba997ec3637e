// Element-wise steps and reductions of the recursion: the Gershgorin start
// Z0 = I / sqrt(max_i sum_j |S_ij|) (Sec. 3: ||X0 - I||_2 < 1), the
// deterministic Frobenius-norm finish Err = ||I - X||_F, and the stop test of
// Algorithm 2 (Sec. 4.1, Eq. stopL2) evaluated on the device in FP64.
#include <math.h>

#include "kernels.h"

namespace zf {
namespace {

__global__ void k_rowabs_max(const double* __restrict__ S, int n, IterState* st) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = S + (size_t)warp * n;
  double s = 0.0;
#pragma unroll 4
  for (int j = lane; j < n; j += 32) s += fabs(row[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  // non-negative doubles order like their bit patterns, and a NaN (or Inf) row sum orders above
  // every finite one, so a non-finite entry of S leaves a non-finite maximum
  if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(&st->amax[0]), __double_as_longlong(s));
}

__global__ void k_gscale(IterState* st) { st->gscale = 1.0 / sqrt(st->amax[0]); }
__global__ void k_set_gscale(IterState* st, double s) { st->gscale = s; }

// Rows i = blockIdx.y, blockIdx.y + gridDim.y, ...; columns across blockIdx.x and the threads (no
// division per element).
__global__ void k_scaled_identity_f64(double* Z, int n, const IterState* st) {
  const double s = st->gscale;
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    double* zr = Z + (size_t)i * n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) zr[j] = (i == j) ? s : 0.0;
  }
}

__global__ void k_finish_err(const double* __restrict__ partials, int np, IterState* st, int idx, int rule,
                             double tol, int n, int check_stop) {
  __shared__ double red[256];
  double s = 0.0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) s += partials[p];  // fixed order per thread
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double err = sqrt(red[0]);
    if (idx < 0) idx = st->loop_iter + 1;  // device-driven loop: the update this residual follows
    if (idx < kHistMax) st->hist[idx] = err;
    st->hist_len = idx + 1;
    if (!isfinite(err)) {
      st->nonfinite = 1;
      st->stop = 1;
    } else if (check_stop) {
      const double prev = st->prev_err;
      if (rule == 1) {
        if (err / sqrt((double)n) <= tol) st->stop = 1;
      } else if (err > prev * prev * prev || err >= prev) {
        st->stop = 1;
      }
    }
    st->prev_err = err;
  }
}

__device__ __forceinline__ uint16_t r16(float x, bool bf16) {
  return bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(x)) : __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ float f16v(uint16_t h, bool bf16) {
  return bf16 ? __bfloat162float(__ushort_as_bfloat16(h)) : __half2float(__ushort_as_half(h));
}

// 32 x 32 tiles through shared memory so that both the read and the (possibly transposed)
// write are coalesced.
template <typename T>
__global__ void k_cvt16(const T* __restrict__ src, int n, int ld_src, uint16_t* __restrict__ hi,
                        uint16_t* __restrict__ lo, int ld16, double scale, const float* scale_ptr, int transpose,
                        int bf16) {
  __shared__ uint16_t th[32][33], tl[32][33];
  const double sc = scale_ptr ? (double)*scale_ptr : scale;
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  // blockDim is (32, 8): four rows per thread, unrolled so that their loads are in flight together
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const int r = threadIdx.y + 8 * rr;
    const int i = bi + r, j = bj + threadIdx.x;
    uint16_t h = 0, l = 0;
    if (i < n && j < n) {
      const float x = (float)((double)src[(size_t)i * ld_src + j] * sc);
      h = r16(x, bf16);
      l = r16(x - f16v(h, bf16), bf16);
    }
    th[r][threadIdx.x] = h;
    tl[r][threadIdx.x] = l;
  }
  __syncthreads();
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const int r = threadIdx.y + 8 * rr;
    int oi, oj;
    uint16_t h, l;
    if (transpose) {
      oi = bj + r;
      oj = bi + threadIdx.x;
      h = th[threadIdx.x][r];
      l = tl[threadIdx.x][r];
    } else {
      oi = bi + r;
      oj = bj + threadIdx.x;
      h = th[r][threadIdx.x];
      l = tl[r][threadIdx.x];
    }
    if (oi < n && oj < n) {
      hi[(size_t)oi * ld16 + oj] = h;
      if (lo) lo[(size_t)oi * ld16 + oj] = l;
    }
  }
}

__global__ void k_split_flat(const double* __restrict__ A, int64_t n, double scale, uint16_t* hi, uint16_t* lo,
                             int bf16) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float x = (float)(A[e] * scale);
    const uint16_t h = r16(x, bf16);
    hi[e] = h;
    lo[e] = r16(x - f16v(h, bf16), bf16);
  }
}

// Row-by-row copies (grid.y strides over rows, grid.x * blockDim over columns): no per-element division.
__global__ void k_f64_to_f32(const double* __restrict__ src, int n, int ld64, float* dst, int ld32) {
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const double* s = src + (size_t)i * ld64;
    float* d = dst + (size_t)i * ld32;
#pragma unroll 4
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) d[j] = (float)s[j];
  }
}

// With amax != null also max |x| into *amax (the bits of a non-negative double; the caller zeroes it).
__global__ void k_f32_to_f64(const float* __restrict__ src, int n, int ld32, double* dst, int ld64,
                             unsigned long long* amax) {
  unsigned long long m = 0ull;
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const float* s = src + (size_t)i * ld32;
    double* d = dst + (size_t)i * ld64;
#pragma unroll 4
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
      const double x = (double)s[j];
      d[j] = x;
      m = max_bits(m, abs_bits(x));
    }
  }
  if (!amax) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(amax, m);
}

// max |A_ij| on the integer pipes (abs_bits): a NaN orders above every number, so a NaN anywhere
// makes the maximum NaN and callers can test the result with isfinite.
__global__ void k_amax_f64(const double* __restrict__ A, size_t total, IterState* st, int slot) {
  unsigned long long m = 0ull;
#pragma unroll 4
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    m = max_bits(m, abs_bits(A[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned long long*>(&st->amax[slot]), m);
}

__device__ float pow2_for(double bound) {
  // largest power of two s with bound * s <= 2^14 (FP16 max is 65504 ~ 2^16: two bits of headroom)
  if (!(bound > 0.0) || !isfinite(bound)) return 1.0f;
  int e;
  frexp(bound, &e);  // bound in [2^(e-1), 2^e)
  int p = 14 - e;
  if (p > 60) p = 60;
  if (p < -60) p = -60;
  return ldexpf(1.0f, p);
}

__global__ void k_pow2_scales(IterState* st, int idx, float c1, float c2) {
  const double ad = st->amax[1];
  const double err = (idx >= 0 && idx < kHistMax) ? st->hist[idx] : ad;
  st->scale[0] = pow2_for(ad);
  st->scale[1] = pow2_for((double)c1 * ad + (double)c2 * err * err);
  st->scale[2] = pow2_for(st->amax[2]);
}

__device__ float pow2_head(double bound, int headroom_log2) {
  if (!(bound > 0.0) || !isfinite(bound)) return 1.0f;
  int e;
  frexp(bound, &e);
  int p = 14 - headroom_log2 - e;
  if (p > 60) p = 60;
  if (p < -60) p = -60;
  return ldexpf(1.0f, p);
}

// head: extra headroom (log2) of every scale; an FP16 accumulator takes operands scaled to at most 1
__global__ void k_fp16_scales(IterState* st, int op, int idx, float c1, float c2, int zslot_next, int head) {
  if (op == 0) {
    if (idx < 0) idx = st->loop_iter + 1;  // device-driven loop, as in k_finish_err
    const double ad = (double)__uint_as_float(st->amaxf[1]);
    const double err = (idx >= 0 && idx < kHistMax) ? st->hist[idx] : ad;
    st->scale[0] = pow2_head(ad, head);
    st->scale[1] = pow2_head((double)c1 * ad + (double)c2 * err * err, head);
  } else if (op == 1) {
    st->scale[4] = pow2_head(st->amax[0] * st->amax[6], head);
  } else if (op == 2) {
    st->scale[zslot_next] = pow2_head(st->amax[6], 4 + head);
  } else {
    st->amax[6] = (double)__uint_as_float(st->amaxf[2]);
  }
}

}  // namespace

cudaError_t launch_fp16_scales(IterState* st, int op, int idx, float c1, float c2, int zslot_next, int head,
                               cudaStream_t s) {
  k_fp16_scales<<<1, 1, 0, s>>>(st, op, idx, c1, c2, zslot_next, head);
  return cudaGetLastError();
}

cudaError_t launch_cvt16(const double* src, int n, int ld_src, uint16_t* hi, uint16_t* lo, int ld16, double scale,
                         const float* scale_ptr, bool transpose, bool bf16, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  k_cvt16<double><<<grid, block, 0, s>>>(src, n, ld_src, hi, lo, ld16, scale, scale_ptr, transpose, bf16);
  return cudaGetLastError();
}

cudaError_t launch_cvt16_f32(const float* src, int n, int ld_src, uint16_t* hi, uint16_t* lo, int ld16,
                             bool transpose, bool bf16, const float* scale_ptr, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  k_cvt16<float><<<grid, block, 0, s>>>(src, n, ld_src, hi, lo, ld16, 1.0, scale_ptr, transpose, bf16);
  return cudaGetLastError();
}

cudaError_t launch_split_flat(const double* A, int64_t n, double scale, uint16_t* hi, uint16_t* lo, bool bf16,
                              cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
  k_split_flat<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(A, n, scale, hi, lo, bf16);
  return cudaGetLastError();
}

// ---- cold start Z0 = s I (s = st->gscale, the Gershgorin scale of the start)
// The first residual needs no product: A^T = Z0^T S = s S and X0 = Z0^T A = s^2 S, so
// d0 = I - s^2 S, formed here from the upper triangle of S (X is defined by its upper triangle,
// mirrored).  Writes d0 in FP32 (D32, leading dimension ld) and, when hi != nullptr, its 16-bit
// hi (and lo, when lo != nullptr) copies; partials[block] = the block's sum of d0_ij^2 over the
// entries it owns (off-diagonal entries twice), amax_bits = max |d0| as FP32 bits.  Blocks of
// 32 x 8 threads walk the upper 32 x 32 tiles; the mirror goes through shared memory.
__global__ void k_cold_resid(const double* __restrict__ S, int n, const IterState* __restrict__ st,
                             float* __restrict__ D32, int ld, uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                             int bf16, double* __restrict__ partials, unsigned int* amax_bits) {
  __shared__ float tile[32][33];
  __shared__ double red[8];
  const double s2 = st->gscale * st->gscale;
  const int tb = (n + 31) / 32;
  const int ntiles = tb * (tb + 1) / 2;
  const int tx = threadIdx.x, ty = threadIdx.y;
  double ss = 0.0;
  float am = 0.0f;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // tile t -> (rb, cb), cb >= rb, row by row of the upper triangle
    int rb = 0, rem = t;
    while (rem >= tb - rb) {
      rem -= tb - rb;
      ++rb;
    }
    const int cb = rb + rem;
    const int bi = rb * 32, bj = cb * 32;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q, i = bi + r, j = bj + tx;
      float d = 0.0f;
      if (i < n && j < n && j >= i) {
        const double dd = (i == j ? 1.0 : 0.0) - s2 * S[(size_t)i * n + j];
        d = (float)dd;
        ss += (i == j ? 1.0 : 2.0) * dd * dd;
        am = fmaxf(am, fabsf(d));
        D32[(size_t)i * ld + j] = d;
        if (hi) {
          const uint16_t h = r16(d, bf16);
          hi[(size_t)i * ld + j] = h;
          if (lo) lo[(size_t)i * ld + j] = r16(d - f16v(h, bf16), bf16);
        }
      }
      tile[r][tx] = d;
    }
    __syncthreads();
    // mirror: (i, j) with j > i to (j, i): rows bj.., columns bi..
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q, oi = bj + r, oj = bi + tx;
      if (oi < n && oj < n && oi > oj) {
        const float d = tile[tx][r];
        D32[(size_t)oi * ld + oj] = d;
        if (hi) {
          const uint16_t h = r16(d, bf16);
          hi[(size_t)oi * ld + oj] = h;
          if (lo) lo[(size_t)oi * ld + oj] = r16(d - f16v(h, bf16), bf16);
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
  }
  if (tx == 0) red[ty] = ss;
  if (tx == 0) atomicMax(amax_bits, __float_as_uint(am));
  __syncthreads();
  if (tx == 0 && ty == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

// The first update from a cold start: Z1 = Z0 + Z0 Q0 = s (I + Q0), elementwise from the FP32 Q0
// (symmetric, both triangles written).  Writes the FP32 master Zm, the 16-bit copies of Z1
// (scaled by *out_scale when given, as the update epilogue does) and the same values as the
// transposed copy (Z1 is symmetric), and max |Z1| (FP32 bits) into amax_bits.
__global__ void k_cold_update(const float* __restrict__ Q, int n, int ld, const IterState* __restrict__ st,
                              float* __restrict__ Zm, uint16_t* zh, uint16_t* zl, uint16_t* th, uint16_t* tl,
                              const float* out_scale, int bf16, unsigned int* amax_bits) {
  const float s = (float)st->gscale;
  const float osc = out_scale ? *out_scale : 1.0f;
  float am = 0.0f;
  // rows across blockIdx.y, columns across blockIdx.x and the threads (no division per element)
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
      const size_t o = (size_t)i * ld + j;
      const float z = s * ((i == j ? 1.0f : 0.0f) + Q[o]);
      Zm[o] = z;
      am = fmaxf(am, fabsf(z));
      const float y = z * osc;
      const uint16_t h = r16(y, bf16);
      zh[o] = h;
      th[o] = h;
      if (zl) {
        const uint16_t l = r16(y - f16v(h, bf16), bf16);
        zl[o] = l;
        tl[o] = l;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, __float_as_uint(am));
}

static int grid_for(size_t total) { return (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192); }

static dim3 rows_grid(int n) {
  const int gx = (n + 255) / 256 < 4 ? (n + 255) / 256 : 4;
  return dim3(gx > 0 ? gx : 1, n < 2048 ? (n > 0 ? n : 1) : 2048);
}

cudaError_t launch_f64_to_f32(const double* src, int n, int ld64, float* dst, int ld32, cudaStream_t s) {
  k_f64_to_f32<<<rows_grid(n), 256, 0, s>>>(src, n, ld64, dst, ld32);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* src, int n, int ld32, double* dst, int ld64, cudaStream_t s,
                              unsigned long long* amax) {
  if (amax) cudaMemsetAsync(amax, 0, sizeof(unsigned long long), s);
  k_f32_to_f64<<<rows_grid(n), 256, 0, s>>>(src, n, ld32, dst, ld64, amax);
  return cudaGetLastError();
}

cudaError_t launch_amax_f64(const double* A, int n, IterState* st, int slot, cudaStream_t s) {
  cudaMemsetAsync(&st->amax[slot], 0, sizeof(double), s);
  const size_t total = (size_t)n * n;
  k_amax_f64<<<grid_for(total) < 1024 ? grid_for(total) : 1024, 256, 0, s>>>(A, total, st, slot);
  return cudaGetLastError();
}

cudaError_t launch_pow2_scales(IterState* st, int idx, float c1, float c2, cudaStream_t s) {
  k_pow2_scales<<<1, 1, 0, s>>>(st, idx, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_gershgorin(const double* S, int n, IterState* st, cudaStream_t s) {
  cudaMemsetAsync(&st->amax[0], 0, sizeof(double), s);
  const int warps_per_block = 8;
  k_rowabs_max<<<(n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(S, n, st);
  k_gscale<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

namespace {
__global__ void k_loop_init(IterState* st, int iters, int limit) {
  st->loop_iter = iters;
  st->loop_limit = limit;
}

// One update of the device-driven bulk loop is done (its residual's Err is in the history): count it and
// decide whether the loop goes on.  Every path ends the loop once loop_limit updates are done.
__global__ void k_loop_cond(IterState* st, cudaGraphConditionalHandle loop, cudaGraphConditionalHandle next,
                            int set_next) {
  const int it = st->loop_iter + 1;
  st->loop_iter = it;
  const unsigned go = (!st->stop && !st->nonfinite && st->error == 0 && it < st->loop_limit) ? 1u : 0u;
  cudaGraphSetConditional(loop, go);
  if (set_next) cudaGraphSetConditional(next, go);
}
}  // namespace

cudaError_t launch_loop_init(IterState* st, int iters, int limit, cudaStream_t s) {
  k_loop_init<<<1, 1, 0, s>>>(st, iters, limit);
  return cudaGetLastError();
}

cudaError_t launch_loop_cond(IterState* st, cudaGraphConditionalHandle loop, cudaGraphConditionalHandle next,
                             bool set_next, cudaStream_t s) {
  k_loop_cond<<<1, 1, 0, s>>>(st, loop, next, set_next ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_set_gscale(IterState* st, double scale, cudaStream_t s) {
  k_set_gscale<<<1, 1, 0, s>>>(st, scale);
  return cudaGetLastError();
}

cudaError_t launch_scaled_identity_f64(double* Z, int n, const IterState* st, cudaStream_t s) {
  k_scaled_identity_f64<<<rows_grid(n), 256, 0, s>>>(Z, n, st);
  return cudaGetLastError();
}

cudaError_t launch_finish_err(const double* partials, int nparts, IterState* st, int idx, int rule, double tol,
                              int n, int check_stop, cudaStream_t s) {
  k_finish_err<<<1, 256, 0, s>>>(partials, nparts, st, idx, rule, tol, n, check_stop);
  return cudaGetLastError();
}

}  // namespace zf

namespace zf {
int cold_resid_blocks(int n) {
  const int tb = (n + 31) / 32, t = tb * (tb + 1) / 2;
  return t < 1024 ? t : 1024;
}

cudaError_t launch_cold_resid(const double* S, int n, const IterState* st, float* D32, int ld, uint16_t* hi,
                              uint16_t* lo, bool bf16, double* partials, unsigned int* amax_bits, cudaStream_t s) {
  k_cold_resid<<<cold_resid_blocks(n), dim3(32, 8), 0, s>>>(S, n, st, D32, ld, hi, lo, bf16 ? 1 : 0, partials,
                                                           amax_bits);
  return cudaGetLastError();
}

cudaError_t launch_cold_update(const float* Q, int n, int ld, const IterState* st, float* Zm, uint16_t* zh,
                               uint16_t* zl, uint16_t* th, uint16_t* tl, const float* out_scale, bool bf16,
                               unsigned int* amax_bits, cudaStream_t s) {
  k_cold_update<<<rows_grid(n), 256, 0, s>>>(Q, n, ld, st, Zm, zh, zl, th, tl, out_scale, bf16 ? 1 : 0, amax_bits);
  return cudaGetLastError();
}
}  // namespace zf

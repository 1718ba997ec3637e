// Element-wise kernels of the batched (grouped) mode: every instance's matrices are
// stacked along the rows of packed buffers (instance i at row offset row0[i], common
// leading dimension), so that one tensor map and one persistent launch cover all of them.
#include <math.h>

#include "batched.h"

namespace zf {
namespace {

__device__ __forceinline__ uint16_t r16b(float x, bool bf16) {
  return bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(x)) : __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ float f16b(uint16_t h, bool bf16) {
  return bf16 ? __bfloat162float(__ushort_as_bfloat16(h)) : __half2float(__ushort_as_half(h));
}

// Gershgorin bound per instance: gmax[i] = max_r sum_c |S_i[r][c]|.  One warp per row,
// grid.y = instance.
__global__ void k_b_rowabs(const BatchTables t, unsigned long long* gmax_bits) {
  const int i = blockIdx.y;
  const int n = t.n[i];
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n || t.Z0[i] != nullptr) return;
  const double* S = t.S[i] + (size_t)row * n;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += fabs(S[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) atomicMax(&gmax_bits[i], (unsigned long long)__double_as_longlong(s));
}

// Dynamic range of every instance for its FP64-accurate residual: g_i = max_r sum_c |S_i[r][c]|
// and z_i = max |Z_i| (the returned FP64 Z).  One warp per row, grid.y = instance.
__global__ void k_b_ranges(const BatchTables t, unsigned long long* gmax_bits, unsigned long long* zmax_bits) {
  const int i = blockIdx.y;
  const int n = t.n[i];
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* S = t.S[i] + (size_t)row * n;
  const double* Z = t.Z[i] + (size_t)row * n;
  double g = 0.0, z = 0.0;
  for (int c = lane; c < n; c += 32) {
    g += fabs(S[c]);
    z = fmax(z, fabs(Z[c]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    g += __shfl_xor_sync(0xffffffffu, g, o);
    z = fmax(z, __shfl_xor_sync(0xffffffffu, z, o));
  }
  if (lane == 0) {
    atomicMax(&gmax_bits[i], (unsigned long long)__double_as_longlong(g));
    atomicMax(&zmax_bits[i], (unsigned long long)__double_as_longlong(z));
  }
}

// Scaled row norms of every instance for the moduli of its residue products (as launch_ozm_rho):
// rho2[i] = max_r sum_c (S_i[r][c] 2^-e_r)^2, e_r the row's exponent bound, FP32 bits, atomic maximum;
// +Inf for a row holding a NaN or Inf or whose largest entry is subnormal.  One warp per row (two passes
// over the row: its maximum, then the scaled sum), grid.y = instance.
__global__ void k_b_rowrho(const BatchTables t, unsigned int* rho2) {
  const int i = blockIdx.y;
  const int n = t.n[i];
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* S = t.S[i] + (size_t)row * n;
  unsigned long long m = 0ull;
  for (int c = lane; c < n; c += 32) m = max_bits(m, abs_bits(S[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (m == 0ull) return;
  if (m >= 0x7FF0000000000000ull || m < (1ull << 52)) {
    if (lane == 0) atomicMax(&rho2[i], 0x7F800000u);
    return;
  }
  const int e = exp_of_bits(m);
  float acc = 0.0f;
  for (int c = lane; c < n; c += 32) {
    const float f = scaled_mag_f32(abs_bits(S[c]), e);
    acc = fmaf(f, f, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) atomicMax(&rho2[i], __float_as_uint(acc));
}

// The same for the columns of every Z_i (the rows of the residual's first operand Z_i^T): blocks of 32
// columns x 256 rows (grid.z = instance), the column maxima and then the scaled sums accumulated with
// atomics into cmax / csum at the instance's packed row offset, then the largest sum per instance.
__global__ void k_b_colmax(const BatchTables t, unsigned long long* cmax) {
  __shared__ unsigned long long red[8][33];
  const int i = blockIdx.z, n = t.n[i];
  const int j = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 256;
  if (blockIdx.x * 32 >= n || r0 >= n) return;
  const int r1 = r0 + 256 < n ? r0 + 256 : n;
  const double* Z = t.Z[i];
  unsigned long long m = 0ull;
  if (j < n)
    for (int r = r0 + threadIdx.y; r < r1; r += 8) m = max_bits(m, abs_bits(Z[(size_t)r * n + j]));
  red[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0 && j < n) {
    for (int y = 1; y < 8; ++y) m = max_bits(m, red[y][threadIdx.x]);
    if (m) atomicMax(&cmax[t.row0[i] + j], m);
  }
}

__device__ __forceinline__ bool b_no_bound(unsigned long long m) {
  return m >= 0x7FF0000000000000ull || (m != 0ull && m < (1ull << 52));
}

__global__ void k_b_colsum(const BatchTables t, const unsigned long long* cmax, float* csum) {
  __shared__ float red[8][33];
  const int i = blockIdx.z, n = t.n[i];
  const int j = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 256;
  if (blockIdx.x * 32 >= n || r0 >= n) return;
  const int r1 = r0 + 256 < n ? r0 + 256 : n;
  const double* Z = t.Z[i];
  const unsigned long long m = j < n ? cmax[t.row0[i] + j] : 0ull;
  float acc = 0.0f;
  if (m != 0ull && !b_no_bound(m)) {
    const int e = exp_of_bits(m);
    for (int r = r0 + threadIdx.y; r < r1; r += 8) {
      const float f = scaled_mag_f32(abs_bits(Z[(size_t)r * n + j]), e);
      acc = fmaf(f, f, acc);
    }
  }
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && m != 0ull && !b_no_bound(m)) {
    for (int y = 1; y < 8; ++y) acc += red[y][threadIdx.x];
    atomicAdd(&csum[t.row0[i] + j], acc);
  }
}

__global__ void k_b_colfin(const BatchTables t, const unsigned long long* cmax, const float* csum,
                           unsigned int* rho2) {
  const int i = blockIdx.y, n = t.n[i];
  const int j = blockIdx.x * 256 + threadIdx.x;
  unsigned u = 0u;
  if (j < n) {
    const unsigned long long m = cmax[t.row0[i] + j];
    u = b_no_bound(m) ? 0x7F800000u : __float_as_uint(csum[t.row0[i] + j]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) u = max(u, __shfl_xor_sync(0xffffffffu, u, o));
  if ((threadIdx.x & 31) == 0 && u) atomicMax(&rho2[i], u);
}

// Pack instance i (grid.z) into the stacked buffers, 32 x 32 tiles through shared memory:
//   mode 0: S16 (hi[, lo]) from S_i
//   mode 1: Z master (FP32) + Z16 and Zt16 (hi[, lo]) from Z0_i, or from s_i I when Z0_i is null
__global__ void k_b_pack(const BatchTables t, int mode, const unsigned long long* gmax_bits, int ld, int bf16,
                         uint16_t* h16, uint16_t* l16, uint16_t* th16, uint16_t* tl16, float* m32) {
  __shared__ float tile[32][33];
  const int inst = blockIdx.z;
  const int n = t.n[inst];
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  if (bi >= n || bj >= n) return;
  const size_t r0 = (size_t)t.row0[inst];
  const double* src = (mode == 0) ? t.S[inst] : t.Z0[inst];
  double gs = 0.0;
  if (mode == 1 && !src) gs = 1.0 / sqrt(__longlong_as_double((long long)gmax_bits[inst]));
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = bi + r, j = bj + threadIdx.x;
    float x = 0.0f;
    if (i < n && j < n) x = src ? (float)src[(size_t)i * n + j] : (i == j ? (float)gs : 0.0f);
    tile[r][threadIdx.x] = x;
    if (i < n && j < n) {
      const uint16_t h = r16b(x, bf16);
      h16[(r0 + i) * ld + j] = h;
      if (l16) l16[(r0 + i) * ld + j] = r16b(x - f16b(h, bf16), bf16);
      if (mode == 1) m32[(r0 + i) * ld + j] = x;
    }
  }
  if (mode == 0) return;
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int oi = bj + r, oj = bi + threadIdx.x;  // transposed position
    if (oi < n && oj < n) {
      const float x = tile[threadIdx.x][r];
      const uint16_t h = r16b(x, bf16);
      th16[(r0 + oi) * ld + oj] = h;
      if (tl16) tl16[(r0 + oi) * ld + oj] = r16b(x - f16b(h, bf16), bf16);
    }
  }
}

// Unpack the FP32 master of instance i (grid.z) into the caller's FP64 Z_i.
__global__ void k_b_unpack(const BatchTables t, const float* m32, int ld) {
  const int inst = blockIdx.z;
  const int n = t.n[inst];
  const size_t r0 = (size_t)t.row0[inst];
  double* Z = t.Z[inst];
  for (int r = blockIdx.y * blockDim.y + threadIdx.y; r < n; r += gridDim.y * blockDim.y)
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
      Z[(size_t)r * n + c] = (double)m32[(r0 + r) * ld + c];
}

// Per-instance Err, history and stop test (Algorithm 2 with the guards of the single-instance
// path; Algorithm 1 with rule 1).  One block per instance; instances already done are left alone.
__global__ void k_b_finish(const double* __restrict__ partials, const BatchTables t, BatchState bs, int initial,
                           int rule, double tol, int check_stop, int limit) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  if (!initial && bs.done[i]) return;
  const int p0 = t.part0[i], np = t.nparts[i];
  double s = 0.0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) s += partials[p0 + p];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double err = sqrt(red[0]);
  const int it = initial ? 0 : bs.iters[i] + 1;
  if (!initial) bs.iters[i] = it;
  if (it < bs.cap) bs.hist[(size_t)i * bs.cap + it] = err;
  bs.hist_len[i] = it + 1;
  const double prev = bs.prev_err[i];
  bs.prev_err[i] = err;
  const double rn = sqrt((double)t.n[i]);
  int stop = 0;
  if (!isfinite(err)) {
    bs.nonfinite[i] = 1;
    stop = 1;
  } else if (initial) {
    stop = (check_stop && rule == 1 && err / rn <= tol) ? 1 : 0;
  } else {
    if (check_stop) {
      if (rule == 1)
        stop = err / rn <= tol;
      else
        stop = (err > prev * prev * prev) || (err >= prev);
    }
    if (it >= limit) stop = 1;
  }
  if (stop) {
    bs.done[i] = 1;
    atomicSub(bs.live, 1);
  }
}

}  // namespace

cudaError_t launch_b_gersh(const BatchTables& t, int count, int max_n, unsigned long long* gmax_bits,
                           cudaStream_t s) {
  cudaMemsetAsync(gmax_bits, 0, sizeof(unsigned long long) * count, s);
  dim3 grid((max_n + 7) / 8, count);
  k_b_rowabs<<<grid, 256, 0, s>>>(t, gmax_bits);
  return cudaGetLastError();
}

cudaError_t launch_b_ranges(const BatchTables& t, int count, int max_n, unsigned long long* gmax_bits,
                            unsigned long long* zmax_bits, cudaStream_t s) {
  cudaMemsetAsync(gmax_bits, 0, sizeof(unsigned long long) * count, s);
  cudaMemsetAsync(zmax_bits, 0, sizeof(unsigned long long) * count, s);
  dim3 grid((max_n + 7) / 8, count);
  k_b_ranges<<<grid, 256, 0, s>>>(t, gmax_bits, zmax_bits);
  return cudaGetLastError();
}

cudaError_t launch_b_rho(const BatchTables& t, int count, int max_n, int rows, unsigned int* rho2,
                        void* scratch, cudaStream_t s) {
  // rho2[0..count): rows of S_i; rho2[count..2 count): columns of Z_i
  unsigned long long* cmax = static_cast<unsigned long long*>(scratch);
  float* csum = reinterpret_cast<float*>(cmax + rows);
  cudaError_t e = cudaMemsetAsync(rho2, 0, sizeof(unsigned int) * 2 * (size_t)count, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, b_rho_scratch_bytes(rows), s);
  if (e != cudaSuccess) return e;
  k_b_rowrho<<<dim3((max_n + 7) / 8, count), 256, 0, s>>>(t, rho2);
  const dim3 grid((max_n + 31) / 32, (max_n + 255) / 256, count), block(32, 8);
  k_b_colmax<<<grid, block, 0, s>>>(t, cmax);
  k_b_colsum<<<grid, block, 0, s>>>(t, cmax, csum);
  k_b_colfin<<<dim3((max_n + 255) / 256, count), 256, 0, s>>>(t, cmax, csum, rho2 + count);
  return cudaGetLastError();
}

size_t b_rho_scratch_bytes(int rows) { return (size_t)rows * (sizeof(unsigned long long) + sizeof(float)); }

cudaError_t launch_b_pack(const BatchTables& t, int count, int max_n, int mode, const unsigned long long* gmax_bits,
                          int ld, bool bf16, uint16_t* h16, uint16_t* l16, uint16_t* th16, uint16_t* tl16, float* m32,
                          cudaStream_t s) {
  dim3 grid((max_n + 31) / 32, (max_n + 31) / 32, count), block(32, 8);
  k_b_pack<<<grid, block, 0, s>>>(t, mode, gmax_bits, ld, bf16 ? 1 : 0, h16, l16, th16, tl16, m32);
  return cudaGetLastError();
}

cudaError_t launch_b_unpack(const BatchTables& t, int count, int max_n, const float* m32, int ld, cudaStream_t s) {
  dim3 grid((max_n + 31) / 32 < 32 ? (max_n + 31) / 32 : 32, (max_n + 7) / 8 < 64 ? (max_n + 7) / 8 : 64, count),
      block(32, 8);
  k_b_unpack<<<grid, block, 0, s>>>(t, m32, ld);
  return cudaGetLastError();
}

cudaError_t launch_b_finish(const double* partials, const BatchTables& t, const BatchState& bs, int count,
                            int initial, int rule, double tol, int check_stop, int limit, cudaStream_t s) {
  k_b_finish<<<count, 256, 0, s>>>(partials, t, bs, initial, rule, tol, check_stop, limit);
  return cudaGetLastError();
}

}  // namespace zf

// FP64-accurate products on the BF16 tensor cores by error-free slicing
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012).
//
// Every row r of an FP64 operand X is scaled by 2^-e_r (e_r: smallest power of two
// bounding the row's largest magnitude) and peeled into s integer slices of b bits:
//     x = 2^e_r * sum_p a_p 2^{-b(p+1)} + remainder,   a_0 in [-2^b, 2^b],
//     a_p in [-2^{b-1}, 2^{b-1}] for p >= 1  (round to nearest at every step),
// so every slice value is an integer that BF16 holds exactly.  The product of two
// sliced operands is  C_ij = 2^{eA_i + eB_j} sum_{t} 2^{-b(t+2)} G_t,ij  with
// G_t = sum_{p+q=t} A_p B_q^T; the terms p + q >= s are dropped (Ozaki's
// truncation).  The tensor-core engine forms each G_t over K-chunks short enough
// that every partial sum is an integer below 2^24, i.e. exact in FP32; the
// combine kernels below add the groups in FP64.
#include <math.h>

#include "kernels.h"

namespace zf {
namespace {

// The same for T > 62 bits (more than ten 6-bit slices): a 128-bit fixed point.
__device__ __forceinline__ __int128 fixed_point128(double x, int e, int T) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (eb == 0 && m == 0) return 0;
  int E;
  if (eb == 0) {
    E = -1074;
  } else {
    m |= 1ull << 52;
    E = eb - 1075;
  }
  const int sh = E - e + T;
  __int128 F;
  if (sh >= 0)
    F = (__int128)m << (sh < 74 ? sh : 74);
  else if (sh > -63)
    F = (__int128)((m + (1ull << (-sh - 1))) >> (-sh));
  else
    F = 0;
  return (bits >> 63) ? -F : F;
}

// Digits of a fixed-point row value: digit p is the next b bits, rounded to nearest.
template <typename I>
__device__ __forceinline__ void slice_digits(I F, int T, int s, int b, uint16_t* out, size_t stride) {
  for (int p = 0; p < s; ++p) {
    const int sh = T - b * (p + 1);
    const I a = sh > 0 ? ((F + ((I)1 << (sh - 1))) >> sh) : F;
    F -= a << sh;
    out[(size_t)p * stride] = __bfloat16_as_ushort(__float2bfloat16((float)(long long)a));
  }
}

// The same digits for T <= 62 in offset binary, with 32-bit operations only.  With
// D = 2^(b-1) sum_{p>=1} 2^(T-b(p+1)) and U = F + D, digit p >= 1 is ((U >> (T-b(p+1))) mod 2^b) - 2^(b-1),
// in [-2^(b-1), 2^(b-1)), and digit 0 is U >> (T-b) (floor), in [-2^b, 2^b]; they sum back to U - D = F.
// (A balanced representation like slice_digits' round-to-nearest one, within the same digit bounds.)
__device__ __forceinline__ long long offset_of(int T, int s, int b) {
  long long D = 0;
  for (int p = 1; p < s; ++p) D += 1ll << (T - b * (p + 1) + b - 1);
  return D;
}
__device__ __forceinline__ uint16_t bf16_of_small_int(int a) {
  // |a| <= 2^b with b <= 7: exact in BF16, whose bits are the top half of the FP32 bits
  return (uint16_t)(__float_as_uint(__int2float_rn(a)) >> 16);
}
__device__ __forceinline__ void slice_digits_offset(long long F, long long D, int T, int s, int b, uint16_t* out,
                                                    size_t stride) {
  const long long U = F + D;
  out[0] = bf16_of_small_int((int)(U >> (T - b)));
  const unsigned lo = (unsigned)U, hi = (unsigned)((unsigned long long)U >> 32);
  const unsigned mask = (1u << b) - 1u;
  const int half = 1 << (b - 1);
  for (int p = 1; p < s; ++p) {
    const int sh = T - b * (p + 1);
    const unsigned u = (sh >= 32 ? (hi >> (sh - 32)) : __funnelshift_r(lo, hi, sh)) & mask;
    out[(size_t)p * stride] = bf16_of_small_int((int)u - half);
  }
}

// Column statistics of X (operand rows = columns of X) in three light passes over a 2-D grid (32 columns
// x 256 rows per block, so that every SM has work): the columns' largest magnitudes (bit patterns,
// integer pipes, atomic maximum per column), optionally the sums of (x 2^-e_j)^2 in FP32 (atomic add per
// column), then e_j and the largest sum.  cmax and csum start at zero.
__global__ void k_oz_colmax(const double* __restrict__ X, int n, int ld, unsigned long long* __restrict__ cmax) {
  __shared__ unsigned long long red[8][33];
  const int j = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 256;
  const int r1 = r0 + 256 < n ? r0 + 256 : n;
  unsigned long long m = 0ull;
  if (j < n)
    for (int i = r0 + threadIdx.y; i < r1; i += 8) m = max_bits(m, abs_bits(X[(size_t)i * ld + j]));
  red[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0 && j < n) {
    for (int y = 1; y < 8; ++y) m = max_bits(m, red[y][threadIdx.x]);
    if (m) atomicMax(&cmax[j], m);
  }
}

__device__ __forceinline__ bool oz_no_bound(unsigned long long m) {
  // NaN or Inf, or a largest entry that is subnormal (its scaled values would read as zero)
  return m >= 0x7FF0000000000000ull || (m != 0ull && m < (1ull << 52));
}

__global__ void k_oz_colsum(const double* __restrict__ X, int n, int ld, const unsigned long long* __restrict__ cmax,
                            float* __restrict__ csum) {
  __shared__ float red[8][33];
  const int j = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 256;
  const int r1 = r0 + 256 < n ? r0 + 256 : n;
  float acc = 0.0f;
  const unsigned long long m = j < n ? cmax[j] : 0ull;
  if (m != 0ull && !oz_no_bound(m)) {
    const int e = exp_of_bits(m);
    for (int i = r0 + threadIdx.y; i < r1; i += 8) {
      const float f = scaled_mag_f32(abs_bits(X[(size_t)i * ld + j]), e);
      acc = fmaf(f, f, acc);
    }
  }
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && m != 0ull && !oz_no_bound(m)) {
    for (int y = 1; y < 8; ++y) acc += red[y][threadIdx.x];
    atomicAdd(&csum[j], acc);
  }
}

__global__ void k_oz_colfin(const unsigned long long* __restrict__ cmax, const float* __restrict__ csum, int n,
                            int* __restrict__ e, unsigned int* __restrict__ rho2) {
  const int j = blockIdx.x * 256 + threadIdx.x;
  unsigned u = 0u;
  if (j < n) {
    const unsigned long long m = cmax[j];
    e[j] = m ? exp_of_bits(m) : -2000000000;
    if (rho2) u = oz_no_bound(m) ? 0x7F800000u : __float_as_uint(csum[j]);
  }
  if (rho2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u = max(u, __shfl_xor_sync(0xffffffffu, u, o));
    if ((threadIdx.x & 31) == 0 && u) atomicMax(rho2, u);
  }
}

// x * 2^(T - e) rounded to the nearest integer (|x| < 2^e, so the result is below 2^T in
// magnitude), from the bits of x alone: integer operations only, since GB300's FP64 pipe
// is far slower than its integer pipes.
__device__ __forceinline__ long long fixed_point(double x, int e, int T) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (eb == 0 && m == 0) return 0;
  int E;
  if (eb == 0) {
    E = -1074;
  } else {
    m |= 1ull << 52;
    E = eb - 1075;
  }
  const int sh = E - e + T;  // value = m 2^E; want m 2^(E - e + T)
  long long F;
  if (sh >= 0)
    F = (long long)(m << (sh < 11 ? sh : 11));
  else if (sh > -63)
    F = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
  else
    F = 0;
  return (bits >> 63) ? -F : F;
}

// Slices of X (TRANS = false: operand rows are rows of X) or of X^T (TRANS = true: operand
// rows are columns of X).  Slice p, operand row r, column k -> out[(p * Rp + r) * ld16 + k].
// The row is held as a fixed-point integer F of T = s*b bits; digit p is F's next b bits
// rounded to nearest (a_0 in [-2^b, 2^b], later digits in [-2^(b-1), 2^(b-1)]).
template <bool TRANS>
__global__ void k_oz_slice(const double* __restrict__ X, int n, int ld, const int* __restrict__ e, int s, int b,
                           uint16_t* __restrict__ out, int ld16, int Rp) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int i = bi + r, j = bj + tx;
    tile[r][tx] = (i < n && j < n) ? X[(size_t)i * ld + j] : 0.0;
  }
  __syncthreads();
  const int T = s * b;
  const long long D = T <= 62 ? offset_of(T, s, b) : 0;
  for (int r = ty; r < 32; r += 8) {
    int row, col;
    double x;
    if (TRANS) {
      row = bj + r;  // operand row = column of X
      col = bi + tx;
      x = tile[tx][r];
    } else {
      row = bi + r;
      col = bj + tx;
      x = tile[r][tx];
    }
    if (row >= n || col >= n) continue;
    const int er = e[row];
    uint16_t* o = out + (size_t)row * ld16 + col;
    const size_t stride = (size_t)Rp * ld16;
    if (T <= 62)
      slice_digits_offset((er > -1000) ? fixed_point(x, er, T) : 0, D, T, s, b, o, stride);
    else
      slice_digits<__int128>((er > -1000) ? fixed_point128(x, er, T) : 0, T, s, b, o, stride);
  }
}

// Slices of X^T (operand rows = columns of X), T <= 62: a 64 x 32 tile of X (rows bi.., columns
// bj..) through shared memory (even and odd rows apart, so the transposed reads are conflict-free);
// each thread forms two adjacent operand columns (X rows) and stores their digits as one 4-byte word.
__global__ void k_oz_tslice2(const double* __restrict__ X, int n, int ld, const int* __restrict__ e, int s, int b,
                             uint16_t* __restrict__ out, int ld16, int Rp) {
  __shared__ double te[32][33], to[32][33];
  const int bi = blockIdx.y * 64, bj = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int rr = ty; rr < 64; rr += 8) {
    const int i = bi + rr, j = bj + tx;
    const double x = (i < n && j < n) ? X[(size_t)i * ld + j] : 0.0;
    if (rr & 1)
      to[rr >> 1][tx] = x;
    else
      te[rr >> 1][tx] = x;
  }
  __syncthreads();
  const int T = s * b;
  const long long D = offset_of(T, s, b);
  const unsigned mask = (1u << b) - 1u;
  const int half = 1 << (b - 1);
  const size_t stride = (size_t)Rp * ld16;
  const int col = bi + 2 * tx;  // operand columns col, col + 1 = X rows
  for (int r = ty; r < 32; r += 8) {
    const int row = bj + r;  // operand row = X column
    if (row >= n || col >= n) continue;
    const int er = e[row];
    const long long U0 = ((er > -1000) ? fixed_point(te[tx][r], er, T) : 0) + D;
    const long long U1 = ((er > -1000) ? fixed_point(to[tx][r], er, T) : 0) + D;
    uint16_t* o = out + (size_t)row * ld16 + col;
    const bool pair = col + 1 < n;
    unsigned w = (unsigned)bf16_of_small_int((int)(U0 >> (T - b))) |
                 ((unsigned)bf16_of_small_int((int)(U1 >> (T - b))) << 16);
    if (pair)
      *reinterpret_cast<unsigned*>(o) = w;
    else
      *o = (uint16_t)w;
    const unsigned lo0 = (unsigned)U0, hi0 = (unsigned)((unsigned long long)U0 >> 32);
    const unsigned lo1 = (unsigned)U1, hi1 = (unsigned)((unsigned long long)U1 >> 32);
    for (int p = 1; p < s; ++p) {
      const int sh = T - b * (p + 1);
      const unsigned u0 = (sh >= 32 ? (hi0 >> (sh - 32)) : __funnelshift_r(lo0, hi0, sh)) & mask;
      const unsigned u1 = (sh >= 32 ? (hi1 >> (sh - 32)) : __funnelshift_r(lo1, hi1, sh)) & mask;
      w = (unsigned)bf16_of_small_int((int)u0 - half) | ((unsigned)bf16_of_small_int((int)u1 - half) << 16);
      uint16_t* op = o + (size_t)p * stride;
      if (pair)
        *reinterpret_cast<unsigned*>(op) = w;
      else
        *op = (uint16_t)w;
    }
  }
}

// Row slices of X (operand rows = rows of X): one warp per row finds the row's exponent and
// then slices the row (two coalesced passes, the second from cache; no atomics).
__global__ void k_oz_rowslice(const double* __restrict__ X, int n, int ld, int* __restrict__ e, int s, int b,
                              uint16_t* __restrict__ out, int ld16, int Rp, int vec) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* xr = X + (size_t)row * ld;
  // vec: the row starts on 16 bytes (X aligned, ld even), so lanes take element pairs
  const int npair = vec ? n / 2 : 0;
  unsigned long long m = 0ull;  // magnitude bit patterns: integer pipes only
  for (int c = lane; c < npair; c += 32) {
    const double2 v = reinterpret_cast<const double2*>(xr)[c];
    m = max_bits(m, max_bits(abs_bits(v.x), abs_bits(v.y)));
  }
  for (int c = 2 * npair + lane; c < n; c += 32) m = max_bits(m, abs_bits(xr[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int er = m ? exp_of_bits(m) : -2000000000;
  if (lane == 0) e[row] = er;
  const int T = s * b;
  const size_t stride = (size_t)Rp * ld16;
  uint16_t* orow = out + (size_t)row * ld16;
  if (T <= 62) {
    const long long D = offset_of(T, s, b);
    for (int c = lane; c < npair; c += 32) {
      const double2 v = reinterpret_cast<const double2*>(xr)[c];
      const long long F0 = (er > -1000) ? fixed_point(v.x, er, T) : 0;
      const long long F1 = (er > -1000) ? fixed_point(v.y, er, T) : 0;
      // both elements' digits, packed into one 4-byte store per slice
      const long long U0 = F0 + D, U1 = F1 + D;
      unsigned* o = reinterpret_cast<unsigned*>(orow + 2 * c);
      *o = (unsigned)bf16_of_small_int((int)(U0 >> (T - b))) |
           ((unsigned)bf16_of_small_int((int)(U1 >> (T - b))) << 16);
      const unsigned lo0 = (unsigned)U0, hi0 = (unsigned)((unsigned long long)U0 >> 32);
      const unsigned lo1 = (unsigned)U1, hi1 = (unsigned)((unsigned long long)U1 >> 32);
      const unsigned mask = (1u << b) - 1u;
      const int half = 1 << (b - 1);
      for (int p = 1; p < s; ++p) {
        const int sh = T - b * (p + 1);
        const unsigned u0 = (sh >= 32 ? (hi0 >> (sh - 32)) : __funnelshift_r(lo0, hi0, sh)) & mask;
        const unsigned u1 = (sh >= 32 ? (hi1 >> (sh - 32)) : __funnelshift_r(lo1, hi1, sh)) & mask;
        o = reinterpret_cast<unsigned*>(orow + (size_t)p * stride + 2 * c);
        *o = (unsigned)bf16_of_small_int((int)u0 - half) | ((unsigned)bf16_of_small_int((int)u1 - half) << 16);
      }
    }
    for (int c = 2 * npair + lane; c < n; c += 32)
      slice_digits_offset((er > -1000) ? fixed_point(xr[c], er, T) : 0, D, T, s, b, orow + c, stride);
  } else {
    for (int c = lane; c < n; c += 32)
      slice_digits<__int128>((er > -1000) ? fixed_point128(xr[c], er, T) : 0, T, s, b, orow + c, stride);
  }
}

// The same with the row held in registers: one block of NT threads per row, each thread up to
// PAIRS element pairs (so n <= 2 NT PAIRS), 16-byte loads (the row starts on 16 bytes), one read of
// X for both the exponent and the digits.  T <= 62 only.
template <int NT, int PAIRS>
__global__ void __launch_bounds__(NT) k_oz_rowslice_reg(const double* __restrict__ X, int n, int ld,
                                                       int* __restrict__ e, int s, int b, uint16_t* __restrict__ out,
                                                       int ld16, int Rp) {
  __shared__ unsigned long long red[NT / 32];
  const int row = blockIdx.x;
  const int tid = threadIdx.x;
  const double* xr = X + (size_t)row * ld;
  const int npair = n / 2;
  double2 v[PAIRS];
  unsigned long long m = 0ull;  // magnitude bit patterns: integer pipes only
#pragma unroll
  for (int k = 0; k < PAIRS; ++k) {
    const int c = tid + NT * k;
    v[k] = c < npair ? reinterpret_cast<const double2*>(xr)[c] : make_double2(0.0, 0.0);
    m = max_bits(m, max_bits(abs_bits(v[k].x), abs_bits(v[k].y)));
  }
  const double last = ((n & 1) && tid == 0) ? xr[n - 1] : 0.0;
  m = max_bits(m, abs_bits(last));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) m = max_bits(m, red[w]);
  const int er = m ? exp_of_bits(m) : -2000000000;
  if (tid == 0) e[row] = er;
  const int T = s * b;
  const size_t stride = (size_t)Rp * ld16;
  uint16_t* orow = out + (size_t)row * ld16;
  const long long D = offset_of(T, s, b);
  const unsigned mask = (1u << b) - 1u;
  const int half = 1 << (b - 1);
#pragma unroll
  for (int k = 0; k < PAIRS; ++k) {
    const int c = tid + NT * k;
    if (c >= npair) break;
    const long long U0 = ((er > -1000) ? fixed_point(v[k].x, er, T) : 0) + D;
    const long long U1 = ((er > -1000) ? fixed_point(v[k].y, er, T) : 0) + D;
    unsigned* o = reinterpret_cast<unsigned*>(orow + 2 * c);
    *o = (unsigned)bf16_of_small_int((int)(U0 >> (T - b))) | ((unsigned)bf16_of_small_int((int)(U1 >> (T - b))) << 16);
    const unsigned lo0 = (unsigned)U0, hi0 = (unsigned)((unsigned long long)U0 >> 32);
    const unsigned lo1 = (unsigned)U1, hi1 = (unsigned)((unsigned long long)U1 >> 32);
    for (int p = 1; p < s; ++p) {
      const int sh = T - b * (p + 1);
      const unsigned u0 = (sh >= 32 ? (hi0 >> (sh - 32)) : __funnelshift_r(lo0, hi0, sh)) & mask;
      const unsigned u1 = (sh >= 32 ? (hi1 >> (sh - 32)) : __funnelshift_r(lo1, hi1, sh)) & mask;
      o = reinterpret_cast<unsigned*>(orow + (size_t)p * stride + 2 * c);
      *o = (unsigned)bf16_of_small_int((int)u0 - half) | ((unsigned)bf16_of_small_int((int)u1 - half) << 16);
    }
  }
  if ((n & 1) && tid == 0)
    slice_digits_offset((er > -1000) ? fixed_point(last, er, T) : 0, D, T, s, b, orow + (n - 1), stride);
}

// The exact groups of four rows of one column: T_t = sum_c G[t * nch + c] as int32 (below nch 2^24 <= 2^31),
// folded into I (t < k0) and J (k0 <= t < k1).  NCH > 0 fixes the chunk count at compile time so the
// chunk loop unrolls; with the group loop unrolled twice, 2 NCH 4 loads are in flight per thread.
template <int NCH>
__device__ __forceinline__ void exact_groups(const float* __restrict__ G, size_t gstride, int nch_rt, int k0, int k1,
                                             int b, const bool (&ok)[4], const size_t (&off)[4], long long (&I)[4],
                                             long long (&J)[4]) {
  const int nch = NCH > 0 ? NCH : nch_rt;
  const long long w = 1ll << b;
#pragma unroll 2
  for (int t = 0; t < k1; ++t) {
    const float* g = G + (size_t)t * nch * gstride;
    int tt[4] = {0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < (NCH > 0 ? NCH : nch); ++c) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (ok[q]) tt[q] += __float2int_rn(__ldcs(g + off[q]));
      g += gstride;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (t < k0)
        I[q] = I[q] * w + tt[q];
      else
        J[q] = J[q] * w + tt[q];
    }
  }
}

// Sum of the groups with the scales: val = 2^{eA_i + eB_j} 2^{-2b} sum_t 2^{-bt} T_t,
// T_t = sum_c G[t * nch + c] (exact integers, |T_t| < 2^30).  Two 64-bit integers hold the
// groups exactly: I = sum_{t<k0} T_t 2^{b(k0-1-t)} and J = sum_{k0<=t<k1} T_t 2^{b(k1-1-t)}
// (each below 2^55), so every group whose weight is above 2^-(b k1) ~ 2^-60 of the leading
// term is exact; only the tail t >= k1 is summed in FP32.  The scale 2^{eA_i + eB_j} belongs to
// the largest entries of row i and column j, so an inexact group here would cost a fixed
// fraction of |Z|^T |S Z| rather than of the result: with ill-conditioned Z, where
// I - Z^T S Z cancels by many orders, the sum has to stay exact well past the 53 bits of the
// result.  Two FP64 roundings join I, J and the tail.
// mode 0: out = val; mode 1: out += val; mode 2 (sym): d = I - val, with the block's sum of
// d^2 (off-diagonal entries twice) in partials[block].  32 x 32 tiles (blockDim 32 x 8): with
// sym only tiles on or above the diagonal run, and the mirrored tile is written through shared
// memory so that both writes are coalesced.
__global__ void k_oz_combine(const float* __restrict__ G, size_t gstride, int ld32, int s, int nch, int b,
                             const int* __restrict__ eA, const int* __restrict__ eB, int n, double* out, int ld64,
                             int mode, int sym, double* partials) {
  __shared__ double tile[32][33];
  __shared__ double red[256];
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const bool active = !(sym && bj < bi);
  double ss = 0.0;
  int k0 = (29 + b - 1) / b;
  if (k0 > s) k0 = s;
  int k1 = k0 + (29 + b - 1) / b;
  if (k1 > s) k1 = s;
  const float wb = ldexpf(1.0f, -b);
  if (active) {
    // the four rows of this thread side by side: four independent loads per (group, chunk)
    const int j = bj + threadIdx.x;
    bool ok[4];
    size_t off[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = bi + threadIdx.y + 8 * q;
      ok[q] = i < n && j < n;
      off[q] = ok[q] ? (size_t)i * ld32 + j : 0;
    }
    long long I[4] = {0, 0, 0, 0}, J[4] = {0, 0, 0, 0};
    switch (nch) {
      case 1: exact_groups<1>(G, gstride, nch, k0, k1, b, ok, off, I, J); break;
      case 2: exact_groups<2>(G, gstride, nch, k0, k1, b, ok, off, I, J); break;
      case 3: exact_groups<3>(G, gstride, nch, k0, k1, b, ok, off, I, J); break;
      case 4: exact_groups<4>(G, gstride, nch, k0, k1, b, ok, off, I, J); break;
      default: exact_groups<0>(G, gstride, nch, k0, k1, b, ok, off, I, J); break;
    }
    float F[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int t = s - 1; t >= k1; --t) {
      float tt[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int c = 0; c < nch; ++c) {
        const float* g = G + (size_t)(t * nch + c) * gstride;
#pragma unroll
        for (int q = 0; q < 4; ++q) tt[q] += ok[q] ? __ldcs(g + off[q]) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) F[q] = (F[q] + tt[q]) * wb;
    }
    const int eb = j < n ? eB[j] : -2000000000;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = threadIdx.y + 8 * q;
      const int i = bi + r;
      double val = 0.0;
      if (ok[q]) {
        const int ea = eA[i];
        if (ea > -1000 && eb > -1000) {
          const int e0 = ea + eb - 2 * b - b * (k0 - 1), e1 = ea + eb - 2 * b - b * (k1 - 1);
          val = ldexp((double)I[q], e0) + ldexp((double)J[q] + (double)F[q], e1);
        }
        if (mode == 2) {
          val = (i == j ? 1.0 : 0.0) - val;
          if (j >= i) ss += (i == j ? 1.0 : 2.0) * val * val;
        }
        double* o = out + (size_t)i * ld64 + j;
        const bool own = !sym || j >= i;  // in a diagonal tile only the upper half is formed
        if (own) {
          if (mode == 1)
            *o += val;
          else
            *o = val;
        }
      }
      tile[r][threadIdx.x] = val;
    }
    if (sym && bj > bi) {
      // the (j, i) mirror of this off-diagonal tile, coalesced through shared memory
      __syncthreads();
      for (int r = threadIdx.y; r < 32; r += 8) {
        const int oi = bj + r, oj = bi + threadIdx.x;
        if (oi < n && oj < n) {
          double* o = out + (size_t)oi * ld64 + oj;
          if (mode == 1)
            *o += tile[threadIdx.x][r];
          else
            *o = tile[threadIdx.x][r];
        }
      }
    } else if (sym) {
      // diagonal tile: mirror its upper half into its lower half
      __syncthreads();
      for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = bi + r, j = bj + threadIdx.x;
        if (i < n && j < n && j < i) {
          double* o = out + (size_t)i * ld64 + j;
          if (mode == 1)
            *o += tile[threadIdx.x][r];
          else
            *o = tile[threadIdx.x][r];
        }
      }
    }
  }
  if (mode == 2) {
    red[tid] = ss;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
  }
}

// d = I - X (X symmetric, FP64), partials[block] = sum over the block's entries of d^2.
__global__ void k_resid_from_x(const double* __restrict__ X, double* __restrict__ D, int n, double* partials) {
  __shared__ double red[256];
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int i = blockIdx.y * 8 + threadIdx.y;
  double ss = 0.0;
  if (i < n && j < n) {
    const double d = (i == j ? 1.0 : 0.0) - X[(size_t)i * n + j];
    D[(size_t)i * n + j] = d;
    ss = d * d;
  }
  const int tid = threadIdx.y * 32 + threadIdx.x;
  red[tid] = ss;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// out = a * X + b * Y (FP64, n x n contiguous)
__global__ void k_axpby64(double* out, double a, const double* X, double b, const double* Y, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    out[e] = a * X[e] + b * Y[e];
}

__global__ void k_pow2_slot(IterState* st, int amax_slot, int scale_slot, int head) {
  const double bound = st->amax[amax_slot];
  float sc = 1.0f;
  if (bound > 0.0 && isfinite(bound)) {
    int e;
    frexp(bound, &e);
    int p = 14 - head - e;
    p = p > 60 ? 60 : (p < -60 ? -60 : p);
    sc = ldexpf(1.0f, p);
  }
  st->scale[scale_slot] = sc;
}

}  // namespace

cudaError_t launch_pow2_slot(IterState* st, int amax_slot, int scale_slot, int head, cudaStream_t s) {
  k_pow2_slot<<<1, 1, 0, s>>>(st, amax_slot, scale_slot, head);
  return cudaGetLastError();
}

cudaError_t launch_oz_colstats(const double* X, int n, int ld, int* e, unsigned int* rho2, void* scratch,
                               cudaStream_t s) {
  if (n < 1 || !scratch) return cudaErrorInvalidValue;
  unsigned long long* cmax = static_cast<unsigned long long*>(scratch);
  float* csum = reinterpret_cast<float*>(cmax + n);
  cudaError_t err = cudaMemsetAsync(scratch, 0, oz_colstats_scratch_bytes(n), s);
  if (err != cudaSuccess) return err;
  const dim3 grid((n + 31) / 32, (n + 255) / 256), block(32, 8);
  k_oz_colmax<<<grid, block, 0, s>>>(X, n, ld, cmax);
  if (rho2) k_oz_colsum<<<grid, block, 0, s>>>(X, n, ld, cmax, csum);
  k_oz_colfin<<<(n + 255) / 256, 256, 0, s>>>(cmax, csum, n, e, rho2);
  return cudaGetLastError();
}

size_t oz_colstats_scratch_bytes(int n) { return (size_t)n * (sizeof(unsigned long long) + sizeof(float)); }

cudaError_t launch_oz_exp(const double* X, int n, int ld, bool cols, int* e, void* scratch, cudaStream_t s) {
  // column exponents only: row exponents are found by the row kernels themselves
  if (!cols) return cudaSuccess;
  return launch_oz_colstats(X, n, ld, e, nullptr, scratch, s);
}

cudaError_t launch_oz_slice(const double* X, int n, int ld, bool trans, const int* e, int sl, int b, uint16_t* out,
                            int ld16, int Rp, cudaStream_t s) {
  // padding rows n..Rp-1 of every slice read as zero: one strided memset over all of them
  if (Rp > n)
    cudaMemset2DAsync(out + (size_t)n * ld16, sizeof(uint16_t) * (size_t)Rp * ld16, 0,
                      sizeof(uint16_t) * (size_t)(Rp - n) * ld16, sl, s);
  if (trans) {
    if (sl * b <= 62 && (ld16 & 1) == 0) {
      dim3 grid((n + 31) / 32, (n + 63) / 64), block(32, 8);
      k_oz_tslice2<<<grid, block, 0, s>>>(X, n, ld, e, sl, b, out, ld16, Rp);
    } else {
      dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
      k_oz_slice<true><<<grid, block, 0, s>>>(X, n, ld, e, sl, b, out, ld16, Rp);
    }
  } else {
    const int vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0 && (ld & 1) == 0 && (ld16 & 1) == 0) ? 1 : 0;
    if (vec && sl * b <= 62 && n <= 2 * 256 * 8)
      k_oz_rowslice_reg<256, 8><<<n, 256, 0, s>>>(X, n, ld, const_cast<int*>(e), sl, b, out, ld16, Rp);
    else if (vec && sl * b <= 62 && n <= 2 * 512 * 16)
      k_oz_rowslice_reg<512, 16><<<n, 512, 0, s>>>(X, n, ld, const_cast<int*>(e), sl, b, out, ld16, Rp);
    else
      k_oz_rowslice<<<(n + 7) / 8, 256, 0, s>>>(X, n, ld, const_cast<int*>(e), sl, b, out, ld16, Rp, vec);
  }
  return cudaGetLastError();
}

int oz_combine_blocks(int n) { return ((n + 31) / 32) * ((n + 31) / 32); }

cudaError_t launch_oz_combine(const float* G, size_t gstride, int ld32, int sl, int nch, int b, const int* eA,
                              const int* eB, int n, double* out, int ld64, int mode, bool sym, double* partials,
                              cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  k_oz_combine<<<grid, block, 0, s>>>(G, gstride, ld32, sl, nch, b, eA, eB, n, out, ld64, mode, sym ? 1 : 0,
                                      partials);
  return cudaGetLastError();
}

int resid_from_x_blocks(int n) { return ((n + 31) / 32) * ((n + 7) / 8); }

cudaError_t launch_resid_from_x(const double* X, double* D, int n, double* partials, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 7) / 8), block(32, 8);
  k_resid_from_x<<<grid, block, 0, s>>>(X, D, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_axpby64(double* out, double a, const double* X, double b, const double* Y, size_t total,
                           cudaStream_t s) {
  const int blocks = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  k_axpby64<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(out, a, X, b, Y, total);
  return cudaGetLastError();
}

}  // namespace zf

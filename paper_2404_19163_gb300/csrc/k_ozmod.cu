// FP64-accurate products on the BF16 tensor cores by modular arithmetic (Ozaki scheme II:
// Ozaki, Uchino, Imamura, "Ozaki Scheme II: A GEMM-oriented emulation of floating-point matrix
// multiplication using an integer modular technique", 2025).
//
// Every row r of an FP64 operand is scaled by 2^(T - e_r) (e_r: the row's exponent bound) and
// rounded to an integer F with |F| <= 2^T.  The product C' = F_A F_B^T of two such integer
// matrices is exact and bounded by K 2^(T_A + T_B).  It is formed modulo pairwise coprime
// moduli m_i <= 127: the symmetric residues of F (|r| <= 63) are exact in BF16, one residue
// product over K <= 4224 terms stays an integer below 2^24 (exact in the FP32 accumulator), and
// the Chinese remainder theorem recovers C' from its residues once M = prod m_i > 4 |C'|.  The
// result is C_ij = 2^(eA_i + eB_j - T_A - T_B) C'_ij: the only errors are the two roundings to
// T-bit fixed point and the final conversion to FP64.  The moduli count grows linearly with the
// bits kept (about 6.4 bits per product), where slicing grows quadratically (s(s+1)/2 pairs).
#include <math.h>

#include "kernels.h"

namespace zf {

namespace {

__device__ __forceinline__ int exp_bound_m(double v) {
  int e;
  frexp(v, &e);
  return e;
}

// round(x 2^(T - e)) for |x| < 2^e and T <= 62, from the bits of x (integer operations only).
__device__ __forceinline__ long long fixed_point_m(double x, int e, int T) {
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
  long long F;
  if (sh >= 0)
    F = (long long)(m << (sh < 11 ? sh : 11));
  else if (sh > -63)
    F = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
  else
    F = 0;
  return (bits >> 63) ? -F : F;
}

// The residues of an element pair for moduli I.. (compile-time moduli, FP32 arithmetic of
// crt_residue_f), each pair packed as two BF16 into one 4-byte store (an integer |r| <= 63
// has its low 16 FP32 bits zero, so the BF16 value is the upper half).
template <int I>
__device__ __forceinline__ void residues_pair_all(const float (&p0)[5], const float (&p1)[5], int nmod, uint16_t* o,
                                                  size_t stride) {
  if constexpr (I < kCrtMax) {
    if (I < nmod) {
      const float r0 = crt_residue_f(p0, crt_modulus(I)), r1 = crt_residue_f(p1, crt_modulus(I));
      *reinterpret_cast<unsigned*>(o + (size_t)I * stride) =
          __byte_perm(__float_as_uint(r0), __float_as_uint(r1), 0x7632);
      residues_pair_all<I + 1>(p0, p1, nmod, o, stride);
    }
  }
}

template <int I>
__device__ __forceinline__ void residues_one_all(const float (&p0)[5], int nmod, uint16_t* o, size_t stride) {
  if constexpr (I < kCrtMax) {
    if (I < nmod) {
      o[(size_t)I * stride] = (uint16_t)(__float_as_uint(crt_residue_f(p0, crt_modulus(I))) >> 16);
      residues_one_all<I + 1>(p0, nmod, o, stride);
    }
  }
}

__device__ __forceinline__ void parts_of(double x, int er, int T, float (&p)[5]) {
  crt_parts(er > -1000 ? fixed_point_m(x, er, T) : 0, p);
}

// Residues of the rows of X (operand rows = rows of X): one block of NT threads per row finds
// the row's exponent and writes the nmod residue planes, two elements per 4-byte store.  With
// PAIRS > 0 the row stays in registers (n <= 2 NT PAIRS); PAIRS = 0 reads it twice.
template <int NT, int PAIRS>
__global__ void __launch_bounds__(NT) k_ozm_rowres(const double* __restrict__ X, int n, int ld, int* __restrict__ e,
                                                  int T, int nmod, uint16_t* __restrict__ out, int ld16, int Rp) {
  __shared__ double red[NT / 32];
  const int row = blockIdx.x;
  const int tid = threadIdx.x;
  const double* xr = X + (size_t)row * ld;
  const int npair = n / 2;
  constexpr int NREG = PAIRS > 0 ? PAIRS : 1;
  double v0[NREG], v1[NREG];
  double m = 0.0;
  if (PAIRS > 0) {
#pragma unroll
    for (int k = 0; k < NREG; ++k) {
      const int c = tid + NT * k;
      v0[k] = c < npair ? xr[2 * c] : 0.0;
      v1[k] = c < npair ? xr[2 * c + 1] : 0.0;
      m = fmax(m, fmax(fabs(v0[k]), fabs(v1[k])));
    }
  } else {
    for (int c = tid; c < n; c += NT) m = fmax(m, fabs(xr[c]));
  }
  if (PAIRS > 0 && (n & 1) && tid == 0) m = fmax(m, fabs(xr[n - 1]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) m = fmax(m, red[w]);
  const int er = m > 0.0 ? exp_bound_m(m) : -2000000000;
  if (tid == 0) e[row] = er;
  const size_t stride = (size_t)Rp * ld16;
  uint16_t* orow = out + (size_t)row * ld16;
  if (PAIRS > 0) {
#pragma unroll
    for (int k = 0; k < NREG; ++k) {
      const int c = tid + NT * k;
      if (c >= npair) break;
      float p0[5], p1[5];
      parts_of(v0[k], er, T, p0);
      parts_of(v1[k], er, T, p1);
      residues_pair_all<0>(p0, p1, nmod, orow + 2 * c, stride);
    }
  } else {
    for (int c = tid; c < npair; c += NT) {
      float p0[5], p1[5];
      parts_of(xr[2 * c], er, T, p0);
      parts_of(xr[2 * c + 1], er, T, p1);
      residues_pair_all<0>(p0, p1, nmod, orow + 2 * c, stride);
    }
  }
  if ((n & 1) && tid == 0) {
    float p0[5];
    parts_of(xr[n - 1], er, T, p0);
    residues_one_all<0>(p0, nmod, orow + (n - 1), stride);
  }
}

// Residues of X^T (operand rows = columns of X; exponents from launch_oz_exp(cols = true)): a
// 64 x 32 tile of X (rows bi.., columns bj..) through shared memory, even and odd rows apart so
// the transposed reads are conflict-free; each thread forms two adjacent operand columns (X rows).
__global__ void k_ozm_tres(const double* __restrict__ X, int n, int ld, const int* __restrict__ e, int T, int nmod,
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
  const size_t stride = (size_t)Rp * ld16;
  const int col = bi + 2 * tx;
  for (int r = ty; r < 32; r += 8) {
    const int row = bj + r;
    if (row >= n || col >= n) continue;
    const int er = e[row];
    float p0[5], p1[5];
    parts_of(te[tx][r], er, T, p0);
    parts_of(to[tx][r], er, T, p1);
    uint16_t* o = out + (size_t)row * ld16 + col;
    if (col + 1 < n)
      residues_pair_all<0>(p0, p1, nmod, o, stride);
    else
      residues_one_all<0>(p0, nmod, o, stride);
  }
}

// The partials of all moduli of one element for K-chunk c (slot t * nch + c), issued together.
__device__ __forceinline__ void load_moduli(const float* __restrict__ g, size_t slot, int nmod, bool ok,
                                            float (&v)[kCrtMax]) {
#pragma unroll
  for (int t = 0; t < kCrtMax; ++t) v[t] = (ok && t < nmod) ? __ldcs(g + (size_t)t * slot) : 0.0f;
}

// C' from the residue products and the scales: per modulus the K-chunk partials (exact FP32
// integers) are reduced (crt_fmod_sym) and summed, the CRT digits y_t = r_t w_t mod m_t weight the
// limbs of M / m_t, and the FP32 sum of y_t / m_t gives the multiple of M to remove (CrtAcc).
// Modes as the slicing combine: 0 out = C, 1 out += C, 2 (sym) d = I - C with the block's sum of
// d^2 in partials[block].  32 x 32 tiles, blockDim 32 x 8, four rows per thread, two blocks per SM;
// with one K-chunk the loads of the next row are in flight while a row is reduced.  With sym only
// tiles on or above the diagonal run and the mirror goes through shared memory.
__global__ void __launch_bounds__(256, 2) k_ozm_combine(const float* __restrict__ G, size_t gstride, int ld32, int nch,
                                                        CrtPlan plan, const int* __restrict__ eA,
                                                        const int* __restrict__ eB, int TA, int TB, int n,
                                                        double* out, int ld64, int mode, int sym, double* partials) {
  __shared__ double tile[32][33];
  __shared__ double red[256];
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const bool active = !(sym && bj < bi);
  const int nmod = plan.nmod;
  double ss = 0.0;
  if (active) {
    const int j = bj + threadIdx.x;
    const int eb = j < n ? eB[j] : -2000000000;
    bool ok[4];
    size_t off[4];
    int ea[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = bi + threadIdx.y + 8 * q;
      ok[q] = i < n && j < n;
      off[q] = ok[q] ? (size_t)i * ld32 + j : 0;
      ea[q] = ok[q] ? eA[i] : -2000000000;
    }
    const size_t slot = (size_t)nch * gstride;
    double val[4];
    float cur[kCrtMax], nxt[kCrtMax];
    if (nch == 1) load_moduli(G + off[0], slot, nmod, ok[0], cur);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float r[kCrtMax];
      if (nch == 1) {
        if (q < 3) load_moduli(G + off[q + 1], slot, nmod, ok[q + 1], nxt);
#pragma unroll
        for (int t = 0; t < kCrtMax; ++t) r[t] = crt_fmod_sym(cur[t], plan.fm[t], plan.inv[t]);
      } else {
#pragma unroll
        for (int t = 0; t < kCrtMax; ++t) r[t] = 0.0f;
        for (int c = 0; c < nch; ++c) {
          float v[kCrtMax];
          load_moduli(G + (size_t)c * gstride + off[q], slot, nmod, ok[q], v);
#pragma unroll
          for (int t = 0; t < kCrtMax; ++t) r[t] += crt_fmod_sym(v[t], plan.fm[t], plan.inv[t]);
        }
      }
      CrtAcc acc;
      acc.clear();
#pragma unroll
      for (int t = 0; t < kCrtMax; ++t)
        if (t < nmod) acc.add_f(plan, t, r[t]);
      const int i = bi + threadIdx.y + 8 * q;
      double v = 0.0;
      if (ok[q]) {
        if (ea[q] > -1000 && eb > -1000) v = acc.value(plan, ea[q] + eb - TA - TB);
        if (mode == 2) {
          v = (i == j ? 1.0 : 0.0) - v;
          if (j >= i) ss += (i == j ? 1.0 : 2.0) * v * v;
        }
      }
      val[q] = v;
      if (nch == 1 && q < 3) {
#pragma unroll
        for (int t = 0; t < kCrtMax; ++t) cur[t] = nxt[t];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = threadIdx.y + 8 * q;
      const int i = bi + r;
      if (ok[q] && (!sym || j >= i)) {
        double* o = out + (size_t)i * ld64 + j;
        if (mode == 1)
          *o += val[q];
        else
          *o = val[q];
      }
      tile[r][threadIdx.x] = val[q];
    }
    if (sym && bj > bi) {
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
      __syncthreads();
      for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = bi + r, j2 = bj + threadIdx.x;
        if (i < n && j2 < n && j2 < i) {
          double* o = out + (size_t)i * ld64 + j2;
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

}  // namespace

cudaError_t launch_ozm_residues(const double* X, int n, int ld, bool trans, int* e, int T, int nmod, uint16_t* out,
                                int ld16, int Rp, cudaStream_t s) {
  if (nmod < 1 || nmod > kCrtMax || T < 1 || T > 62) return cudaErrorInvalidValue;
  for (int p = 0; p < nmod; ++p)  // padding rows n..Rp-1 of every plane read as zero
    if (Rp > n) cudaMemsetAsync(out + ((size_t)p * Rp + n) * ld16, 0, sizeof(uint16_t) * (size_t)(Rp - n) * ld16, s);
  if (trans) {
    dim3 grid((n + 31) / 32, (n + 63) / 64), block(32, 8);
    k_ozm_tres<<<grid, block, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
  } else if (n <= 2 * 256 * 8) {
    k_ozm_rowres<256, 8><<<n, 256, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
  } else {
    k_ozm_rowres<256, 0><<<n, 256, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
  }
  return cudaGetLastError();
}

cudaError_t launch_ozm_combine(const float* G, size_t gstride, int ld32, int nch, const CrtPlan& plan, const int* eA,
                               const int* eB, int TA, int TB, int n, double* out, int ld64, int mode, bool sym,
                               double* partials, cudaStream_t s) {
  if (nch < 1 || nch > kCrtMaxChunks) return cudaErrorInvalidValue;
  dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  k_ozm_combine<<<grid, block, 0, s>>>(G, gstride, ld32, nch, plan, eA, eB, TA, TB, n, out, ld64, mode, sym ? 1 : 0,
                                       partials);
  return cudaGetLastError();
}

}  // namespace zf

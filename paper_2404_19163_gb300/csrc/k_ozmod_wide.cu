// Wider CRT residue products (crt_wide.h): rows of up to 83 bits kept as 128-bit fixed point, up to
// 24 moduli, six-limb reconstruction.  Used by the default scheme for products whose bound passes
// the sixteen moduli of k_ozmod.cu (an ill-conditioned Z, whose residual asks for 60 to 83 bits per
// row).  Same layouts as k_ozmod.cu, whose reconstruction kernel
// takes the wider plan too.
#include <math.h>

#include "crt_wide.h"
#include "kernels.h"

namespace zf {
namespace {

// round(x 2^(T - e)) for |x| < 2^e and T <= 83, as sign and 128-bit magnitude (hi, lo), from the
// bits of x.  For a normal x the shift T - e + E is at most T - 53, so the magnitude stays below 2^84.
__device__ __forceinline__ void parts_w(double x, int er, int T, float (&a)[crtw::kParts]) {
  unsigned long long hi = 0, lo = 0;
  bool neg = false;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (er > -1000 && !(eb == 0 && m == 0)) {
    int E;
    if (eb == 0) {
      E = -1074;
    } else {
      m |= 1ull << 52;
      E = eb - 1075;
    }
    const int sh = E - er + T;
    unsigned __int128 F;
    if (sh >= 0)
      F = (unsigned __int128)m << (sh < 74 ? sh : 74);
    else if (sh > -63)
      F = (unsigned __int128)((m + (1ull << (-sh - 1))) >> (-sh));
    else
      F = 0;
    hi = (unsigned long long)(F >> 64);
    lo = (unsigned long long)F;
    neg = (bits >> 63) != 0;
  }
  crtw::parts(hi, lo, neg, a);
}

template <int I>
__device__ __forceinline__ void wres_pair(const float (&p0)[crtw::kParts], const float (&p1)[crtw::kParts], int nmod,
                                          uint16_t* o, size_t stride) {
  if constexpr (I < crtw::kMax) {
    if (I < nmod) {
      const float r0 = crtw::residue_f(p0, crtw::modulus(I)), r1 = crtw::residue_f(p1, crtw::modulus(I));
      *reinterpret_cast<unsigned*>(o + (size_t)I * stride) =
          __byte_perm(__float_as_uint(r0), __float_as_uint(r1), 0x7632);
      wres_pair<I + 1>(p0, p1, nmod, o, stride);
    }
  }
}

template <int I>
__device__ __forceinline__ void wres_one(const float (&p0)[crtw::kParts], int nmod, uint16_t* o, size_t stride) {
  if constexpr (I < crtw::kMax) {
    if (I < nmod) {
      o[(size_t)I * stride] = (uint16_t)(__float_as_uint(crtw::residue_f(p0, crtw::modulus(I))) >> 16);
      wres_one<I + 1>(p0, nmod, o, stride);
    }
  }
}

// Residues of the rows of X: one block of 256 threads per row, exponent pass then residue pass.
__global__ void __launch_bounds__(256) k_ozmw_rowres(const double* __restrict__ X, int n, int ld, int* __restrict__ e,
                                                     int T, int nmod, uint16_t* __restrict__ out, int ld16, int Rp) {
  __shared__ unsigned long long red[8];
  const int row = blockIdx.x;
  const int tid = threadIdx.x;
  const double* xr = X + (size_t)row * ld;
  unsigned long long m = 0ull;  // the row's largest magnitude, as a bit pattern (integer pipes)
  for (int c = tid; c < n; c += 256) m = max_bits(m, abs_bits(xr[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = max_bits(m, red[w]);
  const int er = m ? exp_of_bits(m) : -2000000000;
  if (tid == 0) e[row] = er;
  const size_t stride = (size_t)Rp * ld16;
  uint16_t* orow = out + (size_t)row * ld16;
  const int npair = n / 2;
  for (int c = tid; c < npair; c += 256) {
    float p0[crtw::kParts], p1[crtw::kParts];
    parts_w(xr[2 * c], er, T, p0);
    parts_w(xr[2 * c + 1], er, T, p1);
    wres_pair<0>(p0, p1, nmod, orow + 2 * c, stride);
  }
  if ((n & 1) && tid == 0) {
    float p0[crtw::kParts];
    parts_w(xr[n - 1], er, T, p0);
    wres_one<0>(p0, nmod, orow + (n - 1), stride);
  }
}

// Residues of X^T (operand rows = columns of X; exponents from launch_oz_exp(cols = true)), through a
// 64 x 32 shared-memory tile as k_ozmod.cu's transposed kernel.
__global__ void k_ozmw_tres(const double* __restrict__ X, int n, int ld, const int* __restrict__ e, int T, int nmod,
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
    float p0[crtw::kParts], p1[crtw::kParts];
    parts_w(te[tx][r], er, T, p0);
    parts_w(to[tx][r], er, T, p1);
    uint16_t* o = out + (size_t)row * ld16 + col;
    if (col + 1 < n)
      wres_pair<0>(p0, p1, nmod, o, stride);
    else
      wres_one<0>(p0, nmod, o, stride);
  }
}

// Grouped forms (the batched mode's final residuals; layouts as k_ozmod.cu's k_gozm_rowres / k_gozm_tres).
__global__ void __launch_bounds__(256) k_gozmw_rowres(const GroupRes g, int nmod, uint16_t* __restrict__ out,
                                                      int ld16, size_t plane) {
  __shared__ unsigned long long red[8];
  const int inst = blockIdx.y, n = g.n[inst], row = blockIdx.x;
  if (row >= n) return;
  const int r0 = g.row0[inst], T = g.T[inst], tid = threadIdx.x;
  const double* xr = g.src ? g.src[inst] + (size_t)row * n : g.packed + (size_t)(r0 + row) * g.ldp;
  unsigned long long m = 0ull;
  for (int c = tid; c < n; c += 256) m = max_bits(m, abs_bits(xr[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = max_bits(m, red[w]);
  const int er = m ? exp_of_bits(m) : -2000000000;
  if (tid == 0) g.e[r0 + row] = er;
  uint16_t* orow = out + (size_t)(r0 + row) * ld16;
  const int ncols = (n + 63) & ~63;
  for (int j = 2 * tid; j < ncols; j += 512) {
    float p0[crtw::kParts], p1[crtw::kParts];
    parts_w(j < n ? xr[j] : 0.0, er, T, p0);
    parts_w(j + 1 < n ? xr[j + 1] : 0.0, er, T, p1);
    wres_pair<0>(p0, p1, nmod, orow + j, plane);
  }
}

__global__ void k_gozmw_tres(const GroupRes g, int nmod, uint16_t* __restrict__ out, int ld16, size_t plane) {
  __shared__ double te[32][33], to[32][33];
  const int inst = blockIdx.z, n = g.n[inst];
  const int bi = blockIdx.y * 64, bj = blockIdx.x * 32;
  const int ncols = (n + 63) & ~63;
  if (bj >= n || bi >= ncols) return;  // the whole block (uniform)
  const int r0 = g.row0[inst], T = g.T[inst];
  const double* X = g.src[inst];
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int rr = ty; rr < 64; rr += 8) {
    const int i = bi + rr, j = bj + tx;
    const double x = (i < n && j < n) ? X[(size_t)i * n + j] : 0.0;
    if (rr & 1)
      to[rr >> 1][tx] = x;
    else
      te[rr >> 1][tx] = x;
  }
  __syncthreads();
  const int col = bi + 2 * tx;
  for (int r = ty; r < 32; r += 8) {
    const int row = bj + r;
    if (row >= n) continue;
    const int er = g.e[r0 + row];
    float p0[crtw::kParts], p1[crtw::kParts];
    parts_w(te[tx][r], er, T, p0);
    parts_w(to[tx][r], er, T, p1);
    wres_pair<0>(p0, p1, nmod, out + (size_t)(r0 + row) * ld16 + col, plane);
  }
}

}  // namespace

cudaError_t launch_ozmw_residues(const double* X, int n, int ld, bool trans, int* e, int T, int nmod, uint16_t* out,
                                 int ld16, int Rp, cudaStream_t s) {
  if (nmod < 1 || nmod > crtw::kMax || T < 1 || T > 83) return cudaErrorInvalidValue;
  // padding rows n..Rp-1 of every plane read as zero: one strided memset over all of them
  if (Rp > n)
    cudaMemset2DAsync(out + (size_t)n * ld16, sizeof(uint16_t) * (size_t)Rp * ld16, 0,
                      sizeof(uint16_t) * (size_t)(Rp - n) * ld16, nmod, s);
  if (trans) {
    dim3 grid((n + 31) / 32, (n + 63) / 64), block(32, 8);
    k_ozmw_tres<<<grid, block, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
  } else {
    k_ozmw_rowres<<<n, 256, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
  }
  return cudaGetLastError();
}

cudaError_t launch_gozmw_rowres(const GroupRes& g, int nmod, uint16_t* out, int ld16, size_t plane, cudaStream_t s) {
  if (nmod < 1 || nmod > crtw::kMax || g.count < 1) return cudaErrorInvalidValue;
  k_gozmw_rowres<<<dim3(g.max_n, g.count), 256, 0, s>>>(g, nmod, out, ld16, plane);
  return cudaGetLastError();
}

cudaError_t launch_gozmw_tres(const GroupRes& g, int nmod, uint16_t* out, int ld16, size_t plane, cudaStream_t s) {
  if (nmod < 1 || nmod > crtw::kMax || g.count < 1 || !g.src) return cudaErrorInvalidValue;
  const dim3 grid((g.max_n + 31) / 32, (g.max_n + 63) / 64, g.count), block(32, 8);
  k_gozmw_tres<<<grid, block, 0, s>>>(g, nmod, out, ld16, plane);
  return cudaGetLastError();
}

}  // namespace zf

// FP64-accurate products on the BF16 tensor cores by modular arithmetic (Ozaki scheme II:
// Ozaki, Uchino, Imamura, "Ozaki Scheme II: A GEMM-oriented emulation of floating-point matrix
// multiplication using an integer modular technique", 2025).
//
// Every row r of an FP64 operand is scaled by 2^(T - e_r) (e_r: the row's exponent bound) and
// rounded to an integer F with |F| <= 2^T.  The product C' = F_A F_B^T of two such integer
// matrices is exact and bounded by K 2^(T_A + T_B).  It is formed modulo pairwise coprime
// moduli m_i <= 256: residues of F within 128 of zero (one FP32 reduction) are exact in BF16, a residue
// product over K <= 1024 terms stays an integer of at most 2^24 (exact in the FP32 accumulator;
// longer products are reduced modulo m_i every 1024 terms inside the product's epilogue), and
// the Chinese remainder theorem recovers C' from its residues once M = prod m_i > 4 |C'|.  The
// result is C_ij = 2^(eA_i + eB_j - T_A - T_B) C'_ij: the only errors are the two roundings to
// T-bit fixed point and the final conversion to FP64.  The moduli count grows linearly with the
// bits kept (about 7.9 bits per product), where slicing grows quadratically (s(s+1)/2 pairs).
#include <math.h>

#include "crt_wide.h"
#include "kernels.h"

namespace zf {

namespace {

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
// crt_residue_f), each pair packed as two BF16 into one 4-byte store (an integer |r| <= 128
// has its low 16 FP32 bits zero, so the BF16 value is the upper half).
template <int I, int NP>
__device__ __forceinline__ void residues_pair_all(const float (&p0)[5], const float (&p1)[5], int nmod, uint16_t* o,
                                                  size_t stride) {
  if constexpr (I < kCrtMax) {
    if (I < nmod) {
      const float r0 = crt_residue_f<NP>(p0, crt_modulus(I)), r1 = crt_residue_f<NP>(p1, crt_modulus(I));
      *reinterpret_cast<unsigned*>(o + (size_t)I * stride) =
          __byte_perm(__float_as_uint(r0), __float_as_uint(r1), 0x7632);
      residues_pair_all<I + 1, NP>(p0, p1, nmod, o, stride);
    }
  }
}

template <int I, int NP>
__device__ __forceinline__ void residues_one_all(const float (&p0)[5], int nmod, uint16_t* o, size_t stride) {
  if constexpr (I < kCrtMax) {
    if (I < nmod) {
      o[(size_t)I * stride] = (uint16_t)(__float_as_uint(crt_residue_f<NP>(p0, crt_modulus(I))) >> 16);
      residues_one_all<I + 1, NP>(p0, nmod, o, stride);
    }
  }
}

__device__ __forceinline__ void parts_of(double x, int er, int T, float (&p)[5]) {
  crt_parts(er > -1000 ? fixed_point_m(x, er, T) : 0, p);
}

// Residues of the rows of X (operand rows = rows of X): one block of NT threads per row finds
// the row's exponent and writes the nmod residue planes, two elements per 4-byte store.  With
// PAIRS > 0 the row stays in registers (n <= 2 NT PAIRS); PAIRS = 0 reads it twice.
template <int NT, int PAIRS, int NP>
__global__ void __launch_bounds__(NT) k_ozm_rowres(const double* __restrict__ X, int n, int ld, int* __restrict__ e,
                                                  int T, int nmod, uint16_t* __restrict__ out, int ld16, int Rp) {
  __shared__ unsigned long long red[NT / 32];
  const int row = blockIdx.x;
  const int tid = threadIdx.x;
  const double* xr = X + (size_t)row * ld;
  const int npair = n / 2;
  constexpr int NREG = PAIRS > 0 ? PAIRS : 1;
  double v0[NREG], v1[NREG];
  unsigned long long m = 0ull;  // the row's largest magnitude, as a bit pattern (integer pipes)
  if (PAIRS > 0) {
#pragma unroll
    for (int k = 0; k < NREG; ++k) {
      const int c = tid + NT * k;
      v0[k] = c < npair ? xr[2 * c] : 0.0;
      v1[k] = c < npair ? xr[2 * c + 1] : 0.0;
      m = max_bits(m, max_bits(abs_bits(v0[k]), abs_bits(v1[k])));
    }
  } else {
    for (int c = tid; c < n; c += NT) m = max_bits(m, abs_bits(xr[c]));
  }
  if (PAIRS > 0 && (n & 1) && tid == 0) m = max_bits(m, abs_bits(xr[n - 1]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) m = max_bits(m, red[w]);
  const int er = m ? exp_of_bits(m) : -2000000000;
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
      residues_pair_all<0, NP>(p0, p1, nmod, orow + 2 * c, stride);
    }
  } else {
    for (int c = tid; c < npair; c += NT) {
      float p0[5], p1[5];
      parts_of(xr[2 * c], er, T, p0);
      parts_of(xr[2 * c + 1], er, T, p1);
      residues_pair_all<0, NP>(p0, p1, nmod, orow + 2 * c, stride);
    }
  }
  if ((n & 1) && tid == 0) {
    float p0[5];
    parts_of(xr[n - 1], er, T, p0);
    residues_one_all<0, NP>(p0, nmod, orow + (n - 1), stride);
  }
}

// Residues of X^T (operand rows = columns of X; exponents from launch_oz_exp(cols = true)): a
// 64 x 32 tile of X (rows bi.., columns bj..) through shared memory, even and odd rows apart so
// the transposed reads are conflict-free; each thread forms two adjacent operand columns (X rows).
template <int NP>
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
      residues_pair_all<0, NP>(p0, p1, nmod, o, stride);
    else
      residues_one_all<0, NP>(p0, nmod, o, stride);
  }
}

// C' from the CRT digits of the residue products, scaled by 2^(eA_i + eB_j - TA - TB).  Plane
// t * nch + c of G holds, for modulus t and K-chunk c, the byte y = (product mod m_t) w_t mod m_t
// (the tensor-core epilogue kEpiCrt8); the digits of a modulus are summed over its chunks and
// accumulated as sum_t y_t P_t in 32-bit limbs with sum_t y_t / m_t in FP32 (CrtAcc / crtw::Acc).
// Modes: 0 out = C, 1 out += C, 2 (sym) d = I - C with the block's sum of d^2 in partials[block].
// Tiles of 32 rows x 128 columns, blockDim 32 x 8: a thread forms 4 adjacent columns of 4 rows and
// reads one 4-byte word per plane per row (a warp reads 128 consecutive bytes of a plane).  With sym
// only entries j >= i are formed (their digits are the only ones written) and mirrored through
// shared memory.
// One 32 x 128 output tile at (bi, bj) of a reconstruction (the kernels below place it); out may be null
// (mode 2: only the tile's sum of d^2 into *partial_out).
template <class Plan, class Acc, int KMAX>
__device__ __forceinline__ void combine8_tile(const uint8_t* __restrict__ G, size_t gstride, int ld8, int nch,
                                              const Plan& plan, const int* __restrict__ eA,
                                              const int* __restrict__ eB, int TA, int TB, int n,
                                              double* __restrict__ out, int ld64, int mode, int sym,
                                              double* partial_out, int bi, int bj,
                                              unsigned long long* amax_out = nullptr) {
  __shared__ double tile[32][129];
  __shared__ double red[8];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool active = !sym || bj + 127 >= bi;
  const int nmod = plan.nmod;
  double ss_off = 0.0, ss_diag = 0.0;  // sums of d_ij^2 over j > i and j = i
  unsigned long long am = 0ull;         // max |d_ij| (bits of a non-negative double) when amax_out is set
  if (active) {
    const int j0 = bj + 4 * tx;
    int eb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) eb[k] = j0 + k < n ? eB[j0 + k] : -2000000000;
    const size_t tstride = (size_t)nch * gstride;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q, i = bi + r;
      const bool rok = i < n && j0 < n;
      const uint8_t* g = G + (rok ? (size_t)i * ld8 + j0 : 0);
      // per modulus the chunk digits summed in two 16-bit lanes per word (even and odd bytes)
      unsigned ev[KMAX], od[KMAX];
#pragma unroll
      for (int t = 0; t < KMAX; ++t) {
        ev[t] = 0u;
        od[t] = 0u;
      }
      for (int c = 0; c < nch; ++c) {
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
          const unsigned w =
              (rok && t < nmod) ? __ldcs(reinterpret_cast<const unsigned*>(g + (size_t)t * tstride + (size_t)c * gstride))
                                : 0u;
          ev[t] += w & 0x00FF00FFu;
          od[t] += (w >> 8) & 0x00FF00FFu;
        }
      }
      Acc acc[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k].clear();
#pragma unroll
      for (int t = 0; t < KMAX; ++t) {
        if (t < nmod) {
          acc[0].add_y(plan, t, ev[t] & 0xFFFFu);
          acc[1].add_y(plan, t, od[t] & 0xFFFFu);
          acc[2].add_y(plan, t, ev[t] >> 16);
          acc[3].add_y(plan, t, od[t] >> 16);
        }
      }
      const int ea = i < n ? eA[i] : -2000000000;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = j0 + k;
        double v = 0.0;
        if (i < n && j < n) {
          if (ea > -1000 && eb[k] > -1000) v = acc[k].value(plan, ea + eb[k] - TA - TB);
          if (mode == 2) {
            // d = I - C: a sign flip off the diagonal (no FP64 arithmetic), one subtraction on it
            if (i == j) {
              v = 1.0 - v;
              ss_diag = fma(v, v, ss_diag);
            } else {
              v = __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
              if (j > i) ss_off = fma(v, v, ss_off);
            }
            if (amax_out && (!sym || j >= i)) am = max_bits(am, abs_bits(v));
          }
          if (out && (!sym || j >= i)) {
            double* o = out + (size_t)i * ld64 + j;
            if (mode == 1)
              *o += v;
            else
              *o = v;
          }
        }
        tile[r][4 * tx + k] = v;
      }
    }
    if (sym && out) {
      // (i, j) with j > i also goes to (j, i): rows bj.. of the output, columns bi..
      __syncthreads();
      for (int rr = ty; rr < 128; rr += 8) {
        const int oi = bj + rr, oj = bi + tx;
        if (oi < n && oj < n && oi > oj) {
          double* o = out + (size_t)oi * ld64 + oj;
          if (mode == 1)
            *o += tile[tx][rr];
          else
            *o = tile[tx][rr];
        }
      }
    }
  }
  if (mode == 2) {
    double ss = fma(2.0, ss_off, ss_diag);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (tx == 0) red[ty] = ss;
    __syncthreads();
    if (ty == 0 && tx == 0) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += red[w];
      if (partial_out) *partial_out = t;
    }
    if (amax_out) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) am = max_bits(am, __shfl_xor_sync(0xffffffffu, am, o));
      if (tx == 0 && am) atomicMax(amax_out, am);
    }
  }
}

template <class Plan, class Acc, int KMAX>
__global__ void __launch_bounds__(256, KMAX > kCrtMax ? 2 : 3) k_ozm_combine8(const uint8_t* __restrict__ G, size_t gstride, int ld8,
                                                         int nch, const __grid_constant__ Plan plan,
                                                         const int* __restrict__ eA, const int* __restrict__ eB, int TA,
                                                         int TB, int n, double* __restrict__ out, int ld64, int mode,
                                                         int sym, double* __restrict__ partials,
                                                         unsigned long long* amax) {
  combine8_tile<Plan, Acc, KMAX>(G, gstride, ld8, nch, plan, eA, eB, TA, TB, n, out, ld64, mode, sym,
                                 partials ? partials + blockIdx.y * gridDim.x + blockIdx.x : nullptr, blockIdx.y * 32,
                                 blockIdx.x * 128, amax);
}

// Every instance of a group (grid.z): its digits, exponents and output rows start at its packed row.
template <class Plan, class Acc, int KMAX>
__global__ void __launch_bounds__(256, KMAX > kCrtMax ? 2 : 3) k_gozm_combine8(const uint8_t* __restrict__ G, size_t gstride, int ld8,
                                                          const __grid_constant__ Plan plan, const GroupRes g,
                                                          const int* __restrict__ eA, const int* __restrict__ eB,
                                                          double* __restrict__ out, int ld64, int mode, int sym,
                                                          double* __restrict__ partials) {
  const int inst = blockIdx.z, r0 = g.row0[inst], T = g.T[inst];
  const size_t nb = (size_t)gridDim.x * gridDim.y;
  combine8_tile<Plan, Acc, KMAX>(G + (size_t)r0 * ld8, gstride, ld8, 1, plan, eA + r0, eB + r0, T, T, g.n[inst],
                                 out ? out + (size_t)r0 * ld64 : nullptr, ld64, mode, sym,
                                 partials ? partials + inst * nb + blockIdx.y * gridDim.x + blockIdx.x : nullptr,
                                 blockIdx.y * 32, blockIdx.x * 128);
}

// rho_r^2 = sum_k (x_rk 2^-e_r)^2 of every row r of X (e_r the row's exponent bound, as in the
// residue kernels), and the largest of them as an FP32 bit pattern into *rho2 (atomic maximum:
// non-negative floats order like their bit patterns).  A row holding a NaN or Inf, or whose
// largest entry is subnormal, writes +Inf (no bound).
// One block of 256 threads per row; the sum runs in FP32 (its error is bounded by the caller).
__global__ void __launch_bounds__(256) k_ozm_rowrho(const double* __restrict__ X, int n, int ld,
                                                    unsigned int* __restrict__ rho2) {
  __shared__ unsigned long long redm[8];
  __shared__ float reds[8];
  const double* xr = X + (size_t)blockIdx.x * ld;
  const int tid = threadIdx.x;
  unsigned long long m = 0ull;
  for (int c = tid; c < n; c += 256) m = max_bits(m, abs_bits(xr[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) redm[tid >> 5] = m;
  __syncthreads();
  m = redm[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = max_bits(m, redm[w]);
  if (m == 0ull) return;
  if (m >= 0x7FF0000000000000ull || m < (1ull << 52)) {
    // NaN or Inf, or a row of subnormals (their scaled values would all read as zero): no bound
    if (tid == 0) atomicMax(rho2, 0x7F800000u);
    return;
  }
  const int e = exp_of_bits(m);
  float acc = 0.0f;
  for (int c = tid; c < n; c += 256) {
    const float f = scaled_mag_f32(abs_bits(xr[c]), e);
    acc = fmaf(f, f, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) reds[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += reds[w];
    atomicMax(rho2, __float_as_uint(t));
  }
}

// ---- grouped forms (the batched mode's final residuals): instance = blockIdx.y (rows) or blockIdx.z (tiles)
template <int NP>
__global__ void __launch_bounds__(256) k_gozm_rowres(const GroupRes g, int nmod, uint16_t* __restrict__ out, int ld16,
                                                     size_t plane) {
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
  const int ncols = (n + 63) & ~63;  // zeros from n up to the K padding the tensor-core loads read
  for (int j = 2 * tid; j < ncols; j += 512) {
    float p0[5], p1[5];
    parts_of(j < n ? xr[j] : 0.0, er, T, p0);
    parts_of(j + 1 < n ? xr[j + 1] : 0.0, er, T, p1);
    residues_pair_all<0, NP>(p0, p1, nmod, orow + j, plane);
  }
}

template <int NP>
__global__ void k_gozm_tres(const GroupRes g, int nmod, uint16_t* __restrict__ out, int ld16, size_t plane) {
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
  const int col = bi + 2 * tx;  // < ncols: bi + 63 < ncols since both are multiples of 64
  for (int r = ty; r < 32; r += 8) {
    const int row = bj + r;
    if (row >= n) continue;
    const int er = g.e[r0 + row];
    float p0[5], p1[5];
    parts_of(te[tx][r], er, T, p0);
    parts_of(to[tx][r], er, T, p1);
    residues_pair_all<0, NP>(p0, p1, nmod, out + (size_t)(r0 + row) * ld16 + col, plane);
  }
}

__global__ void k_gozm_colmax(const GroupRes g, unsigned long long* __restrict__ cmax) {
  __shared__ unsigned long long red[8][33];
  const int inst = blockIdx.z, n = g.n[inst];
  const int j = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 256;
  if (blockIdx.x * 32 >= n || r0 >= n) return;  // the whole block (uniform)
  const int r1 = r0 + 256 < n ? r0 + 256 : n;
  const double* Z = g.src[inst];
  unsigned long long m = 0ull;
  if (j < n)
    for (int r = r0 + threadIdx.y; r < r1; r += 8) m = max_bits(m, abs_bits(Z[(size_t)r * n + j]));
  red[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0 && j < n) {
    for (int y = 1; y < 8; ++y) m = max_bits(m, red[y][threadIdx.x]);
    if (m) atomicMax(&cmax[g.row0[inst] + j], m);
  }
}

__global__ void k_gozm_colfin(const GroupRes g, const unsigned long long* __restrict__ cmax) {
  const int inst = blockIdx.y, n = g.n[inst], j = blockIdx.x * 256 + threadIdx.x;
  if (j >= n) return;
  const unsigned long long m = cmax[g.row0[inst] + j];
  g.e[g.row0[inst] + j] = m ? exp_of_bits(m) : -2000000000;
}

// rho2[inst] = max over the instance's packed rows of rho_r^2 (as k_ozm_rowrho).
__global__ void __launch_bounds__(256) k_gozm_rowrho(const GroupRes g, unsigned int* __restrict__ rho2) {
  __shared__ unsigned long long redm[8];
  __shared__ float reds[8];
  const int inst = blockIdx.y, n = g.n[inst], row = blockIdx.x;
  if (row >= n) return;
  const double* xr = g.packed + (size_t)(g.row0[inst] + row) * g.ldp;
  const int tid = threadIdx.x;
  unsigned long long m = 0ull;
  for (int c = tid; c < n; c += 256) m = max_bits(m, abs_bits(xr[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) redm[tid >> 5] = m;
  __syncthreads();
  m = redm[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = max_bits(m, redm[w]);
  if (m == 0ull) return;
  if (m >= 0x7FF0000000000000ull || m < (1ull << 52)) {
    if (tid == 0) atomicMax(&rho2[inst], 0x7F800000u);
    return;
  }
  const int e = exp_of_bits(m);
  float acc = 0.0f;
  for (int c = tid; c < n; c += 256) {
    const float f = scaled_mag_f32(abs_bits(xr[c]), e);
    acc = fmaf(f, f, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) reds[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += reds[w];
    atomicMax(&rho2[inst], __float_as_uint(t));
  }
}

__global__ void k_gozm_finish(const double* __restrict__ partials, int nb, double* __restrict__ err) {
  __shared__ double red[256];
  const double* p = partials + (size_t)blockIdx.x * nb;
  double s = 0.0;
  for (int k = threadIdx.x; k < nb; k += 256) s += p[k];  // fixed order per thread
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) err[blockIdx.x] = sqrt(red[0]);
}

}  // namespace

cudaError_t launch_ozm_residues(const double* X, int n, int ld, bool trans, int* e, int T, int nmod, uint16_t* out,
                                int ld16, int Rp, cudaStream_t s) {
  if (nmod < 1 || nmod > kCrtMax || T < 1 || T > 62) return cudaErrorInvalidValue;
  // padding rows n..Rp-1 of every plane read as zero: one strided memset over all of them
  if (Rp > n)
    cudaMemset2DAsync(out + (size_t)n * ld16, sizeof(uint16_t) * (size_t)Rp * ld16, 0,
                      sizeof(uint16_t) * (size_t)(Rp - n) * ld16, nmod, s);
  // rows of at most 55 bits (|F| < 2^56) need only four 14-bit parts
  const bool four = T <= 55;
  if (trans) {
    dim3 grid((n + 31) / 32, (n + 63) / 64), block(32, 8);
    if (four)
      k_ozm_tres<4><<<grid, block, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
    else
      k_ozm_tres<5><<<grid, block, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
  } else if (n <= 2 * 256 * 8) {
    if (four)
      k_ozm_rowres<256, 8, 4><<<n, 256, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
    else
      k_ozm_rowres<256, 8, 5><<<n, 256, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
  } else {
    if (four)
      k_ozm_rowres<256, 0, 4><<<n, 256, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
    else
      k_ozm_rowres<256, 0, 5><<<n, 256, 0, s>>>(X, n, ld, e, T, nmod, out, ld16, Rp);
  }
  return cudaGetLastError();
}

cudaError_t launch_ozm_rho(const double* X, int n, int ld, bool cols, unsigned int* rho2, void* scratch,
                           cudaStream_t s) {
  if (n < 1) return cudaErrorInvalidValue;
  if (cols) {
    // column exponents land in the scratch too (after the statistics the passes need)
    char* p = static_cast<char*>(scratch);
    return launch_oz_colstats(X, n, ld, reinterpret_cast<int*>(p + oz_colstats_scratch_bytes(n)), rho2, p, s);
  }
  k_ozm_rowrho<<<n, 256, 0, s>>>(X, n, ld, rho2);
  return cudaGetLastError();
}

int ozm_combine_blocks(int n) { return ((n + 127) / 128) * ((n + 31) / 32); }

cudaError_t launch_ozm_combine8(const uint8_t* G, size_t gstride, int ld8, int nch, const CrtPlan& plan, const int* eA,
                                const int* eB, int TA, int TB, int n, double* out, int ld64, int mode, bool sym,
                                double* partials, cudaStream_t s, unsigned long long* amax) {
  if (nch < 1 || nch > kCrtMaxChunks || plan.nmod < 1 || plan.nmod > kCrtMax || (ld8 % 4) != 0)
    return cudaErrorInvalidValue;
  dim3 grid((n + 127) / 128, (n + 31) / 32), block(32, 8);
  k_ozm_combine8<CrtPlan, CrtAcc, kCrtMax><<<grid, block, 0, s>>>(G, gstride, ld8, nch, plan, eA, eB, TA, TB, n, out,
                                                                  ld64, mode, sym ? 1 : 0, partials, amax);
  return cudaGetLastError();
}

cudaError_t launch_ozmw_combine8(const uint8_t* G, size_t gstride, int ld8, int nch, const crtw::Plan& plan,
                                 const int* eA, const int* eB, int TA, int TB, int n, double* out, int ld64, int mode,
                                 bool sym, double* partials, cudaStream_t s, unsigned long long* amax) {
  if (nch < 1 || nch > kCrtMaxChunks || plan.nmod < 1 || plan.nmod > crtw::kMax || (ld8 % 4) != 0)
    return cudaErrorInvalidValue;
  dim3 grid((n + 127) / 128, (n + 31) / 32), block(32, 8);
  k_ozm_combine8<crtw::Plan, crtw::Acc, crtw::kMax><<<grid, block, 0, s>>>(G, gstride, ld8, nch, plan, eA, eB, TA, TB,
                                                                         n, out, ld64, mode, sym ? 1 : 0, partials,
                                                                         amax);
  return cudaGetLastError();
}

cudaError_t launch_gozm_rowres(const GroupRes& g, int nmod, uint16_t* out, int ld16, size_t plane, int maxT,
                               cudaStream_t s) {
  if (nmod < 1 || nmod > kCrtMax || maxT > 62 || g.count < 1) return cudaErrorInvalidValue;
  const dim3 grid(g.max_n, g.count);
  if (maxT <= 55)
    k_gozm_rowres<4><<<grid, 256, 0, s>>>(g, nmod, out, ld16, plane);
  else
    k_gozm_rowres<5><<<grid, 256, 0, s>>>(g, nmod, out, ld16, plane);
  return cudaGetLastError();
}

cudaError_t launch_gozm_tres(const GroupRes& g, int nmod, uint16_t* out, int ld16, size_t plane, int maxT,
                             cudaStream_t s) {
  if (nmod < 1 || nmod > kCrtMax || maxT > 62 || g.count < 1 || !g.src) return cudaErrorInvalidValue;
  const dim3 grid((g.max_n + 31) / 32, (g.max_n + 63) / 64, g.count), block(32, 8);
  if (maxT <= 55)
    k_gozm_tres<4><<<grid, block, 0, s>>>(g, nmod, out, ld16, plane);
  else
    k_gozm_tres<5><<<grid, block, 0, s>>>(g, nmod, out, ld16, plane);
  return cudaGetLastError();
}

cudaError_t launch_gozm_colexp(const GroupRes& g, unsigned long long* scratch, size_t scratch_rows, cudaStream_t s) {
  if (g.count < 1 || !g.src) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * scratch_rows, s);
  if (e != cudaSuccess) return e;
  k_gozm_colmax<<<dim3((g.max_n + 31) / 32, (g.max_n + 255) / 256, g.count), dim3(32, 8), 0, s>>>(g, scratch);
  k_gozm_colfin<<<dim3((g.max_n + 255) / 256, g.count), 256, 0, s>>>(g, scratch);
  return cudaGetLastError();
}

cudaError_t launch_gozm_rowrho(const GroupRes& g, unsigned int* rho2, cudaStream_t s) {
  if (g.count < 1 || !g.packed) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(rho2, 0, sizeof(unsigned int) * (size_t)g.count, s);
  if (e != cudaSuccess) return e;
  k_gozm_rowrho<<<dim3(g.max_n, g.count), 256, 0, s>>>(g, rho2);
  return cudaGetLastError();
}

cudaError_t launch_gozm_combine8(const uint8_t* G, size_t gstride, int ld8, const CrtPlan& plan, const GroupRes& g,
                                 const int* eA, const int* eB, double* out, int ld64, int mode, bool sym,
                                 double* partials, cudaStream_t s) {
  if (plan.nmod < 1 || plan.nmod > kCrtMax || (ld8 % 4) != 0 || g.count < 1) return cudaErrorInvalidValue;
  dim3 grid((g.max_n + 127) / 128, (g.max_n + 31) / 32, g.count), block(32, 8);
  k_gozm_combine8<CrtPlan, CrtAcc, kCrtMax><<<grid, block, 0, s>>>(G, gstride, ld8, plan, g, eA, eB, out, ld64, mode,
                                                                   sym ? 1 : 0, partials);
  return cudaGetLastError();
}

cudaError_t launch_gozmw_combine8(const uint8_t* G, size_t gstride, int ld8, const crtw::Plan& plan,
                                  const GroupRes& g, const int* eA, const int* eB, double* out, int ld64, int mode,
                                  bool sym, double* partials, cudaStream_t s) {
  if (plan.nmod < 1 || plan.nmod > crtw::kMax || (ld8 % 4) != 0 || g.count < 1) return cudaErrorInvalidValue;
  dim3 grid((g.max_n + 127) / 128, (g.max_n + 31) / 32, g.count), block(32, 8);
  k_gozm_combine8<crtw::Plan, crtw::Acc, crtw::kMax><<<grid, block, 0, s>>>(G, gstride, ld8, plan, g, eA, eB, out,
                                                                            ld64, mode, sym ? 1 : 0, partials);
  return cudaGetLastError();
}

cudaError_t launch_gozm_finish(const double* partials, int nb, int count, double* err, cudaStream_t s) {
  if (count < 1 || nb < 1) return cudaErrorInvalidValue;
  k_gozm_finish<<<count, 256, 0, s>>>(partials, nb, err);
  return cudaGetLastError();
}

}  // namespace zf

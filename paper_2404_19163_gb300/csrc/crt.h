// Modular (Chinese remainder) arithmetic of the residue products in k_ozmod.cu, shared by the
// host planner and the device kernels.  Plain C++ outside nvcc, so the arithmetic can be
// checked on the host.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define ZF_HD __host__ __device__
#else
#define ZF_HD
#endif

namespace zf {

constexpr int kCrtMax = 16;        // moduli available; their product is just below 2^125.38
constexpr int kCrtMaxChunks = 4;   // digit planes per reconstruction (K-chunks reduced outside the product)
constexpr int kCrtMaxResidue = 128;  // largest |residue|: K-chunks of 2^24 / 128^2 = 1024 terms stay exact
constexpr int kCrtSubKb = (1 << 24) / (kCrtMaxResidue * kCrtMaxResidue) / 64;  // 64-wide K-blocks per chunk

// Pairwise coprime moduli up to 256, largest first: 2^8, then products of small primes and primes,
// so that the first k carry about 7.9 bits each and all sixteen multiply to about 2^125.38 (below the
// 2^127 the four-limb reconstruction takes).  Residues |r| <= 128 are exact in BF16 (8 significand bits).
ZF_HD constexpr int crt_modulus(int i) {
  switch (i) {
    case 0: return 256;
    case 1: return 255;  // 3 5 17
    case 2: return 253;  // 11 23
    case 3: return 251;
    case 4: return 247;  // 13 19
    case 5: return 241;
    case 6: return 239;
    case 7: return 233;
    case 8: return 229;
    case 9: return 227;
    case 10: return 223;
    case 11: return 217;  // 7 31
    case 12: return 211;
    case 13: return 199;
    case 14: return 197;
    case 15: return 193;
    default: return 1;
  }
}

ZF_HD inline float crt_bits_f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
ZF_HD inline unsigned crt_f_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
#endif
}

// Nearest integer (ties to even) of |x| < 2^22 with two FP32 additions: adding 1.5 * 2^23 leaves
// no fraction bits.
ZF_HD inline float crt_rint(float x) {
  const float C = 12582912.0f;
  return (x + C) - C;
}

ZF_HD inline double crt_bits_d(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}
ZF_HD inline int crt_clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// The integer nearest (ties to even) to |x| < 2^22 with FP32 and integer operations only.
ZF_HD inline int crt_rint_i(float x) { return (int)(crt_f_bits(x + 12582912.0f) - 0x4B400000u); }
// An integer 0 <= y < 2^23 as a float, exactly (the bits of 2^23 + y, minus 2^23).
ZF_HD inline float crt_u2f(unsigned y) { return crt_bits_f(0x4B000000u | y) - 8388608.0f; }

// (neg ? -x : x) 2^sc for the 128-bit magnitude x = hi 2^64 + lo, rounded once to the nearest double
// (ties to even), with integer operations only: GB300's FP64 pipe runs at a small fraction of its
// integer rate, and a reconstruction converts every entry.  Results outside the normal range go
// through ldexp of the exactly representable rounded significand.
ZF_HD inline double crt_to_double(unsigned long long hi, unsigned long long lo, bool neg, int sc) {
  if ((hi | lo) == 0ull) return 0.0;
  const int lz = hi ? crt_clz64(hi) : 64 + crt_clz64(lo);
  unsigned long long t, r;  // the magnitude shifted so that its leading one is bit 63 of t; r the rest
  if (lz >= 64) {
    t = lo << (lz - 64);
    r = 0ull;
  } else if (lz == 0) {
    t = hi;
    r = lo;
  } else {
    t = (hi << lz) | (lo >> (64 - lz));
    r = lo << lz;
  }
  unsigned long long m = t >> 11;  // 53 significant bits
  const bool round_bit = ((t >> 10) & 1ull) != 0ull, sticky = ((t & 0x3FFull) | r) != 0ull;
  if (round_bit && (sticky || (m & 1ull))) ++m;
  int e = 127 - lz + sc;  // value = m 2^(e - 52)
  if (m >> 53) {
    m >>= 1;
    ++e;
  }
  const int be = e + 1023;
  if (be <= 0 || be >= 2047) {
    const double v = ldexp((double)m, e - 52);
    return neg ? -v : v;
  }
  return crt_bits_d(((unsigned long long)neg << 63) | ((unsigned long long)be << 52) | (m & ((1ull << 52) - 1ull)));
}

// 2^e mod m in symmetric form (|c| <= m/2).
ZF_HD constexpr int crt_pow2_sym(int m, int e) {
  int r = 1 % m;
  for (int i = 0; i < e; ++i) r = (2 * r) % m;
  return 2 * r > m ? r - m : r;
}

// The five 14-bit parts of a fixed-point value F (|F| <= 2^62), signed, as floats:
// F = sum_k a_k 2^(14k), |a_k| < 2^14.
ZF_HD inline void crt_parts(long long F, float (&a)[5]) {
  const unsigned long long u = F < 0 ? 0ull - (unsigned long long)F : (unsigned long long)F;
  const float sg = F < 0 ? -1.0f : 1.0f;
  // a 14-bit integer v as a float: the bits of 2^23 + v, minus 2^23
  for (int k = 0; k < 5; ++k)
    a[k] = sg * (crt_bits_f(0x4B000000u | (unsigned)((u >> (14 * k)) & 0x3FFFu)) - 8388608.0f);
}

// Residue of F modulo m from its first NP parts (NP = 4 when |F| < 2^56), in FP32: x = sum_k a_k
// (2^(14k) mod m), with |a_k| < 2^14 and the symmetric |2^(14k) mod m| <= m/2, is an integer with
// |x / m| < 5 2^13, below 2^24 (exact).  r = x - m rint(x / m) is congruent to F; the FP32 quotient
// (1/m and the product each rounded once) errs by at most |x / m| 2^-23 < 0.0049, so rint is at most one
// step from the nearest integer and |r| <= m (1/2 + 0.0049) < 128.8 for m <= 255, |r| <= 128; for
// m = 256 the quotient is exact and |r| <= 128 too.  (Not always the symmetric residue, but within the
// bound the residue products need.)
template <int NP = 5>
ZF_HD inline float crt_residue_f(const float (&a)[5], int m) {
  const float fm = (float)m;
  float x = fmaf(a[3], (float)crt_pow2_sym(m, 42),
                 fmaf(a[2], (float)crt_pow2_sym(m, 28), fmaf(a[1], (float)crt_pow2_sym(m, 14), a[0])));
  if (NP > 4) x = fmaf(a[4], (float)crt_pow2_sym(m, 56), x);
  return fmaf(-fm, crt_rint(x * (1.0f / fm)), x);
}

// x mod m for an integer-valued float |x| <= 2^24 and m >= 13, inv = FP32(1 / m): congruent, and
// within 0.66 m of 0.  The FP32 quotient x * inv carries a relative error of at most 2^-23 (inv and
// the product each rounded once), so it is off by at most 2^24 / 13 * 2^-23 = 0.154 from x / m (well
// inside crt_rint's range); rint is then at most one step from the nearest integer, |x - m rint| <=
// m (1/2 + 0.154), and the fma is exact because that difference is an integer below 2^24.
ZF_HD inline float crt_fmod_sym(float x, float m, float inv) { return fmaf(-m, crt_rint(x * inv), x); }

// The CRT digit of an exact residue-product sum v (integer-valued float, |v| <= 2^24): y = (v mod m) w
// mod m in [0, m), w = (M / m)^-1 mod m the plan's weight of this modulus.  |v mod m| <= 0.66 m <= 169
// and w < 256, so the product stays an exact integer below 2^16, and its second reduction leaves
// |y| <= 0.66 m, which the shift of negative values by m takes into [0, m).
ZF_HD inline float crt_digit(float v, float m, float inv, float w) {
  float y = crt_fmod_sym(crt_fmod_sym(v, m, inv) * w, m, inv);
  return y < 0.0f ? y + m : y;
}

// Reconstruction constants of the first nmod moduli: M = prod m_i, P_i = M / m_i as four
// 32-bit limbs, w_i = P_i^-1 mod m_i.
struct CrtPlan {
  int nmod;
  int m[kCrtMax];
  int w[kCrtMax];
  float inv[kCrtMax];
  float fm[kCrtMax], fw[kCrtMax];  // m and w as floats
  unsigned P[kCrtMax][4];
  unsigned M[4];
};

// Accumulates sum_i y_i P_i (y_i congruent to (C mod m_i) w_i modulo m_i, y_i < 2^10) per 32-bit limb
// without carries (each limb sum stays below 2^46) and sum_i y_i / m_i in FP32.  That sum equals q + C / M for
// an integer q; with |C| < M / 4 and an FP32 error far below 1/4, q = round(sum) and
// C = sum_i y_i P_i - q M, formed modulo 2^128 (exact, since |C| < 2^125).
struct CrtAcc {
  unsigned long long L[4];
  float S;
  ZF_HD void clear() {
    L[0] = L[1] = L[2] = L[3] = 0ull;
    S = 0.0f;
  }
  // Adds a sum y of CRT digits of modulus t (one per digit plane, each in [0, m_t), so y < 2^10).  The
  // digits need no reduction: any y congruent to (C mod m_t) w_t gives sum_t y_t P_t = C (mod M), and
  // sum_t y_t / m_t is still q + C / M for an integer q (below 2^7 here, far from FP32's limits).
  ZF_HD void add_y(const CrtPlan& p, int t, unsigned y) {
    S = fmaf(crt_u2f(y), p.inv[t], S);
    for (int l = 0; l < 4; ++l) L[l] += (unsigned long long)y * p.P[t][l];
  }
  // C 2^sc in FP64, rounded once (crt_to_double).
  ZF_HD double value(const CrtPlan& p, int sc) const {
    const long long q = crt_rint_i(S);
    long long t0 = (long long)L[0] - q * (long long)p.M[0];
    long long t1 = (long long)L[1] - q * (long long)p.M[1] + (t0 >> 32);
    long long t2 = (long long)L[2] - q * (long long)p.M[2] + (t1 >> 32);
    long long t3 = (long long)L[3] - q * (long long)p.M[3] + (t2 >> 32);
    const unsigned l0 = (unsigned)t0, l1 = (unsigned)t1, l2 = (unsigned)t2, l3 = (unsigned)t3;
    unsigned long long hi = ((unsigned long long)l3 << 32) | l2, lo = ((unsigned long long)l1 << 32) | l0;
    const bool neg = (l3 >> 31) != 0u;
    if (neg) {
      lo = ~lo + 1ull;
      hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    return crt_to_double(hi, lo, neg, sc);
  }
};

// The moduli count that makes M = m_0 ... m_{k-1} exceed 2^bits (0 if all sixteen do not), with
// the reconstruction constants.
inline int crt_plan(double bits, CrtPlan* p) {
  unsigned __int128 M = 1;
  int k = 0;
  double lb = 0.0;
  while (k < kCrtMax && lb <= bits) {
    M *= (unsigned)crt_modulus(k);
    lb += log2((double)crt_modulus(k));
    ++k;
  }
  if (lb <= bits) return 0;
  p->nmod = k;
  for (int i = 0; i < kCrtMax; ++i) {
    const unsigned m = i < k ? (unsigned)crt_modulus(i) : 1u;
    p->m[i] = (int)m;
    p->inv[i] = 1.0f / (float)m;
    p->fm[i] = (float)m;
    p->w[i] = 0;
    p->fw[i] = 0.0f;
    for (int l = 0; l < 4; ++l) p->P[i][l] = 0u;
    if (i >= k) continue;
    const unsigned __int128 P = M / m;
    for (int l = 0; l < 4; ++l) p->P[i][l] = (unsigned)(P >> (32 * l));
    const unsigned pm = (unsigned)(P % m);
    for (unsigned x = 1; x < m; ++x)
      if ((pm * x) % m == 1u) {
        p->w[i] = (int)x;
        p->fw[i] = (float)x;
        break;
      }
  }
  for (int l = 0; l < 4; ++l) p->M[l] = (unsigned)(M >> (32 * l));
  return k;
}

}  // namespace zf

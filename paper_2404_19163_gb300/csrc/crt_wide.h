// Wider CRT arithmetic for residue products whose bound passes the sixteen moduli of crt.h:
// up to 24 pairwise coprime moduli (M about 2^184.6) in six 32-bit limbs, and fixed-point rows of
// up to 84 bits as six 14-bit parts.  The first sixteen moduli are crt.h's, in the same order,
// so a plan of at most sixteen moduli is the same plan.  Every modulus is at most 256, so the
// residues, the K-chunk length (1024) and the FP32 reductions are those of crt.h.
//
// Used by the residue kernels of k_ozmod_wide.cu (residues) and k_ozmod.cu (reconstruction); the
// arithmetic is checked on the host against exact big-integer products (tests/test_crt_host.py).
#pragma once
#include "crt.h"

namespace zf {
namespace crtw {

constexpr int kMax = 24;    // moduli
constexpr int kLimbs = 6;   // 32-bit limbs of M and of the digit sums
constexpr int kParts = 6;   // 14-bit parts of a fixed-point row value (|F| <= 2^84)

// crt.h's sixteen moduli, then the next primes below 193 (coprime to all of them).
ZF_HD constexpr int modulus(int i) {
  if (i < kCrtMax) return crt_modulus(i);
  switch (i) {
    case 16: return 191;
    case 17: return 181;
    case 18: return 179;
    case 19: return 173;
    case 20: return 167;
    case 21: return 163;
    case 22: return 157;
    case 23: return 151;
    default: return 1;
  }
}

// CRT digit weight of modulus t in the plan of the first k moduli: w_t = (M / m_t)^-1 mod m_t,
// M = m_0 ... m_{k-1}, the value plan() stores in w[t] (checked against it on the host), formed
// from small products only.
ZF_HD inline int digit_weight(int t, int k) {
  const int m = modulus(t);
  int p = 1 % m;
  for (int s = 0; s < k; ++s)
    if (s != t) p = (p * (modulus(s) % m)) % m;
  for (int x = 1; x < m; ++x)
    if ((p * x) % m == 1) return x;
  return 0;
}

// The six signed 14-bit parts of F (|F| <= 2^84), as floats: F = sum_k a_k 2^(14k).
ZF_HD inline void parts(unsigned long long mag_hi, unsigned long long mag_lo, bool neg, float (&a)[kParts]) {
  const float sg = neg ? -1.0f : 1.0f;
  for (int k = 0; k < kParts; ++k) {
    const int sh = 14 * k;
    unsigned long long v;
    if (sh + 14 <= 64)
      v = mag_lo >> sh;
    else if (sh >= 64)
      v = mag_hi >> (sh - 64);
    else
      v = (mag_lo >> sh) | (mag_hi << (64 - sh));
    a[k] = sg * (crt_bits_f(0x4B000000u | (unsigned)(v & 0x3FFFu)) - 8388608.0f);
  }
}

// Residue of F modulo m from its six parts: x = sum_k a_k (2^(14k) mod m) has |x / m| < 6 2^13, below
// 2^24 (exact in FP32); crt_residue_f's one reduction then errs by less than 0.0059 in the quotient, so
// |r| <= m (1/2 + 0.0059) < 129 for m <= 255, |r| <= 128 (m = 256: exact quotient).
ZF_HD inline float residue_f(const float (&a)[kParts], int m) {
  const float fm = (float)m;
  float x = a[kParts - 1] * (float)crt_pow2_sym(m, 14 * (kParts - 1));
  for (int k = kParts - 2; k >= 1; --k) x = fmaf(a[k], (float)crt_pow2_sym(m, 14 * k), x);
  x += a[0];
  return fmaf(-fm, crt_rint(x * (1.0f / fm)), x);
}

struct Plan {
  int nmod;
  int m[kMax];
  int w[kMax];
  float inv[kMax], fm[kMax], fw[kMax];
  unsigned P[kMax][kLimbs];
  unsigned M[kLimbs];
};

// sum_t y_t P_t per 32-bit limb (each limb sum below 2^47) and sum_t y_t / m_t in FP32 (error far
// below 1/4 for 24 terms); C = sum_t y_t P_t - q M modulo 2^192, exact while |C| < M / 4 < 2^183.
struct Acc {
  unsigned long long L[kLimbs];
  float S;
  ZF_HD void clear() {
    for (int l = 0; l < kLimbs; ++l) L[l] = 0ull;
    S = 0.0f;
  }
  // A sum y of CRT digits of modulus t (see CrtAcc::add_y): below 2^10, so every limb sum stays
  // below 2^47 over 24 moduli.
  ZF_HD void add_y(const Plan& p, int t, unsigned y) {
    S = fmaf(crt_u2f(y), p.inv[t], S);
    for (int l = 0; l < kLimbs; ++l) L[l] += (unsigned long long)y * p.P[t][l];
  }
  // C 2^sc in FP64, rounded once.  With a non-zero top word the magnitude is at least 2^128, so its
  // 53 leading bits lie in the top two words and the lowest word only decides the sticky bit (folded
  // into the lowest bit of the middle word, far below the rounding position).
  ZF_HD double value(const Plan& p, int sc) const {
    const long long q = crt_rint_i(S);
    unsigned l[kLimbs];
    long long carry = 0;
    for (int k = 0; k < kLimbs; ++k) {
      const long long t = (long long)L[k] - q * (long long)p.M[k] + carry;
      l[k] = (unsigned)t;
      carry = t >> 32;
    }
    unsigned long long w0 = ((unsigned long long)l[1] << 32) | l[0], w1 = ((unsigned long long)l[3] << 32) | l[2],
                       w2 = ((unsigned long long)l[5] << 32) | l[4];
    const bool neg = (l[5] >> 31) != 0u;
    if (neg) {
      w0 = ~w0 + 1ull;
      const unsigned long long c1 = w0 == 0ull ? 1ull : 0ull;
      w1 = ~w1 + c1;
      const unsigned long long c2 = (c1 && w1 == 0ull) ? 1ull : 0ull;
      w2 = ~w2 + c2;
    }
    if (w2 != 0ull) return crt_to_double(w2, w1 | (w0 != 0ull ? 1ull : 0ull), neg, 64 + sc);
    return crt_to_double(w1, w0, neg, sc);
  }
};

// The moduli count that makes M exceed 2^bits (0 if all 24 do not), with the constants.  M and
// M / m_i are formed in 32-bit limbs (products and quotients by small integers only).
inline int plan(double bits, Plan* p) {
  unsigned M[kLimbs + 1] = {1u};
  int k = 0;
  double lb = 0.0;
  while (k < kMax && lb <= bits) {
    const unsigned m = (unsigned)modulus(k);
    unsigned long long c = 0;
    for (int l = 0; l <= kLimbs; ++l) {
      const unsigned long long t = (unsigned long long)M[l] * m + c;
      M[l] = (unsigned)t;
      c = t >> 32;
    }
    lb += log2((double)m);
    ++k;
  }
  if (lb <= bits || M[kLimbs] != 0u) return 0;
  p->nmod = k;
  for (int l = 0; l < kLimbs; ++l) p->M[l] = M[l];
  for (int i = 0; i < kMax; ++i) {
    const unsigned m = i < k ? (unsigned)modulus(i) : 1u;
    p->m[i] = (int)m;
    p->inv[i] = 1.0f / (float)m;
    p->fm[i] = (float)m;
    p->w[i] = 0;
    p->fw[i] = 0.0f;
    for (int l = 0; l < kLimbs; ++l) p->P[i][l] = 0u;
    if (i >= k) continue;
    // P = M / m from the top limb down; the remainder of M / m is 0, and P mod m follows from P's limbs
    unsigned long long rem = 0;
    for (int l = kLimbs - 1; l >= 0; --l) {
      const unsigned long long cur = (rem << 32) | M[l];
      p->P[i][l] = (unsigned)(cur / m);
      rem = cur % m;
    }
    unsigned long long pm = 0;
    for (int l = kLimbs - 1; l >= 0; --l) pm = ((pm << 32) | p->P[i][l]) % m;
    for (unsigned x = 1; x < m; ++x)
      if ((pm * x) % m == 1u) {
        p->w[i] = (int)x;
        p->fw[i] = (float)x;
        break;
      }
  }
  return k;
}

}  // namespace crtw
}  // namespace zf

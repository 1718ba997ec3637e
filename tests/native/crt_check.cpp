// Host check of the CRT arithmetic of the residue products (paper_2404_19163_gb300/csrc/crt.h)
// against exact 128-bit integer products: residues, exact chunked residue dot products (K-chunks of
// 1024 terms, each sum reduced modulo m and the reductions summed, as the tensor-core epilogue does),
// and the reconstruction, including the extreme bound N 2^(2T) where the moduli are used up.
#include <math.h>
#include <stdio.h>

#include <random>
#include <vector>

#include "../../paper_2404_19163_gb300/csrc/crt_wide.h"

using namespace zf;

// Integer reference, independent of the FP32 arithmetic under test.
// Symmetric residue of +-a (a < 2^62) modulo m: |r| <= m / 2.
static int ref_sym_residue(unsigned long long a, bool neg, int m) {
  int v = (int)(a % (unsigned long long)m);
  if (2 * v >= m) v -= m;
  return neg ? -v : v;
}
// R mod m in [0, m).
static int ref_mod(long long R, int m) {
  const long long y = R % m;
  return (int)(y < 0 ? y + m : y);
}
// CrtAcc's sums from an exact integer residue R of C: y = (R mod m) w mod m, y P limbs, y / m.
static void ref_add(CrtAcc& acc, const CrtPlan& p, int t, long long R) {
  const int m = p.m[t];
  const int y = ref_mod((long long)ref_mod(R, m) * p.w[t], m);
  acc.S = fmaf((float)y, p.inv[t], acc.S);
  for (int l = 0; l < 4; ++l) acc.L[l] += (unsigned long long)(unsigned)y * p.P[t][l];
}

static double to_double(__int128 x) {
  const bool neg = x < 0;
  const unsigned __int128 a = neg ? -(unsigned __int128)x : (unsigned __int128)x;
  const long double v =
      (long double)(unsigned long long)(a >> 64) * 18446744073709551616.0L + (long double)(unsigned long long)a;
  return (double)(neg ? -v : v);
}

int main() {
  std::mt19937_64 rng(7);
  int fails = 0;
  long cases = 0;
  const int Ts[] = {24, 40, 47, 53, 54};
  const int Ks[] = {1, 2, 64, 1000, 1024, 1025, 4096, 4224, 16384};
  const int chunk = kCrtSubKb * 64;
  for (int T : Ts)
    for (int K : Ks) {
      CrtPlan p;
      const int k = crt_plan(2.0 * T + log2((double)K) + 2.0, &p);
      if (!k) {
        printf("no plan for T=%d K=%d\n", T, K);
        return 1;
      }
      for (int mode = 0; mode < 4; ++mode) {
        std::vector<long long> a(K), b(K);
        const long long lim = 1ll << T;
        for (int l = 0; l < K; ++l) {
          if (mode == 0) {
            a[l] = (long long)(rng() % (2 * (unsigned long long)lim + 1)) - lim;
            b[l] = (long long)(rng() % (2 * (unsigned long long)lim + 1)) - lim;
          } else if (mode == 1) {  // the largest positive product
            a[l] = lim;
            b[l] = lim;
          } else if (mode == 2) {  // the largest negative product
            a[l] = lim;
            b[l] = -lim;
          } else {  // -1
            a[l] = l == 0 ? -1 : 0;
            b[l] = l == 0 ? 1 : 0;
          }
        }
        __int128 exact = 0;
        for (int l = 0; l < K; ++l) exact += (__int128)a[l] * b[l];
        // two reconstructions: the integer reference (exact residues and reductions), and the FP32
        // path of the kernels (crt_residue_f, the epilogue's per-chunk reduction crt_fmod_sym and the
        // sum of those reductions, its digit crt_digit, add_y)
        CrtAcc acc, accf;
        acc.clear();
        accf.clear();
        for (int t = 0; t < k; ++t) {
          const int m = p.m[t];
          long long R = 0, Rsum = 0;
          for (int c0 = 0; c0 < K; c0 += chunk) {
            long long part = 0, partf = 0;
            for (int l = c0; l < K && l < c0 + chunk; ++l) {
              const int ra = ref_sym_residue((unsigned long long)(a[l] < 0 ? -a[l] : a[l]), a[l] < 0, m);
              const int rb = ref_sym_residue((unsigned long long)(b[l] < 0 ? -b[l] : b[l]), b[l] < 0, m);
              float pa[5], pb[5];
              crt_parts(a[l], pa);
              crt_parts(b[l], pb);
              const float fa = crt_residue_f(pa, m), fb = crt_residue_f(pb, m);
              if (ra > kCrtMaxResidue || ra < -kCrtMaxResidue || rb > kCrtMaxResidue || rb < -kCrtMaxResidue ||
                  fabsf(fa) > (float)kCrtMaxResidue || fabsf(fb) > (float)kCrtMaxResidue || fa != floorf(fa) ||
                  ((long long)fa - ra) % m != 0 || ((long long)fb - rb) % m != 0) {
                printf("residue wrong or out of range (m=%d: %d %g, %d %g)\n", m, ra, fa, rb, fb);
                return 1;
              }
              part += (long long)ra * rb;
              partf += (long long)fa * (long long)fb;
            }
            if (part > (1ll << 24) || part < -(1ll << 24) || partf > (1ll << 24) || partf < -(1ll << 24)) {
              printf("chunk sum %lld / %lld exceeds 2^24\n", part, partf);
              return 1;
            }
            R += part;
            const float rc = crt_fmod_sym((float)partf, p.fm[t], p.inv[t]);
            if (rc != floorf(rc) || fabsf(rc) > 0.66f * m || ((long long)rc - partf) % m != 0) {
              printf("chunk reduction of %lld mod %d wrong: %g\n", partf, m, rc);
              return 1;
            }
            Rsum += (long long)rc;
          }
          if (Rsum > 32767 || Rsum < -32768) {
            printf("summed chunk reductions %lld leave 16 bits\n", Rsum);
            return 1;
          }
          const float y = crt_digit((float)Rsum, p.fm[t], p.inv[t], p.fw[t]);
          if (y != floorf(y) || y < 0.0f || y >= (float)m ||
              ((long long)y - (long long)ref_mod((long long)ref_mod(Rsum, m) * p.w[t], m)) % m != 0) {
            printf("digit of %lld mod %d wrong: %g\n", Rsum, m, y);
            return 1;
          }
          ref_add(acc, p, t, R);
          accf.add_y(p, t, (unsigned)y);
        }
        const double want = to_double(exact);
        for (const CrtAcc* A : {&acc, &accf}) {
          const double got = A->value(p, 0);
          const double rel = want != 0 ? fabs(got - want) / fabs(want) : fabs(got);
          ++cases;
          if (!(rel <= 2.3e-16)) {
            ++fails;
            printf("FAIL T=%d K=%d mode=%d moduli=%d %s: %.17g vs %.17g\n", T, K, mode, k, A == &acc ? "int" : "fp32",
                   got, want);
          }
        }
      }
    }
  for (int it = 0; it < 400000; ++it) {  // residues are congruent to the value and in range
    long long F = (long long)(rng() >> 1) - (1ll << 62);
    if (it % 4 == 1) F >>= (it / 4) % 62;  // all magnitudes
    const int m = crt_modulus(it % kCrtMax);
    const int r = ref_sym_residue((unsigned long long)(F < 0 ? -F : F), F < 0, m);
    float pa[5];
    crt_parts(F, pa);
    const float rf = crt_residue_f(pa, m);
    if ((F - r) % m != 0 || (F - (long long)rf) % m != 0 || fabsf(rf) > 128.0f || rf != floorf(rf)) {
      printf("residue of %lld mod %d wrong: %d / %g\n", F, m, r, rf);
      return 1;
    }
    // four parts for |F| < 2^56 (rows of up to 55 bits): the same residue
    const long long F4 = F >> 7;
    float p4[5];
    crt_parts(F4, p4);
    const int r4 = ref_sym_residue((unsigned long long)(F4 < 0 ? -F4 : F4), F4 < 0, m);
    const float rf4 = crt_residue_f<4>(p4, m);
    if ((F4 - (long long)rf4) % m != 0 || (F4 - r4) % m != 0 || fabsf(rf4) > 128.0f || rf4 != floorf(rf4)) {
      printf("four-part residue of %lld mod %d wrong: %d / %g\n", F4, m, r4, rf4);
      return 1;
    }
  }
  for (int i = 0; i < crtw::kMax; ++i) {  // crt_fmod_sym over |x| <= 2^24, every modulus
    const int m = crtw::modulus(i);
    const float inv = 1.0f / (float)m;
    for (long long x = -(1ll << 24); x <= (1ll << 24); x += (x > -(1ll << 24) + 5000 && x < (1ll << 24) - 5000) ? 331 : 1) {
      const float r = crt_fmod_sym((float)x, (float)m, inv);
      if (r != floorf(r) || ((long long)r - x) % m != 0 || fabsf(r) > 0.66f * m) {
        printf("crt_fmod_sym(%lld, %d) = %g\n", x, m, r);
        return 1;
      }
    }
  }
  for (int k = 1; k <= kCrtMax; ++k) {  // the device's digit weights are the plan's
    // bits = log2 of the first k - 1 moduli, summed as crt_plan sums them: the plan takes k moduli
    double bits = 0.0;
    for (int t = 0; t < k - 1; ++t) bits += log2((double)crt_modulus(t));
    CrtPlan q;
    if (crt_plan(bits, &q) != k) {
      printf("plan of %d moduli not found\n", k);
      return 1;
    }
    for (int t = 0; t < k; ++t)
      if (crtw::digit_weight(t, k) != q.w[t]) {
        printf("digit weight of modulus %d in a %d-moduli plan: %d vs %d\n", t, k, crtw::digit_weight(t, k), q.w[t]);
        return 1;
      }
  }
  // the tables: pairwise coprime, at most 256, products within the reconstructions' limb counts
  {
    double lb = 0.0;
    for (int i = 0; i < crtw::kMax; ++i) {
      const int mi = crtw::modulus(i);
      if (mi < 2 || mi > 256 || (i < kCrtMax && mi != crt_modulus(i))) {
        printf("modulus %d out of range: %d\n", i, mi);
        return 1;
      }
      for (int j = 0; j < i; ++j) {
        int a = mi, b = crtw::modulus(j);
        while (b) {
          const int t = a % b;
          a = b;
          b = t;
        }
        if (a != 1) {
          printf("moduli %d and %d share the factor %d\n", mi, crtw::modulus(j), a);
          return 1;
        }
      }
      lb += log2((double)mi);
      if (i == kCrtMax - 1 && !(lb < 126.0)) {
        printf("the regular set's product 2^%.2f passes the four-limb reconstruction\n", lb);
        return 1;
      }
    }
    if (!(lb < 190.0)) {
      printf("the wide set's product 2^%.2f passes the six-limb reconstruction\n", lb);
      return 1;
    }
  }
  CrtPlan p;
  if (crt_plan(110.0, &p) != 14 || crt_plan(117.0, &p) != 15 || crt_plan(118.0, &p) != 16 ||
      crt_plan(125.5, &p) != 0) {
    printf("moduli counts wrong\n");
    return 1;
  }
  printf("cases %ld fails %d\n", cases, fails);
  return fails != 0;
}

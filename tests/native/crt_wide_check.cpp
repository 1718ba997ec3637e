// Host check of the wider CRT arithmetic (paper_2404_19163_gb300/csrc/crt_wide.h).  Reads cases
// (T, K, then K pairs of fixed-point values as sign, high and low 64-bit words of the magnitude),
// forms the residue products as the tensor cores would (exact chunk sums of K <= 1024 terms, each
// of at most 2^24, reduced modulo m and summed, then that sum's CRT digit, as the tensor-core
// epilogue does) and prints the
// reconstructed product; the Python side compares it with the exact
// big-integer product.  Also checks every residue against the magnitude modulo m.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "../../paper_2404_19163_gb300/csrc/crt_wide.h"

using namespace zf;

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = fopen(argv[1], "r");
  if (!f) return 2;
  int T, K;
  const int chunk = kCrtSubKb * 64;
  while (fscanf(f, "%d %d", &T, &K) == 2) {
    std::vector<float> pa((size_t)K * crtw::kParts), pb((size_t)K * crtw::kParts);
    std::vector<unsigned __int128> ma(K), mb(K);
    std::vector<int> na(K), nb(K);
    for (int l = 0; l < K; ++l) {
      int sa, sb;
      unsigned long long ah, al, bh, bl;
      if (fscanf(f, "%d %llu %llu %d %llu %llu", &sa, &ah, &al, &sb, &bh, &bl) != 6) return 3;
      float a[crtw::kParts], b[crtw::kParts];
      crtw::parts(ah, al, sa < 0, a);
      crtw::parts(bh, bl, sb < 0, b);
      for (int k = 0; k < crtw::kParts; ++k) {
        pa[(size_t)l * crtw::kParts + k] = a[k];
        pb[(size_t)l * crtw::kParts + k] = b[k];
      }
      ma[l] = ((unsigned __int128)ah << 64) | al;
      mb[l] = ((unsigned __int128)bh << 64) | bl;
      na[l] = sa < 0;
      nb[l] = sb < 0;
    }
    crtw::Plan p;
    const int k = crtw::plan(2.0 * T + log2((double)K) + 2.0, &p);
    if (!k) {
      printf("noplan %d %d\n", T, K);
      continue;
    }
    for (int t = 0; t < k; ++t)  // the device's digit weights are the plan's
      if (crtw::digit_weight(t, k) != p.w[t]) {
        printf("digitweight %d %d\n", t, k);
        return 1;
      }
    crtw::Acc acc;
    acc.clear();
    for (int t = 0; t < k; ++t) {
      const int m = p.m[t];
      long long rsum = 0;
      for (int c0 = 0; c0 < K; c0 += chunk) {
        long long part = 0;
        for (int l = c0; l < K && l < c0 + chunk; ++l) {
          float a[crtw::kParts], b[crtw::kParts];
          for (int q = 0; q < crtw::kParts; ++q) {
            a[q] = pa[(size_t)l * crtw::kParts + q];
            b[q] = pb[(size_t)l * crtw::kParts + q];
          }
          const float ra = crtw::residue_f(a, m), rb = crtw::residue_f(b, m);
          // congruence with the exact value and the symmetric range
          const long long ea = (long long)(ma[l] % (unsigned)m) * (na[l] ? -1 : 1);
          const long long eb = (long long)(mb[l] % (unsigned)m) * (nb[l] ? -1 : 1);
          if ((((long long)ra - ea) % m) != 0 || (((long long)rb - eb) % m) != 0 || fabsf(ra) > 128.0f ||
              fabsf(rb) > 128.0f || ra != floorf(ra) || rb != floorf(rb)) {
            printf("badresidue %d %d %d\n", T, K, m);
            return 1;
          }
          part += (long long)ra * (long long)rb;
        }
        if (part > (1ll << 24) || part < -(1ll << 24)) {
          printf("chunk %lld\n", part);
          return 1;
        }
        // the tensor-core epilogue's reduction of this chunk sum, summed over the chunks
        const float rc = crt_fmod_sym((float)part, p.fm[t], p.inv[t]);
        if (rc != floorf(rc) || fabsf(rc) > 0.66f * m || ((long long)rc - part) % m != 0) {
          printf("reduction %d %d %d\n", T, K, m);
          return 1;
        }
        rsum += (long long)rc;
      }
      // the digit of the summed reductions
      const float y = crt_digit((float)rsum, p.fm[t], p.inv[t], p.fw[t]);
      const long long rm = ((rsum % m) + m) % m;
      if (rsum > 32767 || rsum < -32768 || y != floorf(y) || y < 0.0f || y >= (float)m ||
          ((long long)y - (rm * p.w[t]) % m) % m != 0) {
        printf("digit %d %d %d\n", T, K, m);
        return 1;
      }
      acc.add_y(p, t, (unsigned)y);
    }
    printf("%d %d %d %.17g\n", T, K, k, acc.value(p, 0));
  }
  fclose(f);
  return 0;
}

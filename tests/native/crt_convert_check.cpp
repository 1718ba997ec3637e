// Host check of crt_to_double (paper_2404_19163_gb300/csrc/crt.h): reads lines "sign hi lo sc" and
// prints the bits of the double it returns, for the Python side to compare with the correctly rounded
// value of the exact rational.
#include <stdio.h>
#include <string.h>

#include "../../paper_2404_19163_gb300/csrc/crt.h"

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = fopen(argv[1], "r");
  if (!f) return 2;
  int sg, sc;
  unsigned long long hi, lo;
  while (fscanf(f, "%d %llu %llu %d", &sg, &hi, &lo, &sc) == 4) {
    const double v = zf::crt_to_double(hi, lo, sg < 0, sc);
    unsigned long long b;
    memcpy(&b, &v, 8);
    printf("%llu\n", b);
  }
  fclose(f);
  return 0;
}

// The congruence transform H_perp = Z^T H Z (Sec. 2, Eq. standard_form): with Z^T S Z = I it
// turns the generalized eigenproblem H C = S C e into the standard one H_perp C_perp = C_perp e,
// C = Z C_perp.  Both products reuse the factorization's kernels: FP64 CUDA-core products,
// FP64-accurate products on the BF16 tensor cores (CRT residues or error-free slices), or BF16
// (hi/lo) tensor-core products.
#include <math.h>
#include <string.h>

#include "ctx.h"
#include "kernels.h"
#include "tc_gemm.h"

using namespace zf;

int tc_product_public(zfact_ctx* c, TcArgs& a, const uint16_t* Ah, const uint16_t* Al, const uint16_t* Bh,
                      const uint16_t* Bl, int ld, int bn);

namespace {

// A = H Z (general), then Z^T A on upper-triangle tiles, mirrored.
int f64_congruence(zfact_ctx* c, const double* H, const double* Z, double* out, int n) {
  int st = ZFACT_OK;
  double* A = (double*)ctx_buf(c, "cg.A64", sizeof(double) * (size_t)n * n, &st);
  if (!A) return st;
  const double n2 = (double)n * n, n3 = n2 * n;
  F64Gemm g1{H, Z, A, nullptr, nullptr, 0.0, 1.0, nullptr, n, false, false, false};
  if ((st = ctx_cuda(c, klaunch(c, "f64_gemm.hz", 2 * n3, 24 * n2, 1, [&] { return launch_f64_gemm(g1, c->stream); }),
                     "f64 H*Z")))
    return st;
  F64Gemm g2{Z, A, out, nullptr, nullptr, 0.0, 1.0, nullptr, n, true, true, false};
  return ctx_cuda(c, klaunch(c, "f64_gemm.zta", n3, 24 * n2, 1, [&] { return launch_f64_gemm(g2, c->stream); }),
                  "f64 Z^T*A");
}

// BF16 operands (hi, and lo when split) with FP32 accumulation: A^T = Z^T H stored as 16-bit
// hi/lo, then Z^T A with an FP64 epilogue on upper-triangle tiles.
int bf16_congruence(zfact_ctx* c, const double* H, const double* Z, double* out, int n, bool split) {
  int st = ZFACT_OK;
  const int ld = (n + 63) / 64 * 64;
  const size_t bytes = (size_t)n * ld * sizeof(uint16_t);
  const char* names[6] = {"cg.Zt.h", "cg.Zt.l", "cg.H.h", "cg.H.l", "cg.At.h", "cg.At.l"};
  uint16_t* b[6] = {};
  for (int k = 0; k < 6; ++k) {
    if ((k & 1) && !split) continue;
    b[k] = (uint16_t*)ctx_buf(c, names[k], bytes, &st);
    if (!b[k]) return st;
  }
  uint16_t *Zth = b[0], *Ztl = b[1], *Hh = b[2], *Hl = b[3], *Ath = b[4], *Atl = b[5];
  if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 2, [&] {
                       cudaError_t e = launch_cvt16(Z, n, n, Zth, Ztl, ld, 1.0, nullptr, true, true, c->stream);
                       if (e == cudaSuccess) e = launch_cvt16(H, n, n, Hh, Hl, ld, 1.0, nullptr, false, true, c->stream);
                       return e;
                     }),
                     "16-bit Z^T, H")))
    return st;
  const int bn = n <= 128 ? 128 : 256;
  TcArgs k1;
  memset(&k1, 0, sizeof(k1));
  k1.M = k1.N = k1.K = n;
  k1.bf16 = 1;
  k1.unscale = 1.0f;
  k1.epi = kEpiStore16;
  k1.split_out = split ? 1 : 0;
  k1.o16h = Ath;
  k1.o16l = Atl;
  k1.ld16 = ld;
  if ((st = tc_product_public(c, k1, Zth, Ztl, Hh, Hl, ld, bn))) return st;
  TcArgs k2;
  memset(&k2, 0, sizeof(k2));
  k2.M = k2.N = k2.K = n;
  k2.bf16 = 1;
  k2.unscale = 1.0f;
  k2.epi = kEpiF64;
  k2.sym = 1;
  k2.f64 = out;
  k2.ld64 = n;
  return tc_product_public(c, k2, Zth, Ztl, Ath, Atl, ld, bn);
}

}  // namespace

extern "C" int zfact_congruence(zfact_ctx* c, const double* H, const double* Z, int64_t N, int precision,
                                int refine_mode, double* Hp) {
  if (!c) return ZFACT_ERR_ARG;
  if (!H || !Z || !Hp) return ctx_fail(c, ZFACT_ERR_ARG, "null matrix");
  if (N < 1 || N > 65536) return ctx_fail(c, ZFACT_ERR_ARG, "N out of range");
  if (precision == ZFACT_P_FP64 && refine_mode != ZFACT_R_NATIVE && refine_mode != ZFACT_R_OZAKI)
    return ctx_fail(c, ZFACT_ERR_ARG, "unknown refine mode %d", refine_mode);
  if (precision != ZFACT_P_FP64 && precision != ZFACT_P_BF16 && precision != ZFACT_P_BF16_SPLIT) {
    if (precision == ZFACT_P_FP32 || precision == ZFACT_P_FP16 || precision == ZFACT_P_FP16_SPLIT)
      return ctx_fail(c, ZFACT_ERR_UNSUPPORTED, "congruence: precision %d is not offered (FP64, BF16, BF16_SPLIT)",
                      precision);
    return ctx_fail(c, ZFACT_ERR_ARG, "unknown precision %d", precision);
  }
  cudaSetDevice(c->device);
  const int n = (int)N;
  const size_t bytes = sizeof(double) * (size_t)n * n;
  int st = ZFACT_OK;
  c->launches = 0;
  cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
  // host operands are staged through the context's workspace
  const double* Hd = H;
  if (!is_device_ptr(H)) {
    double* w = (double*)ctx_buf(c, "cg.Hin", bytes, &st);
    if (!w) return st;
    if ((st = ctx_cuda(c, cudaMemcpyAsync(w, H, bytes, cudaMemcpyHostToDevice, c->stream), "copy H"))) return st;
    Hd = w;
  }
  const double* Zd = Z;
  if (!is_device_ptr(Z)) {
    double* w = (double*)ctx_buf(c, "cg.Zin", bytes, &st);
    if (!w) return st;
    if ((st = ctx_cuda(c, cudaMemcpyAsync(w, Z, bytes, cudaMemcpyHostToDevice, c->stream), "copy Z"))) return st;
    Zd = w;
  }
  double* out = Hp;
  const bool host_out = !is_device_ptr(Hp);
  if (host_out) {
    out = (double*)ctx_buf(c, "cg.out", bytes, &st);
    if (!out) return st;
  }
  // non-finite inputs are reported, not passed on: the FP64-accurate scheme's row scaling would turn
  // a NaN into a finite fixed-point value
  if ((st = ctx_cuda(c, launch_amax_f64(Hd, n, c->st_dev, 3, c->stream), "amax H"))) return st;
  if ((st = ctx_cuda(c, launch_amax_f64(Zd, n, c->st_dev, 2, c->stream), "amax Z"))) return st;
  if ((st = ctx_read_state(c))) return st;
  if (!isfinite(c->st_host->amax[3]) || !isfinite(c->st_host->amax[2]))
    return ctx_fail(c, ZFACT_ERR_NONFINITE, "H or Z holds a NaN or Inf");
  if (precision == ZFACT_P_FP64)
    st = refine_mode == ZFACT_R_OZAKI ? oz_congruence(c, Hd, Zd, out, n) : f64_congruence(c, Hd, Zd, out, n);
  else
    st = bf16_congruence(c, Hd, Zd, out, n, precision == ZFACT_P_BF16_SPLIT);
  if (st) return st;
  if (host_out &&
      (st = ctx_cuda(c, cudaMemcpyAsync(Hp, out, bytes, cudaMemcpyDeviceToHost, c->stream), "copy H_perp")))
    return st;
  return ctx_read_state(c);
}

// Single steps of the recursion exposed through the C ABI for step-level
// parity tests: a tensor-core product of 16-bit-rounded operands (Sec. 3.2,
// Table I), the hi/lo split of Eq. splitStyle, and d = I - Z^T S Z.
#include <math.h>
#include <string.h>

#include "ctx.h"
#include "kernels.h"
#include "tc_gemm.h"

using namespace zf;

int tc_product_public(zfact_ctx* c, TcArgs& a, const uint16_t* Ah, const uint16_t* Al, const uint16_t* Bh,
                      const uint16_t* Bl, int ld, int bn);

extern "C" int zfact_gemm(zfact_ctx* c, int precision, int64_t N, const double* A, double scale_a, const double* B,
                          double scale_b, double* C) {
  if (!c) return ZFACT_ERR_ARG;
  if (!A || !B || !C) return ctx_fail(c, ZFACT_ERR_ARG, "null matrix");
  if (N < 1 || N > 65536) return ctx_fail(c, ZFACT_ERR_ARG, "N out of range");
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C))
    return ctx_fail(c, ZFACT_ERR_ARG, "zfact_gemm takes device pointers");
  if (!(scale_a > 0) || !(scale_b > 0)) return ctx_fail(c, ZFACT_ERR_ARG, "scales must be positive");
  cudaSetDevice(c->device);
  const int n = (int)N;
  int st = ZFACT_OK;
  cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
  if (precision == ZFACT_P_FP64) {
    F64Gemm g{A, B, C, nullptr, nullptr, 0.0, 1.0, nullptr, n, false, false, false};
    if ((st = ctx_cuda(c, launch_f64_gemm(g, c->stream), "f64 gemm"))) return st;
    return ctx_read_state(c);
  }
  if (precision == ZFACT_P_FP32) {
    // FP32 operands (rounded to nearest), FP32 CUDA-core product, FP64 result
    float* A32 = (float*)ctx_buf(c, "g.A32", sizeof(float) * (size_t)n * n, &st);
    if (!A32) return st;
    float* B32 = (float*)ctx_buf(c, "g.B32", sizeof(float) * (size_t)n * n, &st);
    if (!B32) return st;
    float* C32 = (float*)ctx_buf(c, "g.C32", sizeof(float) * (size_t)n * n, &st);
    if (!C32) return st;
    if ((st = ctx_cuda(c, launch_f64_to_f32(A, n, n, A32, n, c->stream), "A32"))) return st;
    if ((st = ctx_cuda(c, launch_f64_to_f32(B, n, n, B32, n, c->stream), "B32"))) return st;
    F32Gemm g{A32, B32, C32, nullptr, nullptr, 0.0, 1.0, nullptr, n, false, false, false};
    if ((st = ctx_cuda(c, launch_f32_gemm(g, c->stream), "f32 gemm"))) return st;
    if ((st = ctx_cuda(c, launch_f32_to_f64(C32, n, n, C, n, c->stream), "C64"))) return st;
    return ctx_read_state(c);
  }
  const bool bf16 = (precision == ZFACT_P_BF16 || precision == ZFACT_P_BF16_SPLIT);
  const bool split = (precision == ZFACT_P_FP16_SPLIT || precision == ZFACT_P_BF16_SPLIT);
  const bool half = precision == ZFACT_P_FP16_HALF;
  if (!bf16 && !half && precision != ZFACT_P_FP16 && precision != ZFACT_P_FP16_SPLIT)
    return ctx_fail(c, ZFACT_ERR_ARG, "unknown precision %d", precision);
  const int ld = (n + 63) / 64 * 64;
  const size_t bytes = (size_t)n * ld * sizeof(uint16_t);
  uint16_t* Ah = (uint16_t*)ctx_buf(c, "g.Ah", bytes, &st);
  if (!Ah) return st;
  uint16_t* Bh = (uint16_t*)ctx_buf(c, "g.Bh", bytes, &st);
  if (!Bh) return st;
  uint16_t *Al = nullptr, *Bl = nullptr;
  if (split) {
    Al = (uint16_t*)ctx_buf(c, "g.Al", bytes, &st);
    if (!Al) return st;
    Bl = (uint16_t*)ctx_buf(c, "g.Bl", bytes, &st);
    if (!Bl) return st;
  }
  if ((st = ctx_cuda(c, launch_cvt16(A, n, n, Ah, Al, ld, scale_a, nullptr, false, bf16, c->stream), "A16")))
    return st;
  // the right factor is read as B^T (row-major N x K)
  if ((st = ctx_cuda(c, launch_cvt16(B, n, n, Bh, Bl, ld, scale_b, nullptr, true, bf16, c->stream), "B16")))
    return st;
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.M = a.N = a.K = n;
  a.bf16 = bf16;
  a.acc16 = half ? 1 : 0;
  a.epi = kEpiF64;
  a.unscale = (float)(1.0 / (scale_a * scale_b));
  a.f64 = C;
  a.ld64 = n;
  const int bn = n <= 128 ? 128 : 256;
  if ((st = tc_product_public(c, a, Ah, Al, Bh, Bl, ld, bn))) return st;
  return ctx_read_state(c);
}

extern "C" int zfact_split(zfact_ctx* c, int precision, const double* A, int64_t n, double scale, uint16_t* hi,
                           uint16_t* lo) {
  if (!c) return ZFACT_ERR_ARG;
  if (!A || !hi || !lo || n < 0) return ctx_fail(c, ZFACT_ERR_ARG, "bad arguments");
  if (n == 0) return ZFACT_OK;
  const bool bf16 = (precision == ZFACT_P_BF16 || precision == ZFACT_P_BF16_SPLIT);
  if (!bf16 && precision != ZFACT_P_FP16 && precision != ZFACT_P_FP16_SPLIT && precision != ZFACT_P_FP16_HALF)
    return ctx_fail(c, ZFACT_ERR_ARG, "split needs a 16-bit precision");
  cudaSetDevice(c->device);
  int st = ctx_cuda(c, launch_split_flat(A, n, scale, hi, lo, bf16, c->stream), "split");
  if (st) return st;
  return ctx_cuda(c, cudaStreamSynchronize(c->stream), "split sync");
}

extern "C" int zfact_residual(zfact_ctx* c, int mode, const double* S, const double* Z, int64_t N, double* D,
                              double* err) {
  if (!c) return ZFACT_ERR_ARG;
  if (!S || !Z || !err) return ctx_fail(c, ZFACT_ERR_ARG, "null argument");
  if (N < 1 || N > 65536) return ctx_fail(c, ZFACT_ERR_ARG, "N out of range");
  if (mode != ZFACT_R_NATIVE && mode != ZFACT_R_OZAKI)
    return ctx_fail(c, ZFACT_ERR_ARG, "unknown refine mode %d", mode);
  cudaSetDevice(c->device);
  const int n = (int)N;
  int st = ZFACT_OK;
  double* A64 = (double*)ctx_buf(c, "A64", sizeof(double) * (size_t)n * n, &st);
  if (!A64) return st;
  double* Dw = D;
  if (!Dw) {
    Dw = (double*)ctx_buf(c, "D64", sizeof(double) * (size_t)n * n, &st);
    if (!Dw) return st;
  }
  cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
  if (mode == ZFACT_R_OZAKI) {
    // slice count from the dynamic range of Z and S, as in the refinement
    if ((st = ctx_cuda(c, launch_gershgorin(S, n, c->st_dev, c->stream), "gershgorin"))) return st;
    if ((st = ctx_cuda(c, launch_amax_f64(Z, n, c->st_dev, 2, c->stream), "amax Z"))) return st;
    // scaled row norms of S's rows and Z's columns: the moduli of the residue products
    void* cs = ctx_buf(c, "oz.colstats", oz_colstats_scratch_bytes(n) + sizeof(int) * (size_t)n, &st);
    if (!cs) return st;
    if ((st = ctx_cuda(c, launch_ozm_rho(S, n, n, false, &c->st_dev->rho2[0], nullptr, c->stream), "rho S"))) return st;
    if ((st = ctx_cuda(c, launch_ozm_rho(Z, n, n, true, &c->st_dev->rho2[1], cs, c->stream), "rho Z"))) return st;
    if ((st = ctx_read_state(c))) return st;
    // the fixed-point scaling takes row maxima, which would pass a NaN or Inf by as a finite value
    if (!isfinite(c->st_host->amax[0]) || !isfinite(c->st_host->amax[2]))
      return ctx_fail(c, ZFACT_ERR_NONFINITE, "S or Z holds a NaN or Inf");
    if ((st = oz_prepare_S(c, S, n, oz_slices_for(c->st_host->amax[2], c->st_host->amax[0]),
                           oz_rho_from(c->st_host->rho2[0], n))))
      return st;
    if ((st = oz_residual(c, Z, Dw, n, 0, 0, 0.0, 0, oz_rho_from(c->st_host->rho2[1], n)))) return st;
  } else if ((st = f64_residual(c, S, Z, A64, Dw, n, 0, 0, 0.0, 0))) {
    return st;
  }
  if ((st = ctx_read_state(c))) return st;
  *err = c->st_host->hist[0];
  if (!isfinite(*err)) return ctx_fail(c, ZFACT_ERR_NONFINITE, "the residual is not finite");
  return ZFACT_OK;
}

// The paper's "single" scheme (Table I): every product of the recursion in FP32 on the CUDA
// cores (GB300: ~70 TFLOP/s), with the same fused epilogues as the FP64 path, Algorithm 2's
// stop, and (when requested) Algorithm 3's refinement with FP64-accurate sliced products.
#include <math.h>

#include <utility>

#include "ctx.h"
#include "kernels.h"

using namespace zf;

int single_refine(zfact_ctx* c, const double* S, double* Za64, int n, int order, const zfact_opts& o, int* iters_out,
                  int* ridx_out, zfact_info* inf) {
  int st = ZFACT_OK;
  const size_t nn = (size_t)n * n;
  float* S32 = (float*)ctx_buf(c, "s.S", sizeof(float) * nn, &st);
  if (!S32) return st;
  float* Za = (float*)ctx_buf(c, "s.Za", sizeof(float) * nn, &st);
  if (!Za) return st;
  float* Zb = (float*)ctx_buf(c, "s.Zb", sizeof(float) * nn, &st);
  if (!Zb) return st;
  float* A = (float*)ctx_buf(c, "s.A", sizeof(float) * nn, &st);
  if (!A) return st;
  float* D = (float*)ctx_buf(c, "s.D", sizeof(float) * nn, &st);
  if (!D) return st;
  float* Q = (float*)ctx_buf(c, "s.Q", sizeof(float) * nn, &st);
  if (!Q) return st;
  float *P = nullptr, *P2 = nullptr;
  if (order > 2) {
    P = (float*)ctx_buf(c, "s.P", sizeof(float) * nn, &st);
    if (!P) return st;
    P2 = (float*)ctx_buf(c, "s.P2", sizeof(float) * nn, &st);
    if (!P2) return st;
  }
  const int nb = f64_num_blocks(n, true, true);
  double* partials = (double*)ctx_buf(c, "partials", sizeof(double) * (size_t)(nb + 1024), &st);
  if (!partials) return st;
  const double n2 = (double)n * n, n3 = n2 * n;
  auto elem = [&](const char* w, auto&& f) { return ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, f), w); };
  if ((st = elem("S32", [&] { return launch_f64_to_f32(S, n, n, S32, n, c->stream); }))) return st;
  if ((st = elem("Z32", [&] { return launch_f64_to_f32(Za64, n, n, Za, n, c->stream); }))) return st;
  double coef[8];
  coef[0] = 1.0;
  for (int k = 1; k <= order; ++k) coef[k] = coef[k - 1] * (2.0 * k - 1.0) / (2.0 * k);

  auto residual = [&](const float* Z, int idx, int check_stop) -> int {
    int s2;
    F32Gemm g1{S32, Z, A, nullptr, nullptr, 0.0, 1.0, nullptr, n, false, false, false};
    if ((s2 = ctx_cuda(c, klaunch(c, "f32_gemm.sz", 2 * n3, 12 * n2, 1, [&] { return launch_f32_gemm(g1, c->stream); }),
                       "f32 S*Z")))
      return s2;
    F32Gemm g2{Z, A, D, nullptr, nullptr, 0.0, 1.0, partials, n, true, true, true};
    if ((s2 = ctx_cuda(c, klaunch(c, "f32_gemm.resid", n3, 12 * n2, 1,
                                  [&] { return launch_f32_gemm(g2, c->stream); }),
                       "f32 residual")))
      return s2;
    return ctx_cuda(c, klaunch(c, "finish_err", 0, 0, 1, [&] {
                      return launch_finish_err(partials, nb, c->st_dev, idx, o.stop_rule, o.tol, n, check_stop,
                                               c->stream);
                    }),
                    "finish err");
  };
  auto poly = [&]() -> int {
    int s2;
    F32Gemm g{D, D, Q, D, order > 2 ? P : nullptr, coef[1], coef[2], nullptr, n, false, true, false};
    if ((s2 = ctx_cuda(c, klaunch(c, "f32_gemm.poly", n3, 12 * n2, 1, [&] { return launch_f32_gemm(g, c->stream); }),
                       "f32 poly")))
      return s2;
    float *Pa = P, *Pb = P2;
    for (int k = 3; k <= order; ++k) {
      F32Gemm gk{Pa, D, Q, Q, k < order ? Pb : nullptr, 1.0, coef[k], nullptr, n, false, true, false};
      if ((s2 = ctx_cuda(c, klaunch(c, "f32_gemm.poly", n3, 16 * n2, 1,
                                    [&] { return launch_f32_gemm(gk, c->stream); }),
                         "f32 poly chain")))
        return s2;
      std::swap(Pa, Pb);
    }
    return ZFACT_OK;
  };

  float* Zc = Za;
  float* Zn = Zb;
  if ((st = residual(Zc, 0, 0))) return st;
  if ((st = ctx_read_state(c))) return st;
  const double err0 = c->st_host->hist[0];
  if (!(err0 < 1.0)) inf->warn = ZFACT_WARN_NONCONTRACTIVE;
  bool done = c->st_host->nonfinite || (o.fixed_iters <= 0 && o.stop_rule == 1 && err0 / sqrt((double)n) <= o.tol);
  const int limit = o.fixed_iters > 0 ? o.fixed_iters : o.nmax;
  int iters = 0;
  while (!done && iters < limit && iters + 1 + o.refine_steps + 1 < kHistMax) {
    if ((st = poly())) return st;
    F32Gemm gu{Zc, Q, Zn, Zc, nullptr, 1.0, 1.0, nullptr, n, false, false, false};
    if ((st = ctx_cuda(c, klaunch(c, "f32_gemm.update", 2 * n3, 12 * n2, 1,
                                  [&] { return launch_f32_gemm(gu, c->stream); }),
                       "f32 update")))
      return st;
    std::swap(Zc, Zn);
    ++iters;
    if ((st = residual(Zc, iters, o.fixed_iters <= 0 ? 1 : 0))) return st;
    if ((st = ctx_read_state(c))) return st;
    done = c->st_host->nonfinite || c->st_host->stop;
  }
  *iters_out = iters;
  if ((st = elem("Z to FP64", [&] { return launch_f32_to_f64(Zc, n, n, Za64, n, c->stream); }))) return st;
  c->mixed_result = Za64;
  if (c->st_host->nonfinite || (o.refine_steps <= 0 && !o.final_residual)) {
    *ridx_out = 0;
    return ZFACT_OK;
  }
  return refine_ozaki(c, S, Za64, n, order, o, iters, ridx_out, inf);
}

// Algorithm 3's refinement in single precision (Table I "(h)(h)+refi" with its FP32 step): up to
// refine_steps updates of the bulk's Z with d, Q and Z + Z Q formed by FP32 CUDA-core products
// (their Err, FP32-accurate, goes to the history), then the FP64-accurate residual of the result.
int refine_fp32(zfact_ctx* c, const double* S, double* Z64, int n, int order, const zfact_opts& o, int iters,
                int* ridx_out, zfact_info* inf) {
  int st = ZFACT_OK;
  const size_t nn = (size_t)n * n;
  const char* names[6] = {"r32.S", "r32.Za", "r32.Zb", "r32.A", "r32.D", "r32.Q"};
  float* b[6];
  for (int k = 0; k < 6; ++k) {
    b[k] = (float*)ctx_buf(c, names[k], sizeof(float) * nn, &st);
    if (!b[k]) return st;
  }
  float *S32 = b[0], *Zc = b[1], *Zn = b[2], *A = b[3], *D = b[4], *Q = b[5];
  float *P = nullptr, *P2 = nullptr;
  if (order > 2) {
    P = (float*)ctx_buf(c, "r32.P", sizeof(float) * nn, &st);
    if (!P) return st;
    P2 = (float*)ctx_buf(c, "r32.P2", sizeof(float) * nn, &st);
    if (!P2) return st;
  }
  const int nb = f64_num_blocks(n, true, true);
  double* partials = (double*)ctx_buf(c, "partials", sizeof(double) * (size_t)(nb + 1024), &st);
  if (!partials) return st;
  const double n2 = (double)n * n, n3 = n2 * n;
  double coef[8];
  coef[0] = 1.0;
  for (int k = 1; k <= order; ++k) coef[k] = coef[k - 1] * (2.0 * k - 1.0) / (2.0 * k);
  auto elem = [&](const char* w, auto&& f) { return ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, f), w); };
  if ((st = elem("S32", [&] { return launch_f64_to_f32(S, n, n, S32, n, c->stream); }))) return st;
  if ((st = elem("Z32", [&] { return launch_f64_to_f32(Z64, n, n, Zc, n, c->stream); }))) return st;
  int idx = iters, ridx = 0;
  for (int r = 0; r < o.refine_steps && idx + 2 < kHistMax; ++r) {
    ++idx;
    F32Gemm g1{S32, Zc, A, nullptr, nullptr, 0.0, 1.0, nullptr, n, false, false, false};
    F32Gemm g2{Zc, A, D, nullptr, nullptr, 0.0, 1.0, partials, n, true, true, true};
    if ((st = ctx_cuda(c, klaunch(c, "f32_gemm.sz", 2 * n3, 12 * n2, 1, [&] { return launch_f32_gemm(g1, c->stream); }),
                       "f32 S*Z")))
      return st;
    if ((st = ctx_cuda(c, klaunch(c, "f32_gemm.resid", n3, 12 * n2, 1, [&] { return launch_f32_gemm(g2, c->stream); }),
                       "f32 residual")))
      return st;
    if ((st = ctx_cuda(c, klaunch(c, "finish_err", 0, 0, 1, [&] {
                         return launch_finish_err(partials, nb, c->st_dev, idx, o.stop_rule, o.tol, n, 0, c->stream);
                       }),
                       "finish err")))
      return st;
    if ((st = ctx_read_state(c))) return st;
    if (c->st_host->nonfinite) break;
    if (o.tol > 0 && c->st_host->hist[idx] / sqrt((double)n) <= o.tol) break;
    F32Gemm gp{D, D, Q, D, order > 2 ? P : nullptr, coef[1], coef[2], nullptr, n, false, true, false};
    if ((st = ctx_cuda(c, klaunch(c, "f32_gemm.poly", n3, 12 * n2, 1, [&] { return launch_f32_gemm(gp, c->stream); }),
                       "f32 poly")))
      return st;
    float *Pa = P, *Pb = P2;
    for (int k = 3; k <= order; ++k) {
      F32Gemm gk{Pa, D, Q, Q, k < order ? Pb : nullptr, 1.0, coef[k], nullptr, n, false, true, false};
      if ((st = ctx_cuda(c, klaunch(c, "f32_gemm.poly", n3, 16 * n2, 1, [&] { return launch_f32_gemm(gk, c->stream); }),
                         "f32 poly chain")))
        return st;
      std::swap(Pa, Pb);
    }
    F32Gemm gu{Zc, Q, Zn, Zc, nullptr, 1.0, 1.0, nullptr, n, false, false, false};
    if ((st = ctx_cuda(c, klaunch(c, "f32_gemm.update", 2 * n3, 12 * n2, 1, [&] { return launch_f32_gemm(gu, c->stream); }),
                       "f32 update")))
      return st;
    std::swap(Zc, Zn);
    ++ridx;
  }
  *ridx_out = ridx;
  if (ridx > 0 && (st = elem("Z to FP64", [&] { return launch_f32_to_f64(Zc, n, n, Z64, n, c->stream); }))) return st;
  if (!o.final_residual || c->st_host->nonfinite) return ZFACT_OK;
  // the FP64-accurate residual of the returned Z, after the FP32 entries of the history
  zfact_opts of = o;
  of.refine_steps = 0;
  int unused = 0;
  return refine_ozaki(c, S, Z64, n, order, of, idx, &unused, inf);
}

// C-ABI entry points of the learned start proposal: features, MLP training steps
// (forward / backward / Adam) and zfact_propose with its fallback to the plain schedule.
#include <math.h>
#include <string.h>

#include "ctx.h"
#include "kernels.h"
#include "mlp.h"
#include "tc_gemm.h"

using namespace zf;

int tc_product_public(zfact_ctx* c, TcArgs& a, const uint16_t* Ah, const uint16_t* Al, const uint16_t* Bh,
                      const uint16_t* Bl, int ld, int bn);

// 16 features of S into the device array f (see include/zfact.h); st receives the row statistics.
static int features_device(zfact_ctx* c, const double* S, int n, float* f, double** st_out) {
  int st = ZFACT_OK;
  const size_t nn = (size_t)n * n;
  double* rows = (double*)ctx_buf(c, "f.rows", sizeof(double) * 3 * (size_t)n, &st);
  if (!rows) return st;
  double* rst = (double*)ctx_buf(c, "f.st", sizeof(double) * 8, &st);
  if (!rst) return st;
  double* D0 = (double*)ctx_buf(c, "f.D0", sizeof(double) * nn, &st);
  if (!D0) return st;
  double* P = (double*)ctx_buf(c, "f.P", sizeof(double) * nn, &st);
  if (!P) return st;
  double* part = (double*)ctx_buf(c, "f.part", sizeof(double) * 4 * (size_t)feat_trace_blocks(n), &st);
  if (!part) return st;
  const int ld = (n + 63) / 64 * 64;
  uint16_t* Dh = (uint16_t*)ctx_buf(c, "f.Dh", sizeof(uint16_t) * (size_t)n * ld, &st);
  if (!Dh) return st;
  uint16_t* Dl = (uint16_t*)ctx_buf(c, "f.Dl", sizeof(uint16_t) * (size_t)n * ld, &st);
  if (!Dl) return st;
  IterState* sd = c->st_dev;
  if ((st = ctx_cuda(c, klaunch(c, "features", 0, 8.0 * nn, 6, [&] {
                       cudaError_t e = launch_feat_rows(S, n, rows, rst, c->stream);
                       if (e == cudaSuccess) e = launch_feat_d0(S, n, rst, D0, c->stream);
                       if (e == cudaSuccess) e = launch_amax_f64(D0, n, sd, 7, c->stream);
                       if (e == cudaSuccess) e = launch_pow2_slot(sd, 7, 7, 0, c->stream);
                       if (e == cudaSuccess)
                         e = launch_cvt16(D0, n, n, Dh, Dl, ld, 1.0, &sd->scale[7], false, false, c->stream);
                       return e;
                     }),
                     "features")))
    return st;
  // E^2 (E = d0 - t1 I) by an FP16 hi/lo product on symmetric tiles (FP64 output)
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.M = a.N = a.K = n;
  a.epi = kEpiF64;
  a.sym = 1;
  a.bf16 = 0;
  a.unscale = 1.0f;
  a.sa_ptr = &sd->scale[7];
  a.sb_ptr = &sd->scale[7];
  a.f64 = P;
  a.ld64 = n;
  if ((st = tc_product_public(c, a, Dh, Dl, Dh, Dl, ld, n <= 128 ? 128 : 256))) return st;
  if ((st = ctx_cuda(c, klaunch(c, "features", 0, 16.0 * nn, 2,
                                [&] { return launch_feat_traces(D0, P, n, part, rst, f, c->stream); }),
                     "feature traces")))
    return st;
  if (st_out) *st_out = rst;
  return ZFACT_OK;
}

static const double* stage_S(zfact_ctx* c, const double* S, int n, int* st) {
  if (is_device_ptr(S)) return S;
  double* Sd = (double*)ctx_buf(c, "S64", sizeof(double) * (size_t)n * n, st);
  if (!Sd) return nullptr;
  *st = ctx_cuda(c, cudaMemcpyAsync(Sd, S, sizeof(double) * (size_t)n * n, cudaMemcpyHostToDevice, c->stream),
                 "copy S");
  return *st ? nullptr : Sd;
}

extern "C" int zfact_features(zfact_ctx* c, const double* S, int64_t N, float* feat) {
  if (!c) return ZFACT_ERR_ARG;
  if (!S || !feat || N < 2 || N > 65536) return ctx_fail(c, ZFACT_ERR_ARG, "bad arguments");
  cudaSetDevice(c->device);
  int st = ZFACT_OK;
  const int n = (int)N;
  const double* Sd = stage_S(c, S, n, &st);
  if (!Sd) return st;
  float* f = (float*)ctx_buf(c, "f.feat", 64, &st);
  if (!f) return st;
  cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
  if ((st = features_device(c, Sd, n, f, nullptr))) return st;
  if ((st = ctx_cuda(c, cudaMemcpyAsync(feat, f, 16 * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "feat")))
    return st;
  return ctx_read_state(c);
}

extern "C" int zfact_mlp_forward(zfact_ctx* c, const float* params, const float* mean, const float* stdv,
                                 const float* x, int batch, float* y) {
  if (!c) return ZFACT_ERR_ARG;
  if (!params || !mean || !stdv || !x || !y || batch < 1) return ctx_fail(c, ZFACT_ERR_ARG, "bad arguments");
  cudaSetDevice(c->device);
  int st = ctx_cuda(c, klaunch(c, "mlp", 0, 0, 1, [&] {
                      return launch_mlp(params, mean, stdv, x, batch, y, nullptr, nullptr, 0.f, nullptr, nullptr,
                                        c->stream);
                    }),
                    "mlp forward");
  if (st) return st;
  return ctx_cuda(c, cudaStreamSynchronize(c->stream), "mlp sync");
}

extern "C" int zfact_mlp_backward(zfact_ctx* c, const float* params, const float* mean, const float* stdv,
                                  const float* x, const float* target_scale, const int* target_order, int batch,
                                  float w_order, float* grad, double* loss) {
  if (!c) return ZFACT_ERR_ARG;
  if (!params || !mean || !stdv || !x || !target_scale || !target_order || !grad || batch < 1)
    return ctx_fail(c, ZFACT_ERR_ARG, "bad arguments");
  cudaSetDevice(c->device);
  int st = ZFACT_OK;
  const int nc = mlp_chunks(batch);
  float* act = (float*)ctx_buf(c, "mlp.act", sizeof(float) * ((size_t)mlp_act_floats(batch) + (size_t)nc * kMlpParams),
                               &st);
  if (!act) return st;
  float* part = act + mlp_act_floats(batch);
  double* ls = (double*)ctx_buf(c, "mlp.ls", sizeof(double) * ((size_t)batch + nc + 1), &st);
  if (!ls) return st;
  double* lpart = ls + batch;
  double* lmean = lpart + nc;
  if ((st = ctx_cuda(c, klaunch(c, "mlp", 0, 0, 3, [&] {
                       cudaError_t e = launch_mlp(params, mean, stdv, x, batch, nullptr, target_scale, target_order,
                                                  w_order, act, ls, c->stream);
                       if (e == cudaSuccess)
                         e = launch_mlp_reduce(act, batch, part, ls, lpart, grad, lmean, c->stream);
                       return e;
                     }),
                     "mlp backward")))
    return st;
  double l = 0;
  if ((st = ctx_cuda(c, cudaMemcpyAsync(&l, lmean, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "loss")))
    return st;
  if ((st = ctx_cuda(c, cudaStreamSynchronize(c->stream), "mlp sync"))) return st;
  if (loss) *loss = l;
  return ZFACT_OK;
}

extern "C" int zfact_mlp_adam(zfact_ctx* c, float* params, const float* grad, float* m, float* v, int n, int step,
                              float lr, float beta1, float beta2, float eps) {
  if (!c) return ZFACT_ERR_ARG;
  if (!params || !grad || !m || !v || n < 1 || step < 1) return ctx_fail(c, ZFACT_ERR_ARG, "bad arguments");
  cudaSetDevice(c->device);
  int st = ctx_cuda(c, klaunch(c, "adam", 0, 0, 1, [&] {
                      return launch_adam(params, grad, m, v, n, step, lr, beta1, beta2, eps, c->stream);
                    }),
                    "adam");
  if (st) return st;
  return ctx_cuda(c, cudaStreamSynchronize(c->stream), "adam sync");
}

extern "C" int zfact_propose(zfact_ctx* c, const double* S, int64_t N, const float* params, const float* mean,
                             const float* stdv, double* scale, int* order) {
  if (!c) return ZFACT_ERR_ARG;
  if (!S || !scale || !order || N < 2 || N > 65536) return ctx_fail(c, ZFACT_ERR_ARG, "bad arguments");
  cudaSetDevice(c->device);
  int st = ZFACT_OK;
  const int n = (int)N;
  const double* Sd = stage_S(c, S, n, &st);
  if (!Sd) return st;
  float* f = (float*)ctx_buf(c, "f.feat", 64, &st);
  if (!f) return st;
  float* y = (float*)ctx_buf(c, "f.y", 64, &st);
  if (!y) return st;
  double* rst = nullptr;
  cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
  if ((st = features_device(c, Sd, n, f, &rst))) return st;
  const bool have_net = params && mean && stdv;
  if (have_net &&
      (st = ctx_cuda(c, klaunch(c, "mlp", 0, 0, 1, [&] {
                       return launch_mlp(params, mean, stdv, f, 1, y, nullptr, nullptr, 0.f, nullptr, nullptr,
                                         c->stream);
                     }),
                     "propose mlp")))
    return st;
  float yh[5] = {0, 0, 0, 0, 0};
  double g_hi = 0;
  if (have_net) cudaMemcpyAsync(yh, y, sizeof(yh), cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(&g_hi, rst, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if ((st = ctx_read_state(c))) return st;
  // plain schedule: Gershgorin scale, m = 2 (also the fallback)
  const double s0 = 1.0 / sqrt(g_hi);
  double s = s0;
  int m = 2;
  if (have_net) {
    const double cand = s0 * exp((double)yh[0]);
    int best = 0;
    for (int k = 1; k < 4; ++k)
      if (yh[1 + k] > yh[1 + best]) best = k;
    if (isfinite(cand) && cand >= 0.25 * s0 && cand <= 4.0 * s0 && isfinite(yh[1 + best])) {
      s = cand;
      m = 2 + best;
    }
  }
  *scale = s;
  *order = m;
  return ZFACT_OK;
}

// C-ABI entry points of libzfact and the host-side driver of the recursion
// (Sec. 3 Eq. np1; Algorithm 2's stop rule; Algorithm 3's refinement).
// Every arithmetic step runs in this library's kernels; the host only
// sequences launches on the context's stream and reads back the stop flag.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <utility>
#include <stdarg.h>
#include <string>
#include <vector>

#include "ctx.h"
#include "kernels.h"

using namespace zf;

// ----------------------------------------------------------------- context helpers
int ctx_fail(zfact_ctx* c, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof(c->err), fmt, ap);
  va_end(ap);
  return code;
}

int ctx_cuda(zfact_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return ZFACT_OK;
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return ctx_fail(c, ZFACT_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
  return ctx_fail(c, ZFACT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* ctx_buf(zfact_ctx* c, const char* name, size_t bytes, int* status) {
  auto it = c->bufs.find(name);
  if (it != c->bufs.end() && it->second.bytes >= bytes) return it->second.ptr;
  const size_t need = bytes < 256 ? 256 : bytes;
  const size_t held = (it != c->bufs.end()) ? (it->second.bytes < 256 ? 256 : it->second.bytes) : 0;
  if (c->ws_limit && c->ws_bytes - held + need > c->ws_limit) {
    *status = ctx_fail(c, ZFACT_ERR_NOMEM, "%s: workspace limit of %zu bytes reached", name, c->ws_limit);
    return nullptr;
  }
  if (it != c->bufs.end()) {
    c->ws_bytes -= held;
    // the old buffer may still be read by queued work: the context's stream, or the current lane's
    // (lane buffers are private to their lane)
    cudaStreamSynchronize(c->stream);
    if (c->lane >= 0 && c->lane_stream[c->lane]) cudaStreamSynchronize(c->lane_stream[c->lane]);
    cudaFree(it->second.ptr);
    c->bufs.erase(it);
  }
  void* p = nullptr;
  ++c->ws_gen;  // captured loop graphs hold workspace addresses
  cudaError_t e = cudaMalloc(&p, need);
  if (e != cudaSuccess) {
    *status = ctx_cuda(c, e, name);
    return nullptr;
  }
  c->ws_bytes += need;
  c->bufs[name] = DevBuf{p, bytes};
  return p;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int out_copy_start(zfact_ctx* c, const double* Z) {
  if (!c->out_host) return ZFACT_OK;
  if (!c->out_stream && cudaStreamCreateWithFlags(&c->out_stream, cudaStreamNonBlocking) != cudaSuccess)
    return ctx_fail(c, ZFACT_ERR_CUDA, "output stream");
  if (!c->out_ev && cudaEventCreateWithFlags(&c->out_ev, cudaEventDisableTiming) != cudaSuccess)
    return ctx_fail(c, ZFACT_ERR_CUDA, "output event");
  cudaEvent_t e = ev_get(c);
  cudaEventRecord(e, c->stream);
  cudaStreamWaitEvent(c->out_stream, e, 0);
  c->ev_pool.push_back(e);
  int st = ctx_cuda(c, cudaMemcpyAsync(c->out_host, Z, c->out_bytes, cudaMemcpyDeviceToHost, c->out_stream),
                    "early copy of Z");
  if (st) return st;
  cudaEventRecord(c->out_ev, c->out_stream);
  c->out_src = Z;
  return ZFACT_OK;
}

void out_copy_fence(zfact_ctx* c) {
  if (!c->out_src) return;
  cudaStreamWaitEvent(c->stream, c->out_ev, 0);
  c->out_src = nullptr;
}

// ----------------------------------------------------------------- per-kernel accounting
int kstat_id(zfact_ctx* c, const char* name) {
  for (size_t i = 0; i < c->kstats.size(); ++i)
    if (c->kstats[i].name == name) return (int)i;
  KStat k;
  k.name = name;
  c->kstats.push_back(k);
  return (int)c->kstats.size() - 1;
}

void kstat_note(zfact_ctx* c, const char* name, double flops) {
  if (c->profiling) c->kstats[kstat_id(c, name)].flops += flops;
}

cudaEvent_t ev_get(zfact_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void kstats_flush(zfact_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    KStat& k = c->kstats[p.id];
    k.launches += p.count;
    k.ms += ms;
    k.flops += p.flops;
    k.bytes += p.bytes;
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
}

extern "C" int zfact_set_profiling(zfact_ctx* c, int on) {
  if (!c) return ZFACT_ERR_ARG;
  c->profiling = on != 0;
  return ZFACT_OK;
}

extern "C" int zfact_kernel_stats(zfact_ctx* c, zfact_kstat* out, int cap, int* n, int reset) {
  if (!c) return ZFACT_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  kstats_flush(c);
  int cnt = 0;
  for (auto& k : c->kstats) {
    if (out && cnt < cap) {
      memset(&out[cnt], 0, sizeof(zfact_kstat));
      strncpy(out[cnt].name, k.name.c_str(), sizeof(out[cnt].name) - 1);
      out[cnt].launches = k.launches;
      out[cnt].ms = k.ms;
      out[cnt].flops = k.flops;
      out[cnt].bytes = k.bytes;
    }
    ++cnt;
  }
  if (n) *n = cnt;
  if (reset) c->kstats.clear();
  return ZFACT_OK;
}

// ----------------------------------------------------------------- lifecycle
extern "C" void zfact_default_opts(zfact_opts* o) {
  if (!o) return;
  o->nmax = 50;
  o->refine_steps = -1;  // precision-dependent default
  o->refine_mode = -1;   // automatic
  o->stop_rule = 0;
  o->tol = 0.0;
  o->fixed_iters = 0;
  o->final_residual = 1;
  o->tile_cfg = 0;
  o->start_scale = 0.0;
}

extern "C" int zfact_create(zfact_ctx** out, int device, void* stream) {
  if (!out) return ZFACT_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ZFACT_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return ZFACT_ERR_CUDA;
  zfact_ctx* c = new zfact_ctx();
  c->device = device;
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, device);
  c->num_sms = prop.multiProcessorCount;
  c->cc_major = prop.major;
  c->cc_minor = prop.minor;
  if (stream) {
    c->stream = (cudaStream_t)stream;
    c->own_stream = false;
  } else {
    // a blocking stream: its work is ordered after the legacy default stream's, where
    // most callers produce their device inputs
    if (cudaStreamCreate(&c->stream) != cudaSuccess) {
      delete c;
      return ZFACT_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaMalloc(&c->st_dev, sizeof(IterState)) != cudaSuccess ||
      cudaMallocHost(&c->st_host, sizeof(IterState)) != cudaSuccess) {
    delete c;
    return ZFACT_ERR_NOMEM;
  }
  cudaEventCreate(&c->ev0);
  cudaEventCreate(&c->ev1);
  c->err[0] = 0;
  *out = c;
  return ZFACT_OK;
}

extern "C" void zfact_destroy(zfact_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->gr_pinned) cudaFreeHost(c->gr_pinned);
  for (auto& kv : c->loop_graph_cache) cudaGraphExecDestroy(kv.second.exec);
  c->loop_graph_cache.clear();
  for (auto& kv : c->bufs) cudaFree(kv.second.ptr);
  c->bufs.clear();
  kstats_flush(c);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->st_dev) cudaFree(c->st_dev);
  if (c->st_host) cudaFreeHost(c->st_host);
  cudaEventDestroy(c->ev0);
  cudaEventDestroy(c->ev1);
  if (c->out_ev) cudaEventDestroy(c->out_ev);
  if (c->out_stream) cudaStreamDestroy(c->out_stream);
  for (int l = 0; l < zfact_ctx::kLanes; ++l)
    if (c->lane_stream[l]) cudaStreamDestroy(c->lane_stream[l]);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

extern "C" const char* zfact_last_error(zfact_ctx* c) { return c ? c->err : "null context"; }

// ----------------------------------------------------------------- state read-back
int ctx_read_state(zfact_ctx* c) {
  cudaError_t e = cudaMemcpyAsync(c->st_host, c->st_dev, sizeof(IterState), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  int s = ctx_cuda(c, e, "state read-back");
  if (s) return s;
  kstats_flush(c);
  if (c->st_host->error & kErrTimeout)
    return ctx_fail(c, ZFACT_ERR_TIMEOUT, "a bounded device wait gave up (code 0x%x)", c->st_host->error);
  if (c->st_host->error & kErrShape) return ctx_fail(c, ZFACT_ERR_ARG, "kernel shape check failed");
  return ZFACT_OK;
}

// ----------------------------------------------------------------- FP64 building blocks
// d = I - Z^T (S Z); Err -> hist[idx] (and the stop test when check_stop).
int f64_residual(zfact_ctx* c, const double* S, const double* Z, double* A, double* D, int n, int idx,
                 int rule, double tol, int check_stop) {
  int st = ZFACT_OK;
  const int nb = f64_num_blocks(n, true);
  double* partials = (double*)ctx_buf(c, "partials", sizeof(double) * (size_t)(nb + 1024), &st);
  if (!partials) return st;
  const double n2 = (double)n * n, n3 = n2 * n;
  F64Gemm g1{S, Z, A, nullptr, nullptr, 0.0, 1.0, nullptr, n, false, false, false};
  if ((st = ctx_cuda(c, klaunch(c, "f64_gemm.sz", 2 * n3, 24 * n2, 1, [&] { return launch_f64_gemm(g1, c->stream); }),
                     "f64 S*Z")))
    return st;
  F64Gemm g2{Z, A, D, nullptr, nullptr, 0.0, 1.0, partials, n, true, true, true};
  if ((st = ctx_cuda(c, klaunch(c, "f64_gemm.resid", n3, 24 * n2, 1, [&] { return launch_f64_gemm(g2, c->stream); }),
                     "f64 Z^T*A residual")))
    return st;
  return ctx_cuda(c, klaunch(c, "finish_err", 0, 0, 1, [&] {
                    return launch_finish_err(partials, nb, c->st_dev, idx, rule, tol, n, check_stop, c->stream);
                  }),
                  "finish err");
}

// Q = sum_{k=1..m} c_k d^k (powers chain; every product symmetric).
int f64_poly(zfact_ctx* c, const double* D, double* Q, double* P, double* P2, int n, int m) {
  double coef[8];
  coef[0] = 1.0;
  for (int k = 1; k <= m; ++k) coef[k] = coef[k - 1] * (2.0 * k - 1.0) / (2.0 * k);
  int st;
  // P = d*d, Q = c1 d + c2 P
  const double n2 = (double)n * n, n3 = n2 * n;
  F64Gemm g{D, D, Q, D, m > 2 ? P : nullptr, coef[1], coef[2], nullptr, n, false, true, false};
  if ((st = ctx_cuda(c, klaunch(c, "f64_gemm.poly", n3, 24 * n2, 1, [&] { return launch_f64_gemm(g, c->stream); }),
                     "f64 poly")))
    return st;
  for (int k = 3; k <= m; ++k) {
    // P_k = P_{k-1} d ; Q += c_k P_k
    F64Gemm gk{P, D, Q, Q, k < m ? P2 : nullptr, 1.0, coef[k], nullptr, n, false, true, false};
    if ((st = ctx_cuda(c, klaunch(c, "f64_gemm.poly", n3, 32 * n2, 1, [&] { return launch_f64_gemm(gk, c->stream); }),
                       "f64 poly chain")))
      return st;
    double* t = P;
    P = P2;
    P2 = t;
  }
  return ZFACT_OK;
}

// Zn = Z + Z Q
int f64_update(zfact_ctx* c, const double* Z, const double* Q, double* Zn, int n) {
  const double n2 = (double)n * n, n3 = n2 * n;
  F64Gemm g{Z, Q, Zn, Z, nullptr, 1.0, 1.0, nullptr, n, false, false, false};
  return ctx_cuda(c, klaunch(c, "f64_gemm.update", 2 * n3, 24 * n2, 1, [&] { return launch_f64_gemm(g, c->stream); }),
                  "f64 update");
}

// ----------------------------------------------------------------- argument checks
static int check_common(zfact_ctx* c, const double* S, int64_t N, int order, int precision) {
  if (!c) return ZFACT_ERR_ARG;
  if (!S) return ctx_fail(c, ZFACT_ERR_ARG, "S is NULL");
  if (N < 1 || N > 65536) return ctx_fail(c, ZFACT_ERR_ARG, "N=%lld out of range [1, 65536]", (long long)N);
  if (order < 2 || order > 5) return ctx_fail(c, ZFACT_ERR_ARG, "order=%d out of range [2, 5]", order);
  if (precision != ZFACT_P_FP64 && precision != ZFACT_P_FP32 && precision != ZFACT_P_BF16 &&
      precision != ZFACT_P_FP16 && precision != ZFACT_P_FP16_SPLIT && precision != ZFACT_P_BF16_SPLIT &&
      precision != ZFACT_P_FP16_HALF)
    return ctx_fail(c, ZFACT_ERR_ARG, "unknown precision %d", precision);
  if (precision == ZFACT_P_FP16_HALF && N > 32768)
    return ctx_fail(c, ZFACT_ERR_ARG, "an FP16 accumulator takes N <= 32768 (N=%lld)", (long long)N);
  return ZFACT_OK;
}

// ----------------------------------------------------------------- zfact_refine
extern "C" int zfact_refine(zfact_ctx* c, const double* S_in, const double* Z0_in, int64_t N, int order,
                            int precision, const zfact_opts* opts_in, double* Z_out, double* hist, int hist_cap,
                            zfact_info* info) {
  int st = check_common(c, S_in, N, order, precision);
  if (st) return st;
  if (!Z_out) return ctx_fail(c, ZFACT_ERR_ARG, "Z is NULL");
  cudaSetDevice(c->device);
  zfact_opts o;
  zfact_default_opts(&o);
  if (opts_in) o = *opts_in;
  if (o.nmax < 1) o.nmax = 1;
  if (o.refine_steps < 0) o.refine_steps = (precision == ZFACT_P_FP64 || precision == ZFACT_P_FP32) ? 0 : 3;
  if (o.refine_mode < 0) o.refine_mode = ZFACT_R_OZAKI;
  if (o.refine_mode != ZFACT_R_NATIVE && o.refine_mode != ZFACT_R_OZAKI && o.refine_mode != ZFACT_R_FP32)
    return ctx_fail(c, ZFACT_ERR_ARG, "unknown refine mode %d", o.refine_mode);
  const int n = (int)N;
  const size_t nn = (size_t)n * n, bytes = nn * sizeof(double);
  zfact_info inf;
  memset(&inf, 0, sizeof(inf));
  inf.resid_f = NAN;

  c->launches = 0;
  c->ghi_S = nullptr;
  c->zmax_Z = nullptr;
  cudaEventRecord(c->ev0, c->stream);
  // ---- stage inputs (host inputs are copied in; device S is used in place)
  const double* S = S_in;
  if (!is_device_ptr(S_in)) {
    double* Sd = (double*)ctx_buf(c, "S64", bytes, &st);
    if (!Sd) return st;
    if ((st = ctx_cuda(c, cudaMemcpyAsync(Sd, S_in, bytes, cudaMemcpyHostToDevice, c->stream), "copy S")))
      return st;
    S = Sd;
  }
  double* Za = (double*)ctx_buf(c, "Z64a", bytes, &st);
  if (!Za) return st;
  double* Zb = (double*)ctx_buf(c, "Z64b", bytes, &st);
  if (!Zb) return st;
  cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
  if (Z0_in) {
    if ((st = ctx_cuda(c, cudaMemcpyAsync(Za, Z0_in, bytes, cudaMemcpyDefault, c->stream), "copy Z0"))) return st;
  } else {
    if ((st = ctx_cuda(c, klaunch(c, "gershgorin", 2.0 * n * n, 8.0 * n * n, 2,
                                  [&] { return launch_gershgorin(S, n, c->st_dev, c->stream); }),
                       "gershgorin")))
      return st;
    c->ghi_S = S;  // amax[0] holds S's Gershgorin bound for the rest of the call
    if (o.start_scale > 0.0 &&
        (st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1,
                                  [&] { return launch_set_gscale(c->st_dev, o.start_scale, c->stream); }),
                       "start scale")))
      return st;
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 8.0 * n * n, 1,
                                  [&] { return launch_scaled_identity_f64(Za, n, c->st_dev, c->stream); }),
                       "Z0")))
      return st;
  }

  int iters = 0, ridx = 0;
  double* Zcur = Za;
  double* Znext = Zb;
  // whatever happens below, no early copy into the caller's buffer (mixed path) outlives this call
  struct OutGuard {
    zfact_ctx* c;
    ~OutGuard() {
      if (c->out_src) cudaStreamSynchronize(c->out_stream);
      c->out_src = nullptr;
      c->out_host = nullptr;
    }
  } out_guard{c};
  c->out_host = nullptr;
  c->out_src = nullptr;
  if (precision == ZFACT_P_FP64) {
    double* A = (double*)ctx_buf(c, "A64", bytes, &st);
    if (!A) return st;
    double* D = (double*)ctx_buf(c, "D64", bytes, &st);
    if (!D) return st;
    double* Q = (double*)ctx_buf(c, "Q64", bytes, &st);
    if (!Q) return st;
    double *P = nullptr, *P2 = nullptr;
    if (order > 2) {
      P = (double*)ctx_buf(c, "P64", bytes, &st);
      if (!P) return st;
      P2 = (double*)ctx_buf(c, "P64b", bytes, &st);
      if (!P2) return st;
    }
    if ((st = f64_residual(c, S, Zcur, A, D, n, 0, o.stop_rule, o.tol, 0))) return st;
    if ((st = ctx_read_state(c))) return st;
    const double err0 = c->st_host->hist[0];
    if (!(err0 < 1.0)) inf.warn = ZFACT_WARN_NONCONTRACTIVE;
    bool done = c->st_host->nonfinite || (o.fixed_iters <= 0 && o.stop_rule == 1 && err0 / sqrt((double)n) <= o.tol);
    const int limit = o.fixed_iters > 0 ? o.fixed_iters : o.nmax;
    // bulk updates (Algorithm 2; Algorithm 1 with stop_rule 1)
    while (!done && iters < limit && iters + 1 < kHistMax) {
      if ((st = f64_poly(c, D, Q, P, P2, n, order))) return st;
      if ((st = f64_update(c, Zcur, Q, Znext, n))) return st;
      std::swap(Zcur, Znext);
      ++iters;
      if ((st = f64_residual(c, S, Zcur, A, D, n, iters, o.stop_rule, o.tol, o.fixed_iters <= 0 ? 1 : 0)))
        return st;
      if ((st = ctx_read_state(c))) return st;
      done = c->st_host->nonfinite || c->st_host->stop;
    }
    // refinement updates (Algorithm 3); in FP64 these are further plain updates
    for (int r = 0; r < o.refine_steps && !c->st_host->nonfinite && iters + ridx + 1 < kHistMax; ++r) {
      if (o.tol > 0 && c->st_host->hist[iters + ridx] / sqrt((double)n) <= o.tol) break;
      if ((st = f64_poly(c, D, Q, P, P2, n, order))) return st;
      if ((st = f64_update(c, Zcur, Q, Znext, n))) return st;
      std::swap(Zcur, Znext);
      ++ridx;
      if ((st = f64_residual(c, S, Zcur, A, D, n, iters + ridx, o.stop_rule, o.tol, 0))) return st;
      if ((st = ctx_read_state(c))) return st;
    }
    inf.resid_f = c->st_host->hist[c->st_host->hist_len - 1];
  } else if (precision == ZFACT_P_FP32) {
    st = single_refine(c, S, Zcur, n, order, o, &iters, &ridx, &inf);
    if (st) return st;
    Zcur = c->mixed_result;
  } else {
    // a pinned host Z takes the result by an early copy that overlaps the final residual (a pageable
    // one would make that copy block the host, so it is copied at the end as usual)
    cudaPointerAttributes pa;
    const bool pinned = cudaPointerGetAttributes(&pa, Z_out) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    if (!pinned) cudaGetLastError();
    c->out_host = pinned ? (void*)Z_out : nullptr;
    c->out_bytes = bytes;
    st = mixed_refine(c, S, Zcur, Znext, n, order, precision, o, &iters, &ridx, &inf, Z0_in == nullptr);
    if (st == kRetryGershgorin) {
      out_copy_fence(c);  // the retry writes the Z an early copy may be reading
      // the caller's start scale did not contract: the Gershgorin start, as if start_scale were 0
      o.start_scale = 0.0;
      iters = ridx = 0;
      memset(&inf, 0, sizeof(inf));
      inf.resid_f = NAN;
      cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
      if ((st = ctx_cuda(c, klaunch(c, "gershgorin", 2.0 * n * n, 8.0 * n * n, 2,
                                    [&] { return launch_gershgorin(S, n, c->st_dev, c->stream); }),
                         "gershgorin")))
        return st;
      c->ghi_S = S;
      c->zmax_Z = nullptr;
      if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 8.0 * n * n, 1,
                                    [&] { return launch_scaled_identity_f64(Zcur, n, c->st_dev, c->stream); }),
                         "Z0")))
        return st;
      st = mixed_refine(c, S, Zcur, Znext, n, order, precision, o, &iters, &ridx, &inf, true);
    }
    if (st) return st;
    Zcur = c->mixed_result;
  }

  // ---- output (the early copy already holds the final Z when it read this array after its last write)
  if (c->out_src && c->out_src == Zcur) {
    cudaStreamWaitEvent(c->stream, c->out_ev, 0);
  } else {
    out_copy_fence(c);
    if ((st = ctx_cuda(c, cudaMemcpyAsync(Z_out, Zcur, bytes, cudaMemcpyDefault, c->stream), "copy Z out")))
      return st;
  }
  cudaEventRecord(c->ev1, c->stream);
  if ((st = ctx_read_state(c))) return st;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  const int hl = c->st_host->hist_len;
  if (hist)
    for (int i = 0; i < hl && i < hist_cap; ++i) hist[i] = c->st_host->hist[i];
  inf.iters = iters;
  inf.refine_iters = ridx;
  inf.hist_len = hl < hist_cap ? hl : hist_cap;
  inf.ms = ms;
  inf.launches = c->launches;
  if (!(c->st_host->hist[0] < 1.0)) inf.warn = ZFACT_WARN_NONCONTRACTIVE;
  if (info) *info = inf;
  if (c->st_host->nonfinite) return ctx_fail(c, ZFACT_ERR_NONFINITE, "Err became non-finite");
  if (o.tol > 0 && o.final_residual && !(inf.resid_f / sqrt((double)n) <= o.tol))
    return ctx_fail(c, ZFACT_ERR_NOT_CONVERGED, "final residual %.3e > tol %.3e", inf.resid_f / sqrt((double)n),
                    o.tol);
  return inf.warn ? ZFACT_WARN_NONCONTRACTIVE : ZFACT_OK;
}

// ----------------------------------------------------------------- workspace cap and self-test
extern "C" int zfact_set_workspace_limit(zfact_ctx* c, int64_t bytes) {
  if (!c) return ZFACT_ERR_ARG;
  if (bytes < 0) return ctx_fail(c, ZFACT_ERR_ARG, "negative workspace limit");
  c->ws_limit = (size_t)bytes;
  return ZFACT_OK;
}

extern "C" int zfact_set_loop_graphs(zfact_ctx* c, int on) {
  if (!c) return ZFACT_ERR_ARG;
  c->loop_graphs = on != 0;
  return ZFACT_OK;
}

extern "C" int zfact_set_emulation(zfact_ctx* c, int scheme) {
  if (!c) return ZFACT_ERR_ARG;
  if (scheme != ZFACT_EMU_AUTO && scheme != ZFACT_EMU_SLICES && scheme != ZFACT_EMU_WIDE)
    return ctx_fail(c, ZFACT_ERR_ARG, "unknown emulation scheme %d", scheme);
  c->oz_scheme = scheme;
  return ZFACT_OK;
}

namespace {
// One mbarrier that nothing arrives at: the production bounded wait must give up, raise the
// timeout flag and return, leaving the kernel to exit normally.
__global__ void k_selftest_wait(int* err_flag, uint32_t limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, err_flag, 7, limit);
}
}  // namespace

extern "C" int zfact_selftest_timeout(zfact_ctx* c) {
  if (!c) return ZFACT_ERR_ARG;
  cudaSetDevice(c->device);
  cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
  k_selftest_wait<<<1, 32, 0, c->stream>>>(&c->st_dev->error, 1u << 12);
  int st = ctx_cuda(c, cudaGetLastError(), "self-test launch");
  if (st) return st;
  return ctx_read_state(c);
}

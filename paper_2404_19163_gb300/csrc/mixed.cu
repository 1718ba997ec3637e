// Mixed-precision driver: bulk iterations of Eq. np1 on the tensor cores in the
// schemes of Table I ((h)(h) with 16-bit operands and FP32 accumulation, or
// the split (h)(h)+(h)(l)+(l)(h) of Sec. 3.2), stopped by Algorithm 2, then
// Algorithm 3's refinement with d formed in FP64 accuracy.
//
// Per bulk iteration (all products tcgen05, FP32 accumulation in TMEM):
//   K3  Q  = c1 d + c2 d^2 (+ c_k d^k)       symmetric tiles, fused polynomial epilogue
//   K4  Z' = Z + Z Q                          FP32 master update + 16-bit Z and Z^T copies
//   K1  A^T = Z^T S                           16-bit A^T for the next product
//   K2  d  = I - Z^T A, Err = ||d||_F         symmetric tiles, fused residual epilogue
// Z^T S is formed instead of S Z because S is symmetric: both operands of every
// product are then K-major (row-major) 16-bit matrices, which is what a TMA
// box and a tcgen05 shared-memory descriptor read directly.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <utility>
#include <vector>

#include "ctx.h"
#include "kernels.h"
#include "tc_gemm.h"

using namespace zf;

namespace {

struct Mat16 {
  uint16_t* h = nullptr;
  uint16_t* l = nullptr;
};

int round_up(int x, int m) { return (x + m - 1) / m * m; }

int alloc16(zfact_ctx* c, const char* name, int n, int ld, bool split, Mat16* m) {
  int st = ZFACT_OK;
  const size_t bytes = (size_t)n * ld * sizeof(uint16_t);
  std::string nh = std::string(name) + ".h", nl = std::string(name) + ".l";
  m->h = (uint16_t*)ctx_buf(c, nh.c_str(), bytes, &st);
  if (!m->h) return st;
  if (split) {
    m->l = (uint16_t*)ctx_buf(c, nl.c_str(), bytes, &st);
    if (!m->l) return st;
  } else {
    m->l = nullptr;
  }
  return ZFACT_OK;
}

}  // namespace

int ctx_make_map(zfact_ctx* c, CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows,
                 bool bf16) {
  char key[96];
  snprintf(key, sizeof(key), "%p:%d:%d:%d:%d:%d", base, rows, cols, ld, box_rows, bf16 ? 1 : 0);
  auto it = c->map_cache.find(key);
  if (it != c->map_cache.end()) {
    *m = it->second;
    return 0;
  }
  const int r = tc_make_map(m, base, rows, cols, ld, box_rows, bf16);
  if (r == 0) {
    if (c->map_cache.size() > 4096) c->map_cache.clear();
    c->map_cache[key] = *m;
  }
  return r;
}

// A tensor-core product D = sum_s A_s B_s^T (B_s given N x K, i.e. the row-major matrix whose
// rows are the columns of the right factor), with the split segments of Sec. 3.2 when
// A.l / B.l are present: (h)(h) + (h)(l) + (l)(h).
int tc_product(zfact_ctx* c, TcArgs& a, const Mat16& A, const Mat16& B, int ld, int bn) {
  TcMaps maps;
  memset(&maps, 0, sizeof(maps));
  const uint16_t* as[3] = {A.h, A.h, A.l};
  const uint16_t* bs[3] = {B.h, B.l, B.h};
  int nseg = 1;
  if (A.l && B.l) nseg = 3;
  for (int s = 0; s < nseg; ++s) {
    int r1 = ctx_make_map(c, &maps.a[s], as[s], a.M, a.K, ld, 128, a.bf16 != 0);
    int r2 = ctx_make_map(c, &maps.b[s], bs[s], a.N, a.K, ld, bn, a.bf16 != 0);
    if (r1 || r2) return ctx_fail(c, ZFACT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d, %d)", r1, r2);
  }
  a.nseg = nseg;
  a.err_flag = &c->st_dev->error;
  static const char* names[] = {"tc_gemm.store16", "tc_gemm.resid", "tc_gemm.poly", "tc_gemm.zupd",
                                "tc_gemm.f64out", "tc_gemm.zupd64"};
  const double flops = (double)nseg * 2.0 * a.M * a.N * a.K * (a.sym ? 0.5 : 1.0);
  const double in_bytes = (double)nseg * 2.0 * ((double)a.M * a.K + (double)a.N * a.K);
  const double out_elems = (double)a.M * a.N;
  const double out_bytes[] = {2, 4 + 2, 2, 8 + 4, 8, 16 + 4};
  const int e = a.epi >= 0 && a.epi <= 5 ? a.epi : 0;
  return ctx_cuda(c, klaunch(c, names[e], flops, in_bytes + out_elems * out_bytes[e] * (a.split_out ? 1.5 : 1.0), 1,
                             [&] { return launch_tc_gemm(a, maps, bn, c->num_sms, c->stream); }),
                  "tcgen05 gemm");
}

int tc_product_public(zfact_ctx* c, TcArgs& a, const uint16_t* Ah, const uint16_t* Al, const uint16_t* Bh,
                      const uint16_t* Bl, int ld, int bn) {
  Mat16 A, B;
  A.h = const_cast<uint16_t*>(Ah);
  A.l = const_cast<uint16_t*>(Al);
  B.h = const_cast<uint16_t*>(Bh);
  B.l = const_cast<uint16_t*>(Bl);
  return tc_product(c, a, A, B, ld, bn);
}

static TcArgs tc_args(int n, bool bf16) {
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.M = a.N = a.K = n;
  a.bf16 = bf16 ? 1 : 0;
  a.unscale = 1.0f;
  return a;
}

int pick_bn(int n) { return n <= 128 ? 128 : 256; }


// Algorithm 3 with d formed by FP64 CUDA-core products; Q and Z Q by FP16 hi/lo tensor-core
// products (FP32 accumulation) added to the FP64 master.
static int refine_native(zfact_ctx* c, const double* S, double* Z64, int n, int order, const zfact_opts& o,
                         int iters, int* ridx_out, zfact_info* inf, float* D32, int ld, int bn) {
  int st = ZFACT_OK;
  double coef[8];
  coef[0] = 1.0;
  for (int k = 1; k <= order; ++k) coef[k] = coef[k - 1] * (2.0 * k - 1.0) / (2.0 * k);
  int ridx = 0;
  double* A64 = (double*)ctx_buf(c, "A64", sizeof(double) * (size_t)n * n, &st);
  if (!A64) return st;
  double* D64 = (double*)ctx_buf(c, "D64", sizeof(double) * (size_t)n * n, &st);
  if (!D64) return st;
  // FP16 hi/lo operands with power-of-two scales for the refinement products
  Mat16 Dr, Qr, Zr;
  if ((st = alloc16(c, "D16r", n, ld, true, &Dr))) return st;
  if ((st = alloc16(c, "Q16r", n, ld, true, &Qr))) return st;
  if ((st = alloc16(c, "Z16r", n, ld, true, &Zr))) return st;
  int idx = iters;
  for (int r = 0; r <= o.refine_steps; ++r) {
    ++idx;
    if ((st = f64_residual(c, S, Z64, A64, D64, n, idx, o.stop_rule, o.tol, 0))) return st;
    if ((st = ctx_read_state(c))) return st;
    const double err = c->st_host->hist[idx];
    inf->resid_f = err;
    if (c->st_host->nonfinite) break;
    if (r == o.refine_steps) break;
    if (o.tol > 0 && err / sqrt((double)n) <= o.tol) break;
    // Q = c1 d + c2 d^2 with d in FP64 (FP16 hi/lo products for the quadratic term)
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, [&] { return launch_amax_f64(D64, n, c->st_dev, 1, c->stream); }), "amax d"))) return st;
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, [&] { return launch_amax_f64(Z64, n, c->st_dev, 2, c->stream); }), "amax Z"))) return st;
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, [&] { return launch_pow2_scales(c->st_dev, idx, (float)coef[1], (float)coef[2], c->stream); }), "scales")))
      return st;
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, [&] { return launch_f64_to_f32(D64, n, n, D32, ld, c->stream); }), "d to FP32"))) return st;
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, [&] {
                         return launch_cvt16(D64, n, n, Dr.h, Dr.l, ld, 1.0, &c->st_dev->scale[0], false, false,
                                             c->stream);
                       }),
                       "d16")))
      return st;
    TcArgs kq = tc_args(n, false);
    kq.epi = kEpiPoly;
    kq.sym = 1;
    kq.split_out = 1;
    kq.f32_in = D32;
    kq.ld32 = ld;
    kq.c1 = (float)coef[1];
    kq.c2 = (float)coef[2];
    kq.sa_ptr = &c->st_dev->scale[0];
    kq.sb_ptr = &c->st_dev->scale[0];
    kq.out_scale = &c->st_dev->scale[1];
    kq.o16h = Qr.h;
    kq.o16l = Qr.l;
    kq.ld16 = ld;
    if ((st = tc_product(c, kq, Dr, Dr, ld, bn))) return st;
    // Z += Z Q with an FP64 master
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, [&] {
                         return launch_cvt16(Z64, n, n, Zr.h, Zr.l, ld, 1.0, &c->st_dev->scale[2], false, false,
                                             c->stream);
                       }),
                       "Z16 refine")))
      return st;
    TcArgs ku = tc_args(n, false);
    ku.epi = kEpiZupd64;
    ku.f64 = Z64;
    ku.ld64 = n;
    ku.sa_ptr = &c->st_dev->scale[2];
    ku.sb_ptr = &c->st_dev->scale[1];
    if ((st = tc_product(c, ku, Zr, Qr, ld, bn))) return st;
    ++ridx;
  }
  *ridx_out = ridx;
  return ZFACT_OK;
}

// Algorithm 3 with d = I - Z^T S Z and Z + Z Q formed to FP64 accuracy on the BF16 tensor cores
// (CRT residues or error-free slices, ozaki.cu); the polynomial's powers d^k (k >= 2) by FP16
// hi/lo products.
int refine_ozaki(zfact_ctx* c, const double* S, double* Z64, int n, int order, const zfact_opts& o, int iters,
                 int* ridx_out, zfact_info* inf) {
  int st = ZFACT_OK;
  double coef[8];
  coef[0] = 1.0;
  for (int k = 1; k <= 5; ++k) coef[k] = coef[k - 1] * (2.0 * k - 1.0) / (2.0 * k);
  const int ld = round_up(n, 64);
  const int bn = pick_bn(n);
  const size_t nn = (size_t)n * n;
  double* D64 = (double*)ctx_buf(c, "D64", sizeof(double) * nn, &st);
  if (!D64) return st;
  double* Q64 = (double*)ctx_buf(c, "Q64", sizeof(double) * nn, &st);
  if (!Q64) return st;
  double* P64 = (double*)ctx_buf(c, "P64", sizeof(double) * nn, &st);
  if (!P64) return st;
  Mat16 Dr, Pr;
  if ((st = alloc16(c, "D16r", n, ld, true, &Dr))) return st;
  // (the update's order may exceed the bulk's under a tolerance, see below)
  if ((order > 2 || o.tol > 0) && (st = alloc16(c, "P16r", n, ld, true, &Pr))) return st;
  // slice count from the dynamic range of Z and S (see oz_slices_for); the scaled row norms of S's rows
  // and of Z's columns and rows, which set the moduli of the residue products
  void* cs = ctx_buf(c, "oz.colstats", oz_colstats_scratch_bytes(n) + sizeof(int) * (size_t)n, &st);
  if (!cs) return st;
  auto z_norms = [&]() -> cudaError_t {
    cudaError_t e = launch_ozm_rho(Z64, n, n, true, &c->st_dev->rho2[1], cs, c->stream);
    if (e == cudaSuccess) e = launch_ozm_rho(Z64, n, n, false, &c->st_dev->rho2[2], nullptr, c->stream);
    return e;
  };
  cudaMemsetAsync(c->st_dev->rho2, 0, sizeof(c->st_dev->rho2), c->stream);
  // S's Gershgorin bound and max|Z| unless this call's state already holds them (cold start, conversion of Z)
  const bool have_g = c->ghi_S == S, have_z = c->zmax_Z == Z64;
  c->zmax_Z = nullptr;
  if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 5 - (have_g ? 2 : 0) - (have_z ? 1 : 0), [&] {
                       cudaError_t e = have_g ? cudaSuccess : launch_gershgorin(S, n, c->st_dev, c->stream);
                       if (e == cudaSuccess && !have_z) e = launch_amax_f64(Z64, n, c->st_dev, 2, c->stream);
                       if (e == cudaSuccess) e = launch_ozm_rho(S, n, n, false, &c->st_dev->rho2[0], nullptr, c->stream);
                       if (e == cudaSuccess) e = z_norms();
                       return e;
                     }),
                     "dynamic range")))
    return st;
  if ((st = ctx_read_state(c))) return st;
  const int s_res = oz_slices_for(c->st_host->amax[2], c->st_host->amax[0]);
  double rho_zt = oz_rho_from(c->st_host->rho2[1], n), rho_zr = oz_rho_from(c->st_host->rho2[2], n);
  if ((st = oz_prepare_S(c, S, n, s_res, oz_rho_from(c->st_host->rho2[0], n)))) return st;
  int ridx = 0, idx = iters;
  for (int r = 0; r <= o.refine_steps; ++r) {
    ++idx;
    if (r > 0) {
      // Z changed in the update: the column norms again for this residual (a further update, rare,
      // takes the bound for any rows)
      cudaMemsetAsync(&c->st_dev->rho2[1], 0, sizeof(unsigned int), c->stream);
      if ((st = ctx_cuda(c, klaunch(c, "oz_rho", 0, 16.0 * n * n, 3, [&] {
                           return launch_ozm_rho(Z64, n, n, true, &c->st_dev->rho2[1], cs, c->stream);
                         }),
                         "Z norms")))
        return st;
      if ((st = ctx_read_state(c))) return st;
      rho_zt = oz_rho_from(c->st_host->rho2[1], n);
      rho_zr = -1.0;
    }
    // max|d| comes back with Err (from the CRT reconstruction itself, else one pass over d): it scales
    // d's 16-bit copy and bounds Q for the update's moduli or slices
    c->oz_amax = reinterpret_cast<unsigned long long*>(&c->st_dev->amax[1]);
    st = oz_residual(c, Z64, D64, n, idx, o.stop_rule, o.tol, 0, rho_zt);
    c->oz_amax = nullptr;
    if (st) return st;
    if (!c->oz_amax_done &&
        (st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1,
                                  [&] { return launch_amax_f64(D64, n, c->st_dev, 1, c->stream); }),
                       "amax d")))
      return st;
    if ((st = ctx_read_state(c))) return st;
    const double err = c->st_host->hist[idx];
    inf->resid_f = err;
    if (c->st_host->nonfinite || r == o.refine_steps) break;
    if (o.tol > 0 && err / sqrt((double)n) <= o.tol) break;
    // The polynomial of this update: with a tolerance, the lowest order m' >= 2 whose error term, estimated
    // as ||d^(m'+1)||_F ~ Err^(m'+1) / N^(m'/2) (the spectrum of d spread over N eigenvalues), is half the
    // target; else the bulk's order.  Each order costs a product; an estimate that falls short costs one more
    // refinement step, which the loop takes.
    int ord = order;
    if (o.tol > 0) {
      for (int mr = 2; mr <= 5; ++mr)
        if (pow(err, mr + 1.0) / pow((double)n, 0.5 * mr) <= 0.5 * o.tol * sqrt((double)n)) {
          ord = mr;
          break;
        }
    }
    // |Q_ij| <= sum_k c_k |(d^k)_ij| <= sum_k c_k N^(k-1) max|d|^k
    const double dmax = c->st_host->amax[1];
    double qmax = 0.0, dk = dmax;
    for (int k = 1; k <= ord; ++k, dk *= (double)n * dmax) qmax += coef[k] * dk;
    // Q = c1 d + sum_{k>=2} c_k d^k: the linear term exact in FP64, the powers by FP16 hi/lo products
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1,
                                  [&] { return launch_pow2_slot(c->st_dev, 1, 0, 0, c->stream); }),
                       "scale d")))
      return st;
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, [&] {
                         return launch_cvt16(D64, n, n, Dr.h, Dr.l, ld, 1.0, &c->st_dev->scale[0], false, false,
                                             c->stream);
                       }),
                       "d16")))
      return st;
    const double* Pprev = D64;
    for (int k = 2; k <= ord; ++k) {
      Mat16 A = Dr;
      if (k > 2) {
        // 16-bit hi/lo copy of the previous power with its own scale
        if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 3, [&] {
                             cudaError_t e = launch_amax_f64(Pprev, n, c->st_dev, 4, c->stream);
                             if (e != cudaSuccess) return e;
                             e = launch_pow2_slot(c->st_dev, 4, 4, 0, c->stream);
                             if (e != cudaSuccess) return e;
                             return launch_cvt16(Pprev, n, n, Pr.h, Pr.l, ld, 1.0, &c->st_dev->scale[4], false, false,
                                                 c->stream);
                           }),
                           "power16")))
          return st;
        A = Pr;
      }
      TcArgs kp = tc_args(n, false);
      kp.epi = kEpiF64;
      kp.sym = 1;
      kp.f64 = P64;
      kp.ld64 = n;
      kp.sa_ptr = &c->st_dev->scale[k > 2 ? 4 : 0];
      kp.sb_ptr = &c->st_dev->scale[0];
      if (ord == 2) {
        // Q = c1 d + c2 d^2 formed in the product's epilogue (FP64), no power kept
        kp.f64 = Q64;
        kp.f64_in = D64;
        kp.c1 = (float)coef[1];
        kp.c2 = (float)coef[2];
        if ((st = tc_product(c, kp, A, Dr, ld, bn))) return st;
        break;
      }
      if ((st = tc_product(c, kp, A, Dr, ld, bn))) return st;
      const double* first = (k == 2) ? D64 : Q64;
      const double a1 = (k == 2) ? coef[1] : 1.0;
      if ((st = ctx_cuda(c, klaunch(c, "elementwise", 3.0 * nn, 24.0 * nn, 1, [&] {
                           return launch_axpby64(Q64, a1, first, coef[k], P64, nn, c->stream);
                         }),
                         "Q")))
        return st;
      if (k < ord) {
        // keep the power for the next product (P64 is overwritten by it)
        double* keep = (double*)ctx_buf(c, "P64keep", sizeof(double) * nn, &st);
        if (!keep) return st;
        if ((st = ctx_cuda(c, cudaMemcpyAsync(keep, P64, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->stream),
                           "keep power")))
          return st;
        Pprev = keep;
      }
    }
    out_copy_fence(c);  // an early copy of the previous Z reads the array the update writes
    if ((st = oz_update(c, Z64, Q64, n, qmax, rho_zr))) return st;
    if ((st = out_copy_start(c, Z64))) return st;
    ++ridx;
  }
  *ridx_out = ridx;
  return ZFACT_OK;
}

// ---- device-driven bulk loop (zfact_set_loop_graphs)
// Graph: while (cond) { update(Z_c -> Z_n); cond kernel; if (cond) { update(Z_n -> Z_c); cond kernel } }.
// `body(parity)` enqueues one update on the context's stream (parity 0: Z_c -> Z_n, 1: back); it is
// captured, not run.  Every cond kernel counts the update and ends the loop at st->loop_limit updates.
// Returns ZFACT_OK with lg->exec == nullptr when the graph cannot be built (the caller then stays on the
// host loop).
template <class F>
static int loop_graph_build(zfact_ctx* c, F&& body, zfact_ctx::LoopGraph* lg) {
  lg->exec = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle hw = 0, hi = 0;
  cudaGraphNode_t wnode = nullptr, inode = nullptr;
  cudaGraphNodeParams wp = {}, ip = {};
  const bool prof = c->profiling;
  const int l0 = c->launches;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    ok = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp) == cudaSuccess &&
         cudaGraphConditionalHandleCreate(&hi, wp.conditional.phGraph_out[0], 0, cudaGraphCondAssignDefault) ==
             cudaSuccess;
  }
  c->profiling = false;  // no per-launch events inside the graph
  for (int part = 0; ok && part < 2; ++part) {
    cudaGraph_t target = part == 0 ? wp.conditional.phGraph_out[0] : ip.conditional.phGraph_out[0];
    const int lstart = c->launches;
    if (cudaStreamBeginCaptureToGraph(c->stream, target, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess) {
      ok = false;
      break;
    }
    int s2 = body(part);
    if (!s2)
      s2 = ctx_cuda(c, launch_loop_cond(c->st_dev, hw, hi, part == 0, c->stream), "loop condition");
    std::vector<cudaGraphNode_t> leaves;
    if (!s2 && part == 0) {
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      if (cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess)
        leaves.assign(deps, deps + nd);
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->stream, &captured);
    if (s2) {  // nothing is allocated inside an update: a failure here is the capture's, not the math's
      ok = false;
      break;
    }
    if (ec != cudaSuccess || (part == 0 && leaves.empty())) {
      ok = false;
      break;
    }
    lg->launches[part] = c->launches - lstart + 1;
    if (part == 0) {
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = hi;
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      ok = cudaGraphAddNode(&inode, wp.conditional.phGraph_out[0], leaves.data(), nullptr, leaves.size(), &ip) ==
           cudaSuccess;
    }
  }
  c->profiling = prof;
  c->launches = l0;
  if (ok) ok = cudaGraphInstantiate(&lg->exec, g, 0) == cudaSuccess;
  if (!ok) lg->exec = nullptr;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();  // a graph that could not be built leaves no error behind: the host loop runs instead
  return ZFACT_OK;
}

// Runs the loop graph for `key` (built on first use) from update `iters` to at most `lim` updates, waits for
// it, and returns the updates it did in *g_iters (-1: no graph, use the host loop).
template <class F>
static int loop_graph_run(zfact_ctx* c, const std::string& key, int iters, int lim, F&& body, int* g_iters) {
  *g_iters = -1;
  int st = ZFACT_OK;
  auto it = c->loop_graph_cache.find(key);
  if (it == c->loop_graph_cache.end()) {
    zfact_ctx::LoopGraph lg{};
    if ((st = loop_graph_build(c, body, &lg))) return st;
    if (!lg.exec) return ZFACT_OK;
    if (c->loop_graph_cache.size() >= 32) {
      for (auto& kv : c->loop_graph_cache) cudaGraphExecDestroy(kv.second.exec);
      c->loop_graph_cache.clear();
    }
    it = c->loop_graph_cache.emplace(key, lg).first;
  }
  if ((st = ctx_cuda(c, launch_loop_init(c->st_dev, iters, lim, c->stream), "loop init"))) return st;
  if ((st = ctx_cuda(c, klaunch(c, "bulk_graph", 0, 0, 0,
                                [&] { return cudaGraphLaunch(it->second.exec, c->stream); }),
                     "bulk loop graph")))
    return st;
  if ((st = ctx_read_state(c))) return st;
  const int g = c->st_host->loop_iter - iters;
  c->launches += 1 + ((g + 1) / 2) * it->second.launches[0] + (g / 2) * it->second.launches[1];
  *g_iters = g;
  return ZFACT_OK;
}

int mixed_refine(zfact_ctx* c, const double* S, double* Za64, double* Zb64, int n, int order, int precision,
                 const zfact_opts& o, int* iters_out, int* ridx_out, zfact_info* inf, bool cold) {
  const bool bf16 = (precision == ZFACT_P_BF16 || precision == ZFACT_P_BF16_SPLIT);
  const bool split = (precision == ZFACT_P_FP16_SPLIT || precision == ZFACT_P_BF16_SPLIT);
  // (h)(h)half: FP16 operands and an FP16 accumulator in the bulk products
  const bool half = precision == ZFACT_P_FP16_HALF;
  // FP16 has a 5-bit exponent: every FP16 operand carries a power-of-two scale (exact, so it
  // changes no significand bit) chosen from a bound on its magnitude; BF16 needs none.  With an FP16
  // accumulator the scales leave 14 more bits of headroom (operands at most 1, so a product's partial
  // sums stay below its length, far from FP16's 65504, for N up to 32768).
  const bool scaled = !bf16;
  const int head16 = half ? 14 : 0;
  IterState* sd = c->st_dev;
  auto sp = [&](int k) -> const float* { return scaled ? &sd->scale[k] : nullptr; };
  const int ld = round_up(n, 64);
  const int bn = pick_bn(n);
  int st = ZFACT_OK;
  double coef[8];
  coef[0] = 1.0;
  for (int k = 1; k <= order; ++k) coef[k] = coef[k - 1] * (2.0 * k - 1.0) / (2.0 * k);

  // ---- workspace
  Mat16 S16, Za, Zta, Zb, Ztb, At, D16, Q16, Pa, Pb;
  if ((st = alloc16(c, "S16", n, ld, split, &S16))) return st;
  if ((st = alloc16(c, "Z16a", n, ld, split, &Za))) return st;
  if ((st = alloc16(c, "Zt16a", n, ld, split, &Zta))) return st;
  if ((st = alloc16(c, "Z16b", n, ld, split, &Zb))) return st;
  if ((st = alloc16(c, "Zt16b", n, ld, split, &Ztb))) return st;
  if ((st = alloc16(c, "At16", n, ld, split, &At))) return st;
  if ((st = alloc16(c, "D16", n, ld, split, &D16))) return st;
  if ((st = alloc16(c, "Q16", n, ld, split, &Q16))) return st;
  if (order > 2) {
    if ((st = alloc16(c, "P16a", n, ld, split, &Pa))) return st;
    if ((st = alloc16(c, "P16b", n, ld, split, &Pb))) return st;
  }
  float* Zm = (float*)ctx_buf(c, "Zm32", sizeof(float) * (size_t)n * ld, &st);
  if (!Zm) return st;
  float* D32 = (float*)ctx_buf(c, "D32", sizeof(float) * (size_t)n * ld, &st);
  if (!D32) return st;
  float* Q32 = nullptr;
  if (order > 2) {
    Q32 = (float*)ctx_buf(c, "Q32", sizeof(float) * (size_t)n * ld, &st);
    if (!Q32) return st;
  }
  const int max_units = tc_num_units(tc_args(n, bf16), 128) + 16;
  const size_t npart = kTcPartsPerTile * (size_t)max_units > (size_t)cold_resid_blocks(n)
                           ? kTcPartsPerTile * (size_t)max_units
                           : (size_t)cold_resid_blocks(n);
  double* partials = (double*)ctx_buf(c, "tc_partials", sizeof(double) * npart, &st);
  if (!partials) return st;
  // cold start: the first polynomial also keeps Q0 in FP32 for the elementwise first update
  float* Q0 = nullptr;
  if (cold) {
    Q0 = (float*)ctx_buf(c, "Q0f32", sizeof(float) * (size_t)n * ld, &st);
    if (!Q0) return st;
  }

  auto elem = [&](const char* what, int count, auto&& f) -> int {
    return ctx_cuda(c, klaunch(c, "elementwise", 0, 0, count, f), what);
  };
  const int kSlotS = 3, kSlotAt = 4, kSlotD = 0, kSlotQ = 1;
  int zc_slot = 5, zn_slot = 6;

  // ---- set-up: 16-bit S (once), FP32 master Z and its 16-bit copies
  if (scaled) {
    if ((st = elem("scales S", 5 + (cold && o.start_scale > 0.0 ? 1 : 0), [&] {
           cudaError_t e = launch_gershgorin(S, n, sd, c->stream);  // amax[0] = max row sum of |S|
           c->ghi_S = S;
           // (which also resets the start scale: a caller's start_scale applies again)
           if (e == cudaSuccess && cold && o.start_scale > 0.0) e = launch_set_gscale(sd, o.start_scale, c->stream);
           if (e == cudaSuccess) e = launch_amax_f64(S, n, sd, kSlotS, c->stream);
           if (e == cudaSuccess) e = launch_pow2_slot(sd, kSlotS, kSlotS, head16, c->stream);
           if (e == cudaSuccess) e = launch_amax_f64(Za64, n, sd, 6, c->stream);
           if (e == cudaSuccess) e = launch_fp16_scales(sd, 2, 0, 0.f, 0.f, zc_slot, head16, c->stream);
           return e;
         })))
      return st;
  }
  if ((st = elem("S16", 1, [&] {
         return launch_cvt16(S, n, n, S16.h, S16.l, ld, 1.0, sp(kSlotS), false, bf16, c->stream);
       })))
    return st;
  // FP32 master Z and its 16-bit copies from Z0.  A cold start reads neither: its first residual and
  // first update are formed from S and s alone, and the update writes them (they are made from Z0 only
  // if the bulk stops before its first update).
  auto z0_copies = [&]() -> int {
    int s2;
    if ((s2 = elem("Z master", 1, [&] { return launch_f64_to_f32(Za64, n, n, Zm, ld, c->stream); }))) return s2;
    return elem("Z16", 2, [&] {
      cudaError_t e = launch_cvt16(Za64, n, n, Za.h, Za.l, ld, 1.0, sp(zc_slot), false, bf16, c->stream);
      if (e == cudaSuccess) e = launch_cvt16(Za64, n, n, Zta.h, Zta.l, ld, 1.0, sp(zc_slot), true, bf16, c->stream);
      return e;
    });
  };
  if (!cold && (st = z0_copies())) return st;

  Mat16* Zc = &Za;
  Mat16* Ztc = &Zta;
  Mat16* Zn = &Zb;
  Mat16* Ztn = &Ztb;

  // d = I - Z^T S Z from the 16-bit Z^T copy ztc (scale slot zcs); Err -> hist[idx] (idx < 0: the device's
  // loop counter + 1)
  auto residual = [&](int idx, int check_stop, Mat16* ztc, int zcs) -> int {
    int s2;
    if (scaled && (s2 = elem("scale At", 1, [&] { return launch_fp16_scales(sd, 1, 0, 0.f, 0.f, 0, head16, c->stream); })))
      return s2;
    TcArgs k1 = tc_args(n, bf16);
    k1.acc16 = half ? 1 : 0;
    k1.epi = kEpiStore16;
    k1.split_out = split;
    k1.o16h = At.h;
    k1.o16l = At.l;
    k1.ld16 = ld;
    k1.sa_ptr = sp(zcs);
    k1.sb_ptr = sp(kSlotS);
    k1.out_scale = sp(kSlotAt);
    if ((s2 = tc_product(c, k1, *ztc, S16, ld, bn))) return s2;
    cudaMemsetAsync(&sd->amaxf[1], 0, sizeof(unsigned int), c->stream);
    TcArgs k2 = tc_args(n, bf16);
    k2.acc16 = half ? 1 : 0;
    k2.epi = kEpiResid;
    k2.sym = 1;
    k2.split_out = split;
    k2.f32 = D32;
    k2.ld32 = ld;
    if (!scaled) {  // BF16: the 16-bit d is written in the same epilogue
      k2.o16h = D16.h;
      k2.o16l = D16.l;
    }
    k2.ld16 = ld;
    k2.partials = partials;
    k2.amax_bits = &sd->amaxf[1];
    k2.sa_ptr = sp(zcs);
    k2.sb_ptr = sp(kSlotAt);
    if ((s2 = tc_product(c, k2, *ztc, At, ld, bn))) return s2;
    const int np = kTcPartsPerTile * tc_num_units(k2, bn);
    if ((s2 = ctx_cuda(c, klaunch(c, "finish_err", 0, 0, 1, [&] {
                         return launch_finish_err(partials, np, sd, idx, o.stop_rule, o.tol, n, check_stop, c->stream);
                       }),
                       "finish err")))
      return s2;
    if (scaled) {
      // FP16: the scale of d needs its maximum, known only after the residual epilogue
      if ((s2 = elem("d16", 2, [&] {
             cudaError_t e = launch_fp16_scales(sd, 0, idx, (float)coef[1], (float)coef[2], 0, head16, c->stream);
             if (e == cudaSuccess)
               e = launch_cvt16_f32(D32, n, ld, D16.h, D16.l, ld, false, false, sp(kSlotD), c->stream);
             return e;
           })))
        return s2;
    }
    return ZFACT_OK;
  };

  // Cold start Z0 = s I: the first residual is d0 = I - s^2 S (no product; the symmetric X is read
  // from S's upper triangle), with the residual epilogue's outputs: FP32 d, its 16-bit copy, the Err
  // partials and max |d|.
  auto cold_residual = [&]() -> int {
    int s2;
    cudaMemsetAsync(&sd->amaxf[1], 0, sizeof(unsigned int), c->stream);
    if ((s2 = elem("cold residual", 1, [&] {
           return launch_cold_resid(S, n, sd, D32, ld, scaled ? nullptr : D16.h, scaled ? nullptr : D16.l, bf16,
                                    partials, &sd->amaxf[1], c->stream);
         })))
      return s2;
    if ((s2 = ctx_cuda(c, klaunch(c, "finish_err", 0, 0, 1, [&] {
                         return launch_finish_err(partials, cold_resid_blocks(n), sd, 0, o.stop_rule, o.tol, n, 0,
                                                  c->stream);
                       }),
                       "finish err")))
      return s2;
    if (scaled) {
      if ((s2 = elem("d16", 2, [&] {
             cudaError_t e = launch_fp16_scales(sd, 0, 0, (float)coef[1], (float)coef[2], 0, head16, c->stream);
             if (e == cudaSuccess)
               e = launch_cvt16_f32(D32, n, ld, D16.h, D16.l, ld, false, false, sp(kSlotD), c->stream);
             return e;
           })))
        return s2;
    }
    return ZFACT_OK;
  };

  // Q = sum_k c_k d^k (products of commuting symmetric matrices: symmetric tiles); q32 != nullptr
  // also keeps the final Q in FP32
  auto polynomial = [&](float* q32) -> int {
    int s2;
    Mat16* Pin = &D16;
    Mat16* Pout = &Pa;
    for (int k = 2; k <= order; ++k) {
      TcArgs kp = tc_args(n, bf16);
      kp.acc16 = half ? 1 : 0;
      kp.epi = kEpiPoly;
      kp.sym = 1;
      kp.split_out = split;
      kp.f32_in = (k == 2) ? D32 : Q32;
      kp.ld32 = ld;
      kp.c1 = (k == 2) ? (float)coef[1] : 1.0f;
      kp.c2 = (float)coef[k];
      kp.ld16 = ld;
      kp.sa_ptr = sp(kSlotD);  // d^(k-1) carries the scale of d
      kp.sb_ptr = sp(kSlotD);
      if (k == order) {
        kp.o16h = Q16.h;
        kp.o16l = Q16.l;
        kp.out_scale = sp(kSlotQ);
        kp.f32 = q32;
      } else {
        kp.f32 = Q32;
        kp.t16h = Pout->h;
        kp.t16l = Pout->l;
        kp.p_scale = sp(kSlotD);
      }
      if ((s2 = tc_product(c, kp, *Pin, D16, ld, bn))) return s2;
      Pin = Pout;
      Pout = (Pout == &Pa) ? &Pb : &Pa;
    }
    return ZFACT_OK;
  };

  // ---- bulk phase (Algorithm 2)
  if ((st = cold ? cold_residual() : residual(0, 0, Ztc, zc_slot))) return st;
  if ((st = ctx_read_state(c))) return st;
  const double err0 = c->st_host->hist[0];
  if (!(err0 < 1.0)) inf->warn = ZFACT_WARN_NONCONTRACTIVE;
  bool done = c->st_host->nonfinite || (o.fixed_iters <= 0 && o.stop_rule == 1 && err0 / sqrt((double)n) <= o.tol);
  const int limit = o.fixed_iters > 0 ? o.fixed_iters : o.nmax;
  // (the loop below runs no update exactly when this holds)
  if (cold && !(!done && 0 < limit && 0 + 1 + o.refine_steps + 1 < kHistMax) && (st = z0_copies())) return st;
  // One bulk update Z_n = Z_c + Z_c Q (a cold start's first one elementwise: s (I + Q0)), then the residual
  // of Z_n; idx < 0 takes the history index from the device (the graph-driven loop below).
  auto update = [&](Mat16* zc, Mat16* zn, Mat16* ztn, int zcs, int zns, bool cold_update, int idx,
                    int check) -> int {
    int s2;
    if ((s2 = polynomial(cold_update ? Q0 : nullptr))) return s2;
    if (scaled && (s2 = elem("scale Z", 1, [&] { return launch_fp16_scales(sd, 2, 0, 0.f, 0.f, zns, head16, c->stream); })))
      return s2;
    cudaMemsetAsync(&sd->amaxf[2], 0, sizeof(unsigned int), c->stream);
    if (cold_update) {
      if ((s2 = elem("cold update", 1, [&] {
             return launch_cold_update(Q0, n, ld, sd, Zm, zn->h, zn->l, ztn->h, ztn->l, sp(zns), bf16, &sd->amaxf[2],
                                       c->stream);
           })))
        return s2;
    } else {
      TcArgs k4 = tc_args(n, bf16);
      k4.acc16 = half ? 1 : 0;
      k4.epi = kEpiZupd;
      k4.split_out = split;
      k4.f32 = Zm;
      k4.ld32 = ld;
      k4.o16h = zn->h;
      k4.o16l = zn->l;
      k4.t16h = ztn->h;
      k4.t16l = ztn->l;
      k4.ld16 = ld;
      k4.sa_ptr = sp(zcs);
      k4.sb_ptr = sp(kSlotQ);
      k4.out_scale = sp(zns);
      k4.amax_bits = &sd->amaxf[2];
      if ((s2 = tc_product(c, k4, *zc, Q16, ld, bn))) return s2;
    }
    if (scaled && (s2 = elem("amax Z", 1, [&] { return launch_fp16_scales(sd, 3, 0, 0.f, 0.f, 0, head16, c->stream); })))
      return s2;
    return residual(idx, check, ztn, zns);
  };

  int iters = 0;
  const int lim = std::min(limit, kHistMax - o.refine_steps - 2);  // the loop's bound on updates
  const int check = o.fixed_iters <= 0 ? 1 : 0;
  while (!done && iters < lim) {
    if (iters >= 1 && check && c->loop_graphs && c->lane < 0) {
      // The rest of Algorithm 2 on the device: one CUDA graph whose while node runs two updates per
      // pass (Z_c -> Z_n, then, guarded by an if node, Z_n -> Z_c) until the stop test fires or lim
      // updates are done; no host round trip per update.
      int g_iters = -1;
      char key[256];
      snprintf(key, sizeof(key), "%d:%d:%d:%d:%.17g:%p:%p:%d:%llu", n, order, precision, o.stop_rule, o.tol,
               (void*)Zc->h, (const void*)S16.h, ld, (unsigned long long)c->ws_gen);
      if ((st = loop_graph_run(c, key, iters, lim, [&](int parity) {
             return parity == 0 ? update(Zc, Zn, Ztn, zc_slot, zn_slot, false, -1, 1)
                                : update(Zn, Zc, Ztc, zn_slot, zc_slot, false, -1, 1);
           }, &g_iters)))
        return st;
      if (g_iters < 0) {
        c->loop_graphs = false;  // this device or driver cannot build it: the host loop from here on
        continue;
      }
      if (g_iters & 1) {
        std::swap(Zc, Zn);
        std::swap(Ztc, Ztn);
        std::swap(zc_slot, zn_slot);
      }
      iters += g_iters;
      done = true;
      break;
    }
    if ((st = update(Zc, Zn, Ztn, zc_slot, zn_slot, cold && iters == 0, iters + 1, check))) return st;
    std::swap(Zc, Zn);
    std::swap(Ztc, Ztn);
    std::swap(zc_slot, zn_slot);
    ++iters;
    if ((st = ctx_read_state(c))) return st;
    done = c->st_host->nonfinite || c->st_host->stop;
  }
  *iters_out = iters;
  // A caller's start scale (a learned proposal) whose bulk did not bring Err below min(1/4, Err_0):
  // the refinement could not repair it within its steps, so start again from the Gershgorin scale.
  if (cold && o.start_scale > 0.0 && o.fixed_iters <= 0) {
    const double last = c->st_host->hist[iters];
    if (c->st_host->nonfinite || !(last < 0.25) || !(last < err0)) return kRetryGershgorin;
  }
  if (c->st_host->nonfinite) {
    c->mixed_result = Za64;
    return ZFACT_OK;
  }

  // ---- refinement (Algorithm 3): Z = FP64[Z]; X = Z^T S Z in FP64; Z = Z p(X)
  if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 1, [&] {
                       return launch_f32_to_f64(Zm, n, ld, Za64, n, c->stream,
                                                reinterpret_cast<unsigned long long*>(&sd->amax[2]));
                     }),
                     "Z to FP64")))
    return st;
  c->zmax_Z = Za64;  // max|Z| is in the state for the refinement's set-up
  double* Z64 = Za64;
  int ridx = 0;
  if (o.refine_steps <= 0 && !o.final_residual) {
    // bulk only: no refinement and no FP64-accurate residual requested
    *ridx_out = 0;
    c->mixed_result = Z64;
    return ZFACT_OK;
  }
  if (o.refine_mode == ZFACT_R_OZAKI) {
    if ((st = refine_ozaki(c, S, Z64, n, order, o, iters, &ridx, inf))) return st;
  } else if (o.refine_mode == ZFACT_R_FP32) {
    if ((st = refine_fp32(c, S, Z64, n, order, o, iters, &ridx, inf))) return st;
  } else {
    if ((st = refine_native(c, S, Z64, n, order, o, iters, &ridx, inf, D32, ld, bn))) return st;
  }
  *ridx_out = ridx;
  c->mixed_result = Z64;
  return ZFACT_OK;
}

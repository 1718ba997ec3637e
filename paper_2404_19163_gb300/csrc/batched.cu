// zfact_refine_batched: many independent factorizations of uneven N (frames of a
// trajectory, steps of a geometry optimisation: the warm starts of Sec. 6) in grouped
// launches.  Each GEMM stage of an iteration is ONE persistent tcgen05 launch over the
// tiles of every live instance (largest instances first); converged instances drop out on
// the device (their units are skipped by all warp roles); the iteration (K3, K4, K1, K2 and
// the per-instance stop test of Algorithm 2) is a fixed sequence of grouped launches.
// The tile width of the grouped products is picked by timing both candidates on the first
// call for a given set of sizes (autotuner).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "batched.h"
#include "ctx.h"
#include "kernels.h"
#include "tc_gemm.h"

using namespace zf;

namespace {

int rup(int x, int m) { return (x + m - 1) / m * m; }

int tiles_sq(int n, bool sym, int bn) {
  const int tm = (n + 127) / 128, tn = (n + bn - 1) / bn;
  if (!sym) return tm * tn;
  int t = 0;
  for (int r = 0; r < tm; ++r) t += tn - (r * 128) / bn;
  return t;
}

struct Mat16p {
  uint16_t* h;
  uint16_t* l;
};

struct Packs {
  uint16_t *Sh, *Sl, *Zah, *Zal, *Ztah, *Ztal, *Zbh, *Zbl, *Ztbh, *Ztbl, *Ath, *Atl, *Dh, *Dl, *Qh, *Ql, *Pah, *Pal,
      *Pbh, *Pbl;
  float *Zm, *D32, *Q32;
};

}  // namespace

extern "C" int zfact_refine_batched(zfact_ctx* c, int count, const double* const* S, const double* const* Z0,
                                    const int64_t* N, const int* orders, int precision, const zfact_opts* opts_in,
                                    double* const* Z, double* hist, int hist_cap, zfact_info* info, int* status) {
  if (!c) return ZFACT_ERR_ARG;
  if (count < 1 || !S || !N || !Z) return ctx_fail(c, ZFACT_ERR_ARG, "bad batch arguments");
  const int order = orders ? orders[0] : 2;
  if (order < 2 || order > 5) return ctx_fail(c, ZFACT_ERR_ARG, "order out of range");
  for (int i = 0; i < count; ++i) {
    if (orders && orders[i] != order)
      return ctx_fail(c, ZFACT_ERR_UNSUPPORTED, "one order per batched call (group instances by order)");
    if (N[i] < 1 || N[i] > 65536) return ctx_fail(c, ZFACT_ERR_ARG, "N[%d] out of range", i);
    if (!S[i] || !Z[i]) return ctx_fail(c, ZFACT_ERR_ARG, "null matrix for instance %d", i);
    if (!is_device_ptr(S[i]) || !is_device_ptr(Z[i]) || (Z0 && Z0[i] && !is_device_ptr(Z0[i])))
      return ctx_fail(c, ZFACT_ERR_ARG, "batched matrices must be device pointers");
  }
  if (precision != ZFACT_P_BF16 && precision != ZFACT_P_BF16_SPLIT)
    return ctx_fail(c, ZFACT_ERR_UNSUPPORTED, "batched mode runs the BF16 and BF16 hi/lo split bulks");
  const bool split = precision == ZFACT_P_BF16_SPLIT;
  cudaSetDevice(c->device);
  zfact_opts o;
  zfact_default_opts(&o);
  if (opts_in) o = *opts_in;
  if (o.nmax < 1) o.nmax = 1;
  const int limit = o.fixed_iters > 0 ? o.fixed_iters : o.nmax;
  int st = ZFACT_OK;
  c->launches = 0;
  c->ghi_S = nullptr;
  c->zmax_Z = nullptr;
  cudaEventRecord(c->ev0, c->stream);

  // ---- layout: instances stacked along rows, largest first; 256-row slots, common ld
  std::vector<int> n(count), order_idx(count), row0(count), part0(count), nparts(count);
  for (int i = 0; i < count; ++i) n[i] = (int)N[i];
  std::iota(order_idx.begin(), order_idx.end(), 0);
  std::stable_sort(order_idx.begin(), order_idx.end(), [&](int a, int b) { return n[a] > n[b]; });
  const int max_n = n[order_idx[0]];
  const int ld = rup(max_n, 64);
  int rows = 0, parts = 0;
  for (int j = 0; j < count; ++j) {
    const int i = order_idx[j];
    row0[i] = rows;
    rows += rup(n[i], 256);
  }
  for (int i = 0; i < count; ++i) {
    nparts[i] = kTcPartsPerTile * tiles_sq(n[i], true, 128);  // the larger of the two tile widths' counts
    part0[i] = parts;
    parts += nparts[i];
  }
  // layout signature (sizes in order) decides whether the packs must be re-zeroed
  std::string sig = std::to_string(precision) + ":" + std::to_string(order);
  for (int i = 0; i < count; ++i) sig += "," + std::to_string(n[i]);

  // ---- device tables (one allocation): ints then pointers
  const size_t n_int = (size_t)count * 4 + 2 * (size_t)(count + 1) + count;  // n,row0,part0,nparts,prefix x2,order
  const size_t tab_bytes = n_int * sizeof(int) + 256 + (size_t)count * 3 * sizeof(void*);
  char* tab = (char*)ctx_buf(c, "b.tables", tab_bytes, &st);
  if (!tab) return st;
  std::vector<char> host(tab_bytes, 0);
  int* hi = (int*)host.data();
  int* d_n = (int*)tab;
  memcpy(hi, n.data(), sizeof(int) * count);
  memcpy(hi + count, row0.data(), sizeof(int) * count);
  memcpy(hi + 2 * count, part0.data(), sizeof(int) * count);
  memcpy(hi + 3 * count, nparts.data(), sizeof(int) * count);
  int* h_pre_ns = hi + 4 * count;
  int* h_pre_s = h_pre_ns + (count + 1);
  int* h_ord = h_pre_s + (count + 1);
  memcpy(h_ord, order_idx.data(), sizeof(int) * count);
  const size_t ptr_off = rup((int)(n_int * sizeof(int)), 256);
  const double** hS = (const double**)(host.data() + ptr_off);
  const double** hZ0 = hS + count;
  double** hZ = (double**)(hZ0 + count);
  for (int i = 0; i < count; ++i) {
    hS[i] = S[i];
    hZ0[i] = Z0 ? Z0[i] : nullptr;
    hZ[i] = Z[i];
  }
  BatchTables t;
  t.n = d_n;
  t.row0 = d_n + count;
  t.part0 = d_n + 2 * count;
  t.nparts = d_n + 3 * count;
  const int* d_pre_ns = d_n + 4 * count;
  const int* d_pre_s = d_pre_ns + (count + 1);
  const int* d_ord = d_pre_s + (count + 1);
  t.S = (const double* const*)(tab + ptr_off);
  t.Z0 = t.S + count;
  t.Z = (double* const*)(t.Z0 + count);

  // ---- tile width: autotuned per layout (timed on the idempotent product A^T = Z^T S)
  auto& tuned = c->batch_bn;
  int bn = 256;
  int* h_nparts = hi + 3 * count;
  auto fill_prefix = [&](int bnv) {
    h_pre_ns[0] = h_pre_s[0] = 0;
    for (int j = 0; j < count; ++j) {
      const int i = order_idx[j];
      h_pre_ns[j + 1] = h_pre_ns[j] + tiles_sq(n[i], false, bnv);
      h_pre_s[j + 1] = h_pre_s[j] + tiles_sq(n[i], true, bnv);
      h_nparts[i] = kTcPartsPerTile * tiles_sq(n[i], true, bnv);  // partials the residual epilogue writes
    }
  };
  auto it_tuned = tuned.find(sig);
  if (it_tuned != tuned.end()) bn = it_tuned->second;
  fill_prefix(bn);
  if ((st = ctx_cuda(c, cudaMemcpyAsync(tab, host.data(), tab_bytes, cudaMemcpyHostToDevice, c->stream), "tables")))
    return st;
  // the host copy must stay valid until the copy ran
  if ((st = ctx_cuda(c, cudaStreamSynchronize(c->stream), "tables sync"))) return st;

  // ---- packed buffers
  const size_t e16 = (size_t)rows * ld;
  Packs p;
  memset(&p, 0, sizeof(p));
  struct B16 {
    const char* name;
    uint16_t** ptr;
    bool want;
  } b16[] = {{"b.Sh", &p.Sh, true},   {"b.Sl", &p.Sl, split},   {"b.Zah", &p.Zah, true},  {"b.Zal", &p.Zal, split},
             {"b.Ztah", &p.Ztah, true}, {"b.Ztal", &p.Ztal, split}, {"b.Zbh", &p.Zbh, true},  {"b.Zbl", &p.Zbl, split},
             {"b.Ztbh", &p.Ztbh, true}, {"b.Ztbl", &p.Ztbl, split}, {"b.Ath", &p.Ath, true},  {"b.Atl", &p.Atl, split},
             {"b.Dh", &p.Dh, true},     {"b.Dl", &p.Dl, split},     {"b.Qh", &p.Qh, true},    {"b.Ql", &p.Ql, split},
             {"b.Pah", &p.Pah, order > 2}, {"b.Pal", &p.Pal, order > 2 && split},
             {"b.Pbh", &p.Pbh, order > 2}, {"b.Pbl", &p.Pbl, order > 2 && split}};
  const bool relayout = (c->batch_sig != sig);
  for (auto& b : b16) {
    if (!b.want) continue;
    *b.ptr = (uint16_t*)ctx_buf(c, b.name, e16 * 2, &st);
    if (!*b.ptr) return st;
    if (relayout) cudaMemsetAsync(*b.ptr, 0, e16 * 2, c->stream);
  }
  p.Zm = (float*)ctx_buf(c, "b.Zm", e16 * 4, &st);
  if (!p.Zm) return st;
  p.D32 = (float*)ctx_buf(c, "b.D32", e16 * 4, &st);
  if (!p.D32) return st;
  if (order > 2) {
    p.Q32 = (float*)ctx_buf(c, "b.Q32", e16 * 4, &st);
    if (!p.Q32) return st;
  }
  if (relayout) {
    cudaMemsetAsync(p.Zm, 0, e16 * 4, c->stream);
    cudaMemsetAsync(p.D32, 0, e16 * 4, c->stream);
    if (p.Q32) cudaMemsetAsync(p.Q32, 0, e16 * 4, c->stream);
    c->batch_sig = sig;
  }
  double* partials = (double*)ctx_buf(c, "b.partials", sizeof(double) * (size_t)parts, &st);
  if (!partials) return st;
  unsigned long long* gmax = (unsigned long long*)ctx_buf(c, "b.gmax", 8 * (size_t)count, &st);
  if (!gmax) return st;
  // batch state
  const int cap = hist_cap > 0 ? (hist_cap < 1024 ? hist_cap : 1024) : 64;
  char* sbuf = (char*)ctx_buf(c, "b.state", (size_t)count * (cap + 1) * 8 + (size_t)count * 5 * 4 + 64, &st);
  if (!sbuf) return st;
  BatchState bs;
  bs.cap = cap;
  bs.hist = (double*)sbuf;
  bs.prev_err = bs.hist + (size_t)count * cap;
  bs.iters = (int*)(bs.prev_err + count);
  bs.done = bs.iters + count;
  bs.nonfinite = bs.done + count;
  bs.hist_len = bs.nonfinite + count;
  bs.live = bs.hist_len + count;
  cudaMemsetAsync(sbuf, 0, (size_t)count * (cap + 1) * 8 + (size_t)count * 5 * 4 + 64, c->stream);
  cudaMemcpyAsync(bs.live, &count, sizeof(int), cudaMemcpyHostToDevice, c->stream);

  double coef[8];
  coef[0] = 1.0;
  for (int k = 1; k <= order; ++k) coef[k] = coef[k - 1] * (2.0 * k - 1.0) / (2.0 * k);

  // ---- set-up kernels
  if ((st = ctx_cuda(c, klaunch(c, "b_setup", 0, 0, 3, [&] {
                       cudaError_t e = launch_b_gersh(t, count, max_n, gmax, c->stream);
                       if (e == cudaSuccess)
                         e = launch_b_pack(t, count, max_n, 0, gmax, ld, true, p.Sh, p.Sl, nullptr, nullptr, nullptr,
                                           c->stream);
                       if (e == cudaSuccess)
                         e = launch_b_pack(t, count, max_n, 1, gmax, ld, true, p.Zah, p.Zal, p.Ztah, p.Ztal, p.Zm,
                                           c->stream);
                       return e;
                     }),
                     "batched set-up")))
    return st;

  // ---- grouped products
  auto grouped = [&](TcArgs& a, const uint16_t* Ah, const uint16_t* Al, const uint16_t* Bh, const uint16_t* Bl,
                     bool sym, int bnv, const char* name) -> int {
    TcMaps maps;
    memset(&maps, 0, sizeof(maps));
    const uint16_t* as[3] = {Ah, Ah, Al};
    const uint16_t* bs2[3] = {Bh, Bl, Bh};
    const int nseg = (Al && Bl) ? 3 : 1;
    for (int s = 0; s < nseg; ++s) {
      int r1 = ctx_make_map(c, &maps.a[s], as[s], rows, ld, ld, 128, true);
      int r2 = ctx_make_map(c, &maps.b[s], bs2[s], rows, ld, ld, bnv, true);
      if (r1 || r2) return ctx_fail(c, ZFACT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d, %d)", r1, r2);
    }
    a.nseg = nseg;
    a.bf16 = 1;
    a.unscale = 1.0f;
    a.sym = sym ? 1 : 0;
    a.ninst = count;
    a.M = sym ? h_pre_s[count] : h_pre_ns[count];  // total units
    a.N = a.K = max_n;
    a.g_prefix = sym ? d_pre_s : d_pre_ns;
    a.g_inst = d_ord;
    a.g_n = t.n;
    a.g_row0 = t.row0;
    a.g_part0 = t.part0;
    a.g_done = bs.done;
    a.ld16 = ld;
    a.ld32 = ld;
    a.err_flag = &c->st_dev->error;
    double flops = 0;
    for (int i = 0; i < count; ++i) flops += (double)nseg * 2.0 * n[i] * (double)n[i] * n[i] * (sym ? 0.5 : 1.0);
    return ctx_cuda(c, klaunch(c, name, flops, 0, 1, [&] { return launch_tc_gemm(a, maps, bnv, c->num_sms, c->stream); }),
                    "grouped tcgen05");
  };

  Mat16p Zc{p.Zah, p.Zal}, Ztc{p.Ztah, p.Ztal}, Zn{p.Zbh, p.Zbl}, Ztn{p.Ztbh, p.Ztbl};
  auto k1 = [&](int bnv) -> int {
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.epi = kEpiStore16;
    a.split_out = split;
    a.o16h = p.Ath;
    a.o16l = p.Atl;
    return grouped(a, Ztc.h, Ztc.l, p.Sh, p.Sl, false, bnv, "tc_gemm.b_store16");
  };
  auto k2 = [&]() -> int {
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.epi = kEpiResid;
    a.split_out = split;
    a.f32 = p.D32;
    a.o16h = p.Dh;
    a.o16l = p.Dl;
    a.partials = partials;
    return grouped(a, Ztc.h, Ztc.l, p.Ath, p.Atl, true, bn, "tc_gemm.b_resid");
  };
  auto poly = [&]() -> int {
    uint16_t* pin_h = p.Dh;
    uint16_t* pin_l = p.Dl;
    for (int k = 2; k <= order; ++k) {
      TcArgs a;
      memset(&a, 0, sizeof(a));
      a.epi = kEpiPoly;
      a.split_out = split;
      a.f32_in = (k == 2) ? p.D32 : p.Q32;
      a.c1 = (k == 2) ? (float)coef[1] : 1.0f;
      a.c2 = (float)coef[k];
      uint16_t *pout_h = ((k & 1) ? p.Pbh : p.Pah), *pout_l = ((k & 1) ? p.Pbl : p.Pal);
      if (k == order) {
        a.o16h = p.Qh;
        a.o16l = p.Ql;
      } else {
        a.f32 = p.Q32;
        a.t16h = pout_h;
        a.t16l = pout_l;
      }
      int s2 = grouped(a, pin_h, pin_l, p.Dh, p.Dl, true, bn, "tc_gemm.b_poly");
      if (s2) return s2;
      pin_h = pout_h;
      pin_l = pout_l;
    }
    return ZFACT_OK;
  };
  auto k4 = [&]() -> int {
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.epi = kEpiZupd;
    a.split_out = split;
    a.f32 = p.Zm;
    a.o16h = Zn.h;
    a.o16l = Zn.l;
    a.t16h = Ztn.h;
    a.t16l = Ztn.l;
    return grouped(a, Zc.h, Zc.l, p.Qh, p.Ql, false, bn, "tc_gemm.b_zupd");
  };
  auto finish = [&](int initial) -> int {
    return ctx_cuda(c, klaunch(c, "b_finish", 0, 0, 1, [&] {
                      return launch_b_finish(partials, t, bs, count, initial, o.stop_rule, o.tol,
                                             o.fixed_iters <= 0 ? 1 : 0, limit, c->stream);
                    }),
                    "batched finish");
  };

  // autotune the tile width once per layout
  if (it_tuned == tuned.end()) {
    float best = 1e30f;
    int best_bn = 256;
    for (int cand : {256, 128}) {
      fill_prefix(cand);
      cudaMemcpyAsync(tab, host.data(), tab_bytes, cudaMemcpyHostToDevice, c->stream);
      cudaEvent_t e0 = ev_get(c), e1 = ev_get(c);
      if ((st = k1(cand))) return st;  // warm
      cudaEventRecord(e0, c->stream);
      if ((st = k1(cand))) return st;
      cudaEventRecord(e1, c->stream);
      cudaStreamSynchronize(c->stream);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      c->ev_pool.push_back(e0);
      c->ev_pool.push_back(e1);
      if (ms < best) {
        best = ms;
        best_bn = cand;
      }
    }
    bn = best_bn;
    tuned[sig] = bn;
    fill_prefix(bn);
    if ((st = ctx_cuda(c, cudaMemcpyAsync(tab, host.data(), tab_bytes, cudaMemcpyHostToDevice, c->stream), "tables")))
      return st;
    cudaStreamSynchronize(c->stream);
  }

  // ---- bulk (Algorithm 2 per instance)
  if ((st = k1(bn))) return st;
  if ((st = k2())) return st;
  if ((st = finish(1))) return st;
  int* live_h = &c->st_host->pad[0];
  int iters = 0;
  while (iters < limit) {
    if ((st = ctx_cuda(c, cudaMemcpyAsync(live_h, bs.live, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "live")))
      return st;
    if ((st = ctx_cuda(c, cudaStreamSynchronize(c->stream), "live sync"))) return st;
    kstats_flush(c);
    if (*live_h <= 0) break;
    if ((st = poly())) return st;
    if ((st = k4())) return st;
    std::swap(Zc, Zn);
    std::swap(Ztc, Ztn);
    if ((st = k1(bn))) return st;
    if ((st = k2())) return st;
    if ((st = finish(0))) return st;
    ++iters;
  }
  if ((st = ctx_cuda(c, klaunch(c, "b_unpack", 0, 0, 1,
                                [&] { return launch_b_unpack(t, count, max_n, p.Zm, ld, c->stream); }),
                     "unpack")))
    return st;

  // ---- read back per-instance histories
  std::vector<double> hh((size_t)count * cap);
  std::vector<int> hits(count), hlen(count), hnf(count);
  cudaMemcpyAsync(hh.data(), bs.hist, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(hits.data(), bs.iters, sizeof(int) * count, cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(hlen.data(), bs.hist_len, sizeof(int) * count, cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(hnf.data(), bs.nonfinite, sizeof(int) * count, cudaMemcpyDeviceToHost, c->stream);
  if ((st = ctx_cuda(c, cudaStreamSynchronize(c->stream), "batch read-back"))) return st;
  kstats_flush(c);
  const int bulk_launches = c->launches;

  // ---- FP64-accurate final residual of every returned Z (CRT residues or slices), kLanes instances
  // at a time on concurrent streams (each lane with its own workspace and Err slot)
  std::vector<double> resid(count, NAN);
  std::vector<int> rit(count, 0);
  if (o.refine_steps > 0) {
    // Algorithm 3 for every instance, on request only (the default certifies the bulk result): the
    // single-instance refinement on the returned FP64 Z, its Err entries appended to the instance's
    // history; its last residual is the FP64-accurate residual of the returned Z.
    if (o.refine_mode == ZFACT_R_NATIVE)
      return ctx_fail(c, ZFACT_ERR_UNSUPPORTED, "batched refinement offers the sliced and FP32 modes");
    for (int i = 0; i < count; ++i) {
      if (hnf[i]) continue;
      zfact_opts oi = o;
      oi.refine_steps = std::min(o.refine_steps, kHistMax - 3 - hits[i]);
      if (oi.refine_steps < 0) oi.refine_steps = 0;
      const int ord = orders ? orders[i] : 2;
      zfact_info inf;
      memset(&inf, 0, sizeof(inf));
      int ridx = 0;
      cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
      st = (o.refine_mode == ZFACT_R_FP32) ? refine_fp32(c, S[i], Z[i], n[i], ord, oi, hits[i], &ridx, &inf)
                                           : refine_ozaki(c, S[i], Z[i], n[i], ord, oi, hits[i], &ridx, &inf);
      if (st) return st;
      if ((st = ctx_read_state(c))) return st;
      const int end = std::min(c->st_host->hist_len, cap);
      for (int k = hits[i] + 1; k < end; ++k) hh[(size_t)i * cap + k] = c->st_host->hist[k];
      hlen[i] = std::max(hlen[i], end);
      if (c->st_host->nonfinite) hnf[i] = 1;
      resid[i] = inf.resid_f;
      rit[i] = ridx;
    }
  } else if (o.final_residual) {
    const int L = zfact_ctx::kLanes;
    for (int l = 0; l < L; ++l)
      if (!c->lane_stream[l] && cudaStreamCreateWithFlags(&c->lane_stream[l], cudaStreamNonBlocking) != cudaSuccess)
        return ctx_fail(c, ZFACT_ERR_CUDA, "lane stream");
    // every instance's slice count from its dynamic range, as in the single-instance refinement
    // and the scaled row norms of S_i's rows and Z_i's columns, which set the moduli of its residue
    // products (one read-back for all instances)
    unsigned long long* rng = (unsigned long long*)ctx_buf(c, "b.ranges", 16 * (size_t)count + 8 * (size_t)count, &st);
    if (!rng) return st;
    unsigned int* rho2 = reinterpret_cast<unsigned int*>(rng + 2 * (size_t)count);
    void* rscratch = ctx_buf(c, "b.rho_scratch", b_rho_scratch_bytes(rows), &st);
    if (!rscratch) return st;
    std::vector<unsigned long long> hr(3 * (size_t)count);
    if ((st = ctx_cuda(c, klaunch(c, "elementwise", 0, 0, 6, [&] {
                         cudaError_t e = launch_b_ranges(t, count, max_n, rng, rng + count, c->stream);
                         if (e == cudaSuccess) e = launch_b_rho(t, count, max_n, rows, rho2, rscratch, c->stream);
                         return e;
                       }),
                       "batch ranges")))
      return st;
    cudaMemcpyAsync(hr.data(), rng, 24 * (size_t)count, cudaMemcpyDeviceToHost, c->stream);
    if ((st = ctx_cuda(c, cudaStreamSynchronize(c->stream), "ranges read-back"))) return st;
    std::vector<int> slices(count);
    std::vector<double> rho_s(count), rho_z(count);
    const unsigned int* hrho = reinterpret_cast<const unsigned int*>(hr.data() + 2 * (size_t)count);
    for (int i = 0; i < count; ++i) {
      double g, z;
      memcpy(&g, &hr[i], 8);
      memcpy(&z, &hr[count + i], 8);
      slices[i] = oz_slices_for(z, g);
      rho_s[i] = oz_rho_from(hrho[i], n[i]);
      rho_z[i] = oz_rho_from(hrho[count + i], n[i]);
    }
    // Grouped launches over all instances where the batch allows (rows of at most 83 bits, residues
    // rather than slices); else per-instance lanes.
    bool grouped_done = false;
    if ((st = batched_grouped_residuals(c, count, n, order_idx, S, Z, slices, rho_s, rho_z, resid, &grouped_done)))
      return st;
    // Lane l takes instances order_idx[l], order_idx[l + L], ... (largest first: its buffers never
    // grow), one after another on its stream with no host wait in between: each residual's Err, which
    // the lane's next residual overwrites in the state, is copied to the instance's slot on the lane.
    if (!grouped_done) {
      double* rdev = (double*)ctx_buf(c, "b.resid", sizeof(double) * (size_t)count, &st);
      if (!rdev) return st;
      cudaEvent_t fork = ev_get(c);
      cudaEvent_t join[zfact_ctx::kLanes];
      for (int l = 0; l < L; ++l) join[l] = ev_get(c);
      cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);
      cudaEventRecord(fork, c->stream);
      const int nl = std::min(L, count);
      for (int l = 0; l < nl; ++l) cudaStreamWaitEvent(c->lane_stream[l], fork, 0);
      for (int j = 0; j < count; ++j) {
        const int l = j % L, i = order_idx[j];
        c->lane = l;
        double* D64 = (double*)ctx_buf(c, lane_name(c, "D64").c_str(), sizeof(double) * (size_t)n[i] * n[i], &st);
        if (!D64) {
          c->lane = -1;
          return st;
        }
        st = oz_prepare_S(c, S[i], n[i], slices[i], rho_s[i]);
        if (!st) st = oz_residual(c, Z[i], D64, n[i], l, 0, 0.0, 0, rho_z[i]);
        if (!st)
          st = ctx_cuda(c, cudaMemcpyAsync(rdev + i, &c->st_dev->hist[l], sizeof(double), cudaMemcpyDeviceToDevice,
                                           c->lane_stream[l]),
                        "residual slot");
        c->lane = -1;
        if (st) return st;
      }
      for (int l = 0; l < nl; ++l) {
        cudaEventRecord(join[l], c->lane_stream[l]);
        cudaStreamWaitEvent(c->stream, join[l], 0);
      }
      if ((st = ctx_cuda(c, cudaMemcpyAsync(resid.data(), rdev, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost,
                                            c->stream),
                         "residuals")))
        return st;
      if ((st = ctx_read_state(c))) return st;
      c->ev_pool.push_back(fork);
      for (int l = 0; l < L; ++l) c->ev_pool.push_back(join[l]);
    }
  }
  cudaEventRecord(c->ev1, c->stream);
  cudaEventSynchronize(c->ev1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);

  int ret = ZFACT_OK;
  for (int i = 0; i < count; ++i) {
    const int hl = std::min(hlen[i], cap);
    if (hist)
      for (int k = 0; k < hist_cap; ++k) hist[(size_t)i * hist_cap + k] = (k < hl) ? hh[(size_t)i * cap + k] : NAN;
    int sti = ZFACT_OK;
    if (hnf[i]) sti = ZFACT_ERR_NONFINITE;
    else if (!(hh[(size_t)i * cap] < 1.0)) sti = ZFACT_WARN_NONCONTRACTIVE;
    else if (o.tol > 0 && o.final_residual && !(resid[i] / sqrt((double)n[i]) <= o.tol)) sti = ZFACT_ERR_NOT_CONVERGED;
    if (status) status[i] = sti;
    if (sti != ZFACT_OK && sti != ZFACT_WARN_NONCONTRACTIVE && ret == ZFACT_OK) ret = sti;
    if (info) {
      memset(&info[i], 0, sizeof(zfact_info));
      info[i].iters = hits[i];
      info[i].refine_iters = rit[i];
      info[i].hist_len = hl;
      info[i].warn = (sti == ZFACT_WARN_NONCONTRACTIVE) ? ZFACT_WARN_NONCONTRACTIVE : 0;
      info[i].resid_f = resid[i];
      info[i].ms = ms;
      info[i].launches = (i == 0) ? c->launches : 0;
    }
  }
  (void)bulk_launches;
  if (ret) ctx_fail(c, ret, "one or more instances failed (see status)");
  return ret;
}

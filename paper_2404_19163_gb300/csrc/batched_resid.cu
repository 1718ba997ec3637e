// FP64-accurate final residuals of the batched mode as grouped launches: every stage of the residual
// d_i = I - Z_i^T S_i Z_i (the residues of S_i's rows and of Z_i's columns, A_i^T = Z_i^T S_i, A_i's
// residues, X_i = Z_i^T A_i with the fused d = I - X and its Err) is one launch over a group of instances,
// as the bulk's products are.  Instances are grouped in the bulk's order (largest first) under a memory
// budget; within a group every operand's residue planes are stacked by instance along the rows of one
// packed buffer (instance i at row row0[i], one leading dimension), so one tensor map covers all of them and
// one persistent tcgen05 launch forms every instance's residue products (units: instance, modulus, tile).
// The moduli of a product are the largest any instance of the group asks for (each instance's from its
// measured row norms, as in the single-instance refinement).  Two buffer sets on two streams let one
// group's residues and first product run while the host reads the previous group's A norms (which set the
// second product's moduli).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "batched.h"
#include "ctx.h"
#include "kernels.h"
#include "tc_gemm.h"

using namespace zf;

namespace {

int rup(int x, int m) { return (x + m - 1) / m * m; }

int tiles256(int n, bool sym) {
  const int tm = (n + 127) / 128, tn = (n + 255) / 256;
  if (!sym) return tm * tn;
  int t = 0;
  for (int r = 0; r < tm; ++r) t += tn - (r * 128) / 256;
  return t;
}

// the moduli count of `bits` (0: no set holds it) and whether it needs the wider set
int count_of(const zfact_ctx* c, int T, double bits, bool* wide) {
  int w = 0;
  const int k = oz_moduli_count(c, T, T, bits, &w);
  *wide = w != 0;
  return k;
}

struct Group {
  int first, cnt;   // instances order[first .. first + cnt)
  int rows, ld, max_n, maxT;
  int k1, kz;       // moduli of Z^T S, planes of Z^T (enough for Z^T A with any A)
  bool wide_res;    // residues by the wide kernels (rows of more than 62 bits, or more than 20 planes)
  size_t tab_off;   // ints in the device table: n, row0, T, prefix1, prefix2, inst (6 arrays)
  size_t ptr_off;   // pointers: S, Z
};

}  // namespace

int batched_grouped_residuals(zfact_ctx* c, int count, const std::vector<int>& n, const std::vector<int>& order,
                              const double* const* S, double* const* Z, const std::vector<int>& slices,
                              const std::vector<double>& rho_s, const std::vector<double>& rho_z,
                              std::vector<double>& resid, bool* done) {
  *done = false;
  if (c->oz_scheme == ZFACT_EMU_SLICES || count < 1) return ZFACT_OK;
  const int chunk_kb = oz_crt_chunk_kb();
  const size_t budget = (size_t)12 << 30;  // per buffer set; two sets pipeline consecutive groups
  // ---- groups (bulk order, largest first) within the memory budget
  std::vector<Group> groups;
  std::vector<int> T(count), k1i(count), kzi(count);
  for (int j = 0; j < count; ++j) {
    const int i = order[j];
    T[i] = 6 * slices[i];
    if (T[i] > 83) return ZFACT_OK;  // outside the grouped form: lanes
    bool w1 = false, w2 = false;
    const double b1 = oz_product_bits(T[i], T[i], rho_z[i], rho_s[i], n[i]);
    const double b2 = oz_product_bits(T[i], T[i], rho_z[i], -1.0, n[i]);
    k1i[i] = count_of(c, T[i], b1, &w1);
    kzi[i] = count_of(c, T[i], std::max(b1, b2), &w2);
    if (k1i[i] < 1 || kzi[i] < 1) return ZFACT_OK;
  }
  for (int j = 0; j < count;) {
    Group g{};
    g.first = j;
    g.ld = rup(n[order[j]], 64);
    g.max_n = n[order[j]];
    while (j < count) {
      const int i = order[j];
      const int rows = g.rows + rup(n[i], 256);
      const int k1 = std::max(g.k1, k1i[i]), kz = std::max(g.kz, kzi[i]);
      const size_t mem = (size_t)rows * g.ld * (2 * (size_t)(k1 + 2 * kz) + kz + 8);
      if (g.cnt > 0 && mem > budget) break;
      g.rows = rows;
      g.k1 = k1;
      g.kz = kz;
      g.maxT = std::max(g.maxT, T[i]);
      ++g.cnt;
      ++j;
    }
    g.wide_res = g.maxT > 62 || g.kz > kCrtMax;
    groups.push_back(g);
  }
  // ---- device tables of every group: ints n, row0, T, prefix1, prefix2, inst; then pointers S, Z
  size_t nint = 0, nptr = 0;
  for (auto& g : groups) {
    g.tab_off = nint;
    nint += 3 * (size_t)g.cnt + 2 * (size_t)(g.cnt + 1) + g.cnt;
    g.ptr_off = nptr;
    nptr += 2 * (size_t)g.cnt;
  }
  const size_t ptr_bytes_off = (nint * sizeof(int) + 255) / 256 * 256;
  int st = ZFACT_OK;
  char* tab = (char*)ctx_buf(c, "gr.tab", ptr_bytes_off + nptr * sizeof(void*), &st);
  if (!tab) return st;
  std::vector<char> host(ptr_bytes_off + nptr * sizeof(void*), 0);
  int* hi = (int*)host.data();
  const double** hp = (const double**)(host.data() + ptr_bytes_off);
  for (auto& g : groups) {
    int* t = hi + g.tab_off;
    int row = 0;
    for (int q = 0; q < g.cnt; ++q) {
      const int i = order[g.first + q];
      t[q] = n[i];
      t[g.cnt + q] = row;
      t[2 * g.cnt + q] = T[i];
      row += rup(n[i], 256);
      int* pre1 = t + 3 * g.cnt;
      pre1[q + 1] = pre1[q] + tiles256(n[i], false) * g.k1;
      t[3 * g.cnt + 2 * (g.cnt + 1) + q] = q;  // slot q is instance q of the group (largest first)
      hp[g.ptr_off + q] = S[i];
      hp[g.ptr_off + g.cnt + q] = Z[i];
    }
  }
  if ((st = ctx_cuda(c, cudaMemcpyAsync(tab, host.data(), host.size(), cudaMemcpyHostToDevice, c->stream),
                     "grouped tables")))
    return st;
  if ((st = ctx_cuda(c, cudaStreamSynchronize(c->stream), "grouped tables sync"))) return st;


  // ---- two buffer sets (lane 0 and 1, each sized for the largest group), one stream each: group g runs on
  // set g % 2, so one group's products overlap the other's reconstruction and residues
  size_t rmax = 0, res_elems = 0, g_bytes = 0, a64_elems = 0, nparts = 0;
  int cmax_n = 0;
  for (auto& g : groups) {
    const size_t e = (size_t)g.rows * g.ld;
    rmax = std::max(rmax, (size_t)g.rows);
    res_elems = std::max(res_elems, e * (size_t)(g.k1 + 2 * g.kz));
    g_bytes = std::max(g_bytes, e * (size_t)g.kz);
    a64_elems = std::max(a64_elems, e);
    cmax_n = std::max(cmax_n, g.cnt);
    nparts = std::max(nparts, (size_t)g.cnt * ozm_combine_blocks(g.max_n));
  }
  struct Set {
    uint16_t* R;
    uint8_t* G;
    double* A64;
    int* E;
    unsigned long long* cmax;
    unsigned int* rho;
    double* parts;
    int* hbuf;  // pinned: rho read-back (cmax_n words), then the second product's prefix (cmax_n + 1)
    cudaStream_t s;
    cudaEvent_t ev;
  } sets[2];
  const size_t pin_words = 2 * (2 * (size_t)cmax_n + 2);
  if (c->gr_pinned_n < pin_words) {
    if (c->gr_pinned) cudaFreeHost(c->gr_pinned);
    c->gr_pinned = nullptr;
    c->gr_pinned_n = 0;
    if (cudaMallocHost(&c->gr_pinned, sizeof(int) * pin_words) != cudaSuccess)
      return ctx_fail(c, ZFACT_ERR_NOMEM, "pinned host words for the grouped residuals");
    c->gr_pinned_n = pin_words;
  }
  double* err = (double*)ctx_buf(c, "gr.err", sizeof(double) * (size_t)count, &st);
  if (!err) return st;
  for (int l = 0; l < 2; ++l) {
    if (!c->lane_stream[l] && cudaStreamCreateWithFlags(&c->lane_stream[l], cudaStreamNonBlocking) != cudaSuccess)
      return ctx_fail(c, ZFACT_ERR_CUDA, "lane stream");
    Set& b = sets[l];
    c->lane = l;
    b.R = (uint16_t*)ctx_buf(c, lane_name(c, "gr.res").c_str(), sizeof(uint16_t) * res_elems, &st);
    b.G = b.R ? (uint8_t*)ctx_buf(c, lane_name(c, "gr.G").c_str(), g_bytes, &st) : nullptr;
    b.A64 = b.G ? (double*)ctx_buf(c, lane_name(c, "gr.A64").c_str(), sizeof(double) * a64_elems, &st) : nullptr;
    b.E = b.A64 ? (int*)ctx_buf(c, lane_name(c, "gr.e").c_str(), sizeof(int) * 3 * rmax, &st) : nullptr;
    b.cmax = b.E ? (unsigned long long*)ctx_buf(c, lane_name(c, "gr.cmax").c_str(), 8 * rmax, &st) : nullptr;
    b.rho = b.cmax ? (unsigned int*)ctx_buf(c, lane_name(c, "gr.rho").c_str(), 4 * (size_t)cmax_n, &st) : nullptr;
    b.parts = b.rho ? (double*)ctx_buf(c, lane_name(c, "gr.parts").c_str(), 8 * nparts, &st) : nullptr;
    c->lane = -1;
    if (!b.parts) return st;
    b.hbuf = c->gr_pinned + (size_t)l * (2 * (size_t)cmax_n + 2);
    b.s = c->lane_stream[l];
  }

  // the plan of exactly k moduli: the sixteen-moduli one where k fits it, else the wider set's
  struct Plans {
    CrtPlan p;
    crtw::Plan wp;
    bool wide;
    float fw[32];
  };
  auto make_plan = [&](int k, Plans* pl) -> int {
    double bits = 0.0;  // the first k - 1 moduli's bits, summed as the planners sum them: they take k
    for (int t = 0; t + 1 < k; ++t) bits += log2((double)crtw::modulus(t));
    pl->wide = k > kCrtMax;
    const int got = pl->wide ? crtw::plan(bits, &pl->wp) : crt_plan(bits, &pl->p);
    if (got != k) return ctx_fail(c, ZFACT_ERR_ARG, "no plan for %d moduli", k);
    for (int t = 0; t < k; ++t) pl->fw[t] = pl->wide ? pl->wp.fw[t] : pl->p.fw[t];
    return ZFACT_OK;
  };
  struct Run {
    int* dt;
    size_t plane;
    uint16_t *RS, *RZ, *RA;
    int *eS, *eZ, *eA;
    GroupRes gS, gZ, gA;
    Plans p1, p2;
    int k2;
  };
  std::vector<Run> runs(groups.size());
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const Group& g = groups[gi];
    const Set& b = sets[gi & 1];
    Run& r = runs[gi];
    r.dt = (int*)tab + g.tab_off;
    const double* const* dS = (const double* const*)(tab + ptr_bytes_off) + g.ptr_off;
    r.plane = (size_t)g.rows * g.ld;
    r.RS = b.R;
    r.RZ = r.RS + r.plane * g.k1;
    r.RA = r.RZ + r.plane * g.kz;
    r.eS = b.E;
    r.eZ = b.E + g.rows;
    r.eA = b.E + 2 * g.rows;
    GroupRes gb{};
    gb.n = r.dt;
    gb.row0 = r.dt + g.cnt;
    gb.T = r.dt + 2 * g.cnt;
    gb.count = g.cnt;
    gb.max_n = g.max_n;
    r.gS = r.gZ = r.gA = gb;
    r.gS.src = dS;
    r.gS.e = r.eS;
    r.gZ.src = dS + g.cnt;
    r.gZ.e = r.eZ;
    r.gA.packed = b.A64;
    r.gA.ldp = g.ld;
    r.gA.e = r.eA;
    if ((st = make_plan(g.k1, &r.p1))) return st;
  }
  cudaEvent_t fork = ev_get(c);
  for (int l = 0; l < 2; ++l) sets[l].ev = ev_get(c);
  cudaMemsetAsync(c->st_dev, 0, sizeof(IterState), c->stream);  // error flag of the products
  cudaEventRecord(fork, c->stream);  // the lanes start after the bulk and the tables
  for (int l = 0; l < 2; ++l) cudaStreamWaitEvent(sets[l].s, fork, 0);

  // one grouped residue product over k moduli: A's planes (rows of Z_i^T) against B's, digits into G
  auto product = [&](const Group& g, const Run& r, const Set& b, bool sym, int k, const uint16_t* Ap, int kA,
                     const uint16_t* Bp, int kB, const int* prefix, int units, const float* fw) -> int {
    TcMaps maps;
    memset(&maps, 0, sizeof(maps));
    int r1 = ctx_make_map(c, &maps.a[0], Ap, kA * g.rows, g.ld, g.ld, 128, true);
    int r2 = ctx_make_map(c, &maps.b[0], Bp, kB * g.rows, g.ld, g.ld, 256, true);
    if (r1 || r2) return ctx_fail(c, ZFACT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d, %d)", r1, r2);
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.M = units;
    a.N = a.K = g.max_n;
    a.nseg = 1;
    a.sym = sym ? 1 : 0;
    a.epi = kEpiCrt8;
    a.bf16 = 1;
    a.unscale = 1.0f;
    a.d8 = b.G;
    a.ld32 = g.ld;
    a.g_stride = r.plane;
    for (int t = 0; t < k; ++t) a.crt_w[t] = fw[t];
    a.oz_s = k;
    a.oz_diag = 1;
    a.oz_nch = 1;
    a.oz_chunk_kb = (g.max_n + 63) / 64;  // every unit runs over its instance's whole K
    a.oz_sub_kb = chunk_kb;               // in exact sub-chunks reduced in the epilogue
    a.oz_ra = g.rows;
    a.oz_rb = g.rows;
    a.ninst = g.cnt;
    a.g_prefix = prefix;
    a.g_inst = r.dt + 3 * g.cnt + 2 * (g.cnt + 1);
    a.g_n = r.gS.n;
    a.g_row0 = r.gS.row0;
    a.err_flag = &c->st_dev->error;
    double flops = 0.0;
    for (int q = 0; q < g.cnt; ++q) {
      const double nq = n[order[g.first + q]];
      flops += k * 2.0 * nq * nq * nq * (sym ? 0.5 : 1.0);
      kstat_note(c, "fp64_equiv", 2.0 * nq * nq * nq * (sym ? 0.5 : 1.0));
    }
    return ctx_cuda(c, klaunch(c, "tc_gemm.crt", flops, 0, 1,
                               [&] { return launch_tc_gemm(a, maps, 256, c->num_sms, b.s); }),
                    "grouped residue products");
  };
  auto combine = [&](const Group& g, const Run& r, const Set& b, const Plans& pl, const int* eA_, const int* eB_,
                     double* out, int mode, bool sym, double* partials) -> int {
    return ctx_cuda(c, klaunch(c, pl.wide ? "oz_crt.wide" : "oz_crt", 0, 0, 1, [&] {
                      return pl.wide ? launch_gozmw_combine8(b.G, r.plane, g.ld, pl.wp, r.gZ, eA_, eB_, out, g.ld,
                                                             mode, sym, partials, b.s)
                                     : launch_gozm_combine8(b.G, r.plane, g.ld, pl.p, r.gZ, eA_, eB_, out, g.ld, mode,
                                                            sym, partials, b.s);
                    }),
                    "grouped reconstruction");
  };
  auto rows_res = [&](const Group& g, const Run& r, const Set& b, const GroupRes& gr, int k, uint16_t* out) {
    return g.wide_res ? launch_gozmw_rowres(gr, k, out, g.ld, r.plane, b.s)
                      : launch_gozm_rowres(gr, k, out, g.ld, r.plane, g.maxT, b.s);
  };

  // phase A of a group: residues of S_i and Z_i^T, A_i^T = Z_i^T S_i reconstructed into A, A's row norms
  // read back into pinned words (event)
  auto phase_a = [&](size_t gi) -> int {
    const Group& g = groups[gi];
    const Run& r = runs[gi];
    Set& b = sets[gi & 1];
    c->lane = (int)(gi & 1);  // per-launch events (profiling) on this lane's stream
    int s2 = ctx_cuda(c, klaunch(c, "oz_residues", 0, 0, 5, [&] {
                        cudaError_t e = rows_res(g, r, b, r.gS, g.k1, r.RS);
                        if (e == cudaSuccess) e = launch_gozm_colexp(r.gZ, b.cmax, g.rows, b.s);
                        if (e == cudaSuccess)
                          e = g.wide_res ? launch_gozmw_tres(r.gZ, g.kz, r.RZ, g.ld, r.plane, b.s)
                                         : launch_gozm_tres(r.gZ, g.kz, r.RZ, g.ld, r.plane, g.maxT, b.s);
                        return e;
                      }),
                      "grouped residues");
    if (!s2)
      s2 = product(g, r, b, false, g.k1, r.RZ, g.kz, r.RS, g.k1, r.dt + 3 * g.cnt,
                   hi[g.tab_off + 3 * g.cnt + g.cnt], r.p1.fw);
    if (!s2) s2 = combine(g, r, b, r.p1, r.eZ, r.eS, b.A64, 0, false, nullptr);
    if (!s2)
      s2 = ctx_cuda(c, klaunch(c, "oz_rho", 0, 0, 1, [&] { return launch_gozm_rowrho(r.gA, b.rho, b.s); }),
                    "grouped rho A");
    if (!s2)
      s2 = ctx_cuda(c, cudaMemcpyAsync(b.hbuf, b.rho, sizeof(unsigned int) * (size_t)g.cnt, cudaMemcpyDeviceToHost,
                                       b.s),
                    "grouped rho read-back");
    if (!s2) s2 = ctx_cuda(c, cudaEventRecord(b.ev, b.s), "grouped rho event");
    c->lane = -1;
    return s2;
  };
  // phase B: the second product's moduli from A's norms, A's residues, X_i = Z_i^T A_i on upper tiles with
  // d = I - X fused (Err partials only), Err per instance
  auto phase_b = [&](size_t gi) -> int {
    const Group& g = groups[gi];
    Run& r = runs[gi];
    Set& b = sets[gi & 1];
    int s2 = ctx_cuda(c, cudaEventSynchronize(b.ev), "grouped rho wait");
    if (s2) return s2;
    int k2 = 1;
    for (int q = 0; q < g.cnt; ++q) {
      const int i = order[g.first + q];
      bool w = false;
      const double bits = oz_product_bits(T[i], T[i], rho_z[i], oz_rho_from((unsigned int)b.hbuf[q], n[i]), n[i]);
      const int kq = count_of(c, T[i], bits, &w);
      k2 = std::max(k2, kq < 1 ? g.kz : kq);
    }
    r.k2 = std::min(k2, g.kz);
    if ((s2 = make_plan(r.k2, &r.p2))) return s2;
    int* pre2 = b.hbuf + cmax_n;  // pinned: the copy below reads it after this function returns
    pre2[0] = 0;
    for (int q = 0; q < g.cnt; ++q) pre2[q + 1] = pre2[q] + tiles256(n[order[g.first + q]], true) * r.k2;
    int* dpre2 = r.dt + 3 * g.cnt + (g.cnt + 1);
    c->lane = (int)(gi & 1);
    s2 = ctx_cuda(c, cudaMemcpyAsync(dpre2, pre2, sizeof(int) * (size_t)(g.cnt + 1), cudaMemcpyHostToDevice, b.s),
                  "grouped prefix");
    if (!s2)
      s2 = ctx_cuda(c, klaunch(c, "oz_residues", 0, 0, 1, [&] { return rows_res(g, r, b, r.gA, r.k2, r.RA); }),
                    "grouped residues A");
    if (!s2) s2 = product(g, r, b, true, r.k2, r.RZ, g.kz, r.RA, r.k2, dpre2, pre2[g.cnt], r.p2.fw);
    if (!s2) s2 = combine(g, r, b, r.p2, r.eZ, r.eA, nullptr, 2, true, b.parts);
    if (!s2)
      s2 = ctx_cuda(c, klaunch(c, "finish_err", 0, 0, 1, [&] {
                      return launch_gozm_finish(b.parts, ozm_combine_blocks(g.max_n), g.cnt, err + g.first, b.s);
                    }),
                    "grouped Err");
    c->lane = -1;
    return s2;
  };

  // group g + 1's residues and first product run while the host waits for group g's norms; group g's second
  // product then overlaps group g + 1's reconstruction
  auto release = [&] {
    c->ev_pool.push_back(fork);
    for (int l = 0; l < 2; ++l) c->ev_pool.push_back(sets[l].ev);
  };
  st = phase_a(0);
  for (size_t gi = 0; !st && gi < groups.size(); ++gi) {
    if (gi + 1 < groups.size()) st = phase_a(gi + 1);
    if (!st) st = phase_b(gi);
  }
  if (st) {
    // leave no work of these buffers in flight before handing the error back
    for (int l = 0; l < 2; ++l) cudaStreamSynchronize(sets[l].s);
    release();
    return st;
  }
  for (int l = 0; l < 2; ++l) {
    cudaEventRecord(sets[l].ev, sets[l].s);
    cudaStreamWaitEvent(c->stream, sets[l].ev, 0);
  }
  std::vector<double> herr(count);
  st = ctx_cuda(c, cudaMemcpyAsync(herr.data(), err, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost,
                                   c->stream),
                "grouped residuals");
  if (!st) st = ctx_read_state(c);
  release();
  if (st) return st;
  for (int j = 0; j < count; ++j) resid[order[j]] = herr[j];
  *done = true;
  return ZFACT_OK;
}

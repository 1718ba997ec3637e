// FP64-accurate final residuals of the batched mode as grouped launches: every stage of the residual
// d_i = I - Z_i^T S_i Z_i (the residues of S_i's rows and of Z_i's columns, A_i^T = Z_i^T S_i, A_i's
// residues, X_i = Z_i^T A_i with the fused d = I - X and its Err) is one launch over a group of instances,
// as the bulk's products are.  Instances are grouped in the bulk's order (largest first) under a memory
// budget; within a group every operand's residue planes are stacked by instance along the rows of one
// packed buffer (instance i at row row0[i], one leading dimension), so one tensor map covers all of them and
// one persistent tcgen05 launch forms every instance's residue products (units: instance, modulus, tile).
// The moduli of a product are the largest any instance of the group asks for (each instance's from its
// measured row norms, as in the single-instance refinement).
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
  const size_t budget = (size_t)24 << 30;
  // ---- groups (bulk order, largest first) within the memory budget
  std::vector<Group> groups;
  std::vector<int> T(count), k1i(count), kzi(count);
  for (int j = 0; j < count; ++j) {
    const int i = order[j];
    T[i] = 6 * slices[i];
    if (n[i] > chunk_kb * 64 || T[i] > 83) return ZFACT_OK;  // outside the grouped form: lanes
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

  // ---- buffers, sized for the largest group
  size_t rmax = 0, res_elems = 0, g_bytes = 0;
  int cmax_n = 0;
  for (auto& g : groups) {
    const size_t e = (size_t)g.rows * g.ld;
    rmax = std::max(rmax, (size_t)g.rows);
    res_elems = std::max(res_elems, e * (size_t)(g.k1 + 2 * g.kz));
    g_bytes = std::max(g_bytes, e * (size_t)g.kz);
    cmax_n = std::max(cmax_n, g.cnt);
  }
  size_t a64_elems = 0;
  for (auto& g : groups) a64_elems = std::max(a64_elems, (size_t)g.rows * g.ld);
  uint16_t* R = (uint16_t*)ctx_buf(c, "gr.res", sizeof(uint16_t) * res_elems, &st);
  if (!R) return st;
  uint8_t* G = (uint8_t*)ctx_buf(c, "gr.G", g_bytes, &st);
  if (!G) return st;
  double* A64 = (double*)ctx_buf(c, "gr.A64", sizeof(double) * a64_elems, &st);
  if (!A64) return st;
  int* E = (int*)ctx_buf(c, "gr.e", sizeof(int) * 3 * rmax, &st);
  if (!E) return st;
  unsigned long long* cmax = (unsigned long long*)ctx_buf(c, "gr.cmax", sizeof(unsigned long long) * rmax, &st);
  if (!cmax) return st;
  unsigned int* rho = (unsigned int*)ctx_buf(c, "gr.rho", sizeof(unsigned int) * (size_t)cmax_n, &st);
  if (!rho) return st;
  double* err = (double*)ctx_buf(c, "gr.err", sizeof(double) * (size_t)count, &st);
  if (!err) return st;
  size_t nparts = 0;
  for (auto& g : groups) nparts = std::max(nparts, (size_t)g.cnt * ozm_combine_blocks(g.max_n));
  double* parts = (double*)ctx_buf(c, "gr.parts", sizeof(double) * nparts, &st);
  if (!parts) return st;

  std::vector<unsigned int> hrho(cmax_n);
  for (auto& g : groups) {
    int* dt = (int*)tab + g.tab_off;
    const double* const* dS = (const double* const*)(tab + ptr_bytes_off) + g.ptr_off;
    const double* const* dZ = dS + g.cnt;
    const size_t plane = (size_t)g.rows * g.ld;
    uint16_t* RS = R;
    uint16_t* RZ = RS + plane * g.k1;
    uint16_t* RA = RZ + plane * g.kz;
    int *eS = E, *eZ = E + g.rows, *eA = E + 2 * g.rows;
    GroupRes gb{};
    gb.n = dt;
    gb.row0 = dt + g.cnt;
    gb.T = dt + 2 * g.cnt;
    gb.count = g.cnt;
    gb.max_n = g.max_n;
    GroupRes gS = gb, gZ = gb, gA = gb;
    gS.src = dS;
    gS.e = eS;
    gZ.src = (const double* const*)dZ;
    gZ.e = eZ;
    gA.packed = A64;
    gA.ldp = g.ld;
    gA.e = eA;
    auto rows_res = [&](const GroupRes& gr, int k, uint16_t* out) -> cudaError_t {
      return g.wide_res ? launch_gozmw_rowres(gr, k, out, g.ld, plane, c->stream)
                        : launch_gozm_rowres(gr, k, out, g.ld, plane, g.maxT, c->stream);
    };
    // residues of S_i's rows and of Z_i's columns
    if ((st = ctx_cuda(c, klaunch(c, "oz_residues", 0, 0, 5, [&] {
                         cudaError_t e = rows_res(gS, g.k1, RS);
                         if (e == cudaSuccess) e = launch_gozm_colexp(gZ, cmax, g.rows, c->stream);
                         if (e == cudaSuccess)
                           e = g.wide_res ? launch_gozmw_tres(gZ, g.kz, RZ, g.ld, plane, c->stream)
                                          : launch_gozm_tres(gZ, g.kz, RZ, g.ld, plane, g.maxT, c->stream);
                         return e;
                       }),
                       "grouped residues")))
      return st;
    // one grouped residue product over k moduli: A's planes (rows of Z_i^T) against B's, digits into G
    auto product = [&](bool sym, int k, const uint16_t* Ap, int kA, const uint16_t* Bp, int kB, const int* prefix,
                       int units, const float* fw) -> int {
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
      a.d8 = G;
      a.ld32 = g.ld;
      a.g_stride = plane;
      for (int t = 0; t < k; ++t) a.crt_w[t] = fw[t];
      a.oz_s = k;
      a.oz_diag = 1;
      a.oz_nch = 1;
      a.oz_chunk_kb = chunk_kb;
      a.oz_ra = g.rows;
      a.oz_rb = g.rows;
      a.ninst = g.cnt;
      a.g_prefix = prefix;
      a.g_inst = dt + 3 * g.cnt + 2 * (g.cnt + 1);
      a.g_n = gb.n;
      a.g_row0 = gb.row0;
      a.err_flag = &c->st_dev->error;
      double flops = 0.0;
      for (int q = 0; q < g.cnt; ++q) {
        const double nq = n[order[g.first + q]];
        flops += k * 2.0 * nq * nq * nq * (sym ? 0.5 : 1.0);
        kstat_note(c, "fp64_equiv", 2.0 * nq * nq * nq * (sym ? 0.5 : 1.0));
      }
      return ctx_cuda(c, klaunch(c, "tc_gemm.crt", flops, 0, 1,
                                 [&] { return launch_tc_gemm(a, maps, 256, c->num_sms, c->stream); }),
                      "grouped residue products");
    };
    // the plan of exactly k moduli (the twenty-moduli one where k fits it, else the wider set's) and the
    // reconstruction with it
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
    auto combine = [&](const Plans& pl, const int* eA_, const int* eB_, double* out, int mode, bool sym,
                       double* partials) -> int {
      return ctx_cuda(c, klaunch(c, pl.wide ? "oz_crt.wide" : "oz_crt", 0, 0, 1, [&] {
                        return pl.wide ? launch_gozmw_combine8(G, plane, g.ld, pl.wp, gZ, eA_, eB_, out, g.ld, mode,
                                                               sym, partials, c->stream)
                                       : launch_gozm_combine8(G, plane, g.ld, pl.p, gZ, eA_, eB_, out, g.ld, mode, sym,
                                                              partials, c->stream);
                      }),
                      "grouped reconstruction");
    };
    // A_i^T = Z_i^T S_i over k1 moduli, reconstructed into the packed FP64 A
    Plans p1, p2;
    if ((st = make_plan(g.k1, &p1))) return st;
    if ((st = product(false, g.k1, RZ, g.kz, RS, g.k1, dt + 3 * g.cnt, hi[g.tab_off + 3 * g.cnt + g.cnt], p1.fw)))
      return st;
    if ((st = combine(p1, eZ, eS, A64, 0, false, nullptr))) return st;
    // the scaled row norms of every A_i set the second product's moduli (one read-back per group)
    if ((st = ctx_cuda(c, klaunch(c, "oz_rho", 0, 0, 1, [&] { return launch_gozm_rowrho(gA, rho, c->stream); }),
                       "grouped rho A")))
      return st;
    cudaMemcpyAsync(hrho.data(), rho, sizeof(unsigned int) * (size_t)g.cnt, cudaMemcpyDeviceToHost, c->stream);
    if ((st = ctx_cuda(c, cudaStreamSynchronize(c->stream), "grouped rho read-back"))) return st;
    int k2 = 1;
    for (int q = 0; q < g.cnt; ++q) {
      const int i = order[g.first + q];
      bool w = false;
      const double b = oz_product_bits(T[i], T[i], rho_z[i], oz_rho_from(hrho[q], n[i]), n[i]);
      const int kq = count_of(c, T[i], b, &w);
      k2 = std::max(k2, kq < 1 ? g.kz : kq);
    }
    k2 = std::min(k2, g.kz);
    // units of the symmetric products
    std::vector<int> pre2(g.cnt + 1, 0);
    for (int q = 0; q < g.cnt; ++q) pre2[q + 1] = pre2[q] + tiles256(n[order[g.first + q]], true) * k2;
    int* dpre2 = dt + 3 * g.cnt + (g.cnt + 1);
    if ((st = ctx_cuda(c, cudaMemcpyAsync(dpre2, pre2.data(), sizeof(int) * pre2.size(), cudaMemcpyHostToDevice,
                                          c->stream),
                       "grouped prefix")))
      return st;
    if ((st = ctx_cuda(c, klaunch(c, "oz_residues", 0, 0, 1, [&] { return rows_res(gA, k2, RA); }),
                       "grouped residues A")))
      return st;
    // X_i = Z_i^T A_i on upper tiles over k2 moduli, d = I - X fused into the reconstruction: Err only
    if ((st = make_plan(k2, &p2))) return st;
    if ((st = product(true, k2, RZ, g.kz, RA, k2, dpre2, pre2[g.cnt], p2.fw))) return st;
    if ((st = combine(p2, eZ, eA, nullptr, 2, true, parts))) return st;
    if ((st = ctx_cuda(c, klaunch(c, "finish_err", 0, 0, 1, [&] {
                         return launch_gozm_finish(parts, ozm_combine_blocks(g.max_n), g.cnt, err + g.first, c->stream);
                       }),
                       "grouped Err")))
      return st;
  }
  std::vector<double> herr(count);
  cudaMemcpyAsync(herr.data(), err, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, c->stream);
  if ((st = ctx_read_state(c))) return st;
  for (int j = 0; j < count; ++j) resid[order[j]] = herr[j];
  *done = true;
  return ZFACT_OK;
}

// Host driver of the FP64-accurate products used by the refinement of Algorithm 3:
// d = I - Z^T S Z and Z <- Z + Z Q formed to FP64 accuracy on the BF16 tensor cores instead
// of GB300's ~1.1 TFLOP/s FP64 pipe, by CRT residues (k_ozmod.cu) where the product bound fits
// the moduli, else by error-free slices (k_ozaki.cu).
#include <math.h>
#include <string.h>

#include <string>

#include "ctx.h"
#include "kernels.h"
#include "tc_gemm.h"

using namespace zf;

namespace {

constexpr int kOzBits = 6;             // bits per slice
constexpr int kOzSlicesResid = 9;      // 54 bits: residual products of a well-scaled Z
constexpr int kOzSlicesUpdateMin = 4;  // 24 bits: the least Z Q is formed with (see oz_update_slices)
constexpr int kOzSlicesMax = 14;
// Target bytes of the slicing products' group partials per launch: K-chunks are batched up to it.  One
// K-chunk of every group is the least a launch holds, so a product may exceed it: the FP32 partials of one
// slicing chunk take 4 s N^2 bytes (up to 15 GB for 14 slices at N = 16384).  The CRT products keep one digit
// plane per modulus whatever K is, k N^2 bytes (6.4 GB for 24 moduli at N = 16384).  Both fit GB300's HBM
// many times over, and a workspace cap (zfact_set_workspace_limit) turns them into ZFACT_ERR_NOMEM before
// anything is allocated.
constexpr size_t kOzGBudget = (size_t)6 << 30;

struct OzOperand {
  uint16_t* sl = nullptr;
  int* e = nullptr;
  int Rp = 0, s = 0;  // s planes: slices, or CRT residues when nmod > 0
  int T = 0, nmod = 0;  // residues: fixed-point bits of the rows, moduli count (= s)
  int wide = 0;         // residues modulo the wider moduli of crt_wide.h
};


int ld16_of(int n) { return (n + 63) / 64 * 64; }
int rp_of(int n) { return (n + 255) / 256 * 256; }

// K-blocks per chunk: every group sum stays an integer below 2^24.  A group t holds
// pairs with |a_0| <= 2^b, |a_p| <= 2^(b-1) (p >= 1), so its sum over K terms is at
// most K 2^(2b) (1 + (t-1)/4) for t >= 1 and K 2^(2b) for t = 0.
int chunk_kb(int s) {
  const double worst = 1.0 + (s - 2) / 4.0;
  const double kmax = ldexp(1.0, 24 - 2 * kOzBits) / (worst > 1.0 ? worst : 1.0);
  int kb = (int)floor(kmax / 64.0);
  return kb < 1 ? 1 : kb;
}

int oz_make(zfact_ctx* c, const char* name, const double* X, int n, int ldx, bool trans, int s, OzOperand* op) {
  int st = ZFACT_OK;
  const int ld16 = ld16_of(n), Rp = rp_of(n);
  std::string ns = lane_name(c, (std::string("oz.") + name + ".sl").c_str()),
              ne = lane_name(c, (std::string("oz.") + name + ".e").c_str());
  op->sl = (uint16_t*)ctx_buf(c, ns.c_str(), sizeof(uint16_t) * (size_t)s * Rp * ld16, &st);
  if (!op->sl) return st;
  // the exponents, then the scratch of the column-statistics passes
  const size_t e_bytes = (sizeof(int) * (size_t)n + 15) / 16 * 16;
  op->e = (int*)ctx_buf(c, ne.c_str(), e_bytes + oz_colstats_scratch_bytes(n), &st);
  if (!op->e) return st;
  op->Rp = Rp;
  op->s = s;
  if ((st = ctx_cuda(c, klaunch(c, "oz_slice", 0, 8.0 * n * n * 2 + 2.0 * s * n * n, 2, [&] {
                       cudaError_t e = launch_oz_exp(X, n, ldx, trans, op->e, (char*)op->e + e_bytes, cur_stream(c));
                       if (e != cudaSuccess) return e;
                       return launch_oz_slice(X, n, ldx, trans, op->e, s, kOzBits, op->sl, ld16, Rp, cur_stream(c));
                     }),
                     "oz slice")))
    return st;
  return ZFACT_OK;
}

// Bits the moduli product must exceed for C' = F_A F_B^T of T_A- and T_B-bit operand rows with scaled row
// norms at most rhoA, rhoB (rho_r = ||x_r||_2 2^-e_r < sqrt(K)): by Cauchy-Schwarz |C'_ij| <= ||f_i|| ||g_j||,
// and rounding the rows to integers adds at most sqrt(K)/2 to each norm, so |C'| <= 2^(T_A + T_B) rA rB with
// r = rho + sqrt(K) 2^(-T-1); M must exceed four times that.  Never more than the bound K 2^(T_A + T_B)
// that holds for any rows (rho = sqrt(K)).
double oz_prod_bits(int TA, int TB, double rhoA, double rhoB, int n) {
  const double sq = sqrt((double)n);
  const double worst = TA + TB + log2((double)n) + 2.0;
  // an unknown (negative) or implausible norm takes the bound for any rows
  if (!(rhoA >= 0.0 && rhoA <= sq)) rhoA = sq;
  if (!(rhoB >= 0.0 && rhoB <= sq)) rhoB = sq;
  const double ra = rhoA + sq * ldexp(1.0, -TA - 1), rb = rhoB + sq * ldexp(1.0, -TB - 1);
  const double b = TA + TB + log2(ra * rb) + 2.0;
  return b < worst ? b : worst;
}

// Moduli for a product of `bits`: the sixteen of crt.h where they suffice, else the wider ones
// (*wide = 1), else 0 (the product needs slices).
int oz_moduli_for(const zfact_ctx* c, int TA, int TB, double bits, int* wide) {
  *wide = 0;
  if (c->oz_scheme == ZFACT_EMU_SLICES || TA < 1 || TB < 1 || TA > 83 || TB > 83) return 0;
  CrtPlan p;
  int k = crt_plan(bits, &p);
  if (k > 0) return k;
  crtw::Plan wp;
  k = crtw::plan(bits, &wp);
  if (k > 0) *wide = 1;
  return k;
}

}  // namespace

// rho from the FP32 pattern of max_r rho_r^2 that launch_ozm_rho wrote (an FP32 sum whose result lies at
// most (n/8 + 40) 2^-23 below the exact one, enlarged here by twice that); -1 when there is no bound.
double oz_rho_from(unsigned int rho2_bits, int n) {
  float t;
  memcpy(&t, &rho2_bits, sizeof(t));
  if (!(t >= 0.0f) || isinf(t)) return -1.0;
  return sqrt((double)t * (1.0 + (n / 8.0 + 40.0) * ldexp(1.0, -22)));
}

// The bound and moduli choice of the products above, for the grouped residuals of the batched mode.
double oz_product_bits(int TA, int TB, double rhoA, double rhoB, int n) { return oz_prod_bits(TA, TB, rhoA, rhoB, n); }
int oz_moduli_count(const zfact_ctx* c, int TA, int TB, double bits, int* wide) {
  return oz_moduli_for(c, TA, TB, bits, wide);
}
int oz_crt_chunk_kb() { return kCrtSubKb; }

namespace {

int oz_make_mod(zfact_ctx* c, const char* name, const double* X, int n, int ldx, bool trans, int T, int nmod,
                int wide, OzOperand* op) {
  int st = ZFACT_OK;
  const int ld16 = ld16_of(n), Rp = rp_of(n);
  std::string ns = lane_name(c, (std::string("oz.") + name + ".sl").c_str()),
              ne = lane_name(c, (std::string("oz.") + name + ".e").c_str());
  op->sl = (uint16_t*)ctx_buf(c, ns.c_str(), sizeof(uint16_t) * (size_t)nmod * Rp * ld16, &st);
  if (!op->sl) return st;
  // the exponents, then the scratch of the column-statistics passes
  const size_t e_bytes = (sizeof(int) * (size_t)n + 15) / 16 * 16;
  op->e = (int*)ctx_buf(c, ne.c_str(), e_bytes + oz_colstats_scratch_bytes(n), &st);
  if (!op->e) return st;
  op->Rp = Rp;
  op->s = nmod;
  op->T = T;
  op->nmod = nmod;
  // the sixteen-moduli kernel holds rows of up to 62 bits; wider rows or more planes take the wide one
  // (both write the same residues of the same fixed-point rows)
  wide = (wide || T > 62 || nmod > kCrtMax) ? 1 : 0;
  op->wide = wide;
  if ((st = ctx_cuda(c, klaunch(c, wide ? "oz_residues.wide" : "oz_residues", 0, 8.0 * n * n + 2.0 * nmod * n * n, 2, [&] {
                       cudaError_t e = launch_oz_exp(X, n, ldx, trans, op->e, (char*)op->e + e_bytes, cur_stream(c));
                       if (e != cudaSuccess) return e;
                       if (wide)
                         return launch_ozmw_residues(X, n, ldx, trans, op->e, T, nmod, op->sl, ld16, Rp, cur_stream(c));
                       return launch_ozm_residues(X, n, ldx, trans, op->e, T, nmod, op->sl, ld16, Rp, cur_stream(c));
                     }),
                     "oz residues")))
    return st;
  return ZFACT_OK;
}

// out (mode 0: =, 1: +=, fused 2: I - .) A B^T to FP64 accuracy from the CRT residues of A and B:
// one tensor-core product per modulus (group t = pair (t, t)) whose epilogue keeps only the CRT
// digit of each entry (one byte), then the reconstruction from the digits.  A fused residual writes
// *nparts Err partials.
int oz_product_mod(zfact_ctx* c, const OzOperand& A, const OzOperand& B, int n, bool sym, double* out, int ld64,
                   int mode, double bits, double* partials = nullptr, bool* fused_resid = nullptr,
                   int* nparts = nullptr) {
  int st = ZFACT_OK;
  CrtPlan plan;
  crtw::Plan wplan;
  // the first k moduli whose product exceeds 2^bits: crt.h's sixteen where they suffice, else the wider
  // moduli (the same sixteen first); the operands hold at least k residue planes
  bool wide = false;
  int k = crt_plan(bits, &plan);
  if (k < 1) {
    k = crtw::plan(bits, &wplan);
    wide = true;
  }
  if (k < 1 || k > A.nmod || k > B.nmod)
    return ctx_fail(c, ZFACT_ERR_ARG, "residue operands do not match (%d, %d, %d moduli)", k, A.nmod, B.nmod);
  const int ld = ld16_of(n);
  const int kblocks = (n + 63) / 64;
  // one digit plane per modulus: every unit runs over all of K, its exact FP32 sums of kCrtSubKb
  // K-blocks reduced modulo m and summed in the epilogue
  const size_t slot_bytes = (size_t)n * ld;
  uint8_t* G = (uint8_t*)ctx_buf(c, lane_name(c, "oz.G").c_str(), slot_bytes * k, &st);
  if (!G) return st;
  TcMaps maps;
  memset(&maps, 0, sizeof(maps));
  const int bn = 256;
  int r1 = ctx_make_map(c, &maps.a[0], A.sl, k * A.Rp, n, ld, 128, true);
  int r2 = ctx_make_map(c, &maps.b[0], B.sl, k * B.Rp, n, ld, bn, true);
  if (r1 || r2) return ctx_fail(c, ZFACT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d, %d)", r1, r2);
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.M = a.N = a.K = n;
  a.nseg = 1;
  a.sym = sym ? 1 : 0;
  a.epi = kEpiCrt8;
  a.bf16 = 1;
  a.unscale = 1.0f;
  a.d8 = G;
  a.ld32 = ld;
  a.g_stride = (size_t)n * ld;
  for (int t = 0; t < k; ++t) a.crt_w[t] = wide ? wplan.fw[t] : plan.fw[t];
  a.oz_s = k;
  a.oz_diag = 1;
  a.oz_nch = 1;
  a.oz_chunk_kb = kblocks;
  a.oz_sub_kb = kCrtSubKb;
  a.oz_c0 = 0;
  a.oz_ra = A.Rp;
  a.oz_rb = B.Rp;
  a.oz_tiles = tc_num_units(a, bn) / k;
  a.err_flag = &c->st_dev->error;
  // algorithmic work: k residue products
  const double flops = k * 2.0 * n * n * (double)n * (sym ? 0.5 : 1.0);
  const double bytes = k * 2.0 * 2.0 * n * (double)n + 1.0 * k * (double)n * n * (sym ? 0.5 : 1.0);
  kstat_note(c, "fp64_equiv", flops / k);
  if ((st = ctx_cuda(c, klaunch(c, "tc_gemm.crt", flops, bytes, 1,
                                [&] { return launch_tc_gemm(a, maps, bn, c->num_sms, cur_stream(c)); }),
                     "tcgen05 residue products")))
    return st;
  int md = mode;
  if (partials && fused_resid && sym) {
    md = 2;
    *fused_resid = true;
    if (nparts) *nparts = ozm_combine_blocks(n);
  }
  // digits read (the upper triangle when sym), FP64 result written (read too when accumulating)
  const double cbytes = (1.0 * k * n * (double)n + (md == 1 ? 16.0 : 8.0) * n * n) * (sym ? 0.5 : 1.0);
  if ((st = ctx_cuda(c, klaunch(c, wide ? "oz_crt.wide" : "oz_crt", 0, cbytes, 1, [&] {
                       if (wide)
                         return launch_ozmw_combine8(G, (size_t)n * ld, ld, 1, wplan, A.e, B.e, A.T, B.T, n, out, ld64,
                                                     md, sym, partials, cur_stream(c), md == 2 ? c->oz_amax : nullptr);
                       return launch_ozm_combine8(G, (size_t)n * ld, ld, 1, plan, A.e, B.e, A.T, B.T, n, out, ld64, md,
                                                  sym, partials, cur_stream(c), md == 2 ? c->oz_amax : nullptr);
                     }),
                     "oz crt combine")))
    return st;
  return ZFACT_OK;
}

// out (mode 0: =, 1: +=) A B^T to FP64 accuracy, A and B given by their row slices.
// bits: what the moduli product must exceed (residue operands; oz_prod_bits), <= 0 for the bound that holds
// for any rows.
int oz_product(zfact_ctx* c, const OzOperand& A, const OzOperand& B, int n, bool sym, double* out, int ld64,
               int mode, double* partials = nullptr, bool* fused_resid = nullptr, int* nparts = nullptr,
               double bits = 0.0) {
  if (A.nmod > 0 || B.nmod > 0) {
    if (bits <= 0.0) bits = A.T + B.T + log2((double)n) + 2.0;
    return oz_product_mod(c, A, B, n, sym, out, ld64, mode, bits, partials, fused_resid, nparts);
  }
  if (nparts) *nparts = oz_combine_blocks(n);
  int st = ZFACT_OK;
  const int s = A.s < B.s ? A.s : B.s;
  const int ld = ld16_of(n);
  const int ckb = chunk_kb(s);
  const int kblocks = (n + 63) / 64;
  const int nch_total = (kblocks + ckb - 1) / ckb;
  const size_t slot_bytes = sizeof(float) * (size_t)n * ld;
  int nch_b = (int)(kOzGBudget / (slot_bytes * s));
  if (nch_b < 1) nch_b = 1;
  if (nch_b > nch_total) nch_b = nch_total;
  float* G = (float*)ctx_buf(c, lane_name(c, "oz.G").c_str(), slot_bytes * s * nch_b, &st);
  if (!G) return st;
  TcMaps maps;
  memset(&maps, 0, sizeof(maps));
  const int bn = 256;
  int r1 = ctx_make_map(c, &maps.a[0], A.sl, A.s * A.Rp, n, ld, 128, true);
  int r2 = ctx_make_map(c, &maps.b[0], B.sl, B.s * B.Rp, n, ld, bn, true);
  if (r1 || r2) return ctx_fail(c, ZFACT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d, %d)", r1, r2);
  for (int c0 = 0; c0 < nch_total; c0 += nch_b) {
    const int nch = (nch_total - c0) < nch_b ? (nch_total - c0) : nch_b;
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.M = a.N = a.K = n;
    a.nseg = 1;
    a.sym = sym ? 1 : 0;
    a.epi = kEpiG32;
    a.bf16 = 1;
    a.unscale = 1.0f;
    a.f32 = G;
    a.ld32 = ld;
    a.g_stride = (size_t)n * ld;
    a.oz_s = s;
    a.oz_nch = nch;
    a.oz_chunk_kb = ckb;
    a.oz_c0 = c0;
    a.oz_ra = A.Rp;
    a.oz_rb = B.Rp;
    a.oz_tiles = tc_num_units(a, bn) / (s * nch);
    a.err_flag = &c->st_dev->error;
    // algorithmic work: s(s+1)/2 slice pairs over this launch's share of K
    const int kb_lo = c0 * ckb, kb_hi = (c0 + nch) * ckb < kblocks ? (c0 + nch) * ckb : kblocks;
    const double kk = (double)(kb_hi - kb_lo) * 64.0 < n ? (double)(kb_hi - kb_lo) * 64.0 : (double)n;
    const double pairs = s * (s + 1) / 2.0;
    const double flops = pairs * 2.0 * n * n * kk * (sym ? 0.5 : 1.0);
    const double bytes = pairs * 2.0 * 2.0 * n * kk + 4.0 * s * nch * (double)n * n;
    kstat_note(c, "fp64_equiv", flops / pairs);
    if ((st = ctx_cuda(c, klaunch(c, "tc_gemm.ozaki", flops, bytes, 1,
                                  [&] { return launch_tc_gemm(a, maps, bn, c->num_sms, cur_stream(c)); }),
                       "tcgen05 ozaki")))
      return st;
    int md = (c0 == 0) ? mode : 1;
    // a symmetric product that fits one launch goes straight to d = I - X (fused residual)
    const bool fuse = partials && fused_resid && sym && c0 == 0 && nch == nch_total;
    if (fuse) {
      md = 2;
      *fused_resid = true;
    }
    const double cbytes = 4.0 * s * nch * n * (double)n + 16.0 * n * n;
    if ((st = ctx_cuda(c, klaunch(c, "oz_combine", 0, cbytes, 1, [&] {
                         return launch_oz_combine(G, (size_t)n * ld, ld, s, nch, kOzBits, A.e, B.e, n, out, ld64, md,
                                                  sym, partials, cur_stream(c));
                       }),
                       "oz combine")))
      return st;
  }
  return ZFACT_OK;
}

}  // namespace

// Slices per operand for FP64-level accuracy.  Row-scaled slicing is accurate relative to the
// row maxima: an entry of Z^T S Z carries an error ~ 2^(-b s) max|Z|^2 g_hi (g_hi the largest
// absolute row sum of S) where FP64 arithmetic errs by ~ 2^-53 |X_ij| ~ 2^-53.  So b s is made
// at least 53 + log2(max|Z|^2 g_hi) (9 slices for a well-scaled Z, more for an ill-conditioned S).
int oz_slices_for(double zmax, double g_hi) {
  double extra = log2(zmax * zmax * g_hi);
  if (!(extra > 0)) extra = 0;
  int s = (int)ceil((53.0 + extra) / kOzBits);
  if (s < kOzSlicesResid) s = kOzSlicesResid;
  if (s > kOzSlicesMax) s = kOzSlicesMax;
  return s;
}

// The residual's operands keep T = b s bits either way: as s slices, or as CRT residues of the
// T-bit rows where the product bound fits the moduli (then c->oz_nmod > 0).
int oz_prepare_S(zfact_ctx* c, const double* S, int n, int s, double rho_s) {
  OzOperand op;
  c->oz_s = s > 0 ? s : kOzSlicesResid;
  c->oz_T = kOzBits * c->oz_s;
  c->oz_rho_s = rho_s;
  // S's residue planes serve Z^T S for any Z (rho_Z <= sqrt(N)) of this factorization
  const double bits = oz_prod_bits(c->oz_T, c->oz_T, -1.0, rho_s, n);
  c->oz_nmod = oz_moduli_for(c, c->oz_T, c->oz_T, bits, &c->oz_wide);
  if (c->oz_nmod > 0) return oz_make_mod(c, "S", S, n, n, false, c->oz_T, c->oz_nmod, c->oz_wide, &op);
  return oz_make(c, "S", S, n, n, false, c->oz_s, &op);
}

namespace {
// An operand of the current residual products (slices or residues, as oz_prepare_S chose).
int oz_make_resid(zfact_ctx* c, const char* name, const double* X, int n, bool trans, OzOperand* op, int planes = 0,
                  int wide = 0) {
  if (c->oz_nmod > 0)
    return oz_make_mod(c, name, X, n, n, trans, c->oz_T, planes > 0 ? planes : c->oz_nmod, planes > 0 ? wide : c->oz_wide,
                       op);
  return oz_make(c, name, X, n, n, trans, c->oz_s, op);
}
}  // namespace

// d = I - Z^T S Z to FP64 accuracy; Err -> hist[idx].  oz_prepare_S must have run for this S.
int oz_residual(zfact_ctx* c, const double* Z, double* D, int n, int idx, int rule, double tol, int check_stop,
                double rho_zt) {
  int st = ZFACT_OK;
  OzOperand Sop, Zt, At;
  Sop.sl = (uint16_t*)ctx_buf(c, lane_name(c, "oz.S.sl").c_str(), 0, &st);
  Sop.e = (int*)ctx_buf(c, lane_name(c, "oz.S.e").c_str(), 0, &st);
  Sop.Rp = rp_of(n);
  Sop.s = c->oz_s;
  if (c->oz_nmod > 0) {
    Sop.s = Sop.nmod = c->oz_nmod;
    Sop.T = c->oz_T;
    Sop.wide = c->oz_wide;
  }
  double* A64 = (double*)ctx_buf(c, lane_name(c, "oz.At64").c_str(), sizeof(double) * (size_t)n * n, &st);
  if (!A64) return st;
  double* X64 = (double*)ctx_buf(c, lane_name(c, "oz.X64").c_str(), sizeof(double) * (size_t)n * n, &st);
  if (!X64) return st;
  int nb_fused = oz_combine_blocks(n);
  const int nb_sep = resid_from_x_blocks(n), nb_max = nb_fused > ozm_combine_blocks(n) ? nb_fused : ozm_combine_blocks(n);
  double* partials =
      (double*)ctx_buf(c, lane_name(c, "oz.partials").c_str(),
                       sizeof(double) * (size_t)(nb_max > nb_sep ? nb_max : nb_sep), &st);
  if (!partials) return st;
  // Moduli per product from the scaled row norms of its operands (oz_prod_bits): S's from oz_prepare_S,
  // Z's columns from the caller, A's rows measured below (one read-back) when the context runs on its
  // own stream; an unknown norm takes the bound for any rows.
  const int T = c->oz_T;
  double bits1 = 0.0, bits2 = 0.0;
  int planes_zt = 0, wide_zt = 0;
  if (c->oz_nmod > 0) {
    bits1 = oz_prod_bits(T, T, rho_zt, c->oz_rho_s, n);
    bits2 = oz_prod_bits(T, T, rho_zt, -1.0, n);
    planes_zt = oz_moduli_for(c, T, T, bits1 > bits2 ? bits1 : bits2, &wide_zt);
    if (planes_zt < 1) return ctx_fail(c, ZFACT_ERR_ARG, "no moduli for the residual products");
  }
  // rows of Z^T = columns of Z
  if ((st = oz_make_resid(c, "Zt", Z, n, true, &Zt, planes_zt, wide_zt))) return st;
  // A^T = Z^T S  (S symmetric: B operand rows are rows of S)
  if ((st = oz_product(c, Zt, Sop, n, false, A64, n, 0, nullptr, nullptr, nullptr, bits1))) return st;
  int planes_at = 0, wide_at = 0;
  if (c->oz_nmod > 0) {
    if (c->lane < 0 && rho_zt >= 0.0) {
      cudaMemsetAsync(&c->st_dev->rho2[3], 0, sizeof(unsigned int), c->stream);
      if ((st = ctx_cuda(c, klaunch(c, "oz_rho", 0, 8.0 * n * n, 1,
                                    [&] { return launch_ozm_rho(A64, n, n, false, &c->st_dev->rho2[3], nullptr, c->stream); }),
                         "rho A")))
        return st;
      if ((st = ctx_read_state(c))) return st;
      bits2 = oz_prod_bits(T, T, rho_zt, oz_rho_from(c->st_host->rho2[3], n), n);
    }
    planes_at = oz_moduli_for(c, T, T, bits2, &wide_at);
  }
  if ((st = oz_make_resid(c, "At", A64, n, false, &At, planes_at, wide_at))) return st;
  // X = Z^T A = Z^T (A^T)^T, symmetric tiles; d = I - X fused into the combine when possible
  bool fused = false;
  double* Xout = X64;
  // with residues the fused reconstruction also gives max|d| (into st->amax[1]) when the caller asks
  if (c->oz_amax) cudaMemsetAsync(c->oz_amax, 0, sizeof(unsigned long long), cur_stream(c));
  if ((st = oz_product(c, Zt, At, n, true, D, n, 0, partials, &fused, &nb_fused, bits2))) return st;
  c->oz_amax_done = fused && c->oz_nmod > 0 && c->oz_amax;
  if (!fused) {
    // several K-chunk batches: the combine accumulated X into D; form d = I - X from it
    if ((st = ctx_cuda(c, cudaMemcpyAsync(Xout, D, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice, cur_stream(c)),
                       "X copy")))
      return st;
    if ((st = ctx_cuda(c, klaunch(c, "resid_from_x", 2.0 * n * n, 16.0 * n * n, 1,
                                  [&] { return launch_resid_from_x(Xout, D, n, partials, cur_stream(c)); }),
                       "resid from X")))
      return st;
  }
  const int nb = fused ? nb_fused : nb_sep;
  return ctx_cuda(c, klaunch(c, "finish_err", 0, 0, 1, [&] {
                    return launch_finish_err(partials, nb, c->st_dev, idx, rule, tol, n, check_stop, cur_stream(c));
                  }),
                  "finish err");
}

// Slices for Z Q given a bound q >= max|Q_ij|.  Row i of Z and column j of Q are kept to T bits
// below their largest entries (2^ez_i, 2^eq_j); the truncation of either operand and the dropped
// slice pairs leave N error terms of size ~2^(ez_i + eq_j - T) in entry (i, j).  They are rounding
// errors uncorrelated with the other operand, so their sum grows like sqrt(N) (the probabilistic
// model of Higham and Mary, SIAM J. Sci. Comput. 2019, which also describes FP64 GEMM's own error).
// T = 53 + log2(4 sqrt(N) q) keeps that sum a factor 4 below 2^-53 2^ez_i, the rounding unit of row
// i's largest entry: below what storing Z + Z Q in FP64 costs anyway.  A small correction needs
// few bits.
int oz_update_bits(int n, double q) {
  double T = 53.0 + log2(4.0 * sqrt((double)n) * q);
  if (!(T > 0)) T = 0;
  const int t = (int)ceil(T), tmin = kOzBits * kOzSlicesUpdateMin;
  return t < tmin ? tmin : t;
}

int oz_update_slices(int n, double q) {
  double T = 53.0 + log2(4.0 * sqrt((double)n) * q);
  if (!(T > 0)) T = 0;
  int s = (int)ceil(T / kOzBits);
  if (s < kOzSlicesUpdateMin) s = kOzSlicesUpdateMin;
  if (s > kOzSlicesMax) s = kOzSlicesMax;
  return s;
}

// H_perp = Z^T H Z to FP64 accuracy (H symmetric), upper tiles mirrored.  Row-scaled slicing errs
// relative to |Z|^T |H| |Z|, the scale of FP64 GEMM's own error, and H_perp does not cancel the
// way d = I - Z^T S Z does, so the residual's base slice count (54 bits) is the right one.
int oz_congruence(zfact_ctx* c, const double* H, const double* Z, double* out, int n) {
  int st = ZFACT_OK;
  const int s = kOzSlicesResid, T = kOzBits * s;
  int wide = 0;
  const int nm = oz_moduli_for(c, T, T, oz_prod_bits(T, T, -1.0, -1.0, n), &wide);
  OzOperand Hop, Zt, At;
  double* A64 = (double*)ctx_buf(c, lane_name(c, "oz.At64").c_str(), sizeof(double) * (size_t)n * n, &st);
  if (!A64) return st;
  auto make = [&](const char* name, const double* X, bool trans, OzOperand* op) {
    return nm > 0 ? oz_make_mod(c, name, X, n, n, trans, T, nm, wide, op) : oz_make(c, name, X, n, n, trans, s, op);
  };
  if ((st = make("H", H, false, &Hop))) return st;
  if ((st = make("Zt", Z, true, &Zt))) return st;
  // A^T = Z^T H (H symmetric: B operand rows are rows of H), then Z^T (H Z) on upper tiles
  if ((st = oz_product(c, Zt, Hop, n, false, A64, n, 0))) return st;
  if ((st = make("At", A64, false, &At))) return st;
  return oz_product(c, Zt, At, n, true, out, n, 0);
}

// Z <- Z + Z Q to FP64 accuracy (Q symmetric: B operand rows are rows of Q); qmax bounds |Q_ij|.
int oz_update(zfact_ctx* c, double* Z, const double* Q, int n, double qmax, double rho_zr) {
  int st = ZFACT_OK;
  OzOperand Zr, Qr;
  if (qmax == 0.0) return ZFACT_OK;  // Q = 0: Z is unchanged
  if (qmax > 0.0 && isfinite(qmax)) {
    // T = 53 + log2(4 sqrt(N) q) bits as below, kept exactly by CRT residues where they fit; the moduli
    // from the scaled row norms of Z (the caller's, or unknown) and of any Q
    int wide = 0;
    const int Tu = oz_update_bits(n, qmax);
    const double bits = oz_prod_bits(Tu, Tu, rho_zr, -1.0, n);
    const int nm = oz_moduli_for(c, Tu, Tu, bits, &wide);
    if (nm > 0) {
      if ((st = oz_make_mod(c, "Zr", Z, n, n, false, Tu, nm, wide, &Zr))) return st;
      if ((st = oz_make_mod(c, "Qr", Q, n, n, false, Tu, nm, wide, &Qr))) return st;
      return oz_product(c, Zr, Qr, n, false, Z, n, 1, nullptr, nullptr, nullptr, bits);
    }
  }
  const int su = (qmax > 0.0 && isfinite(qmax)) ? oz_update_slices(n, qmax) : kOzSlicesMax;
  if ((st = oz_make(c, "Zr", Z, n, n, false, su, &Zr))) return st;
  if ((st = oz_make(c, "Qr", Q, n, n, false, su, &Qr))) return st;
  return oz_product(c, Zr, Qr, n, false, Z, n, 1);
}

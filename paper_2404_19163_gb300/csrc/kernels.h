// Host-side launchers of libzfact's kernels (C++ linkage, internal to the library).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "crt.h"
#include "crt_wide.h"

namespace zf {

// ----------------------------------------------------------------- FP64 CUDA-core products (k_f64.cu)
// acc = op(A) B for N x N row-major FP64 matrices, op(A) = A or A^T.
// Epilogue:  C = alpha * Add + beta * acc   (Add == nullptr: C = beta * acc),
//            P = acc when P != nullptr (raw product, for power chains),
//            sym: only tiles with row-block <= col-block are formed; entry (i,j), i <= j,
//                 is written to (i,j) and (j,i).
// Residual epilogue (resid == true, requires sym and op(A) = A^T):
//            C = I - acc, and partials[block] = sum of C_ij^2 over the entries the block owns
//            (off-diagonal entries count twice), to be reduced by launch_finish_err.
struct F64Gemm {
  const double* A;
  const double* B;
  double* C;
  const double* Add;
  double* P;
  double alpha, beta;
  double* partials;
  int n;
  bool transA, sym, resid;
};
int f64_num_blocks(int n, bool sym, bool fp32 = false);  // blocks of launch_f64_gemm / launch_f32_gemm (fp32)
cudaError_t launch_f64_gemm(const F64Gemm& g, cudaStream_t s);
// The same product in FP32 (the paper's "single"); Err partials stay FP64.
struct F32Gemm {
  const float* A;
  const float* B;
  float* C;
  const float* Add;
  float* P;
  double alpha, beta;
  double* partials;
  int n;
  bool transA, sym, resid;
};
cudaError_t launch_f32_gemm(const F32Gemm& g, cudaStream_t s);

// ----------------------------------------------------------------- elementwise / reductions (k_elem.cu)
// st->gscale = 1/sqrt(max_i sum_j |S_ij|) (st->amax[0] is used as scratch).
cudaError_t launch_gershgorin(const double* S, int n, IterState* st, cudaStream_t s);
// st->gscale = scale: the scale s of a cold start Z0 = s I chosen by the caller (zfact_opts.start_scale).
cudaError_t launch_set_gscale(IterState* st, double scale, cudaStream_t s);
// Z = st->gscale * I (FP64, N x N).
cudaError_t launch_scaled_identity_f64(double* Z, int n, const IterState* st, cudaStream_t s);
// Err = sqrt(sum of partials in a fixed order) -> st->hist[idx]; if check_stop, evaluate the stop
// rule against st->hist[idx-1] (rule 0: Algorithm 2 with guards; rule 1: Err/sqrt(N) <= tol).
cudaError_t launch_finish_err(const double* partials, int nparts, IterState* st, int idx, int rule,
                              double tol, int n, int check_stop, cudaStream_t s);
// Device-driven bulk loop (a CUDA graph with a while node): st->loop_iter = iters, st->loop_limit = limit;
// then, after each update's residual (whose finish_err takes idx = -1, i.e. loop_iter + 1), count the update
// and set the loop's condition (and `next`, the guard of the graph's second update, when set_next) to
// "no stop, no error, fewer than loop_limit updates".
cudaError_t launch_loop_init(IterState* st, int iters, int limit, cudaStream_t s);
cudaError_t launch_loop_cond(IterState* st, cudaGraphConditionalHandle loop, cudaGraphConditionalHandle next,
                             bool set_next, cudaStream_t s);

// 16-bit operand copies of an FP64 matrix (Eq. splitStyle): x = FP32[scale * src_ij],
// hi = R16(x), lo = R16(x - hi) (lo skipped when lo == nullptr), written at (i, j), or at
// (j, i) when transpose.  scale = *scale_ptr when scale_ptr != nullptr, else `scale`.
cudaError_t launch_cvt16(const double* src, int n, int ld_src, uint16_t* hi, uint16_t* lo, int ld16, double scale,
                         const float* scale_ptr, bool transpose, bool bf16, cudaStream_t s);
// The same from an FP32 source (scale from *scale_ptr when non-null, else 1).
cudaError_t launch_cvt16_f32(const float* src, int n, int ld_src, uint16_t* hi, uint16_t* lo, int ld16,
                             bool transpose, bool bf16, const float* scale_ptr, cudaStream_t s);
// FP16 operand scales of the bulk iteration (powers of two, bound * scale <= 2^14 / headroom):
//   op 0 (after the residual): scale[0] (d) from amaxf[1]; scale[1] (Q) from c1*|d|max + c2*hist[idx]^2
//   op 1 (before K1): scale[4] (A^T) from amax[0] (Gershgorin row sum of S) * amax[6] (|Z|max)
//   op 2 (before K4): scale[zslot_next] from 16 * amax[6]
//   op 3 (after K4): amax[6] = amaxf[2] (|Z|max of the new iterate)
cudaError_t launch_fp16_scales(IterState* st, int op, int idx, float c1, float c2, int zslot_next, int head,
                               cudaStream_t s);
// Flat split of n values (zfact_split).
cudaError_t launch_split_flat(const double* A, int64_t n, double scale, uint16_t* hi, uint16_t* lo, bool bf16,
                              cudaStream_t s);
// dst32 = (float) src64 (n x n, leading dimensions ld64 / ld32) and back.
cudaError_t launch_f64_to_f32(const double* src, int n, int ld64, float* dst, int ld32, cudaStream_t s);
// dst = (double)src; with amax != null also max |src| into *amax (the bits of a double, zeroed first).
cudaError_t launch_f32_to_f64(const float* src, int n, int ld32, double* dst, int ld64, cudaStream_t s,
                              unsigned long long* amax = nullptr);
// st->amax[slot] = max |A_ij| (FP64 bits, non-negative ordering).
cudaError_t launch_amax_f64(const double* A, int n, IterState* st, int slot, cudaStream_t s);
// Power-of-two scales for FP16 operands: st->scale[k] = 2^e with bound_k * 2^e in (2^13, 2^14],
// bound_0 = amax[1] (d), bound_1 = c1*amax[1] + c2*hist[idx]^2 (Q), bound_2 = amax[2] (Z).
cudaError_t launch_pow2_scales(IterState* st, int idx, float c1, float c2, cudaStream_t s);

// Cold start Z0 = s I (s = st->gscale): d0 = I - s^2 S from S's upper triangle, in FP32 (D32) and,
// when hi != nullptr, 16-bit hi (/lo) copies; cold_resid_blocks(n) Err partials; max |d0| (FP32
// bits) into *amax_bits.
int cold_resid_blocks(int n);
cudaError_t launch_cold_resid(const double* S, int n, const IterState* st, float* D32, int ld, uint16_t* hi,
                              uint16_t* lo, bool bf16, double* partials, unsigned int* amax_bits, cudaStream_t s);
// The first update from that start, Z1 = s (I + Q0) from the FP32 Q0: FP32 master, 16-bit copies
// (scaled by *out_scale when given) written to both the row-major and the transposed buffers (Z1 is
// symmetric), max |Z1| (FP32 bits) into *amax_bits.
cudaError_t launch_cold_update(const float* Q, int n, int ld, const IterState* st, float* Zm, uint16_t* zh,
                               uint16_t* zl, uint16_t* th, uint16_t* tl, const float* out_scale, bool bf16,
                               unsigned int* amax_bits, cudaStream_t s);

// ---- modular residues (k_ozmod.cu)
// Residue planes of X's rows (trans = false; e[r] written) or columns (trans = true; e from
// launch_oz_exp): round(x 2^(T - e_r)) modulo crt_modulus(0..nmod-1), symmetric, as BF16; plane t
// of operand row r at out[(t * Rp + r) * ld16 + k]; rows n..Rp-1 of every plane are zeroed.
cudaError_t launch_ozm_residues(const double* X, int n, int ld, bool trans, int* e, int T, int nmod, uint16_t* out,
                                int ld16, int Rp, cudaStream_t s);
// C' from the CRT digits of the residue products (k_tc.cu epilogue kEpiCrt8: plane t * nch + c holds
// the byte (product_t,c mod m_t) w_t mod m_t, row-major with leading dimension ld8), scaled by
// 2^(eA_i + eB_j - TA - TB); modes as launch_oz_combine (mode 2 writes ozm_combine_blocks(n)
// partials, and with amax != null the atomic maximum of |d| as the bits of a double, which the caller
// zeroes); sym forms i <= j and mirrors; nch <= kCrtMaxChunks.
cudaError_t launch_ozm_combine8(const uint8_t* G, size_t gstride, int ld8, int nch, const CrtPlan& plan, const int* eA,
                                const int* eB, int TA, int TB, int n, double* out, int ld64, int mode, bool sym,
                                double* partials, cudaStream_t s, unsigned long long* amax = nullptr);
int ozm_combine_blocks(int n);
// max_r rho_r^2 over the rows (cols = false) or columns (cols = true) of X, rho_r^2 = sum_k (x_rk 2^-e_r)^2
// with e_r the exponent bound of the residue kernels, as an FP32 bit pattern: atomic maximum into
// *rho2 (the caller zeroes it).  Summed in FP32: the result is below the exact value by at most
// (n/8 + 40) 2^-23 of it.  +Inf when X holds a NaN or Inf, or a row whose largest entry is subnormal.
// Columns need scratch of oz_colstats_scratch_bytes(n) + 4 n bytes (8-byte aligned).
cudaError_t launch_ozm_rho(const double* X, int n, int ld, bool cols, unsigned int* rho2, void* scratch,
                           cudaStream_t s);

// Residues with the wider moduli of crt_wide.h (k_ozmod_wide.cu): rows of up to 83 bits, up to
// crtw::kMax planes and moduli; and the reconstruction with the wider plan.
cudaError_t launch_ozmw_residues(const double* X, int n, int ld, bool trans, int* e, int T, int nmod, uint16_t* out,
                                 int ld16, int Rp, cudaStream_t s);
cudaError_t launch_ozmw_combine8(const uint8_t* G, size_t gstride, int ld8, int nch, const crtw::Plan& plan,
                                 const int* eA, const int* eB, int TA, int TB, int n, double* out, int ld64, int mode,
                                 bool sym, double* partials, cudaStream_t s, unsigned long long* amax = nullptr);

// ---- grouped residue products (the batched mode's final residuals, batched.cu)
// Instance i of a group: size n[i], its operand rows at packed rows row0[i] ... (one leading dimension for
// the group), fixed-point bits T[i].  A source is either per-instance matrices src[i] (n_i x n_i, leading
// dimension n_i) or one packed FP64 matrix (rows row0[i] + r, leading dimension ldp).  Exponents e are
// packed like the rows (e[row0[i] + r]).  Residue planes: plane t of operand row row0[i] + r at
// out + t * plane + (row0[i] + r) * ld16; columns n_i ... up to a multiple of 64 are written as zeros.
struct GroupRes {
  const int* n;
  const int* row0;
  const int* T;
  const double* const* src;
  const double* packed;
  int ldp;
  int* e;
  int count, max_n;
};
// Row residues (rows of src[i] or of the packed matrix; e written), T <= 62, nmod <= kCrtMax.
cudaError_t launch_gozm_rowres(const GroupRes& g, int nmod, uint16_t* out, int ld16, size_t plane, int maxT,
                               cudaStream_t s);
// Residues of the columns of src[i] (e from launch_gozm_colexp), T <= 62, nmod <= kCrtMax.
cudaError_t launch_gozm_tres(const GroupRes& g, int nmod, uint16_t* out, int ld16, size_t plane, int maxT,
                             cudaStream_t s);
// The same with the wider moduli (T <= 83, nmod <= crtw::kMax).
cudaError_t launch_gozmw_rowres(const GroupRes& g, int nmod, uint16_t* out, int ld16, size_t plane, cudaStream_t s);
cudaError_t launch_gozmw_tres(const GroupRes& g, int nmod, uint16_t* out, int ld16, size_t plane, cudaStream_t s);
// Column exponents of src[i] into g.e (packed), scratch: 8 * (packed rows) bytes.
cudaError_t launch_gozm_colexp(const GroupRes& g, unsigned long long* scratch, size_t scratch_rows, cudaStream_t s);
// Largest rho_r^2 of the rows of each instance's packed matrix rows (as launch_ozm_rho) into rho2[i].
cudaError_t launch_gozm_rowrho(const GroupRes& g, unsigned int* rho2, cudaStream_t s);
// CRT reconstruction of every instance (plan, modes as launch_ozm_combine8; TA = TB = T[i]); out packed
// (row0[i], leading dimension ld64) or null (mode 2: only the Err partials, ozm_combine_blocks(max_n) per
// instance from partials + i * ozm_combine_blocks(max_n)).
cudaError_t launch_gozm_combine8(const uint8_t* G, size_t gstride, int ld8, const CrtPlan& plan, const GroupRes& g,
                                 const int* eA, const int* eB, double* out, int ld64, int mode, bool sym,
                                 double* partials, cudaStream_t s);
cudaError_t launch_gozmw_combine8(const uint8_t* G, size_t gstride, int ld8, const crtw::Plan& plan,
                                  const GroupRes& g, const int* eA, const int* eB, double* out, int ld64, int mode,
                                  bool sym, double* partials, cudaStream_t s);
// err[i] = sqrt(sum of instance i's nb partials), in a fixed order.
cudaError_t launch_gozm_finish(const double* partials, int nb, int count, double* err, cudaStream_t s);

// ---- error-free slicing (k_ozaki.cu)
// e[r] = exponent bounding column r of X (cols = true; rows: nothing, the row kernels find their own).
// scratch: oz_colstats_scratch_bytes(n) bytes of device memory, 8-byte aligned.
cudaError_t launch_oz_exp(const double* X, int n, int ld, bool cols, int* e, void* scratch, cudaStream_t s);
// The same column exponents, and with rho2 the largest rho_j^2 of the columns as launch_ozm_rho.
cudaError_t launch_oz_colstats(const double* X, int n, int ld, int* e, unsigned int* rho2, void* scratch,
                               cudaStream_t s);
size_t oz_colstats_scratch_bytes(int n);
// Integer slices (b bits each) of X's rows (trans = false) or columns (trans = true); slice p of
// operand row r at out[(p * Rp + r) * ld16 + k]; rows n..Rp-1 of every slice are zeroed.
cudaError_t launch_oz_slice(const double* X, int n, int ld, bool trans, const int* e, int sl, int b, uint16_t* out,
                            int ld16, int Rp, cudaStream_t s);
// val = 2^{eA_i + eB_j} sum_t 2^{-b(t+2)} sum_c G[t * nch + c]; mode 0: out = val, 1: out += val,
// 2: out = I - val with per-block sums of squares in partials (grid of resid_from_x_blocks(n));
// sym: i <= j only, mirrored.
cudaError_t launch_oz_combine(const float* G, size_t gstride, int ld32, int sl, int nch, int b, const int* eA,
                              const int* eB, int n, double* out, int ld64, int mode, bool sym, double* partials,
                              cudaStream_t s);
int resid_from_x_blocks(int n);
int oz_combine_blocks(int n);  // partials written by launch_oz_combine in mode 2
// st->scale[scale_slot] = power of two s with st->amax[amax_slot] * s <= 2^14.
cudaError_t launch_pow2_slot(IterState* st, int amax_slot, int scale_slot, int head, cudaStream_t s);
// D = I - X (FP64), per-block sums of D_ij^2 into partials.
cudaError_t launch_resid_from_x(const double* X, double* D, int n, double* partials, cudaStream_t s);
cudaError_t launch_axpby64(double* out, double a, const double* X, double b, const double* Y, size_t total,
                           cudaStream_t s);

}  // namespace zf

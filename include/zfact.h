/*
 * zfact -- inverse-overlap factorization Z Z^T = S^{-1} on GB300 (sm_103a).
 *
 * C ABI of libzfact.so.  The method is the recursive refinement of
 * arXiv:2404.19163 (Habib, Finkelstein, Niklasson), Sec. 3, Eq. np1, with the
 * parameter-free stopping rule of Sec. 4.1 / Algorithm 2 and the
 * enhanced-precision refinement of Sec. 4.2 / Algorithm 3:
 *
 *   X_n = Z_n^T S Z_n,   d_n = I - X_n,   Err_n = ||d_n||_F
 *   Z_{n+1} = Z_n p_m(d_n),   p_m(d) = sum_{k=0..m} c_k d^k,  c_k = binom(2k,k)/4^k
 *   stop after update n when Err_n > Err_{n-1}^3  (Eq. stopL2, Algorithm 2)
 *
 * For m = 2, p_2(d) = I + d/2 + 3 d^2/8, which equals a0 I + a1 X + a2 X^2 with
 * the paper's a = (15/8, -5/4, 3/8) (Appendix A) under X = I - d.
 *
 * Conventions for every entry point:
 *   - Matrices are dense, row-major, N x N, FP64, contiguous (leading
 *     dimension N).  S must be symmetric positive definite.
 *   - Matrix pointers (S, Z0, Z) may be DEVICE pointers (any allocation on the
 *     context's device) or HOST pointers (pageable or pinned); the library
 *     classifies each with cudaPointerGetAttributes.  Host inputs are copied
 *     to the device and host outputs copied back inside the call.
 *   - Scalar outputs (hist, info, status arrays, scale, order) are HOST pointers.
 *   - The caller owns every pointer it passes.  The context owns its device
 *     workspace, grows it on demand and frees it in zfact_destroy.
 *   - Work is ordered on the context's stream.  Every call that takes a
 *     context synchronises that stream before it returns, so outputs are
 *     complete on return.  Device inputs must be complete when the context's
 *     stream reaches the call: the stream the context creates (cuda_stream
 *     NULL in zfact_create) is a blocking stream, ordered after work on the
 *     legacy default stream; inputs written on any other stream are the
 *     caller's to order (synchronise that stream, or create the context on
 *     it).  An input read while its producer still runs is silently wrong.
 *   - Nothing is thrown across the ABI.  Each call returns a zfact_status;
 *     zfact_last_error() returns a message for the last failure on a context.
 *     On failure, outputs are unspecified except info->hist_len / iters,
 *     which stay valid up to the failure.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef ZFACT_H
#define ZFACT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zfact_ctx zfact_ctx;

typedef enum zfact_status {
    ZFACT_OK = 0,
    ZFACT_ERR_ARG = 1,            /* bad argument (null pointer, N < 1, order out of range, ...) */
    ZFACT_ERR_CUDA = 2,           /* a CUDA runtime/driver call failed */
    ZFACT_ERR_NOMEM = 3,          /* device workspace allocation failed */
    ZFACT_ERR_NONFINITE = 4,      /* Err became NaN/Inf (divergence or non-finite input) */
    ZFACT_ERR_NOT_CONVERGED = 5,  /* the tolerance (stop_rule 1 / final check) was not met within nmax */
    ZFACT_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up (reported by a kernel) */
    ZFACT_ERR_UNSUPPORTED = 7,    /* request not available on this device/build */
    ZFACT_WARN_NONCONTRACTIVE = 100 /* returned with a result: Err_0 >= 1, so ||X0 - I|| < 1
                                       (the convergence condition of Sec. 3) is not guaranteed */
} zfact_status;

/* Arithmetic of the bulk iterations (Table I of the paper, GB300 forms). */
typedef enum zfact_precision {
    ZFACT_P_FP64 = 0,        /* "double": every product in FP64 (CUDA cores) */
    ZFACT_P_FP32 = 1,        /* "single": every bulk product in FP32 (CUDA cores); Algorithm 3's
                                refinement only when refine_steps > 0 */
    ZFACT_P_BF16 = 3,        /* "(h)(h)" with BF16 operands, FP32 accumulation (tcgen05) */
    ZFACT_P_FP16 = 4,        /* "(h)(h)" with FP16 operands (power-of-two scaled), FP32 accumulation */
    ZFACT_P_FP16_SPLIT = 5,  /* "(h)(h)+(h)(l)+(l)(h)": FP16 hi+lo split operands, FP32 accumulation */
    ZFACT_P_BF16_SPLIT = 6,  /* the same split with BF16 hi+lo */
    ZFACT_P_FP16_HALF = 7    /* "(h)(h)half": FP16 operands and FP16 accumulation (tcgen05 with an FP16
                                accumulator); operands scaled by powers of two to at most 1 in
                                magnitude so that sums of up to 65504 terms stay in FP16's range */
} zfact_precision;

/* How the refinement (Algorithm 3) forms d = I - Z^T S Z in FP64 accuracy. */
typedef enum zfact_refine_mode {
    ZFACT_R_NATIVE = 0,      /* FP64 CUDA-core products */
    ZFACT_R_OZAKI = 1,       /* FP64-accurate products on the BF16 tensor cores with exact FP32
                                accumulation: CRT residues of the fixed-point rows (Ozaki scheme
                                II) where they fit, else error-free slices (Ozaki, Ogita, Oishi,
                                Rump, "Error-free transformations of matrix multiplication by
                                using fast routines of matrix multiplication and its
                                applications", Numer. Algorithms 59 (2012)); see
                                zfact_set_emulation */
    ZFACT_R_FP32 = 2         /* single precision, Table I's "(h)(h)+refi" step: d, Q and Z + Z Q by
                                FP32 CUDA-core products (reaches the FP32 floor only); the final
                                residual of the returned Z is still formed to FP64 accuracy.
                                Mixed bulks only (zfact_refine with a 16-bit precision) */
} zfact_refine_mode;

typedef struct zfact_opts {
    int nmax;            /* max bulk updates (default 50) */
    int refine_steps;    /* max FP64-d refinement updates after the bulk stop (Algorithm 3);
                            default 0 for FP64 and FP32, 3 for the 16-bit precisions */
    int refine_mode;     /* zfact_refine_mode (default ZFACT_R_OZAKI when available) */
    int stop_rule;       /* 0: Algorithm 2 (Err_n > Err_{n-1}^3, or Err_n >= Err_{n-1}, or non-finite);
                            1: Algorithm 1 (Err_n / sqrt(N) <= tol) */
    double tol;          /* target for ||I - Z^T S Z||_F / sqrt(N): ends refinement early once met and
                            is checked on the final residual (0 = no check); stop_rule 1 uses it too */
    int fixed_iters;     /* > 0: exactly this many bulk updates, no stop test (parity mode) */
    int final_residual;  /* 1 (default): form ||I - Z^T S Z||_F of the returned Z in FP64 accuracy */
    int tile_cfg;        /* 0 = automatic; otherwise an index into the tuned tile table */
    double start_scale;  /* Z0 = NULL only: > 0 starts from Z0 = start_scale I (a learned proposal,
                            zfact_propose); 0 (default) from the Gershgorin scale I / sqrt(g_hi).  Either
                            way the cold start's first residual d0 = I - s^2 S and first update
                            s (I + Q0) need no products.  With the 16-bit precisions, a start_scale whose
                            bulk ends with Err >= min(1/4, Err_0) (no contraction the refinement could
                            finish) is dropped and the call starts again from the Gershgorin scale; the
                            time of both counts in info->ms, the history is the second run's */
} zfact_opts;

typedef struct zfact_info {
    int iters;           /* bulk updates performed (Algorithm 2's iter) */
    int refine_iters;    /* refinement updates performed (Algorithm 3) */
    int hist_len;        /* entries written to hist */
    int warn;            /* 0 or ZFACT_WARN_NONCONTRACTIVE */
    int launches;        /* kernels this call launched */
    double resid_f;      /* ||I - Z^T S Z||_F of the returned Z (FP64-accurate), NaN if not formed */
    double ms;           /* device time of the call (CUDA events around the work), milliseconds */
} zfact_info;

/* Fill *opts with the defaults listed above. */
void zfact_default_opts(zfact_opts* opts);

/* Create a context on CUDA device `device`, ordered on `cuda_stream`
 * (a cudaStream_t; NULL = a stream the context creates and owns). */
int zfact_create(zfact_ctx** ctx, int device, void* cuda_stream);

/* Destroy a context and free its workspace.  NULL is ignored. */
void zfact_destroy(zfact_ctx* ctx);

/* Message for the last failure on ctx (static storage owned by ctx). */
const char* zfact_last_error(zfact_ctx* ctx);

/* Refine Z0 into Z with Z^T S Z = I (Sec. 3 Eq. np1; Algorithms 2 and 3).
 *   S       N x N SPD overlap matrix (FP64).
 *   Z0      initial guess (FP64, N x N, general), or NULL for the scaled identity
 *           I / sqrt(max_i sum_j |S_ij|) (Gershgorin bound on lambda_max(S)).
 *   order   m in 2..5 (degree of p_m).
 *   precision  zfact_precision of the bulk iterations.
 *   opts    NULL = defaults.
 *   Z       output (FP64, N x N); may alias Z0.  S, Z0 and Z may each be device or host memory
 *           (host data are copied in and out inside the call); a pinned host Z receives the result
 *           by a copy that starts after the last refinement update and overlaps the final residual.
 *   hist    host array of hist_cap doubles: hist[0] = Err_0, then Err after every bulk
 *           update, then after every refinement update, then the final FP64 residual
 *           (when formed).  Entries beyond hist_cap are dropped.
 *   info    host struct (may be NULL). */
int zfact_refine(zfact_ctx* ctx, const double* S, const double* Z0, int64_t N, int order,
                 int precision, const zfact_opts* opts, double* Z, double* hist, int hist_cap,
                 zfact_info* info);

/* Refine `count` independent problems of uneven size in grouped launches
 * (every tile of every live instance in one persistent launch per GEMM stage).
 * S[i], Z0[i], Z[i] are DEVICE pointers of N[i] x N[i] FP64 matrices (Z0[i] may be
 * NULL, Z[i] may alias Z0[i]); orders[i] in 2..5.  hist is a host array of
 * count * hist_cap doubles (row i for instance i), info a host array of count
 * entries (may be NULL), status a host array of count ints (per-instance
 * zfact_status, may be NULL).  Every instance runs the bulk under the stop rule of opts; then, by
 * default (refine_steps < 0 or 0), the FP64-accurate residual of every returned Z is formed
 * (opts->final_residual) by grouped CRT launches over groups of instances (two groups in flight on
 * two streams), or per instance on concurrent streams when the batch is outside that form.  With refine_steps > 0 every instance also gets
 * Algorithm 3's refinement (refine_mode ZFACT_R_OZAKI or ZFACT_R_FP32; ZFACT_R_NATIVE returns
 * ZFACT_ERR_UNSUPPORTED), one instance after another, its Err entries appended to its history.
 * Motivated by the warm starts of Sec. 6 (molecular-dynamics frames, geometry optimisation). */
int zfact_refine_batched(zfact_ctx* ctx, int count, const double* const* S,
                         const double* const* Z0, const int64_t* N, const int* orders,
                         int precision, const zfact_opts* opts, double* const* Z,
                         double* hist, int hist_cap, zfact_info* info, int* status);

/* ---- learned start proposal (not in the paper; its warm-start motivation is Sec. 6) ----
 * Features: 16 floats per matrix, from the Gershgorin bounds of S and the trace moments
 * t_k = tr(d0^k)/N, k = 1..4, of d0 = I - s0^2 S with s0 = 1/sqrt(g_hi):
 *   0 log N, 1 log g_hi, 2 g_lo/g_hi, 3 mean S_ii/g_hi, 4 min S_ii/g_hi,
 *   5 mean row |S| sum/g_hi, 6 min row |S| sum/g_hi, 7..10 t_1..t_4, 11 sqrt(t_2),
 *   12 t_2 - t_1^2, 13 t_3 - 3t_1t_2 + 2t_1^3, 14 t_4 - 4t_1t_3 + 6t_1^2t_2 - 3t_1^4,
 *   15 log ||d0||_F.
 * S is a DEVICE or HOST FP64 N x N matrix; feat a HOST array of 16 floats. */
int zfact_features(zfact_ctx* ctx, const double* S, int64_t N, float* feat);

/* MLP 16 -> 64 -> 64 -> 5 with GELU, FP32.  Parameters are one flat DEVICE array of
 * 5573 floats: W1 (64x16, row-major, out x in), b1 (64), W2 (64x64), b2 (64),
 * W3 (5x64), b3 (5).  Outputs per row: y0 = predicted log(s / s0) for the start
 * Z0 = s I (s0 the Gershgorin scale) and y1..y4 = logits of the order m = 2..5.
 * Inputs are normalised by the caller-supplied feature mean/std (16 floats each,
 * DEVICE) before the first layer. */
#define ZFACT_MLP_NPARAMS 5573
int zfact_mlp_forward(zfact_ctx* ctx, const float* params, const float* feat_mean,
                      const float* feat_std, const float* x, int batch, float* y);
/* Loss L = mean_b[(y0 - t_b)^2 + w CE(softmax(y1..4), m_b)] and its gradient.
 * x (batch x 16), target_scale (batch), target_order (batch, int 0..3 for m = 2..5)
 * and grad (5573) are DEVICE arrays; *loss is written to a HOST double. */
int zfact_mlp_backward(zfact_ctx* ctx, const float* params, const float* feat_mean,
                       const float* feat_std, const float* x, const float* target_scale,
                       const int* target_order, int batch, float w_order, float* grad,
                       double* loss);
/* One Adam step (Kingma & Ba, Algorithm 1) on DEVICE arrays of n floats; step >= 1. */
int zfact_mlp_adam(zfact_ctx* ctx, float* params, const float* grad, float* m, float* v,
                   int n, int step, float lr, float beta1, float beta2, float eps);

/* Proposal for one matrix: features -> MLP -> (scale, order).  Falls back to the plain
 * schedule (Gershgorin scale, m = 2) when the network output is non-finite or outside
 * [s0/4, 4 s0].  params/mean/std are DEVICE arrays as above.  Returns the scale of
 * Z0 = scale * I in *scale and m in *order (HOST). */
int zfact_propose(zfact_ctx* ctx, const double* S, int64_t N, const float* params,
                  const float* feat_mean, const float* feat_std, double* scale, int* order);

/* ---- per-kernel timing ----------------------------------------------------------------
 * When profiling is on, every kernel launch of the context is bracketed by CUDA events
 * on the context's stream; the per-kernel totals (launch count, device milliseconds,
 * algorithmic FLOPs and bytes) accumulate until read with reset != 0. */
typedef struct zfact_kstat {
    char name[40];       /* kernel family, e.g. "tc_gemm.resid" */
    int launches;
    double ms;           /* summed device time of the launches */
    double flops;        /* summed algorithmic floating-point operations */
    double bytes;        /* summed algorithmic DRAM bytes */
} zfact_kstat;
int zfact_set_profiling(zfact_ctx* ctx, int on);
/* Copies up to cap entries into out (HOST), the count into *n (HOST). */
int zfact_kernel_stats(zfact_ctx* ctx, zfact_kstat* out, int cap, int* n, int reset);

/* ---- single steps, exposed for step-level parity tests ----------------------------- */
/* C = A B for N x N FP64 matrices with the operands rounded to the 16-bit format of
 * `precision` (BF16 / FP16 / the hi+lo splits; FP64 = plain FP64 product; FP32 = FP32 operands
 * and CUDA-core FP32 product, scales ignored) and FP32
 * tensor-core accumulation (FP16_HALF: FP16 operands and an FP16 accumulator, rounded to FP16
 * after every K = 16 step; the scaled partial sums must stay below 65504 in magnitude); C returned
 * in FP64.  scale_a / scale_b are the power-of-two
 * factors applied before rounding (undone after).  DEVICE pointers. */
int zfact_gemm(zfact_ctx* ctx, int precision, int64_t N, const double* A, double scale_a,
               const double* B, double scale_b, double* C);
/* Eq. splitStyle: hi = R16[FP32[scale*A]], lo = R16[FP32[scale*A] - hi] elementwise for
 * n values, R16 the BF16 (precision = BF16/BF16_SPLIT) or FP16 (FP16, FP16_SPLIT, FP16_HALF) rounding, round to nearest
 * even.  hi/lo are DEVICE arrays of n uint16 bit patterns. */
int zfact_split(zfact_ctx* ctx, int precision, const double* A, int64_t n, double scale,
                uint16_t* hi, uint16_t* lo);
/* d = I - Z^T S Z with FP64 accuracy by the method of `refine_mode`; returns ||d||_F in
 * *err (HOST) and d in D (DEVICE, may be NULL).  DEVICE S, Z. */
int zfact_residual(zfact_ctx* ctx, int refine_mode, const double* S, const double* Z,
                   int64_t N, double* D, double* err);

/* ---- congruence transform: the consumer of Z ------------------------------------------
 * H_perp = Z^T H Z for a symmetric N x N H (Sec. 2, Eq. standard_form).  With Z^T S Z = I
 * (Eq. Def_Z) it turns the generalized eigenproblem H C = S C e into the standard problem
 * H_perp C_perp = C_perp e, C = Z C_perp.  H_perp is symmetric by definition: its upper
 * triangle is formed and mirrored (as X = Z^T S Z is).
 *   precision ZFACT_P_FP64: FP64 accuracy by the method of refine_mode (ZFACT_R_NATIVE: FP64
 *     CUDA-core products; ZFACT_R_OZAKI: CRT residues or error-free slices on the BF16 tensor
 *     cores, 54 bits per operand row, errors on the scale of FP64 products relative to
 *     |Z|^T |H| |Z|);
 *   ZFACT_P_BF16 / ZFACT_P_BF16_SPLIT: BF16 (hi, or hi/lo) operands with FP32 accumulation
 *     (refine_mode ignored);
 *   FP32 and the FP16 precisions return ZFACT_ERR_UNSUPPORTED.
 * H, Z (inputs) and Hp (output) are row-major FP64, DEVICE or HOST (host operands are staged
 * through the context's workspace); Hp must not alias H or Z.  The call synchronises the
 * context's stream before it returns. */
int zfact_congruence(zfact_ctx* ctx, const double* H, const double* Z, int64_t N, int precision,
                     int refine_mode, double* Hp);

/* ---- workspace cap ------------------------------------------------------------------
 * Caps the device workspace the context may hold at `bytes` (0 = no cap, the default).  A call that
 * would grow the workspace past the cap fails with ZFACT_ERR_NOMEM before allocating, and the
 * context stays usable (raise the cap, or call again with a smaller problem).  Buffers already held
 * are not freed.  No counterpart in the paper: it bounds what a context takes from a shared GPU. */
int zfact_set_workspace_limit(zfact_ctx* ctx, int64_t bytes);

/* ---- FP64-accurate product scheme ----------------------------------------------------
 * How ZFACT_R_OZAKI forms its FP64-accurate products (the refinement's d = I - Z^T S Z and
 * Z + Z Q, zfact_residual's ozaki mode, zfact_congruence).  Both keep the same bits of every row
 * of the operands (rows rounded to T-bit fixed point, relative to the row's largest entry):
 *   ZFACT_EMU_AUTO (default): modular residues (Ozaki, Uchino, Imamura, "Ozaki Scheme II: A
 *     GEMM-oriented emulation of floating-point matrix multiplication using an integer modular
 *     technique", 2025): one BF16 tensor-core product per modulus (<= 256, pairwise coprime)
 *     and a Chinese-remainder reconstruction.  Sixteen moduli (product about 2^125.4) where the
 *     bound on the integer product fits them, up to 24 (product about 2^184.6, rows of up to
 *     83 bits: an ill-conditioned Z) where it does not; error-free slices beyond;
 *   ZFACT_EMU_SLICES: error-free slices always (the Ozaki et al. 2012 scheme above);
 *   ZFACT_EMU_WIDE: the same as ZFACT_EMU_AUTO (kept for callers that asked for the wider moduli
 *     before they were part of the default).
 * Other values return ZFACT_ERR_ARG.  No counterpart in the paper, which refines in FP64. */
typedef enum zfact_emulation {
    ZFACT_EMU_AUTO = 0,
    ZFACT_EMU_SLICES = 1,
    ZFACT_EMU_WIDE = 2
} zfact_emulation;
int zfact_set_emulation(zfact_ctx* ctx, int scheme);

/* ---- device-driven bulk loop ----------------------------------------------------------
 * With the 16-bit precisions, the Algorithm 2 updates after the first run as one CUDA graph: a
 * while node whose body holds two updates (the second under an if node, the two swap Z's buffers),
 * each ending in a one-thread kernel that applies the stop test on the device and sets the loop's
 * condition; the host waits once for the whole loop instead of once per update.  Every path of the
 * loop ends after nmax updates.  The graph is built on first use and kept per problem size, order,
 * precision and workspace layout.  on = 0 runs every update from the host (the same kernels, the
 * same results); the default is 1.  Not in the paper (a GB300 execution choice).  Returns ZFACT_OK. */
int zfact_set_loop_graphs(zfact_ctx* ctx, int on);

/* ---- bounded-wait self-test -----------------------------------------------------------
 * Launches one block whose mbarrier wait, the bounded wait every tensor-core kernel uses, can never
 * complete: nothing arrives at the barrier.  The wait gives up after a short poll limit, records
 * the timeout in the context's device state and returns, and the kernel exits normally.  The call
 * returns ZFACT_ERR_TIMEOUT (how a real timeout is reported) and the context stays usable.  No
 * counterpart in the paper: it checks the failure path without faulting or hanging a GPU. */
int zfact_selftest_timeout(zfact_ctx* ctx);

/* ---- allocation-free residual -------------------------------------------------------
 * d = I - Z^T S Z (FP64 CUDA cores) and ||d||_F, without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc where they need the residual, such as an application whose own memory pool
 * owns the whole device, or a step loop that cannot absorb the device synchronisation an
 * allocation may cause.  S, Z (N x N FP64, row-major) and the outputs D (N x N) and err
 * (one double) are DEVICE pointers owned by the caller.  Work is queued on cuda_stream
 * (a cudaStream_t; NULL = the default stream) and the call returns without waiting.
 * N must be in 1..1024; larger N returns ZFACT_ERR_ARG and launches nothing.  The product
 * S Z and the norm partials live in one static device array of 8 MiB + 8 KiB that every
 * GPU loading this library holds until the process exits; all calls on a device share
 * it, so calls that overlap on the GPU race.  Every call looks up that array's device
 * address in the current context (a host-side query, no allocation); the first lookup in a
 * context may load the library's device code, so make the first call on each device before
 * any stream capture.  No context is needed. */
int zfact_residual_noalloc(const double* S, const double* Z, int64_t N, double* D, double* err,
                           void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ZFACT_H */

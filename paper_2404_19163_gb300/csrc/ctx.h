// The library context (opaque to callers through zfact.h) and the internal
// host helpers shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc_gemm.h"

struct DevBuf {
  void* ptr;
  size_t bytes;
};

struct KStat {
  std::string name;
  int launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};

struct PendingEv {
  int id;
  cudaEvent_t a, b;
  double flops, bytes;
  int count;
};

struct zfact_ctx {
  int device = 0;
  int num_sms = 0;
  int cc_major = 0, cc_minor = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::map<std::string, DevBuf> bufs;  // named device workspace, grown on demand
  zf::IterState* st_dev = nullptr;     // device iteration state
  zf::IterState* st_host = nullptr;    // pinned host mirror
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double* mixed_result = nullptr;      // device FP64 Z produced by the mixed driver
  // The result's copy to a caller's pinned host Z, started on out_stream after each refinement update so
  // that it overlaps the FP64-accurate residual that follows (out_src: the device Z it reads, or null)
  void* out_host = nullptr;
  size_t out_bytes = 0;
  const double* out_src = nullptr;
  cudaStream_t out_stream = nullptr;
  cudaEvent_t out_ev = nullptr;
  char err[512];
  // per-kernel accounting
  bool profiling = false;
  int launches = 0;                  // kernels launched since the counter was last reset
  std::vector<KStat> kstats;
  std::vector<PendingEv> pending;
  std::vector<cudaEvent_t> ev_pool;
  // concurrent lanes (batched verification): while lane >= 0, the sliced-product driver issues
  // its work on lane_stream[lane] and uses workspace buffers suffixed with the lane
  static constexpr int kLanes = 8;
  int oz_s = 9;  // slices per operand of the current residual products
  int oz_T = 54;     // fixed-point bits per operand of the current residual products
  int oz_nmod = 0;   // > 0: those products use this many CRT residues instead of slices
  int oz_wide = 0;   // 1: those residues use the wider moduli of crt_wide.h
  double oz_rho_s = -1.0;  // largest scaled row norm of S's rows (-1: unknown), see oz_prod_bits
  // when set, oz_residual's fused CRT reconstruction writes max|d| there (double bits) and sets oz_amax_done
  unsigned long long* oz_amax = nullptr;
  bool oz_amax_done = false;
  // what the refinement's set-up would measure again, when this call already has it in the state:
  // the Gershgorin bound of S (amax[0]) and max|Z| of the FP64 Z it starts from (amax[2])
  const double* ghi_S = nullptr;
  const double* zmax_Z = nullptr;
  int oz_scheme = 0;  // zfact_emulation: 0 residues where they fit, 1 slices always, 2 also wide residues
  cudaStream_t lane_stream[kLanes] = {};
  int lane = -1;
  size_t ws_limit = 0;  // cap on the workspace bytes (0 = none), zfact_set_workspace_limit
  size_t ws_bytes = 0;  // workspace bytes allocated now
  // encoded TMA descriptors keyed by (address, rows, cols, ld, box rows, type)
  std::map<std::string, CUtensorMap> map_cache;
  // device-driven bulk loop (mixed.cu): instantiated graphs keyed by the loop's configuration and the
  // workspace generation (bumped whenever a workspace buffer is allocated or moved)
  struct LoopGraph {
    cudaGraphExec_t exec;
    int launches[2];  // kernels of the graph's first and second update
  };
  std::map<std::string, LoopGraph> loop_graph_cache;
  bool loop_graphs = true;  // zfact_set_loop_graphs
  unsigned long long ws_gen = 0;
  // pinned host words for the grouped residuals' read-backs and tables (batched_resid.cu)
  int* gr_pinned = nullptr;
  size_t gr_pinned_n = 0;
  // batched mode
  std::map<std::string, int> batch_bn;  // autotuned tile width per set of sizes
  std::string batch_sig;                // layout of the packed buffers (zeroed on change)
};

int kstat_id(zfact_ctx* c, const char* name);
// Adds FLOPs to the statistics of `name` without a launch or a time: the FP64 product count of an
// FP64-accurate product ("fp64_equiv": 2 N^2 K, half on symmetric tiles), whatever scheme formed it.
void kstat_note(zfact_ctx* c, const char* name, double flops);
// Early output copy (see zfact_ctx::out_host): start it from Z after the work queued so far; order the
// context's stream after the copy in flight (before Z is written again, or the call returns).
int out_copy_start(zfact_ctx* c, const double* Z);
void out_copy_fence(zfact_ctx* c);
cudaEvent_t ev_get(zfact_ctx* c);
void kstats_flush(zfact_ctx* c);  // stream must be idle

// Launch `f` (returning cudaError_t) as `count` kernels of family `name` with the given
// algorithmic FLOPs / bytes; bracketed by events when profiling is on.
inline cudaStream_t cur_stream(zfact_ctx* c) { return c->lane >= 0 ? c->lane_stream[c->lane] : c->stream; }
inline std::string lane_name(zfact_ctx* c, const char* name) {
  return c->lane >= 0 ? std::string(name) + ".L" + std::to_string(c->lane) : std::string(name);
}

template <class F>
cudaError_t klaunch(zfact_ctx* c, const char* name, double flops, double bytes, int count, F&& f) {
  c->launches += count;
  if (!c->profiling) return f();
  cudaEvent_t a = ev_get(c), b = ev_get(c);
  cudaEventRecord(a, cur_stream(c));
  cudaError_t e = f();
  cudaEventRecord(b, cur_stream(c));
  c->pending.push_back(PendingEv{kstat_id(c, name), a, b, flops, bytes, count});
  return e;
}

int ctx_fail(zfact_ctx* c, int code, const char* fmt, ...);
int ctx_cuda(zfact_ctx* c, cudaError_t e, const char* what);
void* ctx_buf(zfact_ctx* c, const char* name, size_t bytes, int* status);
bool is_device_ptr(const void* p);
int ctx_read_state(zfact_ctx* c);

// Cached tc_make_map (tc_gemm.h): identical (address, shape, box, type) reuse one encoding.
int ctx_make_map(zfact_ctx* c, CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows, bool bf16);

// FP64 building blocks (capi.cu)
int f64_residual(zfact_ctx* c, const double* S, const double* Z, double* A, double* D, int n, int idx, int rule,
                 double tol, int check_stop);
int f64_poly(zfact_ctx* c, const double* D, double* Q, double* P, double* P2, int n, int m);
int f64_update(zfact_ctx* c, const double* Z, const double* Q, double* Zn, int n);

// FP64-accurate products by error-free slicing (ozaki.cu)
int oz_slices_for(double zmax, double g_hi);
// rho_s, rho_zt, rho_zr: scaled row norms of S's rows and Z's columns and rows (oz_rho_from; -1 when
// unknown), which set the moduli of the CRT products (fewer where the rows are far from the worst case)
int oz_prepare_S(zfact_ctx* c, const double* S, int n, int s = 0, double rho_s = -1.0);
int oz_residual(zfact_ctx* c, const double* Z, double* D, int n, int idx, int rule, double tol, int check_stop,
                double rho_zt = -1.0);
int oz_update(zfact_ctx* c, double* Z, const double* Q, int n, double qmax, double rho_zr = -1.0);
double oz_rho_from(unsigned int rho2_bits, int n);
// Bits the moduli product must exceed for T_A- and T_B-bit rows with scaled row norms rhoA, rhoB (-1:
// unknown) over K = n terms, the moduli count for them (*wide: the wider set; 0: slices), and the K-blocks
// of one residue chunk.
double oz_product_bits(int TA, int TB, double rhoA, double rhoB, int n);
int oz_moduli_count(const zfact_ctx* c, int TA, int TB, double bits, int* wide);
int oz_crt_chunk_kb();  // K-blocks of one exact FP32 residue-product sum
int oz_update_slices(int n, double q);
int oz_update_bits(int n, double q);
int oz_congruence(zfact_ctx* c, const double* H, const double* Z, double* out, int n);

// Algorithm 3 with FP64-accurate sliced products, from the FP64 iterate Z64 (mixed.cu)
int refine_ozaki(zfact_ctx* c, const double* S, double* Z64, int n, int order, const zfact_opts& o, int iters,
                 int* ridx_out, zfact_info* inf);
int refine_fp32(zfact_ctx* c, const double* S, double* Z64, int n, int order, const zfact_opts& o, int iters,
                int* ridx_out, zfact_info* inf);
// The paper's "single": every bulk product in FP32 on the CUDA cores (single.cu)
int single_refine(zfact_ctx* c, const double* S, double* Za64, int n, int order, const zfact_opts& o, int* iters_out,
                  int* ridx_out, zfact_info* inf);

// Mixed-precision driver (mixed.cu): bulk tensor-core iterations, then Algorithm 3's refinement.
// cold: Za holds the Gershgorin start Z0 = s I (s in the device state's gscale), whose first residual
// and first update need no product.
// Returns kRetryGershgorin (before any refinement) when a caller's start_scale left the bulk without
// contraction (see zfact_opts.start_scale); the caller then starts again from the Gershgorin scale.
constexpr int kRetryGershgorin = -100;
int mixed_refine(zfact_ctx* c, const double* S, double* Za, double* Zb, int n, int order, int precision,
                 const zfact_opts& o, int* iters, int* ridx, zfact_info* inf, bool cold = false);

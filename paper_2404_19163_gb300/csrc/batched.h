// Batched (grouped) mode: device tables describing the stacked instances.
#pragma once
#include "common.cuh"

namespace zf {

struct BatchTables {
  const int* n;        // size of instance i
  const int* row0;     // first row of instance i in every packed buffer
  const int* part0;    // first norm partial of instance i
  const int* nparts;   // norm partials of instance i (4 per symmetric tile)
  const double* const* S;   // caller's FP64 S_i (device)
  const double* const* Z0;  // caller's FP64 Z0_i (device) or null: Gershgorin-scaled identity
  double* const* Z;         // caller's FP64 output Z_i (device)
};

struct BatchState {
  double* hist;     // count x cap: Err history per instance
  int cap;
  double* prev_err;
  int* iters;
  int* done;        // instance stopped (Algorithm 2 / 1, nmax, or non-finite)
  int* nonfinite;
  int* hist_len;
  int* live;        // instances not done
};

cudaError_t launch_b_gersh(const BatchTables& t, int count, int max_n, unsigned long long* gmax_bits,
                           cudaStream_t s);
// g_i (largest absolute row sum of S_i) and z_i (largest |Z_i|) as FP64 bits, for every instance.
cudaError_t launch_b_ranges(const BatchTables& t, int count, int max_n, unsigned long long* gmax_bits,
                            unsigned long long* zmax_bits, cudaStream_t s);
// Scaled row norms for the moduli of every instance's residue products (as launch_ozm_rho): rho2[i] over the
// rows of S_i, rho2[count + i] over the columns of Z_i (FP32 bits of the largest squared norm).  rows: the
// packed row count (instance i's columns at scratch offset row0[i]); scratch: b_rho_scratch_bytes(rows).
cudaError_t launch_b_rho(const BatchTables& t, int count, int max_n, int rows, unsigned int* rho2, void* scratch,
                         cudaStream_t s);
size_t b_rho_scratch_bytes(int rows);
cudaError_t launch_b_pack(const BatchTables& t, int count, int max_n, int mode, const unsigned long long* gmax_bits,
                          int ld, bool bf16, uint16_t* h16, uint16_t* l16, uint16_t* th16, uint16_t* tl16, float* m32,
                          cudaStream_t s);
cudaError_t launch_b_unpack(const BatchTables& t, int count, int max_n, const float* m32, int ld, cudaStream_t s);
}  // namespace zf

#include <vector>
struct zfact_ctx;
// The FP64-accurate final residual of every instance as grouped launches (batched_resid.cu): resid[i] =
// ||I - Z_i^T S_i Z_i||_F.  *done = false (nothing queued) when the batch is outside the grouped form (an
// instance above one residue chunk, rows above 83 bits, slices requested): the caller then uses lanes.
int batched_grouped_residuals(zfact_ctx* c, int count, const std::vector<int>& n, const std::vector<int>& order,
                              const double* const* S, double* const* Z, const std::vector<int>& slices,
                              const std::vector<double>& rho_s, const std::vector<double>& rho_z,
                              std::vector<double>& resid, bool* done);

namespace zf {
cudaError_t launch_b_finish(const double* partials, const BatchTables& t, const BatchState& bs, int count,
                            int initial, int rule, double tol, int check_stop, int limit, cudaStream_t s);

}  // namespace zf

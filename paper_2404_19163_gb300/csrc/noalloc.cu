// zfact_residual_noalloc: the FP64 residual d = I - Z^T S Z and its Frobenius norm
// without any device allocation.
//
// Why it exists: some callers of this library cannot call cudaMalloc at the point
// where they need the residual.  A host application that hands out all device
// memory through its own pool (a molecular-dynamics engine that reserves its
// budget at start-up, a framework whose caching allocator owns the device) may
// forbid raw allocations; and cudaMalloc can synchronise the device, which a
// caller running a latency-critical step loop on other streams cannot afford.
// Those callers still pass their own S, Z and output buffers; the intermediate
// product S Z and the per-block norm partials live in the file-scope array below.
//
// The scratch array is a fixed, modest size (8 MiB + 8 KiB) and is held by every
// GPU that loads this library until the process exits.  Every call on a device
// shares it and it keeps the last call's contents: nothing in it has to start at
// zero (every entry a call reads it has written first), and two calls that
// overlap on the GPU (different streams, or different host threads) race on it.
#include <math.h>

#include "ctx.h"
#include "kernels.h"

using namespace zf;

namespace {

constexpr int kNoallocMaxN = 1024;
constexpr size_t kProdDoubles = (size_t)kNoallocMaxN * kNoallocMaxN;  // S Z, N x N
constexpr size_t kPartDoubles = 1024;                                  // >= blocks of the symmetric product
static __device__ __align__(256) double g_noalloc_scratch[kProdDoubles + kPartDoubles];

// Device address of the scratch array in the current context.  It is looked up on every call (a
// host-side query): a cached address would go stale when the module is loaded again, after
// cudaDeviceReset or in another driver context of the same device.  The first lookup in a context
// may load the module, which is why the first call on a device should come before any stream capture.
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

__global__ void k_noalloc_norm(const double* __restrict__ partials, int np, double* err) {
  __shared__ double red[256];
  double s = 0.0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) s += partials[p];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *err = sqrt(red[0]);
}

}  // namespace

extern "C" int zfact_residual_noalloc(const double* S, const double* Z, int64_t N, double* D, double* err,
                                      void* cuda_stream) {
  if (!S || !Z || !D || !err) return ZFACT_ERR_ARG;
  if (N < 1 || N > kNoallocMaxN) return ZFACT_ERR_ARG;
  const int n = (int)N;
  if (f64_num_blocks(n, true) > (int)kPartDoubles) return ZFACT_ERR_ARG;
  // an error left by earlier, unrelated work on this thread is not this call's: clear it before
  // queuing anything (a sticky error still makes the launches below fail, and is reported then)
  cudaGetLastError();
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return ZFACT_ERR_CUDA;
  }
  double* A = scratch;                    // S Z
  double* partials = scratch + kProdDoubles;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  F64Gemm g1{S, Z, A, nullptr, nullptr, 0.0, 1.0, nullptr, n, false, false, false};
  if (launch_f64_gemm(g1, s) != cudaSuccess) return ZFACT_ERR_CUDA;
  F64Gemm g2{Z, A, D, nullptr, nullptr, 0.0, 1.0, partials, n, true, true, true};
  if (launch_f64_gemm(g2, s) != cudaSuccess) return ZFACT_ERR_CUDA;
  k_noalloc_norm<<<1, 256, 0, s>>>(partials, f64_num_blocks(n, true), err);
  if (cudaGetLastError() != cudaSuccess) return ZFACT_ERR_CUDA;
  return ZFACT_OK;
}

// Shared device/host helpers of libzfact: status plumbing, the iteration state
// that lives on the device, and thin inline-PTX wrappers for the Blackwell
// (sm_103a) primitives the tensor-core kernels use: mbarrier, TMA
// (cp.async.bulk.tensor), and tcgen05 (TMEM alloc / mma / commit / ld).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/zfact.h"

namespace zf {

// ---------------------------------------------------------------- device-side iteration state
constexpr int kHistMax = 128;

// Error bits a kernel may raise (never by trapping): the host reads them after the call.
enum : int { kErrTimeout = 1, kErrNonfinite = 2, kErrShape = 4 };

struct IterState {
  double hist[kHistMax];  // Err_n = ||I - X_n||_F for every formed residual
  double prev_err;        // the Err the stop test compares against
  double gscale;          // Gershgorin scale 1/sqrt(max_i sum_j |S_ij|)
  double amax[8];         // running absolute maxima (scaling of 16-bit operands)
  float scale[8];         // power-of-two operand scales (16-bit formats)
  unsigned int amaxf[8];  // absolute maxima written by GEMM epilogues (FP32 bit patterns)
  int stop;               // set by the stop test (Algorithm 2 / 1)
  int nonfinite;          // Err became NaN/Inf
  int error;              // kErr* bits raised by kernels (bounded waits, shape checks)
  int hist_len;           // entries of hist written
  int timeout_where;      // which wait gave up (diagnostics)
  unsigned int rho2[4];   // largest squared scaled row norm of CRT operands (FP32 bits, launch_ozm_rho)
  int loop_iter;          // bulk updates done, when the device drives the loop (mixed.cu loop graph)
  int loop_limit;         // ... and the count it may not reach
  int pad[1];
};

// ---------------------------------------------------------------- small device helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void raise_error(int* flag, int bits) { atomicOr(flag, bits); }

// Magnitudes of doubles on the integer pipes (GB300's FP64 pipe is a small fraction of them): the
// bit pattern with the sign cleared orders like |x| (Inf above every finite value, NaN above Inf),
// and frexp's exponent follows from it.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long max_bits(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
// e with |x| in [2^(e-1), 2^e) for the non-zero, finite magnitude pattern b (frexp's exponent).
__device__ __forceinline__ int exp_of_bits(unsigned long long b) {
  const int eb = (int)(b >> 52);
  return eb ? eb - 1022 : (63 - __clzll((long long)b)) - 1073;
}
// |x| 2^-e rounded toward zero to FP32, for the magnitude pattern b of x with |x| < 2^e (integer
// operations on the bits); values below FP32's normal range read as zero.
__device__ __forceinline__ float scaled_mag_f32(unsigned long long b, int e) {
  const int eb = (int)(b >> 52), fe = eb - 1023 - e + 127;
  if (eb == 0 || fe <= 0) return 0.0f;
  return __uint_as_float(((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit` polls (each try_wait itself blocks for a
// hardware-defined interval), raises kErrTimeout and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err_flag, int where,
                                          uint32_t limit = 1u << 24) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (err_flag && (i & 1023u) == 1023u && *(volatile int*)err_flag & kErrTimeout) return false;
  }
  if (err_flag) raise_error(err_flag, kErrTimeout | (where << 8));
  return false;
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}
// 2-D tiled load of a box into shared memory; completion is signalled on `bar`
// as transaction bytes.  x (innermost, elements) must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* m, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, both K-major, kind::f16 (BF16 or FP16 in, FP32 out).
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive (once) on `bar` when every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 lanes x 32 consecutive 32-bit columns: thread t of the warp receives lane (base + t).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (tcgen05 format): K-major operand tile whose
// rows are 128 bytes, stored with the 128-byte swizzle in 8-row (1024-byte)
// atoms, as a TMA load with CU_TENSOR_MAP_SWIZZLE_128B writes it.
//   bits  0-13 start address >> 4      bits 16-29 leading byte offset >> 4
//   bits 32-45 stride byte offset >> 4 bits 46-47 descriptor version (1)
//   bits 49-51 base offset (0: atoms are 1024-byte aligned)
//   bits 61-63 layout (2 = 128-byte swizzle)
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                    // LBO (unused for swizzled K-major; canonical value 1)
  d |= (uint64_t)(1024 >> 4) << 32;          // SBO: 8 rows x 128 B between 8-row groups
  d |= (uint64_t)1 << 46;                    // version
  d |= (uint64_t)2 << 61;                    // SWIZZLE_128B
  return d;
}

// Instruction descriptor for kind::f16, both operands K-major.
//   bits 4-5 D format (1 = F32, 0 = F16), 7-9 A format, 10-12 B format (0 = F16, 1 = BF16),
//   15/16 A/B major (0 = K), 17-22 N >> 3, 24-28 M >> 4.  An F16 accumulator takes F16 operands.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n, bool bf16, bool acc16 = false) {
  return ((acc16 ? 0u : 1u) << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// An FP16 accumulator occupies one 32-bit tensor-memory column per element, the value in the low 16
// bits (column j holds D[:, j], as with FP32): widen what tmem_ld32 returned to FP32.
__device__ __forceinline__ void widen_acc16(float (&v)[32]) {
#pragma unroll
  for (int i = 0; i < 32; ++i)
    v[i] = __half2float(__ushort_as_half((unsigned short)(__float_as_uint(v[i]) & 0xFFFFu)));
}

}  // namespace zf

// tcgen05 GEMM engine for the recursion's products on GB300 (sm_103a).
//
// One persistent CTA per SM walks a list of output tiles (128 x BN).  Warp 0
// streams K-blocks of the operands into a ring of shared-memory stages with
// TMA (128-byte swizzle); one thread of warp 1 issues tcgen05.mma (kind::f16,
// FP32 accumulation in tensor memory) and releases each stage with
// tcgen05.commit; warps 2-9 read the accumulator back with tcgen05.ld and run
// the fused epilogue while the next tile accumulates in the other half of the
// tensor memory (two accumulator buffers).  Two epilogue warps share each
// 32-lane quadrant of the accumulator (a warp may only read its own quadrant),
// one for each half of the tile's columns: the epilogue stores and conversions
// of a tile then take no longer than its products.  Each epilogue is its own
// instantiation of the kernel, so no epilogue pays for another's registers.
//
// A product may consist of up to four K-concatenated segments accumulated
// into one accumulator: the split scheme (h)(h)+(h)(l)+(l)(h) of Sec. 3.2
// (Eqs. SZn, Xn, Xsq) is three segments.  Symmetric products (X = Z^T S Z and
// the powers of d) form only the tiles that touch the upper triangle and
// write every entry (i, j), i <= j, to both (i, j) and (j, i).
//
// Every wait on an mbarrier is bounded; a wait that gives up raises a flag in
// the device state and the CTA winds down (no trap).
#include <stdio.h>

#include "crt_wide.h"
#include "tc_gemm.h"

namespace zf {
namespace {

constexpr int BM = 128, BK = 64, UK = 16, NEPI_WARPS = 8, NTHREADS = 64 + 32 * NEPI_WARPS;

template <int BN>
struct Cfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int STAGES = BN == 256 ? 4 : 6;
  static constexpr int TMEM_COLS = 2 * BN;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};

__host__ __device__ inline int tiles_of(int M, int N, int sym, int bn_size) {
  const int tm = (M + BM - 1) / BM, tn = (N + bn_size - 1) / bn_size;
  if (!sym) return tm * tn;
  int total = 0;
  for (int r = 0; r < tm; ++r) total += tn - (r * BM) / bn_size;
  return total;
}

__host__ __device__ inline int units_of(const TcArgs& a, int bn_size) {
  if (a.ninst > 0) return a.M;  // grouped: total units passed in M by the host
  const int t = tiles_of(a.M, a.N, a.sym, bn_size);
  return a.oz_s > 0 ? t * a.oz_s * a.oz_nch : t;
}

// Work of one unit: `npairs` operand pairs over K-blocks [kb0, kb1) of the output tile `tile`
// of a problem of size n whose rows start at row0 (grouped mode) or 0.
struct UnitPlan {
  int tile, group, npairs, p0, t, kb0, kb1;
  int inst, n, row0, skip;
};

template <int BN>
__device__ __forceinline__ UnitPlan plan_unit(int u, const TcArgs& a, int kblocks_all) {
  UnitPlan pl;
  pl.inst = 0;
  pl.row0 = 0;
  pl.n = a.N;
  pl.skip = 0;
  int kblocks = kblocks_all;
  if (a.ninst > 0) {
    int lo = 0, hi = a.ninst - 1;  // slot j with g_prefix[j] <= u < g_prefix[j+1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.g_prefix[mid] <= u)
        lo = mid;
      else
        hi = mid - 1;
    }
    pl.inst = a.g_inst[lo];
    pl.n = a.g_n[pl.inst];
    pl.row0 = a.g_row0[pl.inst];
    pl.skip = (a.g_done && a.g_done[pl.inst]) ? 1 : 0;
    u -= a.g_prefix[lo];
    kblocks = (pl.n + BK - 1) / BK;
  }
  if (a.oz_s > 0) {
    // group-major order: the CTAs running at the same time form different tiles of the same
    // (group, K-chunk) and so read the same slice panels, which then stay in L2
    // (grouped residue products: the instance's own tile count; its units are tiles x moduli x chunks)
    const int ntiles = a.ninst > 0 ? tiles_of(pl.n, pl.n, a.sym, BN) : a.oz_tiles;
    pl.group = u / ntiles;
    pl.tile = u % ntiles;
    pl.t = pl.group / a.oz_nch;
    const int c = pl.group % a.oz_nch;
    if (a.oz_diag) {
      // residue products: group t is the single pair (t, t)
      pl.p0 = pl.t;
      pl.npairs = 1;
    } else {
      pl.p0 = pl.t - (a.oz_s - 1) > 0 ? pl.t - (a.oz_s - 1) : 0;
      const int p1 = pl.t < a.oz_s - 1 ? pl.t : a.oz_s - 1;
      pl.npairs = p1 - pl.p0 + 1;
    }
    pl.kb0 = (a.oz_c0 + c) * a.oz_chunk_kb;
    pl.kb1 = pl.kb0 + a.oz_chunk_kb < kblocks ? pl.kb0 + a.oz_chunk_kb : kblocks;
  } else {
    pl.tile = u;
    pl.group = 0;
    pl.t = 0;
    pl.p0 = 0;
    pl.npairs = a.nseg;
    pl.kb0 = 0;
    pl.kb1 = kblocks;
  }
  return pl;
}

__device__ __forceinline__ void decode_unit(int u, const TcArgs& a, int n_inst, int bn_size, int& bm, int& bn) {
  const int M = a.ninst > 0 ? n_inst : a.M, N = a.ninst > 0 ? n_inst : a.N;
  const int tm = (M + BM - 1) / BM, tn = (N + bn_size - 1) / bn_size;
  if (!a.sym) {
    bm = u % tm;
    bn = u / tm;
    return;
  }
  for (int r = 0; r < tm; ++r) {
    const int first = (r * BM) / bn_size, cnt = tn - first;
    if (u < cnt) {
      bm = r;
      bn = first + u;
      return;
    }
    u -= cnt;
  }
  bm = tm;
  bn = tn;
}

__device__ __forceinline__ uint16_t to16(float x, int bf16) {
  return bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(x)) : __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ float from16(uint16_t h, int bf16) {
  return bf16 ? __bfloat162float(__ushort_as_bfloat16(h)) : __half2float(__ushort_as_half(h));
}

// Store 32 16-bit values of row i starting at column col0; entries with j >= n, or
// j < i when `upper`, are skipped.  Mirror: also write (j, i) for i < j.
__device__ __forceinline__ void put16(uint16_t* base, int ld, int i, int col0, int n, bool upper, bool mirror,
                                      const uint16_t (&h)[32]) {
  if (!base) return;
  const bool full = (col0 + 32 <= n) && (!upper || col0 >= i);
  if (full) {
    uint4* dst = reinterpret_cast<uint4*>(base + (size_t)i * ld + col0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 w;
      w.x = (uint32_t)h[q * 8 + 0] | ((uint32_t)h[q * 8 + 1] << 16);
      w.y = (uint32_t)h[q * 8 + 2] | ((uint32_t)h[q * 8 + 3] << 16);
      w.z = (uint32_t)h[q * 8 + 4] | ((uint32_t)h[q * 8 + 5] << 16);
      w.w = (uint32_t)h[q * 8 + 6] | ((uint32_t)h[q * 8 + 7] << 16);
      dst[q] = w;
    }
  } else {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const int j = col0 + jj;
      if (j < n && (!upper || j >= i)) base[(size_t)i * ld + j] = h[jj];
    }
  }
  if (mirror) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const int j = col0 + jj;
      if (j < n && j > i) base[(size_t)j * ld + i] = h[jj];
    }
  }
}

__device__ __forceinline__ void put32(float* base, int ld, int i, int col0, int n, bool upper, bool mirror,
                                      const float (&x)[32]) {
  const bool full = (col0 + 32 <= n) && (!upper || col0 >= i);
  if (full) {
    float4* dst = reinterpret_cast<float4*>(base + (size_t)i * ld + col0);
#pragma unroll
    for (int q = 0; q < 8; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
  } else {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const int j = col0 + jj;
      if (j < n && (!upper || j >= i)) base[(size_t)i * ld + j] = x[jj];
    }
  }
  if (mirror) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const int j = col0 + jj;
      if (j < n && j > i) base[(size_t)j * ld + i] = x[jj];
    }
  }
}

// Transposed store of 32 values of row i: element j goes to (j, i).  Coalesced across the warp.
__device__ __forceinline__ void put16_t(uint16_t* base, int ld, int i, int col0, int n, const uint16_t (&h)[32]) {
  if (!base) return;
#pragma unroll
  for (int jj = 0; jj < 32; ++jj) {
    const int j = col0 + jj;
    if (j < n) base[(size_t)j * ld + i] = h[jj];
  }
}

// Load 32 floats of a row starting at column col0 (16-byte vector loads when the whole chunk is
// inside the row's n columns; entries j >= n read as 0).
__device__ __forceinline__ void load32(const float* row, int col0, int n, float (&x)[32]) {
  if (col0 + 32 <= n) {
    const float4* src = reinterpret_cast<const float4*>(row + col0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 t = src[q];
      x[4 * q] = t.x;
      x[4 * q + 1] = t.y;
      x[4 * q + 2] = t.z;
      x[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) x[jj] = (col0 + jj < n) ? row[col0 + jj] : 0.0f;
  }
}

// Store 32 bytes of row i starting at column col0 (entries j >= n, or j < i when `upper`, skipped).
__device__ __forceinline__ void put8(uint8_t* base, int ld, int i, int col0, int n, bool upper, const uint32_t (&w)[8]) {
  const bool full = (col0 + 32 <= n) && (!upper || col0 >= i);
  uint8_t* row = base + (size_t)i * ld;
  if (full) {
    uint4* dst = reinterpret_cast<uint4*>(row + col0);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
  } else {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const int j = col0 + jj;
      if (j < n && (!upper || j >= i)) row[j] = (uint8_t)(w[jj >> 2] >> (8 * (jj & 3)));
    }
  }
}

// Modulus of a residue product and its reconstruction weight (kEpiCrt8).
struct CrtDigitConst {
  float m, inv, w;
};

__device__ __forceinline__ void split32(const float (&x)[32], float sc, int bf16, bool want_lo, uint16_t (&h)[32],
                                        uint16_t (&l)[32]) {
#pragma unroll
  for (int jj = 0; jj < 32; ++jj) {
    const float y = x[jj] * sc;
    h[jj] = to16(y, bf16);
    l[jj] = want_lo ? to16(y - from16(h[jj], bf16), bf16) : (uint16_t)0;
  }
}

template <int EPI>
__device__ __forceinline__ void epi_chunk(const TcArgs& a, int i, int col0, float (&v)[32], double& ss, float& amax,
                                          float osc, float us, int group, int n, int row0, const CrtDigitConst& cd) {
  // grouped problems are stacked along rows: shift every output/input base to the instance
  const size_t r16 = (size_t)row0 * a.ld16, r32 = (size_t)row0 * a.ld32, r64 = (size_t)row0 * a.ld64;
  uint16_t* o16h = a.o16h ? a.o16h + r16 : nullptr;
  uint16_t* o16l = a.o16l ? a.o16l + r16 : nullptr;
  uint16_t* t16h = a.t16h ? a.t16h + r16 : nullptr;
  uint16_t* t16l = a.t16l ? a.t16l + r16 : nullptr;
  float* f32 = a.f32 ? a.f32 + r32 : nullptr;
  const float* f32_in = a.f32_in ? a.f32_in + r32 : nullptr;
  double* f64 = a.f64 ? a.f64 + r64 : nullptr;
  if (i >= (a.ninst > 0 ? n : a.M)) return;
  const bool lo = a.split_out != 0;
  uint16_t h[32], l[32];
  switch (EPI) {
    case kEpiStore16: {
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) v[jj] *= us;
      split32(v, osc, a.bf16, lo, h, l);
      put16(o16h, a.ld16, i, col0, n, false, false, h);
      if (lo) put16(o16l, a.ld16, i, col0, n, false, false, l);
      break;
    }
    case kEpiResid: {
      // the chunk's sum of squares in FP32 (32 terms: relative error below 2^-19), then one FP64 add:
      // GB300's FP64 pipe would otherwise set the pace of this epilogue
      float cs = 0.0f;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const int j = col0 + jj;
        const float d = (i == j ? 1.0f : 0.0f) - v[jj] * us;
        v[jj] = d;
        if (j < n && j >= i) {
          cs = fmaf(i == j ? d : 2.0f * d, d, cs);
          amax = fmaxf(amax, fabsf(d));
        }
      }
      ss += (double)cs;
      put32(f32, a.ld32, i, col0, n, true, true, v);
      split32(v, osc, a.bf16, lo, h, l);
      put16(o16h, a.ld16, i, col0, n, true, true, h);
      if (lo) put16(o16l, a.ld16, i, col0, n, true, true, l);
      break;
    }
    case kEpiPoly: {
      // r = c1 * f32_in + c2 * v: the running sum of c_k d^k.  Outputs: the running sum in
      // FP32 (f32), its 16-bit copy (o16, the final Q), and the raw power v (t16, P_k for
      // the next product of the chain), all at (i, j) and (j, i).
      float r[32];
      load32(f32_in + (size_t)i * a.ld32, col0, n, r);
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        v[jj] *= us;
        r[jj] = a.c1 * r[jj] + a.c2 * v[jj];
      }
      if (f32) put32(f32, a.ld32, i, col0, n, true, true, r);
      if (o16h) {
        split32(r, osc, a.bf16, lo, h, l);
        put16(o16h, a.ld16, i, col0, n, true, true, h);
        if (lo) put16(o16l, a.ld16, i, col0, n, true, true, l);
      }
      if (t16h) {
        split32(v, a.p_scale ? *a.p_scale : 1.0f, a.bf16, lo, h, l);
        put16(t16h, a.ld16, i, col0, n, true, true, h);
        if (lo) put16(t16l, a.ld16, i, col0, n, true, true, l);
      }
      break;
    }
    case kEpiZupd: {
      float* zrow = f32 + (size_t)i * a.ld32;
      float zo[32];
      load32(zrow, col0, n, zo);
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const float z = (col0 + jj < n) ? zo[jj] + v[jj] * us : 0.0f;
        v[jj] = z;
        amax = fmaxf(amax, fabsf(z));
      }
      put32(zrow - (size_t)i * a.ld32, a.ld32, i, col0, n, false, false, v);
      split32(v, osc, a.bf16, lo, h, l);
      put16(o16h, a.ld16, i, col0, n, false, false, h);
      if (lo) put16(o16l, a.ld16, i, col0, n, false, false, l);
      put16_t(t16h, a.ld16, i, col0, n, h);
      if (lo) put16_t(t16l, a.ld16, i, col0, n, l);
      break;
    }
    case kEpiF64: {
      double* crow = f64 + (size_t)i * a.ld64;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const int j = col0 + jj;
        if (j < n && (!a.sym || j >= i)) {
          double x = (double)v[jj] * (double)us;
          if (a.f64_in) x = fma((double)a.c1, a.f64_in[(size_t)row0 * a.ld64 + (size_t)i * a.ld64 + j], (double)a.c2 * x);
          crow[j] = x;
          if (a.sym && j > i) f64[(size_t)j * a.ld64 + i] = x;
        }
      }
      break;
    }
    case kEpiG32: {
      float* g = f32 + (size_t)group * a.g_stride;
      put32(g, a.ld32, i, col0, n, a.sym != 0, false, v);
      break;
    }
    case kEpiCrt8: {
      // v is an exact integer of at most 2^24 in magnitude (the sub-chunk residue sums of the unit,
      // each reduced modulo m); its CRT digit in [0, m) < 2^8 is all the reconstruction needs
      uint32_t w[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint32_t word = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float y = crt_digit(v[4 * q + b], cd.m, cd.inv, cd.w);
          word |= (__float_as_uint(y + 8388608.0f) & 0xFFu) << (8 * b);
        }
        w[q] = word;
      }
      put8(a.d8 + (size_t)group * a.g_stride + (size_t)row0 * a.ld32, a.ld32, i, col0, n, a.sym != 0, w);
      break;
    }
    case kEpiZupd64: {
      double* zrow = f64 + (size_t)i * a.ld64;
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const int j = col0 + jj;
        if (j < n) {
          const double z = zrow[j] + (double)v[jj] * (double)us;
          zrow[j] = z;
          v[jj] = (float)z;
          amax = fmaxf(amax, fabsf((float)z));
        } else {
          v[jj] = 0.0f;
        }
      }
      if (o16h) {
        split32(v, osc, a.bf16, lo, h, l);
        put16(o16h, a.ld16, i, col0, n, false, false, h);
        if (lo) put16(o16l, a.ld16, i, col0, n, false, false, l);
        put16_t(t16h, a.ld16, i, col0, n, h);
        if (lo) put16_t(t16l, a.ld16, i, col0, n, l);
      }
      break;
    }
    default:
      break;
  }
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

template <int BN, int EPI>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc_gemm(const __grid_constant__ TcMaps maps, const TcArgs a) {
  using C = Cfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* tfull = empty + C::STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* done_bar = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done_bar + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = units_of(a, BN);
  const int kblocks = (a.K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], NEPI_WARPS);
    }
    mbar_init(done_bar, 1);
    mbar_fence_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < a.nseg; ++s) {
      tma_prefetch_desc(&maps.a[s]);
      tma_prefetch_desc(&maps.b[s]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const UnitPlan pl = plan_unit<BN>(u, a, kblocks);
        if (pl.skip) continue;
        int bm, bn;
        decode_unit(pl.tile, a, pl.n, BN, bm, bn);
        for (int pi = 0; pi < pl.npairs && ok; ++pi) {
          int mi = pi, ya = pl.row0 + bm * BM, yb = pl.row0 + bn * BN;
          if (a.oz_s > 0) {
            const int p = pl.p0 + pi, q = a.oz_diag ? p : pl.t - p;
            mi = 0;
            ya += p * a.oz_ra;
            yb += q * a.oz_rb;
          }
          for (int kb = pl.kb0; kb < pl.kb1; ++kb, ++it) {
            const int st = it % C::STAGES;
            const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
            if (!mbar_wait(&empty[st], ph ^ 1u, a.err_flag, 1)) {
              ok = false;
              break;
            }
            uint8_t* sa = smem + st * C::STAGE;
            mbar_arrive_expect_tx(&full[st], C::STAGE);
            tma_load_2d(sa, &maps.a[mi], kb * BK, ya, &full[st]);
            tma_load_2d(sa + C::A_BYTES, &maps.b[mi], kb * BK, yb, &full[st]);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(BM, BN, a.bf16 != 0, a.acc16 != 0);
      int it = 0, ui = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const UnitPlan pl = plan_unit<BN>(u, a, kblocks);
        if (pl.skip) continue;
        // the residue products hand the accumulator to the epilogue every `sub` K-blocks (an exact
        // FP32 sum of at most that many blocks), each time in the other tensor-memory buffer
        const int sub = (EPI == kEpiCrt8 && a.oz_sub_kb > 0) ? a.oz_sub_kb : (1 << 30);
        int buf = 0, done_kb = 0;
        uint32_t dtm = 0, acc = 0;
        auto take_buffer = [&]() -> bool {
          buf = ui & 1;
          const uint32_t uph = (uint32_t)(ui >> 1) & 1u;
          ++ui;
          if (!mbar_wait(&tempty[buf], uph ^ 1u, a.err_flag, 2)) return false;
          tc_fence_after();
          dtm = tmem_base + (uint32_t)(buf * BN);
          acc = 0;
          return true;
        };
        if (!take_buffer()) break;
        for (int pi = 0; pi < pl.npairs && ok; ++pi) {
          for (int kb = pl.kb0; kb < pl.kb1; ++kb, ++it) {
            if (done_kb == sub) {
              tc_commit(&tfull[buf]);
              if (!take_buffer()) {
                ok = false;
                break;
              }
              done_kb = 0;
            }
            ++done_kb;
            const int st = it % C::STAGES;
            const uint32_t ph = (uint32_t)(it / C::STAGES) & 1u;
            if (!mbar_wait(&full[st], ph, a.err_flag, 3)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + st * C::STAGE);
            const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sa + C::A_BYTES);
#pragma unroll
            for (int k = 0; k < BK / UK; ++k) {
              // advance the start address by k * 16 elements * 2 bytes inside the swizzle atom
              tc_mma_f16(dtm, da + (uint64_t)((k * UK * 2) >> 4), db + (uint64_t)((k * UK * 2) >> 4), idesc, acc);
              acc = 1;
            }
            tc_commit(&empty[st]);
          }
        }
        if (ok) tc_commit(&tfull[buf]);
      }
      tc_commit(done_bar);
      mbar_wait(done_bar, 0, a.err_flag, 4);
    }
  } else {
    const int q = warp & 3;                  // TMEM lane quadrant this warp may access
    const int half = (warp - 2) / 4;         // which half of the tile's columns it handles
    constexpr int CH = BN / 64;              // 32-column chunks per half
    int ui = 0;
    const float osc = a.out_scale ? *a.out_scale : 1.0f;
    float us = a.unscale;
    if (a.sa_ptr) us /= *a.sa_ptr;
    if (a.sb_ptr) us /= *a.sb_ptr;
    float amax = 0.0f;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      const UnitPlan pl = plan_unit<BN>(u, a, kblocks);
      if (pl.skip) continue;
      if constexpr (EPI == kEpiCrt8) {
        // the unit's accumulator arrives in sub-chunks (as many as the MMA issuer hands over); each
        // exact FP32 sum is reduced modulo m and added, in 16-bit halves of one int per column pair
        // (|sum| <= 0.66 m per sub-chunk, 64 sub-chunks at most for N <= 65536, so below 2^14 each),
        // to the running residue sum the digit is formed from
        const int sub = a.oz_sub_kb > 0 ? a.oz_sub_kb : (1 << 30);
        const int total_kb = pl.npairs * (pl.kb1 - pl.kb0);
        const int nsub = (int)(((long long)total_kb + sub - 1) / sub);
        int bm, bn;
        decode_unit(pl.tile, a, pl.n, BN, bm, bn);
        const int i = bm * BM + q * 32 + lane;
        CrtDigitConst cd;
        cd.m = (float)crtw::modulus(pl.t);
        cd.inv = 1.0f / cd.m;
        cd.w = 0.0f;
#pragma unroll
        for (int t = 0; t < 32; ++t)
          if (t == pl.t) cd.w = a.crt_w[t];
        int racc[CH][16];
#pragma unroll
        for (int cc = 0; cc < CH; ++cc)
#pragma unroll
          for (int p2 = 0; p2 < 16; ++p2) racc[cc][p2] = 0;
        bool got = true;
        for (int sc = 0; sc < nsub; ++sc) {
          const int buf = ui & 1;
          const uint32_t uph = (uint32_t)(ui >> 1) & 1u;
          ++ui;
          if (!mbar_wait(&tfull[buf], uph, a.err_flag, 5)) {
            got = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int cc = 0; cc < CH; ++cc) {
            const int c = half * CH + cc;
            if (a.sym && bn * BN + c * 32 + 31 < bm * BM) continue;  // chunk entirely below the diagonal
            float v[32];
            tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c * 32), v);
#pragma unroll
            for (int p2 = 0; p2 < 16; ++p2) {
              const int r0 = (int)crt_fmod_sym(v[2 * p2], cd.m, cd.inv);
              const int r1 = (int)crt_fmod_sym(v[2 * p2 + 1], cd.m, cd.inv);
              racc[cc][p2] += r1 * 65536 + r0;
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        if (!got) break;
        double ss_unused = 0.0;
#pragma unroll
        for (int cc = 0; cc < CH; ++cc) {
          const int c = half * CH + cc;
          const int col0 = bn * BN + c * 32;
          if (a.sym && col0 + 31 < bm * BM) continue;
          float v[32];
#pragma unroll
          for (int p2 = 0; p2 < 16; ++p2) {
            const int lo16 = (int)(short)(racc[cc][p2] & 0xFFFF);
            v[2 * p2] = (float)lo16;
            v[2 * p2 + 1] = (float)((racc[cc][p2] - lo16) >> 16);
          }
          epi_chunk<EPI>(a, i, col0, v, ss_unused, amax, osc, us, pl.group, pl.n, pl.row0, cd);
        }
        continue;
      } else {
        const int buf = ui & 1;
        const uint32_t uph = (uint32_t)(ui >> 1) & 1u;
        ++ui;
        if (!mbar_wait(&tfull[buf], uph, a.err_flag, 5)) break;
        tc_fence_after();
        int bm, bn;
        decode_unit(pl.tile, a, pl.n, BN, bm, bn);
        const int i = bm * BM + q * 32 + lane;
        double ss = 0.0;
        const CrtDigitConst cd{1.0f, 1.0f, 0.0f};
        if constexpr (EPI == kEpiPoly || EPI == kEpiZupd) {
          // the FP32 input row segments of this half (one 128-byte line per chunk) into L1 ahead of use
          const float* src = (EPI == kEpiPoly) ? a.f32_in : a.f32;
          if (src && i < (a.ninst > 0 ? pl.n : a.M)) {
            const float* r = src + ((size_t)pl.row0 + i) * a.ld32 + (size_t)bn * BN + half * CH * 32;
#pragma unroll
            for (int c = 0; c < CH; ++c)
              if (bn * BN + (half * CH + c) * 32 < pl.n) asm volatile("prefetch.global.L1 [%0];" ::"l"(r + c * 32));
          }
        }
#pragma unroll 1
        for (int c = half * CH; c < (half + 1) * CH; ++c) {
          float v[32];
          tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c * 32), v);
          if (a.acc16) widen_acc16(v);
          const int col0 = bn * BN + c * 32;
          if (a.sym && col0 + 31 < bm * BM) continue;  // chunk entirely below the diagonal block
          epi_chunk<EPI>(a, i, col0, v, ss, amax, osc, us, pl.group, pl.n, pl.row0, cd);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
        if constexpr (EPI == kEpiResid) {
          // fixed-order warp reduction; one partial per (tile, quadrant, half), summed in order later
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
          const size_t pidx = a.ninst > 0 ? (size_t)a.g_part0[pl.inst] + (size_t)pl.tile * kTcPartsPerTile
                                          : (size_t)u * kTcPartsPerTile;
          if (lane == 0) a.partials[pidx + half * 4 + q] = ss;
        }
      }
    }
    if (a.amax_bits) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if (lane == 0) atomicMax(a.amax_bits, __float_as_uint(amax));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, C::TMEM_COLS);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

// cuTensorMapEncodeTiled is resolved through the runtime's driver entry-point query, so the
// library carries no link-time dependency on libcuda (it loads on machines without a driver).
static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int tc_make_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows, bool bf16) {
  if ((ld % 8) != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return -1;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return -2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

int tc_num_units(const TcArgs& a, int bn) { return units_of(a, bn); }

template <int BN, int EPI>
static cudaError_t launch_bn(const TcArgs& a, const TcMaps& maps, int num_sms, cudaStream_t s) {
  static bool attr_set = false;
  using C = Cfg<BN>;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int units = units_of(a, BN);
  const int grid = units < num_sms ? units : num_sms;
  if (grid <= 0) return cudaSuccess;
  k_tc_gemm<BN, EPI><<<grid, NTHREADS, C::SMEM, s>>>(maps, a);
  return cudaGetLastError();
}

template <int BN>
static cudaError_t launch_epi(const TcArgs& a, const TcMaps& maps, int num_sms, cudaStream_t s) {
  switch (a.epi) {
    case kEpiStore16: return launch_bn<BN, kEpiStore16>(a, maps, num_sms, s);
    case kEpiResid: return launch_bn<BN, kEpiResid>(a, maps, num_sms, s);
    case kEpiPoly: return launch_bn<BN, kEpiPoly>(a, maps, num_sms, s);
    case kEpiZupd: return launch_bn<BN, kEpiZupd>(a, maps, num_sms, s);
    case kEpiF64: return launch_bn<BN, kEpiF64>(a, maps, num_sms, s);
    case kEpiZupd64: return launch_bn<BN, kEpiZupd64>(a, maps, num_sms, s);
    default: break;
  }
  // the emulation epilogues run on 256-wide tiles only
  if constexpr (BN == 256) {
    if (a.epi == kEpiG32) return launch_bn<BN, kEpiG32>(a, maps, num_sms, s);
    if (a.epi == kEpiCrt8) return launch_bn<BN, kEpiCrt8>(a, maps, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_gemm(const TcArgs& a, const TcMaps& maps, int bn, int num_sms, cudaStream_t s) {
  if (a.oz_s <= 0 && (a.nseg < 1 || a.nseg > kTcMaxSeg)) return cudaErrorInvalidValue;
  if (bn == 256) return launch_epi<256>(a, maps, num_sms, s);
  if (bn == 128) return launch_epi<128>(a, maps, num_sms, s);
  return cudaErrorInvalidValue;
}

}  // namespace zf

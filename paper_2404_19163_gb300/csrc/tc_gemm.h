// Host interface of the tcgen05 GEMM engine (k_tc.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace zf {

constexpr int kTcMaxSeg = 4;
// Err partials the residual epilogue writes per output tile (one per TMEM lane quadrant and column half).
constexpr int kTcPartsPerTile = 8;

// Epilogue of a tensor-core product (acc = sum over segments of A_s B_s^T, FP32).
// v = acc * unscale is the product in true units.
enum TcEpi : int {
  kEpiStore16 = 0,  // o16 (hi[, lo]) = R16(v * out_scale), row-major
  kEpiResid = 1,    // sym: d = I - v; f32 (d) + o16 (d, hi[, lo]) at (i,j) and (j,i); Err partials; amax
  kEpiPoly = 2,     // sym: r = c1 * f32_in + c2 * v -> f32 (r), o16 (r); t16 (v, raw power); mirrored
  kEpiZupd = 3,     // f32_io += v; o16 = R16(f32_io * out_scale) row-major and t16 transposed
  kEpiF64 = 4,      // f64_out = v (double), row-major
  kEpiZupd64 = 5,   // f64_io += v (double); o16/t16 as kEpiZupd from the updated FP64 value
  kEpiG32 = 6,      // f32 + slot * g_stride = raw accumulator (Ozaki group partial), upper only when sym
  kEpiCrt8 = 7,     // d8 + slot * g_stride = CRT digit (acc mod m_t) w_t mod m_t of residue product t
                    // as one byte (row-major, leading dimension ld32), upper only when sym
};

struct TcArgs {
  int M, N, K;        // logical sizes of the product (rows of A, rows of B, reduction length)
  int nseg;           // segments accumulated into one accumulator (K-concatenation)
  int sym;            // upper-triangle tiles only; mirrored writes
  int epi;            // TcEpi
  int bf16;           // operand/output 16-bit format: 1 = BF16, 0 = FP16
  int split_out;      // write the lo part of 16-bit outputs too
  int acc16;          // FP16 accumulator (kind::f16 with D format F16; FP16 operands only)
  float unscale;      // 1 / (scale_A * scale_B), a power of two
  const float* sa_ptr;     // device: extra A scale (unscale /= *sa_ptr), nullptr = none
  const float* sb_ptr;     // device: extra B scale
  const float* out_scale;  // device: scale applied before rounding 16-bit outputs (nullptr = 1)
  const float* p_scale;    // device: scale of the raw-power output of kEpiPoly (nullptr = 1)
  // epilogue operands (row-major, leading dimensions in elements)
  float* f32;  int ld32;        // kEpiResid out (d), kEpiZupd in/out (Z master)
  const float* f32_in;          // kEpiPoly: d in FP32
  double* f64; int ld64;        // kEpiF64 out / kEpiZupd64 in-out
  const double* f64_in;         // kEpiF64: when set, out = c1 f64_in + c2 (product), in FP64 (ld64)
  uint16_t* o16h; uint16_t* o16l; int ld16;
  uint16_t* t16h; uint16_t* t16l;  // kEpiZupd: transposed copy
  float c1, c2;
  double* partials;             // kEpiResid: kTcPartsPerTile per tile, in a fixed order
  unsigned int* amax_bits;      // kEpiResid: max |d| as FP32 bits; kEpiZupd: max |Z|
  int* err_flag;
  // Ozaki mode (oz_s > 0): operands are integer slices stacked along rows (slice p of A at
  // rows p * oz_ra, slice q of B at rows q * oz_rb, one tensor map each); a work unit is
  // (tile, group g) with g = t * oz_nch + c: all slice pairs p + q = t over K-chunk c.
  int oz_s, oz_nch, oz_chunk_kb, oz_ra, oz_rb, oz_c0;  // oz_c0: first K-chunk of this launch
  int oz_tiles;                 // output tiles of the product (units = oz_tiles * oz_s * oz_nch)
  int oz_diag;                  // residue mode: group t holds the one pair (t, t), i.e. oz_s
                                // independent products A_t B_t^T (CRT residues)
  size_t g_stride;              // kEpiG32 / kEpiCrt8: elements between group slots
  uint8_t* d8;                  // kEpiCrt8: digit planes (slot t * oz_nch + c)
  float crt_w[32];              // kEpiCrt8: digit weight w_t of modulus t in this product's plan
  int oz_sub_kb;                // kEpiCrt8: K-blocks per exact FP32 accumulation; a unit's K range is
                                // taken in sub-chunks of this many blocks, each reduced modulo m_t in
                                // the epilogue and summed there (0: the whole range at once)
  // Grouped mode (ninst > 0): independent square problems stacked along the rows of every
  // operand and output buffer (common leading dimensions).  Scheduling slot j covers units
  // [g_prefix[j], g_prefix[j+1]) of instance g_inst[j]; instance i has size g_n[i], first row
  // g_row0[i], first partial g_part0[i], and is skipped entirely while g_done[i] != 0.
  int ninst;
  const int* g_prefix;
  const int* g_inst;
  const int* g_n;
  const int* g_row0;
  const int* g_part0;
  const int* g_done;
};

// Tensor maps of the operands: A segment s is a_maps[s] (M x K, K-major = row-major),
// B segment s is b_maps[s] (N x K, row-major).
struct TcMaps {
  CUtensorMap a[kTcMaxSeg];
  CUtensorMap b[kTcMaxSeg];
};

// Encode a tensor map of a row-major 16-bit matrix (rows x cols, leading dimension ld
// elements, ld % 8 == 0) with a 64-column x box_rows box and 128-byte swizzle.
int tc_make_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows, bool bf16);

int tc_num_units(const TcArgs& a, int bn);
cudaError_t launch_tc_gemm(const TcArgs& a, const TcMaps& maps, int bn, int num_sms, cudaStream_t s);

}  // namespace zf

// Grouped BF16 tensor-core GEMM (tc_gemm.cu): parameters and launchers.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace submat {

constexpr int TC_MAX_SLOTS = 8;
constexpr int TC_MAX_PROD = 16;

struct TcGemmParams {
  const int4* items;        // (s, ti, tj, bucket | slot << 8), 128 x 128 tiles
  int nitems;
  const CUtensorMap* maps;  // device array [set][bucket], 128-row boxes (A operands; B when bn = 128)
  const CUtensorMap* maps_b;  // same sets with 256-row boxes (B operands when bn = 256)
  int bn;                   // output tile width: 128 or 256 (then tmem_cols = 512: nacc = 1 double-
                            // buffered, or nacc = 2 integer accumulators single-buffered)
  int nbucket, nmaps;
  int na, nb;               // A-side and B-side operand slices per k-block
  int a_set[TC_MAX_SLOTS];  // tensor-map set of each A slice
  int b_set[TC_MAX_SLOTS];
  int nprod, nacc;
  int prod_a[TC_MAX_PROD], prod_b[TC_MAX_PROD], prod_acc[TC_MAX_PROD], prod_first[TC_MAX_PROD];
  int nstage, tmem_cols;
  // wave geometry
  const int64_t* off;
  const int32_t* ld;
  const int32_t* n;
  const int* state;
  int skip_state;
  // epilogue: C = alpha * acc + beta * C0 + diag * I_n, written as FP32 or as
  // a BF16 (hi, lo) split
  float alpha, beta, diag;
  int sym;                        // symmetric result: items have ti <= tj; the mirrored tile is
                                  // written too unless upper_only (then a separate pass copies it)
  int upper_only;
  float* out_f32;
  __nv_bfloat16* out_hi;
  __nv_bfloat16* out_lo;          // may be null: plain BF16 output
  const float* c0_f32;
  const __nv_bfloat16* c0_hi;
  const __nv_bfloat16* c0_lo;
  double* res2;                   // optional ||acc - I_n||_F^2 per submatrix (before alpha, beta, diag)
  double* dot_c0;                 // optional: 2 <C, C0> per submatrix (C0 = c0_f32, beta unused)
  // Exact integer output (sliced products, full tiles only): with out_i64 set,
  // the tile value is the integer accumulator times 2^i64_shift, written or
  // (i64_accumulate) added to out_i64; row/column scales are applied later.
  // With nacc = 2 the two accumulators hold adjacent levels: the tile value
  // is (acc0 * 2^i64_dshift + acc1) * 2^i64_shift, 0 <= i64_dshift <= 6.
  long long* out_i64;
  int i64_shift;
  int i64_dshift;
  // lean epilogue: accumulator k carries the weight 2^i64_shifts[k] and up to
  // four accumulators are combined in 64-bit integers (any weights)
  int i64_shifts[4];
  int i64_accumulate;
  // operand and pair format: 0 BF16, 1 FP16 (A and B always share one
  // format; the (hi, lo) output pairs and C0 pairs take the same)
  int f16;
  int* flags;
  long long timeout_cycles;
  int test_skip_arrive;           // test hook: epilogue withholds its TMEM release
};

int tc_smem_bytes(int na, int nb, int nstage, int bn = 128);
int tc_pick_stages(int na, int nb, int bn = 128);
cudaError_t launch_tc_gemm(const TcGemmParams& p, int grid, cudaStream_t st);
// 3D map over a bucket [count][ld][ld] of BF16, box 64 x box_rows x 1, 128B swizzle.
int make_bucket_map(CUtensorMap* out, const void* base, int ld, int count, int box_rows = 128);

}  // namespace submat

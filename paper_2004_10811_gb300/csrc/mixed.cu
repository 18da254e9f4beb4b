// Mixed-precision path: FP16 tensor-core Newton-Schulz, then an FP64-anchored
// correction of the iterate (the paper evaluates sign by FP64
// eigendecomposition, Section IV-F, and reports low-precision GPU iterations,
// Section VI-A; this path combines both).
//
// Why a correction is needed.  Newton-Schulz never looks at a_j after X_0, and
// every involution is a fixed point, so rounding errors that anticommute with
// sign(a) survive all later iterations at full size.  BF16 products leave such
// errors of order 1e-3 (1e-5 with the three-term split hi*hi + hi*lo + lo*hi);
// FP16 (hi, lo) pairs with the same split leave ~1e-6, which is what the
// iteration here uses.
// With S~ = S + F, F = F_c + F_a split into the parts that commute /
// anticommute with S = sign(a):
//   I - S~^2 = -2 S F_c + O(F^2)              =>  F_c = -1/2 S~ (I - S~^2)
//   [S~, a] - [F_c, a] = [F_a, a] = (|a| F_a + F_a |a|) S
// so F_a solves the Lyapunov equation |a| F_a + F_a |a| = C with
// C = ([S~, a] - [F_c, a]) S~ and |a| ~ H = (S~ a + a S~) / 2 (SPD).  Only
// I - S~^2 and S~ a must be accurate to ~1e-10 (FP64 products); everything
// else is a small correction computed with BF16x3 tensor-core products, the
// Lyapunov equation by conjugate gradients to a relative residual tol.  One
// round takes the error from delta to O(delta^2 |a|/gap) + delta tol; from
// the FP16x3 iterate (delta ~1e-6) with tol = 1e-2 this is ~1e-8.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pair.cuh"
#include "plan.cuh"
#include "tc_gemm.cuh"

namespace submat {

long long timeout_cycles_for(double seconds);
int num_sms();

// bytes of workspace per dense element (see MixedBufs)
size_t mixed_bytes_per_elem() { return 8 + 8 + 4 + 8 + 8 + 4 + 4 + 4 + 4 * 4; }

namespace {

enum MapSet {
  MS_XH0, MS_XL0, MS_XH1, MS_XL1, MS_YH, MS_YL, MS_AH, MS_AL, MS_HH, MS_HL, MS_Z0, MS_Z1, MS_COUNT
};

struct MixedBufs {
  double* A;               // a_j (FP64)
  __nv_bfloat16* X[2][2];  // [parity][hi/lo] Newton-Schulz iterate
  __nv_bfloat16* Y[2];     // X^2, later reused for other split operands
  double* S;               // FP64 iterate for the correction
  double* T;               // FP64 residual products (I - S^2, then S a)
  __nv_bfloat16* Ah[2];    // split of a
  __nv_bfloat16* Hh[2];    // split of H
  __nv_bfloat16* Z[2];     // two more BF16 operands (slices)
  float* Fc;               // commuting correction
  float* cx;               // CG solution
  float* cr;               // CG residual (the direction lives in Y as a BF16 pair)
  float* cw;               // H * direction
};

MixedBufs carve(void* ws, int64_t E) {
  MixedBufs b;
  char* p = static_cast<char*>(ws);
  auto take = [&](size_t bytes_per) { char* q = p; p += size_t(E) * bytes_per; return q; };
  b.A = reinterpret_cast<double*>(take(8));
  for (int i = 0; i < 2; ++i)
    for (int k = 0; k < 2; ++k) b.X[i][k] = reinterpret_cast<__nv_bfloat16*>(take(2));
  for (int k = 0; k < 2; ++k) b.Y[k] = reinterpret_cast<__nv_bfloat16*>(take(2));
  b.S = reinterpret_cast<double*>(take(8));
  b.T = reinterpret_cast<double*>(take(8));
  for (int k = 0; k < 2; ++k) b.Ah[k] = reinterpret_cast<__nv_bfloat16*>(take(2));
  for (int k = 0; k < 2; ++k) b.Hh[k] = reinterpret_cast<__nv_bfloat16*>(take(2));
  for (int k = 0; k < 2; ++k) b.Z[k] = reinterpret_cast<__nv_bfloat16*>(take(2));
  b.Fc = reinterpret_cast<float*>(take(4));
  b.cx = reinterpret_cast<float*>(take(4));
  b.cr = reinterpret_cast<float*>(take(4));
  b.cw = reinterpret_cast<float*>(take(4));
  return b;
}

#define FOR_SUB_ELEMS(w)                                                                 \
  const int s = blockIdx.y;                                                              \
  const int ld = (w).ld[s];                                                              \
  const int64_t total = int64_t(ld) * ld;                                                \
  const int64_t base = (w).off[s];                                                       \
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;            \
       e += int64_t(gridDim.x) * blockDim.x)

// Four consecutive entries per thread and step (ld is a multiple of 64, so
// every submatrix has a multiple of four entries and 16-byte aligned rows).
#define FOR_SUB_ELEMS4(w)                                                                \
  const int s = blockIdx.y;                                                              \
  const int ld = (w).ld[s];                                                              \
  const int64_t total4 = int64_t(ld) * ld / 4;                                           \
  const int64_t base = (w).off[s];                                                       \
  for (int64_t e4 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e4 < total4;         \
       e4 += int64_t(gridDim.x) * blockDim.x)

__device__ __forceinline__ float4 load4_f64_trunc(const double* p) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  return make_float4(d2f_trunc(a.x), d2f_trunc(a.y), d2f_trunc(b.x), d2f_trunc(b.y));
}

constexpr int HP_SLICES = 6;  // 6-bit slices per operand in the sliced products
constexpr int HP_BITS = 6;
// slice products kept: p + q <= 8 (26 of 36).  The first dropped level weighs
// ~2^-38 relative to the row and column scales; measured on 1518- and 1748-dim
// submatrices the products are then accurate to ~2e-10, against ~1e-8 when
// stopping at p + q <= 7 (which is too coarse for the 1e-9 trace bound).
constexpr int HP_MAX_LEVEL = 8;

struct SlicePtrs {
  __nv_bfloat16* p[HP_SLICES];
};

// (+-) I * 2^k as a double with integer operations only: round-to-nearest of
// the 64-bit integer to 53 bits, exponent set directly (k within the normal
// range for the values produced here).
__device__ __forceinline__ double i64_to_f64_scaled(long long I, int k, bool negate) {
  if (I == 0) return 0.0;
  unsigned long long sign = 0;
  unsigned long long a = static_cast<unsigned long long>(I);
  if (I < 0) { sign = 1; a = 0ull - a; }
  if (negate) sign ^= 1;
  const int lz = __clzll(static_cast<long long>(a));
  const int msb = 63 - lz;              // value = a * 2^k, a in [2^msb, 2^(msb+1))
  unsigned long long mant;
  int ex = msb + k;
  if (msb <= 52) {
    mant = a << (52 - msb);
  } else {
    const int sh = msb - 52;
    const unsigned long long rem = a & ((1ull << sh) - 1);
    const unsigned long long half = 1ull << (sh - 1);
    mant = a >> sh;
    if (rem > half || (rem == half && (mant & 1))) {
      ++mant;
      if (mant >> 53) { mant >>= 1; ++ex; }
    }
  }
  if (ex + 1023 <= 0) return 0.0;  // below the normal range: flush
  const unsigned long long bits = (sign << 63) | (static_cast<unsigned long long>(ex + 1023) << 52) |
                                  (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double(static_cast<long long>(bits));
}

// The final Newton-Schulz iterate as its FP16 (hi, lo) pair, in buffer 0 or
// 1 per submatrix (par).  The value hi + lo is exact in FP32.
struct PairSrc {
  const __half* hi[2];
  const __half* lo[2];
  const int* par;
};

__device__ __forceinline__ float pair_value(const PairSrc& src, int s, int64_t i) {
  const int k = src.par[s] ? 1 : 0;
  return pair_get(src.hi[k], src.lo[k], i);
}

// the Newton-Schulz buffers hold FP16 pairs (the correction reuses them for
// BF16 operands)
__host__ __device__ __forceinline__ __half* as_h(__nv_bfloat16* p) { return reinterpret_cast<__half*>(p); }

// submax[s] = bit pattern of max |hi + lo| over the iterate of submatrix s
__global__ void k_submax_pair(WaveDev w, PairSrc src, unsigned long long* submax) {
  __shared__ float red[32];
  const int s = blockIdx.y;
  const int ld = w.ld[s];
  const int64_t base = w.off[s];
  const int k = src.par[s] ? 1 : 0;
  const int64_t total4 = int64_t(ld) * ld / 4;
  float mx = 0.0f;
  for (int64_t e4 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e4 < total4;
       e4 += int64_t(gridDim.x) * blockDim.x) {
    const float4 v = load_split4(src.hi[k], src.lo[k], base + 4 * e4);
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int q = 0; q < int(blockDim.x) / 32; ++q) t = fmaxf(t, red[q]);
    atomicMax(&submax[s], (unsigned long long)__double_as_longlong(f2d_exact(t)));
  }
}

// Row-scaled integer slices (the splitting of Ozaki et al.): for row r with
// max_c |X_rc| < 2^e,  X_rc = 2^e sum_{p=1..6} t_p 2^{-6p} + O(2^{e-36}), with
// integers |t_p| <= 63, exact in BF16.  A product of two slice matrices is a sum
// of integers below 63^2 * ld, exact in the FP32 accumulator for ld <= 4096
// (two such products for ld <= 2048).
//
// Grid mode (submax != nullptr): one exponent e for the whole submatrix, from
// the largest |X| of the submatrix (bit pattern in submax), and only the top
// `keep` slices: X is truncated to the grid 2^(e - 6 keep), the truncated
// value written back to X (still symmetric for a symmetric X) and represented
// exactly by its slices.  The sign iterate goes through this mode, so that
// its square needs keep^2 slice products, all exact.
//
// With src.par set (grid mode), the input values are read from that BF16 pair
// instead of X, and the rounded values are written to X.
__global__ void k_slice(WaveDev w, double* X, SlicePtrs out, int* __restrict__ rowexp,
                        const int64_t* __restrict__ voff, const unsigned long long* __restrict__ submax,
                        int keep, __nv_bfloat16* split_hi, __nv_bfloat16* split_lo, PairSrc src) {
  const int s = blockIdx.y;
  const int ld = w.ld[s];
  const int64_t base = w.off[s];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long* Xb = reinterpret_cast<unsigned long long*>(X);
  const bool grid = submax != nullptr;
  const int drop = HP_BITS * (HP_SLICES - keep);  // low bits cleared in grid mode
  int eg = 0;
  if (grid) {
    const unsigned long long mb = submax[s] & 0x7FFFFFFFFFFFFFFFull;
    eg = mb ? int(mb >> 52) - 1023 + 1 : 0;
  }
  for (int r = warp; r < ld; r += nwarps) {
    unsigned long long* row = Xb + base + int64_t(r) * ld;
    int e = eg;
    if (!grid) {
      // the largest |x| of the row, compared as bit patterns
      unsigned long long mb = 0;
      for (int c = lane; c < ld; c += 32) mb = max(mb, row[c] & 0x7FFFFFFFFFFFFFFFull);
      for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
      e = mb ? int(mb >> 52) - 1023 + 1 : 0;  // max |x| < 2^e
    }
    if (lane == 0) rowexp[voff[s] + r] = e;
    for (int c = lane; c < ld; c += 32) {
      const unsigned long long b =
          src.par ? static_cast<unsigned long long>(__double_as_longlong(
                        f2d_exact(pair_value(src, s, base + int64_t(r) * ld + c))))
                  : row[c];
      const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
      const int ex = int(a >> 52) - 1023;
      // fixed = trunc(|x| 2^(36 - e)) = mantissa * 2^(ex - 16 - e), ex < e
      unsigned long long fixed = 0;
      const int sh = e - ex + 16;  // right shift, >= 17
      if ((a >> 52) != 0 && sh < 64)
        fixed = ((a & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> sh;
      const bool neg = (b >> 63) != 0;
      const int64_t i = base + int64_t(r) * ld + c;
      if (grid) {
        fixed = (fixed >> drop) << drop;
        const double v = i64_to_f64_scaled(static_cast<long long>(fixed), e - HP_BITS * HP_SLICES, neg);
        row[c] = static_cast<unsigned long long>(__double_as_longlong(v));
        if (split_hi) split2(v, split_hi, split_lo, i);  // the BF16 pair of the rounded value
      }
#pragma unroll
      for (int q = 0; q < HP_SLICES; ++q) {
        if (q < keep) {
          const int d = int((fixed >> (HP_BITS * (HP_SLICES - 1 - q))) & ((1u << HP_BITS) - 1));
          out.p[q][i] = __int2bfloat16_rn(neg ? -d : d);
        }
      }
    }
  }
}

// I - S^2 from the symmetric slice sum Z = sum_{p<q} 2 w s_p s_q + sum_p w s_p^2
// (s_p symmetric, so s_q s_p = (s_p s_q)^T): S^2 = (Z + Z^T) / 2, exact in
// 64-bit integers (Z + Z^T is even).  Written straight to the BF16 (hi, lo)
// split that the next product reads.  32x32 tile pairs through shared memory;
// block (8, 32): thread (x, y) owns columns 4x..4x+3 of row y.  S is on one
// grid per submatrix, so every entry has the scale 2^(2 e - 48).
__global__ void __launch_bounds__(256) k_hp_finalize_sym(WaveDev w, const long long* __restrict__ Z,
                                                         const int* __restrict__ ex,
                                                         const int64_t* __restrict__ voff,
                                                         __nv_bfloat16* hi, __nv_bfloat16* lo) {
  __shared__ long long ta_[32][33], tb_[32][33];
  const int s = blockIdx.y;
  const int ld = w.ld[s];
  const int n = w.n[s];
  const int64_t base = w.off[s];
  const int k2 = 2 * ex[voff[s]] - HP_BITS * HP_MAX_LEVEL;
  const int T = ld / 32;
  const int npair = T * (T + 1) / 2;
  const int x4 = threadIdx.x * 4, y = threadIdx.y;
  for (int pi = blockIdx.x; pi < npair; pi += gridDim.x) {
    int a = 0, rem = pi;
    while (rem >= T - a) { rem -= T - a; ++a; }
    const int b = a + rem;
    const int64_t iab = base + int64_t(a * 32 + y) * ld + b * 32 + x4;
    const int64_t iba = base + int64_t(b * 32 + y) * ld + a * 32 + x4;
    const longlong2 z0 = *reinterpret_cast<const longlong2*>(Z + iab);
    const longlong2 z1 = *reinterpret_cast<const longlong2*>(Z + iab + 2);
    const longlong2 z2 = *reinterpret_cast<const longlong2*>(Z + iba);
    const longlong2 z3 = *reinterpret_cast<const longlong2*>(Z + iba + 2);
    __syncthreads();
    ta_[y][x4] = z0.x; ta_[y][x4 + 1] = z0.y; ta_[y][x4 + 2] = z1.x; ta_[y][x4 + 3] = z1.y;
    tb_[y][x4] = z2.x; tb_[y][x4 + 1] = z2.y; tb_[y][x4 + 2] = z3.x; tb_[y][x4 + 3] = z3.y;
    __syncthreads();
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long z = (ta_[y][x4 + k] + tb_[x4 + k][y]) >> 1;
      double d = i64_to_f64_scaled(z, k2, true);
      if (a == b && y == x4 + k && a * 32 + y < n) d += 1.0;
      v[k] = d2f_trunc(d);
    }
    store_split4(make_float4(v[0], v[1], v[2], v[3]), hi, lo, iab);
    if (a != b) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long long z = (tb_[y][x4 + k] + ta_[x4 + k][y]) >> 1;
        v[k] = d2f_trunc(i64_to_f64_scaled(z, k2, true));
      }
      store_split4(make_float4(v[0], v[1], v[2], v[3]), hi, lo, iba);
    }
  }
}

// X_0 = a / beta as a (hi, lo) pair (FP16 for the forward iteration, BF16 for
// the tensor-core adjoint's)
template <typename H>
__global__ void k_scale_split(WaveDev w, const double* __restrict__ A, const double* __restrict__ beta,
                              H* xh, H* xl) {
  const float ib = float(1.0 / beta[blockIdx.y]);
  FOR_SUB_ELEMS4(w) {
    const int64_t i = base + 4 * e4;
    const float4 a = load4_f64_trunc(A + i);
    store_split4(make_float4(a.x * ib, a.y * ib, a.z * ib, a.w * ib), xh, xl, i);
  }
}

// X <- f X on the split pair (re-split), f = 1 / (1.05 rho) when it tightens
// the scale; beta follows
template <typename H>
__global__ void k_rescale_split(WaveDev w, H* xh, H* xl, const double* rho, double* beta, const int* state) {
  const int sb = blockIdx.y;
  if (state[sb] == ST_DONE) return;
  const double r = rho[sb];
  if (!(r > 0.0) || r * 1.05 >= 1.0) return;
  const double f = 1.0 / (1.05 * r);
  if (threadIdx.x == 0 && blockIdx.x == 0) beta[sb] = beta[sb] / f;
  const float ff = float(f);
  FOR_SUB_ELEMS4(w) {
    const int64_t i = base + 4 * e4;
    const float4 v = load_split4(xh, xl, i);
    store_split4(make_float4(v.x * ff, v.y * ff, v.z * ff, v.w * ff), xh, xl, i);
  }
}

// Bring every final iterate to parity 0 and widen it: S = hi + lo (FP64).
__device__ __forceinline__ void block_max_bits(float mx, unsigned long long* out) {
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int q = 0; q < int(blockDim.x) / 32; ++q) t = fmaxf(t, red[q]);
    // the FP32 value widened exactly: its bit pattern orders like the value
    atomicMax(out, (unsigned long long)__double_as_longlong(f2d_exact(t)));
  }
}

// ... and submax[s] = max |S| of the submatrix (bit pattern of a bound >= it)
__global__ void k_widen(WaveDev w, const int* __restrict__ par, __half* x0h, __half* x0l,
                        const __half* __restrict__ x1h, const __half* __restrict__ x1l,
                        double* __restrict__ S, unsigned long long* submax) {
  const bool one = par[blockIdx.y] != 0;
  float mx = 0.0f;
  FOR_SUB_ELEMS(w) {
    const int64_t i = base + e;
    const __half h = one ? x1h[i] : x0h[i];
    const __half l = one ? x1l[i] : x0l[i];
    if (one) { x0h[i] = h; x0l[i] = l; }
    const float v = __half2float(h) + __half2float(l);  // exact: at most 22 significant bits
    S[i] = f2d_exact(v);
    mx = fmaxf(mx, fabsf(v));
  }
  block_max_bits(mx, &submax[blockIdx.y]);
}

__global__ void k_split64(WaveDev w, const double* __restrict__ src, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  FOR_SUB_ELEMS4(w) {
    const int64_t i = base + 4 * e4;
    store_split4(load4_f64_trunc(src + i), hi, lo, i);
  }
}

__global__ void k_split32(WaveDev w, const float* __restrict__ src, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  FOR_SUB_ELEMS4(w) {
    const int64_t i = base + 4 * e4;
    store_split4(*reinterpret_cast<const float4*>(src + i), hi, lo, i);
  }
}

// For a 32x32 tile pair (a, b), a <= b, with P = S a (FP64) and W = F_c a (FP32):
//   M = (P - P^T) - (W - W^T)  -> BF16 split (the commutator [S, a] - [F_c, a])
//   H = (P + P^T) / 2          -> BF16 split
// P is either FP64 (Pd) or the exact int64 slice sum Z with row exponents ex
// (rows of S) and ey (columns): P_ij = Z_ij 2^(ex_i + ey_j - 48).  Both
// 32x32 tiles of a pair are converted once into shared memory; block (8, 32):
// thread (x, y) owns columns 4x..4x+3 of row y.
__global__ void __launch_bounds__(256) k_comm(WaveDev w, const double* __restrict__ Pd,
                                              const long long* __restrict__ Z, const int* __restrict__ ex,
                                              const int* __restrict__ ey, const int64_t* __restrict__ voff,
                                              const float* __restrict__ W, __nv_bfloat16* mh, __nv_bfloat16* ml,
                                              __nv_bfloat16* hh, __nv_bfloat16* hl) {
  __shared__ double pa[32][33], pb[32][33];
  __shared__ float wa[32][33], wb[32][33];
  const int s = blockIdx.y;
  const int ld = w.ld[s];
  const int64_t base = w.off[s];
  const int64_t vo = Z ? voff[s] : 0;
  const int T = ld / 32;
  const int npair = T * (T + 1) / 2;
  const int x4 = threadIdx.x * 4, y = threadIdx.y;
  // four entries of row `row`, columns col..col+3, into dst
  auto load4 = [&](int row, int col, double* dst) {
    const int64_t i = base + int64_t(row) * ld + col;
    if (!Z) {
      const double2 u = *reinterpret_cast<const double2*>(Pd + i);
      const double2 v = *reinterpret_cast<const double2*>(Pd + i + 2);
      dst[0] = u.x; dst[1] = u.y; dst[2] = v.x; dst[3] = v.y;
      return;
    }
    const longlong2 u = *reinterpret_cast<const longlong2*>(Z + i);
    const longlong2 v = *reinterpret_cast<const longlong2*>(Z + i + 2);
    const long long z[4] = {u.x, u.y, v.x, v.y};
    const int er = ex[vo + row] - HP_BITS * HP_MAX_LEVEL;
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = i64_to_f64_scaled(z[k], er + ey[vo + col + k], false);
  };
  // M = (P - P^T) - (W - W^T), H = (P + P^T) / 2 for four entries; p - pt
  // cancels to O(delta): the one FP64 operation, the rest in FP32
  auto emit4 = [&](int64_t i, const double* p, const double* pt, const float* wv, const float* wt) {
    float m[4], h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      m[k] = d2f_trunc(p[k] - pt[k]) - (wv[k] - wt[k]);
      h[k] = 0.5f * (d2f_trunc(p[k]) + d2f_trunc(pt[k]));
    }
    store_split4(make_float4(m[0], m[1], m[2], m[3]), mh, ml, i);
    store_split4(make_float4(h[0], h[1], h[2], h[3]), hh, hl, i);
  };
  for (int pi = blockIdx.x; pi < npair; pi += gridDim.x) {
    int a = 0, rem = pi;
    while (rem >= T - a) { rem -= T - a; ++a; }
    const int b = a + rem;
    const int64_t iab = base + int64_t(a * 32 + y) * ld + b * 32 + x4;
    const int64_t iba = base + int64_t(b * 32 + y) * ld + a * 32 + x4;
    double p0[4], p1[4];
    load4(a * 32 + y, b * 32 + x4, p0);
    const float4 w0 = *reinterpret_cast<const float4*>(W + iab);
    float4 w1 = w0;
    if (a != b) {
      load4(b * 32 + y, a * 32 + x4, p1);
      w1 = *reinterpret_cast<const float4*>(W + iba);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) pa[y][x4 + k] = p0[k];
    wa[y][x4] = w0.x; wa[y][x4 + 1] = w0.y; wa[y][x4 + 2] = w0.z; wa[y][x4 + 3] = w0.w;
    if (a != b) {
#pragma unroll
      for (int k = 0; k < 4; ++k) pb[y][x4 + k] = p1[k];
      wb[y][x4] = w1.x; wb[y][x4 + 1] = w1.y; wb[y][x4 + 2] = w1.z; wb[y][x4 + 3] = w1.w;
    }
    __syncthreads();
    double pt[4];
    float wv[4], wt[4];
    const double (*pT)[33] = a == b ? pa : pb;  // the partner tile, read transposed
    const float (*wT)[33] = a == b ? wa : wb;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pt[k] = pT[x4 + k][y];
      wv[k] = wa[y][x4 + k];
      wt[k] = wT[x4 + k][y];
    }
    emit4(iab, p0, pt, wv, wt);
    if (a != b) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        pt[k] = pa[x4 + k][y];
        wv[k] = wb[y][x4 + k];
        wt[k] = wa[x4 + k][y];
      }
      emit4(iba, p1, pt, wv, wt);
    }
  }
}

__device__ __forceinline__ double block_sum(float v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = double(v);
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < int(blockDim.x) / 32; ++q) t += red[q];
  __syncthreads();
  return t;
}

// Complete a symmetric BF16 (hi, lo) pair from its upper triangle: entry
// (r, c), r > c, takes (c, r).  32x32 tile pairs, two per iteration so that
// twice the loads are in flight; block (8, 32).
__global__ void __launch_bounds__(256) k_mirror_split(WaveDev w, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                                      const int* __restrict__ state, int skip_state) {
  __shared__ uint32_t th[2][32][33], tl[2][32][33];  // BF16 bits of the upper tiles
  const int s = blockIdx.y;
  if (state && state[s] == skip_state) return;
  const int ld = w.ld[s];
  const int64_t base = w.off[s];
  const int T = ld / 32;
  const int npair = T * (T + 1) / 2;
  const int x4 = threadIdx.x * 4, y = threadIdx.y;
  const unsigned short* h16 = reinterpret_cast<const unsigned short*>(hi);
  const unsigned short* l16 = reinterpret_cast<const unsigned short*>(lo);
  for (int p0 = blockIdx.x; p0 < npair; p0 += 2 * gridDim.x) {
    int ta[2], tb[2];
    uint2 hv[2], lv[2];
    const int np = p0 + int(gridDim.x) < npair ? 2 : 1;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q < np) {
        int a = 0, rem = p0 + q * int(gridDim.x);
        while (rem >= T - a) { rem -= T - a; ++a; }
        ta[q] = a; tb[q] = a + rem;  // upper tile (a, b), a <= b; lower tile (b, a)
        const int64_t iab = base + int64_t(a * 32 + y) * ld + tb[q] * 32 + x4;
        hv[q] = *reinterpret_cast<const uint2*>(h16 + iab);
        lv[q] = *reinterpret_cast<const uint2*>(l16 + iab);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q < np) {
        th[q][y][x4] = hv[q].x & 0xFFFFu; th[q][y][x4 + 1] = hv[q].x >> 16;
        th[q][y][x4 + 2] = hv[q].y & 0xFFFFu; th[q][y][x4 + 3] = hv[q].y >> 16;
        tl[q][y][x4] = lv[q].x & 0xFFFFu; tl[q][y][x4 + 1] = lv[q].x >> 16;
        tl[q][y][x4 + 2] = lv[q].y & 0xFFFFu; tl[q][y][x4 + 3] = lv[q].y >> 16;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= np) continue;
      const int a = ta[q], b = tb[q];
      // lower tile (b, a), row y, columns x4..x4+3 = upper (a, b) column y, rows x4..x4+3
      const int64_t iba = base + int64_t(b * 32 + y) * ld + a * 32 + x4;
      if (a != b) {
        *reinterpret_cast<uint2*>(hi + iba) = make_uint2(th[q][x4][y] | (th[q][x4 + 1][y] << 16),
                                                         th[q][x4 + 2][y] | (th[q][x4 + 3][y] << 16));
        *reinterpret_cast<uint2*>(lo + iba) = make_uint2(tl[q][x4][y] | (tl[q][x4 + 1][y] << 16),
                                                         tl[q][x4 + 2][y] | (tl[q][x4 + 3][y] << 16));
      } else {
        // diagonal tile: only its strict lower triangle (row y > column x4 + k)
        unsigned short* hd = reinterpret_cast<unsigned short*>(hi) + iba;
        unsigned short* ld16 = reinterpret_cast<unsigned short*>(lo) + iba;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (y > x4 + k) {
            hd[k] = static_cast<unsigned short>(th[q][x4 + k][y]);
            ld16[k] = static_cast<unsigned short>(tl[q][x4 + k][y]);
          }
      }
    }
  }
}

// The same for a symmetric FP32 matrix.
__global__ void __launch_bounds__(256) k_mirror_f32(WaveDev w, float* C) {
  __shared__ float t[32][33];
  const int s = blockIdx.y;
  const int ld = w.ld[s];
  const int64_t base = w.off[s];
  const int T = ld / 32;
  const int npair = T * (T + 1) / 2;
  const int x4 = threadIdx.x * 4, y = threadIdx.y;
  for (int pi = blockIdx.x; pi < npair; pi += gridDim.x) {
    int a = 0, rem = pi;
    while (rem >= T - a) { rem -= T - a; ++a; }
    const int b = a + rem;
    const float4 v = *reinterpret_cast<const float4*>(C + base + int64_t(a * 32 + y) * ld + b * 32 + x4);
    __syncthreads();
    t[y][x4] = v.x; t[y][x4 + 1] = v.y; t[y][x4 + 2] = v.z; t[y][x4 + 3] = v.w;
    __syncthreads();
    float* d = C + base + int64_t(b * 32 + y) * ld + a * 32 + x4;
    if (a != b) {
      *reinterpret_cast<float4*>(d) = make_float4(t[x4][y], t[x4 + 1][y], t[x4 + 2][y], t[x4 + 3][y]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (y > x4 + k) d[k] = t[x4 + k][y];
    }
  }
}

// CG step 2, fused with the symmetrisation: TP = W + W^T read through 32x32
// tile pairs; alpha = rr / pTp; R -= alpha TP; rr_new = <R, R>; and, when X is
// given, X += alpha P.  (On large submatrices X moves in the direction kernel
// instead, which reads P anyway; on small ones the direction kernel's blocks
// are short and the extra bytes cost more there.)
// R, X and P are symmetric, so R and X are kept on the upper tiles only (a
// diagonal tile whole); an upper off-diagonal tile counts twice in <R, R>.
// X's lower triangle is filled once CG ends.
// Block (8, 32): thread (x, y) owns columns 4x..4x+3 of row y of each tile
// (float4 accesses).
template <bool MOVE_X>
__global__ void __launch_bounds__(256) k_cg_update_pairs(WaveDev w, const float* __restrict__ W,
                                                         float* __restrict__ X, float* __restrict__ R,
                                                         const __nv_bfloat16* __restrict__ ph,
                                                         const __nv_bfloat16* __restrict__ pl, const double* rr,
                                                         const double* ptp, double* rr_new,
                                                         const int* __restrict__ cg_done, int* cg_count) {
  __shared__ float tb_[2][32][33];  // W's lower tiles (b, a) of the two pairs in flight
  __shared__ double red[8];
  const int s = blockIdx.y;
  if (cg_done[s]) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && tid == 0) ++cg_count[s];
  const double den = ptp[s];
  const float alpha = (den > 0.0 && rr[s] > 0.0) ? float(rr[s] / den) : 0.0f;
  const int ld = w.ld[s];
  const int64_t base = w.off[s];
  const int T = ld / 32;
  const int npair = T * (T + 1) / 2;
  const int x4 = threadIdx.x * 4, y = threadIdx.y;
  float part = 0.0f;
  // two tile pairs per iteration, every load issued before any store
  for (int p0 = blockIdx.x; p0 < npair; p0 += 2 * gridDim.x) {
    const int np = p0 + int(gridDim.x) < npair ? 2 : 1;
    int64_t iab[2];
    float wgt[2];
    float4 wab[2], wba[2], rv[2], xv[2], pv[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= np) continue;
      int a = 0, rem = p0 + q * int(gridDim.x);
      while (rem >= T - a) { rem -= T - a; ++a; }
      const int b = a + rem;
      iab[q] = base + int64_t(a * 32 + y) * ld + b * 32 + x4;
      wgt[q] = a == b ? 1.0f : 2.0f;
      wab[q] = *reinterpret_cast<const float4*>(W + iab[q]);
      wba[q] = *reinterpret_cast<const float4*>(W + base + int64_t(b * 32 + y) * ld + a * 32 + x4);
      rv[q] = *reinterpret_cast<const float4*>(R + iab[q]);
      if constexpr (MOVE_X) {
        xv[q] = *reinterpret_cast<const float4*>(X + iab[q]);
        pv[q] = load_split4(ph, pl, iab[q]);
      }
    }
    __syncthreads();  // the previous iteration's transposes have been read
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= np) continue;
      tb_[q][y][x4] = wba[q].x; tb_[q][y][x4 + 1] = wba[q].y;
      tb_[q][y][x4 + 2] = wba[q].z; tb_[q][y][x4 + 3] = wba[q].w;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= np) continue;
      // TP = W + W^T on the upper tile (a, b)
      const float tp0 = wab[q].x + tb_[q][x4][y], tp1 = wab[q].y + tb_[q][x4 + 1][y];
      const float tp2 = wab[q].z + tb_[q][x4 + 2][y], tp3 = wab[q].w + tb_[q][x4 + 3][y];
      if constexpr (MOVE_X) {
        float4 x = xv[q];
        x.x = fmaf(alpha, pv[q].x, x.x); x.y = fmaf(alpha, pv[q].y, x.y);
        x.z = fmaf(alpha, pv[q].z, x.z); x.w = fmaf(alpha, pv[q].w, x.w);
        *reinterpret_cast<float4*>(X + iab[q]) = x;
      }
      float4 r = rv[q];
      r.x = fmaf(-alpha, tp0, r.x); r.y = fmaf(-alpha, tp1, r.y);
      r.z = fmaf(-alpha, tp2, r.z); r.w = fmaf(-alpha, tp3, r.w);
      *reinterpret_cast<float4*>(R + iab[q]) = r;
      float sq = 0.0f;
      sq = fmaf(r.x, r.x, sq); sq = fmaf(r.y, r.y, sq);
      sq = fmaf(r.z, r.z, sq); sq = fmaf(r.w, r.w, sq);
      part = fmaf(wgt[q], sq, part);
    }
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) red[tid >> 5] = double(part);
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q];
    atomicAdd(&rr_new[s], t);
  }
}

// CG step 3: when X is given, X += alpha P (X = alpha P on the first step);
// then P = R + (rr_new / rr) P, split for the next product.  Runs exactly when
// the step's update ran (cg_done changes only after this kernel).  P is kept
// only as the BF16 (hi, lo) pair that the product reads, in full (the product
// reads its rows); R and X are read and written on the upper tiles only, and
// P's lower tiles are written from the upper ones through shared memory.
// 32x32 tile pairs, block (8, 32) as in the update.
template <bool MOVE_X>
__global__ void __launch_bounds__(256) k_cg_dir(WaveDev w, const float* __restrict__ R, float* __restrict__ X,
                                                const double* rr, const double* ptp, const double* rr_new,
                                                __nv_bfloat16* ph, __nv_bfloat16* pl,
                                                const int* __restrict__ cg_done, int first) {
  __shared__ float tp_[2][32][33];
  const int s = blockIdx.y;
  if (cg_done[s]) return;
  const double d = rr[s];
  const double den = ptp[s];
  const float alpha = (den > 0.0 && d > 0.0) ? float(d / den) : 0.0f;
  const float beta = d > 0.0 ? float(rr_new[s] / d) : 0.0f;
  const int ld = w.ld[s];
  const int64_t base = w.off[s];
  const int T = ld / 32;
  const int npair = T * (T + 1) / 2;
  const int x4 = threadIdx.x * 4, y = threadIdx.y;
  // two tile pairs per iteration, every load issued before any store
  for (int p0 = blockIdx.x; p0 < npair; p0 += 2 * gridDim.x) {
    const int np = p0 + int(gridDim.x) < npair ? 2 : 1;
    int ta[2], tb[2];
    int64_t iab[2];
    float4 r[2], p[2], x[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= np) continue;
      int a = 0, rem = p0 + q * int(gridDim.x);
      while (rem >= T - a) { rem -= T - a; ++a; }
      ta[q] = a; tb[q] = a + rem;
      iab[q] = base + int64_t(a * 32 + y) * ld + tb[q] * 32 + x4;
      r[q] = *reinterpret_cast<const float4*>(R + iab[q]);
      p[q] = load_split4(ph, pl, iab[q]);
      if constexpr (MOVE_X)
        x[q] = first ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(X + iab[q]);
    }
    float4 pn[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= np) continue;
      if constexpr (MOVE_X) {
        float4 xx = x[q];
        xx.x = fmaf(alpha, p[q].x, xx.x); xx.y = fmaf(alpha, p[q].y, xx.y);
        xx.z = fmaf(alpha, p[q].z, xx.z); xx.w = fmaf(alpha, p[q].w, xx.w);
        *reinterpret_cast<float4*>(X + iab[q]) = xx;
      }
      pn[q] = make_float4(fmaf(beta, p[q].x, r[q].x), fmaf(beta, p[q].y, r[q].y), fmaf(beta, p[q].z, r[q].z),
                          fmaf(beta, p[q].w, r[q].w));
      store_split4(pn[q], ph, pl, iab[q]);
    }
    __syncthreads();  // the previous iteration's transposes have been read
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= np || ta[q] == tb[q]) continue;  // a diagonal tile is whole already
      tp_[q][y][x4] = pn[q].x; tp_[q][y][x4 + 1] = pn[q].y; tp_[q][y][x4 + 2] = pn[q].z; tp_[q][y][x4 + 3] = pn[q].w;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= np || ta[q] == tb[q]) continue;
      // lower tile (b, a), row y, columns x4..x4+3 = upper (a, b) column y, rows x4..x4+3
      const int64_t iba = base + int64_t(tb[q] * 32 + y) * ld + ta[q] * 32 + x4;
      store_split4(make_float4(tp_[q][x4][y], tp_[q][x4 + 1][y], tp_[q][x4 + 2][y], tp_[q][x4 + 3][y]), ph, pl,
                   iba);
    }
  }
}

// CG start: R = P = C (already in R), rr = <C, C>, split P; X = 0 when X is
// given (else the first direction update writes it).
__global__ void k_cg_init(WaveDev w, float* __restrict__ X, const float* __restrict__ R, double* rr,
                          __nv_bfloat16* ph, __nv_bfloat16* pl) {
  __shared__ double red[32];
  float part = 0.0f;
  FOR_SUB_ELEMS4(w) {
    const int64_t i = base + 4 * e4;
    const float4 r = *reinterpret_cast<const float4*>(R + i);
    if (X) *reinterpret_cast<float4*>(X + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    store_split4(r, ph, pl, i);
    part = fmaf(r.x, r.x, part); part = fmaf(r.y, r.y, part);
    part = fmaf(r.z, r.z, part); part = fmaf(r.w, r.w, part);
  }
  const double t = block_sum(part, red);
  if (threadIdx.x == 0) atomicAdd(&rr[blockIdx.y], t);
}

// After the direction update: a submatrix whose relative CG residual
// sqrt(rr / rr0) fell below its tolerance sqrt(tol2[s]) stops (its later CG
// launches return at once).  Counts the submatrices still iterating.
__global__ void k_cg_check(int nsub, const double* rr, const double* rr0, int* cg_done,
                           const double* __restrict__ tol2, int* d_active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  int active = 0;
  if (s < nsub && !cg_done[s]) {
    if (!(rr[s] > tol2[s] * rr0[s])) cg_done[s] = 1;
    else active = 1;
  }
  active = __syncthreads_count(active);
  if (threadIdx.x == 0 && active) atomicAdd(d_active, active);
}

__global__ void k_fill_f64(int n, double* v, double value) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) v[s] = value;
}

// Once every submatrix has reached the loose tolerance: the remaining error
// is ~delta * tol with delta = max |F_c + F_a|, so a submatrix with
// delta * tol > target resumes CG at tol = max(target / delta, tol_tight).
// Counts them.
__global__ void k_cg_tighten(int nsub, const unsigned long long* corr, int* cg_done, double* tol2,
                             double target, double tol_tight, int* d_count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  int more = 0;
  if (s < nsub && cg_done[s]) {
    const double c = __longlong_as_double((long long)corr[s]);
    const double t = sqrt(tol2[s]);
    if (!(c * t <= target)) {
      const double tn = c > 0.0 ? fmax(target / c, tol_tight) : tol_tight;  // c is NaN: tight
      if (tn < t) {
        tol2[s] = tn * tn;
        cg_done[s] = 0;
        more = 1;
      }
    }
  }
  more = __syncthreads_count(more);
  if (threadIdx.x == 0 && more) atomicAdd(d_count, more);
}

// S <- S - F_c - F_a, and corr_s = max |F_c + F_a| (bits of a non-negative double)
__global__ void k_apply(WaveDev w, double* __restrict__ S, const float* __restrict__ Fc,
                        const float* __restrict__ Fa, unsigned long long* corr, unsigned long long* submax) {
  __shared__ double red[32];
  __shared__ unsigned long long redb[32];
  float mx = 0.0f;
  unsigned long long mb = 0;
  FOR_SUB_ELEMS(w) {
    const int64_t i = base + e;
    const float f = Fc[i] + Fa[i];
    const double v = S[i] - f2d_exact(f);
    S[i] = v;
    mx = fmaxf(mx, fabsf(f));
    mb = max(mb, static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  }
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = double(mx); redb[threadIdx.x >> 5] = mb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    unsigned long long tb = 0;
    for (int q = 0; q < int(blockDim.x) / 32; ++q) { t = fmax(t, red[q]); tb = max(tb, redb[q]); }
    atomicMax(&corr[blockIdx.y], (unsigned long long)__double_as_longlong(t));
    atomicMax(&submax[blockIdx.y], tb);
  }
}

// Last round: only max |F_c + F_a| per submatrix (the scatter applies the
// correction to the entries it extracts).
__global__ void k_corr_max(WaveDev w, const float* __restrict__ Fc, const float* __restrict__ Fa,
                           unsigned long long* corr) {
  __shared__ float red[32];
  const int s = blockIdx.y;
  const int ld = w.ld[s];
  const int64_t base = w.off[s];
  const int64_t total4 = int64_t(ld) * ld / 4;
  float mx = 0.0f;
  for (int64_t e4 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e4 < total4;
       e4 += int64_t(gridDim.x) * blockDim.x) {
    const float4 a = *reinterpret_cast<const float4*>(Fc + base + 4 * e4);
    const float4 b = *reinterpret_cast<const float4*>(Fa + base + 4 * e4);
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(a.x + b.x), fabsf(a.y + b.y)), fmaxf(fabsf(a.z + b.z), fabsf(a.w + b.w))));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int q = 0; q < int(blockDim.x) / 32; ++q) t = fmaxf(t, red[q]);
    atomicMax(&corr[s], (unsigned long long)__double_as_longlong(f2d_exact(t)));
  }
}

// Submatrices whose last correction was still large, or whose Lyapunov solve
// did not converge (a gap far smaller than the spectral radius), are
// re-solved by FP64 Newton-Schulz: state ACTIVE for those, DONE for the rest.
// With per-submatrix tolerances (tol2 given), a submatrix is accepted when
// its CG met its own tolerance and either delta * tol <= 2 target (the
// correction grows a little after the tolerance was set) or it ran at
// tol_tight with delta <= corr_tol.
__global__ void k_pick_fallback(WaveDev w, NsStateDev ns, const unsigned long long* corr,
                                const double* rr, const double* rr0, double corr_tol,
                                double cg_tol2, const double* __restrict__ tol2, double tol_tight,
                                double target, int* fallback_flag, int* d_count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  int pick = 0;
  if (s < w.nsub) {
    const double c = __longlong_as_double((long long)corr[s]);
    bool bad;
    if (tol2) {
      const double t = sqrt(tol2[s]);
      const bool small = c * t <= 2.0 * target || (t <= tol_tight * 1.0001 && c <= corr_tol);
      bad = !small || (rr[s] > tol2[s] * 1.0001 * rr0[s]);
    } else {
      bad = !(c <= corr_tol) || (rr[s] > cg_tol2 * rr0[s]);
    }
    fallback_flag[s] = bad ? 1 : 0;
    ns.par[s] = 0;
    if (bad) {
      ns.state[s] = ST_ACTIVE;
      ns.res2[s] = 0.0;
      ns.rprev[s] = 1e300;
      pick = 1;
    } else {
      ns.state[s] = ST_DONE;
    }
  }
  pick = __syncthreads_count(pick);
  if (threadIdx.x == 0 && pick) atomicAdd(d_count, pick);
}

// X_0 = a / beta in FP64 for the submatrices picked for the fallback
__global__ void k_scale_picked(WaveDev w, const int* __restrict__ pick, const double* __restrict__ A,
                               const double* __restrict__ beta, double* __restrict__ X) {
  if (!pick[blockIdx.y]) return;
  const double ib = 1.0 / beta[blockIdx.y];
  FOR_SUB_ELEMS(w) X[base + e] = A[base + e] * ib;
}

// 128 x 256 tiles with a sub-tile on or above the diagonal
int sym256_count(int t128, int t256) {
  int c = 0;
  for (int a = 0; a < t128; ++a)
    for (int b = 0; b < t256; ++b)
      if (2 * b + 1 >= a) ++c;
  return c;
}

dim3 elem_grid(const Wave& wv) {
  // about 32 entries per thread: few, long blocks
  int64_t bx = (wv.max_ld2 + 256 * 32 - 1) / (256 * 32);
  bx = std::max<int64_t>(1, std::min<int64_t>(bx, 256));
  return dim3(unsigned(bx), unsigned(wv.count));
}

dim3 pair_grid(const Wave& wv) {
  int64_t t = 1;
  for (int64_t l : wv.bucket_ld) t = std::max<int64_t>(t, l / 32);
  int64_t np = t * (t + 1) / 2;
  return dim3(unsigned(std::min<int64_t>(np, 512)), unsigned(wv.count));
}

// The same for the streaming tile-pair kernels (CG steps, mirrors): about
// eight pairs per block, so that blocks are few and long enough for their
// launch cost to vanish against their traffic.
dim3 pair_grid_stream(const Wave& wv) {
  int64_t t = 1;
  for (int64_t l : wv.bucket_ld) t = std::max<int64_t>(t, l / 32);
  int64_t np = t * (t + 1) / 2;
  return dim3(unsigned(std::max<int64_t>(1, std::min<int64_t>((np + 7) / 8, 512))), unsigned(wv.count));
}

struct MixedState {
  std::vector<CUtensorMap*> d_maps;  // per wave: [MS_COUNT][nbucket], 128-row boxes
  std::vector<CUtensorMap*> d_maps_b;  // per wave: the same with 256-row boxes
  std::vector<int64_t*> d_voff;      // per wave: offset of each submatrix's row-scale vector
  int* rs_x = nullptr;               // row exponents of the first operand's slices
  int* rs_y = nullptr;               // row exponents of the second operand's slices
  double* scal = nullptr;            // per-slot scalars: rr, ptp, rr_new, rr0 (4 x max_wave)
  int* cg_done = nullptr;            // per slot
  int* cg_count = nullptr;           // per slot: CG iterations run (all rounds)
  unsigned long long* submax = nullptr;  // per slot: bit pattern of max |S|
  int* pick = nullptr;               // per slot: FP64 fallback
  unsigned long long* corr = nullptr;  // per slot: max |correction| of the last round
  double* tol2 = nullptr;            // per slot: squared relative CG tolerance
};

}  // namespace

// Launch plan of an exact sliced product: groups of slice products (one level
// and one weight per exact FP32 accumulator, at most per_acc products),
// sorted by decreasing weight, and launches of up to max_acc groups whose
// slices fit in six operand tiles per stage.  With max_acc = 2 the second
// group is at most 2^6 below the first (the pair is combined in 32-bit
// integers); with more, the epilogue combines in 64-bit integers and any
// weights mix.  Each launch starts from the heaviest group left, so the
// int64 sums grow from the top.
void slice_sets(const SliceGroup* const* gs, int ng, int* as, int* na_out, int* bs, int* nb_out) {
  int na = 0, nb = 0;
  for (int k = 0; k < ng; ++k) {
    const SliceGroup* g = gs[k];
    for (int i = 0; i < g->np; ++i) {
      bool fa = false, fb = false;
      for (int t = 0; t < na; ++t) fa |= as[t] == g->pr[i][0];
      for (int t = 0; t < nb; ++t) fb |= bs[t] == g->pr[i][1];
      if (!fa) as[na++] = g->pr[i][0];
      if (!fb) bs[nb++] = g->pr[i][1];
    }
  }
  *na_out = na;
  *nb_out = nb;
}

void slice_plan(int nx, int ny, bool sym_pairs, int per_acc, int max_acc, std::vector<SliceGroup>* groups_out,
                std::vector<SliceLaunch>* launches) {
  std::vector<SliceGroup>& groups = *groups_out;
  groups.clear();
  launches->clear();
  max_acc = std::max(1, std::min(max_acc, kSliceMaxAcc));
  for (int t = 2; t <= HP_MAX_LEVEL; ++t) {
    int pairs[HP_SLICES][2];
    int np = 0;
    int diag_p = 0;
    for (int pp = 1; pp <= nx; ++pp) {
      const int qq = t - pp;
      if (qq < 1 || qq > ny) continue;
      if (sym_pairs && pp > qq) continue;
      if (sym_pairs && pp == qq) { diag_p = pp; continue; }
      pairs[np][0] = pp; pairs[np][1] = qq; ++np;
    }
    const int shift = HP_BITS * (HP_MAX_LEVEL - t);
    for (int c0 = 0; c0 < np; c0 += per_acc) {
      SliceGroup gr{};
      gr.np = std::min(per_acc, np - c0);
      for (int i = 0; i < gr.np; ++i) { gr.pr[i][0] = pairs[c0 + i][0]; gr.pr[i][1] = pairs[c0 + i][1]; }
      gr.shift = shift + (sym_pairs ? 1 : 0);
      groups.push_back(gr);
    }
    if (diag_p) {
      SliceGroup gr{};
      gr.np = 1; gr.pr[0][0] = gr.pr[0][1] = diag_p; gr.shift = shift;
      groups.push_back(gr);
    }
  }
  std::stable_sort(groups.begin(), groups.end(),
                   [](const SliceGroup& x, const SliceGroup& y) { return x.shift > y.shift; });
  std::vector<char> used(groups.size(), 0);
  for (size_t i = 0; i < groups.size(); ++i) {
    if (used[i]) continue;
    used[i] = 1;
    SliceLaunch L{};
    L.ng = 1;
    L.g[0] = int(i);
    int nprod = groups[i].np;
    while (L.ng < max_acc) {
      int best = -1, best_tiles = 1 << 30;
      for (size_t j = i + 1; j < groups.size(); ++j) {
        if (used[j]) continue;
        if (max_acc == 2 && groups[i].shift - groups[j].shift > 6) continue;
        if (nprod + groups[j].np > 2 * max_acc) continue;
        const SliceGroup* gs[kSliceMaxAcc + 1];
        for (int k = 0; k < L.ng; ++k) gs[k] = &groups[size_t(L.g[k])];
        gs[L.ng] = &groups[j];
        int as[16], bs[16], na = 0, nb = 0;
        slice_sets(gs, L.ng + 1, as, &na, bs, &nb);
        if (na + nb <= 6 && na + nb < best_tiles) { best = int(j); best_tiles = na + nb; }
      }
      if (best < 0) break;
      used[size_t(best)] = 1;
      L.g[L.ng++] = best;
      nprod += groups[size_t(best)].np;
    }
    // accumulators in decreasing weight (accumulator 0 the heaviest)
    std::sort(L.g, L.g + L.ng, [&](int x, int y) { return groups[size_t(x)].shift > groups[size_t(y)].shift; });
    launches->push_back(L);
  }
}

int slice_max_slices() { return HP_SLICES; }

submat_status Plan::sign_mixed(const double* K, double mu, double* D, cudaStream_t st) {
  MixedBufs b = carve(ws, ws_elems);
  auto* ms = static_cast<MixedState*>(mixed);
  if (!ms) {
    ms = new MixedState();
    mixed = ms;
    int64_t vec_max = 1;
    for (auto& wv : waves) {
      const int nbk = int(wv.bucket_ld.size());
      std::vector<CUtensorMap> maps(size_t(MS_COUNT) * nbk);
      const void* bases[MS_COUNT] = {b.X[0][0], b.X[0][1], b.X[1][0], b.X[1][1], b.Y[0], b.Y[1],
                                     b.Ah[0],   b.Ah[1],   b.Hh[0],   b.Hh[1],   b.Z[0], b.Z[1]};
      for (int m = 0; m < MS_COUNT; ++m)
        for (int k = 0; k < nbk; ++k) {
          const __nv_bfloat16* base = static_cast<const __nv_bfloat16*>(bases[m]) + wv.bucket_base[k];
          if (make_bucket_map(&maps[size_t(m) * nbk + k], base, int(wv.bucket_ld[k]),
                              wv.bucket_count[k]) != 0) {
            set_error("cuTensorMapEncodeTiled failed");
            return SUBMAT_ERR_CUDA;
          }
        }
      CUtensorMap* d = nullptr;
      SM_TRY(alloc(&d, maps.size(), "tensor maps"));
      SM_CUDA(cudaMemcpyAsync(d, maps.data(), maps.size() * sizeof(CUtensorMap),
                              cudaMemcpyHostToDevice, st));
      ms->d_maps.push_back(d);
      // the same sets with 256-row boxes for B operands of 128 x 256 tiles
      for (int mset = 0; mset < MS_COUNT; ++mset)
        for (int k = 0; k < nbk; ++k) {
          const __nv_bfloat16* base = static_cast<const __nv_bfloat16*>(bases[mset]) + wv.bucket_base[k];
          if (make_bucket_map(&maps[size_t(mset) * nbk + k], base, int(wv.bucket_ld[k]),
                              wv.bucket_count[k], 256) != 0) {
            set_error("cuTensorMapEncodeTiled failed");
            return SUBMAT_ERR_CUDA;
          }
        }
      CUtensorMap* db = nullptr;
      SM_TRY(alloc(&db, maps.size(), "tensor maps"));
      SM_CUDA(cudaMemcpyAsync(db, maps.data(), maps.size() * sizeof(CUtensorMap),
                              cudaMemcpyHostToDevice, st));
      ms->d_maps_b.push_back(db);
      std::vector<int64_t> vo(wv.count);
      int64_t acc = 0;
      for (int s = 0; s < wv.count; ++s) { vo[s] = acc; acc += wv.host_ld[s]; }
      int64_t* dv = nullptr;
      SM_TRY(put(&dv, vo, st, "row-scale offsets"));
      ms->d_voff.push_back(dv);
      vec_max = std::max(vec_max, acc);
    }
    SM_TRY(alloc(&ms->rs_x, size_t(vec_max), "row scales"));
    SM_TRY(alloc(&ms->rs_y, size_t(vec_max), "row scales"));
    SM_TRY(alloc(&ms->scal, size_t(4) * max_wave, "CG scalars"));
    SM_TRY(alloc(&ms->cg_done, size_t(max_wave), "CG flags"));
    SM_TRY(alloc(&ms->cg_count, size_t(max_wave), "CG counts"));
    SM_TRY(alloc(&ms->pick, size_t(max_wave), "fallback flags"));
    SM_TRY(alloc(&ms->corr, size_t(max_wave), "correction sizes"));
    SM_TRY(alloc(&ms->tol2, size_t(max_wave), "CG tolerances"));
    SM_TRY(alloc(&ms->submax, size_t(max_wave), "iterate maxima"));
  }
  const long long tmo = timeout_cycles_for(2.0);
  const int nsm = num_sms();
  const double floor_thr = 1e-3;
  double* rr = ms->scal;
  double* ptp = rr + max_wave;
  double* rrn = ptp + max_wave;
  double* rr0 = rrn + max_wave;
  int fallback_total = 0;

  for (size_t wi = 0; wi < waves.size(); ++wi) {
    Wave& wv = waves[wi];
    const int nbk = int(wv.bucket_ld.size());
    int bn = 128;
    const int4* SYM = nullptr;
    int NSYM = 0;
    const int4* FULL = nullptr;
    int NFULL = 0;
    // tile width of the tensor-core launches that follow (per phase)
    auto use_width = [&](int want) {
      bn = want == 128 || want == 256 ? want : wv.bn;
      SYM = bn == 256 ? wv.sym256 : wv.sym128;
      NSYM = bn == 256 ? wv.n_sym256 : wv.n_sym128;
      FULL = bn == 256 ? wv.full256 : wv.full128;
      NFULL = bn == 256 ? wv.n_full256 : wv.n_full128;
    };
    use_width(opt.tile_n_ns);
    const int ns_width = bn;
    auto tc = [&](const int4* items, int nitems, int sa0, int sa1, int sb0, int sb1, int sym,
                  float alpha, float beta) {
      TcGemmParams p;
      std::memset(&p, 0, sizeof(p));
      p.items = items;
      p.nitems = nitems;
      p.maps = ms->d_maps[wi];
      p.maps_b = ms->d_maps_b[wi];
      p.bn = bn;
      p.nbucket = nbk;
      p.nmaps = MS_COUNT * nbk;
      p.na = 2; p.nb = 2;
      p.a_set[0] = sa0; p.a_set[1] = sa1;
      p.b_set[0] = sb0; p.b_set[1] = sb1;
      p.nprod = 3;
      const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
      for (int i = 0; i < 3; ++i) { p.prod_a[i] = pa[i]; p.prod_b[i] = pb[i]; p.prod_acc[i] = 0; p.prod_first[i] = i == 0; }
      p.nacc = 1;
      p.nstage = tc_pick_stages(2, 2, bn);
      p.tmem_cols = 2 * bn;
      p.off = wv.dev.off; p.ld = wv.dev.ld; p.n = wv.dev.n;
      p.state = nullptr;
      p.skip_state = -1;
      p.alpha = alpha; p.beta = beta;
      p.sym = sym;
      p.flags = d_flags;
      p.timeout_cycles = tmo;
      return p;
    };
    int tc_class = KC_TC_NS;
    auto launch = [&](const TcGemmParams& p) -> cudaError_t {
      size_t tk;
      if (timer.start(tc_class, st, &tk) != SUBMAT_OK) return cudaErrorUnknown;
      cudaError_t e = launch_tc_gemm(p, std::min(p.nitems, nsm), st);
      if (e == cudaSuccess && timer.stop(tk, st) != SUBMAT_OK) return cudaErrorUnknown;
      return e;
    };
    auto f64 = [&](const GemmF64Args& a) -> cudaError_t {
      size_t tk;
      if (timer.start(KC_SIMT, st, &tk) != SUBMAT_OK) return cudaErrorUnknown;
      cudaError_t e = launch_gemm_f64(a, st);
      if (e == cudaSuccess && timer.stop(tk, st) != SUBMAT_OK) return cudaErrorUnknown;
      return e;
    };

    // ---- assemble and scale (Section III-A step 1) ----
    SM_CUDA(cudaEventRecord(ev[0], st));
    SM_TRY(gather_wave(wv, K, mu, b.A, st));
    const dim3 eg = elem_grid(wv);
    k_scale_split<<<eg, 256, 0, st>>>(wv.dev, b.A, ns.beta, as_h(b.X[0][0]), as_h(b.X[0][1]));
    SM_KCHECK();
    if (opt.beta_mode == 0) {
      // tighter scale: beta = 1.05 x a power estimate of rho(a) (fewer iterations)
      SM_CUDA(launch_power_f16(wv.dev, as_h(b.X[0][0]), kPowerIters, ns.state, ns.rprev, max_ld(wv), st));
      k_rescale_split<<<eg, 256, 0, st>>>(wv.dev, as_h(b.X[0][0]), as_h(b.X[0][1]), ns.rprev, ns.beta,
                                          ns.state);
      SM_KCHECK();
      SM_CUDA(launch_reset_rprev(wv.dev, ns, st));
    }
    SM_CUDA(cudaEventRecord(ev[1], st));

    // ---- FP16x3 Newton-Schulz on the tensor cores ----
    // The iterates are FP16 (hi, lo) pairs: their entries stay below 3 in
    // magnitude, and the three-term split carries ~21 bits against BF16's ~16,
    // so the rounding the correction must remove is ~10x smaller.
    // X_{k+1} = X_k Z_k with Z_k = 1.5 I - 0.5 X_k^2: the squaring writes Z
    // (and the residual ||X^2 - I||_F from its raw accumulator), so the
    // update is a plain product whose epilogue loads nothing
    // Third order (Section VI-A): 8 Z = 15 I - 10 X^2 + 3 X^4 = 3 W^2 + (20/3) I
    // with W = X^2 - (5/3) I, so that no epilogue loads a second operand:
    // W from the squaring, Z = 3/8 W^2 + 5/6 I from a second symmetric product.
    const bool third = opt.iteration == 1;
    int cur = 0;
    // a probe (mu search) caps the iteration: its unconverged submatrices
    // only widen the trace bound
    const int ns_cap = probe_mode ? std::min(opt.max_iter, kProbeMaxIter) : opt.max_iter;
    for (int k = 0; k < ns_cap; ++k) {
      TcGemmParams g1 = tc(SYM, NSYM, cur ? MS_XH1 : MS_XH0, cur ? MS_XL1 : MS_XL0,
                           cur ? MS_XH1 : MS_XH0, cur ? MS_XL1 : MS_XL0, 1, third ? 1.0f : -0.5f, 0.0f);
      g1.diag = third ? -5.0f / 3.0f : 1.5f;
      g1.out_hi = b.Y[0]; g1.out_lo = b.Y[1];
      g1.res2 = ns.res2;
      g1.state = ns.state; g1.skip_state = ST_DONE;
      g1.upper_only = 1;
      g1.f16 = 1;
      SM_CUDA(launch(g1));
      k_mirror_split<<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(wv.dev, b.Y[0], b.Y[1], ns.state, ST_DONE);
      SM_KCHECK();
      if (k == 0 && opt.beta_mode == 0) {  // the power estimate's scale, proven from X_0^2 or reduced
        const CertSquare sq{3, b.Y[0], b.Y[1], g1.alpha, g1.diag};
        const CertLinear lin{1, {b.X[0][0], nullptr, nullptr}, {b.X[0][1], nullptr, nullptr}};
        SM_CUDA(launch_certify(wv.dev, ns, sq, lin, cert_limits(third), max_ld(wv), d_flags + 2, st));
      }
      SM_CUDA(launch_ns_update(wv.dev, ns, tol_eff, floor_thr, ns_cap, d_flags, st));
      int z_hi = MS_YH, z_lo = MS_YL;
      if (third) {  // Z = 3/8 W^2 + 5/6 I into H's buffers
        TcGemmParams gw = tc(SYM, NSYM, MS_YH, MS_YL, MS_YH, MS_YL, 1, 0.375f, 0.0f);
        gw.diag = 5.0f / 6.0f;
        gw.out_hi = b.Hh[0]; gw.out_lo = b.Hh[1];
        gw.state = ns.state; gw.skip_state = ST_DONE;
        gw.upper_only = 1;
        gw.f16 = 1;
        SM_CUDA(launch(gw));
        k_mirror_split<<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(wv.dev, b.Hh[0], b.Hh[1], ns.state, ST_DONE);
        SM_KCHECK();
        z_hi = MS_HH;
        z_lo = MS_HL;
      }
      TcGemmParams g2 = tc(SYM, NSYM, cur ? MS_XH1 : MS_XH0, cur ? MS_XL1 : MS_XL0, z_hi, z_lo, 1, 1.0f, 0.0f);
      g2.out_hi = b.X[cur ^ 1][0]; g2.out_lo = b.X[cur ^ 1][1];
      g2.state = ns.state; g2.skip_state = ST_DONE;
      g2.upper_only = 1;
      g2.f16 = 1;
      SM_CUDA(launch(g2));
      k_mirror_split<<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(wv.dev, b.X[cur ^ 1][0], b.X[cur ^ 1][1], ns.state,
                                                           ST_DONE);
      SM_KCHECK();
      SM_CUDA(cudaMemsetAsync(d_active, 0, sizeof(int), st));
      SM_CUDA(launch_ns_post(wv.dev, ns, cur ^ 1, d_active, st));
      SM_CUDA(cudaMemcpyAsync(h_pinned, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
      SM_CUDA(cudaStreamSynchronize(st));
      cur ^= 1;
      if (reinterpret_cast<int*>(h_pinned)[0] == 0) break;
    }
    SM_CUDA(cudaEventRecord(ev[2], st));

    if (probe_mode) {
      // the FP16x3 iterate as it stands (no correction, no FP64 fallback):
      // S = hi + lo, extracted as it is; the trace bound comes from the
      // submatrices' final residuals (Plan::mu_search)
      SM_CUDA(cudaMemsetAsync(ms->submax, 0, sizeof(unsigned long long) * max_wave, st));
      k_widen<<<eg, 256, 0, st>>>(wv.dev, ns.par, as_h(b.X[0][0]), as_h(b.X[0][1]), as_h(b.X[1][0]),
                                  as_h(b.X[1][1]), b.S, ms->submax);
      SM_KCHECK();
      SM_CUDA(cudaEventRecord(ev[3], st));
      SM_CUDA(launch_scatter_f64(g, wv.dev, ns, b.S, b.S, D, d_trpart, geom(wv), st));
      SM_TRY(collect_wave(wv, st));
      continue;
    }

    // ---- correction rounds ----
    tc_class = KC_TC_REF;
    // split products of the correction: 256-wide tiles (measured 12 % faster
    // per launch than 128 on the 1024x23 workload); the sliced products pick
    // their own width below
    use_width(opt.tile_n_corr ? opt.tile_n_corr : 256);
    std::vector<int> lp_iters(wv.count);
    SM_CUDA(cudaMemcpyAsync(lp_iters.data(), ns.iters, sizeof(int) * wv.count, cudaMemcpyDeviceToHost, st));
    SM_CUDA(cudaMemsetAsync(ms->cg_count, 0, sizeof(int) * max_wave, st));
    // sliced products are exact for K extents up to 4096 (two per accumulator up to 2048)
    int64_t max_ld = 0;
    for (int64_t l : wv.bucket_ld) max_ld = std::max(max_ld, l);
    const bool hp_sliced = opt.hp_mode == 0 && max_ld <= 4096;
    const int per_acc = max_ld <= 2048 ? 2 : 1;
    SM_CUDA(cudaMemsetAsync(ms->submax, 0, sizeof(unsigned long long) * max_wave, st));
    // the final iterate: the sliced path reads its FP16 pair directly (the
    // first slicing writes S); the FP64 residual path widens it to S here
    const PairSrc iterate{{as_h(b.X[0][0]), as_h(b.X[1][0])}, {as_h(b.X[0][1]), as_h(b.X[1][1])}, ns.par};
    if (hp_sliced) {
      k_submax_pair<<<eg, 256, 0, st>>>(wv.dev, iterate, ms->submax);
    } else {
      k_widen<<<eg, 256, 0, st>>>(wv.dev, ns.par, as_h(b.X[0][0]), as_h(b.X[0][1]), as_h(b.X[1][0]),
                                  as_h(b.X[1][1]), b.S, ms->submax);
    }
    SM_KCHECK();
    k_split64<<<eg, 256, 0, st>>>(wv.dev, b.A, b.Ah[0], b.Ah[1]);
    SM_KCHECK();
    static const int S_SETS[HP_SLICES] = {MS_XH0, MS_XL0, MS_XH1, MS_XL1, MS_YH, MS_YL};
    static const int A_SETS[HP_SLICES] = {MS_AH, MS_AL, MS_HH, MS_HL, MS_Z0, MS_Z1};
    SlicePtrs sl_s{{b.X[0][0], b.X[0][1], b.X[1][0], b.X[1][1], b.Y[0], b.Y[1]}};
    SlicePtrs sl_a{{b.Ah[0], b.Ah[1], b.Hh[0], b.Hh[1], b.Z[0], b.Z[1]}};
    // about eight rows per warp (k_slice takes one row per warp at a time)
    const dim3 slice_grid(unsigned(std::max<int64_t>(1, std::min<int64_t>(max_ld / 64, 256))), unsigned(wv.count));
    // C (+)= sign * X Y^T from the slices: level t = p + q weighs 2^(-6 t); each
    // launch sums at most per_acc products of one level in one exact accumulator
    int hp_launch_products = 0;  // slice products issued (all residual products, this wave)
    // out (int64) = sum over kept slice pairs (p, q), p + q <= 8, of
    // 2^(6 (8 - p - q)) X_p Y_q^T.  sym_pairs (X = Y, symmetric slices): only
    // p <= q, the p < q ones counted twice; the symmetric part of the sum is
    // then the full one.
    // Products are grouped into exact FP32 accumulators: one level and one
    // weight each, at most per_acc products.  A launch carries one group, or
    // two groups whose weights differ by at most 2^6 (two TMEM accumulators,
    // combined exactly in the epilogue) when their slices fit in <= 6 operand
    // tiles per stage: fewer launches, so fewer int64 passes.
    auto hp_product = [&](const int* xs, int nx, const int* ys, int ny, bool sym_pairs,
                          double* out) -> submat_status {
      // 128-wide tiles carry up to four accumulators (all of TMEM, single-
      // buffered, combined in 64-bit integers); 256-wide ones two
      const int want_w = opt.tile_n_hp == 256 ? 256 : 128;
      std::vector<SliceGroup> groups;
      std::vector<SliceLaunch> launches;
      slice_plan(nx, ny, sym_pairs, per_acc, want_w == 128 ? kSliceMaxAcc : 2, &groups, &launches);
      bool first = true;
      const int saved_bn = bn;
      auto issue = [&](const SliceLaunch& L) -> submat_status {
        const SliceGroup* gs[kSliceMaxAcc];
        for (int k = 0; k < L.ng; ++k) gs[k] = &groups[size_t(L.g[k])];
        int as[16], bs_[16], na = 0, nb = 0;
        slice_sets(gs, L.ng, as, &na, bs_, &nb);
        // 256-wide tiles when two pipeline stages of the launch's slices fit
        int w = want_w;
        if (w == 256 && tc_smem_bytes(na, nb, 2, 256) > 227 * 1024) w = 128;
        use_width(w);
        TcGemmParams p;
        std::memset(&p, 0, sizeof(p));
        p.items = FULL;
        p.nitems = NFULL;
        p.maps = ms->d_maps[wi];
        p.maps_b = ms->d_maps_b[wi];
        p.bn = bn;
        p.nbucket = nbk;
        p.nmaps = MS_COUNT * nbk;
        p.na = na; p.nb = nb;
        for (int k = 0; k < na; ++k) p.a_set[k] = xs[as[k] - 1];
        for (int k = 0; k < nb; ++k) p.b_set[k] = ys[bs_[k] - 1];
        int np = 0;
        for (int acc = 0; acc < L.ng; ++acc) {
          const SliceGroup* g = gs[acc];
          for (int i = 0; i < g->np; ++i, ++np) {
            int ia = 0, ib = 0;
            while (as[ia] != g->pr[i][0]) ++ia;
            while (bs_[ib] != g->pr[i][1]) ++ib;
            p.prod_a[np] = ia; p.prod_b[np] = ib; p.prod_acc[np] = acc; p.prod_first[np] = i == 0;
          }
          p.i64_shifts[acc] = g->shift;
        }
        p.nprod = np;
        p.nacc = L.ng;
        p.nstage = tc_pick_stages(na, nb, bn);
        // TMEM holds 512 columns: two sets of the accumulators when they fit
        // (the next tile's MMAs overlap this one's drain), else one
        p.tmem_cols = std::min(512, 2 * p.nacc * bn);
        p.off = wv.dev.off; p.ld = wv.dev.ld; p.n = wv.dev.n;
        p.skip_state = -1;
        p.flags = d_flags;
        p.timeout_cycles = tmo;
        p.out_i64 = reinterpret_cast<long long*>(out);
        p.i64_shift = L.ng == 2 ? gs[1]->shift : gs[0]->shift;
        p.i64_dshift = L.ng == 2 ? gs[0]->shift - gs[1]->shift : 0;
        p.i64_accumulate = first ? 0 : 1;
        const int saved = tc_class;
        tc_class = KC_TC_HP;
        const cudaError_t e = launch(p);
        tc_class = saved;
        SM_CUDA(e);
        hp_launch_products += np;
        first = false;
        return SUBMAT_OK;
      };
      for (const SliceLaunch& L : launches) SM_TRY(issue(L));
      use_width(saved_bn);
      return SUBMAT_OK;
    };
    const int rounds = std::max(1, opt.refine_rounds);
    const int cg_max = 60;          // CG cap per round
    // relative residual that ends CG for a submatrix (first correction): the
    // remaining error is ~delta * tol, delta ~1e-6 - 5e-6 from the FP16x3
    // iterate.  All submatrices first run to cg_tol; one whose correction
    // makes delta * cg_tol exceed cg_target resumes to cg_target / delta
    // (at most cg_tol_tight).
    const double cg_tol = 1e-2;
    const double cg_tol_tight = 1e-3;
    const double cg_target = 2e-8;
    const double cg_tol_later = 1e-2;  // later rounds correct an O(1e-9) error: 1e-2 suffices
    const double cg_bad = 1e-2;     // above this after cg_max the submatrix falls back
    const double corr_tol = 1e-8;   // largest acceptable last-round correction
    int cg_total = 0;
    for (int rd = 0; rd < rounds; ++rd) {
      // ---- the two high-precision residual products ----
      // T = I - S^2
      // the first round puts S on a 24-bit grid (four slices, S^2 exact): the
      // rounding (<= 2^-24 max|S|) is well below the FP16x3 error that the
      // round corrects; later rounds, correcting O(1e-9) errors, keep 36 bits
      const int s_keep = rd == 0 ? 4 : HP_SLICES;
      if (rd > 0) {  // a's split, overwritten by its slices in the previous round
        k_split64<<<eg, 256, 0, st>>>(wv.dev, b.A, b.Ah[0], b.Ah[1]);
        SM_KCHECK();
      }
      if (hp_sliced) {
        // slices of S in X (and Y for six), S's BF16 split in Z
        k_slice<<<slice_grid, 256, 0, st>>>(wv.dev, b.S, sl_s, ms->rs_x, ms->d_voff[wi], ms->submax, s_keep,
                                            b.Z[0], b.Z[1], rd == 0 ? iterate : PairSrc{});
        SM_KCHECK();
        SM_TRY(hp_product(S_SETS, s_keep, S_SETS, s_keep, true, b.T));
        // (I - S^2) straight to its split in Y
        k_hp_finalize_sym<<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(
            wv.dev, reinterpret_cast<const long long*>(b.T), ms->rs_x, ms->d_voff[wi], b.Y[0], b.Y[1]);
        SM_KCHECK();
      } else {
        // S's BF16 split for the correction products (in the first round X0
        // still holds the iterate's FP16 pair)
        k_split64<<<eg, 256, 0, st>>>(wv.dev, b.S, b.X[0][0], b.X[0][1]);
        SM_KCHECK();
        GemmF64Args f{};
        f.w = wv.dev; f.items = wv.sym64; f.nitems = wv.n_sym64;
        f.A = b.S; f.B = b.S; f.C0 = nullptr; f.C = b.T;
        f.alpha = -1.0; f.beta = 0.0; f.diag = 1.0; f.sym = 1;
        SM_CUDA(f64(f));
        k_split64<<<eg, 256, 0, st>>>(wv.dev, b.T, b.Y[0], b.Y[1]);
        SM_KCHECK();
      }
      // S's split: Z (sliced path) or X0 (FP64 path)
      const int s_hi = hp_sliced ? MS_Z0 : MS_XH0, s_lo = hp_sliced ? MS_Z1 : MS_XL0;
      // F_c = -1/2 S (I - S^2)
      TcGemmParams g = tc(SYM, NSYM, s_hi, s_lo, MS_YH, MS_YL, 1, -0.5f, 0.0f);
      g.out_f32 = b.Fc;
      g.upper_only = 1;
      SM_CUDA(launch(g));
      k_mirror_f32<<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(wv.dev, b.Fc);
      SM_KCHECK();
      // W = F_c a, before S a so that a's split and Y are free for a's slices
      k_split32<<<eg, 256, 0, st>>>(wv.dev, b.Fc, b.Y[0], b.Y[1]);
      SM_KCHECK();
      TcGemmParams g3 = tc(FULL, NFULL, MS_YH, MS_YL, MS_AH, MS_AL, 0, 1.0f, 0.0f);
      g3.out_f32 = b.cw;
      SM_CUDA(launch(g3));
      // T = S a
      int c_hi = s_hi, c_lo = s_lo;  // S's split for C = M S below
      if (hp_sliced) {
        if (s_keep <= 4) {
          // a's six slices in a's split, H's split and Y (all free now); S's
          // split stays in Z
          static const int A_SETS4[HP_SLICES] = {MS_AH, MS_AL, MS_HH, MS_HL, MS_YH, MS_YL};
          SlicePtrs sl_a4{{b.Ah[0], b.Ah[1], b.Hh[0], b.Hh[1], b.Y[0], b.Y[1]}};
          k_slice<<<slice_grid, 256, 0, st>>>(wv.dev, b.A, sl_a4, ms->rs_y, ms->d_voff[wi], nullptr, HP_SLICES,
                                              nullptr, nullptr, PairSrc{});
          SM_KCHECK();
          SM_TRY(hp_product(S_SETS, s_keep, A_SETS4, HP_SLICES, false, b.T));
        } else {
          // six slices of S again (5 and 6 lived in Y), a's slices over Z,
          // then S's split back in X0
          k_slice<<<slice_grid, 256, 0, st>>>(wv.dev, b.S, sl_s, ms->rs_x, ms->d_voff[wi], ms->submax, s_keep,
                                              nullptr, nullptr, PairSrc{});
          SM_KCHECK();
          k_slice<<<slice_grid, 256, 0, st>>>(wv.dev, b.A, sl_a, ms->rs_y, ms->d_voff[wi], nullptr, HP_SLICES,
                                              nullptr, nullptr, PairSrc{});
          SM_KCHECK();
          SM_TRY(hp_product(S_SETS, s_keep, A_SETS, HP_SLICES, false, b.T));
          k_split64<<<eg, 256, 0, st>>>(wv.dev, b.S, b.X[0][0], b.X[0][1]);
          SM_KCHECK();
          c_hi = MS_XH0;
          c_lo = MS_XL0;
        }
      } else {
        GemmF64Args f2{};
        f2.w = wv.dev; f2.items = wv.full64; f2.nitems = wv.n_full64;
        f2.A = b.S; f2.B = b.A; f2.C0 = nullptr; f2.C = b.T;
        f2.alpha = 1.0; f2.beta = 0.0; f2.diag = 0.0; f2.sym = 0;
        SM_CUDA(f64(f2));
      }
      // M = [S, a] - [F_c, a] (split into Y), H = (S a + a S) / 2 (split)
      // (the sliced S a is read as its exact int64 sum, scaled on the fly)
      k_comm<<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(
          wv.dev, hp_sliced ? nullptr : b.T, hp_sliced ? reinterpret_cast<const long long*>(b.T) : nullptr,
          ms->rs_x, ms->rs_y, ms->d_voff[wi], b.cw, b.Y[0], b.Y[1], b.Hh[0], b.Hh[1]);
      SM_KCHECK();
      // C = M S (symmetric to first order) -> CG residual
      TcGemmParams g4 = tc(SYM, NSYM, MS_YH, MS_YL, c_hi, c_lo, 1, 1.0f, 0.0f);
      g4.out_f32 = b.cr;
      g4.upper_only = 1;
      SM_CUDA(launch(g4));
      k_mirror_f32<<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(wv.dev, b.cr);
      SM_KCHECK();
      // CG on L -> H L + L H, per submatrix until the relative residual is below cg_tol
      SM_CUDA(cudaMemsetAsync(rr, 0, sizeof(double) * 4 * max_wave, st));
      SM_CUDA(cudaMemsetAsync(ms->cg_done, 0, sizeof(int) * max_wave, st));
      // where X moves: in the direction kernel on large submatrices, in the
      // update on small ones (measured: 14.5 against 6.9 ms per direction
      // launch on 504-672-dim submatrices when the direction kernel moves X)
      const bool x_in_dir = max_ld >= 1024 && cg_max > 0;
      k_cg_init<<<eg, 256, 0, st>>>(wv.dev, x_in_dir ? nullptr : b.cx, b.cr, rr, b.Y[0], b.Y[1]);
      SM_KCHECK();
      SM_CUDA(cudaMemcpyAsync(rr0, rr, sizeof(double) * max_wave, cudaMemcpyDeviceToDevice, st));
      // with more rounds to come the first one solves to 1e-4, so that its
      // remaining error (~1e-10) is well inside the last round's 1e-8 test
      const double tol_r = rd > 0 ? cg_tol_later : (rounds >= 2 ? 1e-4 : cg_tol);
      k_fill_f64<<<(wv.count + 255) / 256, 256, 0, st>>>(wv.count, ms->tol2, tol_r * tol_r);
      SM_KCHECK();
      // one round: after the loose tolerance, the size of each correction
      // decides whether delta * cg_tol is small enough (else CG resumes at
      // cg_tol_tight)
      bool tighten = rounds == 1;
      for (int it = 0; it < cg_max; ++it) {
        // W = H P; the epilogue also sums pTp = <P, W + W^T> = 2 <P, W>
        SM_CUDA(cudaMemsetAsync(ptp, 0, sizeof(double) * 2 * max_wave, st));  // ptp and rr_new
        TcGemmParams gh = tc(FULL, NFULL, MS_HH, MS_HL, MS_YH, MS_YL, 0, 1.0f, 0.0f);
        gh.out_f32 = b.cw;
        gh.c0_hi = b.Y[0];
        gh.c0_lo = b.Y[1];
        gh.dot_c0 = ptp;
        gh.state = ms->cg_done; gh.skip_state = 1;
        SM_CUDA(launch(gh));
        // the X-free variants compile as lean as the kernels without X
        if (x_in_dir) {
          k_cg_update_pairs<false><<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(
              wv.dev, b.cw, nullptr, b.cr, b.Y[0], b.Y[1], rr, ptp, rrn, ms->cg_done, ms->cg_count);
          SM_KCHECK();
          k_cg_dir<true><<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(wv.dev, b.cr, b.cx, rr, ptp, rrn, b.Y[0], b.Y[1],
                                                                ms->cg_done, it == 0);
        } else {
          k_cg_update_pairs<true><<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(
              wv.dev, b.cw, b.cx, b.cr, b.Y[0], b.Y[1], rr, ptp, rrn, ms->cg_done, ms->cg_count);
          SM_KCHECK();
          k_cg_dir<false><<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(wv.dev, b.cr, nullptr, rr, ptp, rrn, b.Y[0],
                                                                 b.Y[1], ms->cg_done, 0);
        }
        SM_KCHECK();
        SM_CUDA(cudaMemcpyAsync(rr, rrn, sizeof(double) * max_wave, cudaMemcpyDeviceToDevice, st));
        cg_total += 1;
        {  // convergence test after every step (one 4-byte read)
          SM_CUDA(cudaMemsetAsync(d_active, 0, sizeof(int), st));
          k_cg_check<<<(wv.count + 255) / 256, 256, 0, st>>>(wv.count, rr, rr0, ms->cg_done, ms->tol2,
                                                             d_active);
          SM_KCHECK();
          SM_CUDA(cudaMemcpyAsync(h_pinned, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
          SM_CUDA(cudaStreamSynchronize(st));
          if (reinterpret_cast<int*>(h_pinned)[0] != 0) continue;
          if (!tighten) break;
          tighten = false;
          // max |F_c + F_a|: X's lower triangle from its upper tiles first
          k_mirror_f32<<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(wv.dev, b.cx);
          SM_KCHECK();
          SM_CUDA(cudaMemsetAsync(ms->corr, 0, sizeof(unsigned long long) * max_wave, st));
          k_corr_max<<<eg, 256, 0, st>>>(wv.dev, b.Fc, b.cx, ms->corr);
          SM_KCHECK();
          SM_CUDA(cudaMemsetAsync(d_active, 0, sizeof(int), st));
          k_cg_tighten<<<(wv.count + 255) / 256, 256, 0, st>>>(wv.count, ms->corr, ms->cg_done, ms->tol2,
                                                               cg_target, cg_tol_tight, d_active);
          SM_KCHECK();
          SM_CUDA(cudaMemcpyAsync(h_pinned, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
          SM_CUDA(cudaStreamSynchronize(st));
          if (reinterpret_cast<int*>(h_pinned)[0] == 0) break;
        }
      }
      // CG kept X on its upper tiles: the lower triangle from them
      k_mirror_f32<<<pair_grid_stream(wv), dim3(8, 32), 0, st>>>(wv.dev, b.cx);
      SM_KCHECK();
      SM_CUDA(cudaMemsetAsync(ms->corr, 0, sizeof(unsigned long long) * max_wave, st));
      if (rd + 1 < rounds) {  // S itself is needed by the next round
        SM_CUDA(cudaMemsetAsync(ms->submax, 0, sizeof(unsigned long long) * max_wave, st));
        k_apply<<<eg, 256, 0, st>>>(wv.dev, b.S, b.Fc, b.cx, ms->corr, ms->submax);
      } else {
        k_corr_max<<<eg, 256, 0, st>>>(wv.dev, b.Fc, b.cx, ms->corr);
      }
      SM_KCHECK();
    }
    // ---- FP64 Newton-Schulz for the submatrices the correction could not settle ----
    SM_CUDA(cudaMemsetAsync(d_active, 0, sizeof(int), st));
    // the size of the last correction bounds the remaining error only when an
    // earlier round has already been applied (a single round's correction is
    // the low-precision error itself), so with one round only the CG test applies
    // With one round the remaining error is ~delta^2 |a|/gap + delta tol, and
    // CG reaching its tolerance within cg_max = 60 iterations bounds |a|/gap:
    // accept where delta tol <= 2 cg_target, or where CG ran to cg_tol_tight
    // and delta <= 1e-4.
    k_pick_fallback<<<(wv.count + 255) / 256, 256, 0, st>>>(
        wv.dev, ns, ms->corr, rr, rr0, rounds >= 2 ? corr_tol : 1e-4, cg_bad * cg_bad,
        rounds >= 2 ? nullptr : ms->tol2, cg_tol_tight, cg_target, ms->pick, d_active);
    SM_KCHECK();
    SM_CUDA(cudaMemcpyAsync(h_pinned, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    SM_CUDA(cudaStreamSynchronize(st));
    const int npick = reinterpret_cast<int*>(h_pinned)[0];
    fallback_total += npick;
    double* outS0 = b.S;
    double* outS1 = b.S;
    if (npick > 0) {
      k_scale_picked<<<eg, 256, 0, st>>>(wv.dev, ms->pick, b.A, ns.beta, b.S);
      SM_KCHECK();
      // ping-pong between S and T; A serves as the X^2 buffer
      SM_TRY((ns_simt<double, GemmF64Args>(wv, b.S, b.T, b.A, 1e-14, 1e-9, st, launch_gemm_f64, false)));
      outS1 = b.T;
    }
    stats.refine_rounds = rounds;
    SM_CUDA(cudaEventRecord(ev[3], st));
    // ---- extract (Section III-A step 3); ns.par picks S or, for fallbacks, S/T ----
    SM_TRY(scatter_timed(wv, 24.0, [&] {
      return launch_scatter_f64(g, wv.dev, ns, outS0, outS1, D, d_trpart, geom(wv), st, b.Fc, b.cx, ms->pick);
    }, st));
    SM_TRY(collect_wave(wv, st));
    float t01 = 0, t12 = 0, t23 = 0;
    SM_CUDA(cudaEventElapsedTime(&t01, ev[0], ev[1]));
    SM_CUDA(cudaEventElapsedTime(&t12, ev[1], ev[2]));
    SM_CUDA(cudaEventElapsedTime(&t23, ev[2], ev[3]));
    stats.ms_gather += t01;
    stats.ms_ns += t12;
    stats.ms_refine += t23;
    std::vector<int> cgc(wv.count);
    SM_CUDA(cudaMemcpyAsync(cgc.data(), ms->cg_count, sizeof(int) * wv.count, cudaMemcpyDeviceToHost, st));
    SM_CUDA(cudaStreamSynchronize(st));
    double fl = 0.0;
    for (int s = 0; s < wv.count; ++s) {
      const double n = double(wv.host_n[s]);
      // the cost model's standard count: (CG steps + 4) 2 n^3 per round
      fl += (rounds * 8.0 + 2.0 * cgc[s]) * n * n * n;
    }
    stats.flops_refine += fl;
    stats.refine_cg_iters += cg_total;
    for (int s = 0; s < wv.count; ++s) {
      const double n = double(wv.host_n[s]);
      const double n3 = n * n * n;
      const int extra = res_iters[wv.first + s] - lp_iters[s];  // FP64 fallback iterations
      // algorithmic flops at the standard count, 2 n^3 per n x n product,
      // whatever the kernels skip on symmetric results (a split or sliced
      // product counts once): 4 n^3 per Newton-Schulz step (6 n^3 third
      // order), and per correction round (CG steps + 4) 2 n^3 -- the two
      // residual products, two of the three split products (F_c, W = F_c a
      // and C = M S are executed; the round's cost model counts four) and one
      // per CG step
      stats.kernel_work[KC_TC_NS] += (third ? 3.0 : 2.0) * 2.0 * n3 * lp_iters[s];
      stats.kernel_work[KC_TC_REF] += 2.0 * 2.0 * n3 * rounds + 2.0 * n3 * cgc[s];
      // the two residual products I - S^2 and S a
      if (hp_sliced) stats.kernel_work[KC_TC_HP] += 4.0 * n3 * rounds;
      else stats.kernel_work[KC_SIMT] += 4.0 * n3 * rounds;
      stats.kernel_work[KC_SIMT] += 4.0 * n3 * extra;
      // executed MMA work: tiles x 2 * 128 * width * K per product
      const double ldd = double(wv.host_ld[s]);
      const double t128 = std::ceil(ldd / 128.0);
      const double tns = std::ceil(ldd / ns_width);
      const double sym_tiles_ns = ns_width == 256 ? double(sym256_count(int(t128), int(tns))) : t128 * (t128 + 1) / 2;
      const double tile_ns = 2.0 * 128.0 * ns_width * ldd;
      const double tile128 = 2.0 * 128.0 * 128.0 * ldd;
      stats.kernel_exec[KC_TC_NS] += (third ? 3.0 : 2.0) * lp_iters[s] * 3.0 * sym_tiles_ns * tile_ns;
      const double symt = t128 * (t128 + 1) / 2, fullt = t128 * t128;
      stats.kernel_exec[KC_TC_REF] += rounds * 3.0 * (2.0 * symt + fullt) * tile128 + cgc[s] * 3.0 * fullt * tile128;
      if (hp_sliced) stats.kernel_exec[KC_TC_HP] += double(hp_launch_products) * fullt * tile128;
    }
    stats.refine_fallback = fallback_total;
  }
  return SUBMAT_OK;
}

void free_mixed(void* state) { delete static_cast<MixedState*>(state); }

// ---------------------------------------------------------------------------
// The adjoint on the tensor cores (adjoint_mode = 1)
// ---------------------------------------------------------------------------
// The coupled Newton-Schulz iteration of the adjoint (backward.cu: X, E with
// X_0 = a / beta, E_0 = G / beta) with every product a BF16x3 split product on
// tcgen05.  With Z = 1.5 I - 0.5 X^2 one step is
//     E' = E Z + Z E - 1.5 E - 0.5 X E X,      X' = X Z,
// six products in all: Z (symmetric), U = X E, T = E Z - 1.5 E, T += Z E,
// E' = T - 0.5 U X, and X' = X Z (symmetric).  A product C = A B^T reads B by
// rows, so the two products with E on the right read E's transpose, kept as
// a BF16 pair of its own (a tile-pair transpose after each update).  As in
// the SIMT adjoint every submatrix keeps iterating until all X have converged,
// then two more steps let E settle; the last step leaves E in FP32.
namespace {

enum AdjSet {
  AS_X0H, AS_X0L, AS_X1H, AS_X1L, AS_ZH, AS_ZL, AS_E0H, AS_E0L, AS_E1H, AS_E1L,
  AS_TH, AS_TL, AS_UH, AS_UL, AS_COUNT
};

struct AdjState {
  std::vector<CUtensorMap*> d_maps, d_maps_b;  // per adjoint wave: [AS_COUNT][nbucket]
};

// dst = src^T for a BF16 (hi, lo) pair (src and dst distinct): 32x32 tile
// pairs (a, b), a <= b, both loaded before either is written; block (8, 32).
__global__ void __launch_bounds__(256) k_transpose_split(WaveDev w, const __nv_bfloat16* __restrict__ sh,
                                                         const __nv_bfloat16* __restrict__ sl,
                                                         __nv_bfloat16* __restrict__ dh,
                                                         __nv_bfloat16* __restrict__ dl) {
  __shared__ uint32_t th[2][32][33], tl[2][32][33];  // BF16 bits of tiles (a, b) and (b, a)
  const int s = blockIdx.y;
  const int ld = w.ld[s];
  const int64_t base = w.off[s];
  const int T = ld / 32;
  const int npair = T * (T + 1) / 2;
  const int x4 = threadIdx.x * 4, y = threadIdx.y;
  const unsigned short* h16 = reinterpret_cast<const unsigned short*>(sh);
  const unsigned short* l16 = reinterpret_cast<const unsigned short*>(sl);
  for (int pi = blockIdx.x; pi < npair; pi += gridDim.x) {
    int a = 0, rem = pi;
    while (rem >= T - a) { rem -= T - a; ++a; }
    const int b = a + rem;
    const int64_t iab = base + int64_t(a * 32 + y) * ld + b * 32 + x4;
    const int64_t iba = base + int64_t(b * 32 + y) * ld + a * 32 + x4;
    uint2 hv[2], lv[2];
    hv[0] = *reinterpret_cast<const uint2*>(h16 + iab);
    lv[0] = *reinterpret_cast<const uint2*>(l16 + iab);
    hv[1] = a != b ? *reinterpret_cast<const uint2*>(h16 + iba) : hv[0];
    lv[1] = a != b ? *reinterpret_cast<const uint2*>(l16 + iba) : lv[0];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      th[q][y][x4] = hv[q].x & 0xFFFFu; th[q][y][x4 + 1] = hv[q].x >> 16;
      th[q][y][x4 + 2] = hv[q].y & 0xFFFFu; th[q][y][x4 + 3] = hv[q].y >> 16;
      tl[q][y][x4] = lv[q].x & 0xFFFFu; tl[q][y][x4 + 1] = lv[q].x >> 16;
      tl[q][y][x4 + 2] = lv[q].y & 0xFFFFu; tl[q][y][x4 + 3] = lv[q].y >> 16;
    }
    __syncthreads();
    // dst tile (b, a), row y = src tile (a, b), column y
    *reinterpret_cast<uint2*>(dh + iba) = make_uint2(th[0][x4][y] | (th[0][x4 + 1][y] << 16),
                                                     th[0][x4 + 2][y] | (th[0][x4 + 3][y] << 16));
    *reinterpret_cast<uint2*>(dl + iba) = make_uint2(tl[0][x4][y] | (tl[0][x4 + 1][y] << 16),
                                                     tl[0][x4 + 2][y] | (tl[0][x4 + 3][y] << 16));
    if (a != b) {  // dst tile (a, b), row y = src tile (b, a), column y
      *reinterpret_cast<uint2*>(dh + iab) = make_uint2(th[1][x4][y] | (th[1][x4 + 1][y] << 16),
                                                       th[1][x4 + 2][y] | (th[1][x4 + 3][y] << 16));
      *reinterpret_cast<uint2*>(dl + iab) = make_uint2(tl[1][x4][y] | (tl[1][x4 + 1][y] << 16),
                                                       tl[1][x4 + 2][y] | (tl[1][x4 + 3][y] << 16));
    }
  }
}

// out = hi + lo in FP32
__global__ void k_join32(WaveDev w, const __nv_bfloat16* __restrict__ hi, const __nv_bfloat16* __restrict__ lo,
                         float* __restrict__ out) {
  FOR_SUB_ELEMS(w) out[base + e] = __bfloat162float(hi[base + e]) + __bfloat162float(lo[base + e]);
}

}  // namespace

size_t adjoint_tc_bytes_per_elem() { return 8 + 4 + 2 * AS_COUNT; }  // A, T, the BF16 sets

void free_adjoint_tc(void* state) { delete static_cast<AdjState*>(state); }

submat_status Plan::backward_wave_tc(size_t wi, const double* K, double mu, const double* Dbar, double* Kbar,
                                     double* dn_part, cudaStream_t st) {
  Wave& wv = bwaves[wi];
  const int64_t E = bws_elems;
  double* A = static_cast<double*>(bws);
  float* T = reinterpret_cast<float*>(A + E);
  __nv_bfloat16* P[AS_COUNT];
  for (int i = 0; i < AS_COUNT; ++i) P[i] = reinterpret_cast<__nv_bfloat16*>(T + E) + int64_t(i) * E;
  auto* as = static_cast<AdjState*>(adj_tc);
  if (!as) {
    as = new AdjState();
    adj_tc = as;
  }
  // tensor maps of every adjoint wave (128-row boxes; 256-row boxes for the
  // B operands of 128 x 256 tiles), built once
  while (as->d_maps.size() < bwaves.size()) {
    const Wave& mw = bwaves[as->d_maps.size()];
    const int nb2 = int(mw.bucket_ld.size());
    CUtensorMap* d[2] = {nullptr, nullptr};
    for (int v = 0; v < 2; ++v) {
      std::vector<CUtensorMap> maps(size_t(AS_COUNT) * nb2);
      for (int m = 0; m < AS_COUNT; ++m)
        for (int k = 0; k < nb2; ++k)
          if (make_bucket_map(&maps[size_t(m) * nb2 + k], P[m] + mw.bucket_base[k], int(mw.bucket_ld[k]),
                              mw.bucket_count[k], v ? 256 : 128) != 0) {
            set_error("cuTensorMapEncodeTiled failed");
            return SUBMAT_ERR_CUDA;
          }
      SM_TRY(alloc(&d[v], maps.size(), "tensor maps"));
      SM_CUDA(cudaMemcpyAsync(d[v], maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
      SM_CUDA(cudaStreamSynchronize(st));  // the host array goes out of scope
    }
    as->d_maps.push_back(d[0]);
    as->d_maps_b.push_back(d[1]);
  }
  const int nbk = int(wv.bucket_ld.size());
  const long long tmo = timeout_cycles_for(2.0);
  const int nsm = num_sms();
  constexpr int bn = 256;
  const dim3 eg = elem_grid(wv);
  const dim3 pg = pair_grid(wv);
  const double floor_thr = 1e-3;
  // a BF16x3 split product C = alpha (A B^T) + ..., A and B from the pairs at a0, b0
  auto prm = [&](const int4* items, int nitems, int a0, int b0, int sym) {
    TcGemmParams p;
    std::memset(&p, 0, sizeof(p));
    p.items = items;
    p.nitems = nitems;
    p.maps = as->d_maps[wi];
    p.maps_b = as->d_maps_b[wi];
    p.bn = bn;
    p.nbucket = nbk;
    p.nmaps = AS_COUNT * nbk;
    p.na = 2; p.nb = 2;
    p.a_set[0] = a0; p.a_set[1] = a0 + 1;
    p.b_set[0] = b0; p.b_set[1] = b0 + 1;
    p.nprod = 3;
    const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
    for (int i = 0; i < 3; ++i) { p.prod_a[i] = pa[i]; p.prod_b[i] = pb[i]; p.prod_acc[i] = 0; p.prod_first[i] = i == 0; }
    p.nacc = 1;
    p.nstage = tc_pick_stages(2, 2, bn);
    p.tmem_cols = 2 * bn;
    p.off = wv.dev.off; p.ld = wv.dev.ld; p.n = wv.dev.n;
    p.state = nullptr;
    p.skip_state = -1;
    p.alpha = 1.0f; p.beta = 0.0f; p.diag = 0.0f;
    p.sym = sym;
    p.upper_only = sym;  // symmetric results: upper tiles, then a mirror pass
    p.flags = d_flags;
    p.timeout_cycles = tmo;
    return p;
  };
  auto launch = [&](const TcGemmParams& p) -> cudaError_t {
    size_t tk;
    if (timer.start(KC_TC_ADJ, st, &tk) != SUBMAT_OK) return cudaErrorUnknown;
    cudaError_t e = launch_tc_gemm(p, std::min(p.nitems, nsm), st);
    if (e == cudaSuccess && timer.stop(tk, st) != SUBMAT_OK) return cudaErrorUnknown;
    return e;
  };
  const int passes = dn_part ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    // X_0 = a / beta (the power estimate tightens beta as in the forward path)
    SM_TRY(gather_wave(wv, K, mu, A, st));
    k_scale_split<<<eg, 256, 0, st>>>(wv.dev, A, ns.beta, P[AS_X0H], P[AS_X0L]);
    SM_KCHECK();
    if (opt.beta_mode == 0) {
      SM_CUDA(launch_power_bf16(wv.dev, P[AS_X0H], kPowerIters, ns.state, ns.rprev, max_ld(wv), st));
      k_rescale_split<<<eg, 256, 0, st>>>(wv.dev, P[AS_X0H], P[AS_X0L], ns.rprev, ns.beta, ns.state);
      SM_KCHECK();
      SM_CUDA(launch_reset_rprev(wv.dev, ns, st));
    }
    // E_0 = G / beta (pass 1: I / beta) with the final beta, its pair and transpose
    SM_CUDA(launch_bwd_seed_f32(g, wv, Dbar, ns.beta, T, pass, st));
    k_split32<<<eg, 256, 0, st>>>(wv.dev, T, P[AS_E0H], P[AS_E0L]);
    SM_KCHECK();
    k_transpose_split<<<pg, dim3(8, 32), 0, st>>>(wv.dev, P[AS_E0H], P[AS_E0L], P[AS_TH], P[AS_TL]);
    SM_KCHECK();
    int cur = 0, extra = -1, steps = 0, updates = 0;
    bool in_t = false;  // E left in T (FP32) by the last step
    for (int k = 0; k < opt.max_iter + 2; ++k) {
      const bool last = extra == 1;
      const int xs = cur ? AS_X1H : AS_X0H, xn = cur ? AS_X0H : AS_X1H;
      const int es = cur ? AS_E1H : AS_E0H, en = cur ? AS_E0H : AS_E1H;
      // Z = 1.5 I - 0.5 X^2, with the involution residual while X iterates
      TcGemmParams g1 = prm(wv.sym256, wv.n_sym256, xs, xs, 1);
      g1.alpha = -0.5f;
      g1.diag = 1.5f;
      g1.out_hi = P[AS_ZH]; g1.out_lo = P[AS_ZL];
      if (extra < 0) g1.res2 = ns.res2;
      SM_CUDA(launch(g1));
      k_mirror_split<<<pg, dim3(8, 32), 0, st>>>(wv.dev, P[AS_ZH], P[AS_ZL], nullptr, 0);
      SM_KCHECK();
      if (k == 0 && opt.beta_mode == 0) {  // as in the forward path; E_0 and E_0^T follow X_0
        const CertSquare sq{2, P[AS_ZH], P[AS_ZL], g1.alpha, g1.diag};
        const CertLinear lin{3, {P[AS_X0H], P[AS_E0H], P[AS_TH]}, {P[AS_X0L], P[AS_E0L], P[AS_TL]}};
        SM_CUDA(launch_certify(wv.dev, ns, sq, lin, cert_limits(false), max_ld(wv), d_flags + 2, st));
      }
      if (extra < 0) SM_CUDA(launch_ns_update(wv.dev, ns, tol_eff, floor_thr, opt.max_iter, d_flags, st));
      // U = X E (B: E^T)
      TcGemmParams gu = prm(wv.full256, wv.n_full256, xs, AS_TH, 0);
      gu.out_hi = P[AS_UH]; gu.out_lo = P[AS_UL];
      SM_CUDA(launch(gu));
      // T = E Z - 1.5 E
      TcGemmParams ga = prm(wv.full256, wv.n_full256, es, AS_ZH, 0);
      ga.beta = -1.5f;
      ga.c0_hi = P[es]; ga.c0_lo = P[es + 1];
      ga.out_f32 = T;
      SM_CUDA(launch(ga));
      // T += Z E (B: E^T)
      TcGemmParams gb = prm(wv.full256, wv.n_full256, AS_ZH, AS_TH, 0);
      gb.beta = 1.0f;
      gb.c0_f32 = T;
      gb.out_f32 = T;
      SM_CUDA(launch(gb));
      // E' = T - 0.5 U X
      TcGemmParams gc = prm(wv.full256, wv.n_full256, AS_UH, xs, 0);
      gc.alpha = -0.5f;
      gc.beta = 1.0f;
      gc.c0_f32 = T;
      if (last) {
        gc.out_f32 = T;
      } else {
        gc.out_hi = P[en]; gc.out_lo = P[en + 1];
      }
      SM_CUDA(launch(gc));
      ++steps;
      if (last) {
        in_t = true;
        break;
      }
      // X' = X Z, then E'^T for the next step
      TcGemmParams g2 = prm(wv.sym256, wv.n_sym256, xs, AS_ZH, 1);
      g2.out_hi = P[xn]; g2.out_lo = P[xn + 1];
      SM_CUDA(launch(g2));
      ++updates;
      k_mirror_split<<<pg, dim3(8, 32), 0, st>>>(wv.dev, P[xn], P[xn + 1], nullptr, 0);
      SM_KCHECK();
      k_transpose_split<<<pg, dim3(8, 32), 0, st>>>(wv.dev, P[en], P[en + 1], P[AS_TH], P[AS_TL]);
      SM_KCHECK();
      if (extra < 0) {
        SM_CUDA(cudaMemsetAsync(d_active, 0, sizeof(int), st));
        SM_CUDA(launch_ns_post(wv.dev, ns, cur ^ 1, d_active, st));
        SM_CUDA(cudaMemcpyAsync(h_pinned, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        SM_CUDA(cudaStreamSynchronize(st));
        if (reinterpret_cast<int*>(h_pinned)[0] == 0) extra = 2;  // E settles in two more steps
      } else {
        --extra;
      }
      cur ^= 1;
    }
    if (!in_t) {  // the step cap ended the loop: E is the current pair
      const int es = cur ? AS_E1H : AS_E0H;
      k_join32<<<eg, 256, 0, st>>>(wv.dev, P[es], P[es + 1], T);
      SM_KCHECK();
    }
    if (pass == 0) {
      SM_CUDA(launch_bwd_scatter_add_f32(g, wv, nb_max, T, Kbar, st));
    } else {
      SM_CUDA(launch_bwd_dn_f32(g, wv, T, dn_part, st));
      std::vector<double> part(wv.count);
      SM_CUDA(cudaMemcpyAsync(part.data(), dn_part, sizeof(double) * wv.count, cudaMemcpyDeviceToHost, st));
      SM_CUDA(cudaStreamSynchronize(st));
      for (double v : part) dn_acc += v;
    }
    if (timer.on) {  // executed MMA work: three MMAs per split product, tiles x 2 * 128 * 256 * K
      for (int s = 0; s < wv.count; ++s) {
        const double ldd = double(wv.host_ld[s]);
        const int t128 = int(std::ceil(ldd / 128.0)), t256 = int(std::ceil(ldd / 256.0));
        const double tile = 2.0 * 128.0 * 256.0 * ldd;
        stats.kernel_exec[KC_TC_ADJ] +=
            3.0 * tile * (double(sym256_count(t128, t256)) * (steps + updates) + 4.0 * t128 * t256 * steps);
      }
    }
  }
  int fl = 0;
  SM_TRY(read_flags(st, &fl));
  if (fl & FLAG_TIMEOUT) {
    set_error("a bounded device wait timed out (tensor-core adjoint)");
    return SUBMAT_ERR_TIMEOUT;
  }
  SM_TRY(collect_wave(wv, st));
  return SUBMAT_OK;
}

}  // namespace submat

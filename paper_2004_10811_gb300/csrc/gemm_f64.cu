// Grouped FP64 / FP32 GEMM over the submatrix batch (the plain FP64 and FP32
// Newton-Schulz paths and the high-precision residual products of the
// refinement).
//
// One CTA computes one 64x64 tile (s, ti, tj) of C = alpha A B + beta C0 for
// submatrix s; A, B, C0, C are row-major n x n blocks with leading dimension
// ld (a multiple of 64) at the same wave offset in each buffer.  FP64 is
// issued with DFMA from registers (4x4 outputs per thread, 16-deep k slices
// staged in shared memory with a register prefetch of the next slice).
// The FP32 instantiation issues FFMA with the same structure.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace submat {

namespace {

constexpr int TM = 64;
constexpr int TK = 16;

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

template <typename T, typename Args>
__global__ void __launch_bounds__(256) k_gemm_simt(Args a) {
  using V2 = typename Vec2<T>::type;
  __shared__ __align__(16) T As[TK][TM + 2];  // As[k][m]
  __shared__ __align__(16) T Bs[TK][TM];      // Bs[k][n]
  __shared__ double red[8];
  const int4 item = a.items[blockIdx.x];
  const int s = item.x, ti = item.y, tj = item.z;
  if (a.state != nullptr && a.state[s] == a.skip_state) return;
  const int ld = a.w.ld[s];
  const int64_t off = a.w.off[s];
  const T* __restrict__ Ab = a.A + off + int64_t(ti) * TM * ld;
  const T* __restrict__ Bb = a.B + off + int64_t(tj) * TM;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // loader mapping
  const int a_row = tid >> 2, a_k = (tid & 3) * 4;   // A: 64 rows x 16 k
  const int b_k = tid >> 4, b_n = (tid & 15) * 4;    // B: 16 k x 64 n
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  V2 ra0, ra1, rb0, rb1;
  {
    const T* pa = Ab + int64_t(a_row) * ld + a_k;
    ra0 = *reinterpret_cast<const V2*>(pa);
    ra1 = *reinterpret_cast<const V2*>(pa + 2);
    const T* pb = Bb + int64_t(b_k) * ld + b_n;
    rb0 = *reinterpret_cast<const V2*>(pb);
    rb1 = *reinterpret_cast<const V2*>(pb + 2);
  }
  const int nk = ld / TK;
  for (int kt = 0; kt < nk; ++kt) {
    As[a_k + 0][a_row] = ra0.x;
    As[a_k + 1][a_row] = ra0.y;
    As[a_k + 2][a_row] = ra1.x;
    As[a_k + 3][a_row] = ra1.y;
    *reinterpret_cast<V2*>(&Bs[b_k][b_n]) = rb0;
    *reinterpret_cast<V2*>(&Bs[b_k][b_n + 2]) = rb1;
    __syncthreads();
    if (kt + 1 < nk) {
      const int k0 = (kt + 1) * TK;
      const T* pa = Ab + int64_t(a_row) * ld + k0 + a_k;
      ra0 = *reinterpret_cast<const V2*>(pa);
      ra1 = *reinterpret_cast<const V2*>(pa + 2);
      const T* pb = Bb + int64_t(k0 + b_k) * ld + b_n;
      rb0 = *reinterpret_cast<const V2*>(pb);
      rb1 = *reinterpret_cast<const V2*>(pb + 2);
    }
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[k][ty * 4 + i];
      const V2 b01 = *reinterpret_cast<const V2*>(&Bs[k][tx * 4]);
      const V2 b23 = *reinterpret_cast<const V2*>(&Bs[k][tx * 4 + 2]);
      bv[0] = b01.x; bv[1] = b01.y; bv[2] = b23.x; bv[3] = b23.y;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }

  // epilogue
  const int n = a.w.n[s];
  T* Cb = a.C + off;
  const T* C0b = a.C0 ? a.C0 + off : nullptr;
  double part = 0.0;
  const int r0 = ti * TM + ty * 4, c0 = tj * TM + tx * 4;
  T v[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + i;
    V2 z0, z1;
    z0.x = z0.y = z1.x = z1.y = T(0);
    if (C0b) {
      z0 = *reinterpret_cast<const V2*>(C0b + int64_t(r) * ld + c0);
      z1 = *reinterpret_cast<const V2*>(C0b + int64_t(r) * ld + c0 + 2);
    }
    const T zc[4] = {z0.x, z0.y, z1.x, z1.y};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T x = T(a.alpha) * acc[i][j];
      if (C0b) x = fma(T(a.beta), zc[j], x);
      if (a.diag != 0.0 && r == c0 + j && r < n) x += T(a.diag);
      v[i][j] = x;
      if (a.res2) {
        const int c = c0 + j;
        const double e = double(x) - ((r == c && r < n) ? 1.0 : 0.0);
        part = fma(e, e, part);
      }
    }
    V2 w0, w1;
    w0.x = v[i][0]; w0.y = v[i][1]; w1.x = v[i][2]; w1.y = v[i][3];
    *reinterpret_cast<V2*>(Cb + int64_t(r) * ld + c0) = w0;
    *reinterpret_cast<V2*>(Cb + int64_t(r) * ld + c0 + 2) = w1;
  }
  if (a.sym && ti != tj) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T* row = Cb + int64_t(c0 + j) * ld + r0;
      V2 w0, w1;
      w0.x = v[0][j]; w0.y = v[1][j]; w1.x = v[2][j]; w1.y = v[3][j];
      *reinterpret_cast<V2*>(row) = w0;
      *reinterpret_cast<V2*>(row + 2) = w1;
    }
  }
  if (a.res2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += red[q];
      if (a.sym && ti != tj) t *= 2.0;
      atomicAdd(&a.res2[s], t);
    }
  }
}

}  // namespace

cudaError_t launch_gemm_f64(const GemmF64Args& a, cudaStream_t st) {
  if (a.nitems <= 0) return cudaSuccess;
  k_gemm_simt<double, GemmF64Args><<<a.nitems, 256, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gemm_f32(const GemmF32Args& a, cudaStream_t st) {
  if (a.nitems <= 0) return cudaSuccess;
  k_gemm_simt<float, GemmF32Args><<<a.nitems, 256, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace submat

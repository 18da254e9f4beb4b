// Scale certificate for X_0 = f a / beta_bound.
//
// Newton-Schulz X <- X (3I - X^2) / 2 (Section II-B) keeps the sign of an
// eigenvalue x only for |x| < sqrt(3); one in (sqrt 3, sqrt 5) converges to the
// opposite sign, and the result is still an involution that commutes with a,
// so neither the stopping test nor the correction can notice.  The third-order
// iteration X (15I - 10X^2 + 3X^4) / 8 never flips a sign but diverges beyond
// its repelling fixed point sqrt(7/3).
//
// beta_bound = min(max row abs-sum, ||a||_F) >= rho(a) is rigorous, but loose
// (3-5x rho on the water-like workloads).  The power estimate f = 1 / (1.05 r)
// is tight but only a lower bound on rho: a start vector nearly orthogonal to
// the dominant eigenvector underestimates it.  A scale f <= fcap is safe
// whatever the estimate says.  Above fcap the first squaring, which the
// iteration computes anyway, certifies the scale: for any matrix norm
// rho(X_0)^2 = rho(X_0^2) <= ||X_0^2||_inf, the largest row abs-sum.  Where the
// certificate (with a bound on the rounding of the computed square) does not
// prove rho(X_0)^2 <= gmax, X_0 is scaled by
//     c = max(sqrt(gmax / G), fcap / f) < 1,
// either factor alone being safe, and the square, E_0 (the adjoint's seed) and
// beta follow: (cX)^2 = c^2 X^2, so no product is recomputed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "pair.cuh"

namespace submat {

namespace {

__device__ __forceinline__ double bits_to_double(unsigned long long b) {
  return __longlong_as_double(static_cast<long long>(b));
}

// Largest row abs-sum of X^2 per submatrix (rows and columns < n), decoded
// from the square's representation.  One warp per row; FP32 partial sums per
// lane (ld / 32 terms), the warp total in FP64.
__global__ void __launch_bounds__(256) k_cert_rowsum(WaveDev w, CertSquare sq, const int* __restrict__ state,
                                                     unsigned long long* __restrict__ cert) {
  const int s = blockIdx.y;
  if (state[s] != ST_ACTIVE) return;
  const int n = w.n[s], ld = w.ld[s];
  const int64_t base = w.off[s];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float ia = 1.0f / sq.alpha;
  double best = 0.0;
  for (int r = blockIdx.x * 8 + warp; r < n; r += gridDim.x * 8) {
    const int64_t row = base + int64_t(r) * ld;
    float acc = 0.0f;
    if (sq.mode >= 2) {
      for (int c = lane * 4; c < ld; c += 128) {
        const float4 q = sq.mode == 3 ? load_split4(static_cast<const __half*>(sq.hi),
                                                    static_cast<const __half*>(sq.lo), row + c)
                                      : load_split4(static_cast<const __nv_bfloat16*>(sq.hi),
                                                    static_cast<const __nv_bfloat16*>(sq.lo), row + c);
        const float v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float d = (c + k == r) ? sq.diag : 0.0f;  // padding columns hold q = 0
          acc += fabsf((v[k] - d) * ia);
        }
      }
    } else if (sq.mode == 1) {
      const float* x = static_cast<const float*>(sq.hi);
      for (int c = lane; c < ld; c += 32) acc += fabsf(x[row + c]);
    } else {
      const double* x = static_cast<const double*>(sq.hi);
      for (int c = lane; c < ld; c += 32) acc += fabsf(float(x[row + c]));
    }
    double t = double(acc);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    best = fmax(best, t);
  }
  if (lane == 0 && best > 0.0) atomicMax(&cert[s], (unsigned long long)__double_as_longlong(best));
}

// Per submatrix: is the scale proven safe?  If not, the factor c < 1.
//   f  = beta_bound / beta   (the power estimate's tightening)
//   gx = f gersh / beta_bound >= the largest row abs-sum of |X_0|, which bounds
//        the rounding of the computed square: |err_rc| <= eps sum_k |X_rk||X_kc|
__global__ void k_cert_decide(WaveDev w, NsStateDev ns, double gmax, double fcap, double eps0, double eps_ld,
                              int* count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= w.nsub) return;
  ns.cscale[s] = 1.0;
  if (ns.state[s] != ST_ACTIVE) return;
  const double gersh = bits_to_double(ns.gersh[s]);
  const double bound = fmin(gersh, sqrt(ns.fro2[s])) * (1.0 + 1e-4);  // as the bound beta
  const double beta = ns.beta[s];
  if (!(bound > 0.0) || !(beta > 0.0)) return;
  const double f = bound / beta;
  if (f <= fcap) return;  // rho(X_0) <= f rho(a) / beta_bound <= fcap
  const int ld = w.ld[s];
  const double gx = f * gersh / bound;
  const double G = bits_to_double(ns.cert[s]) * (1.0 + ld * 0x1p-24) + (eps0 + eps_ld * ld) * gx * gx;
  if (G <= gmax) return;  // rho(X_0)^2 <= ||X_0^2||_inf <= G <= gmax
  const double c = fmax(sqrt(gmax / G), fcap / f);
  ns.cscale[s] = c;
  ns.beta[s] = beta / c;
  ns.res2[s] = 0.0;  // recomputed for the rescaled square
  atomicAdd(count, 1);
}

// Rescale the submatrices the certificate did not accept: the linear buffers
// by c, the square q = diag I + alpha X^2 to diag I + alpha c^2 X^2, and the
// residual ||X^2 - I||_F^2 recomputed from the new square.  Four consecutive
// entries of a row per thread (ld is a multiple of 64).
template <typename T>
__global__ void __launch_bounds__(256) k_cert_apply(WaveDev w, NsStateDev ns, CertSquare sq, CertLinear lin) {
  __shared__ double red[8];
  const int s = blockIdx.y;
  const double c = ns.cscale[s];
  if (!(c < 1.0)) return;
  const int n = w.n[s], ld = w.ld[s];
  const int64_t base = w.off[s];
  const int64_t total4 = int64_t(ld) * ld / 4;
  const float cf = float(c), c2f = float(c * c);
  const float dshift = sq.diag * (1.0f - c2f);
  double r2 = 0.0;
  for (int64_t e4 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e4 < total4;
       e4 += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = 4 * e4;
    const int r = int(e / ld), col0 = int(e - int64_t(r) * ld);
    const int64_t i = base + e;
    float q[4];
    if constexpr (sizeof(T) == 2) {  // BF16 or FP16 pairs
      T* hi = static_cast<T*>(sq.hi);
      T* lo = static_cast<T*>(sq.lo);
      const float4 v = load_split4(hi, lo, i);
      q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
#pragma unroll
      for (int k = 0; k < 4; ++k) q[k] = c2f * q[k] + ((col0 + k == r && r < n) ? dshift : 0.0f);
      store_split4(make_float4(q[0], q[1], q[2], q[3]), hi, lo, i);
      for (int b = 0; b < lin.count; ++b) {
        T* lh = static_cast<T*>(lin.hi[b]);
        T* ll = static_cast<T*>(lin.lo[b]);
        const float4 x = load_split4(lh, ll, i);
        store_split4(make_float4(cf * x.x, cf * x.y, cf * x.z, cf * x.w), lh, ll, i);
      }
    } else {
      T* x2 = static_cast<T*>(sq.hi);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const T v = T(c * c) * x2[i + k];
        x2[i + k] = v;
        q[k] = float(v);
      }
      for (int b = 0; b < lin.count; ++b) {
        T* x = static_cast<T*>(lin.hi[b]);
#pragma unroll
        for (int k = 0; k < 4; ++k) x[i + k] = T(c) * x[i + k];
      }
    }
    if (r < n) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (col0 + k >= n) break;
        const bool dg = col0 + k == r;
        const float x2v = (q[k] - (dg ? sq.diag : 0.0f)) / sq.alpha;
        const float d = x2v - (dg ? 1.0f : 0.0f);
        r2 += double(d * d);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < int(blockDim.x >> 5); ++k) t += red[k];
    atomicAdd(&ns.res2[s], t);
  }
}

}  // namespace

CertLimits cert_limits(bool third_order) {
  // Newton-Schulz: rho <= sqrt(2.94) = 1.7146 < sqrt(3) = 1.7321;
  // third order: rho <= sqrt(2.2) = 1.4832 < sqrt(7/3) = 1.5275
  return third_order ? CertLimits{2.2, 1.45} : CertLimits{2.94, 1.7};
}

cudaError_t launch_cert_rowsum(const WaveDev& w, NsStateDev ns, CertSquare sq, int max_ld, cudaStream_t st) {
  if (w.nsub <= 0) return cudaSuccess;
  int bx = (max_ld + 63) / 64;  // about eight rows per warp
  if (bx > 32) bx = 32;
  k_cert_rowsum<<<dim3(unsigned(bx), unsigned(w.nsub)), 256, 0, st>>>(w, sq, ns.state, ns.cert);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_certify(const WaveDev& w, NsStateDev ns, CertSquare sq, CertLinear lin, CertLimits lim,
                           int max_ld, int* count, cudaStream_t st) {
  if (w.nsub <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ns.cert, 0, sizeof(unsigned long long) * size_t(w.nsub), st);
  if (e != cudaSuccess) return e;
  int bx = (max_ld + 63) / 64;  // about eight rows per warp
  if (bx > 32) bx = 32;
  k_cert_rowsum<<<dim3(unsigned(bx), unsigned(w.nsub)), 256, 0, st>>>(w, sq, ns.state, ns.cert);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // rounding of the computed square, relative to sum_k |X_rk||X_kc|:
  // FP64 products; FP32 products (ld terms); BF16x3 split products (the
  // dropped lo*lo term and the pair's own rounding, ~2^-16, FP32 sums of ld
  // terms), doubled for q -> X^2.  FP16x3 split products (mode 3) round to
  // ~2^-21 relative plus 2^-25 absolute per entry (FP16's subnormal step);
  // with gx >= rho(X_0) >= 1/1.05 whenever the certificate matters (the power
  // estimate never exceeds rho), the BF16 terms cover them with room to spare
  // and are kept.
  double eps0 = 0x1p-50, eps_ld = 0x1p-52;
  if (sq.mode == 1) { eps0 = 0x1p-22; eps_ld = 0x1p-23; }
  if (sq.mode >= 2) { eps0 = 0x1p-12; eps_ld = 0x1p-22; }
  k_cert_decide<<<(w.nsub + 255) / 256, 256, 0, st>>>(w, ns, lim.gmax, lim.fcap, eps0, eps_ld, count);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int ax = int((int64_t(max_ld) * max_ld + 4095) / 4096);
  if (ax > 32) ax = 32;
  if (ax < 1) ax = 1;
  const dim3 grid(unsigned(ax), unsigned(w.nsub));
  if (sq.mode == 3) k_cert_apply<__half><<<grid, 256, 0, st>>>(w, ns, sq, lin);
  else if (sq.mode == 2) k_cert_apply<__nv_bfloat16><<<grid, 256, 0, st>>>(w, ns, sq, lin);
  else if (sq.mode == 1) k_cert_apply<float><<<grid, 256, 0, st>>>(w, ns, sq, lin);
  else k_cert_apply<double><<<grid, 256, 0, st>>>(w, ns, sq, lin);
  count_launch();
  return cudaGetLastError();
}

}  // namespace submat

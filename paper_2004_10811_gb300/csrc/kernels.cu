// Memory-bound kernels of the submatrix path: assembly (gather), scaling,
// Newton-Schulz bookkeeping, extraction (scatter) and the trace.
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "common.cuh"

namespace submat {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Section III-A step 1 (block-wise, Section IV-C): rows [locoff[t], +bs[i1])
// of the dense a_j = K[N(j), N(j)] - mu I, for local block row t of
// submatrix s.  One CTA per (s, t); the CTA of the last block row also zeroes
// the padding rows n_j..ld-1.  Row abs-sums (Gershgorin) and ||a_j||_F^2 are
// accumulated for the scaling of X_0.  A per-column table (where column c of
// the block row starts in K, and its row stride) is built once in shared
// memory, so each element costs one table read and one load.
__global__ void __launch_bounds__(256) k_gather(PatternDev g, WaveDev w, const int2* items,
                                                const double* __restrict__ K, double mu,
                                                double* __restrict__ A, NsStateDev ns,
                                                int* flags, int ld_max) {
  extern __shared__ __align__(8) unsigned char smraw[];
  long long* colbase = reinterpret_cast<long long*>(smraw);  // [ld_max]: K index of (0, c) or -1
  int* colstride = reinterpret_cast<int*>(colbase + ld_max);  // [ld_max]
  int* sm = colstride + ld_max;
  const int2 it = items[blockIdx.x];
  const int s = it.x, t = it.y;
  const int j = w.sub[s];  // the submatrix (a block column, or a group of them)
  const int64_t rp0 = g.sp[j];
  const int nb = int(g.sp[j + 1] - rp0);
  int* nbr = sm;            // N(j)
  int* blk = sm + nb;       // CSR position of block (i1, N(j)[u]) or -1
  int* loc = sm + 2 * nb;   // local offsets, loc[nb] = n
  const int n = w.n[s];
  const int ld = w.ld[s];
  for (int u = threadIdx.x; u < nb; u += blockDim.x) {
    nbr[u] = g.srows[rp0 + u];
    blk[u] = -1;
    loc[u] = g.sloc[rp0 + u];
  }
  if (threadIdx.x == 0) loc[nb] = n;
  __syncthreads();
  const int i1 = nbr[t];
  const int64_t q0 = g.row_ptr[i1], q1 = g.row_ptr[i1 + 1];
  for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const int c = g.col[q];
    int lo = 0, hi = nb - 1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int v = nbr[mid];
      if (v == c) { blk[mid] = int(q); break; }
      if (v < c) lo = mid + 1; else hi = mid - 1;
    }
  }
  __syncthreads();
  const int r0 = loc[t];
  const int br = g.bs[i1];
  double* Aj = A + w.off[s];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int u = warp; u < nb; u += nw) {  // one warp per column block
    const int q = blk[u];
    const int c0 = loc[u], wd = loc[u + 1] - c0;
    const long long b0 = q >= 0 ? static_cast<long long>(g.valptr[q]) : -1;
    const int stride = g.bs[nbr[u]];
    for (int cc = lane; cc < wd; cc += 32) {
      colbase[c0 + cc] = q >= 0 ? b0 + cc : -1;
      colstride[c0 + cc] = stride;
    }
  }
  __syncthreads();
  const int rows_total = br + ((t == nb - 1) ? (ld - n) : 0);
  float fro = 0.0f;  // norms in FP32 (the FP64 pipe is slow); beta gets a margin
  bool bad = false;
  for (int rr = warp; rr < rows_total; rr += nw) {
    if (rr < br) {
      double* row = Aj + int64_t(r0 + rr) * ld;
      float rs = 0.0f;
      for (int c = lane; c < ld; c += 32) {
        double v = 0.0;
        if (c < n) {
          const long long b = colbase[c];
          if (b >= 0) {
            v = K[b + int64_t(rr) * colstride[c]];
            if (c == r0 + rr) v -= mu;  // same block, same offset: the diagonal
          }
        }
        if (!isfinite(v)) bad = true;
        row[c] = v;
        const float vf = d2f_trunc(v);
        rs += fabsf(vf);
        fro = fmaf(vf, vf, fro);
      }
      const double rsd = warp_sum(double(rs));
      if (lane == 0 && isfinite(rsd)) atomicMax(&ns.gersh[s], (unsigned long long)__double_as_longlong(rsd));
    } else {
      double* row = Aj + int64_t(n + rr - br) * ld;
      for (int c = lane; c < ld; c += 32) row[c] = 0.0;
    }
  }
  const double frod = warp_sum(double(fro));
  if (lane == 0) atomicAdd(&ns.fro2[s], frod);
  if (bad) atomicOr(flags, FLAG_NONFINITE);
}

// beta_s >= rho(a_s): min(max row abs-sum, ||a_s||_F).  A zero submatrix has
// sign 0 (Eq. signevext), so it is finished before any iteration.
__global__ void k_beta(WaveDev w, NsStateDev ns, int beta_mode) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= w.nsub) return;
  const double gersh = __longlong_as_double((long long)ns.gersh[s]);
  const double fro = sqrt(ns.fro2[s]);
  // FP32 sums of truncated values: a relative margin keeps beta above the bound
  double b = fmin(gersh, fro) * (1.0 + 1e-4);
  (void)beta_mode;
  ns.iters[s] = 0;
  ns.notconv[s] = 0;
  ns.par[s] = 0;
  ns.res2[s] = 0.0;
  ns.rprev[s] = 1e300;
  if (!(b > 0.0) || !isfinite(b)) {
    ns.beta[s] = 1.0;
    ns.state[s] = ST_DONE;
  } else {
    ns.beta[s] = b;
    ns.state[s] = ST_ACTIVE;
  }
}

template <typename T>
__global__ void k_scale(WaveDev w, const double* __restrict__ A, T* __restrict__ X,
                        const double* __restrict__ beta) {
  const int s = blockIdx.y;
  const int ld = w.ld[s];
  const int64_t total = int64_t(ld) * ld;
  const int64_t off = w.off[s];
  const double ib = 1.0 / beta[s];
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x)
    X[off + e] = T(A[off + e] * ib);
}

// After the squaring GEMM: r = ||X^2 - I||_F / sqrt(n); decide whether this
// is the last iteration (Section VI-A: involution as the stopping test).
__global__ void k_ns_update(WaveDev w, NsStateDev ns, double tol, double floor_thr,
                            int max_iter, int* flags) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= w.nsub) return;
  if (ns.state[s] != ST_ACTIVE) return;
  const double r = sqrt(ns.res2[s] / double(w.n[s]));
  ns.res2[s] = 0.0;
  const int it = ++ns.iters[s];
  const double prev = ns.rprev[s];
  ns.rprev[s] = r;
  if (!isfinite(r) || r > 1e6) {
    ns.state[s] = ST_DONE;
    ns.notconv[s] = 1;
    atomicOr(flags, FLAG_DIVERGED);
    return;
  }
  const bool converged = r <= tol;
  const bool at_floor = (r < floor_thr) && (r > 0.5 * prev);
  if (converged || at_floor) {
    ns.state[s] = ST_LAST;
  } else if (it >= max_iter) {
    ns.state[s] = ST_LAST;
    ns.notconv[s] = 1;
  }
}

__global__ void k_ns_post(WaveDev w, NsStateDev ns, int par_new, int* d_active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  int active = 0;
  if (s < w.nsub) {
    const int st = ns.state[s];
    if (st == ST_LAST) {
      ns.state[s] = ST_DONE;
      ns.par[s] = par_new;
    } else if (st == ST_ACTIVE) {
      ns.par[s] = par_new;
      active = 1;
    }
  }
  active = __syncthreads_count(active);
  if (threadIdx.x == 0 && active) atomicAdd(d_active, active);
}

// Section III-A step 3: block column j of D from the columns of block j of
// 1/2 (I - S_j).  S_j is symmetric, so row koff + c of S_j is read (coalesced)
// for column koff + c.  The diagonal block's trace is written to trpart[j].
template <typename T>
__global__ void __launch_bounds__(256) k_scatter(PatternDev g, WaveDev w, NsStateDev ns,
                                                 const T* __restrict__ buf0,
                                                 const T* __restrict__ buf1,
                                                 double* __restrict__ D, double* trpart,
                                                 const float* __restrict__ corr_a,
                                                 const float* __restrict__ corr_b,
                                                 const int* __restrict__ fallback,
                                                 double* __restrict__ sqpart) {
  extern __shared__ int sm[];
  __shared__ double red[8], red2[8];
  const int s = blockIdx.x;
  const int j = w.sub[s];
  const int64_t rp0 = g.row_ptr[j];
  const int nb = int(g.row_ptr[j + 1] - rp0);
  int* loc = sm;
  const int n = w.n[s], ld = w.ld[s];
  for (int u = threadIdx.x; u < nb; u += blockDim.x) loc[u] = g.locoff[rp0 + u];
  if (threadIdx.x == 0) loc[nb] = n;
  __syncthreads();
  const T* S = (ns.par[s] ? buf1 : buf0) + w.off[s];
  // the mixed path's last correction, S - (F_c + F_a), applied here for the
  // extracted entries only (not for submatrices re-solved in FP64)
  const bool correct = corr_a && !fallback[s];
  const float* ca = corr_a ? corr_a + w.off[s] : nullptr;
  const float* cb = corr_b ? corr_b + w.off[s] : nullptr;
  const int koff = g.koff[j];
  const int bj = g.bs[j];
  double tr = 0.0, sq = 0.0;
  const int64_t total = int64_t(bj) * n;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int c = int(e / n);
    const int col = int(e - int64_t(c) * n);
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (loc[mid] <= col) lo = mid; else hi = mid - 1;
    }
    const int r = col - loc[lo];
    const int64_t p = g.tpos[rp0 + lo];  // block (N(j)[lo], j)
    const int64_t si = int64_t(koff + c) * ld + col;
    double sv = double(S[si]);
    if (correct) sv -= f2d_exact(ca[si] + cb[si]);
    const bool diag = (col == koff + c);
    const double v = (diag ? 0.5 : 0.0) - 0.5 * sv;
    if (D) D[g.valptr[p] + int64_t(r) * bj + c] = v;  // null: trace and squares only
    if (diag) tr += v;
    if (sqpart) sq = fma(v, v, sq);
  }
  tr = warp_sum(tr);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tr;
  if (sqpart) {
    sq = warp_sum(sq);
    if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = sq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0, acc2 = 0.0;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) { acc += red[q]; acc2 += red2[q]; }
    trpart[j] = acc;
    // sum over the block's columns c of (D^2)_cc = sum_k D_kc^2 (D_j symmetric)
    if (sqpart) sqpart[j] = acc2;
  }
}

__global__ void k_diag_sums(PatternDev g, int nblk, const double* __restrict__ D, double* part) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nblk) return;
  const int64_t p = g.diagpos[j];
  const int b = g.bs[j];
  const double* blk = D + g.valptr[p];
  double acc = 0.0;
  for (int c = 0; c < b; ++c) acc += blk[c * b + c];
  part[j] = acc;
}

// Fixed-order reduction (one CTA): deterministic for a given nblk.
__global__ void k_reduce_fixed(const double* part, int count, double* out) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// (D + D^T) / 2 on the pattern: block p gets 1/2 (D_p + D_{tpos[p]}^T).
__global__ void k_symmetrize(PatternDev g, int64_t nnzb, const double* __restrict__ Din,
                             double* __restrict__ Dout, const int64_t* __restrict__ rowof) {
  const int64_t p = blockIdx.x;
  if (p >= nnzb) return;
  const int r = int(rowof[p]);
  const int c = g.col[p];
  const int br = g.bs[r], bc = g.bs[c];
  const double* a = Din + g.valptr[p];
  const double* b = Din + g.valptr[g.tpos[p]];  // block (c, r): bc x br
  double* o = Dout + g.valptr[p];
  for (int e = threadIdx.x; e < br * bc; e += blockDim.x) {
    const int u = e / bc, v = e - (e / bc) * bc;
    o[e] = 0.5 * (a[e] + b[v * br + u]);
  }
}

__global__ void k_check_finite(const double* __restrict__ v, int64_t count, int* flags) {
  bool bad = false;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
       e += int64_t(gridDim.x) * blockDim.x)
    if (!isfinite(v[e])) bad = true;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, FLAG_NONFINITE);
}

// ||X v|| / ||v|| after `iters` power steps: a lower bound on rho(X) that
// converges to it.  One CTA per submatrix; v lives in shared memory.
// Deterministic start vector (a fixed hash of the index).
template <typename T>
__global__ void __launch_bounds__(1024) k_power(WaveDev w, const T* __restrict__ X, int iters,
                                                const int* __restrict__ state, double* __restrict__ rho) {
  extern __shared__ float pv[];  // v[ld], y[ld]
  __shared__ float red[32];
  const int s = blockIdx.x;
  if (state && state[s] == ST_DONE) { if (threadIdx.x == 0) rho[s] = 0.0; return; }
  const int ld = w.ld[s];
  const int n = w.n[s];
  const T* Xs = X + w.off[s];
  float* v = pv;
  float* y = pv + ld;
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    unsigned h = unsigned(i) * 2654435761u + 12345u;
    h ^= h >> 15;
    v[i] = i < n ? 0.5f + float(h & 0xFFFF) / 65536.0f : 0.0f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float est = 0.0f;
  for (int it = 0; it < iters; ++it) {
    float yy = 0.0f, vv = 0.0f;
    for (int r = warp; r < n; r += nw) {
      const T* row = Xs + int64_t(r) * ld;
      float acc = 0.0f;
      if constexpr (std::is_same<T, __half>::value) {
        // eight FP16 per lane and load (padding columns are zero in X and v)
        for (int c = lane * 8; c < ld; c += 256) {
          const uint4 q = *reinterpret_cast<const uint4*>(row + c);
          const float4 v0 = *reinterpret_cast<const float4*>(v + c);
          const float4 v1 = *reinterpret_cast<const float4*>(v + c + 4);
          const uint32_t qw[4] = {q.x, q.y, q.z, q.w};
          const float vv8[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&qw[k]));
            acc = fmaf(f.x, vv8[2 * k], acc);
            acc = fmaf(f.y, vv8[2 * k + 1], acc);
          }
        }
      } else if constexpr (sizeof(T) == 2) {
        // eight BF16 per lane and load (padding columns are zero in X and v)
        for (int c = lane * 8; c < ld; c += 256) {
          const uint4 q = *reinterpret_cast<const uint4*>(row + c);
          const float4 v0 = *reinterpret_cast<const float4*>(v + c);
          const float4 v1 = *reinterpret_cast<const float4*>(v + c + 4);
          acc = fmaf(__uint_as_float(q.x << 16), v0.x, acc);
          acc = fmaf(__uint_as_float(q.x & 0xFFFF0000u), v0.y, acc);
          acc = fmaf(__uint_as_float(q.y << 16), v0.z, acc);
          acc = fmaf(__uint_as_float(q.y & 0xFFFF0000u), v0.w, acc);
          acc = fmaf(__uint_as_float(q.z << 16), v1.x, acc);
          acc = fmaf(__uint_as_float(q.z & 0xFFFF0000u), v1.y, acc);
          acc = fmaf(__uint_as_float(q.w << 16), v1.z, acc);
          acc = fmaf(__uint_as_float(q.w & 0xFFFF0000u), v1.w, acc);
        }
      } else {
        for (int c = lane; c < n; c += 32) acc = fmaf(float(row[c]), v[c], acc);
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) y[r] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) { yy = fmaf(y[i], y[i], yy); vv = fmaf(v[i], v[i], vv); }
    for (int o = 16; o > 0; o >>= 1) { yy += __shfl_xor_sync(0xffffffffu, yy, o); vv += __shfl_xor_sync(0xffffffffu, vv, o); }
    if (lane == 0) { red[warp] = yy; }
    __syncthreads();
    float ysum = 0.0f;
    for (int q = 0; q < nw; ++q) ysum += red[q];
    __syncthreads();
    if (lane == 0) red[warp] = vv;
    __syncthreads();
    float vsum = 0.0f;
    for (int q = 0; q < nw; ++q) vsum += red[q];
    est = vsum > 0.0f ? sqrtf(ysum / vsum) : 0.0f;
    const float inv = ysum > 0.0f ? rsqrtf(ysum) : 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = y[i] * inv;
    __syncthreads();
  }
  if (threadIdx.x == 0) rho[s] = double(est);
}

}  // namespace

static dim3 scale_grid(const WaveDev& w, int64_t max_ld2) {
  int64_t bx = (max_ld2 + 256 * 8 - 1) / (256 * 8);
  if (bx > 512) bx = 512;
  if (bx < 1) bx = 1;
  return dim3(unsigned(bx), unsigned(w.nsub));
}

template <typename T>
static cudaError_t power_impl(const WaveDev& w, const T* X, int iters, const int* state, double* rho,
                              int max_ld, cudaStream_t st) {
  const size_t smem = size_t(2 * max_ld) * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_power<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k_power<T><<<w.nsub, 1024, smem, st>>>(w, X, iters, state, rho);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_power_bf16(const WaveDev& w, const __nv_bfloat16* X, int iters, const int* state,
                              double* rho, int max_ld, cudaStream_t st) {
  return power_impl(w, X, iters, state, rho, max_ld, st);
}
cudaError_t launch_power_f16(const WaveDev& w, const __half* X, int iters, const int* state, double* rho,
                             int max_ld, cudaStream_t st) {
  return power_impl(w, X, iters, state, rho, max_ld, st);
}
cudaError_t launch_power_f64(const WaveDev& w, const double* X, int iters, const int* state, double* rho,
                             int max_ld, cudaStream_t st) {
  return power_impl(w, X, iters, state, rho, max_ld, st);
}
cudaError_t launch_power_f32(const WaveDev& w, const float* X, int iters, const int* state, double* rho,
                             int max_ld, cudaStream_t st) {
  return power_impl(w, X, iters, state, rho, max_ld, st);
}

// X <- f_s X with f_s = 1 / (1.05 rho_s) when that tightens the scale; beta_s
// follows.  rho_s is the power estimate of rho(X) (X = a / beta_s).
template <typename T>
__global__ void k_rescale(WaveDev w, T* __restrict__ X, const double* __restrict__ rho,
                          double* __restrict__ beta, const int* __restrict__ state) {
  const int s = blockIdx.y;
  if (state && state[s] == ST_DONE) return;
  const double r = rho[s];
  if (!(r > 0.0) || r * 1.05 >= 1.0) return;  // keep the guaranteed bound
  const double f = 1.0 / (1.05 * r);
  if (threadIdx.x == 0 && blockIdx.x == 0) beta[s] = beta[s] / f;
  const int ld = w.ld[s];
  const int64_t total = int64_t(ld) * ld;
  const int64_t off = w.off[s];
  const T fs = T(f);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x)
    X[off + e] = X[off + e] * fs;
}

cudaError_t launch_rescale_f64(const WaveDev& w, double* X, const double* rho, double* beta,
                               const int* state, int64_t max_ld2, cudaStream_t st) {
  k_rescale<double><<<scale_grid(w, max_ld2), 256, 0, st>>>(w, X, rho, beta, state);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_rescale_f32(const WaveDev& w, float* X, const double* rho, double* beta,
                               const int* state, int64_t max_ld2, cudaStream_t st) {
  k_rescale<float><<<scale_grid(w, max_ld2), 256, 0, st>>>(w, X, rho, beta, state);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_reset_rprev(WaveDev w, NsStateDev ns) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < w.nsub) ns.rprev[s] = 1e300;
}

cudaError_t launch_reset_rprev(const WaveDev& w, NsStateDev ns, cudaStream_t st) {
  k_reset_rprev<<<(w.nsub + 255) / 256, 256, 0, st>>>(w, ns);
  count_launch();
  return cudaGetLastError();
}

static std::atomic<long long> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t launch_gather(const PatternDev& g, const WaveDev& w, const int2* items, int nitems,
                          int nb_max, int ld_max, int bs_max, const double* K, double mu, double* A,
                          NsStateDev ns, int* flags, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (gather_rows_fits(nb_max, ld_max, bs_max))
    return launch_gather_rows(g, w, nb_max, ld_max, K, mu, A, ns, flags, st);
  const size_t smem = size_t(ld_max) * (sizeof(long long) + sizeof(int)) + size_t(3 * nb_max + 1) * sizeof(int);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
  }
  k_gather<<<nitems, 256, smem, st>>>(g, w, items, K, mu, A, ns, flags, ld_max);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_beta(const WaveDev& w, NsStateDev ns, int beta_mode, cudaStream_t st) {
  k_beta<<<(w.nsub + 255) / 256, 256, 0, st>>>(w, ns, beta_mode);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale_f64(const WaveDev& w, const double* A, double* X, const double* beta,
                             int64_t max_ld2, cudaStream_t st) {
  k_scale<double><<<scale_grid(w, max_ld2), 256, 0, st>>>(w, A, X, beta);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale_f32(const WaveDev& w, const double* A, float* X, const double* beta,
                             int64_t max_ld2, cudaStream_t st) {
  k_scale<float><<<scale_grid(w, max_ld2), 256, 0, st>>>(w, A, X, beta);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ns_update(const WaveDev& w, NsStateDev ns, double tol, double floor_thr,
                             int max_iter, int* flags, cudaStream_t st) {
  k_ns_update<<<(w.nsub + 255) / 256, 256, 0, st>>>(w, ns, tol, floor_thr, max_iter, flags);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ns_post(const WaveDev& w, NsStateDev ns, int par_new, int* d_active,
                           cudaStream_t st) {
  k_ns_post<<<(w.nsub + 255) / 256, 256, 0, st>>>(w, ns, par_new, d_active);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t scatter_impl(const PatternDev& g, const WaveDev& w, NsStateDev ns,
                                const T* buf0, const T* buf1, double* D, double* trpart,
                                ScatterGeom geo, cudaStream_t st, const float* corr_a = nullptr,
                                const float* corr_b = nullptr, const int* fallback = nullptr,
                                double* sqpart = nullptr) {
  if (geo.members_max > 0)  // groups of block columns per submatrix
    return launch_scatter_members<T>(g, w, ns, buf0, buf1, D, trpart, geo.nbj_max, geo.members_max, st, corr_a,
                                     corr_b, fallback, sqpart);
  // shared-memory staging of the extracted rows (coalesced reads of S and
  // whole-block writes of D), unless a block is too large to stage
  if (scatter_staged_smem(geo.nb_max, geo.ld_max, geo.bs_max) <= 200 * 1024)
    return launch_scatter_staged<T>(g, w, ns, buf0, buf1, D, trpart, geo.nb_max, geo.ld_max, geo.bs_max, st,
                                    corr_a, corr_b, fallback, sqpart);
  const int nb_max = geo.nb_max;
  const size_t smem = size_t(nb_max + 1) * sizeof(int);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_scatter<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k_scatter<T><<<w.nsub, 256, smem, st>>>(g, w, ns, buf0, buf1, D, trpart, corr_a, corr_b, fallback, sqpart);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scatter_f64(const PatternDev& g, const WaveDev& w, NsStateDev ns,
                               const double* buf0, const double* buf1, double* D,
                               double* trpart, ScatterGeom geo, cudaStream_t st, const float* corr_a,
                               const float* corr_b, const int* fallback) {
  return scatter_impl<double>(g, w, ns, buf0, buf1, D, trpart, geo, st, corr_a, corr_b, fallback);
}

cudaError_t launch_scatter_f32(const PatternDev& g, const WaveDev& w, NsStateDev ns,
                               const float* buf0, const float* buf1, double* D,
                               double* trpart, ScatterGeom geo, cudaStream_t st) {
  return scatter_impl<float>(g, w, ns, buf0, buf1, D, trpart, geo, st);
}

template <typename T>
cudaError_t launch_scatter_sq(const PatternDev& g, const WaveDev& w, NsStateDev ns, const T* S, double* D,
                              double* trpart, double* sqpart, ScatterGeom geo, cudaStream_t st) {
  return scatter_impl<T>(g, w, ns, S, S, D, trpart, geo, st, nullptr, nullptr, nullptr, sqpart);
}
template cudaError_t launch_scatter_sq<double>(const PatternDev&, const WaveDev&, NsStateDev, const double*,
                                               double*, double*, double*, ScatterGeom, cudaStream_t);
template cudaError_t launch_scatter_sq<float>(const PatternDev&, const WaveDev&, NsStateDev, const float*,
                                              double*, double*, double*, ScatterGeom, cudaStream_t);

cudaError_t launch_trace(const PatternDev& g, int nblk, const double* D, double* part,
                         double* out, cudaStream_t st) {
  k_diag_sums<<<(nblk + 255) / 256, 256, 0, st>>>(g, nblk, D, part);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_fixed<<<1, 1024, 0, st>>>(part, nblk, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_symmetrize_impl(const PatternDev& g, int64_t nnzb, const double* Din,
                                   double* Dout, const int64_t* rowof, cudaStream_t st) {
  if (nnzb <= 0) return cudaSuccess;
  k_symmetrize<<<unsigned(nnzb), 64, 0, st>>>(g, nnzb, Din, Dout, rowof);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* v, int64_t count, int* flags, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_check_finite<<<unsigned(blocks), 256, 0, st>>>(v, count, flags);
  count_launch();
  return cudaGetLastError();
}

}  // namespace submat

// submat_dense_sign_noalloc: the dense one-block case of the sign evaluation
// that allocates no memory at all.
//
// Who needs it: callers that may not call cudaMalloc or cudaMallocHost --
// codes that reserve the whole device up front for their own memory pool (a
// molecular-dynamics engine that hands out slices of one arena), runtimes
// whose allocator forbids foreign allocations, and code paths where an
// allocation would implicitly synchronise the device in the middle of a
// time step.  They pass device buffers for K and D; all scratch (the
// Newton-Schulz iterates, X^2, the tile list and the convergence state) lives
// in one file-scope device array of fixed size that every GPU loading this
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "common.cuh"
#include "submat.h"

namespace submat {

namespace {

constexpr int NA_MAX_N = SUBMAT_NOALLOC_MAX_N;  // largest accepted dimension
constexpr int NA_LD = NA_MAX_N;                 // buffers are sized for the maximum
constexpr size_t NA_ELEMS = size_t(NA_LD) * NA_LD;
constexpr int NA_MAX_TILES = (NA_LD / 64) * (NA_LD / 64 + 1) / 2;

// small-state block at the end of the scratch array
struct NaSmall {
  int4 items[NA_MAX_TILES];  // upper 64x64 tiles (0, ti, tj, 0)
  int64_t off;               // wave offset of the single matrix (0)
  int32_t sub, ld, n;        // one "submatrix"
  int state, iters, par, notconv, active, flags;
  double res2, rprev, beta, fro2;
  unsigned long long gersh;
};

constexpr size_t NA_SMALL_DOUBLES = (sizeof(NaSmall) + sizeof(double) - 1) / sizeof(double);

// X0 | X1 | Y | small state.  6 MiB for n <= 512.
__device__ __align__(256) double g_noalloc_scratch[3 * NA_ELEMS + NA_SMALL_DOUBLES];

// Device address of g_noalloc_scratch on the current device, looked up on
// every call: the lookup is on the host and allocates nothing, and a cached
// address would go stale if the caller reset the device (the module, and
// with it the array, is then loaded again elsewhere).
submat_status setup(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    set_error("cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
    return SUBMAT_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return SUBMAT_OK;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA: reset the state, and beta = min(max row abs-sum, ||K - mu I||_F).
__global__ void k_na_init(int n, const double* __restrict__ K, double mu, NaSmall* sm) {
  __shared__ double rmax[32], rfro[32];
  double mx = 0.0, fro = 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  bool bad = false;
  for (int r = warp; r < n; r += nw) {
    double rs = 0.0;
    for (int c = lane; c < n; c += 32) {
      double v = K[int64_t(r) * n + c];
      if (r == c) v -= mu;
      if (!isfinite(v)) bad = true;
      rs += fabs(v);
      fro += v * v;
    }
    rs = warp_sum(rs);
    mx = fmax(mx, rs);
  }
  fro = warp_sum(fro);
  if (lane == 0) { rmax[warp] = mx; rfro[warp] = fro; }
  const int anybad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    double m = 0.0, f = 0.0;
    for (int q = 0; q < nw; ++q) { m = fmax(m, rmax[q]); f += rfro[q]; }
    const double b = fmin(m, sqrt(f));
    sm->flags = anybad ? FLAG_NONFINITE : 0;
    sm->iters = 0;
    sm->par = 0;
    sm->notconv = 0;
    sm->active = 0;
    sm->res2 = 0.0;
    sm->rprev = 1e300;
    sm->fro2 = f;
    sm->gersh = 0ull;
    if (b > 0.0 && isfinite(b)) { sm->beta = b; sm->state = ST_ACTIVE; }
    else { sm->beta = 1.0; sm->state = ST_DONE; }
  }
}

// X0 = (K - mu I) / beta, zero padded to ld x ld.
__global__ void k_na_load(int n, int ld, const double* __restrict__ K, double mu,
                          const NaSmall* sm, double* __restrict__ X) {
  const double ib = 1.0 / sm->beta;
  const int64_t total = int64_t(ld) * ld;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(e / ld), c = int(e - int64_t(r) * ld);
    double v = 0.0;
    if (r < n && c < n) {
      v = K[int64_t(r) * n + c];
      if (r == c) v -= mu;
      v *= ib;
    }
    X[e] = v;
  }
}

// D = 1/2 (I - X) on the n x n block of the final iterate.
__global__ void k_na_store(int n, int ld, const NaSmall* sm, const double* __restrict__ X0,
                           const double* __restrict__ X1, double* __restrict__ D) {
  const double* X = sm->par ? X1 : X0;
  const int64_t total = int64_t(n) * n;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(e / n), c = int(e - int64_t(r) * n);
    D[e] = (r == c ? 0.5 : 0.0) - 0.5 * X[int64_t(r) * ld + c];
  }
}

}  // namespace

}  // namespace submat

extern "C" submat_status submat_dense_sign_noalloc(int n, const double* K_dev, double mu,
                                                   double* D_dev, int* iters_out, void* stream) {
  using namespace submat;
  clear_error();
  if (n < 1 || n > NA_MAX_N) {
    set_error("submat_dense_sign_noalloc: n = %d outside [1, %d] (the fixed scratch holds %d x %d)",
              n, NA_MAX_N, NA_MAX_N, NA_MAX_N);
    return SUBMAT_ERR_INVALID_ARG;
  }
  if (!K_dev || !D_dev || !std::isfinite(mu)) {
    set_error("submat_dense_sign_noalloc: null buffer or non-finite mu");
    return SUBMAT_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* base = nullptr;
  submat_status s = setup(&base);
  if (s != SUBMAT_OK) return s;
  double* X0 = base;
  double* X1 = base + NA_ELEMS;
  double* Y = base + 2 * NA_ELEMS;
  NaSmall* sm = reinterpret_cast<NaSmall*>(base + 3 * NA_ELEMS);
  const int ld = (n + 63) / 64 * 64;
  const int T = ld / 64;

  // geometry and tile list: a host staging struct copied into the scratch
  NaSmall h;
  std::memset(&h, 0, sizeof(h));
  int nt = 0;
  for (int a = 0; a < T; ++a)
    for (int b = a; b < T; ++b) h.items[nt++] = make_int4(0, a, b, 0);
  h.off = 0;
  h.sub = 0;
  h.ld = ld;
  h.n = n;
  SM_CUDA(cudaMemcpyAsync(sm, &h, offsetof(NaSmall, state), cudaMemcpyHostToDevice, st));
  k_na_init<<<1, 1024, 0, st>>>(n, K_dev, mu, sm);
  SM_KCHECK();
  k_na_load<<<(ld * ld + 255) / 256 < 1024 ? (ld * ld + 255) / 256 : 1024, 256, 0, st>>>(n, ld, K_dev, mu,
                                                                                       sm, X0);
  SM_KCHECK();
  int flags = 0;
  SM_CUDA(cudaMemcpyAsync(&flags, &sm->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaStreamSynchronize(st));
  if (flags & FLAG_NONFINITE) {
    set_error("K holds a NaN or Inf value");
    return SUBMAT_ERR_NONFINITE;
  }
  WaveDev w{1, &sm->sub, &sm->off, &sm->ld, &sm->n};
  NsStateDev ns{&sm->state, &sm->iters, &sm->par, &sm->notconv, &sm->res2, &sm->rprev,
                &sm->beta,  &sm->gersh, &sm->fro2};
  double* bufs[2] = {X0, X1};
  const int max_iter = 100;
  int cur = 0;
  for (int k = 0; k < max_iter; ++k) {
    GemmF64Args a1{};
    a1.w = w; a1.items = sm->items; a1.nitems = nt;
    a1.A = bufs[cur]; a1.B = bufs[cur]; a1.C0 = nullptr; a1.C = Y;
    a1.alpha = 1.0; a1.beta = 0.0; a1.diag = 0.0; a1.sym = 1; a1.res2 = &sm->res2;
    a1.state = &sm->state; a1.skip_state = ST_DONE;
    SM_CUDA(launch_gemm_f64(a1, st));
    SM_CUDA(launch_ns_update(w, ns, 1e-14, 1e-9, max_iter, &sm->flags, st));
    GemmF64Args a2 = a1;
    a2.B = Y; a2.C0 = bufs[cur]; a2.C = bufs[cur ^ 1];
    a2.alpha = -0.5; a2.beta = 1.5; a2.res2 = nullptr;
    SM_CUDA(launch_gemm_f64(a2, st));
    SM_CUDA(cudaMemsetAsync(&sm->active, 0, sizeof(int), st));
    SM_CUDA(launch_ns_post(w, ns, cur ^ 1, &sm->active, st));
    int active = 0;
    SM_CUDA(cudaMemcpyAsync(&active, &sm->active, sizeof(int), cudaMemcpyDeviceToHost, st));
    SM_CUDA(cudaStreamSynchronize(st));
    cur ^= 1;
    if (active == 0) break;
  }
  k_na_store<<<(n * n + 255) / 256 < 1024 ? (n * n + 255) / 256 : 1024, 256, 0, st>>>(n, ld, sm, X0, X1,
                                                                                     D_dev);
  SM_KCHECK();
  int tail[2] = {0, 0};  // iters, notconv
  SM_CUDA(cudaMemcpyAsync(&tail[0], &sm->iters, sizeof(int), cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(&tail[1], &sm->notconv, sizeof(int), cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = tail[0];
  if (tail[1]) {
    set_error("Newton-Schulz reached %d iterations without converging (D written)", max_iter);
    return SUBMAT_ERR_NOT_CONVERGED;
  }
  return SUBMAT_OK;
}

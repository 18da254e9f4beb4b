// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "submat.h"

namespace submat {

void set_error(const char* fmt, ...);
void clear_error();

// Kernel launches issued by this library in this process (all threads).
void count_launch(int k = 1);
long long launch_count();

#define SM_KCHECK()                         \
  do {                                      \
    ::submat::count_launch();               \
    SM_CUDA(cudaGetLastError());            \
  } while (0)

#define SM_CUDA(x)                                                                   \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) {                                                         \
      ::submat::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #x,            \
                          cudaGetErrorString(e_));                                   \
      return SUBMAT_ERR_CUDA;                                                        \
    }                                                                                \
  } while (0)

#define SM_TRY(x)                                \
  do {                                           \
    submat_status s_ = (x);                      \
    if (s_ != SUBMAT_OK) return s_;              \
  } while (0)

// Device status word bits (plan->d_flags[0]).
enum : int { FLAG_NONFINITE = 1, FLAG_TIMEOUT = 2, FLAG_DIVERGED = 4, FLAG_BOUNDS = 8 };

// Newton-Schulz state of one submatrix.
enum : int { ST_ACTIVE = 0, ST_LAST = 1, ST_DONE = 2 };

// Pattern and per-submatrix maps (device, indexed by global block / CSR position).
struct PatternDev {
  const int32_t* bs;       // [nblk] block sizes
  const int64_t* row_ptr;  // [nblk + 1]
  const int32_t* col;      // [nnzb]; row j lists N(j) (the pattern is symmetric)
  const int64_t* valptr;   // [nnzb + 1] first value of each block
  const int32_t* locoff;   // [nnzb] local row/column offset of local block t of submatrix j
  const int32_t* tpos;     // [nnzb] CSR position of the transposed block
  const int32_t* nsub;     // [nblk] submatrix dimension n_j
  const int32_t* koff;     // [nblk] local offset of block j inside submatrix j
  const int32_t* diagpos;  // [nblk] CSR position of block (j, j)
  // Submatrices (index q = WaveDev::sub[s]): one per block column, or one
  // per group of block columns (Section IV-C) over the union of their rows.
  // Without groups sp / srows / sloc are row_ptr / col / locoff.
  const int64_t* sp;       // [nq + 1] block rows of submatrix q: srows[sp[q] .. sp[q+1])
  const int32_t* srows;    //   ascending block rows N(q)
  const int32_t* sloc;     //   their local offsets inside submatrix q
  // groups only (null otherwise): the member block columns of submatrix q,
  // mcol[mp[q] .. mp[q+1]), block j's local offset mkoff[], and for every
  // stored block p = (i, j) the local offset dloc[p] of block row i in the
  // submatrix of j's group
  const int32_t* mp;
  const int32_t* mcol;
  const int32_t* mkoff;
  const int32_t* dloc;
};

// One wave: a set of submatrices whose dense buffers fit the workspace together.
struct WaveDev {
  int nsub;
  const int32_t* sub;  // [nsub] global block column j of local submatrix s
  const int64_t* off;  // [nsub] element offset of submatrix s in every workspace buffer
  const int32_t* ld;   // [nsub] leading dimension (multiple of 64)
  const int32_t* n;    // [nsub] dimension n_j
};

// Per-submatrix Newton-Schulz state (device, indexed by local s).
struct NsStateDev {
  int* state;       // ST_*
  int* iters;       // iterations done
  int* par;         // buffer (0/1) that holds the current / final iterate
  int* notconv;     // 1 if max_iter was hit
  double* res2;     // ||X^2 - I||_F^2 accumulated by the squaring GEMM
  double* rprev;    // previous ||X^2 - I||_F / sqrt(n)
  double* beta;     // scale of X_0
  unsigned long long* gersh;  // max row abs-sum (bits of a non-negative double)
  double* fro2;     // ||a||_F^2
  unsigned long long* cert;   // scale certificate: max row abs-sum of X_0^2 (bits)
  double* cscale;   // scale certificate: factor applied to X_0 (1 = kept)
};

// geometry bounds for the gather / scatter kernels: the largest number of
// blocks in a submatrix, leading dimension and block size; for grouped
// submatrices (members_max > 0) the largest member count and block-column
// length nbj_max, and the member-wise scatter is used
struct ScatterGeom {
  int nb_max, ld_max, bs_max;
  int members_max = 0, nbj_max = 0;
};

// ---- kernel launchers (kernels.cu) ----
cudaError_t launch_gather(const PatternDev& g, const WaveDev& w, const int2* items, int nitems,
                          int nb_max, int ld_max, int bs_max, const double* K, double mu, double* A,
                          NsStateDev ns, int* flags, cudaStream_t st);
// (gather.cu) the row-wise gather and the staged scatter
bool gather_rows_fits(int nb_max, int ld_max, int bs_max);
cudaError_t launch_gather_rows(const PatternDev& g, const WaveDev& w, int nb_max, int ld_max, const double* K,
                               double mu, double* A, NsStateDev ns, int* flags, cudaStream_t st);
size_t scatter_staged_smem(int nb_max, int ld_max, int bs_max);
template <typename T>
cudaError_t launch_scatter_members(const PatternDev& g, const WaveDev& w, NsStateDev ns, const T* buf0,
                                   const T* buf1, double* D, double* trpart, int nbj_max, int members_max,
                                   cudaStream_t st, const float* corr_a, const float* corr_b, const int* fallback,
                                   double* sqpart);
template <typename T>
cudaError_t launch_scatter_staged(const PatternDev& g, const WaveDev& w, NsStateDev ns, const T* buf0,
                                  const T* buf1, double* D, double* trpart, int nb_max, int ld_max, int bs_max,
                                  cudaStream_t st, const float* corr_a, const float* corr_b, const int* fallback,
                                  double* sqpart);

cudaError_t launch_beta(const WaveDev& w, NsStateDev ns, int beta_mode, cudaStream_t st);
cudaError_t launch_scale_f64(const WaveDev& w, const double* A, double* X, const double* beta,
                             int64_t max_ld2, cudaStream_t st);
cudaError_t launch_scale_f32(const WaveDev& w, const double* A, float* X, const double* beta,
                             int64_t max_ld2, cudaStream_t st);
cudaError_t launch_ns_update(const WaveDev& w, NsStateDev ns, double tol, double floor_thr,
                             int max_iter, int* flags, cudaStream_t st);
cudaError_t launch_ns_post(const WaveDev& w, NsStateDev ns, int par_new, int* d_active,
                           cudaStream_t st);
// corr_a, corr_b, fallback (mixed path, may be null): the extracted entries of
// S become S - (corr_a + corr_b), except in submatrices with fallback[s] set
cudaError_t launch_scatter_f64(const PatternDev& g, const WaveDev& w, NsStateDev ns,
                               const double* buf0, const double* buf1, double* D,
                               double* trpart, ScatterGeom geo, cudaStream_t st, const float* corr_a = nullptr,
                               const float* corr_b = nullptr, const int* fallback = nullptr);
cudaError_t launch_scatter_f32(const PatternDev& g, const WaveDev& w, NsStateDev ns,
                               const float* buf0, const float* buf1, double* D,
                               double* trpart, ScatterGeom geo, cudaStream_t st);
// the same from one buffer S (finite temperature: S = p(X), the polynomial
// for tanh), with sqpart[j] = sum over the block's columns c of (D_j^2)_cc
template <typename T>
cudaError_t launch_scatter_sq(const PatternDev& g, const WaveDev& w, NsStateDev ns, const T* S, double* D,
                              double* trpart, double* sqpart, ScatterGeom geo, cudaStream_t st);
cudaError_t launch_trace(const PatternDev& g, int nblk, const double* D, double* part,
                         double* out, cudaStream_t st);
cudaError_t launch_symmetrize_impl(const PatternDev& g, int64_t nnzb, const double* Din,
                                   double* Dout, const int64_t* rowof, cudaStream_t st);
cudaError_t launch_check_finite(const double* v, int64_t count, int* flags, cudaStream_t st);
// power iteration: rho[s] ~ rho(X_s) (a lower bound converging to it)
cudaError_t launch_power_bf16(const WaveDev& w, const __nv_bfloat16* X, int iters, const int* state,
                              double* rho, int max_ld, cudaStream_t st);
cudaError_t launch_power_f16(const WaveDev& w, const __half* X, int iters, const int* state, double* rho,
                             int max_ld, cudaStream_t st);
cudaError_t launch_power_f64(const WaveDev& w, const double* X, int iters, const int* state, double* rho,
                             int max_ld, cudaStream_t st);
cudaError_t launch_power_f32(const WaveDev& w, const float* X, int iters, const int* state, double* rho,
                             int max_ld, cudaStream_t st);
cudaError_t launch_rescale_f64(const WaveDev& w, double* X, const double* rho, double* beta,
                               const int* state, int64_t max_ld2, cudaStream_t st);
cudaError_t launch_reset_rprev(const WaveDev& w, NsStateDev ns, cudaStream_t st);
cudaError_t launch_rescale_f32(const WaveDev& w, float* X, const double* rho, double* beta,
                               const int* state, int64_t max_ld2, cudaStream_t st);

// ---- scale certificate (certify.cu) ----
// After the first squaring, ||X_0^2||_inf >= rho(X_0)^2 proves that the power
// estimate's scale keeps the spectrum of X_0 inside the iteration's basin;
// where it cannot, X_0 (and everything derived from it) is scaled down.
// Representation of the squared iterate: 0 FP64 X^2, 1 FP32 X^2, 2 a BF16
// (hi, lo) pair holding q = diag I + alpha X^2.
struct CertSquare {
  int mode;        // 0 FP64, 1 FP32, 2 BF16 (hi, lo) pair, 3 FP16 pair
  void* hi;        // the square (FP64 / FP32 array, or the pair's hi)
  void* lo;        // the pair's lo (modes 2 and 3)
  float alpha, diag;
};
// Up to three buffers that scale linearly with X_0 (X_0 itself, E_0, E_0^T),
// in the square's representation (pairs: hi, lo).
struct CertLinear {
  int count;
  void* hi[3];
  void* lo[3];
};
// basin of the iteration: Newton-Schulz (-sqrt 3, sqrt 3), third order
// (-sqrt(7/3), sqrt(7/3)); the certificate keeps rho(X_0) below these with margin
struct CertLimits {
  double gmax;     // certified when the bound on rho(X_0)^2 is <= gmax
  double fcap;     // X_0 = f a / beta_bound with f <= fcap is safe without it
};
CertLimits cert_limits(bool third_order);
// the row-sum pass alone: ns.cert[s] = bits of the largest row abs-sum of X^2
// (ns.cert must be zero beforehand; submatrices not ACTIVE are skipped)
cudaError_t launch_cert_rowsum(const WaveDev& w, NsStateDev ns, CertSquare sq, int max_ld, cudaStream_t st);
cudaError_t launch_certify(const WaveDev& w, NsStateDev ns, CertSquare sq, CertLinear lin, CertLimits lim,
                           int max_ld, int* count, cudaStream_t st);

// ---- FP64 GEMM (gemm_f64.cu) ----
// C = alpha * A * B + beta * C0 on every listed 64x64 tile (s, ti, tj);
// all operands are row-major per submatrix at wave offsets.  With sym != 0
// the listed tiles have ti <= tj and the transposed tile is written as well.
struct GemmF64Args {
  WaveDev w;
  const int4* items;
  int nitems;
  const double* A;
  const double* B;
  const double* C0;
  double* C;
  double alpha, beta;
  double diag;       // added to C on the diagonal of the n x n block (C += diag * I_n)
  int sym;
  double* res2;      // optional: accumulate ||C - I_n||_F^2 per submatrix
  const int* state;  // optional: skip submatrices with state == skip_state
  int skip_state;
};
cudaError_t launch_gemm_f64(const GemmF64Args& a, cudaStream_t st);

// Same contract in FP32 (FFMA).
struct GemmF32Args {
  WaveDev w;
  const int4* items;
  int nitems;
  const float* A;
  const float* B;
  const float* C0;
  float* C;
  double alpha, beta;
  double diag;
  int sym;
  double* res2;
  const int* state;
  int skip_state;
};
cudaError_t launch_gemm_f32(const GemmF32Args& a, cudaStream_t st);

#ifdef __CUDACC__
// FP64 -> FP32 by truncating the mantissa with integer operations (GB300's
// FP64 pipe is ~60x slower than its FP32 pipe, so the bulk kernels avoid it).
// Relative error < 2^-23; values below 2^-126 become 0.  Only used where the
// result feeds a 16-bit split or another low-precision step.
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned sign = unsigned(b >> 63);
  const int ex = int((b >> 52) & 0x7FF) - 1023;
  if (ex < -126) return sign ? -0.0f : 0.0f;
  if (ex > 127) return sign ? -3.402823466e38f : 3.402823466e38f;
  const unsigned mant = unsigned((b >> 29) & 0x7FFFFFu);
  return __uint_as_float((sign << 31) | (unsigned(ex + 127) << 23) | mant);
}

// FP32 -> FP64 exactly, with integer operations
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;  // zero (subnormal floats do not occur here)
  const unsigned long long b = (static_cast<unsigned long long>(u >> 31) << 63) |
                               (static_cast<unsigned long long>(e - 127 + 1023) << 52) |
                               (static_cast<unsigned long long>(u & 0x7FFFFFu) << 29);
  return __longlong_as_double(static_cast<long long>(b));
}

#endif

}  // namespace submat

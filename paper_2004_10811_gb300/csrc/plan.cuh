// The plan object behind the opaque submat_plan handle.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <vector>

#include "common.cuh"

namespace submat {

submat_status dev_alloc(void** p, size_t bytes, const char* what);
submat_status validate_pattern_public(int nblk, const int32_t* bs, const int64_t* rp,
                                      const int32_t* ci);
const char* last_error();
size_t mixed_bytes_per_elem();
size_t adjoint_tc_bytes_per_elem();
constexpr int kPowerIters = 10;  // power steps of the spectral estimate
constexpr int kProbeMaxIter = 40;  // Newton-Schulz cap of a mu-search probe
void free_mixed(void* state);
void free_adjoint_tc(void* state);

// Launch plan of an exact sliced product (mixed.cu).  Slices are numbered
// 1..n; a group is one exact accumulator: np products (pr[i] = (p, q)) of one
// level and weight 2^shift.  A launch carries group g0 and, if g1 >= 0, group
// g1 in a second accumulator (g0's weight the larger).
struct SliceGroup { int np; int pr[2][2]; int shift; };
constexpr int kSliceMaxAcc = 4;  // accumulators (groups) per launch at most
struct SliceLaunch { int ng; int g[kSliceMaxAcc]; };
// max_acc 2: pairs of groups at most 2^6 apart (combined in 32-bit integers);
// max_acc 4: up to four groups of any weights (combined in 64-bit integers)
void slice_plan(int nx, int ny, bool sym_pairs, int per_acc, int max_acc, std::vector<SliceGroup>* groups,
                std::vector<SliceLaunch>* launches);
void slice_sets(const SliceGroup* const* gs, int ng, int* as, int* na, int* bs, int* nb);
int slice_max_slices();

// The mu search's bracketing bisection on any evaluator of N(mu) (driver.cu).
// bound() gives the spectral bound b at mu0 after the first evaluation.
// Returns OK, MU_NO_ROOT (bracket below 1e-10 b), NOT_CONVERGED (max_steps)
// or the evaluator's error; out->mu is the final mu, where the last
// evaluation was made.
struct MuSearchOut {
  double mu = 0, n_best = 0, lo = 0, hi = 0;
  int steps = 0;        // full evaluations
  int probes = 0;       // probe evaluations
  int probe_steps = 0;  // bisection steps that a probe decided
};
// probe (may be empty): a cheaper evaluation returning N_p and a bound B with
// |N(mu) - N_p| <= B; a bisection step takes the probe's side when
// |N_p - n_el| > B, and after the first inconclusive probe only full
// evaluations follow.
using MuProbe = std::function<submat_status(double, double*, double*)>;
submat_status mu_bisect(const std::function<submat_status(double, double*)>& eval,
                        const std::function<double()>& bound, double n_el, double mu0, double tol,
                        int max_steps, MuSearchOut* out, const MuProbe& probe = MuProbe());


// Finite temperature (fermi.cu): the Chebyshev series of tanh(c x) on
// [-1, 1] cut at odd degree m, folded for 16 baby steps: p = sum_j R_j T_j(Y),
// Y = T_16, R_j = sum_{q < 8} r[j * 8 + q] T_{2q+1}.
constexpr int kFermiBaby = 16;
constexpr int kFermiBuffers = kFermiBaby / 2 + 3;  // odd T_k, T_2 / Y, two Clenshaw buffers
constexpr int kFermiMaxDegree = 8191;
struct FermiPoly {
  int m = 0, blocks = 0;
  double trunc = 0.0;  // sum of |c_k| beyond m: bounds the truncation error on [-1, 1]
  std::vector<double> r;
};
submat_status fermi_poly(double c, double tol, int max_degree, FermiPoly* out);
size_t fermi_bytes_per_elem(int prec);

struct Wave {
  int first = 0;           // first global block column of the wave
  int count = 0;           // submatrices in the wave
  int64_t elems = 0;       // sum of ld^2
  int64_t max_ld2 = 0;
  WaveDev dev{};
  int2* gather_items = nullptr;  // (s, t) for every local block row
  int n_gather = 0;
  int4* sym64 = nullptr;   // 64x64 tiles with ti <= tj
  int n_sym64 = 0;
  int4* full64 = nullptr;  // all 64x64 tiles
  int n_full64 = 0;
  int4* sym128 = nullptr;  // 128x128 tiles with ti <= tj: (s, ti, tj, bucket | slot << 8)
  int n_sym128 = 0;
  int4* full128 = nullptr;
  int n_full128 = 0;
  int4* sym256 = nullptr;  // 128x256 tiles (s, ti, tj, tag) covering sub-tiles (ti, 2tj), (ti, 2tj+1)
  int n_sym256 = 0;
  int4* full256 = nullptr;
  int n_full256 = 0;
  int bn = 128;            // tensor-core tile width used for this wave
  std::vector<int64_t> bucket_ld, bucket_base;  // size buckets: [count][ld][ld] each
  std::vector<int> bucket_count;
  std::vector<int32_t> host_ld, host_n;
  std::vector<int64_t> host_off;
  // tensor-core work (filled by the mixed path on first use)
  void* tc = nullptr;
};

// Adjoint helpers (backward.cu) on an FP32 E in the wave layout: the seed
// E_0 = G / beta (or I / beta), the scatter-add of -1/2 E into Kbar, and the
// per-submatrix dN/dmu part.
cudaError_t launch_bwd_seed_f32(const PatternDev& g, const Wave& wv, const double* Dbar, const double* beta,
                                float* E, int identity, cudaStream_t st);
cudaError_t launch_bwd_scatter_add_f32(const PatternDev& g, const Wave& wv, int nb_max, const float* E,
                                       double* Kbar, cudaStream_t st);
cudaError_t launch_bwd_dn_f32(const PatternDev& g, const Wave& wv, const float* E, double* part,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_bwd_seed(const PatternDev& g, const Wave& wv, const double* Dbar, const double* beta, T* E,
                            int identity, cudaStream_t st);
template <typename T>
cudaError_t launch_bwd_scatter_add(const PatternDev& g, const Wave& wv, int nb_max, const T* E, double* Kbar,
                                   cudaStream_t st);

// Event pairs around kernel launches, grouped in classes (submat_stats kernel_*).
struct KernelTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, size_t>> marks;  // (class, index of the start event)
  ~KernelTimer();
  submat_status start(int cls, cudaStream_t st, size_t* tok);
  submat_status stop(size_t tok, cudaStream_t st);
  submat_status collect(double* ms, int32_t* count);  // after a stream sync
};

enum KernelClass {
  KC_TC_NS = 0, KC_TC_REF = 1, KC_SIMT = 2, KC_GATHER = 3, KC_TC_HP = 4, KC_TC_ADJ = 5, KC_SCATTER = 6,
  KC_COUNT = 8
};

int max_ld(const Wave& wv);

struct Plan {
  ~Plan();

  // pattern (host)
  int nblk = 0;
  int64_t nnzb = 0, nvals = 0;
  submat_options opt{};
  double tol_eff = 1e-14;
  std::vector<int32_t> bs, col, locoff, tpos, nsub, koff, diagpos;
  std::vector<int64_t> row_ptr, valptr, rowof;
  int nb_max = 0, n_max = 0, n_min = 0, bs_max = 1;
  // submatrices: nq of them (nblk without groups); per submatrix q its
  // dimension qn[q], extracted width qext[q] (sum of its members' block
  // sizes), block rows qrows[qsp[q] .. qsp[q+1]) with local offsets qloc;
  // qof[j] is the submatrix of block column j
  bool grouped = false;
  int nq = 0, qm_max = 1;
  std::vector<int32_t> qn, qext, qrows, qloc, qof, qmp, qmcol, qmkoff, dloc;
  std::vector<int64_t> qsp;
  int nbj_max = 0;  // most blocks in one block column (the member scatter's tables)
  ScatterGeom geom(const Wave& wv) const {
    return ScatterGeom{nb_max, max_ld(wv), bs_max, grouped ? qm_max : 0, nbj_max};
  }
  int col_lo = 0, col_hi = 0;      // evaluated block columns
  double sum_n2 = 0, sum_n3 = 0;

  // device
  PatternDev g{};
  int64_t* d_rowof = nullptr;
  std::vector<Wave> waves;
  int max_wave = 0;
  void* ws = nullptr;
  int64_t ws_elems = 0;
  size_t ws_bytes = 0;
  NsStateDev ns{};
  int* d_flags = nullptr;
  int* d_active = nullptr;
  double* d_trpart = nullptr;
  double* d_scalar = nullptr;
  double* d_symtmp = nullptr;
  double* d_hostK = nullptr;   // staging for submat_sign_host
  double* d_hostD = nullptr;
  void* h_pinned = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<void*> owned;
  void* mixed = nullptr;       // mixed-path state (mixed.cu)
  void* adj_tc = nullptr;      // tensor-core adjoint state (mixed.cu)
  // adjoint: its own waves and workspace (six dense buffers per submatrix)
  std::vector<Wave> bwaves;
  int max_bwave = 0;
  void* bws = nullptr;
  int64_t bws_elems = 0;
  double* d_dnpart = nullptr;
  double dn_acc = 0.0;
  // finite temperature: per block column sum of squares of the extracted
  // columns, and the last evaluation's polynomial
  double* d_sqpart = nullptr;
  int fermi_degree = 0;
  double fermi_trunc = 0.0, fermi_flops = 0.0;

  // results of the last evaluation (per global block column)
  std::vector<int> res_iters, res_notconv;
  std::vector<double> res_resid, res_beta, res_bound;  // res_bound: min(max row abs-sum, ||a||_F)
  int last_flags = 0;              // status word of the last read_flags
  bool probe_mode = false;         // mixed path: stop after the FP16x3 iteration (mu-search probe)
  submat_stats stats{};
  KernelTimer timer;
  long long launches_at_start = 0;
  std::vector<double> gather_bytes;  // per block column (timing only)

  template <typename T>
  submat_status alloc(T** p, size_t count, const char* what);
  template <typename T>
  submat_status put(T** p, const std::vector<T>& v, cudaStream_t st, const char* what);

  submat_status build(int nblk, const int32_t* bs, const int64_t* rp, const int32_t* ci,
                      const submat_options* o, cudaStream_t st, const int32_t* groups = nullptr);
  submat_status build_groups(const int32_t* groups);
  submat_status sign(const double* K, double mu, double* D, cudaStream_t st);
  submat_status sign_host(const double* K, double mu, double* D, cudaStream_t st);
  submat_status trace(const double* D, double* tr, cudaStream_t st);
  submat_status mu_search(const double* K, double n_el, double mu0, double tol, int max_steps,
                          double* mu_out, double* D, cudaStream_t st);
  submat_status backward(const double* K, double mu, const double* Dbar, double* Kbar,
                         double* dN_dmu, cudaStream_t st);
  submat_status autotune(const double* K, double mu, double* D, int32_t* chosen, cudaStream_t st);

  // internals
  submat_status read_flags(cudaStream_t st, int* out);
  submat_status gather_wave(Wave& wv, const double* K, double mu, double* A, cudaStream_t st);
  submat_status collect_wave(const Wave& wv, cudaStream_t st);
  submat_status add_phase_times();
  // the extraction of one wave, timed as class KC_SCATTER (bytes_per_entry:
  // what one extracted entry reads and writes)
  submat_status scatter_timed(const Wave& wv, double bytes_per_entry, const std::function<cudaError_t()>& launch,
                              cudaStream_t st);
  void reset_stats();
  void finish_stats(bool adjoint = false);
  submat_status sign_fp64(const double* K, double mu, double* D, cudaStream_t st);
  submat_status sign_fp32(const double* K, double mu, double* D, cudaStream_t st);
  submat_status sign_mixed(const double* K, double mu, double* D, cudaStream_t st);
  template <typename T>
  submat_status sign_fermi(const double* K, double mu, double* D, cudaStream_t st);
  // one wave of the finite-temperature evaluation on workspace `w` of E
  // elements per buffer; with Dbar set, the polynomial runs on dual numbers
  // and -1/2 of its derivative part (L_f(a_j, G_j)) is added into Kbar
  template <typename T>
  submat_status fermi_wave(Wave& wv, const double* K, double mu, double* D, const double* Dbar, double* Kbar,
                           void* w, int64_t E, cudaStream_t st);
  submat_status fermi_dn_dmu(cudaStream_t st, double* out);
  submat_status backward_fermi(const double* K, double mu, const double* Dbar, double* Kbar, double* dN_dmu,
                               cudaStream_t st);
  submat_status mu_newton(const double* K, double n_el, double mu0, double tol, int max_steps,
                          double* mu_out, double* D, cudaStream_t st);
  submat_status build_waves(size_t bpe, size_t cap, std::vector<Wave>& out, cudaStream_t st);
  template <typename T>
  submat_status backward_wave(Wave& wv, const double* K, double mu, const double* Dbar, double* Kbar,
                              double* dn_part, void* bws, cudaStream_t st);
  submat_status backward_wave_tc(size_t wi, const double* K, double mu, const double* Dbar, double* Kbar,
                                 double* dn_part, cudaStream_t st);
  submat_status grow_ns_state(int count);
  template <typename T, typename Args>
  submat_status ns_simt(const Wave& wv, T* buf0, T* buf1, T* Y, double tol, double floor_thr,
                        cudaStream_t st, cudaError_t (*gemm)(const Args&, cudaStream_t), bool certify);
};

template <typename T>
submat_status Plan::alloc(T** p, size_t count, const char* what) {
  void* q = nullptr;
  SM_TRY(dev_alloc(&q, count * sizeof(T), what));
  if (q) owned.push_back(q);
  *p = static_cast<T*>(q);
  return SUBMAT_OK;
}

template <typename T>
submat_status Plan::put(T** p, const std::vector<T>& v, cudaStream_t st, const char* what) {
  void* q = nullptr;
  SM_TRY(dev_alloc(&q, v.size() * sizeof(T), what));
  if (q) owned.push_back(q);
  *p = static_cast<T*>(q);
  if (!v.empty())
    SM_CUDA(cudaMemcpyAsync(q, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return SUBMAT_OK;
}

}  // namespace submat

/*
 * submat.h -- C ABI of the GB300 submatrix sign library.
 *
 * The library evaluates the density matrix of a symmetric block-sparse,
 * orthogonalised Kohn-Sham matrix K,
 *
 *     D = 1/2 (I - sign(K - mu I))            (Eq. DsignSym with S = I)
 *
 * by the submatrix method (Section III-A): for every block column j it
 * assembles the principal submatrix a_j = K[N(j), N(j)] - mu I over the block
 * rows N(j) that hold a stored block in column j, evaluates sign(a_j) on the
 * GPU by scaled Newton-Schulz iteration (Section II-B), and copies the columns
 * of block j of 1/2 (I - sign(a_j)) into block column j of D, keeping K's
 * block pattern.
 *
 * Matrix format (both K and D, and the gradients Dbar and Kbar): block CSR
 * over nblk block rows.  row_ptr[nblk + 1] (int64) and col_idx[nnzb] (int32)
 * list the stored blocks; column indices must be strictly increasing inside a
 * row, every diagonal block must be stored and the pattern must be symmetric
 * (block (i, j) stored iff (j, i) stored).  Block p of row r and column c
 * holds block_sizes[r] * block_sizes[c] doubles, row-major; blocks follow
 * one another in CSR order with no padding, so block p starts at
 * sum_{q < p} area(q).  K must be numerically symmetric (K_(j,i) = K_(i,j)^T).
 *
 * Conventions.
 *   - Device pointers are CUDA device memory that the caller owns.  The plan
 *     owns its own workspaces (it allocates them with cudaMalloc when it is
 *     created, and on first use of the host-buffer entry point).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every entry point that returns a status synchronises that
 *     stream before it returns, so results and statuses are final.
 *   - No C++ exception crosses this boundary.  On failure a function returns
 *     a nonzero submat_status and submat_last_error() describes it.
 *   - A plan is not thread-safe: calls on one plan must not overlap.
 */
#ifndef SUBMAT_H
#define SUBMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct submat_plan submat_plan;

typedef enum {
  SUBMAT_OK = 0,
  SUBMAT_ERR_INVALID_ARG = 1,   /* null pointer, bad size or option */
  SUBMAT_ERR_PATTERN = 2,       /* pattern not symmetric / unsorted / out of range / no diagonal */
  SUBMAT_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  SUBMAT_ERR_OOM = 4,           /* workspace does not fit (even one submatrix per wave) */
  SUBMAT_ERR_NONFINITE = 5,     /* K (or a gradient input) holds NaN or Inf */
  SUBMAT_ERR_NOT_CONVERGED = 6, /* some submatrix hit max_iter; D is written, see stats */
  SUBMAT_ERR_MU_NO_ROOT = 7,    /* mu search ended on a step of the electron-count staircase */
  SUBMAT_ERR_TIMEOUT = 8,       /* a bounded device wait gave up */
  SUBMAT_ERR_UNSUPPORTED = 9    /* feature not available for these sizes/options */
} submat_status;

typedef enum {
  SUBMAT_FP64 = 0,               /* Newton-Schulz in FP64 throughout */
  SUBMAT_FP32 = 1,               /* Newton-Schulz in FP32 (no refinement) */
  SUBMAT_MIXED_BF16_REFINE = 2   /* tensor-core Newton-Schulz on FP16 (hi, lo) pairs, then an
                                    FP64-anchored correction from BF16 and exact sliced
                                    tensor-core products (the name predates the FP16 stage) */
} submat_precision;

typedef struct {
  int prec;                    /* submat_precision */
  double tol;                  /* stop when ||X^2 - I||_F <= sqrt(n_j) * tol, then one more
                                  iteration (Section VI-A: involution as stopping test);
                                  0 selects 1e-14 for FP64, 1e-6 for FP32, 2e-5 for the
                                  FP16x3 stage of the mixed path */
  int max_iter;                /* Newton-Schulz iteration cap; 0 selects 100 */
  int beta_mode;               /* X_0 = a / beta.  0 (default): beta = 1.05 x a 10-step
                                  power-iteration estimate of the spectral radius when that
                                  is below the bound of mode 1 (a tighter beta saves
                                  iterations).  The estimate is only a lower bound on rho,
                                  and an eigenvalue of X_0 beyond sqrt(3) would converge to
                                  the wrong sign, so the scale is certified from the first
                                  squaring: rho(X_0)^2 <= ||X_0^2||_inf (largest row
                                  abs-sum, rounding included) must stay below 2.94 (2.2 for
                                  the third-order iteration), else X_0 is scaled down to
                                  meet it, never below 1.7 (1.45) / beta_bound, which is
                                  safe by itself (submat_stats.scale_reduced counts them);
                                  1: beta = min(max row abs-sum, ||a||_F) >= rho(a) only */
  int symmetrize;              /* 1: return (D + D^T) / 2 on the pattern; 0: column-assembled D */
  size_t workspace_cap_bytes;  /* device workspace cap; 0 = 80 % of free memory at plan time */
  int refine_rounds;           /* mixed path: correction rounds; 0 selects 1.  With one
                                  round a submatrix is accepted when its Lyapunov solve
                                  converged (which bounds |a|/gap); with two or more the last
                                  correction must be below 1e-8.  Others are re-solved in
                                  FP64 (submat_stats.refine_fallback). */
  int timing;                  /* 1: time every GEMM launch with CUDA events (submat_stats
                                  kernel_* fields); adds one event pair per launch */
  int col_begin, col_end;      /* evaluate only block columns [col_begin, col_end) of D (one
                                  contiguous chunk, Section IV-E); 0, 0 = all columns.  The
                                  other block columns of D are left untouched, and the
                                  adjoint sums the contributions of these columns only. */
  int hp_mode;                 /* mixed path, the two residual products I - S^2 and S a:
                                  0: BF16 tensor cores on 6-bit integer slices (S on a 24-bit
                                  grid: four slices; a row-scaled: six), exact integer sums
                                  in 64-bit integers, one rounding to FP64;
                                  1: FP64 SIMT GEMM */
  int tile_n_ns;               /* tensor-core output tile width in the Newton-Schulz phase:
                                  0 = chosen per wave, or 128 / 256 */
  int tile_n_corr;             /* the same for the correction phase (0 = 256) */
  int tile_n_hp;               /* the same for the sliced residual products (0 = 128) */
  int iteration;               /* sign iteration of the mixed path: 0 (default) Newton-Schulz
                                  X <- X (3I - X^2) / 2 (Section II-B); 1 the third-order
                                  X <- X (15I - 10X^2 + 3X^4) / 8 of the paper's GPU runs
                                  (Section VI-A), three products per step.  Other
                                  precisions support 0 only (UNSUPPORTED at plan creation) */
  int adjoint_mode;            /* GEMMs of submat_sign_backward: 0 (default) SIMT in the plan's
                                  precision (FP32 for mixed plans); 1 BF16x3 tensor cores, mixed
                                  plans only (UNSUPPORTED otherwise) -- about 15x faster, with
                                  about 10x the error of mode 0 (BF16x3 carries ~16 bits) */
  double kT;                   /* electronic temperature (Section IV-F, last paragraph: the
                                  Fermi function in place of signum), in the units of K;
                                  0 (default) is zero temperature.  With kT > 0 every call
                                  that evaluates D returns D = f(K - mu I),
                                  f(x) = 1 / (1 + exp(x / kT)) = (1 - tanh(x / 2kT)) / 2, per
                                  submatrix by a Chebyshev series of tanh (truncation below
                                  1e-13 for FP64 plans, 1e-8 for FP32) on the SIMT GEMM in the
                                  plan's precision; mixed plans return UNSUPPORTED.  The
                                  series degree grows like (spectral scale) / kT: a degree
                                  above 8191 returns UNSUPPORTED.  submat_mu_search then takes
                                  Newton steps on the smooth Tr D(mu) (submat_stats.dn_dmu),
                                  and submat_sign_backward differentiates the same series */
} submat_options;

/* Aggregate statistics of the last submat_sign / submat_mu_search call. */
typedef struct {
  int32_t nsub;            /* number of submatrices (= nblk) */
  int32_t n_min, n_max;    /* smallest / largest submatrix dimension */
  int32_t waves;           /* workspace waves the batch was split into */
  int32_t iters_min, iters_max; /* Newton-Schulz iterations over submatrices */
  int32_t not_converged;   /* submatrices that hit max_iter */
  int32_t refine_rounds;   /* correction rounds run (mixed path) */
  int32_t refine_cg_iters; /* conjugate-gradient launches over all rounds and waves */
  int32_t refine_fallback; /* submatrices re-solved in FP64 because the correction did not settle */
  double  sum_n2, sum_n3;  /* sum over submatrices of n_j^2 and n_j^3 */
  double  flops_ns;        /* standard-count Newton-Schulz flops: sum_j 4 n_j^3 iters_j
                              (after submat_sign_backward: the adjoint's
                              sum_j 12 n_j^3 (iters_j + 2)) */
  double  flops_refine;    /* standard-count refinement flops */
  double  max_resid;       /* largest final ||X^2 - I||_F / sqrt(n_j) */
  double  ms_gather, ms_ns, ms_refine, ms_scatter; /* phase times (CUDA events) */
  size_t  workspace_bytes; /* device workspace held by the plan */
  int64_t launches;        /* kernel launches issued by the call */
  /* Per kernel class, with options.timing = 1 (else zero):
   *   0 tensor-core GEMM, Newton-Schulz;  1 tensor-core GEMM, correction
   *   (split products and the Lyapunov CG);  2 FP64/FP32 SIMT GEMM;
   *   3 gather (assembly) kernel;  4 tensor-core GEMM, sliced FP64-accurate
   *   residual products;  5 tensor-core GEMM, adjoint (adjoint_mode 1);
   *   6 extraction (scatter) kernel;  7 reserved.
   * kernel_ms: summed launch durations.  kernel_work: algorithmic work of
   * those launches -- flops for the GEMM classes at the standard count (2 n^3
   * per n x n product the method needs, also where the kernels compute only
   * the upper tiles of a symmetric result; a split or sliced product counts
   * once, as the product it represents), bytes moved for the gather (8 per
   * dense element written plus 8 per K value read) and the scatter (per
   * extracted entry: the iterate read, 8 or 4 bytes, the mixed path's two
   * FP32 corrections, and 8 for D written).
   * kernel_exec: MMA flops the tensor cores executed (every slice product,
   * tile padding included); 0 for the other classes. */
  double  kernel_ms[8];
  int32_t kernel_launches[8];
  double  kernel_work[8];
  double  kernel_exec[8];
  int32_t mu_steps;        /* sign evaluations of the last submat_mu_search (0 otherwise) */
  int32_t scale_reduced;   /* submatrices whose power-estimate scale the certificate did not
                              prove safe, so X_0 was scaled down (see beta_mode) */
  int32_t poly_degree;     /* finite temperature: the largest Chebyshev degree of the last
                              evaluation (iters_* then count its matrix products) */
  double  poly_trunc;      /* ... and its truncation bound, sum of |c_k| beyond the degree */
  int32_t mu_probes;       /* probe evaluations of the last submat_mu_search (mixed plans) */
  double  dn_dmu;          /* finite temperature: dN/dmu = sum_j sum_{c in block j}
                              [f(a_j) (1 - f(a_j))]_cc / kT at the last evaluation's mu,
                              over the evaluated block columns (-L_f(a_j, I) summed; the
                              adjoint's quantity); 0 at zero temperature */
} submat_stats;

/* Fill *opt with defaults (FP64, default tolerances, beta_mode 0). */
void submat_options_default(submat_options* opt);

/*
 * Build a plan for one block pattern (Section IV-A: the global pattern and
 * the per-submatrix index maps are computed once and reused).
 *   nblk         number of block rows/columns (>= 1)
 *   block_sizes  host int32[nblk], each >= 1
 *   row_ptr      host int64[nblk + 1], row_ptr[0] = 0, non-decreasing
 *   col_idx      host int32[row_ptr[nblk]]
 *   opt          host options (NULL = defaults)
 *   stream       stream used for the plan's uploads
 *   out          receives the plan (NULL on failure)
 * The host arrays are copied; the caller may free them afterwards.
 * Errors: INVALID_ARG, PATTERN, OOM, CUDA.
 */
submat_status submat_plan_create(int nblk, const int32_t* block_sizes,
                                 const int64_t* row_ptr, const int32_t* col_idx,
                                 const submat_options* opt, void* stream,
                                 submat_plan** out);

/*
 * A plan whose submatrices are shared by groups of block columns (Section
 * IV-C, "Generating Submatrices From Multiple Block Columns"): the block
 * columns j with groups[j] = q share one submatrix over N(q), the ascending
 * union of their row sets N(j), so a_q = K[N(q), N(q)] - mu I, and every
 * member j takes the columns of block j of 1/2 (I - sign(a_q)) into block
 * column j of D (rows N(j): D keeps K's pattern).  Larger submatrices change
 * the method's truncation (they see more of K) and, by the paper's cost model
 * sum_q n_q^3 (Eq. estimatedspeedup), can cost fewer operations when the
 * members are close in space.
 *   groups  host int32[nblk], group ids 0 .. ngroups - 1, every id used;
 *           copied.  paper_2004_10811_gb300.grouping finds groups by
 *           periodic k-means on the molecule centres.
 * Other arguments and errors as submat_plan_create.  Column ranges
 * (col_begin / col_end) and submat_sign_backward are UNSUPPORTED for
 * grouped plans.  Statistics per block column report its group's submatrix.
 */
submat_status submat_plan_create_grouped(int nblk, const int32_t* block_sizes, const int64_t* row_ptr,
                                         const int32_t* col_idx, const int32_t* groups,
                                         const submat_options* opt, void* stream, submat_plan** out);

/* Release the plan and all device memory it owns.  NULL is allowed. */
submat_status submat_plan_destroy(submat_plan* plan);

/*
 * D = 1/2 (I - sign(K - mu I)) by the submatrix method (Section III-A,
 * Eq. DsignSym with S = I, sign(0) = 0 as in Eq. signevext).
 *   K_vals  device double[plan value count], the BSR values of K
 *   mu      chemical potential
 *   D_vals  device double[plan value count], written in K's layout
 * Returns OK, NONFINITE (K holds NaN/Inf; D untouched), NOT_CONVERGED
 * (D written; some submatrix reached max_iter, e.g. a singular one),
 * TIMEOUT, CUDA.
 */
submat_status submat_sign(submat_plan* plan, const double* K_vals, double mu,
                          double* D_vals, void* stream);

/* As submat_sign, but K_vals and D_vals are HOST arrays; the copies to and
 * from the device run inside the call (on plan-owned device buffers). */
submat_status submat_sign_host(submat_plan* plan, const double* K_host, double mu,
                               double* D_host, void* stream);

/*
 * Tr D in FP64 (Section IV-G: the electron count n_elec).  Sums the diagonal
 * entries of the diagonal blocks; the reduction order is fixed, so the
 * result is deterministic.
 *   D_vals  device double[plan value count];  tr  host double (output)
 */
submat_status submat_trace(submat_plan* plan, const double* D_vals, double* tr,
                           void* stream);

/*
 * Find mu with Tr D(mu) = n_el (canonical adaptation, Section IV-G /
 * Algorithm 1), re-evaluating the submatrix signs at each trial mu.
 * Bisection on a bracket [mu0, mu0 + 1.01 b] or [mu0 - 1.01 b, mu0], on the
 * side of n_el given by Tr D(mu0), where b = max_j min(max row abs-sum,
 * ||a_j||_F) is a rigorous bound on the spectra of the submatrices at mu0,
 * so that N at the far end is 0 or n.  (If the bisection closes in on the far
 * end, that end is evaluated, and the bracket moves outward should it not
 * hold n_el.)  At zero temperature dN/dmu = 1/2 sum_j sum_{c in j}
 * L_sign(a_j, I)_cc is exactly zero for nonsingular a_j --
 * submat_sign_backward reports it -- so Newton steps never apply.
 *   n_el       target electron count, 0 <= n_el <= n (else INVALID_ARG)
 *   mu0        starting guess
 *   tol        stop when |Tr D - n_el| <= tol * n_el
 *   max_steps  cap on sign evaluations (>= 1)
 *   mu_out     host double: final mu
 *   D_vals     device double[value count]: D at mu_out
 * At zero temperature Tr D(mu) is a staircase: if the bracket shrinks below
 * 1e-10 x the spectral bound without meeting tol, the call returns
 * MU_NO_ROOT with mu_out and D at the bracket end nearest n_el.
 * Mixed plans probe each step first: the FP16x3 Newton-Schulz iterate alone
 * (no correction, no FP64 fallback, at most 40 iterations), whose trace is
 * within 1/2 sum_q b_q (r_q sqrt(n_q) + 1e-3) of the full result (r_q the
 * final involution residual, b_q the extracted width); the probe decides the
 * step when its count lies farther than that (and tol) from n_el.  After the
 * first inconclusive probe only full evaluations follow, and D and mu_out
 * always come from a full one.  max_steps counts both kinds
 * (submat_stats.mu_steps: full, mu_probes: probes).
 * NOT_CONVERGED: the step cap was reached (mu_out and D at the evaluation
 * nearest n_el), or the evaluation at mu_out left some submatrix
 * unconverged (D written, see submat_get_stats); a submatrix that diverged
 * (its involution residual grew past 1e6) ends the search at once.
 */
submat_status submat_mu_search(submat_plan* plan, const double* K_vals, double n_el,
                               double mu0, double tol, int max_steps, double* mu_out,
                               double* D_vals, void* stream);

/*
 * Vector-Jacobian product of K -> D (the adjoint of the submatrix density
 * map).  Block column j contributes abar_j = -1/2 L_sign(a_j, G_j), where G_j
 * holds Dbar's block column j in its columns of block j and zeros elsewhere,
 * and L_sign is the Frechet derivative of sign (computed by the coupled
 * Newton-Schulz iteration on [[X, E], [0, X]]); abar_j is added into every
 * stored block of K that a_j was assembled from.
 *   Dbar_vals  device double[value count]  (upstream gradient, K's layout)
 *   Kbar_vals  device double[value count]  (output, overwritten)
 *   dN_dmu     host double or NULL: 1/2 sum_j sum_{c in block j} L_sign(a_j, I)_cc
 * The products run on the SIMT GEMM in the plan's precision (FP32 for mixed
 * plans), or with options.adjoint_mode = 1 as BF16x3 split products on the
 * tensor cores, E's transpose kept beside it for the products that read E as
 * their right operand.
 * Finite temperature (options.kT > 0, D = f(K - mu I) with the Fermi
 * function): abar_j = L_f(a_j, G_j), from the Chebyshev evaluation of D run
 * on dual numbers (every matrix M with a derivative part M',
 * (AB)' = A'B + AB', seeded with G_j / sigma), three products for every one
 * of the forward; dN/dmu = sum_j sum_{c in block j} [f(a_j)(1 - f(a_j))]_cc / kT
 * from the same pass.
 */
submat_status submat_sign_backward(submat_plan* plan, const double* K_vals, double mu,
                                   const double* Dbar_vals, double* Kbar_vals,
                                   double* dN_dmu, void* stream);

/*
 * Tile-shape autotuner (the paper has no counterpart: its GPU runs use cuBLAS).
 * For a mixed-precision plan, times full evaluations of D(mu) for this K with
 * CUDA events per kernel class. The candidates are 128- and 256-wide output
 * tiles for each tensor-core phase: Newton-Schulz, correction split products
 * and sliced residual products. One untimed warm-up evaluation runs first.
 * The widths are independent per phase, so the plan keeps the faster width
 * of each, and later calls of submat_sign use them.
 *   K_vals      device double[value count]
 *   D_vals      device double[value count] (caller-owned): receives D(mu)
 *   tile_n_out  host int[3] or NULL: the chosen widths (NS, correction, sliced)
 * FP64 and FP32 plans have no tile choice: the call evaluates D once and
 * reports zeros.  Costs three evaluations; the timing hooks of the `timing`
 * option are used, whatever its value.
 */
submat_status submat_autotune(submat_plan* plan, const double* K_vals, double mu, double* D_vals,
                              int32_t* tile_n_out, void* stream);

/* Number of doubles in K's (and D's) value array for this plan. */
int64_t submat_plan_value_count(const submat_plan* plan);

/* Statistics of the last sign evaluation (host struct). */
submat_status submat_get_stats(const submat_plan* plan, submat_stats* out);

/* Per-submatrix data of the last sign evaluation, host arrays of length nblk
 * (any may be NULL): dimension n_j, Newton-Schulz iterations, final
 * ||X^2 - I||_F / sqrt(n_j), and beta. */
submat_status submat_get_sub_stats(const submat_plan* plan, int32_t* dims, int32_t* iters,
                                   double* resid, double* beta);

/*
 * Dense one-matrix evaluation that allocates nothing (the paper has no
 * counterpart; it is a convenience of this library).
 *
 *   D = 1/2 (I - sign(K - mu I))  for one dense symmetric n x n matrix K,
 *
 * by scaled FP64 Newton-Schulz iteration on the FP64 path's kernels, with
 * X_0 = (K - mu I) / beta and beta = min(max row abs-sum, ||K - mu I||_F),
 * the rigorous bound only (no power-estimate tightening, so it may take a
 * few more iterations than a plan), for callers that may not call
 * cudaMalloc or cudaMallocHost: codes
 * that reserve the whole device for their own memory pool, allocators that
 * forbid foreign allocations, and time steps in which an allocation's
 * implicit device synchronisation is not acceptable.
 *   n         1 <= n <= SUBMAT_NOALLOC_MAX_N; larger n is rejected with
 *             INVALID_ARG
 *   K_dev     device double[n * n], row-major (caller-owned)
 *   D_dev     device double[n * n], row-major (caller-owned output)
 *   iters_out host int or NULL: Newton-Schulz iterations taken
 * All scratch (6 MiB) is one file-scope device array that every GPU loading
 * the library holds until the process exits.  Every call looks up that
 * array's device address on the current device (cudaGetSymbolAddress, a
 * host-side lookup that allocates nothing); the first call on a device also
 * loads the library's device code there, so make that first call before
 * any stream capture on the device.  Every call shares the
 * array and it keeps the previous call's contents, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race; serialise
 * them.  The call synchronises `stream`.
 * Returns OK, INVALID_ARG, NONFINITE, NOT_CONVERGED (D written), CUDA.
 */
#define SUBMAT_NOALLOC_MAX_N 512
submat_status submat_dense_sign_noalloc(int n, const double* K_dev, double mu, double* D_dev,
                                        int* iters_out, void* stream);

/* Message of the last failure on this thread ("" if none). */
const char* submat_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SUBMAT_H */

/*
 * submat_debug.h -- test hooks of the submatrix library.
 *
 * These entry points exercise one kernel in isolation so that tests can
 * compare it with a plain reference of the same operation.  They are not
 * steps of the density-matrix path.  Conventions (status codes, streams,
 * submat_last_error) are those of submat.h.
 */
#ifndef SUBMAT_DEBUG_H
#define SUBMAT_DEBUG_H

#include "submat.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Grouped BF16 tensor-core GEMM (the Newton-Schulz product engine):
 *   C_s = A_s B_s^T,  s = 0..count-1,
 * for square matrices stored back to back as [count][ld][ld] on the device.
 *   ld     leading dimension, a multiple of 64 (<= 8192)
 *   n      logical dimension (n <= ld); only used for the residual
 *   A_hi, A_lo, B_hi, B_lo   device BF16 arrays [count][ld][ld]; the *_lo may be
 *          NULL when split == 0
 *   split  bit 0 clear: C = A_hi B_hi^T;  set: C = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T.
 *          Bit 1 set: the operands are FP16 instead of BF16 (all four alike)
 *   sym    1: only tiles with ti <= tj are computed and each is mirrored
 *          (B must then be symmetric and A B^T symmetric)
 *   C      device FP32 [count][ld][ld] (output)
 *   res2   device double[count] or NULL: accumulates ||C_s - I_n||_F^2
 *   skip_arrive  test hook: nonzero makes the epilogue withhold its release
 *          of the accumulator, so a bounded wait must expire
 *   timeout_s    limit of each device wait (seconds; <= 0 selects 2 s)
 *   tile_n       output tile width: 128 or 256 (0 selects 128)
 * Returns OK, INVALID_ARG, TIMEOUT (a bounded wait expired; the kernel freed
 * its resources and returned), CUDA.
 */
submat_status submat_debug_tc_gemm(int count, int ld, int n, const void* A_hi, const void* A_lo,
                                   const void* B_hi, const void* B_lo, int split, int sym,
                                   float* C, double* res2, int skip_arrive, double timeout_s,
                                   int tile_n, void* stream);

/*
 * Host-only (no GPU needed): the launch plan of an exact sliced residual
 * product of the mixed path.  The product sum over slice pairs (p, q),
 * p + q <= 8, of 2^(6 (8 - p - q)) X_p Y_q^T is grouped into exact FP32
 * accumulators (one level and one weight each, at most per_acc products) and
 * launches of up to max_acc accumulators.
 *   nx, ny     slices of the two operands (1..6)
 *   sym_pairs  1: X = Y with symmetric slices (nx == ny): only p <= q, the
 *              p < q products carry twice the weight (shift + 1)
 *   per_acc    products per accumulator: 2 (K extents up to 2048) or 1
 *   max_acc    accumulators per launch: 2 (256-wide tiles: paired groups at
 *              most 2^6 apart, combined in 32-bit integers) or 4 (128-wide
 *              tiles: any weights, combined in 64-bit integers)
 *   out        host int32[cap][5] or NULL: one record per slice product,
 *              (launch, accumulator, p, q, shift); the product's weight is
 *              2^shift times 2^(-48) in the int64 sum
 *   cap        records out can hold
 *   count      host int32: records of the plan (written even when cap is short)
 * Returns OK, or INVALID_ARG (bad sizes, NULL count, cap too small).
 */
submat_status submat_debug_slice_plan(int nx, int ny, int sym_pairs, int per_acc, int max_acc, int32_t* out,
                                      int cap, int32_t* count);

/*
 * Host-only (no GPU needed): the bisection of submat_mu_search (Section IV-G,
 * Algorithm 1's outer loop) on the electron count of a given set of levels,
 *   N(mu) = sum_i 1/2 (1 - sign(levels[i] - mu))   (sign(0) = 0),
 * i.e. the trace of D for a diagonal K, with the spectral bound
 * bound_scale * max_i |levels[i] - mu0|.
 *   levels     host double[nlev]
 *   n_el, mu0, tol, max_steps   as in submat_mu_search
 *   bound_scale  > 0; 1 gives the exact bound, below 1 a bound that
 *              underestimates the spectrum (the bracket must then grow)
 *   probe_err  >= 0; with probe_err > 0 a probe returns N off by probe_err
 *              (alternating sides) with the bound probe_err, as the mixed
 *              path's probes do with their certified bound
 *   mu_out     host double: the final mu
 *   steps      host int32: full evaluations of N
 *   probes     host int32 or NULL: probe evaluations
 *   n_out      host double or NULL: N(mu_out)
 * Returns what submat_mu_search returns: OK, MU_NO_ROOT, NOT_CONVERGED, or
 * INVALID_ARG.
 */
submat_status submat_debug_mu_bisect(const double* levels, int nlev, double n_el, double mu0, double tol,
                                     int max_steps, double bound_scale, double probe_err, double* mu_out,
                                     int32_t* steps, int32_t* probes, double* n_out);

/*
 * Host-only (no GPU needed): the finite-temperature polynomial (Section IV-F,
 * last paragraph; the Fermi function (1 - tanh(x / 2kT)) / 2).  The
 * Chebyshev series of tanh(c x) on [-1, 1], cut at the smallest odd degree m
 * whose coefficient tail sum_{k > m} |c_k| is <= tol, in the baby-step /
 * giant-step form the GPU evaluates:
 *   p(x) = sum_{j < blocks} R_j(x) T_j(T_16(x)),
 *   R_j(x) = sum_{q < 8} r_out[8 j + q] T_{2q+1}(x).
 *   c          the scale sigma / (2 kT) (> 0)
 *   tol        truncation tolerance (> 0)
 *   max_degree largest accepted degree (1 .. 8191); above it UNSUPPORTED
 *   r_out      host double[8 * blocks] or NULL (cap: its length)
 *   degree, blocks, trunc   host outputs: m, the giant-step count, the tail sum
 */
submat_status submat_debug_fermi_poly(double c, double tol, int max_degree, double* r_out, int cap,
                                      int32_t* degree, int32_t* blocks, double* trunc);

#ifdef __cplusplus
}
#endif

#endif /* SUBMAT_DEBUG_H */

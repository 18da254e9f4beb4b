// Entry points built on the sign evaluation: host-buffer evaluation and the
// search for the chemical potential (Section IV-G, Algorithm 1's outer loop).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "plan.cuh"

namespace submat {

submat_status Plan::sign_host(const double* K, double mu, double* D, cudaStream_t st) {
  if (!d_hostK) SM_TRY(alloc(&d_hostK, size_t(nvals), "host-call K buffer"));
  if (!d_hostD) SM_TRY(alloc(&d_hostD, size_t(nvals), "host-call D buffer"));
  SM_CUDA(cudaMemcpyAsync(d_hostK, K, size_t(nvals) * sizeof(double), cudaMemcpyHostToDevice, st));
  submat_status s = sign(d_hostK, mu, d_hostD, st);
  if (s != SUBMAT_OK && s != SUBMAT_ERR_NOT_CONVERGED) return s;
  SM_CUDA(cudaMemcpyAsync(D, d_hostD, size_t(nvals) * sizeof(double), cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaStreamSynchronize(st));
  return s;
}

// Tr D(mu) is non-decreasing in mu (more levels fall below mu).  At zero
// temperature it is a staircase: flat inside gaps, with jumps where an
// eigenvalue of some submatrix crosses mu.  The search keeps a bracket
// [lo, hi] with N(lo) <= n_el <= N(hi) and bisects it; a Newton step would use
// dN/dmu, which the adjoint gives as exactly 0 at T = 0 for nonsingular
// submatrices (L_sign(a, I) = 0), so bisection is the step that applies.
submat_status Plan::mu_search(const double* K, double n_el, double mu0, double tol, int max_steps,
                              double* mu_out, double* D, cudaStream_t st) {
  auto eval = [&](double mu, double* n) -> submat_status {
    submat_status s = sign(K, mu, D, st);
    if (s != SUBMAT_OK && s != SUBMAT_ERR_NOT_CONVERGED) return s;
    SM_TRY(trace(D, n, st));
    return SUBMAT_OK;
  };
  int steps = 0;
  // every evaluation resets the statistics; the step count is set on return
  auto done = [&](submat_status s) {
    stats.mu_steps = steps;
    return s;
  };
  double n0 = 0;
  SM_TRY(eval(mu0, &n0));
  ++steps;
  double last_mu = mu0;
  if (std::fabs(n0 - n_el) <= tol * std::fabs(n_el)) { *mu_out = mu0; return done(SUBMAT_OK); }
  // spectral bound: every eigenvalue of a_j = K_sub - mu0 I lies in [-beta_j, beta_j]
  double bmax = 0;
  for (double b : res_beta) bmax = std::max(bmax, b);
  const double span = 1.01 * bmax + 1e-12;
  double lo, hi;
  if (n0 < n_el) { lo = mu0; hi = mu0 + span; } else { hi = mu0; lo = mu0 - span; }
  double best_mu = mu0, best_n = n0;
  const double width_floor = 1e-10 * std::max(bmax, 1e-300);
  while (steps < max_steps && (hi - lo) > width_floor) {
    const double mid = 0.5 * (lo + hi);
    double nm = 0;
    SM_TRY(eval(mid, &nm));
    ++steps;
    last_mu = mid;
    if (std::fabs(nm - n_el) < std::fabs(best_n - n_el)) { best_mu = mid; best_n = nm; }
    if (std::fabs(nm - n_el) <= tol * std::fabs(n_el)) { *mu_out = mid; return done(SUBMAT_OK); }
    if (nm < n_el) lo = mid; else hi = mid;
  }
  if (last_mu != best_mu) {
    double nb = 0;
    SM_TRY(eval(best_mu, &nb));
    ++steps;
  }
  *mu_out = best_mu;
  if ((hi - lo) <= width_floor) {
    set_error("Tr D jumps over n_el inside [%.17g, %.17g] (N = %.17g at mu = %.17g)", lo, hi, best_n,
              best_mu);
    return done(SUBMAT_ERR_MU_NO_ROOT);
  }
  set_error("mu search used %d sign evaluations without meeting tol (best N = %.17g)", steps, best_n);
  return done(SUBMAT_ERR_NOT_CONVERGED);
}

}  // namespace submat

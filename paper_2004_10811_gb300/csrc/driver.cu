// Entry points built on the sign evaluation: host-buffer evaluation and the
// search for the chemical potential (Section IV-G, Algorithm 1's outer loop).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>

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
// The bracket is [mu0 - 1.01 b, mu0 + 1.01 b] on the side of n_el, b the
// spectral bound at mu0 (known after the first evaluation).  The last
// evaluation is made at the returned mu, so that its side effects (D) match.
submat_status mu_bisect(const std::function<submat_status(double, double*)>& eval,
                        const std::function<double()>& bound, double n_el, double mu0, double tol,
                        int max_steps, MuSearchOut* out) {
  MuSearchOut& r = *out;
  r = MuSearchOut{};
  double n0 = 0;
  SM_TRY(eval(mu0, &n0));
  ++r.steps;
  double last_mu = mu0;
  r.mu = mu0;
  r.n_best = n0;
  if (std::fabs(n0 - n_el) <= tol * std::fabs(n_el)) return SUBMAT_OK;
  const double bmax = bound();
  const double span = 1.01 * bmax + 1e-12;
  double lo, hi;
  if (n0 < n_el) { lo = mu0; hi = mu0 + span; } else { hi = mu0; lo = mu0 - span; }
  double best_mu = mu0, best_n = n0;
  const double width_floor = 1e-10 * std::max(bmax, 1e-300);
  while (r.steps < max_steps && (hi - lo) > width_floor) {
    const double mid = 0.5 * (lo + hi);
    double nm = 0;
    SM_TRY(eval(mid, &nm));
    ++r.steps;
    last_mu = mid;
    // the latest of the evaluations nearest n_el: at a step of the staircase
    // that is an end of the final bracket
    if (std::fabs(nm - n_el) <= std::fabs(best_n - n_el)) { best_mu = mid; best_n = nm; }
    if (std::fabs(nm - n_el) <= tol * std::fabs(n_el)) {
      r.mu = mid;
      r.n_best = nm;
      r.lo = lo; r.hi = hi;
      return SUBMAT_OK;
    }
    if (nm < n_el) lo = mid; else hi = mid;
  }
  if (last_mu != best_mu) {
    double nb = 0;
    SM_TRY(eval(best_mu, &nb));
    ++r.steps;
  }
  r.mu = best_mu;
  r.n_best = best_n;
  r.lo = lo; r.hi = hi;
  if ((hi - lo) <= width_floor) {
    set_error("Tr D jumps over n_el inside [%.17g, %.17g] (N = %.17g at mu = %.17g)", lo, hi, best_n,
              best_mu);
    return SUBMAT_ERR_MU_NO_ROOT;
  }
  set_error("mu search used %d sign evaluations without meeting tol (best N = %.17g)", r.steps, best_n);
  return SUBMAT_ERR_NOT_CONVERGED;
}

submat_status Plan::mu_search(const double* K, double n_el, double mu0, double tol, int max_steps,
                              double* mu_out, double* D, cudaStream_t st) {
  auto eval = [&](double mu, double* n) -> submat_status {
    submat_status s = sign(K, mu, D, st);
    if (s != SUBMAT_OK && s != SUBMAT_ERR_NOT_CONVERGED) return s;
    SM_TRY(trace(D, n, st));
    return SUBMAT_OK;
  };
  // spectral bound: every eigenvalue of a_j = K_sub - mu0 I lies in [-beta_j, beta_j]
  auto bound = [&]() {
    double bmax = 0;
    for (double b : res_beta) bmax = std::max(bmax, b);
    return bmax;
  };
  MuSearchOut r;
  const submat_status s = mu_bisect(eval, bound, n_el, mu0, tol, max_steps, &r);
  // every evaluation resets the statistics: the step count is set last
  stats.mu_steps = r.steps;
  if (s == SUBMAT_OK || s == SUBMAT_ERR_MU_NO_ROOT || s == SUBMAT_ERR_NOT_CONVERGED) *mu_out = r.mu;
  return s;
}

}  // namespace submat

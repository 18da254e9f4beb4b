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
// The bracket is [mu0, mu0 + 1.01 b] or [mu0 - 1.01 b, mu0] on the side of
// n_el, b = bound() the spectral bound at mu0 (known after the first
// evaluation): with a rigorous bound every eigenvalue of every submatrix lies
// below mu0 + 1.01 b, so N there is the full count.  The far end is evaluated
// only if the bisection closes in on it (the target in the last eighth of the
// bracket); should it not hold n_el (a bound that was too small), the bracket
// moves outward, twice the span each time.  The last evaluation is made at
// the returned mu, so that its side effects (D) match.
submat_status mu_bisect(const std::function<submat_status(double, double*)>& eval,
                        const std::function<double()>& bound, double n_el, double mu0, double tol,
                        int max_steps, MuSearchOut* out, const MuProbe& probe) {
  MuSearchOut& r = *out;
  r = MuSearchOut{};
  // a probe is conclusive when N lies on one side of n_el, outside tol,
  // whatever its error
  bool probing = bool(probe);
  bool last_probe = false;  // the latest evaluation was a probe (D not final)
  auto try_probe = [&](double mu, int* side) -> submat_status {
    *side = 0;
    if (!probing) return SUBMAT_OK;
    double np = 0, b = 0;
    SM_TRY(probe(mu, &np, &b));
    ++r.probes;
    last_probe = true;
    if (std::fabs(np - n_el) > b + tol * std::fabs(n_el)) *side = np < n_el ? -1 : 1;
    else probing = false;  // near n_el: full evaluations from here on
    return SUBMAT_OK;
  };
  double n0 = 0;
  int side0 = 0;
  SM_TRY(try_probe(mu0, &side0));
  double last_mu = mu0;
  if (side0 == 0) {
    SM_TRY(eval(mu0, &n0));
    ++r.steps;
    last_probe = false;
    r.mu = mu0;
    r.n_best = n0;
    if (std::fabs(n0 - n_el) <= tol * std::fabs(n_el)) return SUBMAT_OK;
  } else {
    n0 = side0 < 0 ? -HUGE_VAL : HUGE_VAL;  // only its side is known
    last_mu = HUGE_VAL;
  }
  const double bmax = bound();
  double span = 1.01 * bmax + 1e-12;
  const bool up = n0 < n_el;
  double lo, hi;
  if (up) { lo = mu0; hi = mu0 + span; } else { hi = mu0; lo = mu0 - span; }
  double far = up ? hi : lo;  // not evaluated
  double best_mu = side0 == 0 ? mu0 : HUGE_VAL, best_n = n0;
  double width_floor = 1e-10 * std::max(bmax, 1e-300);
  auto consider = [&](double mu, double nm) {
    last_mu = mu;
    // the latest of the evaluations nearest n_el: at a step of the staircase
    // that is an end of the final bracket
    if (std::fabs(nm - n_el) <= std::fabs(best_n - n_el)) { best_mu = mu; best_n = nm; }
  };
  bool far_ok = false;  // N(far) has been seen on the other side of n_el
  while (r.steps + r.probes < max_steps && (hi - lo) > width_floor) {
    // the bisection has closed in on the unevaluated far end (the last eighth
    // of the bracket): check that it holds n_el, else move the bracket outward
    if (!far_ok && (up ? far - lo : hi - far) <= 0.125 * span) {
      double nf = 0;
      SM_TRY(eval(far, &nf));
      ++r.steps;
      last_probe = false;
      consider(far, nf);
      if (std::fabs(nf - n_el) <= tol * std::fabs(n_el)) {
        r.mu = far;
        r.n_best = nf;
        r.lo = lo; r.hi = hi;
        return SUBMAT_OK;
      }
      if (up ? nf >= n_el : nf <= n_el) {
        far_ok = true;
      } else {
        span *= 2.0;
        width_floor *= 2.0;  // 1e-10 of the grown bound
        if (up) { lo = far; hi = far + span; far = hi; } else { hi = far; lo = far - span; far = lo; }
      }
      continue;
    }
    const double mid = 0.5 * (lo + hi);
    int side = 0;
    SM_TRY(try_probe(mid, &side));
    if (side != 0) {  // the probe decides this step
      ++r.probe_steps;
      if (side < 0) lo = mid; else hi = mid;
      if (up ? hi != far : lo != far) far_ok = true;
      continue;
    }
    double nm = 0;
    SM_TRY(eval(mid, &nm));
    ++r.steps;
    last_probe = false;
    consider(mid, nm);
    if (std::fabs(nm - n_el) <= tol * std::fabs(n_el)) {
      r.mu = mid;
      r.n_best = nm;
      r.lo = lo; r.hi = hi;
      return SUBMAT_OK;
    }
    if (nm < n_el) lo = mid; else hi = mid;
    if (up ? hi != far : lo != far) far_ok = true;  // a mid value on the far side was seen
  }
  if (best_mu == HUGE_VAL || !std::isfinite(best_n)) {  // only probes so far: one full evaluation
    best_mu = 0.5 * (lo + hi);
    SM_TRY(eval(best_mu, &best_n));
    ++r.steps;
    last_probe = false;
    last_mu = best_mu;
  }
  if (last_mu != best_mu || last_probe) {
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

// Finite temperature: N(mu) = Tr f(K - mu I) is smooth and strictly
// increasing, and every evaluation also returns dN/dmu (the adjoint's
// -sum L_f(a_j, I)_cc, from the same build), so the search takes Newton steps
// inside a bracket and bisects when a step would leave it or does not halve
// the error fast enough (the safeguard of rtsafe).  The bracket is
// [mu0, mu0 + s] or [mu0 - s, mu0] on the side of n_el, s = 1.01 b + 40 kT with
// b the rigorous spectral bound at mu0: beyond every eigenvalue by 40 kT the
// Fermi tails are below e^-40.
submat_status Plan::mu_newton(const double* K, double n_el, double mu0, double tol, int max_steps,
                              double* mu_out, double* D, cudaStream_t st) {
  int steps = 0;
  submat_status last = SUBMAT_OK;
  auto eval = [&](double mu, double* n, double* dn) -> submat_status {
    last = sign(K, mu, D, st);
    if (last != SUBMAT_OK) return last;
    SM_TRY(trace(D, n, st));
    *dn = stats.dn_dmu;
    ++steps;
    return SUBMAT_OK;
  };
  auto done = [&](double nv) { return std::fabs(nv - n_el) <= tol * std::fabs(n_el); };
  double mu = mu0, n = 0, dn = 0;
  submat_status s = eval(mu, &n, &dn);
  double best_mu = mu, best_n = n;
  if (s == SUBMAT_OK && !done(n)) {
    double bmax = 0;
    for (int j = col_lo; j < col_hi; ++j) bmax = std::max(bmax, res_bound[j]);
    const double span = 1.01 * bmax + 40.0 * opt.kT;
    double lo = n < n_el ? mu0 : mu0 - span, hi = n < n_el ? mu0 + span : mu0;
    double dx_old = hi - lo, dx = dx_old;
    s = SUBMAT_ERR_NOT_CONVERGED;
    while (steps < max_steps) {
      const double f = n - n_el;
      // Newton from mu, unless it leaves (lo, hi) or the error shrinks too slowly
      const bool out = !((mu - hi) * dn - f < 0.0 && (mu - lo) * dn - f > 0.0);
      if (!(dn > 0.0) || out || std::fabs(2.0 * f) > std::fabs(dx_old * dn)) {
        dx_old = dx;
        dx = 0.5 * (hi - lo);
        mu = lo + dx;
      } else {
        dx_old = dx;
        dx = f / dn;
        mu -= dx;
      }
      SM_TRY(eval(mu, &n, &dn));
      if (std::fabs(n - n_el) <= std::fabs(best_n - n_el)) { best_mu = mu; best_n = n; }
      if (done(n)) { s = SUBMAT_OK; break; }
      if (n < n_el) lo = mu; else hi = mu;
      if (hi - lo <= 1e-15 * std::max(std::fabs(mu), bmax)) break;  // at the rounding floor
    }
    if (s != SUBMAT_OK) {
      if (mu != best_mu) {
        double nb = 0, db = 0;
        SM_TRY(eval(best_mu, &nb, &db));
      }
      mu = best_mu;
      set_error("mu search (finite temperature) used %d evaluations without meeting tol (N = %.17g "
                "at mu = %.17g)", steps, best_n, best_mu);
    }
  }
  stats.mu_steps = steps;
  if (s == SUBMAT_OK || s == SUBMAT_ERR_NOT_CONVERGED) *mu_out = mu;
  return s;
}

submat_status Plan::mu_search(const double* K, double n_el, double mu0, double tol, int max_steps,
                              double* mu_out, double* D, cudaStream_t st) {
  double n_total = 0.0;
  for (int j = 0; j < nblk; ++j) n_total += bs[j];
  if (n_el < 0.0 || n_el > n_total) {
    set_error("n_el = %.17g outside [0, %.17g] (the matrix dimension)", n_el, n_total);
    return SUBMAT_ERR_INVALID_ARG;
  }
  if (opt.kT > 0.0) return mu_newton(K, n_el, mu0, tol, max_steps, mu_out, D, st);
  // status of the latest evaluation: a submatrix that did not converge there
  // leaves D (and the trace) unfinished; one that diverged ends the search
  submat_status last = SUBMAT_OK;
  auto eval = [&](double mu, double* n) -> submat_status {
    last = sign(K, mu, D, st);
    if (last != SUBMAT_OK && last != SUBMAT_ERR_NOT_CONVERGED) return last;
    if (last == SUBMAT_ERR_NOT_CONVERGED && (last_flags & FLAG_DIVERGED)) {
      set_error("mu search: a submatrix diverged at mu = %.17g", mu);
      return SUBMAT_ERR_NOT_CONVERGED;
    }
    SM_TRY(trace(D, n, st));
    return SUBMAT_OK;
  };
  // rigorous spectral bound at mu0: every eigenvalue of a_j = K_sub - mu0 I
  // lies in [-b_j, b_j], b_j = min(max row abs-sum, ||a_j||_F)
  auto bound = [&]() {
    double bmax = 0;
    for (int j = col_lo; j < col_hi; ++j) bmax = std::max(bmax, res_bound[j]);
    return bmax;
  };
  // Mixed plans probe first: the FP16x3 iterate without correction or FP64
  // fallback (a fraction of a build, and none of the slow fallbacks that
  // evaluations inside a band need).  Its trace error is bounded per block
  // column c of submatrix q: with X the final iterate, S = sign(a) and
  // e_l = x_l^2 - 1 in the eigenbasis, |(X - S)_cc| <= sum_l Q_cl^2 |e_l|
  // <= ||X^2 - I||_F = r_q sqrt(n_q) (Newton-Schulz keeps signs and stays in
  // [-1, 1]), plus 1e-3 for the FP16x3 rounding; N = sum_c (1 - S_cc) / 2.
  MuProbe probe;
  if (opt.prec == SUBMAT_MIXED_BF16_REFINE)
    probe = [&](double mu, double* n, double* bnd) -> submat_status {
      probe_mode = true;
      const submat_status ps = sign(K, mu, D, st);
      probe_mode = false;
      if (ps != SUBMAT_OK && ps != SUBMAT_ERR_NOT_CONVERGED) return ps;
      SM_TRY(trace(D, n, st));
      double b = 0.0;
      for (int q = col_lo; q < col_hi; ++q)
        b += 0.5 * qext[q] * (res_resid[q] * std::sqrt(double(qn[q])) + 1e-3);
      *bnd = (last_flags & FLAG_DIVERGED) ? HUGE_VAL : b;
      return SUBMAT_OK;
    };
  MuSearchOut r;
  submat_status s = mu_bisect(eval, bound, n_el, mu0, tol, max_steps, &r, probe);
  // every evaluation resets the statistics: the step counts are set last
  stats.mu_steps = r.steps;
  stats.mu_probes = r.probes;
  if (s == SUBMAT_OK || s == SUBMAT_ERR_MU_NO_ROOT || s == SUBMAT_ERR_NOT_CONVERGED) *mu_out = r.mu;
  if ((s == SUBMAT_OK || s == SUBMAT_ERR_MU_NO_ROOT) && last == SUBMAT_ERR_NOT_CONVERGED) {
    set_error("mu search ended at mu = %.17g, where %d submatrices did not converge (D written)", r.mu,
              stats.not_converged);
    s = SUBMAT_ERR_NOT_CONVERGED;
  }
  return s;
}

}  // namespace submat

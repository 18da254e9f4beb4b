// Finite temperature: D = f(K - mu I) with the Fermi function
// f(x) = 1 / (1 + exp(x / kT)) in place of (1 - signum(x)) / 2 (Section IV-F,
// last paragraph: the eigendecomposition route extends to finite temperature
// by replacing signum; the Conclusion names the generalisation).
//
// f(x) = (1 - tanh(x / (2 kT))) / 2, so every submatrix needs tanh of its
// scaled matrix X = a / sigma, whose spectrum lies in [-1, 1].  tanh(c x),
// c = sigma / (2 kT), is analytic in the strip |Im x| < pi / (2c), so its
// Chebyshev series on [-1, 1] converges geometrically; the series is cut at
// the odd degree m whose tail sum_{k > m} |c_k| (a bound on the truncation
// error, |T_k| <= 1 on [-1, 1]) is below the precision's tolerance.
//
// Evaluation, baby steps and giant steps (all polynomials in X commute and are
// symmetric, so every product is a symmetric one):
//   baby:  T_2 = 2 X^2 - I, T_{k+2} = 2 T_2 T_k - T_{k-2} for the odd
//          k = 1..15 (eight stored), Y = T_16 = 2 T_9 T_7 - T_2;
//   fold:  with k = 16 j + i, T_{16j+i} = 2 T_{16j} T_i - T_{16j-i}, so the
//          series becomes sum_j R_j T_{16j} with R_j a combination of the
//          stored odd T_i, and T_{16j}(X) = T_j(Y);
//   giant: Clenshaw in Y: b_j = R_j + 2 Y b_{j+1} - b_{j+2}, p = R_0 + Y b_1 - b_2.
// That is 9 + ceil((m + 1) / 16) - 1 products for degree m.
//
// The scale sigma is common to a wave (one polynomial per wave): each
// submatrix starts at X = a / beta_bound (beta_bound = min(max row abs-sum,
// ||a||_F)), the first square gives the rigorous bound
// rho(X)^2 <= ||X^2||_inf (rounding included), and sigma is the largest
// beta_bound * sqrt(||X^2||_inf) of the wave, which roughly halves the degree
// against beta_bound alone.
//
// dN/dmu = sum_j sum_{c in block j} [f'(a_j)]_cc with f' = f (1 - f) / kT as a
// matrix function (d/dmu f(a - mu I) = -f'(a - mu I)), i.e. the adjoint's
// L_f(a_j, I): from the extracted columns of F_j = f(a_j) as
// sum_c (F_cc - sum_k F_kc^2) / kT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "plan.cuh"

namespace submat {

// ---------------------------------------------------------------------------
// host: the Chebyshev series of tanh(c x) and its baby-step / giant-step form
// ---------------------------------------------------------------------------

// Coefficients c_k, k < ncoef, of tanh(c x) on [-1, 1] from its values at the
// N Chebyshev nodes x_n = cos(theta_n), theta_n = pi (2n + 1) / (2N) (the
// discrete cosine transform of the first kind; exact for degree < N).
// cos(k theta_n) = cos(pi j / (2N)) with j = k (2n + 1) mod 4N, read from a
// table, so no rounding accumulates with k.
static void cheb_coefficients(double c, int N, int ncoef, std::vector<double>* out) {
  const int64_t P = 4 * int64_t(N);
  std::vector<double> cosv(static_cast<size_t>(P)), g(static_cast<size_t>(N));
  for (int64_t j = 0; j < P; ++j) cosv[size_t(j)] = std::cos(M_PI * double(j) / (2.0 * N));
  for (int n = 0; n < N; ++n) g[n] = std::tanh(c * cosv[size_t(2 * n + 1)]);
  out->assign(ncoef, 0.0);
  for (int k = 0; k < ncoef; ++k) {
    double acc = 0.0;
    int64_t j = k, step = 2 * int64_t(k) % P;  // j = k (2n + 1) mod 4N
    for (int n = 0; n < N; ++n) {
      acc += g[n] * cosv[size_t(j)];
      j += step;
      if (j >= P) j -= P;
    }
    (*out)[k] = (k == 0 ? 1.0 : 2.0) * acc / N;
  }
}

submat_status fermi_poly(double c, double tol, int max_degree, FermiPoly* out) {
  if (!(c > 0.0) || !std::isfinite(c)) {
    set_error("finite temperature: bad scale c = %g", c);
    return SUBMAT_ERR_INVALID_ARG;
  }
  FermiPoly& P = *out;
  P = FermiPoly{};
  std::vector<double> coef;
  int m = -1;
  double tail = 0.0;
  for (int N = 256;; N *= 2) {
    const int ncoef = N / 2;
    cheb_coefficients(c, N, ncoef, &coef);
    // coefficients below the rounding floor of the transform are noise, not
    // truncation: the series counts up to the last one above it
    double cmax = 0.0;
    for (double v : coef) cmax = std::max(cmax, std::fabs(v));
    const double floor = 64.0 * 0x1p-52 * cmax;
    int last = 0;
    for (int k = 0; k < ncoef; ++k)
      if (std::fabs(coef[k]) > floor) last = k;
    // the series must reach the floor inside the first half of the computed range
    if (last > ncoef / 2) {
      if (N / 4 > max_degree + 1) break;  // would need a degree beyond the cap
      continue;
    }
    // smallest odd m with sum_{m < k <= last} |c_k| <= tol
    std::vector<double> suffix(ncoef + 1, 0.0);
    for (int k = last; k >= 0; --k) suffix[k] = suffix[k + 1] + std::fabs(coef[k]);
    for (int k = 1; k < ncoef; k += 2)
      if (suffix[k + 1] <= tol) { m = k; tail = suffix[k + 1]; break; }
    break;
  }
  if (m < 0 || m > max_degree) {
    set_error("finite temperature: tanh(%g x) needs a Chebyshev degree above %d (kT too small for the "
              "spectral scale)", c, max_degree);
    return SUBMAT_ERR_UNSUPPORTED;
  }
  P.m = m;
  P.trunc = tail;
  constexpr int S = kFermiBaby;
  P.blocks = (m + 1 + S - 1) / S;
  std::vector<double> a(size_t(P.blocks) * S, 0.0);
  for (int k = 1; k <= m; k += 2) a[k] = coef[k];  // tanh is odd: even terms vanish
  P.r.assign(size_t(P.blocks) * (S / 2), 0.0);
  for (int j = P.blocks - 1; j >= 1; --j)
    for (int i = 1; i < S; i += 2) {
      const double ck = a[size_t(S) * j + i];
      P.r[size_t(j) * (S / 2) + i / 2] = 2.0 * ck;
      a[size_t(S) * (j - 1) + (S - i)] -= ck;
    }
  for (int i = 1; i < S; i += 2) P.r[i / 2] = a[i];
  return SUBMAT_OK;
}

namespace {

// X <- r_s X and T2 <- r_s^2 (T2 + I) - I (the square rescaled), r_s = ratio[s]
template <typename T>
__global__ void k_fermi_rescale(WaveDev w, T* __restrict__ X, T* __restrict__ T2, const double* __restrict__ ratio) {
  const int s = blockIdx.y;
  const double r = ratio[s];
  if (r == 1.0) return;
  const int ld = w.ld[s], n = w.n[s];
  const int64_t total = int64_t(ld) * ld, base = w.off[s];
  const T rt = T(r), r2 = T(r * r), dshift = T(r * r - 1.0);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int row = int(e / ld), col = int(e - int64_t(row) * ld);
    X[base + e] *= rt;
    if (!T2) continue;
    T v = r2 * T2[base + e];
    if (row == col && row < n) v += dshift;
    T2[base + e] = v;
  }
}

// M <- r_s^2 M (the derivative part of the rescaled square)
template <typename T>
__global__ void k_fermi_scale_sq(WaveDev w, T* __restrict__ M, const double* __restrict__ ratio) {
  const int s = blockIdx.y;
  const double r = ratio[s];
  if (r == 1.0) return;
  const int ld = w.ld[s];
  const int64_t total = int64_t(ld) * ld, base = w.off[s];
  const T r2 = T(r * r);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x)
    M[base + e] *= r2;
}

// W = sum_i r_i T_{2i+1} - B (B may be null): the giant-step coefficient R_j
// less the Clenshaw term b_{j+2}.  W may be B (each entry is read, then
// written by the same thread).
struct CombArgs {
  double r[kFermiBaby / 2];
};

template <typename T>
__global__ void __launch_bounds__(256) k_cheb_comb(WaveDev w, const T* __restrict__ odd, int64_t stride,
                                                   CombArgs ca, const T* B, T* W) {
  const int s = blockIdx.y;
  const int ld = w.ld[s];
  const int64_t total = int64_t(ld) * ld, base = w.off[s];
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = base + e;
    T acc = B ? -B[i] : T(0);
#pragma unroll
    for (int q = 0; q < kFermiBaby / 2; ++q) acc = fma(T(ca.r[q]), odd[int64_t(q) * stride + i], acc);
    W[i] = acc;
  }
}

dim3 fermi_grid(const Wave& wv) {
  int64_t bx = (wv.max_ld2 + 256 * 8 - 1) / (256 * 8);
  bx = std::max<int64_t>(1, std::min<int64_t>(bx, 512));
  return dim3(unsigned(bx), unsigned(wv.count));
}

template <typename T> struct FermiGemm;
template <> struct FermiGemm<double> {
  using Args = GemmF64Args;
  static cudaError_t run(const Args& a, cudaStream_t st) { return launch_gemm_f64(a, st); }
  static cudaError_t scale(const WaveDev& w, const double* A, double* X, const double* b, int64_t m2,
                           cudaStream_t st) { return launch_scale_f64(w, A, X, b, m2, st); }
};
template <> struct FermiGemm<float> {
  using Args = GemmF32Args;
  static cudaError_t run(const Args& a, cudaStream_t st) { return launch_gemm_f32(a, st); }
  static cudaError_t scale(const WaveDev& w, const double* A, float* X, const double* b, int64_t m2,
                           cudaStream_t st) { return launch_scale_f32(w, A, X, b, m2, st); }
};

}  // namespace

size_t fermi_bytes_per_elem(int prec) {
  // A (FP64) + the eight odd T_k, T_2 / Y, and two Clenshaw buffers
  return 8 + size_t(kFermiBuffers) * (prec == SUBMAT_FP64 ? 8 : 4);
}

// The adjoint runs the same buffers twice: values and derivative parts.
size_t fermi_dual_bytes_per_elem(int prec) {
  return 8 + size_t(2 * kFermiBuffers) * (prec == SUBMAT_FP64 ? 8 : 4);
}

// One wave.  Forward: D = (I - p(X)) / 2 on the extracted columns, with the
// trace and sum-of-squares partials for dN/dmu.  With Dbar (the adjoint):
// every matrix M of the evaluation carries a derivative part M' (dual
// numbers), (A B)' = A' B + A B', seeded with X' = G_j / sigma, G_j holding
// Dbar's block column j in the columns of block j; then p' = L_p(X, X') and
// L_f(a_j, G_j) = -1/2 p' is added into every stored block of Kbar that a_j
// came from (L_f(a, .) is self-adjoint in the Frobenius product for
// symmetric a).  The value part is evaluated exactly as in the forward path.
template <typename T>
submat_status Plan::fermi_wave(Wave& wv, const double* K, double mu, double* D, const double* Dbar, double* Kbar,
                               void* w, int64_t E, cudaStream_t st) {
  using G = FermiGemm<T>;
  using Args = typename G::Args;
  constexpr int S = kFermiBaby;
  const bool dual = Dbar != nullptr;
  double* A = static_cast<double*>(w);
  T* base = reinterpret_cast<T*>(A + E);
  T* odd = base;                  // T_1 = X, T_3, ..., T_15 at odd + q E
  T* T2 = base + (S / 2) * E;     // T_2, later Y = T_16
  T* bb[2] = {T2 + E, T2 + 2 * E};    // Clenshaw b_{j+1}, b_{j+2}
  // derivative parts, the same layout kFermiBuffers buffers further on
  const int64_t dofs = int64_t(kFermiBuffers) * E;
  auto dp = [&](const T* v) -> T* { return v ? const_cast<T*>(v) + dofs : nullptr; };
  const bool f64 = sizeof(T) == 8;
  // truncation tolerance of the series: below the products' own rounding
  const double tol_poly = f64 ? 1e-13 : 1e-8;
  SM_CUDA(cudaEventRecord(ev[0], st));
  SM_TRY(gather_wave(wv, K, mu, A, st));
  SM_CUDA(G::scale(wv.dev, A, odd, ns.beta, wv.max_ld2, st));
  if (dual) SM_CUDA(launch_bwd_seed<T>(g, wv, Dbar, ns.beta, dp(odd), 0, st));  // X' = G / beta
  SM_CUDA(cudaEventRecord(ev[1], st));
  int products = 0;
  auto gemm1 = [&](const Args& a) -> submat_status {
    size_t tk;
    SM_TRY(timer.start(KC_SIMT, st, &tk));
    SM_CUDA(G::run(a, st));
    SM_TRY(timer.stop(tk, st));
    return SUBMAT_OK;
  };
  // C = alpha A B + beta C0 + diag I (symmetric: A, B commute), and with
  // dual numbers C' = alpha (A' B + A B') + beta C0' (full tiles)
  auto gemm = [&](const T* Aop, const T* Bop, const T* C0, T* C, double alpha, double beta,
                  double diag) -> submat_status {
    Args a{};
    a.w = wv.dev; a.items = wv.sym64; a.nitems = wv.n_sym64;
    a.A = Aop; a.B = Bop; a.C0 = C0; a.C = C;
    a.alpha = alpha; a.beta = beta; a.diag = diag; a.sym = 1;
    a.res2 = nullptr; a.state = nullptr; a.skip_state = -1;
    if (dual) {  // derivative first: it reads the values of A, B (and C0 may alias C)
      Args d = a;
      d.items = wv.full64; d.nitems = wv.n_full64; d.sym = 0; d.diag = 0.0;
      d.A = dp(Aop); d.B = Bop; d.C0 = dp(C0); d.C = dp(C);
      SM_TRY(gemm1(d));
      d.A = Aop; d.B = dp(Bop); d.C0 = dp(C); d.beta = 1.0;
      SM_TRY(gemm1(d));
    }
    SM_TRY(gemm1(a));
    ++products;
    return SUBMAT_OK;
  };
  // T_2 = 2 X^2 - I at X = a / beta_bound, and from it the tight scale
  SM_TRY(gemm(odd, odd, nullptr, T2, 2.0, 0.0, -1.0));
  const CertSquare sq{f64 ? 0 : 1, T2, nullptr, 2.0f, -1.0f};
  SM_CUDA(cudaMemsetAsync(ns.cert, 0, sizeof(unsigned long long) * wv.count, st));
  SM_CUDA(launch_cert_rowsum(wv.dev, ns, sq, max_ld(wv), st));
  std::vector<unsigned long long> cert(wv.count), gersh(wv.count);
  std::vector<double> fro2(wv.count), beta(wv.count), ratio(wv.count, 1.0);
  SM_CUDA(cudaMemcpyAsync(cert.data(), ns.cert, 8 * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(gersh.data(), ns.gersh, 8 * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(fro2.data(), ns.fro2, 8 * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(beta.data(), ns.beta, 8 * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaStreamSynchronize(st));
  double sigma = 0.0;
  std::vector<double> bound(wv.count, 0.0);
  const double eps0 = f64 ? 0x1p-50 : 0x1p-22, eps_ld = f64 ? 0x1p-52 : 0x1p-23;
  for (int s = 0; s < wv.count; ++s) {
    double cv = 0.0, gv = 0.0;
    std::memcpy(&cv, &cert[s], 8);
    std::memcpy(&gv, &gersh[s], 8);
    const double bnd = std::min(gv, std::sqrt(fro2[s])) * (1.0 + 1e-4);
    if (!(bnd > 0.0)) continue;  // a zero submatrix: f(0) = 1/2 whatever the scale
    const int ld = wv.host_ld[s];
    const double gx = gv / bnd;
    const double Gs = cv * (1.0 + ld * 0x1p-24) + (eps0 + eps_ld * ld) * gx * gx;
    bound[s] = beta[s] * std::min(1.0, std::sqrt(Gs));
    sigma = std::max(sigma, bound[s]);
  }
  sigma *= 1.0 + 1e-6;
  if (!(sigma > 0.0)) sigma = 1.0;
  for (int s = 0; s < wv.count; ++s)
    if (bound[s] > 0.0) ratio[s] = beta[s] / sigma;
  SM_CUDA(cudaMemcpyAsync(ns.cscale, ratio.data(), 8 * wv.count, cudaMemcpyHostToDevice, st));
  k_fermi_rescale<T><<<fermi_grid(wv), 256, 0, st>>>(wv.dev, odd, T2, ns.cscale);
  SM_KCHECK();
  if (dual) {  // X' and T_2' = 2 (X' X + X X') follow the scale linearly / quadratically
    k_fermi_rescale<T><<<fermi_grid(wv), 256, 0, st>>>(wv.dev, dp(odd), nullptr, ns.cscale);
    SM_KCHECK();
    k_fermi_scale_sq<T><<<fermi_grid(wv), 256, 0, st>>>(wv.dev, dp(T2), ns.cscale);
    SM_KCHECK();
  }
  FermiPoly P;
  SM_TRY(fermi_poly(sigma / (2.0 * opt.kT), tol_poly, kFermiMaxDegree, &P));
  fermi_degree = std::max(fermi_degree, P.m);
  fermi_trunc = std::max(fermi_trunc, P.trunc);
  // baby steps: T_3 = 2 T_2 X - X, T_{k+2} = 2 T_2 T_k - T_{k-2}
  for (int q = 1; q < S / 2; ++q)
    SM_TRY(gemm(T2, odd + int64_t(q - 1) * E, q >= 2 ? odd + int64_t(q - 2) * E : odd, odd + int64_t(q) * E,
                2.0, -1.0, 0.0));
  // Y = T_16 = 2 T_9 T_7 - T_2, in T_2's buffer
  SM_TRY(gemm(odd + 4 * E, odd + 3 * E, T2, T2, 2.0, -1.0, 0.0));
  const T* Y = T2;
  // giant steps: Clenshaw in Y with the coefficients R_j
  auto comb = [&](int j, const T* B, T* W) -> submat_status {
    CombArgs ca;
    for (int q = 0; q < S / 2; ++q) ca.r[q] = P.r[size_t(j) * (S / 2) + q];
    k_cheb_comb<T><<<fermi_grid(wv), 256, 0, st>>>(wv.dev, odd, E, ca, B, W);
    SM_KCHECK();
    if (dual) {
      k_cheb_comb<T><<<fermi_grid(wv), 256, 0, st>>>(wv.dev, dp(odd), E, ca, dp(B), dp(W));
      SM_KCHECK();
    }
    return SUBMAT_OK;
  };
  T* out = nullptr;
  if (P.blocks == 1) {
    SM_TRY(comb(0, nullptr, bb[0]));
    out = bb[0];
  } else {
    T* b1 = bb[0];     // b_{j+1}
    T* b2 = nullptr;   // b_{j+2} (b_G = 0 at the start)
    SM_TRY(comb(P.blocks - 1, nullptr, b1));
    for (int j = P.blocks - 2; j >= 0; --j) {
      // W = R_j - b_{j+2} (in place over b_{j+2}), then W += c Y b_{j+1}
      T* W = b2 ? b2 : bb[1];
      SM_TRY(comb(j, b2, W));
      SM_TRY(gemm(Y, b1, W, W, j == 0 ? 1.0 : 2.0, 1.0, 0.0));
      if (j == 0) { out = W; break; }
      b2 = b1;
      b1 = W;
    }
  }
  SM_CUDA(cudaEventRecord(ev[2], st));
  // D = (I - p(X)) / 2 on the extracted columns, Tr and sum of squares
  SM_TRY(scatter_timed(wv, f64 ? 16.0 : 12.0, [&] {
    return launch_scatter_sq<T>(g, wv.dev, ns, out, D, d_trpart, d_sqpart, geom(wv), st);
  }, st));
  if (dual) SM_CUDA(launch_bwd_scatter_add<T>(g, wv, nb_max, dp(out), Kbar, st));
  SM_CUDA(cudaEventRecord(ev[3], st));
  SM_TRY(collect_wave(wv, st));
  SM_TRY(add_phase_times());
  for (int s = 0; s < wv.count; ++s) {
    res_iters[wv.first + s] = products;  // products of the evaluation, for the statistics
    const double n = wv.host_n[s];
    fermi_flops += 2.0 * n * n * n * products * (dual ? 3.0 : 1.0);
  }
  return SUBMAT_OK;
}

template <typename T>
submat_status Plan::sign_fermi(const double* K, double mu, double* D, cudaStream_t st) {
  for (auto& wv : waves) SM_TRY(fermi_wave<T>(wv, K, mu, D, nullptr, nullptr, ws, ws_elems, st));
  return SUBMAT_OK;
}

template submat_status Plan::sign_fermi<double>(const double*, double, double*, cudaStream_t);
template submat_status Plan::sign_fermi<float>(const double*, double, double*, cudaStream_t);

// dN/dmu of the last finite-temperature evaluation: sum over the evaluated
// block columns of (Tr_j - sum of squares_j) / kT, in fixed order.
submat_status Plan::fermi_dn_dmu(cudaStream_t st, double* out) {
  std::vector<double> tr(nblk), sq(nblk);
  SM_CUDA(cudaMemcpyAsync(tr.data(), d_trpart, 8 * size_t(nblk), cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(sq.data(), d_sqpart, 8 * size_t(nblk), cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaStreamSynchronize(st));
  double acc = 0.0;
  // block columns evaluated: all of them for grouped plans (col_lo / col_hi
  // count submatrices there), else the column range
  const int j0 = grouped ? 0 : col_lo, j1 = grouped ? nblk : col_hi;
  for (int j = j0; j < j1; ++j) acc += tr[j] - sq[j];
  *out = acc / opt.kT;
  return SUBMAT_OK;
}

// The adjoint at finite temperature (vector-Jacobian product of K -> D):
// fermi_wave on dual numbers, on the adjoint's own waves and workspace.
// dN/dmu = sum_j sum_{c in block j} [f'(a_j)]_cc comes from the value part
// of the same pass (f' = f (1 - f) / kT is a function of a_j itself).
submat_status Plan::backward_fermi(const double* K, double mu, const double* Dbar, double* Kbar,
                                   double* dN_dmu, cudaStream_t st) {
  reset_stats();
  fermi_degree = 0;
  fermi_trunc = fermi_flops = 0.0;
  SM_CUDA(cudaMemsetAsync(d_flags, 0, 4 * sizeof(int), st));
  SM_CUDA(launch_check_finite(Dbar, nvals, d_flags, st));
  int fl = 0;
  SM_TRY(read_flags(st, &fl));
  if (fl & FLAG_NONFINITE) {
    set_error("Dbar holds a NaN or Inf value");
    return SUBMAT_ERR_NONFINITE;
  }
  const size_t bpe = fermi_dual_bytes_per_elem(opt.prec);
  if (bwaves.empty()) {
    size_t fre = 0, tot = 0;
    SM_CUDA(cudaMemGetInfo(&fre, &tot));
    size_t cap = opt.workspace_cap_bytes ? opt.workspace_cap_bytes : size_t(double(fre) * 0.8);
    SM_TRY(build_waves(bpe, cap, bwaves, st));
    int64_t mx = 0;
    for (auto& wv : bwaves) {
      mx = std::max(mx, wv.elems);
      max_bwave = std::max(max_bwave, wv.count);
    }
    SM_TRY(grow_ns_state(max_bwave));
    bws_elems = mx;
    SM_TRY(dev_alloc(&bws, size_t(mx) * bpe, "adjoint workspace"));
    owned.push_back(bws);
  }
  SM_CUDA(cudaMemsetAsync(Kbar, 0, sizeof(double) * size_t(nvals), st));
  for (auto& wv : bwaves) {
    if (opt.prec == SUBMAT_FP64) SM_TRY(fermi_wave<double>(wv, K, mu, nullptr, Dbar, Kbar, bws, bws_elems, st));
    else SM_TRY(fermi_wave<float>(wv, K, mu, nullptr, Dbar, Kbar, bws, bws_elems, st));
  }
  SM_CUDA(cudaStreamSynchronize(st));
  finish_stats(true);
  stats.flops_ns = fermi_flops;
  stats.poly_degree = fermi_degree;
  stats.poly_trunc = fermi_trunc;
  SM_TRY(fermi_dn_dmu(st, &stats.dn_dmu));
  if (dN_dmu) *dN_dmu = stats.dn_dmu;
  SM_TRY(read_flags(st, &fl));
  if (fl & FLAG_NONFINITE) {
    set_error("K holds a NaN or Inf value");
    return SUBMAT_ERR_NONFINITE;
  }
  return SUBMAT_OK;
}

}  // namespace submat

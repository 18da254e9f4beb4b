// Adjoint of the submatrix density map K -> D (vector-Jacobian product).
//
// D's block column j is 1/2 (I - sign(a_j)) restricted to the columns of
// block j, a_j = K[N(j), N(j)] - mu I (Section III-A, Eq. DsignSym with S = I).
// For an upstream gradient Dbar, block column j contributes
//     abar_j = -1/2 L_sign(a_j, G_j),
// G_j = n_j x n_j, zero except its columns of block j, which hold Dbar's
// block column j.  For symmetric a_j the Frechet derivative L_sign(a_j, .) is
// self-adjoint in the Frobenius product, so no transpose is needed.  It is
// evaluated by Newton-Schulz on the block upper-triangular matrix
// [[X, E], [0, X]] (sign of it is [[S, L], [0, S]]):
//     X <- 1/2 X (3I - X^2)
//     E <- 1/2 [E (3I - X^2) - X (X E + E X)]
// with X_0 = a_j / beta, E_0 = G_j / beta; the iterates are recomputed here,
// not stored by the forward pass.  abar_j is added into every stored block of
// K that a_j was assembled from (atomics: blocks are shared by submatrices).
// dN/dmu = 1/2 sum_j sum_{c in block j} L_sign(a_j, I)_cc comes from a second
// pass with E_0 = I / beta.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "plan.cuh"

namespace submat {

namespace {

// E_0 = G_j / beta: block column j of Dbar placed in the columns of block j;
// or (identity != 0) E_0 = I_n / beta.  One CTA per (s, local block row t).
template <typename T>
__global__ void k_bwd_seed(PatternDev g, WaveDev w, const int2* items, const double* __restrict__ Dbar,
                           const double* __restrict__ beta, T* __restrict__ E, int identity) {
  const int2 it = items[blockIdx.x];
  const int s = it.x, t = it.y;
  const int j = w.sub[s];
  const int64_t rp0 = g.row_ptr[j];
  const int nb = int(g.row_ptr[j + 1] - rp0);
  const int ld = w.ld[s], n = w.n[s];
  const int i1 = g.col[rp0 + t];
  const int r0 = g.locoff[rp0 + t];
  const int br = g.bs[i1];
  const int koff = g.koff[j], bj = g.bs[j];
  const double ib = 1.0 / beta[s];
  T* Es = E + w.off[s];
  const int rows = br + ((t == nb - 1) ? (ld - n) : 0);
  const int64_t p = g.tpos[rp0 + t];  // block (i1, j) of Dbar
  for (int rr = threadIdx.y; rr < rows; rr += blockDim.y) {
    const int row = rr < br ? r0 + rr : n + (rr - br);
    for (int c = threadIdx.x; c < ld; c += blockDim.x) {
      double v = 0.0;
      if (rr < br) {
        if (identity) v = (row == c) ? ib : 0.0;
        else if (c >= koff && c < koff + bj) v = Dbar[g.valptr[p] + int64_t(rr) * bj + (c - koff)] * ib;
      }
      Es[int64_t(row) * ld + c] = T(v);
    }
  }
}

// Kbar_p += -1/2 E[u-block rows, v-block cols] for every stored block p =
// (N(j)[u], N(j)[v]); one CTA per (s, local block row u).
template <typename T>
__global__ void k_bwd_scatter_add(PatternDev g, WaveDev w, const int2* items, const T* __restrict__ E,
                                  double* __restrict__ Kbar) {
  extern __shared__ int sm[];
  const int2 it = items[blockIdx.x];
  const int s = it.x, t = it.y;
  const int j = w.sub[s];
  const int64_t rp0 = g.row_ptr[j];
  const int nb = int(g.row_ptr[j + 1] - rp0);
  int* nbr = sm;
  int* blk = sm + nb;
  int* loc = sm + 2 * nb;
  for (int u = threadIdx.x; u < nb; u += blockDim.x) {
    nbr[u] = g.col[rp0 + u];
    blk[u] = -1;
    loc[u] = g.locoff[rp0 + u];
  }
  __syncthreads();
  const int i1 = nbr[t];
  for (int64_t q = g.row_ptr[i1] + threadIdx.x; q < g.row_ptr[i1 + 1]; q += blockDim.x) {
    const int c = g.col[q];
    int lo = 0, hi = nb - 1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      if (nbr[mid] == c) { blk[mid] = int(q); break; }
      if (nbr[mid] < c) lo = mid + 1; else hi = mid - 1;
    }
  }
  __syncthreads();
  const int ld = w.ld[s];
  const T* Es = E + w.off[s];
  const int br = g.bs[i1];
  const int r0 = loc[t];
  for (int v = 0; v < nb; ++v) {
    const int q = blk[v];
    if (q < 0) continue;
    const int bc = g.bs[nbr[v]];
    const int c0 = loc[v];
    double* dst = Kbar + g.valptr[q];
    for (int e = threadIdx.x; e < br * bc; e += blockDim.x) {
      const int rr = e / bc, cc = e - (e / bc) * bc;
      atomicAdd(dst + e, -0.5 * double(Es[int64_t(r0 + rr) * ld + c0 + cc]));
    }
  }
}

// per submatrix: 1/2 sum over the diagonal entries of block j of L
template <typename T>
__global__ void k_bwd_dn(PatternDev g, WaveDev w, const T* __restrict__ E, double* part) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= w.nsub) return;
  const int j = w.sub[s];
  const int ld = w.ld[s];
  const int koff = g.koff[j], bj = g.bs[j];
  const T* Es = E + w.off[s];
  double acc = 0.0;
  for (int c = 0; c < bj; ++c) acc += double(Es[int64_t(koff + c) * ld + koff + c]);
  part[s] = 0.5 * acc;
}

template <typename T>
struct GemmFor;
template <>
struct GemmFor<double> {
  using Args = GemmF64Args;
  static cudaError_t run(const Args& a, cudaStream_t st) { return launch_gemm_f64(a, st); }
};
template <>
struct GemmFor<float> {
  using Args = GemmF32Args;
  static cudaError_t run(const Args& a, cudaStream_t st) { return launch_gemm_f32(a, st); }
};

}  // namespace

template <typename T>
cudaError_t launch_bwd_seed(const PatternDev& g, const Wave& wv, const double* Dbar, const double* beta, T* E,
                            int identity, cudaStream_t st) {
  k_bwd_seed<T><<<wv.n_gather, dim3(32, 8), 0, st>>>(g, wv.dev, wv.gather_items, Dbar, beta, E, identity);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_bwd_seed<double>(const PatternDev&, const Wave&, const double*, const double*,
                                             double*, int, cudaStream_t);
template cudaError_t launch_bwd_seed<float>(const PatternDev&, const Wave&, const double*, const double*,
                                            float*, int, cudaStream_t);

template <typename T>
cudaError_t launch_bwd_scatter_add(const PatternDev& g, const Wave& wv, int nb_max, const T* E, double* Kbar,
                                   cudaStream_t st) {
  const size_t smem = size_t(3 * nb_max + 1) * sizeof(int);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_bwd_scatter_add<T>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k_bwd_scatter_add<T><<<wv.n_gather, 256, smem, st>>>(g, wv.dev, wv.gather_items, E, Kbar);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_bwd_scatter_add<double>(const PatternDev&, const Wave&, int, const double*, double*,
                                                    cudaStream_t);
template cudaError_t launch_bwd_scatter_add<float>(const PatternDev&, const Wave&, int, const float*, double*,
                                                   cudaStream_t);

cudaError_t launch_bwd_seed_f32(const PatternDev& g, const Wave& wv, const double* Dbar, const double* beta,
                                float* E, int identity, cudaStream_t st) {
  return launch_bwd_seed<float>(g, wv, Dbar, beta, E, identity, st);
}

cudaError_t launch_bwd_scatter_add_f32(const PatternDev& g, const Wave& wv, int nb_max, const float* E,
                                       double* Kbar, cudaStream_t st) {
  return launch_bwd_scatter_add<float>(g, wv, nb_max, E, Kbar, st);
}

cudaError_t launch_bwd_dn_f32(const PatternDev& g, const Wave& wv, const float* E, double* part,
                              cudaStream_t st) {
  k_bwd_dn<float><<<(wv.count + 255) / 256, 256, 0, st>>>(g, wv.dev, E, part);
  count_launch();
  return cudaGetLastError();
}

size_t backward_bytes_per_elem(int prec, int adjoint_mode) {
  if (adjoint_mode == 1) return adjoint_tc_bytes_per_elem();
  return prec == SUBMAT_FP64 ? 8 * 7 : 8 + 4 * 6;
}

template <typename T>
submat_status Plan::backward_wave(Wave& wv, const double* K, double mu, const double* Dbar,
                                  double* Kbar, double* dn_part, void* bws, cudaStream_t st) {
  using G = GemmFor<T>;
  using Args = typename G::Args;
  const int64_t E = bws_elems;
  double* A = static_cast<double*>(bws);
  T* base = reinterpret_cast<T*>(A + E);
  T* X[2] = {base, base + E};
  T* Ed[2] = {base + 2 * E, base + 3 * E};
  T* Y = base + 4 * E;
  T* T1 = base + 5 * E;
  SM_TRY(gather_wave(wv, K, mu, A, st));
  const int passes = dn_part ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    // iteration state and beta (the bound) reset for this pass
    if (pass > 0) SM_CUDA(launch_beta(wv.dev, ns, opt.beta_mode, st));
    // X_0 = a / beta, E_0 = G / beta (or I / beta)
    if (sizeof(T) == 8) SM_CUDA(launch_scale_f64(wv.dev, A, reinterpret_cast<double*>(X[0]), ns.beta, wv.max_ld2, st));
    else SM_CUDA(launch_scale_f32(wv.dev, A, reinterpret_cast<float*>(X[0]), ns.beta, wv.max_ld2, st));
    if (opt.beta_mode == 0) {  // the power estimate tightens beta as in the forward paths
      if (sizeof(T) == 8) {
        double* x0 = reinterpret_cast<double*>(X[0]);
        SM_CUDA(launch_power_f64(wv.dev, x0, kPowerIters, ns.state, ns.rprev, max_ld(wv), st));
        SM_CUDA(launch_rescale_f64(wv.dev, x0, ns.rprev, ns.beta, ns.state, wv.max_ld2, st));
      } else {
        float* x0 = reinterpret_cast<float*>(X[0]);
        SM_CUDA(launch_power_f32(wv.dev, x0, kPowerIters, ns.state, ns.rprev, max_ld(wv), st));
        SM_CUDA(launch_rescale_f32(wv.dev, x0, ns.rprev, ns.beta, ns.state, wv.max_ld2, st));
      }
    }
    k_bwd_seed<T><<<wv.n_gather, dim3(32, 8), 0, st>>>(g, wv.dev, wv.gather_items, Dbar, ns.beta, Ed[0], pass);
    SM_KCHECK();
    // the power kernel used rprev for its estimate
    SM_CUDA(launch_reset_rprev(wv.dev, ns, st));
    int cur = 0, extra = -1;
    for (int k = 0; k < opt.max_iter + 2; ++k) {
      Args a{};
      a.w = wv.dev;
      a.state = nullptr;
      a.skip_state = -1;
      auto gemm = [&](const int4* items, int nitems, const T* Aop, const T* Bop, const T* C0, T* C,
                      double alpha, double beta, int sym, double* res2) -> cudaError_t {
        Args b = a;
        b.items = items; b.nitems = nitems;
        b.A = Aop; b.B = Bop; b.C0 = C0; b.C = C;
        b.alpha = alpha; b.beta = beta; b.diag = 0.0; b.sym = sym; b.res2 = res2;
        size_t tk;
        if (timer.start(KC_SIMT, st, &tk) != SUBMAT_OK) return cudaErrorUnknown;
        cudaError_t e = G::run(b, st);
        if (e == cudaSuccess && timer.stop(tk, st) != SUBMAT_OK) return cudaErrorUnknown;
        return e;
      };
      T* Xc = X[cur];
      T* Ec = Ed[cur];
      // Y = X^2 (symmetric), with the involution residual while still iterating
      SM_CUDA(gemm(wv.sym64, wv.n_sym64, Xc, Xc, nullptr, Y, 1.0, 0.0, 1, extra < 0 ? ns.res2 : nullptr));
      if (k == 0 && opt.beta_mode == 0) {  // as in the forward paths; E_0 follows X_0
        const CertSquare sq{sizeof(T) == 8 ? 0 : 1, Y, nullptr, 1.0f, 0.0f};
        const CertLinear lin{2, {Xc, Ec, nullptr}, {nullptr, nullptr, nullptr}};
        SM_CUDA(launch_certify(wv.dev, ns, sq, lin, cert_limits(false), max_ld(wv), d_flags + 2, st));
      }
      if (extra < 0) SM_CUDA(launch_ns_update(wv.dev, ns, tol_eff, sizeof(T) == 8 ? 1e-9 : 1e-4, opt.max_iter, d_flags, st));
      // T1 = X E + E X
      SM_CUDA(gemm(wv.full64, wv.n_full64, Xc, Ec, nullptr, T1, 1.0, 0.0, 0, nullptr));
      SM_CUDA(gemm(wv.full64, wv.n_full64, Ec, Xc, T1, T1, 1.0, 1.0, 0, nullptr));
      // E' = 3/2 E - 1/2 E X^2 - 1/2 X T1
      SM_CUDA(gemm(wv.full64, wv.n_full64, Ec, Y, Ec, Ed[cur ^ 1], -0.5, 1.5, 0, nullptr));
      SM_CUDA(gemm(wv.full64, wv.n_full64, Xc, T1, Ed[cur ^ 1], Ed[cur ^ 1], -0.5, 1.0, 0, nullptr));
      // X' = 3/2 X - 1/2 X X^2 (every submatrix keeps iterating: a converged
      // X stays at its fixed point while E settles)
      SM_CUDA(gemm(wv.sym64, wv.n_sym64, Xc, Y, Xc, X[cur ^ 1], -0.5, 1.5, 1, nullptr));
      cur ^= 1;
      if (extra < 0) {
        SM_CUDA(cudaMemsetAsync(d_active, 0, sizeof(int), st));
        SM_CUDA(launch_ns_post(wv.dev, ns, cur, d_active, st));
        SM_CUDA(cudaMemcpyAsync(h_pinned, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        SM_CUDA(cudaStreamSynchronize(st));
        if (reinterpret_cast<int*>(h_pinned)[0] == 0) extra = 2;  // E settles in two more steps
      } else if (--extra == 0) {
        break;
      }
    }
    if (pass == 0) {
      const size_t smem = size_t(3 * nb_max + 1) * sizeof(int);
      if (smem > 48 * 1024)
        SM_CUDA(cudaFuncSetAttribute(k_bwd_scatter_add<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      k_bwd_scatter_add<T><<<wv.n_gather, 256, smem, st>>>(
          g, wv.dev, wv.gather_items, Ed[cur], Kbar);
      SM_KCHECK();
    } else {
      k_bwd_dn<T><<<(wv.count + 255) / 256, 256, 0, st>>>(g, wv.dev, Ed[cur], dn_part);
      SM_KCHECK();
      std::vector<double> part(wv.count);
      SM_CUDA(cudaMemcpyAsync(part.data(), dn_part, sizeof(double) * wv.count, cudaMemcpyDeviceToHost, st));
      SM_CUDA(cudaStreamSynchronize(st));
      for (double v : part) dn_acc += v;
    }
  }
  SM_TRY(collect_wave(wv, st));
  return SUBMAT_OK;
}

submat_status Plan::backward(const double* K, double mu, const double* Dbar, double* Kbar,
                             double* dN_dmu, cudaStream_t st) {
  if (grouped) {
    set_error("submat_sign_backward: not available for grouped plans");
    return SUBMAT_ERR_UNSUPPORTED;
  }
  if (opt.kT > 0.0) return backward_fermi(K, mu, Dbar, Kbar, dN_dmu, st);
  reset_stats();
  SM_CUDA(cudaMemsetAsync(d_flags, 0, 4 * sizeof(int), st));
  SM_CUDA(launch_check_finite(Dbar, nvals, d_flags, st));
  int fl = 0;
  SM_TRY(read_flags(st, &fl));
  if (fl & FLAG_NONFINITE) {
    set_error("Dbar holds a NaN or Inf value");
    return SUBMAT_ERR_NONFINITE;
  }
  const bool f64 = opt.prec == SUBMAT_FP64;
  const bool tc = opt.adjoint_mode == 1;  // tensor cores (mixed plans only)
  const size_t bpe = backward_bytes_per_elem(opt.prec, opt.adjoint_mode);
  // the adjoint keeps its own waves and workspace, sized for its six buffers
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
    SM_TRY(alloc(&d_dnpart, size_t(std::max(max_wave, max_bwave)), "dN/dmu partials"));
  }
  SM_CUDA(cudaMemsetAsync(Kbar, 0, sizeof(double) * size_t(nvals), st));
  dn_acc = 0.0;
  for (size_t wi = 0; wi < bwaves.size(); ++wi) {
    Wave& wv = bwaves[wi];
    if (tc) SM_TRY(backward_wave_tc(wi, K, mu, Dbar, Kbar, dN_dmu ? d_dnpart : nullptr, st));
    else if (f64) SM_TRY(backward_wave<double>(wv, K, mu, Dbar, Kbar, dN_dmu ? d_dnpart : nullptr, bws, st));
    else SM_TRY(backward_wave<float>(wv, K, mu, Dbar, Kbar, dN_dmu ? d_dnpart : nullptr, bws, st));
  }
  SM_CUDA(cudaStreamSynchronize(st));
  finish_stats(true);
  if (dN_dmu) *dN_dmu = dn_acc;
  SM_TRY(read_flags(st, &fl));
  if (fl & FLAG_NONFINITE) {
    set_error("K holds a NaN or Inf value");
    return SUBMAT_ERR_NONFINITE;
  }
  return SUBMAT_OK;
}

template submat_status Plan::backward_wave<double>(Wave&, const double*, double, const double*, double*,
                                                   double*, void*, cudaStream_t);
template submat_status Plan::backward_wave<float>(Wave&, const double*, double, const double*, double*,
                                                  double*, void*, cudaStream_t);

}  // namespace submat

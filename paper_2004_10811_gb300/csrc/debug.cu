// Test hooks (include/submat_debug.h): one kernel in isolation.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "plan.cuh"
#include "submat_debug.h"
#include "tc_gemm.cuh"

namespace submat {

long long timeout_cycles_for(double seconds) {
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (khz <= 0) khz = 2000000;
  if (!(seconds > 0)) seconds = 2.0;
  return static_cast<long long>(seconds * double(khz) * 1000.0);
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace submat

namespace {

struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  submat_status put(T** d, const void* src, size_t bytes, cudaStream_t st) {
    void* q = nullptr;
    submat_status s = submat::dev_alloc(&q, bytes, "debug scratch");
    if (s != SUBMAT_OK) return s;
    ptrs.push_back(q);
    *d = static_cast<T*>(q);
    if (src) SM_CUDA(cudaMemcpyAsync(q, src, bytes, cudaMemcpyHostToDevice, st));
    return SUBMAT_OK;
  }
};

}  // namespace

extern "C" submat_status submat_debug_tc_gemm(int count, int ld, int n, const void* A_hi,
                                              const void* A_lo, const void* B_hi, const void* B_lo,
                                              int split, int sym, float* C, double* res2,
                                              int skip_arrive, double timeout_s, int tile_n,
                                              void* stream) {
  using namespace submat;
  clear_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int f16 = (split >> 1) & 1;  // bit 1: FP16 operands
  split &= 1;
  if (count < 1 || count > (1 << 22) || ld < 64 || ld % 64 || ld > 8192 || n < 0 || n > ld ||
      !A_hi || !B_hi || !C || (split && (!A_lo || !B_lo))) {
    set_error("bad argument to submat_debug_tc_gemm");
    return SUBMAT_ERR_INVALID_ARG;
  }
  Scratch sc;
  std::vector<int64_t> off(count);
  std::vector<int32_t> lds(count, ld), ns(count, n);
  for (int s = 0; s < count; ++s) off[s] = int64_t(s) * ld * ld;
  const int bn = tile_n == 256 ? 256 : 128;
  if (tile_n != 0 && tile_n != 128 && tile_n != 256) {
    set_error("tile_n must be 0, 128 or 256");
    return SUBMAT_ERR_INVALID_ARG;
  }
  std::vector<int4> items;
  const int T = (ld + 127) / 128;
  const int TB = (ld + bn - 1) / bn;
  const int H = bn / 128;
  for (int s = 0; s < count; ++s)
    for (int a = 0; a < T; ++a)
      for (int b = 0; b < TB; ++b)
        if (!sym || H * b + H - 1 >= a) items.push_back(make_int4(s, a, b, 0 | (s << 8)));
  CUtensorMap maps[8];
  std::memset(maps, 0, sizeof(maps));
  const void* srcs[4] = {A_hi, split ? A_lo : A_hi, B_hi, split ? B_lo : B_hi};
  for (int m = 0; m < 4; ++m)
    if (make_bucket_map(&maps[m], srcs[m], ld, count) != 0 ||
        make_bucket_map(&maps[4 + m], srcs[m], ld, count, 256) != 0) {
      set_error("cuTensorMapEncodeTiled failed (map %d)", m);
      return SUBMAT_ERR_CUDA;
    }
  int64_t* d_off; int32_t* d_ld; int32_t* d_n; int4* d_items; CUtensorMap* d_maps; int* d_flags;
  SM_TRY(sc.put(&d_off, off.data(), off.size() * 8, st));
  SM_TRY(sc.put(&d_ld, lds.data(), lds.size() * 4, st));
  SM_TRY(sc.put(&d_n, ns.data(), ns.size() * 4, st));
  SM_TRY(sc.put(&d_items, items.data(), items.size() * sizeof(int4), st));
  SM_TRY(sc.put(&d_maps, maps, sizeof(maps), st));
  SM_TRY(sc.put(&d_flags, nullptr, 16, st));
  SM_CUDA(cudaMemsetAsync(d_flags, 0, 16, st));
  if (res2) SM_CUDA(cudaMemsetAsync(res2, 0, sizeof(double) * count, st));

  TcGemmParams p;
  std::memset(&p, 0, sizeof(p));
  p.items = d_items;
  p.nitems = int(items.size());
  p.maps = d_maps;
  p.maps_b = d_maps + 4;
  p.bn = bn;
  p.nbucket = 1;
  p.nmaps = 4;
  p.na = split ? 2 : 1;
  p.nb = split ? 2 : 1;
  p.a_set[0] = 0; p.a_set[1] = 1;
  p.b_set[0] = 2; p.b_set[1] = 3;
  if (split) {
    p.nprod = 3;
    const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
    for (int i = 0; i < 3; ++i) { p.prod_a[i] = pa[i]; p.prod_b[i] = pb[i]; p.prod_acc[i] = 0; p.prod_first[i] = i == 0; }
  } else {
    p.nprod = 1;
    p.prod_a[0] = 0; p.prod_b[0] = 0; p.prod_acc[0] = 0; p.prod_first[0] = 1;
  }
  p.nacc = 1;
  p.nstage = tc_pick_stages(p.na, p.nb, bn);
  p.tmem_cols = 2 * bn;
  p.off = d_off; p.ld = d_ld; p.n = d_n;
  p.state = nullptr;
  p.skip_state = -1;
  p.alpha = 1.0f; p.beta = 0.0f;
  p.sym = sym;
  p.f16 = f16;
  p.out_f32 = C;
  p.res2 = res2;
  p.flags = d_flags;
  p.timeout_cycles = timeout_cycles_for(timeout_s);
  p.test_skip_arrive = skip_arrive;
  // the timeout hook needs several tiles per CTA, so it runs on one CTA
  const int grid = skip_arrive ? 1 : std::min<int>(p.nitems, num_sms());
  SM_CUDA(launch_tc_gemm(p, grid, st));
  int fl = 0;
  SM_CUDA(cudaMemcpyAsync(&fl, d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaStreamSynchronize(st));
  if (fl & FLAG_TIMEOUT) {
    set_error("a bounded wait in the tensor-core GEMM expired");
    return SUBMAT_ERR_TIMEOUT;
  }
  return SUBMAT_OK;
}

extern "C" submat_status submat_debug_slice_plan(int nx, int ny, int sym_pairs, int per_acc, int max_acc,
                                                 int32_t* out, int cap, int32_t* count) {
  using namespace submat;
  clear_error();
  const int smax = slice_max_slices();
  if (!count || nx < 1 || ny < 1 || nx > smax || ny > smax || (per_acc != 1 && per_acc != 2) ||
      (max_acc != 2 && max_acc != kSliceMaxAcc) || (sym_pairs && nx != ny) || cap < 0) {
    set_error("bad argument to submat_debug_slice_plan");
    return SUBMAT_ERR_INVALID_ARG;
  }
  std::vector<SliceGroup> groups;
  std::vector<SliceLaunch> launches;
  slice_plan(nx, ny, sym_pairs != 0, per_acc, max_acc, &groups, &launches);
  int n = 0;
  for (size_t l = 0; l < launches.size(); ++l) {
    for (int acc = 0; acc < launches[l].ng; ++acc) {
      const SliceGroup& gr = groups[size_t(launches[l].g[acc])];
      for (int i = 0; i < gr.np; ++i, ++n) {
        if (out && n < cap) {
          int32_t* r = out + 5 * int64_t(n);
          r[0] = int32_t(l); r[1] = acc; r[2] = gr.pr[i][0]; r[3] = gr.pr[i][1]; r[4] = gr.shift;
        }
      }
    }
  }
  *count = n;
  if (out && n > cap) {
    set_error("submat_debug_slice_plan: %d records, room for %d", n, cap);
    return SUBMAT_ERR_INVALID_ARG;
  }
  return SUBMAT_OK;
}

extern "C" submat_status submat_debug_mu_bisect(const double* levels, int nlev, double n_el, double mu0,
                                                double tol, int max_steps, double bound_scale, double probe_err,
                                                double* mu_out, int32_t* steps, int32_t* probes,
                                                double* n_out) {
  using namespace submat;
  clear_error();
  if (nlev < 0 || (nlev > 0 && !levels) || !mu_out || !steps || max_steps < 1 || !(tol > 0) ||
      !std::isfinite(n_el) || !std::isfinite(mu0) || !(bound_scale > 0) || !(probe_err >= 0)) {
    set_error("bad argument to submat_debug_mu_bisect");
    return SUBMAT_ERR_INVALID_ARG;
  }
  if (n_el < 0.0 || n_el > double(nlev)) {  // as submat_mu_search: outside [0, n]
    set_error("n_el = %.17g outside [0, %d]", n_el, nlev);
    return SUBMAT_ERR_INVALID_ARG;
  }
  auto count = [&](double mu) {
    double c = 0.0;
    for (int i = 0; i < nlev; ++i) c += levels[i] < mu ? 1.0 : (levels[i] == mu ? 0.5 : 0.0);
    return c;
  };
  auto eval = [&](double mu, double* n) -> submat_status {
    *n = count(mu);
    return SUBMAT_OK;
  };
  auto bound = [&]() {
    double b = 0.0;
    for (int i = 0; i < nlev; ++i) b = std::max(b, std::fabs(levels[i] - mu0));
    return b * bound_scale;
  };
  // probe: the count off by up to probe_err (alternating sides), with that bound
  int calls = 0;
  MuProbe probe;
  if (probe_err > 0)
    probe = [&](double mu, double* n, double* b) -> submat_status {
      *n = count(mu) + ((calls++ & 1) ? probe_err : -probe_err);
      *b = probe_err;
      return SUBMAT_OK;
    };
  MuSearchOut r;
  const submat_status s = mu_bisect(eval, bound, n_el, mu0, tol, max_steps, &r, probe);
  *mu_out = r.mu;
  *steps = r.steps;
  if (probes) *probes = r.probes;
  if (n_out) *n_out = count(r.mu);
  return s;
}

extern "C" submat_status submat_debug_fermi_poly(double c, double tol, int max_degree, double* r_out, int cap,
                                                 int32_t* degree, int32_t* blocks, double* trunc) {
  using namespace submat;
  clear_error();
  if (!degree || !blocks || !trunc || cap < 0 || max_degree < 1 || max_degree > kFermiMaxDegree ||
      !(tol > 0)) {
    set_error("bad argument to submat_debug_fermi_poly");
    return SUBMAT_ERR_INVALID_ARG;
  }
  FermiPoly P;
  SM_TRY(fermi_poly(c, tol, max_degree, &P));
  *degree = P.m;
  *blocks = P.blocks;
  *trunc = P.trunc;
  const int n = int(P.r.size());
  if (r_out) {
    if (cap < n) {
      set_error("submat_debug_fermi_poly: %d coefficients, room for %d", n, cap);
      return SUBMAT_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) r_out[i] = P.r[i];
  }
  return SUBMAT_OK;
}

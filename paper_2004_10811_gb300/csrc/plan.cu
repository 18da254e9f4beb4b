// Host side of the submatrix library: the plan (Section IV-A: global pattern,
// per-submatrix index maps, waves), the Newton-Schulz drivers and the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "plan.cuh"

namespace submat {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

const char* last_error() { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// device memory helpers
// ---------------------------------------------------------------------------

submat_status dev_alloc(void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) return SUBMAT_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SUBMAT_ERR_OOM : SUBMAT_ERR_CUDA;
  }
  return SUBMAT_OK;
}

Plan::~Plan() {
  free_mixed(mixed);
  free_adjoint_tc(adj_tc);
  for (void* p : owned) cudaFree(p);
  if (h_pinned) cudaFreeHost(h_pinned);
  for (auto& e : ev) if (e) cudaEventDestroy(e);
}

// bytes of workspace per dense element for each precision
static size_t bytes_per_elem(int prec, double kT) {
  if (kT > 0.0) return fermi_bytes_per_elem(prec);
  switch (prec) {
    case SUBMAT_FP64: return 3 * 8;                 // X ping-pong + X^2
    case SUBMAT_FP32: return 8 + 3 * 4;             // A (FP64) + X ping-pong + X^2
    default: return mixed_bytes_per_elem();
  }
}

// ---------------------------------------------------------------------------
// per-launch timing
// ---------------------------------------------------------------------------

KernelTimer::~KernelTimer() {
  for (auto e : pool) cudaEventDestroy(e);
}

submat_status KernelTimer::start(int cls, cudaStream_t st, size_t* tok) {
  *tok = size_t(-1);
  if (!on) return SUBMAT_OK;
  while (pool.size() < used + 2) {
    cudaEvent_t e;
    SM_CUDA(cudaEventCreate(&e));
    pool.push_back(e);
  }
  *tok = used;
  marks.emplace_back(cls, used);
  SM_CUDA(cudaEventRecord(pool[used], st));
  used += 2;
  return SUBMAT_OK;
}

submat_status KernelTimer::stop(size_t tok, cudaStream_t st) {
  if (!on || tok == size_t(-1)) return SUBMAT_OK;
  SM_CUDA(cudaEventRecord(pool[tok + 1], st));
  return SUBMAT_OK;
}

submat_status KernelTimer::collect(double* ms, int32_t* count) {
  for (auto& m : marks) {
    float t = 0.0f;
    SM_CUDA(cudaEventElapsedTime(&t, pool[m.second], pool[m.second + 1]));
    ms[m.first] += t;
    count[m.first] += 1;
  }
  marks.clear();
  used = 0;
  return SUBMAT_OK;
}

// ---------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------

static submat_status validate_pattern(int nblk, const int32_t* bs, const int64_t* rp,
                                      const int32_t* ci) {
  if (rp[0] != 0) { set_error("row_ptr[0] must be 0"); return SUBMAT_ERR_PATTERN; }
  for (int i = 0; i < nblk; ++i) {
    if (bs[i] < 1) { set_error("block_sizes[%d] = %d < 1", i, bs[i]); return SUBMAT_ERR_INVALID_ARG; }
    if (rp[i + 1] < rp[i]) { set_error("row_ptr decreases at row %d", i); return SUBMAT_ERR_PATTERN; }
  }
  const int64_t nnzb = rp[nblk];
  for (int i = 0; i < nblk; ++i) {
    bool diag = false;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int c = ci[p];
      if (c < 0 || c >= nblk) {
        set_error("col_idx[%lld] = %d out of range [0, %d)", (long long)p, c, nblk);
        return SUBMAT_ERR_PATTERN;
      }
      if (p > rp[i] && ci[p - 1] >= c) {
        set_error("col_idx not strictly increasing in row %d", i);
        return SUBMAT_ERR_PATTERN;
      }
      if (c == i) diag = true;
    }
    if (!diag) { set_error("diagonal block (%d, %d) is not stored", i, i); return SUBMAT_ERR_PATTERN; }
  }
  (void)nnzb;
  return SUBMAT_OK;
}

submat_status validate_pattern_public(int nblk, const int32_t* bs, const int64_t* rp,
                                      const int32_t* ci) {
  return validate_pattern(nblk, bs, rp, ci);
}

static int64_t find_block(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci, int r,
                          int c) {
  auto b = ci.begin() + rp[r], e = ci.begin() + rp[r + 1];
  auto it = std::lower_bound(b, e, c);
  if (it == e || *it != c) return -1;
  return int64_t(it - ci.begin());
}

// Split the evaluated block columns into waves whose dense buffers (bpe bytes
// per element) fit `cap`, and build each wave's maps and work lists.
submat_status Plan::build_waves(size_t bpe, size_t cap, std::vector<Wave>& waves, cudaStream_t st) {
  std::vector<int64_t> ld_of(nq);
  for (int j = 0; j < nq; ++j) ld_of[j] = (qn[j] + 63) / 64 * 64;
  waves.clear();
  {
    int first = col_lo;
    while (first < col_hi) {
      int64_t elems = 0;
      int cnt = 0;
      while (first + cnt < col_hi) {
        const int64_t e = ld_of[first + cnt] * ld_of[first + cnt];
        if (cnt > 0 && size_t(elems + e) * bpe > cap) break;
        if (cnt == 0 && size_t(e) * bpe > cap) {
          set_error("one submatrix (dim %d) needs %zu bytes > workspace cap %zu", qn[first],
                    size_t(e) * bpe, cap);
          return SUBMAT_ERR_OOM;
        }
        elems += e;
        ++cnt;
        if (cnt >= 65535) break;  // grid.y limit of the scaling kernel
      }
      Wave wv;
      wv.first = first;
      wv.count = cnt;
      wv.elems = elems;
      waves.push_back(wv);
      first += cnt;
    }
  }
  // per-wave maps and work lists.  Dense buffers are grouped into size
  // buckets (equal ld) laid out as [count][ld][ld], so that each bucket is one
  // 3D tensor for the TMA loads of the tensor-core GEMM.
  for (auto& wv : waves) {
    std::vector<int32_t> sub(wv.count), ld(wv.count), nn(wv.count);
    std::vector<int64_t> off(wv.count);
    std::vector<int2> gitems;
    std::vector<int4> sym64, full64, sym128, full128, sym256, full256;
    double area128 = 0.0, area256 = 0.0;
    std::vector<int64_t> lds;
    for (int s = 0; s < wv.count; ++s) lds.push_back(ld_of[wv.first + s]);
    std::sort(lds.begin(), lds.end());
    lds.erase(std::unique(lds.begin(), lds.end()), lds.end());
    if (lds.size() > 255) { set_error("more than 255 size buckets in a wave"); return SUBMAT_ERR_UNSUPPORTED; }
    wv.bucket_ld.assign(lds.begin(), lds.end());
    wv.bucket_count.assign(lds.size(), 0);
    std::vector<int> bucket_of(wv.count), slot_of(wv.count);
    for (int s = 0; s < wv.count; ++s) {
      const int b = int(std::lower_bound(lds.begin(), lds.end(), ld_of[wv.first + s]) - lds.begin());
      bucket_of[s] = b;
      slot_of[s] = wv.bucket_count[b]++;
    }
    wv.bucket_base.assign(lds.size(), 0);
    int64_t o = 0;
    for (size_t b = 0; b < lds.size(); ++b) {
      wv.bucket_base[b] = o;
      o += int64_t(wv.bucket_count[b]) * lds[b] * lds[b];
    }
    wv.max_ld2 = 0;
    for (int s = 0; s < wv.count; ++s) {
      const int j = wv.first + s;
      sub[s] = j;
      ld[s] = int32_t(ld_of[j]);
      nn[s] = qn[j];
      off[s] = wv.bucket_base[bucket_of[s]] + int64_t(slot_of[s]) * ld_of[j] * ld_of[j];
      wv.max_ld2 = std::max(wv.max_ld2, ld_of[j] * ld_of[j]);
      const int nbj = int(grouped ? qsp[j + 1] - qsp[j] : row_ptr[j + 1] - row_ptr[j]);
      for (int t = 0; t < nbj; ++t) gitems.push_back(make_int2(s, t));
      const int T = int(ld_of[j] / 64);
      for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
          full64.push_back(make_int4(s, a, b, 0));
          if (a <= b) sym64.push_back(make_int4(s, a, b, 0));
        }
      const int T2 = int((ld_of[j] + 127) / 128);
      const int T4 = int((ld_of[j] + 255) / 256);
      const int tag = bucket_of[s] | (slot_of[s] << 8);
      for (int a = 0; a < T2; ++a)
        for (int b = 0; b < T2; ++b) {
          full128.push_back(make_int4(s, a, b, tag));
          if (a <= b) sym128.push_back(make_int4(s, a, b, tag));
        }
      // 128 x 256 tiles: sub-tiles (a, 2b) and (a, 2b + 1)
      for (int a = 0; a < T2; ++a)
        for (int b = 0; b < T4; ++b) {
          full256.push_back(make_int4(s, a, b, tag));
          if (2 * b + 1 >= a) sym256.push_back(make_int4(s, a, b, tag));
        }
      area128 += double(T2) * T2;
      area256 += double(T2) * T4 * 2;
    }
    // the wider tile when its padding costs at most 8 % more MMA work
    wv.bn = area256 <= 1.08 * area128 ? 256 : 128;
    int32_t* d_sub; int32_t* d_ld; int32_t* d_n; int64_t* d_off;
    SM_TRY(put(&d_sub, sub, st, "wave submatrices"));
    SM_TRY(put(&d_ld, ld, st, "wave ld"));
    SM_TRY(put(&d_n, nn, st, "wave dims"));
    SM_TRY(put(&d_off, off, st, "wave offsets"));
    wv.dev = WaveDev{wv.count, d_sub, d_off, d_ld, d_n};
    SM_TRY(put(&wv.gather_items, gitems, st, "gather items"));
    wv.n_gather = int(gitems.size());
    SM_TRY(put(&wv.sym64, sym64, st, "tile list"));
    wv.n_sym64 = int(sym64.size());
    SM_TRY(put(&wv.full64, full64, st, "tile list"));
    wv.n_full64 = int(full64.size());
    SM_TRY(put(&wv.sym128, sym128, st, "tile list"));
    wv.n_sym128 = int(sym128.size());
    SM_TRY(put(&wv.full128, full128, st, "tile list"));
    wv.n_full128 = int(full128.size());
    SM_TRY(put(&wv.sym256, sym256, st, "tile list"));
    wv.n_sym256 = int(sym256.size());
    SM_TRY(put(&wv.full256, full256, st, "tile list"));
    wv.n_full256 = int(full256.size());
    wv.host_ld = ld;
    wv.host_n = nn;
    wv.host_off = off;
  }
  return SUBMAT_OK;
}

// Submatrices shared by groups of block columns (Section IV-C): submatrix q
// of a group G spans N(G), the ascending union of its members' row sets.
submat_status Plan::build_groups(const int32_t* groups) {
  int ng = 0;
  for (int j = 0; j < nblk; ++j) {
    if (groups[j] < 0 || groups[j] >= nblk) {
      set_error("groups[%d] = %d outside [0, %d)", j, groups[j], nblk);
      return SUBMAT_ERR_INVALID_ARG;
    }
    ng = std::max(ng, groups[j] + 1);
  }
  std::vector<std::vector<int>> mem(ng);
  for (int j = 0; j < nblk; ++j) mem[groups[j]].push_back(j);
  for (int q = 0; q < ng; ++q)
    if (mem[q].empty()) {
      set_error("group %d has no block column (group ids must be 0 .. ngroups - 1, all used)", q);
      return SUBMAT_ERR_INVALID_ARG;
    }
  nq = ng;
  grouped = true;
  qn.assign(nq, 0);
  qext.assign(nq, 0);
  qsp.assign(nq + 1, 0);
  qrows.clear();
  qloc.clear();
  qof.assign(nblk, 0);
  qmp.assign(nq + 1, 0);
  qmcol.clear();
  qmkoff.clear();
  dloc.assign(nnzb, 0);
  qm_max = 1;
  for (int q = 0; q < nq; ++q) {
    std::vector<int32_t> rows;
    for (int j : mem[q]) rows.insert(rows.end(), col.begin() + row_ptr[j], col.begin() + row_ptr[j + 1]);
    std::sort(rows.begin(), rows.end());
    rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
    std::vector<int32_t> lo(rows.size());
    int64_t acc = 0;
    for (size_t t = 0; t < rows.size(); ++t) { lo[t] = int32_t(acc); acc += bs[rows[t]]; }
    if (acc > 32768) {
      set_error("group %d spans a submatrix of dimension %lld > 32768", q, (long long)acc);
      return SUBMAT_ERR_UNSUPPORTED;
    }
    auto local = [&](int i) {
      return lo[size_t(std::lower_bound(rows.begin(), rows.end(), i) - rows.begin())];
    };
    qn[q] = int32_t(acc);
    for (int j : mem[q]) {
      qof[j] = q;
      qmcol.push_back(j);
      qmkoff.push_back(local(j));
      qext[q] += bs[j];
      for (int64_t t = row_ptr[j]; t < row_ptr[j + 1]; ++t) dloc[tpos[t]] = local(col[t]);
    }
    qm_max = std::max<int>(qm_max, int(mem[q].size()));
    qrows.insert(qrows.end(), rows.begin(), rows.end());
    qloc.insert(qloc.end(), lo.begin(), lo.end());
    qsp[q + 1] = int64_t(qrows.size());
    qmp[q + 1] = int32_t(qmcol.size());
  }
  return SUBMAT_OK;
}

submat_status Plan::build(int nblk_, const int32_t* bs_, const int64_t* rp_, const int32_t* ci_,
                          const submat_options* o, cudaStream_t st, const int32_t* groups) {
  nblk = nblk_;
  opt = *o;
  bs.assign(bs_, bs_ + nblk);
  row_ptr.assign(rp_, rp_ + nblk + 1);
  nnzb = row_ptr[nblk];
  col.assign(ci_, ci_ + nnzb);
  // value offsets (CSR order, no padding)
  valptr.assign(nnzb + 1, 0);
  rowof.assign(nnzb, 0);
  for (int r = 0; r < nblk; ++r)
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) {
      rowof[p] = r;
      valptr[p + 1] = valptr[p] + int64_t(bs[r]) * bs[col[p]];
    }
  nvals = valptr[nnzb];
  // symmetry of the pattern and the transpose map
  tpos.assign(nnzb, -1);
  diagpos.assign(nblk, -1);
  for (int r = 0; r < nblk; ++r)
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) {
      const int c = col[p];
      const int64_t q = find_block(row_ptr, col, c, r);
      if (q < 0) {
        set_error("pattern is not symmetric: block (%d, %d) stored but (%d, %d) is not", r, c, c, r);
        return SUBMAT_ERR_PATTERN;
      }
      if (q > INT32_MAX) { set_error("more than 2^31 blocks"); return SUBMAT_ERR_UNSUPPORTED; }
      tpos[p] = int32_t(q);
      if (c == r) diagpos[r] = int32_t(p);
    }
  // submatrices: N(j) = column j's block rows = row j's columns (symmetric)
  locoff.assign(nnzb, 0);
  nsub.assign(nblk, 0);
  koff.assign(nblk, 0);
  nb_max = 0;
  n_max = 0;
  n_min = INT32_MAX;
  bs_max = *std::max_element(bs.begin(), bs.end());
  sum_n2 = sum_n3 = 0.0;
  for (int j = 0; j < nblk; ++j) {
    int64_t acc = 0;
    for (int64_t p = row_ptr[j]; p < row_ptr[j + 1]; ++p) {
      locoff[p] = int32_t(acc);
      if (col[p] == j) koff[j] = int32_t(acc);
      acc += bs[col[p]];
    }
    if (acc > 32768) {
      set_error("submatrix %d has dimension %lld > 32768", j, (long long)acc);
      return SUBMAT_ERR_UNSUPPORTED;
    }
    nsub[j] = int32_t(acc);
    nb_max = std::max<int>(nb_max, int(row_ptr[j + 1] - row_ptr[j]));
    nbj_max = nb_max;
    n_max = std::max<int>(n_max, nsub[j]);
    n_min = std::min<int>(n_min, nsub[j]);
    sum_n2 += double(acc) * acc;
    sum_n3 += double(acc) * acc * acc;
  }
  // submatrices: one per block column, or one per group
  if (groups) {
    SM_TRY(build_groups(groups));
    nb_max = n_max = 0;
    n_min = INT32_MAX;
    sum_n2 = sum_n3 = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double n = qn[q];
      nb_max = std::max<int>(nb_max, int(qsp[q + 1] - qsp[q]));
      n_max = std::max<int>(n_max, qn[q]);
      n_min = std::min<int>(n_min, qn[q]);
      sum_n2 += n * n;
      sum_n3 += n * n * n;
    }
  } else {
    nq = nblk;
    qn = nsub;
    qext = bs;
    qof.resize(nblk);
    for (int j = 0; j < nblk; ++j) qof[j] = j;
  }
  if (nb_max * 3 + 1 > 48 * 1024) {
    set_error("a submatrix spans %d blocks; at most 16383 are supported", nb_max);
    return SUBMAT_ERR_UNSUPPORTED;
  }
  // device copies of the pattern and maps
  {
    int32_t* d_bs; int64_t* d_rp; int32_t* d_col; int64_t* d_vp; int32_t* d_loc; int32_t* d_tp;
    int32_t* d_ns; int32_t* d_ko; int32_t* d_dp;
    SM_TRY(put(&d_bs, bs, st, "block sizes"));
    SM_TRY(put(&d_rp, row_ptr, st, "row_ptr"));
    SM_TRY(put(&d_col, col, st, "col_idx"));
    SM_TRY(put(&d_vp, valptr, st, "value offsets"));
    SM_TRY(put(&d_loc, locoff, st, "local offsets"));
    SM_TRY(put(&d_tp, tpos, st, "transpose map"));
    SM_TRY(put(&d_ns, nsub, st, "submatrix dims"));
    SM_TRY(put(&d_ko, koff, st, "k offsets"));
    SM_TRY(put(&d_dp, diagpos, st, "diagonal positions"));
    SM_TRY(put(&d_rowof, rowof, st, "row of block"));
    g = PatternDev{d_bs, d_rp, d_col, d_vp, d_loc, d_tp, d_ns, d_ko, d_dp,
                   d_rp, d_col, d_loc, nullptr, nullptr, nullptr, nullptr};
    if (grouped) {
      int64_t* d_sp; int32_t* d_sr; int32_t* d_sl; int32_t* d_mp; int32_t* d_mc; int32_t* d_mk; int32_t* d_dl;
      SM_TRY(put(&d_sp, qsp, st, "submatrix rows"));
      SM_TRY(put(&d_sr, qrows, st, "submatrix rows"));
      SM_TRY(put(&d_sl, qloc, st, "submatrix offsets"));
      SM_TRY(put(&d_mp, qmp, st, "group members"));
      SM_TRY(put(&d_mc, qmcol, st, "group members"));
      SM_TRY(put(&d_mk, qmkoff, st, "group member offsets"));
      SM_TRY(put(&d_dl, dloc, st, "group block offsets"));
      g.sp = d_sp; g.srows = d_sr; g.sloc = d_sl;
      g.mp = d_mp; g.mcol = d_mc; g.mkoff = d_mk; g.dloc = d_dl;
    }
  }
  // waves
  const size_t bpe = bytes_per_elem(opt.prec, opt.kT);
  size_t cap = opt.workspace_cap_bytes;
  if (cap == 0) {
    size_t fre = 0, tot = 0;
    SM_CUDA(cudaMemGetInfo(&fre, &tot));
    cap = size_t(double(fre) * 0.8);
  }
  // the evaluated submatrices (a column range without groups)
  col_lo = opt.col_end > opt.col_begin ? opt.col_begin : 0;
  col_hi = opt.col_end > opt.col_begin ? opt.col_end : nq;
  SM_TRY(build_waves(bpe, cap, waves, st));
  int64_t max_elems = 0;
  max_wave = 0;
  for (auto& wv : waves) {
    max_elems = std::max(max_elems, wv.elems);
    max_wave = std::max(max_wave, wv.count);
  }
  // workspace
  ws_elems = max_elems;
  ws_bytes = size_t(max_elems) * bpe;
  SM_TRY(dev_alloc(&ws, ws_bytes, "workspace"));
  if (ws) owned.push_back(ws);
  // Newton-Schulz state (per wave slot) and per-block results
  {
    const int want = max_wave;
    max_wave = 0;
    SM_TRY(grow_ns_state(want));
  }
  SM_TRY(alloc(&d_flags, 4, "flags"));
  SM_TRY(alloc(&d_active, 1, "active count"));
  SM_TRY(alloc(&d_trpart, size_t(nblk), "trace partials"));
  if (opt.kT > 0.0) SM_TRY(alloc(&d_sqpart, size_t(nblk), "sum-of-squares partials"));
  SM_TRY(alloc(&d_scalar, 8, "scalars"));
  SM_CUDA(cudaMallocHost(&h_pinned, 64));
  for (auto& e : ev) SM_CUDA(cudaEventCreate(&e));
  timer.on = opt.timing != 0;
  if (timer.on) {
    // K values each submatrix reads: the stored blocks inside N(q) x N(q)
    const std::vector<int64_t>& sp = grouped ? qsp : row_ptr;
    const std::vector<int32_t>& sr = grouped ? qrows : col;
    gather_bytes.assign(nq, 0.0);
    for (int j = 0; j < nq; ++j) {
      double acc = 0.0;
      for (int64_t t = sp[j]; t < sp[j + 1]; ++t) {
        const int i = sr[t];
        int64_t a = sp[j], e = sp[j + 1];
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
          while (a < e && sr[a] < col[q]) ++a;
          if (a < e && sr[a] == col[q]) acc += double(bs[i]) * bs[col[q]];
        }
      }
      gather_bytes[j] = 8.0 * acc;
    }
  }
  res_iters.assign(nq, 0);
  res_resid.assign(nq, 0.0);
  res_beta.assign(nq, 0.0);
  res_bound.assign(nq, 0.0);
  res_notconv.assign(nq, 0);
  SM_CUDA(cudaStreamSynchronize(st));
  return SUBMAT_OK;
}

// Per-slot Newton-Schulz state for waves of up to `count` submatrices.
submat_status Plan::grow_ns_state(int count) {
  if (count <= max_wave && ns.state) return SUBMAT_OK;
  SM_TRY(alloc(&ns.state, count, "ns state"));
  SM_TRY(alloc(&ns.iters, count, "ns iters"));
  SM_TRY(alloc(&ns.par, count, "ns parity"));
  SM_TRY(alloc(&ns.notconv, count, "ns flags"));
  SM_TRY(alloc(&ns.res2, count, "ns residual"));
  SM_TRY(alloc(&ns.rprev, count, "ns residual"));
  SM_TRY(alloc(&ns.beta, count, "ns beta"));
  SM_TRY(alloc(&ns.gersh, count, "ns gersh"));
  SM_TRY(alloc(&ns.fro2, count, "ns fro"));
  SM_TRY(alloc(&ns.cert, count, "ns certificate"));
  SM_TRY(alloc(&ns.cscale, count, "ns certificate"));
  max_wave = std::max(max_wave, count);
  return SUBMAT_OK;
}

// ---------------------------------------------------------------------------
// sign evaluation
// ---------------------------------------------------------------------------

int max_ld(const Wave& wv) {
  int64_t m = 64;
  for (int64_t l : wv.bucket_ld) m = std::max(m, l);
  return int(m);
}

// d_flags[0] is the status word; d_flags[2] counts the submatrices whose
// scale the certificate reduced (since the last reset of the flags).
submat_status Plan::read_flags(cudaStream_t st, int* out) {
  SM_CUDA(cudaMemcpyAsync(h_pinned, d_flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaStreamSynchronize(st));
  *out = reinterpret_cast<int*>(h_pinned)[0];
  last_flags = *out;
  stats.scale_reduced = reinterpret_cast<int*>(h_pinned)[2];
  return SUBMAT_OK;
}

submat_status Plan::gather_wave(Wave& wv, const double* K, double mu, double* A, cudaStream_t st) {
  SM_CUDA(cudaMemsetAsync(ns.gersh, 0, sizeof(unsigned long long) * wv.count, st));
  SM_CUDA(cudaMemsetAsync(ns.fro2, 0, sizeof(double) * wv.count, st));
  size_t tk;
  SM_TRY(timer.start(KC_GATHER, st, &tk));
  SM_CUDA(launch_gather(g, wv.dev, wv.gather_items, wv.n_gather, nb_max, max_ld(wv), bs_max, K, mu, A, ns, d_flags,
                        st));
  SM_TRY(timer.stop(tk, st));
  if (timer.on)
    for (int s = 0; s < wv.count; ++s)
      stats.kernel_work[KC_GATHER] += 8.0 * double(wv.host_ld[s]) * wv.host_ld[s] + gather_bytes[wv.first + s];
  int fl = 0;
  SM_TRY(read_flags(st, &fl));
  if (fl & FLAG_NONFINITE) {
    set_error("K holds a NaN or Inf value (in the submatrices of wave starting at block %d)",
              wv.first);
    return SUBMAT_ERR_NONFINITE;
  }
  SM_CUDA(launch_beta(wv.dev, ns, opt.beta_mode, st));
  return SUBMAT_OK;
}

submat_status Plan::collect_wave(const Wave& wv, cudaStream_t st) {
  std::vector<int> it(wv.count), nc(wv.count);
  std::vector<double> rp(wv.count), be(wv.count), fr(wv.count);
  std::vector<unsigned long long> gs(wv.count);
  SM_CUDA(cudaMemcpyAsync(it.data(), ns.iters, sizeof(int) * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(nc.data(), ns.notconv, sizeof(int) * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(rp.data(), ns.rprev, sizeof(double) * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(be.data(), ns.beta, sizeof(double) * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(gs.data(), ns.gersh, sizeof(unsigned long long) * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaMemcpyAsync(fr.data(), ns.fro2, sizeof(double) * wv.count, cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaStreamSynchronize(st));
  for (int s = 0; s < wv.count; ++s) {
    const int j = wv.first + s;
    res_iters[j] = it[s];
    res_notconv[j] = nc[s];
    res_resid[j] = rp[s] > 1e299 ? 0.0 : rp[s];
    res_beta[j] = be[s];
    double gersh = 0.0;
    std::memcpy(&gersh, &gs[s], sizeof(double));
    // the bound beta of the gather's FP32 sums, with their margin
    res_bound[j] = std::min(gersh, std::sqrt(fr[s])) * (1.0 + 1e-4);
  }
  return SUBMAT_OK;
}

// Newton-Schulz X <- 1/2 X (3 I - X^2) (Section II-B) on one wave, in T
// (double or float) with the SIMT GEMM.  X_0 is in buf[0]; on return
// ns.par[s] names the buffer that holds sign(a_s).
template <typename T, typename Args>
submat_status Plan::ns_simt(const Wave& wv, T* buf0, T* buf1, T* Y, double tol, double floor_thr,
                            cudaStream_t st, cudaError_t (*gemm)(const Args&, cudaStream_t), bool certify) {
  T* bufs[2] = {buf0, buf1};
  int cur = 0;
  for (int k = 0; k < opt.max_iter; ++k) {
    Args a1{};
    a1.w = wv.dev; a1.items = wv.sym64; a1.nitems = wv.n_sym64;
    a1.A = bufs[cur]; a1.B = bufs[cur]; a1.C0 = nullptr; a1.C = Y;
    a1.alpha = 1.0; a1.beta = 0.0; a1.sym = 1; a1.res2 = ns.res2;
    a1.state = ns.state; a1.skip_state = ST_DONE;
    size_t tk1, tk2;
    SM_TRY(timer.start(KC_SIMT, st, &tk1));
    SM_CUDA(gemm(a1, st));
    SM_TRY(timer.stop(tk1, st));
    if (k == 0 && certify) {  // the power estimate's scale, proven from X_0^2 or reduced
      const CertSquare sq{sizeof(T) == 8 ? 0 : 1, Y, nullptr, 1.0f, 0.0f};
      const CertLinear lin{1, {bufs[cur], nullptr, nullptr}, {nullptr, nullptr, nullptr}};
      SM_CUDA(launch_certify(wv.dev, ns, sq, lin, cert_limits(false), max_ld(wv), d_flags + 2, st));
    }
    SM_CUDA(launch_ns_update(wv.dev, ns, tol, floor_thr, opt.max_iter, d_flags, st));
    Args a2 = a1;
    a2.B = Y; a2.C0 = bufs[cur]; a2.C = bufs[cur ^ 1];
    a2.alpha = -0.5; a2.beta = 1.5; a2.res2 = nullptr;
    SM_TRY(timer.start(KC_SIMT, st, &tk2));
    SM_CUDA(gemm(a2, st));
    SM_TRY(timer.stop(tk2, st));
    SM_CUDA(cudaMemsetAsync(d_active, 0, sizeof(int), st));
    SM_CUDA(launch_ns_post(wv.dev, ns, cur ^ 1, d_active, st));
    SM_CUDA(cudaMemcpyAsync(h_pinned, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    SM_CUDA(cudaStreamSynchronize(st));
    cur ^= 1;
    if (reinterpret_cast<int*>(h_pinned)[0] == 0) break;
  }
  return SUBMAT_OK;
}

submat_status Plan::sign_fp64(const double* K, double mu, double* D, cudaStream_t st) {
  double* B0 = static_cast<double*>(ws);
  double* B1 = B0 + ws_elems;
  double* Y = B1 + ws_elems;
  for (auto& wv : waves) {
    SM_CUDA(cudaEventRecord(ev[0], st));
    SM_TRY(gather_wave(wv, K, mu, B0, st));
    SM_CUDA(launch_scale_f64(wv.dev, B0, B0, ns.beta, wv.max_ld2, st));
    if (opt.beta_mode == 0) {
      SM_CUDA(launch_power_f64(wv.dev, B0, kPowerIters, ns.state, ns.rprev, max_ld(wv), st));
      SM_CUDA(launch_rescale_f64(wv.dev, B0, ns.rprev, ns.beta, ns.state, wv.max_ld2, st));
      SM_CUDA(launch_reset_rprev(wv.dev, ns, st));
    }
    SM_CUDA(cudaEventRecord(ev[1], st));
    SM_TRY((ns_simt<double, GemmF64Args>(wv, B0, B1, Y, tol_eff, 1e-9, st, launch_gemm_f64,
                                         opt.beta_mode == 0)));
    SM_CUDA(cudaEventRecord(ev[2], st));
    SM_TRY(scatter_timed(wv, 16.0, [&] { return launch_scatter_f64(g, wv.dev, ns, B0, B1, D, d_trpart, geom(wv), st); },
                         st));
    SM_CUDA(cudaEventRecord(ev[3], st));
    SM_TRY(collect_wave(wv, st));
    SM_TRY(add_phase_times());
  }
  return SUBMAT_OK;
}

submat_status Plan::sign_fp32(const double* K, double mu, double* D, cudaStream_t st) {
  double* A = static_cast<double*>(ws);
  float* B0 = reinterpret_cast<float*>(A + ws_elems);
  float* B1 = B0 + ws_elems;
  float* Y = B1 + ws_elems;
  for (auto& wv : waves) {
    SM_CUDA(cudaEventRecord(ev[0], st));
    SM_TRY(gather_wave(wv, K, mu, A, st));
    SM_CUDA(launch_scale_f32(wv.dev, A, B0, ns.beta, wv.max_ld2, st));
    if (opt.beta_mode == 0) {
      SM_CUDA(launch_power_f32(wv.dev, B0, kPowerIters, ns.state, ns.rprev, max_ld(wv), st));
      SM_CUDA(launch_rescale_f32(wv.dev, B0, ns.rprev, ns.beta, ns.state, wv.max_ld2, st));
      SM_CUDA(launch_reset_rprev(wv.dev, ns, st));
    }
    SM_CUDA(cudaEventRecord(ev[1], st));
    SM_TRY((ns_simt<float, GemmF32Args>(wv, B0, B1, Y, tol_eff, 1e-4, st, launch_gemm_f32,
                                        opt.beta_mode == 0)));
    SM_CUDA(cudaEventRecord(ev[2], st));
    SM_TRY(scatter_timed(wv, 12.0, [&] { return launch_scatter_f32(g, wv.dev, ns, B0, B1, D, d_trpart, geom(wv), st); },
                         st));
    SM_CUDA(cudaEventRecord(ev[3], st));
    SM_TRY(collect_wave(wv, st));
    SM_TRY(add_phase_times());
  }
  return SUBMAT_OK;
}

submat_status Plan::scatter_timed(const Wave& wv, double bytes_per_entry,
                                  const std::function<cudaError_t()>& launch, cudaStream_t st) {
  size_t tk;
  SM_TRY(timer.start(KC_SCATTER, st, &tk));
  SM_CUDA(launch());
  SM_TRY(timer.stop(tk, st));
  if (timer.on)
    for (int s = 0; s < wv.count; ++s)
      stats.kernel_work[KC_SCATTER] += bytes_per_entry * double(wv.host_n[s]) * qext[wv.first + s];
  return SUBMAT_OK;
}

submat_status Plan::add_phase_times() {
  float t01 = 0, t12 = 0, t23 = 0;
  SM_CUDA(cudaEventSynchronize(ev[3]));
  SM_CUDA(cudaEventElapsedTime(&t01, ev[0], ev[1]));
  SM_CUDA(cudaEventElapsedTime(&t12, ev[1], ev[2]));
  SM_CUDA(cudaEventElapsedTime(&t23, ev[2], ev[3]));
  stats.ms_gather += t01;
  stats.ms_ns += t12;
  stats.ms_scatter += t23;
  return SUBMAT_OK;
}

void Plan::reset_stats() {
  std::memset(&stats, 0, sizeof(stats));
  stats.nsub = col_hi - col_lo;
  int nmin = INT32_MAX, nmax = 0;
  double s2 = 0.0, s3 = 0.0;
  for (int j = col_lo; j < col_hi; ++j) {
    const double n = qn[j];
    nmin = std::min(nmin, qn[j]);
    nmax = std::max(nmax, qn[j]);
    s2 += n * n;
    s3 += n * n * n;
  }
  stats.n_min = nmin == INT32_MAX ? 0 : nmin;
  stats.n_max = nmax;
  stats.waves = int(waves.size());
  stats.sum_n2 = s2;
  stats.sum_n3 = s3;
  stats.workspace_bytes = ws_bytes;
  launches_at_start = launch_count();
}

// adjoint: the coupled iteration runs six products per step, 12 n^3 flops at
// the standard count, for the iterations of X plus the two in which E settles
void Plan::finish_stats(bool adjoint) {
  int imin = INT32_MAX, imax = 0, nc = 0;
  double flops = 0.0, rmax = 0.0;
  for (int j = col_lo; j < col_hi; ++j) {
    imin = std::min(imin, res_iters[j]);
    imax = std::max(imax, res_iters[j]);
    nc += res_notconv[j];
    const double n3 = double(qn[j]) * qn[j] * qn[j];
    if (opt.kT > 0.0) flops += (adjoint ? 6.0 : 2.0) * n3 * res_iters[j];  // res_iters: products
    else flops += adjoint ? 12.0 * n3 * (res_iters[j] + 2) : (opt.iteration == 1 ? 6.0 : 4.0) * n3 * res_iters[j];
    rmax = std::max(rmax, res_resid[j]);
  }
  stats.iters_min = imin == INT32_MAX ? 0 : imin;
  stats.iters_max = imax;
  stats.not_converged = nc;
  stats.flops_ns = flops;
  stats.max_resid = rmax;
  stats.launches = launch_count() - launches_at_start;
  if (timer.on) {
    timer.collect(stats.kernel_ms, stats.kernel_launches);
    if (adjoint) {  // every adjoint product runs on one GEMM kind
      stats.kernel_work[opt.adjoint_mode == 1 && opt.kT == 0.0 ? KC_TC_ADJ : KC_SIMT] += flops;
    } else if (opt.kT > 0.0) {
      stats.kernel_work[KC_SIMT] += flops;
    } else if (opt.prec != SUBMAT_MIXED_BF16_REFINE) {
      // two products per iteration, 2 n^3 flops each at the standard count
      for (int j = col_lo; j < col_hi; ++j) {
        const double n = qn[j];
        stats.kernel_work[KC_SIMT] += 4.0 * n * n * n * res_iters[j];
      }
    }
  }
}

// Tile-width autotuner: a warm-up evaluation, then one evaluation with every
// tensor-core phase at width 128 and one at 256, timed per kernel class; each
// phase keeps its faster width.
submat_status Plan::autotune(const double* K, double mu, double* D, int32_t* chosen, cudaStream_t st) {
  if (!K || !D) { set_error("K_vals and D_vals must be device pointers"); return SUBMAT_ERR_INVALID_ARG; }
  if (opt.prec != SUBMAT_MIXED_BF16_REFINE) {
    SM_TRY(sign(K, mu, D, st));
    if (chosen) chosen[0] = chosen[1] = chosen[2] = 0;
    return SUBMAT_OK;
  }
  const bool timer_was_on = timer.on;
  if (gather_bytes.size() != size_t(nblk)) gather_bytes.assign(nblk, 0.0);
  SM_TRY(sign(K, mu, D, st));  // warm-up: maps, state, caches
  timer.on = true;
  const int widths[2] = {128, 256};
  const int classes[3] = {KC_TC_NS, KC_TC_REF, KC_TC_HP};
  double ms[2][3] = {{0, 0, 0}, {0, 0, 0}};
  submat_status status = SUBMAT_OK;
  for (int w = 0; w < 2 && status == SUBMAT_OK; ++w) {
    opt.tile_n_ns = opt.tile_n_corr = opt.tile_n_hp = widths[w];
    status = sign(K, mu, D, st);
    for (int c = 0; c < 3; ++c) ms[w][c] = stats.kernel_ms[classes[c]];
  }
  timer.on = timer_was_on;
  SM_TRY(status);
  const int best[3] = {ms[1][0] < ms[0][0] ? 256 : 128, ms[1][1] < ms[0][1] ? 256 : 128,
                       ms[1][2] < ms[0][2] ? 256 : 128};
  opt.tile_n_ns = best[0];
  opt.tile_n_corr = best[1];
  opt.tile_n_hp = best[2];
  if (chosen)
    for (int c = 0; c < 3; ++c) chosen[c] = best[c];
  return SUBMAT_OK;
}

submat_status Plan::sign(const double* K, double mu, double* D, cudaStream_t st) {
  if (!K || !D) { set_error("K_vals and D_vals must be device pointers"); return SUBMAT_ERR_INVALID_ARG; }
  reset_stats();
  SM_CUDA(cudaMemsetAsync(d_flags, 0, 4 * sizeof(int), st));
  double* Dout = D;
  if (opt.symmetrize) {
    if (!d_symtmp) SM_TRY(alloc(&d_symtmp, size_t(nvals), "symmetrize buffer"));
    Dout = d_symtmp;
  }
  fermi_degree = 0;
  fermi_trunc = fermi_flops = 0.0;
  if (opt.kT > 0.0) {
    if (opt.prec == SUBMAT_FP64) SM_TRY(sign_fermi<double>(K, mu, Dout, st));
    else SM_TRY(sign_fermi<float>(K, mu, Dout, st));
  } else switch (opt.prec) {
    case SUBMAT_FP64: SM_TRY(sign_fp64(K, mu, Dout, st)); break;
    case SUBMAT_FP32: SM_TRY(sign_fp32(K, mu, Dout, st)); break;
    case SUBMAT_MIXED_BF16_REFINE: SM_TRY(sign_mixed(K, mu, Dout, st)); break;
    default: set_error("unknown precision %d", opt.prec); return SUBMAT_ERR_INVALID_ARG;
  }
  if (opt.symmetrize) SM_CUDA(launch_symmetrize_impl(g, nnzb, d_symtmp, D, d_rowof, st));
  SM_CUDA(cudaStreamSynchronize(st));
  finish_stats();
  if (opt.kT > 0.0) {
    stats.poly_degree = fermi_degree;
    stats.poly_trunc = fermi_trunc;
    SM_TRY(fermi_dn_dmu(st, &stats.dn_dmu));
  }
  int fl = 0;
  SM_TRY(read_flags(st, &fl));
  if (fl & FLAG_TIMEOUT) { set_error("a bounded device wait timed out"); return SUBMAT_ERR_TIMEOUT; }
  if (stats.not_converged > 0) {
    set_error("%d submatrices did not converge within %d iterations (D written)",
              stats.not_converged, opt.max_iter);
    return SUBMAT_ERR_NOT_CONVERGED;
  }
  return SUBMAT_OK;
}

submat_status Plan::trace(const double* D, double* tr, cudaStream_t st) {
  if (!D || !tr) { set_error("null argument"); return SUBMAT_ERR_INVALID_ARG; }
  SM_CUDA(launch_trace(g, nblk, D, d_trpart, d_scalar, st));
  SM_CUDA(cudaMemcpyAsync(h_pinned, d_scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
  SM_CUDA(cudaStreamSynchronize(st));
  *tr = reinterpret_cast<double*>(h_pinned)[0];
  return SUBMAT_OK;
}

}  // namespace submat

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

using submat::Plan;

struct submat_plan {
  Plan impl;
};

#define ABI_GUARD(body)                                                   \
  try {                                                                   \
    body                                                                  \
  } catch (const std::bad_alloc&) {                                       \
    submat::set_error("host allocation failed");                          \
    return SUBMAT_ERR_OOM;                                                \
  } catch (...) {                                                         \
    submat::set_error("unexpected host exception");                       \
    return SUBMAT_ERR_INVALID_ARG;                                        \
  }

extern "C" {

void submat_options_default(submat_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->prec = SUBMAT_FP64;
}

static submat_status plan_create_impl(int nblk, const int32_t* block_sizes, const int64_t* row_ptr,
                                      const int32_t* col_idx, const int32_t* groups, const submat_options* opt,
                                      void* stream, submat_plan** out) {
  ABI_GUARD({
    submat::clear_error();
    if (!out) { submat::set_error("out is NULL"); return SUBMAT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (nblk < 1 || !block_sizes || !row_ptr || !col_idx) {
      submat::set_error("nblk must be >= 1 and the pattern arrays non-NULL");
      return SUBMAT_ERR_INVALID_ARG;
    }
    submat_options o;
    submat_options_default(&o);
    if (opt) o = *opt;
    if (o.prec < 0 || o.prec > 2) { submat::set_error("bad precision %d", o.prec); return SUBMAT_ERR_INVALID_ARG; }
    if (o.max_iter < 0 || o.tol < 0.0 || o.refine_rounds < 0) {
      submat::set_error("negative max_iter, tol or refine_rounds");
      return SUBMAT_ERR_INVALID_ARG;
    }
    if ((o.tile_n_ns != 0 && o.tile_n_ns != 128 && o.tile_n_ns != 256) ||
        (o.tile_n_corr != 0 && o.tile_n_corr != 128 && o.tile_n_corr != 256) ||
        (o.tile_n_hp != 0 && o.tile_n_hp != 128 && o.tile_n_hp != 256)) {
      submat::set_error("tile widths must be 0, 128 or 256");
      return SUBMAT_ERR_INVALID_ARG;
    }
    if (o.iteration != 0 && o.iteration != 1) {
      submat::set_error("iteration must be 0 (Newton-Schulz) or 1 (third order)");
      return SUBMAT_ERR_INVALID_ARG;
    }
    if (o.adjoint_mode != 0 && o.adjoint_mode != 1) {
      submat::set_error("adjoint_mode must be 0 (SIMT GEMM) or 1 (tensor cores)");
      return SUBMAT_ERR_INVALID_ARG;
    }
    if (o.adjoint_mode == 1 && o.prec != SUBMAT_MIXED_BF16_REFINE) {
      submat::set_error("the tensor-core adjoint is available on the mixed path only");
      return SUBMAT_ERR_UNSUPPORTED;
    }
    if (o.iteration == 1 && o.prec != SUBMAT_MIXED_BF16_REFINE) {
      submat::set_error("the third-order iteration is available on the mixed path only");
      return SUBMAT_ERR_UNSUPPORTED;
    }
    if (o.col_begin < 0 || o.col_end < 0 || o.col_end > nblk || (o.col_end > 0 && o.col_begin >= o.col_end)) {
      submat::set_error("bad column range [%d, %d) for %d block columns", o.col_begin, o.col_end, nblk);
      return SUBMAT_ERR_INVALID_ARG;
    }
    if (!(o.kT >= 0.0) || !std::isfinite(o.kT)) {
      submat::set_error("kT must be finite and >= 0");
      return SUBMAT_ERR_INVALID_ARG;
    }
    if (o.kT > 0.0 && o.prec == SUBMAT_MIXED_BF16_REFINE) {
      submat::set_error("finite temperature runs on the FP64 and FP32 paths only");
      return SUBMAT_ERR_UNSUPPORTED;
    }
    if (groups && (o.col_end > 0 || o.col_begin > 0)) {
      submat::set_error("column ranges do not apply to grouped plans");
      return SUBMAT_ERR_UNSUPPORTED;
    }
    if (o.max_iter == 0) o.max_iter = 100;
    if (o.refine_rounds == 0) o.refine_rounds = 1;
    submat_status s = submat::validate_pattern_public(nblk, block_sizes, row_ptr, col_idx);
    if (s != SUBMAT_OK) return s;
    std::unique_ptr<submat_plan> p(new submat_plan());
    p->impl.tol_eff = o.tol > 0 ? o.tol : (o.prec == SUBMAT_FP64 ? 1e-14 : (o.prec == SUBMAT_FP32 ? 1e-6 : 2e-5));
    s = p->impl.build(nblk, block_sizes, row_ptr, col_idx, &o, static_cast<cudaStream_t>(stream), groups);
    if (s != SUBMAT_OK) return s;
    *out = p.release();
    return SUBMAT_OK;
  })
}

submat_status submat_plan_create(int nblk, const int32_t* block_sizes, const int64_t* row_ptr,
                                 const int32_t* col_idx, const submat_options* opt, void* stream,
                                 submat_plan** out) {
  return plan_create_impl(nblk, block_sizes, row_ptr, col_idx, nullptr, opt, stream, out);
}

submat_status submat_plan_create_grouped(int nblk, const int32_t* block_sizes, const int64_t* row_ptr,
                                         const int32_t* col_idx, const int32_t* groups,
                                         const submat_options* opt, void* stream, submat_plan** out) {
  if (!groups) {
    submat::set_error("groups is NULL");
    if (out) *out = nullptr;
    return SUBMAT_ERR_INVALID_ARG;
  }
  return plan_create_impl(nblk, block_sizes, row_ptr, col_idx, groups, opt, stream, out);
}

submat_status submat_plan_destroy(submat_plan* plan) {
  ABI_GUARD({
    delete plan;
    return SUBMAT_OK;
  })
}

submat_status submat_sign(submat_plan* plan, const double* K_vals, double mu, double* D_vals,
                          void* stream) {
  ABI_GUARD({
    submat::clear_error();
    if (!plan) { submat::set_error("plan is NULL"); return SUBMAT_ERR_INVALID_ARG; }
    if (!std::isfinite(mu)) { submat::set_error("mu is not finite"); return SUBMAT_ERR_INVALID_ARG; }
    return plan->impl.sign(K_vals, mu, D_vals, static_cast<cudaStream_t>(stream));
  })
}

submat_status submat_autotune(submat_plan* plan, const double* K_vals, double mu, double* D_vals,
                              int32_t* tile_n_out, void* stream) {
  ABI_GUARD({
    submat::clear_error();
    if (!plan) { submat::set_error("plan is NULL"); return SUBMAT_ERR_INVALID_ARG; }
    if (!std::isfinite(mu)) { submat::set_error("mu is not finite"); return SUBMAT_ERR_INVALID_ARG; }
    return plan->impl.autotune(K_vals, mu, D_vals, tile_n_out, static_cast<cudaStream_t>(stream));
  })
}

submat_status submat_sign_host(submat_plan* plan, const double* K_host, double mu, double* D_host,
                               void* stream) {
  ABI_GUARD({
    submat::clear_error();
    if (!plan || !K_host || !D_host) { submat::set_error("null argument"); return SUBMAT_ERR_INVALID_ARG; }
    if (!std::isfinite(mu)) { submat::set_error("mu is not finite"); return SUBMAT_ERR_INVALID_ARG; }
    return plan->impl.sign_host(K_host, mu, D_host, static_cast<cudaStream_t>(stream));
  })
}

submat_status submat_trace(submat_plan* plan, const double* D_vals, double* tr, void* stream) {
  ABI_GUARD({
    submat::clear_error();
    if (!plan) { submat::set_error("plan is NULL"); return SUBMAT_ERR_INVALID_ARG; }
    return plan->impl.trace(D_vals, tr, static_cast<cudaStream_t>(stream));
  })
}

submat_status submat_mu_search(submat_plan* plan, const double* K_vals, double n_el, double mu0,
                               double tol, int max_steps, double* mu_out, double* D_vals,
                               void* stream) {
  ABI_GUARD({
    submat::clear_error();
    if (!plan || !mu_out || !K_vals || !D_vals || max_steps < 1 || !(tol > 0) ||
        !std::isfinite(n_el) || !std::isfinite(mu0)) {
      submat::set_error("bad argument to submat_mu_search");
      return SUBMAT_ERR_INVALID_ARG;
    }
    return plan->impl.mu_search(K_vals, n_el, mu0, tol, max_steps, mu_out, D_vals,
                                static_cast<cudaStream_t>(stream));
  })
}

submat_status submat_sign_backward(submat_plan* plan, const double* K_vals, double mu,
                                   const double* Dbar_vals, double* Kbar_vals, double* dN_dmu,
                                   void* stream) {
  ABI_GUARD({
    submat::clear_error();
    if (!plan || !K_vals || !Dbar_vals || !Kbar_vals || !std::isfinite(mu)) {
      submat::set_error("bad argument to submat_sign_backward");
      return SUBMAT_ERR_INVALID_ARG;
    }
    return plan->impl.backward(K_vals, mu, Dbar_vals, Kbar_vals, dN_dmu,
                               static_cast<cudaStream_t>(stream));
  })
}

int64_t submat_plan_value_count(const submat_plan* plan) { return plan ? plan->impl.nvals : -1; }

submat_status submat_get_stats(const submat_plan* plan, submat_stats* out) {
  if (!plan || !out) { submat::set_error("null argument"); return SUBMAT_ERR_INVALID_ARG; }
  *out = plan->impl.stats;
  return SUBMAT_OK;
}

submat_status submat_get_sub_stats(const submat_plan* plan, int32_t* dims, int32_t* iters,
                                   double* resid, double* beta) {
  if (!plan) { submat::set_error("plan is NULL"); return SUBMAT_ERR_INVALID_ARG; }
  const Plan& p = plan->impl;
  for (int j = 0; j < p.nblk; ++j) {  // block column j reports its submatrix q
    const int q = p.qof[j];
    if (dims) dims[j] = p.qn[q];
    if (iters) iters[j] = p.res_iters[q];
    if (resid) resid[j] = p.res_resid[q];
    if (beta) beta[j] = p.res_beta[q];
  }
  return SUBMAT_OK;
}

const char* submat_last_error(void) { return submat::last_error(); }

}  // extern "C"

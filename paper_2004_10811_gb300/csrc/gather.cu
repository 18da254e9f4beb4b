// Assembly (gather) and extraction (scatter) of the submatrices, Section
// III-A steps 1 and 3, laid out for full-width HBM traffic.
//
// Gather: a_j = K[N(j), N(j)] - mu I as a dense ld x ld row-major buffer.  One
// CTA takes every gridDim.x-th block row t of one submatrix.  A column table
// (local block u, offset inside the block, block size) is built once per CTA;
// per block row a table of K block offsets, one per local block column u, is
// filled from row N(j)[t] of the CSR pattern.  Each warp then writes whole
// rows of a_j with 16-byte stores, reading K in the row runs of its blocks.
//
// Scatter: block column j of D from the rows k_j .. k_j + b_j - 1 of S_j (S_j
// is symmetric, so they hold the wanted columns).  Those rows are staged in
// shared memory chunk by chunk (coalesced reads of S), then every block
// (N(j)[u], j) of D, b_u x b_j row-major and contiguous, is written in order.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace submat {

namespace {

constexpr int kGatherThreads = 256;

__device__ __forceinline__ int find_block(const int* __restrict__ nbr, int nb, int c) {
  int lo = 0, hi = nb - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = nbr[mid];
    if (v == c) return mid;
    if (v < c) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// column info: local block u (bits 0-13), offset inside the block (14-22),
// the block's size (23-31)
__device__ __forceinline__ uint32_t col_info(int u, int cc, int b) {
  return uint32_t(u) | (uint32_t(cc) << 14) | (uint32_t(b) << 23);
}

__global__ void __launch_bounds__(kGatherThreads) k_gather_rows(PatternDev g, WaveDev w,
                                                                const double* __restrict__ K, double mu,
                                                                double* __restrict__ A, NsStateDev ns,
                                                                int* flags, int nb_max, int ld_max) {
  extern __shared__ __align__(16) unsigned char smraw[];
  long long* blkbase = reinterpret_cast<long long*>(smraw);  // [nb_max]
  int* nbr = reinterpret_cast<int*>(blkbase + nb_max);        // [nb_max]
  int* loc = nbr + nb_max;                                     // [nb_max + 1]
  uint32_t* cinfo = reinterpret_cast<uint32_t*>(loc + nb_max + 1);  // [ld_max]
  __shared__ float red_max[kGatherThreads / 32];
  __shared__ double red_fro[kGatherThreads / 32];
  const int s = blockIdx.y;
  const int j = w.sub[s];  // the submatrix (a block column, or a group of them)
  const int64_t rp0 = g.sp[j];
  const int nb = int(g.sp[j + 1] - rp0);
  const int n = w.n[s], ld = w.ld[s];
  double* Aj = A + w.off[s];
  for (int u = threadIdx.x; u < nb; u += blockDim.x) {
    nbr[u] = g.srows[rp0 + u];
    loc[u] = g.sloc[rp0 + u];
  }
  if (threadIdx.x == 0) loc[nb] = n;
  __syncthreads();
  for (int u = threadIdx.x; u < nb; u += blockDim.x) {
    const int c0 = loc[u], b = loc[u + 1] - c0;
    for (int cc = 0; cc < b; ++cc) cinfo[c0 + cc] = col_info(u, cc, b);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float rsmax = 0.0f;  // row sums in FP32 (the FP64 pipe is slow); beta gets a margin
  double fro = 0.0;    // per row in FP32, rows summed in FP64
  bool bad = false;
  for (int t = blockIdx.x; t < nb; t += gridDim.x) {
    __syncthreads();  // cinfo is complete; the previous block row's table is no longer read
    for (int u = threadIdx.x; u < nb; u += blockDim.x) blkbase[u] = -1;
    __syncthreads();
    const int i1 = nbr[t];
    for (int64_t q = g.row_ptr[i1] + threadIdx.x; q < g.row_ptr[i1 + 1]; q += blockDim.x) {
      const int u = find_block(nbr, nb, g.col[q]);
      if (u >= 0) blkbase[u] = static_cast<long long>(g.valptr[q]);
    }
    __syncthreads();
    const int r0 = loc[t], bt = loc[t + 1] - r0;
    for (int rr = warp; rr < bt; rr += nw) {
      const int row = r0 + rr;
      double* arow = Aj + int64_t(row) * ld;
      float rs = 0.0f, rf = 0.0f;
      for (int c2 = 2 * lane; c2 < ld; c2 += 64) {
        double v[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int c = c2 + k;
          double x = 0.0;
          if (c < n) {
            const uint32_t info = cinfo[c];
            const long long b0 = blkbase[info & 0x3FFFu];
            if (b0 >= 0) x = K[b0 + int64_t(rr) * (info >> 23) + ((info >> 14) & 0x1FFu)];
            if (c == row) x -= mu;  // the diagonal
          }
          if (!isfinite(x)) bad = true;
          const float xf = d2f_trunc(x);
          rs += fabsf(xf);
          rf = fmaf(xf, xf, rf);
          v[k] = x;
        }
        *reinterpret_cast<double2*>(arow + c2) = make_double2(v[0], v[1]);
      }
      for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
      rsmax = fmaxf(rsmax, rs);
      fro += double(rf);
    }
  }
  // the padding rows n .. ld - 1 (zero) go to the last CTA of the submatrix
  if (blockIdx.x == gridDim.x - 1)
    for (int row = n + warp; row < ld; row += nw) {
      double* arow = Aj + int64_t(row) * ld;
      for (int c2 = 2 * lane; c2 < ld; c2 += 64) *reinterpret_cast<double2*>(arow + c2) = make_double2(0.0, 0.0);
    }
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if (lane == 0) { red_max[warp] = rsmax; red_fro[warp] = fro; }
  const int anybad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    float m = 0.0f;
    double f = 0.0;
    for (int q = 0; q < nw; ++q) { m = fmaxf(m, red_max[q]); f += red_fro[q]; }
    // the FP32 row sum widened exactly: its bit pattern orders like the value
    if (m > 0.0f) atomicMax(&ns.gersh[s], (unsigned long long)__double_as_longlong(f2d_exact(m)));
    if (f > 0.0) atomicAdd(&ns.fro2[s], f);
    if (anybad) atomicOr(flags, FLAG_NONFINITE);
  }
}

// Block column j of D = 1/2 (I - S_j) restricted to the columns of block j,
// with S_j - (corr_a + corr_b) for the mixed path's last correction (not for
// submatrices in fallback).  Rows koff .. koff + b_j - 1 of S_j are staged per
// chunk of `chunk` columns (stage[c][x], pitch chunk + 1), then the blocks
// (N(j)[u], j) that the chunk's columns cover are written row-major.  The
// trace of the diagonal block goes to trpart[j] and, with sqpart, the sum of
// squares of the extracted entries to sqpart[j].
template <typename T>
__global__ void __launch_bounds__(256) k_scatter_staged(PatternDev g, WaveDev w, NsStateDev ns,
                                                        const T* __restrict__ buf0, const T* __restrict__ buf1,
                                                        double* __restrict__ D, double* trpart,
                                                        const float* __restrict__ corr_a,
                                                        const float* __restrict__ corr_b,
                                                        const int* __restrict__ fallback, double* sqpart,
                                                        int nb_max, int chunk) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* stage = reinterpret_cast<double*>(smraw);          // [bj_max][chunk + 1]
  int* loc = reinterpret_cast<int*>(stage + 0);               // set below
  __shared__ double red[8], red2[8];
  const int s = blockIdx.x;
  const int j = w.sub[s];
  const int64_t rp0 = g.row_ptr[j];
  const int nb = int(g.row_ptr[j + 1] - rp0);
  const int n = w.n[s], ld = w.ld[s];
  const int koff = g.koff[j], bj = g.bs[j];
  const int pitch = chunk + 1;
  loc = reinterpret_cast<int*>(stage + size_t(bj) * pitch);  // [nb_max + 1]
  int* tp = loc + nb_max + 1;                                  // [nb_max] CSR position of block (N(j)[u], j)
  int* ublk = tp + nb_max;                                     // [chunk] local block of each staged column
  for (int u = threadIdx.x; u < nb; u += blockDim.x) {
    loc[u] = g.locoff[rp0 + u];
    tp[u] = g.tpos[rp0 + u];
  }
  if (threadIdx.x == 0) loc[nb] = n;
  const T* S = (ns.par[s] ? buf1 : buf0) + w.off[s];
  const bool correct = corr_a && !fallback[s];
  const float* ca = corr_a ? corr_a + w.off[s] : nullptr;
  const float* cb = corr_b ? corr_b + w.off[s] : nullptr;
  double tr = 0.0, sq = 0.0;
  for (int col0 = 0; col0 < n; col0 += chunk) {
    const int wd = min(chunk, n - col0);
    __syncthreads();  // loc / tp ready; the previous chunk's stage is written out
    for (int x = threadIdx.x; x < wd; x += blockDim.x) {
      const int col = col0 + x;
      int lo = 0, hi = nb - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (loc[mid] <= col) lo = mid; else hi = mid - 1;
      }
      ublk[x] = lo;
    }
    for (int e = threadIdx.x; e < bj * wd; e += blockDim.x) {
      const int c = e / wd, x = e - c * wd;
      const int col = col0 + x;
      const int64_t si = int64_t(koff + c) * ld + col;
      double sv = double(S[si]);
      if (correct) sv -= f2d_exact(ca[si] + cb[si]);
      const bool diag = col == koff + c;
      const double v = (diag ? 0.5 : 0.0) - 0.5 * sv;
      stage[c * pitch + x] = v;
      if (diag) tr += v;
      if (sqpart) sq = fma(v, v, sq);
    }
    __syncthreads();
    if (D) {
      for (int e = threadIdx.x; e < wd * bj; e += blockDim.x) {
        const int x = e / bj, c = e - x * bj;
        const int col = col0 + x;
        const int u = ublk[x];
        const int r = col - loc[u];
        D[g.valptr[tp[u]] + int64_t(r) * bj + c] = stage[c * pitch + x];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
  }
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = tr; red2[threadIdx.x >> 5] = sq; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0, acc2 = 0.0;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) { acc += red[q]; acc2 += red2[q]; }
    trpart[j] = acc;
    if (sqpart) sqpart[j] = acc2;
  }
}

// Grouped submatrices (Section IV-C): block column j of D from the rows
// mkoff .. mkoff + b_j - 1 of its group's S (by symmetry, the columns of
// block j), one CTA per (member, submatrix).  Block (N(j)[u], j) of D takes
// the rows dloc[p] .. of the submatrix, p its CSR position; entries are walked
// in D's order (row-major blocks), reading b_j-long row runs of S.
template <typename T>
__global__ void __launch_bounds__(256) k_scatter_members(PatternDev g, WaveDev w, NsStateDev ns,
                                                         const T* __restrict__ buf0, const T* __restrict__ buf1,
                                                         double* __restrict__ D, double* trpart,
                                                         const float* __restrict__ corr_a,
                                                         const float* __restrict__ corr_b,
                                                         const int* __restrict__ fallback, double* sqpart) {
  extern __shared__ int smi[];
  __shared__ double red[8], red2[8];
  const int s = blockIdx.y;
  const int q = w.sub[s];
  const int m0 = g.mp[q];
  if (int(blockIdx.x) >= g.mp[q + 1] - m0) return;
  const int j = g.mcol[m0 + blockIdx.x];
  const int kq = g.mkoff[m0 + blockIdx.x];
  const int bj = g.bs[j];
  const int ld = w.ld[s];
  const int64_t rp0 = g.row_ptr[j];
  const int nb = int(g.row_ptr[j + 1] - rp0);
  const int nj = g.nsub[j];
  int* locj = smi;            // [nb + 1] offsets of N(j)'s blocks in n_j-space
  int* tp = locj + nb + 1;    // [nb] CSR position of block (N(j)[u], j)
  int* dl = tp + nb;          // [nb] its row offset inside the submatrix
  for (int u = threadIdx.x; u < nb; u += blockDim.x) {
    locj[u] = g.locoff[rp0 + u];
    tp[u] = g.tpos[rp0 + u];
    dl[u] = g.dloc[tp[u]];
  }
  if (threadIdx.x == 0) locj[nb] = nj;
  __syncthreads();
  const T* S = (ns.par[s] ? buf1 : buf0) + w.off[s];
  const bool correct = corr_a && !fallback[s];
  const float* ca = corr_a ? corr_a + w.off[s] : nullptr;
  const float* cb = corr_b ? corr_b + w.off[s] : nullptr;
  double tr = 0.0, sq = 0.0;
  for (int e = threadIdx.x; e < nj * bj; e += blockDim.x) {
    const int x = e / bj, c = e - x * bj;
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (locj[mid] <= x) lo = mid; else hi = mid - 1;
    }
    const int r = x - locj[lo];
    const int row = dl[lo] + r;
    const int64_t si = int64_t(row) * ld + kq + c;
    double sv = double(S[si]);
    if (correct) sv -= f2d_exact(ca[si] + cb[si]);
    const bool diag = row == kq + c;
    const double v = (diag ? 0.5 : 0.0) - 0.5 * sv;
    if (D) D[g.valptr[tp[lo]] + int64_t(r) * bj + c] = v;
    if (diag) tr += v;
    if (sqpart) sq = fma(v, v, sq);
  }
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
  }
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = tr; red2[threadIdx.x >> 5] = sq; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0, acc2 = 0.0;
    for (int k = 0; k < int(blockDim.x >> 5); ++k) { acc += red[k]; acc2 += red2[k]; }
    trpart[j] = acc;
    if (sqpart) sqpart[j] = acc2;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_scatter_members(const PatternDev& g, const WaveDev& w, NsStateDev ns, const T* buf0,
                                   const T* buf1, double* D, double* trpart, int nbj_max, int members_max,
                                   cudaStream_t st, const float* corr_a, const float* corr_b, const int* fallback,
                                   double* sqpart) {
  if (w.nsub <= 0) return cudaSuccess;
  const size_t smem = size_t(3 * nbj_max + 1) * sizeof(int);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_scatter_members<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(smem));
    if (e != cudaSuccess) return e;
  }
  k_scatter_members<T><<<dim3(unsigned(members_max), unsigned(w.nsub)), 256, smem, st>>>(
      g, w, ns, buf0, buf1, D, trpart, corr_a, corr_b, fallback, sqpart);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_scatter_members<double>(const PatternDev&, const WaveDev&, NsStateDev, const double*,
                                                    const double*, double*, double*, int, int, cudaStream_t,
                                                    const float*, const float*, const int*, double*);
template cudaError_t launch_scatter_members<float>(const PatternDev&, const WaveDev&, NsStateDev, const float*,
                                                   const float*, double*, double*, int, int, cudaStream_t,
                                                   const float*, const float*, const int*, double*);

// Gather through k_gather_rows when its tables fit in shared memory (block
// sizes below 512, as every workload here); the caller falls back otherwise.
bool gather_rows_fits(int nb_max, int ld_max, int bs_max) {
  const size_t smem = size_t(nb_max) * 8 + size_t(2 * nb_max + 1) * 4 + size_t(ld_max) * 4;
  return bs_max < 512 && smem <= 200 * 1024;
}

cudaError_t launch_gather_rows(const PatternDev& g, const WaveDev& w, int nb_max, int ld_max, const double* K,
                               double mu, double* A, NsStateDev ns, int* flags, cudaStream_t st) {
  if (w.nsub <= 0) return cudaSuccess;
  const size_t smem = size_t(nb_max) * 8 + size_t(2 * nb_max + 1) * 4 + size_t(ld_max) * 4;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_gather_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  // about 128 rows of a_j per CTA
  int gx = (ld_max + 127) / 128;
  if (gx > nb_max) gx = nb_max;
  if (gx < 1) gx = 1;
  k_gather_rows<<<dim3(unsigned(gx), unsigned(w.nsub)), kGatherThreads, smem, st>>>(g, w, K, mu, A, ns, flags,
                                                                                      nb_max, ld_max);
  count_launch();
  return cudaGetLastError();
}

int scatter_chunk(int ld_max, int bs_max) {
  int chunk = (48 * 1024) / (8 * bs_max) - 1;  // stage of about 48 KB
  if (chunk > ld_max) chunk = ld_max;
  if (chunk < 32) chunk = 32;
  return chunk;
}

size_t scatter_staged_smem(int nb_max, int ld_max, int bs_max) {
  const int chunk = scatter_chunk(ld_max, bs_max);
  return size_t(bs_max) * (chunk + 1) * 8 + size_t(2 * nb_max + 1) * 4 + size_t(chunk) * 4;
}

template <typename T>
cudaError_t launch_scatter_staged(const PatternDev& g, const WaveDev& w, NsStateDev ns, const T* buf0,
                                  const T* buf1, double* D, double* trpart, int nb_max, int ld_max, int bs_max,
                                  cudaStream_t st, const float* corr_a, const float* corr_b, const int* fallback,
                                  double* sqpart) {
  if (w.nsub <= 0) return cudaSuccess;
  const int chunk = scatter_chunk(ld_max, bs_max);
  const size_t smem = scatter_staged_smem(nb_max, ld_max, bs_max);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_scatter_staged<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(smem));
    if (e != cudaSuccess) return e;
  }
  k_scatter_staged<T><<<w.nsub, 256, smem, st>>>(g, w, ns, buf0, buf1, D, trpart, corr_a, corr_b, fallback, sqpart,
                                                  nb_max, chunk);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_scatter_staged<double>(const PatternDev&, const WaveDev&, NsStateDev, const double*,
                                                   const double*, double*, double*, int, int, int, cudaStream_t,
                                                   const float*, const float*, const int*, double*);
template cudaError_t launch_scatter_staged<float>(const PatternDev&, const WaveDev&, NsStateDev, const float*,
                                                  const float*, double*, double*, int, int, int, cudaStream_t,
                                                  const float*, const float*, const int*, double*);

}  // namespace submat

// Grouped BF16 tensor-core GEMM for sm_103a: tcgen05.mma with TMEM
// accumulators, operands staged by TMA (cp.async.bulk.tensor, 128B swizzle),
// an mbarrier pipeline, and one persistent CTA per SM.
//
// Every work item is one 128x128 output tile (s, ti, tj) of
//     C_s = alpha * sum_p A_{a(p)} B_{b(p)}^T + beta * C0_s
// over the submatrix batch.  Operands are row-major n x n BF16 arrays stored
// per size bucket as [count][ld][ld]; B is read as rows (B^T with K major),
// which equals B for the symmetric operands of Newton-Schulz.  A product table
// lets one launch sum several slice products into the FP32 accumulator, e.g.
// the three-term split hi*hi + hi*lo + lo*hi that carries about 16 bits
// through the tensor cores.
//
// Roles (192 threads): warp 0 issues TMA loads, warp 1 owns TMEM and one of
// its lanes issues the MMAs, warps 2-5 drain the accumulator (one TMEM lane
// quarter each) and write the tile -- and, for symmetric outputs, its mirror
// through a shared-memory transpose.  Every mbarrier wait is bounded; on
// timeout the kernel raises FLAG_TIMEOUT, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tc_gemm.cuh"

namespace submat {

namespace {

constexpr int BM = 128, BK = 64;
constexpr int TILE_BYTES = BM * BK * 2;  // one 128 x 64 BF16 operand tile (A side)
constexpr int STG_PITCH = 33;            // staged row pitch (32-bit words)
// integer outputs: one 16-column int64 row segment per thread, rows 144 bytes
// apart (16-byte aligned for the bulk copy, padded against bank conflicts);
// the buffer doubles as the 32-bit transpose stage of the mirror
constexpr int I64_SEG = 16, I64_PITCH = 144;
constexpr int STG_BYTES = (BM * I64_PITCH > BM * STG_PITCH * 4) ? BM * I64_PITCH : BM * STG_PITCH * 4;

// instruction descriptor: D F32, A and B BF16, both K-major, M = 128, N = BN
// (FP16 operands clear the two format fields, bits 7-9 and 10-12)
template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false on timeout or when another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// K-major operand tile with 128-byte swizzle: rows of 128 bytes, 8-row
// groups 1024 bytes apart; the tile base is 1024-byte aligned.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);   // start address
  d |= uint64_t(1) << 16;                    // leading byte offset (unused here)
  d |= uint64_t(1024 >> 4) << 32;            // stride byte offset: 8 rows
  d |= uint64_t(1) << 46;                    // descriptor version
  d |= uint64_t(2) << 61;                    // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                          uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(accum));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_split(float o) {
  const __nv_bfloat16 h = __float2bfloat16_rn(o);
  const __nv_bfloat16 l = __float2bfloat16_rn(o - __bfloat162float(h));
  return uint32_t(__bfloat16_as_ushort(h)) | (uint32_t(__bfloat16_as_ushort(l)) << 16);
}

// two values as (hi, lo) BF16 pairs: hi = rn(v), lo = rn(v - hi), two
// values per conversion instruction; bit-identical to pack_split
__device__ __forceinline__ void pack_split2(float a, float b, uint32_t* hw, uint32_t* lw) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  *hw = *reinterpret_cast<const uint32_t*>(&h);
  *lw = *reinterpret_cast<const uint32_t*>(&l);
}

// the FP16 forms of the two above (operands in FP16: TcGemmParams::f16)
__device__ __forceinline__ uint32_t pack_split_h(float o) {
  const __half h = __float2half_rn(o);
  const __half l = __float2half_rn(o - __half2float(h));
  return uint32_t(__half_as_ushort(h)) | (uint32_t(__half_as_ushort(l)) << 16);
}

__device__ __forceinline__ void pack_split2_h(float a, float b, uint32_t* hw, uint32_t* lw) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  *hw = *reinterpret_cast<const uint32_t*>(&h);
  *lw = *reinterpret_cast<const uint32_t*>(&l);
}

// one 32-byte store (a full L2 sector); the address is 32-byte aligned
__device__ __forceinline__ void st_v8(void* d, const uint32_t* w) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(d), "r"(w[0]), "r"(w[1]),
               "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
}

// write 32 values (one row segment, 64-byte aligned) in the output format,
// in whole 32-byte sectors
template <bool F16>
__device__ __forceinline__ void store_row(const TcGemmParams& p, int64_t idx, const float* o) {
  if (p.out_f32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) st_v8(p.out_f32 + idx + 8 * q, reinterpret_cast<const uint32_t*>(o + 8 * q));
  } else {
    uint32_t hw[16], lw[16];
    if constexpr (F16) {
#pragma unroll
      for (int q = 0; q < 16; ++q) pack_split2_h(o[2 * q], o[2 * q + 1], &hw[q], &lw[q]);
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) pack_split2(o[2 * q], o[2 * q + 1], &hw[q], &lw[q]);
    }
    st_v8(p.out_hi + idx, hw);
    st_v8(p.out_hi + idx + 16, hw + 8);
    if (p.out_lo) {
      st_v8(p.out_lo + idx, lw);
      st_v8(p.out_lo + idx + 16, lw + 8);
    }
  }
}

// store o[q] for q in [q_lo, q_hi) only (diagonal tiles of symmetric outputs):
// whole segments as vectors, element stores only where the diagonal crosses
template <bool F16>
__device__ __forceinline__ void store_range(const TcGemmParams& p, int64_t idx, const float* o,
                                            int q_lo, int q_hi) {
  if (q_lo >= 32 || q_hi <= 0 || q_lo >= q_hi) return;
  if (q_lo <= 0 && q_hi >= 32) {
    store_row<F16>(p, idx, o);
    return;
  }
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    if (q < q_lo || q >= q_hi) continue;
    if (p.out_f32) {
      p.out_f32[idx + q] = o[q];
    } else {
      const uint32_t w = F16 ? pack_split_h(o[q]) : pack_split(o[q]);
      p.out_hi[idx + q] = __ushort_as_bfloat16(static_cast<unsigned short>(w & 0xFFFFu));
      if (p.out_lo) p.out_lo[idx + q] = __ushort_as_bfloat16(static_cast<unsigned short>(w >> 16));
    }
  }
}

template <bool F16>
__device__ __forceinline__ void load_c0(const TcGemmParams& p, int64_t idx, float* c) {
  if (p.c0_f32) {
    // whole 32-byte sectors per load
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t w[8];
      asm volatile("ld.global.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
                     "=r"(w[7])
                   : "l"(p.c0_f32 + idx + 8 * q));
#pragma unroll
      for (int e = 0; e < 8; ++e) c[8 * q + e] = __uint_as_float(w[e]);
    }
  } else {
    const uint4* sh = reinterpret_cast<const uint4*>(p.c0_hi + idx);
    const uint4* sl = p.c0_lo ? reinterpret_cast<const uint4*>(p.c0_lo + idx) : nullptr;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 h = sh[q];
      const uint4 l = sl ? sl[q] : make_uint4(0, 0, 0, 0);
      const uint32_t hh[4] = {h.x, h.y, h.z, h.w}, ll[4] = {l.x, l.y, l.z, l.w};
      if constexpr (F16) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 fh = __half22float2(*reinterpret_cast<const __half2*>(&hh[e]));
          const float2 fl = __half22float2(*reinterpret_cast<const __half2*>(&ll[e]));
          c[8 * q + 2 * e] = fh.x + fl.x;
          c[8 * q + 2 * e + 1] = fh.y + fl.y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          c[8 * q + 2 * e] = __uint_as_float(hh[e] << 16) + __uint_as_float(ll[e] << 16);
          c[8 * q + 2 * e + 1] =
              __uint_as_float(hh[e] & 0xFFFF0000u) + __uint_as_float(ll[e] & 0xFFFF0000u);
        }
      }
    }
  }
}

// LEAN: the launch has one accumulator, a BF16-pair or FP32 output, no
// mirror and double-buffered TMEM (the host checks), and the epilogue drains
// it 32 columns at a time; the general epilogue is not compiled in.
template <int BN, bool LEAN, bool F16>
__global__ void __launch_bounds__(192, 1) k_tc_gemm(const __grid_constant__ TcGemmParams p) {
  constexpr int TILE_B = BN * BK * 2;  // one BN x 64 BF16 operand tile (B side)
  constexpr int HALVES = BN / 128;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int stage_bytes = p.na * TILE_BYTES + p.nb * TILE_B;
  uint8_t* tiles = smem;
  uint32_t* stg = reinterpret_cast<uint32_t*>(tiles + size_t(p.nstage) * stage_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(stg) + STG_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + p.nstage;
  uint64_t* tfull = empty + p.nstage;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* epi_ok = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < p.nstage; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], BM);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(uint32_t(p.tmem_cols)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const long long limit = p.timeout_cycles;
  // accumulator sets in TMEM: two (MMA of the next tile overlaps the drain of
  // this one) when they fit, else one (freed as soon as the epilogue has read it)
  const int nbuf = p.tmem_cols >= 2 * p.nacc * BN ? 2 : 1;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    for (int m = 0; m < p.nmaps; ++m)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&p.maps[m])) : "memory");
    int stage = 0;
    uint32_t phase = 0;
    uint32_t issued = 0, issued_phase = 0;  // per-stage bits
    bool ok = true;
    for (int it = blockIdx.x; it < p.nitems && ok; it += gridDim.x) {
      const int4 item = p.items[it];
      if (p.state && p.state[item.x] == p.skip_state) continue;
      const int bucket = item.w & 0xFF, slot = item.w >> 8;
      const int nk = p.ld[item.x] / BK;
      const CUtensorMap* mapsa = p.maps + bucket;
      const CUtensorMap* mapsb = (BN == 128 ? p.maps : p.maps_b) + bucket;
      for (int kb = 0; kb < nk; ++kb) {
        if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, limit)) { ok = false; break; }
        uint8_t* st = tiles + size_t(stage) * stage_bytes;
        mbar_expect_tx(&full[stage], uint32_t(stage_bytes));
        for (int a = 0; a < p.na; ++a)
          tma_load_3d(st + a * TILE_BYTES, mapsa + p.a_set[a] * p.nbucket, &full[stage], kb * BK,
                      item.y * BM, slot);
        for (int b = 0; b < p.nb; ++b)
          tma_load_3d(st + p.na * TILE_BYTES + b * TILE_B, mapsb + p.b_set[b] * p.nbucket,
                      &full[stage], kb * BK, item.z * BN, slot);
        issued |= 1u << stage;
        issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
        if (++stage == p.nstage) { stage = 0; phase ^= 1u; }
      }
    }
    if (!ok) {
      atomicOr(p.flags, FLAG_TIMEOUT);
      *abort_flag = 1;
      // let this CTA's copies in flight land before shared memory is released
      for (int i = 0; i < p.nstage; ++i)
        if (issued & (1u << i)) {
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[i], (issued_phase >> i) & 1u) && clock64() - t0 < limit) {
          }
        }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int stage = 0;
    uint32_t phase = 0;
    int tcount = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < p.nitems && ok; it += gridDim.x) {
      const int4 item = p.items[it];
      if (p.state && p.state[item.x] == p.skip_state) continue;
      const int nk = p.ld[item.x] / BK;
      const int ab = nbuf == 2 ? (tcount & 1) : 0;
      const uint32_t tph = nbuf == 2 ? (uint32_t(tcount >> 1) & 1u) : (uint32_t(tcount) & 1u);
      if (!mbar_wait(&tempty[ab], tph ^ 1u, abort_flag, limit)) { ok = false; break; }
      tc_fence_after();
      const uint32_t dbase = tmem_base + uint32_t(ab * p.nacc * BN);
      // symmetric output, 256-wide tile whose left 128 columns lie below the
      // diagonal (odd row block): only the right half is wanted, so the MMAs
      // run at N = 128 on B rows 128..255 into accumulator columns 128..255
      const bool half = BN == 256 && p.sym && item.z * 2 < item.y;
      // operand format: BF16 (A and B fields 1) or FP16 (both 0)
      const uint32_t id = (half ? idesc<128>() : idesc<BN>()) & (F16 ? ~((7u << 7) | (7u << 10)) : ~0u);
      const uint32_t boff = half ? uint32_t(128 * BK * 2) : 0u;
      const uint32_t doff = half ? 128u : 0u;
      for (int kb = 0; kb < nk; ++kb) {
        if (!mbar_wait(&full[stage], phase, abort_flag, limit)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sb = smem_u32(tiles + size_t(stage) * stage_bytes);
        for (int pr = 0; pr < p.nprod; ++pr) {
          const uint64_t ad = sdesc(sb + uint32_t(p.prod_a[pr] * TILE_BYTES));
          const uint64_t bd = sdesc(sb + uint32_t(p.na * TILE_BYTES + p.prod_b[pr] * TILE_B) + boff);
          const uint32_t d = dbase + uint32_t(p.prod_acc[pr] * BN) + doff;
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)
            umma_bf16(d, ad + uint64_t(2 * k), bd + uint64_t(2 * k), id,
                      (kb > 0 || k > 0 || !p.prod_first[pr]) ? 1u : 0u);
        }
        umma_commit(&empty[stage]);
        if (++stage == p.nstage) { stage = 0; phase ^= 1u; }
      }
      if (!ok) break;
      umma_commit(&tfull[ab]);
      ++tcount;
    }
    if (!ok) {
      atomicOr(p.flags, FLAG_TIMEOUT);
      *abort_flag = 1;
    }
    // every MMA issued by this thread has completed once this commit lands
    umma_commit(drain);
    const long long t0 = clock64();
    while (!mbar_try_wait(drain, 0) && clock64() - t0 < limit) {
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;  // tile row == TMEM lane
    int tcount = 0;
    for (int it = blockIdx.x; it < p.nitems; it += gridDim.x) {
      const int4 item = p.items[it];
      const int s = item.x;
      if (p.state && p.state[s] == p.skip_state) continue;
      const int ab = nbuf == 2 ? (tcount & 1) : 0;
      const uint32_t tph = nbuf == 2 ? (uint32_t(tcount >> 1) & 1u) : (uint32_t(tcount) & 1u);
      // one bounded wait, result shared, so the four warps leave together
      if (threadIdx.x == 64) {
        const bool got = mbar_wait(&tfull[ab], tph, abort_flag, limit);
        if (!got) {
          atomicOr(p.flags, FLAG_TIMEOUT);
          *abort_flag = 1;
        }
        *epi_ok = got ? 1 : 0;
      }
      epi_bar();
      if (!*epi_ok) break;
      tc_fence_after();
      ++tcount;
      const int ld = p.ld[s];
      const int n = p.n[s];
      const int64_t base = p.off[s];
      const int rg = item.y * BM + r;
      double part = 0.0;
      const uint32_t tbase = tmem_base + (uint32_t(quarter * 32) << 16) + uint32_t(ab * p.nacc * BN);
      // Lean path for the common launches (one accumulator, BF16-pair or FP32
      // output, no mirror, double-buffered TMEM): 32 columns at a time, so
      // only one chunk is live in registers, and the diagonal handled only
      // on diagonal sub-tiles.  TMEM is released after its last read.
      if constexpr (LEAN) {
        if (p.out_i64) {
          // exact integer sums of slice products (full tiles): per 32-column
          // chunk the sum over the accumulators of acc_k * 2^shift_k in 64-bit
          // integers (|acc_k| < 2^24, shift_k <= 36, at most four terms),
          // handed to the L2 bulk add in 16-column row segments
          const uint32_t tb = tbase;
#pragma unroll 1
          for (int c = 0; c < 4 * HALVES; ++c) {
            long long v[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = 0;
#pragma unroll 1
            for (int k = 0; k < p.nacc; ++k) {
              float a[32];
              tmem_ld32(tb + uint32_t(k * BN + c * 32), a);
              tmem_wait_ld();
              const int sh = p.i64_shifts[k];
#pragma unroll
              for (int q = 0; q < 32; ++q) v[q] += (long long)__float2int_rn(a[q]) << sh;
            }
            if (c == 4 * HALVES - 1) {
              tc_fence_before();
              if (!p.test_skip_arrive) mbar_arrive(&tempty[ab]);
            }
            const int cg0 = item.z * BN + c * 32;
            if (rg >= ld || cg0 >= ld) continue;
            uint8_t* srow = reinterpret_cast<uint8_t*>(stg) + r * I64_PITCH;
#pragma unroll
            for (int seg = 0; seg < 32 / I64_SEG; ++seg) {
              asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
#pragma unroll
              for (int q = 0; q < I64_SEG; ++q)
                *reinterpret_cast<long long*>(srow + 8 * q) = v[seg * I64_SEG + q];
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
              long long* d = p.out_i64 + base + int64_t(rg) * ld + cg0 + seg * I64_SEG;
              if (p.i64_accumulate)
                asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;" ::"l"(d),
                             "r"(smem_u32(srow)), "n"(I64_SEG * 8)
                             : "memory");
              else
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(d),
                             "r"(smem_u32(srow)), "n"(I64_SEG * 8)
                             : "memory");
              asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
          }
        } else
        for (int h = 0; h < HALVES; ++h) {
          const int sub_tj = item.z * HALVES + h;
          const bool last_h = h == HALVES - 1;
          if (p.sym && sub_tj < item.y) {  // below the diagonal: not written
            if (last_h) {
              tc_fence_before();
              if (!p.test_skip_arrive) mbar_arrive(&tempty[ab]);
            }
            continue;
          }
          const bool dtile = item.y == sub_tj;  // the diagonal crosses this sub-tile
          const bool diag_sym = p.sym && dtile;
          const double res_weight = (p.sym && !diag_sym) ? 2.0 : 1.0;
          const uint32_t tb = tbase + uint32_t(h * 128);
#pragma unroll 1
          for (int c = 0; c < 4; ++c) {
            float a[32];
            tmem_ld32(tb + uint32_t(c * 32), a);
            tmem_wait_ld();
            if (last_h && c == 3) {
              tc_fence_before();
              if (!p.test_skip_arrive) mbar_arrive(&tempty[ab]);
            }
            const int cg0 = sub_tj * 128 + c * 32;
            if (rg >= ld || cg0 >= ld) continue;
            const int64_t idx = base + int64_t(rg) * ld + cg0;
            const bool has_c0 = (p.c0_f32 || p.c0_hi) && p.beta != 0.0f && !p.dot_c0;
            float c0[32];
            if (has_c0 || p.dot_c0) load_c0<F16>(p, idx, c0);
            float o[32];
            float pr = 0.0f, pd = 0.0f;
            if (!dtile) {
#pragma unroll
              for (int q = 0; q < 32; ++q) {
                float v = p.alpha * a[q];
                if (has_c0) v = fmaf(p.beta, c0[q], v);
                o[q] = v;
                pr = fmaf(a[q], a[q], pr);
                if (p.dot_c0) pd = fmaf(v, c0[q], pd);
              }
            } else {
              const int dq = (rg < n) ? rg - cg0 : -1;  // diagonal position in this segment
#pragma unroll
              for (int q = 0; q < 32; ++q) {
                float v = p.alpha * a[q];
                if (has_c0) v = fmaf(p.beta, c0[q], v);
                if (q == dq) v += p.diag;
                o[q] = v;
                const float e = a[q] - ((q == dq) ? 1.0f : 0.0f);
                pr = fmaf(e, e, pr);
                if (p.dot_c0) pd = fmaf(v, c0[q], pd);
              }
            }
            if (p.res2) part += res_weight * double(pr);
            if (p.dot_c0) part += 2.0 * double(pd);
            if (diag_sym) store_range<F16>(p, idx, o, r - c * 32, 32);
            else store_row<F16>(p, idx, o);
          }
        }
      } else {
      for (int h = 0; h < HALVES; ++h) {
      float acc[128];
      const uint32_t tb = tbase + uint32_t(h * 128);
#pragma unroll
      for (int c = 0; c < 4; ++c) tmem_ld32(tb + uint32_t(c * 32), acc + c * 32);
      tmem_wait_ld();
      if (p.out_i64 && p.nacc == 2) {
        // two exact integer accumulators of adjacent levels: acc0 * 2^d + acc1
        // (|acc| < 2^24, d <= 6: the sum fits in 31 bits), kept as int bits
        float tmp[32];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          tmem_ld32(tb + uint32_t(BN + c * 32), tmp);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 32; ++q)
            acc[c * 32 + q] = __int_as_float(__float2int_rn(acc[c * 32 + q]) * (1 << p.i64_dshift) +
                                             __float2int_rn(tmp[q]));
        }
      } else {
        for (int a = 1; a < p.nacc; ++a) {
          float tmp[32];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            tmem_ld32(tb + uint32_t(a * BN + c * 32), tmp);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[c * 32 + q] += tmp[q];
          }
        }
      }
      if (h == HALVES - 1) {
        tc_fence_before();
        if (!p.test_skip_arrive) mbar_arrive(&tempty[ab]);
      }
      // this half is the 128 x 128 sub-tile (item.y, sub_tj) of C
      const int sub_tj = item.z * HALVES + h;
      // symmetric output: sub-tiles below the diagonal are not written, those
      // above it are mirrored, diagonal ones keep their upper triangle and take
      // the strict lower one from it, so C is exactly symmetric whatever the
      // accumulation order
      if (p.sym && sub_tj < item.y) continue;
      const bool diag_sym = p.sym && item.y == sub_tj;
      const bool mirror = p.sym != 0 && !p.upper_only;
      const double res_weight = (p.sym && !diag_sym) ? 2.0 : 1.0;  // the mirror counts too
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int cg0 = sub_tj * 128 + c * 32;
        float o[32];
        const bool inside = (rg < ld) && (cg0 < ld);
        if (p.out_i64) {
          // exact integer sums of slice products, accumulated in 64-bit integers
          // (full tiles only: no mirror, no diagonal mask).  Each 16-column row
          // segment is staged in shared memory and handed to a bulk copy (first
          // product) or a bulk add in L2 (later ones): no loads on the SM.
          if (inside) {
            const long long mul = 1LL << p.i64_shift;
            uint8_t* srow = reinterpret_cast<uint8_t*>(stg) + r * I64_PITCH;
#pragma unroll
            for (int seg = 0; seg < 32 / I64_SEG; ++seg) {
              // the previous bulk operation of this thread has read its source
              asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
#pragma unroll
              for (int q = 0; q < I64_SEG; ++q) {
                const float x = acc[c * 32 + seg * I64_SEG + q];
                const long long v = (long long)(p.nacc == 2 ? __float_as_int(x) : __float2int_rn(x)) * mul;
                *reinterpret_cast<long long*>(srow + 8 * q) = v;
              }
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
              long long* d = p.out_i64 + base + int64_t(rg) * ld + cg0 + seg * I64_SEG;
              if (p.i64_accumulate)
                asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;" ::"l"(d),
                             "r"(smem_u32(srow)), "n"(I64_SEG * 8)
                             : "memory");
              else
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(d),
                             "r"(smem_u32(srow)), "n"(I64_SEG * 8)
                             : "memory");
              asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
          }
          continue;
        }
        if (inside) {
          float c0[32];
          const int64_t idx = base + int64_t(rg) * ld + cg0;
          const bool has_c0 = (p.c0_f32 || p.c0_hi) && p.beta != 0.0f && !p.dot_c0;
          if (has_c0 || p.dot_c0) load_c0<F16>(p, idx, c0);
          const int dq = (rg < n) ? rg - cg0 : -1;  // diagonal position in this segment
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            float v = p.alpha * acc[c * 32 + q];
            if (has_c0) v = fmaf(p.beta, c0[q], v);
            if (q == dq) v += p.diag;
            o[q] = v;
          }
          if (p.dot_c0) {
            float pc = 0.0f;
#pragma unroll
            for (int q = 0; q < 32; ++q) pc = fmaf(o[q], c0[q], pc);
            part += 2.0 * double(pc);
          }
          if (p.res2) {
            float pc = 0.0f;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              const int cg = cg0 + q;
              const float e = acc[c * 32 + q] - ((rg == cg && rg < n) ? 1.0f : 0.0f);
              pc = fmaf(e, e, pc);
            }
            part += res_weight * double(pc);
          }
          if (diag_sym) store_range<F16>(p, idx, o, r - c * 32, 32);
          else store_row<F16>(p, idx, o);
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) o[q] = 0.0f;
        }
        if (mirror) {
          // transpose the 128 x 32 chunk through shared memory; column q of
          // row r sits at q ^ 8 (r / 32), so that the row writes and the column
          // reads below both hit 32 distinct banks
#pragma unroll
          for (int q = 0; q < 32; ++q) stg[r * STG_PITCH + (q ^ (8 * quarter))] = __float_as_uint(o[q]);
          epi_bar();
          const int t = threadIdx.x - 64;
          const int q = t >> 2, part4 = t & 3;
          const int mrow = sub_tj * 128 + c * 32 + q;       // row of the mirrored tile
          const int mcol0 = item.y * BM + part4 * 32;      // its first column
          if (mrow < ld && mcol0 < ld) {
            float w[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) w[i] = __uint_as_float(stg[(part4 * 32 + i) * STG_PITCH + (q ^ (8 * part4))]);
            if (diag_sym) store_range<F16>(p, base + int64_t(mrow) * ld + mcol0, w, 0, c * 32 + q - part4 * 32);
            else store_row<F16>(p, base + int64_t(mrow) * ld + mcol0, w);
          }
          epi_bar();
        }
      }
      }  // halves
      }  // general epilogue
      if (p.res2 || p.dot_c0) {
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o2);
        if (lane == 0 && part != 0.0) atomicAdd(p.res2 ? &p.res2[s] : &p.dot_c0[s], part);
      }
    }
    // bulk copies and adds issued by this thread are complete and visible
    if (p.out_i64) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(uint32_t(p.tmem_cols)));
  }
}

}  // namespace

int tc_smem_bytes(int na, int nb, int nstage, int bn) {
  return 1024 + nstage * (na * TILE_BYTES + nb * bn * BK * 2) + STG_BYTES + (2 * nstage + 5) * 8 +
         32;
}

int tc_pick_stages(int na, int nb, int bn) {
  const int budget = 227 * 1024;
  int st = 6;
  while (st > 2 && tc_smem_bytes(na, nb, st, bn) > budget) --st;
  return st;
}

cudaError_t launch_tc_gemm(const TcGemmParams& p, int grid, cudaStream_t st) {
  if (p.nitems <= 0) return cudaSuccess;
  const int bn = p.bn == 256 ? 256 : 128;
  if (bn == 256 && (p.tmem_cols != 512 || !p.maps_b || !(p.nacc == 1 || (p.nacc == 2 && p.out_i64))))
    return cudaErrorInvalidValue;
  if (p.nacc * bn > p.tmem_cols) return cudaErrorInvalidValue;
  if (p.out_i64 && p.sym) return cudaErrorInvalidValue;  // integer outputs: full tiles only
  // the lean epilogue combines up to four integer accumulators in 64 bits
  // (weights 2^i64_shifts[k]); the general one two in 32 bits (d <= 6)
  const bool lean_i64 = p.out_i64 && !p.sym && p.nacc <= 4 && p.nacc * bn <= p.tmem_cols &&
                        (p.nacc > 2 ? bn == 128 : p.tmem_cols >= 2 * p.nacc * bn);
  if (p.out_i64 && !lean_i64 && (p.nacc > 2 || (p.nacc == 2 && (p.i64_dshift < 0 || p.i64_dshift > 6))))
    return cudaErrorInvalidValue;
  if (p.out_i64)
    for (int k = 0; k < p.nacc; ++k)
      if (lean_i64 && (p.i64_shifts[k] < 0 || p.i64_shifts[k] > 36)) return cudaErrorInvalidValue;
  const int smem = tc_smem_bytes(p.na, p.nb, p.nstage, bn);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  // the lean epilogue: one accumulator, double-buffered in TMEM, BF16-pair or
  // FP32 output without a mirror
  const bool lean = (p.out_i64 ? lean_i64
                                : p.tmem_cols >= 2 * bn && p.nacc == 1 && !(p.sym && !p.upper_only) &&
                                      (p.out_f32 || p.out_hi));
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 192, smem, st>>>(p);
    return cudaSuccess;
  };
  // FP16 operands: lean launches only (the Newton-Schulz products)
  if (p.f16 && !lean) return cudaErrorInvalidValue;
  cudaError_t e;
  if (bn == 256)
    e = p.f16 ? run(k_tc_gemm<256, true, true>)
              : (lean ? run(k_tc_gemm<256, true, false>) : run(k_tc_gemm<256, false, false>));
  else
    e = p.f16 ? run(k_tc_gemm<128, true, true>)
              : (lean ? run(k_tc_gemm<128, true, false>) : run(k_tc_gemm<128, false, false>));
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// tensor maps
// ---------------------------------------------------------------------------

typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encoder() {
  static PFN_encodeTiled fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled>(ptr);
  }
  return fn;
}

int make_bucket_map(CUtensorMap* out, const void* base, int ld, int count, int box_rows) {
  PFN_encodeTiled enc = get_encoder();
  if (!enc) return -1;
  const cuuint64_t dims[3] = {cuuint64_t(ld), cuuint64_t(ld), cuuint64_t(count)};
  const cuuint64_t strides[2] = {cuuint64_t(ld) * 2, cuuint64_t(ld) * ld * 2};
  const cuuint32_t box[3] = {BK, cuuint32_t(box_rows), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : int(r);
}

}  // namespace submat

// BF16 (hi, lo) pairs: a float v is carried as hi = bf16(v) and
// lo = bf16(v - hi), so that hi + lo equals v to about 2^-17 relative and the
// three-term split product hi*hi + hi*lo + lo*hi keeps ~16 bits.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"

namespace submat {

__device__ __forceinline__ void split2f(float v, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t i) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[i] = h;
  lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ void split2(double v, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t i) {
  split2f(d2f_trunc(v), hi, lo, i);
}

// four consecutive BF16 (hi, lo) pairs <-> four floats (hi + lo)
__device__ __forceinline__ float4 load_split4(const __nv_bfloat16* hi, const __nv_bfloat16* lo, int64_t i) {
  const uint2 h = *reinterpret_cast<const uint2*>(hi + i);
  const uint2 l = *reinterpret_cast<const uint2*>(lo + i);
  return make_float4(__uint_as_float(h.x << 16) + __uint_as_float(l.x << 16),
                     __uint_as_float(h.x & 0xFFFF0000u) + __uint_as_float(l.x & 0xFFFF0000u),
                     __uint_as_float(h.y << 16) + __uint_as_float(l.y << 16),
                     __uint_as_float(h.y & 0xFFFF0000u) + __uint_as_float(l.y & 0xFFFF0000u));
}

__device__ __forceinline__ void store_split4(float4 v, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t i) {
  const float x[4] = {v.x, v.y, v.z, v.w};
  uint32_t h[4], l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x[k]);
    h[k] = __bfloat16_as_ushort(b);
    l[k] = __bfloat16_as_ushort(__float2bfloat16_rn(x[k] - __bfloat162float(b)));
  }
  *reinterpret_cast<uint2*>(hi + i) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
  *reinterpret_cast<uint2*>(lo + i) = make_uint2(l[0] | (l[1] << 16), l[2] | (l[3] << 16));
}

}  // namespace submat

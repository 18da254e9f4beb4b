// BF16 (hi, lo) pairs: a float v is carried as hi = bf16(v) and
// lo = bf16(v - hi), so that hi + lo equals v to about 2^-17 relative and the
// three-term split product hi*hi + hi*lo + lo*hi keeps ~16 bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

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

// FP16 (hi, lo) pairs, the same construction with 11-bit halves: hi + lo
// carries about 22 bits (down to 2^-24 absolute, FP16's subnormal step), and
// the three-term split product keeps about 21.  FP16's range (|v| < 65504)
// suits the Newton-Schulz iterates, whose entries stay below 3 in magnitude.
__device__ __forceinline__ void split2f(float v, __half* hi, __half* lo, int64_t i) {
  const __half h = __float2half_rn(v);
  hi[i] = h;
  lo[i] = __float2half_rn(v - __half2float(h));
}

__device__ __forceinline__ void split2(double v, __half* hi, __half* lo, int64_t i) {
  split2f(d2f_trunc(v), hi, lo, i);
}

__device__ __forceinline__ float4 load_split4(const __half* hi, const __half* lo, int64_t i) {
  const uint2 h = *reinterpret_cast<const uint2*>(hi + i);
  const uint2 l = *reinterpret_cast<const uint2*>(lo + i);
  const float2 h0 = __half22float2(*reinterpret_cast<const __half2*>(&h.x));
  const float2 h1 = __half22float2(*reinterpret_cast<const __half2*>(&h.y));
  const float2 l0 = __half22float2(*reinterpret_cast<const __half2*>(&l.x));
  const float2 l1 = __half22float2(*reinterpret_cast<const __half2*>(&l.y));
  return make_float4(h0.x + l0.x, h0.y + l0.y, h1.x + l1.x, h1.y + l1.y);
}

__device__ __forceinline__ void store_split4(float4 v, __half* hi, __half* lo, int64_t i) {
  const __half2 h0 = __floats2half2_rn(v.x, v.y), h1 = __floats2half2_rn(v.z, v.w);
  const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
  const __half2 l0 = __floats2half2_rn(v.x - f0.x, v.y - f0.y), l1 = __floats2half2_rn(v.z - f1.x, v.w - f1.y);
  *reinterpret_cast<uint2*>(hi + i) =
      make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
  *reinterpret_cast<uint2*>(lo + i) =
      make_uint2(*reinterpret_cast<const uint32_t*>(&l0), *reinterpret_cast<const uint32_t*>(&l1));
}

// value of one pair element (either format)
__device__ __forceinline__ float pair_get(const __nv_bfloat16* hi, const __nv_bfloat16* lo, int64_t i) {
  return __bfloat162float(hi[i]) + __bfloat162float(lo[i]);
}
__device__ __forceinline__ float pair_get(const __half* hi, const __half* lo, int64_t i) {
  return __half2float(hi[i]) + __half2float(lo[i]);
}

}  // namespace submat

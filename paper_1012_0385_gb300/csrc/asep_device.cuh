// asep_device.cuh -- device helpers shared by the kernel files: the
// Philox4x32-10 generator (Salmon, Moraes, Dror, Shaw, SC'11) with the
// library's counter layout, and a block-wide inclusive scan.  Internal
// linkage: every kernel file gets its own copy.
#pragma once

#include <cstdint>

#include "asep_internal.h"

namespace asep {
namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 and counters
// ---------------------------------------------------------------------------

// 32 x 32 -> 64-bit product as one wide multiply; .x = low word, .y = high word.
__device__ __forceinline__ uint2 mul_wide(uint32_t a, uint32_t b) {
  unsigned long long p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
  return make_uint2(static_cast<uint32_t>(p), static_cast<uint32_t>(p >> 32));
}

// One Philox4x32 round with round key (kx, ky).
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t kx, uint32_t ky) {
  const uint2 p0 = mul_wide(0xD2511F53u, c.x);
  const uint2 p1 = mul_wide(0xCD9E8D57u, c.z);
  return make_uint4(p1.y ^ c.y ^ kx, p1.x, p0.y ^ c.w ^ ky, p0.x);
}

__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    c = philox_round(c, k.x, k.y);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Philox4x32-10 with the round keys precomputed (KeySchedule, filled by the
// host): in a kernel whose descriptor is a parameter the keys are read from
// the constant bank, so a call costs only the multiplies and XORs.
__device__ __forceinline__ uint4 philox10(uint4 c, const KeySchedule& ks) {
#pragma unroll
  for (int round = 0; round < 10; ++round) c = philox_round(c, ks.x[round], ks.y[round]);
  return c;
}

__device__ __forceinline__ uint2 key_of(uint64_t seed) {
  return make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

__device__ __forceinline__ uint4 ctr_of(uint64_t sweep, uint32_t tag, uint32_t call, uint32_t sample, uint32_t d) {
  return make_uint4(static_cast<uint32_t>(sweep),
                    (static_cast<uint32_t>(sweep >> 32) & 0xFFu) | (tag << 8) | (call << 12), sample, d);
}

// Output word i of a Philox call.
__device__ __forceinline__ uint32_t pick(const uint4 x, uint32_t i) {
  return i == 0 ? x.x : (i == 1 ? x.y : (i == 2 ? x.z : x.w));
}

// A draw r accepts a move of threshold t (0, a multiple of 4096 or "always").
__device__ __forceinline__ bool accept(uint32_t r, uint32_t t) { return (r & kAcceptMask) < t; }

// ---------------------------------------------------------------------------
// Block scans (all threads of the block must call; blockDim.x % 32 == 0)
// ---------------------------------------------------------------------------

__device__ long long block_scan_incl(long long v, long long* warp_tot) {
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= static_cast<uint32_t>(o)) v += t;
  }
  if (lane == 31u) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    long long t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= static_cast<uint32_t>(o)) t += u;
    }
    if (lane < nw) warp_tot[lane] = t;
  }
  __syncthreads();
  if (wid > 0) v += warp_tot[wid - 1];
  __syncthreads();
  return v;
}

}  // namespace
}  // namespace asep

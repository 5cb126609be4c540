// asep_balance.cu -- balanced launch of the resident domain schedule.
//
// With one CTA per sample group, a launch of S groups on P SMs that hold two
// CTAs each leaves some SMs with one group and others with two for the whole
// launch (256 samples on 152 SMs: 104 SMs with two, 48 with one).  The SMs
// with two bound the launch, while the others run half loaded.  Here the
// launch's sweeps are cut into chunks and a persistent grid --
// ceil(groups / SMs) CTAs per SM, so one slot per SM beyond the groups'
// share floats -- takes (sample group, chunk) items from a queue in
// chunk-major order.  A CTA runs chunk k of a group once chunk k - 1 of
// that group has published its lattice, so groups move between SMs between
// chunks, and an SM whose second slot is free takes the next item.  Each
// group's sweeps still run in order from the lattice its previous chunk left
// in global memory, with the same random stream, so results are those of the
// one-launch kernel bit for bit.
//
// The wait for the previous chunk is bounded: it gives up after kWaitNs of
// %globaltimer (and kWaitSpins polls), or at once when another CTA has given
// up, sets the context's error flag (asep_sync then reports
// ASEP_ERR_TIMEOUT) and ends the CTA.  No item waits on an item that no
// running CTA holds: items are taken in queue order, so the previous chunk
// of a group was taken earlier, by a CTA that is running it.
#include <algorithm>
#include <cstdint>

#include "asep_device.cuh"
#include "asep_domain.cuh"
#include "asep_internal.h"
#include "asep_resident.cuh"

namespace asep {
namespace {

constexpr uint64_t kWaitNs = 5000000000ull;  // 5 s: far above the longest chunk the host allows
constexpr uint32_t kWaitSpins = 1u << 26;    // backstop if the timer does not advance

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until the group has published at least k chunks; false when the wait
// ran out or another CTA gave up.
__device__ bool wait_published(const uint32_t* flag, uint32_t k, const uint32_t* err) {
  if (ld_acquire(flag) >= k) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kWaitSpins; ++i) {
    __nanosleep(256);
    if (ld_acquire(flag) >= k) return true;
    if (ld_acquire(err)) return false;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT, uint32_t CP>
__global__ void __launch_bounds__(1024) k_domain_bal(const DomainLaunch a, const BalanceLaunch b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_item, s_ok;
  const uint64_t s0 = a.clock->sweep;
  const uint32_t cursor0 = a.clock->next_time;
  const uint32_t groups = a.n_groups;
  const uint32_t n_items = groups * b.chunks;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t i = atomicAdd(b.queue, 1u);
      s_item = i;
      s_ok = 1u;
      if (i < n_items) {
        const uint32_t k = i / groups;
        if (k > 0 && !wait_published(b.progress + (i - k * groups), k, b.err)) {
          s_ok = 0u;
          atomicExch(b.err, 1u);
        }
      }
    }
    __syncthreads();
    const uint32_t i = s_item;
    if (i >= n_items || !s_ok) break;
    const uint32_t k = i / groups, g = i - k * groups;
    const uint32_t first = k * b.chunk;
    const uint32_t n = min(b.chunk, a.n_sweeps - first);
    uint32_t cursor = cursor0;  // first sample time after this chunk's start
    while (cursor < a.n_times && a.times[cursor] <= s0 + first) ++cursor;
    run_group<MODEL, DIS, COUNT, CP>(a, g, smem_raw, s0 + first, cursor, n);
    __threadfence();  // the group's lattice, counters and records are visible device-wide
    __syncthreads();
    if (threadIdx.x == 0 && !(b.stall && g == 0 && k == 0)) st_release(b.progress + g, k + 1);
  }
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT, uint32_t CP>
cudaError_t launch_bal_cp(const DomainLaunch& a, const BalanceLaunch& b, uint32_t threads, size_t smem,
                          cudaStream_t st) {
  (void)cudaGetLastError();
  cudaError_t e = cudaFuncSetAttribute(k_domain_bal<MODEL, DIS, COUNT, CP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_domain_bal<MODEL, DIS, COUNT, CP>,
                                                         static_cast<int>(threads), smem)) != cudaSuccess)
    return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  // As many slots per SM as the groups need (ceil(groups / SMs)), not as many
  // as fit: with more, groups that migrate would pile onto some SMs while
  // others empty.  The slots beyond the groups float between SMs.
  const uint32_t need = (a.n_groups + static_cast<uint32_t>(sms) - 1) / static_cast<uint32_t>(sms);
  const uint32_t slots = std::min<uint32_t>(static_cast<uint32_t>(per_sm), need);
  const uint32_t items = a.n_groups * b.chunks;
  const uint32_t ctas = std::max<uint32_t>(1, std::min<uint32_t>(items, slots * static_cast<uint32_t>(sms)));
  if ((e = cudaMemsetAsync(b.progress, 0, (a.n_groups + 1u) * sizeof(uint32_t), st)) != cudaSuccess) return e;
  k_domain_bal<MODEL, DIS, COUNT, CP><<<ctas, threads, smem, st>>>(a, b);
  return cudaGetLastError();
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT>
cudaError_t launch_bal_t(const DomainLaunch& a, const BalanceLaunch& b, uint32_t threads, size_t smem,
                         cudaStream_t st) {
  if (a.Cp == 256 && DIS == kDisNone && MODEL == kRing) return launch_bal_cp<MODEL, DIS, COUNT, 256>(a, b, threads, smem, st);
  return launch_bal_cp<MODEL, DIS, COUNT, 0>(a, b, threads, smem, st);
}

}  // namespace

cudaError_t launch_domain_balanced(const DomainLaunch& a, const BalanceLaunch& b, uint32_t threads, size_t smem,
                                   cudaStream_t st) {
  const bool count = a.count_hops != 0;
  if (a.model == kRing && a.dis == kDisNone)
    return count ? launch_bal_t<kRing, kDisNone, true>(a, b, threads, smem, st)
                 : launch_bal_t<kRing, kDisNone, false>(a, b, threads, smem, st);
  if (a.model == kRing && a.dis == kDisBimodal)
    return count ? launch_bal_t<kRing, kDisBimodal, true>(a, b, threads, smem, st)
                 : launch_bal_t<kRing, kDisBimodal, false>(a, b, threads, smem, st);
  if (a.model == kRing && a.dis == kDisBimodalPQ)
    return count ? launch_bal_t<kRing, kDisBimodalPQ, true>(a, b, threads, smem, st)
                 : launch_bal_t<kRing, kDisBimodalPQ, false>(a, b, threads, smem, st);
  if (a.model == kTwoLane && a.dis == kDisNone) return launch_bal_t<kTwoLane, kDisNone, true>(a, b, threads, smem, st);
  if (a.model == kTwoLane && a.dis == kDisTurning)
    return launch_bal_t<kTwoLane, kDisTurning, true>(a, b, threads, smem, st);
  if (a.model == kTwoLane && a.dis == kDisCrossing)
    return launch_bal_t<kTwoLane, kDisCrossing, true>(a, b, threads, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace asep

// asep_stream.cu -- the streamed tier of the two-phase Poisson-domain
// schedule, for rings that fit neither one CTA nor a thread-block cluster.
//
// The lattice stays in global memory in its natural layout (bit k of word w
// = site 32 w + k).  A sweep is one launch per phase (plus, for two lanes
// with turning sites, one lane-change launch).  A CTA takes a tile of C
// consecutive super-domains of one sample: it copies the words that cover
// the tile's sites -- and one site beyond, which the last odd bond reaches --
// from global into shared memory with 1-D bulk asynchronous copies (16-byte
// aligned ranges, completion on an mbarrier, bounded wait), builds the same
// column layout as the resident kernel with the sweep's offset applied by
// funnel shifts (so no rotation pass is needed), runs the same half-domain
// phase, and writes the words back.  Words inside the tile's site range are
// stored; the first word and the last two, which the neighbouring tiles
// also touch, get the XOR of the bits this tile changed (atomically), so
// concurrent tiles never overwrite each other's bits.
#include <algorithm>
#include <cstdint>

#include "asep_device.cuh"
#include "asep_domain.cuh"
#include "asep_internal.h"

namespace asep {
namespace {

constexpr uint32_t kWaitSpins = 1u << 24;        // poll bound of the mbarrier wait (a backstop)
constexpr uint64_t kWaitNs = 1000000000ull;      // wall-clock bound: a copy of < 1 MB takes microseconds

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete, for at most one
// second (and kWaitSpins polls); false when it did not.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kWaitSpins; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// Global -> shared bulk copy of `bytes` (both addresses 16-byte aligned,
// bytes a multiple of 16), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// One phase of one tile.  Grid: tiles x S CTAs, blockIdx.x = sample * tiles + tile.
// stall: bytes the tile's copies announce beyond what they carry (0; a test
// of the timeout path sets it, so that the wait for them runs out).
template <uint32_t MODEL, uint32_t DIS, bool COUNT, uint32_t PHASE>
__global__ void __launch_bounds__(1024) k_stream(const DomainLaunch a, uint32_t tiles, uint32_t* err,
                                                 uint32_t stall) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  constexpr uint32_t NOCC = MODEL == kTwoLane ? 2u : 1u;
  constexpr uint32_t NQ = dis_planes(DIS);
  constexpr uint32_t NP = NOCC + NQ;
  const uint32_t R2 = a.R2, Cp = a.Cp, C = a.C, W = a.geo.W, D = a.D;
  const uint32_t sample = blockIdx.x / tiles, tile = blockIdx.x - sample * tiles;
  const uint32_t g0 = tile * C, Cn = min(C, a.G - g0);
  const uint32_t PW = (R2 + 1) * Cp;
  const uint32_t SW = R2 * C + 16;  // staged words per plane (>= the aligned range)
  uint32_t* cols = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* stage = cols + NP * PW;
  uint32_t* tab = stage + NP * SW;
  const uint32_t n_glob = a.geo.first_sample + sample;
  const uint2 key = key_of(a.seed);
  const uint64_t s = a.clock->sweep;
  const uint64_t L = a.geo.L;

  // the sweep's frame: super-domain g starts at site o + 2 D g (mod L)
  const uint32_t o = philox10(ctr_of(s, kTagOff, 0, n_glob, 0), key).x & (2 * D - 1);
  const uint64_t F = (static_cast<uint64_t>(o) + 2ull * D * g0) % L;
  const uint32_t w_first = static_cast<uint32_t>(F >> 5), sh = static_cast<uint32_t>(F & 31u);
  const uint32_t N = R2 * Cn + 2;                     // natural words w_first .. w_first + N - 1 (mod W)
  const uint32_t a0 = w_first & ~3u, off = w_first - a0;
  const uint32_t n_al = (off + N + 3u) & ~3u;         // 16-byte aligned range [a0, a0 + n_al) (mod W)
  const uint32_t part1 = min(n_al, W - a0), part2 = n_al - part1;

  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, NP * n_al * 4u + stall);
    for (uint32_t p = 0; p < NP; ++p) {
      const uint32_t* base = p < NOCC ? a.state + (static_cast<size_t>(sample) * NOCC + p) * W
                                      : a.mask + (static_cast<size_t>(sample / a.geo.samples_per_real) * NQ +
                                                  (p - NOCC)) * W;
      bulk_g2s(stage + p * SW, base + a0, part1 * 4u, &bar);
      if (part2) bulk_g2s(stage + p * SW + part1, base, part2 * 4u, &bar);
    }
  }
  for (uint32_t i = threadIdx.x; i < a.ptab_n; i += blockDim.x) tab[i] = a.ptab[i];
  const bool done = mbar_wait_bounded(&bar, 0);
  if (__syncthreads_or(!done)) {  // copies did not complete: report, let them land, give up
    if (threadIdx.x == 0) atomicExch(err, 1u);
    (void)mbar_wait_bounded(&bar, 0);
    return;
  }

  // columns: frame word f = c R2 + r (row r of column c; f = R2 Cn is the last column's mirror row)
  const uint32_t c = threadIdx.x;
  if (c < Cn) {
    for (uint32_t p = 0; p < NP; ++p) {
      const uint32_t* st = stage + p * SW + off;
      for (uint32_t r = 0; r <= R2; ++r) {
        const uint32_t f = c * R2 + r;
        cols[p * PW + r * Cp + c] = sh ? __funnelshift_r(st[f], st[f + 1], sh) : st[f];
      }
    }
  }
  __syncthreads();

  Lane ln;
  ln.c = c;
  ln.g = g0 + c;
  ln.col0 = 0;
  ln.c_next = 0;
  ln.c_prev = 0;
  ln.sample = sample;
  ln.n_glob = n_glob;
  ln.active = c < Cn;
  Cnt cnt;
  run_phase<MODEL, DIS, COUNT, 0, PHASE>(cols, nullptr, false, a, tab, PW, s, ln, key, cnt);
  __syncthreads();
  if (PHASE == 1) {  // the last bond of column c reached row 0 of column c + 1 through its mirror row
    if (c + 1 < Cn) {
      for (uint32_t p = 0; p < NOCC; ++p) {
        const uint32_t m = cols[p * PW + R2 * Cp + c];
        uint32_t* row0 = &cols[p * PW + (c + 1)];
        *row0 = (*row0 & ~1u) | (m & 1u);
      }
    }
    __syncthreads();
  }

  // write back: natural word w_first + k takes its high 32 - sh bits from
  // frame word k and its low sh bits from frame word k - 1
  const uint32_t last_f = R2 * Cn;
  const uint32_t low = sh ? (1u << sh) - 1u : 0u;
  for (uint32_t p = 0; p < NOCC; ++p) {
    const uint32_t* st = stage + p * SW + off;
    uint32_t* dst_plane = a.state + (static_cast<size_t>(sample) * NOCC + p) * W;
    const uint32_t* cp = cols + p * PW;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
      const uint32_t orig = st[k];
      uint32_t hi, lo;
      if (k <= last_f) {
        const uint32_t fk = k < last_f ? cp[(k & (R2 - 1)) * Cp + (k >> a.logR2)] : cp[R2 * Cp + (Cn - 1)];
        hi = fk << sh;
      } else {
        hi = orig & ~low;
      }
      if (sh == 0) {
        lo = 0;
      } else if (k >= 1 && k - 1 <= last_f) {
        const uint32_t f = k - 1;
        const uint32_t fk = f < last_f ? cp[(f & (R2 - 1)) * Cp + (f >> a.logR2)] : cp[R2 * Cp + (Cn - 1)];
        lo = fk >> (32u - sh);
      } else {
        lo = orig & low;
      }
      const uint32_t v = sh ? (hi | lo) : (k <= last_f ? hi : orig);
      const uint32_t w = (w_first + k) % W;
      if (k == 0 || k + 2 >= N) {
        const uint32_t delta = v ^ orig;
        if (delta) atomicXor(&dst_plane[w], delta);
      } else {
        dst_plane[w] = v;
      }
    }
  }
  if (ln.active) {
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(a.counters + 4ull * sample);
    if (cnt.a) atomicAdd(ctr + 0, static_cast<unsigned long long>(cnt.a));
    if (cnt.b) atomicAdd(ctr + 1, static_cast<unsigned long long>(cnt.b));
  }
}

// Lane changes of the two-lane model after the odd phase, on the natural
// layout: every turning site (DIS = kDisTurning; probability omega) or every
// site (DIS = kDisCrossing; A -> B with u_i, B -> A with v_i, the slow value
// at sites marked in the u and v planes) with exactly one lane occupied moves
// its particle (the draw of the other tiers: tag TURN, ctr3 = site / 4, word
// site mod 4).  One thread per word.
template <uint32_t DIS>
__global__ void k_stream_turn(const DomainLaunch a) {
  const uint32_t W = a.geo.W;
  const size_t total = static_cast<size_t>(a.geo.S) * W;
  const uint2 key = key_of(a.seed);
  const uint64_t s = a.clock->sweep;
  for (size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const uint32_t sample = static_cast<uint32_t>(idx / W), w = static_cast<uint32_t>(idx - size_t(sample) * W);
    uint32_t* A = a.state + static_cast<size_t>(sample) * 2 * W;
    uint32_t* B = A + W;
    const uint32_t real = sample / a.geo.samples_per_real;
    uint32_t av = A[w], bv = B[w];
    uint32_t e = av ^ bv, um = 0, vm = 0;
    if (DIS == kDisCrossing) {
      um = a.mask[(static_cast<size_t>(real) * 2) * W + w];
      vm = a.mask[(static_cast<size_t>(real) * 2 + 1) * W + w];
    } else {
      e &= a.mask[static_cast<size_t>(real) * W + w];
    }
    if (!e) continue;
    const uint32_t n_glob = a.geo.first_sample + sample;
    uint32_t ab = 0, ba = 0;
    while (e) {
      const uint32_t b = __ffs(e) - 1;
      e &= e - 1;
      const uint32_t site = 32u * w + b;
      const uint4 x = philox10(ctr_of(s, kTagTurn, 0, n_glob, site >> 2), key);
      uint32_t t = a.rates.omega;
      if (DIS == kDisCrossing && ((((av >> b) & 1u) ? um : vm) >> b) & 1u) t = a.rates.omega_slow;
      if (accept(pick(x, site & 3u), t)) {
        if (av & (1u << b)) ++ab;
        else ++ba;
        av ^= 1u << b;
        bv ^= 1u << b;
      }
    }
    A[w] = av;
    B[w] = bv;
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(a.counters + 4ull * sample);
    if (ab) atomicAdd(ctr + 2, static_cast<unsigned long long>(ab));
    if (ba) atomicAdd(ctr + 3, static_cast<unsigned long long>(ba));
  }
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT, uint32_t PHASE>
cudaError_t launch_stream_t(const DomainLaunch& a, uint32_t tiles, uint32_t threads, size_t smem, uint32_t* err,
                            uint32_t stall, cudaStream_t st) {
  (void)cudaGetLastError();
  const cudaError_t e = cudaFuncSetAttribute(k_stream<MODEL, DIS, COUNT, PHASE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_stream<MODEL, DIS, COUNT, PHASE><<<tiles * a.geo.S, threads, smem, st>>>(a, tiles, err, stall);
  return cudaGetLastError();
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT>
cudaError_t launch_stream_phases(const DomainLaunch& a, uint32_t tiles, uint32_t threads, size_t smem, uint32_t* err,
                                 uint32_t stall, cudaStream_t st) {
  cudaError_t e = launch_stream_t<MODEL, DIS, COUNT, 0>(a, tiles, threads, smem, err, stall, st);
  if (e != cudaSuccess) return e;
  e = launch_stream_t<MODEL, DIS, COUNT, 1>(a, tiles, threads, smem, err, stall, st);
  if (e != cudaSuccess) return e;
  if (MODEL == kTwoLane && (DIS == kDisTurning || DIS == kDisCrossing)) {
    const size_t total = static_cast<size_t>(a.geo.S) * a.geo.W;
    const uint32_t blocks = static_cast<uint32_t>(std::min<size_t>(152u * 16u, (total + 255) / 256));
    k_stream_turn<DIS><<<blocks, 256, 0, st>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace

size_t stream_smem_bytes(uint32_t model, uint32_t dis, uint32_t R2, uint32_t C, uint32_t ptab_n) {
  const uint32_t np = (model == kTwoLane ? 2u : 1u) + dis_planes(dis);
  const uint32_t Cp = (C + 31) / 32 * 32;
  return 4ull * np * ((R2 + 1) * Cp + R2 * C + 16) + 4ull * ptab_n;
}

// One sweep of the streamed tier (both phases and, for two lanes with
// turning sites, the lane changes) at the sweep index held by a.clock.
cudaError_t launch_stream_sweep(const DomainLaunch& a, uint32_t tiles, uint32_t threads, size_t smem, uint32_t* err,
                                uint32_t stall, cudaStream_t st) {
  const bool count = a.count_hops != 0;
  if (a.model == kTwoLane) {
    if (a.dis == kDisTurning)
      return launch_stream_phases<kTwoLane, kDisTurning, true>(a, tiles, threads, smem, err, stall, st);
    if (a.dis == kDisCrossing)
      return launch_stream_phases<kTwoLane, kDisCrossing, true>(a, tiles, threads, smem, err, stall, st);
    return launch_stream_phases<kTwoLane, kDisNone, true>(a, tiles, threads, smem, err, stall, st);
  }
  if (a.dis == kDisBimodal)
    return count ? launch_stream_phases<kRing, kDisBimodal, true>(a, tiles, threads, smem, err, stall, st)
                 : launch_stream_phases<kRing, kDisBimodal, false>(a, tiles, threads, smem, err, stall, st);
  if (a.dis == kDisBimodalPQ)
    return count ? launch_stream_phases<kRing, kDisBimodalPQ, true>(a, tiles, threads, smem, err, stall, st)
                 : launch_stream_phases<kRing, kDisBimodalPQ, false>(a, tiles, threads, smem, err, stall, st);
  return count ? launch_stream_phases<kRing, kDisNone, true>(a, tiles, threads, smem, err, stall, st)
               : launch_stream_phases<kRing, kDisNone, false>(a, tiles, threads, smem, err, stall, st);
}

}  // namespace asep

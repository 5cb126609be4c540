// asep_kernels.cu -- sm_103a kernels of the bit-packed ASEP / KPZ engine.
//
// Lattices are 32 sites per uint32 (bit k of word w = site 32w + k).  Every
// random number is a Philox4x32-10 output (Salmon et al., SC'11) with key =
// 64-bit seed and counter = (sweep lo, sweep hi | tag << 8 | call << 12,
// sample, domain / site group); nothing of the generator is stored.  A draw r
// accepts a move of threshold t iff (r & 0xfffff000) < t.
//
// Kernels
//   k_init      initial filling: 1010... (paper sec. 2.1) or Bernoulli(1/2)
//               per lane site (paper sec. 3).
//   k_disorder  quenched site classes (Eq. bimodal, paper sec. 2.3) or
//               turning sites (paper sec. 3), one bit per site.
//   k_domain    the resident two-phase Poisson-domain sweep: a CTA holds one
//               or more whole rings in shared memory for a whole launch.
//   (k_serial, the exact serial schedule, is in asep_serial.cu; k_sca, the
//   paper's two-sub-lattice schedule, in asep_sca.cu.)
//   k_heights   h_i = sum_{j<=i} (2 n_j - 1) and the sums of Eq. (W)
//               (k_heights_part + k_heights_combine for long lattices).
//
// Resident layout.  For sweep s with offset o the ring is cut into G = L/2D
// super-domains of 2D sites starting at o; super-domain g is column g of a
// transposed word array, rows r = 0..2D/32-1 (row r holds sites
// o + 2Dg + 32r .. +31).  Rows 0..D/32-1 are the first (even) half-domain,
// the rest the second (odd) half.  In a phase every active lane touches only
// its own column, so plain shared loads and stores are race-free, and lanes
// of a warp hit 32 different banks whatever rows they draw.  The last bond of
// an odd half reaches bit 0 of the next column's row 0: every column has one
// extra row (row 2D/32) that mirrors the next column's row 0 during the odd
// phase (copied in after the even phase, bit 0 written back after the odd
// phase), so that bond is "row + 1" like every other.  At the start of every
// sweep the words are rotated ("realigned") from the previous offset to the
// new one into a second buffer (double buffering), one funnel shift per word.
#include <algorithm>
#include <cstdint>

#include <cooperative_groups.h>

#include "asep_device.cuh"
#include "asep_domain.cuh"
#include "asep_internal.h"
#include "asep_resident.cuh"

namespace asep {
namespace {

// ---------------------------------------------------------------------------
// Initial state and quenched disorder
// ---------------------------------------------------------------------------

__global__ void k_init(const InitLaunch a) {
  const size_t per_sample = static_cast<size_t>(a.geo.planes) * a.geo.W;
  const size_t total = per_sample * a.geo.S;
  const uint2 key = key_of(a.init_seed);
  for (size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint32_t v;
    if (a.init_kind == 0) {
      v = 0x55555555u;  // site i occupied iff i even
    } else {
      const uint32_t sample = static_cast<uint32_t>(idx / per_sample);
      const uint32_t q = static_cast<uint32_t>(idx - static_cast<size_t>(sample) * per_sample);
      const uint4 x = philox10(ctr_of(0, kTagInit, 0, a.geo.first_sample + sample, q >> 2), key);
      v = pick(x, q & 3u);
    }
    a.state[idx] = v;
  }
}

__global__ void k_disorder(const DisorderLaunch a) {
  const size_t per_real = static_cast<size_t>(a.planes) * a.W;
  const size_t total = static_cast<size_t>(a.R) * per_real;
  const uint2 key = key_of(a.dis_seed);
  for (size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const uint32_t r = static_cast<uint32_t>(idx / per_real);
    const uint32_t pw = static_cast<uint32_t>(idx - static_cast<size_t>(r) * per_real);
    const uint32_t pl = pw / a.W, w = pw - pl * a.W;  // plane pl: call pl of the stream
    uint32_t v = 0;
    for (uint32_t q = 0; q < 8; ++q) {  // site group 8w + q holds sites 32w + 4q .. +3
      const uint4 x = philox10(ctr_of(0, kTagDis, pl, a.first_real + r, 8u * w + q), key);
      v |= (static_cast<uint32_t>(accept(x.x, a.thr)) << (4 * q)) |
           (static_cast<uint32_t>(accept(x.y, a.thr)) << (4 * q + 1)) |
           (static_cast<uint32_t>(accept(x.z, a.thr)) << (4 * q + 2)) |
           (static_cast<uint32_t>(accept(x.w, a.thr)) << (4 * q + 3));
    }
    a.mask[idx] = v;
  }
}

// ---------------------------------------------------------------------------
// Heights of natural-order lattices (one CTA per sample and plane)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_heights(const HeightsLaunch a) {
  __shared__ long long warp_tot[32];
  __shared__ unsigned long long warp_s2[32];
  const uint32_t planes = a.geo.planes, W = a.geo.W;
  const uint32_t sample = blockIdx.x / planes, p = blockIdx.x - sample * planes;
  const uint32_t* w = a.state + (static_cast<size_t>(sample) * planes + p) * W;
  const uint32_t chunk = (W + blockDim.x - 1) / blockDim.x;
  const uint32_t w0 = min(W, threadIdx.x * chunk), w1 = min(W, w0 + chunk);
  long long tot = 0;
  for (uint32_t i = w0; i < w1; ++i) tot += 2 * __popc(w[i]) - 32;
  const long long excl = block_scan_incl(tot, warp_tot) - tot;
  long long h = excl, s1 = 0;
  unsigned long long s2 = 0;
  for (uint32_t i = w0; i < w1; ++i) {
    const uint32_t x = w[i];
    for (uint32_t b = 0; b < 32; ++b) {
      h += ((x >> b) & 1u) ? 1 : -1;
      s1 += h;
      s2 += static_cast<unsigned long long>(h * h);
    }
  }
  const long long s1_all = block_scan_incl(s1, warp_tot);  // last thread holds the total
  // sum of h^2 can exceed 2^64 for L = 2^22: warp sums (< 2^63) then 128 bits
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((threadIdx.x & 31u) == 0) warp_s2[threadIdx.x >> 5] = s2;
  __syncthreads();
  if (threadIdx.x == blockDim.x - 1) {
    unsigned __int128 acc = 0;
    for (uint32_t i = 0; i < (blockDim.x >> 5); ++i) acc += warp_s2[i];
    const size_t e = (static_cast<size_t>(a.slot) * a.geo.S + sample) * planes + p;
    a.tab_sh[e] = s1_all;
    a.tab_sh2[2 * e] = static_cast<uint64_t>(acc);
    a.tab_sh2[2 * e + 1] = static_cast<uint64_t>(acc >> 64);
  }
  // the other observables of this record
  if (p == 0 && threadIdx.x == 0 && a.ex.tab_cnt) {
    const size_t ec = (static_cast<size_t>(a.slot) * a.geo.S + sample) * 4;
    for (int k = 0; k < 4; ++k) a.ex.tab_cnt[ec + k] = static_cast<int64_t>(a.counters[4 * static_cast<size_t>(sample) + k]);
  }
  const size_t pbase = (static_cast<size_t>(sample) * planes + p) * W;
  long long ov = 0;
  for (uint32_t i = w0; i < w1; ++i) {
    if (a.ex.profile) a.ex.profile[pbase + i] += __popc(w[i]);
    if (a.ex.snap) {
      if (a.t == a.ex.t0) a.ex.snap[pbase + i] = w[i];
      if (a.t >= a.ex.t0) ov += __popc(w[i] & a.ex.snap[pbase + i]);
    }
  }
  if (a.ex.snap) {
    const long long tot = block_scan_incl(ov, warp_tot);
    if (threadIdx.x == blockDim.x - 1)
      a.ex.tab_ac[(static_cast<size_t>(a.slot) * a.geo.S + sample) * planes + p] = tot;
  }
}

// Long lattices: chunk j of plane p of a sample (kHeightChunkWords words) per
// CTA.  Heights inside the chunk are taken relative to its entry height H_j
// (the sum of the earlier chunks' changes), which the combine step adds back
// exactly: sum (H + h') = sum h' + H n and sum (H + h')^2 = sum h'^2 +
// 2 H sum h' + H^2 n.
__global__ void __launch_bounds__(256) k_heights_part(const HeightsLaunch a, uint32_t chunks) {
  __shared__ long long warp_tot[32];
  __shared__ unsigned long long warp_s2[32];
  const uint32_t planes = a.geo.planes, W = a.geo.W;
  const uint32_t sp = blockIdx.x / chunks, j = blockIdx.x - sp * chunks;  // sp = sample * planes + p
  const uint32_t p = sp % planes;
  const uint32_t* w = a.state + static_cast<size_t>(sp) * W;
  const uint32_t c0 = j * kHeightChunkWords, c1 = min(W, c0 + kHeightChunkWords);
  const uint32_t per = (c1 - c0 + blockDim.x - 1) / blockDim.x;
  const uint32_t w0 = min(c1, c0 + threadIdx.x * per), w1 = min(c1, w0 + per);
  long long tot = 0;
  for (uint32_t i = w0; i < w1; ++i) tot += 2 * __popc(w[i]) - 32;
  const long long incl = block_scan_incl(tot, warp_tot);
  long long h = incl - tot, s1 = 0;
  unsigned long long s2 = 0;
  for (uint32_t i = w0; i < w1; ++i) {
    const uint32_t x = w[i];
    for (uint32_t b = 0; b < 32; ++b) {
      h += ((x >> b) & 1u) ? 1 : -1;
      s1 += h;
      s2 += static_cast<unsigned long long>(h * h);
    }
  }
  const long long s1_all = block_scan_incl(s1, warp_tot);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((threadIdx.x & 31u) == 0) warp_s2[threadIdx.x >> 5] = s2;
  const size_t pbase = static_cast<size_t>(sp) * W;
  long long ov = 0;
  for (uint32_t i = w0; i < w1; ++i) {
    if (a.ex.profile) a.ex.profile[pbase + i] += __popc(w[i]);
    if (a.ex.snap) {
      if (a.t == a.ex.t0) a.ex.snap[pbase + i] = w[i];
      if (a.t >= a.ex.t0) ov += __popc(w[i] & a.ex.snap[pbase + i]);
    }
  }
  const long long ov_all = block_scan_incl(ov, warp_tot);  // also orders warp_s2 before the read below
  if (threadIdx.x == blockDim.x - 1) {
    unsigned __int128 acc = 0;
    for (uint32_t i = 0; i < (blockDim.x >> 5); ++i) acc += warp_s2[i];
    HeightPart& part = a.parts[static_cast<size_t>(sp) * chunks + j];
    part.tot = incl;
    part.s1 = s1_all;
    part.s2lo = static_cast<uint64_t>(acc);
    part.s2hi = static_cast<uint64_t>(acc >> 64);
    part.ov = ov_all;
  }
  (void)p;
}

// One thread per sample and plane: the exact combination of its chunks.
__global__ void k_heights_combine(const HeightsLaunch a, uint32_t chunks) {
  const uint32_t planes = a.geo.planes, W = a.geo.W;
  const uint32_t sp = blockIdx.x * blockDim.x + threadIdx.x;
  if (sp >= a.geo.S * planes) return;
  const uint32_t sample = sp / planes, p = sp - sample * planes;
  __int128 H = 0, sh = 0, sh2 = 0;
  long long ov = 0;
  for (uint32_t j = 0; j < chunks; ++j) {
    const HeightPart& part = a.parts[static_cast<size_t>(sp) * chunks + j];
    const __int128 n = 32 * static_cast<__int128>(min(W, (j + 1) * kHeightChunkWords) - j * kHeightChunkWords);
    const __int128 s2 = (static_cast<__int128>(part.s2hi) << 64) | part.s2lo;
    sh += part.s1 + H * n;
    sh2 += s2 + 2 * H * part.s1 + H * H * n;
    H += part.tot;
    ov += part.ov;
  }
  const size_t e = (static_cast<size_t>(a.slot) * a.geo.S + sample) * planes + p;
  a.tab_sh[e] = static_cast<int64_t>(sh);
  const unsigned __int128 u2 = static_cast<unsigned __int128>(sh2);
  a.tab_sh2[2 * e] = static_cast<uint64_t>(u2);
  a.tab_sh2[2 * e + 1] = static_cast<uint64_t>(u2 >> 64);
  if (a.ex.snap) a.ex.tab_ac[e] = ov;
  if (p == 0 && a.ex.tab_cnt) {
    const size_t ec = (static_cast<size_t>(a.slot) * a.geo.S + sample) * 4;
    for (int k = 0; k < 4; ++k) a.ex.tab_cnt[ec + k] = static_cast<int64_t>(a.counters[4 * static_cast<size_t>(sample) + k]);
  }
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT, uint32_t CP>
__global__ void __launch_bounds__(1024) k_domain(const DomainLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  run_group<MODEL, DIS, COUNT, CP>(a, blockIdx.x, smem_raw, a.clock->sweep, a.clock->next_time, a.n_sweeps);
}

// Runtime dispatch of one group to the matching instantiation.
__device__ __forceinline__ void run_group_any(const DomainLaunch& a, uint32_t group, unsigned char* smem) {
  const uint64_t s0 = a.clock->sweep;
  const uint32_t cur = a.clock->next_time, n = a.n_sweeps;
  if (a.model == kTwoLane) {
    if (a.dis == kDisTurning) run_group<kTwoLane, kDisTurning, true, 0>(a, group, smem, s0, cur, n);
    else if (a.dis == kDisCrossing) run_group<kTwoLane, kDisCrossing, true, 0>(a, group, smem, s0, cur, n);
    else run_group<kTwoLane, kDisNone, true, 0>(a, group, smem, s0, cur, n);
  } else if (a.dis == kDisBimodal) {
    if (a.count_hops) run_group<kRing, kDisBimodal, true, 0>(a, group, smem, s0, cur, n);
    else run_group<kRing, kDisBimodal, false, 0>(a, group, smem, s0, cur, n);
  } else if (a.dis == kDisBimodalPQ) {
    if (a.count_hops) run_group<kRing, kDisBimodalPQ, true, 0>(a, group, smem, s0, cur, n);
    else run_group<kRing, kDisBimodalPQ, false, 0>(a, group, smem, s0, cur, n);
  } else if (a.Cp == 256) {
    if (a.count_hops) run_group<kRing, kDisNone, true, 256>(a, group, smem, s0, cur, n);
    else run_group<kRing, kDisNone, false, 256>(a, group, smem, s0, cur, n);
  } else {
    if (a.count_hops) run_group<kRing, kDisNone, true, 0>(a, group, smem, s0, cur, n);
    else run_group<kRing, kDisNone, false, 0>(a, group, smem, s0, cur, n);
  }
}

// Persistent batch kernel: CTAs take (job, group) items until the queue is
// empty.  Items are ordered largest first by the host.  The descriptor of the
// current item is copied to shared memory once.  Two block-size classes: up
// to 512 threads (128 registers available) and up to 1024.
template <uint32_t MAXT>
__global__ void __maxnreg__(MAXT == 512 ? 104 : 64) k_batch(const DomainLaunch* jobs, const uint32_t* items, uint32_t n_items,
                                                uint32_t* queue) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t item_idx;
  __shared__ DomainLaunch desc;
  for (;;) {
    if (threadIdx.x == 0) item_idx = atomicAdd(queue, 1u);
    __syncthreads();
    const uint32_t i = item_idx;
    if (i >= n_items) break;
    const uint32_t it = items[i];
    if (threadIdx.x == 0) desc = jobs[it >> kItemGroupBits];
    __syncthreads();
    run_group_any(desc, it & (kItemMaxGroups - 1u), smem_raw);
  }
}

__device__ __forceinline__ void advance_clock(Clock* c, const uint64_t* times, uint32_t n_times, uint32_t n) {
  const unsigned long long sweep = c->sweep + n;
  uint32_t next = c->next_time;
  while (next < n_times && times[next] <= sweep) ++next;
  c->sweep = sweep;
  c->next_time = next;
}

__global__ void k_advance(Clock* clock, const uint64_t* times, uint32_t n_times, uint32_t n) {
  if (blockIdx.x == 0 && threadIdx.x == 0) advance_clock(clock, times, n_times, n);
}

__global__ void k_set_clock(Clock* clock, unsigned long long sweep, uint32_t next_time) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clock->sweep = sweep;
    clock->next_time = next_time;
  }
}

__global__ void k_advance_batch(const DomainLaunch* jobs, uint32_t n_jobs) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n_jobs) advance_clock(jobs[j].clock, jobs[j].times, jobs[j].n_times, jobs[j].n_sweeps);
}

// ---------------------------------------------------------------------------
// Cluster tier: one sample spread over a thread-block cluster
// ---------------------------------------------------------------------------
//
// CTA k of the cluster holds columns [k Gc, (k+1) Gc) of the sample in its
// own shared memory, laid out exactly as in the resident kernel, and runs the
// same phases on them.  The few accesses that cross a slice boundary -- the
// rotation (new column g reads old columns g and g+1, or g-1 and g across the
// ring's end), the mirror copy (next column's row 0), the mirror write-back
// (previous column's mirror row) and the height scan -- go to the owning CTA
// through distributed shared memory.  Cluster barriers stand where data
// crosses CTAs: after the even phase, after the odd phase, and at the end of
// each sweep.

namespace cg = cooperative_groups;

// Word (p, row, global column g) of a plane buffer, in whichever CTA holds it.
__device__ __forceinline__ uint32_t* cl_word(const cg::cluster_group& cl, uint32_t* buf, uint32_t p, uint32_t PW,
                                            uint32_t row, uint32_t Cp, uint32_t g, uint32_t Gc, uint32_t my_rank) {
  const uint32_t rank = g / Gc, col = g - rank * Gc;
  uint32_t* base = rank == my_rank ? buf : cl.map_shared_rank(buf, rank);
  return base + p * PW + row * Cp + col;
}

template <uint32_t NP>
__device__ __forceinline__ void realign_cl(const cg::cluster_group& cl, uint32_t* src, uint32_t* dst,
                                           const DomainLaunch& a, const Lane& ln, uint32_t PW, uint32_t delta,
                                           uint32_t my_rank) {
  const uint64_t L = a.geo.L;
  const uint32_t W = a.geo.W, R2 = a.R2, Cp = a.Cp;
  for (uint32_t r = 0; r < R2; ++r) {
    uint64_t pos = delta + 32ull * (ln.g * R2 + r);
    if (pos >= L) pos -= L;
    const uint32_t fa = static_cast<uint32_t>(pos >> 5), sh = static_cast<uint32_t>(pos & 31u);
    const uint32_t fb = (fa + 1 == W) ? 0u : fa + 1;
#pragma unroll
    for (uint32_t p = 0; p < NP; ++p) {
      const uint32_t wa = *cl_word(cl, src, p, PW, fa & (R2 - 1), Cp, fa >> a.logR2, a.Gc, my_rank);
      const uint32_t wb = *cl_word(cl, src, p, PW, fb & (R2 - 1), Cp, fb >> a.logR2, a.Gc, my_rank);
      dst[p * PW + r * Cp + ln.c] = __funnelshift_r(wa, wb, sh);
    }
  }
}

// Heights of the occupancy planes (frame offset 0) of the cluster's sample.
template <uint32_t NOCC>
__device__ void record_heights_cl(const cg::cluster_group& cl, uint32_t* cur, const DomainLaunch& a, uint32_t PW,
                                  uint32_t slot, const Lane& ln, uint32_t my_rank, long long* warp_tot,
                                  long long* cta_sums) {
  const uint32_t last = blockDim.x - 1;
  for (uint32_t p = 0; p < NOCC; ++p) {
    const uint32_t* pl = cur + p * PW;
    long long tot = 0;
    if (ln.active)
      for (uint32_t r = 0; r < a.R2; ++r) tot += 2 * __popc(pl[r * a.Cp + ln.c]) - 32;
    const long long inc = block_scan_incl(tot, warp_tot);
    if (threadIdx.x == last) cta_sums[0] = inc;  // slice total of (2n - 1)
    cl.sync();
    long long h = inc - tot;  // height before this column within the slice
    for (uint32_t k = 0; k < my_rank; ++k) h += *cl.map_shared_rank(cta_sums, k);
    long long s1 = 0;
    unsigned long long s2 = 0;
    if (ln.active) {
      for (uint32_t r = 0; r < a.R2; ++r) {
        const uint32_t x = pl[r * a.Cp + ln.c];
        for (uint32_t b = 0; b < 32; ++b) {
          h += ((x >> b) & 1u) ? 1 : -1;
          s1 += h;
          s2 += static_cast<unsigned long long>(h * h);
        }
      }
    }
    const long long t1 = block_scan_incl(s1, warp_tot);
    const long long t2 = block_scan_incl(static_cast<long long>(s2), warp_tot);  // slice sum < 2^62
    cl.sync();  // every CTA has read the slice totals
    if (threadIdx.x == last) {
      cta_sums[1] = t1;
      cta_sums[2] = t2;
    }
    cl.sync();
    if (my_rank == 0 && threadIdx.x == 0) {
      long long sum1 = 0;
      unsigned __int128 sum2 = 0;
      for (uint32_t k = 0; k < cl.num_blocks(); ++k) {
        const long long* o = cl.map_shared_rank(cta_sums, k);
        sum1 += o[1];
        sum2 += static_cast<unsigned long long>(o[2]);
      }
      const size_t e = (static_cast<size_t>(slot) * a.geo.S + ln.sample) * NOCC + p;
      a.tab_sh[e] = sum1;
      a.tab_sh2[2 * e] = static_cast<uint64_t>(sum2);
      a.tab_sh2[2 * e + 1] = static_cast<uint64_t>(sum2 >> 64);
    }
    cl.sync();  // the slots are reused by the next plane
  }
}

template <uint32_t NOCC>
__device__ void record_extras_cl(const cg::cluster_group& cl, const uint32_t* cur, const DomainLaunch& a,
                                 uint32_t PW, uint32_t slot, uint64_t t, const Lane& ln, uint32_t my_rank,
                                 long long* warp_tot, long long* cta_sums, Cnt& cnt) {
  const Extras& ex = a.ex;
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(a.counters + 4ull * ln.sample);
  if (ln.active) {
    if (cnt.a) atomicAdd(ctr + 0, static_cast<unsigned long long>(cnt.a));
    if (cnt.b) atomicAdd(ctr + 1, static_cast<unsigned long long>(cnt.b));
    if (cnt.c) atomicAdd(ctr + 2, static_cast<unsigned long long>(cnt.c));
    if (cnt.d) atomicAdd(ctr + 3, static_cast<unsigned long long>(cnt.d));
    cnt = Cnt();
  }
  __threadfence();
  cl.sync();  // every CTA of the sample has flushed its counters
  if (my_rank == 0 && threadIdx.x == 0) {
    const size_t e = (static_cast<size_t>(slot) * a.geo.S + ln.sample) * 4;
    for (int k = 0; k < 4; ++k) ex.tab_cnt[e + k] = static_cast<int64_t>(atomicAdd(ctr + k, 0ull));
  }
  const uint32_t W = a.geo.W;
  for (uint32_t p = 0; p < NOCC; ++p) {
    const uint32_t* pl = cur + p * PW;
    const size_t base = (static_cast<size_t>(ln.sample) * a.geo.planes + p) * W + static_cast<size_t>(ln.g) * a.R2;
    long long ov = 0;
    if (ln.active) {
      for (uint32_t r = 0; r < a.R2; ++r) {
        const uint32_t x = pl[r * a.Cp + ln.c];
        if (ex.profile) ex.profile[base + r] += __popc(x);
        if (ex.snap) {
          if (t == ex.t0) ex.snap[base + r] = x;
          if (t >= ex.t0) ov += __popc(x & ex.snap[base + r]);
        }
      }
    }
    if (ex.snap) {
      const long long tot = block_scan_incl(ov, warp_tot);
      if (threadIdx.x == blockDim.x - 1) cta_sums[3] = tot;
      cl.sync();
      if (my_rank == 0 && threadIdx.x == 0) {
        long long sum = 0;
        for (uint32_t k = 0; k < cl.num_blocks(); ++k) sum += cl.map_shared_rank(cta_sums, k)[3];
        ex.tab_ac[(static_cast<size_t>(slot) * a.geo.S + ln.sample) * NOCC + p] = sum;
      }
      cl.sync();
    }
  }
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT>
__global__ void __launch_bounds__(1024) k_cluster(const DomainLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long cta_sums[4];
  constexpr uint32_t NOCC = MODEL == kTwoLane ? 2u : 1u;
  constexpr uint32_t NQ = dis_planes(DIS);
  constexpr uint32_t NP = NOCC + NQ;
  cg::cluster_group cl = cg::this_cluster();
  const uint32_t my_rank = cl.block_rank(), NC = cl.num_blocks();
  const uint32_t R2 = a.R2, Cp = a.Cp, G = a.G, W = a.geo.W, Gc = a.Gc;
  const uint32_t PW = (R2 + 1) * Cp;
  const uint64_t L = a.geo.L;
  uint32_t* bufA = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* bufB = bufA + NP * PW;
  uint32_t* tab = bufB + NP * PW;
  long long* warp_tot = reinterpret_cast<long long*>(tab + ((a.ptab_n + 1u) & ~1u));

  const uint32_t sample = blockIdx.x / NC;
  const uint32_t g_lo = my_rank * Gc;
  const uint32_t g_hi = min(G, g_lo + Gc);
  Lane ln;
  ln.c = threadIdx.x;
  ln.g = g_lo + threadIdx.x;
  ln.active = ln.g < g_hi && sample < a.geo.S;
  ln.col0 = 0;
  ln.c_next = 0;  // not used by the cluster tier
  ln.c_prev = 0;
  ln.sample = sample;
  ln.n_glob = a.geo.first_sample + sample;
  const uint32_t gn = (ln.g + 1 >= G) ? 0u : ln.g + 1;
  const uint32_t gp = (ln.g == 0) ? G - 1 : ln.g - 1;
  const uint2 key = key_of(a.seed);
  const uint64_t s0 = a.clock->sweep;

  // Poisson table and this CTA's slice of the lattice (frame offset 0)
  for (uint32_t i = threadIdx.x; i < a.ptab_n; i += blockDim.x) tab[i] = a.ptab[i];
  const uint32_t w_lo = g_lo * R2, w_hi = g_hi * R2;
  for (uint32_t p = 0; p < NP; ++p) {
    for (uint32_t w = w_lo + threadIdx.x; w < w_hi; w += blockDim.x) {
      const uint32_t v = p < NOCC ? a.state[(static_cast<size_t>(sample) * a.geo.planes + p) * W + w]
                                  : a.mask[(static_cast<size_t>(sample / a.geo.samples_per_real) * NQ + (p - NOCC)) * W + w];
      const uint32_t wl = w - w_lo;
      bufA[p * PW + (wl & (R2 - 1)) * Cp + (wl >> a.logR2)] = v;
    }
  }
  cl.sync();

  uint32_t* cur = bufA;
  uint32_t* nxt = bufB;
  uint32_t R_cur = 0;
  Cnt cnt;
  uint32_t rec = a.clock->next_time;

  for (uint32_t it = 0; it < a.n_sweeps; ++it) {
    const uint64_t s = s0 + it;
    const uint32_t o = philox10(ctr_of(s, kTagOff, 0, ln.n_glob, 0), key).x & (2 * a.D - 1);
    if (ln.active) realign_cl<NP>(cl, cur, nxt, a, ln, PW, static_cast<uint32_t>((o + L - R_cur) % L), my_rank);
    uint32_t* t = cur;
    cur = nxt;
    nxt = t;
    R_cur = o;
    __syncthreads();
    run_phase<MODEL, DIS, COUNT, 0, 0>(cur, nullptr, false, a, tab, PW, s, ln, key, cnt);
    cl.sync();
    if (ln.active) {
#pragma unroll
      for (uint32_t p = 0; p < NP; ++p)
        cur[p * PW + R2 * Cp + ln.c] = *cl_word(cl, cur, p, PW, 0, Cp, gn, Gc, my_rank);
    }
    run_phase<MODEL, DIS, COUNT, 0, 1>(cur, nullptr, false, a, tab, PW, s, ln, key, cnt);
    cl.sync();
    if (ln.active) {
#pragma unroll
      for (uint32_t p = 0; p < NOCC; ++p) {
        const uint32_t m = *cl_word(cl, cur, p, PW, R2, Cp, gp, Gc, my_rank);
        cur[p * PW + ln.c] = (cur[p * PW + ln.c] & ~1u) | (m & 1u);
      }
    }
    __syncthreads();
    if (MODEL == kTwoLane && (DIS == kDisTurning || DIS == kDisCrossing)) {
      if (ln.active) turning<DIS>(cur, a, PW, s, R_cur, ln, key, cnt);
    }
    cl.sync();
    if (rec < a.n_times && a.times[rec] == s + 1) {
      if (ln.active) realign_cl<NP>(cl, cur, nxt, a, ln, PW, static_cast<uint32_t>((L - R_cur) % L), my_rank);
      t = cur;
      cur = nxt;
      nxt = t;
      R_cur = 0;
      __syncthreads();
      record_heights_cl<NOCC>(cl, cur, a, PW, rec, ln, my_rank, warp_tot, cta_sums);
      record_extras_cl<NOCC>(cl, cur, a, PW, rec, s + 1, ln, my_rank, warp_tot, cta_sums, cnt);
      ++rec;
    }
  }

  if (ln.active) realign_cl<NP>(cl, cur, nxt, a, ln, PW, static_cast<uint32_t>((L - R_cur) % L), my_rank);
  cur = nxt;
  __syncthreads();
  for (uint32_t p = 0; p < NOCC; ++p) {
    for (uint32_t w = w_lo + threadIdx.x; w < w_hi; w += blockDim.x) {
      const uint32_t wl = w - w_lo;
      a.state[(static_cast<size_t>(sample) * a.geo.planes + p) * W + w] =
          cur[p * PW + (wl & (R2 - 1)) * Cp + (wl >> a.logR2)];
    }
  }
  if (ln.active) {
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(a.counters + 4ull * ln.sample);
    if (cnt.a) atomicAdd(dst + 0, static_cast<unsigned long long>(cnt.a));
    if (cnt.b) atomicAdd(dst + 1, static_cast<unsigned long long>(cnt.b));
    if (cnt.c) atomicAdd(dst + 2, static_cast<unsigned long long>(cnt.c));
    if (cnt.d) atomicAdd(dst + 3, static_cast<unsigned long long>(cnt.d));
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT, uint32_t CP>
cudaError_t launch_domain_cp(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st) {
  // set per call to what this launch needs: cheap, and right on every device
  (void)cudaGetLastError();
  const cudaError_t e = cudaFuncSetAttribute(k_domain<MODEL, DIS, COUNT, CP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_domain<MODEL, DIS, COUNT, CP><<<a.n_groups, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// The row pitch is a compile-time constant for the common 256-column plan
// (e.g. L = 2^17 with D = 256), a runtime value otherwise.
template <uint32_t MODEL, uint32_t DIS, bool COUNT>
cudaError_t launch_domain_t(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st) {
  if (a.Cp == 256) return launch_domain_cp<MODEL, DIS, COUNT, 256>(a, threads, smem, st);
  return launch_domain_cp<MODEL, DIS, COUNT, 0>(a, threads, smem, st);
}

uint32_t grid_for(size_t total, uint32_t threads) {
  size_t b = (total + threads - 1) / threads;
  if (b > 152u * 32u) b = 152u * 32u;
  return static_cast<uint32_t>(b < 1 ? 1 : b);
}

__global__ void k_philox_bench(uint32_t calls, uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint2 key = key_of(kBenchSeed);
  uint32_t acc = 0;
  for (uint32_t c = 0; c < calls; ++c) {
    const uint4 x = philox10(ctr_of(c >> 4, kTagDom, c & 15u, tid, tid >> 5), key);
    acc ^= x.x ^ x.y ^ x.z ^ x.w;
  }
  sink[tid] = acc;
}

// The attempt stream without lattice memory: the domain kernel's Philox
// calls (round keys from the descriptor-style key schedule, counters in the
// attempt layout) and, for each of a call's four words r, the plain-ring
// update of `attempt` applied to a word pair held in registers: bits j and
// j + 1 (j = r mod 32) of the 64-bit pair w1:w0 are swapped when they read
// 10 and r < p, or 01 and r < q.  The pair carries from attempt to attempt,
// so the chain is as dependent as on the lattice; each thread writes its final
// pair to sink[2 tid], sink[2 tid + 1].
__global__ void k_attempt_bench(uint32_t calls, int32_t pb, int32_t qb, const KeySchedule ks, uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t w0 = 0x55555555u ^ tid;
  uint32_t w1 = 0xAAAAAAAAu ^ (tid * 0x9E3779B9u);
  for (uint32_t c = 0; c < calls; ++c) {
    const uint4 y = philox10(ctr_of(c >> 4, kTagDom, c & 15u, tid, tid >> 5), ks);
    const uint32_t rs[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t r = rs[i];
      // the ring attempt's one-key hop test (asep_domain.cuh)
      const uint32_t key = __funnelshift_l(r, __funnelshift_r(w0, w1, r), 30);
      const bool hop = static_cast<int32_t>(key) < qb || static_cast<int32_t>(key + 0x40000000u) < pb;
      if (hop) {
        w0 ^= __funnelshift_l(0u, 3u, r);
        w1 ^= __funnelshift_l(3u, 0u, r);
      }
    }
  }
  sink[2 * tid] = w0;
  sink[2 * tid + 1] = w1;
}

}  // namespace

cudaError_t launch_attempt_bench(uint32_t blocks, uint32_t threads, uint32_t calls, uint32_t p, uint32_t q,
                                 uint32_t* sink, cudaStream_t st) {
  k_attempt_bench<<<blocks, threads, 0, st>>>(calls, hop_bound(p), hop_bound(q), key_schedule(kBenchSeed), sink);
  return cudaGetLastError();
}

cudaError_t launch_philox_bench(uint32_t blocks, uint32_t threads, uint32_t calls, uint32_t* sink, cudaStream_t st) {
  k_philox_bench<<<blocks, threads, 0, st>>>(calls, sink);
  return cudaGetLastError();
}

size_t domain_smem_bytes(uint32_t model, uint32_t dis, uint32_t R2, uint32_t Cp, uint32_t ptab_n, uint32_t threads) {
  const uint32_t nocc = model == kTwoLane ? 2u : 1u;
  const uint32_t np = nocc + dis_planes(dis);
  return 2ull * np * (R2 + 1ull) * Cp * 4ull + ((ptab_n + 1ull) & ~1ull) * 4ull + (32ull + threads) * 8ull;
}

cudaError_t launch_init(const InitLaunch& a, cudaStream_t st) {
  (void)cudaGetLastError();
  const size_t total = static_cast<size_t>(a.geo.S) * a.geo.planes * a.geo.W;
  k_init<<<grid_for(total, 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_disorder(const DisorderLaunch& a, cudaStream_t st) {
  (void)cudaGetLastError();
  k_disorder<<<grid_for(static_cast<size_t>(a.R) * a.W, 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

uint32_t height_chunks(uint32_t W) { return W > kHeightChunkWords ? (W + kHeightChunkWords - 1) / kHeightChunkWords : 1u; }

cudaError_t launch_heights(const HeightsLaunch& a, cudaStream_t st) {
  (void)cudaGetLastError();
  const uint32_t chunks = height_chunks(a.geo.W);
  if (chunks == 1) {
    k_heights<<<a.geo.S * a.geo.planes, 256, 0, st>>>(a);
  } else {
    if (!a.parts) return cudaErrorInvalidValue;
    const uint32_t sp = a.geo.S * a.geo.planes;
    k_heights_part<<<sp * chunks, 256, 0, st>>>(a, chunks);
    k_heights_combine<<<(sp + 127) / 128, 128, 0, st>>>(a, chunks);
  }
  return cudaGetLastError();
}

cudaError_t launch_domain(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st) {
  const bool count = a.count_hops != 0;
  if (a.model == kRing && a.dis == kDisNone)
    return count ? launch_domain_t<kRing, kDisNone, true>(a, threads, smem, st)
                 : launch_domain_t<kRing, kDisNone, false>(a, threads, smem, st);
  if (a.model == kRing && a.dis == kDisBimodal)
    return count ? launch_domain_t<kRing, kDisBimodal, true>(a, threads, smem, st)
                 : launch_domain_t<kRing, kDisBimodal, false>(a, threads, smem, st);
  if (a.model == kRing && a.dis == kDisBimodalPQ)
    return count ? launch_domain_cp<kRing, kDisBimodalPQ, true, 0>(a, threads, smem, st)
                 : launch_domain_cp<kRing, kDisBimodalPQ, false, 0>(a, threads, smem, st);
  if (a.model == kTwoLane && a.dis == kDisNone) return launch_domain_t<kTwoLane, kDisNone, true>(a, threads, smem, st);
  if (a.model == kTwoLane && a.dis == kDisTurning)
    return launch_domain_t<kTwoLane, kDisTurning, true>(a, threads, smem, st);
  if (a.model == kTwoLane && a.dis == kDisCrossing)
    return launch_domain_cp<kTwoLane, kDisCrossing, true, 0>(a, threads, smem, st);
  return cudaErrorInvalidValue;
}

// Dynamic shared memory opt-in of the batch kernel (its static shared memory
// -- the item index and the descriptor copy -- counts against the same limit).
template <uint32_t MAXT>
cudaError_t batch_attr(size_t smem) {
  return cudaFuncSetAttribute(k_batch<MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}

cudaError_t launch_batch(const DomainLaunch* jobs, const uint32_t* items, uint32_t n_items, uint32_t* queue,
                         uint32_t threads, uint32_t ctas, size_t smem, cudaStream_t st) {
  (void)cudaGetLastError();
  cudaError_t e;
  if ((e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
  if (threads <= 512) {
    if ((e = batch_attr<512>(smem)) != cudaSuccess) return e;
    k_batch<512><<<ctas, threads, smem, st>>>(jobs, items, n_items, queue);
  } else {
    if ((e = batch_attr<1024>(smem)) != cudaSuccess) return e;
    k_batch<1024><<<ctas, threads, smem, st>>>(jobs, items, n_items, queue);
  }
  return cudaGetLastError();
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT>
cudaError_t cluster_attrs(uint32_t cluster, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_cluster<MODEL, DIS, COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e == cudaSuccess && cluster > 8)
    e = cudaFuncSetAttribute(k_cluster<MODEL, DIS, COUNT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT>
cudaError_t launch_cluster_t(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st) {
  (void)cudaGetLastError();
  cudaError_t e = cluster_attrs<MODEL, DIS, COUNT>(a.cluster, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.geo.S * a.cluster, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cluster<MODEL, DIS, COUNT>, a);
}

template <uint32_t MODEL, uint32_t DIS, bool COUNT>
int cluster_fits_t(uint32_t cluster, uint32_t threads, size_t smem) {
  if (cluster_attrs<MODEL, DIS, COUNT>(cluster, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_cluster<MODEL, DIS, COUNT>, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_cluster(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st) {
  const bool count = a.count_hops != 0;
  if (a.model == kRing && a.dis == kDisNone)
    return count ? launch_cluster_t<kRing, kDisNone, true>(a, threads, smem, st)
                 : launch_cluster_t<kRing, kDisNone, false>(a, threads, smem, st);
  if (a.model == kRing && a.dis == kDisBimodal)
    return count ? launch_cluster_t<kRing, kDisBimodal, true>(a, threads, smem, st)
                 : launch_cluster_t<kRing, kDisBimodal, false>(a, threads, smem, st);
  if (a.model == kRing && a.dis == kDisBimodalPQ)
    return count ? launch_cluster_t<kRing, kDisBimodalPQ, true>(a, threads, smem, st)
                 : launch_cluster_t<kRing, kDisBimodalPQ, false>(a, threads, smem, st);
  if (a.model == kTwoLane && a.dis == kDisNone) return launch_cluster_t<kTwoLane, kDisNone, true>(a, threads, smem, st);
  if (a.model == kTwoLane && a.dis == kDisTurning)
    return launch_cluster_t<kTwoLane, kDisTurning, true>(a, threads, smem, st);
  if (a.model == kTwoLane && a.dis == kDisCrossing)
    return launch_cluster_t<kTwoLane, kDisCrossing, true>(a, threads, smem, st);
  return cudaErrorInvalidValue;
}

int cluster_fits(uint32_t model, uint32_t dis, uint32_t cluster, uint32_t threads, size_t smem) {
  if (model == kRing && dis == kDisNone) return cluster_fits_t<kRing, kDisNone, true>(cluster, threads, smem);
  if (model == kRing && dis == kDisBimodal) return cluster_fits_t<kRing, kDisBimodal, true>(cluster, threads, smem);
  if (model == kRing && dis == kDisBimodalPQ)
    return cluster_fits_t<kRing, kDisBimodalPQ, true>(cluster, threads, smem);
  if (model == kTwoLane && dis == kDisNone) return cluster_fits_t<kTwoLane, kDisNone, true>(cluster, threads, smem);
  if (model == kTwoLane && dis == kDisTurning)
    return cluster_fits_t<kTwoLane, kDisTurning, true>(cluster, threads, smem);
  if (model == kTwoLane && dis == kDisCrossing)
    return cluster_fits_t<kTwoLane, kDisCrossing, true>(cluster, threads, smem);
  return 0;
}

cudaError_t launch_advance(Clock* clock, const uint64_t* times, uint32_t n_times, uint32_t n, cudaStream_t st) {
  k_advance<<<1, 32, 0, st>>>(clock, times, n_times, n);
  return cudaGetLastError();
}

cudaError_t launch_set_clock(Clock* clock, uint64_t sweep, uint32_t next_time, cudaStream_t st) {
  k_set_clock<<<1, 32, 0, st>>>(clock, sweep, next_time);
  return cudaGetLastError();
}

cudaError_t launch_advance_batch(const DomainLaunch* jobs, uint32_t n_jobs, cudaStream_t st) {
  k_advance_batch<<<(n_jobs + 127) / 128, 128, 0, st>>>(jobs, n_jobs);
  return cudaGetLastError();
}

// One empty launch of each batch kernel (no items, no jobs) on `st`: loads
// the kernels' code on the current device and lets the driver size their
// per-thread local memory, so later batch steps start without either.
cudaError_t warm_batch_kernels(uint32_t* queue, cudaStream_t st) {
  (void)cudaGetLastError();
  cudaError_t e;
  if ((e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
  k_batch<512><<<1, 32, 0, st>>>(nullptr, nullptr, 0u, queue);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
  k_batch<1024><<<1, 32, 0, st>>>(nullptr, nullptr, 0u, queue);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_advance_batch<<<1, 32, 0, st>>>(nullptr, 0u);
  return cudaGetLastError();
}

int batch_ctas_per_sm(uint32_t threads, size_t smem) {
  int n = 0;
  cudaError_t e;
  if (threads <= 512) {
    if ((e = batch_attr<512>(smem)) == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<512>, static_cast<int>(threads), smem);
  } else {
    if ((e = batch_attr<1024>(smem)) == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<1024>, static_cast<int>(threads), smem);
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();  // do not leave the failure for the next launch check to find
    return 0;
  }
  return n;
}



}  // namespace asep

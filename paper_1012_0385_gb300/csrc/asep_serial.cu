// asep_serial.cu -- plain random-sequential update (paper sec. 2.1), exact:
// the serial schedule of the library, one warp per sample.
#include <algorithm>
#include <cstdint>

#include "asep_device.cuh"
#include "asep_internal.h"
#include "asep_serial.h"

namespace asep {
namespace {

// ---------------------------------------------------------------------------
// Serial random-sequential update, one warp per sample
// ---------------------------------------------------------------------------
//
// The attempts of a sweep form one sequence; the warp takes them 32 at a
// time in sequence order (lane k = attempt base + k).  Two attempts commute
// when their bonds share no site, so the longest prefix of a batch in which
// no attempt shares a site with an earlier one gives the same lattice
// whether applied one after another or all at once.  The warp applies that
// prefix (its flips are disjoint bits, written with shared-memory atomics)
// and starts the next batch at the first attempt that collided.  Bonds i
// and j share a site exactly when i / 2 == j / 2 or (i + 1 mod L) / 2 ==
// (j + 1 mod L) / 2, so two match operations find every collision.  The
// lattice (and the quenched plane) is staged in shared memory when it fits.

template <uint32_t MODEL, uint32_t DIS, bool SMEM>
__global__ void __launch_bounds__(256) k_serial(const SerialLaunch a) {
  extern __shared__ __align__(16) uint32_t serial_smem[];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  const uint32_t sample = blockIdx.x * (blockDim.x >> 5) + wib;
  if (sample >= a.geo.S) return;  // whole warps leave together
  const uint32_t L = static_cast<uint32_t>(a.geo.L), W = a.geo.W;
  constexpr uint32_t NOCC = MODEL == kTwoLane ? 2u : 1u;
  constexpr uint32_t NQ = dis_planes(DIS);  // quenched planes (independent p, q classes: two)
  constexpr uint32_t NPL = NOCC + NQ;
  uint32_t* gA = a.state + static_cast<size_t>(sample) * NOCC * W;
  const uint32_t* gM =
      (DIS != kDisNone) ? a.mask + static_cast<size_t>(sample / a.geo.samples_per_real) * NQ * W : nullptr;
  uint32_t* A = gA;
  const uint32_t* M = gM;
  if (SMEM) {
    uint32_t* mine = serial_smem + static_cast<size_t>(wib) * NPL * W;
    for (uint32_t w = lane; w < NOCC * W; w += 32) mine[w] = gA[w];
    if (DIS != kDisNone)
      for (uint32_t w = lane; w < NQ * W; w += 32) mine[NOCC * W + w] = gM[w];
    A = mine;
    M = mine + NOCC * W;
    __syncwarp();
  }
  uint32_t* B = A + W;
  const uint32_t n_glob = a.geo.first_sample + sample;
  const uint2 key = key_of(a.seed);
  const uint32_t n_att = MODEL == kTwoLane ? 2u * L : L;
  const uint32_t logL = 31u - static_cast<uint32_t>(__clz(static_cast<int>(L)));
  unsigned long long c0 = 0, c1 = 0, c2 = 0, c3 = 0;  // this lane's share of the sample's counters
  const uint64_t s0 = a.clock->sweep;
  uint32_t rec = a.clock->next_time;
  const uint32_t lt_mask = (1u << lane) - 1u;

  for (uint32_t it = 0; it < a.n_sweeps; ++it) {
    const uint64_t s = s0 + it;
    // The two words of attempt att: bond draw and acceptance draw.
    auto draws = [&](uint32_t att, uint32_t& rb, uint32_t& ru) {
      const uint4 x4 = philox10(ctr_of(s, kTagSer, 0, n_glob, att >> 1), key);
      rb = (att & 1u) ? x4.z : x4.x;
      ru = (att & 1u) ? x4.w : x4.y;
    };
    uint32_t base = 0;
    uint32_t rb, ru;  // draws of attempt base + lane
    draws(lane, rb, ru);
    while (base < n_att) {
      const uint32_t b = min(32u, n_att - base);
      const bool active = lane < b;
      // the next batch's draws if all 32 attempts commit, formed while this
      // batch runs (they do not depend on the lattice)
      uint32_t rb_next, ru_next;
      draws(base + 32u + lane, rb_next, ru_next);
      uint32_t pl = 0, i;
      if (MODEL == kTwoLane) {
        const uint32_t j = rb & (n_att - 1u);
        pl = j >> logL;
        i = j & (L - 1u);
      } else {
        i = rb & (L - 1u);
      }
      const uint32_t i1 = (i + 1u) & (L - 1u);
      uint32_t* P = pl ? B : A;
      const uint32_t x = ((P[i >> 5] >> (i & 31u)) & 1u) | (((P[i1 >> 5] >> (i1 & 31u)) & 1u) << 1);
      uint32_t thr;
      if (MODEL == kTwoLane) {
        thr = pl == 0 ? (x == 1u ? a.rates.p : 0u) : (x == 2u ? a.rates.q : 0u);
      } else if (DIS == kDisBimodal || DIS == kDisBimodalPQ) {
        const uint32_t* Mq = DIS == kDisBimodalPQ ? M + W : M;  // the classes of left hops
        thr = x == 1u ? (((M[i >> 5] >> (i & 31u)) & 1u) ? a.rates.p_slow : a.rates.p)
                      : (x == 2u ? (((Mq[i1 >> 5] >> (i1 & 31u)) & 1u) ? a.rates.q_slow : a.rates.q) : 0u);
      } else {
        thr = x == 1u ? a.rates.p : (x == 2u ? a.rates.q : 0u);
      }
      const bool hop = active && accept(ru, thr);
      // collisions with earlier attempts of the batch (inactive lanes get keys no bond has)
      const uint32_t k1 = active ? (pl << 31) | (i >> 1) : 0x7FE00000u | lane;
      const uint32_t k2 = active ? (pl << 31) | (i1 >> 1) : 0x7FF00000u | lane;
      const uint32_t same = __match_any_sync(0xffffffffu, k1) | __match_any_sync(0xffffffffu, k2);
      const uint32_t coll = __ballot_sync(0xffffffffu, active && (same & lt_mask) != 0u);
      const uint32_t c = coll ? static_cast<uint32_t>(__ffs(coll)) - 1u : b;
      if (lane < c && hop) {
        atomicXor(&P[i >> 5], 1u << (i & 31u));
        atomicXor(&P[i1 >> 5], 1u << (i1 & 31u));
        if (MODEL == kTwoLane) {
          c0 += pl == 0u;
          c1 += pl == 1u;
        } else if (a.count_hops) {
          c0 += x == 1u;
          c1 += x != 1u;
        }
      }
      __syncwarp();
      // the next batch starts at attempt base + c: lane k takes the draws of
      // this batch's lane c + k, or of the prefetched lane c + k - 32
      const uint32_t src = lane + c;
      const uint32_t rb_a = __shfl_sync(0xffffffffu, rb, src & 31u), ru_a = __shfl_sync(0xffffffffu, ru, src & 31u);
      const uint32_t rb_b = __shfl_sync(0xffffffffu, rb_next, src & 31u);
      const uint32_t ru_b = __shfl_sync(0xffffffffu, ru_next, src & 31u);
      rb = src < 32u ? rb_a : rb_b;
      ru = src < 32u ? ru_a : ru_b;
      base += c;
    }
    if (MODEL == kTwoLane && (DIS == kDisTurning || DIS == kDisCrossing)) {
      // lane changes: every event touches only (A_i, B_i); words are split over the lanes.  Crossing kind:
      // every site, u_i (plane 0) for a particle in lane A, v_i (plane 1) for one in lane B
      for (uint32_t w = lane; w < W; w += 32) {
        uint32_t e = (DIS == kDisCrossing ? ~0u : M[w]) & (A[w] ^ B[w]);
        while (e) {
          const uint32_t bit = __ffs(e) - 1;
          e &= e - 1;
          const uint32_t site = 32u * w + bit;
          const uint4 r = philox10(ctr_of(s, kTagTurn, 0, n_glob, site >> 2), key);
          uint32_t thr = a.rates.omega;
          if (DIS == kDisCrossing) {
            const uint32_t marked = ((A[w] >> bit) & 1u) ? M[w] : M[W + w];
            thr = ((marked >> bit) & 1u) ? a.rates.omega_slow : a.rates.omega;
          }
          if (accept(pick(r, site & 3u), thr)) {
            if (A[w] & (1u << bit)) ++c2;
            else ++c3;
            A[w] ^= 1u << bit;
            B[w] ^= 1u << bit;
          }
        }
      }
      __syncwarp();
    }
    if (rec < a.n_times && a.times[rec] == s + 1) {
      const uint32_t chunk = (W + 31u) / 32u;
      const uint32_t w0 = min(W, lane * chunk), w1 = min(W, w0 + chunk);
      for (uint32_t p = 0; p < NOCC; ++p) {
        const uint32_t* pw = p ? B : A;
        long long tot = 0;
        for (uint32_t w = w0; w < w1; ++w) tot += 2 * __popc(pw[w]) - 32;
        long long h = tot;  // inclusive warp scan of the chunk totals
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long t = __shfl_up_sync(0xffffffffu, h, o);
          if (lane >= static_cast<uint32_t>(o)) h += t;
        }
        h -= tot;
        long long s1 = 0;
        unsigned long long s2 = 0;
        for (uint32_t w = w0; w < w1; ++w) {
          const uint32_t xw = pw[w];
          for (uint32_t bb = 0; bb < 32; ++bb) {
            h += ((xw >> bb) & 1u) ? 1 : -1;
            s1 += h;
            s2 += static_cast<unsigned long long>(h * h);
          }
        }
        // profile and autocorrelation overlap of this plane
        const size_t pbase = (static_cast<size_t>(sample) * NOCC + p) * W;
        long long ov = 0;
        for (uint32_t w = w0; w < w1; ++w) {
          if (a.ex.profile) a.ex.profile[pbase + w] += __popc(pw[w]);
          if (a.ex.snap) {
            if (s + 1 == a.ex.t0) a.ex.snap[pbase + w] = pw[w];
            if (s + 1 >= a.ex.t0) ov += __popc(pw[w] & a.ex.snap[pbase + w]);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
          ov += __shfl_xor_sync(0xffffffffu, ov, o);
        }
        unsigned __int128 s2_all = 0;
        for (int l = 0; l < 32; ++l) s2_all += __shfl_sync(0xffffffffu, s2, l);
        if (lane == 0) {
          const size_t e = (static_cast<size_t>(rec) * a.geo.S + sample) * NOCC + p;
          a.tab_sh[e] = s1;
          a.tab_sh2[2 * e] = static_cast<uint64_t>(s2_all);
          a.tab_sh2[2 * e + 1] = static_cast<uint64_t>(s2_all >> 64);
          if (a.ex.snap) a.ex.tab_ac[e] = ov;
        }
      }
      const unsigned long long mine[4] = {c0, c1, c2, c3};
      unsigned long long tot_cnt[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        unsigned long long v = mine[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        tot_cnt[k] = v;
      }
      if (lane == 0) {
        const size_t ec = (static_cast<size_t>(rec) * a.geo.S + sample) * 4;
        for (int k = 0; k < 4; ++k) a.ex.tab_cnt[ec + k] = static_cast<int64_t>(a.counters[4ull * sample + k] + tot_cnt[k]);
      }
      __syncwarp();
      ++rec;
    }
  }
  const unsigned long long mine[4] = {c0, c1, c2, c3};
  unsigned long long tot_cnt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    unsigned long long v = mine[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    tot_cnt[k] = v;
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) a.counters[4ull * sample + k] += tot_cnt[k];
  if (SMEM) {
    __syncwarp();
    for (uint32_t w = lane; w < NOCC * W; w += 32) gA[w] = A[w];
  }
}

// ---------------------------------------------------------------------------
// Serial random-sequential update, one CTA per sample, dependency rounds
// ---------------------------------------------------------------------------
//
// The same attempts, drawn the same way, as k_serial, for samples whose
// lattice and sweep of attempts fit one CTA's shared memory.  Attempt k may
// run once every earlier attempt that shares a site with it has run; attempts
// that share no site commute, so running a sweep as rounds of such ready
// attempts gives the sequential result bit for bit.  Round r: every pending
// attempt k writes the key (r << 16) | (0xFFFF - k) to both its sites with an
// atomic max, so each site ends up holding its earliest pending attempt;
// after a barrier, an attempt whose key survived on both its sites runs.  It is
// the earliest pending attempt on each of its sites, so no earlier attempt
// touching them is left, and two attempts that run in one round share no
// site (their flips, possibly in one word, are atomic XORs of disjoint bits).
// The earliest pending attempt always runs, so every round makes progress.
// Keys of earlier rounds are smaller than those of round r, so the site table
// is cleared once per sweep.  A sweep of L random bonds on a ring of L = 4096
// sites takes about ten rounds -- the depth of its dependency graph -- where a
// warp needs about 150 committed prefixes of up to 32 attempts.

// Sums over the block (all threads call): a signed 64-bit value and an
// unsigned 64-bit value summed exactly in 128 bits.  Results valid in thread 0.
__device__ long long block_sum_i64(long long v, long long* red) {
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  long long t = 0;
  if (threadIdx.x == 0)
    for (uint32_t w = 0; w < nw; ++w) t += red[w];
  __syncthreads();
  return t;
}

__device__ unsigned __int128 block_sum_u128(unsigned long long v, unsigned long long* red) {
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned __int128 w = 0;
  for (int l = 0; l < 32; ++l) w += __shfl_sync(0xffffffffu, v, l);
  if (lane == 0) {
    red[2 * wid] = static_cast<unsigned long long>(w);
    red[2 * wid + 1] = static_cast<unsigned long long>(w >> 64);
  }
  __syncthreads();
  unsigned __int128 t = 0;
  if (threadIdx.x == 0)
    for (uint32_t k = 0; k < nw; ++k)
      t += (static_cast<unsigned __int128>(red[2 * k + 1]) << 64) | red[2 * k];
  __syncthreads();
  return t;
}

template <uint32_t MODEL, uint32_t DIS>
__global__ void __launch_bounds__(1024) k_serial_rounds(const SerialLaunch a) {
  extern __shared__ __align__(16) uint32_t serial_smem[];
  __shared__ long long s_i64[32];
  __shared__ unsigned long long s_u64[64];
  const uint32_t sample = blockIdx.x;
  const uint32_t tid = threadIdx.x, T = blockDim.x;
  const uint32_t L = static_cast<uint32_t>(a.geo.L), W = a.geo.W;
  constexpr uint32_t NOCC = MODEL == kTwoLane ? 2u : 1u;
  constexpr uint32_t NQ = dis_planes(DIS);
  constexpr uint32_t NPL = NOCC + NQ;
  const uint32_t n_att = NOCC * L;   // attempts per sweep (a power of two, at most 32 T)
  const uint32_t J = n_att / T;      // attempts per thread: k = j T + tid
  const uint32_t logL = 31u - static_cast<uint32_t>(__clz(static_cast<int>(L)));
  uint32_t* gA = a.state + static_cast<size_t>(sample) * NOCC * W;
  uint32_t* A = serial_smem;         // [NOCC][W] lattice, then [NQ][W] quenched planes
  uint32_t* B = A + W;
  uint32_t* M = A + NOCC * W;
  uint32_t* tab = A + NPL * W;       // [NOCC L] site keys
  uint32_t* dsite = tab + NOCC * L;  // [n_att] site of attempt k (lane L + i for lane B)
  uint32_t* du = dsite + n_att;      // [n_att] acceptance draw of attempt k
  for (uint32_t w = tid; w < NOCC * W; w += T) A[w] = gA[w];
  if (DIS != kDisNone) {
    const uint32_t* gM = a.mask + static_cast<size_t>(sample / a.geo.samples_per_real) * NQ * W;
    for (uint32_t w = tid; w < NQ * W; w += T) M[w] = gM[w];
  }
  const uint32_t n_glob = a.geo.first_sample + sample;
  const uint2 key = key_of(a.seed);
  unsigned long long c0 = 0, c1 = 0, c2 = 0, c3 = 0;  // this thread's share of the sample's counters
  const uint64_t s0 = a.clock->sweep;
  uint32_t rec = a.clock->next_time;
  const uint32_t all = J == 32u ? 0xffffffffu : (1u << J) - 1u;

  for (uint32_t it = 0; it < a.n_sweeps; ++it) {
    const uint64_t s = s0 + it;
    __syncthreads();  // the previous sweep's lane changes and record are done
    for (uint32_t q = tid; q < NOCC * L; q += T) tab[q] = 0u;
    // the sweep's draws, as k_serial takes them: attempt att from call att / 2 (words x, y or z, w); its
    // site is the bond draw modulo the attempts per sweep (two lanes: lane B's sites follow lane A's)
    for (uint32_t q = tid; q < n_att / 2u; q += T) {
      const uint4 x4 = philox10(ctr_of(s, kTagSer, 0, n_glob, q), key);
      dsite[2 * q] = x4.x & (n_att - 1u);
      du[2 * q] = x4.y;
      dsite[2 * q + 1] = x4.z & (n_att - 1u);
      du[2 * q + 1] = x4.w;
    }
    __syncthreads();
    uint32_t pend = all;
    // at most n_att rounds: every round runs at least the earliest pending attempt
    for (uint32_t r = 1; r <= n_att; ++r) {
      for (uint32_t m = pend; m; m &= m - 1u) {
        const uint32_t k = (static_cast<uint32_t>(__ffs(m)) - 1u) * T + tid;
        const uint32_t st = dsite[k];
        const uint32_t pl = MODEL == kTwoLane ? st >> logL : 0u;
        const uint32_t keyk = (r << 16) | (0xFFFFu - k);
        atomicMax(&tab[st], keyk);
        atomicMax(&tab[pl * L + (((st & (L - 1u)) + 1u) & (L - 1u))], keyk);
      }
      __syncthreads();
      for (uint32_t m = pend; m; m &= m - 1u) {
        const uint32_t j = static_cast<uint32_t>(__ffs(m)) - 1u;
        const uint32_t k = j * T + tid;
        const uint32_t st = dsite[k];
        const uint32_t pl = MODEL == kTwoLane ? st >> logL : 0u;
        const uint32_t i = st & (L - 1u), i1 = (i + 1u) & (L - 1u);
        const uint32_t keyk = (r << 16) | (0xFFFFu - k);
        if (tab[st] != keyk || tab[pl * L + i1] != keyk) continue;
        pend &= ~(1u << j);
        uint32_t* P = pl ? B : A;
        const uint32_t x = ((P[i >> 5] >> (i & 31u)) & 1u) | (((P[i1 >> 5] >> (i1 & 31u)) & 1u) << 1);
        uint32_t thr;
        if (MODEL == kTwoLane) {
          thr = pl == 0 ? (x == 1u ? a.rates.p : 0u) : (x == 2u ? a.rates.q : 0u);
        } else if (DIS == kDisBimodal || DIS == kDisBimodalPQ) {
          const uint32_t* Mq = DIS == kDisBimodalPQ ? M + W : M;  // the classes of left hops
          thr = x == 1u ? (((M[i >> 5] >> (i & 31u)) & 1u) ? a.rates.p_slow : a.rates.p)
                        : (x == 2u ? (((Mq[i1 >> 5] >> (i1 & 31u)) & 1u) ? a.rates.q_slow : a.rates.q) : 0u);
        } else {
          thr = x == 1u ? a.rates.p : (x == 2u ? a.rates.q : 0u);
        }
        if (accept(du[k], thr)) {
          atomicXor(&P[i >> 5], 1u << (i & 31u));
          atomicXor(&P[i1 >> 5], 1u << (i1 & 31u));
          if (MODEL == kTwoLane) {
            c0 += pl == 0u;
            c1 += pl == 1u;
          } else if (a.count_hops) {
            c0 += x == 1u;
            c1 += x != 1u;
          }
        }
      }
      if (!__syncthreads_or(pend != 0u)) break;  // also keeps this round's key reads before the next writes
    }
    if (MODEL == kTwoLane && (DIS == kDisTurning || DIS == kDisCrossing)) {
      // lane changes, as in k_serial: each event touches only (A_i, B_i); a thread per word
      for (uint32_t w = tid; w < W; w += T) {
        uint32_t e = (DIS == kDisCrossing ? ~0u : M[w]) & (A[w] ^ B[w]);
        while (e) {
          const uint32_t bit = __ffs(e) - 1;
          e &= e - 1;
          const uint32_t site = 32u * w + bit;
          const uint4 x4 = philox10(ctr_of(s, kTagTurn, 0, n_glob, site >> 2), key);
          uint32_t thr = a.rates.omega;
          if (DIS == kDisCrossing) {
            const uint32_t marked = ((A[w] >> bit) & 1u) ? M[w] : M[W + w];
            thr = ((marked >> bit) & 1u) ? a.rates.omega_slow : a.rates.omega;
          }
          if (accept(pick(x4, site & 3u), thr)) {
            if (A[w] & (1u << bit)) ++c2;
            else ++c3;
            A[w] ^= 1u << bit;
            B[w] ^= 1u << bit;
          }
        }
      }
      __syncthreads();
    }
    if (rec < a.n_times && a.times[rec] == s + 1) {
      // heights h_i = sum_{j <= i} (2 n_j - 1): a chunk of words per thread, their totals scanned over the block
      const uint32_t chunk = (W + T - 1u) / T;
      const uint32_t w0 = min(W, tid * chunk), w1 = min(W, w0 + chunk);
      for (uint32_t p = 0; p < NOCC; ++p) {
        const uint32_t* pw = p ? B : A;
        long long tot = 0;
        for (uint32_t w = w0; w < w1; ++w) tot += 2 * __popc(pw[w]) - 32;
        long long h = block_scan_incl(tot, s_i64) - tot;
        long long s1 = 0;
        unsigned long long s2 = 0;
        for (uint32_t w = w0; w < w1; ++w) {
          const uint32_t xw = pw[w];
          for (uint32_t bb = 0; bb < 32; ++bb) {
            h += ((xw >> bb) & 1u) ? 1 : -1;
            s1 += h;
            s2 += static_cast<unsigned long long>(h * h);
          }
        }
        const size_t pbase = (static_cast<size_t>(sample) * NOCC + p) * W;
        long long ov = 0;
        for (uint32_t w = w0; w < w1; ++w) {
          if (a.ex.profile) a.ex.profile[pbase + w] += __popc(pw[w]);
          if (a.ex.snap) {
            if (s + 1 == a.ex.t0) a.ex.snap[pbase + w] = pw[w];
            if (s + 1 >= a.ex.t0) ov += __popc(pw[w] & a.ex.snap[pbase + w]);
          }
        }
        const long long s1_all = block_sum_i64(s1, s_i64);
        const long long ov_all = block_sum_i64(ov, s_i64);
        const unsigned __int128 s2_all = block_sum_u128(s2, s_u64);
        if (tid == 0) {
          const size_t e = (static_cast<size_t>(rec) * a.geo.S + sample) * NOCC + p;
          a.tab_sh[e] = s1_all;
          a.tab_sh2[2 * e] = static_cast<uint64_t>(s2_all);
          a.tab_sh2[2 * e + 1] = static_cast<uint64_t>(s2_all >> 64);
          if (a.ex.snap) a.ex.tab_ac[e] = ov_all;
        }
      }
      const unsigned long long mine[4] = {c0, c1, c2, c3};
      for (int k = 0; k < 4; ++k) {
        const long long t = block_sum_i64(static_cast<long long>(mine[k]), s_i64);
        if (tid == 0) {
          const size_t ec = (static_cast<size_t>(rec) * a.geo.S + sample) * 4;
          a.ex.tab_cnt[ec + k] = static_cast<int64_t>(a.counters[4ull * sample + k] + static_cast<unsigned long long>(t));
        }
      }
      ++rec;
    }
  }
  const unsigned long long mine[4] = {c0, c1, c2, c3};
  for (int k = 0; k < 4; ++k) {
    const long long t = block_sum_i64(static_cast<long long>(mine[k]), s_i64);
    if (tid == 0) a.counters[4ull * sample + k] += static_cast<unsigned long long>(t);
  }
  __syncthreads();
  for (uint32_t w = tid; w < NOCC * W; w += T) gA[w] = A[w];
}

// Warps (samples) per CTA: up to 8, but no more than spreads the samples
// over all SMs -- each warp's attempts form one dependent chain, so a few
// samples run fastest one per SM.
uint32_t serial_warps_per_cta(uint32_t S) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                               cudaSuccess || sms <= 0) {
    (void)cudaGetLastError();
    sms = 1;
  }
  return std::max<uint32_t>(1, std::min<uint32_t>(8, (S + sms - 1) / static_cast<uint32_t>(sms)));
}

template <uint32_t MODEL, uint32_t DIS>
cudaError_t launch_serial_t(const SerialLaunch& a, cudaStream_t st) {
  constexpr uint32_t NPL = (MODEL == kTwoLane ? 2u : 1u) + dis_planes(DIS);
  const size_t per_sample = static_cast<size_t>(NPL) * a.geo.W * 4u;
  const size_t budget = 200u * 1024u;  // shared memory for the staged lattices of one block
  const uint32_t spread = serial_warps_per_cta(a.geo.S);
  if (per_sample <= budget) {
    const uint32_t warps = static_cast<uint32_t>(std::min<size_t>(spread, budget / per_sample));
    const size_t smem = per_sample * warps;
    const uint32_t blocks = (a.geo.S + warps - 1) / warps;
    (void)cudaGetLastError();
    const cudaError_t e = cudaFuncSetAttribute(k_serial<MODEL, DIS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    k_serial<MODEL, DIS, true><<<blocks, 32 * warps, smem, st>>>(a);
    return cudaGetLastError();
  }
  const uint32_t warps = spread;
  const uint32_t blocks = (a.geo.S + warps - 1) / warps;
  k_serial<MODEL, DIS, false><<<blocks, 32 * warps, 0, st>>>(a);
  return cudaGetLastError();
}

template <uint32_t MODEL, uint32_t DIS>
cudaError_t launch_serial_rounds_t(const SerialLaunch& a, cudaStream_t st) {
  const size_t smem = serial_rounds_smem_bytes(MODEL, DIS, a.geo.L);
  if (smem == 0) return cudaErrorInvalidValue;
  (void)cudaGetLastError();
  const cudaError_t e = cudaFuncSetAttribute(k_serial_rounds<MODEL, DIS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_serial_rounds<MODEL, DIS><<<a.geo.S, serial_rounds_threads(MODEL, a.geo.L), smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t serial_rounds_smem_bytes(uint32_t model, uint32_t dis, uint64_t L) {
  const uint64_t nocc = model == kTwoLane ? 2u : 1u;
  const uint64_t n_att = nocc * L;
  if (L < 64 || n_att > kSerialRoundsMaxAttempts) return 0;
  const uint64_t words = (nocc + dis_planes(dis)) * (L / 32) + nocc * L + 2 * n_att;
  const size_t bytes = static_cast<size_t>(4 * words);
  return bytes <= kSerialRoundsSmem ? bytes : 0;
}

uint32_t serial_rounds_threads(uint32_t model, uint64_t L) {
  const uint64_t n_att = (model == kTwoLane ? 2u : 1u) * L;
  return static_cast<uint32_t>(std::min<uint64_t>(1024, n_att));
}

cudaError_t launch_serial_plan(const SerialLaunch& a, uint32_t model, uint32_t dis, uint32_t plan, cudaStream_t st) {
  if (plan != kSerialRounds) return launch_serial(a, model, dis, st);
  if (model == kRing && dis == kDisNone) return launch_serial_rounds_t<kRing, kDisNone>(a, st);
  if (model == kRing && dis == kDisBimodal) return launch_serial_rounds_t<kRing, kDisBimodal>(a, st);
  if (model == kRing && dis == kDisBimodalPQ) return launch_serial_rounds_t<kRing, kDisBimodalPQ>(a, st);
  if (model == kTwoLane && dis == kDisNone) return launch_serial_rounds_t<kTwoLane, kDisNone>(a, st);
  if (model == kTwoLane && dis == kDisTurning) return launch_serial_rounds_t<kTwoLane, kDisTurning>(a, st);
  if (model == kTwoLane && dis == kDisCrossing) return launch_serial_rounds_t<kTwoLane, kDisCrossing>(a, st);
  return cudaErrorInvalidValue;
}

uint32_t serial_warp_plan_warps(uint32_t S) { return serial_warps_per_cta(S); }

cudaError_t launch_serial(const SerialLaunch& a, uint32_t model, uint32_t dis, cudaStream_t st) {
  if (model == kRing && dis == kDisNone) return launch_serial_t<kRing, kDisNone>(a, st);
  if (model == kRing && dis == kDisBimodal) return launch_serial_t<kRing, kDisBimodal>(a, st);
  if (model == kRing && dis == kDisBimodalPQ) return launch_serial_t<kRing, kDisBimodalPQ>(a, st);
  if (model == kTwoLane && dis == kDisNone) return launch_serial_t<kTwoLane, kDisNone>(a, st);
  if (model == kTwoLane && dis == kDisTurning) return launch_serial_t<kTwoLane, kDisTurning>(a, st);
  if (model == kTwoLane && dis == kDisCrossing) return launch_serial_t<kTwoLane, kDisCrossing>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace asep

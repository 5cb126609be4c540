// asep_domain.cuh -- the attempt and the half-domain phase of the two-phase
// Poisson-domain schedule, shared by the resident/cluster kernels
// (asep_kernels.cu) and the streamed tier (asep_stream.cu).  A CTA holds
// columns of 2D/32 (+1 mirror) rows per plane in shared memory, column g =
// super-domain g of the sweep; see asep_kernels.cu for the layout.
#pragma once

#include <cstdint>

#include "asep_device.cuh"
#include "asep_internal.h"

namespace asep {
namespace {

// K = k_lo + #{ j : tab[j] <= w } (table ascending): inversion of the
// Poisson CDF in u32 fixed point.
__device__ __forceinline__ uint32_t poisson_count(const uint32_t* tab, uint32_t n, uint32_t klo, uint32_t w) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (tab[mid] <= w) lo = mid + 1;
    else hi = mid;
  }
  return klo + lo;
}

struct Cnt {
  uint32_t a = 0, b = 0, c = 0, d = 0;  // ring: right, left; two lanes: A hops, B hops, A->B, B->A
};

struct Lane {
  uint32_t c;        // column in the CTA
  uint32_t g;        // super-domain index within the sample
  uint32_t col0;     // first column of the sample
  uint32_t c_next;   // column of super-domain g+1 (ring)
  uint32_t c_prev;   // column of super-domain g-1 (ring)
  uint32_t sample;   // sample index in the context
  uint32_t n_glob;   // global sample id (Philox counter)
  bool active;
};

// One attempt of a half-domain phase, without branches.  The bond's two
// words are rows `row` and `row + 1` of the lane's own column (row 2D/32 is
// the mirror of the next column's row 0), both loaded unconditionally; the
// 64-bit flip mask (3 << j across the word pair) is applied under one
// predicate.  `valid` is k <= K.
//
// Both hop tests come from one key: bits 31 and 30 hold sites i+1 and i (the
// funnel-shifted word pair), bits 29..0 hold r >> 2.  A left hop (sites 01,
// key bits 10) is accepted iff the key, read as signed, lies below
// INT_MIN + t/4 for the left rate t; adding 2^30 carries a right-hop pattern
// (bits 01) into the same window, tested against the right rate's bound
// (hop_bound: INT_MIN + t/4, INT_MIN + 2^30 for "always", INT_MIN for 0).
// Thresholds are multiples of 4096, for which r < t iff r >> 2 < t >> 2, so
// the test equals u < t of the definition; the other two patterns fall
// outside the window.
template <uint32_t MODEL, uint32_t DIS, bool COUNT, uint32_t CP>
__device__ __forceinline__ void attempt(unsigned char* cur, const DomainLaunch& a, uint32_t PWb, uint32_t base_b,
                                        uint32_t row_scale_b, uint32_t r, bool valid, Cnt& cnt) {
  // byte offset of row (j >> 5) of this half: (r & (D - 1) & ~31) * (4 Cp / 32)
  const uint32_t cpb = CP ? CP * 4u : a.Cp * 4u;  // row pitch in bytes (compile-time when CP != 0)
  uint32_t o0 = base_b + (r & a.row_bits) * row_scale_b;
  int32_t bR = a.rates.pb, bL = a.rates.qb;  // bounds of the right and left hop
  uint32_t laneB = 0;
  if (MODEL == kTwoLane) {
    laneB = (r >> a.logD) & 1u;  // lane A hops right only (p), lane B left only (q)
    o0 += laneB * PWb;
  } else if (DIS == kDisBimodal || DIS == kDisBimodalPQ) {
    const uint32_t c0 = *reinterpret_cast<const uint32_t*>(cur + PWb + o0);
    const uint32_t c1 = *reinterpret_cast<const uint32_t*>(cur + PWb + o0 + cpb);
    const uint32_t pc = __funnelshift_r(c0, c1, r);  // bit0: class of site i, bit1: of site i+1
    uint32_t qc = pc;
    if (DIS == kDisBimodalPQ) {  // left hops take the class of site i+1 from the second quenched plane
      const uint32_t d0 = *reinterpret_cast<const uint32_t*>(cur + 2u * PWb + o0);
      const uint32_t d1 = *reinterpret_cast<const uint32_t*>(cur + 2u * PWb + o0 + cpb);
      qc = __funnelshift_r(d0, d1, r);
    }
    bR = (pc & 1u) ? a.rates.pb_slow : bR;  // right hop across (i, i+1): p_i
    bL = (qc & 2u) ? a.rates.qb_slow : bL;  // left hop: q_{i+1}
  }
  uint32_t* p0 = reinterpret_cast<uint32_t*>(cur + o0);
  uint32_t* p1 = reinterpret_cast<uint32_t*>(cur + o0 + cpb);
  const uint32_t w0 = *p0;
  const uint32_t w1 = *p1;
  const uint32_t key = __funnelshift_l(r, __funnelshift_r(w0, w1, r), 30);
  bool hopL = static_cast<int32_t>(key) < bL;
  bool hopR = static_cast<int32_t>(key + 0x40000000u) < bR;
  if (MODEL == kTwoLane) {
    hopR = hopR && !laneB;
    hopL = hopL && laneB;
  }
  if (valid && (hopR || hopL)) {
    *p0 = w0 ^ __funnelshift_l(0u, 3u, r);  // 3 << (j mod 32), truncated
    *p1 = w1 ^ __funnelshift_l(3u, 0u, r);  // 1 when j mod 32 == 31, else 0
  }
  if (COUNT) {
    cnt.a += valid && hopR;
    cnt.b += valid && hopL;
  }
}

// One half-domain phase of one sweep.  All threads of the block must call.
//
// Lane sort: the lanes of a warp run to the largest Poisson count of the
// warp, so a warp whose domains drew similar counts wastes fewer slots.  With
// `a.lane_sort` (every warp inside one sample, and a scratch area of 5 words
// per column) each thread ranks its domain's count among the domains of the
// same shared-memory bank in its sample (columns lane, lane + 32, ...) and
// warp w runs the domains of rank w.  A domain's attempts are the same
// whichever thread runs them, and a thread stays in its own sample and bank,
// so results and bank mapping are unchanged; only the slots a warp wastes
// shrink.  `scr` is the idle realign buffer (overwritten by the next realign).
// The cluster tier passes sort = false: there other CTAs may still read that
// buffer remotely during the first phase.
template <uint32_t MODEL, uint32_t DIS, bool COUNT, uint32_t CP, uint32_t PHASE>
__device__ __forceinline__ void run_phase(uint32_t* cur, uint32_t* scr, bool sort, const DomainLaunch& a,
                                          const uint32_t* tab, uint32_t PW, uint64_t s, const Lane& ln, uint2 key,
                                          Cnt& cnt) {
  const uint32_t d = 2 * ln.g + PHASE;
  uint4 x0 = make_uint4(0u, 0u, 0u, 0u);
  uint32_t K = 0;
  if (ln.active) {
    x0 = philox10(ctr_of(s, kTagDom, 0, ln.n_glob, d), a.ks);
    K = poisson_count(tab, a.ptab_n, a.ptab_klo, x0.x);
  }
  const uint32_t cp = CP ? CP : a.Cp;
  uint32_t col = ln.c;  // the column (domain pair) this thread runs
  uint32_t dd = d;      // its domain index in the sample
  if (sort) {
    // Only the group's own columns (c < C) take part: a persistent CTA may be
    // wider than the group, and its extra threads keep K = 0 and no column.
    const bool in_group = ln.c < a.C;
    uint32_t* sK = scr;
    uint32_t* sPerm = scr + cp;
    uint32_t* sX = scr + 2 * cp;
    if (in_group) {
      sK[ln.c] = K;
      sX[ln.c] = x0.y;
      sX[cp + ln.c] = x0.z;
      sX[2 * cp + ln.c] = x0.w;
    }
    __syncthreads();
    if (in_group) {
      const uint32_t lane = ln.c & 31u;
      uint32_t rank = 0;
      for (uint32_t q = ln.col0 + lane; q < ln.col0 + a.G; q += 32) {
        const uint32_t kq = sK[q];
        rank += (kq < K || (kq == K && q < ln.c)) ? 1u : 0u;
      }
      sPerm[ln.col0 + (rank << 5) + lane] = ln.c;
    }
    __syncthreads();
    if (in_group) {
      col = sPerm[ln.c];
      dd = 2 * (ln.g - ln.c + col) + PHASE;
      K = sK[col];
      x0.y = sX[col];
      x0.z = sX[cp + col];
      x0.w = sX[2 * cp + col];
    }
  }
  const uint32_t Kmax = __reduce_max_sync(0xffffffffu, K);
  const uint32_t Kmin = __reduce_min_sync(0xffffffffu, K);
  unsigned char* cb = reinterpret_cast<unsigned char*>(cur);
  const uint32_t base_b = (PHASE * (a.D >> 5) * cp + col) * 4u;
  const uint32_t row_scale_b = cp >> 3;  // 4 * Cp / 32
  const uint32_t PWb = PW * 4u;
  attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, x0.y, 1 <= K, cnt);
  attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, x0.z, 2 <= K, cnt);
  attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, x0.w, 3 <= K, cnt);
  // Calls whose four attempts every lane of the warp makes (k + 3 <= Kmin) need
  // no per-attempt count test; the remaining calls up to Kmax test k <= K.  A
  // domain's attempts keep their order either way.  The fast calls are
  // 1 .. (Kmin - 3) / 4; call k's counter is call 1's with k - 1 added at bit 12
  // of word 1 (the call field), so the loop steps that word.  Each iteration
  // draws the next call's words before it applies the current call's four
  // attempts (the random stream does not depend on the lattice), so Philox's
  // rounds overlap the attempts' dependent chain; two iterations per loop trip.
  uint4 ctr = ctr_of(s, kTagDom, 1, ln.n_glob, dd);
  const uint32_t n_fast = Kmin >= 3u ? (Kmin - 3u) >> 2 : 0u;
  const uint32_t y_end = ctr.y + (n_fast << 12);
  uint4 y = philox10(ctr, a.ks);  // call n_fast + 1's words when the fast loop ends
#pragma unroll 2
  for (; ctr.y != y_end;) {
    ctr.y += 1u << 12;
    const uint4 yn = philox10(ctr, a.ks);  // the next call, ahead of this call's attempts
    attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, y.x, true, cnt);
    attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, y.y, true, cnt);
    attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, y.z, true, cnt);
    attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, y.w, true, cnt);
    y = yn;
  }
#pragma unroll 1
  for (uint32_t call = n_fast + 1; (call << 2) <= Kmax; ++call) {
    const uint32_t k = call << 2;
    uint4 yn = y;
    if (k + 4 <= Kmax) {  // warp-uniform
      ctr.y += 1u << 12;
      yn = philox10(ctr, a.ks);
    }
    attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, y.x, k <= K, cnt);
    attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, y.y, k + 1 <= K, cnt);
    attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, y.z, k + 2 <= K, cnt);
    attempt<MODEL, DIS, COUNT, CP>(cb, a, PWb, base_b, row_scale_b, y.w, k + 3 <= K, cnt);
    y = yn;
  }
}

}  // namespace
}  // namespace asep

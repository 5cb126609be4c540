// asep_sca.cu -- the paper's own GPU schedule: the two-sub-lattice stochastic
// cellular automaton of sec. 2.1 (Fig. "parasep"), bit-sliced for sm_103a.
//
// One sweep updates every even bond (i, i+1), i = 0, 2, ..., L-2, in
// parallel, then every odd bond i = 1, 3, ..., L-1 (the last one, (L-1, 0),
// is the paper's ring-closing step; it shares no site with the other odd
// bonds, so it runs with them).  Each bond makes one attempt: 10 -> 01 with
// p_i, 01 -> 10 with q_{i+1}, accepted iff a 20-bit uniform u is below the
// threshold's top 20 bits.
//
// Bit slicing.  A group is 32 bonds of one phase: the 16 bonds of word 2g
// (lanes 0, 2, ..., 30) and the 16 of word 2g + 1 (lanes 1, 3, ..., 31).
// Bit k of every lane's u is bit `lane` of random plane k of the group; call k
// of the stream (tag SCA, ctr3 = 2 * unit + phase) gives plane k of the four
// groups of a unit (8 words).  The comparison u < t runs most significant bit
// first over all 32 lanes at once and stops when no lane is undecided or no
// set bit of any threshold is left (p = 0.75, q = 0.25 need two planes).
//
// Layout.  One CTA per sample; the ring sits in shared memory as plain words
// (bit k of word w = site 32w + k), a thread owns whole units and moves them
// with 128-bit shared loads and stores.  An odd bond (32w + 31, 32w + 32)
// reaches bit 0 of the next word; inside a unit that word is in the thread's
// registers, across units the flip is left in a per-unit carry flag and the
// next unit's owner applies it when it next loads its first word (bit 0 of a
// unit's first word is touched by no odd bond of its own unit, so reading it
// during the odd phase is race-free).
#include <cstdint>

#include "asep_device.cuh"
#include "asep_internal.h"

namespace asep {
namespace {

constexpr uint32_t kEven = 0x55555555u;
constexpr uint32_t kOdd = 0xAAAAAAAAu;

// Sum of per-thread values over the block; every thread gets the total.
__device__ long long block_sum(long long v, long long* warp_tot) {
  const long long inc = block_scan_incl(v, warp_tot);
  __shared__ long long total;
  if (threadIdx.x == blockDim.x - 1) total = inc;
  __syncthreads();
  const long long t = total;
  __syncthreads();
  return t;
}

// Eight consecutive words (16-byte aligned) into registers.
__device__ __forceinline__ void load8(const uint32_t* p, uint32_t (&x)[8]) {
  const uint4 v0 = reinterpret_cast<const uint4*>(p)[0], v1 = reinterpret_cast<const uint4*>(p)[1];
  x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w; x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
}

// All-ones where bit k (0 = most significant of 20) of a 20-bit threshold is set.
__device__ __forceinline__ uint32_t bit_mask(uint32_t t20, uint32_t k) { return 0u - ((t20 >> (19u - k)) & 1u); }

// Applies the accepted moves h[g] of a unit's four groups (bit 2j: bond j
// of word 2g, bit 2j + 1: bond j of word 2g + 1) to its words; returns the
// flip of bit 0 of the next unit's first word that the unit's last odd bond
// makes (odd phase).  The masks ha, hb hold even bits only, so a bond's
// two-bit flip ha | ha << 1 is the product 3 ha (6 ha one site further on),
// which the multiply-add unit forms, sparing the busier integer pipe a shift
// and an OR.
template <uint32_t PHASE>
__device__ __forceinline__ uint32_t apply_moves(uint32_t (&x)[8], const uint32_t (&h)[4]) {
  uint32_t carry_out = 0u;
#pragma unroll
  for (int gi = 0; gi < 4; ++gi) {
    const uint32_t ha = h[gi] & kEven, hb = (h[gi] >> 1) & kEven;  // bonds of word 2g and of word 2g + 1
    if (PHASE == 0) {
      x[2 * gi] ^= ha * 3u;
      x[2 * gi + 1] ^= hb * 3u;
    } else {
      x[2 * gi] ^= ha * 6u;
      x[2 * gi + 1] ^= ((ha >> 30) & 1u) | (hb * 6u);  // bond (32w + 31, 32w + 32) of word 2g
      const uint32_t out = (hb >> 30) & 1u;            // ... and of word 2g + 1
      if (gi < 3) x[2 * gi + 2] ^= out;
      else carry_out = out;
    }
  }
  return carry_out;
}

// One phase over one unit (four groups, global unit index u) held in
// registers: x = its 8 words, c = its 8 class words (DIS: the classes of
// right hops, and of left hops too unless PQ), d = the classes of left hops
// (PQ: independent p and q classes), x_next / c_next / d_next = the next
// unit's first words (only bit 0 is used, odd phase).  Returns the flip of
// bit 0 of the next unit's first word that the unit's last odd bond makes
// (odd phase).
template <bool DIS, bool COUNT, bool FAST2, uint32_t PHASE, bool PQ = false>
__device__ __forceinline__ uint32_t sca_update(uint32_t (&x)[8], const uint32_t (&c)[8], const uint32_t (&d)[8],
                                               uint32_t x_next, uint32_t c_next, uint32_t d_next,
                                               const DomainLaunch& a, uint32_t u, uint64_t s, uint32_t n_glob,
                                               uint32_t kmax, unsigned long long& n_right,
                                               unsigned long long& n_left) {
  uint32_t rc[4], lc[4], acc[4], eq[4];
  if (FAST2) {
    // No disorder, p and q neither 0 nor "always", at most two planes: every
    // candidate lane is compared, and the threshold bit of a plane is p's on
    // right candidates and q's on left ones (uniform per plane).
#pragma unroll
    for (int gi = 0; gi < 4; ++gi) {
      const uint32_t xa = x[2 * gi], xb = x[2 * gi + 1];
      const uint32_t xn = gi < 3 ? x[2 * gi + 2] : x_next;
      const uint32_t ya = PHASE ? __funnelshift_r(xa, xb, 1) : xa;
      const uint32_t yb = PHASE ? __funnelshift_r(xb, xn, 1) : xb;
      // even lanes: bonds of word 2g (ya, ya >> 1); odd lanes: bonds of word 2g + 1 (yb << 1, yb)
      const uint32_t sa = ya >> 1, tb = yb << 1;
      const uint32_t df = ((ya ^ sa) & kEven) | ((tb ^ yb) & kOdd);  // the bond's sites differ
      const uint32_t first = (ya & kEven) | (tb & kOdd);             // its first site
      rc[gi] = df & first;   // 10
      lc[gi] = df & ~first;  // 01
      acc[gi] = 0u;
      eq[gi] = df;
    }
    const uint32_t p20 = a.rates.p >> 12, q20 = a.rates.q >> 12;
#pragma unroll
    for (uint32_t k = 0; k < 2; ++k) {  // FAST2: at most two planes (kmax <= 2)
      if (k >= kmax) break;
      const uint4 y = philox10(ctr_of(s, kTagSca, k, n_glob, 2u * u + PHASE), a.ks);
      const uint32_t U[4] = {y.x, y.y, y.z, y.w};
      const uint32_t pb = (p20 >> (19u - k)) & 1u, qb = (q20 >> (19u - k)) & 1u;
      if (pb && qb) {  // threshold bit 1 on every candidate lane
#pragma unroll
        for (int gi = 0; gi < 4; ++gi) {
          acc[gi] |= eq[gi] & ~U[gi];
          eq[gi] &= U[gi];
        }
      } else if (pb) {  // 1 on right candidates, 0 on left ones
#pragma unroll
        for (int gi = 0; gi < 4; ++gi) {
          acc[gi] |= eq[gi] & rc[gi] & ~U[gi];
          eq[gi] &= ~(rc[gi] ^ U[gi]);
        }
      } else if (qb) {
#pragma unroll
        for (int gi = 0; gi < 4; ++gi) {
          acc[gi] |= eq[gi] & lc[gi] & ~U[gi];
          eq[gi] &= ~(lc[gi] ^ U[gi]);
        }
      } else {  // 0 on every lane: still equal only where u's bit is 0
#pragma unroll
        for (int gi = 0; gi < 4; ++gi) eq[gi] &= ~U[gi];
      }
    }
  } else {
    const Rates& r = a.rates;
    const uint32_t pA = r.p == 0xFFFFFFFFu ? ~0u : 0u, qA = r.q == 0xFFFFFFFFu ? ~0u : 0u;
    const uint32_t psA = r.p_slow == 0xFFFFFFFFu ? ~0u : 0u, qsA = r.q_slow == 0xFFFFFFFFu ? ~0u : 0u;
    const uint32_t pN = r.p == 0u ? ~0u : 0u, qN = r.q == 0u ? ~0u : 0u;
    const uint32_t psN = r.p_slow == 0u ? ~0u : 0u, qsN = r.q_slow == 0u ? ~0u : 0u;
    uint32_t c1[4], c2[4];
    uint32_t any = 0;
#pragma unroll
    for (int gi = 0; gi < 4; ++gi) {
      const uint32_t xa = x[2 * gi], xb = x[2 * gi + 1];
      const uint32_t xn = gi < 3 ? x[2 * gi + 2] : x_next;
      // window: bit 2j = first site of bond j, bit 2j + 1 = its second site
      const uint32_t ya = PHASE ? __funnelshift_r(xa, xb, 1) : xa;
      const uint32_t yb = PHASE ? __funnelshift_r(xb, xn, 1) : xb;
      const uint32_t ra = ya & ~(ya >> 1) & kEven, la = ~ya & (ya >> 1) & kEven;
      const uint32_t rb = yb & ~(yb >> 1) & kEven, lb = ~yb & (yb >> 1) & kEven;
      rc[gi] = ra | (rb << 1);
      lc[gi] = la | (lb << 1);
      if (DIS) {
        const uint32_t ca = c[2 * gi], cb = c[2 * gi + 1];
        const uint32_t cn = gi < 3 ? c[2 * gi + 2] : c_next;
        const uint32_t za = PHASE ? __funnelshift_r(ca, cb, 1) : ca;
        const uint32_t zb = PHASE ? __funnelshift_r(cb, cn, 1) : cb;
        c1[gi] = (za & kEven) | ((zb & kEven) << 1);                   // class of site i
        c2[gi] = ((za >> 1) & kEven) | (((zb >> 1) & kEven) << 1);     // class of site i + 1
        if (PQ) {  // left hops: the q class of site i + 1
          const uint32_t da = d[2 * gi], db = d[2 * gi + 1];
          const uint32_t dn = gi < 3 ? d[2 * gi + 2] : d_next;
          const uint32_t wa = PHASE ? __funnelshift_r(da, db, 1) : da;
          const uint32_t wb = PHASE ? __funnelshift_r(db, dn, 1) : db;
          c2[gi] = ((wa >> 1) & kEven) | (((wb >> 1) & kEven) << 1);
        }
      } else {
        c1[gi] = 0u;
        c2[gi] = 0u;
      }
      const uint32_t rA = rc[gi] & ((~c1[gi] & pA) | (c1[gi] & psA));
      const uint32_t lA = lc[gi] & ((~c2[gi] & qA) | (c2[gi] & qsA));
      const uint32_t rN = rc[gi] & ((~c1[gi] & pN) | (c1[gi] & psN));
      const uint32_t lN = lc[gi] & ((~c2[gi] & qN) | (c2[gi] & qsN));
      acc[gi] = rA | lA;
      eq[gi] = (rc[gi] | lc[gi]) & ~(rA | lA | rN | lN);
      any |= eq[gi];
    }
    // most significant bit first; plane k of the four groups = Philox call k
    const uint32_t p20 = r.p >> 12, q20 = r.q >> 12, ps20 = r.p_slow >> 12, qs20 = r.q_slow >> 12;
    for (uint32_t k = 0; k < kmax && any; ++k) {
      const uint4 y = philox10(ctr_of(s, kTagSca, k, n_glob, 2u * u + PHASE), a.ks);
      const uint32_t P = bit_mask(p20, k), Q = bit_mask(q20, k);
      const uint32_t PS = DIS ? bit_mask(ps20, k) : 0u, QS = DIS ? bit_mask(qs20, k) : 0u;
      const uint32_t U[4] = {y.x, y.y, y.z, y.w};
      any = 0;
#pragma unroll
      for (int gi = 0; gi < 4; ++gi) {
        const uint32_t T = DIS ? ((rc[gi] & ((~c1[gi] & P) | (c1[gi] & PS))) | (lc[gi] & ((~c2[gi] & Q) | (c2[gi] & QS))))
                               : ((rc[gi] & P) | (lc[gi] & Q));
        acc[gi] |= eq[gi] & T & ~U[gi];  // this bit of u is 0 where t's is 1: u < t
        eq[gi] &= ~(T ^ U[gi]);          // equal so far
        any |= eq[gi];
      }
    }
  }
  if (COUNT) {
#pragma unroll
    for (int gi = 0; gi < 4; ++gi) {
      n_right += __popc(acc[gi] & rc[gi]);
      n_left += __popc(acc[gi] & lc[gi]);
    }
  }
  return apply_moves<PHASE>(x, acc);
}

// One phase over unit u of a ring resident in shared memory; the flip of
// bit 0 of the next unit's first word is left in carry[u] for its owner.
template <bool DIS, bool COUNT, bool FAST2, uint32_t PHASE, bool PQ = false>
__device__ __forceinline__ void sca_unit(uint32_t* lat, const uint32_t* cls, uint32_t* carry, const DomainLaunch& a,
                                         uint32_t u, uint32_t n_units, uint32_t W, uint64_t s, uint32_t n_glob,
                                         uint32_t kmax, unsigned long long& n_right, unsigned long long& n_left) {
  uint4* p4 = reinterpret_cast<uint4*>(lat + 8u * u);
  const uint4 v0 = p4[0], v1 = p4[1];
  uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
  if (PHASE == 0) {  // the previous unit's odd phase may have flipped bit 0 of our first word
    const uint32_t prev = (u == 0 ? n_units : u) - 1;
    x[0] ^= carry[prev];
    carry[prev] = 0u;
  }
  uint32_t c[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  if (DIS) {
    const uint4* c4 = reinterpret_cast<const uint4*>(cls + 8u * u);
    const uint4 d0 = c4[0], d1 = c4[1];
    c[0] = d0.x; c[1] = d0.y; c[2] = d0.z; c[3] = d0.w; c[4] = d1.x; c[5] = d1.y; c[6] = d1.z; c[7] = d1.w;
  }
  uint32_t d[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  if (PQ) load8(cls + W + 8u * u, d);  // the q classes follow the p classes
  const uint32_t next_w = (8u * u + 8u == W) ? 0u : 8u * u + 8u;
  const uint32_t x_next = PHASE ? lat[next_w] : 0u;  // only bit 0 is used
  const uint32_t c_next = (PHASE && DIS) ? cls[next_w] : 0u;
  const uint32_t d_next = (PHASE && PQ) ? cls[W + next_w] : 0u;
  const uint32_t carry_out = sca_update<DIS, COUNT, FAST2, PHASE, PQ>(x, c, d, x_next, c_next, d_next, a, u, s,
                                                                      n_glob, kmax, n_right, n_left);
  p4[0] = make_uint4(x[0], x[1], x[2], x[3]);
  p4[1] = make_uint4(x[4], x[5], x[6], x[7]);
  if (PHASE == 1) carry[u] = carry_out;
}

// Apply the pending carries of every plane (before a record or the write-back).
__device__ __forceinline__ void settle_carries(uint32_t* lat, uint32_t* carry, uint32_t n_units, uint32_t W,
                                               uint32_t planes) {
  for (uint32_t p = 0; p < planes; ++p)
    for (uint32_t u = threadIdx.x; u < n_units; u += blockDim.x) {
      const uint32_t prev = (u == 0 ? n_units : u) - 1;
      lat[p * W + 8u * u] ^= carry[p * n_units + prev];
    }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < planes * n_units; i += blockDim.x) carry[i] = 0u;
  __syncthreads();
}

// In-lane bonds of one lane of the two-lane model over one unit: lane A
// (LANE 0) moves particles right (10 -> 01) with threshold t = p, lane B
// (LANE 1) left (01 -> 10) with t = q.  Lane B's planes come from the stream
// with bit 31 of ctr3 set.  Every lane of a group has the same threshold, so
// a plane's threshold bit is uniform.
// Register form: x = the unit's 8 words, x_next = the next unit's first word
// (bit 0, odd phase); returns the flip of that bit (odd phase).
template <uint32_t LANE, uint32_t PHASE>
__device__ __forceinline__ uint32_t sca_lane_update(uint32_t (&x)[8], uint32_t x_next, const DomainLaunch& a,
                                                    uint32_t u, uint64_t s, uint32_t n_glob, uint32_t t,
                                                    unsigned long long& hops) {
  const bool always = t == 0xFFFFFFFFu, never = t == 0u;
  uint32_t acc[4], eq[4];
#pragma unroll
  for (int gi = 0; gi < 4; ++gi) {
    const uint32_t xa = x[2 * gi], xb = x[2 * gi + 1];
    const uint32_t xn = gi < 3 ? x[2 * gi + 2] : x_next;
    const uint32_t ya = PHASE ? __funnelshift_r(xa, xb, 1) : xa;
    const uint32_t yb = PHASE ? __funnelshift_r(xb, xn, 1) : xb;
    const uint32_t sa = ya >> 1, tb = yb << 1;
    const uint32_t cand = LANE == 0 ? ((ya & ~sa & kEven) | (tb & ~yb & kOdd))    // 10
                                    : ((~ya & sa & kEven) | (~tb & yb & kOdd));   // 01
    acc[gi] = always ? cand : 0u;
    eq[gi] = (always || never) ? 0u : cand;
  }
  const uint32_t t20 = t >> 12;
  const uint32_t kmax = (always || never) ? 0u : 21u - static_cast<uint32_t>(__ffs(t20));
  for (uint32_t k = 0; k < kmax; ++k) {
    if (k > 0 && (eq[0] | eq[1] | eq[2] | eq[3]) == 0u) break;
    const uint4 y = philox10(ctr_of(s, kTagSca, k, n_glob, (2u * u + PHASE) | (LANE << 31)), a.ks);
    const uint32_t U[4] = {y.x, y.y, y.z, y.w};
    if ((t20 >> (19u - k)) & 1u) {
#pragma unroll
      for (int gi = 0; gi < 4; ++gi) {
        acc[gi] |= eq[gi] & ~U[gi];
        eq[gi] &= U[gi];
      }
    } else {
#pragma unroll
      for (int gi = 0; gi < 4; ++gi) eq[gi] &= ~U[gi];
    }
  }
#pragma unroll
  for (int gi = 0; gi < 4; ++gi) hops += __popc(acc[gi]);
  return apply_moves<PHASE>(x, acc);
}

// One lane's in-lane phase over unit u of a plane resident in shared memory.
template <uint32_t LANE, uint32_t PHASE>
__device__ __forceinline__ void sca_lane_unit(uint32_t* plane, uint32_t* carry, const DomainLaunch& a, uint32_t u,
                                              uint32_t n_units, uint32_t W, uint64_t s, uint32_t n_glob, uint32_t t,
                                              unsigned long long& hops) {
  uint4* p4 = reinterpret_cast<uint4*>(plane + 8u * u);
  const uint4 v0 = p4[0], v1 = p4[1];
  uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
  if (PHASE == 0) {
    const uint32_t prev = (u == 0 ? n_units : u) - 1;
    x[0] ^= carry[prev];
    carry[prev] = 0u;
  }
  const uint32_t next_w = (8u * u + 8u == W) ? 0u : 8u * u + 8u;
  const uint32_t x_next = PHASE ? plane[next_w] : 0u;
  const uint32_t carry_out = sca_lane_update<LANE, PHASE>(x, x_next, a, u, s, n_glob, t, hops);
  p4[0] = make_uint4(x[0], x[1], x[2], x[3]);
  p4[1] = make_uint4(x[4], x[5], x[6], x[7]);
  if (PHASE == 1) carry[u] = carry_out;
}

// Lane changes of the two-lane model over one unit: STEP 0 (after the even
// phase) moves A -> B, STEP 1 (after the odd phase) B -> A, at turning sites
// whose source lane is occupied and target lane empty, with probability
// omega; one draw per candidate site (tag SCA_TURN, call = STEP, ctr3 =
// site / 4, word site mod 4).  STEP 1 first applies the odd phase's pending
// flips of bit 0 of the unit's first words.
// The lane changes of one word (global word index `word`): candidate sites
// are the set bits of `sel` (turning sites -- or, crossing kind, any site --
// with source occupied and target empty), accepted with omega, or with
// omega_slow where `marked` has the bit set (the crossing kind's reduced u_i
// or v_i); returns the bits that move.
template <uint32_t STEP>
__device__ __forceinline__ uint32_t sca_turn_word(uint32_t sel, uint32_t word, const DomainLaunch& a, uint64_t s,
                                                  uint32_t n_glob, unsigned long long& moves, uint32_t marked = 0u) {
  uint32_t f = 0u;
  while (sel) {
    const uint32_t b = static_cast<uint32_t>(__ffs(sel)) - 1u;
    sel &= sel - 1u;
    const uint32_t site = 32u * word + b;
    const uint4 r = philox10(ctr_of(s, kTagScaTurn, STEP, n_glob, site >> 2), a.ks);
    if (accept(pick(r, site & 3u), ((marked >> b) & 1u) ? a.rates.omega_slow : a.rates.omega)) {
      f |= 1u << b;
      ++moves;
    }
  }
  return f;
}

template <uint32_t STEP>
__device__ __forceinline__ uint32_t turn_candidates(uint32_t xa, uint32_t xb, uint32_t m) {
  return m & (STEP == 0 ? (xa & ~xb) : (xb & ~xa));
}

// XC (crossing kind): every site may cross; M holds the u-class plane, then
// the v-class plane, and STEP selects the one of its direction.
template <uint32_t STEP, bool XC = false>
__device__ __forceinline__ void sca_turn_unit(uint32_t* A, uint32_t* B, const uint32_t* M, uint32_t* carry,
                                              const DomainLaunch& a, uint32_t u, uint32_t n_units, uint32_t W,
                                              uint64_t s, uint32_t n_glob, unsigned long long& moves) {
  uint4* pa = reinterpret_cast<uint4*>(A + 8u * u);
  uint4* pb = reinterpret_cast<uint4*>(B + 8u * u);
  const uint4 a0 = pa[0], a1 = pa[1], b0 = pb[0], b1 = pb[1];
  uint32_t xa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
  uint32_t xb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
  uint32_t m[8], mk[8];  // candidate sites, marked sites
  if (XC) {
    load8(M + STEP * W + 8u * u, mk);
#pragma unroll
    for (int w = 0; w < 8; ++w) m[w] = ~0u;
  } else {
    load8(M + 8u * u, m);
#pragma unroll
    for (int w = 0; w < 8; ++w) mk[w] = 0u;
  }
  if (STEP == 1) {
    const uint32_t prev = (u == 0 ? n_units : u) - 1;
    xa[0] ^= carry[prev];
    xb[0] ^= carry[n_units + prev];
    carry[prev] = 0u;
    carry[n_units + prev] = 0u;
  }
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const uint32_t f =
        sca_turn_word<STEP>(turn_candidates<STEP>(xa[w], xb[w], m[w]), 8u * u + w, a, s, n_glob, moves, mk[w]);
    xa[w] ^= f;
    xb[w] ^= f;
  }
  pa[0] = make_uint4(xa[0], xa[1], xa[2], xa[3]);
  pa[1] = make_uint4(xa[4], xa[5], xa[6], xa[7]);
  pb[0] = make_uint4(xb[0], xb[1], xb[2], xb[3]);
  pb[1] = make_uint4(xb[4], xb[5], xb[6], xb[7]);
}

// Heights, W^2 sums and the other observables of one record, per plane, from
// the lattice in shared memory (contiguous chunks of words per thread), and
// the hop counters of the sample (cnt: this thread's increments since the
// last record, cleared here).
template <uint32_t NOCC, bool COUNT>
__device__ void sca_record(const uint32_t* lat, const DomainLaunch& a, uint32_t slot, uint64_t t, uint32_t sample,
                           long long* warp_tot, unsigned long long* warp_s2, unsigned long long* cnt) {
  const uint32_t W = a.geo.W;
  const uint32_t chunk = (W + blockDim.x - 1) / blockDim.x;
  const uint32_t w0 = min(W, threadIdx.x * chunk), w1 = min(W, w0 + chunk);
  const Extras& ex = a.ex;
  for (uint32_t p = 0; p < NOCC; ++p) {
    const uint32_t* pl = lat + p * W;
    long long tot = 0;
    for (uint32_t i = w0; i < w1; ++i) tot += 2 * __popc(pl[i]) - 32;
    long long h = block_scan_incl(tot, warp_tot) - tot, s1 = 0;
    unsigned long long s2 = 0;
    for (uint32_t i = w0; i < w1; ++i) {
      const uint32_t x = pl[i];
      for (uint32_t b = 0; b < 32; ++b) {
        h += ((x >> b) & 1u) ? 1 : -1;
        s1 += h;
        s2 += static_cast<unsigned long long>(h * h);
      }
    }
    const long long s1_all = block_sum(s1, warp_tot);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if ((threadIdx.x & 31u) == 0) warp_s2[threadIdx.x >> 5] = s2;
    __syncthreads();
    const size_t e = (static_cast<size_t>(slot) * a.geo.S + sample) * NOCC + p;
    if (threadIdx.x == 0) {
      unsigned __int128 acc = 0;
      for (uint32_t i = 0; i < (blockDim.x >> 5); ++i) acc += warp_s2[i];
      a.tab_sh[e] = s1_all;
      a.tab_sh2[2 * e] = static_cast<uint64_t>(acc);
      a.tab_sh2[2 * e + 1] = static_cast<uint64_t>(acc >> 64);
    }
    if (ex.profile || ex.snap) {
      const size_t base = (static_cast<size_t>(sample) * NOCC + p) * W;
      long long ov = 0;
      for (uint32_t i = w0; i < w1; ++i) {
        const uint32_t x = pl[i];
        if (ex.profile) ex.profile[base + i] += __popc(x);
        if (ex.snap) {
          if (t == ex.t0) ex.snap[base + i] = x;
          if (t >= ex.t0) ov += __popc(x & ex.snap[base + i]);
        }
      }
      if (ex.snap) {
        const long long tot_ov = block_sum(ov, warp_tot);
        if (threadIdx.x == 0) ex.tab_ac[e] = tot_ov;
      }
    }
    __syncthreads();
  }
  // hop counters of this sample up to now
  long long tot_cnt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    tot_cnt[k] = COUNT ? block_sum(static_cast<long long>(cnt[k]), warp_tot) : 0;
    cnt[k] = 0;
  }
  if (threadIdx.x == 0) {
    uint64_t* ctr = a.counters + 4ull * sample;
    const size_t ec = (static_cast<size_t>(slot) * a.geo.S + sample) * 4;
    for (int k = 0; k < 4; ++k) {
      ctr[k] += static_cast<uint64_t>(tot_cnt[k]);
      a.ex.tab_cnt[ec + k] = static_cast<int64_t>(ctr[k]);
    }
  }
  __syncthreads();
}

// The SCA kernel.  Ring (MODEL 0): one lattice plane, optionally a bimodal
// class plane (DIS), or the p-class and q-class planes (DIS and PQ).  Two
// lanes (MODEL 1): planes A and B and, with turning sites (DIS), the turning
// plane and the lane-change steps.  A quenched plane costs registers in
// every step: at most 512 threads then, so the compiler may use up to 128
// registers.
template <uint32_t MODEL, bool DIS, bool COUNT, bool FAST2, bool PQ = false>
__global__ void __launch_bounds__(DIS ? 512 : 1024) k_sca(const DomainLaunch a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long warp_tot[32];
  __shared__ unsigned long long warp_s2[32];
  constexpr uint32_t NOCC = MODEL == kTwoLane ? 2u : 1u;
  const uint32_t W = a.geo.W, n_units = W / 8;
  uint32_t* lat = reinterpret_cast<uint32_t*>(smem_raw);  // NOCC planes
  constexpr uint32_t NQ = DIS ? (PQ ? 2u : 1u) : 0u;      // quenched planes
  uint32_t* qp = lat + NOCC * W;                          // class (p, q classes) or turning plane
  uint32_t* carry = qp + NQ * W;                          // NOCC x n_units flags
  const uint32_t sample = blockIdx.x;
  const uint32_t n_glob = a.geo.first_sample + sample;
  const uint64_t s0 = a.clock->sweep;
  uint32_t rec = a.clock->next_time;
  const uint32_t kmax = a.sca_kmax;

  for (uint32_t i = threadIdx.x; i < NOCC * W; i += blockDim.x)
    lat[i] = a.state[static_cast<size_t>(sample) * NOCC * W + i];
  if (DIS)
    for (uint32_t i = threadIdx.x; i < NQ * W; i += blockDim.x)
      qp[i] = a.mask[static_cast<size_t>(sample / a.geo.samples_per_real) * NQ * W + i];
  for (uint32_t i = threadIdx.x; i < NOCC * n_units; i += blockDim.x) carry[i] = 0u;
  __syncthreads();

  unsigned long long cnt[4] = {0ull, 0ull, 0ull, 0ull};
  for (uint32_t it = 0; it < a.n_sweeps; ++it) {
    const uint64_t s = s0 + it;
    if (MODEL == kRing) {
      for (uint32_t u = threadIdx.x; u < n_units; u += blockDim.x)
        sca_unit<DIS, COUNT, FAST2, 0, PQ>(lat, qp, carry, a, u, n_units, W, s, n_glob, kmax, cnt[0], cnt[1]);
      __syncthreads();
      for (uint32_t u = threadIdx.x; u < n_units; u += blockDim.x)
        sca_unit<DIS, COUNT, FAST2, 1, PQ>(lat, qp, carry, a, u, n_units, W, s, n_glob, kmax, cnt[0], cnt[1]);
      __syncthreads();
    } else {
      uint32_t* A = lat;
      uint32_t* B = lat + W;
      for (uint32_t u = threadIdx.x; u < n_units; u += blockDim.x) {
        sca_lane_unit<0, 0>(A, carry, a, u, n_units, W, s, n_glob, a.rates.p, cnt[0]);
        sca_lane_unit<1, 0>(B, carry + n_units, a, u, n_units, W, s, n_glob, a.rates.q, cnt[1]);
      }
      __syncthreads();
      if (DIS) {
        for (uint32_t u = threadIdx.x; u < n_units; u += blockDim.x)
          sca_turn_unit<0, PQ>(A, B, qp, carry, a, u, n_units, W, s, n_glob, cnt[2]);
        __syncthreads();
      }
      for (uint32_t u = threadIdx.x; u < n_units; u += blockDim.x) {
        sca_lane_unit<0, 1>(A, carry, a, u, n_units, W, s, n_glob, a.rates.p, cnt[0]);
        sca_lane_unit<1, 1>(B, carry + n_units, a, u, n_units, W, s, n_glob, a.rates.q, cnt[1]);
      }
      __syncthreads();
      if (DIS) {
        for (uint32_t u = threadIdx.x; u < n_units; u += blockDim.x)
          sca_turn_unit<1, PQ>(A, B, qp, carry, a, u, n_units, W, s, n_glob, cnt[3]);
        __syncthreads();
      }
    }
    if (rec < a.n_times && a.times[rec] == s + 1) {
      settle_carries(lat, carry, n_units, W, NOCC);
      sca_record<NOCC, COUNT>(lat, a, rec, s + 1, sample, warp_tot, warp_s2, cnt);
      ++rec;
    }
  }
  settle_carries(lat, carry, n_units, W, NOCC);
  for (uint32_t i = threadIdx.x; i < NOCC * W; i += blockDim.x)
    a.state[static_cast<size_t>(sample) * NOCC * W + i] = lat[i];
  if (COUNT) {
    long long tot[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) tot[k] = block_sum(static_cast<long long>(cnt[k]), warp_tot);
    if (threadIdx.x == 0)
      for (int k = 0; k < 4; ++k) a.counters[4ull * sample + k] += static_cast<uint64_t>(tot[k]);
  }
}

// Ring without disorder, rates neither 0 nor "always", at most two random
// planes: the specialised comparison.
bool sca_fast2(const DomainLaunch& a) {
  const auto regular = [](uint32_t t) { return t != 0u && t != 0xFFFFFFFFu; };
  return regular(a.rates.p) && regular(a.rates.q) && a.sca_kmax <= 2;
}

template <uint32_t MODEL, bool DIS, bool COUNT, bool FAST2, bool PQ = false>
cudaError_t launch_sca_t(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st) {
  (void)cudaGetLastError();
  const cudaError_t e = cudaFuncSetAttribute(k_sca<MODEL, DIS, COUNT, FAST2, PQ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_sca<MODEL, DIS, COUNT, FAST2, PQ><<<a.geo.S, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Streamed SCA, for rings beyond one CTA's shared memory (the paper's mode of
// one large sample per GPU held in device memory).  The lattice stays in
// global memory in its natural layout; a sweep is one launch per phase, one
// thread per unit (two 128-bit loads per plane).  Even bonds lie inside a
// word, so the even phase needs nothing from other units.  The odd bond
// (32w + 31, 32w + 32) that ends in the next unit flips bit 0 of that unit's
// first word, a bit no bond of its owner touches: the owner merges the bits
// it changed in its first word with an atomic XOR, the previous unit's owner
// flips bit 0 the same way, so the lattice is settled after every launch.
//
// Two lanes: the lane changes that follow a phase are fused into its launch.
// After the even phase a unit's sites depend on that unit alone.  After the
// odd phase site 256(u + 1) also depends on unit u's last bond, so the owner
// of unit u takes the lane changes of sites 256u + 1 .. 256(u + 1) and merges
// them into the next unit's first words with its carry.
constexpr uint32_t kScaStreamThreads = 256;

// Write back a unit: all 8 words after an even phase; after an odd phase
// words 1..7 plainly and word 0 as the XOR of the bits this thread changed
// (`old0` = word 0 as loaded), then the carry into the next unit (`nw`).
template <uint32_t PHASE>
__device__ __forceinline__ void store_unit(uint32_t* p, const uint32_t (&x)[8], uint32_t old0, uint32_t* nw,
                                           uint32_t carry) {
  if (PHASE == 0) {
    reinterpret_cast<uint4*>(p)[0] = make_uint4(x[0], x[1], x[2], x[3]);
    reinterpret_cast<uint4*>(p)[1] = make_uint4(x[4], x[5], x[6], x[7]);
  } else {
    p[1] = x[1];
    *reinterpret_cast<uint2*>(p + 2) = make_uint2(x[2], x[3]);
    reinterpret_cast<uint4*>(p)[1] = make_uint4(x[4], x[5], x[6], x[7]);
    if (x[0] != old0) atomicXor(p, x[0] ^ old0);
    if (carry) atomicXor(nw, carry);
  }
}

// Two lanes: one phase and its lane changes over every sample, a thread per
// unit.  Grid: S x blocks_per_sample CTAs, blockIdx.x = sample *
// blocks_per_sample + block.  DIS: turning sites.
template <bool DIS, uint32_t PHASE, bool XC = false>
__global__ void __launch_bounds__(kScaStreamThreads) k_sca_stream_lanes(const DomainLaunch a,
                                                                         uint32_t blocks_per_sample) {
  __shared__ unsigned long long red[kScaStreamThreads / 32][4];
  const uint32_t W = a.geo.W, n_units = W / 8;
  const uint32_t sample = blockIdx.x / blocks_per_sample;
  const uint32_t u = (blockIdx.x - sample * blocks_per_sample) * kScaStreamThreads + threadIdx.x;
  const uint32_t n_glob = a.geo.first_sample + sample;
  const uint64_t s = a.clock->sweep;
  unsigned long long cnt[4] = {0ull, 0ull, 0ull, 0ull};
  if (u < n_units) {
    const uint32_t nw = (8u * u + 8u == W) ? 0u : 8u * u + 8u;  // the next unit's first word
    const size_t real = sample / a.geo.samples_per_real;
    {
      uint32_t* A = a.state + static_cast<size_t>(sample) * 2u * W;
      uint32_t* B = A + W;
      uint32_t xa[8], xb[8];
      load8(A + 8u * u, xa);
      load8(B + 8u * u, xb);
      const uint32_t a0 = xa[0], b0 = xb[0];
      const uint32_t na = PHASE ? A[nw] : 0u, nb = PHASE ? B[nw] : 0u;
      uint32_t oa = sca_lane_update<0, PHASE>(xa, na, a, u, s, n_glob, a.rates.p, cnt[0]);
      uint32_t ob = sca_lane_update<1, PHASE>(xb, nb, a, u, s, n_glob, a.rates.q, cnt[1]);
      if (DIS) {
        // turning plane, or (XC) every site with the u-class / v-class plane of this phase's direction
        const uint32_t* M = a.mask + real * (XC ? 2u : 1u) * W;
        const uint32_t* Mk = M + PHASE * W;
        uint32_t m[8], mk[8];
        if (XC) {
          load8(Mk + 8u * u, mk);
#pragma unroll
          for (int w = 0; w < 8; ++w) m[w] = ~0u;
        } else {
          load8(M + 8u * u, m);
#pragma unroll
          for (int w = 0; w < 8; ++w) mk[w] = 0u;
        }
        if (PHASE == 1) m[0] &= ~1u;  // site 256u belongs to the previous unit's owner
#pragma unroll
        for (int w = 0; w < 8; ++w) {
          const uint32_t f = sca_turn_word<PHASE>(turn_candidates<PHASE>(xa[w], xb[w], m[w]), 8u * u + w, a, s,
                                                  n_glob, cnt[2 + PHASE], mk[w]);
          xa[w] ^= f;
          xb[w] ^= f;
        }
        if (PHASE == 1) {  // site 256(u + 1) = bit 0 of word nw, after this unit's last bond
          const uint32_t cand = XC ? 1u : (M[nw] & 1u), marked = XC ? (Mk[nw] & 1u) : 0u;
          const uint32_t f = sca_turn_word<1>(turn_candidates<1>(na ^ oa, nb ^ ob, cand), nw, a, s, n_glob,
                                              cnt[3], marked);
          oa ^= f;
          ob ^= f;
        }
      }
      store_unit<PHASE>(A + 8u * u, xa, a0, A + nw, oa);
      store_unit<PHASE>(B + 8u * u, xb, b0, B + nw, ob);
    }
  }
  {
    constexpr int NK = DIS ? 4 : 2;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      unsigned long long v = cnt[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31u) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NK) {
      unsigned long long v = 0;
      for (uint32_t w = 0; w < kScaStreamThreads / 32; ++w) v += red[w][threadIdx.x];
      if (v) atomicAdd(reinterpret_cast<unsigned long long*>(a.counters + 4ull * sample + threadIdx.x), v);
    }
  }
}

// The ring: a thread takes `upt` units, T apart (coalesced), and loads the
// next one's words while it updates the current one, so that two units'
// loads are in flight per thread (the one-unit form stalls on them).  The
// 32 lanes of a warp hold 32 consecutive units, so in the odd phase a lane
// takes bit 0 of the next unit's first word from its neighbour lane and
// passes its carry to it by shuffles, and stores its 8 words plainly after
// merging the carry it received.  Only the warp's ends touch other warps'
// units: the last active lane loads the next unit's first word and merges
// its carry into it atomically, lane 0 merges the bits it changed in its
// first word atomically (that word receives the previous warp's carry).
// A first word lane 0 prefetched may or may not hold that carry already:
// bit 0 is not read by the odd phase.
template <bool DIS, bool COUNT, bool FAST2, uint32_t PHASE, bool PQ = false>
__global__ void __launch_bounds__(kScaStreamThreads, DIS ? 2 : 4) k_sca_stream_ring(const DomainLaunch a,
                                                                        uint32_t blocks_per_sample, uint32_t upt) {
  constexpr uint32_t T = kScaStreamThreads;
  __shared__ unsigned long long red[T / 32][2];
  const uint32_t W = a.geo.W, n_units = W / 8;
  const uint32_t sample = blockIdx.x / blocks_per_sample;
  const uint32_t u_first = (blockIdx.x - sample * blocks_per_sample) * (T * upt) + threadIdx.x;
  const uint32_t n_glob = a.geo.first_sample + sample;
  const uint64_t s = a.clock->sweep;
  const uint32_t kmax = a.sca_kmax;
  uint32_t* lat = a.state + static_cast<size_t>(sample) * W;
  constexpr uint32_t NQ = DIS ? (PQ ? 2u : 1u) : 0u;  // p classes, then (PQ) q classes
  const uint32_t* cls = DIS ? a.mask + static_cast<size_t>(sample / a.geo.samples_per_real) * NQ * W : nullptr;
  unsigned long long nr = 0ull, nl = 0ull;
  const uint32_t lane = threadIdx.x & 31u;
  // active lanes of the warp for unit u (lane `lane`): a prefix of the warp
  auto n_active = [&](uint32_t u) { return min(32u, n_units - (u - lane)); };
  uint32_t px[8], pc[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u}, pd[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  uint32_t pxn = 0u, pcn = 0u, pdn = 0u;  // the next unit's words
  auto fetch = [&](uint32_t u) {
    load8(lat + 8u * u, px);
    if (DIS) load8(cls + 8u * u, pc);
    if (PQ) load8(cls + W + 8u * u, pd);
    if (PHASE && lane + 1 == n_active(u)) {  // the warp's last unit: the next unit's first words
      const uint32_t nw = (8u * u + 8u == W) ? 0u : 8u * u + 8u;
      pxn = lat[nw];  // only bit 0, which only this thread changes
      if (DIS) pcn = cls[nw];
      if (PQ) pdn = cls[W + nw];
    }
  };
  if (u_first < n_units) fetch(u_first);
#pragma unroll 1
  for (uint32_t k = 0; k < upt; ++k) {
    const uint32_t u = u_first + k * T;
    if (u >= n_units) break;
    uint32_t x[8], c[8], d[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      x[w] = px[w];
      c[w] = pc[w];
      d[w] = pd[w];
    }
    uint32_t x_next = pxn, c_next = pcn, d_next = pdn;
    const uint32_t na = n_active(u);
    const unsigned act = na == 32u ? 0xffffffffu : (1u << na) - 1u;
    const bool last = lane + 1 == na;
    if (PHASE) {
      const uint32_t xs = __shfl_down_sync(act, x[0], 1);
      const uint32_t cs = DIS ? __shfl_down_sync(act, c[0], 1) : 0u;
      const uint32_t ds = PQ ? __shfl_down_sync(act, d[0], 1) : 0u;
      if (!last) {
        x_next = xs;
        c_next = cs;
        d_next = ds;
      }
    }
    if (k + 1 < upt && u + T < n_units) fetch(u + T);
    const uint32_t old0 = x[0];
    const uint32_t out = sca_update<DIS, COUNT, FAST2, PHASE, PQ>(x, c, d, x_next, c_next, d_next, a, u, s, n_glob,
                                                                  kmax, nr, nl);
    uint32_t* p = lat + 8u * u;
    if (PHASE == 0) {
      reinterpret_cast<uint4*>(p)[0] = make_uint4(x[0], x[1], x[2], x[3]);
      reinterpret_cast<uint4*>(p)[1] = make_uint4(x[4], x[5], x[6], x[7]);
    } else {
      const uint32_t cin = __shfl_up_sync(act, out, 1);  // the carry of the unit before, from lane - 1
      if (lane > 0) {
        x[0] ^= cin;
        reinterpret_cast<uint4*>(p)[0] = make_uint4(x[0], x[1], x[2], x[3]);
        reinterpret_cast<uint4*>(p)[1] = make_uint4(x[4], x[5], x[6], x[7]);
      } else {
        store_unit<1>(p, x, old0, nullptr, 0u);  // words 1..7 plainly, word 0 by atomic XOR of the change
      }
      if (last && out) atomicXor(lat + ((8u * u + 8u == W) ? 0u : 8u * u + 8u), out);
    }
  }
  if (COUNT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nr += __shfl_xor_sync(0xffffffffu, nr, o);
      nl += __shfl_xor_sync(0xffffffffu, nl, o);
    }
    if ((threadIdx.x & 31u) == 0) {
      red[threadIdx.x >> 5][0] = nr;
      red[threadIdx.x >> 5][1] = nl;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      unsigned long long v = 0;
      for (uint32_t w = 0; w < T / 32; ++w) v += red[w][threadIdx.x];
      if (v) atomicAdd(reinterpret_cast<unsigned long long*>(a.counters + 4ull * sample + threadIdx.x), v);
    }
  }
}

template <uint32_t MODEL, bool DIS, bool COUNT, bool FAST2, bool PQ = false>
cudaError_t launch_sca_stream_t(const DomainLaunch& a, cudaStream_t st) {
  const uint32_t n_units = a.geo.W / 8;
  (void)cudaGetLastError();
  if constexpr (MODEL == kRing) {
    // units per thread: 4, 2 or 1, the most that still leaves eight waves of CTAs (152 SMs x 5), so
    // that the last, partial wave costs little; in practice lattices far beyond L2 get 4, the rest 1
    const uint64_t units = static_cast<uint64_t>(n_units) * a.geo.S;
    uint32_t upt = 4;
    while (upt > 1 && units < static_cast<uint64_t>(upt) * kScaStreamThreads * 8u * 152u * 5u) upt >>= 1;
    const uint32_t per_block = kScaStreamThreads * upt;
    const uint32_t bps = (n_units + per_block - 1) / per_block;
    k_sca_stream_ring<DIS, COUNT, FAST2, 0, PQ><<<bps * a.geo.S, kScaStreamThreads, 0, st>>>(a, bps, upt);
    k_sca_stream_ring<DIS, COUNT, FAST2, 1, PQ><<<bps * a.geo.S, kScaStreamThreads, 0, st>>>(a, bps, upt);
  } else {
    const uint32_t bps = (n_units + kScaStreamThreads - 1) / kScaStreamThreads;
    k_sca_stream_lanes<DIS, 0, PQ><<<bps * a.geo.S, kScaStreamThreads, 0, st>>>(a, bps);
    k_sca_stream_lanes<DIS, 1, PQ><<<bps * a.geo.S, kScaStreamThreads, 0, st>>>(a, bps);
  }
  return cudaGetLastError();
}

}  // namespace

size_t sca_smem_bytes(uint32_t W, uint32_t planes, uint32_t quenched_planes) {
  return static_cast<size_t>(W) * 4u * (planes + quenched_planes) + static_cast<size_t>(planes) * (W / 8u) * 4u;
}

cudaError_t launch_sca(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st) {
  const bool count = a.count_hops != 0;
  if (a.model == kTwoLane) {  // two lanes always count hops and turns
    if (a.dis == kDisCrossing) return launch_sca_t<kTwoLane, true, true, false, true>(a, threads, smem, st);
    return a.dis == kDisTurning ? launch_sca_t<kTwoLane, true, true, false>(a, threads, smem, st)
                                : launch_sca_t<kTwoLane, false, true, false>(a, threads, smem, st);
  }
  if (a.dis == kDisBimodal)
    return count ? launch_sca_t<kRing, true, true, false>(a, threads, smem, st)
                 : launch_sca_t<kRing, true, false, false>(a, threads, smem, st);
  if (a.dis == kDisBimodalPQ)
    return count ? launch_sca_t<kRing, true, true, false, true>(a, threads, smem, st)
                 : launch_sca_t<kRing, true, false, false, true>(a, threads, smem, st);
  if (sca_fast2(a))
    return count ? launch_sca_t<kRing, false, true, true>(a, threads, smem, st)
                 : launch_sca_t<kRing, false, false, true>(a, threads, smem, st);
  return count ? launch_sca_t<kRing, false, true, false>(a, threads, smem, st)
               : launch_sca_t<kRing, false, false, false>(a, threads, smem, st);
}


cudaError_t launch_sca_stream(const DomainLaunch& a, cudaStream_t st) {
  const bool count = a.count_hops != 0;
  if (a.model == kTwoLane) {  // two lanes always count hops and turns
    if (a.dis == kDisCrossing) return launch_sca_stream_t<kTwoLane, true, true, false, true>(a, st);
    return a.dis == kDisTurning ? launch_sca_stream_t<kTwoLane, true, true, false>(a, st)
                                : launch_sca_stream_t<kTwoLane, false, true, false>(a, st);
  }
  if (a.dis == kDisBimodal)
    return count ? launch_sca_stream_t<kRing, true, true, false>(a, st)
                 : launch_sca_stream_t<kRing, true, false, false>(a, st);
  if (a.dis == kDisBimodalPQ)
    return count ? launch_sca_stream_t<kRing, true, true, false, true>(a, st)
                 : launch_sca_stream_t<kRing, true, false, false, true>(a, st);
  if (sca_fast2(a))
    return count ? launch_sca_stream_t<kRing, false, true, true>(a, st)
                 : launch_sca_stream_t<kRing, false, false, true>(a, st);
  return count ? launch_sca_stream_t<kRing, false, true, false>(a, st)
               : launch_sca_stream_t<kRing, false, false, false>(a, st);
}

}  // namespace asep

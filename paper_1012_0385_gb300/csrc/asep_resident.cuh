// asep_resident.cuh -- the resident tier of the two-phase Poisson-domain
// schedule: one or more whole samples in one CTA's shared memory (layout in
// asep_kernels.cu).  run_group advances one sample group for a number of
// sweeps from a given sweep index and record cursor; it is shared by the
// one-launch kernel and the persistent batch kernel (asep_kernels.cu) and by
// the balanced kernel (asep_balance.cu).  Internal linkage: every kernel file
// gets its own copy.
#pragma once

#include <cstdint>

#include "asep_device.cuh"
#include "asep_domain.cuh"
#include "asep_internal.h"

namespace asep {
namespace {

// ---------------------------------------------------------------------------
// Segmented scan (all threads of the block must call)
// ---------------------------------------------------------------------------

// Segmented scan over the columns [col0, col0 + G) of one sample.
__device__ void seg_scan(long long v, uint32_t col0, uint32_t G, long long* warp_tot, long long* arr,
                         long long& excl_in_seg, long long& seg_total) {
  const long long inc = block_scan_incl(v, warp_tot);
  arr[threadIdx.x] = inc;
  __syncthreads();
  const long long before = col0 > 0 ? arr[col0 - 1] : 0;
  excl_in_seg = inc - v - before;
  seg_total = arr[col0 + G - 1] - before;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Resident two-phase Poisson-domain kernel
// ---------------------------------------------------------------------------

// Hop counters of one lane (named fields so they stay in registers).

// Rotate the planes of one column from frame offset R_old to R_new:
// new frame word f = g*R2 + r holds logical sites R_new + 32 f .. + 31.
template <uint32_t NP>
__device__ __forceinline__ void realign(const uint32_t* src, uint32_t* dst, const DomainLaunch& a, const Lane& ln,
                                        uint32_t PW, uint32_t delta) {
  const uint64_t L = a.geo.L;
  const uint32_t W = a.geo.W, R2 = a.R2, Cp = a.Cp;
  for (uint32_t r = 0; r < R2; ++r) {
    uint64_t pos = delta + 32ull * (ln.g * R2 + r);
    if (pos >= L) pos -= L;
    const uint32_t fa = static_cast<uint32_t>(pos >> 5), sh = static_cast<uint32_t>(pos & 31u);
    const uint32_t fb = (fa + 1 == W) ? 0u : fa + 1;
    const uint32_t ia = (fa & (R2 - 1)) * Cp + ln.col0 + (fa >> a.logR2);
    const uint32_t ib = (fb & (R2 - 1)) * Cp + ln.col0 + (fb >> a.logR2);
#pragma unroll
    for (uint32_t p = 0; p < NP; ++p)
      dst[p * PW + r * Cp + ln.c] = __funnelshift_r(src[p * PW + ia], src[p * PW + ib], sh);
  }
}

// Mirror row: copy row 0 of the next column into row R2 of this column (all
// planes), after the even phase and before the odd phase.
template <uint32_t NP>
__device__ __forceinline__ void mirror_in(uint32_t* cur, const DomainLaunch& a, uint32_t PW, const Lane& ln) {
#pragma unroll
  for (uint32_t p = 0; p < NP; ++p) cur[p * PW + a.R2 * a.Cp + ln.c] = cur[p * PW + ln.c_next];
}

// After the odd phase: the only bit of row 0 another lane may have changed is
// bit 0 (the previous column's last odd bond); take it back from its mirror.
template <uint32_t NOCC>
__device__ __forceinline__ void mirror_out(uint32_t* cur, const DomainLaunch& a, uint32_t PW, const Lane& ln) {
#pragma unroll
  for (uint32_t p = 0; p < NOCC; ++p) {
    const uint32_t w = cur[p * PW + ln.c];
    const uint32_t m = cur[p * PW + a.R2 * a.Cp + ln.c_prev];
    cur[p * PW + ln.c] = (w & ~1u) | (m & 1u);
  }
}

// Lane changes of the two-lane model in one column: at every turning site
// (DIS = kDisTurning: the sites of the turning plane, probability omega both
// ways) or every site (DIS = kDisCrossing: A -> B with u_i, B -> A with v_i,
// the slow value at sites marked in the u and v planes) where exactly one
// lane is occupied.
template <uint32_t DIS>
__device__ __forceinline__ void turning(uint32_t* cur, const DomainLaunch& a, uint32_t PW, uint64_t s,
                                        uint32_t R_cur, const Lane& ln, uint2 key, Cnt& cnt) {
  uint32_t* A = cur;
  uint32_t* B = cur + PW;
  const uint32_t* M = cur + 2 * PW;  // turning plane, or the u marks (the v marks follow)
  const uint64_t L = a.geo.L;
  for (uint32_t r = 0; r < a.R2; ++r) {
    const uint32_t idx = r * a.Cp + ln.c;
    uint32_t av = A[idx], bv = B[idx];
    uint32_t e = DIS == kDisCrossing ? (av ^ bv) : M[idx] & (av ^ bv);
    const uint32_t um = DIS == kDisCrossing ? M[idx] : 0u, vm = DIS == kDisCrossing ? M[PW + idx] : 0u;
    while (e) {
      const uint32_t b = __ffs(e) - 1;
      e &= e - 1;
      uint64_t site = static_cast<uint64_t>(R_cur) + 32ull * (ln.g * a.R2 + r) + b;
      if (site >= L) site -= L;
      const uint4 x = philox10(ctr_of(s, kTagTurn, 0, ln.n_glob, static_cast<uint32_t>(site >> 2)), key);
      uint32_t t = a.rates.omega;
      if (DIS == kDisCrossing && ((((av >> b) & 1u) ? um : vm) >> b) & 1u) t = a.rates.omega_slow;
      if (accept(pick(x, static_cast<uint32_t>(site & 3u)), t)) {
        const uint32_t bit = 1u << b;
        if (av & bit) ++cnt.c;
        else ++cnt.d;
        av ^= bit;
        bv ^= bit;
      }
    }
    A[idx] = av;
    B[idx] = bv;
  }
}

// Heights of the occupancy planes (frame offset 0) into table slot `slot`.
template <uint32_t NOCC>
__device__ void record_heights(const uint32_t* cur, const DomainLaunch& a, uint32_t PW, uint32_t slot, const Lane& ln,
                               long long* warp_tot, long long* arr) {
  for (uint32_t p = 0; p < NOCC; ++p) {
    const uint32_t* pl = cur + p * PW;
    long long tot = 0;
    if (ln.active)
      for (uint32_t r = 0; r < a.R2; ++r) tot += 2 * __popc(pl[r * a.Cp + ln.c]) - 32;
    long long h0, seg_unused;
    seg_scan(tot, ln.col0, a.G, warp_tot, arr, h0, seg_unused);
    long long s1 = 0, s2 = 0;
    if (ln.active) {
      long long h = h0;
      for (uint32_t r = 0; r < a.R2; ++r) {
        const uint32_t x = pl[r * a.Cp + ln.c];
        for (uint32_t b = 0; b < 32; ++b) {
          h += ((x >> b) & 1u) ? 1 : -1;
          s1 += h;
          s2 += h * h;
        }
      }
    }
    long long e1, t1, e2, t2;
    seg_scan(s1, ln.col0, a.G, warp_tot, arr, e1, t1);
    seg_scan(s2, ln.col0, a.G, warp_tot, arr, e2, t2);
    if (ln.active && ln.g == 0) {
      const size_t e = (static_cast<size_t>(slot) * a.geo.S + ln.sample) * NOCC + p;
      a.tab_sh[e] = t1;
      a.tab_sh2[2 * e] = static_cast<uint64_t>(t2);
      a.tab_sh2[2 * e + 1] = 0;
    }
  }
}

// Sweeps of one sample group (spc samples, one column per thread) of one
// context, for a.n_sweeps sweeps starting at the context clock.  Used by the
// one-launch-per-context kernel (group = blockIdx.x) and by the persistent
// batch kernel (group from the work queue).  All threads of the block call.
// The other observables at a sample time t (frame offset 0): cumulative hop
// counters (lane counters are flushed first), the occupancy profile, and the
// overlap with the reference lattice of the density autocorrelation.
template <uint32_t NOCC>
__device__ void record_extras(const uint32_t* cur, const DomainLaunch& a, uint32_t PW, uint32_t slot, uint64_t t,
                              const Lane& ln, long long* warp_tot, long long* arr, Cnt& cnt) {
  const Extras& ex = a.ex;
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(a.counters + 4ull * ln.sample);
  if (ln.active) {
    if (cnt.a) atomicAdd(ctr + 0, static_cast<unsigned long long>(cnt.a));
    if (cnt.b) atomicAdd(ctr + 1, static_cast<unsigned long long>(cnt.b));
    if (cnt.c) atomicAdd(ctr + 2, static_cast<unsigned long long>(cnt.c));
    if (cnt.d) atomicAdd(ctr + 3, static_cast<unsigned long long>(cnt.d));
    cnt = Cnt();
  }
  __syncthreads();  // the block's counter updates are visible below
  if (ln.active && ln.g == 0) {
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
        if (ex.profile) ex.profile[base + r] = __ldcg(&ex.profile[base + r]) + __popc(x);
        if (ex.snap) {
          if (t == ex.t0) ex.snap[base + r] = x;
          if (t >= ex.t0) ov += __popc(x & (t == ex.t0 ? x : __ldcg(&ex.snap[base + r])));
        }
      }
    }
    if (ex.snap) {
      long long e_unused, tot;
      seg_scan(ov, ln.col0, a.G, warp_tot, arr, e_unused, tot);
      if (ln.active && ln.g == 0) ex.tab_ac[(static_cast<size_t>(slot) * a.geo.S + ln.sample) * NOCC + p] = tot;
    }
  }
}

// Global data a group reads at its start (lattice) and at records (profile,
// reference lattice) may have been written by another CTA of the same launch
// (the balanced kernel hands groups between CTAs): read them from L2
// (ld.global.cg), never from a possibly stale L1 line.
template <uint32_t MODEL, uint32_t DIS, bool COUNT, uint32_t CP>
__device__ __forceinline__ void run_group(const DomainLaunch& a, uint32_t group, unsigned char* smem_raw,
                                          uint64_t s0, uint32_t cursor, uint32_t n_sweeps) {
  constexpr uint32_t NOCC = MODEL == kTwoLane ? 2u : 1u;
  constexpr uint32_t NQ = dis_planes(DIS);
  constexpr uint32_t NP = NOCC + NQ;
  const uint32_t R2 = a.R2, Cp = a.Cp, G = a.G, W = a.geo.W;
  const uint32_t PW = (R2 + 1) * Cp;  // R2 rows + the mirror row
  const uint64_t L = a.geo.L;
  uint32_t* bufA = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* bufB = bufA + NP * PW;
  uint32_t* tab = bufB + NP * PW;
  long long* warp_tot = reinterpret_cast<long long*>(tab + ((a.ptab_n + 1u) & ~1u));
  long long* arr = warp_tot + 32;

  Lane ln;
  ln.c = threadIdx.x;
  const bool col_ok = ln.c < a.C;
  const uint32_t s_loc = col_ok ? ln.c / G : 0u;
  ln.g = col_ok ? ln.c - s_loc * G : 0u;
  ln.col0 = s_loc * G;
  ln.c_next = ln.col0 + (ln.g + 1 == G ? 0u : ln.g + 1);
  ln.c_prev = ln.col0 + (ln.g == 0 ? G - 1 : ln.g - 1);
  ln.sample = group * a.spc + s_loc;
  ln.active = col_ok && ln.sample < a.geo.S;
  ln.n_glob = a.geo.first_sample + ln.sample;
  const uint2 key = key_of(a.seed);

  // load the Poisson table and the lattices (frame offset 0)
  for (uint32_t i = threadIdx.x; i < a.ptab_n; i += blockDim.x) tab[i] = a.ptab[i];
  const uint32_t first = group * a.spc;
  const uint32_t nloc = min(a.spc, a.geo.S - first);
  for (uint32_t p = 0; p < NP; ++p) {
    for (uint32_t idx = threadIdx.x; idx < nloc * W; idx += blockDim.x) {
      const uint32_t sl = idx / W, w = idx - sl * W;
      const uint32_t smp = first + sl;
      const uint32_t v = p < NOCC ? __ldcg(&a.state[(static_cast<size_t>(smp) * a.geo.planes + p) * W + w])
                                  : a.mask[(static_cast<size_t>(smp / a.geo.samples_per_real) * NQ + (p - NOCC)) * W + w];
      bufA[p * PW + (w & (R2 - 1)) * Cp + sl * G + (w >> a.logR2)] = v;
    }
  }
  __syncthreads();

  uint32_t* cur = bufA;
  uint32_t* nxt = bufB;
  uint32_t R_cur = 0;
  Cnt cnt;
  uint32_t rec = cursor;

  for (uint32_t it = 0; it < n_sweeps; ++it) {
    const uint64_t s = s0 + it;
    uint32_t o = 0;
    if (ln.active) o = philox10(ctr_of(s, kTagOff, 0, ln.n_glob, 0), key).x & (2 * a.D - 1);
    if (ln.active) realign<NP>(cur, nxt, a, ln, PW, static_cast<uint32_t>((o + L - R_cur) % L));
    uint32_t* t = cur;
    cur = nxt;
    nxt = t;
    R_cur = o;
    __syncthreads();
    run_phase<MODEL, DIS, COUNT, CP, 0>(cur, nxt, a.lane_sort != 0, a, tab, PW, s, ln, key, cnt);
    __syncthreads();
    if (ln.active) mirror_in<NP>(cur, a, PW, ln);
    run_phase<MODEL, DIS, COUNT, CP, 1>(cur, nxt, a.lane_sort != 0, a, tab, PW, s, ln, key, cnt);
    __syncthreads();
    if (ln.active) mirror_out<NOCC>(cur, a, PW, ln);
    __syncthreads();
    if (MODEL == kTwoLane && (DIS == kDisTurning || DIS == kDisCrossing)) {
      if (ln.active) turning<DIS>(cur, a, PW, s, R_cur, ln, key, cnt);
      __syncthreads();
    }
    if (rec < a.n_times && a.times[rec] == s + 1) {
      if (ln.active) realign<NP>(cur, nxt, a, ln, PW, static_cast<uint32_t>((L - R_cur) % L));
      t = cur;
      cur = nxt;
      nxt = t;
      R_cur = 0;
      __syncthreads();
      record_heights<NOCC>(cur, a, PW, rec, ln, warp_tot, arr);
      record_extras<NOCC>(cur, a, PW, rec, s + 1, ln, warp_tot, arr, cnt);
      ++rec;
    }
  }

  // back to frame offset 0 and out to global memory
  if (ln.active) realign<NP>(cur, nxt, a, ln, PW, static_cast<uint32_t>((L - R_cur) % L));
  cur = nxt;
  __syncthreads();
  for (uint32_t p = 0; p < NOCC; ++p) {
    for (uint32_t idx = threadIdx.x; idx < nloc * W; idx += blockDim.x) {
      const uint32_t sl = idx / W, w = idx - sl * W;
      a.state[(static_cast<size_t>(first + sl) * a.geo.planes + p) * W + w] =
          cur[p * PW + (w & (R2 - 1)) * Cp + sl * G + (w >> a.logR2)];
    }
  }
  if (ln.active) {
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(a.counters + 4ull * ln.sample);
    if (cnt.a) atomicAdd(dst + 0, static_cast<unsigned long long>(cnt.a));
    if (cnt.b) atomicAdd(dst + 1, static_cast<unsigned long long>(cnt.b));
    if (cnt.c) atomicAdd(dst + 2, static_cast<unsigned long long>(cnt.c));
    if (cnt.d) atomicAdd(dst + 3, static_cast<unsigned long long>(cnt.d));
  }
  __syncthreads();  // the shared memory is reused by the next group of a persistent CTA
}

}  // namespace
}  // namespace asep

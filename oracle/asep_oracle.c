/*
 * asep_oracle.c -- CPU oracle for the bit-packed ASEP / 1+1-d KPZ Monte Carlo.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load it.
 * It shares no code, header or table with the CUDA library: it restates the
 * method from the paper (Schulz, Odor, Odor, Nagy, "Simulation of 1+1
 * dimensional surface growth and lattice gases using GPUs") and from the
 * schedule definition written down for this project, one site at a time.
 *
 * What it computes
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the published
 *     round function and key schedule.
 *   - The roof-top RSOS <-> ASEP mapping (paper sec. 2, Fig. "kpzasep"): an
 *     up slope is a particle (bit 1), a down slope a hole (bit 0); deposition
 *     is a right hop 10 -> 01 with probability p_i, evaporation a left hop
 *     01 -> 10 with probability q_{i+1} (paper sec. 2.1, rates per bond).
 *   - The quenched bimodal site disorder of Eq. (bimodal): a per-site class
 *     bit selects the slow rates (paper sec. 2.3).
 *   - The two-lane opposite-direction model of paper sec. 3: lane A hops
 *     right, lane B hops left, lane changes only at quenched turning sites.
 *   - Height reconstruction h_i = sum_{j<=i} (2 n_j - 1) and the sums that
 *     give W^2 of Eq. (W) (paper sec. 2.1), exactly in 128-bit integers.
 *   - Three update schedules, replayed literally:
 *       SERIAL: plain random-sequential update (RSU, paper sec. 2.1), L (or
 *               2L for two lanes) uniform bond attempts per sweep.
 *       DOMAIN: the two-phase Poisson-domain schedule (no paper counterpart;
 *               the paper's GPU schedule is a two-sub-lattice SCA).  Per
 *               sweep a random offset o in [0, 2D) splits the ring into
 *               super-domains of 2D sites; the even halves (D sites, D bonds
 *               each, the last bond reaching the first site of the odd half)
 *               run first, the odd halves second.  Each domain performs a
 *               Poisson(bonds) number of attempts, each on a uniformly drawn
 *               bond of the domain.
 *       SCA:    the paper's own GPU schedule, the two-sub-lattice cellular
 *               automaton of sec. 2.1 (even bonds, then odd bonds; see
 *               sca_sweep).
 *   - An independent serial RSU reference with its own generator
 *     (xoshiro256**, Blackman & Vigna 2018, seeded by splitmix64), used for
 *     statistical comparisons only.
 *
 * Random-word layout (shared by definition with the GPU path, not by code):
 *   key   = (seed & 0xffffffff, seed >> 32)
 *   ctr0  = sweep & 0xffffffff
 *   ctr1  = ((sweep >> 32) & 0xff) | tag << 8 | call << 12
 *   ctr2  = sample (or disorder realization)
 *   ctr3  = domain / site-group / call index (see each tag below)
 *   word q of a stream is output lane (q & 3) of call (q >> 2).
 *
 * Acceptance of a draw r against a threshold t: (r & 0xfffff000) < t.  A
 * threshold is 0 (never), 0xffffffff (always) or a multiple of 4096, so the
 * probability is exactly t / 2^32 and the low 12 bits of r stay free for the
 * bond slot and the lane bit.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TAG_INIT 1u /* Bernoulli(1/2) initial filling */
#define TAG_DIS 2u  /* quenched disorder: class bit or turning-site bit */
#define TAG_OFF 3u  /* per-sweep domain offset */
#define TAG_DOM 4u  /* per-domain attempt stream */
#define TAG_TURN 5u /* per-site lane-change draw */
#define TAG_SER 6u  /* serial-schedule attempt stream */
#define TAG_SCA 7u  /* two-sub-lattice SCA: random bit-planes of a 32-bond group */
#define TAG_SCA_TURN 8u /* two-lane SCA: one word per lane-change candidate site */

#define MODEL_RING 0u
#define MODEL_TWO_LANE 1u
#define SCHED_DOMAIN 0u
#define SCHED_SERIAL 1u
#define SCHED_SCA 2u
#define DIS_NONE 0u
#define DIS_BIMODAL 1u
#define DIS_TURNING 2u
#define DIS_BIMODAL_PQ 3u /* independent slow classes for right (p) and left (q) hops */
#define DIS_CROSSING 4u   /* two lanes: crossing at every site, u_i (A->B) and v_i (B->A) bimodal */
#define INIT_FLAT_ALT 0u
#define INIT_BERNOULLI_HALF 1u

#define ACCEPT_MASK 0xfffff000u

typedef struct {
  uint32_t model;
  uint32_t schedule;
  uint64_t L;
  uint32_t D;
  uint32_t n_realizations;
  uint32_t samples_per_real;
  uint32_t first_sample;
  uint32_t p_thr;
  uint32_t q_thr;
  uint32_t dis_kind;
  uint32_t dis_a_thr;
  uint32_t dis_b_thr;
  uint32_t dis_c_thr;
  uint32_t init_kind;
  uint64_t seed;
  uint64_t dis_seed;
  uint64_t init_seed;
} orc_params;

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                      */
/* ------------------------------------------------------------------ */

void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* key increments (Weyl) */
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; round++) {
    uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* One stream of random words: word q = lane (q & 3) of Philox call (q >> 2).
 * The current call's output is cached so consecutive words cost one call. */
typedef struct {
  uint32_t key[2];
  uint64_t sweep;
  uint32_t tag;
  uint32_t sample;
  uint32_t d;
  int call_in_ctr3; /* serial stream: call index lives in ctr3, d unused */
  int64_t cached_call;
  uint32_t cached[4];
} stream_t;

static void stream_open(stream_t* st, uint64_t seed, uint64_t sweep, uint32_t tag, uint32_t sample,
                        uint32_t d, int call_in_ctr3) {
  st->key[0] = (uint32_t)(seed & 0xffffffffu);
  st->key[1] = (uint32_t)(seed >> 32);
  st->sweep = sweep;
  st->tag = tag;
  st->sample = sample;
  st->d = d;
  st->call_in_ctr3 = call_in_ctr3;
  st->cached_call = -1;
}

static uint32_t stream_word(stream_t* st, uint64_t q) {
  int64_t call = (int64_t)(q >> 2);
  if (call != st->cached_call) {
    uint32_t ctr[4];
    ctr[0] = (uint32_t)(st->sweep & 0xffffffffu);
    ctr[1] = (uint32_t)((st->sweep >> 32) & 0xffu) | (st->tag << 8);
    ctr[2] = st->sample;
    if (st->call_in_ctr3) {
      ctr[3] = (uint32_t)call;
    } else {
      ctr[1] |= (uint32_t)call << 12;
      ctr[3] = st->d;
    }
    orc_philox(ctr, st->key, st->cached);
    st->cached_call = call;
  }
  return st->cached[q & 3];
}

/* ------------------------------------------------------------------ */
/* Sites                                                              */
/* ------------------------------------------------------------------ */

static int get_site(const uint32_t* w, uint64_t i) { return (int)((w[i >> 5] >> (i & 31)) & 1u); }
static void flip_site(uint32_t* w, uint64_t i) { w[i >> 5] ^= 1u << (i & 31); }

static int accept(uint32_t r, uint32_t t) { return (r & ACCEPT_MASK) < t; }

/* rate for a right hop leaving site i (p_i) and a left hop leaving site i
 * (q_i).  BIMODAL: one slow class per site for both.  BIMODAL_PQ (the paper's
 * separate tag bits for reduced forward and backward rates, Eq. bimodal with
 * the same distribution for q_i): the q classes are the second plane. */
static uint32_t rate_p(const orc_params* P, const uint32_t* cls, uint64_t i) {
  if ((P->dis_kind == DIS_BIMODAL || P->dis_kind == DIS_BIMODAL_PQ) && get_site(cls, i)) return P->dis_b_thr;
  return P->p_thr;
}
static uint32_t rate_q(const orc_params* P, const uint32_t* cls, uint64_t i) {
  if (P->dis_kind == DIS_BIMODAL && get_site(cls, i)) return P->dis_c_thr;
  if (P->dis_kind == DIS_BIMODAL_PQ && get_site(cls + (P->L + 31) / 32, i)) return P->dis_c_thr;
  return P->q_thr;
}

/* Two lanes: may a particle change lanes at site i, and with which
 * probability, A -> B (dir 0) or B -> A (dir 1)?  TURNING: only at turning
 * sites, with omega (dis_b_thr) both ways.  CROSSING (sec. 3: crossing
 * probabilities u_i, v_i, quenched with the distribution of Eq. bimodal, the
 * reduced value at sites marked by separate bits for u and v): every site;
 * u_i from plane 0, v_i from plane 1 of the realization, dis_b_thr unmarked,
 * dis_c_thr marked. */
static int crosses(const orc_params* P, const uint32_t* turn, uint64_t i) {
  return P->dis_kind == DIS_CROSSING ? 1 : get_site(turn, i);
}
static uint32_t cross_thr(const orc_params* P, const uint32_t* turn, uint64_t i, uint32_t dir) {
  if (P->dis_kind == DIS_CROSSING && get_site(turn + dir * ((P->L + 31) / 32), i)) return P->dis_c_thr;
  return P->dis_b_thr;
}
static int lane_changes_on(const orc_params* P) {
  return P->dis_kind == DIS_TURNING || P->dis_kind == DIS_CROSSING;
}

/* One attempt on ring bond (i, i+1): 10 -> 01 with p_i, 01 -> 10 with q_{i+1}. */
static void ring_attempt(const orc_params* P, uint32_t* w, const uint32_t* cls, uint64_t i, uint32_t r,
                         uint64_t* cnt) {
  uint64_t i1 = (i + 1) % P->L;
  int a = get_site(w, i), b = get_site(w, i1);
  if (a == 1 && b == 0) {
    if (accept(r, rate_p(P, cls, i))) {
      flip_site(w, i);
      flip_site(w, i1);
      cnt[0]++;
      if (i == P->L - 1) cnt[4]++; /* across the seam (L-1, 0) */
    }
  } else if (a == 0 && b == 1) {
    if (accept(r, rate_q(P, cls, i1))) {
      flip_site(w, i);
      flip_site(w, i1);
      cnt[1]++;
      if (i == P->L - 1) cnt[5]++;
    }
  }
}

/* One in-lane attempt of the two-lane model on bond (i, i+1) of lane `lane`:
 * lane A (0) moves particles right (10 -> 01, rate p_thr), lane B (1) moves
 * them left (01 -> 10, rate q_thr). */
static void lane_attempt(const orc_params* P, uint32_t* wa, uint32_t* wb, int lane, uint64_t i, uint32_t r,
                         uint64_t* cnt) {
  uint64_t i1 = (i + 1) % P->L;
  if (lane == 0) {
    if (get_site(wa, i) == 1 && get_site(wa, i1) == 0 && accept(r, P->p_thr)) {
      flip_site(wa, i);
      flip_site(wa, i1);
      cnt[0]++;
    }
  } else {
    if (get_site(wb, i) == 0 && get_site(wb, i1) == 1 && accept(r, P->q_thr)) {
      flip_site(wb, i);
      flip_site(wb, i1);
      cnt[1]++;
    }
  }
}

/* Lane changes after the in-lane attempts of a sweep: at every turning site
 * with exactly one lane occupied the particle moves to the empty lane with
 * probability omega (dis_b_thr).  Each event touches only (A_i, B_i). */
static void turning_pass(const orc_params* P, uint32_t* wa, uint32_t* wb, const uint32_t* turn, uint32_t sample,
                         uint64_t sweep, uint64_t* cnt) {
  stream_t st;
  for (uint64_t i = 0; i < P->L; i++) {
    if (!crosses(P, turn, i)) continue;
    int a = get_site(wa, i), b = get_site(wb, i);
    if (a == b) continue;
    stream_open(&st, P->seed, sweep, TAG_TURN, sample, (uint32_t)(i >> 2), 0);
    uint32_t r = stream_word(&st, i & 3);
    if (accept(r, cross_thr(P, turn, i, a ? 0u : 1u))) {
      flip_site(wa, i);
      flip_site(wb, i);
      if (a) cnt[2]++;
      else cnt[3]++;
    }
  }
}

/* K = k_lo + #{ j : tab[j] <= w } : inversion of the Poisson CDF table. */
static uint32_t poisson_count(const uint32_t* tab, uint32_t k_lo, uint32_t n_tab, uint32_t w) {
  uint32_t K = k_lo;
  for (uint32_t j = 0; j < n_tab; j++)
    if (tab[j] <= w) K++;
  return K;
}

static int log2u(uint64_t x) {
  int k = 0;
  while ((1ull << k) < x) k++;
  return k;
}

/* ------------------------------------------------------------------ */
/* Schedules                                                          */
/* ------------------------------------------------------------------ */

static void domain_sweep(const orc_params* P, const uint32_t* ptab, uint32_t ptab_klo, uint32_t ptab_n,
                         uint32_t* words, const uint32_t* mask, uint32_t sample, uint64_t sweep, uint64_t* cnt) {
  const uint64_t L = P->L, D = P->D;
  const uint64_t G = L / (2 * D);
  const int two_lane = (P->model == MODEL_TWO_LANE);
  const uint64_t bonds = two_lane ? 2 * D : D;
  const int logD = log2u(D);
  const uint64_t W = (L + 31) / 32;
  uint32_t* wa = words;
  uint32_t* wb = two_lane ? words + W : NULL;
  stream_t st;

  stream_open(&st, P->seed, sweep, TAG_OFF, sample, 0, 0);
  const uint64_t o = stream_word(&st, 0) & (2 * D - 1);

  for (int phase = 0; phase < 2; phase++) {
    for (uint64_t g = 0; g < G; g++) {
      uint32_t d = (uint32_t)(2 * g + (uint64_t)phase);
      uint64_t base = (o + 2 * D * g + (uint64_t)phase * D) % L;
      stream_open(&st, P->seed, sweep, TAG_DOM, sample, d, 0);
      uint32_t K = poisson_count(ptab, ptab_klo, ptab_n, stream_word(&st, 0));
      for (uint32_t k = 1; k <= K; k++) {
        uint32_t r = stream_word(&st, k);
        uint64_t j = r & (bonds - 1);
        if (!two_lane) {
          ring_attempt(P, wa, mask, (base + j) % L, r, cnt);
        } else {
          int lane = (int)(j >> logD);
          uint64_t slot = j & (D - 1);
          lane_attempt(P, wa, wb, lane, (base + slot) % L, r, cnt);
        }
      }
    }
  }
  if (two_lane && lane_changes_on(P)) turning_pass(P, wa, wb, mask, sample, sweep, cnt);
}

/* The paper's GPU schedule (sec. 2.1, Fig. "parasep"): a two-sub-lattice
 * stochastic cellular automaton.  One sweep updates every even bond
 * (i, i+1), i = 0, 2, ..., L-2, then every odd bond i = 1, 3, ..., L-1; the
 * last odd bond (L-1, 0) is the paper's separate ring-closing step, and as it
 * shares no site with the other odd bonds, updating it among them gives the
 * same result.  The bonds of a phase are disjoint, so the order inside a
 * phase does not matter; here it is ascending.  Each bond makes one attempt
 * with a 20-bit uniform u (accept iff u < t / 4096, i.e. with probability
 * t / 2^32; t = always accepts every u):
 *   bond i = 2m + phase, group g = m / 32, lane = 2 (m mod 16) + (m / 16 mod 2);
 *   bit k of u (k = 0 the most significant) = bit `lane` of plane k of g;
 *   plane k of g = word 4k + (g mod 4) of the stream (tag SCA,
 *   ctr3 = 2 (g / 4) + phase + lane_of_model * 2^31), k = 0 .. 19: Philox
 *   call k of that stream gives plane k of four consecutive groups.
 * Two lanes (paper sec. 3, its five-step SCA sequence): the in-lane bonds of
 * lane A (right hops, p_thr) and of lane B (left hops, q_thr) run in each
 * phase, lane B's planes from the stream with bit 31 of ctr3 set; with
 * turning sites, the even phase is followed by the A -> B lane changes and
 * the odd phase by the B -> A ones (sca_lane_changes). */
static void sca_lane_changes(const orc_params* P, uint32_t* wa, uint32_t* wb, const uint32_t* turn, uint32_t sample,
                             uint64_t sweep, uint32_t step, uint64_t* cnt);

static void sca_sweep(const orc_params* P, uint32_t* words, const uint32_t* mask, uint32_t sample, uint64_t sweep,
                      uint64_t* cnt) {
  const uint64_t L = P->L, bonds = L / 2, W = (L + 31) / 32;
  const int two_lane = (P->model == MODEL_TWO_LANE);
  uint32_t* wa = words;
  uint32_t* wb = two_lane ? words + W : NULL;
  for (uint32_t phase = 0; phase < 2; phase++) {
    for (uint32_t lane = 0; lane < (two_lane ? 2u : 1u); lane++) {
      for (uint64_t g = 0; 32 * g < bonds; g++) {
        stream_t st;
        uint32_t plane[20];
        stream_open(&st, P->seed, sweep, TAG_SCA, sample, (uint32_t)(2 * (g / 4) + phase) | (lane << 31), 0);
        for (int k = 0; k < 20; k++) plane[k] = stream_word(&st, 4 * (uint64_t)k + (g % 4));
        for (uint64_t m = 32 * g; m < 32 * g + 32 && m < bonds; m++) {
          const uint32_t bit = (uint32_t)(2 * (m & 15) + ((m >> 4) & 1));
          uint32_t u = 0;
          for (int k = 0; k < 20; k++) u = (u << 1) | ((plane[k] >> bit) & 1u);
          if (two_lane)
            lane_attempt(P, wa, wb, (int)lane, 2 * m + phase, u << 12, cnt);
          else
            ring_attempt(P, wa, mask, 2 * m + phase, u << 12, cnt);
        }
      }
    }
    if (two_lane && lane_changes_on(P)) sca_lane_changes(P, wa, wb, mask, sample, sweep, phase, cnt);
  }
}

/* Lane changes of the two-lane SCA: step 0 moves A -> B, step 1 B -> A.  At
 * a turning site i whose source lane is occupied and target lane empty, the
 * particle moves with probability omega (dis_b_thr); the draw is word
 * 4 step + (i mod 4) of the stream (tag SCA_TURN, ctr3 = i / 4).  Each event
 * touches only (A_i, B_i), so the order over sites does not matter. */
static void sca_lane_changes(const orc_params* P, uint32_t* wa, uint32_t* wb, const uint32_t* turn, uint32_t sample,
                             uint64_t sweep, uint32_t step, uint64_t* cnt) {
  uint32_t* src = step == 0 ? wa : wb;
  uint32_t* dst = step == 0 ? wb : wa;
  stream_t st;
  for (uint64_t i = 0; i < P->L; i++) {
    if (!crosses(P, turn, i) || !get_site(src, i) || get_site(dst, i)) continue;
    stream_open(&st, P->seed, sweep, TAG_SCA_TURN, sample, (uint32_t)(i >> 2), 0);
    if (accept(stream_word(&st, 4 * (uint64_t)step + (i & 3)), cross_thr(P, turn, i, step))) {
      flip_site(src, i);
      flip_site(dst, i);
      cnt[step == 0 ? 2 : 3]++;
    }
  }
}

static void serial_sweep(const orc_params* P, uint32_t* words, const uint32_t* mask, uint32_t sample, uint64_t sweep,
                         uint64_t* cnt) {
  const uint64_t L = P->L;
  const int two_lane = (P->model == MODEL_TWO_LANE);
  const uint64_t n_att = two_lane ? 2 * L : L;
  const int logL = log2u(L);
  const uint64_t W = (L + 31) / 32;
  uint32_t* wa = words;
  uint32_t* wb = two_lane ? words + W : NULL;
  stream_t st;
  stream_open(&st, P->seed, sweep, TAG_SER, sample, 0, 1);
  for (uint64_t k = 0; k < n_att; k++) {
    uint32_t rb = stream_word(&st, 2 * k);
    uint32_t ru = stream_word(&st, 2 * k + 1);
    uint64_t j = rb & (n_att - 1);
    if (!two_lane) {
      ring_attempt(P, wa, mask, j, ru, cnt);
    } else {
      lane_attempt(P, wa, wb, (int)(j >> logL), j & (L - 1), ru, cnt);
    }
  }
  if (two_lane && lane_changes_on(P)) turning_pass(P, wa, wb, mask, sample, sweep, cnt);
}

/* The oracle accepts tiny rings (exact-enumeration tests use L <= 12);
 * words per plane are ceil(L / 32). */
static int params_ok(const orc_params* P) {
  if (P->L < 2 || P->L > (1ull << 30)) return 0;
  if (P->model > MODEL_TWO_LANE || P->schedule > SCHED_SCA) return 0;
  if (P->schedule == SCHED_DOMAIN) {
    if (P->D < 1 || P->D > 2048 || (P->D & (P->D - 1))) return 0;
    if (P->L % (2ull * P->D)) return 0;
  } else if (P->schedule == SCHED_SCA) {
    if (P->L & 1) return 0; /* rings of even length */
  } else {
    if (P->L & (P->L - 1)) return 0;
  }
  return 1;
}

/* Advance one sample (global id `sample`) from sweep s0 by n_sweeps sweeps.
 * words: [planes][ceil(L/32)], planes = 1 (ring) or 2 (two lanes).
 * mask:  this sample's realization of the class plane (BIMODAL) or of the
 *        turning-site plane (TURNING), or NULL.
 * cnt:   6 entries.  ring: [right hops, left hops, 0, 0, right hops across the
 *        seam bond (L-1, 0), left hops across it]; two lanes: [A hops, B hops,
 *        A->B, B->A, 0, 0]. */
int orc_sweeps(const orc_params* P, const uint32_t* ptab, uint32_t ptab_klo, uint32_t ptab_n, uint32_t* words,
               const uint32_t* mask, uint32_t sample, uint64_t s0, uint64_t n_sweeps, uint64_t* cnt) {
  if (!params_ok(P)) return -1;
  for (uint64_t s = s0; s < s0 + n_sweeps; s++) {
    if (P->schedule == SCHED_DOMAIN)
      domain_sweep(P, ptab, ptab_klo, ptab_n, words, mask, sample, s, cnt);
    else if (P->schedule == SCHED_SCA)
      sca_sweep(P, words, mask, sample, s, cnt);
    else
      serial_sweep(P, words, mask, sample, s, cnt);
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Initial state and quenched disorder                                */
/* ------------------------------------------------------------------ */

/* words: [planes][ceil(L/32)] for one sample with global id `sample`. */
int orc_init(const orc_params* P, uint32_t* words, uint32_t sample) {
  const uint64_t W = (P->L + 31) / 32;
  const uint64_t planes = (P->model == MODEL_TWO_LANE) ? 2 : 1;
  stream_t st;
  if (P->L < 2) return -1;
  if (P->init_kind == INIT_FLAT_ALT) {
    /* alternating 1010... : site i occupied iff i is even (paper sec. 2.1) */
    for (uint64_t pl = 0; pl < planes; pl++)
      for (uint64_t i = 0; i < P->L; i++) {
        uint32_t* w = words + pl * W;
        if ((i & 1) == 0) w[i >> 5] |= 1u << (i & 31);
        else w[i >> 5] &= ~(1u << (i & 31));
      }
    return 0;
  }
  if (P->init_kind == INIT_BERNOULLI_HALF) {
    /* each lane site occupied with probability 1/2 (paper sec. 3): word q of
     * the plane-major sequence is one random word, its 32 bits the sites */
    for (uint64_t q = 0; q < planes * W; q++) {
      stream_open(&st, P->init_seed, 0, TAG_INIT, sample, (uint32_t)(q >> 2), 0);
      words[q] = stream_word(&st, q & 3);
    }
    return 0;
  }
  return -1;
}

/* mask: [planes][ceil(L/32)] for realization `real`.  BIMODAL: bit i = site
 * i is slow (probability Q = dis_a_thr, Eq. bimodal).  BIMODAL_PQ: plane 0
 * the slow sites of right hops, plane 1 (drawn independently, call 1 of the
 * same stream) those of left hops.  TURNING: bit i = site i is a turning
 * site (probability density = dis_a_thr).  CROSSING: plane 0 the sites
 * whose A -> B crossing probability is reduced, plane 1 (call 1) those of
 * B -> A, each with probability dis_a_thr. */
int orc_disorder(const orc_params* P, uint32_t* mask, uint32_t real) {
  stream_t st;
  const uint64_t W = (P->L + 31) / 32;
  const uint32_t planes = (P->dis_kind == DIS_BIMODAL_PQ || P->dis_kind == DIS_CROSSING) ? 2u : 1u;
  memset(mask, 0, (size_t)(W * planes) * sizeof(uint32_t));
  if (P->dis_kind == DIS_NONE) return 0;
  for (uint32_t pl = 0; pl < planes; pl++)
    for (uint64_t i = 0; i < P->L; i++) {
      stream_open(&st, P->dis_seed, 0, TAG_DIS, real, (uint32_t)(i >> 2), 0);
      if (accept(stream_word(&st, 4u * pl + (i & 3)), P->dis_a_thr)) mask[pl * W + (i >> 5)] |= 1u << (i & 31);
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Heights and width (Eq. W)                                          */
/* ------------------------------------------------------------------ */

/* h_i = sum_{j<=i} (2 n_j - 1); returns sum_i h_i and sum_i h_i^2 (128-bit). */
void orc_heights(const uint32_t* w, uint64_t L, int64_t* sum_h, uint64_t* sum_h2_lo, uint64_t* sum_h2_hi) {
  int64_t h = 0, s1 = 0;
  unsigned __int128 s2 = 0;
  for (uint64_t i = 0; i < L; i++) {
    h += 2 * get_site(w, i) - 1;
    s1 += h;
    s2 += (unsigned __int128)((__int128)h * (__int128)h);
  }
  *sum_h = s1;
  *sum_h2_lo = (uint64_t)s2;
  *sum_h2_hi = (uint64_t)(s2 >> 64);
}

/* ------------------------------------------------------------------ */
/* Independent serial RSU reference (own generator, statistics only)  */
/* ------------------------------------------------------------------ */

typedef struct {
  uint64_t s[4];
} xoshiro_t;

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xoshiro_next(xoshiro_t* x) {
  uint64_t* s = x->s;
  uint64_t result = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return result;
}

static void xoshiro_seed(xoshiro_t* x, uint64_t seed) {
  uint64_t z = seed;
  for (int i = 0; i < 4; i++) { /* splitmix64 */
    z += 0x9E3779B97F4A7C15ull;
    uint64_t y = z;
    y = (y ^ (y >> 30)) * 0xBF58476D1CE4E5B9ull;
    y = (y ^ (y >> 27)) * 0x94D049BB133111EBull;
    x->s[i] = y ^ (y >> 31);
  }
}

/* uniform integer in [0, n), Lemire's multiply-shift with rejection (2019) */
static uint64_t uniform_below(xoshiro_t* x, uint64_t n) {
  uint32_t nn = (uint32_t)n;
  uint64_t m = (uint64_t)(uint32_t)(xoshiro_next(x) >> 32) * nn;
  uint32_t l = (uint32_t)m;
  if (l < nn) {
    uint32_t thresh = (uint32_t)(-nn) % nn;
    while (l < thresh) {
      m = (uint64_t)(uint32_t)(xoshiro_next(x) >> 32) * nn;
      l = (uint32_t)m;
    }
  }
  return m >> 32;
}

/* Plain RSU: per sweep L (ring) or 2L (two lanes) attempts, each on a bond
 * drawn uniformly among all bonds, then (two lanes) the turning pass with
 * the same generator.  Any L that is a multiple of 32. */
int orc_serial_reference(const orc_params* P, uint32_t* words, const uint32_t* mask, uint64_t rng_seed,
                         uint64_t n_sweeps, uint64_t* cnt) {
  const uint64_t L = P->L, W = (L + 31) / 32;
  const int two_lane = (P->model == MODEL_TWO_LANE);
  uint32_t* wa = words;
  uint32_t* wb = two_lane ? words + W : NULL;
  xoshiro_t x;
  if (L < 2 || L > 0xffffffffull / 2) return -1;
  xoshiro_seed(&x, rng_seed);
  for (uint64_t s = 0; s < n_sweeps; s++) {
    if (!two_lane) {
      for (uint64_t k = 0; k < L; k++) {
        uint64_t i = uniform_below(&x, L);
        uint32_t r = (uint32_t)(xoshiro_next(&x) >> 32);
        ring_attempt(P, wa, mask, i, r, cnt);
      }
    } else {
      for (uint64_t k = 0; k < 2 * L; k++) {
        uint64_t j = uniform_below(&x, 2 * L);
        uint32_t r = (uint32_t)(xoshiro_next(&x) >> 32);
        lane_attempt(P, wa, wb, (int)(j / L), j % L, r, cnt);
      }
      if (lane_changes_on(P)) {
        for (uint64_t i = 0; i < L; i++) {
          if (!crosses(P, mask, i)) continue;
          int a = get_site(wa, i), b = get_site(wb, i);
          if (a == b) continue;
          uint32_t r = (uint32_t)(xoshiro_next(&x) >> 32);
          if (accept(r, cross_thr(P, mask, i, a ? 0u : 1u))) {
            flip_site(wa, i);
            flip_site(wb, i);
            if (a) cnt[2]++;
            else cnt[3]++;
          }
        }
      }
    }
  }
  return 0;
}

/*
 * asep.h -- C ABI of libasep.so, a GB300 (sm_103a) Monte Carlo engine for the
 * 1+1-d restricted-solid-on-solid (KPZ) surface mapped onto a bit-packed ASEP
 * lattice gas (Schulz, Odor, Odor, Nagy, "Simulation of 1+1 dimensional
 * surface growth and lattice gases using GPUs", arXiv:1012.0385).
 *
 * Model (paper sec. 2, Fig. "kpzasep"): an up slope of the roof-top surface is
 * a particle (bit 1), a down slope a hole (bit 0).  Deposition is a right hop
 * 10 -> 01 across bond (i, i+1) with probability p_i, evaporation a left hop
 * 01 -> 10 with probability q_{i+1} (paper sec. 2.1).  Quenched columnar
 * disorder draws a slow class per site with probability Q (Eq. bimodal,
 * paper sec. 2.3).  The two-lane model (paper sec. 3) couples a right-moving
 * ring A and a left-moving ring B through quenched turning sites.
 *
 * Storage: 32 sites per uint32 word, bit k of word w is site 32 w + k.  A
 * context holds S = n_realizations * samples_per_real independent samples,
 * each with `planes` = 1 (ring) or 2 (lanes A, B) planes of L / 32 words;
 * host copies use the layout [S][planes][L/32].
 *
 * Randomness: Philox4x32-10 keyed by a 64-bit seed, counter = (sweep, tag,
 * call, sample, domain or site group); no generator state is stored, so
 * (words, sweep index, params) is a complete checkpoint.
 *
 * Rates are u32 thresholds t: 0 = never, ASEP_ALWAYS = always, otherwise a
 * multiple of 4096 meaning probability t / 2^32 (see asep_threshold).
 *
 * Schedules:
 *   ASEP_SCHED_SERIAL  plain random-sequential update (RSU, paper sec. 2.1):
 *                      per sweep L (two lanes: 2L) attempts on uniformly drawn
 *                      bonds; L a power of two.  Two plans, both giving the
 *                      sequential result: one CTA per sample, which runs a
 *                      sweep's attempts in rounds, each attempt once every
 *                      earlier attempt sharing a site with it has run (the
 *                      automatic plan when the lattice and a sweep's draws
 *                      fit 200 KB of shared memory -- a ring of up to 16384
 *                      sites, two lanes of up to 8192 -- and the samples
 *                      number at most four per SM); or one warp per sample, which
 *                      applies each batch of 32 consecutive attempts up to
 *                      the first one that shares a site with an earlier one
 *                      of the batch.
 *   ASEP_SCHED_DOMAIN  two-phase Poisson-domain RSU (no paper counterpart; the
 *                      paper's GPU schedule is a two-sub-lattice cellular
 *                      automaton).  Per sweep a random offset splits the ring
 *                      into super-domains of 2D sites; the first halves run,
 *                      then the second halves; each half-domain performs a
 *                      Poisson(D) (two lanes: Poisson(2D)) number of attempts
 *                      on uniformly drawn bonds of its own D (2D) bonds.
 *   ASEP_SCHED_SCA     the paper's own GPU schedule (sec. 2.1): a two-sub-
 *                      lattice stochastic cellular automaton; per sweep one
 *                      attempt on every even bond (i, i+1), i even, then on
 *                      every odd bond (the ring-closing bond (L-1, 0) with
 *                      them).  Each attempt compares a 20-bit uniform u with
 *                      the threshold: bit k of u is bit `lane` of random
 *                      plane k of its 32-bond group (plane k of four groups
 *                      = Philox call k of tag 7, ctr3 = 2 * unit + phase;
 *                      group g = bonds 32g..32g+31 of the phase, lane of bond
 *                      m = 2 (m mod 16) + (m / 16 mod 2)).  Two lanes (sec.
 *                      3, its five-step sequence): the bonds of lane A (right
 *                      hops, p) and of lane B (left hops, q; planes from
 *                      ctr3 with bit 31 set) in each phase, with turning
 *                      sites the A -> B lane changes after the even phase
 *                      and B -> A after the odd one (probability omega, one
 *                      draw per candidate site: tag 8, call = step, ctr3 =
 *                      site / 4).  L a multiple of 256.  The lattice sits
 *                      in one CTA's shared memory while it fits (ring L up
 *                      to about 1.4 * 2^20, bimodal or two lanes 2^19,
 *                      two lanes with turning sites 2^18); beyond that
 *                      (or on request, asep_set_plan) it stays in global
 *                      memory and each phase is one launch over all units
 *                      of 8 words (results identical).
 *
 * Error behaviour: every function returns ASEP_OK (0) or a negative
 * ASEP_ERR_* code and never aborts; the context keeps a message readable with
 * asep_last_error().  A context that saw ASEP_ERR_CUDA may be unusable.
 *
 * Threading: a context is used by one host thread at a time.  Device work is
 * enqueued on the context's stream; functions that return host data
 * synchronise that stream only.
 */
#ifndef ASEP_H
#define ASEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Only the functions declared here are exported by libasep.so. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

#define ASEP_OK 0
#define ASEP_ERR_INVALID (-1) /* bad argument or unsupported combination */
#define ASEP_ERR_NOMEM (-2)   /* device or host allocation failed */
#define ASEP_ERR_CUDA (-3)    /* a CUDA runtime call failed */
#define ASEP_ERR_TIMEOUT (-4) /* a streamed tile's bounded wait for its bulk copy gave up (results invalid) */
#define ASEP_ERR_STATE (-5)   /* call not valid in the context's state */

#define ASEP_MODEL_RING 0u     /* one ring, right rate p_i, left rate q_{i+1} */
#define ASEP_MODEL_TWO_LANE 1u /* lane A right (p_thr), lane B left (q_thr) */

#define ASEP_SCHED_DOMAIN 0u
#define ASEP_SCHED_SERIAL 1u
#define ASEP_SCHED_SCA 2u

#define ASEP_DIS_NONE 0u
#define ASEP_DIS_BIMODAL 1u /* dis_a = Q, dis_b = p_slow, dis_c = q_slow     */
#define ASEP_DIS_TURNING 2u /* two lanes: dis_a = site density, dis_b = omega */
/* Ring model: independent slow classes for right and left
 * hops (sec. 3, Eq. bimodal; the paper tags reduced forward and backward
 * rates with separate bits, the same distribution for q_i as for p_i):
 * dis_a = Q for both, dis_b = p_slow, dis_c = q_slow.  Plane 0 of a
 * realization holds the p classes (the ASEP_DIS_BIMODAL draw), plane 1 the q
 * classes (call 1 of the disorder stream).  Every schedule. */
#define ASEP_DIS_BIMODAL_PQ 3u
/* Two lanes: the paper's crossing probabilities
 * (sec. 3): a particle may change lanes at every site, A -> B with u_i and
 * B -> A with v_i, quenched with the distribution of Eq. bimodal: dis_a =
 * fraction of marked sites (for u and v independently), dis_b = the crossing
 * probability of unmarked sites (0.8 in the paper), dis_c = of marked ones
 * (0.2).  Plane 0 marks u, plane 1 (call 1 of the disorder stream) marks v.
 * Same draws per candidate site as ASEP_DIS_TURNING.  Every schedule (the
 * domain schedule's lane-change pass uses u_i for a particle in lane A, v_i
 * for one in lane B). */
#define ASEP_DIS_CROSSING 4u

#define ASEP_INIT_FLAT_ALT 0u       /* 1010...: site i occupied iff i even (paper sec. 2.1) */
#define ASEP_INIT_BERNOULLI_HALF 1u /* every lane site occupied with probability 1/2 (sec. 3) */

#define ASEP_ALWAYS 0xFFFFFFFFu

/* asep_params.flags */
#define ASEP_FLAG_NO_HOP_COUNTS 1u /* ring model: do not count hops (asep_counters then reports zeros) */
#define ASEP_FLAG_PROFILE 2u       /* accumulate the occupancy profile at every sample time (asep_profile) */
#define ASEP_FLAG_AUTOCORR 4u      /* record the overlap with the lattice at autocorr_t0 (asep_autocorr) */

typedef struct asep_ctx asep_ctx; /* opaque; owns every device buffer it allocates */

/* Device allocator hook: when alloc is non-NULL the context obtains all of
 * its device memory through it (e.g. a framework's caching allocator) and
 * returns it through free_fn; otherwise it uses cudaMalloc / cudaFree.  A
 * block must start on a 256-byte boundary (as cudaMalloc's do): the kernels
 * move the lattice with 16- and 32-byte accesses and bulk copies.  A
 * misaligned block is handed back through free_fn and asep_create fails
 * with ASEP_ERR_NOMEM. */
typedef void* (*asep_alloc_fn)(size_t bytes, void* user);
typedef void (*asep_free_fn)(void* ptr, size_t bytes, void* user);

typedef struct asep_params {
  uint32_t model;            /* ASEP_MODEL_* */
  uint32_t schedule;         /* ASEP_SCHED_* */
  uint64_t L;                /* sites per lane, multiple of 64 in [64, 2^28]; DOMAIN: multiple of
                                2*domain_sites (beyond a 16-CTA cluster, also of 128); SERIAL: power
                                of two; SCA: multiple of 256 */
  uint32_t domain_sites;     /* D: power of two in [32, 2048]; 0 = 256 or the largest that divides L/2 */
  uint32_t n_realizations;   /* quenched-disorder realizations (1 without disorder) */
  uint32_t samples_per_real; /* samples per realization */
  uint32_t first_sample;     /* global id of sample 0 (disjoint ranges make replicas mergeable) */
  uint32_t p_thr;            /* ring: right-hop rate of fast sites; two lanes: lane A rate */
  uint32_t q_thr;            /* ring: left-hop rate of fast sites; two lanes: lane B rate */
  uint32_t dis_kind;         /* ASEP_DIS_* */
  uint32_t dis_a_thr;
  uint32_t dis_b_thr;
  uint32_t dis_c_thr;
  uint32_t init_kind;        /* ASEP_INIT_* */
  uint64_t seed;             /* dynamics key */
  uint64_t dis_seed;         /* quenched-disorder key (realization r uses sample field r) */
  uint64_t init_seed;        /* initial-filling key */
  const uint64_t* sample_times; /* host array, ascending sweep counts at which heights are recorded (0 = start) */
  uint32_t n_sample_times;
  uint32_t flags;            /* ASEP_FLAG_* bits, 0 = default */
  void* stream;              /* cudaStream_t for all work of the context; NULL = default stream */
  asep_alloc_fn alloc;       /* optional allocator hook (with free_fn and alloc_user) */
  asep_free_fn free_fn;
  void* alloc_user;
  uint64_t autocorr_t0;      /* ASEP_FLAG_AUTOCORR: reference sweep count, one of sample_times */
} asep_params;

typedef struct asep_info {
  uint64_t L;
  uint32_t D;             /* effective domain size (DOMAIN schedule) */
  uint32_t planes;        /* 1 or 2 */
  uint32_t S;             /* samples */
  uint32_t n_recorded;    /* sample times recorded so far */
  uint64_t sweep;         /* sweeps done so far (the next sweep's index) */
  uint64_t attempts_per_sweep; /* L * planes per sample */
  uint64_t device_bytes;  /* device memory held by the context */
  uint64_t kernel_launches; /* kernels the context has enqueued so far */
  uint32_t cluster;       /* CTAs per sample: 1 = one CTA holds whole samples, 2..16 = a thread-block
                             cluster, 32 = streamed from global memory */
  uint32_t samples_per_group; /* samples per CTA (resident) or 1 (cluster) */
  uint32_t groups;        /* CTAs (resident) or clusters per sweep launch */
  uint32_t threads;       /* threads per CTA */
  uint32_t smem_bytes;    /* dynamic shared memory per CTA of the sweep kernel */
  uint32_t tile_columns;  /* streamed domain tier: columns (threads) per tile; 0 otherwise */
} asep_info;

/* Validate `params`, allocate device memory, draw the initial state (paper
 * sec. 2.1 flat start, or sec. 3 random half filling) and the quenched
 * disorder (Eq. bimodal or turning sites), and record the heights at sweep 0
 * when 0 is a sample time.  On success *out owns the context; on failure
 * *out is NULL and nothing is leaked.  The sample_times array is copied. */
int asep_create(const asep_params* params, asep_ctx** out);

/* What asep_create would make of `params`, without allocating or launching
 * anything: validates them (same errors as asep_create) and fills `info`
 * with the sizes, the automatic launch plan (cluster, samples_per_group,
 * groups, threads, smem_bytes) and device_bytes = the device memory the
 * context would hold, exactly as asep_get_info reports it after creation;
 * n_recorded, sweep and kernel_launches are 0.  For admission control: a
 * server decides whether a job fits its device-memory and shared-memory
 * budget before creating it.  Host only; plans beyond one CTA query the
 * current device's occupancy.  No counterpart in the paper. */
int asep_plan(const asep_params* params, asep_info* info);

/* Enqueue n_mcs sweeps (Monte Carlo steps, paper sec. 2.1: one sweep = L
 * attempts per lane and sample) of all S samples on the context stream,
 * recording heights after every sweep count listed in sample_times.
 * Asynchronous: returns once the work is enqueued. */
int asep_sweep(asep_ctx* ctx, uint64_t n_mcs);

/* Copy the heights recorded so far.  Entry e = (time index, sample, plane),
 * layout [n_recorded][S][planes]: sum_h[e] = sum_i h_i with
 * h_i = sum_{j<=i} (2 n_j - 1); sum_h2[2e], sum_h2[2e+1] = low and high words
 * of the unsigned 128-bit sum_i h_i^2; w2[e] = W^2 of Eq. (W) (paper sec.
 * 2.1) = (L sum h^2 - (sum h)^2) / L^2, evaluated exactly then rounded.  Any
 * output pointer may be NULL.  n_entries must be >= n_recorded*S*planes.
 * Synchronises the context stream. */
int asep_width(asep_ctx* ctx, int64_t* sum_h, uint64_t* sum_h2, double* w2, size_t n_entries);

/* Copy the packed lattices, layout [S][planes][L/32], and the number of
 * sweeps done.  n_words must be >= S*planes*L/32.  Synchronises. */
int asep_state(asep_ctx* ctx, uint32_t* words, size_t n_words, uint64_t* sweep_out);

/* Replace the lattices and the sweep counter (resume from a checkpoint made
 * by asep_state, or set a test state).  Layout as asep_state.  The hop
 * counters keep running; the loaded lattice becomes the reference of
 * asep_height_offset.  Synchronises. */
int asep_load_state(asep_ctx* ctx, const uint32_t* words, size_t n_words, uint64_t sweep);

/* Start the ensemble again on the same buffers: re-draw the initial state
 * with init_seed, use `seed` for the dynamics from now on, set the sweep
 * counter to 0, clear the hop counters and the height table, and record
 * sweep 0 when it is a sample time.  The quenched disorder is kept.
 * Asynchronous (context stream); allocates nothing. */
int asep_reset(asep_ctx* ctx, uint64_t seed, uint64_t init_seed);

/* Cumulative hop counters per sample, layout [S][4]: ring = (right hops,
 * left hops, 0, 0); two lanes = (lane A hops, lane B hops, A->B lane
 * changes, B->A lane changes).  The net current of paper sec. 3 is
 * J = c[0] - c[1].  Synchronises. */
int asep_counters(asep_ctx* ctx, uint64_t* counters, size_t n);

/* Copy the quenched planes, layout [n_realizations][planes][L/32] (planes =
 * 2 for BIMODAL_PQ: p classes, then q classes, and for CROSSING: u marks,
 * then v marks; else 1; bit = slow site for the bimodal kinds, turning site
 * for TURNING).  Synchronises. */
int asep_disorder(asep_ctx* ctx, uint32_t* words, size_t n_words);

/* Hop counters (layout of asep_counters) at every sample time recorded so
 * far, layout [n_recorded][S][4].  Two lanes: J_A and J_B give the current
 * density c = (J_A - J_B) / L of paper sec. 3 at each time.  Synchronises. */
int asep_currents(asep_ctx* ctx, int64_t* out, size_t n);

/* ASEP_FLAG_PROFILE (an observable the paper does not define): for every
 * sample, plane and word w, the number of occupied sites of word w (sites
 * 32w..32w+31) summed over the sample times recorded so far, layout
 * [S][planes][L/32] -- the density profile in bins of 32 sites,
 * time-averaged by dividing by 32 * n_recorded.  The flag allows at most 2^27
 * sample times, so the counts fit 32 bits.  Synchronises. */
int asep_profile(asep_ctx* ctx, uint32_t* out, size_t n);

/* ASEP_FLAG_AUTOCORR (an observable the paper does not define): overlap
 * sum_i n_i(t0) n_i(t) with the lattice at
 * t0 = autocorr_t0, for every sample time t recorded so far (0 for t < t0),
 * layout [n_recorded][S][planes]; the density autocorrelation is
 * overlap / L - rho^2.  Synchronises. */
int asep_autocorr(asep_ctx* ctx, int64_t* out, size_t n);

/* Ring model with hop counting on: the height H(t) of the surface column
 * between sites L-1 and 0 at every sample time recorded so far, relative to
 * the lattice at the last asep_create, asep_reset or asep_load_state, layout
 * [n_recorded][S]; records taken before the last load read 0.  With h_i the
 * open prefix sum of asep_width, the absolute column heights are H + h_i and
 * their mean H + sum_h / L; its slope in t is the growth velocity (paper
 * sec. 2, Eq. KPZ).  A right hop across a bond
 * lowers that bond's column by 2 and a left hop raises it, so
 * H(t) = (sum_h(ref) - sum_h(t) - 2 [(R - Lh)(t) - (R - Lh)(ref)]) / L exactly,
 * with R, Lh the cumulative right and left hop counters; the division is
 * checked.  ASEP_ERR_STATE for the two-lane model or without hop counts.
 * Synchronises. */
int asep_height_offset(asep_ctx* ctx, int64_t* out, size_t n);

/* Sizes, progress, device memory, launch count and launch plan of the
 * context (no synchronisation; n_recorded and sweep count enqueued work). */
int asep_get_info(const asep_ctx* ctx, asep_info* info);

/* Choose the launch plan of a context (the autotuner's knob; results never
 * depend on it).  Serial schedule: cluster 0 = automatic, 1 = one CTA per
 * sample running each sweep in dependency rounds (ASEP_ERR_INVALID beyond
 * 32768 attempts per sweep or 200 KB of shared memory), 2 = one warp per
 * sample; samples_per_group 0.  SCA: cluster 0 =
 * automatic, 1 = the ring in one CTA's shared memory (ASEP_ERR_INVALID when
 * it does not fit), 32 = streamed from global memory; samples_per_group 0.
 * Domain schedule: cluster 0 = automatic, 1 = whole samples in
 * one CTA, 2/4/8/16 = each sample spread over that many CTAs of a
 * thread-block cluster (columns of 2D sites split evenly), 32 = streamed: the
 * lattice stays in global memory and tiles of columns pass through shared
 * memory once per phase (the automatic choice when a sample fits neither one
 * CTA nor a 16-CTA cluster; one launch per phase, records between sweeps;
 * not in batches).  samples_per_group: samples per CTA of the one-CTA plan
 * (0 = automatic); with cluster = 32 it is instead the tile width in columns
 * (a multiple of 32 up to 1024, at most half the sample's columns; 0 =
 * automatic, 128 or the widest that fits below it).  Returns
 * ASEP_ERR_INVALID, keeping the previous plan, when the plan does not fit the
 * device.  Takes effect for the next launch. */
int asep_set_plan(asep_ctx* ctx, uint32_t cluster, uint32_t samples_per_group);

/* Cap the sweeps one kernel launch (or one batch step) runs for this
 * context: max_sweeps = 0 restores the automatic bound (the 32-bit per-lane
 * hop counters of the domain schedule, 2^20 otherwise).  Longer asep_sweep
 * and batch calls are split into launches of at most this many sweeps; the
 * streamed tiers run one sweep per step whatever the cap.  An autotuner knob:
 * results never depend on it (every sample's randomness is keyed by its
 * sweep index).  Takes effect for the next call. */
int asep_set_launch_sweeps(asep_ctx* ctx, uint32_t max_sweeps);

/* Balanced launches of a domain-schedule context whose samples sit in one
 * CTA each (or a few per CTA): a launch's sweeps are cut into chunks of
 * chunk_sweeps (at most 4096) and a persistent grid, as many CTAs as are
 * resident at once, takes (sample group, chunk) items in chunk-major order;
 * a CTA starts chunk k of a group once chunk k - 1 has written the group's
 * lattice back, so groups move between SMs between chunks and no SM idles
 * half-loaded while others hold two groups (e.g. 256 samples on 152 SMs).
 * 0 (the default) = one CTA per group for the whole launch.  Results never
 * depend on it.  The first nonzero call allocates (S + 1) words of device
 * memory for the chunk flags.  The wait for a previous chunk is bounded (5
 * seconds): if it runs out the launch gives up and asep_sync reports
 * ASEP_ERR_TIMEOUT.  Cluster and streamed plans ignore it; batches do not
 * use it.  No counterpart in the paper (its blocks each keep one chain). */
int asep_set_balance(asep_ctx* ctx, uint32_t chunk_sweeps);

/* Wait for all work of the context.  ASEP_ERR_TIMEOUT: a bounded
 * device-side wait ran out -- a streamed tile's wait for its bulk copy (one
 * second), or a balanced launch's wait for a previous chunk (five seconds);
 * the results since are invalid and every later call reports it until
 * asep_reset or asep_load_state replaces the lattice. */
int asep_sync(asep_ctx* ctx);

/* Fault injection for tests of the timeout path (default ASEP_FAULT_NONE).
 * ASEP_FAULT_COPY_STALL: the streamed domain tier's tile copies announce 16
 * bytes more than they carry, so the bounded wait for them runs out and the
 * sweep reports ASEP_ERR_TIMEOUT at the next synchronising call; nothing
 * faults or hangs.  Takes effect for the next launch. */
#define ASEP_FAULT_NONE 0u
#define ASEP_FAULT_COPY_STALL 1u
/* ASEP_FAULT_BALANCE_STALL: in a balanced launch, sample group 0 never
 * announces its first chunk, so the CTA that takes its second chunk waits
 * until the bound runs out (five seconds), the others stop waiting, and the
 * sweep reports ASEP_ERR_TIMEOUT; nothing faults or hangs. */
#define ASEP_FAULT_BALANCE_STALL 2u
int asep_inject_fault(asep_ctx* ctx, uint32_t fault);

/* Free everything the context owns.  NULL-safe; synchronises first. */
int asep_destroy(asep_ctx* ctx);

/* Last error message of the context (or of the last failed asep_create when
 * ctx is NULL); never NULL. */
const char* asep_last_error(const asep_ctx* ctx);

/* ---- Batched execution ------------------------------------------------- */

typedef struct asep_batch asep_batch; /* opaque; owns device workspace and a CUDA graph cache */

/* A batch runs many contexts -- each with its own L, D, rates, disorder and
 * samples -- in ONE persistent launch whose CTAs take (context, sample group)
 * items, largest first, from a device work queue.  Every sample's randomness
 * depends only on its own Philox counters, so each context's results are
 * bit-identical to running it alone with asep_sweep.  The batch owns device
 * workspace for up to max_jobs contexts (at most 16384) and max_items queue
 * items (a context contributes ceil(S / samples per group) items, at most
 * 2^18 per context: larger contexts run alone with asep_sweep).  Work is
 * enqueued on `stream` (cudaStream_t or NULL); the batch first waits for the
 * work already enqueued on each context's stream, and each context's stream
 * waits for the batch before its later work (contexts that share a stream
 * are ordered once).  Only ASEP_SCHED_DOMAIN contexts whose lattices sit in
 * shared memory (one CTA or a cluster); streamed-tier contexts run with
 * asep_sweep. */
int asep_batch_create(void* stream, uint32_t max_jobs, uint32_t max_items, asep_batch** out);

/* Advance ctxs[i] by n_mcs[i] sweeps (0 allowed) for i < n, in one persistent
 * launch per at most 2^20 sweeps.  Each context may appear once.  Asynchronous. */
int asep_batch_sweep(asep_batch* b, asep_ctx* const* ctxs, const uint64_t* n_mcs, uint32_t n);

/* Capture one batch step (these contexts, these sweep counts) as a CUDA
 * graph on the first call for this set, then launch it `replays` times.
 * The sweep index and the sample-time cursor of each context live in device
 * memory and advance with every replay.  Asynchronous. */
int asep_batch_graph(asep_batch* b, asep_ctx* const* ctxs, const uint64_t* n_mcs, uint32_t n, uint32_t replays);

/* Launch shape of the persistent kernel: threads per CTA (0 = the largest a
 * context needs; must be a multiple of 32 and at least that) and CTAs per SM
 * (0 = as many as fit).  Results do not depend on it. */
int asep_batch_set_launch(asep_batch* b, uint32_t threads, uint32_t ctas_per_sm);

/* Free the batch (NULL-safe); synchronises its stream first. */
int asep_batch_destroy(asep_batch* b);

const char* asep_batch_last_error(const asep_batch* b);

/* Batch sweep that allocates nothing -- for callers that may not allocate
 * device memory when they run work (memory owned by another allocator or a
 * fixed pool, a footprint frozen after start-up, or threads that must stay off
 * cudaMalloc's device-synchronising path).  Same work and bit-identical
 * results as asep_batch_create + asep_batch_sweep with a stream, but the work
 * queue (context descriptors, queue items, queue counter) lives in one static
 * device array of the library, about 80 KB, held on every GPU that loads the
 * library until the process exits.  Limits: at most 64 contexts per call and
 * 16384 sample groups per launch step; larger requests return
 * ASEP_ERR_INVALID.  Every context must use `stream`.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current, so make it before any stream capture.  A call with n = 0
 * (ctxs and n_mcs may then be NULL) does only the set-up on the current
 * device: it looks up the address and enqueues one empty launch of each
 * batch kernel on `stream`, which loads their code and lets the driver size
 * their per-thread local memory; a caller whose device footprint must be
 * fixed after start-up makes this call once per device at start-up.  All calls on one GPU
 * share its array, which keeps the last call's contents (the queue counter is
 * cleared by every call): calls whose work overlaps on the same GPU, e.g. on
 * two streams, race and must be ordered by the caller.  The host side of calls
 * is serialised by a lock.  Calls no allocating function, host or device.
 * No counterpart in the paper. */
int asep_batch_sweep_static(asep_ctx* const* ctxs, const uint64_t* n_mcs, uint32_t n, void* stream);

/* Threshold of probability p: 0 for p <= 0, ASEP_ALWAYS for p >= 1, else
 * round(p * 2^20) * 4096.  Host only. */
uint32_t asep_threshold(double p);

/* The attempt-count table of a domain with m bonds: T_k = floor(2^32 *
 * P(Poisson(m) <= k)); *k_lo = number of leading zero entries, table[j] =
 * T_{k_lo + j} for j < *n_out, ending before the first T_k = 2^32 - 1.  A
 * draw w gives K = k_lo + #{j : table[j] <= w}.  Host only; capacity is the
 * length of `table`. */
int asep_poisson_table(uint32_t m, uint32_t* k_lo, uint32_t* table, uint32_t capacity, uint32_t* n_out);

/* Microbenchmark of the random stream alone (no lattice memory): a grid of
 * `blocks` x `threads` threads, each running `calls` Philox4x32-10 calls in
 * the counter layout of the attempt stream and folding the outputs into one
 * word of `sink` (device buffer of blocks*threads uint32, owned by the
 * caller).  Writes the kernel time in milliseconds (CUDA events on `stream`)
 * to *ms; synchronises `stream`.  It bounds the attempt rate of the domain
 * kernel from above: one call feeds four attempts. */
int asep_philox_bench(void* stream, uint32_t blocks, uint32_t threads, uint32_t calls, uint32_t* sink, float* ms);

/* Microbenchmark of the attempt stream without lattice memory: as
 * asep_philox_bench, and each of a call's four output words r drives the
 * domain schedule's plain-ring update (sec. 2.1 bond rule: right hop iff the
 * bond reads 10 and r < p_thr, left hop iff 01 and r < q_thr) on a 64-bit
 * word pair w1:w0 held in registers, at bits j = r mod 32 and j + 1.  Thread
 * t starts from w0 = 0x55555555 ^ t, w1 = 0xAAAAAAAA ^ (t * 0x9E3779B9 mod
 * 2^32), takes call c with counter (c / 16, tag 4, call c mod 16, sample t,
 * group t / 32) under the key 0x243F6A8885A308D3 (the same as
 * asep_philox_bench), and writes its final pair to sink[2t], sink[2t + 1]
 * (device buffer of 2*blocks*threads uint32, owned by the caller).
 * Thresholds must be below ASEP_ALWAYS (else ASEP_ERR_INVALID).  Writes the
 * kernel time in milliseconds to *ms; synchronises `stream`.  It bounds the
 * domain kernel's attempt rate by the same random stream and bit operations
 * with the shared-memory round trip of each attempt removed. */
int asep_attempt_bench(void* stream, uint32_t blocks, uint32_t threads, uint32_t calls, uint32_t p_thr,
                       uint32_t q_thr, uint32_t* sink, float* ms);

/* Library version string. */
const char* asep_version(void);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* ASEP_H */

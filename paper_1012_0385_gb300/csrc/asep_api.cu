// asep_api.cu -- host runtime behind the C ABI declared in include/asep.h.
//
// A context owns: the packed lattices [S][planes][W], the quenched planes
// [R][W], the attempt-count (Poisson) table, the list of sample times, the
// height table [n_times][S][planes] (sum h as int64, sum h^2 as 128 bits)
// and the hop counters [S][4].  asep_sweep splits the requested sweeps into
// launches of the resident domain kernel (or the serial kernel) so that the
// per-lane 32-bit hop counters cannot wrap, and tells each launch which of
// its sweep counts are sample times.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/asep.h"
#include "asep_internal.h"
#include "asep_serial.h"

using namespace asep;

struct asep_ctx {
  asep_params p{};
  uint64_t L = 0;
  uint32_t D = 0, logD = 0, planes = 1, W = 0, S = 0, R = 0;
  cudaStream_t stream = nullptr;
  std::vector<uint64_t> times;
  uint32_t next_time = 0;  // first sample time not yet recorded
  uint64_t sweep = 0;
  // device buffers
  uint32_t* d_state = nullptr;
  uint32_t* d_mask = nullptr;
  uint32_t* d_ptab = nullptr;
  uint64_t* d_times = nullptr;
  int64_t* d_sh = nullptr;
  uint64_t* d_sh2 = nullptr;
  uint64_t* d_cnt = nullptr;
  Clock* d_clock = nullptr;  // device-side (sweep, next sample time); see asep_internal.h
  int64_t* d_tab_cnt = nullptr;  // [n_times][S][4]
  uint32_t* d_profile = nullptr; // [S][planes][W]
  uint32_t* d_snap = nullptr;    // [S][planes][W]
  int64_t* d_tab_ac = nullptr;   // [n_times][S][planes]
  int64_t* d_href = nullptr;     // [S][planes] sum h of the reference lattice (last create / reset / load)
  uint64_t* d_href2 = nullptr;   // [S][planes][2] its sum h^2 (not used)
  int64_t* d_hrefcnt = nullptr;  // [S][4] hop counters at the reference
  HeightPart* d_parts = nullptr;  // [S][planes][chunks] partial sums of a record over a long lattice
  uint32_t err_seen = 0;
  uint32_t ref_slot = 0;         // first sample-time slot recorded after the reference
  std::vector<std::pair<void*, size_t>> allocs;
  size_t dev_bytes = 0;
  // attempt-count table
  std::vector<uint32_t> ptab;
  uint32_t ptab_klo = 0;
  // resident launch plan
  uint32_t R2 = 0, logR2 = 0, G = 0, spc = 1, C = 0, Cp = 0, threads = 0, blocks = 0;
  uint32_t cluster = 1, Gc = 0;  // cluster tier: CTAs per sample, columns per CTA (kStreamTier: streamed)
  uint32_t tiles = 0;             // streamed tier: tiles per sample
  uint32_t* d_err = nullptr;      // device flag: a streamed tile's copy wait gave up
  uint32_t fault = ASEP_FAULT_NONE;  // injected fault (asep_inject_fault)
  size_t smem = 0;
  uint32_t max_sweeps_per_launch = 1;
  uint32_t launch_sweeps = 0;      // caller's cap on sweeps per launch (0 = none)
  uint32_t balance = 0;            // balanced launches: sweeps per chunk (0 = off)
  uint32_t* d_progress = nullptr;  // balanced launches: [S + 1] chunk flags and queue counter
  uint64_t launches = 0;
  std::string err;
};

namespace {

thread_local std::string g_create_error;

int fail(asep_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_create_error = buf;
  return code;
}

int cuda_fail(asep_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, ASEP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

uint32_t log2u(uint64_t x) {
  uint32_t k = 0;
  while ((1ull << k) < x) ++k;
  return k;
}

// Sweeps one launch (or one batch step) may run for this context: the hop
// counters' bound for the domain schedule, 2^20 otherwise, and the caller's
// cap from asep_set_launch_sweeps when set.
uint32_t sweeps_cap(const asep_ctx* c) {
  uint32_t cap = c->p.schedule == ASEP_SCHED_DOMAIN ? std::min<uint32_t>(c->max_sweeps_per_launch, 1u << 20)
                                                    : (1u << 20);
  if (c->launch_sweeps) cap = std::min(cap, c->launch_sweeps);
  return cap;
}

bool thr_ok(uint32_t t) { return t == ASEP_ALWAYS || (t & 0xFFFu) == 0; }

// T_k = floor(2^32 P(Poisson(m) <= k)).  Weights relative to the mode come
// from the exact ratio recurrence (no large logarithms cancel), and are
// normalised by their sum over mode +- 14 sigma (the mass outside is below
// 1e-40); the upper half is taken from the complementary tail sum.
int poisson_table_host(uint32_t m, std::vector<uint32_t>& tab, uint32_t& k_lo) {
  if (m == 0 || m > (1u << 16)) return ASEP_ERR_INVALID;
  const long double lm = static_cast<long double>(m);
  const long double sd = sqrtl(lm);
  const int64_t kmin = std::max<int64_t>(0, static_cast<int64_t>(lm - 14.0L * sd - 30.0L));
  const int64_t kmax = static_cast<int64_t>(lm + 14.0L * sd + 60.0L);
  const size_t n = static_cast<size_t>(kmax - kmin + 1);
  std::vector<long double> w(n);
  const int64_t mode = m;
  w[static_cast<size_t>(mode - kmin)] = 1.0L;
  for (int64_t k = mode - 1; k >= kmin; --k)
    w[static_cast<size_t>(k - kmin)] = w[static_cast<size_t>(k + 1 - kmin)] * static_cast<long double>(k + 1) / lm;
  for (int64_t k = mode + 1; k <= kmax; ++k)
    w[static_cast<size_t>(k - kmin)] = w[static_cast<size_t>(k - 1 - kmin)] * lm / static_cast<long double>(k);
  std::vector<long double> left(n), right(n);
  long double acc = 0.0L;
  for (size_t i = 0; i < n; ++i) {
    acc += w[i];
    left[i] = acc;  // sum_{j<=k}
  }
  const long double total = acc;
  acc = 0.0L;
  for (size_t i = n; i-- > 0;) {
    right[i] = acc;  // sum_{j>k}
    acc += w[i];
  }
  const long double two32 = 4294967296.0L;
  tab.clear();
  k_lo = static_cast<uint32_t>(kmin);  // every k < kmin has T_k = 0
  for (size_t i = 0; i < n; ++i) {
    const long double F = left[i] / total;
    uint64_t t;
    if (F < 0.5L) {
      t = static_cast<uint64_t>(floorl(F * two32));
    } else {
      const long double Gt = right[i] / total;
      t = 4294967295ull - static_cast<uint64_t>(floorl(Gt * two32));
    }
    if (t >= 4294967295ull) return ASEP_OK;
    if (t == 0) ++k_lo;
    else tab.push_back(static_cast<uint32_t>(t));
  }
  return ASEP_ERR_INVALID;  // the range did not reach the saturated tail
}

void* dev_alloc(asep_ctx* ctx, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* ptr = nullptr;
  if (ctx->p.alloc) {
    ptr = ctx->p.alloc(bytes, ctx->p.alloc_user);
    if (ptr && (reinterpret_cast<uintptr_t>(ptr) & 255u)) {  // the kernels need 256-byte aligned blocks
      ctx->p.free_fn(ptr, bytes, ctx->p.alloc_user);
      ptr = nullptr;
    }
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    ptr = nullptr;
  }
  if (ptr) {
    ctx->allocs.emplace_back(ptr, bytes);
    ctx->dev_bytes += bytes;
  }
  return ptr;
}

void release(asep_ctx* ctx) {
  if (!ctx) return;
  if (!ctx->allocs.empty()) cudaStreamSynchronize(ctx->stream);
  for (auto& a : ctx->allocs) {
    if (ctx->p.alloc) {
      if (ctx->p.free_fn) ctx->p.free_fn(a.first, a.second, ctx->p.alloc_user);
    } else {
      cudaFree(a.first);
    }
  }
  ctx->allocs.clear();
}

int validate(const asep_params* p, asep_ctx* ctx) {
  if (!p) return fail(ctx, ASEP_ERR_INVALID, "params is NULL");
  if (p->model > ASEP_MODEL_TWO_LANE) return fail(ctx, ASEP_ERR_INVALID, "unknown model %u", p->model);
  if (p->schedule > ASEP_SCHED_SCA) return fail(ctx, ASEP_ERR_INVALID, "unknown schedule %u", p->schedule);
  if (p->L < 64 || (p->L & 63) || p->L > (1ull << 28))
    return fail(ctx, ASEP_ERR_INVALID, "L = %llu must be a multiple of 64 in [64, 2^28]", (unsigned long long)p->L);
  if (p->n_realizations == 0 || p->samples_per_real == 0)
    return fail(ctx, ASEP_ERR_INVALID, "n_realizations and samples_per_real must be >= 1");
  const uint64_t S = static_cast<uint64_t>(p->n_realizations) * p->samples_per_real;
  if (S > (1u << 24)) return fail(ctx, ASEP_ERR_INVALID, "too many samples (%llu)", (unsigned long long)S);
  if (p->first_sample % p->samples_per_real)
    return fail(ctx, ASEP_ERR_INVALID, "first_sample must be a multiple of samples_per_real");
  if (static_cast<uint64_t>(p->first_sample) + S > (1ull << 32))
    return fail(ctx, ASEP_ERR_INVALID, "sample ids exceed 32 bits");
  if (!thr_ok(p->p_thr) || !thr_ok(p->q_thr) || !thr_ok(p->dis_a_thr) || !thr_ok(p->dis_b_thr) ||
      !thr_ok(p->dis_c_thr))
    return fail(ctx, ASEP_ERR_INVALID, "thresholds must be 0, ASEP_ALWAYS or multiples of 4096");
  if (p->dis_kind > ASEP_DIS_CROSSING) return fail(ctx, ASEP_ERR_INVALID, "unknown dis_kind %u", p->dis_kind);
  if (p->dis_kind == ASEP_DIS_CROSSING && p->model != ASEP_MODEL_TWO_LANE)
    return fail(ctx, ASEP_ERR_INVALID, "crossing probabilities are defined for the two-lane model");
  if ((p->dis_kind == ASEP_DIS_BIMODAL || p->dis_kind == ASEP_DIS_BIMODAL_PQ) && p->model != ASEP_MODEL_RING)
    return fail(ctx, ASEP_ERR_INVALID, "bimodal disorder is defined for the ring model");
  if (p->dis_kind == ASEP_DIS_TURNING && p->model != ASEP_MODEL_TWO_LANE)
    return fail(ctx, ASEP_ERR_INVALID, "turning sites are defined for the two-lane model");
  if (p->init_kind > ASEP_INIT_BERNOULLI_HALF) return fail(ctx, ASEP_ERR_INVALID, "unknown init_kind %u", p->init_kind);
  if (p->flags & ~(ASEP_FLAG_NO_HOP_COUNTS | ASEP_FLAG_PROFILE | ASEP_FLAG_AUTOCORR))
    return fail(ctx, ASEP_ERR_INVALID, "unknown flags 0x%x", p->flags);
  if ((p->flags & ASEP_FLAG_PROFILE) && p->n_sample_times > (1u << 27))
    return fail(ctx, ASEP_ERR_INVALID, "ASEP_FLAG_PROFILE takes at most 2^27 sample times (32-bit bin counts)");
  if (p->flags & ASEP_FLAG_AUTOCORR) {
    bool found = false;
    for (uint32_t i = 0; i < p->n_sample_times && p->sample_times; ++i) found = found || p->sample_times[i] == p->autocorr_t0;
    if (!found) return fail(ctx, ASEP_ERR_INVALID, "autocorr_t0 must be one of the sample times");
  }
  if ((p->alloc == nullptr) != (p->free_fn == nullptr))
    return fail(ctx, ASEP_ERR_INVALID, "alloc and free_fn must be given together");
  if (p->n_sample_times && !p->sample_times) return fail(ctx, ASEP_ERR_INVALID, "sample_times is NULL");
  for (uint32_t i = 1; i < p->n_sample_times; ++i)
    if (p->sample_times[i] <= p->sample_times[i - 1])
      return fail(ctx, ASEP_ERR_INVALID, "sample_times must be strictly ascending");
  if (p->schedule == ASEP_SCHED_SERIAL && !is_pow2(p->L))
    return fail(ctx, ASEP_ERR_INVALID, "the serial schedule needs L a power of two");
  if (p->schedule == ASEP_SCHED_SCA && p->L % 256)
    return fail(ctx, ASEP_ERR_INVALID, "the SCA schedule needs L a multiple of 256");
  return ASEP_OK;
}

// SCA plan.  Resident: one CTA per sample holding the ring in shared memory,
// a thread per unit of 8 words (at most 1024 threads, 512 with a quenched
// plane).  Streamed (kStreamTier): the ring in global memory, a thread per
// unit, one launch per phase.  force: 0 = resident when it fits, 1 =
// resident, kStreamTier = streamed.
int plan_sca(asep_ctx* ctx, uint32_t force) {
  const uint32_t units = ctx->W / 8;
  const bool quenched = ctx->p.dis_kind != ASEP_DIS_NONE;
  const size_t smem = sca_smem_bytes(ctx->W, ctx->planes, dis_planes(ctx->p.dis_kind));
  const bool fits = smem <= 200u * 1024u;
  if (force == 1 && !fits)
    return fail(ctx, ASEP_ERR_INVALID, "the resident SCA plan needs %zu bytes of shared memory (at most 200 KB)",
                smem);
  if (force == kStreamTier || !fits) {
    ctx->cluster = kStreamTier;
    ctx->threads = 256;
    ctx->smem = 0;
    ctx->blocks = ctx->S * ((units + 255u) / 256u);
  } else {
    const uint32_t cap = quenched ? 512u : 1024u;
    ctx->cluster = 1;
    ctx->threads = std::min<uint32_t>(cap, (units + 31u) / 32u * 32u);
    ctx->smem = smem;
    ctx->blocks = ctx->S;
  }
  return ASEP_OK;
}

// Launch plan.  Resident: columns = super-domains, one thread per column, a
// whole sample (or several small ones) per CTA.  Cluster tier: each sample
// spread over 2..16 CTAs of a thread-block cluster, for samples one CTA
// cannot hold -- or, on request, to spread few large samples over more SMs.
// force_cluster: 0 = choose, 1 = resident only, n > 1 = exactly n CTAs per
// sample.  force_spc: samples per CTA for the resident plan (0 = choose).
// The plan changes only the launch shape, never the results.
// Serial-schedule plan.  kSerialRounds: one CTA per sample, the sweep's
// attempts in dependency rounds (when the lattice and the sweep's draws fit
// shared memory); kSerialWarp: one warp per sample.  force: 0 = the rounds
// plan when it applies and the samples number at most four per SM (measured
// on rings of 4096 sites: 4.6x the warp plan at 8 samples and at 152, 0.77x
// at 1024, where the warps alone fill the GPU), else the warp plan.
int plan_serial(asep_ctx* ctx, uint32_t force) {
  const uint32_t model = ctx->p.model, dis = ctx->p.dis_kind;
  const size_t smem = serial_rounds_smem_bytes(model, dis, ctx->L);
  if (force == kSerialRounds && smem == 0)
    return fail(ctx, ASEP_ERR_INVALID, "the one-CTA serial plan needs at most %u attempts per sweep and 200 KB of "
                "shared memory", kSerialRoundsMaxAttempts);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                               cudaSuccess || sms <= 0) {
    (void)cudaGetLastError();
    sms = 1;
  }
  const bool few = ctx->S <= 4u * static_cast<uint32_t>(sms);
  if (force == kSerialRounds || (force == 0 && smem > 0 && few)) {
    ctx->cluster = kSerialRounds;
    ctx->spc = 1;
    ctx->threads = serial_rounds_threads(model, ctx->L);
    ctx->smem = smem;
    ctx->blocks = ctx->S;
  } else {
    const uint32_t warps = serial_warp_plan_warps(ctx->S);
    ctx->cluster = kSerialWarp;
    ctx->spc = warps;
    ctx->threads = 32 * warps;
    ctx->smem = 0;
    ctx->blocks = (ctx->S + warps - 1) / warps;
  }
  return ASEP_OK;
}

// Automatic tile width of the streamed tier, in columns (one thread each).
constexpr uint32_t kStreamTileColumns = 128;

int plan_domain(asep_ctx* ctx, uint32_t force_cluster, uint32_t force_spc) {
  const uint32_t D = ctx->D;
  ctx->R2 = 2 * D / 32;
  ctx->logR2 = log2u(ctx->R2);
  const uint64_t G = ctx->L / (2ull * D);
  ctx->G = static_cast<uint32_t>(G);
  const uint32_t dis = ctx->p.dis_kind;
  const uint32_t ptab_n = static_cast<uint32_t>(ctx->ptab.size());
  bool placed = false;
  if (G <= 1024 && force_cluster <= 1) {
    uint32_t spc = force_spc ? force_spc : 1;
    if (!force_spc && ctx->G < 128) spc = std::max<uint32_t>(1, std::min<uint32_t>(ctx->S, 128 / ctx->G));
    for (;;) {
      const uint32_t C = spc * ctx->G;
      const uint32_t Cp = (C + 31) / 32 * 32;
      const size_t smem = domain_smem_bytes(ctx->p.model, dis, ctx->R2, Cp, ptab_n, Cp);
      if (smem <= 227 * 1024 && Cp <= 1024) {
        ctx->cluster = 1;
        ctx->Gc = 0;
        ctx->spc = spc;
        ctx->C = C;
        ctx->Cp = Cp;
        ctx->threads = Cp;
        ctx->smem = smem;
        ctx->blocks = (ctx->S + spc - 1) / spc;
        placed = true;
        break;
      }
      if (spc == 1 || force_spc) break;
      spc = std::max<uint32_t>(1, spc / 2);
    }
    if (!placed && (force_cluster == 1 || force_spc))
      return fail(ctx, ASEP_ERR_INVALID, "the requested resident plan does not fit one CTA");
  }
  for (uint32_t nc = force_cluster > 1 ? force_cluster : 2; !placed && nc <= 16 && force_cluster != kStreamTier;
       nc *= 2) {
    const uint32_t Gc = static_cast<uint32_t>((G + nc - 1) / nc);
    const bool ok = Gc <= 1024 && (G + Gc - 1) / Gc == nc;  // every CTA of the cluster holds columns
    const uint32_t Cp = (Gc + 31) / 32 * 32;
    const size_t smem = domain_smem_bytes(ctx->p.model, dis, ctx->R2, Cp, ptab_n, Cp);
    if (ok && smem + 64 <= 227 * 1024 && Cp <= 1024 && cluster_fits(ctx->p.model, dis, nc, Cp, smem) > 0) {
      ctx->cluster = nc;
      ctx->spc = 1;
      ctx->C = Gc;
      ctx->Gc = Gc;
      ctx->Cp = Cp;
      ctx->threads = Cp;
      ctx->smem = smem;
      ctx->blocks = ctx->S;
      placed = true;
    }
    if (force_cluster > 1) break;
  }
  // streamed tier: tiles of C columns (a multiple of 32, at least two tiles) through shared memory.
  // Automatic width kStreamTileColumns: narrow tiles keep several CTAs on every SM, so one CTA's bulk
  // copy and phase tail overlap another's attempts, and the last wave of tiles is short.
  // force_spc with force_cluster == kStreamTier: exactly that width.
  if (!placed && (force_cluster == 0 || force_cluster == kStreamTier) && ctx->W % 4 == 0) {
    const uint32_t C0 = force_cluster == kStreamTier && force_spc ? force_spc : kStreamTileColumns;
    for (uint32_t C = C0; C >= 32 && !placed; C -= 32) {
      if (2ull * C > G || (force_cluster == kStreamTier && force_spc && C != force_spc)) continue;
      const size_t smem = stream_smem_bytes(ctx->p.model, dis, ctx->R2, C, ptab_n);
      if (smem > 200u * 1024u) continue;
      ctx->cluster = kStreamTier;
      ctx->spc = 1;
      ctx->C = C;
      ctx->Gc = 0;
      ctx->Cp = C;
      ctx->threads = C;
      ctx->smem = smem;
      ctx->tiles = static_cast<uint32_t>((G + C - 1) / C);
      ctx->blocks = ctx->tiles * ctx->S;
      placed = true;
    }
  }
  if (!placed)
    return fail(ctx, ASEP_ERR_INVALID, "L = %llu (%llu columns, %u planes) fits neither one CTA, a cluster of "
                "up to 16 CTAs nor streamed tiles on this device%s", (unsigned long long)ctx->L,
                (unsigned long long)G, ctx->planes, force_cluster > 1 ? " with the requested plan" : "");
  // per-lane 32-bit hop counters: at most 2 phases x largest count + 2D turns per sweep
  const uint64_t per_sweep = 2ull * (ctx->ptab_klo + ctx->ptab.size() + 1) + 2ull * D;
  ctx->max_sweeps_per_launch = static_cast<uint32_t>(std::max<uint64_t>(1, 4000000000ull / per_sweep));
  return ASEP_OK;
}

Geometry geometry(const asep_ctx* ctx) {
  Geometry g;
  g.L = ctx->L;
  g.W = ctx->W;
  g.planes = ctx->planes;
  g.S = ctx->S;
  g.samples_per_real = ctx->p.samples_per_real;
  g.first_sample = ctx->p.first_sample;
  return g;
}

Rates rates(const asep_ctx* ctx) {
  Rates r;
  r.p = ctx->p.p_thr;
  r.q = ctx->p.q_thr;
  const bool bimodal = ctx->p.dis_kind == ASEP_DIS_BIMODAL || ctx->p.dis_kind == ASEP_DIS_BIMODAL_PQ;
  r.p_slow = bimodal ? ctx->p.dis_b_thr : ctx->p.p_thr;
  r.q_slow = bimodal ? ctx->p.dis_c_thr : ctx->p.q_thr;
  const bool lanes = ctx->p.dis_kind == ASEP_DIS_TURNING || ctx->p.dis_kind == ASEP_DIS_CROSSING;
  r.omega = lanes ? ctx->p.dis_b_thr : 0u;
  r.omega_slow = ctx->p.dis_kind == ASEP_DIS_CROSSING ? ctx->p.dis_c_thr : r.omega;
  r.p_always = r.p == ASEP_ALWAYS;
  r.q_always = r.q == ASEP_ALWAYS;
  r.pb = hop_bound(r.p);
  r.qb = hop_bound(r.q);
  r.pb_slow = hop_bound(r.p_slow);
  r.qb_slow = hop_bound(r.q_slow);
  return r;
}

int clear_extras(asep_ctx* ctx) {
  const size_t n_times = std::max<size_t>(1, ctx->times.size());
  const size_t state_words = static_cast<size_t>(ctx->S) * ctx->planes * ctx->W;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ctx->d_tab_cnt, 0, n_times * ctx->S * 32, ctx->stream)) != cudaSuccess ||
      (ctx->d_profile && (e = cudaMemsetAsync(ctx->d_profile, 0, state_words * 4, ctx->stream)) != cudaSuccess) ||
      (ctx->d_tab_ac &&
       (e = cudaMemsetAsync(ctx->d_tab_ac, 0, n_times * ctx->S * ctx->planes * 8, ctx->stream)) != cudaSuccess))
    return cuda_fail(ctx, e, "clear observables");
  return ASEP_OK;
}

Extras extras(const asep_ctx* ctx) {
  Extras ex;
  ex.tab_cnt = ctx->d_tab_cnt;
  ex.profile = ctx->d_profile;
  ex.snap = ctx->d_snap;
  ex.tab_ac = ctx->d_tab_ac;
  ex.t0 = ctx->p.autocorr_t0;
  return ex;
}

int copy_out(asep_ctx* ctx, void* dst, const void* src, size_t bytes, const char* what) {
  int rc = asep_sync(ctx);
  if (rc != ASEP_OK) return rc;
  if (bytes == 0) return ASEP_OK;
  const cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return ASEP_OK;
}

// Heights and hop counters of the current lattice as the reference of
// asep_height_offset (a record into the reference tables, no observables).
// Forget a streamed tile's copy timeout (for a call that replaces the
// lattice): wait for the context's work, then clear the device flag.
int clear_timeout(asep_ctx* ctx) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  if (ctx->d_err && (e = cudaMemset(ctx->d_err, 0, 16)) != cudaSuccess) return cuda_fail(ctx, e, "clear error flag");
  ctx->err_seen = 0;
  return ASEP_OK;
}

int record_reference(asep_ctx* ctx) {
  HeightsLaunch h;
  h.geo = geometry(ctx);
  h.state = ctx->d_state;
  h.slot = 0;
  h.t = 0;
  h.tab_sh = ctx->d_href;
  h.tab_sh2 = ctx->d_href2;
  h.counters = ctx->d_cnt;
  h.ex = Extras{};
  h.ex.tab_cnt = ctx->d_hrefcnt;
  h.parts = ctx->d_parts;
  const cudaError_t e = launch_heights(h, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reference heights kernel");
  ctx->launches += height_chunks(ctx->W) > 1 ? 2 : 1;
  return ASEP_OK;
}

int record_now(asep_ctx* ctx, uint32_t slot) {
  HeightsLaunch h;
  h.geo = geometry(ctx);
  h.state = ctx->d_state;
  h.slot = slot;
  h.t = ctx->times.empty() ? 0 : ctx->times[slot];
  h.tab_sh = ctx->d_sh;
  h.tab_sh2 = ctx->d_sh2;
  h.counters = ctx->d_cnt;
  h.ex = extras(ctx);
  h.parts = ctx->d_parts;
  const cudaError_t e = launch_heights(h, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "heights kernel");
  ctx->launches += height_chunks(ctx->W) > 1 ? 2 : 1;
  return ASEP_OK;
}

DomainLaunch domain_desc(const asep_ctx* ctx, uint32_t n) {
  DomainLaunch a{};
  a.geo = geometry(ctx);
  a.model = ctx->p.model;
  a.dis = ctx->p.dis_kind;
  a.count_hops = (ctx->p.model == ASEP_MODEL_TWO_LANE || !(ctx->p.flags & ASEP_FLAG_NO_HOP_COUNTS)) ? 1u : 0u;
  a.state = ctx->d_state;
  a.mask = ctx->d_mask;
  a.ptab = ctx->d_ptab;
  a.ptab_n = static_cast<uint32_t>(ctx->ptab.size());
  a.ptab_klo = ctx->ptab_klo;
  a.D = ctx->D;
  a.logD = ctx->logD;
  a.R2 = ctx->R2;
  a.logR2 = ctx->logR2;
  a.row_bits = (ctx->D - 1) & ~31u;
  a.G = ctx->G;
  a.spc = ctx->spc;
  a.C = ctx->C;
  a.Cp = ctx->Cp;
  a.n_groups = ctx->blocks;
  a.cluster = ctx->cluster;
  a.Gc = ctx->Gc;
  {
    // every warp inside one sample, and the idle realign buffer holds 5 words per column
    const uint32_t np = (ctx->p.model == ASEP_MODEL_TWO_LANE ? 2u : 1u) + dis_planes(ctx->p.dis_kind);
    a.lane_sort = (ctx->cluster <= 1 && ctx->G % 32 == 0 && np * (ctx->R2 + 1) >= 5) ? 1u : 0u;
  }
  a.rates = rates(ctx);
  {
    // SCA: planes needed to decide u < t for every threshold that is neither 0 nor always
    uint32_t tz = 20;
    for (uint32_t t : {a.rates.p, a.rates.q, a.rates.p_slow, a.rates.q_slow}) {
      const uint32_t t20 = t >> 12;
      if (t != 0u && t != ASEP_ALWAYS) tz = std::min<uint32_t>(tz, static_cast<uint32_t>(__builtin_ctz(t20)));
    }
    a.sca_kmax = 20u - tz;
  }
  a.seed = ctx->p.seed;
  a.ks = key_schedule(ctx->p.seed);
  a.n_sweeps = n;
  a.clock = ctx->d_clock;
  a.times = ctx->d_times;
  a.n_times = static_cast<uint32_t>(ctx->times.size());
  a.tab_sh = ctx->d_sh;
  a.tab_sh2 = ctx->d_sh2;
  a.counters = ctx->d_cnt;
  a.ex = extras(ctx);
  return a;
}

// Host mirror of the device clock after n more sweeps.
void advance_host(asep_ctx* ctx, uint64_t n) {
  ctx->sweep += n;
  while (ctx->next_time < ctx->times.size() && ctx->times[ctx->next_time] <= ctx->sweep) ++ctx->next_time;
}

int set_clock(asep_ctx* ctx, uint64_t sweep, uint32_t next_time) {
  const cudaError_t e = launch_set_clock(ctx->d_clock, sweep, next_time, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "set clock");
  ++ctx->launches;
  ctx->sweep = sweep;
  ctx->next_time = next_time;
  return ASEP_OK;
}

// Times one microbenchmark launch with CUDA events on `stream` and
// synchronises it.
template <typename Launch>
int timed_bench(void* stream, float* ms, const char* what, Launch launch) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(nullptr, e, "event create");
  }
  int rc = ASEP_OK;
  if ((e = cudaEventRecord(e0, st)) != cudaSuccess || (e = launch(st)) != cudaSuccess ||
      (e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
      (e = cudaEventElapsedTime(ms, e0, e1)) != cudaSuccess)
    rc = cuda_fail(nullptr, e, what);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

bool bench_shape_ok(uint32_t blocks, uint32_t threads) {
  return blocks != 0 && threads != 0 && threads <= 1024 && (threads & 31) == 0;
}

}  // namespace

extern "C" {

const char* asep_version(void) { return "asep 0.1 (sm_103a)"; }

uint32_t asep_threshold(double p) {
  if (!(p > 0.0)) return 0u;
  if (p >= 1.0) return ASEP_ALWAYS;
  const double q = std::floor(p * 1048576.0 + 0.5);
  if (q >= 1048576.0) return ASEP_ALWAYS;
  return static_cast<uint32_t>(q) << 12;
}

int asep_poisson_table(uint32_t m, uint32_t* k_lo, uint32_t* table, uint32_t capacity, uint32_t* n_out) {
  if (!k_lo || !n_out) return ASEP_ERR_INVALID;
  std::vector<uint32_t> tab;
  uint32_t klo = 0;
  const int rc = poisson_table_host(m, tab, klo);
  if (rc != ASEP_OK) return rc;
  *k_lo = klo;
  *n_out = static_cast<uint32_t>(tab.size());
  if (table) {
    if (capacity < tab.size()) return ASEP_ERR_INVALID;
    std::memcpy(table, tab.data(), tab.size() * sizeof(uint32_t));
  }
  return ASEP_OK;
}

int asep_philox_bench(void* stream, uint32_t blocks, uint32_t threads, uint32_t calls, uint32_t* sink, float* ms) {
  if (!sink || !ms || !bench_shape_ok(blocks, threads))
    return fail(nullptr, ASEP_ERR_INVALID, "philox bench: bad launch shape");
  return timed_bench(stream, ms, "philox bench", [&](cudaStream_t st) {
    return launch_philox_bench(blocks, threads, calls, sink, st);
  });
}

int asep_attempt_bench(void* stream, uint32_t blocks, uint32_t threads, uint32_t calls, uint32_t p_thr,
                       uint32_t q_thr, uint32_t* sink, float* ms) {
  if (!sink || !ms || !bench_shape_ok(blocks, threads))
    return fail(nullptr, ASEP_ERR_INVALID, "attempt bench: bad launch shape");
  if (p_thr == ASEP_ALWAYS || q_thr == ASEP_ALWAYS)
    return fail(nullptr, ASEP_ERR_INVALID, "attempt bench: thresholds below ASEP_ALWAYS only");
  return timed_bench(stream, ms, "attempt bench", [&](cudaStream_t st) {
    return launch_attempt_bench(blocks, threads, calls, p_thr, q_thr, sink, st);
  });
}

const char* asep_last_error(const asep_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

}  // extern "C"

namespace {

// Sizes, attempt-count table and launch plan of a new context (no device
// memory, no stream work).  Used by asep_create and asep_plan.
int plan_context(asep_ctx* ctx, const asep_params* params) {
  ctx->p = *params;
  ctx->p.sample_times = nullptr;
  ctx->L = params->L;
  ctx->W = static_cast<uint32_t>(params->L / 32);
  ctx->planes = params->model == ASEP_MODEL_TWO_LANE ? 2u : 1u;
  ctx->S = params->n_realizations * params->samples_per_real;
  ctx->R = params->dis_kind == ASEP_DIS_NONE ? 0u : params->n_realizations;
  ctx->stream = static_cast<cudaStream_t>(params->stream);
  ctx->times.assign(params->sample_times, params->sample_times + params->n_sample_times);
  if (params->schedule == ASEP_SCHED_DOMAIN) {
    uint32_t D = params->domain_sites;
    if (D == 0) {
      D = 256;
      while (D > 32 && ctx->L % (2ull * D)) D >>= 1;
    }
    if (D < 32 || D > 2048 || !is_pow2(D) || ctx->L % (2ull * D))
      return fail(ctx, ASEP_ERR_INVALID, "domain_sites = %u must be a power of two in [32, 2048] with "
                  "L a multiple of 2*domain_sites", D);
    ctx->D = D;
    ctx->logD = log2u(D);
    const uint32_t bonds = ctx->planes * D;
    if (poisson_table_host(bonds, ctx->ptab, ctx->ptab_klo) != ASEP_OK)
      return fail(ctx, ASEP_ERR_INVALID, "attempt-count table for %u bonds failed", bonds);
    return plan_domain(ctx, 0, 0);
  }
  if (params->schedule == ASEP_SCHED_SCA) return plan_sca(ctx, 0);
  return plan_serial(ctx, 0);
}

// Device bytes asep_create allocates for a planned context: the same list,
// in the same sizes, as its allocations below.
size_t planned_device_bytes(const asep_ctx* ctx) {
  size_t total = 0;
  const auto add = [&](size_t b) { total += b ? b : 16; };
  const size_t state_words = static_cast<size_t>(ctx->S) * ctx->planes * ctx->W;
  const size_t n_times = std::max<size_t>(1, ctx->times.size());
  const size_t entries = n_times * ctx->S * ctx->planes;
  add(state_words * 4);
  add(static_cast<size_t>(ctx->S) * 4 * 8);
  add(entries * 8);
  add(entries * 16);
  add(n_times * 8);
  add(sizeof(Clock));
  add(n_times * ctx->S * 32);
  add(static_cast<size_t>(ctx->S) * ctx->planes * 8);
  add(static_cast<size_t>(ctx->S) * ctx->planes * 16);
  add(static_cast<size_t>(ctx->S) * 32);
  add(16);
  if (height_chunks(ctx->W) > 1) add(static_cast<size_t>(ctx->S) * ctx->planes * height_chunks(ctx->W) * sizeof(HeightPart));
  if (ctx->p.flags & ASEP_FLAG_PROFILE) add(state_words * 4);
  if (ctx->p.flags & ASEP_FLAG_AUTOCORR) {
    add(state_words * 4);
    add(entries * 8);
  }
  if (ctx->R) add(static_cast<size_t>(ctx->R) * dis_planes(ctx->p.dis_kind) * ctx->W * 4);
  if (!ctx->ptab.empty()) add(ctx->ptab.size() * 4);
  return total;
}

void fill_info(const asep_ctx* ctx, asep_info* info) {
  info->L = ctx->L;
  info->D = ctx->D;
  info->planes = ctx->planes;
  info->S = ctx->S;
  info->n_recorded = ctx->next_time;
  info->sweep = ctx->sweep;
  info->attempts_per_sweep = ctx->L * ctx->planes;
  info->device_bytes = ctx->dev_bytes;
  info->kernel_launches = ctx->launches;
  info->cluster = ctx->cluster;
  info->samples_per_group = ctx->spc;
  info->groups = ctx->blocks;
  info->threads = ctx->threads;
  info->smem_bytes = static_cast<uint32_t>(ctx->smem);
  info->tile_columns = ctx->p.schedule == ASEP_SCHED_DOMAIN && ctx->cluster == kStreamTier ? ctx->C : 0;
}

}  // namespace

extern "C" {

int asep_plan(const asep_params* params, asep_info* info) {
  g_create_error.clear();
  if (!info) return fail(nullptr, ASEP_ERR_INVALID, "info is NULL");
  int rc = validate(params, nullptr);
  if (rc != ASEP_OK) return rc;
  asep_ctx ctx;
  rc = plan_context(&ctx, params);
  if (rc != ASEP_OK) {
    g_create_error = ctx.err;
    return rc;
  }
  fill_info(&ctx, info);
  info->device_bytes = planned_device_bytes(&ctx);
  return ASEP_OK;
}

int asep_create(const asep_params* params, asep_ctx** out) {
  if (!out) return fail(nullptr, ASEP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  g_create_error.clear();
  int rc = validate(params, nullptr);
  if (rc != ASEP_OK) return rc;
  asep_ctx* ctx = new (std::nothrow) asep_ctx();
  if (!ctx) return fail(nullptr, ASEP_ERR_NOMEM, "host allocation failed");

  auto bail = [&](int code) {
    g_create_error = ctx->err;
    release(ctx);
    delete ctx;
    return code;
  };
  rc = plan_context(ctx, params);
  if (rc != ASEP_OK) return bail(rc);

  // device memory (planned_device_bytes lists the same sizes)
  const size_t state_words = static_cast<size_t>(ctx->S) * ctx->planes * ctx->W;
  const size_t n_times = std::max<size_t>(1, ctx->times.size());
  const size_t entries = n_times * ctx->S * ctx->planes;
  ctx->d_state = static_cast<uint32_t*>(dev_alloc(ctx, state_words * 4));
  ctx->d_cnt = static_cast<uint64_t*>(dev_alloc(ctx, static_cast<size_t>(ctx->S) * 4 * 8));
  ctx->d_sh = static_cast<int64_t*>(dev_alloc(ctx, entries * 8));
  ctx->d_sh2 = static_cast<uint64_t*>(dev_alloc(ctx, entries * 16));
  ctx->d_times = static_cast<uint64_t*>(dev_alloc(ctx, n_times * 8));
  ctx->d_clock = static_cast<Clock*>(dev_alloc(ctx, sizeof(Clock)));
  ctx->d_tab_cnt = static_cast<int64_t*>(dev_alloc(ctx, n_times * ctx->S * 32));
  ctx->d_href = static_cast<int64_t*>(dev_alloc(ctx, static_cast<size_t>(ctx->S) * ctx->planes * 8));
  ctx->d_href2 = static_cast<uint64_t*>(dev_alloc(ctx, static_cast<size_t>(ctx->S) * ctx->planes * 16));
  ctx->d_hrefcnt = static_cast<int64_t*>(dev_alloc(ctx, static_cast<size_t>(ctx->S) * 32));
  ctx->d_err = static_cast<uint32_t*>(dev_alloc(ctx, 16));
  if (height_chunks(ctx->W) > 1)
    ctx->d_parts = static_cast<HeightPart*>(
        dev_alloc(ctx, static_cast<size_t>(ctx->S) * ctx->planes * height_chunks(ctx->W) * sizeof(HeightPart)));
  if (params->flags & ASEP_FLAG_PROFILE) ctx->d_profile = static_cast<uint32_t*>(dev_alloc(ctx, state_words * 4));
  if (params->flags & ASEP_FLAG_AUTOCORR) {
    ctx->d_snap = static_cast<uint32_t*>(dev_alloc(ctx, state_words * 4));
    ctx->d_tab_ac = static_cast<int64_t*>(dev_alloc(ctx, entries * 8));
  }
  if (ctx->R)
    ctx->d_mask = static_cast<uint32_t*>(
        dev_alloc(ctx, static_cast<size_t>(ctx->R) * dis_planes(params->dis_kind) * ctx->W * 4));
  if (!ctx->ptab.empty()) ctx->d_ptab = static_cast<uint32_t*>(dev_alloc(ctx, ctx->ptab.size() * 4));
  if (!ctx->d_state || !ctx->d_cnt || !ctx->d_sh || !ctx->d_sh2 || !ctx->d_times || !ctx->d_clock ||
      !ctx->d_tab_cnt || !ctx->d_href || !ctx->d_href2 || !ctx->d_hrefcnt || !ctx->d_err ||
      (height_chunks(ctx->W) > 1 && !ctx->d_parts) ||
      ((params->flags & ASEP_FLAG_PROFILE) && !ctx->d_profile) ||
      ((params->flags & ASEP_FLAG_AUTOCORR) && (!ctx->d_snap || !ctx->d_tab_ac)) || (ctx->R && !ctx->d_mask) ||
      (!ctx->ptab.empty() && !ctx->d_ptab))
    return bail(fail(ctx, ASEP_ERR_NOMEM, "device allocation failed (%zu bytes so far)", ctx->dev_bytes));

  cudaError_t e;
  if (!ctx->times.empty() &&
      (e = cudaMemcpyAsync(ctx->d_times, ctx->times.data(), ctx->times.size() * 8, cudaMemcpyHostToDevice,
                           ctx->stream)) != cudaSuccess)
    return bail(cuda_fail(ctx, e, "copy sample times"));
  if (!ctx->ptab.empty() &&
      (e = cudaMemcpyAsync(ctx->d_ptab, ctx->ptab.data(), ctx->ptab.size() * 4, cudaMemcpyHostToDevice,
                           ctx->stream)) != cudaSuccess)
    return bail(cuda_fail(ctx, e, "copy attempt-count table"));
  if ((e = cudaMemsetAsync(ctx->d_cnt, 0, static_cast<size_t>(ctx->S) * 32, ctx->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->d_err, 0, 16, ctx->stream)) != cudaSuccess)
    return bail(cuda_fail(ctx, e, "clear counters"));
  if ((e = cudaMemsetAsync(ctx->d_sh, 0, entries * 8, ctx->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->d_sh2, 0, entries * 16, ctx->stream)) != cudaSuccess)
    return bail(cuda_fail(ctx, e, "clear height table"));
  if ((rc = clear_extras(ctx)) != ASEP_OK) return bail(rc);

  InitLaunch il;
  il.geo = geometry(ctx);
  il.state = ctx->d_state;
  il.init_kind = params->init_kind;
  il.init_seed = params->init_seed;
  if ((e = launch_init(il, ctx->stream)) != cudaSuccess) return bail(cuda_fail(ctx, e, "init kernel"));
  ++ctx->launches;
  if (ctx->R) {
    DisorderLaunch dl;
    dl.L = ctx->L;
    dl.W = ctx->W;
    dl.R = ctx->R;
    dl.planes = dis_planes(params->dis_kind);
    dl.first_real = params->first_sample / params->samples_per_real;
    dl.thr = params->dis_a_thr;
    dl.dis_seed = params->dis_seed;
    dl.mask = ctx->d_mask;
    if ((e = launch_disorder(dl, ctx->stream)) != cudaSuccess) return bail(cuda_fail(ctx, e, "disorder kernel"));
    ++ctx->launches;
  }
  if ((rc = record_reference(ctx)) != ASEP_OK) return bail(rc);
  uint32_t next = 0;
  if (!ctx->times.empty() && ctx->times[0] == 0) {
    rc = record_now(ctx, 0);
    if (rc != ASEP_OK) return bail(rc);
    next = 1;
  }
  rc = set_clock(ctx, 0, next);
  if (rc != ASEP_OK) return bail(rc);
  *out = ctx;
  return ASEP_OK;
}

int asep_sweep(asep_ctx* ctx, uint64_t n_mcs) {
  if (!ctx) return ASEP_ERR_INVALID;
  if (ctx->sweep + n_mcs >= (1ull << 40)) return fail(ctx, ASEP_ERR_INVALID, "sweep index would exceed 2^40");
  uint64_t done = 0;
  while (done < n_mcs) {
    uint64_t n = n_mcs - done;
    const uint32_t cap = sweeps_cap(ctx);
    if (n > cap) n = cap;
    cudaError_t e;
    if (ctx->p.schedule == ASEP_SCHED_DOMAIN && ctx->cluster == kStreamTier) {
      // one sweep per step: both phases, lane changes, the record, the clock
      n = 1;
      e = launch_stream_sweep(domain_desc(ctx, 1), ctx->tiles, ctx->threads, ctx->smem, ctx->d_err,
                              ctx->fault == ASEP_FAULT_COPY_STALL ? 16u : 0u, ctx->stream);
      if (e == cudaSuccess && ctx->next_time < ctx->times.size() && ctx->times[ctx->next_time] == ctx->sweep + 1) {
        const int rc = record_now(ctx, ctx->next_time);
        if (rc != ASEP_OK) return rc;
      }
    } else if (ctx->p.schedule == ASEP_SCHED_DOMAIN && ctx->cluster > 1) {
      e = launch_cluster(domain_desc(ctx, static_cast<uint32_t>(n)), ctx->threads, ctx->smem, ctx->stream);
    } else if (ctx->p.schedule == ASEP_SCHED_SCA && ctx->cluster == kStreamTier) {
      n = 1;  // one sweep per step: both phases, then the record and the clock
      e = launch_sca_stream(domain_desc(ctx, 1), ctx->stream);
      if (e == cudaSuccess && ctx->next_time < ctx->times.size() && ctx->times[ctx->next_time] == ctx->sweep + 1) {
        const int rc = record_now(ctx, ctx->next_time);
        if (rc != ASEP_OK) return rc;
      }
    } else if (ctx->p.schedule == ASEP_SCHED_SCA) {
      e = launch_sca(domain_desc(ctx, static_cast<uint32_t>(n)), ctx->threads, ctx->smem, ctx->stream);
    } else if (ctx->p.schedule == ASEP_SCHED_DOMAIN && ctx->balance && ctx->cluster == 1 && n > ctx->balance) {
      BalanceLaunch b;
      b.chunk = ctx->balance;
      b.chunks = static_cast<uint32_t>((n + ctx->balance - 1) / ctx->balance);
      b.progress = ctx->d_progress;
      b.queue = ctx->d_progress + ctx->blocks;
      b.err = ctx->d_err;
      b.stall = ctx->fault == ASEP_FAULT_BALANCE_STALL ? 1u : 0u;
      e = launch_domain_balanced(domain_desc(ctx, static_cast<uint32_t>(n)), b, ctx->threads, ctx->smem,
                                 ctx->stream);
    } else if (ctx->p.schedule == ASEP_SCHED_DOMAIN) {
      e = launch_domain(domain_desc(ctx, static_cast<uint32_t>(n)), ctx->threads, ctx->smem, ctx->stream);
    } else {
      SerialLaunch a;
      a.geo = geometry(ctx);
      a.count_hops = (ctx->p.model == ASEP_MODEL_TWO_LANE || !(ctx->p.flags & ASEP_FLAG_NO_HOP_COUNTS)) ? 1u : 0u;
      a.state = ctx->d_state;
      a.mask = ctx->d_mask;
      a.rates = rates(ctx);
      a.seed = ctx->p.seed;
      a.n_sweeps = static_cast<uint32_t>(n);
      a.clock = ctx->d_clock;
      a.times = ctx->d_times;
      a.n_times = static_cast<uint32_t>(ctx->times.size());
      a.tab_sh = ctx->d_sh;
      a.tab_sh2 = ctx->d_sh2;
      a.counters = ctx->d_cnt;
      a.ex = extras(ctx);
      e = launch_serial_plan(a, ctx->p.model, ctx->p.dis_kind, ctx->cluster, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sweep kernel launch");
    if ((e = launch_advance(ctx->d_clock, ctx->d_times, static_cast<uint32_t>(ctx->times.size()),
                            static_cast<uint32_t>(n), ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "clock advance");
    // the sweep kernels (streamed tiers: one per phase, plus the lane changes
    // of the streamed domain schedule with turning sites) and the clock
    uint32_t sweep_launches = 1;
    if (ctx->cluster == kStreamTier)
      sweep_launches = (ctx->p.schedule == ASEP_SCHED_DOMAIN &&
                        (ctx->p.dis_kind == ASEP_DIS_TURNING || ctx->p.dis_kind == ASEP_DIS_CROSSING)) ? 3u : 2u;
    ctx->launches += sweep_launches + 1;
    advance_host(ctx, n);
    done += n;
  }
  return ASEP_OK;
}

int asep_reset(asep_ctx* ctx, uint64_t seed, uint64_t init_seed) {
  if (!ctx) return ASEP_ERR_INVALID;
  const int rct = clear_timeout(ctx);  // a new initial state replaces results a timed-out sweep invalidated
  if (rct != ASEP_OK) return rct;
  ctx->p.seed = seed;
  ctx->p.init_seed = init_seed;
  const size_t n_times = std::max<size_t>(1, ctx->times.size());
  const size_t entries = n_times * ctx->S * ctx->planes;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ctx->d_cnt, 0, static_cast<size_t>(ctx->S) * 32, ctx->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->d_sh, 0, entries * 8, ctx->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->d_sh2, 0, entries * 16, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "clear tables");
  const int rcx = clear_extras(ctx);
  if (rcx != ASEP_OK) return rcx;
  InitLaunch il;
  il.geo = geometry(ctx);
  il.state = ctx->d_state;
  il.init_kind = ctx->p.init_kind;
  il.init_seed = init_seed;
  if ((e = launch_init(il, ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "init kernel");
  ++ctx->launches;
  const int rcr = record_reference(ctx);
  if (rcr != ASEP_OK) return rcr;
  ctx->ref_slot = 0;
  uint32_t next = 0;
  if (!ctx->times.empty() && ctx->times[0] == 0) {
    const int rc = record_now(ctx, 0);
    if (rc != ASEP_OK) return rc;
    next = 1;
  }
  return set_clock(ctx, 0, next);
}

int asep_inject_fault(asep_ctx* ctx, uint32_t fault) {
  if (!ctx) return ASEP_ERR_INVALID;
  if (fault > ASEP_FAULT_BALANCE_STALL) return fail(ctx, ASEP_ERR_INVALID, "unknown fault %u", fault);
  ctx->fault = fault;
  return ASEP_OK;
}

int asep_sync(asep_ctx* ctx) {
  if (!ctx) return ASEP_ERR_INVALID;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  if ((ctx->cluster == kStreamTier || ctx->balance) && ctx->d_err && !ctx->err_seen) {
    uint32_t flag = 0;
    if ((e = cudaMemcpy(&flag, ctx->d_err, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(ctx, e, "read the error flag");
    if (flag) {
      ctx->err_seen = 1;
      return fail(ctx, ASEP_ERR_TIMEOUT, "a bounded device-side wait ran out (a streamed tile's bulk copy, or a "
                  "balanced launch's previous chunk); results are invalid");
    }
  }
  return ctx->err_seen ? fail(ctx, ASEP_ERR_TIMEOUT, "a bounded device-side wait ran out earlier") : ASEP_OK;
}

int asep_width(asep_ctx* ctx, int64_t* sum_h, uint64_t* sum_h2, double* w2, size_t n_entries) {
  if (!ctx) return ASEP_ERR_INVALID;
  const size_t need = static_cast<size_t>(ctx->next_time) * ctx->S * ctx->planes;
  if (n_entries < need) return fail(ctx, ASEP_ERR_INVALID, "n_entries = %zu < %zu recorded entries", n_entries, need);
  int rc = asep_sync(ctx);
  if (rc != ASEP_OK) return rc;
  if (need == 0) return ASEP_OK;
  std::vector<int64_t> sh(need);
  std::vector<uint64_t> sh2(2 * need);
  cudaError_t e;
  if ((e = cudaMemcpy(sh.data(), ctx->d_sh, need * 8, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(sh2.data(), ctx->d_sh2, need * 16, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(ctx, e, "copy height table");
  if (sum_h) std::memcpy(sum_h, sh.data(), need * 8);
  if (sum_h2) std::memcpy(sum_h2, sh2.data(), need * 16);
  if (w2) {
    const __int128 L = static_cast<__int128>(ctx->L);
    for (size_t i = 0; i < need; ++i) {
      const unsigned __int128 s2 = (static_cast<unsigned __int128>(sh2[2 * i + 1]) << 64) | sh2[2 * i];
      const __int128 s1 = sh[i];
      const __int128 num = L * static_cast<__int128>(s2) - s1 * s1;  // >= 0, < 2^110
      // num / L^2 with one rounding: split into integer quotient and remainder
      const __int128 L2 = L * L;
      const __int128 qt = num / L2, rm = num % L2;
      w2[i] = static_cast<double>(qt) + static_cast<double>(rm) / static_cast<double>(L2);
    }
  }
  return ASEP_OK;
}

int asep_state(asep_ctx* ctx, uint32_t* words, size_t n_words, uint64_t* sweep_out) {
  if (!ctx) return ASEP_ERR_INVALID;
  const size_t need = static_cast<size_t>(ctx->S) * ctx->planes * ctx->W;
  if (words && n_words < need) return fail(ctx, ASEP_ERR_INVALID, "n_words = %zu < %zu", n_words, need);
  int rc = asep_sync(ctx);
  if (rc != ASEP_OK) return rc;
  if (words) {
    const cudaError_t e = cudaMemcpy(words, ctx->d_state, need * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy state");
  }
  if (sweep_out) *sweep_out = ctx->sweep;
  return ASEP_OK;
}

int asep_load_state(asep_ctx* ctx, const uint32_t* words, size_t n_words, uint64_t sweep) {
  if (!ctx || !words) return ASEP_ERR_INVALID;
  const size_t need = static_cast<size_t>(ctx->S) * ctx->planes * ctx->W;
  if (n_words < need) return fail(ctx, ASEP_ERR_INVALID, "n_words = %zu < %zu", n_words, need);
  if (sweep >= (1ull << 40)) return fail(ctx, ASEP_ERR_INVALID, "sweep index >= 2^40");
  int rc = clear_timeout(ctx);  // the loaded state replaces results a timed-out sweep invalidated
  if (rc != ASEP_OK) return rc;
  const cudaError_t e = cudaMemcpy(ctx->d_state, words, need * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "load state");
  if ((rc = record_reference(ctx)) != ASEP_OK) return rc;
  uint32_t i = 0;
  while (i < ctx->times.size() && ctx->times[i] <= sweep) ++i;
  ctx->ref_slot = i;
  rc = set_clock(ctx, sweep, i);
  if (rc != ASEP_OK) return rc;
  return asep_sync(ctx);
}

int asep_counters(asep_ctx* ctx, uint64_t* counters, size_t n) {
  if (!ctx || !counters) return ASEP_ERR_INVALID;
  const size_t need = static_cast<size_t>(ctx->S) * 4;
  if (n < need) return fail(ctx, ASEP_ERR_INVALID, "n = %zu < %zu", n, need);
  int rc = asep_sync(ctx);
  if (rc != ASEP_OK) return rc;
  const cudaError_t e = cudaMemcpy(counters, ctx->d_cnt, need * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy counters");
  return ASEP_OK;
}

int asep_disorder(asep_ctx* ctx, uint32_t* words, size_t n_words) {
  if (!ctx || !words) return ASEP_ERR_INVALID;
  const size_t need = static_cast<size_t>(ctx->R) * dis_planes(ctx->p.dis_kind) * ctx->W;
  if (n_words < need) return fail(ctx, ASEP_ERR_INVALID, "n_words = %zu < %zu", n_words, need);
  int rc = asep_sync(ctx);
  if (rc != ASEP_OK) return rc;
  if (need == 0) return ASEP_OK;
  const cudaError_t e = cudaMemcpy(words, ctx->d_mask, need * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy disorder");
  return ASEP_OK;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------

}  // extern "C"

struct asep_batch {
  cudaStream_t stream = nullptr;
  uint32_t max_jobs = 0, max_items = 0;
  uint32_t threads_req = 0, ctas_per_sm_req = 0;
  DomainLaunch* d_jobs = nullptr;
  uint32_t* d_items = nullptr;
  uint32_t* d_queue = nullptr;
  DomainLaunch* h_jobs = nullptr;  // pinned staging
  uint32_t* h_items = nullptr;
  cudaEvent_t staged = nullptr;  // the staging buffers may be rewritten once this event is done
  cudaEvent_t order = nullptr;   // cross-stream ordering with the contexts
  cudaStream_t cap_stream = nullptr;  // capture stream (the legacy default stream cannot be captured)
  cudaStream_t aux_stream = nullptr;  // cluster-tier launches run here, beside the persistent kernel
  cudaEvent_t fork = nullptr, join = nullptr;
  // graph cache: one captured step
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> graph_key;
  std::string err;
};

namespace {

int bfail(asep_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  else g_create_error = buf;
  return code;
}

// Build descriptors and the largest-first item list for one step, stage and
// upload them, and compute the launch shape.  n[i] <= the context's cap.
int batch_prepare(asep_batch* b, asep_ctx* const* ctxs, const uint32_t* n, uint32_t nj, uint32_t* n_items_out,
                  uint32_t* threads_out, uint32_t* ctas_out, size_t* smem_out) {
  uint32_t threads = 32;
  for (uint32_t j = 0; j < nj; ++j)
    if (ctxs[j]->cluster == 1) threads = std::max(threads, ctxs[j]->threads);
  if (b->threads_req) {
    if (b->threads_req < threads || (b->threads_req & 31) || b->threads_req > 1024)
      return bfail(b, ASEP_ERR_INVALID, "threads %u: must be a multiple of 32 in [%u, 1024]", b->threads_req, threads);
    threads = b->threads_req;
  }
  size_t smem = 0;
  struct It {
    uint64_t cost;
    uint32_t code;
  };
  std::vector<It> items;
  cudaError_t e = cudaEventSynchronize(b->staged);
  if (e != cudaSuccess) return bfail(b, ASEP_ERR_CUDA, "staging event: %s", cudaGetErrorString(e));
  for (uint32_t j = 0; j < nj; ++j) {
    const asep_ctx* c = ctxs[j];
    b->h_jobs[j] = domain_desc(c, n[j]);
    if (c->cluster > 1) continue;  // cluster-tier contexts get their own cluster launch
    smem = std::max(smem, domain_smem_bytes(c->p.model, c->p.dis_kind, c->R2, c->Cp,
                                            static_cast<uint32_t>(c->ptab.size()), threads));
    if (n[j] == 0) continue;
    const uint64_t cost = static_cast<uint64_t>(n[j]) * c->spc * c->L * c->planes;
    for (uint32_t g = 0; g < c->blocks; ++g) items.push_back({cost, (j << kItemGroupBits) | g});
  }
  if (items.size() > b->max_items)
    return bfail(b, ASEP_ERR_INVALID, "%zu queue items exceed the batch's max_items %u", items.size(), b->max_items);
  std::stable_sort(items.begin(), items.end(), [](const It& x, const It& y) { return x.cost > y.cost; });
  for (size_t i = 0; i < items.size(); ++i) b->h_items[i] = items[i].code;
  // the batch kernel's own static shared memory (item index, descriptor) shares the 227 KB opt-in
  if (smem + sizeof(DomainLaunch) + 64 > 227 * 1024)
    return bfail(b, ASEP_ERR_INVALID, "batch needs %zu bytes of shared memory", smem);
  int per_sm = batch_ctas_per_sm(threads, smem);
  if (per_sm <= 0) return bfail(b, ASEP_ERR_INVALID, "batch kernel does not fit (%u threads, %zu B)", threads, smem);
  if (b->ctas_per_sm_req) per_sm = std::min<int>(per_sm, static_cast<int>(b->ctas_per_sm_req));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t ctas = static_cast<uint32_t>(std::max<size_t>(1, std::min<size_t>(items.size(),
                                                                  static_cast<size_t>(per_sm) * sms)));
  if ((e = cudaMemcpyAsync(b->d_jobs, b->h_jobs, nj * sizeof(DomainLaunch), cudaMemcpyHostToDevice, b->stream)) !=
          cudaSuccess ||
      (items.size() && (e = cudaMemcpyAsync(b->d_items, b->h_items, items.size() * 4, cudaMemcpyHostToDevice,
                                            b->stream)) != cudaSuccess) ||
      (e = cudaEventRecord(b->staged, b->stream)) != cudaSuccess)
    return bfail(b, ASEP_ERR_CUDA, "stage batch: %s", cudaGetErrorString(e));
  *n_items_out = static_cast<uint32_t>(items.size());
  *threads_out = threads;
  *ctas_out = ctas;
  *smem_out = smem;
  return ASEP_OK;
}

int batch_check(asep_batch* b, asep_ctx* const* ctxs, const uint64_t* n_mcs, uint32_t n) {
  if (!b) return ASEP_ERR_INVALID;
  if (n == 0) return ASEP_OK;
  if (!ctxs || !n_mcs) return bfail(b, ASEP_ERR_INVALID, "ctxs or n_mcs is NULL");
  if (n > b->max_jobs) return bfail(b, ASEP_ERR_INVALID, "%u contexts exceed max_jobs %u", n, b->max_jobs);
  if (n > kItemMaxJobs) return bfail(b, ASEP_ERR_INVALID, "at most %u contexts per batch", kItemMaxJobs);
  for (uint32_t j = 0; j < n; ++j) {
    if (!ctxs[j]) return bfail(b, ASEP_ERR_INVALID, "context %u is NULL", j);
    if (ctxs[j]->p.schedule != ASEP_SCHED_DOMAIN)
      return bfail(b, ASEP_ERR_INVALID, "context %u: only the domain schedule runs in a batch", j);
    if (ctxs[j]->cluster == kStreamTier)
      return bfail(b, ASEP_ERR_INVALID, "context %u streams its lattice from global memory; use asep_sweep", j);
    if (ctxs[j]->sweep + n_mcs[j] >= (1ull << 40)) return bfail(b, ASEP_ERR_INVALID, "context %u: sweep >= 2^40", j);
    if (ctxs[j]->blocks > kItemMaxGroups)
      return bfail(b, ASEP_ERR_INVALID, "context %u: more than %u sample groups; use asep_sweep", j, kItemMaxGroups);
    for (uint32_t k = 0; k < j; ++k)
      if (ctxs[k] == ctxs[j]) return bfail(b, ASEP_ERR_INVALID, "context %u appears twice", j);
  }
  return ASEP_OK;
}

// Streams of the contexts of a step, each once (contexts often share one).
bool seen_before(asep_ctx* const* ctxs, uint32_t j) {
  for (uint32_t k = j; k-- > 0 && j - k <= 8;)
    if (ctxs[k]->stream == ctxs[j]->stream) return true;
  return false;
}

int order_in(asep_batch* b, asep_ctx* const* ctxs, uint32_t n) {
  for (uint32_t j = 0; j < n; ++j) {
    if (ctxs[j]->stream == b->stream || seen_before(ctxs, j)) continue;
    cudaError_t e;
    if ((e = cudaEventRecord(b->order, ctxs[j]->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->stream, b->order, 0)) != cudaSuccess)
      return bfail(b, ASEP_ERR_CUDA, "order: %s", cudaGetErrorString(e));
  }
  return ASEP_OK;
}

int order_out(asep_batch* b, asep_ctx* const* ctxs, uint32_t n) {
  cudaError_t e = cudaEventRecord(b->order, b->stream);
  if (e != cudaSuccess) return bfail(b, ASEP_ERR_CUDA, "order: %s", cudaGetErrorString(e));
  for (uint32_t j = 0; j < n; ++j) {
    if (ctxs[j]->stream == b->stream || seen_before(ctxs, j)) continue;
    if ((e = cudaStreamWaitEvent(ctxs[j]->stream, b->order, 0)) != cudaSuccess)
      return bfail(b, ASEP_ERR_CUDA, "order: %s", cudaGetErrorString(e));
  }
  return ASEP_OK;
}

int batch_step_enqueue(asep_batch* b, asep_ctx* const* ctxs, uint32_t nj, uint32_t n_items, uint32_t threads,
                       uint32_t ctas, size_t smem, cudaStream_t st) {
  cudaError_t e;
  // contexts of the cluster tier run as their own cluster launches on an
  // auxiliary stream forked from `st`, beside the persistent kernel, and are
  // joined back before the clocks advance
  bool forked = false;
  for (uint32_t j = 0; j < nj; ++j) {
    const DomainLaunch& d = b->h_jobs[j];
    if (ctxs[j]->cluster == 1 || d.n_sweeps == 0) continue;
    if (!forked) {
      if ((e = cudaEventRecord(b->fork, st)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(b->aux_stream, b->fork, 0)) != cudaSuccess)
        return bfail(b, ASEP_ERR_CUDA, "fork: %s", cudaGetErrorString(e));
      forked = true;
    }
    if ((e = launch_cluster(d, ctxs[j]->threads, ctxs[j]->smem, b->aux_stream)) != cudaSuccess)
      return bfail(b, ASEP_ERR_CUDA, "cluster kernel of context %u: %s", j, cudaGetErrorString(e));
  }
  if (n_items && (e = launch_batch(b->d_jobs, b->d_items, n_items, b->d_queue, threads, ctas, smem, st)) !=
                     cudaSuccess)
    return bfail(b, ASEP_ERR_CUDA, "batch kernel: %s", cudaGetErrorString(e));
  if (forked && ((e = cudaEventRecord(b->join, b->aux_stream)) != cudaSuccess ||
                 (e = cudaStreamWaitEvent(st, b->join, 0)) != cudaSuccess))
    return bfail(b, ASEP_ERR_CUDA, "join: %s", cudaGetErrorString(e));
  if ((e = launch_advance_batch(b->d_jobs, nj, st)) != cudaSuccess)
    return bfail(b, ASEP_ERR_CUDA, "batch clock advance: %s", cudaGetErrorString(e));
  return ASEP_OK;
}

}  // namespace

extern "C" {

int asep_batch_create(void* stream, uint32_t max_jobs, uint32_t max_items, asep_batch** out) {
  if (!out) return bfail(nullptr, ASEP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (max_jobs == 0 || max_jobs > kItemMaxJobs || max_items == 0 || max_items > (1u << 24))
    return bfail(nullptr, ASEP_ERR_INVALID, "max_jobs in [1, %u], max_items in [1, 2^24]", kItemMaxJobs);
  asep_batch* b = new (std::nothrow) asep_batch();
  if (!b) return bfail(nullptr, ASEP_ERR_NOMEM, "host allocation failed");
  b->stream = static_cast<cudaStream_t>(stream);
  b->max_jobs = max_jobs;
  b->max_items = max_items;
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_jobs, max_jobs * sizeof(DomainLaunch))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_items, static_cast<size_t>(max_items) * 4)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_queue, 16)) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_jobs, max_jobs * sizeof(DomainLaunch))) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_items, static_cast<size_t>(max_items) * 4)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->order, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->aux_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming)) != cudaSuccess) {
    const int rc = bfail(nullptr, e == cudaErrorMemoryAllocation ? ASEP_ERR_NOMEM : ASEP_ERR_CUDA,
                         "batch workspace: %s", cudaGetErrorString(e));
    (void)cudaGetLastError();
    asep_batch_destroy(b);
    return rc;
  }
  *out = b;
  return ASEP_OK;
}

int asep_batch_set_launch(asep_batch* b, uint32_t threads, uint32_t ctas_per_sm) {
  if (!b) return ASEP_ERR_INVALID;
  if (threads && ((threads & 31) || threads > 1024)) return bfail(b, ASEP_ERR_INVALID, "threads %u", threads);
  b->threads_req = threads;
  b->ctas_per_sm_req = ctas_per_sm;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_key.clear();
  }
  return ASEP_OK;
}

int asep_batch_sweep(asep_batch* b, asep_ctx* const* ctxs, const uint64_t* n_mcs, uint32_t n) {
  int rc = batch_check(b, ctxs, n_mcs, n);
  if (rc != ASEP_OK || n == 0) return rc;
  if ((rc = order_in(b, ctxs, n)) != ASEP_OK) return rc;
  std::vector<uint64_t> left(n_mcs, n_mcs + n);
  std::vector<uint32_t> step(n);
  for (;;) {
    bool any = false;
    for (uint32_t j = 0; j < n; ++j) {
      step[j] = static_cast<uint32_t>(std::min<uint64_t>(left[j], sweeps_cap(ctxs[j])));
      any = any || step[j] > 0;
    }
    if (!any) break;
    uint32_t n_items, threads, ctas;
    size_t smem;
    if ((rc = batch_prepare(b, ctxs, step.data(), n, &n_items, &threads, &ctas, &smem)) != ASEP_OK) return rc;
    if ((rc = batch_step_enqueue(b, ctxs, n, n_items, threads, ctas, smem, b->stream)) != ASEP_OK) return rc;
    for (uint32_t j = 0; j < n; ++j) {
      left[j] -= step[j];
      advance_host(ctxs[j], step[j]);
      ctxs[j]->launches += 2;
    }
  }
  return order_out(b, ctxs, n);
}

int asep_batch_graph(asep_batch* b, asep_ctx* const* ctxs, const uint64_t* n_mcs, uint32_t n, uint32_t replays) {
  int rc = batch_check(b, ctxs, n_mcs, n);
  if (rc != ASEP_OK || n == 0 || replays == 0) return rc;
  std::vector<uint32_t> step(n);
  std::vector<uintptr_t> key;
  for (uint32_t j = 0; j < n; ++j) {
    if (n_mcs[j] > sweeps_cap(ctxs[j]))
      return bfail(b, ASEP_ERR_INVALID, "context %u: a graph step is at most one launch of sweeps", j);
    step[j] = static_cast<uint32_t>(n_mcs[j]);
    key.push_back(reinterpret_cast<uintptr_t>(ctxs[j]));
    key.push_back(step[j]);
  }
  if ((rc = order_in(b, ctxs, n)) != ASEP_OK) return rc;
  cudaError_t e;
  if (!b->exec || key != b->graph_key) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    uint32_t n_items, threads, ctas;
    size_t smem;
    // descriptors and items are uploaded once, outside the graph
    if ((rc = batch_prepare(b, ctxs, step.data(), n, &n_items, &threads, &ctas, &smem)) != ASEP_OK) return rc;
    // kernel attributes are set before capture begins
    if (batch_ctas_per_sm(threads, smem) <= 0) return bfail(b, ASEP_ERR_INVALID, "batch kernel does not fit");
    // capture on the batch's own stream (nothing runs during capture), launch on b->stream
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
      return bfail(b, ASEP_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    const int rc_enq = batch_step_enqueue(b, ctxs, n, n_items, threads, ctas, smem, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (rc_enq != ASEP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc_enq;
    }
    if (e != cudaSuccess) return bfail(b, ASEP_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return bfail(b, ASEP_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    b->graph_key = key;
  }
  for (uint32_t r = 0; r < replays; ++r) {
    if ((e = cudaGraphLaunch(b->exec, b->stream)) != cudaSuccess)
      return bfail(b, ASEP_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    for (uint32_t j = 0; j < n; ++j) {
      advance_host(ctxs[j], step[j]);
      ctxs[j]->launches += 2;
    }
  }
  return order_out(b, ctxs, n);
}

int asep_batch_destroy(asep_batch* b) {
  if (!b) return ASEP_OK;
  cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->staged) cudaEventDestroy(b->staged);
  if (b->order) cudaEventDestroy(b->order);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->aux_stream) {
    cudaStreamSynchronize(b->aux_stream);
    cudaStreamDestroy(b->aux_stream);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->d_jobs) cudaFree(b->d_jobs);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_queue) cudaFree(b->d_queue);
  if (b->h_jobs) cudaFreeHost(b->h_jobs);
  if (b->h_items) cudaFreeHost(b->h_items);
  delete b;
  return ASEP_OK;
}

const char* asep_batch_last_error(const asep_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

int asep_set_plan(asep_ctx* ctx, uint32_t cluster, uint32_t samples_per_group) {
  if (!ctx) return ASEP_ERR_INVALID;
  if (ctx->p.schedule == ASEP_SCHED_SCA) {
    if (cluster > 1 && cluster != kStreamTier)
      return fail(ctx, ASEP_ERR_INVALID, "SCA plans: cluster 0 (choose), 1 (resident) or 32 (streamed)");
    if (samples_per_group) return fail(ctx, ASEP_ERR_INVALID, "samples_per_group applies to the domain schedule");
    const asep_ctx saved = *ctx;
    const int rc = plan_sca(ctx, cluster);
    if (rc != ASEP_OK) {
      const std::string msg = ctx->err;
      ctx->cluster = saved.cluster;
      ctx->threads = saved.threads;
      ctx->smem = saved.smem;
      ctx->blocks = saved.blocks;
      ctx->err = msg;
    }
    return rc;
  }
  if (ctx->p.schedule == ASEP_SCHED_SERIAL) {
    if (cluster > kSerialWarp || samples_per_group)
      return fail(ctx, ASEP_ERR_INVALID, "serial plans: cluster 0 (choose), 1 (a CTA per sample, dependency rounds) "
                  "or 2 (a warp per sample); samples_per_group 0");
    const asep_ctx saved = *ctx;
    const int rc = plan_serial(ctx, cluster);
    if (rc != ASEP_OK) {
      const std::string msg = ctx->err;
      ctx->cluster = saved.cluster;
      ctx->spc = saved.spc;
      ctx->threads = saved.threads;
      ctx->smem = saved.smem;
      ctx->blocks = saved.blocks;
      ctx->err = msg;
    }
    return rc;
  }
  if (ctx->p.schedule != ASEP_SCHED_DOMAIN)
    return fail(ctx, ASEP_ERR_INVALID, "plans apply to the domain, SCA and serial schedules");
  if (cluster != kStreamTier && (cluster > 16 || (cluster > 1 && (cluster & (cluster - 1)))))
    return fail(ctx, ASEP_ERR_INVALID, "cluster must be 0, 1, 2, 4, 8, 16 or 32 (streamed)");
  if (cluster == kStreamTier) {
    if (samples_per_group % 32 || samples_per_group > 1024)
      return fail(ctx, ASEP_ERR_INVALID, "streamed tile width must be 0 (automatic) or a multiple of 32 up to 1024");
  } else {
    if (samples_per_group && cluster > 1)
      return fail(ctx, ASEP_ERR_INVALID, "samples_per_group applies to the resident plan (cluster 0 or 1)");
    if (samples_per_group > ctx->S) return fail(ctx, ASEP_ERR_INVALID, "samples_per_group exceeds the samples");
  }
  const asep_ctx saved = *ctx;  // restore the previous plan if the new one does not fit
  const int rc = plan_domain(ctx, cluster, samples_per_group);
  if (rc != ASEP_OK) {
    const std::string msg = ctx->err;
    ctx->cluster = saved.cluster;
    ctx->Gc = saved.Gc;
    ctx->spc = saved.spc;
    ctx->C = saved.C;
    ctx->Cp = saved.Cp;
    ctx->threads = saved.threads;
    ctx->smem = saved.smem;
    ctx->blocks = saved.blocks;
    ctx->tiles = saved.tiles;
    ctx->max_sweeps_per_launch = saved.max_sweeps_per_launch;
    ctx->err = msg;
  }
  return rc;
}

int asep_set_launch_sweeps(asep_ctx* ctx, uint32_t max_sweeps) {
  if (!ctx) return ASEP_ERR_INVALID;
  ctx->launch_sweeps = max_sweeps;
  return ASEP_OK;
}

int asep_set_balance(asep_ctx* ctx, uint32_t chunk_sweeps) {
  if (!ctx) return ASEP_ERR_INVALID;
  if (chunk_sweeps && ctx->p.schedule != ASEP_SCHED_DOMAIN)
    return fail(ctx, ASEP_ERR_INVALID, "balanced launches apply to the domain schedule");
  if (chunk_sweeps > kMaxBalanceChunk)
    return fail(ctx, ASEP_ERR_INVALID, "chunk of %u sweeps exceeds %u", chunk_sweeps, kMaxBalanceChunk);
  if (chunk_sweeps && !ctx->d_progress) {
    ctx->d_progress = static_cast<uint32_t*>(dev_alloc(ctx, (static_cast<size_t>(ctx->S) + 1) * sizeof(uint32_t)));
    if (!ctx->d_progress) return fail(ctx, ASEP_ERR_NOMEM, "device allocation of the chunk flags failed");
  }
  ctx->balance = chunk_sweeps;
  return ASEP_OK;
}

int asep_currents(asep_ctx* ctx, int64_t* out, size_t n) {
  if (!ctx || !out) return ASEP_ERR_INVALID;
  const size_t need = static_cast<size_t>(ctx->next_time) * ctx->S * 4;
  if (n < need) return fail(ctx, ASEP_ERR_INVALID, "n = %zu < %zu", n, need);
  return copy_out(ctx, out, ctx->d_tab_cnt, need * 8, "copy currents");
}

int asep_profile(asep_ctx* ctx, uint32_t* out, size_t n) {
  if (!ctx || !out) return ASEP_ERR_INVALID;
  if (!ctx->d_profile) return fail(ctx, ASEP_ERR_STATE, "the context was created without ASEP_FLAG_PROFILE");
  const size_t need = static_cast<size_t>(ctx->S) * ctx->planes * ctx->W;
  if (n < need) return fail(ctx, ASEP_ERR_INVALID, "n = %zu < %zu", n, need);
  return copy_out(ctx, out, ctx->d_profile, need * 4, "copy profile");
}

int asep_autocorr(asep_ctx* ctx, int64_t* out, size_t n) {
  if (!ctx || !out) return ASEP_ERR_INVALID;
  if (!ctx->d_tab_ac) return fail(ctx, ASEP_ERR_STATE, "the context was created without ASEP_FLAG_AUTOCORR");
  const size_t need = static_cast<size_t>(ctx->next_time) * ctx->S * ctx->planes;
  if (n < need) return fail(ctx, ASEP_ERR_INVALID, "n = %zu < %zu", n, need);
  return copy_out(ctx, out, ctx->d_tab_ac, need * 8, "copy autocorrelation");
}

int asep_height_offset(asep_ctx* ctx, int64_t* out, size_t n) {
  if (!ctx || !out) return ASEP_ERR_INVALID;
  if (ctx->p.model != ASEP_MODEL_RING || (ctx->p.flags & ASEP_FLAG_NO_HOP_COUNTS))
    return fail(ctx, ASEP_ERR_STATE, "the height offset needs the ring model with hop counting on");
  const size_t S = ctx->S, nr = ctx->next_time;
  if (n < nr * S) return fail(ctx, ASEP_ERR_INVALID, "n = %zu < %zu", n, nr * S);
  std::vector<int64_t> sh(nr * S), cnt(nr * S * 4), ref(S), refcnt(S * 4);
  int rc;
  if ((rc = copy_out(ctx, sh.data(), ctx->d_sh, sh.size() * 8, "copy heights")) != ASEP_OK ||
      (rc = copy_out(ctx, cnt.data(), ctx->d_tab_cnt, cnt.size() * 8, "copy counters")) != ASEP_OK ||
      (rc = copy_out(ctx, ref.data(), ctx->d_href, ref.size() * 8, "copy reference heights")) != ASEP_OK ||
      (rc = copy_out(ctx, refcnt.data(), ctx->d_hrefcnt, refcnt.size() * 8, "copy reference counters")) != ASEP_OK)
    return rc;
  const int64_t L = static_cast<int64_t>(ctx->L);
  for (size_t t = 0; t < nr; ++t) {
    for (size_t s = 0; s < S; ++s) {
      if (t < ctx->ref_slot) {  // recorded before the reference lattice
        out[t * S + s] = 0;
        continue;
      }
      const int64_t net = (cnt[(t * S + s) * 4] - cnt[(t * S + s) * 4 + 1]) - (refcnt[s * 4] - refcnt[s * 4 + 1]);
      const int64_t num = ref[s] - sh[t * S + s] - 2 * net;
      if (num % L != 0)
        return fail(ctx, ASEP_ERR_STATE, "record %zu sample %zu: heights and hop counters disagree", t, s);
      out[t * S + s] = num / L;
    }
  }
  return ASEP_OK;
}

int asep_get_info(const asep_ctx* ctx, asep_info* info) {
  if (!ctx || !info) return ASEP_ERR_INVALID;
  fill_info(ctx, info);
  return ASEP_OK;
}

int asep_destroy(asep_ctx* ctx) {
  if (!ctx) return ASEP_OK;
  release(ctx);
  delete ctx;
  return ASEP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch sweep without allocation
// ---------------------------------------------------------------------------
//
// Some callers cannot allocate device memory at the moment they want to run
// work: a host application whose device memory is owned by another allocator
// or pool that refuses outside requests, code that must not grow its memory
// footprint after start-up, or a thread that may not enter cudaMalloc
// (which can synchronise the device).  For them the
// batch sweep below keeps its work queue -- context descriptors, the item
// list and the queue counter -- in one fixed static device array instead of
// a batch object's workspace.  The array belongs to the library: every GPU
// that loads libasep.so holds it until the process exits.

namespace {

constexpr uint32_t kStaticMaxJobs = 64;      // contexts per call
constexpr uint32_t kStaticMaxItems = 16384;  // queue items (sample groups) per step
constexpr size_t kStaticJobsBytes = (kStaticMaxJobs * sizeof(DomainLaunch) + 255) / 256 * 256;
constexpr size_t kStaticItemsBytes = kStaticMaxItems * sizeof(uint32_t);
constexpr size_t kStaticBytes = kStaticJobsBytes + kStaticItemsBytes + 256;  // + the queue counter

// In host code this name is only a stand-in for the device array; kernels get
// its device address from cudaGetSymbolAddress (see static_scratch()).
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;  // held for a whole call: serialises the host side of all calls
void* g_static_ptr[kMaxDevices] = {};
// host staging for the uploads (static, so no stack or heap use)
DomainLaunch g_static_jobs[kStaticMaxJobs];
uint32_t g_static_items[kStaticMaxItems];

// Device address of the static array on the current device, looked up once
// per device (with that device current) and cached.  Caller holds g_static_mu.
int static_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, ASEP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, ASEP_ERR_INVALID, "device %d out of range", dev);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return fail(nullptr, ASEP_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    }
    g_static_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_static_ptr[dev]);
  return ASEP_OK;
}

}  // namespace

extern "C" {

int asep_batch_sweep_static(asep_ctx* const* ctxs, const uint64_t* n_mcs, uint32_t n, void* stream) {
  if (n > 0 && (!ctxs || !n_mcs)) return fail(nullptr, ASEP_ERR_INVALID, "ctxs or n_mcs is NULL");
  if (n > kStaticMaxJobs)
    return fail(nullptr, ASEP_ERR_INVALID, "%u contexts exceed the static batch limit of %u", n, kStaticMaxJobs);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (uint32_t j = 0; j < n; ++j) {
    const asep_ctx* c = ctxs[j];
    if (!c) return fail(nullptr, ASEP_ERR_INVALID, "context %u is NULL", j);
    if (c->p.schedule != ASEP_SCHED_DOMAIN)
      return fail(nullptr, ASEP_ERR_INVALID, "context %u: only the domain schedule runs in a batch", j);
    if (c->stream != st) return fail(nullptr, ASEP_ERR_INVALID, "context %u does not use the call's stream", j);
    if (c->cluster > 1)
      return fail(nullptr, ASEP_ERR_INVALID, "context %u is spread over a CTA cluster; use asep_batch_sweep", j);
    if (c->sweep + n_mcs[j] >= (1ull << 40)) return fail(nullptr, ASEP_ERR_INVALID, "context %u: sweep >= 2^40", j);
    for (uint32_t k = 0; k < j; ++k)
      if (ctxs[k] == c) return fail(nullptr, ASEP_ERR_INVALID, "context %u appears twice", j);
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  unsigned char* scratch = nullptr;
  int rc = static_scratch(&scratch);
  if (rc != ASEP_OK) return rc;
  DomainLaunch* d_jobs = reinterpret_cast<DomainLaunch*>(scratch);
  uint32_t* d_items = reinterpret_cast<uint32_t*>(scratch + kStaticJobsBytes);
  uint32_t* d_queue = reinterpret_cast<uint32_t*>(scratch + kStaticJobsBytes + kStaticItemsBytes);
  if (n == 0) {
    // start-up call: the array's address is known now; load the batch kernels
    // and size their local memory with empty launches
    const cudaError_t e = warm_batch_kernels(d_queue, st);
    if (e != cudaSuccess) return fail(nullptr, ASEP_ERR_CUDA, "static batch warm-up: %s", cudaGetErrorString(e));
    return ASEP_OK;
  }

  DomainLaunch* jobs = g_static_jobs;
  uint32_t* items = g_static_items;
  uint32_t order[kStaticMaxJobs];
  uint64_t left[kStaticMaxJobs];
  for (uint32_t j = 0; j < n; ++j) left[j] = n_mcs[j];
  for (;;) {
    uint32_t threads = 32;
    size_t smem = 0;
    bool any = false;
    uint64_t cost[kStaticMaxJobs];
    for (uint32_t j = 0; j < n; ++j) {
      const asep_ctx* c = ctxs[j];
      const uint32_t step = static_cast<uint32_t>(std::min<uint64_t>(left[j], sweeps_cap(c)));
      jobs[j] = domain_desc(c, step);
      threads = std::max(threads, c->threads);
      cost[j] = static_cast<uint64_t>(step) * c->spc * c->L * c->planes;
      order[j] = j;
      any = any || step > 0;
    }
    if (!any) break;
    for (uint32_t j = 0; j < n; ++j) {
      const asep_ctx* c = ctxs[j];
      smem = std::max(smem, domain_smem_bytes(c->p.model, c->p.dis_kind, c->R2, c->Cp,
                                              static_cast<uint32_t>(c->ptab.size()), threads));
    }
    if (smem + sizeof(DomainLaunch) + 64 > 227 * 1024)
      return fail(nullptr, ASEP_ERR_INVALID, "batch needs %zu bytes of shared memory", smem);
    // largest first: contexts by cost per item, each context's groups in order
    std::stable_sort(order, order + n, [&](uint32_t x, uint32_t y) { return cost[x] > cost[y]; });
    uint32_t n_items = 0;
    for (uint32_t k = 0; k < n; ++k) {
      const uint32_t j = order[k];
      if (jobs[j].n_sweeps == 0) continue;
      if (ctxs[j]->blocks > kItemMaxGroups || n_items + ctxs[j]->blocks > kStaticMaxItems)
        return fail(nullptr, ASEP_ERR_INVALID, "more than %u sample groups exceed the static batch limit",
                    kStaticMaxItems);
      for (uint32_t g = 0; g < ctxs[j]->blocks; ++g) items[n_items++] = (j << kItemGroupBits) | g;
    }
    int per_sm = batch_ctas_per_sm(threads, smem);
    if (per_sm <= 0) return fail(nullptr, ASEP_ERR_INVALID, "batch kernel does not fit (%u threads)", threads);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t ctas = std::max<uint32_t>(1, std::min<uint32_t>(n_items, static_cast<uint32_t>(per_sm * sms)));
    // pageable copies: they return once the host buffers have been read, and
    // reach the device in stream order after the previous step's kernels
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_jobs, jobs, n * sizeof(DomainLaunch), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (n_items && (e = cudaMemcpyAsync(d_items, items, n_items * sizeof(uint32_t), cudaMemcpyHostToDevice, st)) !=
                        cudaSuccess))
      return fail(nullptr, ASEP_ERR_CUDA, "static batch upload: %s", cudaGetErrorString(e));
    if (n_items && (e = launch_batch(d_jobs, d_items, n_items, d_queue, threads, ctas, smem, st)) != cudaSuccess)
      return fail(nullptr, ASEP_ERR_CUDA, "static batch kernel: %s", cudaGetErrorString(e));
    if ((e = launch_advance_batch(d_jobs, n, st)) != cudaSuccess)
      return fail(nullptr, ASEP_ERR_CUDA, "static batch clock advance: %s", cudaGetErrorString(e));
    for (uint32_t j = 0; j < n; ++j) {
      left[j] -= jobs[j].n_sweeps;
      advance_host(ctxs[j], jobs[j].n_sweeps);
      ctxs[j]->launches += 2;
    }
  }
  return ASEP_OK;
}

}  // extern "C"

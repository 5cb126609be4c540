// asep_internal.h -- launch descriptors shared by the host runtime
// (asep_api.cu) and the kernels (asep_kernels.cu).  Not installed.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace asep {

// Philox counter tags (ctr1 bits 8..11).
constexpr uint32_t kTagInit = 1;  // Bernoulli(1/2) initial filling
constexpr uint32_t kTagDis = 2;   // quenched class / turning-site bit
constexpr uint32_t kTagOff = 3;   // per-sweep domain offset
constexpr uint32_t kTagDom = 4;   // per-domain attempt stream
constexpr uint32_t kTagTurn = 5;  // per-site lane-change draw
constexpr uint32_t kTagSer = 6;   // serial-schedule stream
constexpr uint32_t kTagSca = 7;   // two-sub-lattice SCA: random planes of four 32-bond groups
constexpr uint32_t kTagScaTurn = 8;  // two-lane SCA: one word per lane-change candidate site

constexpr uint32_t kAcceptMask = 0xFFFFF000u;  // draw bits compared with a threshold

enum Model : uint32_t { kRing = 0, kTwoLane = 1 };
enum Dis : uint32_t { kDisNone = 0, kDisBimodal = 1, kDisTurning = 2, kDisBimodalPQ = 3, kDisCrossing = 4 };

// Quenched planes per realization: the class plane (bimodal), the turning
// plane (two lanes), the p-class and q-class planes (bimodal, independent),
// or the u-class and v-class planes (two lanes, crossing at every site).
constexpr uint32_t dis_planes(uint32_t dis) {
  return dis == kDisNone ? 0u : ((dis == kDisBimodalPQ || dis == kDisCrossing) ? 2u : 1u);
}

// Rates of one context (u32 thresholds).
struct Rates {
  uint32_t p, q;          // ring: fast right/left; two lanes: lane A / lane B
  uint32_t p_slow, q_slow;  // bimodal slow class
  uint32_t omega;         // two lanes: lane-change probability per sweep (crossing kind: unmarked sites)
  uint32_t omega_slow;    // two lanes, crossing kind: lane-change probability at marked sites
  bool p_always, q_always;  // p / q == 0xffffffff (a draw r < t test alone cannot say "always")
  // Signed bounds INT_MIN + t / 4 of p, q, p_slow, q_slow (INT_MIN + 2^30 for "always") for the
  // one-key hop test of the domain attempt (asep_domain.cuh): r < t iff r >> 2 < t >> 2 when t is a
  // multiple of 4096.
  int32_t pb, qb, pb_slow, qb_slow;
};

inline int32_t hop_bound(uint32_t t) {
  return static_cast<int32_t>(0x80000000u + (t == 0xFFFFFFFFu ? (1u << 30) : (t >> 2)));
}

// Device-side clock of a context: the sweep index of the next sweep and the
// index of the first sample time not yet recorded.  Kernels read it; only the
// advance kernel, enqueued after them, writes it -- so an enqueued sequence of
// launches (or a captured CUDA graph of it) needs no host-side sweep value.
struct Clock {
  unsigned long long sweep;
  uint32_t next_time;
  uint32_t pad;
};

struct Geometry {
  uint64_t L;
  uint32_t W;        // words per plane
  uint32_t planes;   // occupancy planes
  uint32_t S;        // samples in the context
  uint32_t samples_per_real;
  uint32_t first_sample;
};

// Observables recorded at every sample time besides the heights.
struct Extras {
  int64_t* tab_cnt;        // [n_times][S][4] cumulative hop counters at each sample time
  uint32_t* profile;       // [S][planes][W] occupied sites per word, summed over sample times (or nullptr)
  uint32_t* snap;          // [S][planes][W] lattice at the autocorrelation reference time (or nullptr)
  int64_t* tab_ac;         // [n_times][S][planes] sum_i n_i(t0) n_i(t), 0 before t0 (or nullptr)
  uint64_t t0;             // autocorrelation reference sweep count
};

// Everything a domain-kernel launch needs about one context ("job").
// Philox4x32-10 round keys for a 64-bit seed: round i uses
// (lo + i * 0x9E3779B9, hi + i * 0xBB67AE85) mod 2^32.
struct KeySchedule {
  uint32_t x[10], y[10];
};

inline KeySchedule key_schedule(uint64_t seed) {
  KeySchedule ks;
  uint32_t kx = static_cast<uint32_t>(seed), ky = static_cast<uint32_t>(seed >> 32);
  for (int i = 0; i < 10; ++i) {
    ks.x[i] = kx;
    ks.y[i] = ky;
    kx += 0x9E3779B9u;
    ky += 0xBB67AE85u;
  }
  return ks;
}

struct DomainLaunch {
  Geometry geo;
  uint32_t model, dis;     // Model, Dis
  uint32_t count_hops;     // ring: count hops (two lanes always count)
  uint32_t* state;         // [S][planes][W]
  const uint32_t* mask;    // [R][W] or nullptr
  const uint32_t* ptab;    // Poisson table entries (device)
  uint32_t ptab_n, ptab_klo;
  uint32_t D, logD;        // domain sites, log2
  uint32_t R2, logR2;      // rows per column = 2D / 32, log2
  uint32_t row_bits;       // (D - 1) & ~31: the row bits of a slot
  uint32_t G;              // super-domains (columns) per sample = L / (2D)
  uint32_t spc;            // samples per sample group (CTA or queue item)
  uint32_t C;              // columns per group = spc * G
  uint32_t Cp;             // row pitch in words (multiple of 32, >= C)
  uint32_t n_groups;       // ceil(S / spc); cluster tier: S (one cluster per sample)
  uint32_t cluster;        // CTAs per sample: 1 = resident in one CTA, 2..16 = a thread-block cluster
  uint32_t Gc;             // cluster tier: columns per CTA (the last CTA may hold fewer)
  uint32_t lane_sort;      // resident tier: warps run domains of similar Poisson count (results unchanged)
  uint32_t sca_kmax;       // SCA: random planes that decide every threshold (20 - fewest trailing zeros)
  Rates rates;
  uint64_t seed;
  KeySchedule ks;          // round keys of `seed`
  uint32_t n_sweeps;       // sweeps of this launch
  Clock* clock;            // device
  const uint64_t* times;   // device, ascending sample times
  uint32_t n_times;
  int64_t* tab_sh;         // [n_times][S][planes]
  uint64_t* tab_sh2;       // [n_times][S][planes][2] (low, high word)
  uint64_t* counters;      // [S][4]
  Extras ex;
};

struct SerialLaunch {
  Geometry geo;
  uint32_t count_hops;     // ring: count hops (two lanes always count)
  uint32_t* state;
  const uint32_t* mask;
  Rates rates;
  uint64_t seed;
  uint32_t n_sweeps;
  Clock* clock;
  const uint64_t* times;
  uint32_t n_times;
  int64_t* tab_sh;
  uint64_t* tab_sh2;
  uint64_t* counters;
  Extras ex;
};

struct InitLaunch {
  Geometry geo;
  uint32_t* state;
  uint32_t init_kind;
  uint64_t init_seed;
};

struct DisorderLaunch {
  uint64_t L;
  uint32_t W, R;
  uint32_t planes;         // 1, or 2 for independent p and q classes (plane 1: call 1 of the stream)
  uint32_t first_real;
  uint32_t thr;
  uint64_t dis_seed;
  uint32_t* mask;
};

// Per-chunk partial sums of a record over a long lattice (see k_heights_part).
struct HeightPart {
  int64_t tot;   // height change across the chunk: sum of (2 n_i - 1)
  int64_t s1;    // sum of the heights relative to the chunk's entry height
  uint64_t s2lo, s2hi;  // sum of their squares (128 bits)
  int64_t ov;    // autocorrelation overlap of the chunk
};

// Lattices of more than this many words per plane are recorded in chunks of
// this size, one CTA each, and combined by a second launch.
constexpr uint32_t kHeightChunkWords = 1u << 14;

struct HeightsLaunch {
  Geometry geo;
  const uint32_t* state;
  uint32_t slot;
  uint64_t t;              // sweep count of this record (0 at creation)
  int64_t* tab_sh;
  uint64_t* tab_sh2;
  const uint64_t* counters;
  Extras ex;
  HeightPart* parts;       // [S][planes][chunks] when W > kHeightChunkWords (else unused)
};

// Balanced launch of the resident tier (asep_balance.cu): persistent CTAs
// take (sample group, chunk of `chunk` sweeps) items in chunk-major order.
struct BalanceLaunch {
  uint32_t chunk;      // sweeps per chunk
  uint32_t chunks;     // chunks of this launch: ceil(n_sweeps / chunk)
  uint32_t* progress;  // [n_groups + 1]: chunks each group has published, then the queue counter
  uint32_t* queue;     // = progress + n_groups
  uint32_t* err;       // set when a wait for a previous chunk runs out
  uint32_t stall;      // fault injection: group 0 never publishes its first chunk
};
// Longest chunk the host allows (the device-side wait bound is sized for it).
constexpr uint32_t kMaxBalanceChunk = 4096;
cudaError_t launch_domain_balanced(const DomainLaunch& a, const BalanceLaunch& b, uint32_t threads, size_t smem,
                                   cudaStream_t st);

// Shared memory of the resident kernel, in bytes (planes of R2 + 1 rows:
// the extra row mirrors the next column's row 0).
size_t domain_smem_bytes(uint32_t model, uint32_t dis, uint32_t R2, uint32_t Cp, uint32_t ptab_n, uint32_t threads);

cudaError_t launch_init(const InitLaunch& a, cudaStream_t st);
cudaError_t launch_disorder(const DisorderLaunch& a, cudaStream_t st);
// Chunks per plane of a record (1: one CTA per sample and plane); a.parts
// must hold S * planes * chunks entries when it is above 1.
uint32_t height_chunks(uint32_t W);
cudaError_t launch_heights(const HeightsLaunch& a, cudaStream_t st);
// One CTA per sample group of one context.
cudaError_t launch_domain(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st);
// Work items of the persistent batch kernel: (context index << kItemGroupBits) | sample group.
constexpr uint32_t kItemGroupBits = 18;
constexpr uint32_t kItemMaxJobs = 1u << (32 - kItemGroupBits);  // contexts per batch step
constexpr uint32_t kItemMaxGroups = 1u << kItemGroupBits;       // sample groups per context and step
// Persistent: `ctas` CTAs of `threads` threads take items (job << kItemGroupBits | group)
// from items[0..n_items) through the queue counter (zeroed here first).
cudaError_t launch_batch(const DomainLaunch* jobs, const uint32_t* items, uint32_t n_items, uint32_t* queue,
                         uint32_t threads, uint32_t ctas, size_t smem, cudaStream_t st);
// Cluster tier: one cluster of a.cluster CTAs per sample (grid S * cluster).
cudaError_t launch_cluster(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st);
// Streamed tier of the domain schedule (lattice in global memory, tiles of
// columns through shared memory); plan code kStreamTier in `cluster`.
constexpr uint32_t kStreamTier = 32;
size_t stream_smem_bytes(uint32_t model, uint32_t dis, uint32_t R2, uint32_t C, uint32_t ptab_n);
// err: set when a tile's copy wait runs out (bounded to one second); stall:
// extra bytes each tile's copies announce (0; fault injection for tests).
cudaError_t launch_stream_sweep(const DomainLaunch& a, uint32_t tiles, uint32_t threads, size_t smem, uint32_t* err,
                                uint32_t stall, cudaStream_t st);
// The two-sub-lattice SCA schedule: one CTA per sample, ring in shared memory.
cudaError_t launch_sca(const DomainLaunch& a, uint32_t threads, size_t smem, cudaStream_t st);
// Streamed SCA: one sweep (both phases; two lanes: with the lane changes)
// over every sample, lattice in global memory; results identical to launch_sca.
cudaError_t launch_sca_stream(const DomainLaunch& a, cudaStream_t st);
size_t sca_smem_bytes(uint32_t W, uint32_t planes, uint32_t quenched_planes);
// How many clusters of the given shape can be resident at once (0 = none).
int cluster_fits(uint32_t model, uint32_t dis, uint32_t cluster, uint32_t threads, size_t smem);
// Advance clocks after n sweeps (one context, or the jobs of a batch).
cudaError_t launch_advance(Clock* clock, const uint64_t* times, uint32_t n_times, uint32_t n, cudaStream_t st);
cudaError_t launch_advance_batch(const DomainLaunch* jobs, uint32_t n_jobs, cudaStream_t st);
cudaError_t launch_set_clock(Clock* clock, uint64_t sweep, uint32_t next_time, cudaStream_t st);
// Occupancy of the persistent kernel (CTAs per SM) for a block size and shared memory.
int batch_ctas_per_sm(uint32_t threads, size_t smem);
// Empty launches of the batch kernels (code loaded, local memory sized); `queue` is a device counter.
cudaError_t warm_batch_kernels(uint32_t* queue, cudaStream_t st);
cudaError_t launch_serial(const SerialLaunch& a, uint32_t model, uint32_t dis, cudaStream_t st);
cudaError_t launch_philox_bench(uint32_t blocks, uint32_t threads, uint32_t calls, uint32_t* sink, cudaStream_t st);
cudaError_t launch_attempt_bench(uint32_t blocks, uint32_t threads, uint32_t calls, uint32_t p, uint32_t q,
                                 uint32_t* sink, cudaStream_t st);
// Philox key of the microbenchmarks (the leading hexadecimal digits of pi).
constexpr uint64_t kBenchSeed = 0x243F6A8885A308D3ull;

}  // namespace asep

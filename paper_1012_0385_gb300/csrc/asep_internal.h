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

constexpr uint32_t kAcceptMask = 0xFFFFF000u;  // draw bits compared with a threshold

enum Model : uint32_t { kRing = 0, kTwoLane = 1 };
enum Dis : uint32_t { kDisNone = 0, kDisBimodal = 1, kDisTurning = 2 };

// Rates of one context (u32 thresholds).
struct Rates {
  uint32_t p, q;          // ring: fast right/left; two lanes: lane A / lane B
  uint32_t p_slow, q_slow;  // bimodal slow class
  uint32_t omega;         // two lanes: lane-change probability per sweep
  bool p_always, q_always;  // p / q == 0xffffffff (a draw r < t test alone cannot say "always")
};

// Heights recorded inside a launch: after the sweep count rec_times[i] the
// kernel writes table slot slot_base + i.
struct Record {
  const uint64_t* rec_times;  // device, ascending
  uint32_t n_rec;
  uint32_t slot_base;
  int64_t* tab_sh;    // [slot][S][planes]
  uint64_t* tab_sh2;  // [slot][S][planes][2] (low, high word)
};

struct Geometry {
  uint64_t L;
  uint32_t W;        // words per plane
  uint32_t planes;   // occupancy planes
  uint32_t S;        // samples in the context
  uint32_t samples_per_real;
  uint32_t first_sample;
};

// Resident two-phase Poisson-domain kernel.
struct DomainLaunch {
  Geometry geo;
  uint32_t* state;         // [S][planes][W]
  const uint32_t* mask;    // [R][W] or nullptr
  const uint32_t* ptab;    // Poisson table entries (device)
  uint32_t ptab_n, ptab_klo;
  uint32_t D, logD;        // domain sites, log2
  uint32_t R2, logR2;      // rows per column = 2D / 32, log2
  uint32_t row_bits;       // (D - 1) & ~31: the row bits of a slot
  uint32_t G;              // super-domains (columns) per sample = L / (2D)
  uint32_t spc;            // samples per CTA
  uint32_t C;              // columns per CTA = spc * G
  uint32_t Cp;             // row pitch in words (multiple of 32, >= C)
  Rates rates;
  uint64_t seed;
  uint64_t s0;             // index of the first sweep of this launch
  uint32_t n_sweeps;
  Record rec;
  uint64_t* counters;      // [S][4]
};

struct SerialLaunch {
  Geometry geo;
  uint32_t* state;
  const uint32_t* mask;
  Rates rates;
  uint64_t seed;
  uint64_t s0;
  uint32_t n_sweeps;
  Record rec;
  uint64_t* counters;
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
  uint32_t first_real;
  uint32_t thr;
  uint64_t dis_seed;
  uint32_t* mask;
};

struct HeightsLaunch {
  Geometry geo;
  const uint32_t* state;
  uint32_t slot;
  int64_t* tab_sh;
  uint64_t* tab_sh2;
};

// Shared memory of the resident kernel, in bytes (planes of R2 + 1 rows:
// the extra row mirrors the next column's row 0).
size_t domain_smem_bytes(uint32_t model, uint32_t dis, uint32_t R2, uint32_t Cp, uint32_t ptab_n, uint32_t threads);

cudaError_t launch_init(const InitLaunch& a, cudaStream_t st);
cudaError_t launch_disorder(const DisorderLaunch& a, cudaStream_t st);
cudaError_t launch_heights(const HeightsLaunch& a, cudaStream_t st);
cudaError_t launch_domain(const DomainLaunch& a, uint32_t model, uint32_t dis, bool count_hops, uint32_t threads,
                          uint32_t blocks, size_t smem, cudaStream_t st);
cudaError_t launch_serial(const SerialLaunch& a, uint32_t model, uint32_t dis, cudaStream_t st);
cudaError_t launch_philox_bench(uint32_t blocks, uint32_t threads, uint32_t calls, uint32_t* sink, cudaStream_t st);

}  // namespace asep

// asep_serial.h -- launch plans of the serial schedule (asep_serial.cu) for
// the host runtime.  Not installed.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "asep_internal.h"

namespace asep {

// Plans of the serial schedule (asep_info.cluster of a serial context).
constexpr uint32_t kSerialRounds = 1;  // one CTA per sample, the sweep's attempts in dependency rounds
constexpr uint32_t kSerialWarp = 2;    // one warp per sample, committed prefixes of up to 32 attempts
constexpr uint32_t kSerialRoundsMaxAttempts = 32u * 1024u;  // attempts per sweep: 32 per thread of a CTA
constexpr size_t kSerialRoundsSmem = 200u * 1024u;

// Dynamic shared memory of the one-CTA plan (lattice, quenched planes, site
// table, the sweep's draws), or 0 when the plan does not apply to L.
size_t serial_rounds_smem_bytes(uint32_t model, uint32_t dis, uint64_t L);
// Threads per CTA of the one-CTA plan.
uint32_t serial_rounds_threads(uint32_t model, uint64_t L);
// Samples (warps) per CTA of the one-warp plan for S samples.
uint32_t serial_warp_plan_warps(uint32_t S);
// Launch a serial sweep with plan kSerialRounds or kSerialWarp.
cudaError_t launch_serial_plan(const SerialLaunch& a, uint32_t model, uint32_t dis, uint32_t plan, cudaStream_t st);

}  // namespace asep

// Kernels of the compiled path.  They follow the emitted program functions
// and the dispatcher `jit_run` in the same translation unit.
#pragma once

#include "device_common.cuh"

#ifndef CUFZ_JIT_MIN_CTAS
#define CUFZ_JIT_MIN_CTAS 3
#endif
#ifndef CUFZ_JIT_CTA_THREADS
#define CUFZ_JIT_CTA_THREADS 256
#endif

// Copies the launch's engine tables into the CTA's shared copy.
static __device__ __forceinline__ void jit_stage_tables(const cufz::EngineTables& T) {
  static_assert(sizeof(cufz::EngineTables) % 4 == 0, "word copy");
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&T);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&cufz::s_T);
  for (uint32_t i = threadIdx.x; i < sizeof(cufz::EngineTables) / 4; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Persistent: CTAs pull work items from the batch until it is drained.
// paths: the launch gives the CTA a path table (kPathTableBytes of dynamic
// shared memory).
extern "C" __global__ void __launch_bounds__(CUFZ_JIT_CTA_THREADS, CUFZ_JIT_MIN_CTAS)
    cufz_jit_persistent(cufz::EngineTables T, cufz::BatchHdr* batch, uint32_t paths) {
  using namespace cufz;
  if (threadIdx.x == 0) s_paths = paths;
  jit_stage_tables(T);
  run_items<true, false>(s_T, batch, 0u, 0u, 0u, s_hash, nullptr, &s_in,
                         [&](const DevInput* in, uint32_t g0, uint32_t cnt, bool) -> bool {
                           return jit_run(in->prog, g0, g0 + cnt);
                         });
}

#if defined(CUFZ_JIT_PLAIN)
// Plain: one launch per input, CTA b runs test block b.
extern "C" __global__ void __launch_bounds__(1024) cufz_jit_plain(cufz::EngineTables T,
                                                                  cufz::BatchHdr* batch,
                                                                  uint32_t input) {
  using namespace cufz;
  if (threadIdx.x == 0) s_paths = 0u;  // no path table: threads replay their own paths
  jit_stage_tables(T);
  run_items<false, false>(s_T, batch, input, 0u, 0u, s_hash, nullptr, &s_in,
                          [&](const DevInput* in, uint32_t g0, uint32_t cnt, bool) -> bool {
                            return jit_run(in->prog, g0, g0 + cnt);
                          });
}
#endif

// Kernels of the compiled path.  They follow the emitted program functions
// and the dispatcher `jit_run` in the same translation unit.
#pragma once

#include "device_common.cuh"

#ifndef CUFZ_JIT_MIN_CTAS
#define CUFZ_JIT_MIN_CTAS 4
#endif

// Persistent: CTAs pull work items from the batch until it is drained.
extern "C" __global__ void __launch_bounds__(256, CUFZ_JIT_MIN_CTAS) cufz_jit_persistent(cufz::EngineTables T,
                                                                      cufz::BatchHdr* batch) {
  using namespace cufz;
  __shared__ __align__(16) uint32_t hash[kHashSlots];
  __shared__ __align__(16) uint8_t sin_raw[kInputSmemBytes];
  DevInput* sin = reinterpret_cast<DevInput*>(sin_raw);
  run_items<true, false>(T, batch, 0u, 0u, 0u, hash, nullptr, sin,
                         [&](const DevInput* in, uint32_t g0, uint32_t cnt, bool) -> bool {
                           return jit_run(in->prog, &T, in, hash, g0, g0 + cnt);
                         });
}

#if defined(CUFZ_JIT_PLAIN)
// Plain: one launch per input, CTA b runs test block b.
extern "C" __global__ void __launch_bounds__(1024) cufz_jit_plain(cufz::EngineTables T,
                                                                  cufz::BatchHdr* batch,
                                                                  uint32_t input) {
  using namespace cufz;
  __shared__ __align__(16) uint32_t hash[kHashSlots];
  __shared__ __align__(16) uint8_t sin_raw[kInputSmemBytes];
  DevInput* sin = reinterpret_cast<DevInput*>(sin_raw);
  run_items<false, false>(T, batch, input, 0u, 0u, hash, nullptr, sin,
                          [&](const DevInput* in, uint32_t g0, uint32_t cnt, bool) -> bool {
                            return jit_run(in->prog, &T, in, hash, g0, g0 + cnt);
                          });
}
#endif

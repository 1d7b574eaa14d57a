// Device engine of cufz (sm_103a): runs a loaded access-index program for
// every test thread of every admitted input, checks every access, compacts
// violation records and counts AFL-style edges.
//
// Mapping.  A work item is a contiguous range of an input's linear test
// threads g = block_lin * T + thread_lin.  A CTA takes one item at a time;
// its warps take 32 consecutive g's per pass (lane = test thread), so one warp
// always runs one program and dispatch is warp-uniform.  This is the paper's
// collapsing transform turned around (Sec. 4.1: a block becomes a CPU thread
// and its threads loop iterations); here test threads become lanes again,
// packed across test-block boundaries so no lane idles when T % 32 != 0.
//
// Structured control flow runs under per-lane activity bits with bit stacks
// (IF/ELSE/ENDIF, LOOP/ENDLOOP); a construct no lane enters is skipped.
//
// Checks (Sec. 4, ASan on every access; exact base and bounds as in Sec. 7.2):
// byte_off = idx << log2(width); a violation iff byte_off < 0 or
// byte_off + width > len.  Violating lanes of a warp are compacted with a
// ballot: one atomicAdd reserves their record slots, ranks come from popc.
//
// Coverage (Sec. 2.1, AFL payload after branches): e = (loc ^ prev) & 0xFFFF,
// prev = loc >> 1.  Lanes whose edge already reached 128 in the CTA's table
// skip it (its bucket is final); the others are merged by equal e with
// __match_any_sync and the group leader adds the group size into the per-CTA
// shared-memory hash table; the table is flushed into the slot's global
// counters after each item, and the last CTA of an input buckets the counts
// into the 64 KiB bitmap and ORs them into the device union.
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_common.cuh"
#include "engine.h"
#include "interp_kernel.cuh"

namespace cufz {

// Shared memory: hash table | program blob | DevInput | register file.
template <bool kPersistent>
__global__ void __launch_bounds__(1024) interp_kernel(EngineTables T, BatchHdr* batch,
                                                      uint32_t plain_input, uint32_t max_regs,
                                                      uint32_t max_prog_bytes) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* hash = reinterpret_cast<uint32_t*>(smem);
  uint8_t* sprog = smem + kEdgeSmemBytes;
  DevInput* sin = reinterpret_cast<DevInput*>(sprog + max_prog_bytes);
  uint8_t* rf = reinterpret_cast<uint8_t*>(sin) + kInputSmemBytes;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t nwarps = blockDim.x >> 5;
  run_items<kPersistent, true>(
      T, batch, plain_input, max_regs, max_prog_bytes, hash, sprog, sin,
      [&](const DevInput* in, uint32_t g0, uint32_t cnt, bool skip) -> bool {
        if (skip) return false;
        run_warp(T, in, sprog, rf + (size_t)warp * max_regs * kRegStride, hash, g0, cnt, warp,
                 nwarps);
        return true;
      });
}

template __global__ void interp_kernel<true>(EngineTables, BatchHdr*, uint32_t, uint32_t, uint32_t);
template __global__ void interp_kernel<false>(EngineTables, BatchHdr*, uint32_t, uint32_t, uint32_t);

uint32_t interp_smem_bytes(const LaunchShape& s) {
  return kEdgeSmemBytes + s.max_prog_bytes + kInputSmemBytes +
         (s.cta_threads / 32) * s.max_regs * kRegStride;
}

cudaError_t set_kernel_smem(uint32_t smem_bytes) {
  cudaError_t e = cudaFuncSetAttribute(interp_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(interp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes);
}

cudaError_t persistent_func_attributes(cudaFuncAttributes* out) {
  return cudaFuncGetAttributes(out, interp_kernel<true>);
}

cudaError_t persistent_occupancy(uint32_t cta_threads, uint32_t smem_bytes, int* ctas_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, interp_kernel<true>,
                                                       (int)cta_threads, smem_bytes);
}

cudaError_t launch_persistent(const EngineTables& T, const BatchHdr* d_batch, const LaunchShape& s,
                              cudaStream_t st) {
  interp_kernel<true><<<s.ctas, s.cta_threads, interp_smem_bytes(s), st>>>(
      T, const_cast<BatchHdr*>(d_batch), 0u, s.max_regs, s.max_prog_bytes);
  return cudaGetLastError();
}

cudaError_t launch_plain(const EngineTables& T, const BatchHdr* d_batch, uint32_t input_index,
                         uint32_t n_blocks_grid, const LaunchShape& s, cudaStream_t st) {
  interp_kernel<false><<<n_blocks_grid, s.cta_threads, interp_smem_bytes(s), st>>>(
      T, const_cast<BatchHdr*>(d_batch), input_index, s.max_regs, s.max_prog_bytes);
  return cudaGetLastError();
}

__global__ void fill_u64_kernel(uint64_t* p, uint64_t n, uint64_t v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

cudaError_t launch_clear(void* p, uint64_t bytes, uint64_t pattern, cudaStream_t st) {
  uint64_t n = bytes / 8;
  if (!n) return cudaSuccess;
  uint32_t blocks = (uint32_t)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  fill_u64_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<uint64_t*>(p), n, pattern);
  return cudaGetLastError();
}

// INT32 issue probe: eight independent chains alternating xor and add, which
// no single integer instruction can fuse; 16 ops per chain per iteration.
__global__ void int32_peak_kernel(uint32_t* out, uint32_t iters, uint32_t y, uint32_t z) {
  uint32_t a0 = threadIdx.x, a1 = a0 ^ 1, a2 = a0 ^ 2, a3 = a0 ^ 3, a4 = a0 ^ 4, a5 = a0 ^ 5,
           a6 = a0 ^ 6, a7 = a0 ^ 7;
#pragma unroll 1
  for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      asm volatile("xor.b32 %0, %0, %8;\n\tadd.u32 %0, %0, %9;\n\t"
                   "xor.b32 %1, %1, %8;\n\tadd.u32 %1, %1, %9;\n\t"
                   "xor.b32 %2, %2, %8;\n\tadd.u32 %2, %2, %9;\n\t"
                   "xor.b32 %3, %3, %8;\n\tadd.u32 %3, %3, %9;\n\t"
                   "xor.b32 %4, %4, %8;\n\tadd.u32 %4, %4, %9;\n\t"
                   "xor.b32 %5, %5, %8;\n\tadd.u32 %5, %5, %9;\n\t"
                   "xor.b32 %6, %6, %8;\n\tadd.u32 %6, %6, %9;\n\t"
                   "xor.b32 %7, %7, %8;\n\tadd.u32 %7, %7, %9;\n\t"
                   : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7)
                   : "r"(y), "r"(z));
    }
  }
  uint32_t r = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
  if (r == 0x12345678u) out[0] = r;  // keeps the chains live
}

cudaError_t launch_int32_peak(uint32_t* out, uint32_t blocks, uint32_t threads, uint32_t iters,
                              cudaStream_t st) {
  int32_peak_kernel<<<blocks, threads, 0, st>>>(out, iters, 0x9E3779B9u, 0x7F4A7C15u);
  return cudaGetLastError();
}

}  // namespace cufz

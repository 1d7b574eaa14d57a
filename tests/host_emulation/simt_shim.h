// TEST-ONLY.  Lets the bytecode interpreter's device code (interp_kernel.cuh
// and the work-item loop, finalize and helpers of device_common.cuh) run on
// the host for tests without a GPU: one CTA of one full warp, its 32 lanes
// as 32 host threads.  The interpreter is warp-synchronous (every lane
// reaches every warp collective in the same order, with the full mask), so
// each collective is emulated exactly as an exchange between the 32 threads
// at a barrier; shared memory is memory all 32 threads share; atomics hold
// one lock.  A lane that waits at a collective longer than a bound aborts
// the process (a lane out of step is a bug the test must report, not a
// hang).  Nothing in the package includes this file.
#pragma once

#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>

#define __device__
#define __global__
#define __host__
#define __shared__ static
#define __noinline__ __attribute__((noinline))
#define __forceinline__ inline
#define __align__(n) __attribute__((aligned(n)))
#define __launch_bounds__(...)

struct shim_dim3 {
  unsigned x, y, z;
};
extern thread_local shim_dim3 threadIdx;
static const shim_dim3 blockIdx = {0, 0, 0};
static const shim_dim3 blockDim = {32, 1, 1};
static const shim_dim3 gridDim = {1, 1, 1};

struct uint4 {
  unsigned x, y, z, w;
};
static inline uint4 make_uint4(unsigned x, unsigned y, unsigned z, unsigned w) {
  return uint4{x, y, z, w};
}

static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static inline int __ffs(unsigned x) { return __builtin_ffs((int)x); }
static inline int32_t min(int32_t a, int32_t b) { return a < b ? a : b; }
static inline int32_t max(int32_t a, int32_t b) { return a > b ? a : b; }

// The warp: 32 slots and a reusable barrier (lanes spin, yielding the core,
// until the last lane of the round arrives).
struct ShimWarp {
  std::atomic<unsigned> arrived{0};
  std::atomic<unsigned long long> generation{0};
  uint64_t slot[32];

  void barrier() {
    const unsigned long long gen = generation.load(std::memory_order_acquire);
    if (arrived.fetch_add(1, std::memory_order_acq_rel) == 31) {
      arrived.store(0, std::memory_order_relaxed);
      generation.fetch_add(1, std::memory_order_acq_rel);
      return;
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (unsigned long long spins = 1; generation.load(std::memory_order_acquire) == gen; spins++) {
      std::this_thread::yield();
      if (spins % 100000 == 0 &&
          std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60)) {
        fprintf(stderr, "simt shim: lane %u waited 60 s at a warp collective\n", threadIdx.x);
        abort();
      }
    }
  }
  // Every lane contributes v; afterwards every lane sees all 32 values.
  void exchange(uint64_t v, uint64_t* all) {
    slot[threadIdx.x] = v;
    barrier();
    memcpy(all, slot, sizeof(slot));
    barrier();
  }
};
extern ShimWarp g_shim_warp;
extern std::mutex g_shim_atomic;

template <class T>
static inline uint64_t shim_bits(T v) {
  uint64_t b = 0;
  memcpy(&b, &v, sizeof(T));
  return b;
}
template <class T>
static inline T shim_value(uint64_t b) {
  T v;
  memcpy(&v, &b, sizeof(T));
  return v;
}

static inline unsigned __ballot_sync(unsigned, int p) {
  uint64_t all[32];
  g_shim_warp.exchange(p ? 1u : 0u, all);
  unsigned m = 0;
  for (int i = 0; i < 32; i++) m |= (all[i] ? 1u : 0u) << i;
  return m;
}
static inline int __any_sync(unsigned mask, int p) { return __ballot_sync(mask, p) != 0; }
static inline int __all_sync(unsigned mask, int p) { return __ballot_sync(mask, p) == 0xFFFFFFFFu; }
static inline unsigned __activemask() { return 0xFFFFFFFFu; }
template <class T>
static inline T __shfl_sync(unsigned, T v, int src, int = 32) {
  uint64_t all[32];
  g_shim_warp.exchange(shim_bits(v), all);
  return shim_value<T>(all[src & 31]);
}
template <class T>
static inline T __shfl_xor_sync(unsigned, T v, int lane_mask, int = 32) {
  uint64_t all[32];
  g_shim_warp.exchange(shim_bits(v), all);
  return shim_value<T>(all[(threadIdx.x ^ (unsigned)lane_mask) & 31]);
}
static inline unsigned __match_any_sync(unsigned, unsigned v) {
  uint64_t all[32];
  g_shim_warp.exchange(v, all);
  unsigned m = 0;
  for (int i = 0; i < 32; i++) m |= (all[i] == v ? 1u : 0u) << i;
  return m;
}
static inline unsigned __reduce_add_sync(unsigned, unsigned v) {
  uint64_t all[32];
  g_shim_warp.exchange(v, all);
  unsigned s = 0;
  for (int i = 0; i < 32; i++) s += (unsigned)all[i];
  return s;
}
static inline void __syncthreads() { g_shim_warp.barrier(); }
static inline int __syncthreads_or(int p) { return __any_sync(0xFFFFFFFFu, p); }
static inline void __syncwarp(unsigned = 0xFFFFFFFFu) { g_shim_warp.barrier(); }
static inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }
static inline void __threadfence_system() { std::atomic_thread_fence(std::memory_order_seq_cst); }

template <class T, class U>
static inline T atomicAdd(T* p, U v) {
  std::lock_guard<std::mutex> g(g_shim_atomic);
  const T old = *p;
  *p = (T)(old + (T)v);
  return old;
}
template <class T, class U>
static inline T atomicOr(T* p, U v) {
  std::lock_guard<std::mutex> g(g_shim_atomic);
  const T old = *p;
  *p = (T)(old | (T)v);
  return old;
}
template <class T, class U>
static inline T atomicMin(T* p, U v) {
  std::lock_guard<std::mutex> g(g_shim_atomic);
  const T old = *p;
  if ((T)v < old) *p = (T)v;
  return old;
}
template <class T, class U, class V>
static inline T atomicCAS(T* p, U cmp, V val) {
  std::lock_guard<std::mutex> g(g_shim_atomic);
  const T old = *p;
  if (old == (T)cmp) *p = (T)val;
  return old;
}

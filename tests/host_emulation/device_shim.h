// TEST-ONLY.  Lets the compiled path's device code compile and run on the
// host for tests without a GPU: the program functions the loader emits and
// the helpers of jit_kernel.cuh and device_common.cuh they call.  One CTA of
// one thread: every warp has a single active lane, so the warp intrinsics
// reduce to their one-lane results (a group of one, a sum over one lane) and
// atomics to plain read-modify-writes.  What this cannot show (lanes that
// merge or race, several CTAs) is covered by the GPU tests.  Nothing in the
// package includes this file.
#pragma once

#include <stdint.h>

#define __device__
#define __global__
#define __host__
#define __shared__
#define __noinline__ __attribute__((noinline))
#define __forceinline__ inline
#define __align__(n) __attribute__((aligned(n)))
#define __launch_bounds__(...)

struct shim_dim3 {
  unsigned x, y, z;
};
static const shim_dim3 threadIdx = {0, 0, 0};
static const shim_dim3 blockIdx = {0, 0, 0};
static const shim_dim3 blockDim = {1, 1, 1};
static const shim_dim3 gridDim = {1, 1, 1};

struct uint2 {
  unsigned x, y;
};
struct uint4 {
  unsigned x, y, z, w;
};
static inline uint4 make_uint4(unsigned x, unsigned y, unsigned z, unsigned w) {
  return uint4{x, y, z, w};
}

static inline unsigned __activemask() { return 1u; }
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static inline int __ffs(unsigned x) { return __builtin_ffs((int)x); }
template <class T>
static inline T __shfl_sync(unsigned, T v, int, int = 32) { return v; }
template <class T>
static inline T __shfl_xor_sync(unsigned, T v, int, int = 32) { return v; }
static inline unsigned __match_any_sync(unsigned, unsigned) { return 1u; }
static inline unsigned __reduce_add_sync(unsigned, unsigned v) { return v; }
static inline int __any_sync(unsigned, int p) { return p; }
static inline void __syncthreads() {}
static inline int __syncthreads_or(int p) { return p; }
static inline void __syncwarp(unsigned = 0xFFFFFFFFu) {}
static inline void __threadfence() {}
static inline void __threadfence_system() {}

template <class T, class U>
static inline T atomicAdd(T* p, U v) {
  const T old = *p;
  *p = (T)(old + (T)v);
  return old;
}
template <class T, class U>
static inline T atomicOr(T* p, U v) {
  const T old = *p;
  *p = (T)(old | (T)v);
  return old;
}
template <class T, class U>
static inline T atomicMin(T* p, U v) {
  const T old = *p;
  if ((T)v < old) *p = (T)v;
  return old;
}
template <class T, class U, class V>
static inline T atomicCAS(T* p, U cmp, V val) {
  const T old = *p;
  if (old == (T)cmp) *p = (T)val;
  return old;
}

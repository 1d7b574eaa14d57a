// The fuzzing campaign's input mutator, host and device code: per input one
// to three mutations of a scalar argument or of the length of one of its
// program's buffers, drawn from a SplitMix64 stream (Steele, Lea and Flood,
// 2014).  The mutations are AFL's deterministic-stage kinds applied at
// random (Sec. 2.1): flip one bit, add or subtract 1..35, or substitute a
// boundary value.  Launch shapes are left alone.  The draws follow
// gen.Mutator of the Python package call for call, so both give the same
// inputs from the same state.
#pragma once

#include <stdint.h>

#include "../../include/cufz.h"

#if defined(__CUDACC__)
#define CUFZ_MHD __host__ __device__
#else
#define CUFZ_MHD
#endif

namespace cufz {

struct SplitMix64 {
  uint64_t s;
  CUFZ_MHD uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // uniform in [0, n) by multiply-shift of the top 32 bits
  CUFZ_MHD uint32_t below(uint32_t n) { return (uint32_t)(((next() >> 32) * (uint64_t)n) >> 32); }
  // true with probability 1/2: the 53-bit uniform in [0, 1) is below 0.5
  CUFZ_MHD bool half() { return (next() >> 11) < (1ull << 52); }
};

// The state that starts child j's mutation stream in round r of a campaign
// seeded with `seed` (one stream per child, so the children of a round are
// mutated independently, on the host or in parallel on the device).
CUFZ_MHD inline uint64_t child_stream(uint64_t seed, uint64_t round, uint32_t j) {
  return seed + ((round << 32) | j) * 0xD1B54A32D192ED03ull;
}

CUFZ_MHD inline int32_t boundary_arg(SplitMix64& r) {
  const uint32_t k = r.below(31);
  const uint32_t base = 1u << k;
  const uint32_t pick[7] = {0u, 0xFFFFFFFFu, 1u, base, base + 1u, base - 1u, 0u - base};
  return (int32_t)pick[r.below(7)];
}

CUFZ_MHD inline uint64_t boundary_len(uint32_t i) {
  const uint64_t lens[29] = {0,   1,   2,   3,   4,    7,    8,    15,   16,    17,
                             31,  32,  63,  64,  100,  127,  128,  129,  255,   256,
                             511, 512, 1000, 1023, 1024, 4095, 4096, 65535, 65536};
  return lens[i];
}
constexpr uint32_t kNumBoundaryLens = 29;

CUFZ_MHD inline void mutate_one(cufz_input& x, uint32_t n_bufs, SplitMix64& r) {
  const uint32_t n_fields = 4 + n_bufs;
  const uint32_t rounds = 1 + r.below(3);
  for (uint32_t i = 0; i < rounds; i++) {
    const uint32_t f = r.below(n_fields);
    const uint32_t kind = r.below(3);
    if (f < 4) {
      uint32_t v = (uint32_t)x.args[f];
      if (kind == 0) {
        v ^= 1u << r.below(32);
      } else if (kind == 1) {
        const uint32_t d = 1 + r.below(35);
        v = r.half() ? v + d : v - d;
      } else {
        v = (uint32_t)boundary_arg(r);
      }
      x.args[f] = (int32_t)v;
    } else {
      uint64_t& v = x.buf_len[f - 4];
      if (kind == 0) {
        v ^= 1ull << r.below(24);
      } else if (kind == 1) {
        const uint64_t d = 1 + r.below(35);
        v = r.half() ? v + d : (v > d ? v - d : 0);
      } else {
        v = boundary_len(r.below(kNumBoundaryLens));
      }
    }
  }
}

}  // namespace cufz

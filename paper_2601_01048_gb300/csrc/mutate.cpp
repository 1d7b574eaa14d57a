// The fuzzing campaign's input mutator, native (host-only): per input one to
// three mutations of a scalar argument or of the length of one of its
// program's buffers, drawn from a SplitMix64 stream (Steele, Lea and Flood,
// 2014).  The mutations are AFL's deterministic-stage kinds applied at
// random (Sec. 2.1): flip one bit, add or subtract 1..35, or substitute a
// boundary value.  Launch shapes are left alone.  The draws follow
// gen.Mutator of the Python package call for call, so both give the same
// inputs from the same state.
#include <stdint.h>
#include <string.h>

#include "../../include/cufz.h"

namespace {

struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // uniform in [0, n) by multiply-shift of the top 32 bits
  uint32_t below(uint32_t n) { return (uint32_t)(((next() >> 32) * (uint64_t)n) >> 32); }
  // true with probability 1/2: the 53-bit uniform in [0, 1) is below 0.5
  bool half() { return (next() >> 11) < (1ull << 52); }
};

const uint64_t kLens[] = {0,   1,   2,   3,   4,    7,    8,    15,   16,    17,
                          31,  32,  63,  64,  100,  127,  128,  129,  255,   256,
                          511, 512, 1000, 1023, 1024, 4095, 4096, 65535, 65536};
constexpr uint32_t kNumLens = sizeof(kLens) / sizeof(kLens[0]);

int32_t boundary_arg(SplitMix64& r) {
  const uint32_t k = r.below(31);
  const uint32_t base = 1u << k;
  const uint32_t pick[7] = {0u, 0xFFFFFFFFu, 1u, base, base + 1u, base - 1u, 0u - base};
  return (int32_t)pick[r.below(7)];
}

void mutate_one(cufz_input& x, uint32_t n_bufs, SplitMix64& r) {
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
        v = kLens[r.below(kNumLens)];
      }
    }
  }
}

}  // namespace

extern "C" cufz_status cufz_mutate_inputs(cufz_input* inputs, uint32_t n, const uint8_t* n_bufs,
                                          uint32_t n_programs, uint64_t* rng_state) {
  if ((!inputs && n) || !rng_state || (!n_bufs && n_programs)) return CUFZ_E_INVALID_ARG;
  for (uint32_t i = 0; i < n; i++)
    if (inputs[i].program_id >= n_programs || n_bufs[inputs[i].program_id] > 9)
      return CUFZ_E_INVALID_ARG;
  SplitMix64 r{*rng_state};
  for (uint32_t i = 0; i < n; i++) mutate_one(inputs[i], n_bufs[inputs[i].program_id], r);
  *rng_state = r.s;
  return CUFZ_OK;
}

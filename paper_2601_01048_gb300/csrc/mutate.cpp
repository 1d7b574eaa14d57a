// The fuzzing campaign's input mutator on the host (the mutation itself is
// in mutate.h, shared with the device campaign).
#include <stdint.h>
#include <string.h>

#include "../../include/cufz.h"
#include "mutate.h"

using cufz::SplitMix64;

extern "C" cufz_status cufz_mutate_inputs(cufz_input* inputs, uint32_t n, const uint8_t* n_bufs,
                                          uint32_t n_programs, uint64_t* rng_state) {
  if ((!inputs && n) || !rng_state || (!n_bufs && n_programs)) return CUFZ_E_INVALID_ARG;
  for (uint32_t i = 0; i < n; i++)
    if (inputs[i].program_id >= n_programs || n_bufs[inputs[i].program_id] > 9)
      return CUFZ_E_INVALID_ARG;
  SplitMix64 r{*rng_state};
  for (uint32_t i = 0; i < n; i++) cufz::mutate_one(inputs[i], n_bufs[inputs[i].program_id], r);
  *rng_state = r.s;
  return CUFZ_OK;
}

extern "C" cufz_status cufz_mutate_children(cufz_input* inputs, uint32_t n, const uint8_t* n_bufs,
                                            uint32_t n_programs, uint64_t seed, uint64_t round) {
  if ((!inputs && n) || (!n_bufs && n_programs)) return CUFZ_E_INVALID_ARG;
  for (uint32_t i = 0; i < n; i++)
    if (inputs[i].program_id >= n_programs || n_bufs[inputs[i].program_id] > 9)
      return CUFZ_E_INVALID_ARG;
  for (uint32_t j = 0; j < n; j++) {
    SplitMix64 r{cufz::child_stream(seed, round, j)};
    cufz::mutate_one(inputs[j], n_bufs[inputs[j].program_id], r);
  }
  return CUFZ_OK;
}

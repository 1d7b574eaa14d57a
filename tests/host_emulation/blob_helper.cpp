// TEST-ONLY: the library's program loading (load_program) behind a plain C
// call, for the interpreter's host runner, whose translation unit cannot
// include the CUDA runtime headers next to the warp emulation.
#include <stdlib.h>
#include <string.h>

#include "engine.h"

extern "C" int shim_load_blob(const void* bytes, size_t nbytes, int prune, uint8_t** blob,
                              uint32_t* blob_bytes, uint32_t* n_regs, uint32_t* n_bufs,
                              uint32_t* shared_mask) {
  cufz::LoadedProgram lp;
  if (cufz::load_program(bytes, nbytes, prune != 0, &lp) != CUFZ_OK) return -1;
  *blob = (uint8_t*)malloc(lp.blob_bytes);
  memcpy(*blob, lp.blob, lp.blob_bytes);
  *blob_bytes = lp.blob_bytes;
  *n_regs = lp.hdr.n_regs;
  *n_bufs = lp.n_bufs;
  *shared_mask = lp.shared_mask;
  cufz::free_program(&lp);
  return 0;
}

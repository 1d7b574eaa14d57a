// Building a batch's per-input descriptor from a cufz_input: launch checks
// and the DevInput fields that follow from the input and its program.  Host
// and device code: the runtime builds batches on the host; the device
// fuzzing campaign (campaign.cu) builds its rounds' batches on the device
// with the same functions.
#pragma once

#include <stdint.h>

#include "layout.h"

#if defined(__CUDACC__)
#define CUFZ_HD __host__ __device__
#else
#define CUFZ_HD
#endif

namespace cufz {

// m = ceil(2^64 / d) for d >= 2; d <= 1 is encoded as 0 (see udiv).
CUFZ_HD inline uint64_t div_magic(uint32_t d) { return d <= 1 ? 0ull : (~0ull / d) + 1ull; }

// Launch shapes CUDA would refuse (a zero dimension, more than 1024 threads
// per block, block.z > 64, grid.x > 2^31 - 1, grid.y or grid.z > 65535):
// such inputs complete as CUFZ_ST_INVALID_CONFIG without running.
CUFZ_HD inline bool launch_rejected(const cufz_input& in) {
  const uint32_t* g = in.grid;
  const uint32_t* b = in.block;
  if (!g[0] || !g[1] || !g[2] || !b[0] || !b[1] || !b[2]) return true;
  if (b[0] > 1024 || b[1] > 1024 || b[2] > 64) return true;
  if ((uint64_t)b[0] * b[1] * b[2] > 1024) return true;
  return g[0] > 0x7FFFFFFFu || g[1] > 65535 || g[2] > 65535;
}

// Whether a launch CUDA accepts has at most max_threads test threads; if so
// their number goes to *n_threads (when not null).  The block count (below
// 2^31 * 2^16 * 2^16 = 2^63) is compared with max_threads / (threads per
// block) before any product, so a grid whose thread count would wrap 64 bits
// is refused, not wrapped.
CUFZ_HD inline bool launch_within(const cufz_input& in, uint64_t max_threads, uint64_t* n_threads) {
  const uint64_t T = (uint64_t)in.block[0] * in.block[1] * in.block[2];
  const uint64_t nb = (uint64_t)in.grid[0] * in.grid[1] * in.grid[2];
  if (T == 0 || nb > max_threads / T) return false;
  if (n_threads) *n_threads = nb * T;
  return true;
}

// The part of a DevInput that follows from the input and its program: launch
// shape, division magics, arguments, buffer lengths, redzone-separated
// virtual bases (per space: base_0 = R, base_k+1 = align256(base_k + len_k
// + R)) and per-width index limits min(len >> lw, 2^31).  Zeroes the rest
// (slot, program placement, items, ticket, sequence), which the caller sets.
CUFZ_HD inline void fill_dev_input(const cufz_input& in, uint32_t n_bufs, uint32_t shared_mask,
                                   uint32_t redzone, DevInput* d) {
  uint32_t* w = reinterpret_cast<uint32_t*>(d);
  for (uint32_t i = 0; i < sizeof(DevInput) / 4; i++) w[i] = 0;
  for (int k = 0; k < 3; k++) {
    d->grid[k] = in.grid[k];
    d->block[k] = in.block[k];
  }
  for (int k = 0; k < 4; k++) d->args[k] = in.args[k];
  const uint32_t Bx = in.block[0], By = in.block[1], Bz = in.block[2];
  d->T = Bx * By * Bz;
  // callers pass inputs that launch_within() accepted; anything larger would
  // wrap, so it is stored as 0 threads rather than as a wrapped count
  uint64_t nt = 0;
  d->n_threads = launch_within(in, ~0ull, &nt) ? nt : 0;
  d->mT = div_magic(d->T);
  d->Bx = Bx;
  d->mBx = div_magic(Bx);
  d->Bxy = Bx * By;
  d->mBxy = div_magic(d->Bxy);
  d->gx = in.grid[0];
  d->mGx = div_magic(in.grid[0]);
  d->gxy = (uint32_t)((uint64_t)in.grid[0] * in.grid[1]);
  d->mGxy = div_magic(d->gxy);
  const int64_t R = (int64_t)redzone;
  int64_t next[2] = {R, R};
  for (uint32_t k = 0; k < n_bufs && k < (uint32_t)kMaxBufs; k++) {
    const int sp = (shared_mask >> k) & 1;
    d->len[k] = (int64_t)in.buf_len[k];
    d->base[k] = next[sp];
    next[sp] = (next[sp] + d->len[k] + R + 255) & ~(int64_t)255;
    for (uint32_t lw = 0; lw < 5; lw++) {
      const uint64_t n = in.buf_len[k] >> lw;
      d->lim[k * 5 + lw] = n < 0x80000000ull ? (uint32_t)n : 0x80000000u;
    }
  }
  d->shared_mask = shared_mask;
  d->n_bufs = n_bufs;
  d->user_tag = in.user_tag;
}

// A launch the block-serial form runs: a block of at most kBlkMaxThreads
// threads, and shared buffers of at most kBlkSharedBytes bytes together.
CUFZ_HD inline bool block_serial_fits(uint32_t n_bufs, uint32_t shared_mask, const cufz_input& x) {
  const uint64_t T = (uint64_t)x.block[0] * x.block[1] * x.block[2];
  uint64_t sh = 0;
  for (uint32_t k = 0; k < n_bufs && k < (uint32_t)kMaxBufs; k++)
    if ((shared_mask >> k) & 1u) sh += x.buf_len[k];
  return T <= kBlkMaxThreads && sh <= kBlkSharedBytes;
}

}  // namespace cufz

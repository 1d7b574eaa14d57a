// Device helpers for programs compiled at load time.  The loader emits one
// function per program (straight-line CUDA: program registers become local
// variables, buffer/width/site/LOC values become constants); these helpers
// are what the emitted code calls for checks, records and coverage.  The
// emitted code runs each test thread as one CUDA thread; lanes that take the
// same path are aggregated with __activemask() groups.
#pragma once

#include "device_common.cuh"

namespace cufz {

// Record path of a violating access, entered by the violating lanes of a
// warp that may still reserve record space: one atomicAdd per group, ranks
// from popc.  `what` packs site | buf << 16 | kind << 20 | log2(width) << 24.
// Returns true once the input's record area is full.
static __device__ __noinline__ bool jit_record(const EngineTables* T, const DevInput* in, uint32_t bl,
                                        uint32_t tl, uint32_t ordinal, uint32_t what,
                                        int64_t off) {
  const uint32_t am = __activemask();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t leader = __ffs(am) - 1;
  const uint32_t k = __popc(am);
  const uint32_t cap = T->record_cap;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&T->slots[in->slot].rec_reserved, k);
  base = __shfl_sync(am, base, leader);
  const uint32_t rank = __popc(am & ((1u << lane) - 1u));
  if (base + rank < cap) {
    const uint32_t site = what & 0xFFFFu, buf = (what >> 16) & 0xFu, kind = (what >> 20) & 1u;
    const uint32_t w = 1u << ((what >> 24) & 7u);
    const uint32_t sm = in->shared_mask;
    const uint32_t cls = classify(in, sm, in->n_bufs, buf, off, w, (int64_t)T->redzone);
    write_record(T->records + (size_t)in->slot * cap + base + rank, bl, tl, ordinal, site, buf,
                 kind, w, (sm >> buf) & 1u, cls, off);
  }
  return base + k >= cap;
}

static __device__ __forceinline__ void jit_violation(const EngineTables* T, const DevInput* in,
                                              LaneAcc& acc, uint32_t bl, uint32_t tl,
                                              uint32_t ordinal, uint32_t what, int64_t off) {
  if (acc.first_key == ~0ull) acc.first_key = first_key_of(bl, tl, ordinal);
  if (!acc.rec_full) acc.rec_full = jit_record(T, in, bl, tl, ordinal, what, off);
}

// Number of in-bounds indices of a buffer of len bytes for accesses of
// width 2^lw, clamped to 2^31 (every int32 index below it is in bounds).
static __device__ __forceinline__ uint32_t jit_index_limit(int64_t len, uint32_t lw) {
  const uint64_t n = (uint64_t)len >> lw;
  return n < 0x80000000ull ? (uint32_t)n : 0x80000000u;
}

// Warp-aggregated edge hit: lanes of the current group with equal e are
// merged and their leader adds the group size into the CTA's edge table.
static __device__ __forceinline__ void jit_cover(const EngineTables* T, uint32_t* hash, uint32_t slot,
                                          uint32_t e) {
  const uint32_t am = __activemask();
  const uint32_t peers = __match_any_sync(am, e);
  if ((threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1)) {
    // first probe inline: the edge is usually already in its home slot
    const uint32_t c = __popc(peers);
    const uint32_t tag = (e + 1u) << kHashTagShift;
    uint32_t* p = &hash[(e * 2654435761u) >> (32 - 11)];
    const uint32_t cur = *p;
    if ((cur & ~kHashCountMask) == tag) {
      if ((cur & kHashCountMask) < 128u) atomicAdd(p, c);
    } else {
      edge_add(hash, *T, slot, e, c);
    }
  }
}

// Seeded content of a global buffer (seedx = program seed ^ buf * 0x9E3779B9).
static __device__ __forceinline__ int32_t jit_content(uint32_t seedx, int64_t off, uint32_t lw) {
  const uint32_t word = mix32(seedx ^ (uint32_t)(off >> 2));
  return lw == 0 ? (int32_t)((word >> (8u * ((uint32_t)off & 3u))) & 0xFFu) : (int32_t)word;
}



}  // namespace cufz

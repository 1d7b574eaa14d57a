// Device helpers for programs compiled at load time.  The loader emits two
// functions per program (straight-line CUDA: program registers become local
// variables, buffer/width/site/LOC values become constants), each running
// one test thread per CUDA thread: a work-item function that counts
// accesses, violations and branch evaluations, folds the digest and updates
// edges, with no record code; and a record function that re-runs one
// violating thread to write its records (jit_record, active-mask groups) and
// find its first violation.  These helpers are what the emitted code calls.
#pragma once

#include "device_common.cuh"

namespace cufz {

// The CTA's engine tables, copy of the current input and edge state.  They
// sit at file scope so that the program functions (which take no pointers)
// reach them as shared memory: 32-bit addresses and shared-memory atomics,
// and no registers held for base pointers.
static __shared__ EngineTables s_T;
static __shared__ __align__(16) DevInput s_in;
static __shared__ __align__(16) uint32_t s_hash[kHashSlots + kSatWords];

// Record path of a violating access, entered by the violating lanes of a
// warp that may still reserve record space: one atomicAdd per group, ranks
// from popc.  `what` packs site | buf << 16 | kind << 20 | log2(width) << 24.
// Returns true once the input's record area is full.
static __device__ __noinline__ bool jit_record(uint32_t bl, uint32_t tl, uint32_t ordinal,
                                               uint32_t what, int64_t off) {
  const uint32_t am = __activemask();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t leader = __ffs(am) - 1;
  const uint32_t k = __popc(am);
  const uint32_t cap = s_T.record_cap;
  const uint32_t slot = s_in.slot;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&s_T.slots[slot].rec_reserved, k);
  base = __shfl_sync(am, base, leader);
  const uint32_t rank = __popc(am & ((1u << lane) - 1u));
  if (base + rank < cap) {
    const uint32_t site = what & 0xFFFFu, buf = (what >> 16) & 0xFu, kind = (what >> 20) & 1u;
    const uint32_t w = 1u << ((what >> 24) & 7u);
    const uint32_t sm = s_in.shared_mask;
    const uint32_t cls = classify(&s_in, sm, s_in.n_bufs, buf, off, w, (int64_t)s_T.redzone);
    write_record(s_T.records + (size_t)slot * cap + base + rank, bl, tl, ordinal, site, buf,
                 kind, w, (sm >> buf) & 1u, cls, off);
  }
  return base + k >= cap;
}

// Records of the compiled path come from a second run of a violating test
// thread (the record function).  A thread is listed for it while the
// violations of the threads listed before it are fewer than the record cap,
// so the listed threads hold min(n_violations, cap) records or more and the
// record area is filled exactly as a single pass would fill it.

// Whether the input's record list had room when the item started.
static __device__ __forceinline__ bool jit_records_open(uint32_t slot) {
  const volatile uint32_t* r = &s_T.slots[slot].rec_listed;
  return *r < s_T.record_cap;
}

// Adds a finished thread's nv violations to the listed total; returns the
// total before it (the thread is listed iff that is below the cap).
static __device__ __forceinline__ uint32_t jit_list_violations(uint32_t slot, uint32_t nv) {
  return atomicAdd(&s_T.slots[slot].rec_listed, nv);
}

// Whether a violating thread that is not listed still has to be re-run for
// its first-violation key: only the lane's first violating thread can hold
// the lane's minimum key, and none can beat a smaller key already published
// by a finished item of the input (the lane then takes that key, which
// leaves the input's minimum unchanged and ends the checks).
static __device__ __forceinline__ bool jit_first_key_wanted(LaneAcc& acc, uint32_t slot,
                                                            uint32_t bl, uint32_t tl) {
  if (acc.first_key != ~0ull) return false;
  const volatile unsigned long long* fk = &s_T.slots[slot].first_key;
  const unsigned long long published = *fk;
  if (published > first_key_of(bl, tl, 0u)) return true;
  acc.first_key = published;
  return false;
}

// Number of in-bounds indices of a buffer of len bytes for accesses of
// width 2^lw, clamped to 2^31 (every int32 index below it is in bounds).
static __device__ __forceinline__ uint32_t jit_index_limit(int64_t len, uint32_t lw) {
  const uint64_t n = (uint64_t)len >> lw;
  return n < 0x80000000ull ? (uint32_t)n : 0x80000000u;
}

// Edge update for n hits of e per lane (a loop's repeated head edge), taken
// only when e is not yet saturated in this CTA's table: lanes with equal e
// are merged (__match_any_sync) and their leader adds the group's hits,
// clamped to 128 (counts only matter up to 128).  Out of line, one copy.
static __device__ __noinline__ void jit_cover_slow(uint32_t slot, uint32_t e, uint32_t n) {
  const uint32_t am = __activemask();
  const uint32_t peers = __match_any_sync(am, e);
  uint32_t c = __reduce_add_sync(peers, n < 128u ? n : 128u);
  if ((threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1)) {
    c = c < 128u ? c : 128u;
    const uint32_t tag = (e + 1u) << kHashTagShift;
    const uint32_t h = (e * 2654435761u) >> (32 - 11);
    if ((s_hash[h] & ~kHashCountMask) == tag)
      edge_hit(s_hash, h, e, c);
    else
      edge_add(s_hash, s_T, slot, e, c);
  }
}

// One hit of e by this lane, for an edge not yet saturated in this CTA's
// table: the lane adds its hit at the edge's home slot (inserting the edge
// there if the slot is empty), or probes on if another edge holds it.  No
// warp-level merging: on divergent branch-heavy code the few lanes that
// arrive together rarely share an edge, and merging them cost more than the
// atomics it saves.  Out of line, one copy for all sites.
static __device__ __noinline__ void jit_cover_lane(uint32_t slot, uint32_t e) {
  const uint32_t tag = (e + 1u) << kHashTagShift;
  const uint32_t h = (e * 2654435761u) >> (32 - 11);
  uint32_t v = s_hash[h];
  if (v == 0) {
    v = atomicCAS(&s_hash[h], 0u, tag | 1u);
    if (v == 0) return;
  }
  if ((v & ~kHashCountMask) == tag)
    edge_hit(s_hash, h, e, 1u);
  else
    edge_add(s_hash, s_T, slot, e, 1u);
}

// One hit of edge e: nothing to do once the edge is saturated in this CTA's
// table, the common case.
static __device__ __forceinline__ void jit_cover(uint32_t slot, uint32_t e) {
  if (!edge_saturated(s_hash, e)) jit_cover_lane(slot, e);
}

// jit_cover for an edge whose word w and bit b in the saturated-edge bitmap
// are known (e >> 5 and 1 << (e & 31), constants of the emitted code).
static __device__ __forceinline__ void jit_cover_k(uint32_t slot, uint32_t e, uint32_t w, uint32_t b) {
  if (!(s_hash[kHashSlots + w] & b)) jit_cover_lane(slot, e);
}

// jit_cover as one shared out-of-line copy, for programs compiled to compact
// code (many branch sites): a call at each site instead of the inline test.
static __device__ __noinline__ void jit_cover_out(uint32_t slot, uint32_t e) { jit_cover(slot, e); }

// Path counting (path-mode programs).  In a loop-free program a thread's
// edges and its counts of ops, accesses and branch evaluations follow from
// its path: the sites it evaluates and their outcomes.  The outcome bits po
// (bit s: site s took its then-arm) fix the path alone: which site comes
// after site s is a function of s and its outcome (the program's
// structure), so the sites evaluated need no bits of their own.  walk[s] =
// {LOC[s][0] | LOC[s][1] << 16, next[s][0] | next[s][1] << 8, seg[s][0],
// seg[s][1]}: for each outcome the site evaluated next (>= 64: none) and the
// counts a thread adds up to that evaluation (ops | accesses << 12 | branch
// evaluations << 24); a thread's counts start at the program's `init`.
// A thread adds its path to a per-CTA table of paths and counts; after its
// work item the CTA replays each distinct path once, adding its count to
// every edge of the path and its counts times that count, so threads on one
// path share one replay.  A path that finds no room in the table is replayed
// by its thread at once.  The table is the launch's dynamic shared memory
// (kPathTableBytes): the persistent kernel gets it when its module holds
// path-mode programs; the plain kernel (a CTA per test block) does not, and
// there every thread replays its own path (s_paths = 0).
#ifndef CUFZ_PATH_SLOTS_LOG2
#define CUFZ_PATH_SLOTS_LOG2 12
#endif
constexpr uint32_t kPathSlots = 1u << CUFZ_PATH_SLOTS_LOG2;
constexpr uint32_t kPathTableBytes = kPathSlots * 12u;
constexpr int kPathProbes = kPathSlots < 8u ? (int)kPathSlots : 8;
extern __shared__ __align__(16) unsigned char s_dyn[];
static __shared__ uint32_t s_paths;  // the CTA has a path table
static __device__ __forceinline__ unsigned long long* path_keys() {
  return reinterpret_cast<unsigned long long*>(s_dyn);  // path + 1, 0 = empty
}
static __device__ __forceinline__ uint32_t* path_counts() {
  return reinterpret_cast<uint32_t*>(s_dyn + kPathSlots * 8u);
}

// Counts of one or more threads: executed ops, accesses, branch evaluations.
struct PathCounts {
  uint32_t ops, acc, branch;
};

// n hits of edge e at once (n may differ between lanes, and be 0).
static __device__ __forceinline__ void jit_cover_n(uint32_t slot, uint32_t e, uint32_t n) {
  if (n != 0 && !edge_saturated(s_hash, e)) jit_cover_slow(slot, e, n);
}

// The edges of path (po1:po0), m threads on it, starting at site s; returns
// the path's packed counts (one thread's).  One shared out-of-line copy.
static __device__ __noinline__ uint32_t jit_path_walk(uint32_t slot, uint32_t po0, uint32_t po1,
                                                      uint32_t m, const uint4* __restrict__ walk,
                                                      uint32_t s, uint32_t init) {
  uint32_t prev = 0, cnt = init;
#pragma unroll 1
  while (s < 64u) {
    const uint4 w = walk[s];
    const uint32_t o = ((s < 32u ? po0 : po1) >> (s & 31u)) & 1u;
    const uint32_t cur = o ? (w.x >> 16) : (w.x & 0xFFFFu);
    if (m == 1u)  // one thread's path: a lane's own hit, no warp merging
      jit_cover(slot, (cur ^ prev) & 0xFFFFu);
    else
      jit_cover_n(slot, (cur ^ prev) & 0xFFFFu, m);
    prev = cur >> 1;
    cnt += o ? w.w : w.z;
    s = o ? (w.y >> 8) & 0xFFu : w.y & 0xFFu;
  }
  return cnt;
}

// Adds m threads of packed counts c.
static __device__ __forceinline__ void path_counts_add(PathCounts& t, uint32_t c, uint32_t m) {
  t.ops += m * (c & 0xFFFu);
  t.acc += m * ((c >> 12) & 0xFFFu);
  t.branch += m * (c >> 24);
}

// Empties the CTA's path table, if it has one; every thread of the CTA
// calls it.
static __device__ __forceinline__ void jit_path_clear() {
  if (!s_paths) return;
  unsigned long long* keys = path_keys();
  uint32_t* cnt = path_counts();
  for (uint32_t i = threadIdx.x; i < kPathSlots; i += blockDim.x) {
    keys[i] = 0ull;
    cnt[i] = 0u;
  }
  __syncthreads();
}

// Counts one thread on path (po1:po0) in the CTA's table; false when the
// CTA has no table or the path found no room (within kPathProbes slots of
// its home).
static __device__ __forceinline__ bool jit_path_count(uint32_t po0, uint32_t po1) {
  const unsigned long long key = (((unsigned long long)po1 << 32) | po0) + 1ull;
  if (!s_paths || key == 0ull) return false;  // key 0: every one of 64 sites taken
  unsigned long long* keys = path_keys();
  uint32_t* cnt = path_counts();
  uint32_t h = ((po0 * 0x9E3779B1u) ^ (po1 * 0x85EBCA77u)) >> (32 - CUFZ_PATH_SLOTS_LOG2);
#pragma unroll 1
  for (int p = 0; p < kPathProbes; p++) {
    unsigned long long k = keys[h];
    if (k == 0ull) {
      k = atomicCAS(&keys[h], 0ull, key);
      if (k == 0ull) k = key;
    }
    if (k == key) {
      atomicAdd(&cnt[h], 1u);
      return true;
    }
    h = (h + 1u) & (kPathSlots - 1u);
  }
  return false;
}

// Replays every path of the table with its count and returns the counts of
// the threads on the paths this CTA thread replayed; every thread of the CTA
// calls it, after its last thread of the work item.
static __device__ __noinline__ PathCounts jit_path_flush(uint32_t slot, const uint4* __restrict__ walk,
                                                         uint32_t first, uint32_t init) {
  PathCounts t{0u, 0u, 0u};
  if (!s_paths) return t;
  const unsigned long long* keys = path_keys();
  const uint32_t* cnt = path_counts();
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kPathSlots; i += blockDim.x) {
    const unsigned long long k = keys[i];
    if (k) {
      const unsigned long long po = k - 1ull;
      const uint32_t m = cnt[i];
      path_counts_add(t, jit_path_walk(slot, (uint32_t)po, (uint32_t)(po >> 32), m, walk, first, init), m);
    }
  }
  __syncthreads();
  return t;
}

// Edges of the head evaluations of one execution of a loop whose body has no
// branch sites: n_true taken evaluations, then one not taken if the loop ran
// to its end (not when the iteration budget stopped the thread inside it).
// Taken evaluations after the first all see prev = lt >> 1, so their edge is
// the same constant; three table updates replace n_true + 1.
static __device__ __forceinline__ void jit_loop_cover(uint32_t slot, uint32_t& prev, LaneAcc& acc,
                                                      uint32_t n_true, bool exited, uint32_t lt,
                                                      uint32_t lf) {
  acc.n_branch += n_true + (exited ? 1u : 0u);
  acc.n_folded += n_true > 1u ? n_true - 1u : 0u;
  const uint32_t p_in = prev;
  jit_cover_n(slot, (lt ^ p_in) & 0xFFFFu, n_true ? 1u : 0u);
  jit_cover_n(slot, (lt ^ (lt >> 1)) & 0xFFFFu, n_true ? n_true - 1u : 0u);
  const uint32_t p_exit = n_true ? (lt >> 1) : p_in;
  jit_cover_n(slot, (lf ^ p_exit) & 0xFFFFu, exited ? 1u : 0u);
  prev = exited ? (lf >> 1) : p_exit;
}

// A performed shared store of width w at p (in bounds): the value's four
// bytes little-endian, then zero bytes for widths 8 and 16.
static __device__ __forceinline__ void blk_store(uint8_t* p, int32_t v, uint32_t w) {
  const uint32_t u = (uint32_t)v;
#pragma unroll 1
  for (uint32_t k = 0; k < w; k++) p[k] = k < 4u ? (uint8_t)(u >> (8u * k)) : (uint8_t)0;
}

// A shared load of width w at p (in bounds): the byte, or the 32-bit word.
static __device__ __forceinline__ int32_t blk_load(const uint8_t* p, uint32_t w) {
  if (w == 1u) return (int32_t)p[0];
  return (int32_t)((uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
                   ((uint32_t)p[3] << 24));
}

// Seeded content of a global buffer (seedx = program seed ^ buf * 0x9E3779B9).
static __device__ __forceinline__ int32_t jit_content(uint32_t seedx, int64_t off, uint32_t lw) {
  const uint32_t word = mix32(seedx ^ (uint32_t)(off >> 2));
  return lw == 0 ? (int32_t)((word >> (8u * ((uint32_t)off & 3u))) & 0xFFu) : (int32_t)word;
}

// The same content for an in-bounds index ix of width 2^lw, from the 32-bit
// index: word (off >> 2) mod 2^32 is ix << (lw - 2) for lw >= 2 and ix >> 2
// for bytes (off = ix * 2^lw < 2^48), so no 64-bit offset is formed.
static __device__ __forceinline__ int32_t jit_content_ix(uint32_t seedx, int32_t ix, uint32_t lw) {
  const uint32_t u = (uint32_t)ix;
  if (lw == 0) return (int32_t)((mix32(seedx ^ (u >> 2)) >> (8u * (u & 3u))) & 0xFFu);
  return (int32_t)mix32(seedx ^ (u << (lw - 2u)));
}

// jit_content_ix as one shared out-of-line copy (compact code).
static __device__ __noinline__ int32_t jit_content_out(uint32_t seedx, int32_t ix, uint32_t lw) {
  return jit_content_ix(seedx, ix, lw);
}



}  // namespace cufz

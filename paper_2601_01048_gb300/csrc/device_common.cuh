// Device code shared by the bytecode interpreter (engine.cu) and by the
// programs compiled at load time (jit_kernel.cuh): hashing, division by launch
// dimensions, the per-CTA edge table, violation classification and records,
// the work-item loop and the per-input finalize.  Compiled both by nvcc and
// by the runtime compiler, so it includes nothing but the layouts.
#pragma once

#include "layout.h"

namespace cufz {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t kFlagEngineError = 0x80000000u;
constexpr uint32_t kHashCountMask = 0x7FFFu;
constexpr int kHashTagShift = 15;
constexpr uint32_t kInputSmemBytes = sizeof(DevInput);  // a CTA's staged input

static __device__ __forceinline__ uint32_t mix32(uint32_t h) {
  // MurmurHash3 fmix32 finalizer
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Digest of the accesses: each test thread folds its accesses, in program
// order, into h (starting at digest_start(block_lin, thread_lin)) with
// h = h * k + idx, k = access_k(site) = (site * 0xC2B2AE3D) | 3, one
// multiply-add per access; the input's digest is the sum over threads of
// digest_end(h) = h ^ (h >> 16), mod 2^64.  k is odd, so a step is a
// bijection of h (a changed index changes h); k - 1 is twice an odd number,
// so an added or dropped access changes h unless h * (k - 1) + idx is 0 mod
// 2^32; digest_end, a bijection that is not linear, binds each thread's h
// to its thread before the sum.
static __device__ __forceinline__ uint32_t digest_start(uint32_t bl, uint32_t tl) {
  return bl * 0x9E3779B1u + tl + 0x7F4A7C15u;
}
static __host__ __device__ __forceinline__ constexpr uint32_t access_k(uint32_t site) {
  return (site * 0xC2B2AE3Du) | 3u;
}
static __device__ __forceinline__ uint32_t access_step(uint32_t h, uint32_t k, int32_t idx) {
  return h * k + (uint32_t)idx;
}
static __device__ __forceinline__ uint32_t digest_end(uint32_t h) { return h ^ (h >> 16); }

// floor(n / d) for n < 2^32 with m = ceil(2^64 / d) (m == 0 means d == 1).
static __device__ __forceinline__ uint32_t udiv(uint32_t n, uint64_t m) {
  if (m == 0) return n;
  uint64_t t = (uint64_t)(uint32_t)m * n;
  uint64_t u = (uint64_t)(uint32_t)(m >> 32) * n + (t >> 32);
  return (uint32_t)(u >> 32);
}

static __device__ __forceinline__ uint32_t afl_bucket(uint32_t n) {
  if (n <= 2) return n;
  if (n == 3) return 4;
  if (n < 8) return 8;
  if (n < 16) return 16;
  if (n < 32) return 32;
  if (n < 128) return 64;
  return 128;
}

// Adds c hits of edge e to the slot's global counters, appending e to the
// touched list the first time it becomes nonzero.
static __device__ __forceinline__ void edge_global_add(const EngineTables& T, uint32_t slot, uint32_t e,
                                                uint32_t c) {
  uint32_t old = atomicAdd(&T.counts[(size_t)slot * kEdgeCount + e], c);
  if (old == 0) {
    uint32_t k = atomicAdd(&T.slots[slot].n_touched, 1u);
    T.touched[(size_t)slot * kEdgeCount + k] = (uint16_t)e;
  }
}

// The CTA's edge state in shared memory: a hash table of kHashSlots entries
// (e + 1) << 15 | count, followed by a bitmap of the edges whose count in
// the table reached 128 (their AFL bucket can no longer change, so later hits
// are skipped).  Counts saturate near 128: a count is added to only while it
// is below 128, by at most one add of <= 128 per warp or of 1 per thread at
// a time, so it stays below 127 + 1024 * 128 / 32 + 1024 < 2^15.
static __device__ __forceinline__ bool edge_saturated(const uint32_t* hash, uint32_t e) {
  return (hash[kHashSlots + (e >> 5)] >> (e & 31u)) & 1u;
}

static __device__ __forceinline__ void edge_hit(uint32_t* hash, uint32_t h, uint32_t e, uint32_t c) {
  const uint32_t cur = hash[h] & kHashCountMask;
  const uint32_t old = cur < 128u ? (atomicAdd(&hash[h], c) & kHashCountMask) : cur;
  if (old + c >= 128u) atomicOr(&hash[kHashSlots + (e >> 5)], 1u << (e & 31u));
}

static __device__ __noinline__ void edge_add(uint32_t* hash, const EngineTables& T, uint32_t slot,
                                      uint32_t e, uint32_t c) {
  uint32_t tag = (e + 1u) << kHashTagShift;
  uint32_t h = (e * 2654435761u) >> (32 - 11);
  static_assert(kHashSlots == 2048, "hash index uses 11 bits");
#pragma unroll 1
  for (int p = 0; p < kHashProbes; p++) {
    uint32_t cur = hash[h];
    if ((cur & ~kHashCountMask) == tag) {
      edge_hit(hash, h, e, c);
      return;
    }
    if (cur == 0) {
      uint32_t old = atomicCAS(&hash[h], 0u, tag | c);
      if (old == 0) return;
      if ((old & ~kHashCountMask) == tag) {
        edge_hit(hash, h, e, c);
        return;
      }
    }
    h = (h + 1) & (kHashSlots - 1);
  }
  edge_global_add(T, slot, e, c);
}

// Violation class from the virtual layout of the input's buffers.
static __device__ __noinline__ uint32_t classify(const DevInput* in, uint32_t shared_mask, uint32_t n_bufs,
                                          uint32_t buf, int64_t off, uint32_t w, int64_t R) {
  int64_t len = in->len[buf];
  if (off < 0 && off >= -R) return CUFZ_CLS_UNDERFLOW_RZ;
  if (off >= 0 && off < len + R) return CUFZ_CLS_OVERFLOW_RZ;
  uint32_t sp = (shared_mask >> buf) & 1u;
  int64_t a = in->base[buf] + off;
  for (uint32_t j = 0; j < n_bufs; j++) {
    if (j == buf || ((shared_mask >> j) & 1u) != sp) continue;
    int64_t lj = in->len[j];
    if (lj > 0 && a < in->base[j] + lj && a + (int64_t)w > in->base[j]) return CUFZ_CLS_OTHER_ALLOC;
  }
  return CUFZ_CLS_WILD;
}

static __device__ __forceinline__ void write_record(cufz_violation* dst, uint32_t bl, uint32_t tl,
                                             uint32_t ordinal, uint32_t site, uint32_t buf,
                                             uint32_t kind, uint32_t w, uint32_t space,
                                             uint32_t cls, int64_t off) {
  uint4 lo, hi;
  lo.x = bl;
  lo.y = tl;
  lo.z = ordinal;
  lo.w = site | (buf << 16) | (kind << 24);
  hi.x = w | (space << 8) | (cls << 16);
  hi.y = 0;
  hi.z = (uint32_t)(uint64_t)off;
  hi.w = (uint32_t)((uint64_t)off >> 32);
  uint4* d = reinterpret_cast<uint4*>(dst);
  d[0] = lo;
  d[1] = hi;
}

static __device__ __forceinline__ unsigned long long first_key_of(uint32_t bl, uint32_t tl,
                                                           uint32_t ordinal) {
  const uint32_t ord = ordinal < 0x3FFFFFu ? ordinal : 0x3FFFFFu;
  return ((unsigned long long)bl << 32) | ((unsigned long long)tl << 22) | ord;
}

// Per-lane accumulators of one work item, reduced per warp at its end.
struct LaneAcc {
  uint32_t n_acc;
  uint32_t n_branch;
  uint32_t n_ops;
  uint32_t n_viol;
  uint32_t n_folded;
  unsigned long long digest;
  unsigned long long first_key;
  bool budget_hit;
  bool rec_full;
};

static __device__ __forceinline__ void acc_init(LaneAcc& a) {
  a.n_acc = a.n_branch = a.n_ops = a.n_viol = a.n_folded = 0;
  a.digest = 0ull;
  a.first_key = ~0ull;
  a.budget_hit = false;
  a.rec_full = false;
}

// Warp-level reduction of the accumulators, one atomic per counter per warp.
// Every lane of the warp must call it.
static __device__ __forceinline__ void acc_flush(const EngineTables& T, uint32_t slot, const LaneAcc& a) {
  unsigned long long dig = a.digest;
  unsigned long long fk = a.first_key;
  uint32_t na = a.n_acc, nb = a.n_branch, no = a.n_ops, nv = a.n_viol, nf = a.n_folded;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    dig += __shfl_xor_sync(FULL, dig, s);
    unsigned long long o = __shfl_xor_sync(FULL, fk, s);
    fk = o < fk ? o : fk;
    na += __shfl_xor_sync(FULL, na, s);
    nb += __shfl_xor_sync(FULL, nb, s);
    no += __shfl_xor_sync(FULL, no, s);
    nv += __shfl_xor_sync(FULL, nv, s);
    nf += __shfl_xor_sync(FULL, nf, s);
  }
  const bool bh = __any_sync(FULL, a.budget_hit);
  if ((threadIdx.x & 31u) == 0) {
    SlotState* S = &T.slots[slot];
    if (na) atomicAdd(&S->n_accesses, (unsigned long long)na);
    if (dig) atomicAdd(&S->digest, dig);
    if (nb) atomicAdd(&S->n_branch, (unsigned long long)nb);
    if (no) atomicAdd(&S->n_ops, (unsigned long long)no);
    if (nv) atomicAdd(&S->n_violations, (unsigned long long)nv);
    if (nf) atomicAdd(&S->n_branch_folded, (unsigned long long)nf);
    if (fk != ~0ull) atomicMin(&S->first_key, fk);
    if (bh) atomicOr(&S->flags, (uint32_t)CUFZ_FL_BUDGET);
  }
}

// Last CTA of an input: bucket the touched edges into the bitmap, OR them
// into the union, compare with the epoch snapshot, publish the result.
// Every thread of the CTA must call it.
static __device__ __noinline__ void finalize_input(const EngineTables& T, const DevInput* in) {
  const uint32_t slot = in->slot;
  SlotState* S = &T.slots[slot];
  const uint32_t nt = *reinterpret_cast<volatile uint32_t*>(&S->n_touched);
  const bool keep = T.flags & CUFZ_CF_KEEP_BITMAPS;
  uint8_t* bm = T.bitmaps ? T.bitmaps + (size_t)slot * kBitmapBytes : nullptr;
  uint32_t* counts = T.counts + (size_t)slot * kEdgeCount;
  const uint16_t* touched = T.touched + (size_t)slot * kEdgeCount;
  if (keep) {
    uint4 z = make_uint4(0, 0, 0, 0);
    for (uint32_t i = threadIdx.x; i < kBitmapBytes / 16; i += blockDim.x)
      reinterpret_cast<uint4*>(bm)[i] = z;
  }
  __syncthreads();
  int newcov = 0;
  for (uint32_t k = threadIdx.x; k < nt; k += blockDim.x) {
    const uint32_t e = touched[k];
    const uint32_t c = counts[e];
    counts[e] = 0;
    const uint32_t b = afl_bucket(c);
    if (keep) bm[e] = (uint8_t)b;
    const uint32_t sh = (e & 3u) * 8u;
    const uint32_t snap = (T.union_snap[e >> 2] >> sh) & 0xFFu;
    if (b & ~snap) newcov = 1;
    atomicOr(&T.union_map[e >> 2], b << sh);
  }
  newcov = __syncthreads_or(newcov);
  if (threadIdx.x == 0) {
    volatile SlotState* vS = S;
    const unsigned long long nviol = vS->n_violations;
    const uint32_t reserved = vS->rec_reserved;
    HostDone* hd = &T.done[slot];
    cufz_result r;
    r.ticket = in->ticket;
    r.user_tag = in->user_tag;
    uint32_t flags = vS->flags;
    r.status = (flags & kFlagEngineError) ? CUFZ_E_DEVICE_FAULT
                                          : (nviol ? CUFZ_ST_VIOLATION : CUFZ_ST_OK);
    flags &= ~kFlagEngineError;
    if (nviol > T.record_cap) flags |= CUFZ_FL_OVERFLOW;
    if (newcov) flags |= CUFZ_FL_NEW_COV;
    r.flags = flags;
    r.n_accesses = vS->n_accesses;
    r.n_violations = nviol;
    r.first_key = vS->first_key;
    r.digest = vS->digest;
    r.n_branch = vS->n_branch;
    r.n_threads = in->n_threads;
    r.n_ops = vS->n_ops;
    r.n_records = reserved < T.record_cap ? reserved : T.record_cap;
    r.n_edges = nt;
    r.n_branch_folded = vS->n_branch_folded;
    // reset the slot for its next input
    vS->n_accesses = 0;
    vS->n_violations = 0;
    vS->digest = 0;
    vS->n_branch = 0;
    vS->n_ops = 0;
    vS->n_branch_folded = 0;
    vS->first_key = ~0ull;
    vS->rec_reserved = 0;
    vS->rec_listed = 0;
    vS->n_touched = 0;
    vS->items_done = 0;
    vS->flags = 0;
    const uint64_t* src = reinterpret_cast<const uint64_t*>(&r);
    volatile uint64_t* dst = reinterpret_cast<volatile uint64_t*>(&hd->res);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(cufz_result) / 8); k++) dst[k] = src[k];
    __threadfence_system();
    hd->seq = in->seq;
    __threadfence_system();
  }
}

// Runs work items until the batch is drained (persistent launch: CTAs pull
// items from the batch counter) or until the CTA's one test block is done
// (plain launch: CTA b runs block b of input `plain_input`).  `run(in, g0,
// count, skip)` executes the item's test threads with every thread of the CTA;
// with kStageProg the input's program blob is copied to `sprog` first.  After
// each item the CTA's edge table is flushed, and the CTA that completes an
// input's last item finalizes it.
template <bool kPersistent, bool kStageProg, class Run>
static __device__ __forceinline__ void run_items(const EngineTables& T, BatchHdr* batch,
                                          uint32_t plain_input, uint32_t max_regs,
                                          uint32_t max_prog_bytes, uint32_t* hash, uint8_t* sprog,
                                          DevInput* sin, Run&& run) {
  __shared__ uint32_t s_item, s_last, s_skip;
  const DevInput* inputs = reinterpret_cast<const DevInput*>(
      reinterpret_cast<const uint8_t*>(batch) + batch->inputs_off);
  const WorkItem* items = reinterpret_cast<const WorkItem*>(
      reinterpret_cast<const uint8_t*>(batch) + batch->items_off);
  const uint32_t n_items = kPersistent ? batch->n_items : 1u;

  for (uint32_t i = threadIdx.x; i < kHashSlots + kSatWords; i += blockDim.x) hash[i] = 0;
  if (threadIdx.x == 0) s_skip = 0;  // only the interpreter's staging sets it
  uint32_t cur_input = 0xFFFFFFFFu, cur_prog = 0xFFFFFFFFu;
  bool first = true;

  for (;;) {
    uint32_t in_idx, g0, cnt;
    if (kPersistent) {
      if (threadIdx.x == 0) s_item = atomicAdd(&batch->next_item, 1u);
      __syncthreads();
      const uint32_t it = s_item;
      if (it >= n_items) break;
      const WorkItem w = items[it];
      in_idx = w.input;
      g0 = w.g0;
      cnt = w.count;
    } else {
      if (!first) break;
      in_idx = plain_input;
      const uint32_t Tb = inputs[in_idx].T;
      g0 = blockIdx.x * Tb;
      cnt = Tb;
    }
    first = false;
    if (in_idx != cur_input) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&inputs[in_idx]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(sin);
      for (uint32_t i = threadIdx.x; i < sizeof(DevInput) / 4; i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      if (kStageProg) {  // the interpreter stages the input's program too
        if (threadIdx.x == 0) s_skip = sin->prog_bytes > max_prog_bytes ? 1u : 0u;
        __syncthreads();
        if (!s_skip && sin->prog_off != cur_prog) {
          const uint4* ps = reinterpret_cast<const uint4*>(T.progs + sin->prog_off);
          uint4* pd = reinterpret_cast<uint4*>(sprog);
          for (uint32_t i = threadIdx.x; i < sin->prog_bytes / 16; i += blockDim.x) pd[i] = ps[i];
          cur_prog = sin->prog_off;
        }
        __syncthreads();
        if (!s_skip && threadIdx.x == 0 &&
            reinterpret_cast<const DevProgHdr*>(sprog)->n_regs > max_regs)
          s_skip = 1;
        __syncthreads();
      }
      cur_input = in_idx;
    }
    const bool ran = run(sin, g0, cnt, s_skip != 0);
    if (!ran && threadIdx.x == 0) {
      atomicOr(&T.slots[sin->slot].flags, kFlagEngineError);
      atomicOr(&batch->error, 1u);
    }
    __syncthreads();
    // flush the CTA's edge table into the slot's counters
    const uint32_t slot = sin->slot;
    for (uint32_t i = threadIdx.x; i < kHashSlots; i += blockDim.x) {
      const uint32_t v = hash[i];
      if (v) {
        const uint32_t e = (v >> kHashTagShift) - 1u;
        const uint32_t c = v & kHashCountMask;
        edge_global_add(T, slot, e, c < 128u ? c : 128u);
        hash[i] = 0;
      }
    }
    for (uint32_t i = threadIdx.x; i < kSatWords; i += blockDim.x) hash[kHashSlots + i] = 0;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t done = atomicAdd(&T.slots[slot].items_done, 1u);
      s_last = (done + 1u == sin->n_items) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      finalize_input(T, sin);
    }
    __syncthreads();
  }
}

}  // namespace cufz

// Device-resident fuzzing campaign: the coverage-guided loop of AFL++ that
// drives the paper's translated kernels (Sec. 2.1, Sec. 4, Fig. 1), with its
// queue, corpus and bug buckets in device memory and every step of a round
// in kernels, so a round needs no host round trip:
//
//   select  one CTA sorts the corpus by (favoured first, least picked,
//           index) and takes `batch` parents round-robin from that order;
//           each parent's pick count grows and it stops being favoured;
//   mutate  child j is a copy of its parent mutated from its own
//           SplitMix64 stream (mutate.h: child_stream(seed, round, j));
//   build   one CTA turns the children into a batch of the engine: launch
//           checks, DevInputs (input_build.h) and work items, grouped by
//           program;
//   engine  the context's compiled persistent kernel runs the batch (checks,
//           coverage, finalize into the campaign's slots);
//   file    one CTA reads the children's results: children with new
//           coverage join the corpus as favoured entries (in child order);
//           violating ones are filed under (program, site, class) of their
//           first violation; hangs (the back-edge budget) with new coverage
//           are kept; the union's snapshot is renewed (the next round's
//           NEW_COV is measured against everything seen so far).
//
// The five launches are captured once as a CUDA graph; a round is one graph
// launch, and cufz_campaign_run enqueues any number of them.  The rules are
// those of the host campaign (paper_2601_01048_gb300/fuzz.py) with
// cufz_mutate_children, so both reach the same corpus, buckets, hangs and
// union from the same seeds.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "engine.h"
#include "mutate.h"

using namespace cufz;

namespace {

constexpr uint32_t kCampThreads = 1024;      // threads of the one-CTA kernels
constexpr uint32_t kCampMaxBatch = 8192;     // children per round
constexpr uint32_t kCampMaxCorpus = 16384;   // corpus entries (sort in shared memory)
constexpr uint32_t kCampMaxPrograms = 256;   // loaded programs of a context
constexpr uint64_t kCampAlign = 256;
constexpr int64_t kCampWaitUs = 120ll * 1000 * 1000;

uint64_t camp_align(uint64_t x) { return (x + kCampAlign - 1) / kCampAlign * kCampAlign; }
__host__ __device__ inline uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// Campaign state in device memory, 128 bytes.
struct CampHdr {
  uint32_t n_corpus, corpus_cap, batch, n_programs;
  uint32_t bucket_cap, n_buckets, hang_cap, n_hangs;
  uint32_t max_items, item_threads, redzone, record_cap;
  uint32_t corpus_dropped, buckets_dropped, hangs_dropped, limit_children;
  unsigned long long seed, round, executed, violating, hang_execs, new_coverage;
  unsigned long long max_threads;
  uint32_t pad[2];
};
static_assert(sizeof(CampHdr) == 128, "CampHdr size");
static_assert(sizeof(cufz_bucket) == 152, "cufz_bucket size");

struct DevHang {
  cufz_input input;
  unsigned long long round;
};

// Per program (4 words): bit 0 loaded, bits 8..15 buffers, bits 16..24
// shared mask, bit 31 block-serial; blob offset; blob bytes; 0.
constexpr uint32_t kProgWords = 4;

struct Layout {
  uint64_t hdr, corpus, fav, picks, parents, kids, kid_status, kid_slot, progs, buckets, hangs,
      batch, inputs, items, total;
};

Layout layout_of(const cufz_campaign_config& c) {
  Layout L{};
  uint64_t o = 0;
  auto take = [&](uint64_t bytes) {
    const uint64_t at = o;
    o = camp_align(o + bytes);
    return at;
  };
  L.hdr = take(sizeof(CampHdr));
  L.corpus = take((uint64_t)c.corpus_cap * sizeof(cufz_input));
  L.fav = take((uint64_t)c.corpus_cap * 4);
  L.picks = take((uint64_t)c.corpus_cap * 4);
  L.parents = take((uint64_t)c.batch * 4);
  L.kids = take((uint64_t)c.batch * sizeof(cufz_input));
  L.kid_status = take((uint64_t)c.batch * 4);
  L.kid_slot = take((uint64_t)c.batch * 4);
  L.progs = take((uint64_t)kCampMaxPrograms * kProgWords * 4);
  L.buckets = take((uint64_t)c.bucket_cap * sizeof(cufz_bucket));
  L.hangs = take((uint64_t)c.hang_cap * sizeof(DevHang));
  L.batch = take(sizeof(BatchHdr) + (uint64_t)c.batch * sizeof(DevInput) +
                 (uint64_t)c.max_items * sizeof(WorkItem));
  L.inputs = L.batch + sizeof(BatchHdr);
  L.items = L.inputs + (uint64_t)c.batch * sizeof(DevInput);
  L.total = o;
  return L;
}

// Exclusive prefix sum over the CTA's threads (every thread calls it);
// *total receives the sum.  Uses s_warp[32].
__device__ uint32_t block_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  __syncthreads();
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, d);
      if (lane >= (uint32_t)d) w += y;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  const uint32_t before = (warp ? s_warp[warp - 1] : 0u) + x - v;
  *total = s_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// ---------------------------------------------------------------- select
// One CTA: the corpus order (favoured first, least picked, lower index) by
// a bitonic sort of 64-bit keys in shared memory, the round's parents
// (that order, repeated), and the parents' pick counts and favoured flags.
__global__ void __launch_bounds__(kCampThreads) camp_select(CampHdr* H, uint32_t* fav,
                                                            uint32_t* picks, uint32_t* parents) {
  extern __shared__ unsigned long long s_keys[];
  const uint32_t n = H->n_corpus;
  uint32_t P = 1;
  while (P < n) P <<= 1;
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
    s_keys[i] = i < n ? ((unsigned long long)(fav[i] ? 0u : 1u) << 63) |
                            ((unsigned long long)picks[i] << 24) | i
                      : ~0ull;
  __syncthreads();
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
      for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint32_t l = i ^ jj;
        if (l > i) {
          const unsigned long long a = s_keys[i], b = s_keys[l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            s_keys[i] = b;
            s_keys[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  const uint32_t batch = H->batch;
  for (uint32_t j = threadIdx.x; j < batch; j += blockDim.x)
    parents[j] = (uint32_t)(s_keys[j % n] & 0xFFFFFFull);
  const uint32_t q = batch / n, r = batch % n;
  for (uint32_t p = threadIdx.x; p < n; p += blockDim.x) {
    const uint32_t idx = (uint32_t)(s_keys[p] & 0xFFFFFFull);
    const uint32_t cnt = q + (p < r ? 1u : 0u);
    if (cnt) {
      picks[idx] += cnt;
      fav[idx] = 0;
    }
  }
}

// ---------------------------------------------------------------- mutate
__global__ void camp_mutate(const CampHdr* H, const cufz_input* corpus, const uint32_t* parents,
                            cufz_input* kids, const uint32_t* progs) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= H->batch) return;
  cufz_input x = corpus[parents[j]];
  if (x.program_id < H->n_programs) {
    SplitMix64 r{child_stream(H->seed, H->round, j)};
    mutate_one(x, (progs[x.program_id * kProgWords] >> 8) & 0xFFu, r);
  }
  kids[j] = x;
}

// ---------------------------------------------------------------- build
__device__ int32_t camp_input_status(const CampHdr* H, const uint32_t* progs, const cufz_input& x) {
  if (x.program_id >= H->n_programs || !(progs[x.program_id * kProgWords] & 1u))
    return CUFZ_ST_BAD_PROGRAM;
  if (launch_rejected(x)) return CUFZ_ST_INVALID_CONFIG;
  if (!launch_within(x, H->max_threads, nullptr)) return CUFZ_ST_LIMIT;
  const uint32_t info = progs[x.program_id * kProgWords];
  const uint32_t nb = (info >> 8) & 0xFFu, sm = (info >> 16) & 0x1FFu;
  for (uint32_t k = 0; k < nb && k < (uint32_t)kMaxBufs; k++)
    if (x.buf_len[k] >= (1ull << 48)) return CUFZ_ST_LIMIT;
  if ((info >> 31) && !block_serial_fits(nb, sm, x)) return CUFZ_ST_LIMIT;
  return CUFZ_ST_OK;
}

// One CTA: statuses, work items (a child whose items would pass max_items,
// counting the children admitted before it in child order, completes as
// CUFZ_ST_LIMIT), DevInputs and the batch header.  Items are grouped by
// program, so CTAs running at the same time mostly run one program.
__global__ void __launch_bounds__(kCampThreads) camp_build(CampHdr* H, const cufz_input* kids,
                                                           int32_t* kid_status, const uint32_t* kid_slot,
                                                           const uint32_t* progs, BatchHdr* B,
                                                           DevInput* din, WorkItem* items) {
  __shared__ uint32_t s_items[kCampMaxBatch];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_pcount[kCampMaxPrograms], s_pcur[kCampMaxPrograms];
  __shared__ uint32_t s_total;
  __shared__ unsigned long long s_want;
  const uint32_t batch = H->batch;
  const uint32_t per = (batch + blockDim.x - 1) / blockDim.x;
  const uint32_t j0 = threadIdx.x * per;
  const uint64_t it0 = H->item_threads;
  for (uint32_t p = threadIdx.x; p < kCampMaxPrograms; p += blockDim.x) s_pcount[p] = 0;
  if (threadIdx.x == 0) s_want = 0;
  __syncthreads();
  unsigned long long mine = 0;
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t j = j0 + q;
    if (j >= batch) break;
    const cufz_input& x = kids[j];
    const int32_t st = camp_input_status(H, progs, x);
    uint32_t n_it = 0;
    if (st == CUFZ_ST_OK) {
      uint64_t nt = 0;
      launch_within(x, ~0ull, &nt);
      const uint64_t T = (uint64_t)x.block[0] * x.block[1] * x.block[2];
      const uint64_t it = (progs[x.program_id * kProgWords] >> 31) ? umax64(T, it0 / T * T) : it0;
      const uint64_t n = (nt + it - 1) / it;
      n_it = n > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)n;
    }
    kid_status[j] = st;
    s_items[j] = n_it;
    mine += n_it;
  }
  atomicAdd(&s_want, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    // admission by the batch's item capacity, in child order
    uint32_t limited = 0;
    if (s_want > H->max_items) {
      uint64_t used = 0;
      for (uint32_t j = 0; j < batch; j++) {
        if (!s_items[j]) continue;
        if (used + s_items[j] > H->max_items) {
          s_items[j] = 0;
          kid_status[j] = CUFZ_ST_LIMIT;
          limited++;
        } else {
          used += s_items[j];
        }
      }
    }
    H->limit_children += limited;
  }
  __syncthreads();
  // dense input index (child order) and per-program item counts
  uint32_t run = 0;
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t j = j0 + q;
    if (j >= batch) break;
    if (s_items[j]) {
      run++;
      atomicAdd(&s_pcount[kids[j].program_id], s_items[j]);
    }
  }
  uint32_t n_in = 0;
  uint32_t d = block_scan(run, s_warp, &n_in);
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (uint32_t p = 0; p < kCampMaxPrograms; p++) {
      s_pcur[p] = acc;
      acc += s_pcount[p];
    }
    s_total = acc;
  }
  __syncthreads();
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t j = j0 + q;
    if (j >= batch) break;
    const uint32_t n_it = s_items[j];
    if (!n_it) continue;
    const cufz_input& x = kids[j];
    const uint32_t p = x.program_id;
    const uint32_t info = progs[p * kProgWords];
    DevInput* D = &din[d];
    fill_dev_input(x, (info >> 8) & 0xFFu, (info >> 16) & 0x1FFu, H->redzone, D);
    D->slot = kid_slot[j];
    D->prog = p;
    D->prog_off = progs[p * kProgWords + 1];
    D->prog_bytes = progs[p * kProgWords + 2];
    D->n_items = n_it;
    D->ticket = (H->round << 32) | j;
    D->seq = 1;
    const uint64_t T = D->T;
    const uint64_t it = (info >> 31) ? umax64(T, it0 / T * T) : it0;
    const uint32_t off = atomicAdd(&s_pcur[p], n_it);
    for (uint32_t k = 0; k < n_it; k++) {
      WorkItem w;
      w.input = d;
      w.g0 = (uint32_t)(k * it);
      const uint64_t rem = D->n_threads - (uint64_t)k * it;
      w.count = (uint32_t)(rem < it ? rem : it);
      w.pad = 0;
      items[off + k] = w;
    }
    d++;
  }
  if (threadIdx.x == 0) {
    B->n_inputs = n_in;
    B->n_items = s_total;
    B->next_item = 0;
    B->epoch = 0;
    B->inputs_off = sizeof(BatchHdr);
    B->items_off = sizeof(BatchHdr) + (uint64_t)batch * sizeof(DevInput);
    B->error = 0;
  }
}

// ---------------------------------------------------------------- file
// The first violation a child's stored records hold: the record of least
// (block, thread, ordinal).
__device__ bool first_record(const cufz_violation* r, uint32_t n, uint32_t* site, uint32_t* cls) {
  if (!n) return false;
  unsigned long long best = ~0ull;
  uint32_t bo = ~0u, bs = 0, bc = 0;
  for (uint32_t i = 0; i < n; i++) {
    const unsigned long long k = ((unsigned long long)r[i].block_lin << 32) | r[i].thread_lin;
    if (k < best || (k == best && r[i].ordinal < bo)) {
      best = k;
      bo = r[i].ordinal;
      bs = r[i].site;
      bc = r[i].cls;
    }
  }
  *site = bs;
  *cls = bc;
  return true;
}

__global__ void __launch_bounds__(kCampThreads) camp_file(CampHdr* H, cufz_input* corpus, uint32_t* fav,
                                                          uint32_t* picks, const cufz_input* kids,
                                                          const int32_t* kid_status, const uint32_t* kid_slot,
                                                          EngineTables T, cufz_bucket* buckets,
                                                          DevHang* hangs) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_newb, s_dropb;
  const uint32_t batch = H->batch;
  const uint32_t per = (batch + blockDim.x - 1) / blockDim.x;
  const uint32_t j0 = threadIdx.x * per;
  const unsigned long long round = H->round;
  if (threadIdx.x == 0) s_newb = s_dropb = 0;
  // the children's outcomes (at most 8 per thread)
  uint32_t fl[kCampMaxBatch / kCampThreads];
  uint32_t n_new = 0, n_hang_new = 0, n_viol = 0, n_hang = 0;
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t j = j0 + q;
    uint32_t f = 0;
    if (j < batch && kid_status[j] == CUFZ_ST_OK) {
      const volatile HostDone* hd = &T.done[kid_slot[j]];
      const uint32_t flags = hd->res.flags;
      const int32_t status = hd->res.status;
      if (flags & CUFZ_FL_NEW_COV) f |= 1u;
      if (status == CUFZ_ST_VIOLATION) f |= 2u;
      if (flags & CUFZ_FL_BUDGET) f |= 4u;
    }
    fl[q] = f;
    n_new += f & 1u;
    n_viol += (f >> 1) & 1u;
    n_hang += (f >> 2) & 1u;
    n_hang_new += (f & 5u) == 5u;
  }
  __syncthreads();
  // corpus entries and unique hangs, in child order
  uint32_t tot_new = 0, tot_hang_new = 0, tot_viol = 0, tot_hang = 0;
  uint32_t at = block_scan(n_new, s_warp, &tot_new);
  uint32_t ah = block_scan(n_hang_new, s_warp, &tot_hang_new);
  block_scan(n_viol, s_warp, &tot_viol);
  block_scan(n_hang, s_warp, &tot_hang);
  const uint32_t nc = H->n_corpus, nh = H->n_hangs;
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t j = j0 + q;
    if (j >= batch) break;
    if (fl[q] & 1u) {
      const uint32_t i = nc + at++;
      if (i < H->corpus_cap) {
        corpus[i] = kids[j];
        fav[i] = 1;
        picks[i] = 0;
      }
    }
    if ((fl[q] & 5u) == 5u) {
      const uint32_t i = nh + ah++;
      if (i < H->hang_cap) {
        hangs[i].input = kids[j];
        hangs[i].round = round;
      }
    }
  }
  // bug buckets: key (program, site, class) of the first stored violation
  const uint32_t cap = H->bucket_cap;
  uint32_t my_slot[kCampMaxBatch / kCampThreads];
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t j = j0 + q;
    my_slot[q] = ~0u;
    if (j >= batch || !(fl[q] & 2u)) continue;
    const uint32_t slot = kid_slot[j];
    const uint32_t n_rec = T.done[slot].res.n_records;
    uint32_t site = 0xFFFFu, cls = 0xFFu;
    first_record(T.records + (size_t)slot * T.record_cap, n_rec < T.record_cap ? n_rec : T.record_cap,
                 &site, &cls);
    const unsigned long long key =
        (((unsigned long long)kids[j].program_id << 32) | (site << 8) | cls) + 1ull;
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 40) & (cap - 1);
    for (uint32_t p = 0; p < cap; p++) {
      unsigned long long k = buckets[h].key;
      if (k == 0ull) {
        k = atomicCAS(reinterpret_cast<unsigned long long*>(&buckets[h].key), 0ull, key);
        if (k == 0ull) {
          atomicAdd(&s_newb, 1u);
          k = key;
        }
      }
      if (k == key) {
        atomicAdd(&buckets[h].hits, 1u);
        atomicMin(reinterpret_cast<unsigned long long*>(&buckets[h].first), (round << 32) | j);
        my_slot[q] = h;
        break;
      }
      h = (h + 1u) & (cap - 1);
    }
    if (my_slot[q] == ~0u) atomicAdd(&s_dropb, 1u);
  }
  __syncthreads();
  // the bucket's representative: its first child
  for (uint32_t q = 0; q < per; q++) {
    const uint32_t j = j0 + q;
    if (j >= batch || my_slot[q] == ~0u) continue;
    cufz_bucket* b = &buckets[my_slot[q]];
    if (b->first == ((round << 32) | j)) b->input = kids[j];
  }
  // the union's snapshot: the next round's NEW_COV is against all seen so far
  for (uint32_t i = threadIdx.x; i < kEdgeCount / 4; i += blockDim.x) T.union_snap[i] = T.union_map[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t c_end = nc + tot_new;
    H->corpus_dropped += c_end > H->corpus_cap ? c_end - (nc > H->corpus_cap ? nc : H->corpus_cap) : 0u;
    H->n_corpus = c_end < H->corpus_cap ? c_end : H->corpus_cap;
    const uint32_t h_end = nh + tot_hang_new;
    H->hangs_dropped += h_end > H->hang_cap ? h_end - (nh > H->hang_cap ? nh : H->hang_cap) : 0u;
    H->n_hangs = h_end < H->hang_cap ? h_end : H->hang_cap;
    H->n_buckets += s_newb;
    H->buckets_dropped += s_dropb;
    H->executed += batch;
    H->violating += tot_viol;
    H->hang_execs += tot_hang;
    H->new_coverage += tot_new;
    H->round = round + 1;
  }
}

}  // namespace

struct cufz_campaign {
  cufz_ctx* ctx = nullptr;
  cufz_campaign_config cfg{};
  CampaignEnv env;
  uint8_t* mem = nullptr;
  Layout L{};
  cudaStream_t stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  uint32_t select_smem = 0;
};

namespace {

template <class T>
T* at(cufz_campaign* c, uint64_t off) {
  return reinterpret_cast<T*>(c->mem + off);
}

cufz_status camp_wait(cufz_campaign* c, int64_t limit_us) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(c->stream);
    if (e == cudaSuccess) return CUFZ_OK;
    if (e != cudaErrorNotReady) {
      cudaGetLastError();
      return CUFZ_E_CUDA;
    }
    const int64_t us = std::chrono::duration_cast<std::chrono::microseconds>(
                           std::chrono::steady_clock::now() - t0)
                           .count();
    if (limit_us >= 0 && us > limit_us) return CUFZ_E_TIMEOUT;
    std::this_thread::yield();
  }
}

bool config_ok(const cufz_campaign_config& c) {
  const bool pow2 = c.bucket_cap && (c.bucket_cap & (c.bucket_cap - 1)) == 0;
  return c.batch >= 1 && c.batch <= kCampMaxBatch && c.corpus_cap >= 1 &&
         c.corpus_cap <= kCampMaxCorpus && pow2 && c.bucket_cap >= 16 && c.bucket_cap <= (1u << 20) &&
         c.hang_cap >= 1 && c.hang_cap <= (1u << 20) && c.max_items >= 1 &&
         c.max_items <= (1u << 24);
}

cufz_campaign_config with_defaults(const cufz_campaign_config& in) {
  cufz_campaign_config c = in;
  if (!c.max_items) c.max_items = c.batch * 64u;
  return c;
}

// Captures the round: select, mutate, build, the engine's persistent
// kernel, file.
cufz_status camp_capture(cufz_campaign* c) {
  CampHdr* H = at<CampHdr>(c, c->L.hdr);
  cudaGraph_t g = nullptr;
  cudaGetLastError();
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  camp_select<<<1, kCampThreads, c->select_smem, c->stream>>>(H, at<uint32_t>(c, c->L.fav),
                                                                at<uint32_t>(c, c->L.picks),
                                                                at<uint32_t>(c, c->L.parents));
  camp_mutate<<<(c->cfg.batch + 255) / 256, 256, 0, c->stream>>>(
      H, at<cufz_input>(c, c->L.corpus), at<uint32_t>(c, c->L.parents), at<cufz_input>(c, c->L.kids),
      at<uint32_t>(c, c->L.progs));
  camp_build<<<1, kCampThreads, 0, c->stream>>>(
      H, at<cufz_input>(c, c->L.kids), at<int32_t>(c, c->L.kid_status), at<uint32_t>(c, c->L.kid_slot),
      at<uint32_t>(c, c->L.progs), at<BatchHdr>(c, c->L.batch), at<DevInput>(c, c->L.inputs),
      at<WorkItem>(c, c->L.items));
  EngineTables T = c->env.T;
  BatchHdr* B = at<BatchHdr>(c, c->L.batch);
  uint32_t paths = c->env.jit_smem ? 1u : 0u;
  void* args[] = {&T, &B, &paths};
  cudaError_t e1 = cudaLaunchKernel(c->env.jit_kernel, dim3(c->env.jit_ctas), dim3(c->env.cta_threads),
                                    args, c->env.jit_smem, c->stream);
  camp_file<<<1, kCampThreads, 0, c->stream>>>(
      H, at<cufz_input>(c, c->L.corpus), at<uint32_t>(c, c->L.fav), at<uint32_t>(c, c->L.picks),
      at<cufz_input>(c, c->L.kids), at<int32_t>(c, c->L.kid_status), at<uint32_t>(c, c->L.kid_slot), T,
      at<cufz_bucket>(c, c->L.buckets), at<DevHang>(c, c->L.hangs));
  cudaError_t e2 = cudaGetLastError();
  cudaError_t e3 = cudaStreamEndCapture(c->stream, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  cudaError_t e4 = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e4 != cudaSuccess) {
    cudaGetLastError();
    c->graph = nullptr;
    return CUFZ_E_CUDA;
  }
  return CUFZ_OK;
}

// Runs the seeds once through the context's ordinary path (AFL's dry run),
// then starts a new coverage epoch: the union holds the seeds' coverage.
cufz_status dry_run(cufz_ctx* ctx, const cufz_input* seeds, uint32_t n) {
  std::vector<cufz_result> got(256);
  uint32_t done = 0, sent = 0;
  const auto t0 = std::chrono::steady_clock::now();
  while (done < n) {
    if (sent < n) {
      uint32_t acc = 0;
      uint64_t first = 0;
      const cufz_status st = cufz_submit_inputs(ctx, seeds + sent, n - sent, &acc, &first);
      if (st != CUFZ_OK && st != CUFZ_E_BUSY) return st;
      sent += acc;
    }
    uint32_t k = 0;
    const cufz_status st = cufz_poll_results(ctx, got.data(), (uint32_t)got.size(), &k, 1000);
    if (st != CUFZ_OK && st != CUFZ_E_TIMEOUT) return st;
    for (uint32_t i = 0; i < k; i++) cufz_release(ctx, got[i].ticket);
    done += k;
    if (std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(kCampWaitUs))
      return CUFZ_E_TIMEOUT;
  }
  return cufz_new_epoch(ctx);
}

}  // namespace

extern "C" {

uint64_t cufz_campaign_bytes(const cufz_campaign_config* cfg) {
  if (!cfg) return 0;
  const cufz_campaign_config c = with_defaults(*cfg);
  if (!config_ok(c)) return 0;
  return layout_of(c).total;
}

cufz_status cufz_campaign_create(cufz_ctx* ctx, const cufz_campaign_config* cfg_in, void* dev_mem,
                                 uint64_t dev_bytes, const cufz_input* seeds, uint32_t n_seeds,
                                 cufz_campaign** out) {
  if (out) *out = nullptr;
  if (!ctx || !cfg_in || !dev_mem || !out || !seeds || !n_seeds) return CUFZ_E_INVALID_ARG;
  const cufz_campaign_config cfg = with_defaults(*cfg_in);
  if (!config_ok(cfg) || n_seeds > cfg.corpus_cap) return CUFZ_E_INVALID_ARG;
  const Layout L = layout_of(cfg);
  if (dev_bytes < L.total || (reinterpret_cast<uintptr_t>(dev_mem) & (kCampAlign - 1)))
    return CUFZ_E_INVALID_ARG;
  cufz_status st = dry_run(ctx, seeds, n_seeds);
  if (st != CUFZ_OK) return st;
  auto* c = new cufz_campaign();
  c->ctx = ctx;
  c->cfg = cfg;
  c->mem = static_cast<uint8_t*>(dev_mem);
  c->L = L;
  st = campaign_attach(ctx, cfg.batch, cfg.item_threads, &c->env);
  if (st != CUFZ_OK) {
    delete c;
    return st;
  }
  auto fail = [&](cufz_status s) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->stream) cudaStreamDestroy(c->stream);
    campaign_detach(ctx, c->env.slots);
    delete c;
    return s;
  };
  if (cudaSetDevice(c->env.device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return fail(CUFZ_E_CUDA);
  }
  if (c->env.n_programs > kCampMaxPrograms) return fail(CUFZ_E_INVALID_ARG);
  // initial state: header, corpus (the seeds, favoured), program table, slots
  std::vector<uint8_t> img(L.progs + kCampMaxPrograms * kProgWords * 4, 0);
  CampHdr H{};
  H.n_corpus = n_seeds;
  H.corpus_cap = cfg.corpus_cap;
  H.batch = cfg.batch;
  H.n_programs = c->env.n_programs;
  H.bucket_cap = cfg.bucket_cap;
  H.hang_cap = cfg.hang_cap;
  H.max_items = cfg.max_items;
  H.item_threads = c->env.item_threads;
  H.redzone = c->env.redzone;
  H.record_cap = c->env.T.record_cap;
  H.seed = cfg.seed;
  H.max_threads = c->env.max_threads;
  memcpy(img.data() + L.hdr, &H, sizeof(H));
  memcpy(img.data() + L.corpus, seeds, (size_t)n_seeds * sizeof(cufz_input));
  uint32_t* fav = reinterpret_cast<uint32_t*>(img.data() + L.fav);
  for (uint32_t i = 0; i < n_seeds; i++) fav[i] = 1;
  uint32_t* slot = reinterpret_cast<uint32_t*>(img.data() + L.kid_slot);
  for (uint32_t j = 0; j < cfg.batch; j++) slot[j] = c->env.slots[j];
  uint32_t* pt = reinterpret_cast<uint32_t*>(img.data() + L.progs);
  for (uint32_t p = 0; p < c->env.n_programs; p++)
    for (uint32_t w = 0; w < kProgWords; w++) pt[p * kProgWords + w] = c->env.progs[p * kProgWords + w];
  cudaError_t e = cudaMemcpyAsync(c->mem, img.data(), img.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->mem + L.buckets, 0, (size_t)cfg.bucket_cap * sizeof(cufz_bucket), c->stream);
  if (e == cudaSuccess) {
    // bucket.first starts at the largest (round, child)
    std::vector<cufz_bucket> b(cfg.bucket_cap);
    memset(b.data(), 0, b.size() * sizeof(cufz_bucket));
    for (auto& x : b) x.first = ~0ull;
    e = cudaMemcpyAsync(c->mem + L.buckets, b.data(), b.size() * sizeof(cufz_bucket),
                        cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CUFZ_E_CUDA);
  }
  uint32_t P = 1;
  while (P < cfg.corpus_cap) P <<= 1;
  c->select_smem = P * 8u;
  if (cudaFuncSetAttribute(camp_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)c->select_smem) != cudaSuccess) {
    cudaGetLastError();
    return fail(CUFZ_E_CUDA);
  }
  st = camp_capture(c);
  if (st != CUFZ_OK) return fail(st);
  *out = c;
  return CUFZ_OK;
}

cufz_status cufz_campaign_run(cufz_campaign* c, uint32_t rounds) {
  if (!c) return CUFZ_E_INVALID_ARG;
  if (!campaign_env_current(c->ctx, c->env)) return CUFZ_E_BUSY;
  if (cudaSetDevice(c->env.device) != cudaSuccess) return CUFZ_E_CUDA;
  for (uint32_t r = 0; r < rounds; r++)
    if (cudaGraphLaunch(c->graph, c->stream) != cudaSuccess) {
      cudaGetLastError();
      return CUFZ_E_CUDA;
    }
  return CUFZ_OK;
}

cufz_status cufz_campaign_sync(cufz_campaign* c, int32_t timeout_us) {
  if (!c) return CUFZ_E_INVALID_ARG;
  return camp_wait(c, timeout_us < 0 ? kCampWaitUs : timeout_us);
}

cufz_status cufz_campaign_get_stats(cufz_campaign* c, cufz_campaign_stats* out) {
  if (!c || !out) return CUFZ_E_INVALID_ARG;
  cufz_status st = camp_wait(c, kCampWaitUs);
  if (st != CUFZ_OK) return st;
  CampHdr H{};
  if (cudaMemcpy(&H, c->mem + c->L.hdr, sizeof(H), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  std::vector<uint32_t> picks(H.n_corpus);
  if (H.n_corpus && cudaMemcpy(picks.data(), c->mem + c->L.picks, H.n_corpus * 4ull,
                               cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  memset(out, 0, sizeof(*out));
  out->rounds = H.round;
  out->executed = H.executed;
  out->violating = H.violating;
  out->hang_execs = H.hang_execs;
  out->new_coverage = H.new_coverage;
  out->corpus = H.n_corpus;
  out->buckets = H.n_buckets;
  out->hangs = H.n_hangs;
  out->corpus_dropped = H.corpus_dropped;
  out->buckets_dropped = H.buckets_dropped;
  out->hangs_dropped = H.hangs_dropped;
  out->limit_children = H.limit_children;
  out->cycles_done = picks.empty() ? 0u : *std::min_element(picks.begin(), picks.end());
  return CUFZ_OK;
}

cufz_status cufz_campaign_corpus(cufz_campaign* c, cufz_input* out, uint8_t* favoured, uint32_t* picks,
                                 uint32_t cap, uint32_t* n) {
  if (!c || !n) return CUFZ_E_INVALID_ARG;
  cufz_status st = camp_wait(c, kCampWaitUs);
  if (st != CUFZ_OK) return st;
  CampHdr H{};
  if (cudaMemcpy(&H, c->mem + c->L.hdr, sizeof(H), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  *n = H.n_corpus;
  const uint32_t k = std::min(cap, H.n_corpus);
  std::vector<uint32_t> fav(k), pk(k);
  cudaError_t e = cudaSuccess;
  if (k && out) e = cudaMemcpy(out, c->mem + c->L.corpus, (size_t)k * sizeof(cufz_input), cudaMemcpyDeviceToHost);
  if (k && e == cudaSuccess) e = cudaMemcpy(fav.data(), c->mem + c->L.fav, k * 4ull, cudaMemcpyDeviceToHost);
  if (k && e == cudaSuccess) e = cudaMemcpy(pk.data(), c->mem + c->L.picks, k * 4ull, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  for (uint32_t i = 0; i < k; i++) {
    if (favoured) favoured[i] = fav[i] ? 1 : 0;
    if (picks) picks[i] = pk[i];
  }
  return CUFZ_OK;
}

cufz_status cufz_campaign_buckets(cufz_campaign* c, cufz_bucket* out, uint32_t cap, uint32_t* n) {
  if (!c || !n || (!out && cap)) return CUFZ_E_INVALID_ARG;
  cufz_status st = camp_wait(c, kCampWaitUs);
  if (st != CUFZ_OK) return st;
  std::vector<cufz_bucket> b(c->cfg.bucket_cap);
  if (cudaMemcpy(b.data(), c->mem + c->L.buckets, b.size() * sizeof(cufz_bucket),
                 cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  std::vector<cufz_bucket> used;
  for (auto& x : b)
    if (x.key) {
      x.key -= 1;  // stored + 1 so that 0 marks an empty entry
      used.push_back(x);
    }
  std::sort(used.begin(), used.end(),
            [](const cufz_bucket& a, const cufz_bucket& b2) { return a.key < b2.key; });
  *n = (uint32_t)used.size();
  std::copy_n(used.begin(), std::min<size_t>(cap, used.size()), out);
  return CUFZ_OK;
}

cufz_status cufz_campaign_hangs(cufz_campaign* c, cufz_input* out, uint64_t* rounds, uint32_t cap,
                                uint32_t* n) {
  if (!c || !n) return CUFZ_E_INVALID_ARG;
  cufz_status st = camp_wait(c, kCampWaitUs);
  if (st != CUFZ_OK) return st;
  CampHdr H{};
  if (cudaMemcpy(&H, c->mem + c->L.hdr, sizeof(H), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  *n = H.n_hangs;
  const uint32_t k = std::min(cap, H.n_hangs);
  std::vector<DevHang> h(k);
  if (k && cudaMemcpy(h.data(), c->mem + c->L.hangs, k * sizeof(DevHang), cudaMemcpyDeviceToHost) !=
               cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  for (uint32_t i = 0; i < k; i++) {
    if (out) out[i] = h[i].input;
    if (rounds) rounds[i] = h[i].round;
  }
  return CUFZ_OK;
}

cufz_status cufz_campaign_restore(cufz_campaign* c, const uint8_t* favoured, const uint32_t* picks,
                                  uint32_t n_corpus, const cufz_bucket* buckets, uint32_t n_buckets,
                                  const cufz_input* hangs, const uint64_t* hang_rounds, uint32_t n_hangs,
                                  const cufz_campaign_stats* counters) {
  if (!c || !counters || (n_corpus && (!favoured || !picks)) || (n_buckets && !buckets) ||
      (n_hangs && (!hangs || !hang_rounds)))
    return CUFZ_E_INVALID_ARG;
  cufz_status st = camp_wait(c, kCampWaitUs);
  if (st != CUFZ_OK) return st;
  CampHdr H{};
  if (cudaMemcpy(&H, c->mem + c->L.hdr, sizeof(H), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  if (n_corpus != H.n_corpus || n_hangs > H.hang_cap || n_buckets > H.bucket_cap / 2)
    return CUFZ_E_INVALID_ARG;
  std::vector<uint32_t> fav(n_corpus), pk(picks, picks + n_corpus);
  for (uint32_t i = 0; i < n_corpus; i++) fav[i] = favoured[i] ? 1u : 0u;
  std::vector<cufz_bucket> table(H.bucket_cap);
  memset(table.data(), 0, table.size() * sizeof(cufz_bucket));
  for (auto& x : table) x.first = ~0ull;
  for (uint32_t i = 0; i < n_buckets; i++) {
    const unsigned long long key = buckets[i].key + 1ull;
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 40) & (H.bucket_cap - 1);
    while (table[h].key) h = (h + 1u) & (H.bucket_cap - 1);
    table[h] = buckets[i];
    table[h].key = key;
  }
  std::vector<DevHang> hv(n_hangs);
  for (uint32_t i = 0; i < n_hangs; i++) {
    hv[i].input = hangs[i];
    hv[i].round = hang_rounds[i];
  }
  H.round = counters->rounds;
  H.executed = counters->executed;
  H.violating = counters->violating;
  H.hang_execs = counters->hang_execs;
  H.new_coverage = counters->new_coverage;
  H.n_buckets = n_buckets;
  H.n_hangs = n_hangs;
  H.corpus_dropped = counters->corpus_dropped;
  H.buckets_dropped = counters->buckets_dropped;
  H.hangs_dropped = counters->hangs_dropped;
  H.limit_children = counters->limit_children;
  cudaError_t e = cudaMemcpy(c->mem + c->L.hdr, &H, sizeof(H), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_corpus)
    e = cudaMemcpy(c->mem + c->L.fav, fav.data(), n_corpus * 4ull, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_corpus)
    e = cudaMemcpy(c->mem + c->L.picks, pk.data(), n_corpus * 4ull, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->mem + c->L.buckets, table.data(), table.size() * sizeof(cufz_bucket),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_hangs)
    e = cudaMemcpy(c->mem + c->L.hangs, hv.data(), hv.size() * sizeof(DevHang), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  return CUFZ_OK;
}

cufz_status cufz_campaign_destroy(cufz_campaign* c) {
  if (!c) return CUFZ_E_INVALID_ARG;
  const cufz_status st = camp_wait(c, kCampWaitUs);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->stream) cudaStreamDestroy(c->stream);
  campaign_detach(c->ctx, c->env.slots);
  delete c;
  return st;
}

}  // extern "C"

// Host runtime of cufz: context over a caller-owned arena, program table,
// admission by free slots, batches on overlapping pipeline lanes (each a
// stream with its own staging buffer and CUDA graph), completion polling
// through pinned mapped memory, and the C ABI of include/cufz.h.
//
// The runtime plays the part of the paper's CPU runtime library and fuzzing
// harness (Sec. 4: emulated cudaMalloc/cudaMemcpy and a thread pool that
// runs blocks; Sec. 2.1: the fuzzer feeds inputs and reads the coverage
// map), rebuilt around one GPU: inputs are admitted while earlier ones still
// run, and each input's work is split into block ranges that persistent
// CTAs pull from a device queue.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <deque>
#include <mutex>
#include <thread>
#include <tuple>
#include <future>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "jit_embed.h"  // generated at build time: header texts for the runtime compiler

using namespace cufz;

namespace {

constexpr uint32_t kMaxLanes = 8;
constexpr uint64_t kProgAreaBytes = 8ull << 20;
constexpr uint64_t kAlign = 256;
constexpr int64_t kWaitLimitUs = 120ll * 1000 * 1000;  // longest host-side wait
constexpr double kAutotuneMargin = 1.25;  // the other path must be 25% faster
constexpr uint64_t kAutotuneMinThreads = 1ull << 24;  // test threads timed per program and path
constexpr size_t kAutotuneMaxInputs = 2048;
// Lane mappings the autotuner tries (test threads per lane per iteration of
// a compiled program's work-item loop), for programs of at most this many
// kept ops; a wider mapping must be 3% faster to be kept.
constexpr uint32_t kLanesMaxOps = 24;
// Inputs of the sample the work-item size is timed on.
constexpr size_t kAutotuneItemInputs = 4096;
constexpr double kLanesMargin = 1.03;

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint64_t now_us() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::microseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct SlotHost {
  uint64_t ticket = 0;
  uint32_t seq = 0;
  int state = 0;  // 0 free, 1 in flight, 2 completed (held until release)
  uint32_t lane = 0;
  uint64_t batch = 0;
  uint32_t prog = 0;  // program of the input in the slot
  bool partial = false;  // PREX: only the planned threads run
};

struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  uint8_t* h_stage = nullptr;
  uint8_t* d_batch = nullptr;
  uint64_t cap = 0;
  bool busy = false;
  bool timed = false;
  uint64_t batch_id = 0;
  // one graph per kernel set a batch needs: bit 0 compiled, bit 1 interpreted
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    uint32_t regs = 0, prog = 0, ctas = 0, threads = 0, launches = 0;
    const void* kernel = nullptr;
  } graphs[4];
};

struct HostOnlyResult {
  cufz_result res;
};

}  // namespace

struct cufz_ctx {
  cufz_config cfg{};
  std::mutex mu;
  int device = 0;
  int n_sms = 0;
  uint8_t* arena = nullptr;
  EngineTables T{};
  uint8_t* d_progs = nullptr;
  uint64_t prog_used = 0;
  std::vector<LoadedProgram> progs;
  std::vector<uint32_t> prog_off;
  std::vector<uint8_t> prog_live;                          // 0 once unloaded
  std::vector<uint64_t> prog_key;                          // autotune-cache key of each program
  std::vector<std::vector<uint8_t>> prog_bytes;            // each program as loaded (unpruned)
  std::string tune_path;                                   // autotune cache file, if any
  // key -> the autotuner's choice: bit 0 compiled (1) or interpreted (0),
  // bits 1..3 the lane mapping (test threads per lane per loop iteration)
  std::unordered_map<uint64_t, uint8_t> tune_cache;
  // the autotuner's work-item size per set of loaded programs (key: the sum
  // of their cache keys), and the one in force (0: the size heuristic)
  std::unordered_map<uint64_t, uint32_t> tune_items;
  uint32_t tuned_item = 0;
  std::vector<std::pair<uint32_t, uint32_t>> prog_free;    // unloaded program-area ranges
  uint32_t max_regs = 1, max_prog_bytes = 16;
  uint32_t max_slots = 0;
  std::vector<SlotHost> slots;
  std::vector<uint32_t> free_slots;
  std::unordered_map<uint64_t, uint32_t> ticket_slot;
  std::unordered_map<uint64_t, cufz_result> host_done;  // tickets completed without device work
  std::deque<uint32_t> inflight;
  std::deque<cufz_result> ready;
  HostDone* done_h = nullptr;
  HostDone* done_d = nullptr;
  Lane lanes[kMaxLanes];
  uint32_t n_lanes = 1;
  uint32_t next_lane = 0;
  uint64_t next_ticket = 1;
  uint32_t next_seq = 1;
  uint64_t next_batch = 1;
  LaunchShape shape{};
  uint32_t smem_set = 0;
  uint32_t lane_max_inputs = 0, lane_max_items = 0;
  uint32_t* d_scratch_word = nullptr;
  cudaStream_t copy_stream = nullptr;
  cufz_stats stats{};
  // device intervals (ms after ev_ref) of the last retired batches, for the
  // overlap statistics: recorded when the stats are reset
  cudaEvent_t ev_ref = nullptr;
  bool ref_recorded = false;
  std::deque<std::pair<float, float>> recent;
  // compiled path
  std::vector<std::string> prog_src;  // CUDA source of each program's item function
  cudaLibrary_t jit_lib = nullptr;
  cudaKernel_t jit_persist = nullptr, jit_plain = nullptr;
  uint32_t jit_progs = 0;             // programs in the loaded module
  std::vector<uint8_t> prog_compiled; // per program: run compiled (1) or interpreted (0)
  std::vector<uint8_t> prog_in_module; // per program: its code is in the loaded module
  std::vector<uint8_t> prog_lanes;     // per program: lane mapping (1, 2 or 4)
  std::vector<uint8_t> lanes_in_module; // the lane mappings the loaded module was built with
  uint32_t jit_ctas_per_sm = 0;
  std::string jit_log;
  uint64_t module_gen = 0;   // compiled modules loaded so far
  uint32_t jit_smem = 0;     // dynamic shared memory of persistent launches (path table)
  uint32_t campaigns = 0;    // device campaigns attached
};

namespace {

// A lane's batch buffer: the compiled path's header, the interpreter's
// header, the inputs, the compiled path's items, the interpreter's items.
uint64_t lane_bytes(uint32_t max_inputs, uint32_t max_items) {
  return align_up(2 * sizeof(BatchHdr) + (uint64_t)max_inputs * sizeof(DevInput) +
                      (uint64_t)max_items * sizeof(WorkItem),
                  kAlign);
}

uint64_t fixed_bytes(const cufz_config& c, uint32_t n_slots, uint32_t* max_inputs,
                     uint32_t* max_items) {
  uint32_t lanes = std::max(1u, std::min(c.n_lanes, kMaxLanes));
  *max_inputs = std::max(1u, std::min(n_slots, 16384u));
  *max_items = c.lane_items ? std::min(c.lane_items, 1u << 24) : 1u << 20;
  return kProgAreaBytes + 2ull * kBitmapBytes + lanes * lane_bytes(*max_inputs, *max_items) + 4096;
}

uint64_t total_bytes(const cufz_config& c, uint32_t n_slots) {
  uint32_t mi, mt;
  uint64_t f = fixed_bytes(c, n_slots, &mi, &mt);
  // per-slot tables, each region 256-aligned
  uint64_t b = f;
  b += align_up((uint64_t)n_slots * sizeof(SlotState), kAlign);
  b += align_up((uint64_t)n_slots * 4ull * kEdgeCount, kAlign);
  b += align_up((uint64_t)n_slots * 2ull * kEdgeCount, kAlign);
  b += align_up((uint64_t)n_slots * c.record_cap * sizeof(cufz_violation), kAlign);
  if (c.flags & CUFZ_CF_KEEP_BITMAPS) b += align_up((uint64_t)n_slots * kBitmapBytes, kAlign);
  return b + 8 * kAlign;
}

cufz_status cuda_err(cudaError_t e) { return e == cudaSuccess ? CUFZ_OK : CUFZ_E_CUDA; }

void lane_reset_graph(Lane& L) {
  for (auto& G : L.graphs) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
}

// Accounts the finished batch of a lane (timing) and marks it free.
// Overlap of a retired batch's device interval [a, b) with the recent
// ones: pairs that intersect, and the most intervals that share a moment.
void note_interval(cufz_ctx* c, float a, float b) {
  constexpr size_t kRecent = 256;
  for (const auto& r : c->recent)
    if (r.first < b && a < r.second) c->stats.overlapping_batch_pairs++;
  c->recent.emplace_back(a, b);
  if (c->recent.size() > kRecent) c->recent.pop_front();
  // the most intervals containing one of the recent start points
  uint32_t most = 0;
  for (const auto& p : c->recent) {
    uint32_t k = 0;
    for (const auto& r : c->recent) k += (r.first <= p.first && p.first < r.second) ? 1u : 0u;
    most = std::max(most, k);
  }
  c->stats.max_concurrent_batches = std::max(c->stats.max_concurrent_batches, most);
}

void lane_retire(cufz_ctx* c, Lane& L) {
  if (!L.busy) return;
  if (L.timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, L.ev_start, L.ev_end) == cudaSuccess) c->stats.kernel_ms += ms;
    float a = 0.f, b = 0.f;
    if (c->ref_recorded && cudaEventElapsedTime(&a, c->ev_ref, L.ev_start) == cudaSuccess &&
        cudaEventElapsedTime(&b, c->ev_ref, L.ev_end) == cudaSuccess)
      note_interval(c, a, b);
    cudaGetLastError();
  }
  L.busy = false;
}

bool lane_done(Lane& L) {
  if (!L.busy) return true;
  return cudaEventQuery(L.ev_end) == cudaSuccess;
}

// Moves completed in-flight slots to the ready queue.
void harvest(cufz_ctx* c) {
  for (uint32_t k = 0; k < c->n_lanes; k++)
    if (c->lanes[k].busy && lane_done(c->lanes[k])) lane_retire(c, c->lanes[k]);
  size_t n = c->inflight.size();
  for (size_t i = 0; i < n; i++) {
    uint32_t s = c->inflight.front();
    c->inflight.pop_front();
    SlotHost& sh = c->slots[s];
    volatile HostDone* hd = &c->done_h[s];
    if (hd->seq == sh.seq) {
      std::atomic_thread_fence(std::memory_order_acquire);
      cufz_result r;
      memcpy(&r, const_cast<const cufz_result*>(&c->done_h[s].res), sizeof(r));
      if (sh.partial) r.flags |= CUFZ_FL_PARTIAL;
      c->ready.push_back(r);
      c->stats.inputs_completed++;
      if (c->cfg.flags & CUFZ_CF_AUTO_RELEASE) {
        c->ticket_slot.erase(sh.ticket);
        sh.state = 0;
        c->free_slots.push_back(s);
      } else {
        sh.state = 2;
      }
    } else {
      c->inflight.push_back(s);
    }
  }
}

uint32_t smem_for(const LaunchShape& s, uint32_t cta_threads) {
  LaunchShape t = s;
  t.cta_threads = cta_threads;
  return interp_smem_bytes(t);
}

// Sets the kernels' dynamic shared memory limit to what the persistent shape
// and the largest plain (one CTA per test block, up to 1024 threads) launch
// need, and derives the persistent grid from occupancy.
cufz_status ensure_smem(cufz_ctx* c) {
  const LaunchShape& s = c->shape;
  const uint32_t kSmemMax = 227u * 1024u;
  uint32_t bytes = smem_for(s, s.cta_threads);
  if (bytes > kSmemMax) return CUFZ_E_NOMEM;
  uint32_t attr = std::min(std::max(bytes, smem_for(s, 1024)), kSmemMax);
  if (attr != c->smem_set) {
    if (set_kernel_smem(attr) != cudaSuccess) return CUFZ_E_CUDA;
    c->smem_set = attr;
  }
  c->shape.smem_bytes = bytes;
  int occ = 0;
  if (persistent_occupancy(s.cta_threads, bytes, &occ) != cudaSuccess || occ < 1) return CUFZ_E_CUDA;
  uint32_t per_sm = c->cfg.ctas_per_sm ? std::min<uint32_t>(c->cfg.ctas_per_sm, occ) : (uint32_t)occ;
  c->shape.ctas = per_sm * (uint32_t)c->n_sms;
  c->stats.ctas_per_sm = per_sm;
  c->stats.smem_bytes = bytes;
  return CUFZ_OK;
}


bool use_jit(const cufz_ctx* c) { return (c->cfg.flags & CUFZ_CF_JIT) != 0; }

// Runtime-compiles the module to sm_103a code (no device needed).
cufz_status jit_nvrtc(const std::string& src, bool fast, std::vector<char>* cubin, std::string* log) {
  nvrtcProgram prog = nullptr;
  if (nvrtcCreateProgram(&prog, src.c_str(), "cufz_programs.cu", kJitHeaderCount, kJitHeaderText,
                         kJitHeaderName) != NVRTC_SUCCESS) {
    *log = "nvrtcCreateProgram failed\n";
    return CUFZ_E_CUDA;
  }
  const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "--diag-suppress=177,550,128",
                        "--Ofast-compile=min"};
  nvrtcResult rc = nvrtcCompileProgram(prog, fast ? 4 : 3, opts);
  size_t log_n = 0;
  nvrtcGetProgramLogSize(prog, &log_n);
  log->assign(log_n, '\0');
  if (log_n) nvrtcGetProgramLog(prog, &(*log)[0]);
  while (!log->empty() && log->back() == '\0') log->pop_back();
  if (rc != NVRTC_SUCCESS) {
    *log += std::string("nvrtc: ") + nvrtcGetErrorString(rc) + "\n";
    nvrtcDestroyProgram(&prog);
    return CUFZ_E_INVALID_PROGRAM;
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  cubin->resize(n);
  nvrtcGetCUBIN(prog, cubin->data());
  nvrtcDestroyProgram(&prog);
  return CUFZ_OK;
}

std::mutex g_jit_cache_mu;
std::unordered_map<std::string, std::vector<char>> g_jit_cache;  // module source -> image

// Compiled image of a module source, cached for the life of the process.
cufz_status jit_build_image(const std::vector<std::string>& prog_src,
                            const std::vector<uint8_t>& include, bool plain_kernel,
                            uint32_t min_ctas, uint32_t cta_threads, bool fast,
                            const std::vector<uint8_t>& lanes, std::vector<char>* image,
                            std::string* log) {
  const std::string src =
      jit_module_source(prog_src, include, plain_kernel, min_ctas, cta_threads, lanes) +
      (fast ? "//fast\n" : "");
  {
    std::lock_guard<std::mutex> g(g_jit_cache_mu);
    auto it = g_jit_cache.find(src);
    if (it != g_jit_cache.end()) {
      *image = it->second;
      log->clear();
      return CUFZ_OK;
    }
  }
  cufz_status st = jit_nvrtc(src, fast, image, log);
  if (st == CUFZ_OK) {
    std::lock_guard<std::mutex> g(g_jit_cache_mu);
    g_jit_cache[src] = *image;
  }
  return st;
}

// Compiles every loaded program into one module and loads it; the
// persistent and plain kernels of the compiled path come from it.
bool jit_current(const cufz_ctx* c) {
  if (!c->jit_lib || c->prog_in_module.size() != c->progs.size()) return false;
  if (c->lanes_in_module.size() != c->progs.size()) return false;
  for (size_t k = 0; k < c->progs.size(); k++)
    if (c->prog_compiled[k] && (!c->prog_in_module[k] || c->lanes_in_module[k] != c->prog_lanes[k]))
      return false;
  return true;
}

cufz_status jit_compile(cufz_ctx* c) {
  if (jit_current(c)) return CUFZ_OK;
  if (c->campaigns) return CUFZ_E_BUSY;  // a campaign's captured rounds run this module
  std::vector<char> cubin;
  const bool plain = (c->cfg.flags & CUFZ_CF_PLAIN_LAUNCH) != 0;
  std::vector<uint8_t> include = c->prog_compiled;
  cufz_status cs = jit_build_image(c->prog_src, include, plain, c->cfg.jit_min_ctas,
                                   c->shape.cta_threads, (c->cfg.flags & CUFZ_CF_JIT_FAST_COMPILE) != 0,
                                   c->prog_lanes, &cubin, &c->jit_log);
  if (cs != CUFZ_OK) return cs;
  // wait for work that may still run on the old module
  for (uint32_t k = 0; k < c->n_lanes; k++) {
    Lane& L = c->lanes[k];
    if (L.busy) cudaEventSynchronize(L.ev_end);
    lane_retire(c, L);
    lane_reset_graph(L);
  }
  if (c->jit_lib) cudaLibraryUnload(c->jit_lib);
  c->jit_lib = nullptr;
  cudaError_t e = cudaLibraryLoadData(&c->jit_lib, cubin.data(), nullptr, nullptr, 0, nullptr,
                                      nullptr, 0);
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&c->jit_persist, c->jit_lib, "cufz_jit_persistent");
  if (e == cudaSuccess && plain) e = cudaLibraryGetKernel(&c->jit_plain, c->jit_lib, "cufz_jit_plain");
  // a module with path-mode programs gives persistent CTAs a path table
  uint32_t smem = 0;
  for (size_t k = 0; k < c->prog_src.size(); k++)
    if (include[k] && c->prog_src[k].find("jit_path_count(") != std::string::npos) smem = kJitPathTableBytes;
  if (e == cudaSuccess && smem)
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(c->jit_persist),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, reinterpret_cast<const void*>(c->jit_persist), (int)c->shape.cta_threads, smem);
  if (e != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  c->jit_ctas_per_sm = c->cfg.ctas_per_sm ? std::min<uint32_t>(c->cfg.ctas_per_sm, occ) : (uint32_t)occ;
  c->jit_progs = (uint32_t)c->progs.size();
  c->jit_smem = smem;
  c->module_gen++;
  c->prog_in_module = include;
  c->lanes_in_module = c->prog_lanes;
  return CUFZ_OK;
}

cudaError_t launch_jit_persistent(cufz_ctx* c, const BatchHdr* d_batch, uint32_t ctas, cudaStream_t st) {
  EngineTables T = c->T;
  BatchHdr* b = const_cast<BatchHdr*>(d_batch);
  uint32_t paths = c->jit_smem ? 1u : 0u;
  void* args[] = {&T, &b, &paths};
  return cudaLaunchKernel(reinterpret_cast<const void*>(c->jit_persist), dim3(ctas), dim3(c->shape.cta_threads),
                          args, c->jit_smem, st);
}

cudaError_t launch_jit_plain(cufz_ctx* c, const BatchHdr* d_batch, uint32_t input, uint32_t blocks,
                             uint32_t threads, cudaStream_t st) {
  EngineTables T = c->T;
  BatchHdr* b = const_cast<BatchHdr*>(d_batch);
  void* args[] = {&T, &b, &input};
  return cudaLaunchKernel(reinterpret_cast<const void*>(c->jit_plain), dim3(blocks), dim3(threads),
                          args, 0, st);
}

uint32_t interp_ctas(const cufz_ctx* c) { return c->shape.ctas; }
uint32_t jit_ctas(const cufz_ctx* c) { return c->jit_ctas_per_sm * (uint32_t)c->n_sms; }
bool has_jit_kernel(const cufz_ctx* c) { return use_jit(c) && c->jit_persist; }

const BatchHdr* jit_hdr(const Lane& L) { return reinterpret_cast<const BatchHdr*>(L.d_batch); }
const BatchHdr* interp_hdr(const Lane& L) {
  return reinterpret_cast<const BatchHdr*>(L.d_batch + sizeof(BatchHdr));
}

// The persistent launches of one batch: the compiled programs' items, then
// the interpreted programs' items (an empty list costs one short launch).
// Launches the persistent kernels of a batch: the compiled programs' items
// (if n_jit) and the interpreted programs' items (if n_int).  With `all`
// (graph capture) each runs on its full grid, for any batch with items of
// that kind.
cudaError_t launch_batch_kernels(cufz_ctx* c, const Lane& L, uint32_t n_jit, uint32_t n_int,
                                 bool all, cudaStream_t st, uint32_t* launches) {
  cudaError_t e = cudaSuccess;
  if (has_jit_kernel(c) && n_jit) {
    uint32_t ctas = all ? jit_ctas(c) : std::min<uint32_t>(jit_ctas(c), n_jit);
    e = launch_jit_persistent(c, jit_hdr(L), ctas, st);
    if (e == cudaSuccess) (*launches)++;
  }
  if (e == cudaSuccess && n_int) {
    LaunchShape s = c->shape;
    s.ctas = all ? interp_ctas(c) : std::min<uint32_t>(interp_ctas(c), n_int);
    e = launch_persistent(c->T, interp_hdr(L), s, st);
    if (e == cudaSuccess) (*launches)++;
  }
  return e;
}

// Captures (or re-captures) the lane's graph for the kernel set `mask` of a
// batch (bit 0: compiled programs' items, bit 1: interpreted programs'
// items), so that a batch launches only the kernels it has items for.
cufz_status lane_graph(cufz_ctx* c, Lane& L, uint32_t mask) {
  const LaunchShape& s = c->shape;
  const uint32_t ctas = interp_ctas(c) ^ (has_jit_kernel(c) ? jit_ctas(c) << 16 : 0);
  const void* kern = has_jit_kernel(c) ? reinterpret_cast<const void*>(c->jit_persist) : nullptr;
  Lane::Graph& G = L.graphs[mask & 3u];
  if (G.exec && G.regs == s.max_regs && G.prog == s.max_prog_bytes && G.ctas == ctas &&
      G.threads == s.cta_threads && G.kernel == kern)
    return CUFZ_OK;
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G.exec = nullptr;
  cudaGraph_t g = nullptr;
  cudaGetLastError();  // a stale error must not be taken for the capture's
  cudaError_t e0 = cudaStreamBeginCapture(L.stream, cudaStreamCaptureModeThreadLocal);
  if (e0 != cudaSuccess) {
    c->stats.last_cuda_error = 70000 + (int32_t)e0;
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  uint32_t nl = 0;
  cudaError_t e1 = cudaSuccess;
  cudaError_t e2 = launch_batch_kernels(c, L, mask & 1u, mask & 2u, true, L.stream, &nl);
  cudaError_t e3 = cudaStreamEndCapture(L.stream, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    c->stats.last_cuda_error = e1 != cudaSuccess ? 10000 + (int32_t)e1
                             : e2 != cudaSuccess ? 20000 + (int32_t)e2
                                                 : 30000 + (int32_t)e3;
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  cudaError_t e4 = cudaGraphInstantiate(&G.exec, g, 0);
  cudaGraphDestroy(g);
  if (e4 != cudaSuccess) {
    c->stats.last_cuda_error = 40000 + (int32_t)e4;
    cudaGetLastError();
    G.exec = nullptr;
    return CUFZ_E_CUDA;
  }
  G.regs = s.max_regs;
  G.prog = s.max_prog_bytes;
  G.ctas = ctas;
  G.threads = s.cta_threads;
  G.kernel = kern;
  G.launches = nl;
  return CUFZ_OK;
}

void build_dev_input(cufz_ctx* c, const cufz_input& in, uint32_t slot, DevInput* d) {
  const LoadedProgram& P = c->progs[in.program_id];
  fill_dev_input(in, P.n_bufs, P.shared_mask, c->cfg.redzone, d);
  d->slot = slot;
  d->prog = in.program_id;
  d->prog_off = c->prog_off[in.program_id];
  d->prog_bytes = P.blob_bytes;
}

// Autotune cache: one "key path lanes" line per program, the key a 64-bit
// FNV-1a hash of the program's bytes and of the kernel shape it was tuned
// for (files of the first version hold "key path" lines: lanes 1).
uint64_t tune_key(const cufz_ctx* c, const void* bytes, size_t n) {
  uint64_t h = 0xCBF29CE484222325ull;
  auto mix = [&](uint8_t b) { h = (h ^ b) * 0x100000001B3ull; };
  const uint8_t* p = static_cast<const uint8_t*>(bytes);
  for (size_t i = 0; i < n; i++) mix(p[i]);
  const uint32_t shape[3] = {c->cfg.cta_threads, c->cfg.jit_min_ctas, c->cfg.flags & (CUFZ_CF_NO_PRUNE | CUFZ_CF_NO_DIGEST)};
  for (uint32_t v : shape)
    for (int k = 0; k < 4; k++) mix((uint8_t)(v >> (8 * k)));
  return h;
}

bool lanes_ok(uint32_t k) { return k == 1 || k == 2 || k == 4; }

// The key of the loaded program set for the work-item size: the sum of the
// live programs' cache keys (independent of load order).
uint64_t workload_key(const cufz_ctx* c) {
  uint64_t k = 0;
  for (size_t p = 0; p < c->progs.size(); p++)
    if (c->prog_live[p]) k += c->prog_key[p];
  return k;
}

// Applies the cached work-item size of the loaded program set, if any.
void apply_tuned_item(cufz_ctx* c) {
  const auto it = c->tune_items.find(workload_key(c));
  c->tuned_item = it == c->tune_items.end() ? 0u : it->second;
}
uint8_t tune_value(bool compiled, uint32_t lanes) {
  return (uint8_t)((compiled ? 1u : 0u) | (lanes << 1));
}
uint32_t tune_lanes(uint8_t v) { return lanes_ok(v >> 1) ? (uint32_t)(v >> 1) : 1u; }

void tune_cache_read(cufz_ctx* c) {
  if (c->tune_path.empty()) return;
  FILE* f = fopen(c->tune_path.c_str(), "r");
  if (!f) return;  // no cache yet
  char line[128];
  if (fgets(line, sizeof line, f)) {
    const bool v1 = strncmp(line, "cufz-autotune 1", 15) == 0;
    const bool v2 = strncmp(line, "cufz-autotune 2", 15) == 0;
    unsigned long long key = 0;
    unsigned path = 0, lanes = 1;
    while ((v1 || v2) && fgets(line, sizeof line, f)) {
      lanes = 1;
      unsigned items = 0;
      if (sscanf(line, "item %16llx %u", &key, &items) == 2) {
        if (items && items % 32 == 0) c->tune_items[(uint64_t)key] = items;
        continue;
      }
      const int got = sscanf(line, "%16llx %u %u", &key, &path, &lanes);
      if (got < 2) break;
      c->tune_cache[(uint64_t)key] = tune_value(path != 0, lanes_ok(lanes) ? lanes : 1u);
    }
  }
  fclose(f);
}

// Rewrites the cache (through a temporary file and a rename, so a reader
// never sees half a file).  False if the file could not be written.
bool tune_cache_write(const cufz_ctx* c) {
  if (c->tune_path.empty()) return true;
  const std::string tmp = c->tune_path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return false;
  bool ok = fprintf(f, "cufz-autotune 2\n") > 0;
  for (const auto& kv : c->tune_cache)
    ok = ok && fprintf(f, "%016llx %u %u\n", (unsigned long long)kv.first, kv.second & 1u,
                       (unsigned)tune_lanes(kv.second)) > 0;
  for (const auto& kv : c->tune_items)
    ok = ok && fprintf(f, "item %016llx %u\n", (unsigned long long)kv.first, kv.second) > 0;
  ok = (fclose(f) == 0) && ok;
  return ok && rename(tmp.c_str(), c->tune_path.c_str()) == 0;
}

// The status an input completes with at once (anything but OK), or OK
// when it needs device work.
int32_t input_status(const cufz_ctx* c, const cufz_input& x) {
  if (x.program_id >= c->progs.size() || !c->prog_live[x.program_id]) return CUFZ_ST_BAD_PROGRAM;
  if (launch_rejected(x)) return CUFZ_ST_INVALID_CONFIG;
  if (!launch_within(x, c->cfg.max_threads, nullptr)) return CUFZ_ST_LIMIT;
  const LoadedProgram& P = c->progs[x.program_id];
  for (uint32_t k = 0; k < P.n_bufs; k++)
    if (x.buf_len[k] >= (1ull << 48)) return CUFZ_ST_LIMIT;
  if (P.block_serial && !block_serial_fits(P.n_bufs, P.shared_mask, x)) return CUFZ_ST_LIMIT;
  return CUFZ_ST_OK;
}

uint32_t choose_item_threads(cufz_ctx* c, uint64_t batch_threads) {
  if (c->cfg.item_threads) return c->cfg.item_threads;
  if (c->tuned_item) return c->tuned_item;
  uint32_t cta = c->shape.cta_threads;
  uint64_t target = batch_threads / (8ull * std::max(std::max(interp_ctas(c), jit_ctas(c)), 1u));
  uint64_t lo = 2ull * cta, hi = 256ull * cta;
  target = std::min(std::max(target, lo), hi);
  return (uint32_t)align_up(target, 32);
}

}  // namespace

// ---------------------------------------------------------------- ABI

extern "C" {

void cufz_config_default(cufz_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->flags = CUFZ_CF_KEEP_BITMAPS;
  cfg->record_cap = 4096;
  cfg->redzone = 256;
  cfg->iter_budget = 4096;
  cfg->max_threads = 1ull << 31;
  cfg->cta_threads = 256;
  cfg->n_lanes = 4;
}

uint64_t cufz_arena_bytes(const cufz_config* cfg, uint32_t n_slots) {
  if (!cfg || !n_slots) return 0;
  return total_bytes(*cfg, n_slots);
}

const char* cufz_status_str(cufz_status s) {
  switch (s) {
    case CUFZ_OK: return "ok";
    case CUFZ_E_INVALID_ARG: return "invalid argument";
    case CUFZ_E_INVALID_PROGRAM: return "invalid program";
    case CUFZ_E_NOMEM: return "out of arena memory or table space";
    case CUFZ_E_BUSY: return "busy: no free slot or lane";
    case CUFZ_E_TIMEOUT: return "timeout";
    case CUFZ_E_CUDA: return "CUDA error";
    case CUFZ_E_NOT_FOUND: return "not found";
    case CUFZ_E_NO_DEVICE: return "no CUDA device";
    case CUFZ_E_DEVICE_FAULT: return "device reported an engine error";
    case CUFZ_E_IO: return "autotune cache file could not be written";
    case CUFZ_E_UNSUPPORTED: return "a shared-memory value that stores set reaches a check";
    default: return "unknown status";
  }
}

cufz_status cufz_create(const cufz_config* cfg_in, cufz_ctx** out) {
  if (!cfg_in || !out) return CUFZ_E_INVALID_ARG;
  *out = nullptr;
  cufz_config cfg = *cfg_in;
  if (!cfg.arena || (reinterpret_cast<uintptr_t>(cfg.arena) & (kAlign - 1))) return CUFZ_E_INVALID_ARG;
  if (!cfg.record_cap) cfg.record_cap = 1;
  if (!cfg.cta_threads) cfg.cta_threads = 256;
  if (cfg.cta_threads < 64 || cfg.cta_threads > 1024 || cfg.cta_threads % 32) return CUFZ_E_INVALID_ARG;
  if (cfg.item_threads % 32) return CUFZ_E_INVALID_ARG;
  if (!cfg.max_threads || cfg.max_threads > (1ull << 31)) cfg.max_threads = 1ull << 31;
  if (cfg.redzone > (1u << 20)) return CUFZ_E_INVALID_ARG;
  cfg.n_lanes = std::max(1u, std::min(cfg.n_lanes, kMaxLanes));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= cfg.device || cfg.device < 0) {
    cudaGetLastError();
    return CUFZ_E_NO_DEVICE;
  }
  if (cudaSetDevice(cfg.device) != cudaSuccess) return CUFZ_E_NO_DEVICE;
  uint32_t n_slots = cfg.max_slots;
  if (!n_slots) {
    // as many as fit, up to 16384
    uint32_t lo = 1, hi = 16384;
    if (total_bytes(cfg, 1) > cfg.arena_bytes) return CUFZ_E_NOMEM;
    while (lo < hi) {
      uint32_t mid = lo + (hi - lo + 1) / 2;
      if (total_bytes(cfg, mid) <= cfg.arena_bytes) lo = mid; else hi = mid - 1;
    }
    n_slots = lo;
  }
  if (total_bytes(cfg, n_slots) > cfg.arena_bytes) return CUFZ_E_NOMEM;
  cufz_ctx* c = new cufz_ctx();
  c->cfg = cfg;
  if (cfg.autotune_cache) c->tune_path = cfg.autotune_cache;
  c->cfg.autotune_cache = nullptr;  // the caller's string need not outlive the call
  tune_cache_read(c);
  c->device = cfg.device;
  cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, cfg.device);
  c->arena = reinterpret_cast<uint8_t*>(cfg.arena);
  c->max_slots = n_slots;
  c->n_lanes = cfg.n_lanes;
  // carve the arena
  uint64_t off = 0;
  auto take = [&](uint64_t bytes) {
    uint8_t* p = c->arena + off;
    off = align_up(off + bytes, kAlign);
    return p;
  };
  uint32_t max_inputs, max_items;
  fixed_bytes(cfg, n_slots, &max_inputs, &max_items);
  c->lane_max_inputs = max_inputs;
  c->lane_max_items = max_items;
  c->d_progs = take(kProgAreaBytes);
  c->T.progs = c->d_progs;
  c->T.union_map = reinterpret_cast<uint32_t*>(take(kBitmapBytes));
  c->T.union_snap = reinterpret_cast<uint32_t*>(take(kBitmapBytes));
  c->d_scratch_word = reinterpret_cast<uint32_t*>(take(4096));
  for (uint32_t k = 0; k < c->n_lanes; k++) {
    c->lanes[k].cap = lane_bytes(max_inputs, max_items);
    c->lanes[k].d_batch = take(c->lanes[k].cap);
  }
  c->T.slots = reinterpret_cast<SlotState*>(take((uint64_t)n_slots * sizeof(SlotState)));
  c->T.counts = reinterpret_cast<uint32_t*>(take((uint64_t)n_slots * 4ull * kEdgeCount));
  c->T.touched = reinterpret_cast<uint16_t*>(take((uint64_t)n_slots * 2ull * kEdgeCount));
  c->T.records = reinterpret_cast<cufz_violation*>(
      take((uint64_t)n_slots * cfg.record_cap * sizeof(cufz_violation)));
  c->T.bitmaps = (cfg.flags & CUFZ_CF_KEEP_BITMAPS) ? take((uint64_t)n_slots * kBitmapBytes) : nullptr;
  c->T.record_cap = cfg.record_cap;
  c->T.redzone = cfg.redzone;
  c->T.iter_budget = cfg.iter_budget;
  c->T.flags = cfg.flags;
  if (off > cfg.arena_bytes) {
    delete c;
    return CUFZ_E_NOMEM;
  }
  cudaStream_t s0 = reinterpret_cast<cudaStream_t>(cfg.stream);
  cudaError_t e = cudaSuccess;
  // host structures
  e = cudaHostAlloc(reinterpret_cast<void**>(&c->done_h), (size_t)n_slots * sizeof(HostDone),
                    cudaHostAllocMapped);
  if (e == cudaSuccess) {
    memset(c->done_h, 0, (size_t)n_slots * sizeof(HostDone));
    e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->done_d), c->done_h, 0);
  }
  c->T.done = c->done_d;
  for (uint32_t k = 0; k < c->n_lanes && e == cudaSuccess; k++) {
    Lane& L = c->lanes[k];
    e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&L.ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&L.ev_end);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&L.h_stage), L.cap, cudaHostAllocDefault);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev_ref);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_ref, c->copy_stream);
  c->ref_recorded = e == cudaSuccess;
  // clear the tables on the caller's stream
  if (e == cudaSuccess) e = cudaMemsetAsync(c->T.union_map, 0, kBitmapBytes, s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->T.union_snap, 0, kBitmapBytes, s0);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->T.counts, 0, (size_t)n_slots * 4ull * kEdgeCount, s0);
  if (e == cudaSuccess) {
    std::vector<SlotState> init(n_slots);
    memset(init.data(), 0, init.size() * sizeof(SlotState));
    for (auto& s : init) s.first_key = ~0ull;
    e = cudaMemcpyAsync(c->T.slots, init.data(), init.size() * sizeof(SlotState),
                        cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    cufz_destroy(c);
    return CUFZ_E_CUDA;
  }
  c->slots.resize(n_slots);
  for (uint32_t s = n_slots; s-- > 0;) c->free_slots.push_back(s);
  c->shape.cta_threads = cfg.cta_threads;
  c->shape.max_regs = 1;
  c->shape.max_prog_bytes = 16;
  c->stats.cta_threads = cfg.cta_threads;
  c->stats.n_sms = (uint32_t)c->n_sms;
  c->stats.max_slots = n_slots;
  *out = c;
  return CUFZ_OK;
}

cufz_status cufz_destroy(cufz_ctx* c) {
  if (!c) return CUFZ_E_INVALID_ARG;
  {
    std::lock_guard<std::mutex> g(c->mu);
    if (c->campaigns) return CUFZ_E_BUSY;  // destroy the campaigns first
    uint64_t t0 = now_us();
    for (uint32_t k = 0; k < c->n_lanes; k++) {
      Lane& L = c->lanes[k];
      while (L.busy && !lane_done(L) && (int64_t)(now_us() - t0) < kWaitLimitUs)
        std::this_thread::sleep_for(std::chrono::microseconds(200));
      lane_reset_graph(L);
      if (L.ev_start) cudaEventDestroy(L.ev_start);
      if (L.ev_end) cudaEventDestroy(L.ev_end);
      if (L.stream) cudaStreamDestroy(L.stream);
      if (L.h_stage) cudaFreeHost(L.h_stage);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->ev_ref) cudaEventDestroy(c->ev_ref);
    if (c->jit_lib) cudaLibraryUnload(c->jit_lib);
    if (c->done_h) cudaFreeHost(c->done_h);
    for (auto& p : c->progs) free_program(&p);
  }
  delete c;
  return CUFZ_OK;
}

namespace {
cufz_status load_into(cufz_ctx* c, const void* bytes, size_t nbytes, bool prune, int path,
                      uint32_t* program_id, cufz_prog_stats* stats);
}

cufz_status cufz_load_program(cufz_ctx* c, const void* bytes, size_t nbytes, uint32_t* program_id,
                              cufz_prog_stats* stats) {
  if (!c || !bytes || !program_id) return CUFZ_E_INVALID_ARG;
  return load_into(c, bytes, nbytes, !(c->cfg.flags & CUFZ_CF_NO_PRUNE), -1, program_id, stats);
}

}  // extern "C"

namespace {

// Loads a program (pruned or not) under the context lock.  path: -1 the
// default (the autotune cache's choice, else compiled), 0 interpreted,
// 1 compiled.
cufz_status load_into(cufz_ctx* c, const void* bytes, size_t nbytes, bool prune, int path,
                      uint32_t* program_id, cufz_prog_stats* stats) {
  std::lock_guard<std::mutex> g(c->mu);
  // the id: the lowest unloaded one, else a new one
  uint32_t id = (uint32_t)c->progs.size();
  for (uint32_t k = 0; k < c->progs.size(); k++)
    if (!c->prog_live[k]) {
      id = k;
      break;
    }
  if (id >= (uint32_t)kMaxPrograms) return CUFZ_E_NOMEM;
  LoadedProgram P;
  cufz_status st = load_program(bytes, nbytes, prune, &P);
  if (st != CUFZ_OK) return st;
  // a program in the block-serial form runs only compiled
  if (P.block_serial && (!use_jit(c) || path == 0)) {
    free_program(&P);
    return CUFZ_E_UNSUPPORTED;
  }
  if (P.block_serial) path = 1;
  // program-area space: the first unloaded range that fits, else the end
  const uint32_t need = (uint32_t)align_up(P.blob_bytes, 16);
  uint32_t off = 0;
  size_t fi = c->prog_free.size();
  for (size_t k = 0; k < c->prog_free.size(); k++)
    if (c->prog_free[k].second >= need) {
      fi = k;
      break;
    }
  if (fi < c->prog_free.size()) {
    off = c->prog_free[fi].first;
  } else if (c->prog_used + need > kProgAreaBytes) {
    free_program(&P);
    return CUFZ_E_NOMEM;
  } else {
    off = (uint32_t)c->prog_used;
  }
  cudaError_t e = cudaMemcpy(c->d_progs + off, P.blob, P.blob_bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_program(&P);
    return CUFZ_E_CUDA;
  }
  std::string fsrc;
  st = jit_source(bytes, nbytes, prune, !(c->cfg.flags & CUFZ_CF_NO_DIGEST), id, &fsrc);
  if (st != CUFZ_OK) {
    free_program(&P);
    return st;
  }
  if (fi < c->prog_free.size()) {
    c->prog_free[fi].first += need;
    c->prog_free[fi].second -= need;
    if (!c->prog_free[fi].second) c->prog_free.erase(c->prog_free.begin() + (long)fi);
  } else {
    c->prog_used += need;
  }
  if (stats) *stats = P.stats;
  *program_id = id;
  const uint64_t key = tune_key(c, bytes, nbytes);
  const auto cached = c->tune_cache.find(key);
  const uint8_t path0 = path >= 0 ? (uint8_t)path : cached == c->tune_cache.end() ? 1 : (cached->second & 1u);
  const uint8_t lanes0 = cached == c->tune_cache.end() ? 1 : (uint8_t)tune_lanes(cached->second);
  std::vector<uint8_t> original(static_cast<const uint8_t*>(bytes), static_cast<const uint8_t*>(bytes) + nbytes);
  // default path: compiled (measured faster than the interpreter on every
  // workload family here, branch-heavy ones included); the autotuner
  // measures and can override
  if (id == c->progs.size()) {
    c->prog_src.push_back(fsrc);
    c->prog_compiled.push_back(path0);
    c->prog_lanes.push_back(lanes0);
    c->progs.push_back(P);
    c->prog_off.push_back(off);
    c->prog_live.push_back(1);
    c->prog_key.push_back(key);
    c->prog_bytes.push_back(std::move(original));
  } else {
    c->prog_src[id] = fsrc;
    c->prog_compiled[id] = path0;
    c->prog_lanes[id] = lanes0;
    c->progs[id] = P;
    c->prog_off[id] = off;
    c->prog_live[id] = 1;
    c->prog_key[id] = key;
    c->prog_bytes[id] = std::move(original);
    if (id < c->prog_in_module.size()) c->prog_in_module[id] = 0;  // the module has the old code
  }
  c->shape.max_regs = std::max(c->shape.max_regs, P.hdr.n_regs);
  c->shape.max_prog_bytes = std::max(c->shape.max_prog_bytes, (uint32_t)align_up(P.blob_bytes, 16));
  apply_tuned_item(c);
  return ensure_smem(c);
}

}  // namespace

extern "C" {

cufz_status cufz_submit_inputs(cufz_ctx* c, const cufz_input* in, uint32_t n, uint32_t* n_accepted,
                               uint64_t* first_ticket) {
  if (!c || (!in && n) || !n_accepted) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  *n_accepted = 0;
  if (first_ticket) *first_ticket = c->next_ticket;
  if (!n) return CUFZ_OK;
  harvest(c);
  // a free lane
  Lane* L = nullptr;
  uint32_t lane_idx = 0;
  for (uint32_t k = 0; k < c->n_lanes; k++) {
    uint32_t li = (c->next_lane + k) % c->n_lanes;
    if (lane_done(c->lanes[li])) {
      lane_retire(c, c->lanes[li]);
      L = &c->lanes[li];
      lane_idx = li;
      break;
    }
  }
  if (!L) return CUFZ_E_BUSY;
  if (use_jit(c) && !jit_current(c)) {
    cufz_status cs = jit_compile(c);
    if (cs != CUFZ_OK) return cs;
  }
  const bool plain = c->cfg.flags & CUFZ_CF_PLAIN_LAUNCH;
  // admission
  BatchHdr* hdr_j = reinterpret_cast<BatchHdr*>(L->h_stage);
  BatchHdr* hdr_i = reinterpret_cast<BatchHdr*>(L->h_stage + sizeof(BatchHdr));
  DevInput* dins = reinterpret_cast<DevInput*>(L->h_stage + 2 * sizeof(BatchHdr));
  uint32_t n_dev = 0;
  const bool prex_on = (c->cfg.flags & CUFZ_CF_PREX) != 0 && !plain;
  std::vector<std::vector<uint32_t>> planned;  // per device input under PREX: its threads
  std::vector<uint32_t> dev_slots;
  uint32_t accepted = 0;
  bool busy = false;
  // The batch's work-item size, fixed before admission from the inputs the
  // lane could take; admission then also stops where the lane's staging
  // memory for work items runs out (a prefix is admitted, the rest gets
  // CUFZ_E_BUSY), so inputs are admitted by memory as well as by slots.
  uint64_t est_threads = 0;
  {
    const uint64_t room = std::min<uint64_t>(c->free_slots.size(), c->lane_max_inputs);
    uint64_t k = 0;
    for (uint32_t i = 0; i < n && k < room; i++) {
      uint64_t nt = 0;
      if (input_status(c, in[i]) == CUFZ_ST_OK && launch_within(in[i], ~0ull, &nt)) {
        est_threads += nt;
        k++;
      }
    }
  }
  const uint32_t item = choose_item_threads(c, est_threads);
  // an input's item size: a multiple of its block size for block-serial
  // programs (their items are whole test blocks)
  auto item_of = [&](uint32_t prog, uint32_t T) -> uint32_t {
    if (!c->progs[prog].block_serial) return item;
    return std::max<uint32_t>(T, item / T * T);
  };
  uint64_t items_taken = 0;
  for (uint32_t i = 0; i < n; i++) {
    const cufz_input& x = in[i];
    int32_t status = input_status(c, x);
    std::vector<uint32_t> plan;
    bool part = false;
    uint64_t need = 0;  // work items of this input
    if (status == CUFZ_ST_OK) {
      if (c->free_slots.empty() || n_dev >= c->lane_max_inputs) {
        busy = true;
        break;
      }
      part = prex_on && c->progs[x.program_id].prex &&
             prex_plan(*c->progs[x.program_id].prex, x, c->T.iter_budget, &plan) &&
             plan.size() <= CUFZ_PREX_MAX_PLAN;
      uint64_t nt = 0;
      launch_within(x, ~0ull, &nt);
      const uint32_t T = x.block[0] * x.block[1] * x.block[2];
      const uint64_t it = item_of(x.program_id, T);
      need = plain ? 0 : part ? plan.size() : (nt + it - 1) / it;
      if (items_taken + need > c->lane_max_items) {
        if (n_dev > 0) {
          busy = true;
          break;
        }
        status = CUFZ_ST_LIMIT;  // more work items than a lane holds, even alone
      }
    }
    uint64_t ticket = c->next_ticket;
    if (status != CUFZ_ST_OK) {
      cufz_result r;
      memset(&r, 0, sizeof(r));
      r.ticket = ticket;
      r.user_tag = x.user_tag;
      r.status = status;
      r.first_key = ~0ull;
      c->host_done[ticket] = r;
      c->ready.push_back(r);
      c->next_ticket++;
      accepted++;
      c->stats.inputs_submitted++;
      c->stats.inputs_completed++;
      continue;
    }
    if (c->free_slots.empty() || n_dev >= c->lane_max_inputs) {
      busy = true;
      break;
    }
    uint32_t s = c->free_slots.back();
    c->free_slots.pop_back();
    DevInput* d = &dins[n_dev];
    build_dev_input(c, x, s, d);
    d->ticket = ticket;
    d->seq = c->next_seq++;
    if (c->next_seq == 0) c->next_seq = 1;
    SlotHost& sh = c->slots[s];
    sh.ticket = ticket;
    sh.seq = d->seq;
    sh.state = 1;
    sh.lane = lane_idx;
    sh.prog = x.program_id;
    sh.partial = false;
    if (part) {
      // these threads decide the verdict: run only them
      planned.resize(n_dev + 1);
      planned[n_dev] = std::move(plan);
      d->n_threads = planned[n_dev].size();
      sh.partial = true;
    }
    items_taken += need;
    c->ticket_slot[ticket] = s;
    dev_slots.push_back(s);
    n_dev++;
    c->next_ticket++;
    accepted++;
    c->stats.inputs_submitted++;
  }
  *n_accepted = accepted;
  if (n_dev) {
    // work items: one list per path, each grouped by program (stable), so
    // CTAs running at the same time mostly run the same program
    uint8_t* items_base = reinterpret_cast<uint8_t*>(dins) + (uint64_t)n_dev * sizeof(DevInput);
    c->stats.item_threads = item;
    std::vector<uint32_t> order(n_dev);
    for (uint32_t i = 0; i < n_dev; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return dins[x].prog < dins[y].prog; });
    auto compiled = [&](uint32_t prog) { return use_jit(c) && c->prog_compiled[prog]; };
    uint64_t want[2] = {0, 0};
    planned.resize(n_dev);
    for (uint32_t i = 0; i < n_dev; i++) {
      DevInput* d = &dins[i];
      const uint32_t it = item_of(d->prog, d->T);
      d->n_items = plain ? (uint32_t)(d->n_threads / d->T)
                 : !planned[i].empty() ? (uint32_t)planned[i].size()  // one item per planned thread
                                       : (uint32_t)((d->n_threads + it - 1) / it);
      if (!plain) want[compiled(d->prog) ? 0 : 1] += d->n_items;
    }
    // (admission kept want[0] + want[1] within the lane's lane_max_items)
    WorkItem* lists[2] = {reinterpret_cast<WorkItem*>(items_base),
                          reinterpret_cast<WorkItem*>(items_base) + want[0]};
    uint32_t counts[2] = {0, 0};
    if (!plain) {
      for (uint32_t oi = 0; oi < n_dev; oi++) {
        const uint32_t i = order[oi];
        const DevInput* d = &dins[i];
        const int li = compiled(d->prog) ? 0 : 1;
        for (uint32_t k = 0; k < d->n_items; k++) {
          WorkItem& w = lists[li][counts[li]++];
          w.input = i;
          if (!planned[i].empty()) {
            w.g0 = planned[i][k];
            w.count = 1;
          } else {
            const uint32_t it = item_of(d->prog, d->T);
            w.g0 = k * it;
            uint64_t rem = d->n_threads - (uint64_t)k * it;
            w.count = (uint32_t)std::min<uint64_t>(rem, it);
          }
          w.pad = 0;
        }
      }
    }
    const uint32_t n_items = counts[0] + counts[1];
    memset(hdr_j, 0, 2 * sizeof(BatchHdr));
    hdr_j->n_inputs = hdr_i->n_inputs = n_dev;
    hdr_j->n_items = counts[0];
    hdr_i->n_items = counts[1];
    hdr_j->inputs_off = 2 * sizeof(BatchHdr);
    hdr_i->inputs_off = sizeof(BatchHdr);
    hdr_j->items_off = (uint64_t)(items_base - L->h_stage);
    hdr_i->items_off = hdr_j->items_off - sizeof(BatchHdr) + (uint64_t)counts[0] * sizeof(WorkItem);
    uint64_t bytes = (uint64_t)(items_base - L->h_stage) + (uint64_t)n_items * sizeof(WorkItem);
    cufz_status st = CUFZ_OK;
    L->batch_id = c->next_batch++;
    cudaError_t e = cudaEventRecord(L->ev_start, L->stream);
    bool use_graph = !plain && !(c->cfg.flags & CUFZ_CF_NO_GRAPH);
    const uint32_t kmask = (counts[0] ? 1u : 0u) | (counts[1] ? 2u : 0u);
    if (kmask == 0) use_graph = false;  // no device items (not reached: every device input has one)
    if (use_graph && lane_graph(c, *L, kmask) != CUFZ_OK) {
      use_graph = false;
      c->stats.graph_failures++;
    }
    if (e == cudaSuccess) {
      // the batch image goes up on the lane's stream, then its kernels run
      e = cudaMemcpyAsync(L->d_batch, L->h_stage, bytes, cudaMemcpyHostToDevice, L->stream);
      if (use_graph && e == cudaSuccess) {
        e = cudaGraphLaunch(L->graphs[kmask].exec, L->stream);
        if (e == cudaSuccess) {
          c->stats.graph_launches++;
          c->stats.kernel_launches += L->graphs[kmask].launches;
        } else {
          // the graph cannot run this batch: drop it and launch directly
          c->stats.last_cuda_error = 60000 + (int32_t)e;
          c->stats.graph_failures++;
          cudaGetLastError();
          lane_reset_graph(*L);
          use_graph = false;
          e = cudaSuccess;
        }
      }
      if (!use_graph && e == cudaSuccess) {
        if (!plain) {
          uint32_t nl = 0;
          e = launch_batch_kernels(c, *L, counts[0], counts[1], false, L->stream, &nl);
          c->stats.kernel_launches += nl;
        } else {
          for (uint32_t i = 0; i < n_dev && e == cudaSuccess; i++) {
            LaunchShape s = c->shape;
            s.cta_threads = (uint32_t)align_up(dins[i].T, 32);
            if (compiled(dins[i].prog)) {
              e = launch_jit_plain(c, jit_hdr(*L), i, dins[i].n_items, s.cta_threads, L->stream);
            } else {
              if (smem_for(s, s.cta_threads) > c->smem_set) {
                e = cudaErrorInvalidConfiguration;
                break;
              }
              e = launch_plain(c->T, interp_hdr(*L), i, dins[i].n_items, s, L->stream);
            }
            if (e == cudaSuccess) c->stats.kernel_launches++;
          }
        }
      }
    }
    if (e == cudaSuccess) e = cudaEventRecord(L->ev_end, L->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = CUFZ_E_CUDA;
    }
    L->busy = true;
    L->timed = (e == cudaSuccess);
    c->stats.batches++;
    c->next_lane = (lane_idx + 1) % c->n_lanes;
    for (uint32_t s : dev_slots) c->inflight.push_back(s);
    if (st != CUFZ_OK) return st;
  }
  return busy ? CUFZ_E_BUSY : CUFZ_OK;
}

cufz_status cufz_poll_results(cufz_ctx* c, cufz_result* out, uint32_t max, uint32_t* n_out,
                              int32_t timeout_us) {
  if (!c || !n_out || (!out && max)) return CUFZ_E_INVALID_ARG;
  *n_out = 0;
  uint64_t t0 = now_us();
  int64_t limit = timeout_us < 0 ? kWaitLimitUs : (int64_t)timeout_us;
  for (;;) {
    {
      std::lock_guard<std::mutex> g(c->mu);
      harvest(c);
      bool all_done = c->inflight.empty();
      uint32_t k = 0;
      if (timeout_us >= 0 || all_done) {
        while (k < max && !c->ready.empty()) {
          out[k++] = c->ready.front();
          c->ready.pop_front();
        }
      }
      if (k) {
        *n_out = k;
        return CUFZ_OK;
      }
      if (timeout_us < 0 && all_done) return CUFZ_OK;
      if (timeout_us == 0) return CUFZ_OK;
    }
    if ((int64_t)(now_us() - t0) >= limit) return timeout_us < 0 ? CUFZ_E_TIMEOUT : CUFZ_OK;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

cufz_status cufz_sync(cufz_ctx* c, int32_t timeout_us) {
  if (!c) return CUFZ_E_INVALID_ARG;
  uint64_t t0 = now_us();
  int64_t limit = timeout_us < 0 ? kWaitLimitUs : (int64_t)timeout_us;
  for (;;) {
    {
      std::lock_guard<std::mutex> g(c->mu);
      harvest(c);
      bool lanes_idle = true;
      for (uint32_t k = 0; k < c->n_lanes; k++)
        if (c->lanes[k].busy) lanes_idle = false;
      if (c->inflight.empty() && lanes_idle) return CUFZ_OK;
    }
    if ((int64_t)(now_us() - t0) >= limit) return CUFZ_E_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

static cufz_status lookup_completed(cufz_ctx* c, uint64_t ticket, uint32_t* slot, bool* host_only) {
  harvest(c);
  *host_only = false;
  auto it = c->ticket_slot.find(ticket);
  if (it == c->ticket_slot.end()) {
    if (c->host_done.count(ticket)) {
      *host_only = true;
      return CUFZ_OK;
    }
    return CUFZ_E_NOT_FOUND;
  }
  if (c->slots[it->second].state != 2) return CUFZ_E_BUSY;
  *slot = it->second;
  return CUFZ_OK;
}

cufz_status cufz_get_records(cufz_ctx* c, uint64_t ticket, cufz_violation* out, uint32_t cap,
                             uint32_t* n) {
  if (!c || !n || (!out && cap)) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  uint32_t s = 0;
  bool host_only = false;
  cufz_status st = lookup_completed(c, ticket, &s, &host_only);
  if (st != CUFZ_OK) return st;
  *n = 0;
  if (host_only) return CUFZ_OK;
  uint32_t have = c->done_h[s].res.n_records;
  uint32_t k = std::min(have, cap);
  if (k) {
    cudaError_t e = cudaMemcpyAsync(out, c->T.records + (size_t)s * c->cfg.record_cap,
                                     (size_t)k * sizeof(cufz_violation), cudaMemcpyDeviceToHost,
                                     c->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->copy_stream);
    if (e != cudaSuccess) return CUFZ_E_CUDA;
  }
  *n = k;
  return CUFZ_OK;
}

cufz_status cufz_get_bitmap(cufz_ctx* c, uint64_t ticket, uint8_t* out65536) {
  if (!c || !out65536) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  if (!(c->cfg.flags & CUFZ_CF_KEEP_BITMAPS)) return CUFZ_E_INVALID_ARG;
  uint32_t s = 0;
  bool host_only = false;
  cufz_status st = lookup_completed(c, ticket, &s, &host_only);
  if (st != CUFZ_OK) return st;
  if (host_only) {
    memset(out65536, 0, kBitmapBytes);
    return CUFZ_OK;
  }
  cudaError_t e = cudaMemcpyAsync(out65536, c->T.bitmaps + (size_t)s * kBitmapBytes, kBitmapBytes,
                                   cudaMemcpyDeviceToHost, c->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->copy_stream);
  return cuda_err(e);
}

cufz_status cufz_get_union(cufz_ctx* c, uint8_t* out65536) {
  if (!c || !out65536) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  cudaError_t e = cudaMemcpyAsync(out65536, c->T.union_map, kBitmapBytes, cudaMemcpyDeviceToHost,
                                   c->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->copy_stream);
  return cuda_err(e);
}

cufz_status cufz_new_epoch(cufz_ctx* c) {
  if (!c) return CUFZ_E_INVALID_ARG;
  cufz_status st = cufz_sync(c, -1);
  if (st != CUFZ_OK) return st;
  std::lock_guard<std::mutex> g(c->mu);
  cudaError_t e = cudaMemcpyAsync(c->T.union_snap, c->T.union_map, kBitmapBytes,
                                   cudaMemcpyDeviceToDevice, c->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->copy_stream);
  return cuda_err(e);
}

cufz_status cufz_release(cufz_ctx* c, uint64_t ticket) {
  if (!c) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  if (c->host_done.erase(ticket)) return CUFZ_OK;
  auto it = c->ticket_slot.find(ticket);
  if (it == c->ticket_slot.end()) return CUFZ_E_NOT_FOUND;
  harvest(c);
  SlotHost& sh = c->slots[it->second];
  if (sh.state != 2) return CUFZ_E_BUSY;
  sh.state = 0;
  c->free_slots.push_back(it->second);
  c->ticket_slot.erase(it);
  return CUFZ_OK;
}

cufz_status cufz_program_cuda(const void* bytes, size_t nbytes, uint32_t flags, char* out,
                              size_t out_cap, size_t* out_bytes) {
  if (!bytes || !out_bytes) return CUFZ_E_INVALID_ARG;
  std::string f;
  cufz_status st = jit_source(bytes, nbytes, !(flags & CUFZ_CF_NO_PRUNE),
                              !(flags & CUFZ_CF_NO_DIGEST), 0, &f);
  if (st != CUFZ_OK) return st;
  *out_bytes = f.size() + 1;
  if (!out || out_cap < f.size() + 1) return CUFZ_E_NOMEM;
  memcpy(out, f.c_str(), f.size() + 1);
  return CUFZ_OK;
}

cufz_status cufz_compile_check(const void* const* progs, const size_t* sizes, uint32_t n,
                               uint32_t flags, char* log, uint32_t log_cap, size_t* cubin_bytes) {
  if ((!progs || !sizes) && n) return CUFZ_E_INVALID_ARG;
  std::vector<std::string> srcs(n);
  for (uint32_t k = 0; k < n; k++) {
    cufz_status st = jit_source(progs[k], sizes[k], !(flags & CUFZ_CF_NO_PRUNE),
                                !(flags & CUFZ_CF_NO_DIGEST), k, &srcs[k]);
    if (st != CUFZ_OK) return st;
  }
  std::vector<char> image;
  std::string lg;
  cufz_status st = jit_build_image(srcs, std::vector<uint8_t>(n, 1),
                                   (flags & CUFZ_CF_PLAIN_LAUNCH) != 0, 0, 256,
                                   (flags & CUFZ_CF_JIT_FAST_COMPILE) != 0,
                                   std::vector<uint8_t>(n, 1), &image, &lg);
  if (log && log_cap) {
    size_t m = std::min<size_t>(lg.size(), log_cap - 1);
    memcpy(log, lg.data(), m);
    log[m] = 0;
  }
  if (cubin_bytes) *cubin_bytes = image.size();
  return st;
}

cufz_status cufz_compile_programs(cufz_ctx* c, char* log, uint32_t log_cap) {
  if (!c) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  cufz_status st = jit_compile(c);
  if (log && log_cap) {
    size_t n = std::min<size_t>(c->jit_log.size(), log_cap - 1);
    memcpy(log, c->jit_log.data(), n);
    log[n] = 0;
  }
  return st;
}

cufz_status cufz_set_program_lanes(cufz_ctx* c, uint32_t program_id, uint32_t lanes) {
  if (!c || !lanes_ok(lanes)) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  if (program_id >= c->progs.size() || !c->prog_live[program_id]) return CUFZ_E_NOT_FOUND;
  c->prog_lanes[program_id] = (uint8_t)lanes;
  return CUFZ_OK;
}

cufz_status cufz_get_program_lanes(cufz_ctx* c, uint32_t program_id, uint32_t* lanes) {
  if (!c || !lanes) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  if (program_id >= c->progs.size() || !c->prog_live[program_id]) return CUFZ_E_NOT_FOUND;
  *lanes = c->prog_lanes[program_id];
  return CUFZ_OK;
}

cufz_status cufz_set_program_path(cufz_ctx* c, uint32_t program_id, uint32_t compiled) {
  if (!c) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  if (program_id >= c->progs.size() || !c->prog_live[program_id]) return CUFZ_E_NOT_FOUND;
  if (!compiled && c->progs[program_id].block_serial) return CUFZ_E_UNSUPPORTED;
  c->prog_compiled[program_id] = compiled ? 1 : 0;
  return CUFZ_OK;
}

cufz_status cufz_unload_program(cufz_ctx* c, uint32_t program_id) {
  if (!c) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  if (program_id >= c->progs.size() || !c->prog_live[program_id]) return CUFZ_E_NOT_FOUND;
  // in flight = submitted and not yet collected by a poll or sync
  for (const SlotHost& sh : c->slots)
    if (sh.state == 1 && sh.prog == program_id) return CUFZ_E_BUSY;
  LoadedProgram& P = c->progs[program_id];
  c->prog_free.emplace_back(c->prog_off[program_id], (uint32_t)align_up(P.blob_bytes, 16));
  free_program(&P);
  c->prog_live[program_id] = 0;
  c->prog_compiled[program_id] = 0;
  c->prog_src[program_id].clear();
  apply_tuned_item(c);
  return CUFZ_OK;
}

namespace {

// What a run of one input leaves: its result, bitmap (if kept) and records.
struct Outcome {
  cufz_result res{};
  std::vector<uint8_t> bitmap;
  std::vector<cufz_violation> recs;
};

// Runs inputs on an idle context and collects their outcomes, releasing
// their slots.
cufz_status run_collect(cufz_ctx* c, const std::vector<cufz_input>& in, std::vector<Outcome>* out) {
  out->assign(in.size(), Outcome{});
  const bool keep = (c->cfg.flags & CUFZ_CF_KEEP_BITMAPS) != 0;
  const bool auto_rel = (c->cfg.flags & CUFZ_CF_AUTO_RELEASE) != 0;
  std::unordered_map<uint64_t, size_t> index;
  std::vector<cufz_result> got(256);
  size_t pos = 0, done = 0;
  while (done < in.size()) {
    if (pos < in.size()) {
      uint32_t acc = 0;
      uint64_t first = 0;
      cufz_status st = cufz_submit_inputs(c, in.data() + pos, (uint32_t)(in.size() - pos), &acc, &first);
      if (st != CUFZ_OK && st != CUFZ_E_BUSY) return st;
      for (uint32_t k = 0; k < acc; k++) index[first + k] = pos + k;
      pos += acc;
    }
    cufz_status st = cufz_sync(c, -1);
    if (st != CUFZ_OK) return st;
    for (;;) {
      uint32_t n = 0;
      st = cufz_poll_results(c, got.data(), (uint32_t)got.size(), &n, 0);
      if (st != CUFZ_OK) return st;
      if (!n) break;
      for (uint32_t k = 0; k < n; k++) {
        const auto it = index.find(got[k].ticket);
        if (it == index.end()) continue;
        Outcome& o = (*out)[it->second];
        o.res = got[k];
        if (!auto_rel) {
          if (keep) {
            o.bitmap.resize(kBitmapBytes);
            if (cufz_get_bitmap(c, o.res.ticket, o.bitmap.data()) != CUFZ_OK) o.bitmap.clear();
          }
          o.recs.resize(o.res.n_records);
          uint32_t nr = 0;
          if (o.res.n_records &&
              cufz_get_records(c, o.res.ticket, o.recs.data(), o.res.n_records, &nr) != CUFZ_OK)
            nr = 0;
          o.recs.resize(nr);
          cufz_release(c, o.res.ticket);
        }
        done++;
      }
    }
  }
  return CUFZ_OK;
}

bool same_outcome(const Outcome& a, const Outcome& b, uint32_t cap) {
  const cufz_result &x = a.res, &y = b.res;
  const uint32_t fl = CUFZ_FL_BUDGET | CUFZ_FL_OVERFLOW;
  if (x.status != y.status || (x.flags & fl) != (y.flags & fl) || x.n_accesses != y.n_accesses ||
      x.n_violations != y.n_violations || x.first_key != y.first_key || x.digest != y.digest ||
      x.n_branch != y.n_branch || x.n_threads != y.n_threads || x.n_records != y.n_records ||
      x.n_edges != y.n_edges || a.bitmap != b.bitmap)
    return false;
  if (x.n_violations > cap) return true;  // any cap records of the violations: not unique
  auto key = [](const cufz_violation& v) {
    return std::make_tuple(v.block_lin, v.thread_lin, v.ordinal, v.site, v.buf, v.kind, v.width,
                           v.space, v.cls, v.byte_off);
  };
  std::vector<decltype(key(cufz_violation{}))> ka, kb;
  for (const auto& v : a.recs) ka.push_back(key(v));
  for (const auto& v : b.recs) kb.push_back(key(v));
  std::sort(ka.begin(), ka.end());
  std::sort(kb.begin(), kb.end());
  return ka == kb;
}

}  // namespace

cufz_status cufz_verify_prune(cufz_ctx* c, uint32_t program_id, const cufz_input* inputs, uint32_t n,
                              uint32_t* n_mismatch) {
  if (!c || (!inputs && n) || !n_mismatch) return CUFZ_E_INVALID_ARG;
  *n_mismatch = 0;
  std::vector<uint8_t> bytes;
  bool serial = false;
  {
    std::lock_guard<std::mutex> g(c->mu);
    if (program_id >= c->progs.size() || !c->prog_live[program_id]) return CUFZ_E_NOT_FOUND;
    if (!c->inflight.empty() || !c->ready.empty()) return CUFZ_E_BUSY;
    bytes = c->prog_bytes[program_id];
    serial = c->progs[program_id].block_serial;
  }
  uint32_t full = 0;
  // the unpruned program on the interpreter (block-serial programs: compiled)
  cufz_status st = load_into(c, bytes.data(), bytes.size(), false, serial ? 1 : 0, &full, nullptr);
  if (st != CUFZ_OK) return st;
  std::vector<cufz_input> a(inputs, inputs + n), b(inputs, inputs + n);
  for (auto& x : a) x.program_id = program_id;
  for (auto& x : b) x.program_id = full;
  std::vector<Outcome> ra, rb;
  st = run_collect(c, a, &ra);
  if (st == CUFZ_OK) st = run_collect(c, b, &rb);
  const cufz_status su = cufz_unload_program(c, full);
  if (st != CUFZ_OK) return st;
  if (su != CUFZ_OK) return su;
  for (uint32_t i = 0; i < n; i++)
    if (!same_outcome(ra[i], rb[i], c->cfg.record_cap)) (*n_mismatch)++;
  return CUFZ_OK;
}

cufz_status cufz_get_program_path(cufz_ctx* c, uint32_t program_id, uint32_t* compiled) {
  if (!c || !compiled) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  if (program_id >= c->progs.size() || !c->prog_live[program_id]) return CUFZ_E_NOT_FOUND;
  *compiled = use_jit(c) && c->prog_compiled[program_id];
  return CUFZ_OK;
}

// Runs inputs to completion for the autotuner; their results and slots are
// taken back so that they never reach the caller.  Returns the device time.
static cufz_status autotune_run(cufz_ctx* c, const cufz_input* in, uint32_t n, double* ms) {
  {
    std::lock_guard<std::mutex> g(c->mu);
    harvest(c);
    c->stats.kernel_ms = 0;
  }
  uint32_t pos = 0;
  std::vector<uint64_t> tickets;
  while (pos < n) {
    uint32_t acc = 0;
    uint64_t first = 0;
    cufz_status st = cufz_submit_inputs(c, in + pos, n - pos, &acc, &first);
    for (uint32_t k = 0; k < acc; k++) tickets.push_back(first + k);
    pos += acc;
    if (st != CUFZ_OK && st != CUFZ_E_BUSY) return st;
    if (st == CUFZ_E_BUSY || acc == 0) {
      cufz_status s2 = cufz_sync(c, -1);
      if (s2 != CUFZ_OK) return s2;
      std::lock_guard<std::mutex> g(c->mu);
      harvest(c);
      std::unordered_map<uint64_t, bool> mine;
      for (uint64_t t : tickets) mine[t] = true;
      std::deque<cufz_result> keep;
      for (auto& r : c->ready) {
        if (!mine.count(r.ticket)) {
          keep.push_back(r);
          continue;
        }
        c->host_done.erase(r.ticket);
        auto it = c->ticket_slot.find(r.ticket);
        if (it != c->ticket_slot.end()) {
          c->slots[it->second].state = 0;
          c->free_slots.push_back(it->second);
          c->ticket_slot.erase(it);
        }
      }
      c->ready.swap(keep);
      tickets.clear();
    }
  }
  cufz_status st = cufz_sync(c, -1);
  if (st != CUFZ_OK) return st;
  std::lock_guard<std::mutex> g(c->mu);
  harvest(c);
  std::unordered_map<uint64_t, bool> mine;
  for (uint64_t t : tickets) mine[t] = true;
  std::deque<cufz_result> keep;
  for (auto& r : c->ready) {
    if (!mine.count(r.ticket)) {
      keep.push_back(r);
      continue;
    }
    c->host_done.erase(r.ticket);
    auto it = c->ticket_slot.find(r.ticket);
    if (it != c->ticket_slot.end()) {
      c->slots[it->second].state = 0;
      c->free_slots.push_back(it->second);
      c->ticket_slot.erase(it);
    }
  }
  c->ready.swap(keep);
  *ms = c->stats.kernel_ms;
  return CUFZ_OK;
}

cufz_status cufz_autotune(cufz_ctx* c, const cufz_input* sample, uint32_t n, uint32_t* n_compiled) {
  if (!c || (!sample && n)) return CUFZ_E_INVALID_ARG;
  if (n_compiled) *n_compiled = 0;
  if (!use_jit(c)) return CUFZ_OK;
  std::vector<uint8_t> before;
  {
    std::lock_guard<std::mutex> g(c->mu);
    if (!c->inflight.empty()) return CUFZ_E_BUSY;
    before = c->prog_compiled;
    for (auto& b : c->prog_compiled) b = 1;  // one module with every program
    cufz_status cs = jit_compile(c);
    c->prog_compiled = before;
    if (cs != CUFZ_OK) return cs;
  }
  cufz_stats saved;
  cufz_get_stats(c, &saved);
  std::unordered_map<uint32_t, std::vector<cufz_input>> by_prog;
  for (uint32_t i = 0; i < n; i++) by_prog[sample[i].program_id].push_back(sample[i]);
  std::unordered_map<uint32_t, std::array<double, 3>> lanes_ms;  // compiled: ms at 1, 2, 4 lanes
  // a few small inputs measure launch and finalize costs, not the paths:
  // repeat each program's sample until it fills the GPU many times over
  for (auto& kv : by_prog) {
    std::vector<cufz_input>& v = kv.second;
    uint64_t threads = 0;
    for (const cufz_input& in : v)
      threads += (uint64_t)in.grid[0] * in.grid[1] * in.grid[2] * in.block[0] * in.block[1] * in.block[2];
    const size_t n0 = v.size();
    for (size_t k = 0; threads && threads < kAutotuneMinThreads && v.size() < kAutotuneMaxInputs; k++) {
      const cufz_input& in = v[k % n0];
      threads += (uint64_t)in.grid[0] * in.grid[1] * in.grid[2] * in.block[0] * in.block[1] * in.block[2];
      v.push_back(in);
    }
  }
  for (auto& kv : by_prog) {
    const uint32_t p = kv.first;
    if (p >= c->progs.size() || !c->prog_live[p]) continue;
    if (c->progs[p].block_serial) continue;  // compiled only
    const uint32_t dflt = before[p];
    double best[2] = {1e30, 1e30};
    for (int rep = 0; rep < 3; rep++)
      for (uint32_t path = 0; path < 2; path++) {
        cufz_set_program_path(c, p, path);
        double ms = 0;
        cufz_status st = autotune_run(c, kv.second.data(), (uint32_t)kv.second.size(), &ms);
        if (st != CUFZ_OK) return st;
        best[path] = std::min(best[path], ms);
      }
    // leave the load-time choice only for a clear win
    const uint32_t other = 1u - dflt;
    const uint32_t chosen = best[other] * kAutotuneMargin < best[dflt] ? other : dflt;
    cufz_set_program_path(c, p, chosen);
    c->prog_lanes[p] = 1;
    c->tune_cache[c->prog_key[p]] = tune_value(chosen != 0, 1);
    if (chosen) lanes_ms[p][0] = best[1];
  }
  // Lane mapping of short compiled programs: their sample again with 2 and
  // 4 test threads per lane per loop iteration.  The module for these runs
  // holds only the short programs (the others are set aside, not run).
  std::vector<uint32_t> small;
  for (auto& kv : lanes_ms)
    if (c->progs[kv.first].stats.n_ops_kept <= kLanesMaxOps) small.push_back(kv.first);
  if (!small.empty()) {
    std::vector<uint8_t> paths = c->prog_compiled;
    for (auto& b : c->prog_compiled) b = 0;
    for (uint32_t p : small) c->prog_compiled[p] = 1;
    const uint32_t ks[2] = {2, 4};
    for (int ki = 0; ki < 2; ki++) {
      for (uint32_t p : small) c->prog_lanes[p] = (uint8_t)ks[ki];
      for (uint32_t p : small) {
        double b = 1e30;
        for (int rep = 0; rep < 3; rep++) {
          double ms = 0;
          cufz_status st = autotune_run(c, by_prog[p].data(), (uint32_t)by_prog[p].size(), &ms);
          if (st != CUFZ_OK) {
            c->prog_compiled = paths;
            return st;
          }
          b = std::min(b, ms);
        }
        lanes_ms[p][1 + ki] = b;
      }
    }
    c->prog_compiled = paths;
    for (uint32_t p : small) {
      const std::array<double, 3>& t = lanes_ms[p];
      uint32_t k = 1;
      double tk = t[0];
      if (t[1] * kLanesMargin < tk) k = 2, tk = t[1];
      if (t[2] * kLanesMargin < tk) k = 4;
      c->prog_lanes[p] = (uint8_t)k;
      c->tune_cache[c->prog_key[p]] = tune_value(true, k);
    }
  }
  // The work-item size (test threads a CTA takes at a time, so how many
  // inputs a CTA serves): the whole sample, an equal share of every
  // program's and at most 4096 inputs, timed at a few sizes; a size other
  // than the heuristic's must be 3% faster.  Kept for this set of programs.
  if (!c->cfg.item_threads && !by_prog.empty()) {
    std::vector<cufz_input> all;
    for (size_t k = 0; all.size() < kAutotuneItemInputs; k++) {
      bool more = false;
      for (auto& kv : by_prog)
        if (k < kv.second.size() && all.size() < kAutotuneItemInputs) {
          all.push_back(kv.second[k]);
          more = true;
        }
      if (!more) break;
    }
    const uint32_t cands[] = {0u, 4096u, 16384u, 65536u, 262144u};
    double base = 1e30, best_ms = 1e30;
    uint32_t best = 0;
    for (uint32_t cand : cands) {
      c->tuned_item = cand;
      double b = 1e30;
      for (int rep = 0; rep < 2; rep++) {
        double ms = 0;
        cufz_status st = autotune_run(c, all.data(), (uint32_t)all.size(), &ms);
        if (st != CUFZ_OK) {
          apply_tuned_item(c);
          return st;
        }
        b = std::min(b, ms);
      }
      if (cand == 0) base = b;
      if (b < best_ms) best_ms = b, best = cand;
    }
    if (best && best_ms * kLanesMargin >= base) best = 0;
    c->tuned_item = best;
    if (best)
      c->tune_items[workload_key(c)] = best;
    else
      c->tune_items.erase(workload_key(c));
  }
  std::lock_guard<std::mutex> g(c->mu);
  c->stats = saved;
  if (!tune_cache_write(c)) return CUFZ_E_IO;
  if (n_compiled)
    for (uint8_t b : c->prog_compiled) *n_compiled += b;
  return CUFZ_OK;
}

cufz_status cufz_get_stats(cufz_ctx* c, cufz_stats* out) {
  if (!c || !out) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  harvest(c);
  *out = c->stats;
  return CUFZ_OK;
}

cufz_status cufz_reset_stats(cufz_ctx* c) {
  if (!c) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  harvest(c);
  cufz_stats keep = c->stats;
  memset(&c->stats, 0, sizeof(c->stats));
  c->stats.cta_threads = keep.cta_threads;
  c->stats.ctas_per_sm = keep.ctas_per_sm;
  c->stats.item_threads = keep.item_threads;
  c->stats.n_sms = keep.n_sms;
  c->stats.max_slots = keep.max_slots;
  c->stats.smem_bytes = keep.smem_bytes;
  c->recent.clear();
  c->ref_recorded = cudaEventRecord(c->ev_ref, c->copy_stream) == cudaSuccess;
  return CUFZ_OK;
}

cufz_status cufz_int32_peak(int32_t device, void* stream, double* lane_ops_per_s) {
  if (!lane_ops_per_s) return CUFZ_E_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return CUFZ_E_NO_DEVICE;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* h = nullptr;
  uint32_t* d = nullptr;
  cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&h), 64, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&d), h, 0);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const uint32_t threads = 256, blocks = (uint32_t)sms * 8, iters = 4096;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
    e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = launch_int32_peak(d, blocks, threads, iters, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && rep > 0) best = std::min(best, ms);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (h) cudaFreeHost(h);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  double ops = (double)blocks * threads * iters * 8.0 * 16.0;
  *lane_ops_per_s = ops / (best * 1e-3);
  return CUFZ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- campaign
namespace cufz {

cufz_status campaign_attach(cufz_ctx* c, uint32_t n_slots, uint32_t item_threads, CampaignEnv* env) {
  if (!c || !env || !n_slots) return CUFZ_E_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  if (!use_jit(c) || (c->cfg.flags & CUFZ_CF_PLAIN_LAUNCH)) return CUFZ_E_UNSUPPORTED;
  harvest(c);
  if (c->free_slots.size() < n_slots) return CUFZ_E_BUSY;
  // a campaign runs every loaded program compiled
  for (size_t k = 0; k < c->progs.size(); k++)
    if (c->prog_live[k]) c->prog_compiled[k] = 1;
  const cufz_status st = jit_compile(c);
  if (st != CUFZ_OK) return st;
  if (!c->jit_persist) return CUFZ_E_CUDA;
  env->device = c->device;
  env->T = c->T;
  env->jit_kernel = reinterpret_cast<const void*>(c->jit_persist);
  env->jit_ctas = jit_ctas(c);
  env->cta_threads = c->shape.cta_threads;
  env->item_threads = item_threads ? item_threads
                    : c->cfg.item_threads ? c->cfg.item_threads
                    : c->tuned_item ? c->tuned_item
                                    : 64u * c->shape.cta_threads;
  env->max_threads = c->cfg.max_threads;
  env->redzone = c->cfg.redzone;
  env->n_programs = (uint32_t)c->progs.size();
  env->progs.assign(c->progs.size() * 4, 0u);
  for (size_t k = 0; k < c->progs.size(); k++) {
    const LoadedProgram& P = c->progs[k];
    if (!c->prog_live[k]) continue;
    env->progs[k * 4] = 1u | (P.n_bufs << 8) | ((P.shared_mask & 0x1FFu) << 16) |
                        (P.block_serial ? 1u << 31 : 0u);
    env->progs[k * 4 + 1] = c->prog_off[k];
    env->progs[k * 4 + 2] = P.blob_bytes;
  }
  env->slots.clear();
  for (uint32_t k = 0; k < n_slots; k++) {
    const uint32_t s = c->free_slots.back();
    c->free_slots.pop_back();
    c->slots[s].state = 3;  // held by a campaign
    env->slots.push_back(s);
  }
  env->module_gen = c->module_gen;
  env->jit_smem = c->jit_smem;
  c->campaigns++;
  return CUFZ_OK;
}

void campaign_detach(cufz_ctx* c, const std::vector<uint32_t>& slots) {
  if (!c) return;
  std::lock_guard<std::mutex> g(c->mu);
  for (uint32_t s : slots) {
    c->slots[s].state = 0;
    c->free_slots.push_back(s);
  }
  if (c->campaigns) c->campaigns--;
}

bool campaign_env_current(cufz_ctx* c, const CampaignEnv& env) {
  std::lock_guard<std::mutex> g(c->mu);
  return c->module_gen == env.module_gen &&
         reinterpret_cast<const void*>(c->jit_persist) == env.jit_kernel;
}

}  // namespace cufz

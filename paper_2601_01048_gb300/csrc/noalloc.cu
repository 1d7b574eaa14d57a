// Allocation-free entry point: one checked execution of one input with all
// of the engine's scratch memory in a fixed device array of this library.
//
// Some callers cannot allocate device memory at all: plugins whose host
// framework owns every device allocation and hands out only the buffers of
// one call, and services that must not grow their device footprint after
// start-up.  They cannot create a context (which sub-allocates an arena the
// caller owns), so this entry point takes only the buffers of the call --
// the input record, the record, bitmap and result outputs -- and keeps the
// scratch (edge counters, touched-edge list, union maps, slot state, the
// loaded program and the work items) in `g_noalloc_scratch`, a file-scope
// __device__ array that every GPU loading this library holds until exit.
// The first call on a device looks up the array's device address (the
// host-side name of a __device__ variable is not a device address).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>

#include "engine.h"

namespace {

using namespace cufz;

constexpr size_t kScratchBytes = 2u << 20;  // 2 MiB
constexpr size_t kOffCounts = 0;                                   // u32[65536]
constexpr size_t kOffTouched = kOffCounts + 4u * kEdgeCount;       // u16[65536]
constexpr size_t kOffUnion = kOffTouched + 2u * kEdgeCount;        // u8[65536]
constexpr size_t kOffSnap = kOffUnion + kBitmapBytes;              // u8[65536]
constexpr size_t kOffSlot = kOffSnap + kBitmapBytes;               // SlotState
constexpr size_t kOffDone = kOffSlot + 256;                        // HostDone
constexpr size_t kOffProg = kOffDone + 256;                        // program blob
constexpr size_t kMaxProgBytes = 64u << 10;
constexpr size_t kOffBatch = kOffProg + kMaxProgBytes;             // BatchHdr, DevInput, items
constexpr size_t kMaxItems =
    (kScratchBytes - kOffBatch - sizeof(BatchHdr) - sizeof(DevInput)) / sizeof(WorkItem);
constexpr int kMaxDevices = 64;

__device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
uint8_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per
// device; the array's host-side name is not a device address).
cudaError_t scratch_on(int dev, uint8_t** out) {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = reinterpret_cast<uint8_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" cufz_status cufz_run_noalloc(const void* program, size_t nbytes,
                                        const cufz_input* input, uint32_t flags, uint32_t redzone,
                                        uint32_t iter_budget, cufz_violation* records,
                                        uint32_t record_cap, uint8_t* bitmap, cufz_result* result,
                                        void* stream) {
  if (!program || !input || !result || (!records && record_cap) || redzone > (1u << 20))
    return CUFZ_E_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return CUFZ_E_NO_DEVICE;
  }
  LoadedProgram P;
  cufz_status ls = load_program(program, nbytes, !(flags & CUFZ_CF_NO_PRUNE), &P);
  if (ls != CUFZ_OK) return ls;
  struct Freer {
    LoadedProgram* p;
    ~Freer() { free_program(p); }
  } freer{&P};
  // a valid program's loaded form is at most about 34 KB (2,048 ops of 16
  // bytes, header, LOC table, zero list), so this only guards the limit
  if (P.blob_bytes > kMaxProgBytes) return CUFZ_E_NOMEM;
  if (P.block_serial) return CUFZ_E_UNSUPPORTED;  // runs only compiled, in a context

  cufz_result r0;
  memset(&r0, 0, sizeof(r0));
  r0.user_tag = input->user_tag;
  r0.first_key = ~0ull;
  uint64_t n_threads = 0;
  int32_t status = CUFZ_ST_OK;
  if (launch_rejected(*input)) status = CUFZ_ST_INVALID_CONFIG;
  else if (!launch_within(*input, 1ull << 31, &n_threads)) status = CUFZ_ST_LIMIT;
  for (uint32_t k = 0; k < P.n_bufs && status == CUFZ_ST_OK; k++)
    if (input->buf_len[k] >= (1ull << 48)) status = CUFZ_ST_LIMIT;
  if (status != CUFZ_ST_OK) {
    r0.status = status;
    cudaError_t e = cudaMemcpyAsync(result, &r0, sizeof(r0), cudaMemcpyDefault, st);
    if (e == cudaSuccess && bitmap) e = cudaMemsetAsync(bitmap, 0, kBitmapBytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? CUFZ_OK : CUFZ_E_CUDA;
  }

  uint8_t* S = nullptr;
  if (scratch_on(dev, &S) != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  // the batch image: header, the one input, its work items
  uint64_t item = std::max<uint64_t>(2048, (n_threads + kMaxItems - 1) / kMaxItems);
  item = (item + 31) / 32 * 32;
  const uint32_t n_items = (uint32_t)((n_threads + item - 1) / item);
  const size_t bytes = sizeof(BatchHdr) + sizeof(DevInput) + (size_t)n_items * sizeof(WorkItem);
  struct Image {
    uint8_t* p;
    explicit Image(size_t n) : p(new (std::nothrow) uint8_t[n]()) {}
    ~Image() { delete[] p; }
  } img(bytes);
  if (!img.p) return CUFZ_E_NOMEM;
  BatchHdr* hdr = reinterpret_cast<BatchHdr*>(img.p);
  DevInput* d = reinterpret_cast<DevInput*>(img.p + sizeof(BatchHdr));
  WorkItem* items = reinterpret_cast<WorkItem*>(img.p + sizeof(BatchHdr) + sizeof(DevInput));
  hdr->n_inputs = 1;
  hdr->n_items = n_items;
  hdr->inputs_off = sizeof(BatchHdr);
  hdr->items_off = sizeof(BatchHdr) + sizeof(DevInput);
  fill_dev_input(*input, P.n_bufs, P.shared_mask, redzone, d);
  d->n_items = n_items;
  d->prog_bytes = P.blob_bytes;
  d->seq = 1;
  for (uint32_t k = 0; k < n_items; k++) {
    items[k].input = 0;
    items[k].g0 = (uint32_t)(k * item);
    items[k].count = (uint32_t)std::min<uint64_t>(item, n_threads - k * item);
  }
  SlotState s0;
  memset(&s0, 0, sizeof(s0));
  s0.first_key = ~0ull;

  EngineTables tab;
  memset(&tab, 0, sizeof(tab));
  tab.progs = S + kOffProg;
  tab.slots = reinterpret_cast<SlotState*>(S + kOffSlot);
  tab.records = records;
  tab.bitmaps = bitmap;
  tab.counts = reinterpret_cast<uint32_t*>(S + kOffCounts);
  tab.touched = reinterpret_cast<uint16_t*>(S + kOffTouched);
  tab.union_map = reinterpret_cast<uint32_t*>(S + kOffUnion);
  tab.union_snap = reinterpret_cast<uint32_t*>(S + kOffSnap);
  tab.done = reinterpret_cast<HostDone*>(S + kOffDone);
  tab.record_cap = record_cap;
  tab.redzone = redzone;
  tab.iter_budget = iter_budget;
  tab.flags = (flags & (CUFZ_CF_NO_DIGEST)) | (bitmap ? CUFZ_CF_KEEP_BITMAPS : 0);

  LaunchShape shape;
  memset(&shape, 0, sizeof(shape));
  shape.cta_threads = 256;
  shape.max_regs = P.hdr.n_regs;
  shape.max_prog_bytes = (P.blob_bytes + 15u) & ~15u;
  const uint32_t smem = interp_smem_bytes(shape);
  cudaError_t e = cudaSuccess;
  // raise (never lower) the kernel's dynamic shared memory limit
  cudaFuncAttributes fa;
  if (persistent_func_attributes(&fa) != cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && (uint32_t)fa.maxDynamicSharedSizeBytes < smem) e = set_kernel_smem(smem);
  int occ = 0, sms = 0;
  if (e == cudaSuccess) e = persistent_occupancy(shape.cta_threads, smem, &occ);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
  shape.ctas = std::min<uint32_t>((uint32_t)(occ * sms), n_items);
  shape.smem_bytes = smem;
  // everything that must start at zero (the last call's contents stay otherwise)
  if (e == cudaSuccess) e = cudaMemsetAsync(S + kOffCounts, 0, 4u * kEdgeCount, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S + kOffUnion, 0, 2u * kBitmapBytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S + kOffDone, 0, sizeof(HostDone), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S + kOffSlot, &s0, sizeof(s0), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S + kOffProg, P.blob, P.blob_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S + kOffBatch, img.p, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = launch_persistent(tab, reinterpret_cast<const BatchHdr*>(S + kOffBatch), shape, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(result, S + kOffDone, sizeof(cufz_result), cudaMemcpyDefault, st);
  // the host-side images above are freed on return: wait for the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CUFZ_E_CUDA;
  }
  return CUFZ_OK;
}

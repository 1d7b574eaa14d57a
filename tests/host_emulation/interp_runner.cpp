// TEST-ONLY host runner for the bytecode interpreter (tests/test_interp_host.py):
// the interpreter's warp loop (interp_kernel.cuh) inside the work-item loop
// of device_common.cuh, as the persistent interpreter kernel runs it, on one
// CTA of one warp whose 32 lanes are host threads (simt_shim.h).  Every input
// of the job has its own slot; all of them form one batch whose items the
// CTA pulls in turn, and the CTA that completes an input's last item
// finalizes it (bitmap, union, result), as on the device.  Programs are
// loaded with the library's load_program and inputs built with its
// fill_dev_input (input_build.h).
//
// Job file (little-endian u32 unless noted): n_programs, record_cap,
// redzone, iter_budget, item_threads, flags (CUFZ_CF_NO_PRUNE,
// CUFZ_CF_NO_DIGEST); per program its byte size and bytes; n_inputs; per
// input the 128-byte cufz_input, n_planned and the planned thread ids.
// Output per input: the result (as the compiled path's host runner writes
// it), its records and its bitmap.
#include "simt_shim.h"

#include "interp_kernel.cuh"

#include <thread>
#include <vector>

thread_local shim_dim3 threadIdx = {0, 0, 0};
ShimWarp g_shim_warp;
std::mutex g_shim_atomic;

#include "input_build.h"  // the library's own fill_dev_input
extern "C" int shim_load_blob(const void* bytes, size_t nbytes, int prune, uint8_t** blob,
                              uint32_t* blob_bytes, uint32_t* n_regs, uint32_t* n_bufs,
                              uint32_t* shared_mask);

struct HostResult {
  int32_t status;
  uint32_t flags;
  uint64_t n_accesses, n_violations, first_key, digest, n_branch, n_ops, n_threads;
  uint32_t n_records, n_edges;
};

static bool rd(FILE* f, void* p, size_t n) { return fread(p, 1, n, f) == n; }

static size_t up16(size_t n) { return (n + 15) & ~(size_t)15; }

int main(int argc, char** argv) {
  using namespace cufz;
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  FILE* o = fopen(argv[2], "wb");
  if (!f || !o) return 2;
  uint32_t h[6];
  if (!rd(f, h, sizeof h)) return 3;
  const uint32_t n_progs = h[0], cap = h[1], redzone = h[2], budget = h[3], item = h[4];
  const uint32_t flags = h[5];

  // programs: loaded blobs, one after another in the program area
  std::vector<uint8_t> area;
  std::vector<uint32_t> prog_off(n_progs), prog_bytes(n_progs), n_bufs(n_progs), shared(n_progs);
  uint32_t max_regs = 1, max_prog_bytes = 16;
  for (uint32_t p = 0; p < n_progs; p++) {
    uint32_t nb = 0;
    if (!rd(f, &nb, 4)) return 3;
    std::vector<uint8_t> bytes(nb);
    if (!rd(f, bytes.data(), nb)) return 3;
    uint8_t* blob = nullptr;
    uint32_t bb = 0, regs = 0;
    if (shim_load_blob(bytes.data(), nb, !(flags & CUFZ_CF_NO_PRUNE), &blob, &bb, &regs,
                       &n_bufs[p], &shared[p]) != 0)
      return 4;
    prog_off[p] = (uint32_t)area.size();
    prog_bytes[p] = bb;
    area.insert(area.end(), blob, blob + bb);
    area.resize(up16(area.size()), 0);
    free(blob);
    if (regs > max_regs) max_regs = regs;
    if (up16(bb) > max_prog_bytes) max_prog_bytes = (uint32_t)up16(bb);
  }

  // inputs and their work items
  uint32_t n = 0;
  if (!rd(f, &n, 4)) return 3;
  std::vector<DevInput> dins(n);
  std::vector<WorkItem> items;
  std::vector<uint64_t> planned(n, 0);
  for (uint32_t i = 0; i < n; i++) {
    cufz_input in;
    uint32_t n_plan = 0;
    if (!rd(f, &in, sizeof in) || !rd(f, &n_plan, 4)) return 3;
    std::vector<uint32_t> plan(n_plan);
    if (n_plan && !rd(f, plan.data(), 4ull * n_plan)) return 3;
    if (in.program_id >= n_progs) return 4;
    DevInput& d = dins[i];
    fill_dev_input(in, n_bufs[in.program_id], shared[in.program_id], redzone, &d);
    d.slot = i;
    d.prog = in.program_id;
    d.prog_off = prog_off[in.program_id];
    d.prog_bytes = prog_bytes[in.program_id];
    d.seq = 1;
    const size_t first = items.size();
    if (n_plan) {
      for (uint32_t g : plan) items.push_back(WorkItem{i, g, 1u, 0u});
      planned[i] = n_plan;
    } else {
      for (uint64_t g = 0; g < d.n_threads; g += item)
        items.push_back(WorkItem{i, (uint32_t)g,
                                 (uint32_t)(d.n_threads - g < item ? d.n_threads - g : item), 0u});
    }
    d.n_items = (uint32_t)(items.size() - first);
  }
  std::vector<uint8_t> batch_buf(sizeof(BatchHdr) + n * sizeof(DevInput) +
                                 items.size() * sizeof(WorkItem));
  BatchHdr* batch = reinterpret_cast<BatchHdr*>(batch_buf.data());
  batch->n_inputs = n;
  batch->n_items = (uint32_t)items.size();
  batch->inputs_off = sizeof(BatchHdr);
  batch->items_off = sizeof(BatchHdr) + n * sizeof(DevInput);
  memcpy(batch_buf.data() + batch->inputs_off, dins.data(), n * sizeof(DevInput));
  memcpy(batch_buf.data() + batch->items_off, items.data(), items.size() * sizeof(WorkItem));

  // per-slot tables
  std::vector<SlotState> slots(n);
  for (SlotState& s : slots) {
    memset(&s, 0, sizeof s);
    s.first_key = ~0ull;
  }
  std::vector<cufz_violation> records((size_t)n * (cap ? cap : 1));
  std::vector<uint8_t> bitmaps((size_t)n * kBitmapBytes, 0);
  std::vector<uint32_t> counts((size_t)n * kEdgeCount, 0);
  std::vector<uint16_t> touched((size_t)n * kEdgeCount, 0);
  std::vector<uint32_t> union_map(kEdgeCount / 4, 0), union_snap(kEdgeCount / 4, 0);
  std::vector<HostDone> done(n);
  memset(done.data(), 0, n * sizeof(HostDone));
  EngineTables T;
  memset(&T, 0, sizeof T);
  T.progs = area.data();
  T.slots = slots.data();
  T.records = records.data();
  T.bitmaps = bitmaps.data();
  T.counts = counts.data();
  T.touched = touched.data();
  T.union_map = union_map.data();
  T.union_snap = union_snap.data();
  T.done = done.data();
  T.record_cap = cap;
  T.redzone = redzone;
  T.iter_budget = budget;
  T.flags = CUFZ_CF_KEEP_BITMAPS | (flags & CUFZ_CF_NO_DIGEST);

  // the CTA: shared memory for hash table | program | DevInput | registers
  std::vector<uint8_t> smem_buf(kEdgeSmemBytes + max_prog_bytes + kInputSmemBytes +
                                (size_t)max_regs * kRegStride + 16);
  uint8_t* smem = reinterpret_cast<uint8_t*>(up16((size_t)smem_buf.data()));
  auto lane = [&](uint32_t x) {
    threadIdx.x = x;
    uint32_t* hash = reinterpret_cast<uint32_t*>(smem);
    uint8_t* sprog = smem + kEdgeSmemBytes;
    DevInput* sin = reinterpret_cast<DevInput*>(sprog + max_prog_bytes);
    uint8_t* rf = reinterpret_cast<uint8_t*>(sin) + kInputSmemBytes;
    run_items<true, true>(T, batch, 0u, max_regs, max_prog_bytes, hash, sprog, sin,
                          [&](const DevInput* in, uint32_t g0, uint32_t cnt, bool skip) -> bool {
                            if (skip) return false;
                            run_warp(T, in, sprog, rf, hash, g0, cnt, 0u, 1u);
                            return true;
                          });
  };
  std::vector<std::thread> warp;
  for (uint32_t x = 0; x < 32; x++) warp.emplace_back(lane, x);
  for (std::thread& t : warp) t.join();

  for (uint32_t i = 0; i < n; i++) {
    const cufz_result& r = done[i].res;
    if (done[i].seq != 1) return 5;  // never finalized
    HostResult w;
    memset(&w, 0, sizeof w);
    w.status = r.status;
    w.flags = r.flags;
    w.n_accesses = r.n_accesses;
    w.n_violations = r.n_violations;
    w.first_key = r.first_key;
    w.digest = r.digest;
    w.n_branch = r.n_branch;
    w.n_ops = r.n_ops;
    w.n_threads = planned[i] ? planned[i] : r.n_threads;
    w.n_records = r.n_records;
    w.n_edges = r.n_edges;
    fwrite(&w, sizeof w, 1, o);
    fwrite(records.data() + (size_t)i * cap, sizeof(cufz_violation), w.n_records, o);
    fwrite(bitmaps.data() + (size_t)i * kBitmapBytes, 1, kBitmapBytes, o);
  }
  fclose(o);
  fclose(f);
  return 0;
}

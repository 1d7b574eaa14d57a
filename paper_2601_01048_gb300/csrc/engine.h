// Internal layouts of the cufz engine: the loaded (pruned, register-allocated)
// device program, the per-input descriptor a batch carries to the device, the
// per-slot device state and the arena layout.  Host runtime, loader and
// kernels include this; the CPU oracle does not.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "input_build.h"
#include "layout.h"

namespace cufz {

// ---------------------------------------------------------------- loader
// A program's decoded form for the PREX check (Sec. 5.1).
struct PrexInfo;

// Whether the corner threads of input `in` decide its verdict: every branch
// and loop trip uniform, every access index uniform or affine in the thread
// and block indices, no affine value leaving int32 in the launch box.
bool prex_input_ok(const PrexInfo& p, const cufz_input& in, uint32_t iter_budget);

// The corner threads of `in` (every coordinate first or last) as linear ids
// g = block_lin * T + thread_lin, sorted.
std::vector<uint32_t> prex_corners(const cufz_input& in);

// The threads whose verdict is the whole grid's: the corners when
// prex_input_ok holds, else, for a launch whose values are affine in the
// thread and block indices and whose branch conditions are guards on one
// dimension's coordinates each, the corners of the cells the guards cut the
// launch box into.  False when neither holds.
bool prex_plan(const PrexInfo& p, const cufz_input& in, uint32_t iter_budget,
               std::vector<uint32_t>* threads);

// ---------------------------------------------------------------- inputs
// launch_rejected, launch_within, fill_dev_input, block_serial_fits: see
// input_build.h (host and device code).

struct LoadedProgram {
  DevProgHdr hdr;
  uint8_t* blob = nullptr;   // host copy of the device blob
  uint32_t blob_bytes = 0;
  cufz_prog_stats stats{};
  uint32_t n_bufs = 0;
  uint32_t shared_mask = 0;
  std::shared_ptr<const PrexInfo> prex;  // the program as given, for the PREX check
  // runs only in the block-serial form (compiled path; see prepare_barriers),
  // for launches of at most kBlkMaxThreads threads per block and
  // kBlkSharedBytes bytes of shared buffers
  bool block_serial = false;
};

// Decodes and validates program bytes; fills `out` (device blob built with or
// without pruning).  Returns CUFZ_OK or CUFZ_E_INVALID_PROGRAM.
cufz_status load_program(const void* bytes, size_t nbytes, bool prune, LoadedProgram* out);
void free_program(LoadedProgram* p);

// Dynamic shared memory of a persistent compiled-kernel launch whose module
// holds path-mode programs: the path table (4096 slots of 12 bytes; the
// kPathTableBytes of jit_kernel.cuh).
constexpr uint32_t kJitPathTableBytes = 4096u * 12u;

// Resident CTAs per SM the compiled kernel's registers must allow when the
// config leaves it open: 3 x 256 threads gives it 85 registers a thread.
constexpr uint32_t kJitMinCtasDefault = 3;

// The compiled path's module source: the included programs' functions (from
// jit_source), the dispatcher and the kernels.
// lanes[k] is program k's lane mapping: test threads per lane per
// iteration of its work-item loop (1, 2 or 4; 1 where absent).
std::string jit_module_source(const std::vector<std::string>& prog_src,
                              const std::vector<uint8_t>& include, bool plain_kernel,
                              uint32_t min_ctas, uint32_t cta_threads,
                              const std::vector<uint8_t>& lanes);

// CUDA source of one program's work-item function `cufz_prog_<index>` for
// the compiled path (see jit_kernel.cuh).
cufz_status jit_source(const void* bytes, size_t nbytes, bool prune, bool digest,
                       uint32_t index, std::string* out);

// ---------------------------------------------------------------- kernels
struct LaunchShape {
  uint32_t cta_threads;
  uint32_t ctas;
  uint32_t smem_bytes;
  uint32_t max_regs;     // register-file registers per lane to reserve
  uint32_t max_prog_bytes;
};

// Dynamic shared memory of an interpreter launch of shape s: the CTA's
// edge table, the staged program, the staged input and the warps' register
// files.
uint32_t interp_smem_bytes(const LaunchShape& s);

cudaError_t launch_persistent(const EngineTables& T, const BatchHdr* d_batch, const LaunchShape& s,
                              cudaStream_t st);
cudaError_t launch_plain(const EngineTables& T, const BatchHdr* d_batch, uint32_t input_index,
                         uint32_t n_blocks_grid, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_clear(void* p, uint64_t bytes, uint64_t pattern, cudaStream_t st);
cudaError_t launch_int32_peak(uint32_t* out, uint32_t blocks, uint32_t threads, uint32_t iters,
                              cudaStream_t st);
cudaError_t persistent_occupancy(uint32_t cta_threads, uint32_t smem_bytes, int* ctas_per_sm);
cudaError_t persistent_func_attributes(cudaFuncAttributes* out);
cudaError_t set_kernel_smem(uint32_t smem_bytes);

// ---------------------------------------------------------------- campaign
// What the device fuzzing campaign (campaign.cu) takes from a context: the
// tables and compiled kernel its rounds launch, the launch limits, a table
// of the loaded programs (4 words each: bit 0 loaded, bits 8..15 buffers,
// bits 16..24 shared mask, bit 31 block-serial; blob offset; blob bytes; 0)
// and the slots reserved for its children.
struct CampaignEnv {
  int device = 0;
  EngineTables T{};
  const void* jit_kernel = nullptr;
  uint32_t jit_ctas = 0, cta_threads = 0;
  uint32_t item_threads = 0;
  uint64_t max_threads = 0;
  uint32_t redzone = 0;
  uint32_t n_programs = 0;
  std::vector<uint32_t> progs;
  std::vector<uint32_t> slots;
  uint64_t module_gen = 0;
  uint32_t jit_smem = 0;  // the persistent kernel's dynamic shared memory (path table)
};

// Reserves n_slots free slots for a campaign, sets every loaded program to
// the compiled path and builds the module if needed.  While a campaign is
// attached the module is not rebuilt: a change of programs, paths or lane
// mappings makes later submits return CUFZ_E_BUSY until it detaches.
cufz_status campaign_attach(cufz_ctx* c, uint32_t n_slots, uint32_t item_threads, CampaignEnv* env);
void campaign_detach(cufz_ctx* c, const std::vector<uint32_t>& slots);
// Whether the context still runs the module the campaign captured.
bool campaign_env_current(cufz_ctx* c, const CampaignEnv& env);

}  // namespace cufz

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
// Launch shapes CUDA would refuse (a zero dimension, more than 1024 threads
// per block, block.z > 64, grid.x > 2^31 - 1, grid.y or grid.z > 65535):
// such inputs complete as CUFZ_ST_INVALID_CONFIG without running.
bool launch_rejected(const cufz_input& in);

// Whether a launch CUDA accepts has at most max_threads test threads; if so
// their number goes to *n_threads (when not null).  The block count is
// compared with max_threads / (threads per block) before any product, so a
// grid whose thread count would wrap 64 bits is refused, not wrapped.
bool launch_within(const cufz_input& in, uint64_t max_threads, uint64_t* n_threads);

// The part of a DevInput that follows from the input and its program: launch
// shape, division magics, arguments, buffer lengths, redzone-separated
// virtual bases (per space: base_0 = R, base_k+1 = align256(base_k + len_k
// + R)) and per-width index limits.  Zeroes the rest (slot, program
// placement, items, ticket, sequence), which the caller sets.
void fill_dev_input(const cufz_input& in, uint32_t n_bufs, uint32_t shared_mask, uint32_t redzone,
                    DevInput* d);

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

// unsigned division helpers shared by host (magic computation) and device
__host__ __device__ inline uint64_t div_magic(uint32_t d) {
  return d <= 1 ? 0ull : (~0ull / d) + 1ull;
}

}  // namespace cufz

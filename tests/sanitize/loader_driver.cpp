// Host-only driver for the loader and the PREX analysis built with
// AddressSanitizer and UndefinedBehaviorSanitizer
// (tests/test_loader_sanitized.py).  Reads a
// corpus of (program, inputs) records and runs every host-side analysis on
// each: validation, pruning, code generation for both pruning modes,
// loading, the PREX check and the PREX plan, and the input mutator.  Any sanitizer report aborts
// the process with a non-zero status.
//
// Corpus record: u32 program bytes, u32 input count, the program, then the
// 128-byte cufz_input records.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

using namespace cufz;

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  std::vector<uint8_t> buf;
  uint8_t chunk[65536];
  size_t n;
  while ((n = fread(chunk, 1, sizeof chunk, f)) > 0) buf.insert(buf.end(), chunk, chunk + n);
  fclose(f);
  size_t pos = 0;
  long programs = 0, valid = 0, planned = 0;
  while (pos + 8 <= buf.size()) {
    uint32_t plen, nin;
    memcpy(&plen, &buf[pos], 4);
    memcpy(&nin, &buf[pos + 4], 4);
    pos += 8;
    if (pos + plen + (size_t)nin * sizeof(cufz_input) > buf.size()) return 3;
    // exact-size copies, so that any read past the program is caught
    std::vector<uint8_t> prog(buf.begin() + pos, buf.begin() + pos + plen);
    pos += plen;
    std::vector<cufz_input> ins(nin);
    memcpy(ins.data(), &buf[pos], (size_t)nin * sizeof(cufz_input));
    pos += (size_t)nin * sizeof(cufz_input);
    programs++;
    if (cufz_validate_program(prog.data(), plen) != CUFZ_OK) continue;
    valid++;
    std::vector<uint8_t> pruned(plen);
    size_t pruned_bytes = 0;
    cufz_prog_stats stats;
    cufz_prune_program(prog.data(), plen, pruned.data(), pruned.size(), &pruned_bytes, &stats);
    for (int prune = 0; prune < 2; prune++) {
      std::string src;
      jit_source(prog.data(), plen, prune != 0, true, 0, &src);
    }
    LoadedProgram lp;
    if (load_program(prog.data(), plen, true, &lp) == CUFZ_OK) free_program(&lp);
    std::vector<uint32_t> threads(4096);
    std::vector<cufz_input> mutated(ins);
    for (cufz_input& in : mutated) in.program_id = 0;
    const uint8_t n_bufs = prog[9];
    uint64_t state = (uint64_t)programs;
    cufz_mutate_inputs(mutated.data(), (uint32_t)mutated.size(), &n_bufs, 1, &state);
    for (const cufz_input& in : ins) {
      uint32_t eligible = 0, nt = 0;
      cufz_prex_check(prog.data(), plen, &in, 0, &eligible);
      cufz_prex_plan(prog.data(), plen, &in, 0, threads.data(), (uint32_t)threads.size(), &nt);
      cufz_prex_plan(prog.data(), plen, &in, 3, threads.data(), 0, &nt);
      planned += nt > 0;
    }
  }
  printf("programs %ld valid %ld planned %ld\n", programs, valid, planned);
  return 0;
}

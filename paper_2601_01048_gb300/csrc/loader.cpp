// Program loader of the cufz engine: decodes and validates the program
// format, prunes it (AXIPrune's MathElimination, Sec. 5.2, Alg. 2: an op
// whose result reaches no memory-access index and no branch stays out),
// allocates device registers and emits the device program blob.
//
// The prune is a backward slice computed by liveness over the structured
// control-flow graph: roots are every load/store index, every IF condition
// and every LOOP trip expression; stored values are not roots (stores are
// checked, not performed); loads stay as checked accesses even when their
// value is dead.  Every access of every thread therefore keeps its index,
// site and ordinal, and every branch keeps its decision (Sec. 5.2, "all
// memory accesses are preserved exactly as in the original GPU program").
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <string>
#include <array>
#include <vector>

#include "checked_ops.h"
#include "ir.h"

namespace cufz {
namespace {

uint16_t get16(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }
uint32_t get32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

bool width_ok(int32_t w) { return w == 1 || w == 4 || w == 8 || w == 16; }

}  // namespace

bool decode(const uint8_t* p, size_t n, Ir* ir) {
  if (!p || n < 32) return false;
  if (get32(p) != kMagic || get16(p + 4) != 1) return false;
  int n_ops = get16(p + 6);
  ir->n_regs = p[8];
  ir->n_bufs = p[9];
  ir->n_sites = p[10];
  ir->shared_mask = get16(p + 12);
  ir->seed = get32(p + 16);
  ir->flags = p[11];
  if ((ir->flags & ~kPfSharedStores) || get16(p + 14) || get32(p + 20) || get32(p + 24) ||
      get32(p + 28))
    return false;
  if (n_ops < 1 || n_ops > kMaxOps || ir->n_bufs > kMaxBufs) return false;
  if (ir->shared_mask >> ir->n_bufs) return false;
  if (n != 32u + 4u * (size_t)ir->n_sites + 8u * (size_t)n_ops) return false;
  ir->loc0.resize(ir->n_sites);
  ir->loc1.resize(ir->n_sites);
  for (int s = 0; s < ir->n_sites; s++) {
    ir->loc0[s] = get16(p + 32 + 4 * s);
    ir->loc1[s] = get16(p + 34 + 4 * s);
  }
  const uint8_t* q = p + 32 + 4 * ir->n_sites;
  ir->ops.resize(n_ops);
  std::vector<int> open;
  int bsites = 0, asites = 0, dsites = 0, hsites = 0, fsites = 0, loops = 0;
  const int R = ir->n_regs;
  auto reg = [R](int r) { return r < R; };
  for (int pc = 0; pc < n_ops; pc++) {
    const uint8_t* w = q + 8 * pc;
    IrOp& o = ir->ops[pc];
    uint8_t opc = w[0];
    int d = w[1], a = w[2], b = w[3];
    int32_t imm = (int32_t)get32(w + 4);
    o.opc = opc;
    o.imm = imm;
    o.depth = (int)open.size();
    bool ok = false;
    if (is_alu_reg(opc)) {
      ok = reg(d) && reg(a) && reg(b) && imm == 0;
      o.dst = d; o.a = a; o.b = b;
    } else if (is_alu_imm(opc)) {
      ok = reg(d) && reg(a) && b == 0;
      o.dst = d; o.a = a;
    } else {
      switch (opc) {
        case B_NOP:
          ok = !d && !a && !b && !imm;
          o.kept = false;
          break;
        case B_BAR:  // top level only; never executed (see barriers_eliminable)
          ok = !d && !a && !b && !imm && open.empty();
          o.kept = false;
          break;
        case B_SREG:
          ok = reg(d) && !a && !b && imm >= 0 && imm <= 15;
          o.dst = d; o.sreg = imm;
          break;
        case B_IMM:
          ok = reg(d) && !a && !b;
          o.dst = d;
          break;
        case B_MOV:
          ok = reg(d) && reg(a) && !b && !imm;
          o.dst = d; o.a = a;
          break;
        case B_SEL:
          ok = reg(d) && reg(a) && reg(b) && imm >= 0 && imm < R;
          o.dst = d; o.a = a; o.b = b; o.c = imm;
          break;
        case B_DIV:
        case B_REM:
          ok = reg(d) && reg(a) && reg(b) && !imm;
          o.dst = d; o.a = a; o.b = b; o.site = dsites++;
          break;
        case B_HALLOC:
          ok = reg(d) && reg(a) && !b && !imm;
          o.dst = d; o.a = a; o.site = hsites++;
          break;
        case B_HFREE:
          ok = !d && reg(a) && !b && !imm;
          o.a = a; o.site = fsites++;
          break;
        case B_HLD:
        case B_HST:  // b: the handle; HST's value register (d) is never a root
          ok = reg(d) && reg(a) && reg(b) && width_ok(imm);
          if (opc == B_HLD) o.dst = d;
          o.a = a; o.b = b; o.width = imm; o.site = asites++;
          break;
        case B_LD:
        case B_ST:
          ok = reg(d) && reg(a) && b < ir->n_bufs && width_ok(imm);
          if (opc == B_LD) o.dst = d; else o.b = d;  // ST: value register, never a root
          o.a = a; o.buf = b; o.width = imm; o.site = asites++;
          break;
        case B_IF:
          ok = !d && reg(a) && !b && !imm && (int)open.size() < kMaxDepth;
          o.a = a; o.site = bsites++;
          if (ok) open.push_back(pc);
          break;
        case B_LOOP:
          ok = reg(d) && reg(a) && !b && imm >= 0 && imm <= 65535 && (int)open.size() < kMaxDepth;
          o.dst = d; o.a = a; o.site = bsites++; o.trip = kTripBase + loops++;
          if (ok) open.push_back(pc);
          break;
        case B_ELSE:
          ok = !d && !a && !b && !imm && !open.empty() && ir->ops[open.back()].opc == B_IF &&
               ir->ops[open.back()].else_pc < 0;
          if (ok) {
            ir->ops[open.back()].else_pc = pc;
            o.head_pc = open.back();
            o.depth = (int)open.size() - 1;
          }
          break;
        case B_ENDIF:
          ok = !d && !a && !b && !imm && !open.empty() && ir->ops[open.back()].opc == B_IF;
          if (ok) {
            o.head_pc = open.back();
            ir->ops[open.back()].end_pc = pc;
            open.pop_back();
            o.depth = (int)open.size();
          }
          break;
        case B_ENDLOOP:
          ok = !d && !a && !b && !imm && !open.empty() && ir->ops[open.back()].opc == B_LOOP;
          if (ok) {
            o.head_pc = open.back();
            ir->ops[open.back()].end_pc = pc;
            open.pop_back();
            o.depth = (int)open.size();
          }
          break;
        default:
          ok = false;
      }
    }
    if (!ok) return false;
  }
  if (!open.empty() || bsites != ir->n_sites) return false;
  for (auto& o : ir->ops) {
    if (o.opc == B_ELSE) o.end_pc = ir->ops[o.head_pc].end_pc;
    if (o.opc == B_ENDLOOP) {
      const IrOp& h = ir->ops[o.head_pc];
      o.dst = h.dst;
      o.trip = h.trip;
      o.site = h.site;
    }
  }
  // a loop counter is read-only in its own body
  for (int pc = 0; pc < n_ops; pc++) {
    const IrOp& h = ir->ops[pc];
    if (h.opc != B_LOOP) continue;
    for (int j = pc + 1; j < h.end_pc; j++) {
      const IrOp& o = ir->ops[j];
      bool writes = (o.opc == B_SREG || o.opc == B_IMM || o.opc == B_MOV || o.opc == B_SEL ||
                     o.opc == B_LD || o.opc == B_LOOP || o.opc == B_DIV || o.opc == B_REM ||
                     o.opc == B_HALLOC || o.opc == B_HLD || is_alu_reg(o.opc) ||
                     is_alu_imm(o.opc));
      if (writes && o.dst == h.dst) return false;
    }
  }
  ir->n_access = asites;
  ir->n_div = dsites;
  ir->n_alloc = hsites;
  ir->n_free = fsites;
  ir->n_loops = loops;
  ir->nv = kTripBase + loops;
  return true;
}

namespace {

// ------------------------------------------------------------ dataflow

struct Bits {
  std::vector<uint64_t> w;
  explicit Bits(int n = 0) : w((n + 63) / 64, 0) {}
  void set(int i) { w[i >> 6] |= 1ull << (i & 63); }
  void clr(int i) { w[i >> 6] &= ~(1ull << (i & 63)); }
  bool get(int i) const { return (w[i >> 6] >> (i & 63)) & 1; }
  bool operator==(const Bits& o) const { return w == o.w; }
  void or_with(const Bits& o) {
    for (size_t k = 0; k < w.size(); k++) w[k] |= o.w[k];
  }
};

// Uses and defs of one op.  `sreg_as_pseudo`: SREG reads its special
// register (device IR) instead of being a constant def (format level).
void uses_defs(const IrOp& o, bool device_ir, int* U, int* nu, int* D, int* nd) {
  *nu = *nd = 0;
  if (!o.kept) return;
  uint8_t opc = o.opc;
  if (is_alu_reg(opc)) {
    U[(*nu)++] = o.a; U[(*nu)++] = o.b; D[(*nd)++] = o.dst;
    return;
  }
  if (is_alu_imm(opc)) {
    U[(*nu)++] = o.a; D[(*nd)++] = o.dst;
    return;
  }
  switch (opc) {
    case B_SREG:
      if (device_ir) U[(*nu)++] = kSregBase + o.sreg;
      D[(*nd)++] = o.dst;
      break;
    case B_IMM: D[(*nd)++] = o.dst; break;
    case B_MOV: U[(*nu)++] = o.a; D[(*nd)++] = o.dst; break;
    case B_SEL: U[(*nu)++] = o.a; U[(*nu)++] = o.b; U[(*nu)++] = o.c; D[(*nd)++] = o.dst; break;
    case B_LD:
      U[(*nu)++] = o.a;
      if (!(device_ir && o.value_dead)) D[(*nd)++] = o.dst;
      break;
    case B_ST:
      U[(*nu)++] = o.a;
      if (o.value_live) U[(*nu)++] = o.b;
      break;
    case B_HALLOC: U[(*nu)++] = o.a; D[(*nd)++] = o.dst; break;
    case B_HFREE: U[(*nu)++] = o.a; break;
    case B_HLD:  // the handle and the index decide the check; the value reads 0
      U[(*nu)++] = o.a; U[(*nu)++] = o.b;
      if (!(device_ir && o.value_dead)) D[(*nd)++] = o.dst;
      break;
    case B_HST: U[(*nu)++] = o.a; U[(*nu)++] = o.b; break;
    case B_DIV:
    case B_REM:  // a check: the divisor always, the dividend while the result is live
      U[(*nu)++] = o.b;
      if (!o.value_dead) U[(*nu)++] = o.a;
      if (!(device_ir && o.value_dead)) D[(*nd)++] = o.dst;
      break;
    case B_IF: U[(*nu)++] = o.a; break;
    case B_LOOP:
      U[(*nu)++] = o.a;
      D[(*nd)++] = o.dst;
      if (device_ir) D[(*nd)++] = o.trip;
      break;
    case B_ENDLOOP:
      U[(*nu)++] = o.dst;
      if (device_ir) U[(*nu)++] = o.trip;
      D[(*nd)++] = o.dst;
      break;
    default: break;
  }
}

int successors(const Ir& ir, int pc, int* S) {
  const IrOp& o = ir.ops[pc];
  int n = 0;
  int N = (int)ir.ops.size();
  auto push = [&](int t) {
    if (t < N) S[n++] = t;
  };
  switch (o.opc) {
    case B_IF:
      push(pc + 1);
      push(o.else_pc >= 0 ? o.else_pc + 1 : o.end_pc);
      break;
    case B_ELSE: push(o.end_pc); break;
    case B_LOOP: push(pc + 1); push(o.end_pc + 1); break;
    case B_ENDLOOP: push(o.head_pc + 1); push(pc + 1); break;
    default: push(pc + 1); break;
  }
  return n;
}

struct Liveness {
  std::vector<Bits> in, out;
};

Liveness liveness(const Ir& ir, bool device_ir) {
  int N = (int)ir.ops.size();
  Liveness L;
  L.in.assign(N, Bits(ir.nv));
  L.out.assign(N, Bits(ir.nv));
  bool changed = true;
  int U[4], D[4], S[2], nu, nd;
  while (changed) {
    changed = false;
    for (int pc = N - 1; pc >= 0; pc--) {
      Bits out(ir.nv);
      int ns = successors(ir, pc, S);
      for (int k = 0; k < ns; k++) out.or_with(L.in[S[k]]);
      uses_defs(ir.ops[pc], device_ir, U, &nu, D, &nd);
      Bits in = out;
      for (int k = 0; k < nd; k++) in.clr(D[k]);
      for (int k = 0; k < nu; k++) in.set(U[k]);
      if (!(out == L.out[pc]) || !(in == L.in[pc])) {
        L.out[pc] = std::move(out);
        L.in[pc] = std::move(in);
        changed = true;
      }
    }
  }
  return L;
}

bool is_value_op(uint8_t opc) {
  return opc == B_SREG || opc == B_IMM || opc == B_MOV || opc == B_SEL || is_alu_reg(opc) ||
         is_alu_imm(opc);
}

// MathElimination: drop value ops whose result is dead, to a fixed point.
// A division stays as a check (its divisor decides the fault); once its
// result is dead its dividend is no longer a use.
void prune(Ir* ir) {
  for (;;) {
    Liveness L = liveness(*ir, false);
    bool changed = false;
    for (size_t pc = 0; pc < ir->ops.size(); pc++) {
      IrOp& o = ir->ops[pc];
      if (o.kept && is_value_op(o.opc) && !L.out[pc].get(o.dst)) {
        o.kept = false;
        changed = true;
      }
      if ((o.opc == B_DIV || o.opc == B_REM) && !o.value_dead && !L.out[pc].get(o.dst)) {
        o.value_dead = true;
        changed = true;
      }
    }
    if (!changed) {
      for (size_t pc = 0; pc < ir->ops.size(); pc++) {
        IrOp& o = ir->ops[pc];
        if (o.opc == B_LD || o.opc == B_HLD) o.value_dead = !L.out[pc].get(o.dst);
      }
      return;
    }
  }
}

// Replaces uses of a register defined once, at depth 0, by SREG id, with the
// special register itself (the def dominates every later use).
void propagate_sregs(Ir* ir) {
  int N = (int)ir->ops.size();
  std::vector<int> ndefs(256, 0), defpc(256, -1);
  int U[4], D[4], nu, nd;
  for (int pc = 0; pc < N; pc++) {
    uses_defs(ir->ops[pc], true, U, &nu, D, &nd);
    for (int k = 0; k < nd; k++)
      if (D[k] < 256) {
        ndefs[D[k]]++;
        defpc[D[k]] = pc;
      }
  }
  for (int r = 0; r < 256; r++) {
    if (ndefs[r] != 1) continue;
    IrOp& def = ir->ops[defpc[r]];
    if (def.opc != B_SREG || def.depth != 0) continue;
    int pseudo = kSregBase + def.sreg;
    bool early_use = false;
    for (int pc = 0; pc <= defpc[r] && !early_use; pc++) {
      uses_defs(ir->ops[pc], true, U, &nu, D, &nd);
      for (int k = 0; k < nu; k++) early_use |= (U[k] == r);
    }
    if (early_use) continue;
    for (int pc = defpc[r] + 1; pc < N; pc++) {
      IrOp& o = ir->ops[pc];
      if (!o.kept) continue;
      if (o.a == r) o.a = pseudo;
      if (o.c == r) o.c = pseudo;
      if (o.b == r && o.opc != B_ST) o.b = pseudo;
      if (o.opc == B_ST && o.b == r) o.b = o.value_live ? pseudo : -1;
    }
    def.kept = false;
  }
}

// Interval register allocation: each vreg's live range is the hull of the
// pcs where it is live or defined; overlapping hulls get distinct registers.
// Returns the register count; map[v] = register or -1.
int allocate(const Ir& ir, bool device_ir, std::vector<int>* map, Bits* live_at_entry) {
  int N = (int)ir.ops.size();
  Liveness L = liveness(ir, device_ir);
  std::vector<int> lo(ir.nv, N + 1), hi(ir.nv, -1);
  int U[4], D[4], nu, nd;
  auto touch = [&](int v, int pc) {
    lo[v] = std::min(lo[v], pc);
    hi[v] = std::max(hi[v], pc);
  };
  for (int pc = 0; pc < N; pc++) {
    for (int v = 0; v < ir.nv; v++)
      if (L.in[pc].get(v) || L.out[pc].get(v)) touch(v, pc);
    uses_defs(ir.ops[pc], device_ir, U, &nu, D, &nd);
    for (int k = 0; k < nu; k++) touch(U[k], pc);
    for (int k = 0; k < nd; k++) touch(D[k], pc);
  }
  *live_at_entry = N ? L.in[0] : Bits(ir.nv);
  std::vector<int> order;
  for (int v = 0; v < ir.nv; v++)
    if (hi[v] >= 0) {
      if (v >= kSregBase && v < kTripBase) lo[v] = -1;  // defined by the prologue
      order.push_back(v);
    }
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    return lo[x] != lo[y] ? lo[x] < lo[y] : x < y;
  });
  map->assign(ir.nv, -1);
  std::vector<int> reg_end;  // last pc of the interval occupying each register
  for (int v : order) {
    int r = -1;
    for (size_t k = 0; k < reg_end.size(); k++)
      if (reg_end[k] < lo[v]) {
        r = (int)k;
        break;
      }
    if (r < 0) {
      r = (int)reg_end.size();
      reg_end.push_back(0);
    }
    reg_end[r] = hi[v];
    (*map)[v] = r;
  }
  return (int)reg_end.size();
}

void put16(std::vector<uint8_t>& v, uint16_t x) {
  v.push_back(x & 0xFF);
  v.push_back(x >> 8);
}
void put32(std::vector<uint8_t>& v, uint32_t x) {
  for (int k = 0; k < 4; k++) v.push_back((x >> (8 * k)) & 0xFF);
}

int log2w(int w) { return w == 1 ? 0 : w == 4 ? 2 : w == 8 ? 3 : 4; }

void fill_stats(const Ir& ir, int n_in, int regs_alloc, cufz_prog_stats* st) {
  if (!st) return;
  memset(st, 0, sizeof(*st));
  st->n_ops_in = (uint32_t)n_in;
  uint32_t kept = 0, dead = 0;
  for (const auto& o : ir.ops) {
    if (o.kept && o.opc != B_NOP) kept++;
    if (o.kept && o.opc == B_LD && o.value_dead) dead++;
  }
  st->n_ops_kept = kept;
  st->n_regs_in = (uint32_t)ir.n_regs;
  st->n_regs_alloc = (uint32_t)regs_alloc;
  st->n_access_sites = (uint32_t)ir.n_access;
  st->n_branch_sites = (uint32_t)ir.n_sites;
  st->n_loads_value_dead = dead;
}

}  // namespace

// A shared load whose value is dead after MathElimination reaches no root
// on any path (the liveness over the structured control flow may only
// over-approximate), and stored values are not roots.
bool barriers_eliminable(const Ir& ir) {
  if (!(ir.flags & kPfSharedStores)) return true;
  Ir pruned = ir;
  prune(&pruned);
  for (const IrOp& o : pruned.ops)
    if (o.opc == B_LD && ((ir.shared_mask >> o.buf) & 1u) && !o.value_dead) return false;
  return true;
}

bool prepare_barriers(Ir* ir) {
  if (barriers_eliminable(*ir)) return true;
  for (const IrOp& o : ir->ops)
    if (o.opc == B_DIV || o.opc == B_REM || is_heap_op(o.opc)) return false;
  ir->block_serial = true;
  for (IrOp& o : ir->ops)
    if (o.opc == B_ST && ((ir->shared_mask >> o.buf) & 1u)) o.value_live = true;
  return true;
}


// ------------------------------------------------------------ code generator
// Emits two __device__ functions for program `index`, both with the pruned
// program as straight-line CUDA: program registers become int32 locals (all 0
// at thread start, as in the program semantics), structured IF/LOOP become
// C++ if/for, and every access is an inline bounds check with constant
// buffer, width and site.
//  - cufz_prog_K(g0, g_end) runs a work item (one test thread per CUDA
//    thread): counts, digest and AFL edges (constant LOC values) inline, and
//    no record code, so the per-access path is compare-and-count.  A thread
//    that violated calls the record function at its end while the input's
//    record area still has room, and the first violating thread of each lane
//    calls it for the first-violation key.
//  - cufz_prog_K_rec(g, write) re-runs test thread g with no coverage, digest
//    or counts: it writes the thread's violation records (if `write`) and
//    returns the ordinal of its first violation.
namespace {

// Programs with at least this many kept branch sites get compact code.
constexpr int kCompactSites = 24;
// Programs of at most this many kept ops read their launch constants and
// arguments once per work item, before the loop over the lane's test
// threads; larger ones read them inside it (from the CTA's shared copy of
// the input), which keeps them out of registers the program needs.
constexpr int kHoistMaxOps = 24;

struct Gen {
  const Ir& ir;
  std::string& o;
  int index;
  bool digest_ = true;
  bool rec_ = false;  // emitting the record function
  bool no_counts_ = false;  // a loop body whose counts are added after the loop
  // Compact code for programs with many branch sites: the edge update and
  // the seeded-content hash of a live load become calls of one shared copy
  // instead of inline code at every site, so the program's code stays small
  // enough for the instruction caches (a branch-heavy program's warps
  // diverge and walk most of its code).
  bool compact_ = false;
  bool hoist_ = false;  // launch constants and arguments read before the loop
  // Path mode, for compact programs without loops and with at most 64 branch
  // sites: each site runs at most once per test thread and sites run in
  // program order, so a thread's edges and counts follow from its path, which
  // its sites' outcome bits fix (po0/po1, the two halves of a 64-bit mask,
  // set in taken arms).  At its end a thread counts its path in the CTA's
  // path table (jit_path_count); after the work item the CTA replays each
  // distinct path once through the program's walk table (jit_path_flush),
  // adding the path's count to its edges and counts.  A loop-free thread's
  // ops, accesses and branch evaluations are bounded by the program (12, 12
  // and 8 bits of the walk table's packed counts).
  bool path_ = false;
  // Block-serial function (a program whose performed shared stores need
  // their barriers): accesses perform shared stores and loads in the block's
  // bytes and write their records at once; a budget stop ends the thread's
  // part of the current phase (stop_code_ and its label).
  bool blk_ = false;
  std::string stop_code_ = "acc.budget_hit = true; goto cufz_done;";
  bool has_loop = false;
  // The AFL state prev where the code being emitted runs, when the
  // generator knows it (count function, not in path mode): kp_ with value
  // pv_, else the run-time variable prev holds it.  After a branch site each
  // successor knows it (LOC[site][outcome] >> 1), so a site's edge is a
  // choice between two constants wherever the site before it is known,
  // and prev is written only where paths with different values join (the
  // end of an IF, a loop head).
  bool sp_ = false;
  bool kp_ = false;
  uint32_t pv_ = 0;

  // Makes the run-time variable hold prev (at a join or a loop head).
  void materialize(int ind) {
    if (sp_ && kp_) line(ind, "prev = " + hex32(pv_) + ";");
    kp_ = false;
  }

  void line(int ind, const std::string& t) {
    o.append((size_t)ind * 2, ' ');
    o += t;
    o += '\n';
  }
  static std::string hex32(uint32_t v) {
    char b[24];
    snprintf(b, sizeof b, "0x%08Xu", v);
    return b;
  }
  static std::string r(int v) { return "r" + std::to_string(v); }
  static std::string imm(int32_t v) { return "((int32_t)" + hex32((uint32_t)v) + ")"; }

  std::string alu_expr(int op, const std::string& x, const std::string& y) {
    switch (op) {
      case 0: return "(int32_t)((uint32_t)" + x + " + (uint32_t)" + y + ")";
      case 1: return "(int32_t)((uint32_t)" + x + " - (uint32_t)" + y + ")";
      case 2: return "(int32_t)((uint32_t)" + x + " * (uint32_t)" + y + ")";
      case 3: return "(int32_t)((uint32_t)" + x + " << ((uint32_t)" + y + " & 31u))";
      case 4: return "(int32_t)(" + x + " >> ((uint32_t)" + y + " & 31u))";
      case 5: return "(int32_t)((uint32_t)" + x + " >> ((uint32_t)" + y + " & 31u))";
      case 6: return "(int32_t)(" + x + " & " + y + ")";
      case 7: return "(int32_t)(" + x + " | " + y + ")";
      case 8: return "(int32_t)(" + x + " ^ " + y + ")";
      case 9: return "(" + x + " < " + y + " ? " + x + " : " + y + ")";
      case 10: return "(" + x + " > " + y + " ? " + x + " : " + y + ")";
      case 11: return "(int32_t)(" + x + " < " + y + ")";
      case 12: return "(int32_t)(" + x + " <= " + y + ")";
      case 13: return "(int32_t)(" + x + " == " + y + ")";
      case 14: return "(int32_t)(" + x + " != " + y + ")";
      default: return "(int32_t)((uint32_t)" + x + " < (uint32_t)" + y + ")";
    }
  }

  static const char* sreg_name(int id) {
    static const char* n[16] = {"s_tx", "s_ty", "s_tz", "s_ntx", "s_nty", "s_ntz", "s_bx", "s_by",
                                "s_bz", "s_ngx", "s_ngy", "s_ngz", "s_a0", "s_a1", "s_a2", "s_a3"};
    return n[id];
  }

  bool counted(const IrOp& o2) const {
    return o2.kept && ((o2.opc != B_SREG && is_value_op(o2.opc)) || o2.opc == B_DIV ||
                       o2.opc == B_REM || o2.opc == B_HALLOC || o2.opc == B_HFREE);
  }

  // whether ops [pc, end) hold a kept IF or LOOP (a branch site)
  bool has_branch_sites(int pc, int end) const {
    for (; pc < end; pc++)
      if (ir.ops[pc].kept && (ir.ops[pc].opc == B_IF || ir.ops[pc].opc == B_LOOP)) return true;
    return false;
  }

  // ops and accesses of the straight-line run starting at pc (up to the
  // next IF/LOOP or end)
  int run_ops(int pc, int end) const {
    int k = 0;
    while (pc < end) {
      const IrOp& o2 = ir.ops[pc];
      if (o2.opc == B_IF || o2.opc == B_LOOP) break;
      if (counted(o2)) k++;
      pc++;
    }
    return k;
  }
  int run_acc(int pc, int end) const {
    int k = 0;
    while (pc < end) {
      const IrOp& o2 = ir.ops[pc];
      if (o2.opc == B_IF || o2.opc == B_LOOP) break;
      if (o2.kept && (o2.opc == B_LD || o2.opc == B_ST || o2.opc == B_HLD || o2.opc == B_HST)) k++;
      pc++;
    }
    return k;
  }
  // the counter increments of the run starting at pc, including the
  // evaluation of the IF that ends it (always reached once the run starts:
  // a run holds no loop, so no budget stop)
  void run_counts(int ind, int pc, int end) {
    if (rec_ || no_counts_) return;
    const int k = run_ops(pc, end), m = run_acc(pc, end);
    int q = pc;
    while (q < end && ir.ops[q].opc != B_IF && ir.ops[q].opc != B_LOOP) q++;
    const bool ends_at_if = q < end && ir.ops[q].opc == B_IF && ir.ops[q].kept;
    if (path_) return;  // the walk adds the path's counts (seg_)
    if (k) line(ind, "acc.n_ops += " + std::to_string(k) + "u;");
    if (m) line(ind, "acc.n_acc += " + std::to_string(m) + "u;");
    if (ends_at_if) line(ind, "acc.n_branch += 1u;");
  }

  // One branch evaluation's edge.  count: add it to n_branch here (loop
  // heads); an IF's evaluation is counted with the run that ends at it.
  void cover(int ind, int site, const std::string& cond, bool count) {
    if (rec_) return;
    if (path_) return;  // the outcome bit is set in the taken arm; the walk does the rest
    uint32_t l0 = ir.loc0[site], l1 = ir.loc1[site];
    const std::string upd = std::string(count ? " acc.n_branch++;" : "") +
                            (compact_ ? " jit_cover_out(slot, e); }" : " jit_cover(slot, e); }");
    if (!sp_) {
      line(ind, "{ const uint32_t cur = (" + cond + ") ? " + hex32(l1) + " : " + hex32(l0) +
                    "; const uint32_t e = (cur ^ prev) & 0xFFFFu; prev = cur >> 1;" + upd);
      return;
    }
    // prev is not written here: the caller sets what each successor knows
    if (kp_ && !compact_) {
      // both edges are constants: so are their words and bits in the
      // saturated-edge bitmap
      const uint32_t e1 = (l1 ^ pv_) & 0xFFFFu, e0 = (l0 ^ pv_) & 0xFFFFu;
      line(ind, "{ const uint32_t e = (" + cond + ") ? " + hex32(e1) + " : " + hex32(e0) + ";" +
                    (count ? " acc.n_branch++;" : "") + " jit_cover_k(slot, e, (" + cond + ") ? " +
                    std::to_string(e1 >> 5) + "u : " + std::to_string(e0 >> 5) + "u, (" + cond +
                    ") ? " + hex32(1u << (e1 & 31)) + " : " + hex32(1u << (e0 & 31)) + "); }");
    } else if (kp_)
      line(ind, "{ const uint32_t e = (" + cond + ") ? " + hex32((l1 ^ pv_) & 0xFFFFu) + " : " +
                    hex32((l0 ^ pv_) & 0xFFFFu) + ";" + upd);
    else
      line(ind, "{ const uint32_t e = ((" + cond + " ? " + hex32(l1) + " : " + hex32(l0) +
                    ") ^ prev) & 0xFFFFu;" + upd);
  }

  // index limits are read once per function call into constants (a
  // program uses a few (buffer, width) pairs)
  static std::string lim_name(int buf, int lw) { return "L" + std::to_string(buf * 5 + lw); }
  void lim_decls(int ind) {
    for (int k = 0; k < kMaxBufs * 5; k++) {
      bool used = false;
      for (const auto& op : ir.ops)
        if (op.kept && (op.opc == B_LD || op.opc == B_ST) && op.buf * 5 + log2w(op.width) == k) used = true;
      if (used) line(ind, "const uint32_t L" + std::to_string(k) + " = lim[" + std::to_string(k) + "];");
    }
  }

  // An access of width w = 2^lw at index ix is in bounds iff
  // 0 <= ix < floor(len / w); with the limit clamped to 2^31 a single
  // unsigned compare decides it for every int32 index (negative indices
  // wrap to >= 2^31).
  void access(int ind, const IrOp& o2) {
    int lw = log2w(o2.width);
    bool shared = (ir.shared_mask >> o2.buf) & 1u;
    if (blk_) {
      block_access(ind, o2, lw, shared);
      return;
    }
    line(ind, "{");
    line(ind + 1, "const int32_t ix = " + r(o2.a) + ";");
    line(ind + 1, "const bool viol = (uint32_t)ix >= " + lim_name(o2.buf, lw) + ";");
    if (rec_) line(ind + 1, "const int64_t off = (int64_t)ix * " + std::to_string(1 << lw) + ";");
    uint32_t what = (uint32_t)o2.site | ((uint32_t)o2.buf << 16) |
                    ((o2.opc == B_ST ? 1u : 0u) << 20) | ((uint32_t)lw << 24);
    if (rec_) {
      line(ind + 1, "if (viol) {");
      line(ind + 2, "if (fo == ~0u) fo = ordinal;");
      line(ind + 2, "if (write) write = !jit_record(bl, tl, ordinal, " + hex32(what) + ", off);");
      line(ind + 1, "}");
    } else {
      line(ind + 1, "if (dig) dh = access_step(dh, " + hex32(((uint32_t)o2.site * 0xC2B2AE3Du) | 3u) +
                        ", ix);");
      line(ind + 1, "nv += viol ? 1u : 0u;");
    }
    if (o2.opc == B_LD && !o2.value_dead) {
      if (shared) {
        line(ind + 1, r(o2.dst) + " = 0;");
      } else {
        uint32_t seedx = ir.seed ^ ((uint32_t)o2.buf * 0x9E3779B9u);
        // the record function has the 64-bit offset; the count function
        // derives the word from the 32-bit index
        // (inline in path mode: measured faster there than one shared copy)
        const std::string fnc =
            rec_ ? "jit_content(" : (compact_ && !path_) ? "jit_content_out(" : "jit_content_ix(";
        line(ind + 1, r(o2.dst) + " = viol ? 0 : " + fnc + hex32(seedx) + (rec_ ? ", off, " : ", ix, ") +
                          std::to_string(lw) + "u);");
      }
    }
    if (rec_) line(ind + 1, "ordinal++;");
    line(ind, "}");
  }

  // An access of the block-serial function: the check, the digest, the
  // record written at once, and the shared bytes stored or read in bounds
  // (little-endian; a store of width 8 or 16 writes the 32-bit value and
  // zero bytes, a load of width > 1 reads the 32-bit word at the offset).
  void block_access(int ind, const IrOp& o2, int lw, bool shared) {
    line(ind, "{");
    line(ind + 1, "const int32_t ix = " + r(o2.a) + ";");
    line(ind + 1, "const bool viol = (uint32_t)ix >= " + lim_name(o2.buf, lw) + ";");
    line(ind + 1, "const int64_t off = (int64_t)ix * " + std::to_string(1 << lw) + ";");
    line(ind + 1, "if (dig) dh = access_step(dh, " + hex32(((uint32_t)o2.site * 0xC2B2AE3Du) | 3u) + ", ix);");
    const uint32_t what = (uint32_t)o2.site | ((uint32_t)o2.buf << 16) |
                          ((o2.opc == B_ST ? 1u : 0u) << 20) | ((uint32_t)lw << 24);
    line(ind + 1, "if (viol) {");
    line(ind + 2, "acc.n_viol++;");
    line(ind + 2, "const unsigned long long fk = first_key_of(bl, tl, ordinal);");
    line(ind + 2, "if (fk < acc.first_key) acc.first_key = fk;");
    line(ind + 2, "if (!rec_full) rec_full = jit_record(bl, tl, ordinal, " + hex32(what) + ", off);");
    line(ind + 1, "}");
    const std::string at = "shb + SB" + std::to_string(o2.buf) + " + (uint32_t)off";
    if (o2.opc == B_ST && shared && o2.value_live)
      line(ind + 1, "if (!viol) blk_store(" + at + ", " + r(o2.b) + ", " + std::to_string(1 << lw) + "u);");
    if (o2.opc == B_LD && !o2.value_dead) {
      if (shared)
        line(ind + 1, r(o2.dst) + " = viol ? 0 : blk_load(" + at + ", " + std::to_string(1 << lw) + "u);");
      else
        line(ind + 1, r(o2.dst) + " = viol ? 0 : jit_content_ix(" +
                          hex32(ir.seed ^ ((uint32_t)o2.buf * 0x9E3779B9u)) + ", ix, " +
                          std::to_string(lw) + "u);");
    }
    line(ind + 1, "ordinal++;");
    line(ind, "}");
  }

  // A checked division: a zero divisor is a violation (its record written
  // by the program's fault helper in the record function) and gives 0;
  // INT_MIN / -1 wraps.
  void divide(int ind, const IrOp& o2) {
    line(ind, "{");
    line(ind + 1, "const int32_t dv = " + r(o2.b) + ";");
    if (rec_) {
      line(ind + 1, "if (dv == 0) {");
      line(ind + 2, "if (fo == ~0u) fo = ordinal;");
      line(ind + 2, "if (write) write = !cufz_prog_" + std::to_string(index) +
                        "_div_fault(bl, tl, ordinal, " + std::to_string(o2.site) + "u);");
      line(ind + 1, "}");
      line(ind + 1, "ordinal++;");
    } else {
      line(ind + 1, "nv += dv == 0 ? 1u : 0u;");
    }
    if (!o2.value_dead) {
      const bool rem = o2.opc == B_REM;
      const std::string x = r(o2.a), mn = "(int32_t)0x80000000u";
      line(ind + 1, r(o2.dst) + " = dv == 0 ? 0 : (" + x + " == " + mn + " && dv == -1) ? " +
                        (rem ? "0" : mn) + " : " + x + (rem ? " % dv;" : " / dv;"));
    }
    line(ind, "}");
  }

  // The device heap: hp[s] is allocation site s's block (0 never
  // allocated, its size while live, -1 once freed), reset per test thread.
  // A fault's record is written by the program's heap-fault helper in the
  // record function.
  void heap_fault(int ind, const std::string& site, const std::string& buf,
                  const std::string& kind, const std::string& w, const std::string& cls,
                  const std::string& off) {
    line(ind, "if (fo == ~0u) fo = ordinal;");
    line(ind, "if (write) write = !cufz_prog_" + std::to_string(index) + "_heap_fault(bl, tl, ordinal, " +
                  site + ", " + buf + ", " + kind + ", " + w + ", " + cls + ", " + off + ");");
  }
  void heap(int ind, const IrOp& o2) {
    // with no HALLOC every handle is one of no block
    const std::string st_expr =
        ir.n_alloc ? "hs < " + std::to_string(ir.n_alloc) + "u ? hp[hs] : 0" : std::string("0");
    line(ind, "{");
    if (o2.opc == B_HALLOC) {
      line(ind + 1, "const int32_t hn = " + r(o2.a) + ";");
      line(ind + 1, "if (hn >= 1) hp[" + std::to_string(o2.site) + "] = hn;");
      line(ind + 1, r(o2.dst) + " = hn >= 1 ? " + std::to_string(o2.site + 1) + " : 0;");
    } else if (o2.opc == B_HFREE) {
      line(ind + 1, "const int32_t hh = " + r(o2.a) + ";");
      line(ind + 1, "const uint32_t hs = (uint32_t)hh - 1u;");
      line(ind + 1, "const int32_t st = " + st_expr + ";");
      line(ind + 1, "if (hh != 0 && st > 0) hp[hs] = -1;");
      if (rec_) {
        line(ind + 1, "if (hh != 0 && st <= 0) {");
        heap_fault(ind + 2, std::to_string(o2.site) + "u", "0u", "3u", "0u",
                   "st == 0 ? " + std::to_string(CUFZ_CLS_INVALID_FREE) + "u : " +
                       std::to_string(CUFZ_CLS_DOUBLE_FREE) + "u",
                   "0");
        line(ind + 1, "}");
        line(ind + 1, "ordinal++;");
      } else {
        line(ind + 1, "nv += (hh != 0 && st <= 0) ? 1u : 0u;");
      }
    } else {
      const int w = o2.width;
      line(ind + 1, "const int32_t ix = " + r(o2.a) + ";");
      line(ind + 1, "const uint32_t hs = (uint32_t)" + r(o2.b) + " - 1u;");
      line(ind + 1, "const int32_t st = " + st_expr + ";");
      line(ind + 1, "(void)hs;");
      line(ind + 1, "const int64_t off = (int64_t)ix * " + std::to_string(w) + ";");
      line(ind + 1, "const bool viol = st <= 0 || off < 0 || off + " + std::to_string(w) +
                        " > (int64_t)st;");
      if (rec_) {
        line(ind + 1, "if (viol) {");
        line(ind + 2, "const int64_t R = (int64_t)s_T.redzone;");
        line(ind + 2, "const uint32_t cls = st == 0 ? " + std::to_string(CUFZ_CLS_WILD) +
                          "u : st < 0 ? " + std::to_string(CUFZ_CLS_USE_AFTER_FREE) +
                          "u : (off < 0 && off >= -R) ? " + std::to_string(CUFZ_CLS_UNDERFLOW_RZ) +
                          "u : (off >= 0 && off < (int64_t)st + R) ? " +
                          std::to_string(CUFZ_CLS_OVERFLOW_RZ) + "u : " +
                          std::to_string(CUFZ_CLS_WILD) + "u;");
        heap_fault(ind + 2, std::to_string(o2.site) + "u", "st == 0 ? 0u : hs",
                   o2.opc == B_HST ? "1u" : "0u", std::to_string(w) + "u", "cls", "off");
        line(ind + 1, "}");
        line(ind + 1, "ordinal++;");
      } else {
        line(ind + 1, "if (dig) dh = access_step(dh, " + hex32(((uint32_t)o2.site * 0xC2B2AE3Du) | 3u) +
                          ", ix);");
        line(ind + 1, "nv += viol ? 1u : 0u;");
      }
      if (o2.opc == B_HLD && !o2.value_dead) line(ind + 1, r(o2.dst) + " = 0;");
    }
    line(ind, "}");
  }

  void range(int ind, int pc, int end) {
    run_counts(ind, pc, end);
    while (pc < end) {
      const IrOp& o2 = ir.ops[pc];
      if (!o2.kept) {
        pc++;
        continue;
      }
      uint8_t opc = o2.opc;
      if (is_alu_reg(opc)) {
        line(ind, r(o2.dst) + " = " + alu_expr(opc - 0x10, r(o2.a), r(o2.b)) + ";");
      } else if (is_alu_imm(opc)) {
        line(ind, r(o2.dst) + " = " + alu_expr(opc - 0x30, r(o2.a), imm(o2.imm)) + ";");
      } else if (opc == B_SREG) {
        line(ind, r(o2.dst) + " = " + sreg_name(o2.sreg) + ";");
      } else if (opc == B_IMM) {
        line(ind, r(o2.dst) + " = " + imm(o2.imm) + ";");
      } else if (opc == B_MOV) {
        line(ind, r(o2.dst) + " = " + r(o2.a) + ";");
      } else if (opc == B_SEL) {
        line(ind, r(o2.dst) + " = " + r(o2.a) + " != 0 ? " + r(o2.b) + " : " + r(o2.c) + ";");
      } else if (opc == B_LD || opc == B_ST) {
        access(ind, o2);
      } else if (opc == B_DIV || opc == B_REM) {
        divide(ind, o2);
      } else if (is_heap_op(opc)) {
        heap(ind, o2);
      } else if (opc == B_IF) {
        std::string c = "c" + std::to_string(o2.site);
        line(ind, "{");
        line(ind + 1, "const bool " + c + " = " + r(o2.a) + " != 0;");
        cover(ind + 1, o2.site, c, false);
        line(ind + 1, "if (" + c + ") {");
        if (path_ && !rec_)
          line(ind + 2, "po" + std::to_string(o2.site >> 5) + " |= " + hex32(1u << (o2.site & 31)) + ";");
        kp_ = true;
        pv_ = ir.loc1[o2.site] >> 1;
        range(ind + 2, pc + 1, o2.else_pc >= 0 ? o2.else_pc : o2.end_pc);
        const bool kt = kp_;
        const uint32_t vt = pv_;
        kp_ = true;
        pv_ = ir.loc0[o2.site] >> 1;
        if (o2.else_pc >= 0) {
          line(ind + 1, "} else {");
          range(ind + 2, o2.else_pc + 1, o2.end_pc);
        }
        line(ind + 1, "}");
        if (sp_) {
          // the join: prev stays known if both paths agree on a constant
          if (kt && kp_ && vt != pv_)
            line(ind + 1, "prev = " + c + " ? " + hex32(vt) + " : " + hex32(pv_) + ";");
          else if (kt && !kp_)
            line(ind + 1, "if (" + c + ") prev = " + hex32(vt) + ";");
          else if (!kt && kp_)
            line(ind + 1, "if (!" + c + ") prev = " + hex32(pv_) + ";");
          kp_ = kt && kp_ && vt == pv_;
        }
        line(ind, "}");
        pc = o2.end_pc + 1;
        run_counts(ind, pc, end);
        continue;
      } else if (opc == B_LOOP && !rec_ && !has_branch_sites(pc + 1, o2.end_pc)) {
        // A loop without branch sites in its body.  Its body is one
        // straight-line run, so everything but the body's own values is
        // known before it starts: the budget stop (each iteration ends with
        // a back-edge; the thread stops at back-edge budget + 1, so a loop
        // of trip iterations entered with `back` taken stops iff trip >
        // budget - back, after budget - back + 1 bodies), the counts (the
        // run's counts times the iterations) and the head edges (in closed
        // form after the loop).  The body runs without per-iteration checks.
        has_loop = true;
        const std::string sfx = std::to_string(o2.site);
        const std::string t = "trip" + sfx, n = "n" + sfx, stop = "stop" + sfx, it = "it" + sfx;
        const std::string lt = hex32(ir.loc1[o2.site]), lf = hex32(ir.loc0[o2.site]);
        line(ind, "{");
        line(ind + 1, "const int32_t " + n + " = " + r(o2.a) + ";");
        line(ind + 1, "const uint32_t " + t + " = " + n + " < 0 ? 0u : (" + n + " > " +
                          std::to_string(o2.imm) + " ? " + std::to_string(o2.imm) + "u : (uint32_t)" + n + ");");
        line(ind + 1, "const bool " + stop + " = " + t + " > budget - back;");
        line(ind + 1, "const uint32_t " + it + " = " + stop + " ? budget - back + 1u : " + t + ";");
        line(ind + 1, "#pragma unroll 4");
        line(ind + 1, "for (" + r(o2.dst) + " = 0; (uint32_t)" + r(o2.dst) + " < " + it + "; " + r(o2.dst) + "++) {");
        no_counts_ = true;
        range(ind + 2, pc + 1, o2.end_pc);
        no_counts_ = false;
        line(ind + 1, "}");
        const int k = run_ops(pc + 1, o2.end_pc), m = run_acc(pc + 1, o2.end_pc);
        if (k) line(ind + 1, "acc.n_ops += " + std::to_string(k) + "u * " + it + ";");
        if (m) line(ind + 1, "acc.n_acc += " + std::to_string(m) + "u * " + it + ";");
        line(ind + 1, "back += " + it + ";");
        if (sp_ && kp_) {
          // the entering prev is a constant: the loop's edges fold to constants
          line(ind + 1, "{ uint32_t pin = " + hex32(pv_) + "; jit_loop_cover(slot, pin, acc, " + it +
                            ", !" + stop + ", " + lt + ", " + lf + "); }");
        } else {
          line(ind + 1, "jit_loop_cover(slot, prev, acc, " + it + ", !" + stop + ", " + lt + ", " + lf + ");");
        }
        line(ind + 1, "if (" + stop + ") { " + stop_code_ + " }");
        line(ind, "}");
        // a loop that did not stop the thread left through its exit edge
        kp_ = true;
        pv_ = ir.loc0[o2.site] >> 1;
        pc = o2.end_pc + 1;
        run_counts(ind, pc, end);
        continue;
      } else if (opc == B_LOOP) {
        has_loop = true;
        std::string t = "trip" + std::to_string(o2.site), c = "cont" + std::to_string(o2.site);
        std::string n = "n" + std::to_string(o2.site);
        line(ind, "{");
        line(ind + 1, "const int32_t " + n + " = " + r(o2.a) + ";");
        line(ind + 1, "const int32_t " + t + " = " + n + " < 0 ? 0 : (" + n + " > " +
                          std::to_string(o2.imm) + " ? " + std::to_string(o2.imm) + " : " + n + ");");
        line(ind + 1, r(o2.dst) + " = 0;");
        materialize(ind + 1);  // the head is reached from the entry and the back-edge
        line(ind + 1, "#pragma unroll 1");
        line(ind + 1, "for (;;) {");
        line(ind + 2, "const bool " + c + " = " + r(o2.dst) + " < " + t + ";");
        cover(ind + 2, o2.site, c, true);
        line(ind + 2, "if (!" + c + ") break;");
        kp_ = true;
        pv_ = ir.loc1[o2.site] >> 1;
        range(ind + 2, pc + 1, o2.end_pc);
        materialize(ind + 2);
        line(ind + 2, rec_ ? "if (++back > budget) goto cufz_done;"
                           : "if (++back > budget) { " + stop_code_ + " }");
        line(ind + 2, r(o2.dst) + "++;");
        line(ind + 1, "}");
        line(ind, "}");
        kp_ = true;
        pv_ = ir.loc0[o2.site] >> 1;
        pc = o2.end_pc + 1;
        run_counts(ind, pc, end);
        continue;
      }
      pc++;
    }
  }

  // Decodes test thread g into bl, tl and the used special registers, with
  // only the divisions those need: x = lin % n_x, y = (lin / n_x) % n_y,
  // z = lin / (n_x * n_y) for the thread (tl) and the block (bl).  (The
  // record function's single thread; the count function's work-item loop
  // steps its coordinates instead, see stepped_pre.)
  void thread_setup(int ind, const std::vector<bool>& sreg_used) {
    line(ind, "const uint32_t bl = udiv(g, vin->mT);");
    line(ind, "const uint32_t tl = g - bl * vin->T;");
    const char* lin[2] = {"tl", "bl"};
    const char* m1[2] = {"vin->mBx", "vin->mGx"};
    const char* m2[2] = {"vin->mBxy", "vin->mGxy"};
    const char* n1[2] = {"vin->Bx", "vin->gx"};
    const char* ny[2] = {"vin->block[1]", "vin->grid[1]"};
    const char* nm[2][3] = {{"s_tx", "s_ty", "s_tz"}, {"s_bx", "s_by", "s_bz"}};
    for (int k = 0; k < 2; k++) {
      const bool ux = sreg_used[k * 6 + 0], uy = sreg_used[k * 6 + 1], uz = sreg_used[k * 6 + 2];
      const std::string q = std::string("q") + lin[k], z = std::string("z") + lin[k];
      if (ux || uy) line(ind, "const uint32_t " + q + " = udiv(" + lin[k] + ", " + m1[k] + ");");
      if (uy || uz) line(ind, "const uint32_t " + z + " = udiv(" + lin[k] + ", " + m2[k] + ");");
      if (ux) line(ind, std::string("const int32_t ") + nm[k][0] + " = (int32_t)(" + lin[k] + " - " + q + " * " + n1[k] + ");");
      if (uy) line(ind, std::string("const int32_t ") + nm[k][1] + " = (int32_t)(" + q + " - " + z + " * " + ny[k] + ");");
      if (uz) line(ind, std::string("const int32_t ") + nm[k][2] + " = (int32_t)" + z + ";");
    }
    for (int k = 0; k < 3; k++) {
      if (sreg_used[3 + k]) line(ind, std::string("const int32_t ") + sreg_name(3 + k) + " = (int32_t)vin->block[" + std::to_string(k) + "];");
      if (sreg_used[9 + k]) line(ind, std::string("const int32_t ") + sreg_name(9 + k) + " = (int32_t)vin->grid[" + std::to_string(k) + "];");
    }
    for (int k = 0; k < 4; k++)
      if (sreg_used[12 + k]) line(ind, std::string("const int32_t ") + sreg_name(12 + k) + " = vin->args[" + std::to_string(k) + "];");
  }

  // The work-item loop's coordinates (count function).  A lane runs test
  // threads g, g + blockDim.x, ...  With inc (a block has at least as many
  // threads as the CTA) bl and tl are carried across steps and bl grows by at
  // most one per step, so the block coordinates are stepped too (x, then the
  // carry into y, then z) instead of divided out; with fix_t (a block has
  // exactly the CTA's threads) tl never changes and the thread coordinates
  // are computed once.  Quotients by a unit extent (b1/g1: 1D; bz1/gz1: no
  // z extent) are 0 and skipped.
  void stepped_pre(int ind, const std::vector<bool>& u) {
    const bool tx = u[0], ty = u[1], tz = u[2], bx = u[6], by = u[7], bz = u[8];
    line(ind, "const bool fix_t = inc && vin->T == blockDim.x;");
    if (hoist_) {
      launch_consts(ind, u);
      line(ind, "const uint32_t T_ = vin->T, gx_ = vin->gx, gy_ = vin->grid[1];");
    }
    line(ind, "const bool bz1 = vin->block[2] == 1u, gz1 = vin->grid[2] == 1u;");
    line(ind, "(void)fix_t; (void)bz1; (void)gz1;");
    if (tx || ty) line(ind, "uint32_t qtl = 0;");
    if (ty || tz) line(ind, "uint32_t ztl = 0;");
    if (tx || ty || tz) {
      std::string t = "if (fix_t && !b1) {";
      if (tx || ty) t += " qtl = udiv(tl, vin->mBx);";
      if (ty || tz) t += " ztl = bz1 ? 0u : udiv(tl, vin->mBxy);";
      line(ind, t + " }");
    }
    if (bx || by || bz) line(ind, "uint32_t cbx = 0;");
    if (by || bz) line(ind, "uint32_t cby = 0;");
    if (bz) line(ind, "uint32_t cbz = 0;");
    if (bx || by || bz) {
      line(ind, "if (inc) {");
      block_coords(ind + 1, u);
      line(ind, "}");
    }
  }
  // cbx, cby, cbz of block bl by division
  void block_coords(int ind, const std::vector<bool>& u) {
    const bool by = u[7], bz = u[8];
    line(ind, "const uint32_t qb = g1 ? 0u : udiv(bl, vin->mGx);");
    line(ind, "cbx = bl - qb * vin->gx;");
    if (by || bz) line(ind, "const uint32_t zb = (g1 || gz1) ? 0u : udiv(bl, vin->mGxy);");
    if (by || bz) line(ind, "cby = qb - zb * vin->grid[1];");
    if (bz) line(ind, "cbz = zb;");
  }
  void stepped_in(int ind, const std::vector<bool>& u) {
    const bool tx = u[0], ty = u[1], tz = u[2], bx = u[6], by = u[7], bz = u[8];
    line(ind, "if (!inc) { bl = udiv(g, vin->mT); tl = g - bl * vin->T; }");
    if (tx || ty || tz) {
      std::string t = "if (!fix_t && !b1) {";
      if (tx || ty) t += " qtl = udiv(tl, vin->mBx);";
      if (ty || tz) t += " ztl = bz1 ? 0u : udiv(tl, vin->mBxy);";
      line(ind, t + " }");
    }
    if (tx) line(ind, "const int32_t s_tx = (int32_t)(tl - qtl * vin->Bx);");
    if (ty) line(ind, "const int32_t s_ty = (int32_t)(qtl - ztl * vin->block[1]);");
    if (tz) line(ind, "const int32_t s_tz = (int32_t)ztl;");
    if (bx || by || bz) {
      line(ind, "if (!inc) {");
      block_coords(ind + 1, u);
      line(ind, "}");
    }
    if (bx) line(ind, "const int32_t s_bx = (int32_t)cbx;");
    if (by) line(ind, "const int32_t s_by = (int32_t)cby;");
    if (bz) line(ind, "const int32_t s_bz = (int32_t)cbz;");
    if (!hoist_) launch_consts(ind, u);
  }
  // the used launch dimensions and arguments
  void launch_consts(int ind, const std::vector<bool>& u) {
    for (int k = 0; k < 3; k++) {
      if (u[3 + k]) line(ind, std::string("const int32_t ") + sreg_name(3 + k) + " = (int32_t)vin->block[" + std::to_string(k) + "];");
      if (u[9 + k]) line(ind, std::string("const int32_t ") + sreg_name(9 + k) + " = (int32_t)vin->grid[" + std::to_string(k) + "];");
    }
    for (int k = 0; k < 4; k++)
      if (u[12 + k]) line(ind, std::string("const int32_t ") + sreg_name(12 + k) + " = vin->args[" + std::to_string(k) + "];");
  }
  void stepped_tail(int ind, const std::vector<bool>& u) {
    const bool bx = u[6], by = u[7], bz = u[8];
    const std::string T = hoist_ ? "T_" : "vin->T", gx = hoist_ ? "gx_" : "vin->gx",
                      gy = hoist_ ? "gy_" : "vin->grid[1]";
    line(ind, "tl += blockDim.x;");
    std::string t = "if (tl >= " + T + ") { tl -= " + T + "; bl++;";
    if (bz) t += " if (++cbx == " + gx + ") { cbx = 0; if (++cby == " + gy + ") { cby = 0; cbz++; } }";
    else if (by) t += " if (++cbx == " + gx + ") { cbx = 0; if (++cby == " + gy + ") cby = 0; }";
    else if (bx) t += " if (++cbx == " + gx + ") cbx = 0;";
    line(ind, t + " }");
    if (hoist_) line(ind, "(void)gx_; (void)gy_;");
  }

  void reg_decls(int ind, const std::vector<bool>& used) {
    std::string decl;
    for (int v = 0; v < 256; v++)
      if (used[v]) decl += (decl.empty() ? "int32_t " : ", ") + r(v) + " = 0";
    if (!decl.empty()) line(ind, decl + ";");
  }

  // The block-serial function cufz_prog_<index>(g0, g_end) of a program whose
  // performed shared stores need their barriers (prepare_barriers): its work
  // items are whole test blocks; each CUDA thread takes one block at a time
  // and runs its threads in thread_lin order through the first phase (the
  // ops up to the first BAR), then all of them through the next phase, and
  // so on, as the oracle does.  Between phases a thread keeps its registers
  // live across the barriers, ordinal, prev, back-edges and digest state in
  // local arrays; the block's shared buffers are one local byte array (all
  // zero at the block's start) in which in-bounds shared stores are
  // performed and shared loads read.  A thread stopped by the budget runs no
  // later phase.  Records are written at each violation.
  bool too_many_saved_ = false;
  void emit_block_serial(const std::vector<bool>& used, const std::vector<bool>& u,
                         const std::string& fn) {
    blk_ = true;
    compact_ = path_ = hoist_ = false;
    // registers live at a barrier: the state a thread carries between phases
    Liveness Lv = liveness(ir, false);
    std::vector<int> saved;
    std::vector<int> bars;
    for (int pc = 0; pc < (int)ir.ops.size(); pc++)
      if (ir.ops[pc].opc == B_BAR) bars.push_back(pc);
    for (int v = 0; v < kSregBase; v++) {
      bool live = false;
      for (int pc : bars) live |= Lv.in[pc].get(v);
      if (live) saved.push_back(v);
    }
    if ((uint32_t)saved.size() > kBlkMaxSaved) {
      too_many_saved_ = true;
      return;
    }
    const int ns = std::max((int)saved.size(), 1);
    const std::string NS = std::to_string(ns);
    line(0, "__device__ __noinline__ void " + fn + "(uint32_t g0, uint32_t g_end) {");
    line(1, "const uint32_t slot = s_in.slot;");
    line(1, "LaneAcc acc;");
    line(1, "acc_init(acc);");
    line(1, "const uint32_t budget = s_T.iter_budget;");
    line(1, std::string("constexpr bool dig = ") + (digest_ ? "true;" : "false;"));
    line(1, "const DevInput* vin = &s_in;");
    line(1, "const uint32_t* lim = s_in.lim;");
    lim_decls(1);
    // offsets of the shared buffers in the block's bytes
    std::string sb = "0u";
    for (int k = 0; k < ir.n_bufs; k++)
      if ((ir.shared_mask >> k) & 1u) {
        line(1, "const uint32_t SB" + std::to_string(k) + " = " + sb + ";");
        sb = "SB" + std::to_string(k) + " + (uint32_t)vin->len[" + std::to_string(k) + "]";
      }
    line(1, "const uint32_t sb_total = " + sb + ";");
    line(1, "const uint32_t T = vin->T;");
    line(1, "const uint32_t b_first = udiv(g0, vin->mT), b_end = udiv(g_end, vin->mT);");
    line(1, "bool rec_full = false;");
    line(1, "#pragma unroll 1");
    line(1, "for (uint32_t bl = b_first + threadIdx.x; bl < b_end; bl += blockDim.x) {");
    // block coordinates
    if (u[6] || u[7]) line(2, "const uint32_t qbl = udiv(bl, vin->mGx);");
    if (u[7] || u[8]) line(2, "const uint32_t zbl = udiv(bl, vin->mGxy);");
    if (u[6]) line(2, "const int32_t s_bx = (int32_t)(bl - qbl * vin->gx);");
    if (u[7]) line(2, "const int32_t s_by = (int32_t)(qbl - zbl * vin->grid[1]);");
    if (u[8]) line(2, "const int32_t s_bz = (int32_t)zbl;");
    launch_consts(2, u);
    line(2, "uint8_t shb[" + std::to_string(kBlkSharedBytes) + "];");
    line(2, "for (uint32_t i = 0; i < sb_total; i++) shb[i] = 0;");
    line(2, "int32_t sv[" + std::to_string(kBlkMaxThreads) + "][" + NS + "];");
    line(2, "uint32_t s_ord[" + std::to_string(kBlkMaxThreads) + "], s_prev[" +
                std::to_string(kBlkMaxThreads) + "], s_back[" + std::to_string(kBlkMaxThreads) +
                "], s_dh[" + std::to_string(kBlkMaxThreads) + "];");
    line(2, "uint8_t s_stop[" + std::to_string(kBlkMaxThreads) + "];");
    line(2, "#pragma unroll 1");
    line(2, "for (uint32_t t = 0; t < T; t++) {");
    line(3, "s_ord[t] = 0; s_prev[t] = 0; s_back[t] = 0; s_dh[t] = digest_start(bl, t); s_stop[t] = 0;");
    line(3, "for (int j = 0; j < " + NS + "; j++) sv[t][j] = 0;");
    line(2, "}");
    // phases
    std::vector<std::pair<int, int>> phases;
    int begin = 0;
    for (int pc : bars) {
      phases.emplace_back(begin, pc);
      begin = pc + 1;
    }
    phases.emplace_back(begin, (int)ir.ops.size());
    for (size_t p = 0; p < phases.size(); p++) {
      const std::string label = "blk_stop_" + std::to_string(p);
      stop_code_ = "acc.budget_hit = true; s_stop[tl] = 1; goto " + label + ";";
      line(2, "// phase " + std::to_string(p));
      line(2, "#pragma unroll 1");
      line(2, "for (uint32_t tl = 0; tl < T; tl++) {");
      line(3, "if (s_stop[tl]) continue;");
      if (u[0] || u[1]) line(3, "const uint32_t qtl = udiv(tl, vin->mBx);");
      if (u[1] || u[2]) line(3, "const uint32_t ztl = udiv(tl, vin->mBxy);");
      if (u[0]) line(3, "const int32_t s_tx = (int32_t)(tl - qtl * vin->Bx);");
      if (u[1]) line(3, "const int32_t s_ty = (int32_t)(qtl - ztl * vin->block[1]);");
      if (u[2]) line(3, "const int32_t s_tz = (int32_t)ztl;");
      line(3, "uint32_t ordinal = s_ord[tl], prev = s_prev[tl], back = s_back[tl], dh = s_dh[tl];");
      line(3, "(void)prev; (void)back; (void)dh;");
      reg_decls(3, used);
      for (size_t j = 0; j < saved.size(); j++)
        line(3, r(saved[j]) + " = sv[tl][" + std::to_string(j) + "];");
      has_loop = false;
      range(3, phases[p].first, phases[p].second);
      if (has_loop) line(2, label + ":");
      for (size_t j = 0; j < saved.size(); j++)
        line(3, "sv[tl][" + std::to_string(j) + "] = " + r(saved[j]) + ";");
      line(3, "s_ord[tl] = ordinal; s_prev[tl] = prev; s_back[tl] = back; s_dh[tl] = dh;");
      line(2, "}");
    }
    line(2, "#pragma unroll 1");
    line(2, "for (uint32_t t = 0; t < T; t++)");
    line(3, "if (dig) acc.digest += digest_end(s_dh[t]);");
    line(1, "}");
    line(1, "__syncwarp();");
    line(1, "acc_flush(s_T, slot, acc);");
    line(0, "}");
    blk_ = false;
  }

  void emit() {
    std::vector<bool> used(ir.nv, false), sreg_used(16, false);
    int U[4], D[4], nu, nd;
    for (const auto& op : ir.ops) {
      uses_defs(op, false, U, &nu, D, &nd);
      for (int k = 0; k < nu; k++) used[U[k]] = true;
      for (int k = 0; k < nd; k++) used[D[k]] = true;
      if (op.kept && op.opc == B_SREG) sreg_used[op.sreg] = true;
    }
    const std::string fn = "cufz_prog_" + std::to_string(index);
    if (ir.block_serial) {
      emit_block_serial(used, sreg_used, fn);
      return;
    }
    int n_sites_kept = 0;
    for (const auto& op : ir.ops) n_sites_kept += op.kept && (op.opc == B_IF || op.opc == B_LOOP);
    compact_ = n_sites_kept >= kCompactSites;
    bool loops = false;
    for (const auto& op : ir.ops) loops |= op.kept && op.opc == B_LOOP;
    path_ = compact_ && !loops && ir.n_sites <= 64;
    if (path_) {
      // the walk table: LOC pair, the next site and the counts up to it for
      // each outcome
      path_next();
      std::string t = "static __device__ const uint4 " + fn + "_walk[" +
                      std::to_string(std::max(ir.n_sites, 1)) + "] = {";
      for (int s = 0; s < ir.n_sites; s++)
        t += std::string(s ? ", " : "") + "{" +
             hex32((uint32_t)ir.loc0[s] | ((uint32_t)ir.loc1[s] << 16)) + ", " +
             hex32((uint32_t)next_[s][0] | ((uint32_t)next_[s][1] << 8)) + ", " +
             hex32(seg_[s][0]) + ", " + hex32(seg_[s][1]) + "}";
      line(0, t + (ir.n_sites ? "};" : "{0u, 0u, 0u, 0u}};"));
    }
    int n_kept = 0;
    for (const auto& op : ir.ops) n_kept += op.kept && op.opc != B_NOP;
    hoist_ = n_kept <= kHoistMaxOps;

    // division faults: records of kind 2 (division), class DIV_ZERO, written
    // like access records (one atomicAdd per active-mask group)
    bool divides = false;
    for (const auto& op : ir.ops) divides |= op.kept && (op.opc == B_DIV || op.opc == B_REM);
    if (divides) {
      line(0, "__device__ __noinline__ bool " + fn +
                  "_div_fault(uint32_t bl, uint32_t tl, uint32_t ordinal, uint32_t site) {");
      line(1, "const uint32_t am = __activemask();");
      line(1, "const uint32_t lane = threadIdx.x & 31u;");
      line(1, "const uint32_t leader = __ffs(am) - 1;");
      line(1, "const uint32_t k = __popc(am);");
      line(1, "const uint32_t cap = s_T.record_cap;");
      line(1, "const uint32_t slot = s_in.slot;");
      line(1, "uint32_t base = 0;");
      line(1, "if (lane == leader) base = atomicAdd(&s_T.slots[slot].rec_reserved, k);");
      line(1, "base = __shfl_sync(am, base, leader);");
      line(1, "const uint32_t rank = __popc(am & ((1u << lane) - 1u));");
      line(1, "if (base + rank < cap)");
      line(2, "write_record(s_T.records + (size_t)slot * cap + base + rank, bl, tl, ordinal, site, "
              "0u, 2u, 0u, 0u, CUFZ_CLS_DIV_ZERO, 0);");
      line(1, "return base + k >= cap;");
      line(0, "}");
    }

    // heap faults: records of space 2 (kind 3 for a bad free), written
    // like access records
    bool heap_ops = false;
    for (const auto& op : ir.ops) heap_ops |= op.kept && is_heap_op(op.opc);
    const std::string heap_decl =
        "int32_t hp[" + std::to_string(std::max(ir.n_alloc, 1)) + "] = {};";
    if (heap_ops) {
      line(0, "__device__ __noinline__ bool " + fn +
                  "_heap_fault(uint32_t bl, uint32_t tl, uint32_t ordinal, uint32_t site, "
                  "uint32_t buf, uint32_t kind, uint32_t w, uint32_t cls, int64_t off) {");
      line(1, "const uint32_t am = __activemask();");
      line(1, "const uint32_t lane = threadIdx.x & 31u;");
      line(1, "const uint32_t leader = __ffs(am) - 1;");
      line(1, "const uint32_t k = __popc(am);");
      line(1, "const uint32_t cap = s_T.record_cap;");
      line(1, "const uint32_t slot = s_in.slot;");
      line(1, "uint32_t base = 0;");
      line(1, "if (lane == leader) base = atomicAdd(&s_T.slots[slot].rec_reserved, k);");
      line(1, "base = __shfl_sync(am, base, leader);");
      line(1, "const uint32_t rank = __popc(am & ((1u << lane) - 1u));");
      line(1, "if (base + rank < cap)");
      line(2, "write_record(s_T.records + (size_t)slot * cap + base + rank, bl, tl, ordinal, site, "
              "buf, kind, w, 2u, cls, off);");
      line(1, "return base + k >= cap;");
      line(0, "}");
    }

    // record function: one test thread, records and the first violation
    rec_ = true;
    has_loop = false;
    line(0, "__device__ __noinline__ uint32_t " + fn + "_rec(uint32_t g, bool write) {");
    line(1, "const uint32_t budget = s_T.iter_budget;");
    line(1, "const DevInput* vin = &s_in;");
    line(1, "const uint32_t* lim = vin->lim;");
    lim_decls(1);
    thread_setup(1, sreg_used);
    line(1, "uint32_t ordinal = 0, back = 0, fo = ~0u;");
    line(1, "(void)back;");
    reg_decls(1, used);
    if (heap_ops) line(1, heap_decl);
    range(1, 0, (int)ir.ops.size());
    if (has_loop) line(0, "cufz_done:");
    line(1, "return fo;");
    line(0, "}");

    // count function: a work item.  Its loop over the lane's test threads
    // is unrolled CUFZ_LANES_<index> times (1 unless the module defines it):
    // the lane mapping, k test threads per lane per iteration, which the
    // autotuner chooses for short programs.
    rec_ = false;
    has_loop = false;
    const std::string lanes = "CUFZ_LANES_" + std::to_string(index);
    line(0, "#ifndef " + lanes);
    line(0, "#define " + lanes + " 1");
    line(0, "#endif");
    line(0, "__device__ __noinline__ void " + fn + "(uint32_t g0, uint32_t g_end) {");
    line(1, "const uint32_t slot = s_in.slot;");
    line(1, "LaneAcc acc;");
    line(1, "acc_init(acc);");
    line(1, "const uint32_t budget = s_T.iter_budget;");
    line(1, "bool rec_open = jit_records_open(slot);");
    line(1, std::string("constexpr bool dig = ") + (digest_ ? "true;" : "false;"));
    // launch constants and index limits are plain loads from the CTA's
    // shared copy of the input, which the compiler may keep or reload
    line(1, "const DevInput* vin = &s_in;");
    line(1, "const uint32_t* lim = s_in.lim;");
    lim_decls(1);
    line(1, "const bool inc = vin->T >= blockDim.x;");
    line(1, "const bool b1 = vin->block[1] == 1u && vin->block[2] == 1u;");
    line(1, "const bool g1 = vin->grid[1] == 1u && vin->grid[2] == 1u;");
    line(1, "(void)b1; (void)g1;");
    line(1, "uint32_t bl = 0, tl = 0;");
    line(1, "if (inc) { bl = udiv(g0 + threadIdx.x, vin->mT); tl = g0 + threadIdx.x - bl * vin->T; }");
    stepped_pre(1, sreg_used);
    if (path_) line(1, "jit_path_clear();");
    line(1, "constexpr int lanes_k = " + lanes + ";");
    line(1, "#pragma unroll lanes_k");
    line(1, "for (uint32_t g = g0 + threadIdx.x; g < g_end; g += blockDim.x) {");
    stepped_in(2, sreg_used);
    // dh = the thread's digest state, nv = its violations
    line(2, "uint32_t dh = digest_start(bl, tl);");
    line(2, "uint32_t prev = 0, back = 0, nv = 0;");
    line(2, "(void)prev; (void)back; (void)dh;");
    if (path_) line(2, "uint32_t po0 = 0, po1 = 0;");
    reg_decls(2, used);
    if (heap_ops) line(2, heap_decl);
    sp_ = !path_;  // prev is 0 at each test thread's start
    kp_ = true;
    pv_ = 0;
    range(2, 0, (int)ir.ops.size());
    sp_ = kp_ = false;
    if (has_loop) line(1, "cufz_done:");
    if (path_) {
      line(2, "if (!jit_path_count(po0, po1)) {");
      line(3, "const uint32_t pc_ = jit_path_walk(slot, po0, po1, 1u, " + fn + "_walk, " +
                  std::to_string(first_site_) + "u, " + hex32(init_) + ");");
      line(3, "acc.n_ops += pc_ & 0xFFFu; acc.n_acc += (pc_ >> 12) & 0xFFFu; acc.n_branch += pc_ >> 24;");
      line(2, "}");
    }
    line(2, "if (dig) acc.digest += digest_end(dh);");
    line(2, "if (nv) {");
    line(3, "acc.n_viol += nv;");
    line(3, "bool listed = false;");
    line(3, "if (rec_open) {");
    line(4, "const uint32_t old = jit_list_violations(slot, nv);");
    line(4, "listed = old < s_T.record_cap;");
    line(4, "rec_open = old + nv < s_T.record_cap;");
    line(3, "}");
    line(3, "if (listed || jit_first_key_wanted(acc, slot, bl, tl)) {");
    line(4, "const uint32_t f = " + fn + "_rec(g, listed);");
    line(4, "if (acc.first_key == ~0ull) acc.first_key = first_key_of(bl, tl, f);");
    line(3, "}");
    line(2, "}");
    stepped_tail(2, sreg_used);
    line(1, "}");
    if (path_) {
      line(1, "{");
      line(2, "const PathCounts t_ = jit_path_flush(slot, " + fn + "_walk, " +
                  std::to_string(first_site_) + "u, " + hex32(init_) + ");");
      line(2, "acc.n_ops += t_.ops; acc.n_acc += t_.acc; acc.n_branch += t_.branch;");
      line(1, "}");
    }
    line(1, "__syncwarp();");
    line(1, "acc_flush(s_T, slot, acc);");
    line(0, "}");
  }

  // The walk of a loop-free program's sites: next_[s][o], the site
  // evaluated after site s when its outcome is o (255: none), and
  // first_site_, the first site a thread evaluates.  Control flow is
  // structured, so what follows an IF statement is fixed: the first site of
  // the arm taken, else the first site after the IF, else what follows the
  // enclosing arm.
  // seg_[s][o] packs the counts (ops | accesses << 12 | branch evaluations
  // << 24) of the runs a thread executes from outcome o at site s to its
  // next site evaluation (that evaluation included), init_ those before its
  // first: the counts run_counts adds at each run, summed along a path.
  std::vector<std::array<uint8_t, 2>> next_;
  std::vector<std::array<uint32_t, 2>> seg_;
  int first_site_ = 255;
  uint32_t init_ = 0;
  struct To {
    uint32_t cnt;
    int site;
  };
  // From the start of a run at pc in [pc, end) to the next site evaluation:
  // the first IF of the range, else what follows the range (cont).
  To to_site(int pc, int end, To cont) const {
    int q = pc;
    while (q < end && ir.ops[q].opc != B_IF && ir.ops[q].opc != B_LOOP) q++;
    const bool at_if = q < end && ir.ops[q].opc == B_IF && ir.ops[q].kept;
    const uint32_t c = (uint32_t)run_ops(pc, end) | ((uint32_t)run_acc(pc, end) << 12) |
                       ((at_if ? 1u : 0u) << 24);
    if (at_if) return {c, ir.ops[q].site};
    return {c + cont.cnt, cont.site};
  }
  void walk_range(int pc, int end, To cont) {
    while (pc < end) {
      const IrOp& o2 = ir.ops[pc];
      if (!o2.kept || o2.opc != B_IF) {
        pc++;
        continue;
      }
      const To after = to_site(o2.end_pc + 1, end, cont);
      const int then_end = o2.else_pc >= 0 ? o2.else_pc : o2.end_pc;
      const To t1 = to_site(pc + 1, then_end, after);
      const To t0 = o2.else_pc >= 0 ? to_site(o2.else_pc + 1, o2.end_pc, after) : after;
      next_[o2.site] = {(uint8_t)t0.site, (uint8_t)t1.site};
      seg_[o2.site] = {t0.cnt, t1.cnt};
      walk_range(pc + 1, then_end, after);
      if (o2.else_pc >= 0) walk_range(o2.else_pc + 1, o2.end_pc, after);
      pc = o2.end_pc + 1;
    }
  }
  void path_next() {
    next_.assign(std::max(ir.n_sites, 1), {255, 255});
    seg_.assign(std::max(ir.n_sites, 1), {0u, 0u});
    const int n = (int)ir.ops.size();
    const To start = to_site(0, n, To{0u, 255});
    first_site_ = start.site;
    init_ = start.cnt;
    walk_range(0, n, To{0u, 255});
  }
};

}  // namespace

// The compiled path's module: every program's item function, the dispatcher
// and the kernels, compiled as one translation unit so the program functions
// are register-allocated together with the kernel that calls them.
std::string jit_module_source(const std::vector<std::string>& prog_src,
                              const std::vector<uint8_t>& include, bool plain_kernel,
                              uint32_t min_ctas, uint32_t cta_threads,
                              const std::vector<uint8_t>& lanes) {
  // the persistent kernel's launch bounds follow the context's CTA size;
  // at most 2048 resident threads per SM
  min_ctas = std::max(1u, std::min(min_ctas ? min_ctas : kJitMinCtasDefault, 2048u / cta_threads));
  std::string src = "#define CUFZ_JIT_MIN_CTAS " + std::to_string(min_ctas) +
                    "\n#define CUFZ_JIT_CTA_THREADS " + std::to_string(cta_threads) + "\n";
  // each program's lane mapping (test threads per lane per loop iteration)
  for (size_t k = 0; k < prog_src.size() && k < lanes.size(); k++)
    if (include[k] && lanes[k] > 1)
      src += "#define CUFZ_LANES_" + std::to_string(k) + " " + std::to_string(lanes[k]) + "\n";
  src += "#include \"jit_kernel.cuh\"\nnamespace cufz {\n";
  for (size_t k = 0; k < prog_src.size(); k++)
    if (include[k]) src += prog_src[k];
  src += "static __device__ bool jit_run(uint32_t prog, uint32_t g0, uint32_t g_end) {\n"
         "  switch (prog) {\n";
  for (size_t k = 0; k < prog_src.size(); k++)
    if (include[k])
      src += "    case " + std::to_string(k) + ": cufz_prog_" + std::to_string(k) +
             "(g0, g_end); return true;\n";
  src += "    default: return false;\n  }\n}\n}  // namespace cufz\n";
  if (plain_kernel) src += "#define CUFZ_JIT_PLAIN 1\n";
  src += "#include \"jit_launch.cuh\"\n";
  return src;
}

cufz_status jit_source(const void* bytes, size_t nbytes, bool do_prune, bool digest,
                       uint32_t index, std::string* out) {
  Ir ir;
  if (!decode((const uint8_t*)bytes, nbytes, &ir)) return CUFZ_E_INVALID_PROGRAM;
  if (!prepare_barriers(&ir)) return CUFZ_E_UNSUPPORTED;
  if (do_prune) {
    prune(&ir);
  } else {
    Liveness L = liveness(ir, false);
    for (size_t pc = 0; pc < ir.ops.size(); pc++)
      if (ir.ops[pc].opc == B_LD || ir.ops[pc].opc == B_HLD)
        ir.ops[pc].value_dead = !L.out[pc].get(ir.ops[pc].dst);
  }
  out->clear();
  Gen g{ir, *out, (int)index};
  g.digest_ = digest;
  g.emit();
  return g.too_many_saved_ ? CUFZ_E_UNSUPPORTED : CUFZ_OK;
}



// ---------------------------------------------------------------- public

cufz_status load_program(const void* bytes, size_t nbytes, bool do_prune, LoadedProgram* out) {
  Ir ir;
  if (!decode((const uint8_t*)bytes, nbytes, &ir)) return CUFZ_E_INVALID_PROGRAM;
  if (!prepare_barriers(&ir)) return CUFZ_E_UNSUPPORTED;
  auto prex = std::make_shared<PrexInfo>();
  prex->ir = ir;
  int n_in = (int)ir.ops.size();
  if (do_prune) prune(&ir);
  propagate_sregs(&ir);
  std::vector<int> map;
  Bits entry;
  int n_regs = allocate(ir, true, &map, &entry);
  // the heap state: one register per allocation site after the program's
  const int heap_base = n_regs, n_heap = ir.n_alloc;
  if (n_regs + n_heap > kMaxPhysRegs) return CUFZ_E_INVALID_PROGRAM;

  // device ops
  int N = (int)ir.ops.size();
  std::vector<int> dpc(N + 1, -1);
  int nd = 0;
  for (int pc = 0; pc < N; pc++) {
    dpc[pc] = nd;
    if (ir.ops[pc].kept) nd++;
  }
  dpc[N] = nd;
  int n_dev = nd + 1;  // + END
  if (n_dev > kMaxDevOps) return CUFZ_E_INVALID_PROGRAM;
  std::vector<DevOp> dops;
  dops.reserve(n_dev);
  auto off = [&](int v) -> uint16_t { return v < 0 ? 0 : (uint16_t)(map[v] * kRegStride); };
  uint32_t sreg_mask = 0;
  DevProgHdr hdr;
  memset(&hdr, 0, sizeof(hdr));
  for (int s = 0; s < 16; s++)
    if (map[kSregBase + s] >= 0) {
      sreg_mask |= 1u << s;
      hdr.sreg_reg[s] = (uint8_t)map[kSregBase + s];
    }
  for (int pc = 0; pc < N; pc++) {
    const IrOp& o = ir.ops[pc];
    if (!o.kept) continue;
    DevOp d;
    memset(&d, 0, sizeof(d));
    uint8_t opc = o.opc;
    if (is_alu_reg(opc)) {
      d.opc = D_ALU0 + (opc - 0x10);
      d.d = off(o.dst); d.a = off(o.a); d.b = off(o.b);
    } else if (is_alu_imm(opc)) {
      d.opc = D_ALUI0 + (opc - 0x30);
      d.d = off(o.dst); d.a = off(o.a); d.imm = o.imm;
    } else {
      switch (opc) {
        case B_SREG:  // x = 1: not counted as an executed op
          d.opc = D_MOV; d.d = off(o.dst); d.a = off(kSregBase + o.sreg); d.x = 1;
          break;
        case B_IMM: d.opc = D_IMM; d.d = off(o.dst); d.imm = o.imm; break;
        case B_MOV: d.opc = D_MOV; d.d = off(o.dst); d.a = off(o.a); break;
        case B_SEL:
          d.opc = D_SEL; d.d = off(o.dst); d.a = off(o.a); d.b = off(o.b);
          d.imm = (int32_t)off(o.c);
          break;
        case B_DIV:
        case B_REM:
          d.opc = D_DIVREM;
          d.b = off(o.b);
          d.x = (uint8_t)((opc == B_REM ? 1u : 0u) | (o.value_dead ? 0u : 2u));
          if (!o.value_dead) {
            d.d = off(o.dst);
            d.a = off(o.a);
          }
          d.imm = o.site;
          break;
        case B_HALLOC:
        case B_HFREE:
        case B_HLD:
        case B_HST:
          d.opc = opc == B_HALLOC ? D_HALLOC : opc == B_HFREE ? D_HFREE : D_HACC;
          if (opc == B_HALLOC || (opc == B_HLD && !o.value_dead)) d.d = off(o.dst);
          d.a = off(o.a);
          if (d.opc == D_HACC) {
            d.b = off(o.b);
            d.x = (uint8_t)(log2w(o.width) | (opc == B_HST ? 8u : 0u) |
                            (opc == B_HLD && !o.value_dead ? 16u : 0u));
          }
          d.imm = o.site;
          d.j0 = (uint16_t)heap_base;
          d.j1 = (uint16_t)n_heap;
          break;
        case B_LD:
        case B_ST:
          d.opc = opc == B_ST ? D_ST : (o.value_dead ? D_LDX : D_LD);
          if (d.opc == D_LD) d.d = off(o.dst);
          d.a = off(o.a);
          d.b = (uint16_t)o.buf;
          d.x = (uint8_t)log2w(o.width);
          d.imm = o.site;
          break;
        case B_IF:
          d.opc = D_IF; d.a = off(o.a); d.x = (uint8_t)o.site;
          d.j0 = (uint16_t)(o.else_pc >= 0 ? dpc[o.else_pc] : dpc[o.end_pc]);
          break;
        case B_ELSE: d.opc = D_ELSE; d.j0 = (uint16_t)dpc[o.end_pc]; break;
        case B_ENDIF: d.opc = D_ENDIF; break;
        case B_LOOP:
        case B_ENDLOOP: {
          const IrOp& h = opc == B_LOOP ? o : ir.ops[o.head_pc];
          d.opc = opc == B_LOOP ? D_LOOP : D_ENDLOOP;
          d.d = off(h.dst);
          d.a = opc == B_LOOP ? off(h.a) : 0;
          d.b = off(h.trip);
          d.imm = opc == B_LOOP ? h.imm : 0;
          d.x = (uint8_t)h.site;
          d.j0 = (uint16_t)(dpc[h.end_pc] + 1);
          d.j1 = (uint16_t)(dpc[o.opc == B_LOOP ? pc : o.head_pc] + 1);
          break;
        }
        default: continue;
      }
    }
    dops.push_back(d);
  }
  DevOp end;
  memset(&end, 0, sizeof(end));
  end.opc = D_END;
  dops.push_back(end);

  std::vector<uint16_t> zero;
  for (int v = 0; v < kSregBase; v++)
    if (entry.get(v) && map[v] >= 0) zero.push_back((uint16_t)(map[v] * kRegStride));
  for (int v = kTripBase; v < ir.nv; v++)
    if (entry.get(v) && map[v] >= 0) zero.push_back((uint16_t)(map[v] * kRegStride));
  for (int s = 0; s < n_heap; s++) zero.push_back((uint16_t)((heap_base + s) * kRegStride));
  std::sort(zero.begin(), zero.end());
  zero.erase(std::unique(zero.begin(), zero.end()), zero.end());

  hdr.n_ops = (uint32_t)dops.size();
  hdr.n_regs = (uint32_t)std::max(n_regs + n_heap, 1);
  hdr.n_bufs = (uint32_t)ir.n_bufs;
  hdr.shared_mask = ir.shared_mask;
  hdr.seed = ir.seed;
  hdr.n_sites = (uint32_t)ir.n_sites;
  hdr.sreg_mask = sreg_mask;
  hdr.n_zero = (uint32_t)zero.size();
  hdr.n_loops = (uint32_t)ir.n_loops;
  uint32_t ops_off = sizeof(DevProgHdr);
  uint32_t loc_off = ops_off + (uint32_t)(dops.size() * sizeof(DevOp));
  uint32_t zero_off = loc_off + 4u * (uint32_t)ir.n_sites;
  uint32_t bytes_total = zero_off + 2u * (uint32_t)zero.size();
  bytes_total = (bytes_total + 15u) & ~15u;
  hdr.ops_off = ops_off;
  hdr.loc_off = loc_off;
  hdr.zero_off = zero_off;
  hdr.bytes = bytes_total;

  uint8_t* blob = (uint8_t*)calloc(1, bytes_total);
  if (!blob) return CUFZ_E_NOMEM;
  memcpy(blob, &hdr, sizeof(hdr));
  memcpy(blob + ops_off, dops.data(), dops.size() * sizeof(DevOp));
  for (int s = 0; s < ir.n_sites; s++) {
    uint32_t w = (uint32_t)ir.loc0[s] | ((uint32_t)ir.loc1[s] << 16);
    memcpy(blob + loc_off + 4 * s, &w, 4);
  }
  if (!zero.empty()) memcpy(blob + zero_off, zero.data(), 2 * zero.size());
  out->hdr = hdr;
  out->blob = blob;
  out->blob_bytes = bytes_total;
  out->n_bufs = (uint32_t)ir.n_bufs;
  out->shared_mask = ir.shared_mask;
  out->prex = std::move(prex);
  out->block_serial = ir.block_serial;
  fill_stats(ir, n_in, n_regs, &out->stats);
  return CUFZ_OK;
}

void free_program(LoadedProgram* p) {
  free(p->blob);
  p->blob = nullptr;
  p->prex.reset();
}

}  // namespace cufz

using namespace cufz;

extern "C" cufz_status cufz_validate_program(const void* bytes, size_t nbytes) {
  Ir ir;
  return decode((const uint8_t*)bytes, nbytes, &ir) ? CUFZ_OK : CUFZ_E_INVALID_PROGRAM;
}

extern "C" cufz_status cufz_prune_program(const void* bytes, size_t nbytes, void* out,
                                          size_t out_cap, size_t* out_bytes,
                                          cufz_prog_stats* stats) {
  if ((!out && out_cap) || !out_bytes) return CUFZ_E_INVALID_ARG;
  Ir ir;
  if (!decode((const uint8_t*)bytes, nbytes, &ir)) return CUFZ_E_INVALID_PROGRAM;
  if (!prepare_barriers(&ir)) return CUFZ_E_UNSUPPORTED;
  int n_in = (int)ir.ops.size();
  prune(&ir);
  std::vector<int> map;
  Bits entry;
  int n_regs = allocate(ir, false, &map, &entry);
  if (n_regs > 255) return CUFZ_E_INVALID_PROGRAM;
  std::vector<uint8_t> v;
  std::vector<IrOp> kept;
  // a block-serial program keeps its barriers (they order its stores)
  for (const auto& o : ir.ops)
    if ((o.kept && o.opc != B_NOP) || (ir.block_serial && o.opc == B_BAR)) kept.push_back(o);
  if (kept.empty()) {  // the format needs one op
    IrOp nop;
    nop.opc = B_NOP;
    kept.push_back(nop);
  }
  put32(v, kMagic);
  put16(v, 1);
  put16(v, (uint16_t)kept.size());
  v.push_back((uint8_t)std::max(n_regs, 1));
  v.push_back((uint8_t)ir.n_bufs);
  v.push_back((uint8_t)ir.n_sites);
  v.push_back((uint8_t)ir.flags);  // the flag stays; eliminated barriers are gone
  put16(v, (uint16_t)ir.shared_mask);
  put16(v, 0);
  put32(v, ir.seed);
  put32(v, 0);
  put32(v, 0);
  put32(v, 0);
  for (int s = 0; s < ir.n_sites; s++) {
    put16(v, ir.loc0[s]);
    put16(v, ir.loc1[s]);
  }
  auto R = [&](int r) -> uint8_t { return r < 0 ? 0 : (uint8_t)map[r]; };
  for (const auto& o : kept) {
    uint8_t d = 0, a = 0, b = 0;
    int32_t imm = 0;
    uint8_t opc = o.opc;
    if (is_alu_reg(opc)) {
      d = R(o.dst); a = R(o.a); b = R(o.b);
    } else if (is_alu_imm(opc)) {
      d = R(o.dst); a = R(o.a); imm = o.imm;
    } else {
      switch (opc) {
        case B_SREG: d = R(o.dst); imm = o.sreg; break;
        case B_IMM: d = R(o.dst); imm = o.imm; break;
        case B_MOV: d = R(o.dst); a = R(o.a); break;
        case B_SEL: d = R(o.dst); a = R(o.a); b = R(o.b); imm = R(o.c); break;
        case B_DIV:
        case B_REM: d = R(o.dst); a = o.value_dead ? 0 : R(o.a); b = R(o.b); break;
        case B_LD: d = R(o.dst); a = R(o.a); b = (uint8_t)o.buf; imm = o.width; break;
        case B_ST:  // a stored value that is not performed is dropped (the index stands in)
          d = o.value_live ? R(o.b) : R(o.a); a = R(o.a); b = (uint8_t)o.buf; imm = o.width;
          break;
        case B_HALLOC: d = R(o.dst); a = R(o.a); break;
        case B_HFREE: a = R(o.a); break;
        case B_HLD: d = R(o.dst); a = R(o.a); b = R(o.b); imm = o.width; break;
        case B_HST: d = R(o.a); a = R(o.a); b = R(o.b); imm = o.width; break;
        case B_IF: a = R(o.a); break;
        case B_LOOP: d = R(o.dst); a = R(o.a); imm = o.imm; break;
        default: break;
      }
    }
    v.push_back(opc);
    v.push_back(d);
    v.push_back(a);
    v.push_back(b);
    put32(v, (uint32_t)imm);
  }
  *out_bytes = v.size();
  fill_stats(ir, n_in, n_regs, stats);
  if (v.size() > out_cap) return CUFZ_E_NOMEM;
  memcpy(out, v.data(), v.size());
  return CUFZ_OK;
}

// The bytecode interpreter's warp loop (run_warp): one warp runs 32
// consecutive test threads of a work item per pass, lane = test thread,
// warp-uniform dispatch over the device ops with per-lane activity bits.
// Included by engine.cu, whose kernels wrap it in the work-item loop of
// device_common.cuh.
#pragma once

#include "device_common.cuh"
#include "checked_ops.h"

namespace cufz {

__device__ __forceinline__ int32_t rf_ld(const uint8_t* rf, uint32_t off) {
  return *reinterpret_cast<const int32_t*>(rf + off);
}
__device__ __forceinline__ void rf_st(uint8_t* rf, uint32_t off, int32_t v) {
  *reinterpret_cast<int32_t*>(rf + off) = v;
}

// Runs the test threads [g0, g0 + count) of one input on this warp's lanes.
__device__ __forceinline__ void run_warp(const EngineTables& T, const DevInput* in,
                                         const uint8_t* sprog, uint8_t* rf_warp, uint32_t* hash,
                                         uint32_t g0, uint32_t count, uint32_t warp,
                                         uint32_t nwarps) {
  const uint32_t lane = threadIdx.x & 31u;
  const DevProgHdr* ph = reinterpret_cast<const DevProgHdr*>(sprog);
  const DevOp* ops = reinterpret_cast<const DevOp*>(sprog + ph->ops_off);
  const uint32_t* loc = reinterpret_cast<const uint32_t*>(sprog + ph->loc_off);
  const uint16_t* zero = reinterpret_cast<const uint16_t*>(sprog + ph->zero_off);
  const uint32_t slot = in->slot;
  const uint32_t shared_mask = ph->shared_mask;
  const uint32_t n_bufs = ph->n_bufs;
  const uint32_t seed = ph->seed;
  const uint32_t sreg_mask = ph->sreg_mask;
  const uint32_t n_zero = ph->n_zero;
  const uint32_t budget = T.iter_budget;
  const bool do_digest = !(T.flags & CUFZ_CF_NO_DIGEST);
  const uint32_t cap = T.record_cap;
  cufz_violation* recs = T.records + (size_t)slot * cap;
  SlotState* S = &T.slots[slot];
  uint8_t* rf = rf_warp + lane * kLaneBytes;
  const uint32_t lanemask_lt = (1u << lane) - 1u;

  LaneAcc acc;
  acc_init(acc);
  bool full = false;  // warp-uniform: record area known to be full
  // Reserves record slots for the violating lanes vm of the warp (every
  // lane calls it): one atomicAdd by the first of them; the group's base,
  // or ~0 once the record area is known to be full.
  auto reserve = [&](uint32_t vm) -> uint32_t {
    const uint32_t k = __popc(vm);
    const uint32_t leader = __ffs(vm) - 1;
    uint32_t rbase = 0xFFFFFFFFu;
    if (!full) {
      if (lane == leader) rbase = atomicAdd(&S->rec_reserved, k);
      rbase = __shfl_sync(FULL, rbase, leader);
      if (rbase + k >= cap) full = true;
    }
    return rbase;
  };

  const uint32_t g_end = g0 + count;
  for (uint32_t base = g0 + warp * 32u; base < g_end; base += nwarps * 32u) {
    const uint32_t g = base + lane;
    const bool valid = g < g_end;
    const uint32_t bl = udiv(g, in->mT);
    const uint32_t tl = g - bl * in->T;
    // special registers into their registers
    if (sreg_mask) {
      uint32_t q1 = udiv(tl, in->mBx);
      uint32_t tz = udiv(tl, in->mBxy);
      uint32_t tx = tl - q1 * in->Bx;
      uint32_t ty = q1 - tz * in->block[1];
      uint32_t p1 = udiv(bl, in->mGx);
      uint32_t bz = udiv(bl, in->mGxy);
      uint32_t bx = bl - p1 * in->gx;
      uint32_t by = p1 - bz * in->grid[1];
      uint32_t m = sreg_mask;
      while (m) {
        uint32_t id = __ffs(m) - 1;
        m &= m - 1;
        int32_t v;
        switch (id) {
          case 0: v = (int32_t)tx; break;
          case 1: v = (int32_t)ty; break;
          case 2: v = (int32_t)tz; break;
          case 3: case 4: case 5: v = (int32_t)in->block[id - 3]; break;
          case 6: v = (int32_t)bx; break;
          case 7: v = (int32_t)by; break;
          case 8: v = (int32_t)bz; break;
          case 9: case 10: case 11: v = (int32_t)in->grid[id - 9]; break;
          default: v = in->args[id - 12]; break;
        }
        rf_st(rf, (uint32_t)ph->sreg_reg[id] * kRegStride, v);
      }
    }
    for (uint32_t k = 0; k < n_zero; k++) rf_st(rf, zero[k], 0);

    bool act = valid, alive = valid;
    uint32_t stk_act = 0, stk_aux = 0;
    uint32_t prev = 0, ordinal = 0, back = 0;
    uint32_t dh = digest_start(bl, tl);  // digest state of the thread

    uint32_t pc = 0;
#pragma unroll 1
    for (;;) {
      const DevOp op = ops[pc];
      const uint32_t opc = op.opc;
      // value ops: one dispatch, the op inline, a predicated store
      int32_t r;
      switch (opc) {
#define CUFZ_ALU_CASES(ID, EXPR)                                        \
  case D_ALU0 + ID: {                                                   \
    const int32_t x = rf_ld(rf, op.a), y = rf_ld(rf, op.b);             \
    const uint32_t ux = (uint32_t)x, uy = (uint32_t)y;                  \
    (void)ux; (void)uy;                                                 \
    r = (EXPR);                                                         \
    goto value_done;                                                    \
  }                                                                     \
  case D_ALUI0 + ID: {                                                  \
    const int32_t x = rf_ld(rf, op.a), y = op.imm;                      \
    const uint32_t ux = (uint32_t)x, uy = (uint32_t)y;                  \
    (void)ux; (void)uy;                                                 \
    r = (EXPR);                                                         \
    goto value_done;                                                    \
  }
        CUFZ_ALU_CASES(A_ADD, (int32_t)(ux + uy))
        CUFZ_ALU_CASES(A_SUB, (int32_t)(ux - uy))
        CUFZ_ALU_CASES(A_MUL, (int32_t)(ux * uy))
        CUFZ_ALU_CASES(A_SHL, (int32_t)(ux << (uy & 31u)))
        CUFZ_ALU_CASES(A_SHR, x >> (int)(uy & 31u))
        CUFZ_ALU_CASES(A_SHRU, (int32_t)(ux >> (uy & 31u)))
        CUFZ_ALU_CASES(A_AND, (int32_t)(ux & uy))
        CUFZ_ALU_CASES(A_OR, (int32_t)(ux | uy))
        CUFZ_ALU_CASES(A_XOR, (int32_t)(ux ^ uy))
        CUFZ_ALU_CASES(A_MIN, min(x, y))
        CUFZ_ALU_CASES(A_MAX, max(x, y))
        CUFZ_ALU_CASES(A_SETLT, (int32_t)(x < y))
        CUFZ_ALU_CASES(A_SETLE, (int32_t)(x <= y))
        CUFZ_ALU_CASES(A_SETEQ, (int32_t)(x == y))
        CUFZ_ALU_CASES(A_SETNE, (int32_t)(x != y))
        CUFZ_ALU_CASES(A_SETLTU, (int32_t)(ux < uy))
#undef CUFZ_ALU_CASES
        case D_MOV:  // x = 1: a special-register read, not an executed op
          r = rf_ld(rf, op.a);
          if (op.x) goto value_store;
          goto value_done;
        case D_IMM:
          r = op.imm;
          goto value_done;
        case D_SEL:
          r = rf_ld(rf, op.a) != 0 ? rf_ld(rf, op.b) : rf_ld(rf, (uint32_t)op.imm);
          goto value_done;
        default:
          break;
      }
      if (false) {
      value_done:
        if (act) acc.n_ops++;
      value_store:
        if (act) rf_st(rf, op.d, r);
        pc++;
        continue;
      }
      bool head = false;
      switch (opc) {
        case D_LD:
        case D_LDX:
        case D_ST: {
          const int32_t idx = rf_ld(rf, op.a);
          const uint32_t buf = op.b;
          const uint32_t lw = op.x;
          const uint32_t w = 1u << lw;
          const int64_t off = (int64_t)idx * (int64_t)w;
          const int64_t len = in->len[buf];
          const bool viol = act && (idx < 0 || off + (int64_t)w > len);
          if (act) {
            acc.n_acc++;
            if (do_digest) dh = access_step(dh, access_k((uint32_t)op.imm), idx);
          }
          const uint32_t vm = __ballot_sync(FULL, viol);
          if (vm) {
            const uint32_t rbase = reserve(vm);
            if (viol) {
              acc.n_viol++;
              if (acc.first_key == ~0ull) acc.first_key = first_key_of(bl, tl, ordinal);
              const uint32_t rank = __popc(vm & lanemask_lt);
              if (rbase != 0xFFFFFFFFu && rbase + rank < cap) {
                const uint32_t cls =
                    classify(in, shared_mask, n_bufs, buf, off, w, (int64_t)T.redzone);
                write_record(recs + rbase + rank, bl, tl, ordinal, (uint32_t)op.imm, buf,
                             opc == D_ST ? 1u : 0u, w, (shared_mask >> buf) & 1u, cls, off);
              }
            }
          }
          if (opc == D_LD && act) {
            int32_t v = 0;
            if (!viol && !((shared_mask >> buf) & 1u)) {
              uint32_t word = mix32(seed ^ (buf * 0x9E3779B9u) ^ (uint32_t)(off >> 2));
              v = lw == 0 ? (int32_t)((word >> (8u * ((uint32_t)off & 3u))) & 0xFFu) : (int32_t)word;
            }
            rf_st(rf, op.d, v);
          }
          if (act) ordinal++;
          pc++;
          break;
        }
        case D_DIVREM: {  // a checked division: a zero divisor is a violation of kind 2
          const int32_t y = rf_ld(rf, op.b);
          const bool fault = act && y == 0;
          if (act) acc.n_ops++;
          const uint32_t vm = __ballot_sync(FULL, fault);
          if (vm) {
            const uint32_t rbase = reserve(vm);
            if (fault) {
              acc.n_viol++;
              if (acc.first_key == ~0ull) acc.first_key = first_key_of(bl, tl, ordinal);
              const uint32_t rank = __popc(vm & lanemask_lt);
              if (rbase != 0xFFFFFFFFu && rbase + rank < cap)
                write_record(recs + rbase + rank, bl, tl, ordinal, (uint32_t)op.imm, 0u, 2u, 0u,
                             0u, CUFZ_CLS_DIV_ZERO, 0);
            }
          }
          if (act && (op.x & 2u)) {
            const int32_t x = rf_ld(rf, op.a);
            const int32_t mn = (int32_t)0x80000000u;
            int32_t v = 0;
            if (y != 0) v = (x == mn && y == -1) ? ((op.x & 1u) ? 0 : mn) : ((op.x & 1u) ? x % y : x / y);
            rf_st(rf, op.d, v);
          }
          if (act) ordinal++;
          pc++;
          break;
        }
        case D_HALLOC: {  // block of n >= 1 bytes at site s: state n, handle s + 1
          if (act) {
            const int32_t n = rf_ld(rf, op.a);
            int32_t h = 0;
            if (n >= 1) {
              rf_st(rf, ((uint32_t)op.j0 + (uint32_t)op.imm) * kRegStride, n);
              h = op.imm + 1;
            }
            rf_st(rf, op.d, h);
            acc.n_ops++;
          }
          pc++;
          break;
        }
        case D_HFREE: {  // NULL: no-op; no allocated block or a freed one: kind 3
          uint32_t cls = 0;
          if (act) {
            const int32_t h = rf_ld(rf, op.a);
            if (h != 0) {
              const uint32_t s = (uint32_t)h - 1u;
              const uint32_t so = ((uint32_t)op.j0 + s) * kRegStride;
              const int32_t st = s < op.j1 ? rf_ld(rf, so) : 0;
              if (st == 0)
                cls = CUFZ_CLS_INVALID_FREE;
              else if (st < 0)
                cls = CUFZ_CLS_DOUBLE_FREE;
              else
                rf_st(rf, so, -1);
            }
            acc.n_ops++;
          }
          const uint32_t vm = __ballot_sync(FULL, cls != 0);
          if (vm) {
            const uint32_t rbase = reserve(vm);
            if (cls) {
              acc.n_viol++;
              if (acc.first_key == ~0ull) acc.first_key = first_key_of(bl, tl, ordinal);
              const uint32_t rank = __popc(vm & lanemask_lt);
              if (rbase != 0xFFFFFFFFu && rbase + rank < cap)
                write_record(recs + rbase + rank, bl, tl, ordinal, (uint32_t)op.imm, 0u, 3u, 0u,
                             2u, cls, 0);
            }
          }
          if (act) ordinal++;
          pc++;
          break;
        }
        case D_HACC: {  // an access through a heap handle (space 2)
          const int32_t idx = rf_ld(rf, op.a);
          const int32_t h = rf_ld(rf, op.b);
          const uint32_t w = 1u << (op.x & 7u);
          const int64_t off = (int64_t)idx * (int64_t)w;
          const uint32_t s = (uint32_t)h - 1u;
          const int32_t st = s < op.j1 ? rf_ld(rf, ((uint32_t)op.j0 + s) * kRegStride) : 0;
          uint32_t cls = 0;
          if (act) {
            acc.n_acc++;
            if (do_digest) dh = access_step(dh, access_k((uint32_t)op.imm), idx);
            const int64_t len = st, R = (int64_t)T.redzone;
            if (st == 0)
              cls = CUFZ_CLS_WILD;
            else if (st < 0)
              cls = CUFZ_CLS_USE_AFTER_FREE;
            else if (off < 0 || off + (int64_t)w > len)
              cls = (off < 0 && off >= -R)       ? CUFZ_CLS_UNDERFLOW_RZ
                    : (off >= 0 && off < len + R) ? CUFZ_CLS_OVERFLOW_RZ
                                                  : CUFZ_CLS_WILD;
          }
          const uint32_t vm = __ballot_sync(FULL, cls != 0);
          if (vm) {
            const uint32_t rbase = reserve(vm);
            if (cls) {
              acc.n_viol++;
              if (acc.first_key == ~0ull) acc.first_key = first_key_of(bl, tl, ordinal);
              const uint32_t rank = __popc(vm & lanemask_lt);
              if (rbase != 0xFFFFFFFFu && rbase + rank < cap)
                write_record(recs + rbase + rank, bl, tl, ordinal, (uint32_t)op.imm,
                             st == 0 ? 0u : s, (op.x & 8u) ? 1u : 0u, w, 2u, cls, off);
            }
          }
          if (act && (op.x & 16u)) rf_st(rf, op.d, 0);
          if (act) ordinal++;
          pc++;
          break;
        }
        case D_IF: {
          const bool c = rf_ld(rf, op.a) != 0;
          if (__any_sync(FULL, act)) {
            const uint32_t lw2 = loc[op.x];
            const uint32_t cur = c ? (lw2 >> 16) : (lw2 & 0xFFFFu);
            const uint32_t e = (cur ^ prev) & 0xFFFFu;
            if (act) {
              prev = cur >> 1;
              acc.n_branch++;
            }
            const bool hit = act && !edge_saturated(hash, e);
            if (__any_sync(FULL, hit)) {
              const uint32_t peers = __match_any_sync(FULL, hit ? e : 0xFFFFFFFFu);
              if (hit && lane == (uint32_t)(__ffs(peers) - 1)) edge_add(hash, T, slot, e, __popc(peers));
            }
          }
          stk_act = (stk_act << 1) | (act ? 1u : 0u);
          stk_aux = (stk_aux << 1) | ((act && !c) ? 1u : 0u);
          act = act && c;
          pc = __any_sync(FULL, act) ? pc + 1 : op.j0;
          break;
        }
        case D_ELSE: {
          act = (stk_aux & 1u) && alive;
          stk_aux &= ~1u;
          pc = __any_sync(FULL, act) ? pc + 1 : op.j0;
          break;
        }
        case D_ENDIF: {
          act = (stk_act & 1u) && alive;
          stk_act >>= 1;
          stk_aux >>= 1;
          pc++;
          break;
        }
        case D_LOOP: {
          if (act) {
            int32_t n = rf_ld(rf, op.a);
            int32_t trip = n < 0 ? 0 : (n > op.imm ? op.imm : n);
            rf_st(rf, op.b, trip);
            rf_st(rf, op.d, 0);
          }
          stk_act = (stk_act << 1) | (act ? 1u : 0u);
          stk_aux = (stk_aux << 1) | (act ? 1u : 0u);
          head = true;
          break;
        }
        case D_ENDLOOP: {
          if (act) {
            back++;
            if (back > budget) {
              alive = false;
              act = false;
              acc.budget_hit = true;
              stk_aux &= ~1u;
            } else {
              rf_st(rf, op.d, rf_ld(rf, op.d) + 1);
            }
          }
          head = true;
          break;
        }
        default:  // D_END
          break;
      }
      if (opc == D_END) break;
      if (head) {
        const bool inl = (stk_aux & 1u) && alive;
        const bool cont = inl && rf_ld(rf, op.d) < rf_ld(rf, op.b);
        if (__any_sync(FULL, inl)) {
          const uint32_t lw2 = loc[op.x];
          const uint32_t cur = cont ? (lw2 >> 16) : (lw2 & 0xFFFFu);
          const uint32_t e = (cur ^ prev) & 0xFFFFu;
          if (inl) {
            prev = cur >> 1;
            acc.n_branch++;
          }
          const bool hit = inl && !edge_saturated(hash, e);
          if (__any_sync(FULL, hit)) {
            const uint32_t peers = __match_any_sync(FULL, hit ? e : 0xFFFFFFFFu);
            if (hit && lane == (uint32_t)(__ffs(peers) - 1)) edge_add(hash, T, slot, e, __popc(peers));
          }
        }
        if (inl && !cont) stk_aux &= ~1u;
        act = cont;
        if (__any_sync(FULL, act)) {
          pc = op.j1;
        } else {
          act = (stk_act & 1u) && alive;
          stk_act >>= 1;
          stk_aux >>= 1;
          pc = op.j0;
        }
      }
    }
    if (valid && do_digest) acc.digest += digest_end(dh);
  }

  acc_flush(T, slot, acc);
}

}  // namespace cufz

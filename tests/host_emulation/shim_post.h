// TEST-ONLY, included after jit_kernel.cuh: the end-of-item reduction of the
// per-lane accumulators for a warp of one lane (device_common.cuh's
// acc_flush reduces over 32 lanes with shuffles), put in its place for the
// program functions that follow.
#pragma once

namespace cufz {
static void shim_acc_flush(const EngineTables& T, uint32_t slot, const LaneAcc& a) {
  SlotState* S = &T.slots[slot];
  S->n_accesses += a.n_acc;
  S->digest += a.digest;
  S->n_branch += a.n_branch;
  S->n_ops += a.n_ops;
  S->n_violations += a.n_viol;
  if (a.first_key < S->first_key) S->first_key = a.first_key;
  if (a.budget_hit) S->flags |= (uint32_t)CUFZ_FL_BUDGET;
}
}  // namespace cufz

#define acc_flush shim_acc_flush

// ots_batch.cuh -- device-side description of a batch of independent instances.
//
// A batch keeps many instances of the multi-commodity problem resident at once and advances
// all of them with one kernel launch per "tick": in every tick each running instance executes
// the next step of its own sequence of Algorithm 2 steps (set-up, initial backward sweep,
// then passes of source update, forward steps t = 2..T-1, sink update, backward steps
// t = T-1..2, and after convergence one flows pass).  Instances therefore sit at different
// steps and horizons in the same launch, and an instance that finishes frees its slot
// without stopping the others.  The work of a tick is a list of items (slot, item index);
// item k of an instance covers nodes [k npi, (k+1) npi) of its node panels (npi = rounds x
// npb, one round being one node row per G-thread group of the block), or a slice of its
// states or boundary triples, depending on the step.
#pragma once

#include "ots_device.cuh"

namespace ots {

constexpr int kTickBlock = 256;   // threads per block of the batched kernel

// slot states (BatchCtl::status)
enum : int {
  kSlotIdle = 0,
  kSlotRunning = 1,        // Sinkhorn passes
  kSlotFlows = 2,          // flows pass after the last Sinkhorn pass
  kSlotConverged = 3,      // final: converged, flows ready
  kSlotNotConverged = 4,   // final: max passes reached, flows of the last duals ready
  kSlotInfeasible = 5,     // final: a source or sink message vanished
  kSlotNumeric = 6,        // final: NaN in the convergence measures
  kSlotStopped = 7         // final: stopped by the host (timeout)
};
// Epsilon continuation: an instance admitted with shift k > 0 runs its passes at eps 2^k until
// the stage tolerance, then at eps 2^(k-1), ..., and at eps to its tolerance.  Halving epsilon
// doubles log2 K_L's divisor and every log dual exactly (powers of two), so a stage change is a
// set-up step that doubles the duals and rebuilds W, the boundary panels and the backward
// messages, with the pass count carried on.

struct BndSide {
  int n_seg, n_tri;
  const int *seg_ptr, *seg_node, *seg_l, *tri_other, *tri_l;
  const double *tri_R, *tri_logR;
  double *tri_logU, *tri_flow;
};

// Static description of one resident instance (written by the host at admission; copied
// into shared memory by every item, 16 bytes per lane).
struct alignas(16) BatchInst {
  int V, S, T, Lp, G, C, n_items, npb;   // npb: nodes per round = kTickBlock / G
  int rounds, npi, pad1, pad2;           // npi: nodes per item = rounds * npb
  QScale qs;
  double mass, eps, tol;
  double stage_tol;              // tolerance of the warm-start stages (epsilon continuation)
  int max_passes;
  int kl_stride;                 // S when the costs vary with the interval t (row t of kl), else 0
  int cap_stride;                // S when the capacities vary with t (row t of logd, cap), else 0
  int pad3;
  const int *in_ptr, *in_state, *in_nbr, *out_ptr, *out_state, *out_nbr;
  const float *kl_hi, *kl_lo, *logd_hi, *logd_lo;
  const float2 *cap;             // [S] d as a float-float
  float2 *lu;                    // [T+1][S] log2 u_t as a float-float
  float *w_hi, *w_lo;            // [T+1][S] W_t
  double *flow;                  // [T+1][S] P_t
  float *a0_hi, *a1_hi, *a2_hi;  // A_1, and A_t for even / odd t
  lo_t *a0_lo, *a1_lo, *a2_lo;
  float *b_hi;                   // [T-1][V][Lp], row t-2 holds B_t
  lo_t *b_lo;
  BndSide src, snk;
  double *partials;              // [3 n_items] per-item partial sums of the current step
};

// Dynamic state of one slot (device-resident; the host reads a copy after every launch).
struct alignas(16) BatchCtl {
  int status;
  int step;                      // position in the step sequence of the current status
  int passes;                    // completed Sinkhorn passes
  int final_status;              // status to enter after the flows pass
  unsigned int counter;          // items of this instance finished in the current tick
  int shift;                     // epsilon continuation: this stage runs at eps 2^shift
  long long ticks;               // ticks this instance has executed
  DevStats stats;
  PassReport report;
};

static_assert(sizeof(BatchInst) % 16 == 0, "BatchInst is copied in 16-byte words");

struct TickArgs {
  const BatchInst *inst;         // [slots]
  BatchCtl *ctl;                 // [slots]
  const int2 *items;             // (slot, item index within the instance)
  const int *n_items;            // device scalar: number of items in the list
};

}  // namespace ots

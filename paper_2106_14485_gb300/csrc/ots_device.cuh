// ots_device.cuh -- device-side types and helpers of the GB300 Sinkhorn solver.
//
// Representation.  Every message, dual and weight is a base-2 logarithm ("bits"): the
// exponentials of Algorithm 2 become ex2 and the logarithms lg2 on the SFU.  A message
// entry is stored as an unevaluated pair hi + lo with hi an FP32 value and lo an FP16
// value, |lo| <= ulp(hi) / 2: about 35 significant bits in 6 bytes.  Plain FP32 logs
// carry an absolute error of |x| * 2^-24, which at eps = 0.005 (|x| ~ 1e4 bits) is far
// above the 1e-5 relative flow tolerance; the pair keeps the absolute error near 1e-7.
// Arithmetic on pairs is float-float (two_sum), all in FP32 instructions.
//
// log 0 is represented by the finite sentinel kNeg (-1e30): no inf or NaN ever enters the
// float-float operations (two_sum of infinities would produce NaN).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ots {

constexpr float kNeg = -1e30f;        // log2 0
constexpr float kNegThresh = -1e29f;  // anything below is treated as log2 0
constexpr int kBlock = 256;           // threads per block of the message kernels

struct alignas(16) DevStats {
  double src_resid;   // sum |U01 .* Psi_1 - R01| (taken before the source update)
  double cap_viol;    // sum_t sum_i (P_t - d)_+ (taken before each capacity update)
  double dual_src;    // sum R01 log2 U01
  double dual_snk;    // sum R0T log2 U0T
  double dual_cap;    // sum_t sum_i d_i log2 u_t[i]   (finite d only)
  double mass_snk;    // <K, U> right after the sink update
  double bad;         // > 0 if a source or sink had a vanishing message (infeasible)
  double pad;
};

// Per-pass summary written by the last kernel of a pass (host reads it every few passes).
struct alignas(16) PassReport {
  double src_resid_rel;
  double cap_viol_rel;
  double dual_objective;   // natural units (Theorem 3 convention)
  double bad;
  long long passes;        // passes completed since creation
  long long pad;
};

// Arguments of the node-level message kernels.
//   forward  (fwd = true):  out[v] = LSE_{j in in(v)}  (x[tail j] + W_t[j])   and, per in-state
//                           j, the capacity update from LSE_l(x[tail j] + y[v]) (Corollary 7)
//   backward (fwd = false): out[v] = LSE_{j in out(v)} (x[head j] + W_t[j])
struct StepArgs {
  int V;
  int Lp;                     // padded commodity count (row length of a panel)
  const int *ptr;             // [V+1] CSR over nodes: in-states (fwd) / out-states (bwd)
  const int *state;           // state id of each listed state
  const int *nbr;             // tail (fwd) / head (bwd) node of each listed state
  const float *x_hi;          // input panel [V][Lp]
  const __half *x_lo;
  const float *y_hi;          // fwd only: B_{t+1} panel [V][Lp]
  const __half *y_lo;
  float *out_hi;              // output panel [V][Lp]
  __half *out_lo;
  const float *kl_hi;         // [S] log2 K_L (commodity-independent rows)
  const float *kl_lo;
  const float *klc_hi;        // [S][Lp] log2 K_L per commodity (nullptr if rank-1)
  const __half *klc_lo;
  const float *logd_hi;       // [S] log2 d (kNeg for d = 0)
  const float *logd_lo;
  const double *cap;          // [S] d (inf allowed)
  double *logu_t;             // [S] log2 u_t (row t)
  float *w_hi_t;              // [S] W_t = log2 K_L + log2 u_t (row t)
  float *w_lo_t;
  double *flow_t;             // [S] aggregate P_t (flows mode)
  double *partials;           // [2 * gridDim.x] per-block partial sums
  unsigned int *counter;      // last-block counter
  DevStats *stats;
  int mode;                   // 0: Sinkhorn update, 1: flows only (no update)
};

// Boundary kernels (sources, sinks): segments of (node, commodity) with their triples.
struct BndArgs {
  int n_seg;
  const int *seg_ptr;         // [n_seg+1] into the triple arrays
  const int *seg_node;        // node of the segment (head of the source state / tail of the sink state)
  const int *seg_l;           // commodity of the segment
  const int *tri_node_other;  // node whose message row is read for each triple:
                              //   sources: head(state) (Psi_1 = B_2[head]); sinks: tail(state)
  const double *tri_R;        // mass
  const double *tri_logR;     // log2 mass
  double *tri_logU;           // log2 U (in/out)
  int Lp;
  const float *msg_hi;        // message panel read (B_2 for sources, A_{T-1} for sinks)
  const __half *msg_lo;
  float *out_hi;              // boundary panel written (A_1 for sources, B_T for sinks)
  __half *out_lo;
  double *partials;
  unsigned int *counter;
  DevStats *stats;
  int mode;                   // 0: update U, 1: rebuild the panel from the current U only
  int is_source;
};

// ------------------------------------------------------------------------------------
// scalar helpers
// ------------------------------------------------------------------------------------

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no overflow).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Merge two (max, scaled-sum) pairs of a log-sum-exp: value = m + log2(s).
__device__ __forceinline__ void lse_merge(float &m, float &s, float om, float os) {
  float d = m - om;
  float f = ex2(-fabsf(d));
  if (d >= 0.f) {
    s = fmaf(os, f, s);
  } else {
    s = fmaf(s, f, os);
    m = om;
  }
}

// Online log-sum-exp accumulation of one float-float term (s, e) into (m, acc).  Terms at
// log 0 are skipped: two_sum(kNeg, x) returns (kNeg, x), whose error part x must not reach
// ex2 (it can overflow).
__device__ __forceinline__ void lse_push(float &m, float &acc, float s, float e) {
  if (s < kNegThresh) return;
  if (s > m) {
    acc = fmaf(acc, ex2(m - s), ex2(e));
    m = s;
  } else {
    acc += ex2((s - m) + e);
  }
}

// Finish a log-sum-exp: (m + log2(acc)) as a normalised float-float pair.
__device__ __forceinline__ void lse_finish(float m, float acc, float &hi, float &lo) {
  if (m < kNegThresh || !(acc > 0.f)) {
    hi = kNeg;
    lo = 0.f;
    return;
  }
  two_sum(m, lg2(acc), hi, lo);
}

__device__ __forceinline__ void store_pair(float *hp, __half *lp, float hi, float lo) {
  if (hi < kNegThresh) { hi = kNeg; lo = 0.f; }
  *hp = hi;
  *lp = __float2half_rn(lo);
}

}  // namespace ots

// ots_device.cuh -- device-side types and helpers of the GB300 Sinkhorn solver.
//
// Representation.  Every message, dual and weight is a base-2 logarithm ("bits"): the
// exponentials of Algorithm 2 become ex2 on the SFU and the logarithms log2f.  A message
// entry x is stored in 6 bytes as x = hi + (lo - 32768) * q / 65536 with
//   hi : FP32, an integer multiple of the per-problem quantum q = 2^k (k < 0),
//   lo : uint16, the remainder in units of q / 65536 (|remainder| <= q / 2), biased by 32768
//        so that OR-ing it into the mantissa of 2^23 yields the float 2^23 + lo exactly
//        (decoding costs one logic instruction, no integer-to-float conversion).
// Sums of two hi values are then exact in FP32 (while |sum| < 2^24 q), so the inner loops
// need no compensated additions, and the stored value has an absolute resolution of
// q / 2^17 regardless of its magnitude.  Plain FP32 logs would carry an absolute error of
// |x| 2^-24, which at eps = 0.005 (|x| ~ 1e4 bits) is far above the 1e-5 relative flow
// tolerance.  Per-state weights W = log2 K_L + log2 u keep hi on the same grid and a float lo.
//
// log 0 is represented by the finite sentinel kNeg (-1e30) with lo = 0; terms whose hi part is
// below kNegThresh are skipped by every reduction.
//
// Per-state duals log2 u_t and capacities d are float-float pairs (float2: value = x + y), and
// per-thread sums that decide convergence are float-float too; FP64 appears only in the
// per-block totals, the boundary updates and the flows.  (The FP64 pipe of this GPU issues a
// warp instruction in tens of cycles, so FP64 on the per-state path dominated the step.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ots {

constexpr float kNeg = -1e30f;        // log2 0
constexpr float kNegThresh = -1e29f;  // anything below is treated as log2 0
constexpr int kBlock = 256;           // threads per block of the message kernels

typedef uint16_t lo_t;
constexpr float kLoBias = 8421376.0f;   // 2^23 + 32768: float(2^23 | lo) - kLoBias = signed remainder
constexpr lo_t kLoZero = 32768;

// The quantum of the hi parts and the unit of the lo parts (all powers of two).
struct QScale {
  float q;        // 2^k
  float inv_q;    // 2^-k
  float lo_unit;  // q / 65536
  float lo_inv;   // 65536 / q
};

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
//   forward:  out[v] = LSE_{j in in(v)}  (x[tail j] + W_t[j])   and, per in-state j, the
//             capacity update from LSE_l(x[tail j] + y[v]) (Corollary 7)
//   backward: out[v] = LSE_{j in out(v)} (x[head j] + W_t[j])
struct StepArgs {
  int V;
  int Lp;                     // padded commodity count (row length of a panel)
  QScale qs;
  const int *ptr;             // [V+1] CSR over nodes: in-states (fwd) / out-states (bwd)
  const int *state;           // state id of each listed state
  const int *nbr;             // tail (fwd) / head (bwd) node of each listed state
  const float *x_hi;          // input panel [V][Lp]
  const lo_t *x_lo;
  const float *y_hi;          // fwd only: B_{t+1} panel [V][Lp]
  const lo_t *y_lo;
  float *out_hi;              // output panel [V][Lp]
  lo_t *out_lo;
  const float *kl_hi;         // [S] log2 K_L (commodity-independent rows), float-float
  const float *kl_lo;
  const float *klc_hi;        // [S][Lp] log2 K_L per commodity, panel format (nullptr if rank-1)
  const lo_t *klc_lo;
  const float *logd_hi;       // [S] log2 d (kNeg for d = 0)
  const float *logd_lo;
  const float2 *cap;          // [S] d as a float-float (x = +inf for no capacity)
  float2 *lu_t;               // [S] log2 u_t (row t) as a float-float; (kNeg, 0) for u = 0
  float *w_hi_t;              // [S] W_t hi (on the q grid)
  float *w_lo_t;              // [S] W_t lo
  double *flow_t;             // [S] aggregate P_t (flows mode)
  double *partials;           // [2 * gridDim.x] per-block partial sums
  unsigned int *counter;      // last-block counter
  DevStats *stats;
  int mode;                   // 0: Sinkhorn update, 1: flows only (no update)
  int persist_grid_fwd;       // > 0: pipelined persistent forward kernel with this grid
  int persist_grid_bwd;       // > 0: pipelined persistent backward kernel with this grid
  // CSR-ordered copies for the pipelined kernels (one independent load per work item):
  const float *in_kl_hi;      // [S] log2 K_L of the state at in-CSR position j
  const float *in_kl_lo;
  const float *in_logd_hi;    // [S] log2 d at in-CSR position j
  const float *in_logd_lo;
  const float2 *in_cap;       // [S] d at in-CSR position j
  const int *in_outpos;       // [S] out-CSR position of the state at in-CSR position j
  float2 *lu_in_t;            // [S] log2 u_t by in-CSR position
  float *wout_hi_t;           // [S] W_t by out-CSR position
  float *wout_lo_t;
  float *cref_in_t;           // [S] by in-CSR position: column maximum of an earlier pass (NaN: none)
  // commodity-dependent capacities (register kernels with per-commodity K_L):
  const float2 *dc;           // [S][Lp] log2 D^(0,t) as float-float (x = +inf: none; log2 0 = kNeg)
  float *uc_t;                // [S][Lp] log2 U^(0,t) of row t (nullptr: no commodity capacities)
  int kl_shift;               // log2 K_L is read as kl * 2^-kl_shift (epsilon 2^kl_shift times larger)
  double *slot;               // [2 * blocks] or nullptr: each block's FP64 sums of this step, added up at
                              // the end of the pass (nullptr: a last-block reduction into stats)
  const unsigned char *fixed_w; // [S] or nullptr: 1 = a storage state, whose capacity update ran before this
                              // step (its W_t is read back here, nothing about it is stored)
  unsigned int wait_tries;    // pipelined kernels: tries of each bounded mbarrier wait (each <= 2 us)
  int withhold_stage;         // test switch: the consumers never release their first stage, so that the
                              // bounded waits of the pipelined kernels run out (no copy stays in flight)
};

// Storage states (a state that may follow itself, K_ss = 1: storage on an edge, the source and
// sink states of the traffic-routing model; Section 3.3).  K = B_in B_out + D with D diagonal
// over those states, so a storage state k (state s) owns message row row0 + k of every panel:
//   forward:  A_t[row0 + k] = hatPsi_{t+1}[s] = A_t[tail s] (+) (A_{t-1}[row0 + k] + W_t[s])
//   backward: B_t[row0 + k] = Psi_{t-1}[s]    = B_t[head s] (+) (B_{t+1}[row0 + k] + W_t[s])
// ((+): log-sum-exp; a missing tail or head contributes log 0).
struct StoreRowArgs {
  int n, Lp, row0;            // storage states, row length, first storage row (= number of nodes)
  QScale qs;
  const int *state;           // [n] state index
  const int *node;            // [n] tail (forward) or head (backward) node, -1 for none
  float *p_hi;                // panel of this step: node rows read, storage rows written
  lo_t *p_lo;
  const float *q_hi;          // panel of the step before (nullptr at a boundary: copy only)
  const lo_t *q_lo;
  const float *w_hi, *w_lo;   // W of this step by state
};

// Boundary terms of storage states: row row0 + k[i] of commodity l[i] takes (+) log2 U of triple q[i].
struct StoreTriArgs {
  int n, Lp, row0;
  QScale qs;
  const int *k, *l, *q;
  const double *tri_logU;
  float *p_hi;
  lo_t *p_lo;
};

// Capacity update of the storage states before forward step t: their column sums read the
// storage rows of A_{t-1} (x) and B_{t+1} (y).
struct StoreUpdArgs {
  int n, Lp, row0;
  const int *state;
  const float *x_hi, *y_hi;
  const lo_t *x_lo, *y_lo;
};

// Boundary kernels (sources, sinks): segments of (node, commodity) with their triples.
struct BndArgs {
  int n_seg;
  QScale qs;
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
  const lo_t *msg_lo;
  float *out_hi;              // boundary panel written (A_1 for sources, B_T for sinks); nullptr: none
  lo_t *out_lo;
  double *partials;
  unsigned int *counter;
  DevStats *stats;
  int mode;                   // 0: update U, 1: rebuild the panel from the current U only
  int skip_node;              // segments of this node write no panel entry (a boundary state
                              // without a head (sources) or tail (sinks); -1: none)
  int is_source;
  int accumulate;             // mode 0: add the measures to the pass totals instead of setting them
};

// ------------------------------------------------------------------------------------
// scalar helpers
// ------------------------------------------------------------------------------------

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2 for the one logarithm of every log-sum-exp output (and column sum).  The SFU's
// lg2.approx errs by about +4e-8 on average for arguments in [1, 2), where these sums mostly
// lie (the largest term contributes 1); a message passes through one such logarithm per time
// step, so over a horizon of T steps the bias adds up to about T * 3e-8 of relative flow error,
// the same sign at every step.  The libm-accurate log2f has no measurable mean error there.
__device__ __forceinline__ float log2_unbiased(float x) { return log2f(x); }

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no overflow).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Round to the q grid (exact scalings by powers of two).
__device__ __forceinline__ float quant(float x, const QScale &s) {
  return __fmul_rn(rintf(__fmul_rn(x, s.inv_q)), s.q);
}

// Mantissa-injected float of a stored lo: 2^23 + lo (exact).
__device__ __forceinline__ float lo_word0(uint32_t w) { return __uint_as_float((w & 0xffffu) | 0x4B000000u); }
__device__ __forceinline__ float lo_word1(uint32_t w) { return __uint_as_float((w >> 16) | 0x4B000000u); }

__device__ __forceinline__ lo_t lo_from_units(float li) {
  li = fminf(fmaxf(li, -32767.f), 32767.f);
  return (lo_t)((int)li + 32768);
}

// Stored form of the float-float value (h + l): hi on the q grid, lo in biased units.
__device__ __forceinline__ void encode(float h, float l, const QScale &s, float &hi, lo_t &lo) {
  if (h < kNegThresh) {
    hi = kNeg;
    lo = kLoZero;
    return;
  }
  float hq = quant(__fadd_rn(h, l), s);
  float rem = __fadd_rn(__fsub_rn(h, hq), l);         // h - hq is exact
  // h + l rounded to FP32 is h itself when l is below half an ulp of h, and h can sit exactly
  // halfway between two grid points: the grid point then chosen may be the far one for the
  // value h + l, leaving |rem| up to q/2 + ulp(h)/2, past the 16-bit range.  Moving one whole
  // quantum brings rem back to [-q/2, q/2] (both steps exact: q is a power of two, hq stays on
  // the grid and rem - q is a difference of numbers within a factor of two).
  if (rem > 0.5f * s.q) {
    hq = __fadd_rn(hq, s.q);
    rem = __fsub_rn(rem, s.q);
  } else if (rem < -0.5f * s.q) {
    hq = __fsub_rn(hq, s.q);
    rem = __fadd_rn(rem, s.q);
  }
  hi = hq;
  lo = lo_from_units(rintf(__fmul_rn(rem, s.lo_inv)));
}

// log-sum-exp result m + log2(acc), m on the q grid, in stored form.
__device__ __forceinline__ void lse_encode(float m, float acc, const QScale &s, float &hi, lo_t &lo) {
  if (m < kNegThresh || !(acc > 0.f)) {
    hi = kNeg;
    lo = kLoZero;
    return;
  }
  const float f = log2_unbiased(acc);
  const float fq = quant(f, s);
  hi = __fadd_rn(m, fq);                       // exact: both on the grid
  lo = lo_from_units(rintf(__fmul_rn(__fsub_rn(f, fq), s.lo_inv)));
}

}  // namespace ots

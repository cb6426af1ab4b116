// ots_step.cuh -- device helpers shared by the per-instance and the batched message kernels:
// packed panel loads and stores, deterministic block reductions, group reductions over the
// commodities of a node row, the batched log-sum-exp accumulation of Theorem 6 and the
// capacity update of Algorithm 2 (Corollary 7).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ots_device.cuh"

namespace ots {
namespace {

// 4 consecutive entries of a panel row: hi values and the packed biased lo words.
__device__ __forceinline__ void load4(const float *hp, const lo_t *lp, float h[4], uint32_t w[2]) {
  const float4 a = *reinterpret_cast<const float4 *>(hp);
  const uint2 b = *reinterpret_cast<const uint2 *>(lp);
  h[0] = a.x; h[1] = a.y; h[2] = a.z; h[3] = a.w;
  w[0] = b.x;
  w[1] = b.y;
}

// 2^23 + lo of entry q (0..3) of a packed pair of words.
__device__ __forceinline__ float lo_inj(const uint32_t w[2], int q) {
  return (q & 1) ? lo_word1(w[q >> 1]) : lo_word0(w[q >> 1]);
}

__device__ __forceinline__ void store4(float *hp, lo_t *lp, const float h[4], const lo_t l[4]) {
  *reinterpret_cast<float4 *>(hp) = make_float4(h[0], h[1], h[2], h[3]);
  uint2 b;
  b.x = (uint32_t)l[0] | ((uint32_t)l[1] << 16);
  b.y = (uint32_t)l[2] | ((uint32_t)l[3] << 16);
  *reinterpret_cast<uint2 *>(lp) = b;
}

// ---- float-float accumulation (value = x + y) ------------------------------------------------

// a += (bh + bl), renormalised (the pair stays non-overlapping).
__device__ __forceinline__ void ff_add(float2 &a, float bh, float bl) {
  float s, e;
  two_sum(a.x, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, bl));
  const float h = __fadd_rn(s, e);
  a.y = __fsub_rn(e, __fsub_rn(h, s));
  a.x = h;
}

// acc += c * u for float-float c and u (exact product of the hi parts via fma).
__device__ __forceinline__ void ff_mac(float2 &acc, float2 c, float2 u) {
  const float p = __fmul_rn(c.x, u.x);
  const float pe = fmaf(c.x, u.x, -p);
  ff_add(acc, p, __fadd_rn(pe, __fadd_rn(__fmul_rn(c.x, u.y), __fmul_rn(c.y, u.x))));
}

__device__ __forceinline__ float2 to_ff(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

__device__ __forceinline__ double from_ff(float2 v) { return (double)v.x + (double)v.y; }

// Butterfly sum of a float-float over the warp (fixed order; every lane ends with the total).
__device__ __forceinline__ float2 warp_sum_ff(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, v.x, o);
    const float l = __shfl_xor_sync(0xffffffffu, v.y, o);
    ff_add(v, h, l);
  }
  return v;
}

// Sum of two float-floats over the block (fixed order: warp shuffles, then warps in order).
__device__ __forceinline__ void block_sum2(float2 &v0, float2 &v1, float2 *s0, float2 *s1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v0 = warp_sum_ff(v0);
  v1 = warp_sum_ff(v1);
  __syncthreads();
  if (lane == 0) { s0[wid] = v0; s1[wid] = v1; }
  __syncthreads();
  v0 = s0[0];
  v1 = s1[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    ff_add(v0, s0[w].x, s0[w].y);
    ff_add(v1, s1[w].x, s1[w].y);
  }
}

// Sum of two doubles over the block (FP64; used once per launch, by the last block).
__device__ __forceinline__ void block_sum2_f64(double &v0, double &v1, double *s0, double *s1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  __syncthreads();
  if (lane == 0) { s0[wid] = v0; s1[wid] = v1; }
  __syncthreads();
  v0 = 0.0;
  v1 = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { v0 += s0[w]; v1 += s1[w]; }
}

// The FP64 sums (capacity residual, dual term) of a step: with a slot, every block writes its two
// totals there and the pass-end kernels add the slots of all steps in a fixed order (no grid-wide
// reduction at the end of each step); without one, the last block adds them to the pass statistics.
__device__ __forceinline__ void step_sums(double *slot, float2 v0, float2 v1, double *partials, unsigned int *counter,
                                          double *dst0, double *dst1);

// Deterministic grid reduction of two values: every block sums its threads' float-float
// values and writes the block total as FP64; the last block to finish reduces all partials in
// FP64 with a fixed assignment to threads and a fixed tree, then adds the totals to dst0 /
// dst1 (or assigns, when assign != 0) and resets the counter for the next kernel.
__device__ void block_sum2_last(float2 v0, float2 v1, double *partials, unsigned int *counter,
                                double *dst0, double *dst1, int assign) {
  __shared__ float2 f0[32], f1[32];   // one slot per warp of any block size up to 1024 threads
  __shared__ double s0[32], s1[32];
  __shared__ bool is_last;
  block_sum2(v0, v1, f0, f1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = from_ff(v0);
    partials[2 * blockIdx.x + 1] = from_ff(v1);
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
    a += __ldcg(partials + 2 * k);
    b += __ldcg(partials + 2 * k + 1);
  }
  block_sum2_f64(a, b, s0, s1);
  if (threadIdx.x == 0) {
    if (assign) { *dst0 = a; *dst1 = b; } else { *dst0 += a; *dst1 += b; }
    *counter = 0u;
  }
}

__device__ __forceinline__ void step_sums(double *slot, float2 v0, float2 v1, double *partials, unsigned int *counter,
                                          double *dst0, double *dst1) {
  if (!slot) {
    block_sum2_last(v0, v1, partials, counter, dst0, dst1, 0);
    return;
  }
  __shared__ float2 g0[32], g1[32];
  block_sum2(v0, v1, g0, g1);
  if (threadIdx.x == 0) {
    slot[2 * blockIdx.x] = from_ff(v0);
    slot[2 * blockIdx.x + 1] = from_ff(v1);
  }
}

// Group-wide (G threads) reductions of KB values at once.  For G <= 32 the group is a slice
// of one warp (shuffles only); for G > 32 the block is one node and the warps exchange their
// partial results through shared memory (sm holds G/32 x KB floats).
template <int G, int KB, bool MAX>
__device__ __forceinline__ void group_reduce(float (&x)[KB], float *sm) {
  if (G == 1) return;
  const unsigned lane = threadIdx.x & 31u;
  constexpr int W = G < 32 ? G : 32;
  const unsigned base = lane & ~(unsigned)(W - 1);
  const unsigned mask = (W >= 32) ? 0xffffffffu : (((1u << (W & 31)) - 1u) << base);
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const float y = __shfl_xor_sync(mask, x[k], o, 32);
      x[k] = MAX ? fmaxf(x[k], y) : x[k] + y;
    }
  }
  if (G > 32) {
    constexpr int NW = G / 32;
    const int wid = threadIdx.x >> 5;
    __syncthreads();                              // earlier readers of sm are done
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < KB; ++k) sm[k * NW + wid] = x[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      float r = sm[k * NW];
#pragma unroll
      for (int w = 1; w < NW; ++w) r = MAX ? fmaxf(r, sm[k * NW + w]) : r + sm[k * NW + w];
      x[k] = r;
    }
  }
}

// A log2 value as (hi on the q grid, remainder in lo units); the remainder is rounded to the
// units (|error| <= q / 2^17, the resolution of the stored messages).
__device__ __forceinline__ void split_units(float v, const QScale &qs, float &h, float &units) {
  h = quant(v, qs);
  units = rintf(__fmul_rn(__fsub_rn(v, h), qs.lo_inv));
}

// Bring a sum of up to three remainders back to [-32768, 32767] units, moving whole quanta
// into the hi part (exact: q is a power of two and h stays on its grid).
__device__ __forceinline__ void carry_units(float &u, float &h, float q) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (u > 32767.f) { u -= 65536.f; h += q; }
    if (u < -32768.f) { u += 65536.f; h -= q; }
  }
}

// Gather the thread's slice of up to KB input rows (row index nbr[j0 + k]).  With
// per-commodity costs the row of log2 K_L[., state] (same stored format) is added: hi sums are
// exact; the two remainders are added in signed units and re-biased (|sum| <= 2^16 units, one
// more unit of rounding when the sum leaves the int16 range is avoided by carrying into hi).
template <int G, int C, int KB, bool PC>
__device__ __forceinline__ void gather_rows(const StepArgs &a, int j0, int nb, int g, int (&st)[KB],
                                            float (&xh)[KB][C][4], uint32_t (&xw)[KB][C][2]) {
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    if (k < nb) {
      st[k] = a.state[j0 + k];
      const size_t row = (size_t)a.nbr[j0 + k] * a.Lp;
#pragma unroll
      for (int c = 0; c < C; ++c) load4(a.x_hi + row + 4 * (c * G + g), a.x_lo + row + 4 * (c * G + g), xh[k][c], xw[k][c]);
    } else {
      st[k] = 0;
#pragma unroll
      for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int q = 0; q < 4; ++q) xh[k][c][q] = kNeg;
        xw[k][c][0] = 0x80008000u;
        xw[k][c][1] = 0x80008000u;
      }
    }
  }
  if (PC) {
    const float q = a.qs.q;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      if (k < nb) {
        const size_t row = (size_t)st[k] * a.Lp;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          float ch[4];
          uint32_t cw[2];
          load4(a.klc_hi + row + 4 * (c * G + g), a.klc_lo + row + 4 * (c * G + g), ch, cw);
          float ucv[4] = {0.f, 0.f, 0.f, 0.f};
          if (a.uc_t) {
            const float4 u4 = *reinterpret_cast<const float4 *>(a.uc_t + row + 4 * (c * G + g));
            ucv[0] = u4.x; ucv[1] = u4.y; ucv[2] = u4.z; ucv[3] = u4.w;
          }
          lo_t nl[4];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            // signed remainders in units, exact; log2 U^(0,t) enters split on the same grid
            float uh, un;
            split_units(ucv[qq], a.qs, uh, un);
            float u = (lo_inj(xw[k][c], qq) - kLoBias) + (lo_inj(cw, qq) - kLoBias) + un;
            float h = xh[k][c][qq] + ch[qq] + uh;
            carry_units(u, h, q);
            xh[k][c][qq] = h;
            nl[qq] = (lo_t)((int)u + 32768);
          }
          xw[k][c][0] = (uint32_t)nl[0] | ((uint32_t)nl[1] << 16);
          xw[k][c][1] = (uint32_t)nl[2] | ((uint32_t)nl[3] << 16);
        }
      }
    }
  }
}

// Accumulate one batch of terms x[k] + w[k] into the running log-sum-exp (M, acc) of each
// commodity: hi sums are exact, batch maximum first, one ex2 per term.  Absent or unreachable
// terms have hi sums near -1e30 and vanish in ex2 without a branch.
template <int C, int KB>
__device__ __forceinline__ void aggregate_batch(const float (&xh)[KB][C][4], const uint32_t (&xw)[KB][C][2],
                                                const float (&wh)[KB], const float (&wl)[KB], float lo_unit,
                                                float (&M)[C][4], float (&acc)[C][4]) {
  float wlb[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) wlb[k] = wl[k] - kLoBias * lo_unit;
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float sv[KB];
      float m = 2.f * kNeg;
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        sv[k] = xh[k][c][q] + wh[k];
        m = fmaxf(m, sv[k]);
      }
      if (m < kNegThresh) continue;               // nothing reachable in this batch
      float sum = 0.f;
#pragma unroll
      for (int k = 0; k < KB; ++k) sum += ex2(fmaf(lo_inj(xw[k][c], q), lo_unit, (sv[k] - m) + wlb[k]));
      const float Mo = M[c][q];
      if (m > Mo) {
        acc[c][q] = fmaf(acc[c][q], ex2(Mo - m), sum);
        M[c][q] = m;
      } else {
        acc[c][q] = fmaf(sum, ex2(m - Mo), acc[c][q]);
      }
    }
}

// Merge two (max, scaled-sum) pairs of a log-sum-exp: value = m + log2(s).
__device__ __forceinline__ void lse_merge(float &m, float &s, float om, float os) {
  if (om > m) {
    s = fmaf(s, ex2(m - om), os);
    m = om;
  } else {
    s = fmaf(os, ex2(om - m), s);
  }
}

// W = log2 K_L + log2 u as (hi on the q grid, float lo).
__device__ __forceinline__ void make_w(float kl_hi, float kl_lo, float lu_hi, float lu_lo, const QScale &qs,
                                       float &w_hi, float &w_lo) {
  if (lu_hi < kNegThresh || kl_hi < kNegThresh) {   // u = 0, or the state is closed in this interval
    w_hi = kNeg;
    w_lo = 0.f;
    return;
  }
  float s, e;
  two_sum(kl_hi, lu_hi, s, e);
  e += kl_lo + lu_lo;
  w_hi = quant(s, qs);
  w_lo = (s - w_hi) + e;
}

// Adds |P_new - P_old| of one state's capacity update to viol, where P = 2^(log2 u + col) is the
// state's flow under the old and the new u_t: the excess (P_old - d)_+ where the update lowers
// u_t, and the flow a too small u_t withheld where it raises u_t (a warm start can begin below
// the fixed point, where the excess alone reads zero).  Evaluated as P_old |2^delta - 1| with
// delta = log2 u_new - log2 u_old formed in float-float (its terms cancel near convergence);
// 2^delta - 1 from exp2 for |delta| > 0.5, else from the Taylor series of exp(x) - 1 at
// x = delta ln 2 (|x| <= 0.35, truncation below 2e-7 relative).  A state that closes or
// reopens moves all of its flow.
__device__ __forceinline__ void add_residual(float2 lu_old, float2 lu_new, float col_hi, float col_lo, float &viol) {
  const bool c_old = lu_old.x < kNegThresh, c_new = lu_new.x < kNegThresh;
  if (c_old && c_new) return;
  if (c_old || c_new) {
    const float2 lu = c_old ? lu_new : lu_old;
    viol += ex2(fminf((lu.x + col_hi) + (lu.y + col_lo), 126.f));
    return;
  }
  float s, e;
  two_sum(lu_new.x, -lu_old.x, s, e);
  const float dl = __fadd_rn(s, __fadd_rn(e, __fsub_rn(lu_new.y, lu_old.y)));
  if (dl == 0.f) return;
  float r;
  if (fabsf(dl) > 0.5f) {
    r = fabsf(ex2(fminf(dl, 126.f)) - 1.f);
  } else {
    const float x = dl * 0.69314718f;
    r = fabsf(x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.f / 720.f, 1.f / 120.f), 1.f / 24.f), 1.f / 6.f), 0.5f), 1.f));
  }
  const float p_old = ex2(fminf((lu_old.x + col_hi) + (lu_old.y + col_lo), 126.f));
  viol += fminf(p_old * r, 1e30f);                // huge residuals stay finite (reported, not NaN)
}

// Capacity update of one state from its column log-sum-exp (cm + log2 cs) (Algorithm 2,
// Corollary 7): W_t for the aggregation and, when `write`, the stored log2 u_t, W_t, the
// excess (P_t - d)_+ with the old u_t (viol) and the dual term d log2 u_t (Theorem 3; dual,
// float-float).  In flows mode (a.mode == 1) W_t is read back and, when `write`, P_t is
// stored.
template <bool PC>
__device__ __forceinline__ void update_state(const StepArgs &a, int sk, float cm, float cs, bool write, float &w_hi,
                                             float &w_lo, float &viol, float2 &dual) {
  if (a.fixed_w && a.fixed_w[sk]) {              // a storage state: updated by its own kernel
    w_hi = a.w_hi_t[sk];
    w_lo = a.w_lo_t[sk];
    return;
  }
  float col_hi = kNeg, col_lo = 0.f;
  if (cm > kNegThresh && cs > 0.f) two_sum(cm, log2_unbiased(cs), col_hi, col_lo);  // log2 (hatPsi .* Psi (.* K_L))^T 1
  const float klh = PC ? 0.f : ldexpf(a.kl_hi[sk], -a.kl_shift), kll = PC ? 0.f : ldexpf(a.kl_lo[sk], -a.kl_shift);
  if (!PC && col_hi > kNegThresh) {
    float s, e;
    two_sum(col_hi, klh, s, e);
    col_hi = s;
    col_lo += e + kll;
  }
  if (a.mode != 0) {
    w_hi = a.w_hi_t[sk];
    w_lo = a.w_lo_t[sk];
    if (write) {
      const float2 lu = a.lu_t[sk];
      a.flow_t[sk] = col_hi > kNegThresh && w_hi > kNegThresh
                         ? exp2((double)lu.x + (double)lu.y + (double)col_hi + (double)col_lo) : 0.0;
    }
    return;
  }
  const float2 cap = a.cap[sk];
  const bool fin = cap.x < INFINITY;
  float lu_hi = 0.f, lu_lo = 0.f;
  if (fin && col_hi > kNegThresh) {
    if (a.logd_hi[sk] < kNegThresh) {
      lu_hi = kNeg;                                // d = 0: the state is closed
    } else {
      // log2 u = min(log2 d - col, 0) in float-float
      float s1, e1, s2, e2;
      two_sum(a.logd_hi[sk], -col_hi, s1, e1);
      e1 += a.logd_lo[sk] - col_lo;
      two_sum(s1, e1, s2, e2);
      if (s2 < 0.f) { lu_hi = s2; lu_lo = e2; }
    }
  }
  make_w(klh, kll, lu_hi, lu_lo, a.qs, w_hi, w_lo);
  if (!write) return;
  const float2 lu_old = a.lu_t[sk];
  const float2 lu_new = lu_hi < kNegThresh ? make_float2(kNeg, 0.f) : make_float2(lu_hi, lu_lo);
  if (col_hi > kNegThresh && fin) add_residual(lu_old, lu_new, col_hi, col_lo, viol);
  if (col_hi != col_hi || col_lo != col_lo) viol = __int_as_float(0x7fc00000);   // NaN: reported
  if (fin && cap.x > 0.f && lu_new.x > kNegThresh) ff_mac(dual, cap, lu_new);
  a.lu_t[sk] = lu_new;
  a.w_hi_t[sk] = w_hi;
  a.w_lo_t[sk] = w_lo;
}

// One (node, commodity) segment of boundary triples (Algorithm 2, source and sink updates):
// in mode 0, U <- R ./ message (log2: log2 U = log2 R - msg) with the mismatch before the
// update (sources: r0 += |U msg - R|), <R, log2 U> (r1), the mass <K, U> after a sink update
// (r0) and a count of vanishing messages (r2); in both modes the segment's entry of the
// boundary panel is rebuilt as log2 sum_q U_q.  FP64 throughout.
__device__ __forceinline__ void boundary_segment(const BndArgs &b, int sidx, double &r0, double &r1, double &r2) {
  const int l = b.seg_l[sidx];
  const int q0 = b.seg_ptr[sidx], q1 = b.seg_ptr[sidx + 1];
  double m = -INFINITY;
  for (int q = q0; q < q1; ++q) {
    double lu = b.tri_logU[q];
    if (b.mode == 0) {
      const size_t idx = (size_t)b.tri_node_other[q] * b.Lp + l;
      const double msg = (double)b.msg_hi[idx] + ((double)b.msg_lo[idx] - 32768.0) * (double)b.qs.lo_unit;
      // mismatch before the update; a term is capped at 1e30 so that the far-from-feasible first
      // passes (messages of 2^1000 and more at large epsilon) give a huge finite measure
      if (b.is_source) r0 += fmin(fabs(exp2(fmin(lu + msg, 1000.0)) - b.tri_R[q]), 1e30);
      if (b.msg_hi[idx] < kNegThresh) r2 += 1.0;                   // vanishing message
      lu = b.tri_logR[q] - msg;
      b.tri_logU[q] = lu;
      r1 += b.tri_R[q] * lu;                                       // <R, log2 U>
      if (!b.is_source) r0 += exp2(lu + msg);                      // <K, U> after the update
    }
    m = fmax(m, lu);
  }
  double sum = 0.0;
  for (int q = q0; q < q1; ++q) sum += exp2(b.tri_logU[q] - m);
  if (!b.out_hi || b.seg_node[sidx] == b.skip_node) return;
  const double r = m + log2(sum);
  const float h = (float)r;
  float oh;
  lo_t ol;
  encode(h, (float)(r - (double)h), b.qs, oh, ol);
  const size_t o = (size_t)b.seg_node[sidx] * b.Lp + l;
  b.out_hi[o] = oh;
  b.out_lo[o] = ol;
}

// Capacity update of one in-state from its column log-sum-exp (cm + log2 cs), FP32 part:
// the column sum col = log2 (hatPsi_t .* Psi_t .* K_L)^T 1 as a float-float (col_hi, col_lo),
// the new log2 u_t = min(log2 d - col, 0) as a float-float (lu_hi, lu_lo; cap_finite = 0 for
// d = inf), and W_t = log2 K_L + log2 u_t (w_hi, w_lo).  In flows mode (mode != 0) W_t is the
// stored win and u_t is not changed.
__device__ __forceinline__ void update_w(int mode, const QScale &qs, float cm, float cs, float klh, float kll,
                                         float ldh, float ldl, bool cap_finite, float win_hi, float win_lo,
                                         float &w_hi, float &w_lo, float &col_hi, float &col_lo, float &lu_hi,
                                         float &lu_lo) {
  col_hi = kNeg;
  col_lo = 0.f;
  if (cm > kNegThresh && cs > 0.f) two_sum(cm, log2_unbiased(cs), col_hi, col_lo);
  if (col_hi > kNegThresh) {
    float s, e;
    two_sum(col_hi, klh, s, e);
    col_hi = s;
    col_lo += e + kll;
  }
  lu_hi = 0.f;
  lu_lo = 0.f;
  if (mode != 0) {
    w_hi = win_hi;
    w_lo = win_lo;
    return;
  }
  if (cap_finite && col_hi > kNegThresh) {
    if (ldh < kNegThresh) {
      lu_hi = kNeg;
    } else {
      float s1, e1, s2, e2;
      two_sum(ldh, -col_hi, s1, e1);
      e1 += ldl - col_lo;
      two_sum(s1, e1, s2, e2);
      if (s2 < 0.f) { lu_hi = s2; lu_lo = e2; }
    }
  }
  make_w(klh, kll, lu_hi, lu_lo, qs, w_hi, w_lo);
}

// Per-state part of the same update (one thread per state): the new log2 u_t, the flow P_t
// in flows mode (FP64: once per solve), the excess (P_t - d)_+ with the old u_t (viol) and the
// dual term d log2 u_t of Theorem 3 (dual, float-float).
__device__ __forceinline__ void update_stats(int mode, float col_hi, float col_lo, float lu_hi, float lu_lo, float ldh,
                                             float ldl, float w_hi, float2 cap, float2 lu_old, float2 &lu_new,
                                             double &flow, float &viol, float2 &dual) {
  if (mode != 0) {
    flow = col_hi > kNegThresh && w_hi > kNegThresh
               ? exp2((double)lu_old.x + (double)lu_old.y + (double)col_hi + (double)col_lo) : 0.0;
    lu_new = lu_old;
    return;
  }
  const bool fin = cap.x < INFINITY;
  lu_new = lu_hi < kNegThresh ? make_float2(kNeg, 0.f) : make_float2(lu_hi, lu_lo);
  if (col_hi > kNegThresh && fin) add_residual(lu_old, lu_new, col_hi, col_lo, viol);
  if (col_hi != col_hi || col_lo != col_lo) viol = __int_as_float(0x7fc00000);
  if (fin && cap.x > 0.f && lu_new.x > kNegThresh) ff_mac(dual, cap, lu_new);
}

// Both parts at once (same arithmetic as update_state, with the per-state inputs loaded
// ahead by the caller).
__device__ __forceinline__ void update_meta(int mode, const QScale &qs, float cm, float cs, float klh, float kll,
                                            float ldh, float ldl, float2 cap, float2 lu_old, float win_hi,
                                            float win_lo, float &w_hi, float &w_lo, float2 &lu_new, double &flow,
                                            float &viol, float2 &dual) {
  float col_hi, col_lo, lu_hi, lu_lo;
  update_w(mode, qs, cm, cs, klh, kll, ldh, ldl, cap.x < INFINITY, win_hi, win_lo, w_hi, w_lo, col_hi, col_lo, lu_hi,
           lu_lo);
  update_stats(mode, col_hi, col_lo, lu_hi, lu_lo, ldh, ldl, w_hi, cap, lu_old, lu_new, flow, viol, dual);
}

}  // namespace

}  // namespace ots

// ots_kernels.cu -- sm_103a kernels of the Sinkhorn iterations of Algorithm 2.
//
// Node-level form of the message products.  The transition kernel of the state graph is
// the line graph, K_ij = 1 iff head(i) == tail(j) (Section 3.1), so K = B_in B_out with
// B_in[i, v] = [head(i) = v] and B_out[v, j] = [tail(j) = v].  Every forward message
// hatPsi_{t+1}[l, j] therefore depends on j only through tail(j), and every backward
// message Psi_{t-1}[l, i] only through head(i).  The kernels keep one row per NODE:
//     A_t[v][l] = hatPsi_{t+1}[l, j] for any j leaving v       (t = 1..T-1)
//     B_t[v][l] = Psi_{t-1}[l, i]  for any i entering v        (t = 2..T)
// and compute (eq. psi_hat, eq. psi of Theorem 6)
//     A_t[v] = LSE_{j: head(j) = v} (A_{t-1}[tail j] + log2 K_L[j] + log2 u_t[j])
//     B_t[v] = LSE_{j: tail(j) = v} (B_{t+1}[head j] + log2 K_L[j] + log2 u_t[j])
// with one term per state instead of one per line-graph transition.  The capacity update
// of Algorithm 2 (u_t <- min(d ./ ((hatPsi_t .* Psi_t .* K_L)^T 1), 1), with K_L as in
// Corollary 7) needs, for state j = (y -> v), the column sum over commodities of
//     hatPsi_t[l, j] Psi_t[l, j] K_L[l, j] = A_{t-1}[y][l] B_{t+1}[v][l] K_L[l, j],
// which the forward kernel of node v evaluates for all its in-states before forming A_t[v].
//
// Thread mapping: G threads cooperate on one node row; thread g owns commodities
// 4 (c G + g) + k, k < 4, c < C (float4 / 4 x half loads, coalesced along the row).
// Column sums over commodities are warp-shuffle (and, for G > 32, shared-memory)
// log-sum-exp reductions.  Everything is FP32 float-float; reductions that decide
// convergence are FP64 and deterministic (per-block partials summed by the last block in
// block order).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ots_device.cuh"

namespace ots {

namespace {

__device__ __forceinline__ void load4(const float *hp, const __half *lp, float h[4], float l[4]) {
  float4 a = *reinterpret_cast<const float4 *>(hp);
  uint2 b = *reinterpret_cast<const uint2 *>(lp);
  h[0] = a.x; h[1] = a.y; h[2] = a.z; h[3] = a.w;
  __half2 b0 = *reinterpret_cast<__half2 *>(&b.x);
  __half2 b1 = *reinterpret_cast<__half2 *>(&b.y);
  float2 f0 = __half22float2(b0), f1 = __half22float2(b1);
  l[0] = f0.x; l[1] = f0.y; l[2] = f1.x; l[3] = f1.y;
}

__device__ __forceinline__ void store4(float *hp, __half *lp, const float h[4], const float l[4]) {
  float hh[4], ll[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    hh[k] = h[k] < kNegThresh ? kNeg : h[k];
    ll[k] = h[k] < kNegThresh ? 0.f : l[k];
  }
  *reinterpret_cast<float4 *>(hp) = make_float4(hh[0], hh[1], hh[2], hh[3]);
  __half2 b0 = __floats2half2_rn(ll[0], ll[1]);
  __half2 b1 = __floats2half2_rn(ll[2], ll[3]);
  uint2 b;
  b.x = *reinterpret_cast<unsigned int *>(&b0);
  b.y = *reinterpret_cast<unsigned int *>(&b1);
  *reinterpret_cast<uint2 *>(lp) = b;
}

// Sum of two doubles over the block (fixed order: warp shuffles, then warps in order).
__device__ __forceinline__ void block_sum2(double &v0, double &v1, double *s0, double *s1) {
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

// Deterministic FP64 grid reduction of two values: every block writes its partial sums, the
// last block to finish reduces all partials with a fixed assignment to threads and a fixed
// tree, then adds the totals to dst0 / dst1 (or assigns, when assign != 0) and resets the
// counter for the next kernel.
__device__ void block_sum2_last(double v0, double v1, double *partials, unsigned int *counter,
                                double *dst0, double *dst1, int assign) {
  __shared__ double s0[kBlock / 32], s1[kBlock / 32];
  __shared__ bool is_last;
  block_sum2(v0, v1, s0, s1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = v0;
    partials[2 * blockIdx.x + 1] = v1;
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
  block_sum2(a, b, s0, s1);
  if (threadIdx.x == 0) {
    if (assign) { *dst0 = a; *dst1 = b; } else { *dst0 += a; *dst1 += b; }
    *counter = 0u;
  }
}

// Group-wide (G threads) reductions of KB values at once.  For G <= 32 the group is a slice
// of one warp (shuffles only); for G > 32 the block is one node and the warps exchange their
// partial results through shared memory (sm holds BS/32 x KB floats).
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

// Gather the thread's slice of up to KB input rows (row index nbr[j0 + k]) and, with
// per-commodity costs, fold log2 K_L[., state] into them.
template <int G, int C, int KB, bool PC>
__device__ __forceinline__ void gather_rows(const StepArgs &a, int j0, int nb, int g, int (&st)[KB],
                                            float (&xh)[KB][C][4], float (&xl)[KB][C][4]) {
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    if (k < nb) {
      st[k] = a.state[j0 + k];
      const size_t row = (size_t)a.nbr[j0 + k] * a.Lp;
#pragma unroll
      for (int c = 0; c < C; ++c) load4(a.x_hi + row + 4 * (c * G + g), a.x_lo + row + 4 * (c * G + g), xh[k][c], xl[k][c]);
    } else {
      st[k] = 0;
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) { xh[k][c][q] = kNeg; xl[k][c][q] = 0.f; }
    }
  }
  if (PC) {
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      if (k < nb) {
        const size_t row = (size_t)st[k] * a.Lp;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          float ch[4], cl[4];
          load4(a.klc_hi + row + 4 * (c * G + g), a.klc_lo + row + 4 * (c * G + g), ch, cl);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float s, e;
            two_sum(xh[k][c][q], ch[q], s, e);
            xh[k][c][q] = s;
            xl[k][c][q] += e + cl[q];
          }
        }
      }
    }
  }
}

// Accumulate one batch of terms x[k] + w[k] into the running log-sum-exp (M, acc) of each
// commodity: exact float-float terms, batch maximum first, one ex2 per term.
template <int C, int KB>
__device__ __forceinline__ void aggregate_batch(int nb, float (&xh)[KB][C][4], const float (&xl)[KB][C][4],
                                                const float (&wh)[KB], const float (&wl)[KB], float (&M)[C][4],
                                                float (&acc)[C][4]) {
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float sv[KB], ev[KB];
      float m = 2.f * kNeg;
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        float s, e;
        two_sum(xh[k][c][q], wh[k], s, e);
        sv[k] = s;
        ev[k] = e + (xl[k][c][q] + wl[k]);
        if (k < nb) m = fmaxf(m, s);
      }
      if (m < kNegThresh) continue;               // nothing reachable in this batch
      float sum = 0.f;
#pragma unroll
      for (int k = 0; k < KB; ++k)
        if (k < nb && sv[k] > kNegThresh) sum += ex2((sv[k] - m) + ev[k]);
      // merge (m, sum) into (M, acc)
      const float Mo = M[c][q];
      if (m > Mo) {
        acc[c][q] = fmaf(acc[c][q], ex2(Mo - m), sum);
        M[c][q] = m;
      } else {
        acc[c][q] = fmaf(sum, ex2(m - Mo), acc[c][q]);
      }
    }
}

}  // namespace

// ------------------------------------------------------------------------------------
// forward step t (t = 2..T-1): capacity update of every state entering v, then A_t[v]
//
// W_t[j] is log2 K_L[j] + log2 u_t[j] when the rows of C_L are shared by all commodities,
// and log2 u_t[j] alone when a per-commodity K_L panel (klc) is given.
// ------------------------------------------------------------------------------------
template <int G>
struct BlockOf { static constexpr int value = G > 32 ? G : kBlock; };

constexpr int kBatch = 4;   // in-states gathered per batch

template <int G, int C, bool PC>
__global__ void __launch_bounds__(BlockOf<G>::value, 2 * 256 / BlockOf<G>::value) k_forward(const StepArgs a) {
  constexpr int BS = BlockOf<G>::value;
  constexpr int NPB = BS / G;  // nodes per block (1 when G > 32)
  constexpr int KB = kBatch;
  __shared__ float sm[(BS / 32 > 0 ? BS / 32 : 1) * KB];
  const int g = threadIdx.x % G;
  const int v = blockIdx.x * NPB + threadIdx.x / G;
  const bool active = v < a.V;
  const size_t rowv = (size_t)(active ? v : 0) * a.Lp;

  float bh[C][4], bl[C][4];
#pragma unroll
  for (int c = 0; c < C; ++c) load4(a.y_hi + rowv + 4 * (c * G + g), a.y_lo + rowv + 4 * (c * G + g), bh[c], bl[c]);

  float M[C][4], acc[C][4];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) { M[c][q] = 2.f * kNeg; acc[c][q] = 0.f; }

  double viol = 0.0, dual = 0.0;
  const int jb = active ? a.ptr[v] : 0;
  const int je = active ? a.ptr[v + 1] : 0;
  // G > 32: the block is one node, so trip counts are uniform across the block.
  for (int j0 = jb; j0 < je; j0 += KB) {
    const int nb = min(KB, je - j0);
    int st[KB];
    float xh[KB][C][4], xl[KB][C][4];
    gather_rows<G, C, KB, PC>(a, j0, nb, g, st, xh, xl);

    // (1) column log-sum-exp over commodities of A_{t-1}[y] (+ K_L) + B_{t+1}[v], for each
    //     in-state of the batch: group maximum of the rounded sums, then group sum.
    float cm[KB], cs[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      float m = 2.f * kNeg;
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) m = fmaxf(m, __fadd_rn(xh[k][c][q], bh[c][q]));
      cm[k] = m;
    }
    group_reduce<G, KB, true>(cm, sm);
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      float sum = 0.f;
      if (cm[k] > kNegThresh) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float s, e;
            two_sum(xh[k][c][q], bh[c][q], s, e);
            if (s > kNegThresh) sum += ex2((s - cm[k]) + (e + (xl[k][c][q] + bl[c][q])));
          }
      }
      cs[k] = sum;
    }
    group_reduce<G, KB, false>(cs, sm);

    // (2) capacity update of each in-state (Algorithm 2), or flows of the current iterate
    float wh[KB], wl[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      wh[k] = kNeg;
      wl[k] = 0.f;
      if (k >= nb) continue;
      const int sk = st[k];
      float col_hi, col_lo;
      lse_finish(cm[k], cs[k], col_hi, col_lo);   // log2 of (hatPsi_t .* Psi_t (.* K_L))^T 1
      const float klh = PC ? 0.f : a.kl_hi[sk], kll = PC ? 0.f : a.kl_lo[sk];
      if (!PC && col_hi > kNegThresh) {
        float s, e;
        two_sum(col_hi, klh, s, e);
        col_hi = s;
        col_lo += e + kll;
      }
      if (a.mode == 0) {
        const double cap = a.cap[sk];
        float lu_hi = 0.f, lu_lo = 0.f;
        if (isfinite(cap) && col_hi > kNegThresh) {
          if (a.logd_hi[sk] < kNegThresh) {
            lu_hi = kNeg;                            // d = 0: the state is closed
          } else {
            // log2 u = min(log2 d - col, 0) in float-float
            float s1, e1, s2, e2;
            two_sum(a.logd_hi[sk], -col_hi, s1, e1);
            e1 += a.logd_lo[sk] - col_lo;
            two_sum(s1, e1, s2, e2);
            if (s2 < 0.f) { lu_hi = s2; lu_lo = e2; }
          }
        }
        if (lu_hi > kNegThresh) {
          two_sum(klh, lu_hi, wh[k], wl[k]);
          wl[k] += kll + lu_lo;
        }
        if (g == 0) {
          const double lu_old = a.logu_t[sk];
          if (col_hi > kNegThresh && isfinite(cap)) {
            // excess (P_t - d)_+ with the old u_t; exact FP64 only near or above capacity
            const float q = (float)lu_old + col_hi - a.logd_hi[sk];
            if (q > -1e-3f) {
              const double p_old = exp2(lu_old + (double)col_hi + (double)col_lo);
              if (p_old > cap) viol += p_old - cap;
            }
          }
          if (col_hi != col_hi || col_lo != col_lo) viol = __longlong_as_double(0x7ff8000000000000LL);  // NaN
          const double lu_new = lu_hi < kNegThresh ? -1e30 : (double)lu_hi + (double)lu_lo;
          if (isfinite(cap) && cap > 0.0) dual += cap * lu_new;
          a.logu_t[sk] = lu_new;
          a.w_hi_t[sk] = wh[k];
          a.w_lo_t[sk] = wl[k];
        }
      } else {
        wh[k] = a.w_hi_t[sk];
        wl[k] = a.w_lo_t[sk];
        if (g == 0)
          a.flow_t[sk] = col_hi > kNegThresh && wh[k] > kNegThresh
                             ? exp2(a.logu_t[sk] + (double)col_hi + (double)col_lo) : 0.0;
      }
    }

    // (3) A_t[v] accumulates A_{t-1}[y] + W_t[state] over the batch
    aggregate_batch<C, KB>(nb, xh, xl, wh, wl, M, acc);
  }

  if (active) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float oh[4], ol[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) lse_finish(M[c][q], acc[c][q], oh[q], ol[q]);
      store4(a.out_hi + rowv + 4 * (c * G + g), a.out_lo + rowv + 4 * (c * G + g), oh, ol);
    }
  }
  if (a.mode == 0) block_sum2_last(viol, dual, a.partials, a.counter, &a.stats->cap_viol, &a.stats->dual_cap, 0);
}

// ------------------------------------------------------------------------------------
// backward step t (t = T-1..2): B_t[v] = LSE_{j: tail j = v} (B_{t+1}[head j] + W_t[j] (+ K_L))
// ------------------------------------------------------------------------------------
template <int G, int C, bool PC>
__global__ void __launch_bounds__(BlockOf<G>::value, 3 * 256 / BlockOf<G>::value) k_backward(const StepArgs a) {
  constexpr int BS = BlockOf<G>::value;
  constexpr int NPB = BS / G;
  constexpr int KB = kBatch;
  const int g = threadIdx.x % G;
  const int v = blockIdx.x * NPB + threadIdx.x / G;
  if (v >= a.V) return;
  float M[C][4], acc[C][4];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) { M[c][q] = 2.f * kNeg; acc[c][q] = 0.f; }
  const int jb = a.ptr[v], je = a.ptr[v + 1];
  for (int j0 = jb; j0 < je; j0 += KB) {
    const int nb = min(KB, je - j0);
    int st[KB];
    float xh[KB][C][4], xl[KB][C][4];
    gather_rows<G, C, KB, PC>(a, j0, nb, g, st, xh, xl);
    float wh[KB], wl[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      wh[k] = k < nb ? a.w_hi_t[st[k]] : kNeg;
      wl[k] = k < nb ? a.w_lo_t[st[k]] : 0.f;
    }
    aggregate_batch<C, KB>(nb, xh, xl, wh, wl, M, acc);
  }
  const size_t rowo = (size_t)v * a.Lp;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float oh[4], ol[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) lse_finish(M[c][q], acc[c][q], oh[q], ol[q]);
    store4(a.out_hi + rowo + 4 * (c * G + g), a.out_lo + rowo + 4 * (c * G + g), oh, ol);
  }
}

// ------------------------------------------------------------------------------------
// boundary updates: U01 <- R01 ./ Psi_1 (sources), U0T <- R0T ./ hatPsi_T (sinks), and the
// boundary panels A_1 = (U01 K) by tail node, B_T = (U0T K^T) by head node.
// One thread per (node, commodity) segment of triples.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_boundary(const BndArgs b) {
  const int sidx = blockIdx.x * blockDim.x + threadIdx.x;
  double r0 = 0.0, r1 = 0.0, r2 = 0.0;
  if (sidx < b.n_seg) {
    const int l = b.seg_l[sidx];
    float m = 2.f * kNeg, acc = 0.f;
    for (int q = b.seg_ptr[sidx]; q < b.seg_ptr[sidx + 1]; ++q) {
      const size_t idx = (size_t)b.tri_node_other[q] * b.Lp + l;
      const double msg = (double)b.msg_hi[idx] + (double)__half2float(b.msg_lo[idx]);
      double lu = b.tri_logU[q];
      if (b.mode == 0) {
        if (b.is_source) r0 += fabs(exp2(lu + msg) - b.tri_R[q]);   // mismatch before the update
        if (b.msg_hi[idx] < kNegThresh) r2 += 1.0;                   // vanishing message
        lu = b.tri_logR[q] - msg;
        b.tri_logU[q] = lu;
        r1 += b.tri_R[q] * lu;                                       // <R, log2 U>
        if (!b.is_source) r0 += exp2(lu + msg);                      // <K, U> after the update
      }
      // segment log-sum-exp of log2 U in float-float
      const float hi = (float)lu;
      const float lo = (float)(lu - (double)hi);
      lse_push(m, acc, hi, lo);
    }
    float oh, ol;
    lse_finish(m, acc, oh, ol);
    const size_t o = (size_t)b.seg_node[sidx] * b.Lp + l;
    store_pair(b.out_hi + o, b.out_lo + o, oh, ol);
  }
  if (b.mode == 0) {
    // three sums through two reductions: (r0, r1) then r2 folded into stats->bad
    if (b.is_source) {
      block_sum2_last(r0, r1, b.partials, b.counter, &b.stats->src_resid, &b.stats->dual_src, 1);
    } else {
      block_sum2_last(r0, r1, b.partials, b.counter, &b.stats->mass_snk, &b.stats->dual_snk, 1);
    }
    if (r2 > 0.0) atomicAdd(&b.stats->bad, r2);
  }
}

// Start of a pass: clear the accumulators the forward sweep adds into.
__global__ void k_pass_begin(DevStats *st) {
  st->cap_viol = 0.0;
  st->dual_cap = 0.0;
  st->bad = 0.0;
}

// End of a pass: relative measures and the dual objective of Theorem 3 in natural units:
//   -eps <K,U> + eps ln2 (<R01, log2 U01> + <R0T, log2 U0T> + sum_t <d, log2 u_t>).
__global__ void k_pass_end(const DevStats *st, PassReport *rep, double mass, double eps) {
  rep->src_resid_rel = st->src_resid / mass;
  rep->cap_viol_rel = st->cap_viol / mass;
  rep->dual_objective = -eps * st->mass_snk + eps * 0.69314718055994530942 * (st->dual_src + st->dual_snk + st->dual_cap);
  rep->bad = st->bad;
  rep->passes += 1;
}

// Initial duals: log2 u_t = 0 and W_t = log2 K_L for t = 2..T-1.
__global__ void k_init_weights(int S, int T, const float *kl_hi, const float *kl_lo, double *logu,
                               float *w_hi, float *w_lo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  for (int t = 2; t <= T - 1; ++t) {
    logu[(size_t)t * S + s] = 0.0;
    w_hi[(size_t)t * S + s] = kl_hi ? kl_hi[s] : 0.f;
    w_lo[(size_t)t * S + s] = kl_lo ? kl_lo[s] : 0.f;
  }
}

// W_t = log2 K_L + log2 u_t from given log2 u (after ots_set_duals).
__global__ void k_weights_from_logu(int S, int T, const float *kl_hi, const float *kl_lo, const double *logu,
                                    float *w_hi, float *w_lo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  for (int t = 2; t <= T - 1; ++t) {
    const double lu = logu[(size_t)t * S + s];
    float luh = (float)lu;
    float lul = (float)(lu - (double)luh);
    if (lu < -1e29) { w_hi[(size_t)t * S + s] = kNeg; w_lo[(size_t)t * S + s] = 0.f; continue; }
    float hi, lo;
    two_sum(kl_hi ? kl_hi[s] : 0.f, luh, hi, lo);
    lo += (kl_lo ? kl_lo[s] : 0.f) + lul;
    w_hi[(size_t)t * S + s] = hi;
    w_lo[(size_t)t * S + s] = lo;
  }
}

__global__ void k_fill_panel(size_t n, float *hi, __half *lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    hi[i] = kNeg;
    lo[i] = __float2half_rn(0.f);
  }
}

// Per-commodity flows P_{0,t}[l, j] = 2^(A_{t-1}[tail j][l] + B_{t+1}[head j][l] + log2 K_L + log2 u_t)
// for commodities [l0, l1), all states j; out[(l - l0) * S + j].
__global__ void k_commodity_flows(int S, int Lp, int l0, int l1, const int *tail, const int *head,
                                  const float *a_hi, const __half *a_lo, const float *b_hi, const __half *b_lo,
                                  const float *kl_hi, const float *kl_lo, const float *klc_hi, const __half *klc_lo,
                                  const double *logu_t, double *out) {
  const size_t n = (size_t)S * (l1 - l0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % S);
    const int l = l0 + (int)(i / S);
    const size_t ia = (size_t)tail[j] * Lp + l, ib = (size_t)head[j] * Lp + l;
    const float ah = a_hi[ia], bh = b_hi[ib];
    if (ah < kNegThresh || bh < kNegThresh) { out[i] = 0.0; continue; }
    double x = (double)ah + (double)__half2float(a_lo[ia]) + (double)bh + (double)__half2float(b_lo[ib]) + logu_t[j];
    if (klc_hi) x += (double)klc_hi[(size_t)j * Lp + l] + (double)__half2float(klc_lo[(size_t)j * Lp + l]);
    else x += (double)kl_hi[j] + (double)kl_lo[j];
    out[i] = exp2(x);
  }
}

// Boundary flows of one triple list: P = 2^(log2 U + msg) per triple (t = 1 or t = T).
__global__ void k_boundary_flows(int n, int Lp, const int *tri_l, const int *tri_node_other, const double *tri_logU,
                                 const float *msg_hi, const __half *msg_lo, double *out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const size_t idx = (size_t)tri_node_other[q] * Lp + tri_l[q];
  if (msg_hi[idx] < kNegThresh) { out[q] = 0.0; return; }
  const double msg = (double)msg_hi[idx] + (double)__half2float(msg_lo[idx]);
  out[q] = exp2(tri_logU[q] + msg);
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------

int nodes_per_block(int G) { return (G > 32 ? G : kBlock) / G; }

template <bool FWD, int G, int C, bool PC>
static cudaError_t launch_step_t(const StepArgs &a, cudaStream_t s) {
  constexpr int BS = BlockOf<G>::value;
  const int npb = BS / G;
  const int grid = (a.V + npb - 1) / npb;
  if (FWD) k_forward<G, C, PC><<<grid, BS, 0, s>>>(a);
  else k_backward<G, C, PC><<<grid, BS, 0, s>>>(a);
  return cudaGetLastError();
}

template <bool FWD, bool PC>
static cudaError_t launch_step_g(int G, int C, const StepArgs &a, cudaStream_t s) {
#define OTS_CASE(GG, CC) if (G == GG && C == CC) return launch_step_t<FWD, GG, CC, PC>(a, s);
  OTS_CASE(1, 1) OTS_CASE(2, 1) OTS_CASE(4, 1) OTS_CASE(8, 1) OTS_CASE(16, 1) OTS_CASE(32, 1)
  OTS_CASE(64, 1) OTS_CASE(128, 1) OTS_CASE(256, 1)
  OTS_CASE(256, 2) OTS_CASE(256, 3) OTS_CASE(256, 4)
#undef OTS_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_step(bool fwd, bool pc, int G, int C, const StepArgs &a, cudaStream_t s) {
  if (fwd) return pc ? launch_step_g<true, true>(G, C, a, s) : launch_step_g<true, false>(G, C, a, s);
  return pc ? launch_step_g<false, true>(G, C, a, s) : launch_step_g<false, false>(G, C, a, s);
}

int step_grid(int V, int G) { const int npb = nodes_per_block(G); return (V + npb - 1) / npb; }

cudaError_t launch_boundary(const BndArgs &b, cudaStream_t s) {
  const int grid = (b.n_seg + kBlock - 1) / kBlock;
  k_boundary<<<grid > 0 ? grid : 1, kBlock, 0, s>>>(b);
  return cudaGetLastError();
}

int boundary_grid(int n_seg) { int g = (n_seg + kBlock - 1) / kBlock; return g > 0 ? g : 1; }

cudaError_t launch_pass_begin(DevStats *st, cudaStream_t s) {
  k_pass_begin<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_pass_end(const DevStats *st, PassReport *rep, double mass, double eps, cudaStream_t s) {
  k_pass_end<<<1, 1, 0, s>>>(st, rep, mass, eps);
  return cudaGetLastError();
}

cudaError_t launch_init_weights(int S, int T, const float *kl_hi, const float *kl_lo, double *logu, float *w_hi,
                                float *w_lo, cudaStream_t s) {
  k_init_weights<<<(S + 255) / 256, 256, 0, s>>>(S, T, kl_hi, kl_lo, logu, w_hi, w_lo);
  return cudaGetLastError();
}

cudaError_t launch_weights_from_logu(int S, int T, const float *kl_hi, const float *kl_lo, const double *logu,
                                     float *w_hi, float *w_lo, cudaStream_t s) {
  k_weights_from_logu<<<(S + 255) / 256, 256, 0, s>>>(S, T, kl_hi, kl_lo, logu, w_hi, w_lo);
  return cudaGetLastError();
}

cudaError_t launch_fill_panel(size_t n, float *hi, __half *lo, cudaStream_t s) {
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks == 0) blocks = 1;
  k_fill_panel<<<(unsigned)blocks, 256, 0, s>>>(n, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_commodity_flows(int S, int Lp, int l0, int l1, const int *tail, const int *head, const float *a_hi,
                                   const __half *a_lo, const float *b_hi, const __half *b_lo, const float *kl_hi,
                                   const float *kl_lo, const float *klc_hi, const __half *klc_lo, const double *logu_t,
                                   double *out, cudaStream_t s) {
  size_t n = (size_t)S * (l1 - l0);
  size_t blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks == 0) blocks = 1;
  k_commodity_flows<<<(unsigned)blocks, 256, 0, s>>>(S, Lp, l0, l1, tail, head, a_hi, a_lo, b_hi, b_lo, kl_hi, kl_lo,
                                                     klc_hi, klc_lo, logu_t, out);
  return cudaGetLastError();
}

cudaError_t launch_boundary_flows(int n, int Lp, const int *tri_l, const int *tri_node_other, const double *tri_logU,
                                  const float *msg_hi, const __half *msg_lo, double *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_boundary_flows<<<(n + 255) / 256, 256, 0, s>>>(n, Lp, tri_l, tri_node_other, tri_logU, msg_hi, msg_lo, out);
  return cudaGetLastError();
}

}  // namespace ots

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
// 4 (c G + g) + k, k < 4, c < C (16-byte hi / 8-byte lo loads, coalesced along the row).
// In-states are processed in batches of kBatch rows gathered up front.  Column sums over
// commodities are two group reductions (maximum, then sum of ex2 terms): warp shuffles, and
// one shared-memory exchange when G > 32.  For G >= kBatch the capacity update of in-state k
// is done by thread k of the group and broadcast; smaller groups do all updates in every thread.  Sums that decide convergence are FP64 and
// deterministic (per-block partials, reduced by the last block in a fixed order).
#include <cuda_runtime.h>
#include <algorithm>
#include <math.h>
#include <stdint.h>

#include "ots_device.cuh"
#include "ots_step.cuh"

namespace ots {

template <int G>
struct BlockOf { static constexpr int value = G > 32 ? G : kBlock; };
template <int G>
struct MinBlocks { static constexpr int value = G > 32 ? 768 / G : 3; };
template <int G>
struct MinBlocksFwd { static constexpr int value = G > 32 ? 512 / G : 2; };

constexpr int kBatch = 6;   // in-states gathered per batch (grid nodes have 5)

// Programmatic dependent launch: a step kernel launched with programmatic stream serialisation
// may start while the previous step's grid finishes.  Before pdl_wait a kernel touches only
// shared memory and data no kernel of the pass writes before it (static per-state data, or data
// of the previous pass); pdl_wait returns once the previous grid has completed and its writes
// are visible, and pdl_trigger then lets the next step's grid launch (its blocks take the SM
// slots this grid's blocks free).  The next grid starts only after every block of this one has
// triggered or exited, so its blocks never hold slots this grid still needs.  Both are no-ops
// for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------------------------------
// forward step t (t = 2..T-1): capacity update of every state entering v, then A_t[v]
//
// W_t[j] is log2 K_L[j] + log2 u_t[j] when the rows of C_L are shared by all commodities,
// and log2 u_t[j] alone when a per-commodity K_L panel (klc) is given.
// ------------------------------------------------------------------------------------
template <int G, int C, bool PC>
__global__ void __launch_bounds__(BlockOf<G>::value, MinBlocksFwd<G>::value) k_forward(const StepArgs a) {
  constexpr int BS = BlockOf<G>::value;
  constexpr int NPB = BS / G;  // nodes per block (1 when G > 32)
  constexpr int KB = kBatch;
  constexpr int NW = G > 32 ? G / 32 : 1;
  __shared__ float red[1];                   // unused: reductions above stay within a warp
  __shared__ float xch[2 * 2 * KB * NW];     // per-warp (max, sum) pairs, two batch buffers
  pdl_wait();
  pdl_trigger();
  const float lo_unit = a.qs.lo_unit;
  int batch = 0;
  const int g = threadIdx.x % G;
  const int v = blockIdx.x * NPB + threadIdx.x / G;
  const bool active = v < a.V;
  const size_t rowv = (size_t)(active ? v : 0) * a.Lp;

  float bh[C][4], bl[C][4];   // B_{t+1}[v]: hi, signed remainder in units
#pragma unroll
  for (int c = 0; c < C; ++c) {
    uint32_t w[2];
    load4(a.y_hi + rowv + 4 * (c * G + g), a.y_lo + rowv + 4 * (c * G + g), bh[c], w);
#pragma unroll
    for (int q = 0; q < 4; ++q) bl[c][q] = lo_inj(w, q) - kLoBias;
  }

  float M[C][4], acc[C][4];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) { M[c][q] = 2.f * kNeg; acc[c][q] = 0.f; }

  float viol = 0.f;
  float2 dual = make_float2(0.f, 0.f);
  const int jb = active ? a.ptr[v] : 0;
  const int je = active ? a.ptr[v + 1] : 0;
  // G > 32: the block is one node, so trip counts are uniform across the block.
  for (int j0 = jb; j0 < je; j0 += KB) {
    const int nb = min(KB, je - j0);
    int st[KB];
    float xh[KB][C][4];
    uint32_t xw[KB][C][2];
    gather_rows<G, C, KB, PC>(a, j0, nb, g, st, xh, xw);

    // (1) column log-sum-exp over commodities of A_{t-1}[y] (+ K_L) + B_{t+1}[v] for every
    //     in-state of the batch.  Per warp (or per group when G < 32): maximum, then sum of
    //     ex2 terms, by shuffles; exact hi sums.
    float cm[KB], cs[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      float m = 2.f * kNeg;
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) m = fmaxf(m, xh[k][c][q] + bh[c][q]);
      cm[k] = m;
    }
    group_reduce<(G < 32 ? G : 32), KB, true>(cm, red);
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      float sum = 0.f;
      if (cm[k] > kNegThresh) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float s = xh[k][c][q] + bh[c][q];
            const float e = (lo_inj(xw[k][c], q) - kLoBias) + bl[c][q];   // exact, in units
            sum += ex2(fmaf(e, lo_unit, s - cm[k]));
          }
      }
      cs[k] = sum;
    }
    group_reduce<(G < 32 ? G : 32), KB, false>(cs, red);

    // (2) capacity update of each in-state and the weights W_t of the batch
    float wh[KB], wl[KB];
    if (G >= 32) {
      // lane k of every warp merges the warps' (max, sum) pairs of in-state k (one shared
      // memory exchange, double-buffered by batch parity) and derives W_t[state k]; warp 0
      // stores the update and the FP64 sums.  W is then broadcast by shuffles.
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      float mk = cm[0], sk_ = cs[0];
      int stk = st[0];
#pragma unroll
      for (int k = 1; k < KB; ++k)
        if (k == lane) { mk = cm[k]; sk_ = cs[k]; stk = st[k]; }
      if (G > 32) {
        float *xb = xch + (batch & 1) * (2 * KB * NW);
        if (lane < nb) { xb[(2 * lane) * NW + wid] = mk; xb[(2 * lane + 1) * NW + wid] = sk_; }
        __syncthreads();
        if (lane < nb) {
          mk = xb[(2 * lane) * NW];
          sk_ = xb[(2 * lane + 1) * NW];
#pragma unroll
          for (int w = 1; w < NW; ++w) lse_merge(mk, sk_, xb[(2 * lane) * NW + w], xb[(2 * lane + 1) * NW + w]);
        }
      }
      float mh = kNeg, ml = 0.f;
      // G == 32: each warp is its own node and stores its own updates
      if (lane < nb) update_state<PC>(a, stk, mk, sk_, G == 32 || wid == 0, mh, ml, viol, dual);
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const float h = __shfl_sync(0xffffffffu, mh, k);
        const float l = __shfl_sync(0xffffffffu, ml, k);
        wh[k] = k < nb ? h : kNeg;
        wl[k] = k < nb ? l : 0.f;
      }
    } else if (G >= KB) {
      // groups of at least KB threads: thread k of the group updates in-state k (its loads of
      // the per-state inputs run in parallel with the other threads') and W is broadcast
      // within the group by shuffles
      float mk = cm[0], sk_ = cs[0];
      int stk = st[0];
#pragma unroll
      for (int k = 1; k < KB; ++k)
        if (k == g) { mk = cm[k]; sk_ = cs[k]; stk = st[k]; }
      float mh = kNeg, ml = 0.f;
      if (g < nb) update_state<PC>(a, stk, mk, sk_, true, mh, ml, viol, dual);
      // the group's lanes only: groups of one warp run different numbers of batches
      const unsigned gmask = (G >= 32) ? 0xffffffffu : (((1u << (G & 31)) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const float h = __shfl_sync(gmask, mh, k, G);
        const float l = __shfl_sync(gmask, ml, k, G);
        wh[k] = k < nb ? h : kNeg;
        wl[k] = k < nb ? l : 0.f;
      }
    } else {
      // small groups: every thread derives all updates; thread 0 of the group stores them
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        wh[k] = kNeg;
        wl[k] = 0.f;
        if (k < nb) update_state<PC>(a, st[k], cm[k], cs[k], g == 0, wh[k], wl[k], viol, dual);
      }
    }
    ++batch;

    // (2b) commodity-dependent capacities (Section 3.3): after u_t, the dual of
    //      P_{0,t} <= D of every (in-state, commodity) of the batch,
    //      log2 U^(0,t) <- min(log2 D - log2 (P_{0,t} ./ U^(0,t)), 0), with P_{0,t} under the
    //      new u_t; the change of P_{0,t} joins the capacity residual, and the gathered rows
    //      take the new U^(0,t) for the aggregation.
    if constexpr (PC) {
      if (a.uc_t && a.mode == 0 && active) {
        const float q = a.qs.q;
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          if (k >= nb) continue;
          const size_t row = (size_t)st[k] * a.Lp;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int col0 = 4 * (c * G + g);
            const float4 u4 = *reinterpret_cast<const float4 *>(a.uc_t + row + col0);
            const float uo[4] = {u4.x, u4.y, u4.z, u4.w};
            float un4[4];
            lo_t nl[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              float uh, uu;
              split_units(uo[qq], a.qs, uh, uu);
              // log2 P_{0,t} / U^(0,t): hi on the grid (exact), lo in units plus W's lo
              const float ph = (xh[k][c][qq] - uh) + bh[c][qq] + wh[k];
              const float pu = (lo_inj(xw[k][c], qq) - kLoBias) - uu + bl[c][qq];
              const float pl = fmaf(pu, lo_unit, wl[k]);
              float unew = 0.f;
              const float2 d = a.dc[row + col0 + qq];
              if (xh[k][c][qq] > kNegThresh && bh[c][qq] > kNegThresh && wh[k] > kNegThresh && d.x < INFINITY) {
                if (d.x < kNegThresh) {
                  unew = kNeg;                               // D = 0: closed for this commodity
                } else {
                  float s1, e1;
                  two_sum(d.x, -ph, s1, e1);
                  unew = fminf(s1 + (e1 + (d.y - pl)), 0.f);
                }
                // |P_new - P_old| = P_old |2^(unew - uold) - 1|, P_old = 2^(log2 P / U + uold)
                const bool co = uo[qq] < kNegThresh, cn = unew < kNegThresh;
                if (!(co && cn)) {
                  const float lp = (ph + pl);
                  if (co || cn) {
                    viol += ex2(fminf(lp + (co ? unew : uo[qq]), 126.f));
                  } else {
                    const float dl = unew - uo[qq];
                    if (dl != 0.f)
                      viol += fminf(ex2(fminf(lp + uo[qq], 126.f)) * fabsf(ex2(fminf(dl, 126.f)) - 1.f), 1e30f);
                  }
                }
              }
              un4[qq] = unew;
              // the gathered row with the new dual: x - old + new, on the grid
              float nh, nu;
              split_units(unew, a.qs, nh, nu);
              float u = (lo_inj(xw[k][c], qq) - kLoBias) - uu + nu;
              float h = (xh[k][c][qq] - uh) + nh;
              carry_units(u, h, q);
              xh[k][c][qq] = h;
              nl[qq] = (lo_t)((int)u + 32768);
            }
            *reinterpret_cast<float4 *>(a.uc_t + row + col0) = make_float4(un4[0], un4[1], un4[2], un4[3]);
            xw[k][c][0] = (uint32_t)nl[0] | ((uint32_t)nl[1] << 16);
            xw[k][c][1] = (uint32_t)nl[2] | ((uint32_t)nl[3] << 16);
          }
        }
      }
    }

    // (3) A_t[v] accumulates A_{t-1}[y] + W_t[state] over the batch
    aggregate_batch<C, KB>(xh, xw, wh, wl, lo_unit, M, acc);
  }

  if (active) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float oh[4];
      lo_t ol[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) lse_encode(M[c][q], acc[c][q], a.qs, oh[q], ol[q]);
      store4(a.out_hi + rowv + 4 * (c * G + g), a.out_lo + rowv + 4 * (c * G + g), oh, ol);
    }
  }
  if (a.mode == 0)
    step_sums(a.slot, make_float2(viol, 0.f), dual, a.partials, a.counter, &a.stats->cap_viol, &a.stats->dual_cap);
}

// ------------------------------------------------------------------------------------
// backward step t (t = T-1..2): B_t[v] = LSE_{j: tail j = v} (B_{t+1}[head j] + W_t[j] (+ K_L))
// ------------------------------------------------------------------------------------
template <int G, int C, bool PC>
__global__ void __launch_bounds__(BlockOf<G>::value, MinBlocks<G>::value) k_backward(const StepArgs a) {
  constexpr int BS = BlockOf<G>::value;
  constexpr int NPB = BS / G;
  constexpr int KB = kBatch;
  pdl_wait();
  pdl_trigger();
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
    float xh[KB][C][4];
    uint32_t xw[KB][C][2];
    gather_rows<G, C, KB, PC>(a, j0, nb, g, st, xh, xw);
    float wh[KB], wl[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      wh[k] = k < nb ? a.w_hi_t[st[k]] : kNeg;
      wl[k] = k < nb ? a.w_lo_t[st[k]] : 0.f;
    }
    aggregate_batch<C, KB>(xh, xw, wh, wl, a.qs.lo_unit, M, acc);
  }
  const size_t rowo = (size_t)v * a.Lp;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float oh[4];
    lo_t ol[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) lse_encode(M[c][q], acc[c][q], a.qs, oh[q], ol[q]);
    store4(a.out_hi + rowo + 4 * (c * G + g), a.out_lo + rowo + 4 * (c * G + g), oh, ol);
  }
}

// ------------------------------------------------------------------------------------
// boundary updates: U01 <- R01 ./ Psi_1 (sources), U0T <- R0T ./ hatPsi_T (sinks), and the
// boundary panels A_1 = (U01 K) by tail node, B_T = (U0T K^T) by head node.
// One thread per (node, commodity) segment of triples; FP64 throughout.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_boundary(const BndArgs b) {
  const int sidx = blockIdx.x * blockDim.x + threadIdx.x;
  double r0 = 0.0, r1 = 0.0, r2 = 0.0;
  if (sidx < b.n_seg) boundary_segment(b, sidx, r0, r1, r2);
  if (b.mode == 0) {
    const int assign = b.accumulate ? 0 : 1;
    if (b.is_source) {
      block_sum2_last(to_ff(r0), to_ff(r1), b.partials, b.counter, &b.stats->src_resid, &b.stats->dual_src, assign);
    } else {
      block_sum2_last(to_ff(r0), to_ff(r1), b.partials, b.counter, &b.stats->mass_snk, &b.stats->dual_snk, assign);
    }
    if (r2 > 0.0) atomicAdd(&b.stats->bad, r2);
  }
}

// ------------------------------------------------------------------------------------
// Storage states (the rows of StoreRowArgs): after each step, and at the boundaries.
// One thread per (storage state, 4 commodities); same arithmetic as the node rows (exact hi
// sums on the q grid, one ex2 per term).
// ------------------------------------------------------------------------------------
__global__ void k_store_rows(const StoreRowArgs a) {
  const int n4 = a.Lp / 4;
  const size_t total = (size_t)a.n * n4;
  const float lo_unit = a.qs.lo_unit;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / n4), c = (int)(i % n4);
    const int v = a.node[k];
    float h1[4];
    uint32_t w1[2] = {0x80008000u, 0x80008000u};
    if (v >= 0) {
      load4(a.p_hi + (size_t)v * a.Lp + 4 * c, a.p_lo + (size_t)v * a.Lp + 4 * c, h1, w1);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) h1[q] = kNeg;
    }
    float oh[4];
    lo_t ol[4];
    if (!a.q_hi) {                                   // boundary: the node row's value
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        oh[q] = h1[q];
        ol[q] = (lo_t)((w1[q >> 1] >> (16 * (q & 1))) & 0xffffu);
      }
    } else {
      const int st = a.state[k];
      const float wh = a.w_hi[st], wlb = a.w_lo[st] - kLoBias * lo_unit, nlb = -kLoBias * lo_unit;
      const size_t r = (size_t)(a.row0 + k) * a.Lp + 4 * c;
      float h2[4];
      uint32_t w2[2];
      load4(a.q_hi + r, a.q_lo + r, h2, w2);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float s1 = h1[q], s2 = h2[q] + wh;     // exact (q grid); a closed self term is log 0
        const float m = fmaxf(s1, s2);
        float acc = 0.f;
        if (m > kNegThresh)
          acc = ex2(fmaf(lo_inj(w1, q), lo_unit, (s1 - m) + nlb)) + ex2(fmaf(lo_inj(w2, q), lo_unit, (s2 - m) + wlb));
        lse_encode(m, acc, a.qs, oh[q], ol[q]);
      }
    }
    const size_t o = (size_t)(a.row0 + k) * a.Lp + 4 * c;
    store4(a.p_hi + o, a.p_lo + o, oh, ol);
  }
}

// Boundary terms of storage states: (+) log2 U of their own triples, in FP64 (as the node rows'
// boundary entries); the (row, commodity) pairs are distinct, so no two threads share an entry.
__global__ void k_store_triples(const StoreTriArgs a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const size_t idx = (size_t)(a.row0 + a.k[i]) * a.Lp + a.l[i];
    const double cur = a.p_hi[idx] < kNegThresh ? -INFINITY
                                                 : (double)a.p_hi[idx] + ((double)a.p_lo[idx] - 32768.0) * (double)a.qs.lo_unit;
    const double u = a.tri_logU[a.q[i]];
    const double m = fmax(cur, u);
    const double r = m + log2(exp2(cur - m) + exp2(u - m));
    const float h = (float)r;
    float oh;
    lo_t ol;
    encode(h, (float)(r - (double)h), a.qs, oh, ol);
    a.p_hi[idx] = oh;
    a.p_lo[idx] = ol;
  }
}

// Capacity update of the storage states before forward step t (Corollary 7 with their own
// message rows): one warp per state, the column log-sum-exp over commodities of
// A_{t-1}[row0 + k] + B_{t+1}[row0 + k], then the same update as every other state (a.fixed_w is
// not set here).  The FP64 sums join the pass totals.
__global__ void __launch_bounds__(256) k_store_update(const StepArgs a, const StoreUpdArgs u) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  float viol = 0.f;
  float2 dual = make_float2(0.f, 0.f);
  const int n4 = u.Lp / 4;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < u.n; k += warps) {
    const size_t r = (size_t)(u.row0 + k) * u.Lp;
    float cm = 2.f * kNeg;
    for (int c = lane; c < n4; c += 32) {
      float hx[4], hy[4];
      uint32_t wx[2], wy[2];
      load4(u.x_hi + r + 4 * c, u.x_lo + r + 4 * c, hx, wx);
      load4(u.y_hi + r + 4 * c, u.y_lo + r + 4 * c, hy, wy);
#pragma unroll
      for (int q = 0; q < 4; ++q) cm = fmaxf(cm, hx[q] + hy[q]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    float cs = 0.f;
    if (cm > kNegThresh) {
      for (int c = lane; c < n4; c += 32) {
        float hx[4], hy[4];
        uint32_t wx[2], wy[2];
        load4(u.x_hi + r + 4 * c, u.x_lo + r + 4 * c, hx, wx);
        load4(u.y_hi + r + 4 * c, u.y_lo + r + 4 * c, hy, wy);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float bl = lo_inj(wy, q) - 2.f * kLoBias;                     // exact
          cs += ex2(fmaf(lo_inj(wx, q) + bl, a.qs.lo_unit, (hx[q] + hy[q]) - cm));
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
    if (lane == 0) {
      float wh, wl;
      update_state<false>(a, u.state[k], cm, cs, true, wh, wl, viol, dual);
    }
  }
  block_sum2_last(make_float2(viol, 0.f), dual, a.partials, a.counter, &a.stats->cap_viol, &a.stats->dual_cap, 0);
}

// Start of a pass: clear the accumulators the forward sweep adds into.
__global__ void k_pass_begin(DevStats *st) {
  st->cap_viol = 0.0;
  st->dual_cap = 0.0;
  st->bad = 0.0;
}

// End of a pass, first part: block t adds the per-block sums the forward step t left in its slot
// (fixed assignment of blocks to threads, fixed tree), giving one pair of totals per step.
__global__ void k_step_totals(const double *slots, int stride, int nblk, int T, double *tot) {
  __shared__ double s0[32], s1[32];
  const int t = blockIdx.x;
  double v0 = 0.0, v1 = 0.0;
  if (t >= 2 && t <= T - 1)
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      v0 += slots[(size_t)t * stride + 2 * b];
      v1 += slots[(size_t)t * stride + 2 * b + 1];
    }
  block_sum2_f64(v0, v1, s0, s1);
  if (threadIdx.x == 0) { tot[2 * t] = v0; tot[2 * t + 1] = v1; }
}

// End of a pass: relative measures and the dual objective of Theorem 3 in natural units:
//   -eps <K,U> + eps ln2 (<R01, log2 U01> + <R0T, log2 U0T> + sum_t <d, log2 u_t>).
// The forward steps' sums come from tot (steps 2..T-1, added in order; nullptr: already in st).
__global__ void k_pass_end(const DevStats *st, PassReport *rep, double mass, double eps, const double *tot, int T) {
  double cap = st->cap_viol, dcap = st->dual_cap;
  if (tot)
    for (int t = 2; t <= T - 1; ++t) { cap += tot[2 * t]; dcap += tot[2 * t + 1]; }
  rep->src_resid_rel = st->src_resid / mass;
  rep->cap_viol_rel = cap / mass;
  rep->dual_objective = -eps * st->mass_snk + eps * 0.69314718055994530942 * (st->dual_src + st->dual_snk + dcap);
  rep->bad = st->bad;
  rep->passes += 1;
}

// W_t = log2 K_L + log2 u_t for t = 2..T-1 from log2 u (set to 0 first when reset).
__global__ void k_weights(int S, int T, QScale qs, const float *kl_hi, const float *kl_lo, int kl_stride, float2 *lu2,
                          float *w_hi,
                          float *w_lo, int reset, const int *st_inpos, const int *st_outpos, float2 *lu2_in,
                          float *wout_hi, float *wout_lo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  for (int t = 2; t <= T - 1; ++t) {
    if (reset) lu2[(size_t)t * S + s] = make_float2(0.f, 0.f);
    float2 lu = lu2[(size_t)t * S + s];
    if (lu.x < kNegThresh) lu = make_float2(kNeg, 0.f);
    float hi, lo;
    const size_t kq = (size_t)t * kl_stride + s;   // kl_stride = S for time-varying costs, else 0
    make_w(kl_hi ? kl_hi[kq] : 0.f, kl_lo ? kl_lo[kq] : 0.f, lu.x, lu.y, qs, hi, lo);
    w_hi[(size_t)t * S + s] = hi;
    w_lo[(size_t)t * S + s] = lo;
    lu2_in[(size_t)t * S + st_inpos[s]] = lu;
    wout_hi[(size_t)t * S + st_outpos[s]] = hi;
    wout_lo[(size_t)t * S + st_outpos[s]] = lo;
  }
}

__global__ void k_fill_panel(size_t n, float *hi, lo_t *lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    hi[i] = kNeg;
    lo[i] = kLoZero;
  }
}

// Per-commodity flows P_{0,t}[l, j] = 2^(A_{t-1}[tail j][l] + B_{t+1}[head j][l] + log2 K_L + log2 u_t)
// for commodities [l0, l1), all states j; out[(l - l0) * S + j].
__global__ void k_commodity_flows(int S, int Lp, QScale qs, int l0, int l1, const int *tail, const int *head,
                                  const float *a_hi, const lo_t *a_lo, const float *b_hi, const lo_t *b_lo,
                                  const float *kl_hi, const float *kl_lo, const float *klc_hi, const lo_t *klc_lo,
                                  const float *uc_t, const float2 *lu_t, double *out) {
  const size_t n = (size_t)S * (l1 - l0);
  const double unit = qs.lo_unit;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % S);
    const int l = l0 + (int)(i / S);
    const size_t ia = (size_t)tail[j] * Lp + l, ib = (size_t)head[j] * Lp + l;
    const float ah = a_hi[ia], bh = b_hi[ib];
    const float2 lu = lu_t[j];
    if (ah < kNegThresh || bh < kNegThresh || lu.x < kNegThresh) { out[i] = 0.0; continue; }
    double x = (double)ah + ((double)a_lo[ia] - 32768.0) * unit + (double)bh + ((double)b_lo[ib] - 32768.0) * unit +
               (double)lu.x + (double)lu.y;
    if (klc_hi) x += (double)klc_hi[(size_t)j * Lp + l] + ((double)klc_lo[(size_t)j * Lp + l] - 32768.0) * unit;
    else x += (double)kl_hi[j] + (double)kl_lo[j];
    if (uc_t) {
      const float u = uc_t[(size_t)j * Lp + l];
      if (u < kNegThresh) { out[i] = 0.0; continue; }
      x += (double)u;
    }
    out[i] = exp2(x);
  }
}

// Boundary flows of one triple list: P = 2^(log2 U + msg) per triple (t = 1 or t = T).
__global__ void k_boundary_flows(int n, int Lp, QScale qs, const int *tri_l, const int *tri_node_other,
                                 const double *tri_logU, const float *msg_hi, const lo_t *msg_lo, double *out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const size_t idx = (size_t)tri_node_other[q] * Lp + tri_l[q];
  if (msg_hi[idx] < kNegThresh) { out[q] = 0.0; return; }
  const double msg = (double)msg_hi[idx] + ((double)msg_lo[idx] - 32768.0) * (double)qs.lo_unit;
  out[q] = exp2(tri_logU[q] + msg);
}

// ------------------------------------------------------------------------------------
// Pipelined persistent variants for G >= 64 (one node row of Lp = 4 G commodities per
// block iteration; rank-1 K_L).  A work item is a node and up to kBatchTma of its in-states
// (forward) or out-states (backward).  The rows an item gathers are fetched with TMA bulk
// copies (cp.async.bulk) into one of two shared-memory stages while the block computes on the
// other; an mbarrier with an expected byte count signals each stage.  Waits are bounded: a
// wait that gives up records an error in the pass statistics instead of hanging.
// ------------------------------------------------------------------------------------
constexpr int kBatchTma = 5;
constexpr int kBatchBwd = 5;      // out-states per work item of the backward kernel (<= kBatchTma)

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up.  Each try may suspend
// the thread for up to 2 us (returning as soon as the phase completes), so a waiting warp
// does not spin on the issue slots; the default 2^20 tries bound the wait to about two seconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t tries) {
  for (uint32_t i = 0; i < tries; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(2000u)
        : "memory");
    if (ok) return true;
  }
  return false;
}

struct TmaItem {
  int v, j0, nb, first;
};
__device__ __forceinline__ bool item_first(const int *ptr, int V, int KB, TmaItem &it) {
  it.v = blockIdx.x;
  it.first = 1;
  if (it.v >= V) return false;
  it.j0 = ptr[it.v];
  it.nb = min(KB, ptr[it.v + 1] - it.j0);
  return true;
}
__device__ __forceinline__ bool item_next(const int *ptr, int V, int KB, TmaItem &it) {
  const int je = ptr[it.v + 1];
  if (it.j0 + it.nb < je) {
    it.first = 0;
    it.j0 += it.nb;
    it.nb = min(KB, je - it.j0);
    return true;
  }
  it.v += gridDim.x;
  it.first = 1;
  if (it.v >= V) return false;
  it.j0 = ptr[it.v];
  it.nb = min(KB, ptr[it.v + 1] - it.j0);
  return true;
}

// Thread g's 4 entries of a staged row.
__device__ __forceinline__ void srow(const float *hi, const lo_t *lo, int g, float h[4], uint32_t w[2]) {
  const float4 x = reinterpret_cast<const float4 *>(hi)[g];
  const uint2 y = reinterpret_cast<const uint2 *>(lo)[g];
  h[0] = x.x; h[1] = x.y; h[2] = x.z; h[3] = x.w;
  w[0] = y.x;
  w[1] = y.y;
}

}  // namespace

// Shared-memory stages per block of the pipelined kernels.  The forward kernel runs three blocks
// per SM with two stages each (more warps for its issue-bound consumers); the backward kernel,
// bound by the bytes in flight, runs two blocks with three stages each.
constexpr int kTmaChunks256 = 2;   // chunks of 4 commodities per consumer thread for rows of 1024
constexpr int kStagesFwd = 2;
constexpr int kStagesBwd = 2;
template <bool FWD>
struct StagesOf { static constexpr int value = FWD ? kStagesFwd : kStagesBwd; };

// Per-stage metadata written by the producer warp: the work item and everything the consumers
// would otherwise fetch with dependent global loads.
struct FwdMeta {
  int v, j0, nb, first, last, valid;
  int st[kBatchTma], outpos[kBatchTma], nbr[kBatchTma];
  float kl_hi[kBatchTma], kl_lo[kBatchTma], logd_hi[kBatchTma], logd_lo[kBatchTma];
  float w_hi[kBatchTma], w_lo[kBatchTma];      // flows mode: the stored weights
  float2 cap[kBatchTma], lu_old[kBatchTma];
  int fin[kBatchTma];                           // capacity finite
  float cref[kBatchTma];                        // column references (0 for k >= nb)
  int use_ref;                                  // every in-state of the item has a reference
};

struct BwdMeta {
  int v, j0, nb, first, last, valid;
  int nbr[kBatchTma];
  float w_hi[kBatchTma], w_lo[kBatchTma];
};

namespace {

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Named barrier among the G consumer threads (the producer warp does not take part).
template <int G>
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(G) : "memory");
}

// Per-lane metadata of one work item (lane k < nb holds in-state / out-state k).
struct LaneMeta {
  int nbr, st, outpos;
  float kl_hi, kl_lo, logd_hi, logd_lo, w_hi, w_lo, cref;
  float2 cap, lu_old;
};

// One independent round of loads per item: everything is stored in CSR order.
template <bool FWD>
__device__ __forceinline__ LaneMeta load_lane_meta(const StepArgs &a, const TmaItem &it, bool have, int lane) {
  LaneMeta r{};
  if (have && lane < it.nb) {
    const int j = it.j0 + lane;
    r.nbr = a.nbr[j];
    if (FWD) {
      r.st = a.state[j];
      r.outpos = a.in_outpos[j];
      r.kl_hi = a.in_kl_hi[j];
      r.kl_lo = a.in_kl_lo[j];
      r.logd_hi = a.in_logd_hi[j];
      r.logd_lo = a.in_logd_lo[j];
      r.cap = a.in_cap[j];
      r.lu_old = a.lu_in_t[j];
      r.cref = a.cref_in_t[j];
    } else {
      r.w_hi = a.wout_hi_t[j];
      r.w_lo = a.wout_lo_t[j];
    }
  }
  return r;
}

// Producer warp: metadata of item i (loaded one iteration ahead) into stage s, then the bulk
// copies of its rows (lane 0).  An exhausted item list writes a stop record.
template <bool FWD, int Lp, typename Meta>
__device__ __forceinline__ void producer_loop(const StepArgs &a, Meta *meta, float *st_hi, lo_t *st_lo,
                                              uint64_t *full, uint64_t *empty, int rows, bool &timed_out) {
  constexpr int KB = FWD ? kBatchTma : kBatchBwd;
  constexpr int NS = StagesOf<FWD>::value;
  const int lane = threadIdx.x & 31;
  TmaItem it;
  bool have = item_first(a.ptr, a.V, KB, it);
  LaneMeta lm = load_lane_meta<FWD>(a, it, have, lane);   // static data or the previous pass's
  pdl_wait();
  pdl_trigger();
  for (int i = 0;; ++i) {
    const int s = i % NS;
    TmaItem nx = it;
    const bool have_nx = have && item_next(a.ptr, a.V, KB, nx);
    const LaneMeta lm_nx = load_lane_meta<FWD>(a, nx, have_nx, lane);   // in flight during the wait
    if (FWD && a.mode != 0 && have && lane < it.nb) {      // flows mode: stored weights
      lm.w_hi = a.wout_hi_t[lm.outpos];
      lm.w_lo = a.wout_lo_t[lm.outpos];
    }
    int ok = 1;
    if (i >= NS && lane == 0) ok = mbar_wait(smem_u32(&empty[s]), ((i / NS) - 1) & 1, a.wait_tries) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) { timed_out = true; return; }
    Meta &m = meta[s];
    int use_ref = 0;
    if constexpr (FWD) use_ref = __all_sync(0xffffffffu, !(have && lane < it.nb) || lm.cref > kNegThresh) ? 1 : 0;
    if (have && lane < it.nb) {
      m.nbr[lane] = lm.nbr;
      if constexpr (FWD) {
        m.st[lane] = lm.st; m.outpos[lane] = lm.outpos;
        m.kl_hi[lane] = lm.kl_hi; m.kl_lo[lane] = lm.kl_lo;
        m.logd_hi[lane] = lm.logd_hi; m.logd_lo[lane] = lm.logd_lo;
        m.cap[lane] = lm.cap; m.lu_old[lane] = lm.lu_old;
        m.fin[lane] = lm.cap.x < INFINITY ? 1 : 0;
        m.w_hi[lane] = lm.w_hi; m.w_lo[lane] = lm.w_lo;
        m.cref[lane] = lm.cref;
      } else {
        m.w_hi[lane] = lm.w_hi; m.w_lo[lane] = lm.w_lo;
      }
    }
    if constexpr (FWD) {
      if (have && lane >= it.nb && lane < KB) m.cref[lane] = 0.f;
    }
    if (lane == 0) {
      m.valid = have ? 1 : 0;
      if constexpr (FWD) m.use_ref = use_ref;
      if (have) {
        m.v = it.v; m.j0 = it.j0; m.nb = it.nb; m.first = it.first;
        m.last = (!have_nx || nx.v != it.v) ? 1 : 0;
      }
    }
    __syncwarp();
    if (lane == 0) {
      const uint32_t bar = smem_u32(&full[s]);
      if (!have) {
        mbar_expect_tx(bar, 0);
      } else {
        float *hi = st_hi + s * rows * Lp;
        lo_t *lo = st_lo + s * rows * Lp;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int nrows = (FWD ? 1 : 0) + it.nb;
        mbar_expect_tx(bar, (uint32_t)(nrows * Lp * (int)(sizeof(float) + sizeof(lo_t))));
        int r = 0;
        if (FWD) {
          bulk_g2s(smem_u32(hi), a.y_hi + (size_t)it.v * Lp, Lp * sizeof(float), bar);
          bulk_g2s(smem_u32(lo), a.y_lo + (size_t)it.v * Lp, Lp * sizeof(lo_t), bar);
          r = 1;
        }
        for (int k = 0; k < it.nb; ++k) {
          const size_t row = (size_t)m.nbr[k] * Lp;
          bulk_g2s(smem_u32(hi + (r + k) * Lp), a.x_hi + row, Lp * sizeof(float), bar);
          bulk_g2s(smem_u32(lo + (r + k) * Lp), a.x_lo + row, Lp * sizeof(lo_t), bar);
        }
      }
    }
    if (!have) return;
    it = nx;
    have = have_nx;
    lm = lm_nx;
  }
}

// Consumer aggregation of one staged item into the running (M, acc) of the thread's 4 entries
// (first: the node's first item, which replaces them; uniform over the block).
// Branch-free: rows k >= nb hold finite stale data and carry wh[k] = log2 0, so their terms
// vanish; a batch with nothing reachable leaves M below kNegThresh (encoded as log2 0).
template <int KB>
__device__ __forceinline__ void aggregate_staged(const float *hs, const lo_t *ls, int Lp, int g,
                                                 const float (&wh)[KB], const float (&wlb)[KB], float lo_unit,
                                                 bool first, float *M, float *acc) {
  float hk[KB][4];
  uint32_t wk[KB][2];
#pragma unroll
  for (int k = 0; k < KB; ++k) srow(hs + k * Lp, ls + k * Lp, g, hk[k], wk[k]);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float sv[KB];
    float m = 2.f * kNeg;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      sv[k] = hk[k][q] + wh[k];
      m = fmaxf(m, sv[k]);
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < KB; ++k) sum += ex2(fmaf(lo_inj(wk[k], q), lo_unit, (sv[k] - m) + wlb[k]));
    if (first) {                      // the node's first item: nothing to merge with
      acc[q] = sum;
      M[q] = m;
    } else {
      const float Mo = M[q];
      const bool up = m > Mo;
      const float e = ex2(-fabsf(Mo - m));
      acc[q] = fmaf(up ? acc[q] : sum, e, up ? sum : acc[q]);
      M[q] = fmaxf(Mo, m);
    }
  }
}

}  // namespace

// Forward step, warp-specialised: G consumer threads (one node row, CH chunks of 4 commodities
// per thread: entries 4 (c G + g) .. + 3) + one producer warp.
template <int G, int CH>
__global__ void __launch_bounds__(G + 32, G * CH == 256 ? 3 : 1) k_forward_tma(const StepArgs a) {
  constexpr int Lp = 4 * G * CH;
  constexpr int KB = kBatchTma;
  constexpr int ROWS = KB + 1;
  constexpr int NW = G / 32;
  constexpr int NS = kStagesFwd;
  extern __shared__ __align__(128) unsigned char smem[];
  float *st_hi = reinterpret_cast<float *>(smem);                                    // [NS][ROWS][Lp]
  lo_t *st_lo = reinterpret_cast<lo_t *>(smem + NS * ROWS * Lp * sizeof(float));    // [NS][ROWS][Lp]
  __shared__ __align__(8) uint64_t full[NS], empty[NS];
  __shared__ FwdMeta meta[NS];
  __shared__ float xch[2][2 * KB * NW], xref[2][KB * NW];
  const int g = threadIdx.x, lane = g & 31, wid = g >> 5;
  if (g == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init(smem_u32(&full[k]), 1);
      mbar_init(smem_u32(&empty[k]), NW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    // finite contents for the rows an item does not fill (the consumers read all KB rows)
    float4 *z = reinterpret_cast<float4 *>(smem);
    constexpr int n16 = (int)(NS * ROWS * Lp * (sizeof(float) + sizeof(lo_t)) / 16);
    for (int k = g; k < n16; k += G + 32) z[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  float viol = 0.f;
  float2 dual = make_float2(0.f, 0.f);
  bool timed_out = false;
  if (wid == NW) {
    // ---------------- producer warp ----------------
    producer_loop<true, Lp, FwdMeta>(a, meta, st_hi, st_lo, full, empty, ROWS, timed_out);
  } else {
    // ---------------- consumers ----------------
    pdl_wait();      // the outputs overwrite a panel the previous step may still read
    pdl_trigger();
    const float lo_unit = a.qs.lo_unit;
    float M[CH][4], acc[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) { M[c][q] = 2.f * kNeg; acc[c][q] = 0.f; }
    for (int i = 0;; ++i) {
      const int s = i % NS;
      if (!mbar_wait(smem_u32(&full[s]), (i / NS) & 1, a.wait_tries)) { timed_out = true; break; }
      const FwdMeta &m = meta[s];
      if (!m.valid) break;
      const int nb = m.nb;
      const float *hs = st_hi + s * ROWS * Lp;
      const lo_t *ls = st_lo + s * ROWS * Lp;
      float bh[CH][4], blb[CH][4];
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        uint32_t w[2];
        srow(hs, ls, c * G + g, bh[c], w);
#pragma unroll
        for (int q = 0; q < 4; ++q) blb[c][q] = lo_inj(w, q) - 2.f * kLoBias;   // exact
      }
      // (1) column log-sum-exp per in-state, log2 sum_l 2^(A_{t-1}[tail, l] + B_{t+1}[v, l]).
      // With a stored reference r (the column maximum of an earlier pass, on the q grid) the
      // sum is taken as 2^r sum_l 2^(x_l - r): one warp sum per in-state and no maximum.  It
      // is kept when the total lies in [2^-8, 2^12] (no overflow, nothing significant below
      // the FP32 range, arguments of the dominant terms within a few tens of bits); otherwise,
      // or without a reference, the maximum is taken first.  The decision is the same in every
      // warp (identical sums in the same order), so the barriers match.
      float mk = 0.f, sk_ = 0.f;
      bool exact = m.use_ref == 0;
      if (!exact) {
        float cs[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const float r = m.cref[k];
          float sum = 0.f;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            float h[4];
            uint32_t w[2];
            srow(hs + (1 + k) * Lp, ls + (1 + k) * Lp, c * G + g, h, w);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              sum += ex2(fmaf(lo_inj(w, q) + blb[c][q], lo_unit, (h[q] + bh[c][q]) - r));
          }
          cs[k] = sum;
        }
        group_reduce<32, KB, false>(cs, nullptr);
        sk_ = cs[0];
#pragma unroll
        for (int k = 1; k < KB; ++k)
          if (k == lane) sk_ = cs[k];
        float *xb = xref[i & 1];
        if (lane < nb) xb[lane * NW + wid] = sk_;
        consumers_sync<G>();
        bool ok = true;
        if (lane < nb) {
          sk_ = xb[lane * NW];
#pragma unroll
          for (int w = 1; w < NW; ++w) sk_ += xb[lane * NW + w];
          mk = m.cref[lane];
          ok = sk_ >= 0x1p-8f && sk_ <= 0x1p12f;
        }
        exact = !__all_sync(0xffffffffu, ok);
      }
      if (exact) {
        // warp max, then warp sum of ex2 terms (all KB rows, branch-free; the pairs of rows
        // k >= nb are finite and never used)
        float cm[KB], cs[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          float mm = 2.f * kNeg;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const float4 x = reinterpret_cast<const float4 *>(hs + (1 + k) * Lp)[c * G + g];
            mm = fmaxf(mm, fmaxf(fmaxf(x.x + bh[c][0], x.y + bh[c][1]), fmaxf(x.z + bh[c][2], x.w + bh[c][3])));
          }
          cm[k] = mm;
        }
        group_reduce<32, KB, true>(cm, nullptr);
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          float sum = 0.f;
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            float h[4];
            uint32_t w[2];
            srow(hs + (1 + k) * Lp, ls + (1 + k) * Lp, c * G + g, h, w);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              sum += ex2(fmaf(lo_inj(w, q) + blb[c][q], lo_unit, (h[q] + bh[c][q]) - cm[k]));
          }
          cs[k] = sum;
        }
        group_reduce<32, KB, false>(cs, nullptr);
        // exchange the warps' pairs; lane k of every warp merges in-state k
        mk = cm[0];
        sk_ = cs[0];
#pragma unroll
        for (int k = 1; k < KB; ++k)
          if (k == lane) { mk = cm[k]; sk_ = cs[k]; }
        float *xb = xch[i & 1];
        if (lane < nb) { xb[(2 * lane) * NW + wid] = mk; xb[(2 * lane + 1) * NW + wid] = sk_; }
        consumers_sync<G>();
        if (lane < nb) {
          mk = xb[(2 * lane) * NW];
          sk_ = xb[(2 * lane + 1) * NW];
#pragma unroll
          for (int w = 1; w < NW; ++w) lse_merge(mk, sk_, xb[(2 * lane) * NW + w], xb[(2 * lane + 1) * NW + w]);
        }
      }
      // (2) lane k of every warp derives W for in-state k
      float mh = kNeg, ml = 0.f;
      if (lane < nb) {
        // every warp derives W (FP32); warp 0 alone does the FP64 part and the stores
        float col_hi, col_lo, lu_hi, lu_lo;
        update_w(a.mode, a.qs, mk, sk_, m.kl_hi[lane], m.kl_lo[lane], m.logd_hi[lane], m.logd_lo[lane],
                 m.fin[lane] != 0, m.w_hi[lane], m.w_lo[lane], mh, ml, col_hi, col_lo, lu_hi, lu_lo);
        if (wid == 0) {
          float2 lu_new;
          double flow = 0.0;
          update_stats(a.mode, col_hi, col_lo, lu_hi, lu_lo, m.logd_hi[lane], m.logd_lo[lane], mh, m.cap[lane],
                       m.lu_old[lane], lu_new, flow, viol, dual);
          const int st = m.st[lane];
          if (exact) a.cref_in_t[m.j0 + lane] = mk;    // the column maximum: next pass's reference
          if (a.mode == 0) {
            a.lu_t[st] = lu_new;
            a.lu_in_t[m.j0 + lane] = lu_new;
            a.w_hi_t[st] = mh;
            a.w_lo_t[st] = ml;
            a.wout_hi_t[m.outpos[lane]] = mh;
            a.wout_lo_t[m.outpos[lane]] = ml;
          } else {
            a.flow_t[st] = flow;
          }
        }
      }
      float wh[KB], wlb[KB];
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        wh[k] = __shfl_sync(0xffffffffu, mh, k);
        wlb[k] = __shfl_sync(0xffffffffu, ml, k) - kLoBias * lo_unit;
      }
      // (3) A_t[v] accumulates A_{t-1}[y] + W_t[state] over the item's in-states
#pragma unroll
      for (int c = 0; c < CH; ++c)
        // the generic merge on every item (a branch on the node's first item measured slower here)
        aggregate_staged<KB>(hs + Lp, ls + Lp, Lp, c * G + g, wh, wlb, lo_unit, false, M[c], acc[c]);
      if (m.last) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          float oh[4];
          lo_t ol[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            lse_encode(M[c][q], acc[c][q], a.qs, oh[q], ol[q]);
            M[c][q] = 2.f * kNeg;
            acc[c][q] = 0.f;
          }
          const size_t o = (size_t)m.v * Lp + 4 * (c * G + g);
          store4(a.out_hi + o, a.out_lo + o, oh, ol);
        }
      }
      __syncwarp();
      if (lane == 0 && !(a.withhold_stage && i == 0)) mbar_arrive(smem_u32(&empty[s]));
    }
  }
  if (timed_out) atomicAdd(&a.stats->bad, 1e6);
  step_sums(a.slot, make_float2(viol, 0.f), dual, a.partials, a.counter, &a.stats->cap_viol, &a.stats->dual_cap);
}

// Backward step, warp-specialised like the forward step.
template <int G, int CH>
__global__ void __launch_bounds__(G + 32, G * CH == 256 ? 3 : 1) k_backward_tma(const StepArgs a) {
  constexpr int Lp = 4 * G * CH;
  constexpr int KB = kBatchBwd;
  constexpr int ROWS = KB;
  constexpr int NW = G / 32;
  constexpr int NS = kStagesBwd;
  extern __shared__ __align__(128) unsigned char smem[];
  float *st_hi = reinterpret_cast<float *>(smem);
  lo_t *st_lo = reinterpret_cast<lo_t *>(smem + NS * ROWS * Lp * sizeof(float));
  __shared__ __align__(8) uint64_t full[NS], empty[NS];
  __shared__ BwdMeta meta[NS];
  const int g = threadIdx.x, lane = g & 31, wid = g >> 5;
  if (g == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init(smem_u32(&full[k]), 1);
      mbar_init(smem_u32(&empty[k]), NW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    // finite contents for the rows an item does not fill (the consumers read all KB rows)
    float4 *z = reinterpret_cast<float4 *>(smem);
    constexpr int n16 = (int)(NS * ROWS * Lp * (sizeof(float) + sizeof(lo_t)) / 16);
    for (int k = g; k < n16; k += G + 32) z[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  bool timed_out = false;
  if (wid == NW) {
    producer_loop<false, Lp, BwdMeta>(a, meta, st_hi, st_lo, full, empty, ROWS, timed_out);
  } else {
    pdl_wait();      // the outputs overwrite a panel the previous step may still read
    pdl_trigger();
    const float lo_unit = a.qs.lo_unit;
    float M[CH][4], acc[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) { M[c][q] = 2.f * kNeg; acc[c][q] = 0.f; }
    for (int i = 0;; ++i) {
      const int s = i % NS;
      if (!mbar_wait(smem_u32(&full[s]), (i / NS) & 1, a.wait_tries)) { timed_out = true; break; }
      const BwdMeta &m = meta[s];
      if (!m.valid) break;
      const int nb = m.nb;
      float wh[KB], wlb[KB];
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        wh[k] = k < nb ? m.w_hi[k] : kNeg;
        wlb[k] = (k < nb ? m.w_lo[k] : 0.f) - kLoBias * lo_unit;
      }
#pragma unroll
      for (int c = 0; c < CH; ++c)
        aggregate_staged<KB>(st_hi + s * ROWS * Lp, st_lo + s * ROWS * Lp, Lp, c * G + g, wh, wlb, lo_unit,
                             m.first != 0, M[c], acc[c]);
      if (m.last) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          float oh[4];
          lo_t ol[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            lse_encode(M[c][q], acc[c][q], a.qs, oh[q], ol[q]);
            M[c][q] = 2.f * kNeg;
            acc[c][q] = 0.f;
          }
          const size_t o = (size_t)m.v * Lp + 4 * (c * G + g);
          store4(a.out_hi + o, a.out_lo + o, oh, ol);
        }
      }
      __syncwarp();
      if (lane == 0 && !(a.withhold_stage && i == 0)) mbar_arrive(smem_u32(&empty[s]));
    }
  }
  if (timed_out) atomicAdd(&a.stats->bad, 1e6);
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------

int nodes_per_block(int G) { return (G > 32 ? G : kBlock) / G; }

// Launch with programmatic stream serialisation (see pdl_wait).
template <typename... Args>
static cudaError_t launch_pdl(void (*kernel)(Args...), int grid, int block, size_t smem, cudaStream_t s,
                              const StepArgs &a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3((unsigned)block, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <bool FWD, int G, int C, bool PC>
static cudaError_t launch_step_t(const StepArgs &a, cudaStream_t s) {
  constexpr int BS = BlockOf<G>::value;
  const int npb = BS / G;
  const int grid = (a.V + npb - 1) / npb;
  if (FWD) return launch_pdl(k_forward<G, C, PC>, grid, BS, 0, s, a);
  return launch_pdl(k_backward<G, C, PC>, grid, BS, 0, s, a);
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

template <int G, int CH>
static size_t tma_smem(bool fwd) {
  return (size_t)(fwd ? kStagesFwd : kStagesBwd) * (fwd ? kBatchTma + 1 : kBatchBwd) * 4 * G * CH *
         (sizeof(float) + sizeof(lo_t));
}

template <int G, int CH>
static cudaError_t launch_tma_t(bool fwd, const StepArgs &a, int grid, cudaStream_t s) {
  if (fwd) return launch_pdl(k_forward_tma<G, CH>, grid, G + 32, tma_smem<G, CH>(true), s, a);
  return launch_pdl(k_backward_tma<G, CH>, grid, G + 32, tma_smem<G, CH>(false), s, a);
}

template <int G, int CH>
static cudaError_t prepare_tma_t(int n_sm, int V, int *grid_fwd, int *grid_bwd) {
  cudaError_t e = cudaFuncSetAttribute(k_forward_tma<G, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tma_smem<G, CH>(true));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_backward_tma<G, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tma_smem<G, CH>(false));
  if (e != cudaSuccess) return e;
  int bf = 0, bb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_forward_tma<G, CH>, G + 32, tma_smem<G, CH>(true));
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_backward_tma<G, CH>, G + 32, tma_smem<G, CH>(false));
  if (e != cudaSuccess) return e;
  *grid_fwd = bf > 0 ? min(V, n_sm * bf) : 0;
  *grid_bwd = bb > 0 ? min(V, n_sm * bb) : 0;
  return cudaSuccess;
}

// Consumer threads and chunks per thread of the pipelined kernels for a row of Lp = 4 G
// commodities: rows of 1024 commodities run 128 threads with two chunks each.
static int tma_chunks(int G) { return G == 256 ? kTmaChunks256 : 1; }

// Set up the pipelined persistent kernels for this problem (before any graph capture):
// grid sizes 0 mean "use the register kernels".
cudaError_t prepare_step_kernels(int G, int C, bool pc, int V, int *grid_fwd, int *grid_bwd) {
  *grid_fwd = 0;
  *grid_bwd = 0;
  if (pc || C != 1 || (G != 64 && G != 128 && G != 256)) return cudaSuccess;
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (G == 64) return prepare_tma_t<64, 1>(n_sm, V, grid_fwd, grid_bwd);
  if (G == 128) return prepare_tma_t<128, 1>(n_sm, V, grid_fwd, grid_bwd);
  if (tma_chunks(256) == 2) return prepare_tma_t<128, 2>(n_sm, V, grid_fwd, grid_bwd);
  return prepare_tma_t<256, 1>(n_sm, V, grid_fwd, grid_bwd);
}

cudaError_t launch_step(bool fwd, bool pc, int G, int C, const StepArgs &a, cudaStream_t s) {
  const int pgrid = fwd ? a.persist_grid_fwd : a.persist_grid_bwd;
  if (pgrid > 0 && !pc && C == 1) {
    if (G == 64) return launch_tma_t<64, 1>(fwd, a, pgrid, s);
    if (G == 128) return launch_tma_t<128, 1>(fwd, a, pgrid, s);
    if (G == 256) return tma_chunks(256) == 2 ? launch_tma_t<128, 2>(fwd, a, pgrid, s) : launch_tma_t<256, 1>(fwd, a, pgrid, s);
  }
  if (fwd) return pc ? launch_step_g<true, true>(G, C, a, s) : launch_step_g<true, false>(G, C, a, s);
  return pc ? launch_step_g<false, true>(G, C, a, s) : launch_step_g<false, false>(G, C, a, s);
}

int step_grid(int V, int G) { const int npb = nodes_per_block(G); return (V + npb - 1) / npb; }

cudaError_t launch_boundary(const BndArgs &b, cudaStream_t s) {
  const int grid = (b.n_seg + kBlock - 1) / kBlock;
  k_boundary<<<grid > 0 ? grid : 1, kBlock, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_store_rows(const StoreRowArgs &a, cudaStream_t s) {
  const size_t total = (size_t)a.n * (a.Lp / 4);
  const int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
  k_store_rows<<<grid > 0 ? grid : 1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_store_triples(const StoreTriArgs &a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  k_store_triples<<<(a.n + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_store_update(const StepArgs &a, const StoreUpdArgs &u, int max_grid, cudaStream_t s) {
  int grid = (u.n + 7) / 8;                       // 8 warps per block, one state per warp
  grid = std::max(1, std::min(grid, max_grid));   // the partial sums hold max_grid blocks
  k_store_update<<<grid, 256, 0, s>>>(a, u);
  return cudaGetLastError();
}

int boundary_grid(int n_seg) { int g = (n_seg + kBlock - 1) / kBlock; return g > 0 ? g : 1; }

cudaError_t launch_pass_begin(DevStats *st, cudaStream_t s) {
  k_pass_begin<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_pass_end(const DevStats *st, PassReport *rep, double mass, double eps, const double *slots,
                            int stride, int nblk, int T, double *tot, cudaStream_t s) {
  if (slots) {
    k_step_totals<<<T, 256, 0, s>>>(slots, stride, nblk, T, tot);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_pass_end<<<1, 1, 0, s>>>(st, rep, mass, eps, slots ? tot : nullptr, T);
  return cudaGetLastError();
}

cudaError_t launch_weights(int S, int T, QScale qs, const float *kl_hi, const float *kl_lo, int kl_stride, float2 *logu,
                           float *w_hi, float *w_lo, int reset, const int *st_inpos, const int *st_outpos,
                           float2 *logu_in, float *wout_hi, float *wout_lo, cudaStream_t s) {
  k_weights<<<(S + 255) / 256, 256, 0, s>>>(S, T, qs, kl_hi, kl_lo, kl_stride, logu, w_hi, w_lo, reset, st_inpos, st_outpos,
                                            logu_in, wout_hi, wout_lo);
  return cudaGetLastError();
}

// Continuation in epsilon: the duals lambda = -eps ln u are carried to a new epsilon, so
// every log u (float-float) and log U (FP64) is multiplied by r = eps_old / eps_new; log 0
// stays the sentinel.
__global__ void k_scale_duals(float2 *lu, size_t n_lu, float2 *lu_in, size_t n_in, double *ua, int na, double *ub,
                              int nb, double r) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_lu + n_in; i += stride) {
    float2 *p = i < n_lu ? lu + i : lu_in + (i - n_lu);
    const float2 x = *p;
    if (x.x < kNegThresh) continue;
    const double v = ((double)x.x + (double)x.y) * r;
    const float h = (float)v;
    *p = make_float2(h, (float)(v - (double)h));
  }
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)na + nb; i += stride) {
    double *p = i < (size_t)na ? ua + i : ub + (i - na);
    if (isfinite(*p)) *p *= r;
  }
}

cudaError_t launch_scale_duals(float2 *lu, size_t n_lu, float2 *lu_in, size_t n_in, double *ua, int na, double *ub,
                               int nb, double r, cudaStream_t s) {
  size_t n = std::max(n_lu + n_in, (size_t)na + nb);
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks == 0) blocks = 1;
  k_scale_duals<<<(unsigned)blocks, 256, 0, s>>>(lu, n_lu, lu_in, n_in, ua, na, ub, nb, r);
  return cudaGetLastError();
}

cudaError_t launch_fill_panel(size_t n, float *hi, lo_t *lo, cudaStream_t s) {
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks == 0) blocks = 1;
  k_fill_panel<<<(unsigned)blocks, 256, 0, s>>>(n, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_commodity_flows(int S, int Lp, QScale qs, int l0, int l1, const int *tail, const int *head,
                                   const float *a_hi, const lo_t *a_lo, const float *b_hi, const lo_t *b_lo,
                                   const float *kl_hi, const float *kl_lo, const float *klc_hi, const lo_t *klc_lo,
                                   const float *uc_t, const float2 *logu_t, double *out, cudaStream_t s) {
  size_t n = (size_t)S * (l1 - l0);
  size_t blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks == 0) blocks = 1;
  k_commodity_flows<<<(unsigned)blocks, 256, 0, s>>>(S, Lp, qs, l0, l1, tail, head, a_hi, a_lo, b_hi, b_lo, kl_hi,
                                                     kl_lo, klc_hi, klc_lo, uc_t, logu_t, out);
  return cudaGetLastError();
}

cudaError_t launch_boundary_flows(int n, int Lp, QScale qs, const int *tri_l, const int *tri_node_other,
                                  const double *tri_logU, const float *msg_hi, const lo_t *msg_lo, double *out,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_boundary_flows<<<(n + 255) / 256, 256, 0, s>>>(n, Lp, qs, tri_l, tri_node_other, tri_logU, msg_hi, msg_lo, out);
  return cudaGetLastError();
}

}  // namespace ots

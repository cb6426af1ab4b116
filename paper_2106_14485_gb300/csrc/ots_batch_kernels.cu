// ots_batch_kernels.cu -- the batched tick kernel: one launch advances every resident
// instance of a batch by one step of Algorithm 2.
//
// Each instance follows its own step sequence (decode_phase): set-up (u_t = 1, W_t = log2 K_L,
// U = 1 on the supports, boundary panels at log 0), the initial boundary panels and backward
// sweep ("Compute Psi_t"), then passes of the while loop of Algorithm 2 -- source update,
// forward steps t = 2..T-1 (capacity update of u_t, Corollary 7, and hatPsi_{t+1}, Theorem
// 6), sink update, backward steps t = T-1..2 -- and, once the pass-end test finds the
// relative source mismatch and capacity excess below the instance's tolerance (or its pass
// limit is reached), one flows pass (Corollary 7) before the slot becomes final.
//
// The message arithmetic is that of the per-instance kernels (node-level rows, quantised
// hi/lo storage, batched log-sum-exp), with the thread mapping as a runtime parameter of the
// instance: G threads per node (G <= 32, so a node row is a slice of one warp) and C = 1 or 2
// chunks of 4 commodities per thread, panel width Lp = 4 G C.  Blocks are persistent: block b
// takes items b, b + grid, b + 2 grid, ... of the tick's list, and stages the next item's
// header and instance description in shared memory while it works on the current one.  The
// last item of an instance to finish reduces the items' FP64 partial sums in a fixed order
// and advances the instance, so every result is deterministic and independent of the other
// instances in the batch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ots_batch.cuh"
#include "ots_device.cuh"
#include "ots_step.cuh"

namespace ots {

namespace {

enum : int { kPhSetup, kPhInitBnd, kPhSrc, kPhFwd, kPhSnk, kPhBwd, kPhFlowFwd, kPhFlowBnd };

struct Phase {
  int kind;
  int t;
  bool pass_end;   // last backward step of a Sinkhorn pass
};

// Step `step` of an instance with horizon T in slot state `status`.
__device__ __forceinline__ Phase decode_phase(int status, int step, int T) {
  if (status == kSlotFlows) {
    if (step < T - 2) return {kPhFlowFwd, step + 2, false};
    return {kPhFlowBnd, 0, false};
  }
  if (step == 0) return {kPhSetup, 0, false};
  if (step == 1) return {kPhInitBnd, 0, false};
  if (step < T) return {kPhBwd, T + 1 - step, false};          // initial sweep t = T-1..2
  const int p = step - T;                                       // position in the pass, 0..2T-3
  if (p == 0) return {kPhSrc, 0, false};
  if (p <= T - 2) return {kPhFwd, p + 1, false};
  if (p == T - 1) return {kPhSnk, 0, false};
  return {kPhBwd, 2 * T - 1 - p, p == 2 * T - 3};
}

__device__ __forceinline__ float *a_hi_of(const BatchInst &I, int t) {
  return t == 1 ? I.a0_hi : ((t & 1) ? I.a2_hi : I.a1_hi);
}
__device__ __forceinline__ lo_t *a_lo_of(const BatchInst &I, int t) {
  return t == 1 ? I.a0_lo : ((t & 1) ? I.a2_lo : I.a1_lo);
}
__device__ __forceinline__ size_t panel_of(const BatchInst &I) { return (size_t)I.V * I.Lp; }

__device__ __forceinline__ StepArgs step_of(const BatchInst &I, bool fwd, int t, int mode, int shift) {
  StepArgs a{};
  a.kl_shift = shift;
  a.V = I.V;
  a.Lp = I.Lp;
  a.qs = I.qs;
  const size_t pan = panel_of(I);
  if (fwd) {
    a.ptr = I.in_ptr; a.state = I.in_state; a.nbr = I.in_nbr;
    a.x_hi = a_hi_of(I, t - 1); a.x_lo = a_lo_of(I, t - 1);
    a.y_hi = I.b_hi + (size_t)(t - 1) * pan; a.y_lo = I.b_lo + (size_t)(t - 1) * pan;   // B_{t+1}
    a.out_hi = a_hi_of(I, t); a.out_lo = a_lo_of(I, t);
  } else {
    a.ptr = I.out_ptr; a.state = I.out_state; a.nbr = I.out_nbr;
    a.x_hi = I.b_hi + (size_t)(t - 1) * pan; a.x_lo = I.b_lo + (size_t)(t - 1) * pan;   // B_{t+1}
    a.out_hi = I.b_hi + (size_t)(t - 2) * pan; a.out_lo = I.b_lo + (size_t)(t - 2) * pan;
  }
  a.kl_hi = I.kl_hi + (size_t)t * I.kl_stride; a.kl_lo = I.kl_lo + (size_t)t * I.kl_stride;
  a.logd_hi = I.logd_hi + (size_t)t * I.cap_stride; a.logd_lo = I.logd_lo + (size_t)t * I.cap_stride;
  a.cap = I.cap + (size_t)t * I.cap_stride;
  a.lu_t = I.lu + (size_t)t * I.S;
  a.w_hi_t = I.w_hi + (size_t)t * I.S;
  a.w_lo_t = I.w_lo + (size_t)t * I.S;
  a.flow_t = I.flow + (size_t)t * I.S;
  a.mode = mode;
  return a;
}

__device__ __forceinline__ BndArgs bnd_of(const BatchInst &I, bool source, int mode) {
  const BndSide &s = source ? I.src : I.snk;
  BndArgs b{};
  b.skip_node = -1;
  b.n_seg = s.n_seg;
  b.qs = I.qs;
  b.seg_ptr = s.seg_ptr; b.seg_node = s.seg_node; b.seg_l = s.seg_l;
  b.tri_node_other = s.tri_other;
  b.tri_R = s.tri_R; b.tri_logR = s.tri_logR; b.tri_logU = s.tri_logU;
  b.Lp = I.Lp;
  const size_t pan = panel_of(I);
  if (source) {
    b.msg_hi = I.b_hi; b.msg_lo = I.b_lo;                                   // B_2 = Psi_1 by head
    b.out_hi = I.a0_hi; b.out_lo = I.a0_lo;                                 // A_1
  } else {
    b.msg_hi = a_hi_of(I, I.T - 1); b.msg_lo = a_lo_of(I, I.T - 1);         // hatPsi_T by tail
    b.out_hi = I.b_hi + (size_t)(I.T - 2) * pan; b.out_lo = I.b_lo + (size_t)(I.T - 2) * pan;   // B_T
  }
  b.mode = mode;
  b.is_source = source ? 1 : 0;
  return b;
}

// Sum of three float-floats over the block, fixed order.
__device__ __forceinline__ void block_sum3(float2 &v0, float2 &v1, float2 &v2, float2 *s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v0 = warp_sum_ff(v0);
  v1 = warp_sum_ff(v1);
  v2 = warp_sum_ff(v2);
  __syncthreads();
  if (lane == 0) { s[3 * wid] = v0; s[3 * wid + 1] = v1; s[3 * wid + 2] = v2; }
  __syncthreads();
  v0 = s[0]; v1 = s[1]; v2 = s[2];
  for (int w = 1; w < kTickBlock / 32; ++w) {
    ff_add(v0, s[3 * w].x, s[3 * w].y);
    ff_add(v1, s[3 * w + 1].x, s[3 * w + 1].y);
    ff_add(v2, s[3 * w + 2].x, s[3 * w + 2].y);
  }
}

template <int C>
struct KBOf { static constexpr int value = C == 1 ? 6 : 3; };   // rows per batch (same registers)

// Slice of KB gathered rows for thread g of a G-thread group (runtime G).
template <int C, int KB>
__device__ __forceinline__ void gather_rt(const StepArgs &a, int G, int j0, int nb, int g, int (&st)[KB],
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
}

// Butterfly reduction over the G lanes of an aligned group of one warp (runtime G <= 32).
template <int KB, bool MAX>
__device__ __forceinline__ void group_reduce_rt(float (&x)[KB], int G, unsigned mask) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (o < G) {
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const float y = __shfl_xor_sync(mask, x[k], o);
        x[k] = MAX ? fmaxf(x[k], y) : x[k] + y;
      }
    }
  }
}

// Forward step t for the nodes [v0, v0 + kTickBlock / G) of one round: capacity update of
// each in-state j of a node (thread j mod G of the node's group owns it) and A_t of the node.
// [jb, je) is the node's in-state range (loaded by the caller one round ahead).  When the
// group has at least KB threads, each owner loads its state's inputs together with the
// gathered rows, so the update waits for no further load.
template <int C>
__device__ __forceinline__ void fwd_round(const StepArgs &a, int G, int v0, int jb, int je, float2 (*s_w)[6],
                                          float &viol, float2 &dual) {
  constexpr int KB = KBOf<C>::value;
  const int g = threadIdx.x & (G - 1);
  const int nib = threadIdx.x / G;                 // node within the round
  const int v = v0 + nib;
  const bool active = v < a.V;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned base = lane & ~(unsigned)(G - 1);
  const unsigned mask = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << base);
  const float lo_unit = a.qs.lo_unit;
  const size_t rowv = (size_t)(active ? v : 0) * a.Lp;
  const bool own1 = G >= KB;                       // at most one in-state per thread

  float bh[C][4], bl[C][4];
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

  if (!active) je = jb;
  for (int j0 = jb; j0 < je; j0 += KB) {           // uniform within the group
    const int nb = min(KB, je - j0);
    int st[KB];
    float xh[KB][C][4];
    uint32_t xw[KB][C][2];
    gather_rt<C, KB>(a, G, j0, nb, g, st, xh, xw);

    // inputs of the owned in-state (one per thread when own1)
    int sk = 0;
    float klh = 0.f, kll = 0.f, ldh = 0.f, ldl = 0.f, wih = kNeg, wil = 0.f;
    float2 capk = make_float2(0.f, 0.f), luo = make_float2(0.f, 0.f);
    if (own1 && g < nb) {
#pragma unroll
      for (int k = 0; k < KB; ++k)
        if (k == g) sk = st[k];
      klh = ldexpf(a.kl_hi[sk], -a.kl_shift); kll = ldexpf(a.kl_lo[sk], -a.kl_shift);
      ldh = a.logd_hi[sk]; ldl = a.logd_lo[sk];
      capk = a.cap[sk];
      luo = a.lu_t[sk];
      if (a.mode != 0) { wih = a.w_hi_t[sk]; wil = a.w_lo_t[sk]; }
    }

    // column log-sum-exp over the commodities of A_{t-1}[tail j] + B_{t+1}[v] per in-state
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
    group_reduce_rt<KB, true>(cm, G, mask);
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      float sum = 0.f;
      if (cm[k] > kNegThresh) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float s = xh[k][c][q] + bh[c][q];
            const float e = (lo_inj(xw[k][c], q) - kLoBias) + bl[c][q];
            sum += ex2(fmaf(e, lo_unit, s - cm[k]));
          }
      }
      cs[k] = sum;
    }
    group_reduce_rt<KB, false>(cs, G, mask);

    // capacity updates; W goes to the group through shared memory
    if (own1) {
      if (g < nb) {
        float m = cm[0], sm = cs[0];
#pragma unroll
        for (int k = 1; k < KB; ++k)
          if (k == g) { m = cm[k]; sm = cs[k]; }
        float h, l;
        float2 lu_new;
        double flow = 0.0;
        update_meta(a.mode, a.qs, m, sm, klh, kll, ldh, ldl, capk, luo, wih, wil, h, l, lu_new, flow, viol, dual);
        if (a.mode == 0) {
          a.lu_t[sk] = lu_new;
          a.w_hi_t[sk] = h;
          a.w_lo_t[sk] = l;
        } else {
          a.flow_t[sk] = flow;
        }
        s_w[nib][g] = make_float2(h, l);
      }
    } else {
      for (int mk = g; mk < nb; mk += G) {
        float m = cm[0], sm = cs[0];
        int skk = st[0];
#pragma unroll
        for (int k = 1; k < KB; ++k)
          if (k == mk) { m = cm[k]; sm = cs[k]; skk = st[k]; }
        float h, l;
        update_state<false>(a, skk, m, sm, true, h, l, viol, dual);
        s_w[nib][mk] = make_float2(h, l);
      }
    }
    __syncwarp(mask);
    float wh[KB], wl[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const float2 wv = k < nb ? s_w[nib][k] : make_float2(kNeg, 0.f);
      wh[k] = wv.x;
      wl[k] = wv.y;
    }
    __syncwarp(mask);
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
}

// Backward step t for the nodes [v0, v0 + kTickBlock / G) of one round: B_t[v] over the
// out-states of v.
template <int C>
__device__ __forceinline__ void bwd_round(const StepArgs &a, int G, int v0, int jb, int je) {
  constexpr int KB = KBOf<C>::value;
  const int g = threadIdx.x & (G - 1);
  const int v = v0 + threadIdx.x / G;
  if (v >= a.V) return;
  float M[C][4], acc[C][4];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) { M[c][q] = 2.f * kNeg; acc[c][q] = 0.f; }
  for (int j0 = jb; j0 < je; j0 += KB) {
    const int nb = min(KB, je - j0);
    int st[KB];
    float xh[KB][C][4];
    uint32_t xw[KB][C][2];
    gather_rt<C, KB>(a, G, j0, nb, g, st, xh, xw);
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

// Set-up slice k: boundary panels A_1, B_T at log 0 for the item's nodes; u_t = 1 and
// W_t = log2 K_L for its share of the states; U01 = U0T = 1 for its share of the triples.
__device__ void setup_item(const BatchInst &I, int k, int shift, bool restage) {
  const size_t pan = panel_of(I);
  float *bt_hi = I.b_hi + (size_t)(I.T - 2) * pan;
  lo_t *bt_lo = I.b_lo + (size_t)(I.T - 2) * pan;
  const int v0 = k * I.npi, v1 = min(I.V, v0 + I.npi);
  for (size_t e = (size_t)v0 * I.Lp + threadIdx.x; e < (size_t)v1 * I.Lp; e += kTickBlock) {
    I.a0_hi[e] = kNeg;
    I.a0_lo[e] = kLoZero;
    bt_hi[e] = kNeg;
    bt_lo[e] = kLoZero;
  }
  const int s0 = (int)((long long)k * I.S / I.n_items), s1 = (int)((long long)(k + 1) * I.S / I.n_items);
  for (int s = s0 + threadIdx.x; s < s1; s += kTickBlock) {
    for (int t = 2; t <= I.T - 1; ++t) {
      const size_t kq = (size_t)t * I.kl_stride + s;
      float wh, wl;
      float2 lu = make_float2(0.f, 0.f);
      if (restage) {                               // epsilon halved: log u doubles (exact)
        lu = I.lu[(size_t)t * I.S + s];
        lu = lu.x < kNegThresh ? make_float2(kNeg, 0.f) : make_float2(2.f * lu.x, 2.f * lu.y);
      }
      make_w(ldexpf(I.kl_hi[kq], -shift), ldexpf(I.kl_lo[kq], -shift), lu.x, lu.y, I.qs, wh, wl);
      I.lu[(size_t)t * I.S + s] = lu;
      I.w_hi[(size_t)t * I.S + s] = wh;
      I.w_lo[(size_t)t * I.S + s] = wl;
    }
  }
  const BndSide *sides[2] = {&I.src, &I.snk};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int n = sides[h]->n_tri;
    const int q0 = (int)((long long)k * n / I.n_items), q1 = (int)((long long)(k + 1) * n / I.n_items);
    for (int q = q0 + threadIdx.x; q < q1; q += kTickBlock)
      sides[h]->tri_logU[q] = restage ? 2.0 * sides[h]->tri_logU[q] : 0.0;
  }
}

// Boundary segments of slice k (segments k * kTickBlock + thread, strided by the item count).
__device__ __forceinline__ void bnd_item(const BndArgs &b, int k, int n_items, double &r0, double &r1, double &r2) {
  for (int sidx = k * kTickBlock + threadIdx.x; sidx < b.n_seg; sidx += n_items * kTickBlock)
    boundary_segment(b, sidx, r0, r1, r2);
}

// Boundary flows P = 2^(log2 U + msg) of the triples of slice k, both sides.
__device__ void flow_bnd_item(const BatchInst &I, int k) {
  const BndSide *sides[2] = {&I.src, &I.snk};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const BndSide &sd = *sides[h];
    const float *mh = h == 0 ? I.b_hi : a_hi_of(I, I.T - 1);
    const lo_t *ml = h == 0 ? I.b_lo : a_lo_of(I, I.T - 1);
    for (int q = k * kTickBlock + threadIdx.x; q < sd.n_tri; q += I.n_items * kTickBlock) {
      const size_t idx = (size_t)sd.tri_other[q] * I.Lp + sd.tri_l[q];
      if (mh[idx] < kNegThresh) { sd.tri_flow[q] = 0.0; continue; }
      const double msg = (double)mh[idx] + ((double)ml[idx] - 32768.0) * (double)I.qs.lo_unit;
      sd.tri_flow[q] = exp2(sd.tri_logU[q] + msg);
    }
  }
}

// The last item of an instance in this tick: reduce the items' partials (fixed order),
// fold them into the pass statistics, and advance the step sequence.
__device__ void finalise(const BatchInst &I, BatchCtl *c, const Phase &ph, float2 *s_red) {
  __threadfence();
  float2 fa = make_float2(0.f, 0.f), fb = fa, fd = fa;
  for (int q = threadIdx.x; q < I.n_items; q += kTickBlock) {
    const float2 x = to_ff(__ldcg(I.partials + 3 * q));
    const float2 y = to_ff(__ldcg(I.partials + 3 * q + 1));
    const float2 z = to_ff(__ldcg(I.partials + 3 * q + 2));
    ff_add(fa, x.x, x.y);
    ff_add(fb, y.x, y.y);
    ff_add(fd, z.x, z.y);
  }
  block_sum3(fa, fb, fd, s_red);
  if (threadIdx.x != 0) return;
  const double a = from_ff(fa), b = from_ff(fb), d = from_ff(fd);
  DevStats &st = c->stats;
  int status = c->status;
  int step = c->step + 1;
  switch (ph.kind) {
    case kPhSrc:
      st.src_resid = a; st.dual_src = b; st.bad = d;
      st.cap_viol = 0.0; st.dual_cap = 0.0;
      break;
    case kPhFwd:
      st.cap_viol += a; st.dual_cap += b;
      break;
    case kPhSnk:
      st.mass_snk = a; st.dual_snk = b; st.bad += d;
      break;
    case kPhFlowBnd:
      status = c->final_status;
      step = 0;
      break;
    default:
      break;
  }
  if (ph.pass_end) {
    const int passes = c->passes + 1;
    c->passes = passes;
    PassReport &r = c->report;
    r.src_resid_rel = st.src_resid / I.mass;
    r.cap_viol_rel = st.cap_viol / I.mass;
    const double eps_now = ldexp(I.eps, c->shift);
    r.dual_objective = -eps_now * st.mass_snk + eps_now * 0.69314718055994530942 * (st.dual_src + st.dual_snk + st.dual_cap);
    r.bad = st.bad;
    r.passes = passes;
    const double tol_now = c->shift > 0 ? I.stage_tol : I.tol;
    if (st.bad > 0.0) {
      status = kSlotInfeasible;
    } else if (isnan(r.src_resid_rel) || isnan(r.cap_viol_rel) || isnan(r.dual_objective)) {
      status = kSlotNumeric;
    } else if (c->shift > 0 && passes < I.max_passes) {
      if (r.src_resid_rel <= tol_now && r.cap_viol_rel <= tol_now) {
        c->shift -= 1;                              // next stage: epsilon halved, set-up rescales
        step = 0;
      } else {
        step = I.T;                                 // next pass of this stage
      }
    } else if (c->shift == 0 && r.src_resid_rel <= tol_now && r.cap_viol_rel <= tol_now) {
      status = kSlotFlows;
      c->final_status = kSlotConverged;
      step = 0;
    } else if (passes >= I.max_passes) {
      status = kSlotFlows;
      c->final_status = kSlotNotConverged;
      step = 0;
    } else {
      step = I.T;                                   // next pass
    }
  }
  c->counter = 0u;
  c->ticks += 1;
  c->step = step;
  c->status = status;
}

// Fetch-and-add with release (orders this thread's earlier writes, here the item's partial
// sums, before the increment) and acquire (the last item then sees every item's partials).
__device__ __forceinline__ unsigned int atomic_add_acq_rel(unsigned int *p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Warp 0 stages the header (slot, item, status, step) and the instance description of
// item `it` into shared memory; w is the item's (slot, index) on every lane.
__device__ __forceinline__ void stage_item(const TickArgs &ta, int2 w, int *hdr, BatchInst *si) {
  const int lane = threadIdx.x & 31;
  constexpr int kWords = (int)(sizeof(BatchInst) / 16);
  static_assert(kWords <= 32, "one 16-byte word per lane");
  if (lane < kWords)
    reinterpret_cast<int4 *>(si)[lane] = __ldg(reinterpret_cast<const int4 *>(ta.inst + w.x) + lane);
  if (lane == 0) {
    const BatchCtl *c = ta.ctl + w.x;
    hdr[0] = w.x;
    hdr[1] = w.y;
    hdr[2] = c->status;
    hdr[3] = c->step;
    hdr[4] = c->shift;
    hdr[5] = c->passes;
  }
}

}  // namespace

__global__ void __launch_bounds__(kTickBlock, 2) k_batch_tick(const TickArgs ta) {
  __shared__ BatchInst s_inst[2];                  // current and next item's instance
  __shared__ int s_hdr[2][8];
  __shared__ int s_last;
  __shared__ float2 s_red[3 * (kTickBlock / 32)];
  __shared__ float2 s_w[kTickBlock][6];            // W of the in-states of each node (fwd)
  const int n = *ta.n_items;
  int it = blockIdx.x;                             // items it, it + grid, it + 2 grid, ...
  if (it >= n) return;
  if (threadIdx.x < 32) {
    int2 w = make_int2(0, 0);
    if (threadIdx.x == 0) w = ta.items[it];
    w.x = __shfl_sync(0xffffffffu, w.x, 0);
    w.y = __shfl_sync(0xffffffffu, w.y, 0);
    stage_item(ta, w, s_hdr[0], &s_inst[0]);
  }
  __syncthreads();
  int buf = 0;
  for (;;) {
    const int nxt = it + gridDim.x;
    int2 wn = make_int2(0, 0);
    if (threadIdx.x == 0 && nxt < n) wn = ta.items[nxt];   // used after this item's work
    const int slot = s_hdr[buf][0], k = s_hdr[buf][1], status = s_hdr[buf][2];
    const int c_shift = s_hdr[buf][4], c_passes = s_hdr[buf][5];
    const BatchInst &I = s_inst[buf];
    const bool running = status == kSlotRunning || status == kSlotFlows;
    const Phase ph = decode_phase(status, s_hdr[buf][3], I.T);
    BatchCtl *c = ta.ctl + slot;
    if (running) {
      const int G = I.G, C = I.C;
      double r0 = 0.0, r1 = 0.0, r2 = 0.0;          // boundary steps (FP64)
      float fviol = 0.f;                             // forward steps: excess, dual (float-float)
      float2 fdual = make_float2(0.f, 0.f);
      switch (ph.kind) {
        case kPhSetup:
          setup_item(I, k, c_shift, c_passes > 0);
          break;
        case kPhInitBnd:
          bnd_item(bnd_of(I, true, 1), k, I.n_items, r0, r1, r2);
          bnd_item(bnd_of(I, false, 1), k, I.n_items, r0, r1, r2);
          break;
        case kPhSrc:
          bnd_item(bnd_of(I, true, 0), k, I.n_items, r0, r1, r2);
          break;
        case kPhSnk:
          bnd_item(bnd_of(I, false, 0), k, I.n_items, r0, r1, r2);
          break;
        case kPhFwd:
        case kPhFlowFwd:
        case kPhBwd: {
          const bool fwd = ph.kind != kPhBwd;
          const StepArgs a = step_of(I, fwd, ph.t, ph.kind == kPhFlowFwd ? 1 : 0, c_shift);
          const int v_end = min(I.V, (k + 1) * I.npi);
          const int nib = threadIdx.x / G;
          int v0 = k * I.npi;
          int vv = min(v0 + nib, I.V - 1);
          int jb = a.ptr[vv], je = a.ptr[vv + 1];
          for (; v0 < v_end; v0 += I.npb) {
            // CSR range of this thread's node in the next round, loaded ahead
            const int vn = min(v0 + I.npb + nib, I.V - 1);
            int jbn = 0, jen = 0;
            if (v0 + I.npb < v_end) { jbn = a.ptr[vn]; jen = a.ptr[vn + 1]; }
            if (fwd) {
              if (C == 1) fwd_round<1>(a, G, v0, jb, je, s_w, fviol, fdual);
              else fwd_round<2>(a, G, v0, jb, je, s_w, fviol, fdual);
            } else {
              if (C == 1) bwd_round<1>(a, G, v0, jb, je);
              else bwd_round<2>(a, G, v0, jb, je);
            }
            jb = jbn;
            je = jen;
          }
          break;
        }
        case kPhFlowBnd:
          flow_bnd_item(I, k);
          break;
        default:
          break;
      }
      const bool bnd = ph.kind == kPhSrc || ph.kind == kPhSnk || ph.kind == kPhInitBnd;
      float2 p0 = bnd ? to_ff(r0) : make_float2(fviol, 0.f);
      float2 p1 = bnd ? to_ff(r1) : fdual;
      float2 p2 = bnd ? to_ff(r2) : make_float2(0.f, 0.f);
      block_sum3(p0, p1, p2, s_red);
      if (threadIdx.x == 0) {
        I.partials[3 * k] = from_ff(p0);
        I.partials[3 * k + 1] = from_ff(p1);
        I.partials[3 * k + 2] = from_ff(p2);
        s_last = atomic_add_acq_rel(&c->counter, 1u) == (unsigned)(I.n_items - 1);
      }
    }
    if (threadIdx.x < 32 && nxt < n) {
      wn.x = __shfl_sync(0xffffffffu, wn.x, 0);
      wn.y = __shfl_sync(0xffffffffu, wn.y, 0);
      stage_item(ta, wn, s_hdr[buf ^ 1], &s_inst[buf ^ 1]);
    }
    __syncthreads();
    if (running && s_last) finalise(I, c, ph, s_red);
    if (nxt >= n) break;
    it = nxt;
    buf ^= 1;
  }
}

// Grid of the persistent tick kernel: resident blocks per SM times the SM count.
cudaError_t batch_tick_grid(int *grid) {
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_tick, kTickBlock, 0);
  if (e != cudaSuccess) return e;
  *grid = n_sm * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

cudaError_t launch_batch_tick(const TickArgs &ta, int grid, cudaStream_t s) {
  k_batch_tick<<<grid, kTickBlock, 0, s>>>(ta);
  return cudaGetLastError();
}

}  // namespace ots

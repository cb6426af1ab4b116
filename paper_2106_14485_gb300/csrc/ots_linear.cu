// ots_linear.cu -- the single-commodity problem (L = 1, Section 4.2) with FP32 messages in
// the linear domain, one thread block per problem (a cluster of up to 8 blocks for problems of
// more than 4096 states) for whole runs of passes.
//
// Algorithm 1 works with the messages themselves (products of K and the duals), not their
// logarithms; Algorithm 2 at L = 1 is the same iteration (the boundary duals absorb the costs of
// t = 1 and t = T).  In FP32 the plain form loses every entry more than about 2^-126 below the
// largest one, which at small epsilon is most of them.  Here each message keeps its own
// power-of-two scale per node and interval, and the duals u_t one per state:
//   A_t[v] = a_t[v] 2^alpha_t[v],   B_t[v] = b_t[v] 2^beta_t[v],   u_t(i) = w_t(i) 2^nu_t(i)
// (a, b, w: FP32; alpha, beta: FP32 scales; nu: integers).  The scales are folded into per-state
// factors once per rescaling (float-float exponents, one exp2f each):
//   Gf_t(i) = 2^(alpha_{t-1}[tail i] + log2 K(i) + nu_t(i) - alpha_t[head i])
//   Gb_t(i) = 2^(beta_{t+1}[head i] + log2 K(i) + nu_t(i) - beta_t[tail i])
//   Fc_t(i) = 2^(alpha_{t-1}[tail i] + beta_{t+1}[head i] + log2 K(i) + nu_t(i)),   Dc_t(i) = d_t(i) / Fc_t(i)
// and a pass of Algorithm 2 (node-level form: A_t[v] sums the states with head v, B_t[v] the
// states with tail v) is then, per state and interval, one multiply-add in each sweep and, on a
// capacitated state, one divide:
//   backward   b_t[v] = sum_{tail j = v} b_{t+1}[head j] w_t(j) Gb_t(j)
//   capacity   w_t(i) <- min(Dc_t(i) / (a_{t-1}[tail i] b_{t+1}[head i]), 2^-nu_t(i))
//   forward    a_t[v] = sum_{head i = v} a_{t-1}[tail i] w_t(i) Gf_t(i)
// (the capacity update is u_t <- min(d_t / P_t(u_t = 1), 1) of Algorithm 2, written in the scaled
// quantities).  The boundary duals stay float-float base-2 logarithms: U01 <- R01 / Psi_1 with
// Psi_1(i) = B_2[head i], U0T <- R0T / hatPsi_T with hatPsi_T(j) = A_{T-1}[tail j].
//
// The scales are taken from the messages themselves by a sweep in FP32 log arithmetic at the
// current duals (no update; the iterate does not change), so that after it every a and b is 1.
// A pass in which some scaled value leaves [2^-60, 2^60] (or is not finite) is thrown away and
// run again in FP32 log arithmetic (with updates), which re-takes the scales; one that stays
// inside but leaves [2^-30, 2^30] re-takes them before the next pass.  The measures are those
// of Algorithm 2 (relative source mismatch before the U01 update, capacity residual
// sum |P_t after - P_t before|), summed in float-float in a fixed order.
//
// A step is two phases: one thread per state entry forms its term, then one thread per node adds
// its entries' terms from shared memory.  On a cluster every block owns a node range and the
// state entries of those nodes, keeps the step rows in its shared memory (its own nodes' entries
// written, the others read from the owning block through distributed shared memory), and the
// blocks meet at a cluster barrier between steps; every block takes the same decisions from sums
// that all of them add in rank order.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <algorithm>
#include <memory>
#include <vector>

#include "ots_internal.h"

namespace ots {

struct LinArgs {
  int V, S, T, krs, drs;             // krs / drs: row strides of kappa / logd (S if per interval, else 0)
  int n_src, n_snk, n_sseg, n_zseg;
  int mode;                          // arrays in shared memory: 0 none, 1 index arrays, 2 all (see lin_layout)
  float mass;                        // sum of R01
  const int *in_ptr, *in_tail, *in_head, *in_state, *in_to_out;   // in-CSR by head node (entry k = state in_state[k])
  const int *out_ptr, *out_tail, *out_head, *out_to_in;           // out-CSR by tail node
  const float2 *kappa;               // [rows][S] log2 K of in-entry k (float-float); x = -inf: closed
  const float2 *logd;                // [rows][S] log2 d of in-entry k; x = +inf: no capacity, -inf: d = 0
  float *Gf, *Gb, *Dc, *Fc;          // [(T+1) S] by in-entry
  int *nu;                           // [(T+1) S] by in-entry
  float *w[2];                       // [(T+1) S] by in-entry: w_t (two buffers: current, next)
  float *gbw;                        // [(T+1) S] by out-entry: Gb_t w_t of the state
  float *alpha, *beta, *bm;          // [(T+1) V]: scales and the scaled backward messages
  const int *sseg_node, *sseg_ptr, *zseg_node, *zseg_ptr;   // boundary entries grouped by node
  const float *src_R, *snk_R;        // per entry
  const float2 *src_logR, *snk_logR; // per entry, log2 R (float-float)
  float2 *lU01[2], *lU0T[2];         // per entry, log2 U01 / U0T (float-float, two buffers)
  const int *src_tri, *snk_tri;      // entry -> boundary triple of the problem
  float2 *p_logu;                    // problem's log2 u_t [(T+1) S] by state (float-float)
  double *p_src_logU, *p_snk_logU;   // problem's log2 U01 / U0T per triple
  float2 *cred;                      // [4][16] cluster reduction slots
  LinReport *rep;
  int cur, done;                     // state kept between launches
};

// Shared-memory layout of one problem (offsets in 4-byte words, 16-byte aligned): always the two
// message rows and one value per entry (the per-entry terms of a step before the node sums);
// mode >= 1 adds the index arrays, mode 2 every per-(t, entry) and per-(t, node) array.
struct LinLayout {
  size_t rows, c, in_ptr, out_ptr, in_tail, in_head, in_to_out, out_head;
  size_t Gf, Gb, Dc, Fc, nu, w0, w1, gbw, bm, alpha, beta, words;
};

__host__ __device__ inline size_t lin_take(size_t &o, size_t n) {
  const size_t r = o;
  o += (n + 3) & ~(size_t)3;
  return r;
}

__host__ __device__ inline LinLayout lin_layout(int V, int S, int T, int mode) {
  LinLayout L{};
  size_t o = 0;
  L.rows = lin_take(o, 2 * (size_t)V);
  L.c = lin_take(o, (size_t)S);
  if (mode >= 1) {
    L.in_ptr = lin_take(o, (size_t)V + 1);
    L.out_ptr = lin_take(o, (size_t)V + 1);
    L.in_tail = lin_take(o, (size_t)S);
    L.in_head = lin_take(o, (size_t)S);
    L.in_to_out = lin_take(o, (size_t)S);
    L.out_head = lin_take(o, (size_t)S);
  }
  if (mode >= 2) {
    const size_t TS = (size_t)(T + 1) * S, TV = (size_t)(T + 1) * V;
    L.Gf = lin_take(o, TS); L.Gb = lin_take(o, TS); L.Dc = lin_take(o, TS); L.Fc = lin_take(o, TS);
    L.nu = lin_take(o, TS); L.w0 = lin_take(o, TS); L.w1 = lin_take(o, TS); L.gbw = lin_take(o, TS);
    L.bm = lin_take(o, TV); L.alpha = lin_take(o, TV); L.beta = lin_take(o, TV);
  }
  L.words = o;
  return L;
}

namespace {

constexpr int kLinThreads = 512;
constexpr int kBatch = 4;   // state entries per thread whose loads are in flight together
constexpr float kLost = 0x1p60f, kDrift = 0x1p30f;
constexpr float kLn2f = 0.693147180559945309f;
constexpr float kNegLog = -1e30f;    // log 0 in the problem's float-float duals

// Where the working arrays of a problem live for one launch (shared or global memory).
struct Ptrs {
  const int *in_ptr, *out_ptr, *in_tail, *in_head, *in_to_out, *out_head;
  float *Gf, *Gb, *Dc, *Fc, *w[2], *gbw, *bm, *alpha, *beta, *rows, *c;
  int *nu;
};

__device__ Ptrs make_ptrs(const LinArgs &a, float *dyn) {
  const LinLayout L = lin_layout(a.V, a.S, a.T, a.mode);
  Ptrs P;
  P.rows = dyn + L.rows;
  P.c = dyn + L.c;
  if (a.mode >= 1) {
    P.in_ptr = (const int *)(dyn + L.in_ptr); P.out_ptr = (const int *)(dyn + L.out_ptr);
    P.in_tail = (const int *)(dyn + L.in_tail); P.in_head = (const int *)(dyn + L.in_head);
    P.in_to_out = (const int *)(dyn + L.in_to_out); P.out_head = (const int *)(dyn + L.out_head);
  } else {
    P.in_ptr = a.in_ptr; P.out_ptr = a.out_ptr; P.in_tail = a.in_tail; P.in_head = a.in_head;
    P.in_to_out = a.in_to_out; P.out_head = a.out_head;
  }
  if (a.mode >= 2) {
    P.Gf = dyn + L.Gf; P.Gb = dyn + L.Gb; P.Dc = dyn + L.Dc; P.Fc = dyn + L.Fc; P.nu = (int *)(dyn + L.nu);
    P.w[0] = dyn + L.w0; P.w[1] = dyn + L.w1; P.gbw = dyn + L.gbw; P.bm = dyn + L.bm;
    P.alpha = dyn + L.alpha; P.beta = dyn + L.beta;
  } else {
    P.Gf = a.Gf; P.Gb = a.Gb; P.Dc = a.Dc; P.Fc = a.Fc; P.nu = a.nu; P.w[0] = a.w[0]; P.w[1] = a.w[1];
    P.gbw = a.gbw; P.bm = a.bm; P.alpha = a.alpha; P.beta = a.beta;
  }
  return P;
}

__device__ void copy_words(void *dst, const void *src, size_t n) {
  const int *s = (const int *)src;
  int *d = (int *)dst;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

// Index arrays (mode >= 1) and the duals' working copies (mode 2) into shared memory.
__device__ void stage_in(const LinArgs &a, const Ptrs &P, bool duals) {
  const int V = a.V, S = a.S;
  if (a.mode >= 1) {
    copy_words((void *)P.in_ptr, a.in_ptr, V + 1);
    copy_words((void *)P.out_ptr, a.out_ptr, V + 1);
    copy_words((void *)P.in_tail, a.in_tail, S);
    copy_words((void *)P.in_head, a.in_head, S);
    copy_words((void *)P.in_to_out, a.in_to_out, S);
    copy_words((void *)P.out_head, a.out_head, S);
  }
  if (a.mode >= 2 && duals) {
    const size_t TS = (size_t)(a.T + 1) * S;
    copy_words(P.w[0], a.w[0], TS);
    copy_words(P.w[1], a.w[1], TS);
    copy_words(P.nu, a.nu, TS);
  }
  __syncthreads();
}

// The duals' working copies back to global memory (mode 2), for the next launch.
__device__ void stage_out(const LinArgs &a, const Ptrs &P) {
  if (a.mode >= 2) {
    const size_t TS = (size_t)(a.T + 1) * a.S;
    copy_words(a.w[0], P.w[0], TS);
    copy_words(a.w[1], P.w[1], TS);
    copy_words(a.nu, P.nu, TS);
  }
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct FF {
  float h, l;
};

__device__ __forceinline__ FF ff_add(FF a, float b) {
  FF r;
  float e;
  two_sum(a.h, b, r.h, e);
  r.l = __fadd_rn(a.l, e);
  return r;
}

__device__ __forceinline__ FF ff_add(FF a, float2 b) {
  FF r = ff_add(a, b.x);
  r.l = __fadd_rn(r.l, b.y);
  return r;
}

// a + b for float-float values, renormalised (the boundary duals and the measures)
__device__ __forceinline__ FF ff_sum(FF a, FF b) {
  FF r;
  float e;
  two_sum(a.h, b.h, r.h, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  two_sum(r.h, e, r.h, r.l);
  return r;
}

__device__ __forceinline__ FF ff_of(float2 x) { return FF{x.x, x.y}; }
__device__ __forceinline__ float2 f2_of(FF x) { return make_float2(x.h, x.l); }
__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.h, -x.l}; }

// log2 x of a positive float as float-float: the exponent exactly, log2f of the mantissa in [1/2, 1)
__device__ __forceinline__ FF ff_log2(float x) {
  int e;
  const float m = frexpf(x, &e);
  FF r;
  two_sum((float)e, log2f(m), r.h, r.l);
  return r;
}

// 2^(h + l + n) for a float-float exponent (h, l) (|l| small) and an integer n: the integer part of
// h is applied exactly by ldexpf, the rest by exp2f on [-1/2, 1/2] and a first-order term in l.
__device__ __forceinline__ float exp2_ff(FF e, int n) {
  float r = fminf(fmaxf(rintf(e.h), -1024.f), 1024.f);
  const float f = __fsub_rn(e.h, r);
  const float y = exp2f(f);
  const float z = fmaf(y, e.l * kLn2f, y);
  const int k = max(min((int)r + n, 2048), -2048);
  return ldexpf(z, k);
}

// Block reductions in a fixed order (all threads get the result).  Sums are float-float: FP64 on
// this part issues a warp instruction every 16 cycles, too slow for per-pass reductions.
__device__ FF block_sum(FF v, float2 *red) {
  for (int o = 16; o; o >>= 1) {
    const FF w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    v = ff_sum(v, w);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f2_of(v);
  __syncthreads();
  FF s{0.f, 0.f};
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = ff_sum(s, ff_of(red[i]));
  return s;
}

__device__ float block_max(float v, float *red) {
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = red[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) s = fmaxf(s, red[i]);
  return s;
}

// The part of a problem one block owns: a node range, the state entries of those nodes (in-CSR
// range for the forward step, out-CSR range for the backward step) and the boundary segments of
// those nodes.  A problem on one block owns everything; on a cluster of R blocks the node ranges
// split the in-entries evenly.
struct Part {
  int rank, R;
  int v0, v1, in0, in1, out0, out1, s0, s1, z0, z1;
  int slot;                          // next reduction slot (cluster)
  const int *vb;                     // [9] first node of every rank (vb[R] = V), in shared memory
};

__device__ int first_node_at(const int *ptr, int V, int target) {   // smallest v with ptr[v] >= target
  int lo = 0, hi = V;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ptr[mid] < target) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ int first_seg_at(const int *node, int n, int v) {        // first segment whose node >= v
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (node[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ Part make_part(const LinArgs &a, int rank, int R, int *vb) {
  Part p;
  p.rank = rank;
  p.R = R;
  p.slot = 0;
  const long long S = a.S;
  for (int r = 0; r <= 8; ++r)
    vb[r] = r == 0 ? 0 : (r >= R ? a.V : first_node_at(a.in_ptr, a.V, (int)(S * r / R)));
  p.vb = vb;
  p.v0 = vb[rank];
  p.v1 = vb[rank + 1];
  p.in0 = a.in_ptr[p.v0];
  p.in1 = a.in_ptr[p.v1];
  p.out0 = a.out_ptr[p.v0];
  p.out1 = a.out_ptr[p.v1];
  p.s0 = first_seg_at(a.sseg_node, a.n_sseg, p.v0);
  p.s1 = first_seg_at(a.sseg_node, a.n_sseg, p.v1);
  p.z0 = first_seg_at(a.zseg_node, a.n_zseg, p.v0);
  p.z1 = first_seg_at(a.zseg_node, a.n_zseg, p.v1);
  return p;
}

// Barrier between the steps: the block, or every block of the cluster (release / acquire at
// cluster scope, so the rows one block wrote are seen by the others).
template <bool CL>
__device__ __forceinline__ void step_sync() {
  if constexpr (CL) {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
  } else {
    __syncthreads();
  }
}

// Load of a value another block of the cluster may have written (L2, not a stale L1 line).
template <bool CL, typename X>
__device__ __forceinline__ X ldx(const X *p) {
  if constexpr (CL) return __ldcg(p);
  else return *p;
}

// Value of node x in a step row.  On a cluster every block keeps a whole row array in its shared
// memory but writes only the entries of its own nodes; the entry of node x is read from the shared
// memory of the block that owns x (distributed shared memory, same offset in every block).
template <bool CL>
__device__ __forceinline__ float ld_row(const float *rows, int x, const Part &pt) {
  if constexpr (!CL) {
    return rows[x];
  } else {
    int r = 0;
#pragma unroll
    for (int k = 1; k < 8; ++k) r += (k < pt.R && x >= pt.vb[k]) ? 1 : 0;
    const uint32_t la = (uint32_t)__cvta_generic_to_shared(rows + x);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(r));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
    return v;
  }
}

// Sum / maximum over the whole problem: the block's value, then (cluster) every block adds the R
// block values in rank order from a slot in global memory, so every block gets the same result.
template <bool CL>
__device__ FF part_sum(FF v, float2 *red, float2 *cred, Part &pt) {
  const FF b = block_sum(v, red);
  if constexpr (!CL) {
    return b;
  } else {
    float2 *sl = cred + (pt.slot & 3) * 16;
    ++pt.slot;
    if (threadIdx.x == 0) sl[pt.rank] = f2_of(b);
    step_sync<true>();
    FF s{0.f, 0.f};
    for (int r = 0; r < pt.R; ++r) s = ff_sum(s, ff_of(__ldcg(sl + r)));
    return s;
  }
}

template <bool CL>
__device__ float part_max(float v, float *redf, float2 *cred, Part &pt) {
  const float b = block_max(v, redf);
  if constexpr (!CL) {
    return b;
  } else {
    float2 *sl = cred + (pt.slot & 3) * 16;
    ++pt.slot;
    if (threadIdx.x == 0) sl[pt.rank] = make_float2(b, 0.f);
    step_sync<true>();
    float s = 0.f;
    for (int r = 0; r < pt.R; ++r) s = fmaxf(s, __ldcg(sl + r).x);
    return s;
  }
}

// Range of the scaled values a pass produced (non-zero ones; any non-finite value counts as
// out of range).
struct Range {
  float hi = 0.f, lo = FLT_MAX;
  bool bad = false;
  __device__ __forceinline__ void see(float x) {
    if (!(x >= 0.f && x <= FLT_MAX)) bad = true;
    else if (x > 0.f) { hi = fmaxf(hi, x); lo = fminf(lo, x); }
  }
};

// |P_new - P_old| of one capacity update with P = 2^(log2 u + ls) (FP32 terms).
__device__ __forceinline__ float flow_change(float lo, float ln, float ls) {
  if (lo == -INFINITY && ln == -INFINITY) return 0.f;
  if (lo == -INFINITY) return exp2f(ln + ls);
  if (ln == -INFINITY) return exp2f(lo + ls);
  return exp2f(lo + ls) * fabsf(exp2f(ln - lo) - 1.f);
}

__device__ __forceinline__ double dbl(float2 x) { return (double)x.x + (double)x.y; }
__device__ __forceinline__ float2 split(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// log2 of the sum of 2^c[k] over k in [k0, k1) (two passes over shared memory; log 0 = -inf)
__device__ __forceinline__ float lse_range(const float *c, int k0, int k1) {
  float m = -INFINITY;
  for (int k = k0; k < k1; ++k) m = fmaxf(m, c[k]);
  if (!(m > -INFINITY)) return -INFINITY;
  float sum = 0.f;
  for (int k = k0; k < k1; ++k) sum += exp2f(c[k] - m);
  return m + log2f(sum);
}

// log2 u_t of an entry from its stored pair (w, nu): 0 without a capacity, -inf for u = 0
__device__ __forceinline__ float log2_u(float2 ld, float wv, int nu) {
  if (ld.x == INFINITY) return 0.f;
  return wv > 0.f ? (float)nu + log2f(wv) : -INFINITY;
}

// Scale sweep (update = false) or a whole pass of Algorithm 2 in FP32 log arithmetic
// (update = true): alpha_t, beta_t become the base-2 logarithms of the messages.  With updates,
// the new duals go to the next buffers (w[nxt], lU01/lU0T[nxt], nu in place) and the measures
// to *mism, *resid; returns an ots_status (OTS_ERR_INFEASIBLE if a boundary state has no path).
// Same two phases per step as the linear pass (per-entry terms, then per-node log-sum-exp).
template <bool CL>
__device__ int log_sweep(const LinArgs &a, const Ptrs &P, Part &pt, int cur, bool update, FF *mism_out, FF *res_out,
                         float2 *red) {
  const int V = a.V, S = a.S, T = a.T, nxt = cur ^ 1, nt = blockDim.x;
  float *rp = P.rows, *rc = P.rows + V, *c = P.c;
  int bad = 0;
  FF mism{0.f, 0.f}, res{0.f, 0.f};
  // beta_T[v] = log2 sum_{sink j, tail j = v} U0T(j)
  for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) rp[v] = -INFINITY;
  __syncthreads();
  for (int s = pt.z0 + threadIdx.x; s < pt.z1; s += nt) {
    // (this sweep runs once per rescaling: FP64 for the few boundary entries)
    double m = -INFINITY;
    for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) m = fmax(m, dbl(a.lU0T[cur][e]));
    double acc = 0.0;
    for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) acc += exp2(dbl(a.lU0T[cur][e]) - m);
    rp[a.zseg_node[s]] = (float)(m + log2(acc));
  }
  __syncthreads();
  for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) P.beta[(size_t)T * V + v] = rp[v];
  step_sync<CL>();
  // beta_t[v] = log2 sum_{tail j = v} 2^(beta_{t+1}[head j] + log2 K(j) + log2 u_t(j)),  t = T-1..2
  for (int t = T - 1; t >= 2; --t) {
    for (int k0 = pt.out0 + threadIdx.x; k0 < pt.out1; k0 += kBatch * nt) {
      int hd[kBatch], ki[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j * nt;
        hd[j] = k < pt.out1 ? P.out_head[k] : 0;
        ki[j] = k < pt.out1 ? a.out_to_in[k] : 0;
      }
      float2 kap[kBatch], ld[kBatch];
      float wv[kBatch];
      int nu[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const size_t q = (size_t)t * S + ki[j];
        kap[j] = a.kappa[(size_t)t * a.krs + ki[j]];
        ld[j] = a.logd[(size_t)t * a.drs + ki[j]];
        wv[j] = ldx<CL>(P.w[cur] + q);
        nu[j] = ldx<CL>(P.nu + q);
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j * nt;
        if (k < pt.out1) c[k] = ld_row<CL>(rp, hd[j], pt) + kap[j].x + log2_u(ld[j], wv[j], nu[j]);
      }
    }
    __syncthreads();
    for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) {
      const float r = lse_range(c, P.out_ptr[v], P.out_ptr[v + 1]);
      rc[v] = r;
      P.beta[(size_t)t * V + v] = r;
    }
    step_sync<CL>();
    float *tmp = rp; rp = rc; rc = tmp;
  }
  // source update U01 <- R01 / Psi_1, then alpha_1[v] = log2 sum_{source i, head i = v} U01(i)
  const int su = update ? nxt : cur;
  for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) rc[v] = -INFINITY;
  __syncthreads();
  for (int s = pt.s0 + threadIdx.x; s < pt.s1; s += nt) {
    const int v = a.sseg_node[s];
    if (update) {
      const double p1 = (double)ldx<CL>(P.beta + (size_t)2 * V + v);
      for (int e = a.sseg_ptr[s]; e < a.sseg_ptr[s + 1]; ++e) {
        if (!(p1 > -INFINITY)) { bad = 1; a.lU01[nxt][e] = a.lU01[cur][e]; continue; }
        const double ln = dbl(a.src_logR[e]) - p1;
        mism = ff_add(mism, (float)(a.src_R[e] * fabs(exp2(dbl(a.lU01[cur][e]) - ln) - 1.0)));
        a.lU01[nxt][e] = split(ln);
      }
    }
    double m = -INFINITY;
    for (int e = a.sseg_ptr[s]; e < a.sseg_ptr[s + 1]; ++e) m = fmax(m, dbl(a.lU01[su][e]));
    double acc = 0.0;
    for (int e = a.sseg_ptr[s]; e < a.sseg_ptr[s + 1]; ++e) acc += exp2(dbl(a.lU01[su][e]) - m);
    rc[v] = (float)(m + log2(acc));
  }
  __syncthreads();
  { float *tmp = rp; rp = rc; rc = tmp; }
  for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) P.alpha[(size_t)V + v] = rp[v];
  step_sync<CL>();
  // forward: capacity update of u_t (update) and alpha_t[v] = log2 sum_{head i = v} 2^(alpha_{t-1}[tail i]
  // + log2 K(i) + log2 u_t(i)),  t = 2..T-1
  for (int t = 2; t <= T - 1; ++t) {
    const size_t o = (size_t)t * S;
    float rsum = 0.f;
    for (int k0 = pt.in0 + threadIdx.x; k0 < pt.in1; k0 += kBatch * nt) {
      int ti[kBatch], hi[kBatch], nu[kBatch];
      float2 kap[kBatch], ld[kBatch];
      float wv[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j * nt;
        const bool in = k < pt.in1;
        ti[j] = in ? P.in_tail[k] : 0;
        hi[j] = in ? P.in_head[k] : 0;
        kap[j] = in ? a.kappa[(size_t)t * a.krs + k] : make_float2(-INFINITY, 0.f);
        ld[j] = in ? a.logd[(size_t)t * a.drs + k] : make_float2(INFINITY, 0.f);
        wv[j] = in ? P.w[cur][o + k] : 1.f;
        nu[j] = in ? P.nu[o + k] : 0;
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j * nt;
        if (k >= pt.in1) continue;
        const float al = ld_row<CL>(rp, ti[j], pt);
        float lu = log2_u(ld[j], wv[j], nu[j]);
        if (update && ld[j].x != INFINITY) {
          const float ls = al + ldx<CL>(P.beta + (size_t)(t + 1) * V + hi[j]) + kap[j].x;
          float ln = 0.f;
          if (ls > -INFINITY) {
            ln = ld[j].x == -INFINITY ? -INFINITY : fminf(ld[j].x - ls, 0.f);
            rsum += flow_change(lu, ln, ls);
          }
          if (ln == -INFINITY) { P.w[nxt][o + k] = 0.f; P.nu[o + k] = 0; }
          else { const float n = floorf(ln); P.w[nxt][o + k] = exp2f(ln - n); P.nu[o + k] = (int)n; }
          lu = ln;
        }
        c[k] = al + kap[j].x + lu;
      }
    }
    res = ff_add(res, rsum);
    __syncthreads();
    for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) {
      const float r = lse_range(c, P.in_ptr[v], P.in_ptr[v + 1]);
      rc[v] = r;
      P.alpha[(size_t)t * V + v] = r;
    }
    step_sync<CL>();
    float *tmp = rp; rp = rc; rc = tmp;
  }
  // sink update U0T <- R0T / hatPsi_T
  if (update) {
    for (int s = pt.z0 + threadIdx.x; s < pt.z1; s += nt) {
      const double p = (double)rp[a.zseg_node[s]];   // own node
      for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) {
        if (!(p > -INFINITY)) { bad = 1; a.lU0T[nxt][e] = a.lU0T[cur][e]; continue; }
        a.lU0T[nxt][e] = split(dbl(a.snk_logR[e]) - p);
      }
    }
  }
  __syncthreads();
  const FF ms = part_sum<CL>(mism, red, a.cred, pt);
  const FF rs = part_sum<CL>(res, red, a.cred, pt);
  const FF bd = part_sum<CL>(FF{(float)bad, 0.f}, red, a.cred, pt);
  if (mism_out) *mism_out = ms;
  if (res_out) *res_out = rs;
  return bd.h > 0.f ? OTS_ERR_INFEASIBLE : OTS_OK;
}

// Scale fold: w_t(i) = m 2^e with m in [1/2, 1) -> w = m, nu += e (exact).  Then the per-state
// factors Gf, Gb, Dc, Fc and the backward weights gbw = Gb w from the current scales (entries of
// the block's own nodes).
template <bool CL>
__device__ void rebuild(const LinArgs &a, const Ptrs &P, const Part &pt, int cur) {
  const int V = a.V, S = a.S, T = a.T;
  const int nown = pt.in1 - pt.in0;
  const int n = (T - 2) * nown;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int t = 2 + idx / nown, k = pt.in0 + idx - (t - 2) * nown;
    const size_t q = (size_t)t * S + k;
    const float2 kap = a.kappa[(size_t)t * a.krs + k];
    const float2 ld = a.logd[(size_t)t * a.drs + k];
    const int y = P.in_tail[k], v = P.in_head[k];
    float wv = P.w[cur][q];
    int nu = P.nu[q];
    if (ld.x != INFINITY && wv > 0.f) {
      int e;
      wv = frexpf(wv, &e);
      nu += e;
      P.w[cur][q] = wv;
      P.nu[q] = nu;
    }
    const float al0 = ldx<CL>(P.alpha + (size_t)(t - 1) * V + y), al1 = ldx<CL>(P.alpha + (size_t)t * V + v);
    const float be1 = ldx<CL>(P.beta + (size_t)(t + 1) * V + v), be0 = ldx<CL>(P.beta + (size_t)t * V + y);
    const bool open = kap.x > -INFINITY;
    float gf = 0.f, gb = 0.f;
    if (open && al0 > -INFINITY && al1 > -INFINITY) gf = exp2_ff(ff_add(ff_add(FF{al0, 0.f}, -al1), kap), nu);
    if (open && be1 > -INFINITY && be0 > -INFINITY) gb = exp2_ff(ff_add(ff_add(FF{be1, 0.f}, -be0), kap), nu);
    P.Gf[q] = gf;
    P.Gb[q] = gb;
    P.gbw[(size_t)t * S + P.in_to_out[k]] = gb * wv;
    if (ld.x == INFINITY) {
      P.Dc[q] = INFINITY;   // no capacity: w stays 1
      P.Fc[q] = 0.f;
    } else {
      float fc = 0.f, dc = FLT_MAX;
      if (open && al0 > -INFINITY && be1 > -INFINITY) {
        const FF e = ff_add(ff_add(FF{al0, 0.f}, be1), kap);
        fc = fminf(exp2_ff(e, nu), FLT_MAX);
        if (ld.x == -INFINITY) dc = 0.f;
        else {
          FF g = ff_add(FF{ld.x, ld.y}, -e.h);
          g.l = __fsub_rn(g.l, e.l);
          dc = fminf(exp2_ff(g, -nu), FLT_MAX);
        }
      }
      P.Fc[q] = fc;
      P.Dc[q] = dc;
    }
  }
  step_sync<CL>();
}

// One pass of Algorithm 2 on the scaled quantities; new duals to the next buffers.  Each step
// has two phases: one thread per state entry computes its term (independent loads, several
// entries' loads issued before any is used), then one thread per node adds the terms of its
// entries in a fixed order.  Returns 1 if a scaled value left [2^-60, 2^60] (the pass must be
// redone), sets *drift if one left [2^-30, 2^30], and the measures (unnormalised) in *mism,
// *resid.  The boundary duals are float-float base-2 logarithms (about 48 bits).
template <bool CL>
__device__ int linear_pass(const LinArgs &a, const Ptrs &P, Part &pt, int cur, FF *mism_out, FF *res_out, int *drift,
                           float2 *red, float *redf) {
  const int V = a.V, S = a.S, T = a.T, nxt = cur ^ 1;
  float *rp = P.rows, *rc = P.rows + V, *c = P.c;
  const int nt = blockDim.x;
  Range rg;
  int lost = 0;
  FF mism{0.f, 0.f}, res{0.f, 0.f};
  // b_T[v] = sum_{sink j, tail j = v} U0T(j) 2^-beta_T[v]
  for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) rp[v] = 0.f;
  __syncthreads();
  for (int s = pt.z0 + threadIdx.x; s < pt.z1; s += nt) {
    const int v = a.zseg_node[s];
    const float sc = ldx<CL>(P.beta + (size_t)T * V + v);
    float acc = 0.f;
    for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) acc += exp2_ff(ff_add(ff_of(a.lU0T[cur][e]), -sc), 0);
    rg.see(acc);
    rp[v] = acc;
  }
  __syncthreads();
  for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) P.bm[(size_t)T * V + v] = rp[v];
  step_sync<CL>();
  // backward sweep, t = T-1..2: term of out-entry j = b_{t+1}[head j] Gb_t(j) w_t(j)
  for (int t = T - 1; t >= 2; --t) {
    const float *gw = P.gbw + (size_t)t * S;
    for (int k0 = pt.out0 + threadIdx.x; k0 < pt.out1; k0 += kBatch * nt) {
      int hd[kBatch];
      float g[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j * nt;
        hd[j] = k < pt.out1 ? P.out_head[k] : 0;
        g[j] = k < pt.out1 ? ldx<CL>(gw + k) : 0.f;
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j * nt;
        if (k < pt.out1) c[k] = ld_row<CL>(rp, hd[j], pt) * g[j];
      }
    }
    __syncthreads();
    for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) {
      float acc = 0.f;
      for (int k = P.out_ptr[v]; k < P.out_ptr[v + 1]; ++k) acc += c[k];
      rg.see(acc);
      rc[v] = acc;
      P.bm[(size_t)t * V + v] = acc;
    }
    step_sync<CL>();
    float *tmp = rp; rp = rc; rc = tmp;
  }
  // rp = b_2.  Source update U01 <- R01 / Psi_1 (mismatch taken before), then
  // a_1[v] = sum_{source i, head i = v} U01(i) 2^-alpha_1[v]
  for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) rc[v] = 0.f;
  __syncthreads();
  for (int s = pt.s0 + threadIdx.x; s < pt.s1; s += nt) {
    const int v = a.sseg_node[s];
    const float bb = rp[v];   // own node
    const FF p1 = bb > 0.f ? ff_add(ff_log2(bb), ldx<CL>(P.beta + (size_t)2 * V + v)) : FF{0.f, 0.f};
    const float sc = ldx<CL>(P.alpha + (size_t)V + v);
    float acc = 0.f;
    for (int e = a.sseg_ptr[s]; e < a.sseg_ptr[s + 1]; ++e) {
      const FF lo = ff_of(a.lU01[cur][e]);
      FF ln = lo;
      if (bb > 0.f) {
        ln = ff_sum(ff_of(a.src_logR[e]), ff_neg(p1));
        const FF d = ff_sum(lo, ff_neg(ln));
        mism = ff_add(mism, a.src_R[e] * fabsf(expm1f((d.h + d.l) * kLn2f)));
      } else {
        lost = 1;
      }
      a.lU01[nxt][e] = f2_of(ln);
      acc += exp2_ff(ff_add(ln, -sc), 0);
    }
    rg.see(acc);
    rc[v] = acc;
  }
  step_sync<CL>();
  { float *tmp = rp; rp = rc; rc = tmp; }
  // forward sweep with the capacity updates, t = 2..T-1: term of in-entry i =
  // a_{t-1}[tail i] Gf_t(i) w_t(i), w_t(i) updated first where the state has a capacity
  for (int t = 2; t <= T - 1; ++t) {
    const size_t o = (size_t)t * S;
    const float *bn = P.bm + (size_t)(t + 1) * V;
    FF rsum{0.f, 0.f};
    for (int k0 = pt.in0 + threadIdx.x; k0 < pt.in1; k0 += kBatch * nt) {
      int ti[kBatch], hi[kBatch], nu[kBatch];
      float gf[kBatch], dc[kBatch], wo[kBatch], fc[kBatch], gb[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j * nt;
        const bool in = k < pt.in1;
        ti[j] = in ? P.in_tail[k] : 0;
        hi[j] = in ? P.in_head[k] : 0;
        gf[j] = in ? P.Gf[o + k] : 0.f;
        dc[j] = in ? P.Dc[o + k] : INFINITY;
        nu[j] = in ? P.nu[o + k] : 0;
        wo[j] = in ? P.w[cur][o + k] : 0.f;
        fc[j] = in ? P.Fc[o + k] : 0.f;
        gb[j] = in ? P.Gb[o + k] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j * nt;
        if (k >= pt.in1) continue;
        const float a0 = ld_row<CL>(rp, ti[j], pt);
        float g = gf[j];
        if (dc[j] != INFINITY) {
          const float x = a0 * ldx<CL>(bn + hi[j]);
          const float uc = ldexpf(1.f, -nu[j]);
          const float un = x > 0.f ? fminf(__fdiv_rn(dc[j], x), uc) : uc;
          rsum = ff_add(rsum, fabsf(un - wo[j]) * fminf(x * fc[j], FLT_MAX));
          P.w[nxt][o + k] = un;
          P.gbw[o + P.in_to_out[k]] = gb[j] * un;
          if (un > 0.f) rg.lo = fminf(rg.lo, un);   // u_t must not drop out of the FP32 range
          g *= un;
        }
        c[k] = a0 * g;
      }
    }
    res = ff_sum(res, rsum);
    __syncthreads();
    for (int v = pt.v0 + threadIdx.x; v < pt.v1; v += nt) {
      float acc = 0.f;
      for (int k = P.in_ptr[v]; k < P.in_ptr[v + 1]; ++k) acc += c[k];
      rg.see(acc);
      rc[v] = acc;
    }
    step_sync<CL>();
    float *tmp = rp; rp = rc; rc = tmp;
  }
  // rp = a_{T-1}.  Sink update U0T <- R0T / hatPsi_T
  for (int s = pt.z0 + threadIdx.x; s < pt.z1; s += nt) {
    const int v = a.zseg_node[s];
    const float aa = rp[v];   // own node
    const FF p = aa > 0.f ? ff_add(ff_log2(aa), ldx<CL>(P.alpha + (size_t)(T - 1) * V + v)) : FF{0.f, 0.f};
    for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) {
      if (aa > 0.f) a.lU0T[nxt][e] = f2_of(ff_sum(ff_of(a.snk_logR[e]), ff_neg(p)));
      else { a.lU0T[nxt][e] = a.lU0T[cur][e]; lost = 1; }
    }
  }
  __syncthreads();
  *mism_out = part_sum<CL>(mism, red, a.cred, pt);
  *res_out = part_sum<CL>(res, red, a.cred, pt);
  const FF nlost = part_sum<CL>(FF{(float)(lost | (rg.bad ? 1 : 0)), 0.f}, red, a.cred, pt);
  const float hi = part_max<CL>(rg.hi, redf, a.cred, pt);
  const float inv_lo = part_max<CL>(rg.lo > 0.f ? 1.f / rg.lo : 0.f, redf, a.cred, pt);
  *drift = (hi > kDrift || inv_lo > kDrift) ? 1 : 0;
  return (nlost.h > 0.f || hi > kLost || inv_lo > kLost) ? 1 : 0;
}

// Duals in from the problem (init = 2), or the initialisation of Algorithm 2 (init = 1:
// u_t = 1, U01 = U0T = 1 on the supports).  States without a capacity at t keep w = 1, nu = 0 in
// both buffers.  Entries and boundary segments of the block's own nodes.
__device__ void load_duals(const LinArgs &a, const Ptrs &P, const Part &pt, int cur, int init) {
  const int S = a.S, T = a.T, nown = pt.in1 - pt.in0, n = (T - 2) * nown;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int t = 2 + idx / nown, k = pt.in0 + idx - (t - 2) * nown;
    const size_t q = (size_t)t * S + k;
    const float2 ld = a.logd[(size_t)t * a.drs + k];
    float wv = 1.f;
    int nu = 0;
    if (ld.x != INFINITY && init == 2) {
      const float2 lu = a.p_logu[(size_t)t * S + a.in_state[k]];
      if (lu.x < -1e29f) wv = 0.f;
      else {
        const float n0 = floorf(lu.x);
        wv = exp2f(__fadd_rn(__fsub_rn(lu.x, n0), lu.y));
        nu = (int)n0;
      }
    }
    P.w[cur][q] = wv;
    P.nu[q] = nu;
    if (ld.x == INFINITY) P.w[cur ^ 1][q] = 1.f;
  }
  const int e0 = a.sseg_ptr[pt.s0], e1 = a.sseg_ptr[pt.s1];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x)
    a.lU01[cur][e] = init == 2 ? split(a.p_src_logU[a.src_tri[e]]) : make_float2(0.f, 0.f);
  const int f0 = a.zseg_ptr[pt.z0], f1 = a.zseg_ptr[pt.z1];
  for (int e = f0 + threadIdx.x; e < f1; e += blockDim.x)
    a.lU0T[cur][e] = init == 2 ? split(a.p_snk_logU[a.snk_tri[e]]) : make_float2(0.f, 0.f);
  __syncthreads();
}

// Duals out to the problem: log2 u_t = nu + log2 w as a float-float pair; U01, U0T per triple.
__device__ void store_duals(const LinArgs &a, const Ptrs &P, const Part &pt, int cur) {
  const int S = a.S, T = a.T, nown = pt.in1 - pt.in0, n = (T - 2) * nown;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int t = 2 + idx / nown, k = pt.in0 + idx - (t - 2) * nown;
    const size_t q = (size_t)t * S + k;
    const float2 ld = a.logd[(size_t)t * a.drs + k];
    float2 lu = make_float2(0.f, 0.f);
    if (ld.x != INFINITY) {
      const float wv = P.w[cur][q];
      if (wv > 0.f) {
        float h, l;
        two_sum((float)P.nu[q], log2f(wv), h, l);
        lu = make_float2(h, l);
      } else {
        lu = make_float2(kNegLog, 0.f);
      }
    }
    a.p_logu[(size_t)t * S + a.in_state[k]] = lu;
  }
  const int e0 = a.sseg_ptr[pt.s0], e1 = a.sseg_ptr[pt.s1];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) a.p_src_logU[a.src_tri[e]] = dbl(a.lU01[cur][e]);
  const int f0 = a.zseg_ptr[pt.z0], f1 = a.zseg_ptr[pt.z1];
  for (int e = f0 + threadIdx.x; e < f1; e += blockDim.x) a.p_snk_logU[a.snk_tri[e]] = dbl(a.lU0T[cur][e]);
}

struct LinShared {
  LinArgs a;
  Ptrs P;
  Part pt;
  int vb[9];
  float2 red[32];
  float redf[32];
};

// Up to max_passes passes on one problem, stopping at tol (tol < 0: never).  init: 0 = continue
// the previous launch, 1 = initial duals, 2 = the problem's duals.  Every launch starts with a
// scale sweep (it does not change the iterate).  CL: the problem runs on a cluster of R blocks
// (blockIdx.x / R is the problem, the rank in the cluster its part); otherwise on one block.
template <bool CL>
__global__ void __launch_bounds__(kLinThreads) k_linear(LinArgs *const *args, int max_passes, double tol, int init,
                                                        int R) {
  __shared__ LinShared sh;
  extern __shared__ __align__(16) float dyn[];
  const int prob = CL ? blockIdx.x / R : blockIdx.x;
  const int rank = CL ? blockIdx.x % R : 0;
  LinArgs *g = args[prob];
  if (threadIdx.x == 0) sh.a = *g;
  __syncthreads();
  const LinArgs &a = sh.a;
  // (uniform over the cluster: every block reads the same flag)
  if (init == 0 && a.done) {   // finished in an earlier launch: report no new passes
    if (threadIdx.x == 0 && rank == 0) { a.rep->passes = 0; a.rep->log_passes = 0; a.rep->rescalings = 0; }
    return;
  }
  if (threadIdx.x == 0) {
    if (CL) sh.a.mode = 0;         // a cluster keeps the per-entry arrays in global memory
    sh.P = make_ptrs(sh.a, dyn);
    sh.pt = make_part(a, rank, CL ? R : 1, sh.vb);
  }
  __syncthreads();
  const Ptrs &P = sh.P;
  Part pt = sh.pt;                 // per-thread copy: the reduction slot advances in every thread
  stage_in(a, P, init == 0);
  int cur = a.cur, need = 1;
  if (init) load_duals(a, P, pt, cur, init);
  step_sync<CL>();
  int passes = 0, log_passes = 0, rescalings = 0, status = OTS_OK, converged = 0;
  const float tolf = (float)tol;
  FF mism{0.f, 0.f}, res{0.f, 0.f};
  int log_run = 0, backoff = 1;    // passes still to run in log arithmetic after a thrown-away pass
  while (passes < max_passes) {
    int lost = 0;
    if (log_run > 0) {
      // a problem whose duals keep leaving the range (e.g. they diverge, with no feasible flow)
      // runs in log arithmetic for a while before the linear form is tried again
      status = log_sweep<CL>(a, P, pt, cur, true, &mism, &res, sh.red);
      cur ^= 1;
      ++log_passes;
      lost = 1;
      if (status) { ++passes; break; }
      if (--log_run == 0) { rebuild<CL>(a, P, pt, cur); ++rescalings; }
    } else {
      if (need) {
        status = log_sweep<CL>(a, P, pt, cur, false, nullptr, nullptr, sh.red);
        if (status) break;
        rebuild<CL>(a, P, pt, cur);
        ++rescalings;
        need = 0;
      }
      int drift = 0;
      lost = linear_pass<CL>(a, P, pt, cur, &mism, &res, &drift, sh.red, sh.redf);
      if (lost) {
        // thrown away: the same pass again in log arithmetic, from the same duals; the next
        // 1, 2, 4, ... 64 passes too while the linear form keeps failing
        status = log_sweep<CL>(a, P, pt, cur, true, &mism, &res, sh.red);
        cur ^= 1;
        ++log_passes;
        if (status) { ++passes; break; }
        log_run = backoff - 1;
        backoff = min(2 * backoff, 64);
        if (log_run == 0) { rebuild<CL>(a, P, pt, cur); ++rescalings; }
      } else {
        cur ^= 1;
        need = drift;
        backoff = 1;
      }
    }
    ++passes;
    const float srcf = (mism.h + mism.l) / a.mass, capf = (res.h + res.l) / a.mass;
    if (!(srcf == srcf) || !(capf == capf)) { status = OTS_ERR_NUMERIC; break; }
    if (!lost && srcf <= tolf && capf <= tolf) { converged = 1; break; }
  }
  step_sync<CL>();
  store_duals(a, P, pt, cur);
  stage_out(a, P);
  if (threadIdx.x == 0 && rank == 0) {
    g->cur = cur;
    g->done = converged || status != OTS_OK;
    LinReport r;
    r.passes = passes; r.log_passes = log_passes; r.rescalings = rescalings; r.status = status;
    r.converged = converged; r.pad = 0;
    r.src = ((double)mism.h + (double)mism.l) / a.mass;
    r.cap = ((double)res.h + (double)res.l) / a.mass;
    *a.rep = r;
  }
}

}  // namespace
}  // namespace ots

// ---------------------------------------------------------------------------------------
// Host side: the per-problem argument block and arrays, and the launch.

using namespace ots;

namespace ots_host {

struct LinearData {
  void *arena = nullptr;
  LinArgs h{};                  // argument block with device pointers
  LinArgs *d_args = nullptr;    // its device copy (also holds the state kept between launches)
  LinArgs **d_argp = nullptr;   // one-entry pointer array for single-problem launches
  LinReport *d_rep = nullptr;
  LinReport *h_rep = nullptr;   // pinned
  int smem = 0;
};

namespace {

constexpr size_t kLinSmemAll = 96 * 1024;     // whole problem in shared memory up to this size
constexpr size_t kLinSmemIndex = 96 * 1024;   // index arrays too up to this size
constexpr int kLinSmemMax = 200 * 1024;       // two message rows + per-entry terms must fit

struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = align_up(off, 256);
    off = o + bytes;
    return o;
  }
};

void split_log2(double x, float2 &out) {
  float h, l;
  split_ff(x, h, l);
  out = make_float2(h, l);
}

}  // namespace

ots_status linear_prepare(ots_problem *p) {
  if (p->lin) return OTS_OK;
  if (p->L != 1) return fail(OTS_ERR_INVALID_ARG, "the linear-domain path solves single-commodity problems (L = 1), not L = %d", p->L);
  if (p->xgraph || p->win || p->pc || p->cc)
    return fail(OTS_ERR_INVALID_ARG, "the linear-domain path takes the node-level state graph with state costs and "
                                     "capacities only (no explicit state graph, windows or per-commodity data)");
  if (p->member) return fail(OTS_ERR_INVALID_ARG, "problem belongs to a batch");
  const int V = p->V, S = p->S, T = p->T;
  // in-CSR by head node, out-CSR by tail node
  std::vector<int> in_ptr(V + 1, 0), out_ptr(V + 1, 0), in_state(S), in_tail(S), in_head(S), pos_in(S);
  std::vector<int> out_tail(S), out_head(S), out_to_in(S), in_to_out(S);
  for (int s = 0; s < S; ++s) { ++in_ptr[p->head[s] + 1]; ++out_ptr[p->tail[s] + 1]; }
  for (int v = 0; v < V; ++v) { in_ptr[v + 1] += in_ptr[v]; out_ptr[v + 1] += out_ptr[v]; }
  {
    std::vector<int> fi(in_ptr.begin(), in_ptr.end() - 1), fo(out_ptr.begin(), out_ptr.end() - 1);
    for (int s = 0; s < S; ++s) {
      const int k = fi[p->head[s]]++;
      in_state[k] = s; in_tail[k] = p->tail[s]; in_head[k] = p->head[s]; pos_in[s] = k;
    }
    for (int s = 0; s < S; ++s) {
      const int k = fo[p->tail[s]]++;
      out_tail[k] = p->tail[s]; out_head[k] = p->head[s]; out_to_in[k] = pos_in[s]; in_to_out[pos_in[s]] = k;
    }
  }
  // log2 K and log2 d per in-entry (rows t when they vary with t)
  const int KR = p->tv ? T + 1 : 1, DR = p->cv ? T + 1 : 1;
  std::vector<float2> kappa((size_t)KR * S), logd((size_t)DR * S);
  for (int r = 0; r < KR; ++r)
    for (int k = 0; k < S; ++k) {
      const double c = p->cost_nat[(size_t)r * S + in_state[k]];
      if (c == INFINITY) kappa[(size_t)r * S + k] = make_float2(-INFINITY, 0.f);
      else split_log2(-c / p->eps * kInvLn2, kappa[(size_t)r * S + k]);
    }
  for (int r = 0; r < DR; ++r)
    for (int k = 0; k < S; ++k) {
      const double d = p->cap_nat[(size_t)r * S + in_state[k]];
      if (std::isinf(d)) logd[(size_t)r * S + k] = make_float2(INFINITY, 0.f);
      else if (d == 0.0) logd[(size_t)r * S + k] = make_float2(-INFINITY, 0.f);
      else split_log2(std::log2(d), logd[(size_t)r * S + k]);
    }
  // boundary entries grouped by node (head of a source state, tail of a sink state)
  struct Side {
    std::vector<int> seg_node, seg_ptr, tri;
    std::vector<float> R;
    std::vector<float2> logR;
  } side[2];
  double mass = 0.0;
  for (int b = 0; b < 2; ++b) {
    const Boundary &bd = b == 0 ? p->src : p->snk;
    std::vector<int> order(bd.n);
    for (int q = 0; q < bd.n; ++q) order[q] = q;
    auto node = [&](int q) { return b == 0 ? p->head[bd.tri_state[q]] : p->tail[bd.tri_state[q]]; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return node(x) < node(y); });
    Side &sd = side[b];
    for (int i = 0; i < bd.n; ++i) {
      const int q = order[i];
      if (i == 0 || node(q) != node(order[i - 1])) { sd.seg_node.push_back(node(q)); sd.seg_ptr.push_back(i); }
      sd.tri.push_back(q);
      sd.R.push_back((float)bd.tri_R[q]);
      float2 lr;
      split_log2(std::log2(bd.tri_R[q]), lr);
      sd.logR.push_back(lr);
      if (b == 0) mass += bd.tri_R[q];
    }
    sd.seg_ptr.push_back(bd.n);
  }
  // one arena
  Bump m;
  const size_t TS = (size_t)(T + 1) * S, TV = (size_t)(T + 1) * V;
  const int ns = p->src.n, nz = p->snk.n;
  const int nss = (int)side[0].seg_node.size(), nzs = (int)side[1].seg_node.size();
  const size_t o_in_ptr = m.take(4 * (V + 1)), o_in_tail = m.take(4 * S), o_in_head = m.take(4 * S),
               o_in_state = m.take(4 * S), o_out_ptr = m.take(4 * (V + 1)), o_out_tail = m.take(4 * S),
               o_out_head = m.take(4 * S), o_out_to_in = m.take(4 * S), o_in_to_out = m.take(4 * S),
               o_gbw = m.take(4 * TS), o_kappa = m.take(8 * kappa.size()),
               o_logd = m.take(8 * logd.size()), o_gf = m.take(4 * TS), o_gb = m.take(4 * TS), o_dc = m.take(4 * TS),
               o_fc = m.take(4 * TS), o_nu = m.take(4 * TS), o_w0 = m.take(4 * TS), o_w1 = m.take(4 * TS),
               o_alpha = m.take(4 * TV), o_beta = m.take(4 * TV), o_bm = m.take(4 * TV),
               o_ssn = m.take(4 * std::max(nss, 1)), o_ssp = m.take(4 * (nss + 1)), o_zsn = m.take(4 * std::max(nzs, 1)),
               o_zsp = m.take(4 * (nzs + 1)), o_sR = m.take(4 * std::max(ns, 1)), o_slR = m.take(8 * std::max(ns, 1)),
               o_zR = m.take(4 * std::max(nz, 1)), o_zlR = m.take(8 * std::max(nz, 1)), o_u01a = m.take(8 * std::max(ns, 1)),
               o_u01b = m.take(8 * std::max(ns, 1)), o_u0ta = m.take(8 * std::max(nz, 1)), o_u0tb = m.take(8 * std::max(nz, 1)),
               o_stri = m.take(4 * std::max(ns, 1)), o_ztri = m.take(4 * std::max(nz, 1)), o_args = m.take(sizeof(LinArgs)),
               o_argp = m.take(sizeof(LinArgs *)), o_rep = m.take(sizeof(LinReport)),
               o_cred = m.take(8 * 4 * 16);
  std::unique_ptr<LinearData> L(new LinearData);
  L->arena = problem_alloc(p, m.off);
  if (!L->arena) return fail(OTS_ERR_OOM, "device allocation of %zu bytes failed", m.off);
  if (cudaMallocHost(&L->h_rep, sizeof(LinReport)) != cudaSuccess) {
    problem_free(p, L->arena);
    return fail(OTS_ERR_OOM, "pinned allocation failed");
  }
  char *base = (char *)L->arena;
  auto at = [&](size_t o) { return (void *)(base + o); };
  LinArgs &h = L->h;
  h.V = V; h.S = S; h.T = T; h.krs = p->tv ? S : 0; h.drs = p->cv ? S : 0;
  h.n_src = ns; h.n_snk = nz; h.n_sseg = nss; h.n_zseg = nzs; h.mass = (float)mass;
  h.in_ptr = (int *)at(o_in_ptr); h.in_tail = (int *)at(o_in_tail); h.in_head = (int *)at(o_in_head);
  h.in_state = (int *)at(o_in_state); h.out_ptr = (int *)at(o_out_ptr); h.out_tail = (int *)at(o_out_tail);
  h.out_head = (int *)at(o_out_head); h.out_to_in = (int *)at(o_out_to_in); h.in_to_out = (int *)at(o_in_to_out);
  h.gbw = (float *)at(o_gbw);
  h.kappa = (float2 *)at(o_kappa); h.logd = (float2 *)at(o_logd);
  h.Gf = (float *)at(o_gf); h.Gb = (float *)at(o_gb); h.Dc = (float *)at(o_dc); h.Fc = (float *)at(o_fc);
  h.nu = (int *)at(o_nu); h.w[0] = (float *)at(o_w0); h.w[1] = (float *)at(o_w1);
  h.alpha = (float *)at(o_alpha); h.beta = (float *)at(o_beta); h.bm = (float *)at(o_bm);
  h.sseg_node = (int *)at(o_ssn); h.sseg_ptr = (int *)at(o_ssp); h.zseg_node = (int *)at(o_zsn); h.zseg_ptr = (int *)at(o_zsp);
  h.src_R = (float *)at(o_sR); h.src_logR = (float2 *)at(o_slR); h.snk_R = (float *)at(o_zR); h.snk_logR = (float2 *)at(o_zlR);
  h.lU01[0] = (float2 *)at(o_u01a); h.lU01[1] = (float2 *)at(o_u01b); h.lU0T[0] = (float2 *)at(o_u0ta); h.lU0T[1] = (float2 *)at(o_u0tb);
  h.src_tri = (int *)at(o_stri); h.snk_tri = (int *)at(o_ztri);
  h.p_logu = p->d_logu; h.p_src_logU = p->src.d_tri_logU; h.p_snk_logU = p->snk.d_tri_logU;
  h.cred = (float2 *)at(o_cred);
  L->d_rep = (LinReport *)at(o_rep);
  h.rep = L->d_rep;
  h.cur = 0; h.done = 0;
  L->d_args = (LinArgs *)at(o_args);
  L->d_argp = (LinArgs **)at(o_argp);
  // shared-memory mode: everything when it fits in kLinSmemAll, else the index arrays when they
  // fit in kLinSmemIndex, else only the two message rows and the per-entry terms
  h.mode = 0;
  if (lin_layout(V, S, T, 2).words * 4 <= kLinSmemAll) h.mode = 2;
  else if (lin_layout(V, S, T, 1).words * 4 <= kLinSmemIndex) h.mode = 1;
  L->smem = (int)(lin_layout(V, S, T, h.mode).words * 4);
  if (L->smem > kLinSmemMax) {
    cudaFreeHost(L->h_rep);
    problem_free(p, L->arena);
    return fail(OTS_ERR_INVALID_ARG, "the linear-domain path needs %d bytes of shared memory (at most %d)", L->smem, kLinSmemMax);
  }
  LinArgs *argp = L->d_args;
  cudaStream_t s = p->stream;
  size_t up = 0;
  auto put = [&](size_t o, const void *src, size_t bytes) {
    up += bytes;
    return bytes ? cudaMemcpyAsync(at(o), src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  cudaError_t e = cudaMemsetAsync(L->arena, 0, m.off, s);
  if (!e) e = put(o_in_ptr, in_ptr.data(), 4 * in_ptr.size());
  if (!e) e = put(o_in_tail, in_tail.data(), 4 * S);
  if (!e) e = put(o_in_head, in_head.data(), 4 * S);
  if (!e) e = put(o_in_state, in_state.data(), 4 * S);
  if (!e) e = put(o_out_ptr, out_ptr.data(), 4 * out_ptr.size());
  if (!e) e = put(o_out_tail, out_tail.data(), 4 * S);
  if (!e) e = put(o_out_head, out_head.data(), 4 * S);
  if (!e) e = put(o_out_to_in, out_to_in.data(), 4 * S);
  if (!e) e = put(o_in_to_out, in_to_out.data(), 4 * S);
  if (!e) e = put(o_kappa, kappa.data(), 8 * kappa.size());
  if (!e) e = put(o_logd, logd.data(), 8 * logd.size());
  if (!e) e = put(o_ssn, side[0].seg_node.data(), 4 * nss);
  if (!e) e = put(o_ssp, side[0].seg_ptr.data(), 4 * (nss + 1));
  if (!e) e = put(o_zsn, side[1].seg_node.data(), 4 * nzs);
  if (!e) e = put(o_zsp, side[1].seg_ptr.data(), 4 * (nzs + 1));
  if (!e) e = put(o_sR, side[0].R.data(), 4 * ns);
  if (!e) e = put(o_slR, side[0].logR.data(), 8 * ns);
  if (!e) e = put(o_zR, side[1].R.data(), 4 * nz);
  if (!e) e = put(o_zlR, side[1].logR.data(), 8 * nz);
  if (!e) e = put(o_stri, side[0].tri.data(), 4 * ns);
  if (!e) e = put(o_ztri, side[1].tri.data(), 4 * nz);
  if (!e) e = put(o_args, &h, sizeof(LinArgs));
  if (!e) e = put(o_argp, &argp, sizeof(LinArgs *));
  if (!e) e = cudaStreamSynchronize(s);   // the host vectors above go out of scope
  if (e) {
    cudaFreeHost(L->h_rep);
    problem_free(p, L->arena);
    return fail(OTS_ERR_CUDA, "linear-domain set-up: %s", cudaGetErrorString(e));
  }
  p->h2d_bytes += (long long)up;
  p->lin = L.release();
  return OTS_OK;
}

const LinReport &linear_report(const ots_problem *p) { return *p->lin->h_rep; }

void linear_release(ots_problem *p) {
  if (!p->lin) return;
  if (p->lin->h_rep) cudaFreeHost(p->lin->h_rep);
  problem_free(p, p->lin->arena);
  delete p->lin;
  p->lin = nullptr;
}

// Blocks per problem: one up to kLinClusterMin states (a cluster's barriers cost more than they
// gain there: 0.40 against 0.32 ms per pass at 2800 states), else a cluster with about
// kLinClusterStates state entries per block (at most 8 blocks, the portable cluster size).
constexpr int kLinClusterMin = 4096;
constexpr int kLinClusterStates = 2048;

int linear_blocks_per_problem(int S) {
  if (S <= kLinClusterMin) return 1;
  int R = 1;
  while (R < 8 && (long long)R * kLinClusterStates < S) R <<= 1;
  return R;
}

ots_status linear_run(ots_problem *const *ps, int n, int max_passes, double tol, int init, double *kernel_ms) {
  int smax = 0;
  for (int i = 0; i < n; ++i) smax = std::max(smax, ps[i]->S);
  const int R = linear_blocks_per_problem(smax);
  int smem = 0;
  for (int i = 0; i < n; ++i) {
    const LinArgs &h = ps[i]->lin->h;
    smem = std::max(smem, R > 1 ? (int)(lin_layout(h.V, h.S, h.T, 0).words * 4) : ps[i]->lin->smem);
  }
  // threads per block: enough for one state entry each up to kLinThreads (small problems take
  // fewer warps, so their barriers are cheaper)
  const int threads = R > 1 ? kLinThreads : std::min(kLinThreads, std::max(64, (smax + 31) / 32 * 32));
  if (smem > 48 * 1024) {
    OTS_CUDA(cudaFuncSetAttribute(k_linear<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    OTS_CUDA(cudaFuncSetAttribute(k_linear<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  }
  cudaStream_t s = ps[0]->stream;
  for (int i = 1; i < n; ++i) OTS_CUDA(cudaStreamSynchronize(ps[i]->stream));
  LinArgs **argp = ps[0]->lin->d_argp;
  if (n > 1) {
    std::vector<LinArgs *> hp(n);
    for (int i = 0; i < n; ++i) hp[i] = ps[i]->lin->d_args;
    OTS_CUDA(cudaMallocAsync((void **)&argp, sizeof(LinArgs *) * n, s));
    OTS_CUDA(cudaMemcpyAsync(argp, hp.data(), sizeof(LinArgs *) * n, cudaMemcpyHostToDevice, s));
    OTS_CUDA(cudaStreamSynchronize(s));
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  OTS_CUDA(cudaEventCreate(&e0));
  OTS_CUDA(cudaEventCreate(&e1));
  OTS_CUDA(cudaEventRecord(e0, s));
  cudaError_t le = cudaSuccess;
  if (R == 1) {
    k_linear<false><<<n, threads, smem, s>>>(argp, max_passes, tol, init, 1);
    le = cudaGetLastError();
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n * R), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)R;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    le = cudaLaunchKernelEx(&cfg, k_linear<true>, argp, max_passes, tol, init, R);
  }
  OTS_CUDA(cudaEventRecord(e1, s));
  for (int i = 0; i < n; ++i)
    OTS_CUDA(cudaMemcpyAsync(ps[i]->lin->h_rep, ps[i]->lin->d_rep, sizeof(LinReport), cudaMemcpyDeviceToHost, s));
  if (n > 1) OTS_CUDA(cudaFreeAsync(argp, s));
  OTS_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (le != cudaSuccess) return fail(OTS_ERR_CUDA, "linear-domain kernel: %s", cudaGetErrorString(le));
  if (kernel_ms) *kernel_ms = ms;
  for (int i = 0; i < n; ++i) {
    ots_problem *p = ps[i];
    p->stale = true;   // duals changed: the log-domain messages are recomputed before use
    p->kernels_launched += 1;
    p->passes_total += p->lin->h_rep->passes;
    p->d2h_bytes += sizeof(LinReport);
  }
  return OTS_OK;
}

}  // namespace ots_host

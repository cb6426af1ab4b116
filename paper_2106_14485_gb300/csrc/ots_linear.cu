// ots_linear.cu -- the single-commodity problem (L = 1, Section 4.2) with FP32 messages in
// the linear domain, one thread block per problem for whole runs of passes.
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
// quantities).  The boundary duals stay FP64 base-2 logarithms: U01 <- R01 / Psi_1 with
// Psi_1(i) = B_2[head i], U0T <- R0T / hatPsi_T with hatPsi_T(j) = A_{T-1}[tail j].
//
// The scales are taken from the messages themselves by a sweep in FP32 log arithmetic at the
// current duals (no update; the iterate does not change), so that after it every a and b is 1.
// A pass in which some scaled value leaves [2^-60, 2^60] (or is not finite) is thrown away and
// run again in FP32 log arithmetic (with updates), which re-takes the scales; one that stays
// inside but leaves [2^-30, 2^30] re-takes them before the next pass.  The measures are those
// of Algorithm 2 (relative source mismatch before the U01 update, capacity residual
// sum |P_t after - P_t before|), summed per block in a fixed order.
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
  double mass;                       // sum of R01
  const int *in_ptr, *in_tail, *in_head, *in_state;   // in-CSR by head node (entry k = state in_state[k])
  const int *out_ptr, *out_tail, *out_head, *out_to_in;  // out-CSR by tail node
  const float2 *kappa;               // [rows][S] log2 K of in-entry k (float-float); x = -inf: closed
  const float2 *logd;                // [rows][S] log2 d of in-entry k; x = +inf: no capacity, -inf: d = 0
  float *Gf, *Gb, *Dc, *Fc;          // [(T+1) S]: Gf, Dc, Fc by in-entry, Gb by out-entry
  int *nu;                           // [(T+1) S] by in-entry
  float *w[2];                       // [(T+1) S] by in-entry: w_t (two buffers: current, next)
  float *alpha, *beta, *bm;          // [(T+1) V]: scales and the scaled backward messages
  const int *sseg_node, *sseg_ptr, *zseg_node, *zseg_ptr;   // boundary entries grouped by node
  const double *src_R, *src_logR, *snk_R, *snk_logR;       // per entry, log2
  double *lU01[2], *lU0T[2];         // per entry, log2 (two buffers)
  const int *src_tri, *snk_tri;      // entry -> boundary triple of the problem
  float2 *p_logu;                    // problem's log2 u_t [(T+1) S] by state (float-float)
  double *p_src_logU, *p_snk_logU;   // problem's log2 U01 / U0T per triple
  LinReport *rep;
  int cur, need, done, pad;          // state kept between launches
};

namespace {

constexpr int kLinThreads = 512;
constexpr float kLost = 0x1p60f, kDrift = 0x1p30f;
constexpr float kLn2f = 0.693147180559945309f;
constexpr float kNegLog = -1e30f;    // log 0 in the problem's float-float duals

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

// Block reductions in a fixed order (all threads get the result).
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
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

// Scale sweep (update = false) or a whole pass of Algorithm 2 in FP32 log arithmetic
// (update = true): alpha_t, beta_t become the base-2 logarithms of the messages.  With updates,
// the new duals go to the next buffers (w[nxt], lU01/lU0T[nxt], nu in place) and the measures
// to *mism, *resid; returns an ots_status (OTS_ERR_INFEASIBLE if a boundary state has no path).
__device__ int log_sweep(const LinArgs &a, int cur, bool update, float *rows, double *mism_out, double *res_out,
                         double *red) {
  const int V = a.V, S = a.S, T = a.T, nxt = cur ^ 1;
  float *rp = rows, *rc = rows + V;
  int bad = 0;
  double mism = 0.0, res = 0.0;
  // beta_T[v] = log2 sum_{sink j, tail j = v} U0T(j)
  for (int v = threadIdx.x; v < V; v += blockDim.x) rp[v] = -INFINITY;
  __syncthreads();
  for (int s = threadIdx.x; s < a.n_zseg; s += blockDim.x) {
    double m = -INFINITY;
    for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) m = fmax(m, a.lU0T[cur][e]);
    double acc = 0.0;
    for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) acc += exp2(a.lU0T[cur][e] - m);
    rp[a.zseg_node[s]] = (float)(m + log2(acc));
  }
  __syncthreads();
  for (int v = threadIdx.x; v < V; v += blockDim.x) a.beta[(size_t)T * V + v] = rp[v];
  // beta_t[v] = log2 sum_{tail j = v} 2^(beta_{t+1}[head j] + log2 K(j) + log2 u_t(j)),  t = T-1..2
  for (int t = T - 1; t >= 2; --t) {
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      float m = -INFINITY, sum = 0.f;
      for (int k = a.out_ptr[v]; k < a.out_ptr[v + 1]; ++k) {
        const int ki = a.out_to_in[k];
        const size_t q = (size_t)t * S + ki;
        const float2 kap = a.kappa[(size_t)t * a.krs + ki];
        const float wv = a.w[cur][q];
        const float lu = wv > 0.f ? (float)a.nu[q] + log2f(wv) : -INFINITY;
        const float x = rp[a.out_head[k]] + kap.x + lu;
        if (x > m) { sum = sum * exp2f(m - x) + 1.f; m = x; }
        else if (x > -INFINITY) sum += exp2f(x - m);
      }
      const float r = m > -INFINITY ? m + log2f(sum) : -INFINITY;
      rc[v] = r;
      a.beta[(size_t)t * V + v] = r;
    }
    __syncthreads();
    float *tmp = rp; rp = rc; rc = tmp;
  }
  // source update U01 <- R01 / Psi_1, then alpha_1[v] = log2 sum_{source i, head i = v} U01(i)
  const int su = update ? nxt : cur;
  for (int v = threadIdx.x; v < V; v += blockDim.x) rc[v] = -INFINITY;
  __syncthreads();
  for (int s = threadIdx.x; s < a.n_sseg; s += blockDim.x) {
    const int v = a.sseg_node[s];
    if (update) {
      const double p1 = (double)a.beta[(size_t)2 * V + v];
      for (int e = a.sseg_ptr[s]; e < a.sseg_ptr[s + 1]; ++e) {
        if (!(p1 > -INFINITY)) { bad = 1; a.lU01[nxt][e] = a.lU01[cur][e]; continue; }
        const double ln = a.src_logR[e] - p1;
        mism += a.src_R[e] * fabs(exp2(a.lU01[cur][e] - ln) - 1.0);
        a.lU01[nxt][e] = ln;
      }
    }
    double m = -INFINITY;
    for (int e = a.sseg_ptr[s]; e < a.sseg_ptr[s + 1]; ++e) m = fmax(m, a.lU01[su][e]);
    double acc = 0.0;
    for (int e = a.sseg_ptr[s]; e < a.sseg_ptr[s + 1]; ++e) acc += exp2(a.lU01[su][e] - m);
    rc[v] = (float)(m + log2(acc));
  }
  __syncthreads();
  { float *tmp = rp; rp = rc; rc = tmp; }
  for (int v = threadIdx.x; v < V; v += blockDim.x) a.alpha[(size_t)V + v] = rp[v];
  // forward: capacity update of u_t (update) and alpha_t[v] = log2 sum_{head i = v} 2^(alpha_{t-1}[tail i]
  // + log2 K(i) + log2 u_t(i)),  t = 2..T-1
  for (int t = 2; t <= T - 1; ++t) {
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      const float bb = a.beta[(size_t)(t + 1) * V + v];
      float m = -INFINITY, sum = 0.f;
      for (int k = a.in_ptr[v]; k < a.in_ptr[v + 1]; ++k) {
        const size_t q = (size_t)t * S + k;
        const float al = rp[a.in_tail[k]];
        const float2 kap = a.kappa[(size_t)t * a.krs + k];
        const float2 ld = a.logd[(size_t)t * a.drs + k];
        float lu = 0.f;
        if (ld.x != INFINITY) {
          const float wv = a.w[cur][q];
          const float lo = wv > 0.f ? (float)a.nu[q] + log2f(wv) : -INFINITY;
          lu = lo;
          if (update) {
            const float ls = al + bb + kap.x;
            float ln = 0.f;
            if (ls > -INFINITY) {
              ln = ld.x == -INFINITY ? -INFINITY : fminf(ld.x - ls, 0.f);
              // |P_new - P_old| with P = 2^(log2 u + ls)
              if (lo == -INFINITY && ln == -INFINITY) {}
              else if (lo == -INFINITY) res += exp2((double)ln + ls);
              else if (ln == -INFINITY) res += exp2((double)lo + ls);
              else res += exp2((double)lo + ls) * fabs(exp2((double)ln - lo) - 1.0);
            }
            if (ln == -INFINITY) { a.w[nxt][q] = 0.f; a.nu[q] = 0; }
            else { const float n = floorf(ln); a.w[nxt][q] = exp2f(ln - n); a.nu[q] = (int)n; }
            lu = ln;
          }
        }
        const float x = al + kap.x + lu;
        if (x > m) { sum = sum * exp2f(m - x) + 1.f; m = x; }
        else if (x > -INFINITY) sum += exp2f(x - m);
      }
      const float r = m > -INFINITY ? m + log2f(sum) : -INFINITY;
      rc[v] = r;
      a.alpha[(size_t)t * V + v] = r;
    }
    __syncthreads();
    float *tmp = rp; rp = rc; rc = tmp;
  }
  // sink update U0T <- R0T / hatPsi_T
  if (update) {
    for (int s = threadIdx.x; s < a.n_zseg; s += blockDim.x) {
      const double p = (double)rp[a.zseg_node[s]];
      for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) {
        if (!(p > -INFINITY)) { bad = 1; a.lU0T[nxt][e] = a.lU0T[cur][e]; continue; }
        a.lU0T[nxt][e] = a.snk_logR[e] - p;
      }
    }
  }
  __syncthreads();
  const double ms = block_sum(mism, red);
  const double rs = block_sum(res, red);
  const double bd = block_sum((double)bad, red);
  if (mism_out) *mism_out = ms;
  if (res_out) *res_out = rs;
  return bd > 0.0 ? OTS_ERR_INFEASIBLE : OTS_OK;
}

// Scale fold: w_t(i) = m 2^e with m in [1/2, 1) -> w = m, nu += e (exact).  Then the per-state
// factors Gf, Gb, Dc, Fc from the current scales alpha, beta, nu.
__device__ void rebuild(const LinArgs &a, int cur) {
  const int V = a.V, S = a.S, T = a.T;
  const int n = (T - 2) * S;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int t = 2 + idx / S, k = idx - (t - 2) * S;
    const size_t q = (size_t)t * S + k;
    const float2 ld = a.logd[(size_t)t * a.drs + k];
    if (ld.x != INFINITY) {
      const float wv = a.w[cur][q];
      if (wv > 0.f) {
        int e;
        const float m = frexpf(wv, &e);
        a.w[cur][q] = m;
        a.nu[q] += e;
      }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int t = 2 + idx / S, k = idx - (t - 2) * S;
    const size_t q = (size_t)t * S + k;
    const float2 kap = a.kappa[(size_t)t * a.krs + k];
    const float2 ld = a.logd[(size_t)t * a.drs + k];
    const float al0 = a.alpha[(size_t)(t - 1) * V + a.in_tail[k]];
    const float al1 = a.alpha[(size_t)t * V + a.in_head[k]];
    const float be1 = a.beta[(size_t)(t + 1) * V + a.in_head[k]];
    const int nu = a.nu[q];
    const bool open = kap.x > -INFINITY;
    float gf = 0.f;
    if (open && al0 > -INFINITY && al1 > -INFINITY) gf = exp2_ff(ff_add(ff_add(FF{al0, 0.f}, -al1), kap), nu);
    a.Gf[q] = gf;
    if (ld.x == INFINITY) {
      a.Dc[q] = INFINITY;   // no capacity: w stays 1
      a.Fc[q] = 0.f;
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
      a.Fc[q] = fc;
      a.Dc[q] = dc;
    }
  }
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int t = 2 + idx / S, k = idx - (t - 2) * S;
    const int ki = a.out_to_in[k];
    const float2 kap = a.kappa[(size_t)t * a.krs + ki];
    const float b1 = a.beta[(size_t)(t + 1) * V + a.out_head[k]];
    const float b0 = a.beta[(size_t)t * V + a.out_tail[k]];
    float gb = 0.f;
    if (kap.x > -INFINITY && b1 > -INFINITY && b0 > -INFINITY)
      gb = exp2_ff(ff_add(ff_add(FF{b1, 0.f}, -b0), kap), a.nu[(size_t)t * S + ki]);
    a.Gb[(size_t)t * S + k] = gb;
  }
  __syncthreads();
}

// One pass of Algorithm 2 on the scaled quantities; new duals to the next buffers.  Returns
// 1 if a scaled value left [2^-60, 2^60] (the pass must be redone), sets *drift if one left
// [2^-30, 2^30], and the measures (unnormalised) in *mism, *resid.
__device__ int linear_pass(const LinArgs &a, int cur, float *rows, double *mism_out, double *res_out, int *drift,
                           double *red, float *redf) {
  const int V = a.V, S = a.S, T = a.T, nxt = cur ^ 1;
  float *rp = rows, *rc = rows + V;
  Range rg;
  int lost = 0;
  double mism = 0.0, res = 0.0;
  // b_T[v] = sum_{sink j, tail j = v} U0T(j) 2^-beta_T[v]
  for (int v = threadIdx.x; v < V; v += blockDim.x) rp[v] = 0.f;
  __syncthreads();
  for (int s = threadIdx.x; s < a.n_zseg; s += blockDim.x) {
    const int v = a.zseg_node[s];
    const double sc = (double)a.beta[(size_t)T * V + v];
    double acc = 0.0;
    for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) acc += exp2(a.lU0T[cur][e] - sc);
    const float f = (float)acc;
    rg.see(f);
    rp[v] = f;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < V; v += blockDim.x) a.bm[(size_t)T * V + v] = rp[v];
  // backward sweep, t = T-1..2
  for (int t = T - 1; t >= 2; --t) {
    const float *Gb = a.Gb + (size_t)t * S;
    const float *wt = a.w[cur] + (size_t)t * S;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      float acc = 0.f;
      for (int k = a.out_ptr[v]; k < a.out_ptr[v + 1]; ++k)
        acc = fmaf(rp[a.out_head[k]], Gb[k] * wt[a.out_to_in[k]], acc);
      rg.see(acc);
      rc[v] = acc;
      a.bm[(size_t)t * V + v] = acc;
    }
    __syncthreads();
    float *tmp = rp; rp = rc; rc = tmp;
  }
  // rp = b_2.  Source update U01 <- R01 / Psi_1 (mismatch taken before), then
  // a_1[v] = sum_{source i, head i = v} U01(i) 2^-alpha_1[v]
  for (int v = threadIdx.x; v < V; v += blockDim.x) rc[v] = 0.f;
  __syncthreads();
  for (int s = threadIdx.x; s < a.n_sseg; s += blockDim.x) {
    const int v = a.sseg_node[s];
    const float bb = rp[v];
    const double p1 = (double)a.beta[(size_t)2 * V + v] + (bb > 0.f ? log2((double)bb) : 0.0);
    const double sc = (double)a.alpha[(size_t)V + v];
    double acc = 0.0;
    for (int e = a.sseg_ptr[s]; e < a.sseg_ptr[s + 1]; ++e) {
      double ln = a.lU01[cur][e];
      if (bb > 0.f) {
        ln = a.src_logR[e] - p1;
        mism += a.src_R[e] * fabs(exp2(a.lU01[cur][e] - ln) - 1.0);
      } else {
        lost = 1;
      }
      a.lU01[nxt][e] = ln;
      acc += exp2(ln - sc);
    }
    const float f = (float)acc;
    rg.see(f);
    rc[v] = f;
  }
  __syncthreads();
  { float *tmp = rp; rp = rc; rc = tmp; }
  // forward sweep with the capacity updates, t = 2..T-1
  for (int t = 2; t <= T - 1; ++t) {
    const size_t o = (size_t)t * S;
    const float *bn = a.bm + (size_t)(t + 1) * V;
    float rsum = 0.f;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      const float bb = bn[v];
      float acc = 0.f;
      for (int k = a.in_ptr[v]; k < a.in_ptr[v + 1]; ++k) {
        const float a0 = rp[a.in_tail[k]];
        float g = a.Gf[o + k];
        const float dc = a.Dc[o + k];
        if (dc != INFINITY) {
          const float x = a0 * bb;
          const float uc = ldexpf(1.f, -a.nu[o + k]);
          const float un = x > 0.f ? fminf(__fdiv_rn(dc, x), uc) : uc;
          rsum += fabsf(un - a.w[cur][o + k]) * fminf(x * a.Fc[o + k], FLT_MAX);
          a.w[nxt][o + k] = un;
          if (un > 0.f) rg.lo = fminf(rg.lo, un);   // u_t must not drop out of the FP32 range
          g *= un;
        }
        acc = fmaf(a0, g, acc);
      }
      rg.see(acc);
      rc[v] = acc;
    }
    res += (double)rsum;
    __syncthreads();
    float *tmp = rp; rp = rc; rc = tmp;
  }
  // rp = a_{T-1}.  Sink update U0T <- R0T / hatPsi_T
  for (int s = threadIdx.x; s < a.n_zseg; s += blockDim.x) {
    const int v = a.zseg_node[s];
    const float aa = rp[v];
    const double p = (double)a.alpha[(size_t)(T - 1) * V + v] + (aa > 0.f ? log2((double)aa) : 0.0);
    for (int e = a.zseg_ptr[s]; e < a.zseg_ptr[s + 1]; ++e) {
      if (aa > 0.f) a.lU0T[nxt][e] = a.snk_logR[e] - p;
      else { a.lU0T[nxt][e] = a.lU0T[cur][e]; lost = 1; }
    }
  }
  __syncthreads();
  *mism_out = block_sum(mism, red);
  *res_out = block_sum(res, red);
  const double nlost = block_sum((double)(lost | (rg.bad ? 1 : 0)), red);
  const float hi = block_max(rg.hi, redf);
  const float inv_lo = block_max(rg.lo > 0.f ? 1.f / rg.lo : 0.f, redf);
  *drift = (hi > kDrift || inv_lo > kDrift) ? 1 : 0;
  return (nlost > 0.0 || hi > kLost || inv_lo > kLost) ? 1 : 0;
}

// Duals in from the problem (init = 2), or the initialisation of Algorithm 2 (init = 1:
// u_t = 1, U01 = U0T = 1 on the supports).  States without a capacity at t keep w = 1, nu = 0 in
// both buffers.
__device__ void load_duals(const LinArgs &a, int cur, int init) {
  const int S = a.S, T = a.T, n = (T - 2) * S;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int t = 2 + idx / S, k = idx - (t - 2) * S;
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
    a.w[cur][q] = wv;
    a.nu[q] = nu;
    if (ld.x == INFINITY) a.w[cur ^ 1][q] = 1.f;
  }
  for (int e = threadIdx.x; e < a.n_src; e += blockDim.x) a.lU01[cur][e] = init == 2 ? a.p_src_logU[a.src_tri[e]] : 0.0;
  for (int e = threadIdx.x; e < a.n_snk; e += blockDim.x) a.lU0T[cur][e] = init == 2 ? a.p_snk_logU[a.snk_tri[e]] : 0.0;
  __syncthreads();
}

// Duals out to the problem: log2 u_t = nu + log2 w as a float-float pair; U01, U0T per triple.
__device__ void store_duals(const LinArgs &a, int cur) {
  const int S = a.S, T = a.T, n = (T - 2) * S;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int t = 2 + idx / S, k = idx - (t - 2) * S;
    const size_t q = (size_t)t * S + k;
    const float2 ld = a.logd[(size_t)t * a.drs + k];
    float2 lu = make_float2(0.f, 0.f);
    if (ld.x != INFINITY) {
      const float wv = a.w[cur][q];
      if (wv > 0.f) {
        float h, l;
        two_sum((float)a.nu[q], log2f(wv), h, l);
        lu = make_float2(h, l);
      } else {
        lu = make_float2(kNegLog, 0.f);
      }
    }
    a.p_logu[(size_t)t * S + a.in_state[k]] = lu;
  }
  for (int e = threadIdx.x; e < a.n_src; e += blockDim.x) a.p_src_logU[a.src_tri[e]] = a.lU01[cur][e];
  for (int e = threadIdx.x; e < a.n_snk; e += blockDim.x) a.p_snk_logU[a.snk_tri[e]] = a.lU0T[cur][e];
}

struct LinShared {
  LinArgs a;
  double red[32];
  float redf[32];
};

// Up to max_passes passes on problem blockIdx.x, stopping at tol (tol < 0: never).  init: 0 =
// continue (state kept in the argument block), 1 = initial duals, 2 = the problem's duals.
__global__ void __launch_bounds__(kLinThreads) k_linear(LinArgs *const *args, int max_passes, double tol, int init) {
  __shared__ LinShared sh;
  extern __shared__ float rows[];   // [2][V]
  LinArgs *g = args[blockIdx.x];
  if (threadIdx.x == 0) sh.a = *g;
  __syncthreads();
  const LinArgs &a = sh.a;
  if (init == 0 && a.done) {   // finished in an earlier launch: report no new passes
    if (threadIdx.x == 0) { a.rep->passes = 0; a.rep->log_passes = 0; a.rep->rescalings = 0; }
    return;
  }
  int cur = a.cur, need = init ? 1 : a.need;
  if (init) load_duals(a, cur, init);
  int passes = 0, log_passes = 0, rescalings = 0, status = OTS_OK, converged = 0;
  double src = 0.0, cap = 0.0;
  while (passes < max_passes) {
    if (need) {
      status = log_sweep(a, cur, false, rows, nullptr, nullptr, sh.red);
      if (status) break;
      rebuild(a, cur);
      ++rescalings;
      need = 0;
    }
    double mism, res;
    int drift = 0;
    const int lost = linear_pass(a, cur, rows, &mism, &res, &drift, sh.red, sh.redf);
    if (lost) {
      // thrown away: the same pass again in log arithmetic, from the same duals
      status = log_sweep(a, cur, true, rows, &mism, &res, sh.red);
      cur ^= 1;
      ++log_passes;
      if (status) { ++passes; break; }
      rebuild(a, cur);
      ++rescalings;
    } else {
      cur ^= 1;
      need = drift;
    }
    ++passes;
    src = mism / a.mass;
    cap = res / a.mass;
    if (!(src == src) || !(cap == cap)) { status = OTS_ERR_NUMERIC; break; }
    if (!lost && src <= tol && cap <= tol) { converged = 1; break; }
  }
  __syncthreads();
  store_duals(a, cur);
  if (threadIdx.x == 0) {
    g->cur = cur;
    g->need = need;
    g->done = converged || status != OTS_OK;
    LinReport r;
    r.passes = passes; r.log_passes = log_passes; r.rescalings = rescalings; r.status = status;
    r.converged = converged; r.pad = 0; r.src = src; r.cap = cap;
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
  if (p->V > 16384) return fail(OTS_ERR_INVALID_ARG, "the linear-domain path holds two message rows of %d nodes in shared memory (at most 16384)", p->V);
  const int V = p->V, S = p->S, T = p->T;
  // in-CSR by head node, out-CSR by tail node
  std::vector<int> in_ptr(V + 1, 0), out_ptr(V + 1, 0), in_state(S), in_tail(S), in_head(S), pos_in(S);
  std::vector<int> out_tail(S), out_head(S), out_to_in(S);
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
      out_tail[k] = p->tail[s]; out_head[k] = p->head[s]; out_to_in[k] = pos_in[s];
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
    std::vector<double> R, logR;
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
      sd.R.push_back(bd.tri_R[q]);
      sd.logR.push_back(std::log2(bd.tri_R[q]));
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
               o_out_head = m.take(4 * S), o_out_to_in = m.take(4 * S), o_kappa = m.take(8 * kappa.size()),
               o_logd = m.take(8 * logd.size()), o_gf = m.take(4 * TS), o_gb = m.take(4 * TS), o_dc = m.take(4 * TS),
               o_fc = m.take(4 * TS), o_nu = m.take(4 * TS), o_w0 = m.take(4 * TS), o_w1 = m.take(4 * TS),
               o_alpha = m.take(4 * TV), o_beta = m.take(4 * TV), o_bm = m.take(4 * TV),
               o_ssn = m.take(4 * std::max(nss, 1)), o_ssp = m.take(4 * (nss + 1)), o_zsn = m.take(4 * std::max(nzs, 1)),
               o_zsp = m.take(4 * (nzs + 1)), o_sR = m.take(8 * std::max(ns, 1)), o_slR = m.take(8 * std::max(ns, 1)),
               o_zR = m.take(8 * std::max(nz, 1)), o_zlR = m.take(8 * std::max(nz, 1)), o_u01a = m.take(8 * std::max(ns, 1)),
               o_u01b = m.take(8 * std::max(ns, 1)), o_u0ta = m.take(8 * std::max(nz, 1)), o_u0tb = m.take(8 * std::max(nz, 1)),
               o_stri = m.take(4 * std::max(ns, 1)), o_ztri = m.take(4 * std::max(nz, 1)), o_args = m.take(sizeof(LinArgs)),
               o_argp = m.take(sizeof(LinArgs *)), o_rep = m.take(sizeof(LinReport));
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
  h.n_src = ns; h.n_snk = nz; h.n_sseg = nss; h.n_zseg = nzs; h.mass = mass;
  h.in_ptr = (int *)at(o_in_ptr); h.in_tail = (int *)at(o_in_tail); h.in_head = (int *)at(o_in_head);
  h.in_state = (int *)at(o_in_state); h.out_ptr = (int *)at(o_out_ptr); h.out_tail = (int *)at(o_out_tail);
  h.out_head = (int *)at(o_out_head); h.out_to_in = (int *)at(o_out_to_in);
  h.kappa = (float2 *)at(o_kappa); h.logd = (float2 *)at(o_logd);
  h.Gf = (float *)at(o_gf); h.Gb = (float *)at(o_gb); h.Dc = (float *)at(o_dc); h.Fc = (float *)at(o_fc);
  h.nu = (int *)at(o_nu); h.w[0] = (float *)at(o_w0); h.w[1] = (float *)at(o_w1);
  h.alpha = (float *)at(o_alpha); h.beta = (float *)at(o_beta); h.bm = (float *)at(o_bm);
  h.sseg_node = (int *)at(o_ssn); h.sseg_ptr = (int *)at(o_ssp); h.zseg_node = (int *)at(o_zsn); h.zseg_ptr = (int *)at(o_zsp);
  h.src_R = (double *)at(o_sR); h.src_logR = (double *)at(o_slR); h.snk_R = (double *)at(o_zR); h.snk_logR = (double *)at(o_zlR);
  h.lU01[0] = (double *)at(o_u01a); h.lU01[1] = (double *)at(o_u01b); h.lU0T[0] = (double *)at(o_u0ta); h.lU0T[1] = (double *)at(o_u0tb);
  h.src_tri = (int *)at(o_stri); h.snk_tri = (int *)at(o_ztri);
  h.p_logu = p->d_logu; h.p_src_logU = p->src.d_tri_logU; h.p_snk_logU = p->snk.d_tri_logU;
  L->d_rep = (LinReport *)at(o_rep);
  h.rep = L->d_rep;
  h.cur = 0; h.need = 1; h.done = 0; h.pad = 0;
  L->d_args = (LinArgs *)at(o_args);
  L->d_argp = (LinArgs **)at(o_argp);
  L->smem = 2 * V * (int)sizeof(float);
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
  if (!e) e = put(o_kappa, kappa.data(), 8 * kappa.size());
  if (!e) e = put(o_logd, logd.data(), 8 * logd.size());
  if (!e) e = put(o_ssn, side[0].seg_node.data(), 4 * nss);
  if (!e) e = put(o_ssp, side[0].seg_ptr.data(), 4 * (nss + 1));
  if (!e) e = put(o_zsn, side[1].seg_node.data(), 4 * nzs);
  if (!e) e = put(o_zsp, side[1].seg_ptr.data(), 4 * (nzs + 1));
  if (!e) e = put(o_sR, side[0].R.data(), 8 * ns);
  if (!e) e = put(o_slR, side[0].logR.data(), 8 * ns);
  if (!e) e = put(o_zR, side[1].R.data(), 8 * nz);
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

ots_status linear_run(ots_problem *const *ps, int n, int max_passes, double tol, int init, double *kernel_ms) {
  int smem = 0;
  for (int i = 0; i < n; ++i) smem = std::max(smem, ps[i]->lin->smem);
  if (smem > 48 * 1024)
    OTS_CUDA(cudaFuncSetAttribute(k_linear, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
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
  k_linear<<<n, kLinThreads, smem, s>>>(argp, max_passes, tol, init);
  cudaError_t le = cudaGetLastError();
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

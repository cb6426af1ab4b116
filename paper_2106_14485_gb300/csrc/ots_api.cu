// ots_api.cu -- host side of the C ABI declared in include/ots.h.
//
// Builds the state graph of the road network (directed edges plus wait loops, Sections 3.1
// and 3.3), its node-level CSR views (states entering / leaving each node), the boundary
// triples of R01 and R0T, uploads everything into one device arena, captures one pass of
// Algorithm 2 as a CUDA graph, and runs the passes until the convergence measures reach
// the tolerance.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ots.h"
#include "ots_device.cuh"
#include "ots_internal.h"

using namespace ots;
using namespace ots_host;

namespace ots_host {

thread_local std::string g_last_error;

ots_status fail(ots_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

void clear_error() { g_last_error.clear(); }

void *problem_alloc(ots_problem *p, size_t bytes) {
  if (p->alloc) return p->alloc(bytes, p->actx);
  void *ptr = nullptr;
  if (cudaMalloc(&ptr, bytes) != cudaSuccess) return nullptr;
  return ptr;
}

void problem_free(ots_problem *p, void *ptr) {
  if (!ptr) return;
  if (p->free_fn) p->free_fn(ptr, p->actx);
  else cudaFree(ptr);
}

}  // namespace ots_host

namespace {

void *dev_alloc(ots_problem *p, size_t bytes) { return problem_alloc(p, bytes); }

void dev_free(ots_problem *p, void *ptr) { problem_free(p, ptr); }

// Thread mapping for L commodities: G threads per node (power of two <= 256), C chunks of 4.
bool choose_mapping(int L, int want_G, int &G, int &C, int &Lp) {
  int q = (L + 3) / 4;
  if (want_G > 0) {
    if ((want_G & (want_G - 1)) != 0 || want_G > 256) return false;
    G = want_G;
    C = (q + G - 1) / G;
    if (G < 256 && C != 1) return false;
  } else if (q <= 256) {
    G = 1;
    while (G < q) G <<= 1;
    C = 1;
  } else {
    G = 256;
    C = (q + 255) / 256;
  }
  if (C > 4 || (C == 3 && G != 256)) return false;
  Lp = 4 * G * C;
  return true;
}

StepArgs step_args(ots_problem *p, bool fwd, int t, int mode) {
  StepArgs a{};
  a.V = p->V;
  a.Lp = p->Lp;
  a.qs = p->qs;
  if (fwd) {
    a.ptr = p->d_in_ptr; a.state = p->d_in_state; a.nbr = p->d_in_nbr;
    a.x_hi = p->a_hi(t - 1); a.x_lo = p->a_lo(t - 1);
    a.y_hi = p->b_hi(t + 1); a.y_lo = p->b_lo(t + 1);
    a.out_hi = p->a_hi(t); a.out_lo = p->a_lo(t);
  } else {
    a.ptr = p->d_out_ptr; a.state = p->d_out_state; a.nbr = p->d_out_nbr;
    a.x_hi = p->b_hi(t + 1); a.x_lo = p->b_lo(t + 1);
    a.out_hi = p->b_hi(t); a.out_lo = p->b_lo(t);
  }
  const size_t klo = p->tv ? (size_t)t * p->S : 0;   // time-varying costs: row t
  a.kl_hi = p->d_kl_hi + klo; a.kl_lo = p->d_kl_lo + klo;
  a.klc_hi = p->d_klc_hi; a.klc_lo = p->d_klc_lo;
  const size_t dlo = p->cv ? (size_t)t * p->S : 0;   // per-interval capacities: row t
  a.logd_hi = p->d_logd_hi + dlo; a.logd_lo = p->d_logd_lo + dlo;
  a.cap = p->d_cap + dlo;
  a.lu_t = p->d_logu + (size_t)t * p->S;
  a.w_hi_t = p->d_w_hi + (size_t)t * p->S;
  a.w_lo_t = p->d_w_lo + (size_t)t * p->S;
  a.flow_t = p->d_flow + (size_t)t * p->S;
  a.persist_grid_fwd = p->pgrid_fwd;
  a.persist_grid_bwd = p->pgrid_bwd;
  a.in_kl_hi = p->d_in_kl_hi ? p->d_in_kl_hi + klo : nullptr;
  a.in_kl_lo = p->d_in_kl_lo ? p->d_in_kl_lo + klo : nullptr;
  a.in_logd_hi = p->d_in_logd_hi ? p->d_in_logd_hi + dlo : nullptr;
  a.in_logd_lo = p->d_in_logd_lo ? p->d_in_logd_lo + dlo : nullptr;
  a.in_cap = p->d_in_cap ? p->d_in_cap + dlo : nullptr;
  a.in_outpos = p->d_in_outpos;
  a.lu_in_t = p->d_logu_in + (size_t)t * p->S;
  a.cref_in_t = p->d_cref_in ? p->d_cref_in + (size_t)t * p->S : nullptr;
  a.dc = p->d_dc;
  a.uc_t = p->d_uc ? p->d_uc + (size_t)t * p->S * p->Lp : nullptr;
  a.wout_hi_t = p->d_wout_hi + (size_t)t * p->S;
  a.wout_lo_t = p->d_wout_lo + (size_t)t * p->S;
  a.partials = p->d_partials;
  a.counter = p->d_counter;
  a.stats = p->d_stats;
  a.mode = mode;
  a.wait_tries = p->wait_tries;
  a.withhold_stage = p->withhold_stage;
  a.fixed_w = p->d_fixed_w;
  a.slot = fwd && p->d_slots ? p->d_slots + (size_t)t * 2 * p->max_grid : nullptr;
  return a;
}

// Boundary kernel arguments for all segments of a side (g < 0), or for group g of a problem
// with commodity windows: the segments whose commodities enter (sources) or leave (sinks) at
// time t.  Sources read Psi_t = B_{t+1} and write hatPsi_{t+1} = A_t; sinks read hatPsi_t =
// A_{t-1} and write Psi_{t-1} = B_t.  An update (mode 0) of a group that enters after t = 1
// or leaves before T writes no panel: its rows are put into A_t / B_t when the sweep gets there
// (mode 1).  Groups after the first add their measures to the pass totals.
BndArgs bnd_args(ots_problem *p, bool source, int mode, int g) {
  Boundary &b = source ? p->src : p->snk;
  int s0 = 0, s1 = b.n_seg, t = source ? 1 : p->T;
  if (g >= 0) { s0 = b.grp_seg[g]; s1 = b.grp_seg[g + 1]; t = b.grp_t[g]; }
  BndArgs a{};
  a.skip_node = p->null_row;                   // -1 unless the state graph is explicit
  a.n_seg = s1 - s0;
  a.qs = p->qs;
  a.seg_ptr = b.d_seg_ptr + s0; a.seg_node = b.d_seg_node + s0; a.seg_l = b.d_seg_l + s0;
  a.tri_node_other = b.d_tri_other;
  a.tri_R = b.d_tri_R; a.tri_logR = b.d_tri_logR; a.tri_logU = b.d_tri_logU;
  a.Lp = p->Lp;
  if (source) {
    a.msg_hi = p->b_hi(t + 1); a.msg_lo = p->b_lo(t + 1);
    if (mode == 1 || t == 1) { a.out_hi = p->a_hi(t); a.out_lo = p->a_lo(t); }
  } else {
    a.msg_hi = p->a_hi(t - 1); a.msg_lo = p->a_lo(t - 1);
    if (mode == 1 || t == p->T) { a.out_hi = p->b_hi(t); a.out_lo = p->b_lo(t); }
  }
  a.partials = p->d_partials; a.counter = p->d_counter; a.stats = p->d_stats;
  a.mode = mode;
  a.is_source = source ? 1 : 0;
  a.accumulate = g > 0 ? 1 : 0;
  return a;
}

BndArgs bnd_args(ots_problem *p, bool source, int mode) { return bnd_args(p, source, mode, -1); }

int n_groups(const Boundary &b) { return (int)b.grp_t.size(); }

// ---- storage states of an explicit state graph (one row each, see StoreRowArgs) ----
StoreRowArgs store_rows(ots_problem *p, bool fwd, int t, bool boundary) {
  StoreRowArgs a{};
  a.n = p->nstore; a.Lp = p->Lp; a.row0 = p->V; a.qs = p->qs;
  a.state = p->d_store_state;
  a.node = fwd ? p->d_store_tail : p->d_store_head;
  a.p_hi = fwd ? p->a_hi(t) : p->b_hi(t);
  a.p_lo = fwd ? p->a_lo(t) : p->b_lo(t);
  if (!boundary) {
    a.q_hi = fwd ? p->a_hi(t - 1) : p->b_hi(t + 1);
    a.q_lo = fwd ? p->a_lo(t - 1) : p->b_lo(t + 1);
    a.w_hi = p->d_w_hi + (size_t)t * p->S;
    a.w_lo = p->d_w_lo + (size_t)t * p->S;
  }
  return a;
}

// The storage rows of A_1 (sources) or B_T (sinks) once its node rows are written: the row of the
// state's tail (head), then (+) log2 U of the boundary triples on the state itself.
cudaError_t store_boundary(ots_problem *p, bool source) {
  if (!p->nstore) return cudaSuccess;
  cudaError_t e = launch_store_rows(store_rows(p, source, source ? 1 : p->T, true), p->stream);
  if (e != cudaSuccess) return e;
  const int n = (int)(source ? p->sst_k.size() : p->zst_k.size());
  if (n == 0) return cudaSuccess;
  StoreTriArgs a{};
  const int *d = source ? p->d_sst : p->d_zst;
  a.n = n; a.Lp = p->Lp; a.row0 = p->V; a.qs = p->qs;
  a.k = d; a.l = d + n; a.q = d + 2 * n;
  a.tri_logU = (source ? p->src : p->snk).d_tri_logU;
  a.p_hi = source ? p->a_hi(1) : p->b_hi(p->T);
  a.p_lo = source ? p->a_lo(1) : p->b_lo(p->T);
  return launch_store_triples(a, p->stream);
}

// Forward step t (mode 0: update, 1: flows): the storage states' own capacity update first (the
// step reads their W_t back), then the node rows, then the storage rows of A_t.
cudaError_t forward_step(ots_problem *p, int t, int mode) {
  if (p->nstore) {
    StepArgs a = step_args(p, true, t, mode);
    a.fixed_w = nullptr;
    StoreUpdArgs u{};
    u.n = p->nstore; u.Lp = p->Lp; u.row0 = p->V; u.state = p->d_store_state;
    u.x_hi = p->a_hi(t - 1); u.x_lo = p->a_lo(t - 1);
    u.y_hi = p->b_hi(t + 1); u.y_lo = p->b_lo(t + 1);
    cudaError_t e = launch_store_update(a, u, p->max_grid, p->stream);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = launch_step(true, p->pc, p->G, p->C, step_args(p, true, t, mode), p->stream);
  if (e != cudaSuccess || !p->nstore) return e;
  return launch_store_rows(store_rows(p, true, t, false), p->stream);
}

// Backward step t: the node rows of B_t, then its storage rows.
cudaError_t backward_step(ots_problem *p, int t) {
  cudaError_t e = launch_step(false, p->pc, p->G, p->C, step_args(p, false, t, 0), p->stream);
  if (e != cudaSuccess || !p->nstore) return e;
  return launch_store_rows(store_rows(p, false, t, false), p->stream);
}

// Kernels a storage state graph adds to a pass (update and rows per forward step, rows per
// backward step, rows and triples at each boundary).
long long store_kernels_per_pass(const ots_problem *p) {
  if (!p->nstore) return 0;
  return 3LL * (p->T - 2) + 2 + (p->sst_k.empty() ? 0 : 1) + (p->zst_k.empty() ? 0 : 1);
}

// Panels of the first sweep step: A_1 from the sources entering at t = 1 (all of them
// without windows), B_T from the sinks leaving at T.
cudaError_t launch_boundary_rebuild(ots_problem *p, bool source) {
  if (!p->win) {
    cudaError_t e = launch_boundary(bnd_args(p, source, 1), p->stream);
    if (e != cudaSuccess) return e;
    return store_boundary(p, source);
  }
  const Boundary &b = source ? p->src : p->snk;
  const int t0 = source ? 1 : p->T;
  for (int g = 0; g < n_groups(b); ++g)
    if (b.grp_t[g] == t0) return launch_boundary(bnd_args(p, source, 1, g), p->stream);
  return cudaSuccess;
}

// Commodity windows, after forward step t (A_t written): rows of the commodities entering at t
// into A_t; the update (or, in flows mode, the boundary flows) of the sinks leaving at t+1 < T,
// which read A_t.
cudaError_t after_forward_step(ots_problem *p, int t, bool flows) {
  if (!p->win) return cudaSuccess;
  for (int g = 0; g < n_groups(p->src); ++g)
    if (p->src.grp_t[g] == t) {
      cudaError_t e = launch_boundary(bnd_args(p, true, 1, g), p->stream);
      if (e != cudaSuccess) return e;
      p->kernels_launched += 1;
    }
  for (int g = 0; g < n_groups(p->snk); ++g)
    if (p->snk.grp_t[g] == t + 1 && t + 1 < p->T) {
      cudaError_t e;
      if (!flows) {
        e = launch_boundary(bnd_args(p, false, 0, g), p->stream);
      } else {
        const Boundary &b = p->snk;
        const int q0 = b.seg_ptr[b.grp_seg[g]], q1 = b.seg_ptr[b.grp_seg[g + 1]];
        e = launch_boundary_flows(q1 - q0, p->Lp, p->qs, b.d_tri_l + q0, b.d_tri_other + q0, b.d_tri_logU + q0,
                                  p->a_hi(t), p->a_lo(t), b.d_flow + q0, p->stream);
      }
      if (e != cudaSuccess) return e;
      p->kernels_launched += 1;
    }
  return cudaSuccess;
}

// Commodity windows, after backward step t (B_t written): rows of the commodities leaving at t.
cudaError_t after_backward_step(ots_problem *p, int t) {
  if (!p->win) return cudaSuccess;
  for (int g = 0; g < n_groups(p->snk); ++g)
    if (p->snk.grp_t[g] == t) {
      cudaError_t e = launch_boundary(bnd_args(p, false, 1, g), p->stream);
      if (e != cudaSuccess) return e;
      p->kernels_launched += 1;
    }
  return cudaSuccess;
}

// Source update at the start of a pass (mode 0): every group reads its own Psi_t.
cudaError_t launch_source_update(ots_problem *p) {
  if (!p->win) {
    cudaError_t e = launch_boundary(bnd_args(p, true, 0), p->stream);
    if (e != cudaSuccess) return e;
    return store_boundary(p, true);
  }
  for (int g = 0; g < n_groups(p->src); ++g) {
    cudaError_t e = launch_boundary(bnd_args(p, true, 0, g), p->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Sink update after the forward sweep (mode 0): the sinks leaving at T.
cudaError_t launch_sink_update(ots_problem *p) {
  if (!p->win) {
    cudaError_t e = launch_boundary(bnd_args(p, false, 0), p->stream);
    if (e != cudaSuccess) return e;
    return store_boundary(p, false);
  }
  for (int g = 0; g < n_groups(p->snk); ++g)
    if (p->snk.grp_t[g] == p->T) return launch_boundary(bnd_args(p, false, 0, g), p->stream);
  return cudaSuccess;
}

// Boundary flows of the sources (all groups; each reads its Psi_t) and of the sinks leaving at T.
cudaError_t launch_boundary_flows_all(ots_problem *p) {
  const Boundary &bs = p->src, &bz = p->snk;
  for (int g = 0; g < std::max(1, n_groups(bs)); ++g) {
    const int s0 = bs.grp_seg.empty() ? 0 : bs.grp_seg[g], s1 = bs.grp_seg.empty() ? bs.n_seg : bs.grp_seg[g + 1];
    const int t = bs.grp_t.empty() ? 1 : bs.grp_t[g];
    const int q0 = bs.seg_ptr.empty() ? 0 : bs.seg_ptr[s0], q1 = bs.seg_ptr.empty() ? 0 : bs.seg_ptr[s1];
    cudaError_t e = launch_boundary_flows(q1 - q0, p->Lp, p->qs, bs.d_tri_l + q0, bs.d_tri_other + q0,
                                          bs.d_tri_logU + q0, p->b_hi(t + 1), p->b_lo(t + 1), bs.d_flow + q0, p->stream);
    if (e != cudaSuccess) return e;
  }
  for (int g = 0; g < std::max(1, n_groups(bz)); ++g) {
    const int t = bz.grp_t.empty() ? p->T : bz.grp_t[g];
    if (t != p->T) continue;                     // earlier exits: after_forward_step
    const int s0 = bz.grp_seg.empty() ? 0 : bz.grp_seg[g], s1 = bz.grp_seg.empty() ? bz.n_seg : bz.grp_seg[g + 1];
    const int q0 = bz.seg_ptr.empty() ? 0 : bz.seg_ptr[s0], q1 = bz.seg_ptr.empty() ? 0 : bz.seg_ptr[s1];
    cudaError_t e = launch_boundary_flows(q1 - q0, p->Lp, p->qs, bz.d_tri_l + q0, bz.d_tri_other + q0,
                                          bz.d_tri_logU + q0, p->a_hi(p->T - 1), p->a_lo(p->T - 1), bz.d_flow + q0,
                                          p->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Backward sweep of Algorithm 2 ("Compute Psi_t"), from the current duals.
ots_status enqueue_backward_sweep(ots_problem *p) {
  OTS_CUDA(launch_boundary_rebuild(p, false));
  for (int t = p->T - 1; t >= 2; --t) {
    OTS_CUDA(backward_step(p, t));
    OTS_CUDA(after_backward_step(p, t));
  }
  p->kernels_launched += p->T - 1;
  return OTS_OK;
}

// With backward panels kept only every bk-th t, a forward step t whose B_{t+1} has no slot of
// its own starts a segment: the panels up to the next kept one are recomputed by backward steps
// from it, with the weights the last backward sweep used (the forward sweep has not updated
// them yet), so they equal the panels that sweep computed.
cudaError_t enqueue_segment(ots_problem *p, int t) {
  if (p->bk <= 1 || p->b_stored(t + 1) || !p->b_stored(t)) return cudaSuccess;
  int hi = t + 2;
  while (!p->b_stored(hi)) ++hi;
  for (int tt = hi - 1; tt >= t + 1; --tt) {
    cudaError_t e = launch_step(false, p->pc, p->G, p->C, step_args(p, false, tt, 0), p->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

long long kernels_per_pass(const ots_problem *p) {
  return 2LL * p->T + p->b_recompute + store_kernels_per_pass(p) + (p->d_slots ? 1 : 0);
}

// One pass of the while loop of Algorithm 2 (enqueued directly or captured into a graph),
// with phase events around the source update, the forward sweep, the sink update and the
// backward sweep.
ots_status enqueue_pass(ots_problem *p, bool capture) {
  // inside a graph the marks become external event-record nodes, usable for timing
  const unsigned flags = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
  OTS_CUDA(launch_pass_begin(p->d_stats, p->stream));
  OTS_CUDA(cudaEventRecordWithFlags(p->ev[0], p->stream, flags));
  OTS_CUDA(launch_source_update(p));                                           // U01, hatPsi_2
  OTS_CUDA(cudaEventRecordWithFlags(p->ev[1], p->stream, flags));
  for (int t = 2; t <= p->T - 1; ++t) {                                        // u_t, hatPsi_{t+1}
    OTS_CUDA(enqueue_segment(p, t));
    OTS_CUDA(forward_step(p, t, 0));
    OTS_CUDA(after_forward_step(p, t, false));
  }
  OTS_CUDA(cudaEventRecordWithFlags(p->ev[2], p->stream, flags));
  OTS_CUDA(launch_sink_update(p));                                             // U0T, Psi_{T-1}
  OTS_CUDA(cudaEventRecordWithFlags(p->ev[3], p->stream, flags));
  for (int t = p->T - 1; t >= 2; --t) {                                        // Psi_{t-1}
    OTS_CUDA(backward_step(p, t));
    OTS_CUDA(after_backward_step(p, t));
  }
  OTS_CUDA(cudaEventRecordWithFlags(p->ev[4], p->stream, flags));
  OTS_CUDA(launch_pass_end(p->d_stats, p->d_report, p->mass, p->eps, p->d_slots, 2 * p->max_grid, p->max_grid, p->T,
                           p->d_step_tot, p->stream));
  return OTS_OK;
}

ots_status build_pass_graph(ots_problem *p) {
  if (p->pass_exec) return OTS_OK;
  cudaGraph_t g = nullptr;
  OTS_CUDA(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  ots_status st = enqueue_pass(p, true);
  cudaError_t e = cudaStreamEndCapture(p->stream, &g);
  if (st != OTS_OK) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) return fail(OTS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&p->pass_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { p->pass_exec = nullptr; return fail(OTS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
  return OTS_OK;
}

// Reset the duals to the initialisation of Algorithm 2 (u_t = 1, U01 = U0T = 1 on the
// supports) and recompute the backward messages.
ots_status reset_duals(ots_problem *p) {
  p->kernels_launched += 2;
  OTS_CUDA(launch_weights(p->S, p->T, p->qs, p->pc ? nullptr : p->d_kl_hi, p->pc ? nullptr : p->d_kl_lo,
                          p->tv ? p->S : 0, p->d_logu, p->d_w_hi, p->d_w_lo, 1, p->d_st_inpos, p->d_st_outpos,
                          p->d_logu_in, p->d_wout_hi, p->d_wout_lo, p->stream));
  if (p->src.n) OTS_CUDA(cudaMemsetAsync(p->src.d_tri_logU, 0, sizeof(double) * p->src.n, p->stream));
  if (p->snk.n) OTS_CUDA(cudaMemsetAsync(p->snk.d_tri_logU, 0, sizeof(double) * p->snk.n, p->stream));
  if (p->d_uc) OTS_CUDA(cudaMemsetAsync(p->d_uc, 0, sizeof(float) * (size_t)(p->T + 1) * p->S * p->Lp, p->stream));
  // column references of the pipelined forward step are dropped too (NaN: none), so that a
  // reset problem repeats a fresh one bit for bit whatever ran on it before
  if (p->d_cref_in)
    OTS_CUDA(cudaMemsetAsync(p->d_cref_in, 0xff, sizeof(float) * (size_t)(p->T + 1) * p->S, p->stream));
  OTS_CUDA(cudaMemsetAsync(p->d_report, 0, sizeof(PassReport), p->stream));
  OTS_CUDA(launch_boundary_rebuild(p, true));
  ots_status st = enqueue_backward_sweep(p);
  if (st) return st;
  p->stale = false;
  return OTS_OK;
}

ots_status refresh_if_stale(ots_problem *p) {
  if (!p->stale) return OTS_OK;
  p->kernels_launched += 2;
  OTS_CUDA(launch_weights(p->S, p->T, p->qs, p->pc ? nullptr : p->d_kl_hi, p->pc ? nullptr : p->d_kl_lo,
                          p->tv ? p->S : 0, p->d_logu, p->d_w_hi, p->d_w_lo, 0, p->d_st_inpos, p->d_st_outpos,
                          p->d_logu_in, p->d_wout_hi, p->d_wout_lo, p->stream));
  OTS_CUDA(launch_boundary_rebuild(p, true));
  ots_status st = enqueue_backward_sweep(p);
  if (st) return st;
  p->stale = false;
  return OTS_OK;
}

ots_status run_passes(ots_problem *p, int n, bool use_graph) {
  if (use_graph) {
    ots_status st = build_pass_graph(p);
    if (st) return st;
    for (int k = 0; k < n; ++k) OTS_CUDA(cudaGraphLaunch(p->pass_exec, p->stream));
  } else {
    for (int k = 0; k < n; ++k) {
      ots_status st = enqueue_pass(p, false);
      if (st) return st;
    }
  }
  p->passes_total += n;
  p->kernels_launched += (long long)n * kernels_per_pass(p);
  return OTS_OK;
}

ots_status read_report(ots_problem *p, ots_solve_report *rep) {
  OTS_CUDA(cudaMemcpyAsync(p->h_report, p->d_report, sizeof(PassReport), cudaMemcpyDeviceToHost, p->stream));
  p->d2h_bytes += sizeof(PassReport);
  OTS_CUDA(cudaStreamSynchronize(p->stream));
  rep->src_residual = p->h_report->src_resid_rel;
  rep->cap_violation = p->h_report->cap_viol_rel;
  rep->dual_objective = p->h_report->dual_objective;
  // a wait that gave up adds 1e6 per thread, a vanishing boundary message 1 per triple
  if (p->h_report->bad >= 1e6)
    return fail(OTS_ERR_DEVICE_WAIT, "a bounded wait in a pipelined step kernel gave up (the pass is invalid)");
  if (p->h_report->bad > 0) return fail(OTS_ERR_INFEASIBLE, "a source or sink message vanished (infeasible instance)");
  if (std::isnan(rep->src_residual) || std::isnan(rep->cap_violation) || std::isnan(rep->dual_objective))
    return fail(OTS_ERR_NUMERIC, "NaN in the convergence measures");
  return OTS_OK;
}


// Necessary feasibility condition: every sink state is reached by a source state of the same
// commodity, and every source reaches a sink, in exactly T-1 transitions.  With wait loops a
// walk of length k <= T-1 can be padded to T-1, so the test is on hop distances: state j is
// reachable from state i after T-1 transitions iff 1 + dist(head(i), tail(j)) <= T-1 (or
// i == j needs a loop to stay; covered by the same rule when loops exist).
bool feasible(ots_problem *p, const std::vector<int> &eptr, const std::vector<int> &enbr, std::string &why) {
  std::map<int, std::vector<int>> cache;
  auto dist_from = [&](int s) -> const std::vector<int> & {
    auto it = cache.find(s);
    if (it != cache.end()) return it->second;
    std::vector<int> d(p->V, -1);
    std::vector<int> q;
    q.reserve(p->V);
    d[s] = 0;
    q.push_back(s);
    for (size_t h = 0; h < q.size(); ++h) {
      int u = q[h];
      for (int k = eptr[u]; k < eptr[u + 1]; ++k) {
        int w = enbr[k];
        if (d[w] < 0) { d[w] = d[u] + 1; q.push_back(w); }
      }
    }
    return cache.emplace(s, std::move(d)).first->second;
  };
  // group triples by commodity
  std::vector<std::vector<int>> src_by_l(p->L), snk_by_l(p->L);
  for (int q = 0; q < p->src.n; ++q) src_by_l[p->src.tri_l[q]].push_back(q);
  for (int q = 0; q < p->snk.n; ++q) snk_by_l[p->snk.tri_l[q]].push_back(q);
  for (int l = 0; l < p->L; ++l) {
    std::vector<char> snk_hit(snk_by_l[l].size(), 0);
    for (int qs : src_by_l[l]) {
      const std::vector<int> &d = dist_from(p->head[p->src.tri_state[qs]]);
      bool any = false;
      for (size_t k = 0; k < snk_by_l[l].size(); ++k) {
        int j = p->snk.tri_state[snk_by_l[l][k]];
        int dd = d[p->tail[j]];
        if (dd >= 0 && 1 + dd <= p->tb[l] - p->ta[l]) { any = true; snk_hit[k] = 1; }
      }
      if (!any) {
        char buf[160];
        snprintf(buf, sizeof(buf), "commodity %d: source state %d reaches no sink within t_out - t_in transitions", l,
                 p->src.tri_state[qs]);
        why = buf;
        return false;
      }
    }
    for (size_t k = 0; k < snk_hit.size(); ++k) {
      if (!snk_hit[k]) {
        char buf[160];
        snprintf(buf, sizeof(buf), "commodity %d: sink state %d is reached by no source within t_out - t_in transitions", l,
                 p->snk.tri_state[snk_by_l[l][k]]);
        why = buf;
        return false;
      }
    }
  }
  return true;
}

// Explicit state graphs (storage states, states without a tail or head): the same necessary
// condition on exact walks, without the hop-distance shortcut (waiting is possible only where
// a state may follow itself).  Layered reachability over the states: after a state s comes every
// state j with tail(j) = head(s) >= 0, and s itself when it may follow itself (a storage flag, or
// head(s) = tail(s)); a state with capacity 0 in every interval is closed in the interior layers.
bool feasible_states(ots_problem *p, const std::vector<int> &hold, const std::vector<double> &cap, std::string &why) {
  const int S = p->S, T = p->T;
  std::vector<char> open(S, 0);
  for (int s = 0; s < S; ++s) {
    if (!p->cv) open[s] = cap[s] > 0.0;
    else
      for (int t = 2; t <= T - 1; ++t) open[s] |= cap[(size_t)t * S + s] > 0.0;
  }
  std::vector<std::vector<int>> leaving(p->V);
  for (int s = 0; s < S; ++s)
    if (p->tail[s] >= 0) leaving[p->tail[s]].push_back(s);
  auto reach = [&](int s0) {                      // states reachable from s0 in exactly T-1 steps
    std::vector<char> cur(S, 0), nxt(S, 0);
    cur[s0] = 1;
    for (int step = 1; step <= T - 1; ++step) {
      std::fill(nxt.begin(), nxt.end(), 0);
      const bool last = step == T - 1;
      for (int s = 0; s < S; ++s) {
        if (!cur[s]) continue;
        if ((hold[s] || (p->head[s] >= 0 && p->head[s] == p->tail[s])) && (last || open[s])) nxt[s] = 1;
        if (p->head[s] >= 0)
          for (int j : leaving[p->head[s]])
            if (last || open[j]) nxt[j] = 1;
      }
      cur.swap(nxt);
    }
    return cur;
  };
  std::vector<std::vector<int>> src_by_l(p->L), snk_by_l(p->L);
  for (int q = 0; q < p->src.n; ++q) src_by_l[p->src.tri_l[q]].push_back(q);
  for (int q = 0; q < p->snk.n; ++q) snk_by_l[p->snk.tri_l[q]].push_back(q);
  char buf[160];
  for (int l = 0; l < p->L; ++l) {
    std::vector<char> hit(snk_by_l[l].size(), 0);
    for (int qs : src_by_l[l]) {
      const std::vector<char> r = reach(p->src.tri_state[qs]);
      bool any = false;
      for (size_t k = 0; k < snk_by_l[l].size(); ++k)
        if (r[p->snk.tri_state[snk_by_l[l][k]]]) { any = true; hit[k] = 1; }
      if (!any) {
        snprintf(buf, sizeof(buf), "commodity %d: source state %d reaches no sink in T-1 transitions", l,
                 p->src.tri_state[qs]);
        why = buf;
        return false;
      }
    }
    for (size_t k = 0; k < hit.size(); ++k)
      if (!hit[k]) {
        snprintf(buf, sizeof(buf), "commodity %d: sink state %d is reached by no source in T-1 transitions", l,
                 p->snk.tri_state[snk_by_l[l][k]]);
        why = buf;
        return false;
      }
  }
  return true;
}

ots_status build_boundary(ots_problem *p, Boundary &b, int n, const int32_t *comm, const int32_t *state,
                          const double *mass, bool source) {
  std::map<std::pair<int, int>, int> uniq;  // (l, state) -> unique index
  std::vector<std::pair<int, int>> keys;
  std::vector<double> R;
  b.input_to_tri.resize(n);
  for (int q = 0; q < n; ++q) {
    if (comm[q] < 0 || comm[q] >= p->L) return fail(OTS_ERR_INVALID_ARG, "triple %d: commodity %d out of range", q, comm[q]);
    if (state[q] < 0 || state[q] >= p->S) return fail(OTS_ERR_INVALID_ARG, "triple %d: state %d out of range", q, state[q]);
    if (!(mass[q] > 0.0) || !std::isfinite(mass[q]))
      return fail(OTS_ERR_INVALID_ARG, "triple %d: mass must be positive and finite", q);
    auto key = std::make_pair((int)comm[q], (int)state[q]);
    auto it = uniq.find(key);
    if (it == uniq.end()) {
      uniq[key] = (int)keys.size();
      b.input_to_tri[q] = (int)keys.size();
      keys.push_back(key);
      R.push_back(mass[q]);
    } else {
      b.input_to_tri[q] = it->second;
      R[it->second] += mass[q];
    }
  }
  // order unique triples by (time of the commodity, segment node, commodity, state); the time
  // is the entry time for sources and the exit time for sinks (1 and T without windows)
  const int nu = (int)keys.size();
  std::vector<int> order(nu);
  for (int k = 0; k < nu; ++k) order[k] = k;
  auto seg_node_of = [&](int k) {   // the node row the boundary panel entry goes to (log-0 row: none)
    const int v = source ? p->head[keys[k].second] : p->tail[keys[k].second];
    return v >= 0 ? v : p->null_row;
  };
  auto time_of = [&](int l) { return source ? p->ta[l] : p->tb[l]; };
  std::sort(order.begin(), order.end(), [&](int a, int c) {
    const int ta = time_of(keys[a].first), tc = time_of(keys[c].first);
    if (ta != tc) return ta < tc;
    int na = seg_node_of(a), nc = seg_node_of(c);
    if (na != nc) return na < nc;
    if (keys[a].first != keys[c].first) return keys[a].first < keys[c].first;
    return keys[a].second < keys[c].second;
  });
  std::vector<int> rank(nu);
  for (int k = 0; k < nu; ++k) rank[order[k]] = k;
  for (int q = 0; q < n; ++q) b.input_to_tri[q] = rank[b.input_to_tri[q]];
  b.n = nu;
  b.tri_l.resize(nu); b.tri_state.resize(nu); b.tri_other.resize(nu); b.tri_R.resize(nu);
  b.seg_ptr.clear(); b.seg_node.clear(); b.seg_l.clear();
  for (int k = 0; k < nu; ++k) {
    int u = order[k];
    b.tri_l[k] = keys[u].first;
    b.tri_state[k] = keys[u].second;
    // message row read at the boundary: Psi_1 = B_2[head(i)] for sources, hatPsi_T = A_{T-1}[tail(j)]
    // for sinks (a storage state's own row, or the log-0 row without head / tail)
    b.tri_other[k] = source ? p->brow[keys[u].second] : p->frow[keys[u].second];
    b.tri_R[k] = R[u];
    int node = seg_node_of(u);
    if (k == 0 || node != b.seg_node.back() || keys[u].first != b.seg_l.back()) {
      b.seg_ptr.push_back(k);
      b.seg_node.push_back(node);
      b.seg_l.push_back(keys[u].first);
    }
  }
  b.seg_ptr.push_back(nu);
  b.n_seg = (int)b.seg_node.size();
  b.grp_t.clear();
  b.grp_seg.clear();
  for (int g = 0; g < b.n_seg; ++g) {
    const int t = time_of(b.seg_l[g]);
    if (b.grp_t.empty() || b.grp_t.back() != t) {
      b.grp_t.push_back(t);
      b.grp_seg.push_back(g);
    }
  }
  b.grp_seg.push_back(b.n_seg);
  return OTS_OK;
}

// Arena carving helper.
struct Carver {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    size_t o = align_up(off, 256);
    off = o + align_up(count * sizeof(T), 256);
    return o;
  }
};

}  // namespace

extern "C" {

const char *ots_status_string(ots_status s) {
  switch (s) {
    case OTS_OK: return "OTS_OK";
    case OTS_ERR_INVALID_ARG: return "OTS_ERR_INVALID_ARG";
    case OTS_ERR_INFEASIBLE: return "OTS_ERR_INFEASIBLE";
    case OTS_ERR_NOT_CONVERGED: return "OTS_ERR_NOT_CONVERGED";
    case OTS_ERR_TIMEOUT: return "OTS_ERR_TIMEOUT";
    case OTS_ERR_OOM: return "OTS_ERR_OOM";
    case OTS_ERR_CUDA: return "OTS_ERR_CUDA";
    case OTS_ERR_NUMERIC: return "OTS_ERR_NUMERIC";
    case OTS_PENDING: return "OTS_PENDING";
    case OTS_ERR_DEVICE_WAIT: return "OTS_ERR_DEVICE_WAIT";
  }
  return "OTS_ERR_UNKNOWN";
}

const char *ots_last_error(void) { return g_last_error.c_str(); }

ots_status ots_default_solve_opts(ots_solve_opts *o) {
  if (!o) return fail(OTS_ERR_INVALID_ARG, "opts is NULL");
  o->tol = 1e-6;
  o->max_iters = 100000;
  o->check_every = 10;
  o->timeout_ms = 0.0;
  o->warm_start = 0;
  o->use_graph = 1;
  o->threads_per_node = 0;
  o->eps_stages = 0;
  o->eps_start = 0.0;
  o->eps_stage_tol = 0.0;
  return OTS_OK;
}

void ots_destroy_problem(ots_problem *p) {
  if (!p) return;
  DeviceGuard guard(p->dev);
  if (p->stream && !p->member) cudaStreamSynchronize(p->stream);   // a batch orders its own frees
  if (p->pass_exec) cudaGraphExecDestroy(p->pass_exec);
  for (int k = 0; k < 5; ++k)
    if (p->ev[k]) cudaEventDestroy(p->ev[k]);
  linear_release(p);
  if (p->arena) dev_free(p, p->arena);
  if (p->h_report) cudaFreeHost(p->h_report);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

ots_status ots_create_problem(const ots_problem_desc *d, ots_problem **out) {
  g_last_error.clear();
  return create_problem_impl(d, CreateOpts{}, out);
}

ots_status ots_check_problem(const ots_problem_desc *d) {
  g_last_error.clear();
  ots_problem *p = nullptr;
  const ots_status st = build_problem_host(d, CreateOpts{}, &p);
  if (st) return st;
  delete p;   // the host part holds no device resource: no stream, arena, events or pinned memory yet
  return OTS_OK;
}

}  // extern "C"

// Host part of the construction (no CUDA call): validation, state graph, per-state data,
// boundary triples, feasibility; the arrays to upload stay in p->host.
ots_status ots_host::build_problem_host(const ots_problem_desc *d, const CreateOpts &co, ots_problem **out) {
  if (!d || !out) return fail(OTS_ERR_INVALID_ARG, "desc or out is NULL");
  *out = nullptr;
  if (d->n_nodes < 1 || d->n_edges < 0) return fail(OTS_ERR_INVALID_ARG, "n_nodes must be >= 1 and n_edges >= 0");
  if (d->n_edges > 0 && (!d->edge_src || !d->edge_dst)) return fail(OTS_ERR_INVALID_ARG, "edge_src / edge_dst missing");
  if (d->T < 3) return fail(OTS_ERR_INVALID_ARG, "T must be >= 3 (Algorithm 2 needs hatPsi_2 and Psi_{T-1})");
  if (d->L < 1 || d->L > 4096) return fail(OTS_ERR_INVALID_ARG, "L must be in [1, 4096]");
  if (!(d->eps > 0.0) || !std::isfinite(d->eps)) return fail(OTS_ERR_INVALID_ARG, "eps must be > 0");
  if ((d->alloc == nullptr) != (d->free_fn == nullptr)) return fail(OTS_ERR_INVALID_ARG, "alloc and free_fn go together");
  if (d->n_sources < 1 || d->n_sinks < 1) return fail(OTS_ERR_INVALID_ARG, "need at least one source and one sink");
  if (!d->src_commodity || !d->src_state || !d->src_mass || !d->snk_commodity || !d->snk_state || !d->snk_mass)
    return fail(OTS_ERR_INVALID_ARG, "source / sink arrays missing");

  ots_problem *p = new (std::nothrow) ots_problem();
  if (!p) return fail(OTS_ERR_OOM, "host allocation failed");
  p->dev = d->device;
  p->alloc = d->alloc;
  p->free_fn = d->free_fn;
  p->actx = d->alloc_ctx;
  p->V = d->n_nodes;
  p->rows = p->V;
  p->E = d->n_edges;
  p->S = d->n_edges + (d->add_wait_loops ? d->n_nodes : 0);
  p->L = d->L;
  p->T = d->T;
  p->eps = d->eps;
  p->pc = d->commodity_cost != nullptr || d->commodity_capacity != nullptr;
  p->cc = d->commodity_capacity != nullptr;
  p->member = co.member;
  if (p->S < 1) { delete p; return fail(OTS_ERR_INVALID_ARG, "no states"); }
  if (d->psi_stride < 0) { delete p; return fail(OTS_ERR_INVALID_ARG, "psi_stride must be >= 0"); }
  p->bk = co.member ? 1 : std::max(1, (int)d->psi_stride);
  {
    // slots of the backward panels: one per kept t, then k - 1 shared recompute slots (a
    // t between two kept ones uses slot first_recompute + (next kept above t) - 1 - t)
    p->bslot.assign((size_t)p->T + 1, 0);
    int nk = 0;
    for (int t = 2; t <= p->T; ++t)
      if (p->b_stored(t)) p->bslot[t] = nk++;
    int maxgap = 0;
    p->b_recompute = 0;
    for (int t = 2; t <= p->T; ++t) {
      if (p->b_stored(t)) continue;
      int hi = t + 1;
      while (!p->b_stored(hi)) ++hi;
      p->bslot[t] = nk + (hi - 1 - t);
      maxgap = std::max(maxgap, hi - t);
      ++p->b_recompute;
    }
    p->nbslots = nk + maxgap;
  }
  if (co.member) {
    if (p->pc) { delete p; return fail(OTS_ERR_INVALID_ARG, "batched instances take commodity-independent costs"); }
    if (!d->stream) { delete p; return fail(OTS_ERR_INVALID_ARG, "batch member without a stream"); }
    p->G = co.G;
    p->C = co.C;
    p->Lp = 4 * co.G * co.C;
    if (p->Lp < p->L) { delete p; return fail(OTS_ERR_INVALID_ARG, "mapping too narrow for L"); }
  } else if (!choose_mapping(p->L, 0, p->G, p->C, p->Lp)) {
    delete p;
    return fail(OTS_ERR_INVALID_ARG, "unsupported L");
  }

  auto bail = [&](ots_status s) { ots_destroy_problem(p); return s; };

  // ---- state graph (Sections 3.1, 3.3) ----
  p->tail.resize(p->S);
  p->head.resize(p->S);
  for (int e = 0; e < p->E; ++e) {
    if (d->edge_src[e] < 0 || d->edge_src[e] >= p->V || d->edge_dst[e] < 0 || d->edge_dst[e] >= p->V)
      return bail(fail(OTS_ERR_INVALID_ARG, "edge %d: node index out of range", e));
    p->tail[e] = d->edge_src[e];
    p->head[e] = d->edge_dst[e];
  }
  if (d->add_wait_loops)
    for (int v = 0; v < p->V; ++v) { p->tail[p->E + v] = v; p->head[p->E + v] = v; }

  // ---- explicit state graph (Section 3.3: storage on edges, the traffic-routing model) ----
  std::vector<int> hold(p->S, 0);
  if (d->state_tail || d->state_head || d->state_hold) {
    if (!d->state_tail || !d->state_head) return bail(fail(OTS_ERR_INVALID_ARG, "state_tail and state_head go together"));
    for (int s = 0; s < p->S; ++s) {
      const int tl = d->state_tail[s], hd = d->state_head[s], h = d->state_hold ? d->state_hold[s] : 0;
      if (tl < -1 || tl >= p->V || hd < -1 || hd >= p->V)
        return bail(fail(OTS_ERR_INVALID_ARG, "state %d: tail / head must be -1 or a node", s));
      if (h != 0 && h != 1) return bail(fail(OTS_ERR_INVALID_ARG, "state %d: state_hold must be 0 or 1", s));
      p->tail[s] = tl;
      p->head[s] = hd;
      hold[s] = h;
    }
    p->xgraph = true;
  }
  if (p->xgraph) {
    if (co.member) return bail(fail(OTS_ERR_INVALID_ARG, "the batched solver takes no explicit state graph"));
    if (p->pc) return bail(fail(OTS_ERR_INVALID_ARG, "an explicit state graph does not combine with per-commodity costs or capacities"));
    if (p->bk > 1) return bail(fail(OTS_ERR_INVALID_ARG, "an explicit state graph needs psi_stride <= 1"));
    if (d->commodity_t_in || d->commodity_t_out)
      return bail(fail(OTS_ERR_INVALID_ARG, "an explicit state graph does not combine with commodity windows"));
    // a state that may follow itself other than through its own node needs a row of its own
    for (int s = 0; s < p->S; ++s)
      if (hold[s] && !(p->head[s] >= 0 && p->head[s] == p->tail[s])) {
        p->store_state.push_back(s);
        p->store_tail.push_back(p->tail[s]);
        p->store_head.push_back(p->head[s]);
      }
    p->nstore = (int)p->store_state.size();
    p->null_row = p->V + p->nstore;
    p->rows = p->V + p->nstore + 1;
  }
  // message rows gathered for each state: its tail's (forward) / head's (backward) node row, its
  // own row when it is a storage state, the log-0 row when it has no tail / head
  p->frow.resize(p->S);
  p->brow.resize(p->S);
  {
    std::vector<int> sidx(p->S, -1);
    for (int k = 0; k < p->nstore; ++k) sidx[p->store_state[k]] = k;
    for (int s = 0; s < p->S; ++s) {
      p->frow[s] = sidx[s] >= 0 ? p->V + sidx[s] : (p->tail[s] >= 0 ? p->tail[s] : p->null_row);
      p->brow[s] = sidx[s] >= 0 ? p->V + sidx[s] : (p->head[s] >= 0 ? p->head[s] : p->null_row);
    }
  }

  std::vector<int> in_ptr(p->V + 1, 0), out_ptr(p->V + 1, 0);
  for (int s = 0; s < p->S; ++s) {
    if (p->head[s] >= 0) in_ptr[p->head[s] + 1]++;
    if (p->tail[s] >= 0) out_ptr[p->tail[s] + 1]++;
  }
  for (int v = 0; v < p->V; ++v) { in_ptr[v + 1] += in_ptr[v]; out_ptr[v + 1] += out_ptr[v]; }
  // in_state / out_state list every state once: the node lists first, then (explicit graphs)
  // the states with no head / tail, which no node gathers
  std::vector<int> in_state(p->S), in_nbr(p->S), out_state(p->S), out_nbr(p->S);
  {
    std::vector<int> fi(in_ptr.begin(), in_ptr.end() - 1), fo(out_ptr.begin(), out_ptr.end() - 1);
    int xi = in_ptr[p->V], xo = out_ptr[p->V];
    for (int s = 0; s < p->S; ++s) {
      int k = p->head[s] >= 0 ? fi[p->head[s]]++ : xi++;
      in_state[k] = s; in_nbr[k] = p->frow[s];
      k = p->tail[s] >= 0 ? fo[p->tail[s]]++ : xo++;
      out_state[k] = s; out_nbr[k] = p->brow[s];
    }
  }
  // node adjacency for the feasibility BFS (edges with positive capacity)
  std::vector<int> eptr(p->V + 1, 0), enbr;
  {
    std::vector<std::vector<int>> adj(p->V);
    for (int e = 0; e < p->E; ++e) {
      double cap = d->edge_capacity ? d->edge_capacity[e] : INFINITY;
      if (d->state_capacity_t) {   // usable if open in some interval
        cap = 0.0;
        for (int t = 2; t <= p->T - 1; ++t) cap = std::max(cap, d->state_capacity_t[(size_t)(t - 2) * (p->E + p->V) + e]);
      }
      if (cap > 0.0 && p->tail[e] >= 0 && p->head[e] >= 0 && p->tail[e] != p->head[e]) adj[p->tail[e]].push_back(p->head[e]);
    }
    for (int v = 0; v < p->V; ++v) { eptr[v + 1] = eptr[v] + (int)adj[v].size(); enbr.insert(enbr.end(), adj[v].begin(), adj[v].end()); }
  }

  // ---- per-state data (costs, capacities) in log2 units ----
  p->tv = d->state_cost_t != nullptr;
  if (p->tv && p->pc) return bail(fail(OTS_ERR_INVALID_ARG, "state_cost_t does not combine with commodity_cost or commodity_capacity"));
  const size_t KR = p->tv ? (size_t)(p->T + 1) : 1;   // rows of log2 K_L (row t for interval t)
  p->cv = d->state_capacity_t != nullptr;
  const size_t DR = p->cv ? (size_t)(p->T + 1) : 1;   // rows of the capacities (row t for interval t)
  std::vector<float> kl_hi(KR * p->S, 0.f), kl_lo(KR * p->S, 0.f), logd_hi(DR * p->S, 0.f), logd_lo(DR * p->S, 0.f);
  p->cost_nat.assign(KR * p->S, 0.0);
  std::vector<double> cap(DR * p->S, INFINITY);
  auto set_cap = [&](size_t q, double dd) {
    cap[q] = dd;
    if (dd == 0.0) { logd_hi[q] = kNeg; logd_lo[q] = 0.f; }
    else if (std::isinf(dd)) { logd_hi[q] = 0.f; logd_lo[q] = 0.f; }
    else split_ff(std::log2(dd), logd_hi[q], logd_lo[q]);
  };
  if (p->cv) {
    for (int t = 2; t <= p->T - 1; ++t)
      for (int s = 0; s < p->S; ++s) {
        const double dd = d->state_capacity_t[(size_t)(t - 2) * p->S + s];
        if (std::isnan(dd) || dd < 0.0)
          return bail(fail(OTS_ERR_INVALID_ARG, "state_capacity_t[%d][%d] must be >= 0 (inf for none)", t - 2, s));
        set_cap((size_t)t * p->S + s, dd);
      }
  }
  double cmax_tv = 0.0;
  if (p->tv) {
    for (int t = 2; t <= p->T - 1; ++t)
      for (int s = 0; s < p->S; ++s) {
        const double c = d->state_cost_t[(size_t)(t - 2) * p->S + s];
        const size_t q = (size_t)t * p->S + s;
        if (std::isnan(c) || c == -INFINITY)
          return bail(fail(OTS_ERR_INVALID_ARG, "state_cost_t[%d][%d] must be finite or +inf", t - 2, s));
        p->cost_nat[q] = c;
        if (c == INFINITY) { kl_hi[q] = kNeg; kl_lo[q] = 0.f; continue; }   // closed in interval t
        split_ff(-c / d->eps * kInvLn2, kl_hi[q], kl_lo[q]);
        cmax_tv = std::max(cmax_tv, std::fabs(c) / d->eps * kInvLn2);
      }
  }
  for (int s = 0; s < p->S; ++s) {
    double c = 0.0, dd = INFINITY;
    if (s < p->E) {
      if (d->edge_cost) c = d->edge_cost[s];
      if (d->edge_capacity) dd = d->edge_capacity[s];
    } else {
      int v = s - p->E;
      if (d->wait_cost) c = d->wait_cost[v];
      if (d->wait_capacity) dd = d->wait_capacity[v];
    }
    if (!p->tv && !std::isfinite(c)) return bail(fail(OTS_ERR_INVALID_ARG, "state %d: cost must be finite", s));
    if (std::isnan(dd) || dd < 0.0) return bail(fail(OTS_ERR_INVALID_ARG, "state %d: capacity must be >= 0", s));
    if (!p->tv) {
      split_ff(-c / d->eps * kInvLn2, kl_hi[s], kl_lo[s]);
      p->cost_nat[s] = c;
    }
    if (!p->cv) set_cap(s, dd);
  }
  p->cap_nat = cap;
  // quantum of the hi parts: the magnitude of any message is bounded by about (T+1) times the
  // largest per-interval cost in bits; q = 2^k with that bound below 2^24 q keeps hi sums exact
  {
    double cmax = cmax_tv;
    if (!p->tv)
      for (int s = 0; s < p->S; ++s) cmax = std::max(cmax, std::fabs((double)kl_hi[s]));
    if (d->commodity_cost)
      for (size_t k = 0; k < (size_t)p->L * p->S; ++k) cmax = std::max(cmax, std::fabs(d->commodity_cost[k]) / d->eps * kInvLn2);
    const double bound = (p->T + 1.0) * std::max(cmax, 1.0) + 256.0;
    int k = (int)std::ceil(std::log2(bound)) - 23;
    k = std::min(std::max(k, -40), -2);
    p->qs.q = std::ldexp(1.0f, k);
    p->qs.inv_q = std::ldexp(1.0f, -k);
    p->qs.lo_unit = std::ldexp(1.0f, k - 16);
    p->qs.lo_inv = std::ldexp(1.0f, 16 - k);
  }
  std::vector<float> klc_hi;
  std::vector<lo_t> klc_lo;
  if (p->pc) {
    klc_hi.assign((size_t)p->S * p->Lp, kNeg);
    klc_lo.assign((size_t)p->S * p->Lp, kLoZero);
    const double q = p->qs.q;
    for (int l = 0; l < p->L; ++l)
      for (int s = 0; s < p->S; ++s) {
        // per-commodity costs, or the state costs for every commodity (commodity capacities alone)
        double c = d->commodity_cost ? d->commodity_cost[(size_t)l * p->S + s]
                   : s < p->E ? (d->edge_cost ? d->edge_cost[s] : 0.0)
                              : (d->wait_cost ? d->wait_cost[s - p->E] : 0.0);
        if (!std::isfinite(c)) return bail(fail(OTS_ERR_INVALID_ARG, "commodity_cost must be finite"));
        const double x = -c / d->eps * kInvLn2;
        double h = std::nearbyint(x / q) * q;
        int units = (int)std::nearbyint((x - h) * 65536.0 / q);   // in [-32768, 32768]
        if (units > 32767) { units -= 65536; h += q; }            // x - h = q/2 exactly
        klc_hi[(size_t)s * p->Lp + l] = (float)h;
        klc_lo[(size_t)s * p->Lp + l] = (lo_t)(units + 32768);
      }
  }

  // ---- CSR-ordered copies (positions of every state in the in / out lists) ----
  std::vector<int> st_inpos(p->S), st_outpos(p->S), in_outpos(p->S);
  for (int k = 0; k < p->S; ++k) { st_inpos[in_state[k]] = k; st_outpos[out_state[k]] = k; }
  p->in_state_h = in_state;
  for (int k = 0; k < p->S; ++k) in_outpos[k] = st_outpos[in_state[k]];
  std::vector<float> in_kl_hi(KR * p->S), in_kl_lo(KR * p->S), in_logd_hi(DR * p->S), in_logd_lo(DR * p->S);
  std::vector<float2> in_cap(DR * p->S), cap2(DR * p->S);
  auto split_cap = [](double dd) {
    if (!(dd < 3.0e38)) return make_float2(INFINITY, 0.f);        // no capacity (or beyond FP32)
    const float h = (float)dd;
    return make_float2(h, (float)(dd - (double)h));
  };
  for (size_t q = 0; q < DR * p->S; ++q) cap2[q] = split_cap(cap[q]);
  for (int k = 0; k < p->S; ++k) {
    const int st = in_state[k];
    for (size_t r = 0; r < KR; ++r) {
      in_kl_hi[r * p->S + k] = kl_hi[r * p->S + st];
      in_kl_lo[r * p->S + k] = kl_lo[r * p->S + st];
    }
    for (size_t r = 0; r < DR; ++r) {
      in_logd_hi[r * p->S + k] = logd_hi[r * p->S + st];
      in_logd_lo[r * p->S + k] = logd_lo[r * p->S + st];
      in_cap[r * p->S + k] = cap2[r * p->S + st];
    }
  }

  // ---- commodity windows (entry / exit times) ----
  p->ta.assign(p->L, 1);
  p->tb.assign(p->L, p->T);
  for (int l = 0; l < p->L; ++l) {
    if (d->commodity_t_in) p->ta[l] = d->commodity_t_in[l];
    if (d->commodity_t_out) p->tb[l] = d->commodity_t_out[l];
    if (p->ta[l] < 1 || p->tb[l] > p->T || p->ta[l] >= p->tb[l])
      return bail(fail(OTS_ERR_INVALID_ARG, "commodity %d: need 1 <= t_in < t_out <= T", l));
    if (p->ta[l] != 1 || p->tb[l] != p->T) p->win = true;
  }
  if (p->win && p->member) return bail(fail(OTS_ERR_INVALID_ARG, "the batched solver takes no commodity windows"));
  if (p->win && p->bk > 1) return bail(fail(OTS_ERR_INVALID_ARG, "commodity windows need psi_stride <= 1"));

  // ---- boundary triples ----
  ots_status st = build_boundary(p, p->src, d->n_sources, d->src_commodity, d->src_state, d->src_mass, true);
  if (st) return bail(st);
  st = build_boundary(p, p->snk, d->n_sinks, d->snk_commodity, d->snk_state, d->snk_mass, false);
  if (st) return bail(st);
  if (p->nstore) {                               // boundary triples on storage states
    std::vector<int> sidx(p->S, -1);
    for (int k = 0; k < p->nstore; ++k) sidx[p->store_state[k]] = k;
    for (int q = 0; q < p->src.n; ++q)
      if (sidx[p->src.tri_state[q]] >= 0) {
        p->sst_k.push_back(sidx[p->src.tri_state[q]]); p->sst_l.push_back(p->src.tri_l[q]); p->sst_q.push_back(q);
      }
    for (int q = 0; q < p->snk.n; ++q)
      if (sidx[p->snk.tri_state[q]] >= 0) {
        p->zst_k.push_back(sidx[p->snk.tri_state[q]]); p->zst_l.push_back(p->snk.tri_l[q]); p->zst_q.push_back(q);
      }
  }
  {
    std::vector<double> ms(p->L, 0.0), mz(p->L, 0.0);
    for (int q = 0; q < p->src.n; ++q) ms[p->src.tri_l[q]] += p->src.tri_R[q];
    for (int q = 0; q < p->snk.n; ++q) mz[p->snk.tri_l[q]] += p->snk.tri_R[q];
    p->mass = 0.0;
    for (int l = 0; l < p->L; ++l) {
      if (ms[l] <= 0.0 || mz[l] <= 0.0)
        return bail(fail(OTS_ERR_INVALID_ARG, "commodity %d has no source or no sink", l));
      if (std::fabs(ms[l] - mz[l]) > 1e-9 * std::max(ms[l], mz[l]))
        return bail(fail(OTS_ERR_INVALID_ARG, "commodity %d: source mass %.17g != sink mass %.17g", l, ms[l], mz[l]));
      p->mass += ms[l];
    }
  }
  {
    std::string why;
    if (p->xgraph ? !feasible_states(p, hold, cap, why) : !feasible(p, eptr, enbr, why))
      return bail(fail(OTS_ERR_INFEASIBLE, "%s", why.c_str()));
  }

  p->stream = (cudaStream_t)d->stream;          // NULL: the device step creates one
  p->host.reset(new (std::nothrow) HostArrays());
  if (!p->host) return bail(fail(OTS_ERR_OOM, "host allocation failed"));
  HostArrays &H = *p->host;
  H.in_ptr = std::move(in_ptr);
  H.out_ptr = std::move(out_ptr);
  H.in_state = std::move(in_state);
  H.in_nbr = std::move(in_nbr);
  H.out_state = std::move(out_state);
  H.out_nbr = std::move(out_nbr);
  H.st_inpos = std::move(st_inpos);
  H.st_outpos = std::move(st_outpos);
  H.in_outpos = std::move(in_outpos);
  H.kl_hi = std::move(kl_hi);
  H.kl_lo = std::move(kl_lo);
  H.logd_hi = std::move(logd_hi);
  H.logd_lo = std::move(logd_lo);
  H.in_kl_hi = std::move(in_kl_hi);
  H.in_kl_lo = std::move(in_kl_lo);
  H.in_logd_hi = std::move(in_logd_hi);
  H.in_logd_lo = std::move(in_logd_lo);
  H.klc_hi = std::move(klc_hi);
  H.in_cap = std::move(in_cap);
  H.cap = std::move(cap2);
  H.klc_lo = std::move(klc_lo);
  if (p->cc) {
    // log2 D per (state, commodity) in the panel layout: +inf none, log 0 closed
    H.dc.assign((size_t)p->S * p->Lp, make_float2(INFINITY, 0.f));
    for (int l = 0; l < p->L; ++l)
      for (int s = 0; s < p->S; ++s) {
        const double dd = d->commodity_capacity[(size_t)l * p->S + s];
        if (std::isnan(dd) || dd < 0.0)
          return bail(fail(OTS_ERR_INVALID_ARG, "commodity_capacity[%d][%d] must be >= 0 (inf for none)", l, s));
        float2 &v = H.dc[(size_t)s * p->Lp + l];
        if (dd == 0.0) v = make_float2(kNeg, 0.f);
        else if (std::isfinite(dd)) split_ff(std::log2(dd), v.x, v.y);
      }
  }
  *out = p;
  return OTS_OK;
}

// Device part of the construction: stream, kernel set-up, one arena for all device arrays,
// uploads of the host arrays kept by the host part (released at the end), initial duals.
// On failure the caller destroys p.
ots_status ots_host::build_problem_device(ots_problem *p) {
  if (!p || !p->host) return fail(OTS_ERR_INVALID_ARG, "problem has no host arrays to upload");
  HostArrays &H = *p->host;
  auto &in_ptr = H.in_ptr;
  auto &out_ptr = H.out_ptr;
  auto &in_state = H.in_state;
  auto &in_nbr = H.in_nbr;
  auto &out_state = H.out_state;
  auto &out_nbr = H.out_nbr;
  auto &st_inpos = H.st_inpos;
  auto &st_outpos = H.st_outpos;
  auto &in_outpos = H.in_outpos;
  auto &kl_hi = H.kl_hi;
  auto &kl_lo = H.kl_lo;
  auto &logd_hi = H.logd_hi;
  auto &logd_lo = H.logd_lo;
  auto &in_kl_hi = H.in_kl_hi;
  auto &in_kl_lo = H.in_kl_lo;
  auto &in_logd_hi = H.in_logd_hi;
  auto &in_logd_lo = H.in_logd_lo;
  auto &klc_hi = H.klc_hi;
  auto &cap = H.cap;
  auto &in_cap = H.in_cap;
  auto &klc_lo = H.klc_lo;
  auto bail = [&](ots_status s) { return s; };
  ots_status st = OTS_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return bail(fail(OTS_ERR_CUDA, "no CUDA device"));
  if (p->dev < 0 || p->dev >= ndev) return bail(fail(OTS_ERR_INVALID_ARG, "device %d out of range", p->dev));
  DeviceGuard guard(p->dev);
  if (p->stream) {
    p->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(OTS_ERR_CUDA, "stream creation failed"));
    p->own_stream = true;
  }
  if (!p->member) {
    if (cudaMallocHost(&p->h_report, sizeof(PassReport)) != cudaSuccess) return bail(fail(OTS_ERR_OOM, "pinned alloc failed"));
    cudaError_t e = prepare_step_kernels(p->G, p->C, p->pc, p->V, &p->pgrid_fwd, &p->pgrid_bwd);
    if (e != cudaSuccess) return bail(fail(OTS_ERR_CUDA, "kernel setup: %s", cudaGetErrorString(e)));
    if (p->xgraph) p->pgrid_fwd = p->pgrid_bwd = 0;   // explicit graphs run on the register kernels
    for (int k = 0; k < 5; ++k)
      if (cudaEventCreate(&p->ev[k]) != cudaSuccess) return bail(fail(OTS_ERR_CUDA, "event creation failed"));
  }
  const bool csr_copies = !p->member;   // in- / out-CSR-ordered copies of the per-state data

  const size_t S = p->S, V = p->V, T = p->T, panel = p->panel();
  const int max_grid = std::max(std::max(step_grid(p->V, p->G), boundary_grid(p->src.n_seg)),
                                std::max(boundary_grid(p->snk.n_seg), 1));
  p->max_grid = max_grid;
  Carver cv;
  size_t o_in_ptr = cv.take<int>(V + 1), o_in_state = cv.take<int>(S), o_in_nbr = cv.take<int>(S);
  size_t o_out_ptr = cv.take<int>(V + 1), o_out_state = cv.take<int>(S), o_out_nbr = cv.take<int>(S);
  size_t o_tail = cv.take<int>(S), o_head = cv.take<int>(S);
  const size_t KR = p->tv ? T + 1 : 1;
  const size_t DR = p->cv ? T + 1 : 1;
  size_t o_kl_hi = cv.take<float>(KR * S), o_kl_lo = cv.take<float>(KR * S), o_ld_hi = cv.take<float>(DR * S),
         o_ld_lo = cv.take<float>(DR * S);
  size_t o_cap = cv.take<float2>(DR * S);
  size_t o_klc_hi = p->pc ? cv.take<float>(S * p->Lp) : 0, o_klc_lo = p->pc ? cv.take<lo_t>(S * p->Lp) : 0;
  size_t o_dc = p->cc ? cv.take<float2>(S * p->Lp) : 0, o_uc = p->cc ? cv.take<float>((T + 1) * S * p->Lp) : 0;
  size_t o_w_hi = cv.take<float>((T + 1) * S), o_w_lo = cv.take<float>((T + 1) * S);
  size_t o_logu = cv.take<float2>((T + 1) * S), o_flow = cv.take<double>((T + 1) * S);
  const size_t Sc = csr_copies ? S : 0;
  size_t o_st_inpos = cv.take<int>(Sc), o_st_outpos = cv.take<int>(Sc), o_in_outpos = cv.take<int>(Sc);
  size_t o_in_kl_hi = cv.take<float>(KR * Sc), o_in_kl_lo = cv.take<float>(KR * Sc),
         o_in_ld_hi = cv.take<float>(DR * Sc), o_in_ld_lo = cv.take<float>(DR * Sc), o_in_cap = cv.take<float2>(DR * Sc);
  size_t o_logu_in = cv.take<float2>((T + 1) * Sc), o_wout_hi = cv.take<float>((T + 1) * Sc),
         o_wout_lo = cv.take<float>((T + 1) * Sc), o_cref_in = cv.take<float>((T + 1) * Sc);
  size_t o_a_hi[3], o_a_lo[3];
  for (int k = 0; k < 3; ++k) { o_a_hi[k] = cv.take<float>(panel); o_a_lo[k] = cv.take<lo_t>(panel); }
  size_t o_b_hi = cv.take<float>((size_t)p->nbslots * panel), o_b_lo = cv.take<lo_t>((size_t)p->nbslots * panel);
  const size_t NS = p->nstore;
  size_t o_store = cv.take<int>(3 * NS), o_fixed = cv.take<unsigned char>(NS ? S : 0);
  size_t o_sst = cv.take<int>(3 * p->sst_k.size()), o_zst = cv.take<int>(3 * p->zst_k.size());
  size_t o_stats = cv.take<DevStats>(1), o_report = cv.take<PassReport>(1);
  size_t o_partials = cv.take<double>(3 * (size_t)max_grid), o_counter = cv.take<unsigned int>(4);
  const size_t n_slots = p->member ? 0 : (T + 1) * 2 * (size_t)max_grid;
  size_t o_slots = cv.take<double>(n_slots), o_step_tot = cv.take<double>(p->member ? 0 : 2 * (T + 1));
  struct BOff { size_t seg_ptr, seg_node, seg_l, other, l, R, logR, logU, flow; } bo[2];
  Boundary *sides[2] = {&p->src, &p->snk};
  for (int k = 0; k < 2; ++k) {
    Boundary &b = *sides[k];
    bo[k].seg_ptr = cv.take<int>(b.n_seg + 1); bo[k].seg_node = cv.take<int>(b.n_seg); bo[k].seg_l = cv.take<int>(b.n_seg);
    bo[k].other = cv.take<int>(b.n); bo[k].l = cv.take<int>(b.n);
    bo[k].R = cv.take<double>(b.n); bo[k].logR = cv.take<double>(b.n); bo[k].logU = cv.take<double>(b.n);
    bo[k].flow = cv.take<double>(b.n);
  }
  p->arena_bytes = cv.off;
  p->arena = dev_alloc(p, p->arena_bytes);
  if (!p->arena) return bail(fail(OTS_ERR_OOM, "device allocation of %zu bytes failed", p->arena_bytes));
  char *base = (char *)p->arena;
  auto at = [&](size_t off) { return (void *)(base + off); };
  p->d_in_ptr = (int *)at(o_in_ptr); p->d_in_state = (int *)at(o_in_state); p->d_in_nbr = (int *)at(o_in_nbr);
  p->d_out_ptr = (int *)at(o_out_ptr); p->d_out_state = (int *)at(o_out_state); p->d_out_nbr = (int *)at(o_out_nbr);
  p->d_tail = (int *)at(o_tail); p->d_head = (int *)at(o_head);
  p->d_kl_hi = (float *)at(o_kl_hi); p->d_kl_lo = (float *)at(o_kl_lo);
  p->d_logd_hi = (float *)at(o_ld_hi); p->d_logd_lo = (float *)at(o_ld_lo);
  p->d_cap = (float2 *)at(o_cap);
  if (p->pc) { p->d_klc_hi = (float *)at(o_klc_hi); p->d_klc_lo = (lo_t *)at(o_klc_lo); }
  if (p->cc) { p->d_dc = (float2 *)at(o_dc); p->d_uc = (float *)at(o_uc); }
  p->d_w_hi = (float *)at(o_w_hi); p->d_w_lo = (float *)at(o_w_lo);
  p->d_logu = (float2 *)at(o_logu); p->d_flow = (double *)at(o_flow);
  if (csr_copies) {
    p->d_st_inpos = (int *)at(o_st_inpos); p->d_st_outpos = (int *)at(o_st_outpos); p->d_in_outpos = (int *)at(o_in_outpos);
    p->d_in_kl_hi = (float *)at(o_in_kl_hi); p->d_in_kl_lo = (float *)at(o_in_kl_lo);
    p->d_in_logd_hi = (float *)at(o_in_ld_hi); p->d_in_logd_lo = (float *)at(o_in_ld_lo);
    p->d_in_cap = (float2 *)at(o_in_cap);
    p->d_logu_in = (float2 *)at(o_logu_in); p->d_wout_hi = (float *)at(o_wout_hi); p->d_wout_lo = (float *)at(o_wout_lo);
    p->d_cref_in = (float *)at(o_cref_in);
  }
  for (int k = 0; k < 3; ++k) { p->d_a_hi[k] = (float *)at(o_a_hi[k]); p->d_a_lo[k] = (lo_t *)at(o_a_lo[k]); }
  p->d_b_hi = (float *)at(o_b_hi); p->d_b_lo = (lo_t *)at(o_b_lo);
  if (NS) {
    p->d_store_state = (int *)at(o_store);
    p->d_store_tail = p->d_store_state + NS;
    p->d_store_head = p->d_store_state + 2 * NS;
    p->d_fixed_w = (unsigned char *)at(o_fixed);
    if (!p->sst_k.empty()) p->d_sst = (int *)at(o_sst);
    if (!p->zst_k.empty()) p->d_zst = (int *)at(o_zst);
  }
  p->d_stats = (DevStats *)at(o_stats); p->d_report = (PassReport *)at(o_report);
  p->d_partials = (double *)at(o_partials); p->d_counter = (unsigned int *)at(o_counter);
  if (n_slots) { p->d_slots = (double *)at(o_slots); p->d_step_tot = (double *)at(o_step_tot); }
  for (int k = 0; k < 2; ++k) {
    Boundary &b = *sides[k];
    b.d_seg_ptr = (int *)at(bo[k].seg_ptr); b.d_seg_node = (int *)at(bo[k].seg_node); b.d_seg_l = (int *)at(bo[k].seg_l);
    b.d_tri_other = (int *)at(bo[k].other); b.d_tri_l = (int *)at(bo[k].l);
    b.d_tri_R = (double *)at(bo[k].R); b.d_tri_logR = (double *)at(bo[k].logR); b.d_tri_logU = (double *)at(bo[k].logU);
    b.d_flow = (double *)at(bo[k].flow);
  }

  auto up = [&](void *dst, const void *srcp, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    p->h2d_bytes += (long long)bytes;
    return cudaMemcpyAsync(dst, srcp, bytes, cudaMemcpyHostToDevice, p->stream);
  };
#define UP(dst, vec) \
  if (up(dst, vec.data(), vec.size() * sizeof(vec[0])) != cudaSuccess) return bail(fail(OTS_ERR_CUDA, "upload " #vec))
  UP(p->d_in_ptr, in_ptr); UP(p->d_in_state, in_state); UP(p->d_in_nbr, in_nbr);
  UP(p->d_out_ptr, out_ptr); UP(p->d_out_state, out_state); UP(p->d_out_nbr, out_nbr);
  UP(p->d_tail, p->frow); UP(p->d_head, p->brow);     // rows gathered for each state (flow queries)
  std::vector<int> stv, sst, zst;                      // kept until the end: the copies are asynchronous
  std::vector<unsigned char> fixed;
  if (NS) {
    stv = p->store_state;
    stv.insert(stv.end(), p->store_tail.begin(), p->store_tail.end());
    stv.insert(stv.end(), p->store_head.begin(), p->store_head.end());
    fixed.assign(S, 0);
    for (int s : p->store_state) fixed[s] = 1;
    sst = p->sst_k;
    zst = p->zst_k;
    sst.insert(sst.end(), p->sst_l.begin(), p->sst_l.end()); sst.insert(sst.end(), p->sst_q.begin(), p->sst_q.end());
    zst.insert(zst.end(), p->zst_l.begin(), p->zst_l.end()); zst.insert(zst.end(), p->zst_q.begin(), p->zst_q.end());
    UP(p->d_store_state, stv); UP(p->d_fixed_w, fixed);
    if (p->d_sst) UP(p->d_sst, sst);
    if (p->d_zst) UP(p->d_zst, zst);
  }
  UP(p->d_kl_hi, kl_hi); UP(p->d_kl_lo, kl_lo); UP(p->d_logd_hi, logd_hi); UP(p->d_logd_lo, logd_lo);
  UP(p->d_cap, cap);
  if (csr_copies) {
    UP(p->d_st_inpos, st_inpos); UP(p->d_st_outpos, st_outpos); UP(p->d_in_outpos, in_outpos);
    UP(p->d_in_kl_hi, in_kl_hi); UP(p->d_in_kl_lo, in_kl_lo); UP(p->d_in_logd_hi, in_logd_hi);
    UP(p->d_in_logd_lo, in_logd_lo); UP(p->d_in_cap, in_cap);
  }
  if (p->pc) { UP(p->d_klc_hi, klc_hi); UP(p->d_klc_lo, klc_lo); }
  if (p->cc) { UP(p->d_dc, H.dc); }
  std::vector<std::vector<double>> logR(2);
  for (int k = 0; k < 2; ++k) {
    Boundary &b = *sides[k];
    logR[k].resize(b.n);
    for (int q = 0; q < b.n; ++q) logR[k][q] = std::log2(b.tri_R[q]);
    UP(b.d_seg_ptr, b.seg_ptr); UP(b.d_seg_node, b.seg_node); UP(b.d_seg_l, b.seg_l);
    UP(b.d_tri_other, b.tri_other); UP(b.d_tri_l, b.tri_l); UP(b.d_tri_R, b.tri_R); UP(b.d_tri_logR, logR[k]);
  }
#undef UP
  p->host.reset();                             // pageable copies have completed
  if (p->member) return OTS_OK;  // duals, panels, accumulators: the batched kernel's set-up step
  // slots of blocks that never run stay 0, so the pass end may add all max_grid of them
  if (n_slots && cudaMemsetAsync(p->d_slots, 0, sizeof(double) * n_slots, p->stream) != cudaSuccess)
    return bail(fail(OTS_ERR_CUDA, "memset failed"));
  if (cudaMemsetAsync(p->d_stats, 0, sizeof(DevStats), p->stream) != cudaSuccess ||
      cudaMemsetAsync(p->d_counter, 0, 4 * sizeof(unsigned int), p->stream) != cudaSuccess ||
      cudaMemsetAsync(p->d_flow, 0, sizeof(double) * (T + 1) * S, p->stream) != cudaSuccess)
    return bail(fail(OTS_ERR_CUDA, "memset failed"));
  // logu rows outside 2..T-1 stay 0; W rows likewise unused
  if (cudaMemsetAsync(p->d_logu, 0, sizeof(float2) * (T + 1) * S, p->stream) != cudaSuccess ||
      cudaMemsetAsync(p->d_logu_in, 0, sizeof(float2) * (T + 1) * S, p->stream) != cudaSuccess ||
      cudaMemsetAsync(p->d_cref_in, 0xff, sizeof(float) * (T + 1) * S, p->stream) != cudaSuccess)   // NaN: none yet
    return bail(fail(OTS_ERR_CUDA, "memset failed"));
  // boundary panels start at log 0 everywhere; only the support entries are rewritten
  p->kernels_launched += 2;
  if (launch_fill_panel(panel, p->a_hi(1), p->a_lo(1), p->stream) != cudaSuccess ||
      launch_fill_panel(panel, p->b_hi(p->T), p->b_lo(p->T), p->stream) != cudaSuccess)
    return bail(fail(OTS_ERR_CUDA, "panel fill failed"));
  if (p->xgraph) {
    // every panel: the log-0 row is never written, and storage rows are read before their first write
    bool ok = true;
    for (int k = 0; k < 3; ++k) ok &= launch_fill_panel(panel, p->d_a_hi[k], p->d_a_lo[k], p->stream) == cudaSuccess;
    ok &= launch_fill_panel((size_t)p->nbslots * panel, p->d_b_hi, p->d_b_lo, p->stream) == cudaSuccess;
    if (!ok) return bail(fail(OTS_ERR_CUDA, "panel fill failed"));
    p->kernels_launched += 4;
  }
  st = reset_duals(p);
  if (st) return bail(st);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return bail(fail(OTS_ERR_CUDA, "%s", cudaGetErrorString(cudaGetLastError())));
  return OTS_OK;
}

ots_status ots_host::create_problem_impl(const ots_problem_desc *d, const CreateOpts &co, ots_problem **out) {
  ots_problem *p = nullptr;
  ots_status st = build_problem_host(d, co, &p);
  if (st) return st;
  st = build_problem_device(p);
  if (st) {
    ots_destroy_problem(p);
    return st;
  }
  *out = p;
  return OTS_OK;
}

extern "C" {

ots_status ots_problem_info(const ots_problem *p, ots_problem_stats *o) {
  if (!p || !o) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  o->n_states = p->S;
  o->n_nodes = p->V;
  o->T = p->T;
  o->L = p->L;
  o->padded_L = p->Lp;
  o->threads_per_node = p->G;
  o->device_bytes = (int64_t)p->arena_bytes;
  o->kernels_per_pass = kernels_per_pass(p);
  o->kernels_launched = p->kernels_launched;
  o->passes_total = p->passes_total;
  o->h2d_bytes = p->h2d_bytes;
  o->d2h_bytes = p->d2h_bytes;
  return OTS_OK;
}

ots_status ots_last_pass_timing(ots_problem *p, double *ms) {
  if (!p || !ms) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  if (p->passes_total == 0) return fail(OTS_ERR_INVALID_ARG, "no pass has run");
  DeviceGuard guard(p->dev);
  OTS_CUDA(cudaStreamSynchronize(p->stream));
  for (int k = 0; k < 4; ++k) {
    float v = 0.f;
    OTS_CUDA(cudaEventElapsedTime(&v, p->ev[k], p->ev[k + 1]));
    ms[k] = v;
  }
  return OTS_OK;
}

ots_status ots_iterate(ots_problem *p, int32_t n, int32_t reset, ots_solve_report *rep) {
  g_last_error.clear();
  if (!p || n < 0) return fail(OTS_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard guard(p->dev);
  auto t0 = std::chrono::steady_clock::now();
  ots_status st = reset ? reset_duals(p) : refresh_if_stale(p);
  if (st) return st;
  st = run_passes(p, n, true);
  if (st) return st;
  ots_solve_report r{};
  st = read_report(p, &r);
  r.iterations = n;
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  r.status = st;
  if (rep) *rep = r;
  return st;
}

namespace {

// Continuation in epsilon (warm starts at larger epsilon; the fixed point at the problem's own
// epsilon is unique, so the final result does not depend on them): rebuild log2 K_L for
// epsilon e, carry the duals over with lambda = -eps ln u held fixed, and mark the messages
// stale.  The quantum of the hi parts, chosen for the smallest epsilon, stays valid.
ots_status set_eps(ots_problem *p, double e) {
  if (e == p->eps) return OTS_OK;
  const size_t S = p->S, KR = p->tv ? (size_t)p->T + 1 : 1;
  std::vector<float> kh(KR * S, 0.f), kl(KR * S, 0.f);
  for (size_t q = 0; q < KR * S; ++q) {
    const size_t t = q / S;
    if (p->tv && (t < 2 || t > (size_t)p->T - 1)) continue;
    const double c = p->cost_nat[q];
    if (c == INFINITY) { kh[q] = kNeg; kl[q] = 0.f; }
    else split_ff(-c / e * kInvLn2, kh[q], kl[q]);
  }
  OTS_CUDA(cudaMemcpyAsync(p->d_kl_hi, kh.data(), sizeof(float) * KR * S, cudaMemcpyHostToDevice, p->stream));
  OTS_CUDA(cudaMemcpyAsync(p->d_kl_lo, kl.data(), sizeof(float) * KR * S, cudaMemcpyHostToDevice, p->stream));
  std::vector<float> ih, il;
  if (p->d_in_kl_hi) {
    ih.resize(KR * S);
    il.resize(KR * S);
    for (size_t r = 0; r < KR; ++r)
      for (size_t k = 0; k < S; ++k) {
        ih[r * S + k] = kh[r * S + p->in_state_h[k]];
        il[r * S + k] = kl[r * S + p->in_state_h[k]];
      }
    OTS_CUDA(cudaMemcpyAsync(p->d_in_kl_hi, ih.data(), sizeof(float) * KR * S, cudaMemcpyHostToDevice, p->stream));
    OTS_CUDA(cudaMemcpyAsync(p->d_in_kl_lo, il.data(), sizeof(float) * KR * S, cudaMemcpyHostToDevice, p->stream));
  }
  const size_t n_lu = (size_t)(p->T + 1) * S;
  OTS_CUDA(launch_scale_duals(p->d_logu, n_lu, p->d_logu_in, p->d_logu_in ? n_lu : 0, p->src.d_tri_logU, p->src.n,
                              p->snk.d_tri_logU, p->snk.n, p->eps / e, p->stream));
  if (p->d_cref_in) OTS_CUDA(cudaMemsetAsync(p->d_cref_in, 0xff, sizeof(float) * n_lu, p->stream));
  p->kernels_launched += 1;
  OTS_CUDA(cudaStreamSynchronize(p->stream));   // the host staging vectors go out of scope
  p->eps = e;
  if (p->pass_exec) {                            // epsilon is an argument of the pass graph
    cudaGraphExecDestroy(p->pass_exec);
    p->pass_exec = nullptr;
  }
  p->stale = true;
  return OTS_OK;
}

}  // namespace

ots_status ots_sinkhorn_solve(ots_problem *p, const ots_solve_opts *opts, ots_solve_report *rep) {
  g_last_error.clear();
  if (!p) return fail(OTS_ERR_INVALID_ARG, "problem is NULL");
  ots_solve_opts o;
  ots_default_solve_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_iters < 1 || o.check_every < 1) return fail(OTS_ERR_INVALID_ARG, "bad solve options");
  if (o.threads_per_node != 0) {
    int G, C, Lp;
    if (!choose_mapping(p->L, o.threads_per_node, G, C, Lp) || Lp != p->Lp)
      return fail(OTS_ERR_INVALID_ARG, "threads_per_node %d is not usable with L = %d", o.threads_per_node, p->L);
  }
  const bool anneal = o.eps_start > p->eps;
  if (anneal && (p->pc || !std::isfinite(o.eps_start) || o.eps_stages < 0))
    return fail(OTS_ERR_INVALID_ARG, "epsilon continuation needs commodity-independent costs and a finite eps_start");
  DeviceGuard guard(p->dev);
  auto t0 = std::chrono::steady_clock::now();
  const double target = p->eps;
  ots_status st = anneal ? set_eps(p, o.eps_start) : OTS_OK;
  if (!st) st = o.warm_start ? refresh_if_stale(p) : reset_duals(p);
  if (st) { if (anneal) set_eps(p, target); return st; }
  ots_solve_report r{};
  int done = 0;
  if (anneal) {
    // stages eps_start * (eps / eps_start)^(k / n), k = 0..n-1, each to the stage tolerance,
    // then the problem's own epsilon below
    const int ns = o.eps_stages > 0 ? o.eps_stages : 3;
    const double stol = o.eps_stage_tol > 0.0 ? o.eps_stage_tol : 1e-4;
    for (int k = 0; k < ns && done < o.max_iters && !st; ++k) {
      st = set_eps(p, o.eps_start * std::pow(target / o.eps_start, (double)k / ns));
      if (!st) st = refresh_if_stale(p);
      while (!st && done < o.max_iters) {
        const int n = std::min(o.check_every, o.max_iters - done);
        st = run_passes(p, n, o.use_graph != 0);
        if (st) break;
        done += n;
        st = read_report(p, &r);
        if (st || (r.src_residual <= stol && r.cap_violation <= stol)) break;
      }
    }
    const ots_status back = set_eps(p, target);
    if (!st) st = back;
    if (!st) st = refresh_if_stale(p);
    if (st) {
      r.iterations = done;
      r.status = st;
      if (rep) *rep = r;
      return st;
    }
  }
  st = OTS_ERR_NOT_CONVERGED;
  while (done < o.max_iters) {
    int k = std::min(o.check_every, o.max_iters - done);
    ots_status e = run_passes(p, k, o.use_graph != 0);
    if (e) return e;
    done += k;
    e = read_report(p, &r);
    if (e) { st = e; break; }
    if (r.src_residual <= o.tol && r.cap_violation <= o.tol) { st = OTS_OK; break; }
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (o.timeout_ms > 0 && ms > o.timeout_ms) { st = fail(OTS_ERR_TIMEOUT, "timeout after %d passes", done); break; }
  }
  if (st == OTS_ERR_NOT_CONVERGED) fail(st, "not converged after %d passes (src %.3e, cap %.3e)", done, r.src_residual, r.cap_violation);
  r.iterations = done;
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  r.status = st;
  if (rep) *rep = r;
  return st;
}

namespace {

constexpr int kLinearChunk = 2000;   // passes per launch of the linear-domain kernel

void add_stats(ots_linear_stats *st, const LinReport &r, double ms) {
  if (!st) return;
  st->linear_passes += r.passes - r.log_passes;
  st->log_passes += r.log_passes;
  st->rescalings += r.rescalings;
  st->kernel_ms += ms;
}

// Linear-domain passes on n problems until each is converged (tol) or has run max_passes, in
// launches of kLinearChunk passes.  done[i]: passes run on problem i.
ots_status linear_phase(ots_problem *const *ps, int n, int max_passes, double tol, int init, double timeout_ms,
                        std::chrono::steady_clock::time_point t0, std::vector<int> &done, ots_linear_stats *stats) {
  done.assign(n, 0);
  int ran = 0;
  for (bool first = true; ran < max_passes; first = false) {
    const int chunk = std::min(kLinearChunk, max_passes - ran);
    double ms = 0.0;
    ots_status st = linear_run(ps, n, chunk, tol, first ? init : 0, &ms);
    if (st) return st;
    bool open = false;
    for (int i = 0; i < n; ++i) {
      const LinReport &r = linear_report(ps[i]);
      done[i] += r.passes;
      add_stats(stats, r, i == 0 ? ms : 0.0);
      if (r.status == OTS_OK && !r.converged && r.passes > 0) open = true;
    }
    ran += chunk;
    if (!open) break;
    const double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_ms > 0 && el > timeout_ms) break;
  }
  return OTS_OK;
}

// Log-domain passes from the duals the linear phase left, until the measures of a pass are
// <= tol: the result and its measures are those of the log-domain path.
ots_status confirm(ots_problem *p, const ots_solve_opts &o, int budget, ots_solve_report &r, int &passes) {
  passes = 0;
  ots_status st = refresh_if_stale(p);
  if (st) return st;
  int k = 1;
  while (true) {
    st = run_passes(p, k, o.use_graph != 0);
    if (st) return st;
    passes += k;
    st = read_report(p, &r);
    if (st) return st;
    if (r.src_residual <= o.tol && r.cap_violation <= o.tol) return OTS_OK;
    if (passes >= budget) return fail(OTS_ERR_NOT_CONVERGED, "not converged (src %.3e, cap %.3e)", r.src_residual, r.cap_violation);
    k = std::min(std::min(2 * k, o.check_every), budget - passes);   // 1, 2, 4, ... up to check_every
  }
}

ots_status linear_opts(const ots_solve_opts *opts, ots_solve_opts &o) {
  ots_default_solve_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_iters < 1 || o.check_every < 1) return fail(OTS_ERR_INVALID_ARG, "bad solve options");
  if (o.eps_start > 0.0) return fail(OTS_ERR_INVALID_ARG, "epsilon continuation is not part of the linear-domain path");
  return OTS_OK;
}

}  // namespace

extern "C" {

ots_status ots_linear_iterate(ots_problem *p, int32_t n, int32_t reset, ots_solve_report *rep, ots_linear_stats *stats) {
  g_last_error.clear();
  if (!p || n < 0) return fail(OTS_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard guard(p->dev);
  if (stats) *stats = ots_linear_stats{};
  auto t0 = std::chrono::steady_clock::now();
  ots_status st = linear_prepare(p);
  if (st) return st;
  if (n == 0) {                     // nothing to run: an empty report
    if (rep) *rep = ots_solve_report{};
    return OTS_OK;
  }
  std::vector<int> done;
  st = linear_phase(&p, 1, n, -1.0, reset ? 1 : 2, 0.0, t0, done, stats);
  if (st) return st;
  const LinReport &lr = linear_report(p);
  ots_solve_report r{};
  r.iterations = done[0];
  r.src_residual = lr.src;
  r.cap_violation = lr.cap;
  r.dual_objective = NAN;
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  r.status = lr.status;
  if (r.status) fail((ots_status)r.status, "linear-domain pass failed (status %d)", r.status);
  if (rep) *rep = r;
  return (ots_status)r.status;
}

ots_status ots_linear_solve_many(ots_problem *const *ps, int32_t n, const ots_solve_opts *opts, ots_solve_report *reps,
                                 ots_linear_stats *stats) {
  g_last_error.clear();
  if (!ps || n < 1) return fail(OTS_ERR_INVALID_ARG, "bad arguments");
  for (int i = 0; i < n; ++i) {
    if (!ps[i]) return fail(OTS_ERR_INVALID_ARG, "problem %d is NULL", i);
    if (ps[i]->dev != ps[0]->dev) return fail(OTS_ERR_INVALID_ARG, "problems on different devices");
    for (int j = 0; j < i; ++j)
      if (ps[j] == ps[i]) return fail(OTS_ERR_INVALID_ARG, "problem %d appears twice", i);
  }
  ots_solve_opts o;
  ots_status st = linear_opts(opts, o);
  if (st) return st;
  DeviceGuard guard(ps[0]->dev);
  if (stats) *stats = ots_linear_stats{};
  auto t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < n; ++i) {
    st = linear_prepare(ps[i]);
    if (st) return fail(st, "problem %d: %s", i, ots_last_error());
  }
  std::vector<int> done;
  st = linear_phase(ps, n, o.max_iters, o.tol, o.warm_start ? 2 : 1, o.timeout_ms, t0, done, stats);
  if (st) return st;
  ots_status worst = OTS_OK;
  for (int i = 0; i < n; ++i) {
    ots_solve_report r{};
    const LinReport &lr = linear_report(ps[i]);
    int cp = 0;
    ots_status si = (ots_status)lr.status;
    if (!si) {
      DeviceGuard g(ps[i]->dev);
      si = confirm(ps[i], o, std::max(1, o.max_iters - done[i]), r, cp);
    } else {
      r.src_residual = lr.src;
      r.cap_violation = lr.cap;
    }
    if (stats) stats->confirm_passes += cp;
    r.iterations = done[i] + cp;
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    r.status = si;
    if (reps) reps[i] = r;
    if (si && !worst) worst = si;
  }
  if (worst) fail(worst, "%s", n > 1 ? "not every problem was solved (see the per-problem reports)" : ots_last_error());
  return worst;
}

ots_status ots_linear_solve(ots_problem *p, const ots_solve_opts *opts, ots_solve_report *rep, ots_linear_stats *stats) {
  return ots_linear_solve_many(&p, 1, opts, rep, stats);
}

}  // extern "C"

// Flows pass: recompute the forward messages at the current duals, writing the aggregate
// flows P_t for t = 2..T-1 (Corollary 7).
static ots_status flows_pass(ots_problem *p) {
  ots_status st = refresh_if_stale(p);
  if (st) return st;
  p->kernels_launched += 1 + (p->T - 2) + 2 + p->b_recompute;
  OTS_CUDA(launch_boundary_rebuild(p, true));
  for (int t = 2; t <= p->T - 1; ++t) {
    OTS_CUDA(enqueue_segment(p, t));
    OTS_CUDA(forward_step(p, t, 1));
    OTS_CUDA(after_forward_step(p, t, true));
  }
  OTS_CUDA(launch_boundary_flows_all(p));
  return OTS_OK;
}

ots_status ots_get_flows(ots_problem *p, int32_t t_begin, int32_t t_end, double *out) {
  g_last_error.clear();
  if (!p || !out) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  if (t_begin < 1 || t_end > p->T + 1 || t_begin >= t_end) return fail(OTS_ERR_INVALID_ARG, "bad t range");
  DeviceGuard guard(p->dev);
  ots_status st = flows_pass(p);
  if (st) return st;
  const size_t S = p->S;
  std::vector<double> sf(p->src.n), zf(p->snk.n);
  for (int t = t_begin; t < t_end; ++t) {
    double *row = out + (size_t)(t - t_begin) * S;
    if (t >= 2 && t <= p->T - 1) {
      OTS_CUDA(cudaMemcpyAsync(row, p->d_flow + (size_t)t * S, sizeof(double) * S, cudaMemcpyDeviceToHost, p->stream));
      p->d2h_bytes += (long long)(sizeof(double) * S);
    }
  }
  if (p->src.n) OTS_CUDA(cudaMemcpyAsync(sf.data(), p->src.d_flow, sizeof(double) * p->src.n, cudaMemcpyDeviceToHost, p->stream));
  if (p->snk.n) OTS_CUDA(cudaMemcpyAsync(zf.data(), p->snk.d_flow, sizeof(double) * p->snk.n, cudaMemcpyDeviceToHost, p->stream));
  p->d2h_bytes += (long long)(sizeof(double) * (p->src.n + p->snk.n));
  OTS_CUDA(cudaStreamSynchronize(p->stream));
  // rows t = 1 and T hold only boundary flows; each source (sink) triple adds its flow at its
  // commodity's entry (exit) time, where the interior rows leave that commodity out
  for (int t = t_begin; t < t_end; ++t)
    if (t == 1 || t == p->T) std::fill(out + (size_t)(t - t_begin) * S, out + (size_t)(t - t_begin + 1) * S, 0.0);
  for (int side = 0; side < 2; ++side) {
    const Boundary &b = side == 0 ? p->src : p->snk;
    const std::vector<double> &f = side == 0 ? sf : zf;
    for (int q = 0; q < b.n; ++q) {
      const int t = side == 0 ? p->ta[b.tri_l[q]] : p->tb[b.tri_l[q]];
      if (t >= t_begin && t < t_end) out[(size_t)(t - t_begin) * S + b.tri_state[q]] += f[q];
    }
  }
  return OTS_OK;
}

ots_status ots_get_commodity_flows(ots_problem *p, int32_t t_begin, int32_t t_end, int32_t l_begin, int32_t l_end,
                                   double *out) {
  g_last_error.clear();
  if (!p || !out) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  if (t_begin < 1 || t_end > p->T + 1 || t_begin >= t_end) return fail(OTS_ERR_INVALID_ARG, "bad t range");
  if (l_begin < 0 || l_end > p->L || l_begin >= l_end) return fail(OTS_ERR_INVALID_ARG, "bad commodity range");
  DeviceGuard guard(p->dev);
  ots_status st = refresh_if_stale(p);
  if (st) return st;
  const size_t S = p->S, nl = l_end - l_begin, blk = S * nl;
  double *d_tmp = (double *)dev_alloc(p, sizeof(double) * blk);
  if (!d_tmp) return fail(OTS_ERR_OOM, "device allocation failed");
  std::vector<double> sf(p->src.n), zf(p->snk.n);
  ots_status rc = OTS_OK;
  auto check = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == OTS_OK) rc = fail(OTS_ERR_CUDA, "%s", cudaGetErrorString(e));
  };
  check(launch_boundary_rebuild(p, true));
  for (int t = 2; t <= p->T - 1 && rc == OTS_OK; ++t) {
    check(enqueue_segment(p, t));
    if (t >= t_begin && t < t_end) {
      // A_{t-1} is current here (written by the previous forward step of this pass)
      check(launch_commodity_flows(p->S, p->Lp, p->qs, l_begin, l_end, p->d_tail, p->d_head, p->a_hi(t - 1), p->a_lo(t - 1),
                                   p->b_hi(t + 1), p->b_lo(t + 1), p->d_kl_hi + (p->tv ? t * S : 0),
                                   p->d_kl_lo + (p->tv ? t * S : 0), p->d_klc_hi, p->d_klc_lo,
                                   p->d_uc ? p->d_uc + (size_t)t * S * p->Lp : nullptr,
                                   p->d_logu + (size_t)t * S, d_tmp, p->stream));
      check(cudaMemcpyAsync(out + (size_t)(t - t_begin) * blk, d_tmp, sizeof(double) * blk, cudaMemcpyDeviceToHost,
                            p->stream));
      check(cudaStreamSynchronize(p->stream));
    }
    check(forward_step(p, t, 1));
    check(after_forward_step(p, t, true));
  }
  check(launch_boundary_flows_all(p));
  if (p->src.n) check(cudaMemcpyAsync(sf.data(), p->src.d_flow, sizeof(double) * p->src.n, cudaMemcpyDeviceToHost, p->stream));
  if (p->snk.n) check(cudaMemcpyAsync(zf.data(), p->snk.d_flow, sizeof(double) * p->snk.n, cudaMemcpyDeviceToHost, p->stream));
  check(cudaStreamSynchronize(p->stream));
  dev_free(p, d_tmp);
  if (rc) return rc;
  for (int t : {1, p->T})
    if (t >= t_begin && t < t_end) std::fill(out + (size_t)(t - t_begin) * blk, out + (size_t)(t - t_begin + 1) * blk, 0.0);
  for (int side = 0; side < 2; ++side) {
    const Boundary &b = side == 0 ? p->src : p->snk;
    const std::vector<double> &f = side == 0 ? sf : zf;
    for (int q = 0; q < b.n; ++q) {
      const int l = b.tri_l[q];
      const int t = side == 0 ? p->ta[l] : p->tb[l];
      if (l >= l_begin && l < l_end && t >= t_begin && t < t_end)
        out[(size_t)(t - t_begin) * blk + (size_t)(l - l_begin) * S + b.tri_state[q]] += f[q];
    }
  }
  return OTS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Allocation-free per-commodity flows.
//
// ots_get_commodity_flows obtains a temporary device buffer on every call.  Some callers
// cannot allow that: a real-time loop that must not stall on the device allocator (cudaMalloc
// can synchronise the whole device) between solver passes, or an application that gives this
// library a fixed device-memory budget when the problem is created.  The variant
// below computes the same flows with its scratch in one fixed array that lives in this
// library's device image: kNoAllocMaxDoubles doubles (8 MiB) on every GPU that loads the
// library, held until the process exits.
// ---------------------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocMaxDoubles = size_t(1) << 20;     // flow slice: n_states x commodities
constexpr size_t kNoAllocMaxTriples = 65536;               // boundary triples per side

struct NoAllocScratch {
  double flows[kNoAllocMaxDoubles];                        // [commodity - l0][state]
  int tri_state[kNoAllocMaxTriples];                       // states of one side's triples
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Scatter the per-triple boundary flows of commodities [l0, l1) into a zeroed
// [commodity - l0][state] slice (triples are unique per (commodity, state)).
__global__ void k_noalloc_scatter(int n, int l0, int l1, int S, const int *tri_l, const int *tri_state,
                                  const double *flow, double *slice) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int l = tri_l[q];
  if (l >= l0 && l < l1) slice[(size_t)(l - l0) * S + tri_state[q]] = flow[q];
}

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
NoAllocScratch *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
ots_status noalloc_scratch(int dev, NoAllocScratch **out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(OTS_ERR_INVALID_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(OTS_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = (NoAllocScratch *)ptr;
  }
  *out = g_noalloc_ptr[dev];
  return OTS_OK;
}

}  // namespace

extern "C" {

ots_status ots_get_commodity_flows_noalloc(ots_problem *p, int32_t t_begin, int32_t t_end, int32_t l_begin,
                                           int32_t l_end, double *out) {
  g_last_error.clear();
  if (!p || !out) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  if (t_begin < 1 || t_end > p->T + 1 || t_begin >= t_end) return fail(OTS_ERR_INVALID_ARG, "bad t range");
  if (l_begin < 0 || l_end > p->L || l_begin >= l_end) return fail(OTS_ERR_INVALID_ARG, "bad commodity range");
  const size_t S = p->S, nl = l_end - l_begin, blk = S * nl;
  if (blk > kNoAllocMaxDoubles)
    return fail(OTS_ERR_INVALID_ARG,
                "n_states x commodities = %zu exceeds the static buffer of %zu doubles; request fewer commodities",
                blk, kNoAllocMaxDoubles);
  if ((size_t)p->src.n > kNoAllocMaxTriples || (size_t)p->snk.n > kNoAllocMaxTriples)
    return fail(OTS_ERR_INVALID_ARG, "more than %zu source or sink triples", kNoAllocMaxTriples);
  if (p->win) return fail(OTS_ERR_INVALID_ARG, "commodity windows: use ots_get_commodity_flows");
  DeviceGuard guard(p->dev);
  NoAllocScratch *scr = nullptr;
  ots_status st = noalloc_scratch(p->dev, &scr);
  if (st) return st;
  st = refresh_if_stale(p);
  if (st) return st;
  double *slice = scr->flows;
  // forward pass at the current duals; interior rows come from the message panels
  OTS_CUDA(launch_boundary_rebuild(p, true));
  for (int t = 2; t <= p->T - 1; ++t) {
    OTS_CUDA(enqueue_segment(p, t));
    if (t >= t_begin && t < t_end) {
      OTS_CUDA(launch_commodity_flows(p->S, p->Lp, p->qs, l_begin, l_end, p->d_tail, p->d_head, p->a_hi(t - 1),
                                      p->a_lo(t - 1), p->b_hi(t + 1), p->b_lo(t + 1),
                                      p->d_kl_hi + (p->tv ? t * S : 0), p->d_kl_lo + (p->tv ? t * S : 0),
                                      p->d_klc_hi, p->d_klc_lo, p->d_uc ? p->d_uc + (size_t)t * S * p->Lp : nullptr,
                                   p->d_logu + (size_t)t * S, slice, p->stream));
      OTS_CUDA(cudaMemcpyAsync(out + (size_t)(t - t_begin) * blk, slice, sizeof(double) * blk,
                               cudaMemcpyDeviceToHost, p->stream));
      OTS_CUDA(cudaStreamSynchronize(p->stream));      // the slice is reused for the next t
      p->kernels_launched += 1;
      p->d2h_bytes += (long long)(sizeof(double) * blk);
    }
    OTS_CUDA(forward_step(p, t, 1));
    OTS_CUDA(after_forward_step(p, t, true));
  }
  OTS_CUDA(launch_boundary_flows_all(p));
  p->kernels_launched += 1 + (p->T - 2) + 2 + p->b_recompute;
  // boundary rows t = 1 (sources) and t = T (sinks): scatter the per-triple flows into the
  // zeroed slice; the states of the triples are copied from the problem's host-side list
  for (int t : {1, p->T}) {
    if (t < t_begin || t >= t_end) continue;
    const Boundary &b = t == 1 ? p->src : p->snk;
    OTS_CUDA(cudaMemsetAsync(slice, 0, sizeof(double) * blk, p->stream));
    if (b.n > 0) {
      OTS_CUDA(cudaMemcpyAsync(scr->tri_state, b.tri_state.data(), sizeof(int) * b.n, cudaMemcpyHostToDevice,
                               p->stream));
      k_noalloc_scatter<<<(b.n + 255) / 256, 256, 0, p->stream>>>(b.n, l_begin, l_end, p->S, b.d_tri_l,
                                                                  scr->tri_state, b.d_flow, slice);
      OTS_CUDA(cudaGetLastError());
      p->kernels_launched += 1;
      p->h2d_bytes += (long long)(sizeof(int) * b.n);
    }
    OTS_CUDA(cudaMemcpyAsync(out + (size_t)(t - t_begin) * blk, slice, sizeof(double) * blk, cudaMemcpyDeviceToHost,
                             p->stream));
    OTS_CUDA(cudaStreamSynchronize(p->stream));       // the slice is reused next
    p->d2h_bytes += (long long)(sizeof(double) * blk);
  }
  return OTS_OK;
}

ots_status ots_get_duals(ots_problem *p, double *log_u, double *log_U01, double *log_U0T) {
  g_last_error.clear();
  if (!p) return fail(OTS_ERR_INVALID_ARG, "problem is NULL");
  DeviceGuard guard(p->dev);
  const size_t S = p->S;
  std::vector<float2> lu;
  std::vector<double> su(p->src.n), zu(p->snk.n);
  if (log_u) {
    lu.resize((size_t)(p->T - 2) * S);
    OTS_CUDA(cudaMemcpyAsync(lu.data(), p->d_logu + 2 * S, sizeof(float2) * lu.size(), cudaMemcpyDeviceToHost, p->stream));
  }
  if (p->src.n) OTS_CUDA(cudaMemcpyAsync(su.data(), p->src.d_tri_logU, sizeof(double) * p->src.n, cudaMemcpyDeviceToHost, p->stream));
  if (p->snk.n) OTS_CUDA(cudaMemcpyAsync(zu.data(), p->snk.d_tri_logU, sizeof(double) * p->snk.n, cudaMemcpyDeviceToHost, p->stream));
  OTS_CUDA(cudaStreamSynchronize(p->stream));
  if (log_u)
    for (size_t k = 0; k < lu.size(); ++k)
      log_u[k] = lu[k].x < -1e29f ? -INFINITY : ((double)lu[k].x + (double)lu[k].y) * kLn2;
  if (log_U01)
    for (size_t q = 0; q < p->src.input_to_tri.size(); ++q) log_U01[q] = su[p->src.input_to_tri[q]] * kLn2;
  if (log_U0T)
    for (size_t q = 0; q < p->snk.input_to_tri.size(); ++q) log_U0T[q] = zu[p->snk.input_to_tri[q]] * kLn2;
  return OTS_OK;
}

ots_status ots_set_duals(ots_problem *p, const double *log_u, const double *log_U01, const double *log_U0T) {
  g_last_error.clear();
  if (!p || !log_u || !log_U01 || !log_U0T) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(p->dev);
  const size_t S = p->S;
  std::vector<float2> lu((size_t)(p->T - 2) * S);
  std::vector<double> su(p->src.n, 0.0), zu(p->snk.n, 0.0);
  for (size_t k = 0; k < lu.size(); ++k) {
    if (std::isnan(log_u[k]) || log_u[k] > 0.0) return fail(OTS_ERR_INVALID_ARG, "log_u must be <= 0");
    if (std::isinf(log_u[k])) {
      lu[k] = make_float2(kNeg, 0.f);
    } else {
      const double x = log_u[k] * kInvLn2;
      const float h = (float)x;
      lu[k] = make_float2(h, (float)(x - (double)h));
    }
  }
  for (size_t q = 0; q < p->src.input_to_tri.size(); ++q) {
    if (!std::isfinite(log_U01[q])) return fail(OTS_ERR_INVALID_ARG, "log_U01 must be finite");
    su[p->src.input_to_tri[q]] = log_U01[q] * kInvLn2;
  }
  for (size_t q = 0; q < p->snk.input_to_tri.size(); ++q) {
    if (!std::isfinite(log_U0T[q])) return fail(OTS_ERR_INVALID_ARG, "log_U0T must be finite");
    zu[p->snk.input_to_tri[q]] = log_U0T[q] * kInvLn2;
  }
  OTS_CUDA(cudaMemcpyAsync(p->d_logu + 2 * S, lu.data(), sizeof(float2) * lu.size(), cudaMemcpyHostToDevice, p->stream));
  if (p->src.n) OTS_CUDA(cudaMemcpyAsync(p->src.d_tri_logU, su.data(), sizeof(double) * p->src.n, cudaMemcpyHostToDevice, p->stream));
  if (p->snk.n) OTS_CUDA(cudaMemcpyAsync(p->snk.d_tri_logU, zu.data(), sizeof(double) * p->snk.n, cudaMemcpyHostToDevice, p->stream));
  OTS_CUDA(cudaStreamSynchronize(p->stream));
  p->stale = true;
  return OTS_OK;
}

ots_status ots_set_wait_limit(ots_problem *p, int32_t tries, int32_t withhold_stage) {
  g_last_error.clear();
  if (!p || tries < 0) return fail(OTS_ERR_INVALID_ARG, "NULL problem or negative tries");
  p->wait_tries = tries == 0 ? (1u << 20) : (unsigned int)tries;
  p->withhold_stage = withhold_stage != 0 ? 1 : 0;
  if (p->pass_exec) {                               // the pass graph holds the old arguments
    cudaGraphExecDestroy(p->pass_exec);
    p->pass_exec = nullptr;
  }
  return OTS_OK;
}

// Stream of the problem (for callers that time or order work around it).
void *ots_problem_stream(const ots_problem *p) { return p ? (void *)p->stream : nullptr; }

}  // extern "C"

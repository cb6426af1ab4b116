// ots_internal.h -- host-side internals shared by the translation units of the library:
// the problem object behind the opaque ots_problem handle, error reporting, and the kernel
// launchers.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "ots.h"
#include "ots_device.cuh"

namespace ots {
cudaError_t launch_step(bool fwd, bool pc, int G, int C, const StepArgs &a, cudaStream_t s);
cudaError_t prepare_step_kernels(int G, int C, bool pc, int V, int *grid_fwd, int *grid_bwd);
int step_grid(int V, int G);
cudaError_t launch_boundary(const BndArgs &b, cudaStream_t s);
cudaError_t launch_store_rows(const StoreRowArgs &a, cudaStream_t s);
cudaError_t launch_store_triples(const StoreTriArgs &a, cudaStream_t s);
cudaError_t launch_store_update(const StepArgs &a, const StoreUpdArgs &u, int max_grid, cudaStream_t s);
int boundary_grid(int n_seg);
cudaError_t launch_pass_begin(DevStats *st, cudaStream_t s);
cudaError_t launch_pass_end(const DevStats *st, PassReport *rep, double mass, double eps, const double *slots,
                            int stride, int nblk, int T, double *tot, cudaStream_t s);
cudaError_t launch_weights(int S, int T, QScale qs, const float *kl_hi, const float *kl_lo, int kl_stride, float2 *logu,
                           float *w_hi, float *w_lo, int reset, const int *st_inpos, const int *st_outpos,
                           float2 *logu_in, float *wout_hi, float *wout_lo, cudaStream_t s);
cudaError_t launch_fill_panel(size_t n, float *hi, lo_t *lo, cudaStream_t s);
cudaError_t launch_scale_duals(float2 *lu, size_t n_lu, float2 *lu_in, size_t n_in, double *ua, int na, double *ub,
                               int nb, double r, cudaStream_t s);
cudaError_t launch_commodity_flows(int S, int Lp, QScale qs, int l0, int l1, const int *tail, const int *head,
                                   const float *a_hi, const lo_t *a_lo, const float *b_hi, const lo_t *b_lo,
                                   const float *kl_hi, const float *kl_lo, const float *klc_hi, const lo_t *klc_lo,
                                   const float *uc_t, const float2 *logu_t, double *out, cudaStream_t s);
cudaError_t launch_boundary_flows(int n, int Lp, QScale qs, const int *tri_l, const int *tri_node_other,
                                  const double *tri_logU, const float *msg_hi, const lo_t *msg_lo, double *out,
                                  cudaStream_t s);
}  // namespace ots

namespace ots {
// Result of the last launch of the linear-domain kernel on a problem (ots_linear.cu).
struct LinReport {
  int passes;       // passes of the launch
  int log_passes;   // of which redone in log arithmetic
  int rescalings;   // scale sweeps of the launch
  int status;       // ots_status
  int converged;    // measures <= tol after the last pass
  int pad;
  double src, cap;  // measures of the last pass (relative)
};
}  // namespace ots

namespace ots_host {

struct LinearData;   // device arrays of the linear-domain path (ots_linear.cu)

// Records a formatted message for ots_last_error (per thread) and returns s.
ots_status fail(ots_status s, const char *fmt, ...);
void clear_error();

#define OTS_CUDA(expr)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return ::ots_host::fail(e_ == cudaErrorMemoryAllocation ? OTS_ERR_OOM : OTS_ERR_CUDA,     \
                              "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kInvLn2 = 1.44269504088896340736;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline void split_ff(double x, float &hi, float &lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// One side of the boundary (sources or sinks): unique (commodity, state) triples grouped in
// segments of equal (node, commodity).
struct Boundary {
  int n = 0;                      // unique triples
  int n_seg = 0;
  std::vector<int> seg_ptr, seg_node, seg_l;
  std::vector<int> tri_l, tri_state, tri_other;
  std::vector<double> tri_R;
  std::vector<int> input_to_tri;  // descriptor triple -> unique triple
  // groups of segments with the same time (entry time of the commodity for sources, exit time
  // for sinks), in increasing time: group g holds segments [grp_seg[g], grp_seg[g+1])
  std::vector<int> grp_t, grp_seg;
  // device
  int *d_seg_ptr = nullptr, *d_seg_node = nullptr, *d_seg_l = nullptr, *d_tri_other = nullptr, *d_tri_l = nullptr;
  double *d_tri_R = nullptr, *d_tri_logR = nullptr, *d_tri_logU = nullptr, *d_flow = nullptr;
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Options of the internal constructor.  A batch member is an instance that lives in a batch
// (ots_batch / ots_server): it uses the batch's stream and device pool, is initialised by
// the batched kernel rather than here, and has the thread mapping the batch chose.
struct CreateOpts {
  bool member = false;
  int G = 0, C = 0;          // forced mapping (member only): G threads per node, C chunks of 4
};

// Host arrays of a problem between its host build and its upload.
struct HostArrays {
  std::vector<int> in_ptr, out_ptr, in_state, in_nbr, out_state, out_nbr, st_inpos, st_outpos, in_outpos;
  std::vector<float> kl_hi, kl_lo, logd_hi, logd_lo, in_kl_hi, in_kl_lo, in_logd_hi, in_logd_lo, klc_hi;
  std::vector<float2> cap, in_cap;          // capacities as float-float pairs (x = inf: none)
  std::vector<float2> dc;                   // [S][Lp] log2 of the commodity capacities
  std::vector<ots::lo_t> klc_lo;
};

// create_problem_impl = build_problem_host (no CUDA call; may run on any thread) followed by
// build_problem_device (allocation, uploads and initial duals on p->stream).
ots_status build_problem_host(const ots_problem_desc *d, const CreateOpts &co, ots_problem **out);
ots_status build_problem_device(ots_problem *p);
ots_status create_problem_impl(const ots_problem_desc *d, const CreateOpts &co, ots_problem **out);

// Device memory through the problem's allocator (ots_api.cu).
void *problem_alloc(ots_problem *p, size_t bytes);
void problem_free(ots_problem *p, void *ptr);

// Linear-domain path for L = 1 (ots_linear.cu).  linear_prepare builds the problem's arrays once
// (OTS_ERR_INVALID_ARG where the path does not apply); linear_run runs up to max_passes passes on
// each of the n problems in one launch (one thread block each; all on one device, launched on
// ps[0]'s stream), stopping each at tol (tol < 0: never).  init: 1 = from the initial duals,
// 2 = from the problem's duals, 0 = continue the previous launch.  The duals are written back
// to each problem (which is then marked stale); per-problem results in linear_report.
ots_status linear_prepare(ots_problem *p);
ots_status linear_run(ots_problem *const *ps, int n, int max_passes, double tol, int init, double *kernel_ms);
const ots::LinReport &linear_report(const ots_problem *p);
void linear_release(ots_problem *p);

// Batch internals used by the server (ots_batch.cu).
struct Pool;
Pool *batch_pool(ots_batch *b);
void *pool_alloc_cb(size_t bytes, void *ctx);   // ots_alloc_fn / ots_free_fn over a Pool
void pool_free_cb(void *p, void *ctx);
ots_status batch_prepare(ots_batch *b, const ots_problem_desc *desc, cudaStream_t upload_stream, ots_problem **out);
ots_status batch_admit(ots_batch *b, ots_problem *p, const ots_solve_opts *opts, int32_t *id);
int batch_free_slots(const ots_batch *b);

}  // namespace ots_host

struct ots_problem {
  using QScale = ots::QScale;
  using lo_t = ots::lo_t;
  using DevStats = ots::DevStats;
  using PassReport = ots::PassReport;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ots_alloc_fn alloc = nullptr;
  ots_free_fn free_fn = nullptr;
  void *actx = nullptr;

  int V = 0, E = 0, S = 0, L = 0, T = 0, G = 1, C = 1, Lp = 4;
  double eps = 1.0, mass = 0.0;
  QScale qs{};                                 // quantum of the message hi parts
  int pgrid_fwd = 0, pgrid_bwd = 0;            // grids of the pipelined persistent kernels (0 = not used)
  int max_grid = 1;                            // blocks the per-block partial sums hold
  unsigned int wait_tries = 1u << 20;          // tries of each bounded device wait (ots_set_wait_limit)
  int withhold_stage = 0;                      // test switch of ots_set_wait_limit
  bool pc = false;
  bool member = false;                         // lives in a batch (see CreateOpts)
  bool tv = false;                             // time-varying costs: K_L rows per interval t
  bool cv = false;                             // per-interval capacities: d rows per interval t
  bool win = false;                            // commodities with their own entry / exit times
  bool cc = false;                             // commodity-dependent capacities D^(0,t)
  float2 *d_dc = nullptr;                      // [S][Lp] log2 D, float-float
  float *d_uc = nullptr;                       // [T+1][S][Lp] log2 U^(0,t)
  std::vector<int> ta, tb;                     // [L] entry and exit time of each commodity
  std::vector<double> cost_nat;                // state costs in natural units ([S], or [T+1][S] rows when tv)
  std::vector<double> cap_nat;                 // capacities ([S], or [T+1][S] rows when cv; inf: none)
  ots_host::LinearData *lin = nullptr;         // linear-domain path (L = 1), built on first use
  std::vector<int> in_state_h;                 // in-CSR order of the states (host copy)
  std::unique_ptr<ots_host::HostArrays> host;  // between the host build and the upload

  std::vector<int> tail, head;                 // -1: none (explicit state graphs)
  ots_host::Boundary src, snk;
  // Explicit state graph (Section 3.3): storage state k owns row V + k of every panel, and row
  // null_row = V + nstore stays log 0 (the row a state without a tail / head gathers).
  bool xgraph = false;
  int nstore = 0, null_row = -1, rows = 0;     // rows per panel: V, or V + nstore + 1
  std::vector<int> store_state, store_tail, store_head, frow, brow;
  std::vector<int> sst_k, sst_l, sst_q, zst_k, zst_l, zst_q;   // storage triples of sources / sinks
  int *d_store_state = nullptr, *d_store_tail = nullptr, *d_store_head = nullptr;
  int *d_sst = nullptr, *d_zst = nullptr;      // [3][n] (k, l, triple) of the storage triples
  unsigned char *d_fixed_w = nullptr;          // [S] 1 = storage state

  void *arena = nullptr;
  size_t arena_bytes = 0;

  int *d_in_ptr = nullptr, *d_in_state = nullptr, *d_in_nbr = nullptr;
  int *d_out_ptr = nullptr, *d_out_state = nullptr, *d_out_nbr = nullptr;
  int *d_tail = nullptr, *d_head = nullptr;
  float *d_kl_hi = nullptr, *d_kl_lo = nullptr, *d_logd_hi = nullptr, *d_logd_lo = nullptr;
  float2 *d_cap = nullptr;                     // [S] float-float
  float *d_klc_hi = nullptr;
  lo_t *d_klc_lo = nullptr;
  float *d_w_hi = nullptr, *d_w_lo = nullptr;  // [T+1][S]
  float2 *d_logu = nullptr;                    // [T+1][S] log2 u_t, float-float
  // CSR-ordered copies used by the pipelined kernels
  int *d_st_inpos = nullptr, *d_st_outpos = nullptr, *d_in_outpos = nullptr;
  float *d_in_kl_hi = nullptr, *d_in_kl_lo = nullptr, *d_in_logd_hi = nullptr, *d_in_logd_lo = nullptr;
  float2 *d_in_cap = nullptr;
  float2 *d_logu_in = nullptr;                 // [T+1][S] by in-CSR position
  float *d_cref_in = nullptr;                  // [T+1][S] column references by in-CSR position
  float *d_wout_hi = nullptr, *d_wout_lo = nullptr;  // [T+1][S] by out-CSR position
  double *d_flow = nullptr;                    // [T+1][S]
  float *d_a_hi[3] = {nullptr, nullptr, nullptr};
  lo_t *d_a_lo[3] = {nullptr, nullptr, nullptr};
  float *d_b_hi = nullptr;                     // [nbslots][V][Lp]
  lo_t *d_b_lo = nullptr;
  DevStats *d_stats = nullptr;
  PassReport *d_report = nullptr;
  double *d_partials = nullptr;
  double *d_slots = nullptr;                   // [T+1][2 max_grid] per-block sums of each forward step
  double *d_step_tot = nullptr;                // [T+1][2] their totals per step
  unsigned int *d_counter = nullptr;
  PassReport *h_report = nullptr;              // pinned

  cudaGraphExec_t pass_exec = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // phase marks of a pass
  bool stale = true;                           // backward messages not consistent with duals
  long long passes_total = 0;
  long long kernels_launched = 0;
  long long h2d_bytes = 0, d2h_bytes = 0;

  size_t panel() const { return (size_t)rows * Lp; }
  float *a_hi(int t) { return t == 1 ? d_a_hi[0] : d_a_hi[1 + (t & 1)]; }
  lo_t *a_lo(int t) { return t == 1 ? d_a_lo[0] : d_a_lo[1 + (t & 1)]; }
  // backward panels: B_t lives in slot bslot[t]; with bk > 1 only t = 2, T and every bk-th t
  // below T keep their own slot, the others share k - 1 recompute slots
  int bk = 1;
  int nbslots = 0;
  int b_recompute = 0;                         // backward steps a forward sweep adds
  std::vector<int> bslot;
  bool b_stored(int t) const { return bk <= 1 || t == 2 || t == T || (T - t) % bk == 0; }
  float *b_hi(int t) { return d_b_hi + (size_t)bslot[t] * panel(); }
  lo_t *b_lo(int t) { return d_b_lo + (size_t)bslot[t] * panel(); }
};

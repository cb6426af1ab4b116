/*
 * ots.h -- C ABI of the GB300 solver for entropy-regularised dynamic multi-commodity
 * minimum-cost flow by graph-structured multi-marginal optimal transport
 * (Haasler, Ringh, Chen, Karlsson, arXiv 2106.14485).
 *
 * The library solves problem eq. multicommodity_reg (Section 4.3): minimise
 *     <C, M> + eps D(M)  over M >= 0 (L x n^T),
 *     P_{0,1}(M) = R01,  P_{0,T}(M) = R0T,  P_t(M) <= d  (t = 2..T-1),
 * with the Sinkhorn iterations of Algorithm 2, all on one CUDA device.
 *
 * State model.  A state is a directed edge of the road network (Section 3.1: marginals
 * live on edges, n = |E|).  With add_wait_loops = 1 the library adds one self-loop state
 * per node (storage in the vertices, Section 3.3), so
 *     state e in [0, n_edges)          is edge e (edge_src[e] -> edge_dst[e]),
 *     state n_edges + v                 is the wait loop of node v.
 * The transition kernel is the line graph: state i may be followed by state j iff the
 * head of i is the tail of j (Section 3.1, C_ij = 0 or infinity).  Costs are per state
 * and per time interval (the matrix C_L of Section 3.2, eq. cost_multicommodity) and
 * apply at t = 2..T-1; capacities d are per state and bind at t = 2..T-1.
 *
 * Memory and ownership.  Every pointer in ots_problem_desc is a HOST pointer; the library
 * copies what it needs during ots_create_problem and keeps no reference to the caller's
 * arrays.  Device memory is obtained once per problem, either from the optional allocator
 * callbacks in the descriptor or from cudaMalloc.  Output buffers of the getters are host
 * buffers allocated by the caller.
 *
 * Errors.  Every entry point returns an ots_status (no exceptions cross the ABI, nothing
 * aborts).  ots_last_error() gives a human-readable message for the calling thread.
 *
 * Threads.  One problem handle must not be used by two threads at once; distinct handles
 * are independent.  All device work of a handle runs on its stream (desc.stream, or a
 * stream the library creates); the getters synchronise that stream.
 */
#ifndef OTS_H
#define OTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ots_status {
  OTS_OK = 0,
  OTS_ERR_INVALID_ARG = 1,   /* bad size, index out of range, eps <= 0, T < 3, negative
                                mass or capacity, per-commodity source mass != sink mass
                                (relative 1e-9), unsupported option */
  OTS_ERR_INFEASIBLE = 2,    /* a sink state no source of its commodity reaches in T-1
                                transitions, or a source that reaches no sink */
  OTS_ERR_NOT_CONVERGED = 3, /* max_iters passes without reaching tol (e.g. capacities
                                that admit no feasible flow: the duals then diverge) */
  OTS_ERR_TIMEOUT = 4,       /* timeout_ms elapsed before convergence */
  OTS_ERR_OOM = 5,           /* device or host allocation failed */
  OTS_ERR_CUDA = 6,          /* a CUDA runtime call failed (see ots_last_error) */
  OTS_ERR_NUMERIC = 7,       /* a NaN appeared in the convergence measures */
  OTS_PENDING = 8,           /* batch / server: the instance has not finished yet */
  OTS_ERR_DEVICE_WAIT = 9    /* a bounded wait inside a pipelined step kernel gave up (its
                                data did not arrive in time); the pass's results are invalid,
                                the problem stays usable (reset the duals or load them again) */
} ots_status;

typedef struct ots_problem ots_problem;

/* Optional device allocator: returns a device pointer (256-byte aligned) or NULL. */
typedef void *(*ots_alloc_fn)(size_t bytes, void *ctx);
typedef void (*ots_free_fn)(void *ptr, void *ctx);

/* Problem description (Section 3.2, eq. multicommodity; Section 3.3 wait loops). */
typedef struct ots_problem_desc {
  int32_t n_nodes;               /* |V| >= 1 */
  int32_t n_edges;               /* |E| >= 0, directed */
  const int32_t *edge_src;       /* [n_edges] tail node of each edge */
  const int32_t *edge_dst;       /* [n_edges] head node of each edge */
  const double *edge_cost;       /* [n_edges] cost per interval on the edge (row of C_L,
                                    identical for every commodity); NULL = 0 */
  const double *edge_capacity;   /* [n_edges] d on edges, INFINITY = none; NULL = none */
  int32_t add_wait_loops;        /* 1: add a wait-loop state per node; 0: states = edges */
  const double *wait_cost;       /* [n_nodes] cost per interval on the wait loop; NULL = 0 */
  const double *wait_capacity;   /* [n_nodes] d on wait loops, INFINITY = none; NULL = none */
  const double *commodity_cost;  /* optional [L x n_states] row-major C_L with per-commodity
                                    rows; overrides edge_cost / wait_cost when non-NULL */
  int32_t T;                     /* number of marginals / time intervals, T >= 3 */
  int32_t L;                     /* number of commodities, L >= 1 */
  double eps;                    /* entropy regularisation eps > 0 (eq. omt_multi_graph_reg) */
  int32_t n_sources;             /* non-zeros of R01 as (commodity, state, mass) triples;   */
  const int32_t *src_commodity;  /* repeated (commodity, state) pairs add up              */
  const int32_t *src_state;
  const double *src_mass;        /* > 0 */
  int32_t n_sinks;               /* non-zeros of R0T, same layout */
  const int32_t *snk_commodity;
  const int32_t *snk_state;
  const double *snk_mass;
  int32_t device;                /* CUDA device ordinal */
  void *stream;                  /* cudaStream_t for all work of this problem; NULL = own */
  ots_alloc_fn alloc;            /* optional device allocator (both or neither) */
  ots_free_fn free_fn;
  void *alloc_ctx;
  const double *state_cost_t;    /* optional [(T-2) x n_states] row-major: a time-varying
                                    network (Section 3.3, C replaced by time-dependent C_t):
                                    the cost of every state in interval t = 2..T-1, the same
                                    for all commodities; +INFINITY closes a state during that
                                    interval.  When given, edge_cost and wait_cost are not used;
                                    not combinable with commodity_cost. */
  const double *state_capacity_t; /* optional [(T-2) x n_states] row-major: per-interval
                                    capacities d_t (the problem statements of Section 3 and
                                    eq. multicommodity_reg bound P_t by d_t for t = 2..T-1):
                                    row t-2 holds d_t, >= 0, +INFINITY for none, 0 closes the
                                    state in that interval.  When given, edge_capacity and
                                    wait_capacity are not used.  NaN or negative entries give
                                    OTS_ERR_INVALID_ARG. */
  int32_t psi_stride;            /* k > 1: keep the backward messages Psi_t only for t = 2, T and
                                    every k-th t below T, and recompute the others (k - 1 at a
                                    time, from the kept one above) whenever a forward sweep needs
                                    them: about T/k + k message panels instead of T - 1, for about
                                    (k-1)/k more backward steps per pass; results are bitwise the
                                    same.  0 or 1 = keep all (default).  Ignored in a batch.
                                    Negative values give OTS_ERR_INVALID_ARG. */
  const int32_t *commodity_t_in;  /* optional [L]: entry time a_l of each commodity (the
                                    multi-tensor scheme of the Remark after Algorithm 2, where
                                    commodities enter and leave at different times): its sources
                                    are its marginal at a_l, its sinks its marginal at b_l
                                    (commodity_t_out), 1 <= a_l < b_l <= T; it is absent outside
                                    [a_l, b_l] and counts in the capacity sums at a_l < t < b_l.
                                    NULL: a_l = 1.  Not with psi_stride > 1; the batched solver
                                    rejects windows (the server solves them one at a time). */
  const int32_t *commodity_t_out; /* optional [L]: exit time b_l; NULL: b_l = T */
  const double *commodity_capacity; /* optional [L x n_states] row-major: commodity-dependent
                                    capacities D^(0,t) (Section 3.3), P_{0,t} <= D for
                                    t = 2..T-1 with the same D for every t; +INFINITY for none, 0
                                    closes the state for that commodity.  Adds one dual per
                                    (t, state, commodity), updated after u_t in each forward step;
                                    the capacity residual includes its changes.  Runs on the
                                    per-commodity kernels (as commodity_cost does); not with
                                    state_cost_t, epsilon continuation or the batched solver.
                                    The reported dual objective leaves out the D term. */
  const int32_t *state_tail;     /* optional [n_states]: an explicit state graph (Section 3.3:
                                    storage on edges; the source and sink states of the
                                    traffic-routing model, eq. cost_traffic_routing).  Tail node
                                    of each state, -1 for none (no state leads into it); replaces
                                    edge_src and the wait loops' nodes.  State j may follow state
                                    i iff head(i) = tail(j) >= 0, or i = j when state_hold[i] = 1.
                                    Given together with state_head. */
  const int32_t *state_head;     /* optional [n_states]: head node of each state, -1 for none (it
                                    leads to no state) */
  const int32_t *state_hold;     /* optional [n_states] of 0 / 1: 1 = the state may follow itself
                                    (storage; implied when head = tail >= 0, e.g. a wait loop).
                                    Each such state with head != tail gets one message row of its
                                    own.  Runs on the register kernels; not with per-commodity costs
                                    or capacities, commodity windows, psi_stride > 1 or the batched
                                    solver (OTS_ERR_INVALID_ARG).  Feasibility is checked on the
                                    states (exact walks of T-1 transitions). */
} ots_problem_desc;

/* Options of ots_sinkhorn_solve. */
typedef struct ots_solve_opts {
  double tol;            /* stop when the relative L1 source mismatch and the relative
                            capacity residual are both <= tol (default 1e-6) */
  int32_t max_iters;     /* Sinkhorn passes (default 100000) */
  int32_t check_every;   /* passes between host reads of the measures (default 10) */
  double timeout_ms;     /* 0 = none */
  int32_t warm_start;    /* 1: continue from the current duals; 0: start from u = 1,
                            U01 = U0T = 1 on the supports (default 0) */
  int32_t use_graph;     /* 1: run each pass as one captured CUDA graph (default 1) */
  int32_t threads_per_node; /* tuning knob: threads cooperating on one node row
                               (power of two <= 256); 0 = automatic */
  int32_t eps_stages;    /* epsilon continuation: number of warm-start stages (default 3) */
  double eps_start;      /* > eps: run the passes first at eps_start, eps_start (eps /
                            eps_start)^(1/n), ... (n = eps_stages stages, each to
                            eps_stage_tol), carrying the duals lambda = -eps ln u from stage
                            to stage, then at the problem's eps to tol.  The fixed point at eps
                            is unique, so the result is the same; the pass count usually drops.
                            0 (default) = off.  Not with per-commodity costs
                            (OTS_ERR_INVALID_ARG).  The batched solver halves epsilon per
                            stage: stages at eps 2^k, ..., 2 eps, eps with
                            k = round(log2(eps_start / eps)) (eps_stages is not used there). */
  double eps_stage_tol;  /* tolerance of the warm-start stages (default 1e-4) */
} ots_solve_opts;

/* Report of ots_sinkhorn_solve / ots_iterate. */
typedef struct ots_solve_report {
  int32_t iterations;      /* passes done by this call */
  double src_residual;     /* ||U01 .* Psi_1 - R01||_1 / ||R01||_1, taken just before the
                              last source update */
  double cap_violation;    /* capacity residual of the last pass: sum_t sum_i |P_t after the
                              capacity update u_t - P_t before it| / ||R01||_1 (from u_t = 1
                              this is the excess sum (P_t - d)_+; at a fixed point it is 0) */
  double dual_objective;   /* dual objective of Theorem 3 (u = exp(-lambda/eps)) after the
                              last pass, without the constant of the entropy term */
  double seconds;          /* wall time of the call */
  int32_t status;          /* same as the return value */
} ots_solve_report;

/* Fill opts with the defaults above. */
ots_status ots_default_solve_opts(ots_solve_opts *opts);

/* Validate and copy a problem to the device (Section 3.2 problem statement, eq.
 * multicommodity; state graph of Sections 3.1 and 3.3).  On success *out owns all device
 * memory of the problem; release it with ots_destroy_problem.  Also checks reachability of
 * every sink from its commodity's sources within T-1 transitions (OTS_ERR_INFEASIBLE). */
ots_status ots_create_problem(const ots_problem_desc *desc, ots_problem **out);

/* The host part of ots_create_problem alone: every check of the descriptor (arguments, state
 * graph, costs, capacities, masses, windows) and the reachability test, with no device, stream
 * or allocator call (desc->device, stream and allocator are not used).  OTS_OK when
 * ots_create_problem would get past its host part; otherwise the same status and message
 * (ots_last_error).  Runs on machines without a GPU. */
ots_status ots_check_problem(const ots_problem_desc *desc);

/* Run Algorithm 2 (Section 4.3) until convergence: source update U01 <- R01 ./ Psi_1,
 * forward sweep with the capacity updates u_t <- min(d ./ ((hatPsi_t .* Psi_t .* K_L)^T 1), 1),
 * sink update U0T <- R0T ./ hatPsi_T, backward sweep (eq. psi_hat, eq. psi, Corollary 7).
 * opts may be NULL (defaults); rep may be NULL.  Returns OTS_OK on convergence,
 * OTS_ERR_NOT_CONVERGED / OTS_ERR_TIMEOUT otherwise (the duals are kept either way). */
ots_status ots_sinkhorn_solve(ots_problem *p, const ots_solve_opts *opts, ots_solve_report *rep);

/* Run exactly n passes of Algorithm 2 from the current duals (no convergence test); the
 * measures of the last pass go to rep (may be NULL).  With reset = 1 the duals are first
 * set to their initial values.  Used for benchmarking and iterate-by-iterate checks. */
ots_status ots_iterate(ots_problem *p, int32_t n, int32_t reset, ots_solve_report *rep);

/* Aggregate flows P_t(M) = sum_l P_{0,t}(M) (Corollary 7; eq. proj_0t for t = 1, T) of the
 * current iterate, for t in [t_begin, t_end) with 1 <= t_begin < t_end <= T + 1.
 * out: host buffer [(t_end - t_begin) x n_states], row-major, FP64.  The flow of state i
 * at t is the amount on edge / wait loop i during the interval (t-1, t). */
ots_status ots_get_flows(ots_problem *p, int32_t t_begin, int32_t t_end, double *out);

/* Per-commodity flows P_{0,t}(M) (Theorem 6, eq. proj_0t) for t in [t_begin, t_end) and
 * commodities [l_begin, l_end).  out: host [(t_end-t_begin) x (l_end-l_begin) x n_states]. */
ots_status ots_get_commodity_flows(ots_problem *p, int32_t t_begin, int32_t t_end,
                                   int32_t l_begin, int32_t l_end, double *out);

/* Same values as ots_get_commodity_flows, computed without allocating memory.  The paper has
 * no counterpart; this entry point is for callers that cannot allocate while they read
 * results: a real-time loop that must not wait on the device allocator (cudaMalloc can
 * synchronise the whole device) between solver passes, or an application that fixes this
 * library's device memory when it creates the problem and has no room for more.  ots_get_commodity_flows takes a temporary
 * device buffer per call; this variant uses one static device array of 8 MiB for the flows
 * of one t plus 256 KiB for triple indices, present on every GPU that loads the library
 * until the process exits.  Limits: (l_end - l_begin) x n_states <= 1048576 and at most
 * 65536 source and 65536 sink triples, else OTS_ERR_INVALID_ARG.  Arguments and layout as
 * in ots_get_commodity_flows (out is a host buffer).  The first call on a device looks up
 * the array's device address; make that first call before any stream capture.  All calls
 * share the one array: calls that overlap on the GPU (two problems on different streams,
 * two host threads) race on it and must be serialised by the caller.  Problems with commodity
 * windows (commodity_t_in / commodity_t_out) give OTS_ERR_INVALID_ARG here. */
ots_status ots_get_commodity_flows_noalloc(ots_problem *p, int32_t t_begin, int32_t t_end,
                                           int32_t l_begin, int32_t l_end, double *out);

/* Current duals in natural-log form (Theorem 3 convention u = exp(-lambda/eps), so
 * lambda = -eps * log u).  log_u: host [(T-2) x n_states], rows t = 2..T-1;
 * log_U01: host [n_sources] aligned with the descriptor's source triples;
 * log_U0T: host [n_sinks] aligned with the sink triples.  Any pointer may be NULL. */
ots_status ots_get_duals(ots_problem *p, double *log_u, double *log_U01, double *log_U0T);

/* Set the duals (same layout as ots_get_duals), e.g. to resume from a checkpoint; the
 * next solve or iterate call first recomputes the backward messages.  log_u entries must
 * be <= 0. */
ots_status ots_set_duals(ots_problem *p, const double *log_u, const double *log_U01,
                         const double *log_U0T);

/* Limit of the device-side waits of the pipelined step kernels (no counterpart in the paper:
 * an execution safeguard).  Each wait on a shared-memory stage (an mbarrier) is tried at most
 * `tries` times, each try suspending the waiting thread for up to 2 us; a wait that runs out
 * makes the kernel finish its own work and return, and the pass reports OTS_ERR_DEVICE_WAIT.
 * tries = 0 restores the default (2^20, about two seconds).  withhold_stage != 0 is a test
 * switch: the consumers of every block never release their first stage, so the producer's
 * next wait for it and the consumers' next wait for data run out; every copy that was
 * started has been waited for by then, so none is left in flight.  Kernels that are not
 * pipelined (narrow rows, per-commodity costs) have no such waits.  The next solve or
 * iterate call rebuilds its pass graph.  OTS_ERR_INVALID_ARG for NULL or tries < 0. */
ots_status ots_set_wait_limit(ots_problem *p, int32_t tries, int32_t withhold_stage);

/* Counters of the linear-domain path (ots_linear_iterate, ots_linear_solve[_many]); summed over
 * the problems of one call. */
typedef struct ots_linear_stats {
  int32_t linear_passes;   /* passes run in scaled FP32 linear arithmetic */
  int32_t log_passes;      /* passes thrown away and run again in FP32 log arithmetic because a
                              scaled message or dual left [2^-60, 2^60] */
  int32_t rescalings;      /* sweeps that re-took the per-node scales from the messages */
  int32_t confirm_passes;  /* log-domain passes of the confirmation (ots_linear_solve[_many]) */
  double kernel_ms;        /* device time of the linear-domain kernel launches */
} ots_linear_stats;

/* Single-commodity problems (L = 1: eq. singlecommodity_reg, Algorithm 1 of Section 4.2, which is
 * Algorithm 2 with one commodity) with FP32 messages in the linear domain: no exponential per
 * term, a multiply-add per state and interval in each sweep, and a divide per capacitated state
 * in the capacity update.  Every message keeps a power-of-two scale per node and interval and
 * every dual u_t(i) an integer exponent, re-taken from the messages by a sweep in log arithmetic
 * whenever a scaled value drifts out of [2^-30, 2^30]; a pass whose values leave [2^-60, 2^60]
 * is run again in log arithmetic.  So the iteration is Algorithm 2's at any epsilon; the linear
 * form pays off while rescalings are rare (epsilon not far below the cost differences that the
 * duals move by per pass).  One thread block runs whole passes of one problem, or a cluster of up
 * to 8 blocks above 4096 states; every block holds two message rows of n_nodes floats and one
 * float per state in shared memory, so 4 (2 n_nodes + n_states) bytes must not exceed 200 KB
 * (about 5600 nodes on a road graph; larger problems give OTS_ERR_INVALID_ARG and stay on the
 * log-domain path).  Applies to problems with L = 1, state
 * costs (also per interval) and capacities (also per interval); explicit state graphs, commodity
 * windows, per-commodity costs or capacities and batch members give OTS_ERR_INVALID_ARG.
 * The problem's device memory grows by about 36 bytes per state and interval on first use.
 *
 * ots_linear_iterate: exactly n linear-domain passes from the current duals (reset = 1: from the
 * initial duals); rep gets the measures of the last pass (dual_objective = NaN).  The duals are
 * written back to the problem (ots_get_duals, ots_get_flows read them).
 *
 * ots_linear_solve: linear-domain passes until the measures are <= tol (or max_iters passes),
 * then log-domain passes of ots_sinkhorn_solve from those duals until a pass has measures <= tol
 * (normally one): the reported measures and the flows are the log-domain path's.  opts as for
 * ots_sinkhorn_solve (warm_start, tol, max_iters, check_every for the confirmation, timeout_ms
 * between launches); epsilon continuation gives OTS_ERR_INVALID_ARG.  rep, stats may be NULL.
 *
 * ots_linear_solve_many: the same for n independent problems in one launch (one thread block
 * each, so a whole set of small problems fills the GPU); all on one device, the launch on ps[0]'s
 * stream after the other problems' streams have been synchronised.  reps: [n] or NULL.  Returns
 * OTS_OK if every problem converged, else the first failing status (per-problem statuses in
 * reps[i].status). */
ots_status ots_linear_iterate(ots_problem *p, int32_t n, int32_t reset, ots_solve_report *rep,
                              ots_linear_stats *stats);
ots_status ots_linear_solve(ots_problem *p, const ots_solve_opts *opts, ots_solve_report *rep,
                            ots_linear_stats *stats);
ots_status ots_linear_solve_many(ots_problem *const *ps, int32_t n, const ots_solve_opts *opts,
                                 ots_solve_report *reps, ots_linear_stats *stats);

/* Sizes and counters of a created problem. */
typedef struct ots_problem_stats {
  int32_t n_states;         /* states (edges plus wait loops) */
  int32_t n_nodes;
  int32_t T;
  int32_t L;
  int32_t padded_L;         /* row length of a device message panel (L rounded up) */
  int32_t threads_per_node; /* threads cooperating on one node row */
  int64_t device_bytes;     /* device memory held by the problem */
  int64_t kernels_per_pass; /* kernels of one pass of Algorithm 2 */
  int64_t kernels_launched; /* kernels of this library launched for the problem so far */
  int64_t passes_total;     /* passes run so far */
  int64_t h2d_bytes;        /* host-to-device bytes copied so far */
  int64_t d2h_bytes;        /* device-to-host bytes copied so far */
} ots_problem_stats;

ots_status ots_problem_info(const ots_problem *p, ots_problem_stats *out);

/* Device time in milliseconds of the phases of the most recent pass, from CUDA events
 * recorded on the problem's stream: ms[0] source update, ms[1] forward sweep (T-2
 * forward kernels), ms[2] sink update, ms[3] backward sweep (T-2 backward kernels).
 * Synchronises the stream.  OTS_ERR_INVALID_ARG if no pass has run yet. */
ots_status ots_last_pass_timing(ots_problem *p, double *ms);

/* The cudaStream_t (as void*) on which all device work of the problem runs, so a caller can
 * order its own work or record timing events around the solver's.  NULL if p is NULL. */
void *ots_problem_stream(const ots_problem *p);

/* ------------------------------------------------------------------------------------
 * Batches: many independent instances resident on one device, advanced together.
 *
 * The paper solves one instance at a time; a batch is this library's way of running many
 * small instances at once without one kernel launch per Sinkhorn step of each.  Every
 * instance in a batch runs Algorithm 2 exactly as ots_sinkhorn_solve does (same updates,
 * convergence measured after every pass), but all resident instances advance by one
 * step per launch of one persistent kernel, each at its own position in its own step
 * sequence, and launches are replayed from a captured CUDA graph.  When an instance has
 * converged (or reached its pass limit) the batch also computes its flows; its slot can
 * then be reused.  Results do not depend on which other instances share the batch.
 *
 * Limits of batched instances: L <= 256 commodities, commodity-independent costs
 * (commodity_cost must be NULL), duals start from the initialisation of Algorithm 2
 * (no warm start).  Device memory of the instances comes from one pool allocated at
 * ots_batch_create (admission by memory: ots_batch_add returns OTS_ERR_OOM when the
 * instance does not fit in what is free).
 * ------------------------------------------------------------------------------------ */
typedef struct ots_batch ots_batch;

typedef struct ots_batch_desc {
  int32_t device;
  void *stream;              /* cudaStream_t for all work of the batch; NULL = own stream */
  int64_t pool_bytes;        /* device memory for resident instances */
  int32_t max_instances;     /* instances resident at once (slots) */
  int32_t max_items;         /* work items per tick (0 = 1 << 20); an instance of V nodes
                                with thread mapping G takes ceil(V G / 256) items */
  int32_t ticks_per_launch;  /* steps per graph launch (0 = 32) */
  ots_alloc_fn alloc;        /* optional allocator for the pool (both or neither) */
  ots_free_fn free_fn;
  void *alloc_ctx;
} ots_batch_desc;

/* Counters of a batch. */
typedef struct ots_batch_stats {
  int32_t resident;          /* instances holding a slot (running or finished, not removed) */
  int32_t running;           /* instances still iterating */
  int64_t pool_bytes;
  int64_t pool_used;         /* bytes of the pool held by resident instances */
  int64_t launches;          /* graph launches so far */
  int64_t ticks;             /* tick kernels launched so far */
  int64_t items;             /* items in the current tick list */
  int64_t h2d_bytes;
  int64_t d2h_bytes;
} ots_batch_stats;

/* Fill d with defaults: device 0, own stream, 4 GiB pool, 256 slots. */
ots_status ots_default_batch_desc(ots_batch_desc *d);

ots_status ots_batch_create(const ots_batch_desc *desc, ots_batch **out);

/* Validate and copy an instance into the batch (same descriptor as ots_create_problem;
 * its device, stream and allocator fields are ignored).  opts may be NULL: tol and
 * max_iters (a pass limit) are used, the other fields are ignored.  The instance starts
 * iterating with the next ots_batch_run.  *id identifies it until ots_batch_remove.
 * OTS_ERR_OOM: no free slot or not enough free pool memory (nothing is kept). */
ots_status ots_batch_add(ots_batch *b, const ots_problem_desc *desc, const ots_solve_opts *opts, int32_t *id);

/* Advance the batch by up to max_launches graph launches, returning early once no
 * instance is running; *n_running (may be NULL) receives the number still running. */
ots_status ots_batch_run(ots_batch *b, int32_t max_launches, int32_t *n_running);

/* OTS_PENDING while the instance runs; afterwards its final status (OTS_OK,
 * OTS_ERR_NOT_CONVERGED, OTS_ERR_INFEASIBLE, OTS_ERR_NUMERIC, OTS_ERR_TIMEOUT) with the
 * measures of its last pass in rep (may be NULL; seconds = time from add to the launch
 * that finished it). */
ots_status ots_batch_status(ots_batch *b, int32_t id, ots_solve_report *rep);

/* Flows of a finished instance (OTS_OK or OTS_ERR_NOT_CONVERGED), computed by the batch at
 * its final duals; same layout as ots_get_flows.  OTS_PENDING while it runs. */
ots_status ots_batch_get_flows(ots_batch *b, int32_t id, int32_t t_begin, int32_t t_end, double *out);

/* Duals of an instance, same layout as ots_get_duals (any pointer may be NULL). */
ots_status ots_batch_get_duals(ots_batch *b, int32_t id, double *log_u, double *log_U01, double *log_U0T);

/* Stop (if running) and release an instance: its slot and pool memory become free. */
ots_status ots_batch_remove(ots_batch *b, int32_t id);

ots_status ots_batch_info(const ots_batch *b, ots_batch_stats *out);

/* Thread mapping used for instances with L commodities: G threads per node row (a power of
 * two <= 32, 32 / G node rows per warp) and C = 1 or 2 chunks of 4 commodities per thread
 * (panel width 4 G C >= L).  Without tuning: C = 1 up to L = 128, then C = 2. */
ots_status ots_batch_mapping(const ots_batch *b, int32_t L, int32_t *G, int32_t *C);

/* Autotuner: for every class of commodity counts (L up to 4, 8, 16, ..., 256) time the tick
 * kernel with each admissible chunk count C in {1, 2} on a synthetic grid instance and
 * keep the fastest per class.  With cache_path != NULL the table is read from that JSON
 * file when it exists and was made on the same device model, else measured and written
 * there.  Only affects instances added afterwards.  The batch must hold no instance. */
ots_status ots_batch_autotune(ots_batch *b, const char *cache_path);

/* Release everything of the batch (NULL is ignored). */
void ots_batch_destroy(ots_batch *b);

/* ------------------------------------------------------------------------------------
 * Server: a request loop with continuous batching on one device.
 *
 * The paper has no counterpart; this is how the library serves a stream of routing solves
 * of different sizes, horizons and commodity counts.  ots_server_submit copies a request
 * and returns at once.  Builder threads build and upload each request into the batch's
 * device pool as soon as it fits (admission by memory) and a slot is free; a driver thread
 * admits built requests into the running batch between graph launches, so requests that
 * arrive while others are on the GPU join them and their work overlaps; finished requests
 * leave with their flows and free their slot and memory.  Requests the batch does not take
 * (L > 256 or per-commodity costs) are solved one at a time by the single-instance solver on
 * a stream of their own, next to the batch, with memory from the same pool.  Every result is
 * the one the request gets alone (the batch computes each instance independently).
 * With mode = 1 every request is instead solved to completion, in arrival order, by the
 * single-instance solver: the one-at-a-time baseline behind the same interface.
 * ------------------------------------------------------------------------------------ */
typedef struct ots_server ots_server;

typedef struct ots_server_desc {
  ots_batch_desc batch;      /* device, stream, pool, slots, steps per launch of the batch */
  int32_t builder_threads;   /* host threads building requests (0 = 2) */
  int32_t max_queued;        /* open requests accepted at once (0 = unlimited); beyond it
                                ots_server_submit returns OTS_ERR_OOM */
  int32_t mode;              /* 0: continuous batching; 1: one request at a time */
} ots_server_desc;

typedef struct ots_server_stats {
  int64_t submitted, completed, failed;
  int32_t queued;            /* submitted, not yet built or admitted */
  int32_t building;          /* being built by a builder thread */
  int32_t resident;          /* in the batch */
  int32_t large_running;     /* being solved by the single-instance lane */
  int64_t pool_bytes, pool_used;
  int64_t batch_launches, batch_ticks;
} ots_server_stats;

/* Defaults: ots_default_batch_desc with 8 steps per launch, 2 builder threads, mode 0. */
ots_status ots_default_server_desc(ots_server_desc *d);

/* Start the server's threads (and create its batch in mode 0). */
ots_status ots_server_create(const ots_server_desc *desc, ots_server **out);

/* Submit a request: the descriptor's host arrays are copied (device, stream and allocator
 * fields are ignored); opts as for ots_batch_add (tol, max_iters, timeout_ms) or
 * ots_sinkhorn_solve (large and plain requests).  *ticket names the request.  Validation
 * errors of the instance surface as its final status. */
ots_status ots_server_submit(ots_server *s, const ots_problem_desc *desc, const ots_solve_opts *opts,
                             int64_t *ticket);

/* OTS_PENDING while the request is open, then its final status; rep (may be NULL) gets the
 * measures of its last pass, rep->seconds = time from submit to result. */
ots_status ots_server_poll(ots_server *s, int64_t ticket, ots_solve_report *rep);

/* Block until the request is finished (timeout_ms <= 0: no limit), then as ots_server_poll. */
ots_status ots_server_wait(ots_server *s, int64_t ticket, double timeout_ms, ots_solve_report *rep);

/* Flows of a finished request (OTS_OK or OTS_ERR_NOT_CONVERGED), same layout as ots_get_flows
 * (copied from the host-side result; no device work). */
ots_status ots_server_get_flows(ots_server *s, int64_t ticket, int32_t t_begin, int32_t t_end, double *out);

/* Milliseconds of a finished request: ms[0] from submit to admission (queueing, building),
 * ms[1] from admission to result, ms[2] from submit to result. */
ots_status ots_server_timing(ots_server *s, int64_t ticket, double *ms);

/* Drop a finished request's result. */
ots_status ots_server_release(ots_server *s, int64_t ticket);

ots_status ots_server_info(ots_server *s, ots_server_stats *out);

/* Stop the threads (a single-instance solve in progress runs to its end first) and free
 * everything; open requests are dropped. */
void ots_server_destroy(ots_server *s);

/* Free all device and host memory of the problem (NULL is ignored). */
void ots_destroy_problem(ots_problem *p);

/* Static string naming a status code. */
const char *ots_status_string(ots_status s);

/* Message of the last failed call on this thread ("" if none). */
const char *ots_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OTS_H */

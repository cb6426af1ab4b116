/*
 * ots_oracle.c -- FP64 CPU oracle for the Sinkhorn iterations of Algorithm 2
 * (Haasler, Ringh, Chen, Karlsson, "Scalable computation of dynamic flow problems via
 * multi-marginal graph-structured optimal transport", Section 4.3).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, plain reference that the GPU solver is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code with the GPU path.
 *
 * Everything is FP64 and in the log domain (a linear-domain FP64 evaluation underflows:
 * path costs divided by eps reach 1e4 nats).  Plain loops, one OpenMP parallel-for per
 * step; no blocking, fusion or reordering beyond the order of Algorithm 2.
 *
 * Notation (Section 3.2 / Theorem 6):
 *   states s = directed edges plus one wait loop per node (Section 3.3 vertex augmentation),
 *            or an explicit list of states with a head and a tail node each (-1: none) and a
 *            storage flag (orc_set_state_graph; Section 3.3 storage on edges and the
 *            source / sink states of eq. cost_traffic_routing)
 *   K      : line graph, K_ij = 1 iff edge i leads to edge j (head(i) == tail(j)), else 0
 *            (Section 3.1, C_ij = 0 or infinity), plus K_ii = 1 for a storage state
 *   K_L    : exp(-C_L / eps), L x S (Section 3.2, eq. K_multicommodity); with time-varying
 *            costs (a time-dependent network, Section 3.3) one K_L per interval t = 2..T-1
 *   d      : capacities per state (inf = none)
 *   R01,R0T: source / sink matrices L x S
 *   duals  : u_t (t = 2..T-1), U01, U0T  (eq. U_multicommodity); stored as logs
 *   messages (eq. psi_hat, eq. psi):
 *     hatPsi_2     = U01 K
 *     hatPsi_t     = (hatPsi_{t-1} .* K_L) diag(u_{t-1}) K          t = 3..T
 *     Psi_{T-1}    = U0T K^T
 *     Psi_t        = (Psi_{t+1} .* K_L) diag(u_{t+1}) K^T           t = 1..T-2
 *   projections (eq. proj_0t, Corollary 7):
 *     P_{0,1} = U01 .* Psi_1,  P_{0,T} = U0T .* hatPsi_T,
 *     P_{0,t} = (hatPsi_t .* Psi_t .* K_L) diag(u_t),  P_t = u_t .* (hatPsi_t .* Psi_t .* K_L)^T 1
 *   updates (eq. sinkhorn_multicommodity, Proposition 5):
 *     U01 <- R01 ./ Psi_1,  u_t <- min(d ./ ((hatPsi_t .* Psi_t .* K_L)^T 1), 1),  U0T <- R0T ./ hatPsi_T
 *
 * Readings where the paper is silent or garbled:
 *   - Algorithm 2 writes K inside the capacity update; K_L is meant (Corollary 7).
 *   - Initialisation: u_t = 1, U0T = 1 on the support of R0T, U01 = 1 on the support of R01.
 *   - Zero column sum (state unreachable) gives u_t = 1; d = inf gives u_t = 1;
 *     R = 0 gives U = 0 (Theorem 4, eq. u_augment); 0 * inf = 0.
 *   - Convergence measures: relative L1 source mismatch taken just before the U01 update,
 *     and the relative capacity residual sum_t sum_i |P_t after - P_t before| of each u_t
 *     update: from the initialisation (u_t = 1) this is the capacity excess (P_t - d)_+; from
 *     a warm start below the fixed point it also counts the flow a too small u_t withheld.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct orc {
  int V, E, S, L, T;
  double eps;
  int *tail, *head;            /* [S] */
  int64_t *pred_ptr;           /* [S+1]  pred(j) = { i : head(i) == tail(j) } */
  int *pred_idx;
  int64_t *succ_ptr;           /* [S+1]  succ(i) = { j : head(i) == tail(j) } */
  int *succ_idx;
  double *logKL;               /* [L*S], or [(T+1)*L*S] (rows t = 2..T-1) when tv */
  int tv;                      /* time-varying costs set by orc_set_time_costs */
  double *d;                   /* [S] */
  double *dt;                  /* [(T+1)*S] per-interval capacities (row t), or NULL */
  int *ta, *tb;                /* [L] entry and exit time of each commodity, or NULL (1 and T) */
  double *logD;                /* [L*S] log of the commodity capacities D^(0,t), or NULL */
  double *logUc;               /* [(T+1)*L*S] log U^(0,t), the duals of P_{0,t} <= D^(0,t) */
  double *R01, *R0T;           /* [L*S] dense */
  double *logu;                /* [T*S], row t (1-based) used for t = 2..T-1 */
  double *logU01, *logU0T;     /* [L*S] */
  double *psi;                 /* [T*L*S], Psi_t stored at row t for t = 1..T-1 */
  double *ph_a, *ph_b;         /* [L*S] rolling forward messages */
  double mass01, mass0T;
} orc;

#define IDX(l, s) ((size_t)(l) * (size_t)o->S + (size_t)(s))
#define PSI(t, l, s) o->psi[((size_t)(t) * (size_t)o->L + (size_t)(l)) * (size_t)o->S + (size_t)(s)]

enum { ORC_OK = 0, ORC_BAD_ARG = 1, ORC_NOMEM = 2, ORC_INFEASIBLE = 3 };

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_destroy(orc *o) {
  if (!o) return;
  free(o->tail); free(o->head); free(o->pred_ptr); free(o->pred_idx);
  free(o->succ_ptr); free(o->succ_idx); free(o->logKL); free(o->d); free(o->dt); free(o->ta); free(o->tb); free(o->logD); free(o->logUc);
  free(o->R01); free(o->R0T); free(o->logu); free(o->logU01); free(o->logU0T);
  free(o->psi); free(o->ph_a); free(o->ph_b);
  free(o);
}

/* State-level CSR of K: K_ij = 1 iff head(i) == tail(j) (Section 3.1), plus K_jj = 1 for the
 * states marked in hold (storage on a state, Section 3.3; already present when head == tail).
 * A state whose head (tail) is -1 leads to (is reached from) no other state.  pred(j) lists the
 * states i with K_ij = 1, succ(i) the states j with K_ij = 1, each in increasing state order. */
static int build_csr(orc *o, const int *hold) {
  const int S = o->S, V = o->V;
  free(o->pred_ptr); free(o->pred_idx); free(o->succ_ptr); free(o->succ_idx);
  o->pred_ptr = NULL; o->pred_idx = NULL; o->succ_ptr = NULL; o->succ_idx = NULL;
  int64_t *in_cnt = (int64_t *)calloc((size_t)V + 1, sizeof(int64_t));
  int64_t *out_cnt = (int64_t *)calloc((size_t)V + 1, sizeof(int64_t));
  int *in_list = (int *)malloc(sizeof(int) * (size_t)S), *out_list = (int *)malloc(sizeof(int) * (size_t)S);
  o->pred_ptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)S + 1));
  o->succ_ptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)S + 1));
  if (!in_cnt || !out_cnt || !in_list || !out_list || !o->pred_ptr || !o->succ_ptr) {
    free(in_cnt); free(out_cnt); free(in_list); free(out_list);
    return ORC_NOMEM;
  }
  /* per node v: the states entering v (head == v) and leaving v (tail == v), in state order */
  for (int s = 0; s < S; ++s) {
    if (o->head[s] >= 0) in_cnt[o->head[s] + 1]++;
    if (o->tail[s] >= 0) out_cnt[o->tail[s] + 1]++;
  }
  for (int v = 0; v < V; ++v) { in_cnt[v + 1] += in_cnt[v]; out_cnt[v + 1] += out_cnt[v]; }
  {
    int64_t *in_fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(V > 0 ? V : 1));
    int64_t *out_fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(V > 0 ? V : 1));
    if (!in_fill || !out_fill) {
      free(in_fill); free(out_fill); free(in_cnt); free(out_cnt); free(in_list); free(out_list);
      return ORC_NOMEM;
    }
    for (int v = 0; v < V; ++v) { in_fill[v] = in_cnt[v]; out_fill[v] = out_cnt[v]; }
    for (int s = 0; s < S; ++s) {
      if (o->head[s] >= 0) in_list[in_fill[o->head[s]]++] = s;
      if (o->tail[s] >= 0) out_list[out_fill[o->tail[s]]++] = s;
    }
    free(in_fill); free(out_fill);
  }
  /* a storage state adds itself unless head == tail already puts it there */
#define EXTRA(s) ((hold && hold[s] && !(o->head[s] >= 0 && o->head[s] == o->tail[s])) ? 1 : 0)
  o->pred_ptr[0] = 0; o->succ_ptr[0] = 0;
  for (int s = 0; s < S; ++s) {
    const int u = o->tail[s], w = o->head[s];
    o->pred_ptr[s + 1] = o->pred_ptr[s] + (u >= 0 ? in_cnt[u + 1] - in_cnt[u] : 0) + EXTRA(s);
    o->succ_ptr[s + 1] = o->succ_ptr[s] + (w >= 0 ? out_cnt[w + 1] - out_cnt[w] : 0) + EXTRA(s);
  }
  o->pred_idx = (int *)malloc(sizeof(int) * (size_t)(o->pred_ptr[S] > 0 ? o->pred_ptr[S] : 1));
  o->succ_idx = (int *)malloc(sizeof(int) * (size_t)(o->succ_ptr[S] > 0 ? o->succ_ptr[S] : 1));
  if (!o->pred_idx || !o->succ_idx) { free(in_cnt); free(out_cnt); free(in_list); free(out_list); return ORC_NOMEM; }
  for (int s = 0; s < S; ++s) {
    const int u = o->tail[s], w = o->head[s];
    int64_t k = o->pred_ptr[s];
    int placed = !EXTRA(s);
    if (u >= 0)
      for (int64_t q = in_cnt[u]; q < in_cnt[u + 1]; ++q) {
        if (!placed && in_list[q] > s) { o->pred_idx[k++] = s; placed = 1; }
        o->pred_idx[k++] = in_list[q];
      }
    if (!placed) o->pred_idx[k++] = s;
    k = o->succ_ptr[s];
    placed = !EXTRA(s);
    if (w >= 0)
      for (int64_t q = out_cnt[w]; q < out_cnt[w + 1]; ++q) {
        if (!placed && out_list[q] > s) { o->succ_idx[k++] = s; placed = 1; }
        o->succ_idx[k++] = out_list[q];
      }
    if (!placed) o->succ_idx[k++] = s;
  }
#undef EXTRA
  free(in_cnt); free(out_cnt); free(in_list); free(out_list);
  return ORC_OK;
}

/* Build the state graph and the dense problem data.
 * state_cost: C_L, either [S] (same for every commodity) or [L*S] when per_commodity != 0.
 * state_cap : [S], INFINITY for none.  Sources / sinks: (commodity, state, mass) triples,
 * repeated (commodity, state) pairs add up. */
orc *orc_create(int V, int E, const int *esrc, const int *edst, int L, int T, double eps,
                const double *state_cost, int per_commodity, const double *state_cap,
                int nsrc, const int *scomm, const int *sstate, const double *smass,
                int nsnk, const int *zcomm, const int *zstate, const double *zmass) {
  if (V <= 0 || E < 0 || L <= 0 || T < 3 || !(eps > 0)) return NULL;
  orc *o = (orc *)calloc(1, sizeof(orc));
  if (!o) return NULL;
  o->V = V; o->E = E; o->S = E + V; o->L = L; o->T = T; o->eps = eps;
  int S = o->S;
  o->tail = (int *)malloc(sizeof(int) * S);
  o->head = (int *)malloc(sizeof(int) * S);
  for (int e = 0; e < E; ++e) { o->tail[e] = esrc[e]; o->head[e] = edst[e]; }
  for (int v = 0; v < V; ++v) { o->tail[E + v] = v; o->head[E + v] = v; }
  for (int s = 0; s < S; ++s)
    if (o->tail[s] < 0 || o->tail[s] >= V || o->head[s] < 0 || o->head[s] >= V) { orc_destroy(o); return NULL; }

  if (build_csr(o, NULL)) { orc_destroy(o); return NULL; }

  size_t LS = (size_t)L * S;
  o->logKL = (double *)malloc(sizeof(double) * LS);
  for (int l = 0; l < L; ++l)
    for (int s = 0; s < S; ++s)
      o->logKL[IDX(l, s)] = -(per_commodity ? state_cost[IDX(l, s)] : state_cost[s]) / eps;
  o->d = (double *)malloc(sizeof(double) * S);
  for (int s = 0; s < S; ++s) o->d[s] = state_cap ? state_cap[s] : INFINITY;

  o->R01 = (double *)calloc(LS, sizeof(double));
  o->R0T = (double *)calloc(LS, sizeof(double));
  for (int k = 0; k < nsrc; ++k) {
    if (scomm[k] < 0 || scomm[k] >= L || sstate[k] < 0 || sstate[k] >= S || smass[k] < 0) { orc_destroy(o); return NULL; }
    o->R01[IDX(scomm[k], sstate[k])] += smass[k];
  }
  for (int k = 0; k < nsnk; ++k) {
    if (zcomm[k] < 0 || zcomm[k] >= L || zstate[k] < 0 || zstate[k] >= S || zmass[k] < 0) { orc_destroy(o); return NULL; }
    o->R0T[IDX(zcomm[k], zstate[k])] += zmass[k];
  }
  o->mass01 = 0; o->mass0T = 0;
  for (size_t q = 0; q < LS; ++q) { o->mass01 += o->R01[q]; o->mass0T += o->R0T[q]; }

  o->logu = (double *)calloc((size_t)T * S, sizeof(double));
  o->logU01 = (double *)malloc(sizeof(double) * LS);
  o->logU0T = (double *)malloc(sizeof(double) * LS);
  o->ph_a = (double *)malloc(sizeof(double) * LS);
  o->ph_b = (double *)malloc(sizeof(double) * LS);
  if (!o->logKL || !o->R01 || !o->R0T || !o->logu || !o->logU01 || !o->logU0T || !o->ph_a || !o->ph_b) {
    orc_destroy(o); return NULL;
  }
  return o;
}

/* Replace the state graph by explicit heads and tails (-1: none) and a storage flag per state
 * (Section 3.3: storage on edges, and the source / sink states of eq. cost_traffic_routing, which
 * nothing enters and nothing leaves).  hold may be NULL.  Call before orc_init_duals. */
int orc_set_state_graph(orc *o, const int *tail, const int *head, const int *hold) {
  for (int s = 0; s < o->S; ++s)
    if (tail[s] < -1 || tail[s] >= o->V || head[s] < -1 || head[s] >= o->V) return ORC_BAD_ARG;
  memcpy(o->tail, tail, sizeof(int) * (size_t)o->S);
  memcpy(o->head, head, sizeof(int) * (size_t)o->S);
  return build_csr(o, hold);
}

/* log K_L row of commodity l in interval t (t >= 2). */
static const double *kl_row(const orc *o, int t, int l) {
  return o->logKL + ((size_t)(o->tv ? t : 0) * o->L + l) * o->S;
}

/* Time-varying network (Section 3.3: C replaced by time-dependent C_t): per-interval state
 * costs cost_t[(t-2)*S + s] for t = 2..T-1, the same for every commodity; +INFINITY closes
 * state s during interval t.  Replaces the costs given at creation. */
int orc_set_time_costs(orc *o, const double *cost_t) {
  const int S = o->S, L = o->L, T = o->T;
  double *k = (double *)malloc(sizeof(double) * (size_t)(T + 1) * L * S);
  if (!k) return ORC_NOMEM;
  for (size_t q = 0; q < (size_t)(T + 1) * L * S; ++q) k[q] = 0.0;
  for (int t = 2; t <= T - 1; ++t)
    for (int l = 0; l < L; ++l)
      for (int s = 0; s < S; ++s) k[((size_t)t * L + l) * S + s] = -cost_t[(size_t)(t - 2) * S + s] / o->eps;
  free(o->logKL);
  o->logKL = k;
  o->tv = 1;
  return ORC_OK;
}

/* Per-interval capacities d_t (the problem statements of Section 3 give one capacity vector
 * per interval t = 2..T-1): cap_t is [(T-2)*S], row t-2 for interval t, INFINITY for none. */
int orc_set_time_capacities(orc *o, const double *cap_t) {
  const int S = o->S, T = o->T;
  double *d = (double *)malloc(sizeof(double) * (size_t)(T + 1) * S);
  if (!d) return ORC_NOMEM;
  for (size_t q = 0; q < (size_t)(T + 1) * S; ++q) d[q] = INFINITY;
  for (int t = 2; t <= T - 1; ++t)
    for (int s = 0; s < S; ++s) {
      const double c = cap_t[(size_t)(t - 2) * S + s];
      if (!(c >= 0)) { free(d); return ORC_BAD_ARG; }
      d[(size_t)t * S + s] = c;
    }
  free(o->dt);
  o->dt = d;
  return ORC_OK;
}

/* Per-commodity entry and exit times (the multi-tensor scheme of the Remark after
 * Algorithm 2, where commodities enter and leave at different times): commodity l has its
 * source marginal at time a[l] and its sink marginal at b[l], 1 <= a[l] < b[l] <= T; it is
 * absent before a[l] and after b[l] and counts in the capacity sums at a[l] < t < b[l]. */
int orc_set_windows(orc *o, const int *a, const int *b) {
  for (int l = 0; l < o->L; ++l)
    if (a[l] < 1 || b[l] > o->T || a[l] >= b[l]) return ORC_BAD_ARG;
  free(o->ta); free(o->tb);
  o->ta = (int *)malloc(sizeof(int) * o->L);
  o->tb = (int *)malloc(sizeof(int) * o->L);
  if (!o->ta || !o->tb) return ORC_NOMEM;
  memcpy(o->ta, a, sizeof(int) * o->L);
  memcpy(o->tb, b, sizeof(int) * o->L);
  return ORC_OK;
}

/* Commodity-dependent capacities (Section 3.3): P_{0,t}(M) <= D^(0,t) for t = 2..T-1, with one
 * D (L x S, INFINITY for none) for every t.  Each adds a dual U^(0,t) per (commodity, state)
 * that multiplies K_L like u_t does; its Sinkhorn update (Proposition 5 with the commodity mode)
 * follows the update of u_t in each forward step:
 * U^(0,t) <- min(U^(0,t) .* D ./ P_{0,t}, 1). */
int orc_set_commodity_capacities(orc *o, const double *D) {
  const size_t LS = (size_t)o->L * o->S;
  double *ld = (double *)malloc(sizeof(double) * LS);
  double *lu = (double *)calloc((size_t)(o->T + 1) * LS, sizeof(double));
  if (!ld || !lu) { free(ld); free(lu); return ORC_NOMEM; }
  for (size_t q = 0; q < LS; ++q) {
    if (!(D[q] >= 0)) { free(ld); free(lu); return ORC_BAD_ARG; }
    ld[q] = log(D[q]);
  }
  free(o->logD); free(o->logUc);
  o->logD = ld;
  o->logUc = lu;
  return ORC_OK;
}

/* log of the weight of state i for commodity l in interval t: log K_L (+ log U^(0,t)) */
static double wlog(const orc *o, int t, int l, int i) {
  double w = kl_row(o, t, l)[i];
  if (o->logUc && t >= 2 && t <= o->T - 1) w += o->logUc[((size_t)t * o->L + l) * o->S + i];
  return w;
}

static int t_in(const orc *o, int l) { return o->ta ? o->ta[l] : 1; }
static int t_out(const orc *o, int l) { return o->tb ? o->tb[l] : o->T; }

/* commodity l's row of a message array is log 0 (the commodity is absent at that time) */
static void set_absent(const orc *o, double *x, int l) {
  for (int s = 0; s < o->S; ++s) x[(size_t)l * o->S + s] = -INFINITY;
}

/* capacity of state s in interval t */
static double cap_at(const orc *o, int t, int s) { return o->dt ? o->dt[(size_t)t * o->S + s] : o->d[s]; }

int orc_num_states(const orc *o) { return o->S; }
int64_t orc_nnz(const orc *o) { return o->pred_ptr[o->S]; }

/* ---- duals ---------------------------------------------------------------------- */

/* Initialisation (reading of the unspecified first line of Algorithm 2):
 * u_t = 1, U01 = U0T = 1 on the supports of R01 / R0T and 0 elsewhere. */
void orc_init_duals(orc *o) {
  size_t LS = (size_t)o->L * o->S;
  for (size_t q = 0; q < (size_t)o->T * o->S; ++q) o->logu[q] = 0.0;
  if (o->logUc)
    for (size_t q = 0; q < (size_t)(o->T + 1) * o->L * o->S; ++q) o->logUc[q] = 0.0;
  for (size_t q = 0; q < LS; ++q) {
    o->logU01[q] = o->R01[q] > 0 ? 0.0 : -INFINITY;
    o->logU0T[q] = o->R0T[q] > 0 ? 0.0 : -INFINITY;
  }
}

/* logu: [(T-2)*S] rows t = 2..T-1; logU01, logU0T: [L*S] (values off the supports are ignored) */
void orc_set_duals(orc *o, const double *logu, const double *logU01, const double *logU0T) {
  size_t LS = (size_t)o->L * o->S;
  for (int t = 2; t <= o->T - 1; ++t)
    memcpy(o->logu + (size_t)t * o->S, logu + (size_t)(t - 2) * o->S, sizeof(double) * o->S);
  for (size_t q = 0; q < LS; ++q) {
    o->logU01[q] = o->R01[q] > 0 ? logU01[q] : -INFINITY;
    o->logU0T[q] = o->R0T[q] > 0 ? logU0T[q] : -INFINITY;
  }
}

void orc_get_duals(const orc *o, double *logu, double *logU01, double *logU0T) {
  size_t LS = (size_t)o->L * o->S;
  for (int t = 2; t <= o->T - 1; ++t)
    memcpy(logu + (size_t)(t - 2) * o->S, o->logu + (size_t)t * o->S, sizeof(double) * o->S);
  memcpy(logU01, o->logU01, sizeof(double) * LS);
  memcpy(logU0T, o->logU0T, sizeof(double) * LS);
}

/* ---- message products (Theorem 6) ------------------------------------------------ */

/* out[l][j] = log sum_{i in pred(j)} exp(x[l][i] + logKL[l][i] + logu_t[i])   (one forward
 * product (X .* K_L) diag(u_t) K); with t == 0 the weights are dropped (X K). */
static void fwd_product(const orc *o, const double *x, int t, double *out, int l0, int l1) {
  const int S = o->S;
  const double *lu = t > 0 ? o->logu + (size_t)t * S : NULL;
#pragma omp parallel for schedule(static) collapse(2)
  for (int l = l0; l < l1; ++l) {
    for (int j = 0; j < S; ++j) {
      const double *xl = x + (size_t)(l - l0) * S;
      double m = -INFINITY;
      for (int64_t k = o->pred_ptr[j]; k < o->pred_ptr[j + 1]; ++k) {
        int i = o->pred_idx[k];
        double v = xl[i] + (lu ? wlog(o, t, l, i) + lu[i] : 0.0);
        if (v > m) m = v;
      }
      double r = -INFINITY;
      if (m > -INFINITY) {
        double acc = 0.0;
        for (int64_t k = o->pred_ptr[j]; k < o->pred_ptr[j + 1]; ++k) {
          int i = o->pred_idx[k];
          double v = xl[i] + (lu ? wlog(o, t, l, i) + lu[i] : 0.0);
          acc += exp(v - m);
        }
        r = m + log(acc);
      }
      out[(size_t)(l - l0) * S + j] = r;
    }
  }
}

/* out[l][i] = log sum_{j in succ(i)} exp(x[l][j] + logKL[l][j] + logu_t[j])   (one backward
 * product (X .* K_L) diag(u_t) K^T); with t == 0 the weights are dropped (X K^T). */
static void bwd_product(const orc *o, const double *x, int t, double *out, int l0, int l1) {
  const int S = o->S;
  const double *lu = t > 0 ? o->logu + (size_t)t * S : NULL;
#pragma omp parallel for schedule(static) collapse(2)
  for (int l = l0; l < l1; ++l) {
    for (int i = 0; i < S; ++i) {
      const double *xl = x + (size_t)(l - l0) * S;
      double m = -INFINITY;
      for (int64_t k = o->succ_ptr[i]; k < o->succ_ptr[i + 1]; ++k) {
        int j = o->succ_idx[k];
        double v = xl[j] + (lu ? wlog(o, t, l, j) + lu[j] : 0.0);
        if (v > m) m = v;
      }
      double r = -INFINITY;
      if (m > -INFINITY) {
        double acc = 0.0;
        for (int64_t k = o->succ_ptr[i]; k < o->succ_ptr[i + 1]; ++k) {
          int j = o->succ_idx[k];
          double v = xl[j] + (lu ? wlog(o, t, l, j) + lu[j] : 0.0);
          acc += exp(v - m);
        }
        r = m + log(acc);
      }
      out[(size_t)(l - l0) * S + i] = r;
    }
  }
}

/* log of the column sums of (hatPsi_t .* Psi_t .* K_L) over commodities: ls[i]. */
static void col_lse(const orc *o, int t, const double *ph, const double *ps, double *ls) {
  const int S = o->S, L = o->L;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < S; ++i) {
    double m = -INFINITY;
    for (int l = 0; l < L; ++l) {
      double v = ph[(size_t)l * S + i] + ps[(size_t)l * S + i] + wlog(o, t, l, i);
      if (v > m) m = v;
    }
    double r = -INFINITY;
    if (m > -INFINITY) {
      double acc = 0.0;
      for (int l = 0; l < L; ++l)
        acc += exp(ph[(size_t)l * S + i] + ps[(size_t)l * S + i] + wlog(o, t, l, i) - m);
      r = m + log(acc);
    }
    ls[i] = r;
  }
}

/* 0 * inf = 0 and 0 * (-inf) = 0 (the paper's convention for the dual objective). */
static double xlogy(double x, double logy) { return x == 0.0 ? 0.0 : x * logy; }

/* eps * ( <R01, log U01> + <R0T, log U0T> + sum_t <d, log u_t> ): the linear part of the
 * dual objective of Theorem 3 (u = exp(-lambda / eps)). */
static double dual_linear_part(const orc *o) {
  size_t LS = (size_t)o->L * o->S;
  double a = 0.0;
  for (size_t q = 0; q < LS; ++q) a += xlogy(o->R01[q], o->logU01[q]) + xlogy(o->R0T[q], o->logU0T[q]);
  for (int t = 2; t <= o->T - 1; ++t)
    for (int s = 0; s < o->S; ++s)
      if (isfinite(cap_at(o, t, s))) a += xlogy(cap_at(o, t, s), o->logu[(size_t)t * o->S + s]);
  if (o->logD)
    for (int t = 2; t <= o->T - 1; ++t)
      for (size_t q = 0; q < LS; ++q)
        if (isfinite(o->logD[q])) a += xlogy(exp(o->logD[q]), o->logUc[(size_t)t * LS + q]);
  return o->eps * a;
}

/* ---- Algorithm 2 ------------------------------------------------------------------ */

static int ensure_psi(orc *o) {
  if (o->psi) return ORC_OK;
  o->psi = (double *)malloc(sizeof(double) * (size_t)o->T * o->L * o->S);
  return o->psi ? ORC_OK : ORC_NOMEM;
}

/* "Compute Psi_t, for t = 1..T-1" from the current duals. */
int orc_backward_sweep(orc *o) {
  if (ensure_psi(o)) return ORC_NOMEM;
  const int T = o->T;
  size_t LS = (size_t)o->L * o->S;
  bwd_product(o, o->logU0T, 0, o->psi + (size_t)(T - 1) * LS, 0, o->L);        /* Psi_{T-1} = U0T K^T */
  for (int l = 0; l < o->L; ++l)                   /* commodities that leave before T are absent */
    if (t_out(o, l) != T) set_absent(o, o->psi + (size_t)(T - 1) * LS, l);
  for (int t = T - 1; t >= 2; --t) {                                           /* Psi_{t-1} */
    bwd_product(o, o->psi + (size_t)t * LS, t, o->psi + (size_t)(t - 1) * LS, 0, o->L);
    for (int l = 0; l < o->L; ++l)                 /* leaving at t: Psi_{t-1} = U0T K^T */
      if (t_out(o, l) == t)
        bwd_product(o, o->logU0T + (size_t)l * o->S, 0, o->psi + (size_t)(t - 1) * LS + (size_t)l * o->S, l, l + 1);
  }
  return ORC_OK;
}

/* |P_new - P_old| of one capacity update, P = exp(log u + ls): the excess (P_old - d)_+ where
 * u_t drops, the withheld flow where it rises (from a warm start below the fixed point). */
static double flow_change(double lu_old, double lu_new, double ls) {
  if (lu_old == -INFINITY && lu_new == -INFINITY) return 0.0;
  if (lu_old == -INFINITY) return exp(lu_new + ls);
  if (lu_new == -INFINITY) return exp(lu_old + ls);
  return exp(lu_old + ls) * fabs(expm1(lu_new - lu_old));
}

/* One pass of the while loop of Algorithm 2.  Requires orc_backward_sweep to have been run
 * for the current duals (orc_solve does this).  Outputs the two convergence measures and,
 * if trace != NULL, the dual objective after every block update (T entries: after U01,
 * after u_2 .. u_{T-1}, after U0T). */
int orc_iteration(orc *o, double *src_resid, double *cap_viol, double *trace) {
  if (!o->psi) return ORC_BAD_ARG;
  const int S = o->S, L = o->L, T = o->T;
  size_t LS = (size_t)L * S;
  int bad = 0;

  /* U01 <- R01 ./ Psi_1 (Psi_a for a commodity entering at a), with the mismatch
   * |U01 .* Psi_1 - R01| taken just before. */
  double resid = 0.0, mass_now = 0.0;
  for (size_t q = 0; q < LS; ++q) {
    if (o->R01[q] > 0) {
      const double p1 = o->psi[(size_t)t_in(o, (int)(q / S)) * LS + q];
      resid += fabs(exp(o->logU01[q] + p1) - o->R01[q]);
      if (!(p1 > -INFINITY)) bad = 1;
      o->logU01[q] = log(o->R01[q]) - p1;
      mass_now += exp(o->logU01[q] + p1);
    }
  }
  if (bad) return ORC_INFEASIBLE;
  if (src_resid) *src_resid = resid / o->mass01;
  if (trace) trace[0] = -o->eps * mass_now + dual_linear_part(o);

  /* hatPsi_2 <- U01 K (commodities entering later are absent) */
  double *ph = o->ph_a, *pn = o->ph_b;
  fwd_product(o, o->logU01, 0, ph, 0, L);
  for (int l = 0; l < L; ++l)
    if (t_in(o, l) != 1) set_absent(o, ph, l);

  double *ls = (double *)malloc(sizeof(double) * S);
  double viol = 0.0;
  for (int t = 2; t <= T - 1; ++t) {
    /* u_t <- min(d ./ ((hatPsi_t .* Psi_t .* K_L)^T 1), 1), excess (P_t - d)_+ taken before */
    col_lse(o, t, ph, o->psi + (size_t)t * LS, ls);
    double *lu = o->logu + (size_t)t * S;
    double mass_t = 0.0;
    for (int i = 0; i < S; ++i) {
      if (ls[i] > -INFINITY) {
        const double di = cap_at(o, t, i);
        const double lu_old = lu[i];
        lu[i] = isfinite(di) ? fmin(log(di) - ls[i], 0.0) : 0.0;
        viol += flow_change(lu_old, lu[i], ls[i]);
        mass_t += exp(lu[i] + ls[i]);
      } else {
        lu[i] = 0.0;
      }
    }
    if (o->logD) {
      /* U^(0,t) <- min(U^(0,t) .* D ./ P_{0,t}, 1), P_{0,t} under the new u_t */
      double *lc = o->logUc + (size_t)t * LS;
      for (int l = 0; l < L; ++l)
        for (int i = 0; i < S; ++i) {
          const size_t q = (size_t)l * S + i;
          const double base = ph[q] + o->psi[(size_t)t * LS + q] + kl_row(o, t, l)[i] + lu[i];
          if (!(base > -INFINITY)) { lc[q] = 0.0; continue; }
          const double old = lc[q];
          lc[q] = isfinite(o->logD[q]) ? fmin(o->logD[q] - base, 0.0) : 0.0;
          viol += flow_change(old, lc[q], base);
        }
    }
    if (trace) trace[t - 1] = -o->eps * mass_t + dual_linear_part(o);
    /* hatPsi_{t+1} <- (hatPsi_t .* K_L) diag(u_t) K */
    fwd_product(o, ph, t, pn, 0, L);
    for (int l = 0; l < L; ++l) {
      if (t_in(o, l) == t)                         /* entering at t: hatPsi_{t+1} = U01 K */
        fwd_product(o, o->logU01 + (size_t)l * S, 0, pn + (size_t)l * S, l, l + 1);
      if (t_out(o, l) == t + 1 && t + 1 < T)       /* leaving at t+1 < T: U0T <- R0T ./ hatPsi_{t+1} */
        for (int s = 0; s < S; ++s) {
          const size_t q = (size_t)l * S + s;
          if (o->R0T[q] > 0) {
            if (!(pn[q] > -INFINITY)) bad = 1;
            o->logU0T[q] = log(o->R0T[q]) - pn[q];
          }
        }
    }
    double *tmp = ph; ph = pn; pn = tmp;
  }
  free(ls);

  /* U0T <- R0T ./ hatPsi_T  (commodities leaving at T) */
  mass_now = 0.0;
  for (size_t q = 0; q < LS; ++q) {
    if (o->R0T[q] > 0 && t_out(o, (int)(q / S)) == T) {
      if (!(ph[q] > -INFINITY)) bad = 1;
      o->logU0T[q] = log(o->R0T[q]) - ph[q];
      mass_now += exp(o->logU0T[q] + ph[q]);
    }
  }
  if (bad) return ORC_INFEASIBLE;
  if (trace) trace[T - 1] = -o->eps * mass_now + dual_linear_part(o);
  if (cap_viol) *cap_viol = viol / o->mass01;

  /* Psi_{T-1} <- U0T K^T;  Psi_{t-1} <- (Psi_t .* K_L) diag(u_t) K^T,  t = T-1..2 */
  return orc_backward_sweep(o);
}

/* Dual objective of Theorem 3 at the current duals (needs the backward messages):
 * -eps <K, U> + eps (<R01, log U01> + <R0T, log U0T> + sum_t <d, log u_t>),  <K,U> = 1^T P_{0,1} 1. */
double orc_dual_objective(orc *o) {
  size_t LS = (size_t)o->L * o->S;
  double mass_now = 0.0;
  for (size_t q = 0; q < LS; ++q)
    if (o->R01[q] > 0) mass_now += exp(o->logU01[q] + o->psi[(size_t)t_in(o, (int)(q / o->S)) * LS + q]);
  return -o->eps * mass_now + dual_linear_part(o);
}

/* Run Algorithm 2 from the current duals until both relative measures are <= tol or
 * max_iters passes are done.  Returns ORC_OK; *iters = passes done. */
int orc_solve(orc *o, int max_iters, double tol, int *iters, double *src_resid, double *cap_viol) {
  int rc = orc_backward_sweep(o);
  if (rc) return rc;
  double r = INFINITY, c = INFINITY;
  int k = 0;
  while (k < max_iters) {
    rc = orc_iteration(o, &r, &c, NULL);
    ++k;
    if (rc) break;
    if (r <= tol && c <= tol) break;
  }
  if (iters) *iters = k;
  if (src_resid) *src_resid = r;
  if (cap_viol) *cap_viol = c;
  return rc;
}

/* ---- projections at fixed duals (Theorem 6, Corollary 7) ---------------------------- */

/* Messages for commodities [l0, l1) at the current duals, recomputed from scratch (does not
 * touch the stored Psi).  psihat: rows t = 2..T  ([T-1][l1-l0][S], row 0 = hatPsi_2);
 * psi: rows t = 1..T-1 ([T-1][l1-l0][S], row 0 = Psi_1).  Either pointer may be NULL. */
int orc_messages(orc *o, int l0, int l1, double *psihat, double *psi) {
  if (l0 < 0 || l1 > o->L || l0 >= l1) return ORC_BAD_ARG;
  const int S = o->S, T = o->T, nl = l1 - l0;
  size_t blk = (size_t)nl * S;
  double *h = (double *)malloc(sizeof(double) * blk * (T - 1));
  double *b = (double *)malloc(sizeof(double) * blk * (T - 1));
  if (!h || !b) { free(h); free(b); return ORC_NOMEM; }
  /* forward: hatPsi_2 = U01 K, hatPsi_{t+1} = (hatPsi_t .* K_L) diag(u_t) K */
  fwd_product(o, o->logU01 + (size_t)l0 * S, 0, h, l0, l1);
  for (int l = l0; l < l1; ++l)
    if (t_in(o, l) != 1) set_absent(o, h, l - l0);
  for (int t = 2; t <= T - 1; ++t) {
    fwd_product(o, h + (size_t)(t - 2) * blk, t, h + (size_t)(t - 1) * blk, l0, l1);
    for (int l = l0; l < l1; ++l)                  /* entering at t: hatPsi_{t+1} = U01 K */
      if (t_in(o, l) == t)
        fwd_product(o, o->logU01 + (size_t)l * S, 0, h + (size_t)(t - 1) * blk + (size_t)(l - l0) * S, l, l + 1);
  }
  /* backward: Psi_{T-1} = U0T K^T, Psi_{t-1} = (Psi_t .* K_L) diag(u_t) K^T  (row t-1 holds Psi_t) */
  bwd_product(o, o->logU0T + (size_t)l0 * S, 0, b + (size_t)(T - 2) * blk, l0, l1);
  for (int l = l0; l < l1; ++l)
    if (t_out(o, l) != T) set_absent(o, b + (size_t)(T - 2) * blk, l - l0);
  for (int t = T - 1; t >= 2; --t) {
    bwd_product(o, b + (size_t)(t - 1) * blk, t, b + (size_t)(t - 2) * blk, l0, l1);
    for (int l = l0; l < l1; ++l)                  /* leaving at t: Psi_{t-1} = U0T K^T */
      if (t_out(o, l) == t)
        bwd_product(o, o->logU0T + (size_t)l * S, 0, b + (size_t)(t - 2) * blk + (size_t)(l - l0) * S, l, l + 1);
  }
  if (psihat) memcpy(psihat, h, sizeof(double) * blk * (T - 1));
  if (psi) memcpy(psi, b, sizeof(double) * blk * (T - 1));
  free(h); free(b);
  return ORC_OK;
}

/* P_{0,t} for t = 1..T and commodities [l0, l1) at the current duals:
 * out[(t-1)][l-l0][s]  (eq. proj_0t). */
int orc_projections(orc *o, int l0, int l1, double *out) {
  if (l0 < 0 || l1 > o->L || l0 >= l1) return ORC_BAD_ARG;
  const int S = o->S, T = o->T, nl = l1 - l0;
  size_t blk = (size_t)nl * S;
  double *h = (double *)malloc(sizeof(double) * blk * (T - 1));
  double *b = (double *)malloc(sizeof(double) * blk * (T - 1));
  if (!h || !b) { free(h); free(b); return ORC_NOMEM; }
  int rc = orc_messages(o, l0, l1, h, b);
  if (rc) { free(h); free(b); return rc; }
#pragma omp parallel for schedule(static)
  for (int l = l0; l < l1; ++l) {
    const int a = t_in(o, l), z = t_out(o, l);
    for (int s = 0; s < S; ++s) {
      size_t q = (size_t)(l - l0) * S + s;
      for (int t = 1; t <= T; ++t) out[(size_t)(t - 1) * blk + q] = 0.0;
      /* t = a: U01 .* Psi_a  (row a-1 of b holds Psi_a) */
      out[(size_t)(a - 1) * blk + q] = exp(o->logU01[(size_t)l * S + s] + b[(size_t)(a - 1) * blk + q]);
      /* a < t < z: hatPsi_t .* Psi_t .* K_L .* u_t */
      for (int t = a + 1; t <= z - 1; ++t)
        out[(size_t)(t - 1) * blk + q] = exp(h[(size_t)(t - 2) * blk + q] + b[(size_t)(t - 1) * blk + q] +
                                             wlog(o, t, l, s) + o->logu[(size_t)t * S + s]);
      /* t = z: U0T .* hatPsi_z  (row z-2 of h holds hatPsi_z) */
      out[(size_t)(z - 1) * blk + q] = exp(o->logU0T[(size_t)l * S + s] + h[(size_t)(z - 2) * blk + q]);
    }
  }
  free(h); free(b);
  return ORC_OK;
}

/* Time-only entry: k backward products of the sweep Psi_{t-1} = (Psi_t .* K_L) diag(u_t) K^T
 * starting from t = T-1 on commodities [0, L), written into a scratch pair; used to measure
 * the oracle's update rate on a bounded sample of a large instance. */
int orc_sample_backward_products(orc *o, int k, int l1) {
  if (l1 <= 0 || l1 > o->L) return ORC_BAD_ARG;
  size_t blk = (size_t)l1 * o->S;
  double *a = (double *)malloc(sizeof(double) * blk), *b = (double *)malloc(sizeof(double) * blk);
  if (!a || !b) { free(a); free(b); return ORC_NOMEM; }
  bwd_product(o, o->logU0T, 0, a, 0, l1);
  int t = o->T - 1;
  for (int r = 0; r < k; ++r) {
    bwd_product(o, a, t, b, 0, l1);
    double *tmp = a; a = b; b = tmp;
    if (--t < 2) t = o->T - 1;
  }
  free(a); free(b);
  return ORC_OK;
}

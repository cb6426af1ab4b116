/* solve_grid.c -- the C ABI of include/ots.h used from plain C: a 6 x 6 grid road network
 * (both directions of every street, plus a wait loop at every node), two commodities
 * crossing it in opposite directions through capacitated streets, T = 14 time steps.
 * Builds the problem from host arrays, runs Algorithm 2 to a tolerance, reads the aggregate
 * flows P_t and the duals, and prints a short report.  Exit code 0 on OTS_OK. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "ots.h"

#define ROWS 6
#define COLS 6
#define NODES (ROWS * COLS)
#define HORIZON 14
#define COMMODITIES 2

int main(void) {
  int32_t src[4 * NODES], dst[4 * NODES];
  double cost[4 * NODES], cap[4 * NODES], wait_cost[NODES];
  int E = 0;
  for (int r = 0; r < ROWS; ++r)
    for (int c = 0; c < COLS; ++c) {
      const int v = r * COLS + c;
      const int dr[4] = {0, 1, 0, -1}, dc[4] = {1, 0, -1, 0};
      for (int k = 0; k < 4; ++k) {
        const int rr = r + dr[k], cc = c + dc[k];
        if (rr < 0 || rr >= ROWS || cc < 0 || cc >= COLS) continue;
        src[E] = v;
        dst[E] = rr * COLS + cc;
        cost[E] = 1.0 + 0.1 * ((v + 3 * k) % 5);   /* a little variation per street */
        cap[E] = 0.35;                              /* each street carries at most 0.35 per step */
        ++E;
      }
      wait_cost[v] = 0.2;
    }
  /* commodity 0: corner (0,0) -> (5,5); commodity 1: (5,0) -> (0,5); sources and sinks on the
   * wait-loop states (state E + node) */
  const int32_t s_comm[2] = {0, 1}, s_state[2] = {E + 0, E + (ROWS - 1) * COLS};
  const int32_t z_comm[2] = {0, 1}, z_state[2] = {E + NODES - 1, E + COLS - 1};
  const double mass[2] = {1.0, 0.8};

  ots_problem_desc d = {0};
  d.n_nodes = NODES;
  d.n_edges = E;
  d.edge_src = src;
  d.edge_dst = dst;
  d.edge_cost = cost;
  d.edge_capacity = cap;
  d.add_wait_loops = 1;
  d.wait_cost = wait_cost;
  d.wait_capacity = NULL;                          /* waiting is not capacitated */
  d.T = HORIZON;
  d.L = COMMODITIES;
  d.eps = 0.05;
  d.n_sources = 2; d.src_commodity = s_comm; d.src_state = s_state; d.src_mass = mass;
  d.n_sinks = 2; d.snk_commodity = z_comm; d.snk_state = z_state; d.snk_mass = mass;
  d.device = 0;

  ots_problem *p = NULL;
  ots_status st = ots_create_problem(&d, &p);
  if (st != OTS_OK) {
    fprintf(stderr, "create: %s: %s\n", ots_status_string(st), ots_last_error());
    return 1;
  }
  ots_solve_opts o;
  ots_default_solve_opts(&o);
  o.tol = 1e-7;
  ots_solve_report rep;
  st = ots_sinkhorn_solve(p, &o, &rep);
  printf("solve: %s after %d passes (source mismatch %.2e, capacity residual %.2e)\n", ots_status_string(st),
         rep.iterations, rep.src_residual, rep.cap_violation);
  const int S = E + NODES;
  double *flows = (double *)malloc(sizeof(double) * (size_t)HORIZON * S);
  ots_status sf = ots_get_flows(p, 1, HORIZON + 1, flows);
  int ok = st == OTS_OK && sf == OTS_OK;
  if (sf == OTS_OK) {
    double worst = 0.0, busiest = 0.0;
    for (int t = 1; t <= HORIZON; ++t) {
      double total = 0.0;
      for (int s = 0; s < S; ++s) total += flows[(size_t)(t - 1) * S + s];
      worst = fmax(worst, fabs(total - 1.8));
      if (t >= 2 && t <= HORIZON - 1)
        for (int e = 0; e < E; ++e) busiest = fmax(busiest, flows[(size_t)(t - 1) * S + e]);
    }
    printf("mass at every t: 1.8 (largest deviation %.1e); busiest street carries %.4f (capacity 0.35)\n", worst,
           busiest);
    ok = ok && worst < 1e-5 && busiest <= 0.35 + 1e-5;
  }
  double log_u[(HORIZON - 2) * (4 * NODES + NODES)];
  if (ots_get_duals(p, log_u, NULL, NULL) == OTS_OK) {
    int binding = 0;
    for (int k = 0; k < (HORIZON - 2) * S; ++k) binding += log_u[k] < -1e-9;
    printf("capacity duals below 1 (binding street-steps): %d\n", binding);
  }
  free(flows);
  ots_destroy_problem(p);
  return ok ? 0 : 2;
}

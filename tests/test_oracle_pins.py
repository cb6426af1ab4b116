"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test compares the oracle (Algorithm 2, state-level line graph, log domain) with a
computation that shares no code with it (``tests/pins_math.py``): brute force over the full
tensor, the generic Sinkhorn scheme of Proposition 5 on that tensor, closed forms, a
two-marginal reduction, the exact LP, and invariants the paper states.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, build
from paper_2106_14485_gb300 import instances as I
from tests import pins_math as PM

build()


def tiny_instance(seed=0, rows=2, cols=2, L=2, T=4, eps=0.7, cap_scale=None, per_commodity=True,
                  edge_sources=True):
    """Small grid with random per-commodity costs, optional capacities, sources/sinks on
    random states (wait loops and edges)."""
    rng = np.random.default_rng(seed)
    src, dst, pos = I.grid_graph(rows, cols)
    V, E = rows * cols, len(src)
    S = V + E
    states = np.arange(S) if edge_sources else np.arange(E, S)
    sc, ss, sm, zc, zs, zm = [], [], [], [], [], []
    for l in range(L):
        a = rng.choice(states, 2, replace=False)
        b = rng.choice(states, 2, replace=False)
        m = rng.uniform(0.5, 1.5)
        w = rng.dirichlet(np.ones(2)) * m
        w2 = rng.dirichlet(np.ones(2)) * m
        sc += [l, l]; ss += list(a); sm += list(w)
        zc += [l, l]; zs += list(b); zm += list(w2)
    cap = np.full(E, np.inf) if cap_scale is None else rng.uniform(0.3, 1.0, E) * cap_scale
    inst = I.Instance(name="tiny", n_nodes=V, edge_src=src, edge_dst=dst,
                      edge_cost=rng.uniform(0, 1, E), edge_cap=cap,
                      wait_cost=rng.uniform(0, 0.3, V), wait_cap=np.full(V, np.inf),
                      L=L, T=T, eps=eps,
                      src_comm=np.array(sc, np.int32), src_state=np.array(ss, np.int32), src_mass=np.array(sm),
                      snk_comm=np.array(zc, np.int32), snk_state=np.array(zs, np.int32), snk_mass=np.array(zm))
    if per_commodity:
        inst.commodity_cost = rng.uniform(0, 1, (L, S))
    return inst


def test_line_graph_matches_definition():
    for inst in (tiny_instance(), I.grid_single_commodity(0), I.rgg_instance(seed=3, n=60, L=4, T=12)):
        o = Oracle(inst)
        assert o.nnz == int(PM.dense_K(inst).sum())
        assert o.nnz == inst.nnz_line_graph()


@pytest.mark.parametrize("T", [3, 4, 5])
def test_projections_match_brute_force(T):
    """Theorem 6 / eq. proj_0t against direct summation over the tensor, random duals."""
    inst = tiny_instance(seed=T, T=T)
    o = Oracle(inst)
    rng = np.random.default_rng(10 + T)
    S, L = inst.n_states, inst.L
    R01, R0T = PM.dense_marginals(inst)
    logu = -rng.uniform(0, 2, (T - 2, S))
    U01 = rng.uniform(-2, 2, (L, S))
    U0T = rng.uniform(-2, 2, (L, S))
    o.set_duals(logu, U01, U0T)
    P = o.projections()
    tz = PM.Tensor(inst)
    u = np.ones((T + 1, S))
    u[2:T] = np.exp(logu)
    M = tz.M(u, np.where(R01 > 0, np.exp(U01), 0), np.where(R0T > 0, np.exp(U0T), 0))
    for t in range(1, T + 1):
        ref = tz.proj0t(M, t)
        np.testing.assert_allclose(P[t - 1], ref, rtol=1e-12, atol=1e-14 * ref.max())
    # the messages equal the partial sums of Theorem 6 over partial paths
    h, b = o.messages()
    assert h.shape == (T - 1, L, S) and b.shape == (T - 1, L, S)
    if T <= 4:
        hat, psi = PM.brute_messages(inst, u, np.where(R01 > 0, np.exp(U01), 0), np.where(R0T > 0, np.exp(U0T), 0))
        for t in range(2, T + 1):
            ref = hat[t]
            with np.errstate(divide="ignore"):
                np.testing.assert_allclose(np.exp(h[t - 2]), ref, rtol=1e-12, atol=1e-14 * ref.max())
        for t in range(1, T):
            ref = psi[t]
            np.testing.assert_allclose(np.exp(b[t - 1]), ref, rtol=1e-12, atol=1e-14 * ref.max())


def test_fixed_point_matches_tensor_sinkhorn():
    """Proposition 5 on the full tensor (reverse block order) reaches the same M_eps."""
    inst = tiny_instance(seed=7, T=5, L=2, cap_scale=0.8, eps=0.5)
    o = Oracle(inst)
    r = o.solve(max_iters=50000, tol=1e-13)
    assert r["status"] == 0 and r["src_resid"] < 1e-12 and r["cap_viol"] < 1e-12
    P = o.projections()
    tz, M, _ = PM.tensor_sinkhorn(inst)
    d = PM.capacity(inst)
    binding = 0
    for t in range(1, inst.T + 1):
        ref = tz.proj0t(M, t)
        np.testing.assert_allclose(P[t - 1], ref, rtol=1e-7, atol=1e-9)
        if 2 <= t <= inst.T - 1:
            binding += int(np.sum(np.isclose(ref.sum(0), d, rtol=1e-6)))
    assert binding > 0, "capacities should bind in this pin"


def test_bridge_closed_form_one_iteration():
    """No capacities, one source and one sink per commodity: Sinkhorn is exact after one
    pass, and the flows are the Markov bridge (Remark, Section 4.2)."""
    inst = I.rgg_instance(seed=5, n=30, L=3, T=9, eps=0.2)
    inst.edge_cap[:] = np.inf
    o = Oracle(inst)
    o.backward_sweep()
    o.iteration()
    r2, c2, _ = o.iteration()
    assert r2 < 1e-13 and c2 == 0.0
    P = o.projections()
    for l in range(inst.L):
        ref = PM.bridge_flows(inst, l)
        np.testing.assert_allclose(P[:, l, :], ref, rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grid5x5_two_marginal_reduction(seed):
    """The 5x5-grid workload (multi-source, single commodity, no capacities) equals textbook
    two-marginal Sinkhorn on K_eff = K (diag(k) K)^(T-2)."""
    inst = I.grid_single_commodity(seed)
    o = Oracle(inst)
    r = o.solve(max_iters=100000, tol=1e-13)
    assert r["status"] == 0 and r["src_resid"] < 1e-12
    P = o.projections()[:, 0, :]
    ref = PM.two_marginal_flows(inst)
    np.testing.assert_allclose(P, ref, rtol=1e-8, atol=1e-12)


def test_decoupling_nonbinding_capacities():
    """Capacities that never bind: the L-commodity solution equals L separate solves."""
    inst = I.rgg_instance(seed=11, n=40, L=4, T=10, eps=0.1)
    inst.edge_cap[:] = 1e6
    o = Oracle(inst)
    o.solve(max_iters=10, tol=1e-14)
    P = o.projections()
    for l in range(inst.L):
        one = I.Instance(**{**inst.__dict__})
        one.L = 1
        m = inst.src_comm == l
        one.src_comm = np.zeros(m.sum(), np.int32); one.src_state = inst.src_state[m]; one.src_mass = inst.src_mass[m]
        m2 = inst.snk_comm == l
        one.snk_comm = np.zeros(m2.sum(), np.int32); one.snk_state = inst.snk_state[m2]; one.snk_mass = inst.snk_mass[m2]
        o1 = Oracle(one)
        o1.solve(max_iters=10, tol=1e-14)
        np.testing.assert_allclose(P[:, l, :], o1.projections()[:, 0, :], rtol=1e-11, atol=1e-14)
    logu, _, _ = o.get_duals()
    assert np.all(logu == 0.0)


def test_lp_limit_eps_to_zero():
    """Theorems 1-2 and Section 5.1: <C, M_eps> decreases to the LP optimum as eps -> 0,
    with 0 <= gap <= eps * mass * log(#paths)."""
    inst = tiny_instance(seed=3, rows=3, cols=3, L=2, T=6, cap_scale=0.9, per_commodity=True,
                         edge_sources=False)
    lp = PM.lp_optimum(inst)
    C = PM.cost_matrix(inst)
    mass = inst.total_mass()
    gaps = []
    for eps in (0.2, 0.1, 0.05, 0.02, 0.01):
        inst.eps = eps
        o = Oracle(inst)
        r = o.solve(max_iters=200000, tol=1e-10)
        assert r["status"] == 0 and r["src_resid"] <= 1e-10 and r["cap_viol"] <= 1e-10
        P = o.projections()
        cost = sum(float(np.sum(C * P[t - 1])) for t in range(2, inst.T))
        gap = cost - lp
        bound = eps * mass * inst.T * np.log(inst.n_states)
        assert -1e-7 <= gap <= bound, (eps, gap, bound)
        gaps.append(gap)
    assert all(a >= b - 1e-9 for a, b in zip(gaps, gaps[1:])), gaps
    assert gaps[-1] < 0.1 * gaps[0]


def test_invariants_every_iterate():
    """Section 5.1 / Corollary 7 / Proposition 5 proof: on every iterate the sink mismatch is
    at rounding level, every commodity carries the same mass at every t, and the dual
    objective does not decrease after any block update; at convergence P_t <= d and
    u_t < 1 only where P_t = d (complementary slackness)."""
    inst = I.rgg_instance(seed=2, n=50, L=6, T=18, eps=0.05, cap_lo=0.15, cap_hi=0.4)
    o = Oracle(inst)
    o.backward_sweep()
    R01, R0T = PM.dense_marginals(inst)
    last = -np.inf
    for k in range(25):
        _, _, tr = o.iteration(trace=True)
        seq = np.concatenate([[last], tr])
        assert np.all(np.diff(seq) >= -1e-9 * np.abs(seq[1:]).max()), (k, np.diff(seq).min())
        last = tr[-1]
        P = o.projections()
        np.testing.assert_allclose(P[-1], R0T, rtol=1e-10, atol=1e-13)
        mass_t = P.sum(axis=2)                       # [T, L]
        np.testing.assert_allclose(mass_t, np.broadcast_to(mass_t[-1], mass_t.shape), rtol=1e-10)
    r = o.solve(max_iters=100000, tol=1e-11)
    assert r["status"] == 0
    P = o.projections()
    d = PM.capacity(inst)
    logu, _, _ = o.get_duals()
    Pt = P[1:-1].sum(axis=1)                         # [T-2, S]
    excess = np.max(Pt - d[None, :])
    assert excess <= 1e-8, excess
    tight = logu < -1e-6
    assert tight.any(), "capacities should bind"
    np.testing.assert_allclose(Pt[tight], np.broadcast_to(d, Pt.shape)[tight], rtol=1e-7)


def test_zero_marginals_give_zero_duals():
    """Theorem 4 (eq. u_augment): U = 0 wherever R = 0."""
    inst = tiny_instance(seed=4, T=4)
    o = Oracle(inst)
    o.solve(max_iters=50, tol=1e-12)
    _, U01, U0T = o.get_duals()
    R01, R0T = PM.dense_marginals(inst)
    assert np.all(np.isneginf(U01[R01 == 0])) and np.all(np.isfinite(U01[R01 > 0]))
    assert np.all(np.isneginf(U0T[R0T == 0])) and np.all(np.isfinite(U0T[R0T > 0]))


def test_degenerate_source_equals_sink_and_T3():
    """T = 3 (the smallest horizon Algorithm 2 covers) and a commodity whose source and sink
    are the same wait loop (it can only wait, or leave and come back)."""
    inst = I.rgg_instance(seed=8, n=20, L=3, T=3, eps=0.1)
    inst.snk_state = inst.src_state.copy()
    o = Oracle(inst)
    r = o.solve(max_iters=1000, tol=1e-12)
    assert r["status"] == 0 and r["src_resid"] < 1e-12
    P = o.projections()
    R01, R0T = PM.dense_marginals(inst)
    np.testing.assert_allclose(P[0], R01, rtol=1e-10)
    np.testing.assert_allclose(P[-1], R0T, rtol=1e-10)
    # the middle interval: with wait cost 0.05 vs. leaving-and-returning impossible in 2 steps
    # (needs edge then loop), all mass stays on the source loop
    np.testing.assert_allclose(P[1], R01, rtol=1e-10)


def test_infeasible_sink_is_reported():
    """A sink that no source reaches within T-1 transitions makes Psi_1 vanish on the source."""
    inst = I.grid_single_commodity(0, T=3)
    far = inst.n_edges + 24
    near = inst.n_edges + 0
    inst.src_state = np.array([near], np.int32); inst.src_mass = np.array([1.0]); inst.src_comm = np.zeros(1, np.int32)
    inst.snk_state = np.array([far], np.int32); inst.snk_mass = np.array([1.0]); inst.snk_comm = np.zeros(1, np.int32)
    o = Oracle(inst)
    o.backward_sweep()
    with pytest.raises(RuntimeError):
        o.iteration()


# ---------------------------------------------------------------------------------------
# time-varying network (Section 3.3: C replaced by time-dependent C_t)
# ---------------------------------------------------------------------------------------

def time_varying(inst, seed=0, closures=1):
    """Per-interval state costs: the static costs scaled per (t, state) by U[0.5, 2], with
    `closures` random moving edges closed (+inf) in one interval each."""
    rng = np.random.default_rng(seed)
    base = np.concatenate([inst.edge_cost, inst.wait_cost]).astype(np.float64)
    ct = base[None, :] * rng.uniform(0.5, 2.0, (inst.T - 2, base.size))
    for _ in range(closures):
        ct[rng.integers(inst.T - 2), rng.integers(inst.n_edges)] = np.inf
    inst.state_cost_t = ct
    return inst


@pytest.mark.parametrize("T", [4, 5])
def test_time_varying_projections_match_brute_force(T):
    inst = time_varying(tiny_instance(seed=20 + T, T=T, per_commodity=False), seed=T, closures=2)
    o = Oracle(inst)
    rng = np.random.default_rng(30 + T)
    S, L = inst.n_states, inst.L
    R01, R0T = PM.dense_marginals(inst)
    logu = -rng.uniform(0, 2, (T - 2, S))
    U01 = rng.uniform(-2, 2, (L, S))
    U0T = rng.uniform(-2, 2, (L, S))
    o.set_duals(logu, U01, U0T)
    P = o.projections()
    tz = PM.Tensor(inst)
    u = np.ones((T + 1, S))
    u[2:T] = np.exp(logu)
    M = tz.M(u, np.where(R01 > 0, np.exp(U01), 0), np.where(R0T > 0, np.exp(U0T), 0))
    for t in range(1, T + 1):
        ref = tz.proj0t(M, t)
        np.testing.assert_allclose(P[t - 1], ref, rtol=1e-12, atol=1e-14 * max(ref.max(), 1e-300))


def test_time_varying_fixed_point_matches_tensor_sinkhorn():
    inst = time_varying(tiny_instance(seed=7, T=5, L=2, cap_scale=0.8, eps=0.5, per_commodity=False), seed=3,
                        closures=1)
    o = Oracle(inst)
    r = o.solve(max_iters=50000, tol=1e-13)
    assert r["status"] == 0 and r["src_resid"] < 1e-12 and r["cap_viol"] < 1e-12
    P = o.projections()
    tz, M, _ = PM.tensor_sinkhorn(inst)
    for t in range(1, inst.T + 1):
        np.testing.assert_allclose(P[t - 1], tz.proj0t(M, t), rtol=1e-7, atol=1e-9)


def test_time_constant_costs_and_per_interval_shifts():
    """Costs that do not vary with t reproduce the static solution; adding a constant to every
    state's cost in one interval multiplies every path by the same factor, so M_eps does not
    change; a state closed in an interval carries no flow there."""
    base = I.rgg_instance(seed=4, n=40, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    o0 = Oracle(base)
    o0.solve(max_iters=100000, tol=1e-12)
    F0 = o0.flows()
    c = np.concatenate([base.edge_cost, base.wait_cost]).astype(np.float64)
    inst = I.rgg_instance(seed=4, n=40, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    inst.state_cost_t = np.tile(c, (inst.T - 2, 1))
    o1 = Oracle(inst)
    o1.solve(max_iters=100000, tol=1e-12)
    np.testing.assert_allclose(o1.flows(), F0, rtol=1e-10, atol=1e-12)
    shift = np.linspace(-0.3, 0.7, inst.T - 2)[:, None]
    inst.state_cost_t = np.tile(c, (inst.T - 2, 1)) + shift
    o2 = Oracle(inst)
    o2.solve(max_iters=100000, tol=1e-12)
    np.testing.assert_allclose(o2.flows(), F0, rtol=1e-8, atol=1e-10)
    # close the busiest moving edge in interval t = 4
    ct = np.tile(c, (inst.T - 2, 1))
    e = int(np.argmax(F0[3, :inst.n_edges]))
    ct[4 - 2, e] = np.inf
    inst.state_cost_t = ct
    o3 = Oracle(inst)
    r3 = o3.solve(max_iters=100000, tol=1e-12)
    assert r3["status"] == 0
    F3 = o3.flows()
    assert F3[3, e] == 0.0 and F0[3, e] > 1e-3
    assert abs(F3[0].sum() - F0[0].sum()) < 1e-9 * F0[0].sum()


# ---------------------------------------------------------------------------------------
# per-interval capacities d_t (the capacity vectors of the problem statements, one per
# interval t = 2..T-1; Algorithm 2 writes a single d)
# ---------------------------------------------------------------------------------------

def test_per_interval_capacities_fixed_point_matches_tensor_sinkhorn():
    inst = tiny_instance(seed=9, T=5, L=2, cap_scale=0.9, eps=0.5, per_commodity=False)
    rng = np.random.default_rng(2)
    d = PM.capacity(inst)
    dt = np.tile(d, (inst.T - 2, 1))
    fin = np.isfinite(dt)
    dt[fin] *= rng.uniform(0.4, 1.6, int(fin.sum()))
    dt[1, 0] = 0.0                                      # edge 0 closed in interval t = 3
    inst.state_capacity_t = dt
    o = Oracle(inst)
    r = o.solve(max_iters=50000, tol=1e-13)
    assert r["status"] == 0 and r["src_resid"] < 1e-12 and r["cap_viol"] < 1e-12
    P = o.projections()
    tz, M, _ = PM.tensor_sinkhorn(inst)
    for t in range(1, inst.T + 1):
        np.testing.assert_allclose(P[t - 1], tz.proj0t(M, t), rtol=1e-7, atol=1e-9)
    assert np.all(P[2, :, 0] == 0.0)


def test_per_interval_capacities_kkt_and_reductions():
    """At the fixed point P_t <= d_t, and a state's dual is active (u_t < 1) only where its
    capacity binds (complementary slackness of Theorem 3); d_t equal for every t reproduces
    the single-capacity solution and d_t = inf the uncapacitated one."""
    base = I.rgg_instance(seed=4, n=40, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    o0 = Oracle(base)
    o0.solve(max_iters=100000, tol=1e-12)
    F0 = o0.flows()
    inst = I.rgg_instance(seed=4, n=40, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    inst.state_capacity_t = np.tile(PM.capacity(inst), (inst.T - 2, 1))
    o1 = Oracle(inst)
    o1.solve(max_iters=100000, tol=1e-12)
    np.testing.assert_allclose(o1.flows(), F0, rtol=1e-10, atol=1e-12)
    free = I.rgg_instance(seed=4, n=40, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    free.edge_cap = np.full_like(free.edge_cap, np.inf)
    of = Oracle(free)
    of.solve(max_iters=100000, tol=1e-12)
    inst.state_capacity_t = np.full((inst.T - 2, inst.n_states), np.inf)
    o2 = Oracle(inst)
    o2.solve(max_iters=100000, tol=1e-12)
    np.testing.assert_allclose(o2.flows(), of.flows(), rtol=1e-10, atol=1e-12)
    I.with_time_varying_capacities(inst, seed=5, lo=0.8, hi=1.5, closures=1)
    o3 = Oracle(inst)
    r3 = o3.solve(max_iters=200000, tol=1e-12)
    assert r3["status"] == 0 and r3["cap_viol"] < 1e-12 and r3["iters"] < 200000
    F3 = o3.flows()
    logu, _, _ = o3.get_duals()
    dt = inst.state_capacity_t
    n_active = 0
    for t in range(2, inst.T):
        P, d, lu = F3[t - 1], dt[t - 2], logu[t - 2]
        assert np.all(P <= d + 1e-8)                   # feasible up to the solve tolerance
        act = lu < -1e-6
        n_active += int(act.sum())
        np.testing.assert_allclose(P[act], d[act], rtol=1e-6, atol=1e-8)
    assert n_active > 0
    zero = dt == 0.0
    assert zero.any() and np.all(F3[1:-1][zero] == 0.0)


# ---------------------------------------------------------------------------------------
# per-commodity entry and exit times (the multi-tensor scheme of the Remark after Algorithm 2)
# ---------------------------------------------------------------------------------------

def test_windows_fixed_point_matches_the_multi_tensor_problem():
    inst = tiny_instance(seed=11, T=6, L=3, cap_scale=0.8, eps=0.5, per_commodity=False)
    inst.commodity_t_in = np.array([2, 1, 3], np.int32)
    inst.commodity_t_out = np.array([6, 4, 6], np.int32)
    o = Oracle(inst)
    r = o.solve(max_iters=50000, tol=1e-13)
    assert r["status"] == 0 and r["src_resid"] < 1e-12 and r["cap_viol"] < 1e-12
    P = o.projections()
    proj = PM.window_tensor_sinkhorn(inst)
    for l in range(inst.L):
        for t in range(1, inst.T + 1):
            np.testing.assert_allclose(P[t - 1, l], proj(l, t), rtol=1e-7, atol=1e-9)
    R01, R0T = PM.dense_marginals(inst)
    for l in range(inst.L):                             # marginals at the commodity's own times
        np.testing.assert_allclose(P[inst.commodity_t_in[l] - 1, l], R01[l], atol=1e-12)
        np.testing.assert_allclose(P[inst.commodity_t_out[l] - 1, l], R0T[l], atol=1e-11)


def test_windows_shifted_in_time_reproduce_the_shorter_horizon():
    """All commodities present from t = 3 to t = 9 of a T = 11 horizon solve the T = 7 problem
    (time-invariant costs and capacities), shifted by two intervals; nothing flows outside."""
    short = I.rgg_instance(seed=4, n=40, L=3, T=7, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    o0 = Oracle(short)
    o0.solve(max_iters=100000, tol=1e-12)
    F0 = o0.flows()
    long = I.rgg_instance(seed=4, n=40, L=3, T=7, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    long.T = 11
    long.commodity_t_in = np.full(3, 3, np.int32)
    long.commodity_t_out = np.full(3, 9, np.int32)
    o1 = Oracle(long)
    r = o1.solve(max_iters=100000, tol=1e-12)
    assert r["status"] == 0
    F1 = o1.flows()
    np.testing.assert_allclose(F1[2:9], F0, rtol=1e-9, atol=1e-12)
    assert np.all(F1[:2] == 0.0) and np.all(F1[9:] == 0.0)


# ---------------------------------------------------------------------------------------
# commodity-dependent capacities D^(0,t) (Section 3.3), one D for every t
# ---------------------------------------------------------------------------------------

def test_commodity_capacities_fixed_point_matches_tensor_sinkhorn():
    inst = tiny_instance(seed=7, T=5, L=2, cap_scale=1.2, eps=0.5, per_commodity=False)
    rng = np.random.default_rng(4)
    D = np.full((inst.L, inst.n_states), np.inf)
    D[:, :inst.n_edges] = rng.uniform(0.08, 0.25, (inst.L, inst.n_edges))
    inst.commodity_capacity = D
    o = Oracle(inst)
    r = o.solve(max_iters=50000, tol=1e-13)
    assert r["status"] == 0 and r["iters"] < 50000 and r["cap_viol"] < 1e-12
    P = o.projections()
    tz, M, _ = PM.tensor_sinkhorn(inst, reverse=False)
    for t in range(1, inst.T + 1):
        np.testing.assert_allclose(P[t - 1], tz.proj0t(M, t), rtol=1e-7, atol=1e-9)
    act = 0
    for t in range(2, inst.T):                          # KKT of the commodity mode
        assert np.all(P[t - 1] <= D + 1e-9)
        act += int((np.abs(P[t - 1] - D) < 1e-7).sum())
    assert act > 0


def test_commodity_capacities_reductions():
    """D = inf changes nothing; with one commodity, D = d repeats the aggregate constraint and
    the fixed point is the one without D."""
    base = I.rgg_instance(seed=4, n=40, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    o0 = Oracle(base)
    o0.solve(max_iters=100000, tol=1e-12)
    inst = I.rgg_instance(seed=4, n=40, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    inst.commodity_capacity = np.full((inst.L, inst.n_states), np.inf)
    o1 = Oracle(inst)
    o1.solve(max_iters=100000, tol=1e-12)
    np.testing.assert_allclose(o1.flows(), o0.flows(), rtol=1e-12, atol=1e-14)
    single = I.single_commodity_instance(seed=1, per_interval=False)
    os_ = Oracle(single)
    os_.solve(max_iters=100000, tol=1e-13)
    single.commodity_capacity = PM.capacity(single)[None, :].copy()
    od = Oracle(single)
    r = od.solve(max_iters=100000, tol=1e-13)
    assert r["status"] == 0 and r["iters"] < 100000
    np.testing.assert_allclose(od.flows(), os_.flows(), rtol=1e-8, atol=1e-11)


@pytest.mark.parametrize("cap_scale", [None, 0.8])
def test_dual_objective_equals_the_primal_at_the_optimum(cap_scale):
    """Strong duality (Theorem 3): at the optimum the dual objective the oracle reports equals the
    entropic primal objective evaluated directly on the optimal tensor (both without the constant
    of the entropy term), with and without binding capacities."""
    inst = tiny_instance(seed=7, T=5, L=2, cap_scale=cap_scale, eps=0.5)
    o = Oracle(inst)
    r = o.solve(max_iters=100000, tol=1e-13)
    assert r["status"] == 0 and r["src_resid"] < 1e-12 and r["cap_viol"] < 1e-12
    tz, M, _ = PM.tensor_sinkhorn(inst)
    primal = PM.primal_objective(inst, tz, M)
    assert o.dual_objective() == pytest.approx(primal, rel=1e-9, abs=1e-12)

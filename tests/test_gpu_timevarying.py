"""Time-varying network (Section 3.3: C replaced by time-dependent C_t, here per-interval state
costs, +inf closing a state during an interval) and per-interval capacities d_t (eq.
multicommodity_reg), on every GPU path, against the FP64 oracle."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2106_14485_gb300 import instances as I

pytestmark = pytest.mark.gpu

FLOW_TOL = 1e-5


@pytest.fixture(scope="module")
def O():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14485_gb300 import build, ots
    build.build()
    ots.load_library()
    return ots


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def closed_cells(inst):
    t_idx, s_idx = np.nonzero(np.isinf(inst.state_cost_t))
    return t_idx + 2, s_idx                       # 1-based interval, state


@pytest.mark.parametrize("L,seed", [(9, 31), (300, 32)])
def test_single_instance_paths(O, L, seed):
    """Register kernels (L = 9) and pipelined kernels (L = 300)."""
    inst = I.with_time_varying_costs(I.rgg_instance(seed=seed, n=50, L=L, T=12, eps=0.05, cap_lo=2.0, cap_hi=6.0),
                                     seed=seed, closures=3)
    o = Oracle(inst)
    ro = o.solve(max_iters=100000, tol=1e-11)
    assert ro["status"] == 0
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-7, max_iters=50000)
    assert r["status"] == 0
    F = O.ots_get_flows(h)
    Fref = o.flows()
    assert rel_l1(F, Fref) <= FLOW_TOL
    t, s = closed_cells(inst)
    assert np.all(F[t - 1, s] == 0.0)
    O.ots_destroy_problem(h)


def test_batched_path_with_capacities(O):
    insts = [I.with_time_varying_costs(I.rgg_instance(seed=200, n=45, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0),
                                       seed=1, closures=2),
             I.with_time_varying_costs(I.rgg_instance(seed=202, n=40, L=30, T=8, eps=0.05, cap_lo=0.3, cap_hi=1.0),
                                       seed=2, lo=0.8, hi=1.25, closures=1)]
    b = O.ots_batch_create(pool_bytes=256 << 20, max_instances=4)
    ids = [O.ots_batch_add(b, x, tol=1e-7, max_iters=50000) for x in insts]
    assert O.ots_batch_run(b) == 0
    for x, i in zip(insts, ids):
        o = Oracle(x)
        ro = o.solve(max_iters=200000, tol=1e-12)
        st = O.ots_batch_status(b, i)
        if ro["status"] != 0 or st["status"] != 0:
            pytest.skip("time-varying draw made this instance capacity-infeasible")
        F = O.ots_batch_get_flows(b, i)
        assert rel_l1(F, o.flows()) <= FLOW_TOL
        t, s = closed_cells(x)
        assert np.all(F[t - 1, s] == 0.0)
    O.ots_batch_destroy(b)


def capacity_closed_cells(inst):
    t_idx, s_idx = np.nonzero(inst.state_capacity_t == 0.0)
    return t_idx + 2, s_idx


def with_capacities(inst, seed):
    return I.with_time_varying_capacities(inst, seed=seed, lo=0.8, hi=1.5, closures=1)


@pytest.mark.parametrize("L,seed,cseed", [(9, 31, 1), (300, 32, 2)])
def test_per_interval_capacities_single_instance(O, L, seed, cseed):
    inst = with_capacities(I.rgg_instance(seed=seed, n=50, L=L, T=12, eps=0.05, cap_lo=0.3, cap_hi=1.0), cseed)
    o = Oracle(inst)
    assert o.solve(max_iters=100000, tol=1e-11)["status"] == 0
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-7, max_iters=50000)
    assert r["status"] == 0
    F = O.ots_get_flows(h)
    assert rel_l1(F, o.flows()) <= FLOW_TOL
    t, s = capacity_closed_cells(inst)
    assert np.all(F[t - 1, s] == 0.0)
    # the dual objective of Theorem 3 (with d_t in its capacity term) at the two fixed points
    ref = o.dual_objective()
    assert abs(r["dual_objective"] - ref) <= 1e-6 * abs(ref)
    O.ots_destroy_problem(h)


def test_per_interval_capacities_and_costs_batched_and_served(O):
    """Batched kernel and the server (which copies the per-interval arrays at submission: the
    caller's arrays are overwritten right after submitting)."""
    insts = [with_capacities(I.rgg_instance(seed=200, n=45, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0), 3),
             with_capacities(I.rgg_instance(seed=202, n=40, L=30, T=8, eps=0.05, cap_lo=0.3, cap_hi=1.0), 4)]
    I.with_time_varying_costs(insts[1], seed=5, lo=0.9, hi=1.1)
    refs = []
    for x in insts:
        o = Oracle(x)
        assert o.solve(max_iters=200000, tol=1e-12)["status"] == 0
        refs.append(o.flows())
    b = O.ots_batch_create(pool_bytes=256 << 20, max_instances=4)
    ids = [O.ots_batch_add(b, x, tol=1e-7, max_iters=50000) for x in insts]
    assert O.ots_batch_run(b) == 0
    for x, i, ref in zip(insts, ids, refs):
        assert O.ots_batch_status(b, i)["status"] == 0
        F = O.ots_batch_get_flows(b, i)
        assert rel_l1(F, ref) <= FLOW_TOL
        t, s = capacity_closed_cells(x)
        assert np.all(F[t - 1, s] == 0.0)
    O.ots_batch_destroy(b)
    srv = O.ots_server_create(pool_bytes=256 << 20, max_instances=4)
    tickets = []
    for x in insts:
        tickets.append(O.ots_server_submit(srv, x, tol=1e-7))
    saved = [(x.state_capacity_t.copy(), None if x.state_cost_t is None else x.state_cost_t.copy()) for x in insts]
    for x in insts:                      # the server must not read the caller's arrays any more
        x.state_capacity_t[...] = np.nan
        if x.state_cost_t is not None:
            x.state_cost_t[...] = np.nan
    for tk, ref in zip(tickets, refs):
        assert O.ots_server_wait(srv, tk, 60000)["status"] == 0
        assert rel_l1(O.ots_server_get_flows(srv, tk), ref) <= FLOW_TOL
    O.ots_server_destroy(srv)
    for x, (dt, ct) in zip(insts, saved):
        x.state_capacity_t, x.state_cost_t = dt, ct

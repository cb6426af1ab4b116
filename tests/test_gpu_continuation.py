"""Continuation in epsilon (warm starts at larger epsilon, carried with lambda = -eps ln u):
the fixed point at the problem's epsilon is unique (the entropic objective is strictly
convex), so an annealed solve must end at the oracle's solution."""
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


@pytest.mark.parametrize("L,tv,seed", [(9, False, 5), (300, False, 4), (40, True, 4)])
def test_annealed_solve_reaches_the_oracle_fixed_point(O, L, tv, seed):
    inst = I.rgg_instance(seed=seed, n=60, L=L, T=14, eps=0.02, cap_lo=0.3, cap_hi=1.0)
    if tv:
        I.with_time_varying_costs(inst, seed=2, lo=0.7, hi=1.4, closures=1)
    o = Oracle(inst)
    ro = o.solve(max_iters=50000, tol=1e-12)
    assert ro["status"] == 0 and ro["iters"] < 50000
    h = O.ots_create_problem(inst)
    plain = O.ots_sinkhorn_solve(h, tol=1e-7, max_iters=100000)
    F0 = O.ots_get_flows(h)
    ann = O.ots_sinkhorn_solve(h, tol=1e-7, max_iters=100000, eps_start=8 * inst.eps, eps_stages=3)
    assert plain["status"] == 0 and ann["status"] == 0
    F1 = O.ots_get_flows(h)
    assert rel_l1(F1, o.flows()) <= FLOW_TOL
    assert rel_l1(F1, F0) <= FLOW_TOL
    # the problem is back at its own epsilon: more passes leave the converged duals alone
    r = O.ots_iterate(h, 3)
    assert r["src_residual"] <= 1e-6 and r["cap_violation"] <= 1e-6
    assert abs(r["dual_objective"] - o.dual_objective()) <= 1e-6 * abs(o.dual_objective())
    O.ots_destroy_problem(h)


def test_batched_continuation_reaches_the_oracle_fixed_point(O):
    """The batch halves epsilon per stage (eps 8x -> eps); the instances next to it run without
    continuation, and each result matches the oracle at its own epsilon."""
    insts = [I.rgg_instance(seed=5, n=60, L=9, T=14, eps=0.02, cap_lo=0.3, cap_hi=1.0),
             I.rgg_instance(seed=4, n=40, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0),
             I.rgg_instance(seed=11, n=90, L=40, T=13, eps=0.03, cap_lo=0.3, cap_hi=1.0)]
    refs = []
    for x in insts:
        o = Oracle(x)
        ro = o.solve(max_iters=100000, tol=1e-12)
        assert ro["status"] == 0 and ro["iters"] < 100000
        refs.append(o.flows())
    b = O.ots_batch_create(pool_bytes=256 << 20, max_instances=8)
    ids = [O.ots_batch_add(b, insts[0], tol=1e-8, eps_start=8 * insts[0].eps),
           O.ots_batch_add(b, insts[1], tol=1e-8),
           O.ots_batch_add(b, insts[2], tol=1e-8, eps_start=4 * insts[2].eps)]
    assert O.ots_batch_run(b) == 0
    for i, ref in zip(ids, refs):
        r = O.ots_batch_status(b, i)
        assert r["status"] == 0
        assert rel_l1(O.ots_batch_get_flows(b, i), ref) <= FLOW_TOL
    O.ots_batch_destroy(b)


def test_continuation_is_rejected_where_unsupported(O):
    import ctypes
    o = O.ots_default_solve_opts()
    o.eps_start = 0.2
    pc = I.rgg_instance(seed=4, n=40, L=3, T=9, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    pc.commodity_cost = np.ones((pc.L, pc.n_states))
    h = O.ots_create_problem(pc)
    code = O.load_library().ots_sinkhorn_solve(h.ptr, ctypes.byref(o), None)
    assert code == O.OTS_ERR_INVALID_ARG
    O.ots_destroy_problem(h)


def test_served_request_with_continuation(O):
    inst = I.rgg_instance(seed=11, n=90, L=40, T=13, eps=0.03, cap_lo=0.3, cap_hi=1.0)
    o = Oracle(inst)
    o.solve(max_iters=200000, tol=1e-12)
    s = O.ots_server_create(pool_bytes=256 << 20, max_instances=4)
    t = O.ots_server_submit(s, inst, tol=1e-7, eps_start=0.24, eps_stages=3)
    assert O.ots_server_wait(s, t, 60000)["status"] == 0
    assert rel_l1(O.ots_server_get_flows(s, t), o.flows()) <= FLOW_TOL
    O.ots_server_destroy(s)

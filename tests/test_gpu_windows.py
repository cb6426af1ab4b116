"""Per-commodity entry and exit times (the multi-tensor scheme of the Remark after
Algorithm 2) on the GPU, against the FP64 oracle: fixed points, per-commodity flows with the
marginals at each commodity's own times, iterate-by-iterate measures, and the server."""
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


def windowed(L, seed, wseed, slack, clo):
    inst = I.rgg_instance(seed=seed, n=60, L=L, T=14, eps=0.03, cap_lo=clo, cap_hi=3 * clo)
    return I.with_commodity_windows(inst, seed=wseed, slack=slack)


@pytest.mark.parametrize("L,seed,wseed,slack,clo", [(9, 5, 2, 2, 0.3), (9, 6, 1, 2, 0.3), (40, 4, 1, 1, 0.2),
                                                    (300, 4, 1, 1, 0.3)])
def test_windows_fixed_point(O, L, seed, wseed, slack, clo):
    inst = windowed(L, seed, wseed, slack, clo)
    o = Oracle(inst)
    ro = o.solve(max_iters=50000, tol=1e-12)
    assert ro["status"] == 0 and ro["iters"] < 50000
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=50000)
    assert r["status"] == 0
    assert rel_l1(O.ots_get_flows(h), o.flows()) <= FLOW_TOL
    l1 = min(L, 6)
    P = O.ots_get_commodity_flows(h, 1, inst.T + 1, 0, l1)
    assert rel_l1(P, o.projections(0, l1)) <= FLOW_TOL
    for l in range(l1):                                # nothing outside the window, marginals inside
        a, b = inst.commodity_t_in[l], inst.commodity_t_out[l]
        assert np.all(P[:a - 1, l] == 0.0) and np.all(P[b:, l] == 0.0)
        m = inst.src_mass[inst.src_comm == l].sum()
        assert abs(P[a - 1, l].sum() - m) <= 1e-6 * m and abs(P[b - 1, l].sum() - m) <= 1e-6 * m
    O.ots_destroy_problem(h)


def test_windows_iterates_and_default_windows(O):
    inst = windowed(9, 6, 1, 2, 0.3)
    o = Oracle(inst)
    o.backward_sweep()
    h = O.ots_create_problem(inst)
    done = 0
    for target in (1, 3):
        r = O.ots_iterate(h, target - done, reset=(done == 0))
        for _ in range(target - done):
            ro, co, _ = o.iteration()
        done = target
        assert abs(r["src_residual"] - ro) <= 1e-6 + 1e-4 * ro
        assert abs(r["cap_violation"] - co) <= 1e-6 + 1e-4 * co
        assert rel_l1(O.ots_get_flows(h), o.flows()) <= FLOW_TOL
        assert abs(r["dual_objective"] - o.dual_objective()) <= 1e-6 * abs(o.dual_objective())
    O.ots_destroy_problem(h)
    # windows covering 1..T are the plain problem, bitwise
    base = I.rgg_instance(seed=6, n=60, L=9, T=14, eps=0.03, cap_lo=0.3, cap_hi=0.9)
    h0 = O.ots_create_problem(base)
    r0 = O.ots_iterate(h0, 5, reset=True)
    base.commodity_t_in = np.ones(9, np.int32)
    base.commodity_t_out = np.full(9, 14, np.int32)
    h1 = O.ots_create_problem(base)
    r1 = O.ots_iterate(h1, 5, reset=True)
    assert r0["src_residual"] == r1["src_residual"] and r0["cap_violation"] == r1["cap_violation"]
    assert np.array_equal(O.ots_get_flows(h0), O.ots_get_flows(h1))


def test_windows_served_and_rejected_by_the_batch(O):
    inst = windowed(9, 5, 2, 2, 0.3)
    o = Oracle(inst)
    o.solve(max_iters=50000, tol=1e-12)
    s = O.ots_server_create(pool_bytes=128 << 20, max_instances=4)
    t = O.ots_server_submit(s, inst, tol=1e-8)
    assert O.ots_server_wait(s, t, 60000)["status"] == 0
    assert rel_l1(O.ots_server_get_flows(s, t), o.flows()) <= FLOW_TOL
    O.ots_server_destroy(s)
    b = O.ots_batch_create(pool_bytes=64 << 20, max_instances=2)
    with pytest.raises(O.OTSError) as e:
        O.ots_batch_add(b, inst)
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    O.ots_batch_destroy(b)

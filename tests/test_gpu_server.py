"""Serving (ots_server_*): continuous batching of a request stream, admission by memory, the
single-instance lane for wide instances, and results that are the same alone and in the mix.
"""
import time

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


def stream_of_requests():
    """Uneven feasible instances (same seeds as the batch tests)."""
    shapes = [(30, 1, 7, 100), (45, 3, 9, 200), (60, 7, 12, 102), (50, 13, 10, 103), (40, 30, 8, 202),
              (70, 61, 11, 105), (36, 120, 9, 106), (32, 200, 8, 107)]
    return [I.rgg_instance(seed=sd, n=n, L=L, T=T, eps=0.05, cap_lo=0.3, cap_hi=1.0) for n, L, T, sd in shapes]


def test_alone_and_in_the_mix_give_the_same_result(O):
    """A request's result is identical (bitwise) whether it is served alone or arrives while
    other requests are on the GPU, and matches the oracle."""
    target = I.rgg_instance(seed=11, n=90, L=40, T=13, eps=0.03, cap_lo=0.3, cap_hi=1.0)
    others = stream_of_requests()
    s = O.ots_server_create(pool_bytes=1 << 30, max_instances=16, ticks_per_launch=4)
    t0 = O.ots_server_submit(s, target, tol=1e-7)
    r0 = O.ots_server_wait(s, t0, 60000)
    F0 = O.ots_server_get_flows(s, t0)
    assert r0["status"] == 0
    # now the same request arrives in the middle of a stream, behind a request whose capacities
    # admit no feasible flow (it runs to its pass limit, so it is resident while the target runs)
    from tests.test_gpu_parity import capped_rgg
    blocker = O.ots_server_submit(s, capped_rgg(seed=17, L=5, T=12), tol=1e-9, max_iters=4000)
    tickets = [O.ots_server_submit(s, x, tol=1e-7) for x in others[:4]]
    time.sleep(0.002)
    t1 = O.ots_server_submit(s, target, tol=1e-7)
    tickets += [O.ots_server_submit(s, x, tol=1e-7) for x in others[4:]]
    most = 0
    while O.ots_server_poll(s, t1)["status"] == O.OTS_PENDING:
        most = max(most, O.ots_server_info(s)["resident"])
        time.sleep(0.0005)
    r1 = O.ots_server_wait(s, t1, 60000)
    assert most >= 2, "the target never shared the GPU with another request"
    for t in tickets:
        assert O.ots_server_wait(s, t, 60000)["status"] == 0
    assert O.ots_server_wait(s, blocker, 60000)["status"] == O.OTS_ERR_NOT_CONVERGED
    F1 = O.ots_server_get_flows(s, t1)
    assert r1["status"] == 0 and r1["iterations"] == r0["iterations"]
    assert np.array_equal(F0, F1)
    o = Oracle(target)
    o.solve(max_iters=200000, tol=1e-12)
    assert rel_l1(F1, o.flows()) <= FLOW_TOL
    for x, t in zip(others, tickets[:4] + tickets[4:]):
        ox = Oracle(x)
        ox.solve(max_iters=200000, tol=1e-12)
        assert rel_l1(O.ots_server_get_flows(s, t), ox.flows()) <= FLOW_TOL
    info = O.ots_server_info(s)
    assert info["completed"] + info["failed"] == 3 + len(others) and info["failed"] <= 1 and info["resident"] == 0
    O.ots_server_destroy(s)


def test_admission_by_memory_and_slots(O):
    """A pool that holds only a few instances at once and two slots: every request still
    completes (requests wait for memory and slots instead of failing)."""
    reqs = stream_of_requests()[:6]
    s = O.ots_server_create(pool_bytes=48 << 20, max_instances=2, ticks_per_launch=4)
    tickets = [O.ots_server_submit(s, x, tol=1e-7) for x in reqs]
    peak = 0
    while True:
        info = O.ots_server_info(s)
        peak = max(peak, info["resident"])
        assert info["pool_used"] <= info["pool_bytes"]
        if info["completed"] + info["failed"] == len(reqs):
            break
        time.sleep(0.001)
    assert peak <= 2
    for x, t in zip(reqs, tickets):
        r = O.ots_server_poll(s, t)
        assert r["status"] == 0
        tm = O.ots_server_timing(s, t)
        assert tm["total_ms"] >= tm["wait_ms"] >= 0.0
        ox = Oracle(x)
        ox.solve(max_iters=200000, tol=1e-12)
        assert rel_l1(O.ots_server_get_flows(s, t), ox.flows()) <= FLOW_TOL
        O.ots_server_release(s, t)
    # a request larger than the whole pool fails with OTS_ERR_OOM instead of waiting forever
    big = I.rgg_instance(seed=3, n=400, L=250, T=120, eps=0.05, cap_lo=2.0, cap_hi=6.0)   # ~75 MB
    t = O.ots_server_submit(s, big)
    assert O.ots_server_wait(s, t, 60000)["status"] == O.OTS_ERR_OOM
    O.ots_server_destroy(s)


def test_wide_requests_use_the_single_instance_lane(O):
    """L > 256 goes to the single-instance solver next to the batch; same fixed point."""
    wide = I.rgg_instance(seed=3, n=40, L=300, T=8, eps=0.1, cap_lo=2.0, cap_hi=6.0)
    small = stream_of_requests()[2]
    s = O.ots_server_create(pool_bytes=1 << 30, max_instances=8)
    tw = O.ots_server_submit(s, wide, tol=1e-6)
    ts = O.ots_server_submit(s, small, tol=1e-7)
    assert O.ots_server_wait(s, tw, 60000)["status"] == 0
    assert O.ots_server_wait(s, ts, 60000)["status"] == 0
    o = Oracle(wide)
    o.solve(max_iters=20000, tol=1e-10)
    assert rel_l1(O.ots_server_get_flows(s, tw), o.flows()) <= FLOW_TOL
    O.ots_server_destroy(s)


def test_plain_mode_and_failures(O):
    """mode 1 solves one request at a time with the single-instance solver (same results);
    invalid or infeasible requests finish with their error status."""
    reqs = stream_of_requests()[:3]
    plain = O.ots_server_create(mode=1)
    batched = O.ots_server_create(pool_bytes=256 << 20, max_instances=8)
    tp = [O.ots_server_submit(plain, x, tol=1e-7) for x in reqs]
    tb = [O.ots_server_submit(batched, x, tol=1e-7) for x in reqs]
    for a, b in zip(tp, tb):
        assert O.ots_server_wait(plain, a, 60000)["status"] == 0
        assert O.ots_server_wait(batched, b, 60000)["status"] == 0
        assert rel_l1(O.ots_server_get_flows(batched, b), O.ots_server_get_flows(plain, a)) <= 1e-6
    bad = I.grid_single_commodity(0)
    bad.snk_mass = bad.snk_mass * 2.0                      # unbalanced masses
    t = O.ots_server_submit(batched, bad)
    assert O.ots_server_wait(batched, t, 60000)["status"] == O.OTS_ERR_INVALID_ARG
    t = O.ots_server_submit(plain, bad)
    assert O.ots_server_wait(plain, t, 60000)["status"] == O.OTS_ERR_INVALID_ARG
    far = I.grid_single_commodity(0, T=3)                                # sinks out of reach in T-1 steps
    t = O.ots_server_submit(batched, far)
    assert O.ots_server_wait(batched, t, 60000)["status"] == O.OTS_ERR_INFEASIBLE
    O.ots_server_destroy(plain)
    O.ots_server_destroy(batched)

"""The oracle on the storage state models of Section 3.3 (explicit heads and tails, states that
may follow themselves): storage on edges and the traffic-routing model of eq.
cost_traffic_routing, in which nothing enters a source and nothing leaves a sink.  Pinned against
brute force over the full tensor with K built from the definition (tests/pins_math.py), the
fixed point of Proposition 5 on that tensor, and the properties the model fixes.  The CUDA solver
takes these models through the explicit state graph of its descriptor; its parity with this oracle
is tested on the GPU (tests/test_gpu_storage.py)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2106_14485_gb300 import instances as I
from tests import pins_math as PM


def tiny(edge_storage=False, seed=0, T=5, L=2, cap_lo=0.2, cap_hi=0.6, eps=0.3):
    return I.traffic_routing_instance(seed=seed, rows=1, cols=3, L=L, T=T, eps=eps, cap_lo=cap_lo, cap_hi=cap_hi,
                                      edge_storage=edge_storage)


def test_line_graph_counts_storage():
    for es in (False, True):
        inst = tiny(es)
        o = Oracle(inst)
        assert o.nnz == int(PM.dense_K(inst).sum()) == inst.nnz_line_graph()


@pytest.mark.parametrize("edge_storage", [False, True])
@pytest.mark.parametrize("T", [3, 4, 5])
def test_projections_match_brute_force(edge_storage, T):
    inst = tiny(edge_storage, seed=T, T=T)
    o = Oracle(inst)
    rng = np.random.default_rng(20 + T)
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


@pytest.mark.parametrize("edge_storage", [False, True])
def test_fixed_point_matches_tensor_sinkhorn(edge_storage):
    inst = tiny(edge_storage, seed=3, T=5, cap_lo=1.45, cap_hi=1.45)      # street 0 binds at t = 2, 3
    o = Oracle(inst)
    r = o.solve(max_iters=200000, tol=1e-13)
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


def test_traffic_model_properties():
    """Nothing enters a source and nothing leaves a sink: per commodity, the mass on its source
    never grows and the mass on its sink never shrinks; junctions hold nothing; streets carry at
    most their capacity; every P_t has the total mass."""
    inst = I.traffic_routing_instance(seed=4, rows=4, cols=4, L=3, T=9, eps=0.1)
    o = Oracle(inst)
    r = o.solve(max_iters=200000, tol=1e-12)
    assert r["status"] == 0 and r["src_resid"] < 1e-11 and r["cap_viol"] < 1e-11
    P = o.projections()                                           # [T, L, S]
    E, V = inst.n_edges, 16
    for l in range(inst.L):
        s_src, s_snk = inst.src_state[l], inst.snk_state[l]
        src = P[:, l, s_src]
        snk = P[:, l, s_snk]
        assert np.all(np.diff(src) <= 1e-12) and np.all(np.diff(snk) >= -1e-12)
        assert src[0] == pytest.approx(inst.src_mass[l], rel=1e-11)
        assert snk[-1] == pytest.approx(inst.snk_mass[l], rel=1e-11)
        others = np.setdiff1d(np.arange(E, inst.n_states), [s_src, s_snk])
        assert np.all(P[:, l, others] == 0.0)                     # other commodities' and junction states
    F = P.sum(1)
    np.testing.assert_allclose(F.sum(1), inst.src_mass.sum(), rtol=1e-11)
    assert np.all(F[1:-1, :E] <= inst.edge_cap[None, :] * (1 + 1e-9))
    assert np.all(F[:, E:E + V] == 0.0)


def test_storage_on_a_wait_loop_changes_nothing():
    """A wait loop already follows itself (head == tail): marking it as storage leaves K, and
    every result, as they are; the explicit graph equal to the default one gives the same bits."""
    inst = I.rgg_instance(seed=3, n=30, L=3, T=8, eps=0.1, cap_lo=1.0, cap_hi=2.0)
    o0 = Oracle(inst)
    o0.solve(max_iters=2000, tol=1e-12)
    F0 = o0.flows()
    tail, head = inst.state_tail_head()
    for hold in (None, np.concatenate([np.zeros(inst.n_edges), np.ones(inst.n_nodes)]).astype(np.int32)):
        x = I.Instance(**{**inst.__dict__})
        x.state_tail, x.state_head, x.state_hold = tail.copy(), head.copy(), hold
        o = Oracle(x)
        o.solve(max_iters=2000, tol=1e-12)
        assert o.nnz == o0.nnz
        assert np.array_equal(o.flows(), F0)


def test_cuda_binding_passes_the_state_graph_through():
    """The binding hands tail, head and storage flag of every state to the library, whose host
    checks accept the model (the device path is checked against the oracle on the GPU)."""
    from paper_2106_14485_gb300 import ots
    inst = tiny()
    d, arr = ots._problem_desc(inst)
    assert np.array_equal(arr["state_tail"], inst.state_tail) and np.array_equal(arr["state_head"], inst.state_head)
    assert np.array_equal(arr["state_hold"], inst.state_hold)
    ots.load_library()
    ots.ots_check_problem(inst)

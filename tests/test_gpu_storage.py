"""Storage states on the GPU (Section 3.3): storage on edges, and the source / sink states of the
traffic-routing model (eq. cost_traffic_routing), given as an explicit state graph.  A storage
state owns one message row of its own (K = B_in B_out + D, D diagonal over those states); its
capacity update runs before each forward step.  Parity with the FP64 oracle, which builds K from
the same definition state by state: iterates after 1 and 3 passes (flows and both measures), the
fixed point (aggregate and per-commodity flows, entry by entry), and the served path."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2106_14485_gb300 import instances as I

pytestmark = pytest.mark.gpu


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


def elementwise(F, Fref):
    return float((np.abs(F - Fref) / (1e-5 * np.abs(Fref) + 1e-9 * np.abs(Fref).max())).max())


def road_with_edge_storage(seed, L, T=12, n=40, frac=0.3):
    """A random geometric road graph with wait loops, where a random share of the edges may also
    hold flow from one interval to the next (storage on edges)."""
    inst = I.rgg_instance(seed=seed, n=n, L=L, T=T, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    rng = np.random.default_rng(seed + 100)
    V, E = inst.n_nodes, len(inst.edge_src)
    inst.state_tail = np.concatenate([inst.edge_src, np.arange(V)]).astype(np.int32)
    inst.state_head = np.concatenate([inst.edge_dst, np.arange(V)]).astype(np.int32)
    inst.state_hold = np.concatenate([(rng.random(E) < frac).astype(np.int32), np.ones(V, np.int32)])
    return inst


CASES = {
    "traffic routing": lambda: I.traffic_routing_instance(seed=1, rows=4, cols=4, L=3, T=9, eps=0.1),
    "traffic routing, storage on streets": lambda: I.traffic_routing_instance(seed=2, rows=4, cols=5, L=4, T=10,
                                                                               eps=0.1, edge_storage=True),
    "road, storage on edges, L=6": lambda: road_with_edge_storage(3, 6),
    "road, storage on edges, L=300": lambda: road_with_edge_storage(4, 300, T=9),
}


@pytest.mark.parametrize("name", list(CASES))
def test_storage_iterates_and_fixed_point(O, name):
    inst = CASES[name]()
    o = Oracle(inst)
    o.backward_sweep()
    h = O.ots_create_problem(inst)
    done = 0
    for target in (1, 3):
        r = O.ots_iterate(h, target - done, reset=(done == 0))
        for _ in range(target - done):
            ro, co, _ = o.iteration()
        done = target
        assert rel_l1(O.ots_get_flows(h), o.flows()) <= 1e-5, (name, target)
        assert abs(r["src_residual"] - ro) <= 1e-6 + 1e-4 * ro, (name, target, r["src_residual"], ro)
        assert abs(r["cap_violation"] - co) <= 1e-6 + 1e-4 * co, (name, target, r["cap_violation"], co)
    r = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=50000, warm_start=True)
    assert r["status"] == 0, r
    o2 = Oracle(inst)
    ro = o2.solve(max_iters=200000, tol=1e-12)
    assert ro["status"] == 0
    F, Fref = O.ots_get_flows(h), o2.flows()
    assert rel_l1(F, Fref) <= 1e-5 and elementwise(F, Fref) <= 1.0, (name, rel_l1(F, Fref), elementwise(F, Fref))
    l1 = min(inst.L, 4)
    P, Pref = O.ots_get_commodity_flows(h, 1, inst.T + 1, 0, l1), o2.projections(0, l1)
    assert rel_l1(P, Pref) <= 1e-5 and elementwise(P, Pref) <= 1.0, name
    if "traffic" in name:
        # the model's own properties: nothing enters a source, nothing leaves a sink, so a source
        # only loses mass over time and a sink only gains it
        src = F[:, inst.src_state]
        snk = F[:, inst.snk_state]
        assert np.all(np.diff(src, axis=0) <= 1e-9) and np.all(np.diff(snk, axis=0) >= -1e-9)
    O.ots_destroy_problem(h)


def test_storage_served_and_refused_by_the_batch(O):
    inst = CASES["traffic routing, storage on streets"]()
    o = Oracle(inst)
    assert o.solve(max_iters=200000, tol=1e-12)["status"] == 0
    srv = O.ots_server_create(pool_bytes=256 << 20, max_instances=4)
    tk = O.ots_server_submit(srv, inst, tol=1e-8)
    r = O.ots_server_wait(srv, tk, 60000.0)
    assert r["status"] == 0, r
    assert rel_l1(O.ots_server_get_flows(srv, tk), o.flows()) <= 1e-5
    O.ots_server_destroy(srv)
    b = O.ots_batch_create(pool_bytes=64 << 20, max_instances=2)
    with pytest.raises(O.OTSError) as e:
        O.ots_batch_add(b, inst)
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    O.ots_batch_destroy(b)

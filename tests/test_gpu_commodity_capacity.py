"""Commodity-dependent capacities D^(0,t) (Section 3.3, one D for every t) on the GPU's
per-commodity kernels, against the FP64 oracle: fixed points, per-commodity flows within D,
iterate-by-iterate measures, and the reductions D = inf and batch rejection."""
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


def with_D(inst, seed=1, lo=0.2, hi=0.6):
    rng = np.random.default_rng(seed)
    D = np.full((inst.L, inst.n_states), np.inf)
    D[:, :inst.n_edges] = rng.uniform(lo, hi, (inst.L, inst.n_edges)) * inst.src_mass[:, None]
    inst.commodity_capacity = D
    return inst


def base(seed):
    return I.rgg_instance(seed=seed, n=60, L=9, T=14, eps=0.03, cap_lo=0.5, cap_hi=1.5)


@pytest.mark.parametrize("seed,per_commodity_costs", [(5, False), (6, False), (5, True)])
def test_commodity_capacities_fixed_point(O, seed, per_commodity_costs):
    inst = with_D(base(seed))
    if per_commodity_costs:
        rng = np.random.default_rng(3)
        c = np.concatenate([inst.edge_cost, inst.wait_cost])
        inst.commodity_cost = c[None, :] * rng.uniform(0.8, 1.25, (inst.L, inst.n_states))
    o = Oracle(inst)
    ro = o.solve(max_iters=50000, tol=1e-12)
    assert ro["status"] == 0 and ro["iters"] < 50000
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=50000)
    assert r["status"] == 0
    assert rel_l1(O.ots_get_flows(h), o.flows()) <= FLOW_TOL
    P = O.ots_get_commodity_flows(h)
    assert rel_l1(P, o.projections()) <= FLOW_TOL
    D = inst.commodity_capacity
    for t in range(2, inst.T):
        assert np.all(P[t - 1] <= D * (1 + 1e-5) + 1e-9)
    O.ots_destroy_problem(h)


def test_commodity_capacities_iterates(O):
    inst = with_D(base(6))
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
    O.ots_destroy_problem(h)


def test_infinite_commodity_capacities_change_nothing(O):
    inst = base(5)
    h0 = O.ots_create_problem(inst)
    O.ots_sinkhorn_solve(h0, tol=1e-8)
    F0 = O.ots_get_flows(h0)
    inst.commodity_capacity = np.full((inst.L, inst.n_states), np.inf)
    h1 = O.ots_create_problem(inst)
    O.ots_sinkhorn_solve(h1, tol=1e-8)
    assert rel_l1(O.ots_get_flows(h1), F0) <= 1e-6
    b = O.ots_batch_create(pool_bytes=64 << 20, max_instances=2)
    with pytest.raises(O.OTSError) as e:
        O.ots_batch_add(b, inst)
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    O.ots_batch_destroy(b)

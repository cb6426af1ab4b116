"""Pins of the single-commodity oracle (Algorithm 1, Section 4.2, linear domain, FP64): it is
checked against the multi-commodity oracle with L = 1 (Algorithm 2 in log domain, a different
recursion and arithmetic), the full tensor on a tiny instance, the two-marginal reduction of
the uncapacitated problem, the KKT conditions, and the boundary reading (k_1, k_T)."""
import numpy as np
import pytest

from tests import pins_math as PM
from oracle.oracle import Oracle
from oracle.single_commodity import cyclic_projections
from paper_2106_14485_gb300 import instances as I


def alg1_inputs(inst, k1=None, kT=None):
    S, T = inst.n_states, inst.T
    K = PM.dense_K(inst)
    c = np.concatenate([inst.edge_cost, inst.wait_cost]).astype(np.float64)
    k = np.tile(np.exp(-c / inst.eps), (T + 1, 1))
    if k1 is not None:
        k[1] = k1
    if kT is not None:
        k[T] = kT
    mu1 = np.zeros(S)
    np.add.at(mu1, inst.src_state, inst.src_mass)
    muT = np.zeros(S)
    np.add.at(muT, inst.snk_state, inst.snk_mass)
    d = np.full((T + 1, S), np.inf)
    for t in range(2, T):
        d[t] = PM.capacity_at(inst, t)
    return K, k, mu1, muT, d


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_algorithm1_matches_the_multicommodity_oracle(seed):
    inst = I.single_commodity_instance(seed=seed)
    u, P, it, src, cap = cyclic_projections(*alg1_inputs(inst))
    assert src < 1e-12 and cap < 1e-12
    o = Oracle(inst)
    r = o.solve(max_iters=100000, tol=1e-13)
    assert r["status"] == 0 and r["iters"] < 100000
    np.testing.assert_allclose(P[1:], o.flows(), rtol=1e-10, atol=1e-13)
    lu, _, _ = o.get_duals()
    assert (lu < -1e-6).sum() > 0                     # capacities bind somewhere


def test_algorithm1_matches_the_full_tensor():
    inst = I.single_commodity_instance(seed=4, rows=2, cols=2, T=4, eps=0.5, n_src=2, n_snk=2, cap_scale=0.3)
    u, P, it, src, cap = cyclic_projections(*alg1_inputs(inst))
    tz, M, _ = PM.tensor_sinkhorn(inst)
    for t in range(1, inst.T + 1):
        np.testing.assert_allclose(P[t], tz.proj0t(M, t)[0], rtol=1e-7, atol=1e-10)


def test_uncapacitated_algorithm1_is_two_marginal_ot():
    inst = I.single_commodity_instance(seed=4, rows=3, cols=3, T=6, eps=0.4, per_interval=False, cap_scale=np.inf)
    inst.edge_cap = np.full_like(inst.edge_cap, np.inf)
    u, P, it, src, cap = cyclic_projections(*alg1_inputs(inst))
    np.testing.assert_allclose(P[1:], PM.two_marginal_flows(inst), rtol=1e-9, atol=1e-12)


def test_kkt_at_the_fixed_point():
    inst = I.single_commodity_instance(seed=5)
    K, k, mu1, muT, d = alg1_inputs(inst)
    u, P, it, src, cap = cyclic_projections(K, k, mu1, muT, d)
    np.testing.assert_allclose(P[1], mu1, atol=1e-12)
    np.testing.assert_allclose(P[inst.T], muT, atol=1e-12)
    for t in range(2, inst.T):
        assert np.all(P[t] <= d[t] + 1e-12)
        act = u[t] < 1 - 1e-9
        np.testing.assert_allclose(P[t][act], d[t][act], rtol=1e-9)


def test_boundary_costs_do_not_change_the_flows_and_need_the_reading():
    """M does not depend on k_1 and k_T (the fixed marginals absorb them); the boundary updates
    as printed in Algorithm 1 (without k_1, k_T) miss the marginals when k_1, k_T != 1."""
    inst = I.single_commodity_instance(seed=6)
    rng = np.random.default_rng(0)
    S = inst.n_states
    base = cyclic_projections(*alg1_inputs(inst))[1]
    k1, kT = rng.uniform(0.2, 3.0, S), rng.uniform(0.2, 3.0, S)
    P = cyclic_projections(*alg1_inputs(inst, k1, kT))[1]
    np.testing.assert_allclose(P, base, rtol=1e-9, atol=1e-13)
    K, k, mu1, muT, d = alg1_inputs(inst, k1, kT)
    u, P_lit, it, src, cap = cyclic_projections(K, k, mu1, muT, d, iters=200, literal_boundary=True)
    assert np.abs(P_lit[1] - mu1).sum() > 1e-3

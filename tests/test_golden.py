"""Stored expected values (tests/golden/): the oracle reproduces them, and they satisfy on their
own what the paper fixes for the optimum: equal mass at every t (Corollary 7: every P_t is a
marginal of the same M), flow conservation at every node between consecutive intervals (a
state i at t can only be followed at t+1 by a state leaving head(i); Section 3.1), and the
capacities P_t <= d for t = 2..T-1 (eq. multicommodity_reg)."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden as G                                   # noqa: E402

from paper_2106_14485_gb300 import instances as I         # noqa: E402,F401


def tail_head(inst):
    E = inst.edge_src.shape[0]
    v = np.arange(inst.n_nodes)
    return (np.concatenate([inst.edge_src, v]).astype(int), np.concatenate([inst.edge_dst, v]).astype(int))


@pytest.mark.parametrize("name", sorted(G.CASES))
def test_stored_flows_satisfy_the_constraints(name):
    inst = G.CASES[name][0]()
    F, _ = G.load(name)
    T, S = F.shape
    assert T == inst.T and S == inst.n_states
    mass = inst.src_mass.sum()
    np.testing.assert_allclose(F.sum(axis=1), mass, rtol=1e-11)
    assert np.isclose(inst.snk_mass.sum(), mass)
    tail, head = tail_head(inst)
    for t in range(T - 1):
        into = np.bincount(head, weights=F[t], minlength=inst.n_nodes)
        out = np.bincount(tail, weights=F[t + 1], minlength=inst.n_nodes)
        np.testing.assert_allclose(into, out, atol=1e-12 * mass)
    d = np.concatenate([inst.edge_cap, inst.wait_cap])
    assert (F[1:-1] <= d[None, :] * (1 + 1e-11) + 1e-14).all()
    assert (F >= 0).all()


@pytest.mark.parametrize("name", sorted(G.CASES))
def test_oracle_reproduces_the_stored_values(name):
    _, _, F, dual = G.solve(name)
    Fs, dual_s = G.load(name)
    assert np.abs(F - Fs).sum() <= 1e-10 * np.abs(Fs).sum()
    assert dual == pytest.approx(dual_s, rel=1e-11)


def test_capacities_bind_in_the_capacitated_case():
    inst = G.CASES["rgg30_L4_capped"][0]()
    F, _ = G.load("rgg30_L4_capped")
    d = np.concatenate([inst.edge_cap, inst.wait_cap])
    tight = np.isclose(F[1:-1], d[None, :], rtol=1e-9)
    assert tight.sum() >= 10

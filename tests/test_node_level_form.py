"""The node-level form of the messages is an exact rewriting of Theorem 6.

K_ij = [head(i) = tail(j)] factors through the nodes, so the forward message of a state depends on
the state only through its tail node and the backward message only through its head node; the
GPU kernels keep one row per node (A_t[v], B_t[v]) instead of one per state.  With storage states
(K_jj = 1, Section 3.3) a storage state needs a row of its own on top.  Here both forms are written
out in FP64 numpy (natural logs) from those definitions and compared with the oracle's state-level
messages (eq. psi_hat, eq. psi) at random duals."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2106_14485_gb300 import instances as I
from tests import pins_math as PM


def lse(a, axis=0):
    m = np.max(a, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    with np.errstate(divide="ignore"):
        return np.squeeze(m, axis) + np.log(np.sum(np.exp(a - m), axis=axis))


def node_lse(vals, node, V):
    """[L, S] values -> [L, V]: log-sum-exp over the states whose node is v (-1: none)."""
    out = np.full((vals.shape[0], V), -np.inf)
    for v in range(V):
        sel = node == v
        if sel.any():
            out[:, v] = lse(vals[:, sel], axis=1)
    return out


def node_level_messages(inst, logu, logU01, logU0T):
    """hatPsi_t (t = 2..T) and Psi_t (t = 1..T-1) of every state from node rows plus storage rows."""
    tail, head = PM.tail_head(inst)
    tail, head = np.asarray(tail), np.asarray(head)
    hold = np.asarray(getattr(inst, "state_hold", None) if getattr(inst, "state_hold", None) is not None
                      else np.zeros(len(tail)), bool)
    own = hold & ~((head >= 0) & (head == tail))              # storage rows beyond the node rows
    L, T, V, S = inst.L, inst.T, inst.n_nodes, len(tail)
    logKL = -PM.cost_matrix(inst) / inst.eps                  # [L, S]
    w = {t: logKL + logu[t - 2][None, :] for t in range(2, T)}

    def from_node(rows, node):
        out = np.full((L, S), -np.inf)
        ok = node >= 0
        out[:, ok] = rows[:, node[ok]]
        return out

    # forward: x_t = hatPsi_t; node row A[v] = LSE over states entering v of (x_t + w_t)
    hat = {}
    A = node_lse(logU01, head, V)                              # A_1 = U01 summed into the head nodes
    x = from_node(A, tail)
    x[:, own] = np.logaddexp(x[:, own], logU01[:, own])        # a storage state may start where it is
    hat[2] = x
    for t in range(2, T):
        y = hat[t] + w[t]
        A = node_lse(y, head, V)
        x = from_node(A, tail)
        x[:, own] = np.logaddexp(x[:, own], y[:, own])
        hat[t + 1] = x
    # backward: z_t = Psi_t; node row B[v] = LSE over states leaving v of (z_t + w_t)
    psi = {}
    B = node_lse(logU0T, tail, V)
    z = from_node(B, head)
    z[:, own] = np.logaddexp(z[:, own], logU0T[:, own])
    psi[T - 1] = z
    for t in range(T - 1, 1, -1):
        y = psi[t] + w[t]
        B = node_lse(y, tail, V)
        z = from_node(B, head)
        z[:, own] = np.logaddexp(z[:, own], y[:, own])
        psi[t - 1] = z
    return hat, psi


CASES = {
    "wait loops (the GPU's model)": lambda: I.rgg_instance(seed=3, n=30, L=3, T=8, eps=0.1),
    "traffic routing (source and sink storage)": lambda: I.traffic_routing_instance(seed=1, rows=3, cols=3, L=3, T=8),
    "traffic routing with storage on edges": lambda: I.traffic_routing_instance(seed=2, rows=3, cols=3, L=3, T=8,
                                                                                edge_storage=True),
}


@pytest.mark.parametrize("name", list(CASES))
def test_node_rows_reproduce_the_state_level_messages(name):
    inst = CASES[name]()
    o = Oracle(inst)
    rng = np.random.default_rng(5)
    S, L, T = inst.n_states, inst.L, inst.T
    R01, R0T = PM.dense_marginals(inst)
    logu = -rng.uniform(0, 2, (T - 2, S))
    U01 = np.where(R01 > 0, rng.uniform(-2, 2, (L, S)), -np.inf)
    U0T = np.where(R0T > 0, rng.uniform(-2, 2, (L, S)), -np.inf)
    o.set_duals(logu, np.where(R01 > 0, U01, 0.0), np.where(R0T > 0, U0T, 0.0))
    h, b = o.messages()                                        # natural logs: h[t-2] = hatPsi_t, b[t-1] = Psi_t
    hat, psi = node_level_messages(inst, logu, U01, U0T)
    for t in range(2, T + 1):
        fin = np.isfinite(h[t - 2])
        assert np.array_equal(fin, np.isfinite(hat[t])), t
        np.testing.assert_allclose(hat[t][fin], h[t - 2][fin], rtol=1e-12, atol=1e-9)
    for t in range(1, T):
        fin = np.isfinite(b[t - 1])
        assert np.array_equal(fin, np.isfinite(psi[t])), t
        np.testing.assert_allclose(psi[t][fin], b[t - 1][fin], rtol=1e-12, atol=1e-9)

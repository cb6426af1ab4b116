"""The seeded input generators (host only): the single-commodity family drawn with the uneven
batch's sizes is the same whether drawn in one process or in a spawn pool, stays within its
recipe, and every member passes the library's host-side checks (graph, masses, reachability)."""
import numpy as np
import pytest

from paper_2106_14485_gb300 import instances as I


def _same(a, b):
    for k in ("edge_src", "edge_dst", "edge_cost", "edge_cap", "wait_cost", "src_state", "src_mass", "snk_state",
              "snk_mass"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k), err_msg=k)
    assert (a.n_nodes, a.T, a.L, a.eps) == (b.n_nodes, b.T, b.L, b.eps)


def _connected(inst):
    adj = [[] for _ in range(inst.n_nodes)]
    for s, d in zip(inst.edge_src, inst.edge_dst):
        adj[s].append(d)
        adj[d].append(s)
    seen, stack = {0}, [0]
    while stack:
        v = stack.pop()
        for w in adj[v]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == inst.n_nodes


def test_uneven_single_batch_recipe_and_determinism():
    serial = I.uneven_single_batch(0, count=4, workers=1)
    pooled = I.uneven_single_batch(0, count=4, workers=2)
    for a, b in zip(serial, pooled):
        _same(a, b)
    for x in serial:
        assert x.L == 1 and 50 <= x.n_nodes <= 2000 and 10 <= x.T <= 80 and x.eps == 0.01
        assert _connected(x)
        m = float(np.sum(x.src_mass))
        assert 0.5 <= m <= 2.0
        cap = x.edge_cap
        assert np.all(cap >= 0.2 * m / 2 - 1e-12) and np.all(cap <= 1.0 * m / 2 + 1e-12)


def test_single_commodity_members_pass_the_host_checks():
    ots = pytest.importorskip("paper_2106_14485_gb300.ots")
    from paper_2106_14485_gb300 import build
    build.build()
    ots.load_library()
    for x in I.uneven_single_batch(1, count=3, workers=1) + [I.grid_single_commodity(0)]:
        ots.ots_check_problem(x)

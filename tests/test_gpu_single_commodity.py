"""The single-commodity problem (eq. singlecommodity_reg) on the GPU as L = 1 (one thread per
node row), against the Algorithm 1 oracle: single-instance, batched and continuation paths."""
import numpy as np
import pytest

from oracle.single_commodity import cyclic_projections
from paper_2106_14485_gb300 import instances as I
from tests.test_single_commodity_pins import alg1_inputs

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


@pytest.mark.parametrize("seed,rows,T", [(0, 6, 12), (1, 6, 12), (2, 16, 30)])
def test_single_commodity_matches_algorithm1(O, seed, rows, T):
    inst = I.single_commodity_instance(seed=seed, rows=rows, cols=rows, T=T)
    u, P, it, src, cap = cyclic_projections(*alg1_inputs(inst))
    assert src < 1e-12 and cap < 1e-12
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=100000)
    assert r["status"] == 0
    assert rel_l1(O.ots_get_flows(h), P[1:]) <= FLOW_TOL
    r = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=100000, eps_start=4 * inst.eps, eps_stages=2)
    assert r["status"] == 0
    assert rel_l1(O.ots_get_flows(h), P[1:]) <= FLOW_TOL
    O.ots_destroy_problem(h)


def test_single_commodity_batched(O):
    insts = [I.single_commodity_instance(seed=s, rows=5 + s, cols=6, T=10 + s) for s in range(4)]
    refs = [cyclic_projections(*alg1_inputs(x))[1][1:] for x in insts]
    b = O.ots_batch_create(pool_bytes=128 << 20, max_instances=8)
    ids = [O.ots_batch_add(b, x, tol=1e-8, max_iters=100000) for x in insts]
    assert O.ots_batch_run(b) == 0
    for i, ref in zip(ids, refs):
        assert O.ots_batch_status(b, i)["status"] == 0
        assert rel_l1(O.ots_batch_get_flows(b, i), ref) <= FLOW_TOL
    O.ots_batch_destroy(b)

"""Backward messages kept every k-th t and recomputed in between (f4, horizon scaling): the
recomputed panels are the same computation on the same inputs, so every result is bitwise the
one of the full storage, on less device memory."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("L", [9, 300])
def test_kept_every_k_is_bitwise_the_full_storage(O, L):
    inst = I.rgg_instance(seed=4, n=60, L=L, T=17, eps=0.02, cap_lo=0.3, cap_hi=1.0)
    ref = None
    for k in (0, 2, 3, 7, 40):
        h = O.ots_create_problem(inst, psi_stride=k)
        r = O.ots_iterate(h, 25, reset=True)
        F = O.ots_get_flows(h)
        P = O.ots_get_commodity_flows(h, 1, inst.T + 1, 0, min(L, 5))
        lu, U01, U0T = O.ots_get_duals(h)
        info = O.ots_problem_info(h)
        out = (r["src_residual"], r["cap_violation"], r["dual_objective"], F, P, lu, U01, U0T)
        if ref is None:
            ref, full_bytes = out, info["device_bytes"]
        else:
            assert out[:3] == ref[:3], k
            for a, b in zip(out[3:], ref[3:]):
                assert np.array_equal(a, b), k
            if 1 < k < inst.T - 3:
                assert info["device_bytes"] < full_bytes
        O.ots_destroy_problem(h)


def test_kept_every_k_solves_and_continues(O):
    inst = I.rgg_instance(seed=5, n=60, L=9, T=14, eps=0.02, cap_lo=0.3, cap_hi=1.0)
    h0 = O.ots_create_problem(inst)
    h1 = O.ots_create_problem(inst, psi_stride=4)
    r0 = O.ots_sinkhorn_solve(h0, tol=1e-8, eps_start=0.16, eps_stages=3)
    r1 = O.ots_sinkhorn_solve(h1, tol=1e-8, eps_start=0.16, eps_stages=3)
    assert r0["status"] == 0 and r1["iterations"] == r0["iterations"]
    assert np.array_equal(O.ots_get_flows(h0), O.ots_get_flows(h1))
    assert np.array_equal(O.ots_get_commodity_flows_noalloc(h0), O.ots_get_commodity_flows_noalloc(h1))
    O.ots_destroy_problem(h0)
    O.ots_destroy_problem(h1)


@pytest.mark.parametrize("L,k", [(9, 3), (300, 5)])
def test_kept_every_k_against_the_oracle(O, L, k):
    """Recomputed segments (stride k >= 3, horizon 24) against the FP64 oracle, not only against the
    GPU's own full storage: iterates after 1 and 4 passes (flows and both measures) and the
    converged flows, relative L1 <= 1e-5 and entry by entry."""
    from oracle.oracle import Oracle
    from tests.test_gpu_parity import assert_elementwise, rel_l1
    inst = I.rgg_instance(seed=6, n=60, L=L, T=24, eps=0.03, cap_lo=0.3, cap_hi=1.0)
    o = Oracle(inst)
    o.backward_sweep()
    h = O.ots_create_problem(inst, psi_stride=k)
    done = 0
    for target in (1, 4):
        r = O.ots_iterate(h, target - done, reset=(done == 0))
        for _ in range(target - done):
            ro, co, _ = o.iteration()
        done = target
        assert rel_l1(O.ots_get_flows(h), o.flows()) <= 1e-5, target
        assert abs(r["src_residual"] - ro) <= 1e-6 + 1e-4 * ro
        assert abs(r["cap_violation"] - co) <= 1e-6 + 1e-4 * co
    r = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=20000, warm_start=True)
    assert r["status"] == 0
    o2 = Oracle(inst)
    assert o2.solve(max_iters=100000, tol=1e-11)["status"] == 0
    F, Fref = O.ots_get_flows(h), o2.flows()
    assert rel_l1(F, Fref) <= 1e-5
    assert_elementwise(F, Fref, f"psi_stride {k}")
    O.ots_destroy_problem(h)

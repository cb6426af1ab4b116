"""The allocation-free flow query (ots_get_commodity_flows_noalloc).

It serves callers that cannot allocate device memory while they read results, such as a
real-time loop between solver passes or an application with a fixed memory budget.  It must
return the same per-commodity flows as ots_get_commodity_flows, call after call, although
its scratch space is one static device array shared by every call.  This file is collected
last so that a failure here never hides the other GPU tests.
"""
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


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def test_noalloc_flows_match_the_allocating_query_twice(O):
    inst = I.rgg_instance(seed=13, n=60, L=8, T=16, eps=0.05, cap_lo=0.15, cap_hi=0.4)
    h = O.ots_create_problem(inst)
    O.ots_iterate(h, 6, reset=True)
    for _ in range(2):   # two calls in a row: the shared array keeps the previous call's data
        ref = O.ots_get_commodity_flows(h, 1, inst.T + 1, 2, 7)
        got = O.ots_get_commodity_flows_noalloc(h, 1, inst.T + 1, 2, 7)
        assert got.shape == ref.shape
        assert rel_l1(got, ref) <= 1e-12
        O.ots_iterate(h, 1)
    # a different, smaller slice after a larger one: stale entries must not leak through
    ref = O.ots_get_commodity_flows(h, 1, 4, 0, 1)
    got = O.ots_get_commodity_flows_noalloc(h, 1, 4, 0, 1)
    assert rel_l1(got, ref) <= 1e-12
    O.ots_destroy_problem(h)


def test_noalloc_rejects_requests_beyond_the_static_buffer(O):
    inst = I.grid_traffic_instance(seed=3, rows=60, cols=60, L=128, T=8, eps=0.05)
    h = O.ots_create_problem(inst)
    O.ots_iterate(h, 1, reset=True)
    assert inst.n_states * inst.L > (1 << 20)
    with pytest.raises(O.OTSError) as e:
        O.ots_get_commodity_flows_noalloc(h, 2, 3, 0, inst.L)
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    # within the limit it still works
    lmax = (1 << 20) // inst.n_states
    ref = O.ots_get_commodity_flows(h, 2, 3, 0, lmax)
    got = O.ots_get_commodity_flows_noalloc(h, 2, 3, 0, lmax)
    assert rel_l1(got, ref) <= 1e-12
    O.ots_destroy_problem(h)


def test_noalloc_with_kept_panels_and_refusal_of_windows(O):
    """Backward panels kept every 3rd t (the query recomputes the others segment by segment in
    its problem's own memory): exactly the allocating query's values, which run the same
    kernels.  Commodity windows are refused with OTS_ERR_INVALID_ARG before any device work."""
    inst = I.rgg_instance(seed=14, n=60, L=8, T=16, eps=0.05, cap_lo=0.15, cap_hi=0.4)
    h = O.ots_create_problem(inst, psi_stride=3)
    O.ots_iterate(h, 5, reset=True)
    for _ in range(2):
        ref = O.ots_get_commodity_flows(h, 1, inst.T + 1, 1, 8)
        got = O.ots_get_commodity_flows_noalloc(h, 1, inst.T + 1, 1, 8)
        assert np.array_equal(got, ref)
    O.ots_destroy_problem(h)
    win = I.with_commodity_windows(I.rgg_instance(seed=5, n=60, L=9, T=14, eps=0.03, cap_lo=0.3, cap_hi=0.9),
                                   seed=2, slack=2)
    h = O.ots_create_problem(win)
    O.ots_iterate(h, 1, reset=True)
    with pytest.raises(O.OTSError) as e:
        O.ots_get_commodity_flows_noalloc(h, 1, win.T + 1, 0, 2)
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    O.ots_destroy_problem(h)

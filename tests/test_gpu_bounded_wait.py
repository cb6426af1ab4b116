"""The bounded device-side waits of the pipelined step kernels give up with a status instead of
hanging.  A test switch (ots_set_wait_limit) makes the consumers of every block withhold their
first shared-memory stage: the producer's next wait for that stage runs out, it stops issuing
copies, and the consumers' next wait for data runs out too.  Every copy that was issued had
been waited for, so none is in flight when the kernel returns.  With a short limit (2000 tries
of at most 2 us) the failing pass takes milliseconds; the process and the problem stay usable,
and the next passes match those of a fresh problem bit for bit."""
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


def test_withheld_stage_makes_the_waits_give_up(O):
    # rows of 512 commodities: the pipelined kernels; 2500 nodes: several work items per block
    inst = I.grid_traffic_instance(seed=2, rows=50, cols=50, L=300, T=12, eps=0.05)
    h = O.ots_create_problem(inst)
    assert O.ots_problem_info(h)["threads_per_node"] >= 64
    O.ots_set_wait_limit(h, 2000, True)
    with pytest.raises(O.OTSError) as e:
        O.ots_iterate(h, 1, reset=True)
    assert e.value.code == O.OTS_ERR_DEVICE_WAIT
    O.ots_set_wait_limit(h, 0, False)                 # default limit, no switch
    r = O.ots_iterate(h, 20, reset=True)
    h2 = O.ots_create_problem(inst)
    r2 = O.ots_iterate(h2, 20, reset=True)
    assert (r["src_residual"], r["cap_violation"]) == (r2["src_residual"], r2["cap_violation"])
    assert np.array_equal(O.ots_get_flows(h), O.ots_get_flows(h2))
    with pytest.raises(O.OTSError) as e:
        O.ots_set_wait_limit(h, -1, False)
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    O.ots_destroy_problem(h)
    O.ots_destroy_problem(h2)

"""Host-side pieces of bench.py (no GPU): the algorithmic bytes behind the roofline figure, the
metric's update count and the committed traffic figure it reads."""
import os

import bench
from paper_2106_14485_gb300 import instances as I


def test_algorithmic_bytes_of_the_message_steps():
    """Forward step: read A_{t-1} and B_{t+1}, write A_t (6 B per node-commodity entry each) plus
    56 B per state and the node CSR; backward step: read B_{t+1}, write B_t plus 16 B per state.
    On the 100x100 grid with L = 1024: 187.1 MB and 123.7 MB per launch."""
    info = {"n_nodes": 10000, "n_states": 49600}

    class L1024:
        L = 1024
    assert bench.forward_bytes_per_launch(info, L1024) == 18 * 10000 * 1024 + 56 * 49600 + 4 * 10001 == 187137604
    assert bench.backward_bytes_per_launch(info, L1024) == 12 * 10000 * 1024 + 16 * 49600 + 4 * 10001 == 123713604


def test_update_count_of_the_metric():
    """One update = one (non-zero of K, commodity, step) term; 2 (T-1) nnz(K) L per pass.  For an
    R x C grid with wait loops nnz(K) = sum_v (deg_v + 1)^2: 5x5 -> 453, 100x100 -> 246408."""
    g = I.grid_single_commodity(0)
    assert g.nnz_line_graph() == 4 * 3 ** 2 + 12 * 4 ** 2 + 9 * 5 ** 2 == 453
    assert g.n_updates_per_iteration() == 2 * (g.T - 1) * 453 * g.L
    src, dst, _ = I.grid_graph(100, 100)
    x = I.Instance(name="g", n_nodes=10000, edge_src=src, edge_dst=dst, edge_cost=src * 0.0, edge_cap=src * 0.0,
                   wait_cost=None, wait_cap=None, L=1024, T=100, eps=1.0, src_comm=None, src_state=None,
                   src_mass=None, snk_comm=None, snk_state=None, snk_mass=None)
    assert x.nnz_line_graph() == 4 * 9 + 392 * 16 + 9604 * 25 == 246408
    assert x.n_updates_per_iteration() == 2 * 99 * 246408 * 1024


def test_committed_traffic_figure_is_read_only_for_the_current_sources():
    """bench.py reports the ncu DRAM traffic of the forward step only while the kernel sources hash
    to the version the counters were taken on."""
    path = os.path.join(os.path.dirname(bench.__file__), "profiles", "k_forward_tma-grid100x100-L1024.md")
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith(("|", " ")):
            k, _, v = line.partition(":")
            vals[k.strip()] = v.strip()
    got = bench.measured_traffic(100)
    if vals.get("kernel_source_sha256_16") == bench.kernel_sources_hash():
        assert got == int(vals["traffic_bytes_per_launch"])
    else:
        assert got is None

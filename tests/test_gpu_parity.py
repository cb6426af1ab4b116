"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 float-float log-domain messages against the FP64 oracle):
  relative L1 flow error  ||F - F*||_1 / ||F*||_1  <= 1e-5   over all (t, state) flows,
  marginal violation (source mismatch, capacity excess) <= 1e-6 at the GPU's stopping point.
"""
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2106_14485_gb300 import instances as I

pytestmark = pytest.mark.gpu

FLOW_TOL = 1e-5
ELEM_REL, ELEM_ABS = 1e-5, 1e-9     # entry-wise: |F - F*| <= ELEM_REL F* + ELEM_ABS max F*


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


def assert_elementwise(F, Fref, what=""):
    """Every entry within ELEM_REL of the oracle's, plus ELEM_ABS of the largest entry (so that
    low-flow states cannot hide under an L1 norm dominated by the corridors); names the worst."""
    r = np.abs(F - Fref) / (ELEM_REL * np.abs(Fref) + ELEM_ABS * np.abs(Fref).max())
    k = int(np.argmax(r))
    idx = np.unravel_index(k, r.shape)
    assert r.flat[k] <= 1.0, f"{what}: worst entry {idx}: gpu {F[idx]!r} oracle {Fref[idx]!r} (ratio {r.flat[k]:.3g})"
    return float(r.flat[k])


def assert_duals_relative(lu, lu_ref, Fref, bound, what=""):
    """log u is the relative error of u: compare it on the states that carry flow."""
    carry = Fref[1:-1] > 1e-6 * Fref.max()
    d = np.abs(lu - lu_ref)[carry]
    k = int(np.argmax(d))
    assert d[k] <= bound, f"{what}: log u differs by {d[k]:.3g} on a flow-carrying state (bound {bound})"
    return float(d[k])


def dense_duals(inst, U01, U0T):
    S = inst.n_states
    a = np.full((inst.L, S), -np.inf)
    b = np.full((inst.L, S), -np.inf)
    a[inst.src_comm, inst.src_state] = U01
    b[inst.snk_comm, inst.snk_state] = U0T
    return a, b


def capped_rgg(seed=4, n=60, L=9, T=16, eps=0.05, lo=0.15, hi=0.4):
    return I.rgg_instance(seed=seed, n=n, L=L, T=T, eps=eps, cap_lo=lo, cap_hi=hi)


# ---------------------------------------------------------------------------------------
# converged parity on instances the oracle solves in seconds
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grid5x5_converged(O, seed):
    inst = I.grid_single_commodity(seed)
    o = Oracle(inst)
    ro = o.solve(max_iters=200000, tol=1e-12)
    assert ro["status"] == 0
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=200000)
    assert r["src_residual"] <= 1e-8 and r["cap_violation"] <= 1e-8
    F = O.ots_get_flows(h)
    Fref = o.flows()
    assert rel_l1(F, Fref) <= FLOW_TOL
    assert_elementwise(F, Fref, "grid5x5")
    lu, _, _ = O.ots_get_duals(h)
    assert_duals_relative(lu, o.get_duals()[0], Fref, 1e-5, "grid5x5")
    O.ots_destroy_problem(h)


@pytest.mark.parametrize("L,eps,seed,lo,hi", [(9, 0.05, 9, 0.15, 0.4), (37, 0.02, 37, 0.15, 0.4),
                                              (64, 0.01, 64, 0.15, 0.4), (200, 0.05, 7, 0.05, 0.15),
                                              (500, 0.05, 7, 0.05, 0.15), (1000, 0.05, 7, 0.05, 0.15)])
def test_capacitated_converged(O, L, eps, seed, lo, hi):
    """Binding capacities, several commodities (ragged L: 9 -> 16, 37 -> 64, 200 -> 256,
    500 -> 512 padded lanes; L >= 200 runs the pipelined persistent kernels)."""
    inst = capped_rgg(seed=seed, L=L, eps=eps, T=18, lo=lo, hi=hi)
    o = Oracle(inst)
    ro = o.solve(max_iters=100000, tol=1e-11)
    assert ro["status"] == 0 and ro["cap_viol"] <= 1e-11
    logu_ref, _, _ = o.get_duals()
    assert (logu_ref < -1e-6).any(), "capacities should bind"
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-6, max_iters=20000)
    assert r["src_residual"] <= 1e-6 and r["cap_violation"] <= 1e-6
    F = O.ots_get_flows(h)
    Fref = o.flows()
    assert rel_l1(F, Fref) <= FLOW_TOL
    # duals where they are determined (states that carry flow)
    lu, U01, U0T = O.ots_get_duals(h)
    carry = Fref[1:-1] > 1e-6 * Fref.max()
    np.testing.assert_allclose(lu[carry], logu_ref[carry], atol=1e-4 * max(1.0, np.abs(logu_ref[carry]).max()))
    # per-commodity flows agree too
    P = O.ots_get_commodity_flows(h)
    Pref = o.projections()
    assert rel_l1(P, Pref) <= FLOW_TOL
    # Entry by entry.  (1) Arithmetic: the oracle evaluates Theorem 6 at the GPU's own duals, so
    # only the message arithmetic differs.  (2) The fixed point: at the stopping tolerance 1e-6 a
    # low-flow entry can still be 2e-5 away from the optimum (convergence, not arithmetic), so the
    # solve continues from its duals to 1e-8 first.
    od = Oracle(inst)
    od.set_duals(lu, *dense_duals(inst, U01, U0T))
    e_ar = assert_elementwise(P, od.projections(), f"L={L} per commodity at the GPU's duals")
    r8 = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=20000, warm_start=True)
    assert r8["status"] == 0
    F8, P8 = O.ots_get_flows(h), O.ots_get_commodity_flows(h)
    e_agg = assert_elementwise(F8, Fref, f"L={L} aggregate")
    e_com = assert_elementwise(P8, Pref, f"L={L} per commodity")
    e_dual = assert_duals_relative(O.ots_get_duals(h)[0], logu_ref, Fref, 1e-5, f"L={L}")
    print(f"capacitated L={L}: elementwise at duals {e_ar:.3g}, at 1e-8 {e_agg:.3g} / {e_com:.3g}, "
          f"max dlog u {e_dual:.3g}")
    O.ots_destroy_problem(h)


def test_per_commodity_costs(O):
    """C_L with a different row per commodity (Section 3.2; the paper's experiments draw
    c_e^l ~ U[0,1] per commodity)."""
    inst = capped_rgg(seed=21, L=12, T=14, eps=0.05)
    rng = np.random.default_rng(0)
    inst.commodity_cost = rng.uniform(0.0, 1.0, (inst.L, inst.n_states))
    o = Oracle(inst)
    ro = o.solve(max_iters=100000, tol=1e-11)
    assert ro["status"] == 0
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-6, max_iters=20000)
    assert r["status"] == 0
    assert rel_l1(O.ots_get_flows(h), o.flows()) <= FLOW_TOL
    assert rel_l1(O.ots_get_commodity_flows(h), o.projections()) <= FLOW_TOL


def test_wide_panel_more_than_1024_commodities(O):
    """L = 1100 commodities: 256 threads per node, two chunks per thread, ragged tail."""
    inst = I.rgg_instance(seed=3, n=40, L=1100, T=8, eps=0.1, cap_lo=2.0, cap_hi=6.0)
    o = Oracle(inst)
    o.solve(max_iters=20000, tol=1e-10)
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-6, max_iters=20000)
    assert r["status"] == 0
    assert rel_l1(O.ots_get_flows(h), o.flows()) <= FLOW_TOL


def test_pipelined_rows_of_1024_commodities(O):
    """L = 1000 (rows of 1024, ragged tail): the pipelined kernels with two 4-commodity chunks
    per consumer thread, against the oracle's fixed point."""
    inst = I.rgg_instance(seed=5, n=48, L=1000, T=9, eps=0.08, cap_lo=0.3, cap_hi=1.0, cap_div=40.0)
    o = Oracle(inst)
    o.solve(max_iters=20000, tol=1e-10)
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-7, max_iters=20000)
    assert r["status"] == 0
    F, Fref = O.ots_get_flows(h), o.flows()
    assert rel_l1(F, Fref) <= FLOW_TOL
    assert_elementwise(F, Fref, "L=1000 aggregate")
    P = O.ots_get_commodity_flows(h, 1, inst.T + 1, 990, 1000)
    Pref = o.projections(990, 1000)
    assert rel_l1(P, Pref) <= FLOW_TOL
    assert_elementwise(P, Pref, "L=1000 commodities 990..999")


# ---------------------------------------------------------------------------------------
# iterate-by-iterate parity (same initialisation, same number of passes)
# ---------------------------------------------------------------------------------------

def test_rgg400_iterates_and_converged(O):
    inst = I.rgg400(0)
    o = Oracle(inst)
    o.backward_sweep()
    h = O.ots_create_problem(inst)
    done = 0
    for target in (1, 3):
        n = target - done
        r = O.ots_iterate(h, n, reset=(done == 0))
        for _ in range(n):
            ro, co, _ = o.iteration()
        done = target
        F = O.ots_get_flows(h)
        assert rel_l1(F, o.flows()) <= FLOW_TOL, target
        assert abs(r["src_residual"] - ro) <= 1e-6 + 1e-4 * ro
        assert abs(r["cap_violation"] - co) <= 1e-6 + 1e-4 * co
    # converged
    r = O.ots_sinkhorn_solve(h, tol=1e-6)
    assert r["status"] == 0 and r["src_residual"] <= 1e-6 and r["cap_violation"] <= 1e-6
    o2 = Oracle(inst)
    o2.solve(max_iters=10000, tol=1e-10)
    assert rel_l1(O.ots_get_flows(h), o2.flows()) <= FLOW_TOL


def test_widest_rows_L4096(O):
    """The largest commodity count the ABI takes (L = 4096: 256 threads per node row, four chunks
    of 4 commodities per thread) with binding capacities: passes 1 and 3 from the initialisation
    against the oracle's (aggregate flows, the pass measures, log u on flow-carrying states), and
    every commodity's flows entry by entry where the oracle evaluates Theorem 6 at the GPU's duals."""
    inst = I.rgg_instance(seed=41, n=30, L=4096, T=8, eps=0.05, cap_lo=0.05, cap_hi=0.15, connect="bridge")
    h = O.ots_create_problem(inst)
    st = O.ots_problem_info(h)
    assert st["padded_L"] == 4096 and st["threads_per_node"] == 256
    o = Oracle(inst)
    o.backward_sweep()
    done = 0
    for target in (1, 3):
        n = target - done
        r = O.ots_iterate(h, n, reset=(done == 0))
        for _ in range(n):
            ro, co, _ = o.iteration()
        done = target
        Fo = o.flows()
        assert rel_l1(O.ots_get_flows(h), Fo) <= FLOW_TOL, target
        assert abs(r["src_residual"] - ro) <= 1e-6 + 1e-4 * ro
        assert abs(r["cap_violation"] - co) <= 1e-6 + 1e-4 * co
    lu, U01, U0T = O.ots_get_duals(h)
    logu_ref = o.get_duals()[0]
    carry = Fo[1:-1] > 1e-6 * Fo.max()
    assert (logu_ref[carry] < -1e-3).any(), "capacities should bind"
    assert np.abs(lu - logu_ref)[carry].max() <= 1e-5
    od = Oracle(inst)
    od.set_duals(lu, *dense_duals(inst, U01, U0T))
    e = assert_elementwise(O.ots_get_commodity_flows(h), od.projections(), "L=4096 per commodity at the GPU's duals")
    print(f"L=4096: worst entry {e:.3g} of the bound")
    O.ots_destroy_problem(h)


def test_dual_objective_matches_and_increases(O):
    """Dual objective of Theorem 3 after each pass equals the oracle's and does not decrease
    (block-coordinate ascent, proof of Proposition 5)."""
    inst = capped_rgg(seed=9, L=8, T=16)
    o = Oracle(inst)
    o.backward_sweep()
    h = O.ots_create_problem(inst)
    last = -np.inf
    for k in range(12):
        r = O.ots_iterate(h, 1, reset=(k == 0))
        o.iteration()
        ref = o.dual_objective()
        assert abs(r["dual_objective"] - ref) <= 1e-6 * abs(ref) + 1e-9
        assert r["dual_objective"] >= last - 1e-7 * abs(last)
        last = r["dual_objective"]


# ---------------------------------------------------------------------------------------
# traffic-scale workload (100x100 grid, L = 1024, T = 100): sampled outputs and properties
# ---------------------------------------------------------------------------------------

def test_traffic_grid_sampled_commodities_and_properties(O):
    inst = I.traffic_grid(0)
    h = O.ots_create_problem(inst)
    O.ots_iterate(h, 2, reset=True)
    lu, U01, U0T = O.ots_get_duals(h)
    F = O.ots_get_flows(h)
    # properties that hold at any size: exact sink marginal after the sink update, equal mass
    # at every t (Corollary 7), non-negative flows
    snk = np.zeros(inst.n_states)
    np.add.at(snk, inst.snk_state, inst.snk_mass)
    np.testing.assert_allclose(F[-1], snk, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(F.sum(axis=1), inst.total_mass(), rtol=1e-6)
    assert (F >= 0).all()
    # sampled commodities: the oracle evaluates Theorem 6 at the GPU's duals
    o = Oracle(inst)
    a, b = dense_duals(inst, U01, U0T)
    o.set_duals(lu, a, b)
    for l0, l1 in ((0, 3), (1021, 1024)):
        P = O.ots_get_commodity_flows(h, 1, inst.T + 1, l0, l1)
        Pref = o.projections(l0, l1)
        assert rel_l1(P, Pref) <= FLOW_TOL, (l0, rel_l1(P, Pref))
    O.ots_destroy_problem(h)


# ---------------------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------------------

def test_smallest_horizon_and_source_equals_sink(O):
    inst = I.rgg_instance(seed=8, n=20, L=3, T=3, eps=0.1)
    inst.snk_state = inst.src_state.copy()
    o = Oracle(inst)
    o.solve(max_iters=1000, tol=1e-12)
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-8)
    assert r["status"] == 0
    assert rel_l1(O.ots_get_flows(h), o.flows()) <= FLOW_TOL


def test_duplicate_triples_and_closed_states(O):
    """Repeated (commodity, state) triples add up; d = 0 closes a state."""
    inst = capped_rgg(seed=5, L=4, T=16)
    inst.edge_cap[:5] = 0.0
    m0 = float(inst.src_mass[0])
    inst.src_comm = np.concatenate([inst.src_comm, inst.src_comm[:1]])
    inst.src_state = np.concatenate([inst.src_state, inst.src_state[:1]])
    inst.src_mass = np.concatenate([inst.src_mass, [m0 / 2]])
    inst.src_mass[0] = m0 / 2
    o = Oracle(inst)
    ro = o.solve(max_iters=100000, tol=1e-11)
    assert ro["status"] == 0 and ro["cap_viol"] <= 1e-11, ro
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-6)
    assert r["status"] == 0
    F = O.ots_get_flows(h)
    assert rel_l1(F, o.flows()) <= FLOW_TOL
    assert np.all(F[1:-1, :5] == 0.0)
    lu, U01, _ = O.ots_get_duals(h)
    assert U01[0] == U01[-1]


def test_invalid_and_infeasible_inputs(O):
    inst = I.grid_single_commodity(0)
    bad = I.Instance(**{**inst.__dict__})
    bad.eps = -1.0
    with pytest.raises(O.OTSError) as e:
        O.ots_create_problem(bad)
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    bad = I.Instance(**{**inst.__dict__})
    bad.snk_mass = bad.snk_mass * 2
    with pytest.raises(O.OTSError) as e:
        O.ots_create_problem(bad)
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    far = I.grid_single_commodity(0, T=3)
    far.src_state = np.array([far.n_edges + 0], np.int32); far.src_mass = np.array([1.0]); far.src_comm = np.zeros(1, np.int32)
    far.snk_state = np.array([far.n_edges + 24], np.int32); far.snk_mass = np.array([1.0]); far.snk_comm = np.zeros(1, np.int32)
    with pytest.raises(O.OTSError) as e:
        O.ots_create_problem(far)
    assert e.value.code == O.OTS_ERR_INFEASIBLE
    # capacities that admit no feasible flow: the solver stops with NOT_CONVERGED, no fault
    tight = capped_rgg(seed=17, L=5, T=12)
    h = O.ots_create_problem(tight)
    r = O.ots_sinkhorn_solve(h, tol=1e-6, max_iters=300, raise_on_error=False)
    assert r["status"] == O.OTS_ERR_NOT_CONVERGED and r["cap_violation"] > 1e-2
    o = Oracle(tight)
    ro = o.solve(max_iters=300, tol=1e-6)
    assert abs(ro["cap_viol"] - r["cap_violation"]) <= 1e-3 * ro["cap_viol"]


def test_checkpoint_resume_and_determinism(O):
    inst = capped_rgg(seed=13, L=8, T=16)
    h1 = O.ots_create_problem(inst)
    O.ots_iterate(h1, 20, reset=True)
    F20 = O.ots_get_flows(h1)
    # same run again: bitwise equal
    h2 = O.ots_create_problem(inst)
    O.ots_iterate(h2, 20, reset=True)
    assert np.array_equal(O.ots_get_flows(h2), F20)
    # resume: 10 passes, checkpoint the duals, load them into a fresh problem, 10 more passes
    h3 = O.ots_create_problem(inst)
    O.ots_iterate(h3, 10, reset=True)
    duals = O.ots_get_duals(h3)
    h4 = O.ots_create_problem(inst)
    O.ots_set_duals(h4, *duals)
    O.ots_iterate(h4, 10, reset=False)
    assert rel_l1(O.ots_get_flows(h4), F20) <= 1e-6


def test_flows_at_duals_loaded_from_the_oracle(O):
    """Theorem 6 at duals the GPU did not produce: the oracle's iterate after three passes on a
    traffic-like grid with binding capacities, loaded through ots_set_duals.  The boundary panels
    are rebuilt from FP64 duals of ~1e4 bits; a remainder that once overflowed its 16-bit field
    there (a float part exactly halfway between two grid points) cost whole commodities 1e-4 of
    their flow at t >= 2.  Checked: every flow entry, every commodity's mass at every t, and a
    shift of one commodity's U01 far below an FP32 ulp of log2 U01 moving its flows at every t."""
    inst = I.grid_traffic_instance(seed=0, rows=30, cols=30, L=64, T=100, cap_lo=0.05, cap_hi=0.3)
    o = Oracle(inst)
    o.backward_sweep()
    for _ in range(3):
        o.iteration()
    lu, a, b = o.get_duals()
    U01, U0T = a[inst.src_comm, inst.src_state], b[inst.snk_comm, inst.snk_state]
    h = O.ots_create_problem(inst)
    O.ots_set_duals(h, lu, U01, U0T)
    P, Pref = O.ots_get_commodity_flows(h), o.projections()
    assert_elementwise(P, Pref, "per commodity at loaded duals")
    np.testing.assert_allclose(P.sum(axis=2), Pref.sum(axis=2), rtol=1e-5)
    m0 = P[1:3].sum(axis=2)                           # GPU masses at t = 2, 3 (read off A_1, A_2)
    for l in range(inst.L):
        k = int(np.where(inst.src_comm == l)[0][0])
        for d in (1e-6, 3e-5):
            U = U01.copy()
            U[k] += d
            O.ots_set_duals(h, lu, U, U0T)
            m = O.ots_get_commodity_flows(h, 2, 4, l, l + 1).sum(axis=2)[:, 0]
            np.testing.assert_allclose(np.log(m / m0[:, l]), d, atol=5e-7, err_msg=f"commodity {l}")
    O.ots_destroy_problem(h)


def test_solver_without_graph_and_with_cuda_allocator(O):
    inst = capped_rgg(seed=21, L=6, T=16)
    h1 = O.ots_create_problem(inst, allocator="cuda")
    r1 = O.ots_sinkhorn_solve(h1, tol=1e-6, use_graph=False)
    h2 = O.ots_create_problem(inst)
    r2 = O.ots_sinkhorn_solve(h2, tol=1e-6)
    assert r1["iterations"] == r2["iterations"]
    assert np.array_equal(O.ots_get_flows(h1), O.ots_get_flows(h2))


def test_plain_c_program_through_the_abi(O):
    """The C example drives the library without Python: create, solve, flows, duals."""
    import subprocess
    from tests.test_abi import build_c_example
    r = subprocess.run([build_c_example()], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "OTS_OK" in r.stdout


@pytest.mark.parametrize("name", ["grid5x5_seed0", "rgg30_L4_capped"])
def test_stored_golden_flows(O, name):
    """The GPU fixed point against the stored oracle values of tests/golden/ (no oracle run)."""
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_golden as G
    inst = G.CASES[name][0]()
    Fs, dual_s = G.load(name)
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=50000)
    assert r["status"] == 0
    assert rel_l1(O.ots_get_flows(h), Fs) <= FLOW_TOL
    assert r["dual_objective"] == pytest.approx(dual_s, rel=1e-5)
    O.ots_destroy_problem(h)

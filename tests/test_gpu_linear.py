"""The linear-domain path for single-commodity problems (L = 1; Algorithm 1 of Section 4.2 as
Algorithm 2 with one commodity) against the FP64 oracles, through the C ABI.

Iterates: the oracle runs the same passes of Algorithm 2 from the same initial duals, so after
k passes the duals agree up to the FP32 rounding of the GPU's messages (each pass multiplies
about T rounded factors per message: relative 1e-6 at T = 12).  Fixed points: the Algorithm 1
oracle (oracle/single_commodity.py, cyclic projections in FP64) and the log-domain oracle,
flows within the parity bounds of the log-domain path (relative L1 <= 1e-5, every entry within
1e-5 F* + 1e-9 max F*)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from oracle.single_commodity import cyclic_projections
from paper_2106_14485_gb300 import instances as I
from tests.test_single_commodity_pins import alg1_inputs

pytestmark = pytest.mark.gpu

FLOW_TOL = 1e-5
ELEM_REL, ELEM_ABS = 1e-5, 1e-9


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


def elementwise(F, Fref, what=""):
    r = np.abs(F - Fref) / (ELEM_REL * np.abs(Fref) + ELEM_ABS * np.abs(Fref).max())
    k = int(np.argmax(r))
    idx = np.unravel_index(k, r.shape)
    assert r.flat[k] <= 1.0, f"{what}: worst entry {idx}: gpu {F[idx]!r} oracle {Fref[idx]!r} (ratio {r.flat[k]:.3g})"
    return float(r.flat[k])


def oracle_after(inst, k):
    o = Oracle(inst)
    o.init_duals()
    o.backward_sweep()
    for _ in range(k):
        r = o.iteration()
    return o, r


def c4_single(seed, n, T, eps=0.01):
    """An L = 1 instance shaped like the uneven random-geometric family (bridged graph, eps = 0.01)
    with capacities U[0.2, 1] x mass / 2: binding, and feasible for these seeds (mass / 8 is
    below the cut a single commodity needs)."""
    return I.rgg_instance(seed=seed, n=n, L=1, T=T, eps=eps, cap_div=2.0, connect="bridge")


@pytest.mark.parametrize("seed,k", [(0, 1), (0, 3), (1, 3), (2, 5)])
def test_iterates_match_oracle(O, seed, k):
    """k passes from the initialisation: duals (on flow-carrying states and the boundary) and the
    measures of the last pass against the oracle's k passes."""
    inst = I.single_commodity_instance(seed=seed)
    o, (src_o, cap_o, _) = oracle_after(inst, k)
    h = O.ots_create_problem(inst)
    r = O.ots_linear_iterate(h, k, reset=True)
    assert r["iterations"] == k and r["linear"]["log_passes"] == 0
    lu, U01, U0T = O.ots_get_duals(h)
    lu_o, U01_o, U0T_o = o.get_duals()
    Fo = o.flows()
    carry = Fo[1:-1] > 1e-6 * Fo.max()
    assert np.abs(lu - lu_o)[carry].max() <= 5e-6
    assert np.abs(U01 - U01_o[0, inst.src_state]).max() <= 5e-6
    assert np.abs(U0T - U0T_o[0, inst.snk_state]).max() <= 5e-6
    assert r["src_residual"] == pytest.approx(src_o, rel=1e-4, abs=1e-9)
    assert r["cap_violation"] == pytest.approx(cap_o, rel=1e-4, abs=1e-9)
    # flows at the GPU's duals, evaluated by the log-domain kernels, against the oracle's
    elementwise(O.ots_get_flows(h), Fo, f"seed {seed}, {k} passes")
    O.ots_destroy_problem(h)


@pytest.mark.parametrize("seed,rows,T", [(0, 6, 12), (1, 6, 12), (2, 16, 30)])
def test_fixed_point_matches_algorithm1(O, seed, rows, T):
    inst = I.single_commodity_instance(seed=seed, rows=rows, cols=rows, T=T)
    u, P, it, src, cap = cyclic_projections(*alg1_inputs(inst))
    assert src < 1e-12 and cap < 1e-12
    h = O.ots_create_problem(inst)
    r = O.ots_linear_solve(h, tol=1e-8, max_iters=100000)
    assert r["status"] == 0 and r["src_residual"] <= 1e-8 and r["cap_violation"] <= 1e-8
    st = r["linear"]
    # the FP32 linear and the log-domain fixed points differ by about 1e-7: a few confirming passes
    assert st["linear_passes"] > 0 and st["confirm_passes"] <= 20
    F = O.ots_get_flows(h)
    assert rel_l1(F, P[1:]) <= FLOW_TOL
    elementwise(F, P[1:], f"single {rows}x{rows} T={T}")
    O.ots_destroy_problem(h)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grid5x5_small_eps(O, seed):
    """The 5x5 grid at eps = 0.05: message entries span far more than the FP32 range (the plain
    linear form loses flows), so the per-node scales must be taken and re-taken."""
    inst = I.grid_single_commodity(seed)
    o = Oracle(inst)
    assert o.solve(max_iters=200000, tol=1e-12)["status"] == 0
    Fref = o.flows()
    K, k, mu1, muT, d = alg1_inputs(inst)
    _, P, _, src, cap = cyclic_projections(K, k, mu1, muT, d, iters=200000, tol=1e-12)
    np.testing.assert_allclose(P[1:], Fref, rtol=1e-8, atol=1e-12)
    h = O.ots_create_problem(inst)
    r = O.ots_linear_solve(h, tol=1e-8, max_iters=200000)
    assert r["status"] == 0
    st = r["linear"]
    assert st["rescalings"] >= 1 and st["log_passes"] <= 0.1 * st["linear_passes"] + 2
    F = O.ots_get_flows(h)
    assert rel_l1(F, Fref) <= FLOW_TOL
    elementwise(F, Fref, f"grid5x5 seed {seed}")
    print(f"grid5x5 seed {seed}: {r['iterations']} passes, {st}")
    O.ots_destroy_problem(h)


@pytest.mark.parametrize("seed,n,T", [(3, 120, 20), (5, 300, 40), (13, 70, 33)])
def test_capacitated_rgg_l1(O, seed, n, T):
    """L = 1 instances of the uneven random-geometric family (eps = 0.01, binding capacities):
    the linear-domain solve, the log-domain solve and the oracle agree."""
    inst = c4_single(seed, n, T)
    o = Oracle(inst)
    ro = o.solve(max_iters=200000, tol=1e-11)
    assert ro["status"] == 0
    Fref = o.flows()
    h = O.ots_create_problem(inst)
    r = O.ots_linear_solve(h, tol=1e-8, max_iters=200000)
    assert r["status"] == 0
    F = O.ots_get_flows(h)
    assert rel_l1(F, Fref) <= FLOW_TOL
    elementwise(F, Fref, f"rgg n={n} T={T}")
    lu, _, _ = O.ots_get_duals(h)
    carry = Fref[1:-1] > 1e-6 * Fref.max()
    assert np.abs(lu - o.get_duals()[0])[carry].max() <= 1e-4
    O.ots_destroy_problem(h)


@pytest.mark.parametrize("seed,n,T", [(22, 800, 20), (24, 700, 30)])
def test_cluster_path(O, seed, n, T):
    """Problems of more than 4096 states run on a cluster of blocks (node ranges per block, step
    rows read across the cluster, cluster-wide sums): iterates after 3 passes and the fixed
    point against the oracle."""
    inst = c4_single(seed, n, T)
    assert inst.n_states > 4096
    o3, (src3, cap3, _) = oracle_after(inst, 3)
    h = O.ots_create_problem(inst)
    r = O.ots_linear_iterate(h, 3, reset=True)
    lu, U01, U0T = O.ots_get_duals(h)
    F3 = o3.flows()
    carry = F3[1:-1] > 1e-6 * F3.max()
    assert np.abs(lu - o3.get_duals()[0])[carry].max() <= 5e-6
    assert np.abs(U01 - o3.get_duals()[1][0, inst.src_state]).max() <= 5e-6
    assert r["cap_violation"] == pytest.approx(cap3, rel=1e-4, abs=1e-9)
    elementwise(O.ots_get_flows(h), F3, f"cluster n={n}, 3 passes")
    o = Oracle(inst)
    assert o.solve(max_iters=200000, tol=1e-11)["status"] == 0
    Fref = o.flows()
    r = O.ots_linear_solve(h, tol=1e-8, max_iters=200000)
    assert r["status"] == 0
    F = O.ots_get_flows(h)
    assert rel_l1(F, Fref) <= FLOW_TOL
    elementwise(F, Fref, f"cluster n={n} T={T}")
    O.ots_destroy_problem(h)


def test_solve_many_matches_one_at_a_time(O):
    """Several L = 1 problems of different sizes in one launch: each result equals its own
    log-domain solve within the parity bound, and the oracle's."""
    insts = [c4_single(10 + s, n, T) for s, (n, T) in enumerate([(50, 10), (90, 25), (160, 17), (70, 33), (120, 20)])]
    insts.append(I.grid_single_commodity(4))
    insts.append(c4_single(21, 800, 20))          # > 4096 states: the launch runs on clusters
    hs = [O.ots_create_problem(x) for x in insts]
    reps, st = O.ots_linear_solve_many(hs, tol=1e-8, max_iters=200000)
    assert all(r["status"] == 0 for r in reps)
    assert st["linear_passes"] > 0
    for x, h in zip(insts, hs):
        o = Oracle(x)
        assert o.solve(max_iters=200000, tol=1e-11)["status"] == 0
        Fref = o.flows()
        F = O.ots_get_flows(h)
        assert rel_l1(F, Fref) <= FLOW_TOL
        elementwise(F, Fref, x.name)
        O.ots_destroy_problem(h)


def test_time_varying_costs_and_closures(O):
    """Per-interval state costs (Section 3.3, C_t) with moving edges closed (+inf) in single
    intervals, on top of per-interval capacities: iterates and the fixed point against the oracle."""
    inst = I.with_time_varying_costs(I.single_commodity_instance(seed=5, rows=6, cols=6, T=14), seed=3,
                                     lo=0.5, hi=2.0, closures=6)
    assert np.isinf(inst.state_cost_t).sum() >= 1
    o3, _ = oracle_after(inst, 3)
    h = O.ots_create_problem(inst)
    O.ots_linear_iterate(h, 3, reset=True)
    lu = O.ots_get_duals(h)[0]
    F3 = o3.flows()
    carry = F3[1:-1] > 1e-6 * F3.max()
    assert np.abs(lu - o3.get_duals()[0])[carry].max() <= 5e-6
    elementwise(O.ots_get_flows(h), F3, "time-varying, 3 passes")
    o = Oracle(inst)
    assert o.solve(max_iters=200000, tol=1e-12)["status"] == 0
    Fref = o.flows()
    r = O.ots_linear_solve(h, tol=1e-8, max_iters=200000)
    assert r["status"] == 0
    F = O.ots_get_flows(h)
    assert rel_l1(F, Fref) <= FLOW_TOL
    elementwise(F, Fref, "time-varying fixed point")
    O.ots_destroy_problem(h)


def test_warm_start_and_iterate_continue(O):
    """Passes split over calls (warm start from the problem's duals) give the iterate of one call,
    and a linear-domain solve from a log-domain iterate ends at the same fixed point."""
    inst = I.single_commodity_instance(seed=3)
    h = O.ots_create_problem(inst)
    O.ots_linear_iterate(h, 4, reset=True)
    a = O.ots_get_duals(h)
    O.ots_linear_iterate(h, 2, reset=True)
    O.ots_linear_iterate(h, 2, reset=False)
    b = O.ots_get_duals(h)
    fin = np.isfinite(a[0])
    assert np.abs(a[0][fin] - b[0][fin]).max() <= 1e-6
    assert np.abs(a[1] - b[1]).max() <= 1e-6
    O.ots_iterate(h, 7, reset=True)
    r = O.ots_linear_solve(h, tol=1e-8, warm_start=True)
    assert r["status"] == 0
    F = O.ots_get_flows(h)
    u, P, _, _, _ = cyclic_projections(*alg1_inputs(inst))
    assert rel_l1(F, P[1:]) <= FLOW_TOL
    O.ots_destroy_problem(h)


def test_refusals(O):
    """The path applies to L = 1 with state costs and capacities; other problems are refused with
    OTS_ERR_INVALID_ARG and are left usable."""
    multi = I.rgg_instance(seed=1, n=40, L=3, T=10, eps=0.05)
    h = O.ots_create_problem(multi)
    with pytest.raises(O.OTSError) as e:
        O.ots_linear_iterate(h, 1, reset=True)
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    assert O.ots_iterate(h, 3, reset=True)["status"] == 0
    O.ots_destroy_problem(h)
    one = I.single_commodity_instance(seed=0)
    h = O.ots_create_problem(one)
    with pytest.raises(O.OTSError) as e:
        O.ots_linear_solve_many([h, h])          # the same problem twice
    assert e.value.code == O.OTS_ERR_INVALID_ARG
    O.ots_destroy_problem(h)

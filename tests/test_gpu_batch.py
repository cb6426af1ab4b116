"""Batched solving (ots_batch_*) against the FP64 oracle and the single-instance solver.

Every instance in a batch runs Algorithm 2 with its convergence test after every pass; the
batch also computes its flows.  Tolerances as for the single-instance path: relative L1 flow
error <= 1e-5 against the oracle, marginal measures <= tol at the stopping point.
"""
import json
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2106_14485_gb300 import instances as I

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


def assert_elementwise(F, Fref, what=""):
    """|F - F*| <= 1e-5 F* + 1e-9 max F* on every entry; names the worst."""
    r = np.abs(F - Fref) / (1e-5 * np.abs(Fref) + 1e-9 * np.abs(Fref).max())
    k = int(np.argmax(r))
    idx = np.unravel_index(k, r.shape)
    assert r.flat[k] <= 1.0, f"{what}: worst entry {idx}: gpu {F[idx]!r} oracle {Fref[idx]!r} (ratio {r.flat[k]:.3g})"


def mixed_instances():
    """Uneven sizes, horizons and commodity counts covering every thread mapping of the
    batch kernel (G = 1..32 with C = 1, and C = 2 for L > 128), binding capacities."""
    out = [I.grid_single_commodity(0), I.grid_single_commodity(1)]
    shapes = [(30, 1, 7, 100), (45, 3, 9, 200), (60, 7, 12, 102), (50, 13, 10, 103), (40, 30, 8, 202),
              (70, 61, 11, 105), (36, 120, 9, 106), (32, 200, 8, 107)]
    for n, L, T, seed in shapes:     # seeds whose capacities admit a feasible flow
        out.append(I.rgg_instance(seed=seed, n=n, L=L, T=T, eps=0.05, cap_lo=0.3, cap_hi=1.0))
    return out


def run_all(O, b, max_launches=20000):
    left = O.ots_batch_run(b, max_launches)
    assert left == 0, "instances still running"


def test_batch_matches_oracle_on_mixed_instances(O):
    insts = mixed_instances()
    b = O.ots_batch_create(pool_bytes=1 << 30, max_instances=16, ticks_per_launch=16)
    ids = [O.ots_batch_add(b, inst, tol=1e-7, max_iters=50000) for inst in insts]
    run_all(O, b)
    for inst, i in zip(insts, ids):
        st = O.ots_batch_status(b, i)
        assert st["status"] == 0, (inst.name, st)
        assert st["src_residual"] <= 1e-7 and st["cap_violation"] <= 1e-7
        o = Oracle(inst)
        ro = o.solve(max_iters=200000, tol=1e-12)
        assert ro["status"] == 0
        F = O.ots_batch_get_flows(b, i)
        assert F.shape == (inst.T, inst.n_states)
        Fref = o.flows()
        assert rel_l1(F, Fref) <= FLOW_TOL, inst.name
        assert_elementwise(F, Fref, inst.name)
    info = O.ots_batch_info(b)
    assert info["running"] == 0 and info["resident"] == len(insts)
    O.ots_batch_destroy(b)


def test_batch_equals_single_instance_solver(O):
    """Same fixed point as ots_sinkhorn_solve (both at tol 1e-8), same duals on the flow support."""
    inst = I.rgg_instance(seed=7, n=80, L=24, T=14, eps=0.03, cap_lo=0.3, cap_hi=1.0)
    h = O.ots_create_problem(inst)
    r = O.ots_sinkhorn_solve(h, tol=1e-8, max_iters=50000, check_every=1)
    assert r["status"] == 0
    F1 = O.ots_get_flows(h)
    lu1, _, _ = O.ots_get_duals(h)
    b = O.ots_batch_create(pool_bytes=256 << 20, max_instances=4)
    i = O.ots_batch_add(b, inst, tol=1e-8, max_iters=50000)
    run_all(O, b)
    st = O.ots_batch_status(b, i)
    assert st["status"] == 0
    # the convergence test after every pass stops at the same pass as check_every = 1
    assert abs(st["iterations"] - r["iterations"]) <= 1
    F2 = O.ots_batch_get_flows(b, i)
    assert rel_l1(F2, F1) <= 1e-6
    lu2, _, _ = O.ots_batch_get_duals(b, i)
    carry = F1[1:-1] > 1e-6 * F1.max()
    np.testing.assert_allclose(lu2[carry], lu1[carry], atol=1e-4 * max(1.0, np.abs(lu1[carry]).max()))
    O.ots_batch_destroy(b)
    O.ots_destroy_problem(h)


def test_result_is_the_same_alone_and_in_the_mix(O):
    """An instance's result does not depend on the instances that share the batch: bitwise
    equal flows, duals and pass counts alone, in a mix, and re-admitted into a reused slot."""
    target = I.rgg_instance(seed=11, n=90, L=40, T=13, eps=0.03, cap_lo=0.3, cap_hi=1.0)
    others = mixed_instances()[2:8]

    def solve(mix_before, mix_after, slots):
        b = O.ots_batch_create(pool_bytes=1 << 30, max_instances=slots, ticks_per_launch=8)
        for inst in mix_before:
            O.ots_batch_add(b, inst, tol=1e-7)
        i = O.ots_batch_add(b, target, tol=1e-7)
        for inst in mix_after:
            O.ots_batch_add(b, inst, tol=1e-7)
        run_all(O, b)
        out = (O.ots_batch_status(b, i), O.ots_batch_get_flows(b, i), O.ots_batch_get_duals(b, i))
        O.ots_batch_destroy(b)
        return out

    s0, F0, d0 = solve([], [], 1)
    s1, F1, d1 = solve(others[:3], others[3:], 8)
    s2, F2, d2 = solve(others[::-1], [], 8)
    assert s0["status"] == 0
    for s, F, d in ((s1, F1, d1), (s2, F2, d2)):
        assert s["iterations"] == s0["iterations"]
        assert np.array_equal(F, F0)
        for a, c in zip(d, d0):
            assert np.array_equal(a, c)


def test_slot_reuse_and_memory_admission(O):
    """Admission by memory and slots: a full batch refuses (OTS_ERR_OOM) and admits again once
    a finished instance is removed; the reused slot and pool memory give correct results."""
    a = I.rgg_instance(seed=200, n=60, L=16, T=12, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    c = I.rgg_instance(seed=22, n=50, L=8, T=10, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    b = O.ots_batch_create(pool_bytes=64 << 20, max_instances=1)
    ia = O.ots_batch_add(b, a, tol=1e-7)
    assert O.ots_batch_add(b, c, tol=1e-7, raise_on_error=False) == -O.OTS_ERR_OOM    # no slot
    assert O.ots_batch_status(b, ia)["status"] == O.OTS_PENDING
    run_all(O, b)
    Fa = O.ots_batch_get_flows(b, ia)
    O.ots_batch_remove(b, ia)
    ic = O.ots_batch_add(b, c, tol=1e-7)
    run_all(O, b)
    assert O.ots_batch_status(b, ic)["status"] == 0
    oc = Oracle(c)
    oc.solve(max_iters=200000, tol=1e-12)
    assert rel_l1(O.ots_batch_get_flows(b, ic), oc.flows()) <= FLOW_TOL
    oa = Oracle(a)
    oa.solve(max_iters=200000, tol=1e-12)
    assert rel_l1(Fa, oa.flows()) <= FLOW_TOL
    O.ots_batch_destroy(b)
    # pool too small for the instance: refused, nothing kept
    tiny = O.ots_batch_create(pool_bytes=1 << 16, max_instances=4)
    assert O.ots_batch_add(tiny, a, raise_on_error=False) == -O.OTS_ERR_OOM
    assert O.ots_batch_info(tiny)["resident"] == 0 and O.ots_batch_info(tiny)["pool_used"] == 0
    O.ots_batch_destroy(tiny)


def test_capacity_infeasible_instance_stops_at_pass_limit(O):
    """Capacities that admit no feasible flow: the batch stops at the pass limit with
    OTS_ERR_NOT_CONVERGED (as ots_sinkhorn_solve does) while a feasible neighbour converges."""
    bad = I.rgg_instance(seed=17, n=40, L=5, T=12, eps=0.05, cap_lo=0.01, cap_hi=0.02)
    good = I.grid_single_commodity(2)
    b = O.ots_batch_create(pool_bytes=256 << 20, max_instances=4)
    ib = O.ots_batch_add(b, bad, tol=1e-7, max_iters=300)
    ig = O.ots_batch_add(b, good, tol=1e-8, max_iters=100000)
    run_all(O, b)
    sb, sg = O.ots_batch_status(b, ib), O.ots_batch_status(b, ig)
    assert sb["status"] == O.OTS_ERR_NOT_CONVERGED and sb["iterations"] == 300
    assert sb["cap_violation"] > 1e-7
    assert sg["status"] == 0
    o = Oracle(good)
    o.solve(max_iters=200000, tol=1e-12)
    assert rel_l1(O.ots_batch_get_flows(b, ig), o.flows()) <= FLOW_TOL
    O.ots_batch_destroy(b)


def test_timeout_and_remove_while_running(O):
    inst = I.rgg_instance(seed=17, n=40, L=5, T=12, eps=0.05, cap_lo=0.01, cap_hi=0.02)
    b = O.ots_batch_create(pool_bytes=256 << 20, max_instances=4, ticks_per_launch=4)
    i = O.ots_batch_add(b, inst, tol=1e-7, max_iters=1 << 30, timeout_ms=50.0)
    j = O.ots_batch_add(b, inst, tol=1e-7, max_iters=1 << 30)
    O.ots_batch_run(b, 5000)
    assert O.ots_batch_status(b, i)["status"] == O.OTS_ERR_TIMEOUT
    assert O.ots_batch_status(b, j)["status"] == O.OTS_PENDING
    O.ots_batch_remove(b, j)                     # stops it and frees its slot
    assert O.ots_batch_info(b)["running"] == 0
    assert O.ots_batch_run(b, 10) == 0
    O.ots_batch_destroy(b)


def test_autotuner_writes_and_reads_its_table(O, tmp_path):
    b = O.ots_batch_create(pool_bytes=2 << 30, max_instances=64)
    path = str(tmp_path / "tune.json")
    O.ots_batch_autotune(b, path)
    tab = json.load(open(path))
    assert len(tab["classes"]) == 7
    for row in tab["classes"]:
        g, c = O.ots_batch_mapping(b, row["L_max"])
        assert (g, c) == (row["G"], row["C"]) and 4 * g * c >= row["L_max"] and g <= 32
    # a second batch reads the cached table instead of measuring
    b2 = O.ots_batch_create(pool_bytes=64 << 20, max_instances=4)
    os.utime(path, None)
    O.ots_batch_autotune(b2, path)
    for row in tab["classes"]:
        assert O.ots_batch_mapping(b2, row["L_max"]) == (row["G"], row["C"])
    # tuned mappings still solve correctly
    inst = I.rgg_instance(seed=5, n=50, L=20, T=10, eps=0.05, cap_lo=0.3, cap_hi=1.0)
    i = O.ots_batch_add(b2, inst, tol=1e-7)
    run_all(O, b2)
    o = Oracle(inst)
    o.solve(max_iters=200000, tol=1e-12)
    assert rel_l1(O.ots_batch_get_flows(b2, i), o.flows()) <= FLOW_TOL
    O.ots_batch_destroy(b)
    O.ots_batch_destroy(b2)

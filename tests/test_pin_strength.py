"""The pins catch plausible mistakes in the oracle.  Each case compiles a copy of
``oracle/ots_oracle.c`` with one planted mistake (a dropped term, a wrong sign, a wrong index, a
transposed operand, a convergence measure taken at the wrong moment or scaled wrongly), on the
CPU, and checks that at least one of four fast pins rejects it: projections and messages against
brute force at random duals (Theorem 6), the fixed point against Proposition 5 on the full tensor
with binding capacities, strong duality at the optimum (Theorem 3), and the two convergence
measures of a pass against the same pass done on the tensor.  The unmodified oracle passes all
four."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle.oracle import Oracle
from tests import pins_math as PM
from tests.test_oracle_pins import tiny_instance

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "ots_oracle.c")

# name: [(text, replacement, expected number of occurrences)]
MUTANTS = {
    "forward product without K_L": [
        ("double v = xl[i] + (lu ? wlog(o, t, l, i) + lu[i] : 0.0);", "double v = xl[i] + (lu ? lu[i] : 0.0);", 2)],
    "backward product with the dual of the wrong state": [
        ("double v = xl[j] + (lu ? wlog(o, t, l, j) + lu[j] : 0.0);", "double v = xl[j] + (lu ? wlog(o, t, l, j) + lu[i] : 0.0);", 2)],
    "forward product over successors instead of predecessors": [
        ("o->pred_ptr[j]; k < o->pred_ptr[j + 1]", "o->succ_ptr[j]; k < o->succ_ptr[j + 1]", 2),
        ("int i = o->pred_idx[k];", "int i = o->succ_idx[k];", 2)],
    "capacity update without the projection min(., 1)": [
        ("lu[i] = isfinite(di) ? fmin(log(di) - ls[i], 0.0) : 0.0;", "lu[i] = isfinite(di) ? log(di) - ls[i] : 0.0;", 1)],
    "column sums without Psi_t": [
        ("ph[(size_t)l * S + i] + ps[(size_t)l * S + i] + wlog(o, t, l, i)", "ph[(size_t)l * S + i] + wlog(o, t, l, i)", 2)],
    "column sums against Psi_{t+1}": [
        ("col_lse(o, t, ph, o->psi + (size_t)t * LS, ls);", "col_lse(o, t, ph, o->psi + (size_t)(t + 1) * LS, ls);", 1)],
    "source update with the wrong sign": [
        ("o->logU01[q] = log(o->R01[q]) - p1;", "o->logU01[q] = log(o->R01[q]) + p1;", 1)],
    "sink update with the wrong sign": [
        ("o->logU0T[q] = log(o->R0T[q]) - ph[q];", "o->logU0T[q] = log(o->R0T[q]) + ph[q];", 1)],
    "source mismatch taken after the source update": [
        ("resid += fabs(exp(o->logU01[q] + p1) - o->R01[q]);\n      if (!(p1 > -INFINITY)) bad = 1;\n"
         "      o->logU01[q] = log(o->R01[q]) - p1;",
         "if (!(p1 > -INFINITY)) bad = 1;\n      o->logU01[q] = log(o->R01[q]) - p1;\n"
         "      resid += fabs(exp(o->logU01[q] + p1) - o->R01[q]);", 1)],
    "source mismatch without the absolute value": [
        ("resid += fabs(exp(o->logU01[q] + p1) - o->R01[q]);", "resid += exp(o->logU01[q] + p1) - o->R01[q];", 1)],
    "capacity residual as the excess left after the update": [
        ("viol += flow_change(lu_old, lu[i], ls[i]);", "viol += fmax(exp(lu[i] + ls[i]) - di, 0.0);", 1)],
    "capacity residual counting only the duals that drop": [
        ("return exp(lu_old + ls) * fabs(expm1(lu_new - lu_old));",
         "return lu_new < lu_old ? exp(lu_old + ls) * fabs(expm1(lu_new - lu_old)) : 0.0;", 1)],
    "capacity residual not relative to the source mass": [
        ("if (cap_viol) *cap_viol = viol / o->mass01;", "if (cap_viol) *cap_viol = viol;", 1)],
    "dual objective without the capacity term": [
        ("if (isfinite(cap_at(o, t, s))) a += xlogy(cap_at(o, t, s), o->logu[(size_t)t * o->S + s]);",
         "if (isfinite(cap_at(o, t, s))) a += 0.0;", 1)],
}


def build_variant(text, d, name):
    c = os.path.join(d, name + ".c")
    so = os.path.join(d, name + ".so")
    with open(c, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", c, "-o", so, "-lm"])
    return so


def pin_projections(lib):
    """Theorem 6 at random duals: projections and messages against brute force."""
    T = 4
    inst = tiny_instance(seed=T, T=T)
    o = Oracle(inst, lib_path=lib)
    rng = np.random.default_rng(10 + T)
    S, L = inst.n_states, inst.L
    R01, R0T = PM.dense_marginals(inst)
    logu = -rng.uniform(0, 2, (T - 2, S))
    U01 = rng.uniform(-2, 2, (L, S))
    U0T = rng.uniform(-2, 2, (L, S))
    o.set_duals(logu, U01, U0T)
    P = o.projections()
    tz = PM.Tensor(inst)
    u = np.ones((T + 1, S))
    u[2:T] = np.exp(logu)
    eU01, eU0T = np.where(R01 > 0, np.exp(U01), 0), np.where(R0T > 0, np.exp(U0T), 0)
    M = tz.M(u, eU01, eU0T)
    ok = all(np.allclose(P[t - 1], tz.proj0t(M, t), rtol=1e-10, atol=1e-13) for t in range(1, T + 1))
    h, b = o.messages()
    hat, psi = PM.brute_messages(inst, u, eU01, eU0T)
    ok &= all(np.allclose(np.exp(h[t - 2]), hat[t], rtol=1e-10, atol=1e-13) for t in range(2, T + 1))
    ok &= all(np.allclose(np.exp(b[t - 1]), psi[t], rtol=1e-10, atol=1e-13) for t in range(1, T))
    return bool(ok)


_CACHE = {}


def _solved(lib):
    """(instance, oracle, solve report) of the capacitated pin instance, once per library."""
    if lib not in _CACHE:
        inst = tiny_instance(seed=7, T=5, L=2, cap_scale=0.8, eps=0.5)
        o = Oracle(inst, lib_path=lib)
        r = o.solve(max_iters=20000, tol=1e-13)
        _CACHE[lib] = (inst, o, r)
    return _CACHE[lib]


def _reference(inst):
    """Proposition 5 on the full tensor, once."""
    if "tensor" not in _CACHE:
        _CACHE["tensor"] = PM.tensor_sinkhorn(inst)
    return _CACHE["tensor"]


def pin_fixed_point(lib):
    """Proposition 5 on the full tensor (binding capacities) reaches the same flows."""
    try:
        inst, o, r = _solved(lib)
        if r["status"] != 0:
            return False
        P = o.projections()
    except (RuntimeError, ValueError):
        return False
    tz, M, _ = _reference(inst)
    return bool(all(np.allclose(P[t - 1], tz.proj0t(M, t), rtol=1e-6, atol=1e-8) for t in range(1, inst.T + 1)))


def pin_strong_duality(lib):
    """Theorem 3: dual objective = entropic primal objective at the optimum."""
    try:
        inst, o, r = _solved(lib)
        if r["status"] != 0:
            return False
        dual = o.dual_objective()
    except (RuntimeError, ValueError):
        return False
    tz, M, _ = _reference(inst)
    return bool(np.isclose(dual, PM.primal_objective(inst, tz, M), rtol=1e-8, atol=1e-12))


def pin_measures(lib):
    """The two convergence measures and the duals of one pass against the same pass done on the
    full tensor: two cold passes, then one pass from duals pulled below the fixed point."""
    from tests.test_measure_pins import binding_instance, check_pass
    try:
        inst = binding_instance(5)
        tz = _reference(inst)[0]
        o = Oracle(inst, lib_path=lib)
        o.backward_sweep()
        check_pass(o, inst, tz)
        check_pass(o, inst, tz)
        _, o2, r = _solved(lib)
        if r["status"] != 0:
            return False
        lu, a, b = o2.get_duals()
        o3 = Oracle(inst, lib_path=lib)
        o3.set_duals(lu - 0.5, a, b)
        check_pass(o3, inst, tz)
    except (AssertionError, RuntimeError, ValueError):
        return False
    return True


PINS = (pin_projections, pin_fixed_point, pin_strong_duality, pin_measures)


@pytest.fixture(scope="module")
def variants():
    src = open(SRC).read()
    d = tempfile.mkdtemp(prefix="orc_mut_")
    libs = {"control": build_variant(src, d, "control")}
    for k, (name, edits) in enumerate(MUTANTS.items()):
        text = src
        for old, new, count in edits:
            assert text.count(old) == count, (name, old)
            text = text.replace(old, new)
        libs[name] = build_variant(text, d, f"m{k}")
    return libs


def test_unmodified_oracle_passes_every_pin(variants):
    assert [p(variants["control"]) for p in PINS] == [True, True, True, True]


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(variants, name):
    results = [p(variants[name]) for p in PINS]
    assert not all(results), f"no pin rejects: {name}"

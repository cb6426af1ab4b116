"""Pins for the oracle's two convergence measures (the stopping rule, which Algorithm 2 leaves
open: the relative L1 source mismatch taken just before the U01 update, and the relative
capacity residual sum_t sum_i |P_t after - P_t before| of every u_t update).

Both are recomputed here from projections of the full transport tensor (direct summation over
all L * S^T paths, eq. proj_discrete_bi), with Proposition 5's block updates applied to the
tensor in Algorithm 2's order, and must equal the numbers ``orc_iteration`` returns to 1e-12
relative.  The duals after the pass must agree as well (an iterate-level check of the pass).
Three starting points: the initialisation after k cold passes, random duals, and duals pulled
below the fixed point (a warm start, where a capacity dual rises and the residual counts the
flow it gives back)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from tests import pins_math as PM
from tests.test_oracle_pins import tiny_instance


def linear_duals(inst, logu, logU01, logU0T):
    T, S = inst.T, inst.n_states
    R01, R0T = PM.dense_marginals(inst)
    u = np.ones((T + 1, S))
    u[2:T] = np.exp(logu)
    return u, np.where(R01 > 0, np.exp(logU01), 0.0), np.where(R0T > 0, np.exp(logU0T), 0.0)


def check_pass(o, inst, tz=None, rtol=1e-12):
    """Run one oracle pass from its current duals and compare both measures and the new duals
    with the same pass done on the tensor.  Returns (mismatch, residual) of the oracle."""
    tz = tz or PM.Tensor(inst)
    u, U01, U0T = linear_duals(inst, *o.get_duals())
    src_t, cap_t, u2, U01b, U0Tb = PM.tensor_pass_with_measures(inst, tz, u, U01, U0T)
    o.backward_sweep()
    src_o, cap_o, _ = o.iteration()
    assert src_o == pytest.approx(src_t, rel=rtol, abs=1e-15), (src_o, src_t)
    assert cap_o == pytest.approx(cap_t, rel=rtol, abs=1e-15), (cap_o, cap_t)
    lu, a, b = o.get_duals()
    np.testing.assert_allclose(np.exp(lu), u2[2:inst.T], rtol=1e-10, atol=1e-14)
    R01, R0T = PM.dense_marginals(inst)
    np.testing.assert_allclose(np.where(R01 > 0, np.exp(a), 0.0), U01b, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(np.where(R0T > 0, np.exp(b), 0.0), U0Tb, rtol=1e-10, atol=1e-14)
    return src_o, cap_o


def binding_instance(T=5):
    return tiny_instance(seed=7, T=T, L=2, cap_scale=0.8, eps=0.5)


@pytest.mark.parametrize("T", [4, 5])
def test_measures_after_cold_passes(T):
    """From the initialisation u_t = 1, passes 1..4 and pass 305: the measures are the tensor's source
    mismatch and capacity excess, and both have shrunk by pass 305 (linear convergence)."""
    inst = binding_instance(T)
    tz = PM.Tensor(inst)
    o = Oracle(inst)
    o.backward_sweep()
    seen = [check_pass(o, inst, tz) for _ in range(4)]
    assert seen[0][1] > 1e-3, "capacities should bind in the first pass"
    for _ in range(300):
        o.iteration()
    late = check_pass(o, inst, tz)
    assert late[0] < 1e-3 * seen[0][0] and late[1] < 1e-3 * seen[0][1]


def test_measures_at_random_duals():
    """Arbitrary duals (not an iterate of the method): the definitions still hold exactly."""
    inst = binding_instance(5)
    rng = np.random.default_rng(3)
    S, L, T = inst.n_states, inst.L, inst.T
    o = Oracle(inst)
    o.set_duals(-rng.uniform(0, 2, (T - 2, S)), rng.uniform(-2, 2, (L, S)), rng.uniform(-2, 2, (L, S)))
    src, cap = check_pass(o, inst)
    assert src > 1e-2 and cap > 1e-2


def test_measures_from_below_the_fixed_point():
    """A warm start with every capacity dual pulled down: updates raise u_t on states that are
    below their capacity, and the residual counts that withheld flow (the excess alone would
    read zero there)."""
    inst = binding_instance(5)
    o = Oracle(inst)
    assert o.solve(max_iters=20000, tol=1e-13)["status"] == 0
    lu, a, b = o.get_duals()
    o.set_duals(lu - 0.5, a, b)
    tz = PM.Tensor(inst)
    u, U01, U0T = linear_duals(inst, *o.get_duals())
    # the capacity excess of this state is zero everywhere: only the residual sees the gap
    M = tz.M(u, U01, U0T)
    excess = sum(np.maximum(tz.proj0t(M, t).sum(0) - PM.capacity_at(inst, t), 0).sum() for t in range(2, inst.T))
    assert excess == 0.0
    src, cap = check_pass(o, inst, tz)
    assert cap > 1e-2

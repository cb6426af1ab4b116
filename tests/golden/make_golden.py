"""Write the stored expected values of tests/golden/ from the FP64 oracle.

The paper prints no numeric worked example (its experiments report their results as figures), so
the stored values here are the oracle's fixed point (Algorithm 2 run to a relative marginal
residual of 1e-13) on two seeded instances.  They pin the oracle against later changes of its
arithmetic (test_golden.py re-solves and compares) and let the GPU tests compare against stored
numbers without running the oracle.  Only ``oracle/`` and the seeded input generators are used.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.oracle import Oracle                     # noqa: E402
from paper_2106_14485_gb300 import instances as I     # noqa: E402

CASES = {
    # name: (builder, description)
    "grid5x5_seed0": (lambda: I.grid_single_commodity(0),
                      "5x5 grid, one commodity, Dirichlet(1) sources and sinks on 3 nodes each, T=10, eps=0.05, "
                      "no capacities (instances.grid_single_commodity(0))"),
    "rgg30_L4_capped": (lambda: I.rgg_instance(seed=4, n=30, L=4, T=12, eps=0.05, cap_lo=0.15, cap_hi=0.4),
                        "random geometric graph n=30 (mean degree 6), L=4 single-pair commodities, T=12, eps=0.05, "
                        "edge capacities U[0.15,0.4]*mass/8, 50 binding state-steps (instances.rgg_instance(seed=4, "
                        "n=30, L=4, T=12, eps=0.05, cap_lo=0.15, cap_hi=0.4))"),
}
TOL = 1e-13


def solve(name):
    inst = CASES[name][0]()
    o = Oracle(inst)
    r = o.solve(max_iters=500000, tol=TOL)
    if r["status"] != 0 or r["src_resid"] > TOL or r["cap_viol"] > TOL:
        raise RuntimeError(f"{name}: oracle did not converge ({r})")
    return inst, o, o.flows(), o.dual_objective()


def write(name):
    inst, o, F, dual = solve(name)
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write(f"# {CASES[name][1]}\n")
        f.write("# Aggregate flows P_t(M) (Corollary 7; eq. proj_0t for t = 1, T) at the oracle's fixed point of\n")
        f.write(f"# Algorithm 2 (relative source and capacity residuals <= {TOL:g}); rows t = 1..T, columns the\n")
        f.write("# states (directed edges, then the wait loop of each node).  Written by tests/golden/make_golden.py.\n")
        f.write(f"# T {inst.T} S {F.shape[1]} dual_objective {dual:.17g}\n")
        np.savetxt(f, F, fmt="%.17g")
    return path


def load(name):
    """(flows [T, S], dual objective) of a stored case."""
    path = os.path.join(HERE, name + ".txt")
    dual = None
    with open(path) as f:
        for line in f:
            if line.startswith("# T "):
                dual = float(line.split()[-1])
    return np.loadtxt(path, comments="#"), dual


if __name__ == "__main__":
    for n in CASES:
        print(write(n))

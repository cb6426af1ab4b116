"""FP64 CPU oracle of the single-commodity scheme (Algorithm 1, Section 4.2).

TEST INFRASTRUCTURE.  Only ``tests/`` use this module; it imports nothing from the GPU package.

Problem (eq. singlecommodity_reg): one commodity on n states over T times, marginals
``mu_1`` and ``mu_T`` fixed, ``P_t(M) <= d_t`` for t = 2..T-1, cost
``sum_{t=1}^{T} c_{i_t} + sum_{t=1}^{T-1} C_{i_t i_{t+1}}``.  With ``k_t = exp(-c_t / eps)`` and
``K = exp(-C / eps)`` the solution is ``M = K .* (u_1 x ... x u_T)`` and the projections are
``P_t = u_t .* k_t .* hatphi_t .* phi_t`` (eq. proj_bridge) with the recursions of
eq. phi_hat / eq. phi.  The iteration follows Algorithm 1 in the paper's order: a backward
sweep for phi_{T-1..1}, the update of u_1, then for t = 2..T-1 hatphi_t and u_t, then
hatphi_T and u_T.

Reading: Algorithm 1 writes ``u_1 <- mu_1 ./ phi_1`` and ``u_T <- mu_T ./ hatphi_T`` without
``k_1`` and ``k_T``, while eq. proj_bridge has ``P_1 = u_1 .* k_1 .* phi_1``; the updates here
divide by ``k_1 .* phi_1`` and ``k_T .* hatphi_T`` so that the marginals hold.  (M itself does
not depend on k_1 or k_T: the fixed marginals absorb them.)

Linear domain in FP64 (the paper's form): valid while no product under- or overflows, which
the caller keeps by choosing epsilon and T; every result is checked to be finite.
"""
from __future__ import annotations

import numpy as np


def algorithm1(K, k, mu1, muT, d, iters: int = 100000, tol: float = 1e-13, literal_boundary: bool = False):
    """K: [n, n] (dense or scipy sparse), K_ij > 0 iff state i may be followed by j;
    k: [T+1, n], row t = k_t for t = 1..T (row 0 unused); mu1, muT: [n];
    d: [T+1, n], row t = d_t for t = 2..T-1 (inf for none).
    literal_boundary: use the boundary updates exactly as Algorithm 1 prints them (without k_1,
    k_T) -- only for the test that shows why the reading is needed.
    Returns (u [T+1, n], P [T+1, n] with rows 1..T, iterations, src mismatch, capacity residual)."""
    T = k.shape[0] - 1
    n = mu1.shape[0]
    Kt = K.T
    u = np.ones((T + 1, n))
    phi = np.ones((T + 1, n))       # phi_T = 1
    phih = np.ones((T + 1, n))      # hatphi_1 = 1
    mass = float(mu1.sum())
    src = cap = np.inf
    it = 0
    for it in range(1, iters + 1):
        for t in range(T - 1, 0, -1):                                   # phi_t = K (u_{t+1} k_{t+1} phi_{t+1})
            phi[t] = K @ (u[t + 1] * k[t + 1] * phi[t + 1])
        P1 = u[1] * k[1] * phi[1]
        src = float(np.abs(P1 - mu1).sum() / mass)
        with np.errstate(divide="ignore", invalid="ignore"):
            u[1] = np.where(mu1 > 0, mu1 / ((1.0 if literal_boundary else k[1]) * phi[1]), 0.0)
        cap = 0.0
        for t in range(2, T):
            phih[t] = Kt @ (u[t - 1] * k[t - 1] * phih[t - 1])
            col = k[t] * phih[t] * phi[t]
            p_old = u[t] * col
            with np.errstate(divide="ignore", invalid="ignore"):
                u_new = np.where(col > 0, np.minimum(d[t] / col, 1.0), 1.0)
            cap += float(np.abs(u_new * col - p_old).sum())
            u[t] = u_new
        phih[T] = Kt @ (u[T - 1] * k[T - 1] * phih[T - 1])
        with np.errstate(divide="ignore", invalid="ignore"):
            u[T] = np.where(muT > 0, muT / ((1.0 if literal_boundary else k[T]) * phih[T]), 0.0)
        cap /= mass
        if not np.all(np.isfinite(u)):
            raise FloatingPointError("linear-domain range exceeded (raise epsilon)")
        if src <= tol and cap <= tol:
            break
    # projections at the final duals (eq. proj_bridge), with a fresh backward sweep
    for t in range(T - 1, 0, -1):
        phi[t] = K @ (u[t + 1] * k[t + 1] * phi[t + 1])
    P = np.zeros((T + 1, n))
    for t in range(2, T + 1):
        phih[t] = Kt @ (u[t - 1] * k[t - 1] * phih[t - 1])
    for t in range(1, T + 1):
        P[t] = u[t] * k[t] * phih[t] * phi[t]
    return u, P, it, src, cap

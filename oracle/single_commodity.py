"""FP64 CPU oracle of the single-commodity problem (Section 4.2).

TEST INFRASTRUCTURE.  Only ``tests/`` use this module; it imports nothing from the GPU package.

Problem (eq. singlecommodity_reg): one commodity on n states over T times, marginals ``mu_1``
and ``mu_T`` fixed, ``P_t(M) <= d_t`` for t = 2..T-1, cost
``sum_{t=1}^{T} c_{i_t} + sum_{t=1}^{T-1} C_{i_t i_{t+1}}``.  With ``k_t = exp(-c_t / eps)`` and
``K = exp(-C / eps)`` the optimum has the form ``M = K .* (u_1 x ... x u_T)`` (Proposition 5
applied to this problem).

What is computed here, written from the definitions rather than from a listing:

* the messages of eq. phi (backward, ``phi_T = 1``, ``phi_t = K (u_{t+1} k_{t+1} phi_{t+1})``)
  and eq. phi_hat (forward, ``hatphi_1 = 1``, ``hatphi_t = K^T (u_{t-1} k_{t-1} hatphi_{t-1})``);
* the projections of eq. proj_bridge, ``P_t = u_t k_t hatphi_t phi_t`` (``project``);
* Proposition 5's block-coordinate scheme: the blocks (the marginal at t = 1, the capacity
  constraint at each t = 2..T-1, the marginal at t = T) are visited cyclically, and each visit
  is the Bregman projection onto that block: ``u_t <- u_t mu_t / P_t`` for a marginal and
  ``u_t <- min(u_t d_t / P_t, 1)`` elementwise for a capacity (the dual of an inequality stays
  non-negative, ``u_t <= 1``, and rises back towards 1 where the flow is below the capacity).
  Only the messages a visit depends on are recomputed: a cycle starts from a full backward
  recursion and carries the forward one along.

Reading: the boundary factors ``k_1`` and ``k_T`` enter ``P_1`` and ``P_T`` through
eq. proj_bridge, so the multiplicative updates above keep them; Algorithm 1 prints the boundary
updates without them (``literal_boundary`` reproduces that form, for the test that shows the
marginals then fail when the boundary costs are not zero).  M itself does not depend on k_1 or
k_T: the fixed marginals absorb them.

Linear domain in FP64, as the paper writes the method: valid while no product under- or
overflows, which the caller keeps by choosing epsilon and T; every result is checked to be
finite.
"""
from __future__ import annotations

import numpy as np


class SingleCommodity:
    """The problem data and its duals u (rows 1..T; row 0 unused)."""

    def __init__(self, K, k, mu1, muT, d):
        self.K, self.Kt = K, K.T
        self.k = np.asarray(k, np.float64)
        self.T = self.k.shape[0] - 1
        self.mu = {1: np.asarray(mu1, np.float64), self.T: np.asarray(muT, np.float64)}
        self.d = np.asarray(d, np.float64)
        n = self.k.shape[1]
        self.u = np.ones((self.T + 1, n))
        self.phi = np.ones((self.T + 1, n))       # eq. phi, phi_T = 1
        self.phih = np.ones((self.T + 1, n))      # eq. phi_hat, hatphi_1 = 1

    def backward(self):
        """phi_t for t = T-1..1 at the current u (eq. phi)."""
        for t in range(self.T - 1, 0, -1):
            self.phi[t] = self.K @ (self.u[t + 1] * self.k[t + 1] * self.phi[t + 1])

    def forward_to(self, t):
        """hatphi_t from hatphi_{t-1} at the current u (eq. phi_hat), t >= 2."""
        self.phih[t] = self.Kt @ (self.u[t - 1] * self.k[t - 1] * self.phih[t - 1])

    def project(self, t):
        """P_t(M) at the current u and messages (eq. proj_bridge)."""
        return self.u[t] * self.k[t] * self.phih[t] * self.phi[t]

    def visit_marginal(self, t, literal=False):
        """Projection onto {P_t(M) = mu_t}: u_t <- u_t mu_t / P_t (0 where mu_t = 0)."""
        with np.errstate(divide="ignore", invalid="ignore"):
            if literal:           # the boundary update as printed, without k_t
                self.u[t] = np.where(self.mu[t] > 0, self.mu[t] / (self.phih[t] * self.phi[t]), 0.0)
            else:
                P = self.project(t)
                self.u[t] = np.where(self.mu[t] > 0, self.u[t] * self.mu[t] / P, 0.0)

    def visit_capacity(self, t):
        """Projection onto {P_t(M) <= d_t}: u_t <- min(u_t d_t / P_t, 1); returns sum |P_new - P_old|."""
        P_old = self.project(t)
        with np.errstate(divide="ignore", invalid="ignore"):
            # states no path reaches get u = 1; d = 0 closes a state
            self.u[t] = np.where(P_old > 0, np.minimum(self.u[t] * self.d[t] / P_old, 1.0),
                                 np.where(self.d[t] == 0, 0.0, 1.0))
        return float(np.abs(self.project(t) - P_old).sum())

    def cycle(self, literal=False):
        """One cycle over the blocks t = 1, 2..T-1, T.  Returns the relative source mismatch
        taken before the t = 1 visit and the relative capacity residual of the cycle."""
        T, mass = self.T, float(self.mu[1].sum())
        self.backward()
        mismatch = float(np.abs(self.project(1) - self.mu[1]).sum()) / mass
        self.visit_marginal(1, literal)
        resid = 0.0
        for t in range(2, T):
            self.forward_to(t)
            resid += self.visit_capacity(t)
        self.forward_to(T)
        self.visit_marginal(T, literal)
        if not np.all(np.isfinite(self.u)):
            raise FloatingPointError("linear-domain range exceeded (raise epsilon)")
        return mismatch, resid / mass

    def all_projections(self):
        """P_t for t = 1..T at the current u, from fresh messages in both directions."""
        self.backward()
        for t in range(2, self.T + 1):
            self.forward_to(t)
        P = np.zeros_like(self.u)
        for t in range(1, self.T + 1):
            P[t] = self.project(t)
        return P


def cyclic_projections(K, k, mu1, muT, d, iters: int = 100000, tol: float = 1e-13, literal_boundary: bool = False):
    """Solve the single-commodity problem by the cyclic projections above.

    K: [n, n] (dense or scipy sparse), K_ij > 0 iff state i may be followed by j;
    k: [T+1, n], row t = k_t for t = 1..T (row 0 unused); mu1, muT: [n];
    d: [T+1, n], row t = d_t for t = 2..T-1 (inf for none).
    literal_boundary: the boundary updates exactly as Algorithm 1 prints them (without k_1, k_T).
    Stops when both measures of a cycle are <= tol.
    Returns (u [T+1, n], P [T+1, n] with rows 1..T, cycles, src mismatch, capacity residual)."""
    prob = SingleCommodity(K, k, mu1, muT, d)
    src = cap = np.inf
    it = 0
    for it in range(1, iters + 1):
        src, cap = prob.cycle(literal_boundary)
        if src <= tol and cap <= tol:
            break
    return prob.u, prob.all_projections(), it, src, cap

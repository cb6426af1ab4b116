"""Independent mathematics used to pin the oracle (no code shared with the oracle).

Everything here is written from the definitions in the paper, in FP64 linear domain, on
tiny instances only:

* the transport tensor M = K .* U over all L * S^T paths and its projections by direct
  summation (eq. proj_discrete, eq. proj_discrete_bi, eq. K_multicommodity, eq. U_multicommodity);
* the generic Sinkhorn scheme of Proposition 5 run on that full tensor;
* the Markov bridge for one source and one sink (Remark in Section 4.2);
* the reduction of an uncapacitated single-commodity problem to a two-marginal OT problem
  with the dense kernel K_eff = K (diag(k) K)^(T-2), solved by textbook Sinkhorn;
* the exact LP of problem eq. multicommodity (Theorem 2) via scipy's HiGHS.
"""
from __future__ import annotations

import itertools

import numpy as np


def tail_head(inst):
    if getattr(inst, "state_tail", None) is not None:            # explicit state graph (-1: none)
        return np.asarray(inst.state_tail), np.asarray(inst.state_head)
    V = inst.n_nodes
    tail = np.concatenate([np.asarray(inst.edge_src), np.arange(V)])
    head = np.concatenate([np.asarray(inst.edge_dst), np.arange(V)])
    return tail, head


def dense_K(inst) -> np.ndarray:
    """K_ij = 1 if edge i leads to edge j (second vertex of i is the first vertex of j), and
    K_ii = 1 for a state that may hold its flow (storage, Section 3.3)."""
    tail, head = tail_head(inst)
    K = ((head[:, None] == tail[None, :]) & (head[:, None] >= 0)).astype(np.float64)
    hold = getattr(inst, "state_hold", None)
    if hold is not None:
        K[np.arange(K.shape[0]), np.arange(K.shape[0])] = np.maximum(np.diag(K), np.asarray(hold, np.float64))
    return K


def dense_marginals(inst):
    S = inst.n_edges + inst.n_nodes
    R01 = np.zeros((inst.L, S))
    R0T = np.zeros((inst.L, S))
    for c, s, m in zip(inst.src_comm, inst.src_state, inst.src_mass):
        R01[c, s] += m
    for c, s, m in zip(inst.snk_comm, inst.snk_state, inst.snk_mass):
        R0T[c, s] += m
    return R01, R0T


def cost_matrix(inst) -> np.ndarray:
    """C_L as an L x S matrix."""
    if getattr(inst, "commodity_cost", None) is not None:
        return np.asarray(inst.commodity_cost, np.float64)
    c = np.concatenate([inst.edge_cost, inst.wait_cost]).astype(np.float64)
    return np.tile(c, (inst.L, 1))


def cost_at(inst, t: int) -> np.ndarray:
    """C_L in interval t (1-based, 2..T-1) as an L x S matrix: the per-interval costs of a
    time-varying network when the instance has them (same for every commodity)."""
    ct = getattr(inst, "state_cost_t", None)
    if ct is not None:
        return np.tile(np.asarray(ct[t - 2], np.float64), (inst.L, 1))
    return cost_matrix(inst)


def capacity(inst) -> np.ndarray:
    return np.concatenate([inst.edge_cap, inst.wait_cap]).astype(np.float64)


def capacity_at(inst, t: int) -> np.ndarray:
    """d_t for interval t (1-based, 2..T-1): the per-interval capacities when the instance has
    them, else the single capacity vector."""
    dt = getattr(inst, "state_capacity_t", None)
    if dt is not None:
        return np.asarray(dt[t - 2], np.float64)
    return capacity(inst)


def all_paths(S: int, T: int) -> np.ndarray:
    return np.array(list(itertools.product(range(S), repeat=T)), dtype=np.int64)


class Tensor:
    """The full tensor of eq. K_multicommodity for a tiny instance (L x S^T entries)."""

    def __init__(self, inst):
        self.inst = inst
        self.L, self.T, self.S = inst.L, inst.T, inst.n_edges + inst.n_nodes
        self.paths = all_paths(self.S, self.T)                     # [N, T]
        K = dense_K(inst)
        p = self.paths
        kpath = np.ones(len(p))
        for t in range(self.T - 1):                                 # prod_{t=1}^{T-1} K_{i_t i_{t+1}}
            kpath *= K[p[:, t], p[:, t + 1]]
        keep = kpath > 0                                            # drop infeasible paths
        self.paths = p[keep]
        self.kpath = kpath[keep]
        # prod_{t=2}^{T-1} (K_L,t)_{i_0 i_t}  (K_L,t = K_L unless the costs vary with t)
        self.kl = np.ones((self.L, len(self.paths)))
        for t in range(1, self.T - 1):
            KL = np.exp(-cost_at(inst, t + 1) / inst.eps)          # [L, S], 1-based time t + 1
            self.kl *= KL[:, self.paths[:, t]]

    def M(self, u, U01, U0T):
        """K .* U (eq. U_multicommodity); u is [T+1, S] with rows 2..T-1 used."""
        p = self.paths
        w = self.kl * self.kpath[None, :] * U01[:, p[:, 0]] * U0T[:, p[:, -1]]
        for t in range(1, self.T - 1):
            w = w * u[t + 1][p[:, t]][None, :]
        return w

    def proj0t(self, M, t):
        """P_{0,t}(M), 1-based t (eq. proj_discrete_bi with the commodity mode)."""
        out = np.zeros((self.L, self.S))
        for l in range(self.L):
            out[l] = np.bincount(self.paths[:, t - 1], weights=M[l], minlength=self.S)
        return out

    def proj_tt(self, M, t):
        """P_{t,t+1}(M) summed over commodities, [S, S]."""
        out = np.zeros((self.S, self.S))
        np.add.at(out, (self.paths[:, t - 1], self.paths[:, t]), M.sum(0))
        return out


def tensor_sinkhorn(inst, iters=20000, tol=1e-13, reverse=True):
    """Proposition 5 on the full tensor: U01, then u_t (reverse order by default; each followed by
    the commodity-capacity duals U^(0,t) when the instance has D), then U0T."""
    tz = Tensor(inst)
    L, S, T = tz.L, tz.S, tz.T
    R01, R0T = dense_marginals(inst)
    D = getattr(inst, "commodity_capacity", None)
    u = np.ones((T + 1, S))
    Uc = np.ones((T + 1, L, S))
    U01 = (R01 > 0).astype(float)
    U0T = (R0T > 0).astype(float)
    order = list(range(T - 1, 1, -1)) if reverse else list(range(2, T))

    def Mc():
        M = tz.M(u, U01, U0T)
        if D is not None:
            for t in range(2, T):
                M = M * Uc[t][:, tz.paths[:, t - 1]]
        return M

    for k in range(iters):
        M = Mc()
        P1 = tz.proj0t(M, 1)
        err = np.abs(P1 - R01).sum() / R01.sum()
        U01 = np.where(R01 > 0, U01 * R01 / np.where(P1 > 0, P1, 1), 0.0)
        for t in order:
            M = Mc()
            Pt = tz.proj0t(M, t).sum(0)
            dt = capacity_at(inst, t)
            with np.errstate(divide="ignore", invalid="ignore"):
                upd = np.where(Pt > 0, u[t] * dt / Pt, 1.0)
            upd = np.where(dt == 0, 0.0, upd)                       # d = 0 closes the state
            u[t] = np.minimum(upd, 1.0)
            if D is not None:                                       # U^(0,t) <- min(U D ./ P_{0,t}, 1)
                P0t = tz.proj0t(Mc(), t)
                with np.errstate(divide="ignore", invalid="ignore"):
                    updc = np.where(P0t > 0, Uc[t] * D / P0t, 1.0)
                Uc[t] = np.minimum(np.where(D == 0, 0.0, updc), 1.0)
        M = Mc()
        PT = tz.proj0t(M, T)
        U0T = np.where(R0T > 0, U0T * R0T / np.where(PT > 0, PT, 1), 0.0)
        M = Mc()
        excess = sum(np.maximum(tz.proj0t(M, t).sum(0) - capacity_at(inst, t), 0).sum() for t in range(2, T))
        if D is not None:
            excess += sum(np.maximum(tz.proj0t(M, t) - D, 0).sum() for t in range(2, T))
        if err < tol and excess / R01.sum() < tol:
            break
    M = Mc()
    return tz, M, (u, U01, U0T)


def bridge_flows(inst, l=0):
    """Single source s, single sink z, no capacities: P_{0,t} by dense linear products.

    F_1 = e_s, F_t = (F_{t-1} .* k_{t-1}) K;  G_T = e_z, G_t = K (k_{t+1} .* G_{t+1});
    k_t = (K_L)_l for t = 2..T-1 and 1 at t = 1, T;  P_{0,t} = mass F_t .* k_t .* G_t / F_T[z].
    """
    K = dense_K(inst)
    S, T = K.shape[0], inst.T
    kl = np.exp(-cost_matrix(inst)[l] / inst.eps)
    s = int(inst.src_state[list(inst.src_comm).index(l)])
    z = int(inst.snk_state[list(inst.snk_comm).index(l)])
    mass = float(inst.src_mass[list(inst.src_comm).index(l)])
    k = [None] + [np.ones(S)] + [kl] * (T - 2) + [np.ones(S)]   # 1-based k[t]
    F = [None] * (T + 1)
    G = [None] * (T + 1)
    F[1] = np.eye(S)[s]
    for t in range(2, T + 1):
        F[t] = (F[t - 1] * k[t - 1]) @ K
    G[T] = np.eye(S)[z]
    for t in range(T - 1, 0, -1):
        G[t] = K @ (k[t + 1] * G[t + 1])
    Z = F[T][z]
    return np.array([mass * F[t] * k[t] * G[t] / Z for t in range(1, T + 1)])


def two_marginal_flows(inst, iters=200000, tol=1e-14):
    """Uncapacitated single commodity: the coupling of (t=1, t=T) is two-marginal entropic OT
    with K_eff = K diag(k) K ... diag(k) K  (T-1 factors K); textbook Sinkhorn a <- mu1 ./ (K_eff b),
    b <- muT ./ (K_eff^T a); then P_t = (a^T K D..K)_s k_t (K D..K b)_s."""
    K = dense_K(inst)
    S, T = K.shape[0], inst.T
    kl = np.exp(-cost_matrix(inst)[0] / inst.eps)
    D = np.diag(kl)
    R01, R0T = dense_marginals(inst)
    mu1, muT = R01[0], R0T[0]
    Keff = K.copy()
    for _ in range(T - 2):
        Keff = Keff @ D @ K
    sup1, supT = mu1 > 0, muT > 0
    A = Keff[np.ix_(sup1, supT)]
    a = np.ones(sup1.sum())
    b = np.ones(supT.sum())
    for _ in range(iters):
        a = mu1[sup1] / (A @ b)
        b_new = muT[supT] / (A.T @ a)
        if np.max(np.abs(b_new - b) / b) < tol:
            b = b_new
            break
        b = b_new
    af = np.zeros(S); af[sup1] = a
    bf = np.zeros(S); bf[supT] = b
    fw = [None] * (T + 1)
    bw = [None] * (T + 1)
    fw[1] = af
    for t in range(2, T + 1):
        fw[t] = (fw[t - 1] * (kl if t - 1 >= 2 else 1.0)) @ K
    bw[T] = bf
    for t in range(T - 1, 0, -1):
        bw[t] = K @ ((kl if t + 1 <= T - 1 else 1.0) * bw[t + 1])
    out = []
    for t in range(1, T + 1):
        kt = kl if 2 <= t <= T - 1 else 1.0
        out.append(fw[t] * kt * bw[t])
    return np.array(out)


def lp_optimum(inst):
    """Exact LP of eq. multicommodity in node-edge form on the time-expanded state graph.

    Variables y[l, t, (i,j)] >= 0: flow of commodity l moving from state i at interval t to
    state j at interval t+1 (t = 1..T-1, K_ij = 1).  Constraints: out-flow at t = 1 equals
    R01, in-flow at t = T equals R0T, conservation at t = 2..T-1, and
    sum_l (flow in state j at t) <= d_j for t = 2..T-1.  Cost: sum_{t=2}^{T-1} C_L[l, j] x flow.
    Returns the optimal value."""
    import scipy.sparse as sp
    from scipy.optimize import linprog

    K = dense_K(inst)
    I, J = np.nonzero(K)
    nnz = len(I)
    L, T, S = inst.L, inst.T, K.shape[0]
    R01, R0T = dense_marginals(inst)
    C = cost_matrix(inst)
    d = capacity(inst)
    nvar = L * (T - 1) * nnz
    var = lambda l, t: (l * (T - 1) + (t - 1)) * nnz   # t = 1..T-1
    rows, cols, vals, beq = [], [], [], []
    r = 0
    for l in range(L):
        for i in range(S):                                   # t = 1 out-flow = R01
            m = I == i
            rows += [r] * m.sum(); cols += list(var(l, 1) + np.nonzero(m)[0]); vals += [1.0] * m.sum()
            beq.append(R01[l, i]); r += 1
        for j in range(S):                                   # t = T in-flow = R0T
            m = J == j
            rows += [r] * m.sum(); cols += list(var(l, T - 1) + np.nonzero(m)[0]); vals += [1.0] * m.sum()
            beq.append(R0T[l, j]); r += 1
        for t in range(2, T):                                # conservation in state s at interval t
            for s in range(S):
                mi, mo = J == s, I == s
                rows += [r] * (mi.sum() + mo.sum())
                cols += list(var(l, t - 1) + np.nonzero(mi)[0]) + list(var(l, t) + np.nonzero(mo)[0])
                vals += [1.0] * mi.sum() + [-1.0] * mo.sum()
                beq.append(0.0); r += 1
    Aeq = sp.csr_matrix((vals, (rows, cols)), shape=(r, nvar))
    rows, cols, vals, bub = [], [], [], []
    r = 0
    for t in range(2, T):
        for s in range(S):
            if not np.isfinite(d[s]):
                continue
            mo = np.nonzero(I == s)[0]
            for l in range(L):
                rows += [r] * len(mo); cols += list(var(l, t) + mo); vals += [1.0] * len(mo)
            bub.append(d[s]); r += 1
    Aub = sp.csr_matrix((vals, (rows, cols)), shape=(r, nvar)) if r else None
    c = np.zeros(nvar)
    for l in range(L):
        for t in range(2, T):
            c[var(l, t):var(l, t) + nnz] = C[l, I]
    res = linprog(c, A_ub=Aub, b_ub=bub if r else None, A_eq=Aeq, b_eq=beq, bounds=(0, None), method="highs")
    assert res.status == 0, res.message
    return float(res.fun)


def window_tensor_sinkhorn(inst, iters=20000, tol=1e-13):
    """Proposition 5 on the multi-tensor problem of the Remark after Algorithm 2, with each
    commodity's tensor over its own times a_l..b_l (paths of length b_l - a_l + 1, K_L and the
    shared u_t at its interior times) and the capacity sums over the commodities inside their
    windows; full enumeration for tiny instances.  Returns a function P(l, t) -> [S] (zero
    outside the window)."""
    K = dense_K(inst)
    L, T, S = inst.L, inst.T, inst.n_edges + inst.n_nodes
    a = np.asarray(inst.commodity_t_in)
    b = np.asarray(inst.commodity_t_out)
    R01, R0T = dense_marginals(inst)
    KL = np.exp(-cost_matrix(inst) / inst.eps)
    paths, base = [], []
    for l in range(L):
        p = all_paths(S, int(b[l] - a[l] + 1))
        w = np.ones(len(p))
        for k in range(p.shape[1] - 1):
            w *= K[p[:, k], p[:, k + 1]]
        for k in range(1, p.shape[1] - 1):
            w *= KL[l, p[:, k]]
        keep = w > 0
        paths.append(p[keep])
        base.append(w[keep])
    u = np.ones((T + 1, S))
    U01 = (R01 > 0).astype(float)
    U0T = (R0T > 0).astype(float)

    def M(l):
        p = paths[l]
        w = base[l] * U01[l, p[:, 0]] * U0T[l, p[:, -1]]
        for k in range(1, p.shape[1] - 1):
            w = w * u[a[l] + k][p[:, k]]
        return w

    def proj(l, t):
        if t < a[l] or t > b[l]:
            return np.zeros(S)
        return np.bincount(paths[l][:, t - a[l]], weights=M(l), minlength=S)

    for _ in range(iters):
        err = 0.0
        for l in range(L):
            P = proj(l, a[l])
            err += np.abs(P - R01[l]).sum()
            U01[l] = np.where(R01[l] > 0, U01[l] * R01[l] / np.where(P > 0, P, 1), 0.0)
        excess = 0.0
        for t in range(T - 1, 1, -1):
            Pt = sum(proj(l, t) for l in range(L) if a[l] < t < b[l]) + np.zeros(S)
            d = capacity_at(inst, t)
            with np.errstate(divide="ignore", invalid="ignore"):
                upd = np.where(Pt > 0, u[t] * d / Pt, 1.0)
            u_new = np.minimum(upd, 1.0)
            excess += np.abs((u_new - u[t]) * np.where(u[t] > 0, Pt / np.where(u[t] > 0, u[t], 1), 0)).sum()
            u[t] = u_new
        for l in range(L):
            P = proj(l, b[l])
            U0T[l] = np.where(R0T[l] > 0, U0T[l] * R0T[l] / np.where(P > 0, P, 1), 0.0)
        if err / R01.sum() < tol and excess / R01.sum() < tol:
            break
    return proj


def primal_objective(inst, tz, M) -> float:
    """Entropic primal objective of eq. multicommodity_reg on the full tensor, without the constant
    of the entropy term: sum over paths of M (path cost) + eps M (log M - 1), with the state
    costs C_L applied at t = 2..T-1 (the transitions of K cost nothing)."""
    cost = np.zeros((tz.L, len(tz.paths)))
    for t in range(1, tz.T - 1):
        C = cost_at(inst, t + 1)                                    # [L, S], 1-based time t + 1
        cost += C[:, tz.paths[:, t]]
    pos = M > 0
    return float(np.sum(M * cost) + inst.eps * np.sum(M[pos] * (np.log(M[pos]) - 1.0)))


def brute_messages(inst, u, U01, U0T):
    """The messages of Theorem 6 by direct summation over partial paths (linear domain):
    hatPsi_t[l, j] sums U01[l, i_1] prod_s K[i_s, i_{s+1}] prod_{s=2}^{t-1} K_L[l, i_s] u_s[i_s] over the
    paths (i_1, ..., i_t = j), t = 2..T; Psi_t[l, i] sums prod_s K[i_s, i_{s+1}]
    prod_{s=t+1}^{T-1} K_L[l, i_s] u_s[i_s] U0T[l, i_T] over the paths (i = i_t, ..., i_T), t = 1..T-1.
    u is [T+1, S] (rows 2..T-1 used).  Returns (hat [T+1, L, S], psi [T+1, L, S]) by row t."""
    K = dense_K(inst)
    L, T, S = inst.L, inst.T, K.shape[0]
    KL = {s: np.exp(-cost_at(inst, s) / inst.eps) for s in range(2, T)}
    hat = np.zeros((T + 1, L, S))
    psi = np.zeros((T + 1, L, S))
    for t in range(2, T + 1):
        for p in itertools.product(range(S), repeat=t):
            k = np.prod([K[p[s], p[s + 1]] for s in range(t - 1)])
            if k == 0:
                continue
            w = U01[:, p[0]] * k
            for s in range(2, t):                                  # 1-based interval s at p[s - 1]
                w = w * KL[s][:, p[s - 1]] * u[s][p[s - 1]]
            hat[t, :, p[-1]] += w
    for t in range(1, T):
        for p in itertools.product(range(S), repeat=T - t + 1):
            k = np.prod([K[p[s], p[s + 1]] for s in range(T - t)])
            if k == 0:
                continue
            w = U0T[:, p[-1]] * k
            for s in range(t + 1, T):
                w = w * KL[s][:, p[s - t]] * u[s][p[s - t]]
            psi[t, :, p[0]] += w
    return hat, psi


def tensor_pass_with_measures(inst, tz, u, U01, U0T):
    """One pass of Algorithm 2 done on the full tensor (Proposition 5's block updates in the
    order U01, u_2 .. u_{T-1}, U0T), with the two convergence measures taken from the tensor's
    projections: the relative L1 source mismatch ||P_{0,1} - R01||_1 / ||R01||_1 of the tensor
    before the U01 update, and the relative capacity residual
    sum_t sum_i |P_t(after the u_t update) - P_t(before it)| / ||R01||_1.

    u is [T+1, S] (rows 2..T-1 used), U01 and U0T are L x S linear duals (0 off the supports).
    Returns (mismatch, residual, u, U01, U0T) with the updated duals (new arrays)."""
    R01, R0T = dense_marginals(inst)
    T = tz.T
    u, U01, U0T = u.copy(), U01.copy(), U0T.copy()
    mass = R01.sum()
    P1 = tz.proj0t(tz.M(u, U01, U0T), 1)
    mismatch = np.abs(P1 - R01).sum() / mass
    with np.errstate(divide="ignore", invalid="ignore"):
        U01 = np.where(R01 > 0, U01 * R01 / np.where(P1 > 0, P1, 1.0), 0.0)
    resid = 0.0
    for t in range(2, T):
        before = tz.proj0t(tz.M(u, U01, U0T), t).sum(0)
        with np.errstate(divide="ignore", invalid="ignore"):
            column = np.where(u[t] > 0, before / np.where(u[t] > 0, u[t], 1.0), 0.0)
            d = capacity_at(inst, t)
            new = np.where(column > 0, np.minimum(d / np.where(column > 0, column, 1.0), 1.0), 1.0)
        u[t] = new
        after = tz.proj0t(tz.M(u, U01, U0T), t).sum(0)
        resid += np.abs(after - before).sum()
    PT = tz.proj0t(tz.M(u, U01, U0T), T)
    with np.errstate(divide="ignore", invalid="ignore"):
        U0T = np.where(R0T > 0, U0T * R0T / np.where(PT > 0, PT, 1.0), 0.0)
    return mismatch, resid / mass, u, U01, U0T

"""Seeded synthetic instances of the dynamic multi-commodity min-cost flow problem.

This module only builds input data (graphs, costs, capacities, marginals).  It holds
none of the method's arithmetic: both the CUDA solver and the FP64 oracle consume the
``Instance`` objects built here.

Conventions (shared by every consumer, restated in ``include/ots.h``):

* The road network is a directed graph with ``n_nodes`` nodes and ``n_edges`` directed
  edges ``edge_src[e] -> edge_dst[e]``.
* A *state* is a directed edge (the edge-state model of Section 3.1, marginals on edges).
  Waiting is modelled by one self-loop state per node (the vertex augmentation of
  Section 3.3): states ``0..n_edges-1`` are the edges, state ``n_edges + v`` is the wait
  loop of node ``v``.  ``n_states = n_edges + n_nodes``.
* Costs are per state and per time interval (``C_L`` of Section 3.2, identical rows for
  every commodity unless ``commodity_cost`` is given), capacities are per state
  (``d`` of Section 3.2, ``inf`` = uncapacitated).
* Sources / sinks are ``(commodity, state, mass)`` triples: the non-zeros of
  ``R^(0,1)`` and ``R^(0,T)`` of Section 3.2.  All sources and sinks sit on wait-loop
  states of nodes.

Workload recipes of the benchmark (see ``WORKLOADS``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Instance:
    name: str
    n_nodes: int
    edge_src: np.ndarray          # int32 [E]
    edge_dst: np.ndarray          # int32 [E]
    edge_cost: np.ndarray         # float64 [E], cost per interval on the edge
    edge_cap: np.ndarray          # float64 [E], inf = none
    wait_cost: np.ndarray         # float64 [V], cost per interval on the node's wait loop
    wait_cap: np.ndarray          # float64 [V], inf = none
    L: int
    T: int
    eps: float
    src_comm: np.ndarray          # int32 [n_src]
    src_state: np.ndarray         # int32 [n_src]
    src_mass: np.ndarray          # float64 [n_src]
    snk_comm: np.ndarray          # int32 [n_snk]
    snk_state: np.ndarray         # int32 [n_snk]
    snk_mass: np.ndarray          # float64 [n_snk]
    pos: Optional[np.ndarray] = None              # [V, 2] node positions (not used by solvers)
    commodity_cost: Optional[np.ndarray] = None   # [L, S] per-commodity state costs
    state_cost_t: Optional[np.ndarray] = None     # [T-2, S] per-interval state costs (t = 2..T-1)
    state_capacity_t: Optional[np.ndarray] = None  # [T-2, S] per-interval capacities d_t (inf: none)
    commodity_t_in: Optional[np.ndarray] = None   # [L] entry time of each commodity (1..T-1)
    commodity_t_out: Optional[np.ndarray] = None  # [L] exit time of each commodity (t_in+1..T)
    commodity_capacity: Optional[np.ndarray] = None  # [L, S] D^(0,t), the same for every t (inf: none)
    # explicit state graph (Section 3.3 storage models), replacing edges + wait loops: tail and head
    # node of every state (-1: none) and a storage flag (the state may follow itself)
    state_tail: Optional[np.ndarray] = None       # int32 [S]
    state_head: Optional[np.ndarray] = None       # int32 [S]
    state_hold: Optional[np.ndarray] = None       # int32 [S], 1 = storage
    meta: dict = field(default_factory=dict)

    # ---- derived sizes / per-state views (data assembly only) ----
    @property
    def n_edges(self) -> int:
        return int(self.edge_src.shape[0])

    @property
    def n_states(self) -> int:
        return self.n_edges + self.n_nodes

    def state_cost(self) -> np.ndarray:
        """Per-state cost vector [S]: edge costs then wait-loop costs."""
        return np.concatenate([self.edge_cost, self.wait_cost]).astype(np.float64)

    def state_cap(self) -> np.ndarray:
        """Per-state capacity vector [S]: edge capacities then wait-loop capacities."""
        return np.concatenate([self.edge_cap, self.wait_cap]).astype(np.float64)

    def state_tail_head(self):
        """(tail, head) node of every state; a wait loop has tail == head (-1: none, with an
        explicit state graph)."""
        if self.state_tail is not None:
            return np.asarray(self.state_tail, np.int32), np.asarray(self.state_head, np.int32)
        loops = np.arange(self.n_nodes, dtype=np.int32)
        tail = np.concatenate([self.edge_src, loops]).astype(np.int32)
        head = np.concatenate([self.edge_dst, loops]).astype(np.int32)
        return tail, head

    def total_mass(self) -> float:
        return float(np.sum(self.src_mass))

    def n_updates_per_iteration(self) -> int:
        """Work units of one Sinkhorn sweep: 2 (T-1) nnz(K) L.

        nnz(K) counts the transitions of the line graph with wait loops, i.e. the
        ordered state pairs (i, j) with head(i) == tail(j).
        """
        return 2 * (self.T - 1) * self.nnz_line_graph() * self.L

    def nnz_line_graph(self) -> int:
        """Ordered state pairs (i, j) with head(i) == tail(j), plus the storage states that do
        not already follow themselves."""
        tail, head = self.state_tail_head()
        indeg = np.bincount(head[head >= 0], minlength=self.n_nodes).astype(np.int64)
        outdeg = np.bincount(tail[tail >= 0], minlength=self.n_nodes).astype(np.int64)
        extra = 0
        if self.state_hold is not None:
            hold = np.asarray(self.state_hold) != 0
            extra = int(np.sum(hold & ~((head >= 0) & (head == tail))))
        return int(np.sum(indeg * outdeg)) + extra


# ----------------------------------------------------------------------------------
# graph builders
# ----------------------------------------------------------------------------------

def grid_graph(rows: int, cols: int):
    """4-neighbour grid, both directions.  Node id = r * cols + c."""
    src, dst = [], []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            for dr, dc in ((0, 1), (1, 0), (0, -1), (-1, 0)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < rows and 0 <= cc < cols:
                    src.append(v)
                    dst.append(rr * cols + cc)
    pos = np.stack(np.meshgrid(np.arange(cols, dtype=np.float64),
                               np.arange(rows, dtype=np.float64)), -1).reshape(-1, 2)
    return np.asarray(src, np.int32), np.asarray(dst, np.int32), pos


def _connected(n: int, src: np.ndarray, dst: np.ndarray) -> bool:
    return bool(np.all(hop_distances(n, src, dst, 0) >= 0))


def _components(n: int, src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Connected-component label of every node (undirected edge lists in both directions)."""
    label = np.full(n, -1, np.int64)
    order = np.argsort(src, kind="stable")
    ptr = np.zeros(n + 1, np.int64)
    np.add.at(ptr, src.astype(np.int64) + 1, 1)
    ptr = np.cumsum(ptr)
    nbr = dst[order]
    c = 0
    for s0 in range(n):
        if label[s0] >= 0:
            continue
        label[s0] = c
        stack = [s0]
        while stack:
            v = stack.pop()
            for w in nbr[ptr[v]:ptr[v + 1]]:
                if label[w] < 0:
                    label[w] = c
                    stack.append(int(w))
        c += 1
    return label


def rgg_graph(n: int, mean_degree: float, rng: np.random.Generator, max_tries: int = 200,
              connect: str = "reject"):
    """Random geometric graph in the unit square.

    The radius is calibrated per draw so that the mean degree is exactly ``mean_degree``
    (the ``n * mean_degree / 2`` shortest pairs become undirected edges).  A draw that is not
    connected is rejected (connect="reject"), or (connect="bridge", used where graphs of up
    to thousands of nodes are drawn and almost never come out connected at this degree)
    kept and made connected by repeatedly joining the smallest component to the rest with
    its shortest edge, as a road network would be.  Nodes are renumbered along a coarse
    spatial sort so that neighbouring nodes have nearby ids.
    """
    n_und = int(round(n * mean_degree / 2))
    for _ in range(max_tries if connect == "reject" else 1):
        pos = rng.random((n, 2))
        d = np.sqrt(((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1))
        iu, ju = np.triu_indices(n, 1)
        dist = d[iu, ju]
        # the n_und shortest pairs in ascending order (ties by pair index)
        sel = np.argpartition(dist, n_und - 1)[:n_und] if n_und < dist.size else np.arange(dist.size)
        order = sel[np.lexsort((sel, dist[sel]))]
        a, b = iu[order], ju[order]
        src = np.concatenate([a, b]).astype(np.int32)
        dst = np.concatenate([b, a]).astype(np.int32)
        r = float(dist[order[-1]])
        if connect == "bridge":
            label = _components(n, src, dst)
            extra_a, extra_b = [], []
            while label.max() > 0:
                sizes = np.bincount(label)
                small = int(np.argmin(sizes))
                inside = np.flatnonzero(label == small)
                outside = np.flatnonzero(label != small)
                sub = d[np.ix_(inside, outside)]
                k = int(np.argmin(sub))
                u, w = int(inside[k // outside.size]), int(outside[k % outside.size])
                extra_a.append(u)
                extra_b.append(w)
                label[label == small] = label[w]
                _, label = np.unique(label, return_inverse=True)
            if extra_a:
                ea, eb = np.asarray(extra_a, np.int32), np.asarray(extra_b, np.int32)
                src = np.concatenate([src, ea, eb]).astype(np.int32)
                dst = np.concatenate([dst, eb, ea]).astype(np.int32)
        elif not _connected(n, src, dst):
            continue
        # spatial renumbering: strips of width ~ radius, snake order inside
        nstrip = max(1, int(1.0 / max(r, 1e-3)))
        strip = np.minimum((pos[:, 1] * nstrip).astype(np.int64), nstrip - 1)
        key = np.where(strip % 2 == 0, pos[:, 0], -pos[:, 0])
        perm = np.lexsort((key, strip))          # new order -> old id
        inv = np.empty(n, np.int64)
        inv[perm] = np.arange(n)
        src2, dst2 = inv[src].astype(np.int32), inv[dst].astype(np.int32)
        eorder = np.lexsort((dst2, src2))
        length = np.sqrt(((pos[src] - pos[dst]) ** 2).sum(-1))
        return src2[eorder], dst2[eorder], pos[perm], length[eorder], r
    raise RuntimeError("could not draw a connected random geometric graph")


def hop_distances(n: int, src: np.ndarray, dst: np.ndarray, s: int) -> np.ndarray:
    """BFS hop distance from node s (-1 = unreachable)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    g = csr_matrix((np.ones(src.shape[0]), (src.astype(np.int64), dst.astype(np.int64))), shape=(n, n))
    d = shortest_path(g, method="D", unweighted=True, indices=int(s))
    out = np.full(n, -1, np.int64)
    ok = np.isfinite(d)
    out[ok] = d[ok].astype(np.int64)
    return out


def _od_pairs(n: int, src, dst, L: int, max_hops: int, rng, grid_cols: Optional[int] = None):
    """L origin-destination node pairs, uniform over pairs with 1 <= hops <= max_hops."""
    out = []
    cache = {}
    while len(out) < L:
        s = int(rng.integers(n))
        z = int(rng.integers(n))
        if s == z:
            continue
        if grid_cols is not None:
            hops = abs(s // grid_cols - z // grid_cols) + abs(s % grid_cols - z % grid_cols)
        else:
            if s not in cache:
                cache[s] = hop_distances(n, src, dst, s)
            hops = int(cache[s][z])
        if 1 <= hops <= max_hops:
            out.append((s, z))
    return out


def _single_pair_instance(name, n, src, dst, edge_cost, edge_cap, wait_cost, L, T, eps,
                          pairs, masses, pos=None, meta=None):
    E = src.shape[0]
    comm = np.arange(L, dtype=np.int32)
    s_state = np.asarray([E + s for s, _ in pairs], np.int32)
    z_state = np.asarray([E + z for _, z in pairs], np.int32)
    return Instance(
        name=name, n_nodes=n, edge_src=src, edge_dst=dst,
        edge_cost=np.asarray(edge_cost, np.float64), edge_cap=np.asarray(edge_cap, np.float64),
        wait_cost=np.full(n, wait_cost, np.float64), wait_cap=np.full(n, np.inf),
        L=L, T=T, eps=eps,
        src_comm=comm.copy(), src_state=s_state, src_mass=np.asarray(masses, np.float64),
        snk_comm=comm.copy(), snk_state=z_state, snk_mass=np.asarray(masses, np.float64).copy(),
        pos=pos, meta=dict(meta or {}))


# ----------------------------------------------------------------------------------
# workload recipes
# ----------------------------------------------------------------------------------

def grid_single_commodity(seed: int = 0, rows: int = 5, cols: int = 5, T: int = 10, eps: float = 0.05,
            move_cost: float = 1.0, wait_cost: float = 0.1, n_src: int = 3, n_snk: int = 3):
    """Single commodity on a grid: Dirichlet(1) sources and sinks over 3 nodes each."""
    rng = np.random.default_rng(seed)
    src, dst, pos = grid_graph(rows, cols)
    n, E = rows * cols, src.shape[0]
    s_nodes = rng.choice(n, n_src, replace=False)
    z_nodes = rng.choice(n, n_snk, replace=False)
    s_mass = rng.dirichlet(np.ones(n_src))
    z_mass = rng.dirichlet(np.ones(n_snk))
    return Instance(
        name=f"grid{rows}x{cols}-L1-T{T}", n_nodes=n, edge_src=src, edge_dst=dst,
        edge_cost=np.full(E, move_cost), edge_cap=np.full(E, np.inf),
        wait_cost=np.full(n, wait_cost), wait_cap=np.full(n, np.inf),
        L=1, T=T, eps=eps,
        src_comm=np.zeros(n_src, np.int32), src_state=(E + s_nodes).astype(np.int32),
        src_mass=s_mass.astype(np.float64),
        snk_comm=np.zeros(n_snk, np.int32), snk_state=(E + z_nodes).astype(np.int32),
        snk_mass=z_mass.astype(np.float64),
        pos=pos, meta={"workload": "grid5x5", "seed": seed})


def single_commodity_instance(seed: int = 0, rows: int = 6, cols: int = 6, T: int = 12, eps: float = 0.3,
                              n_src: int = 6, n_snk: int = 6, cap_scale: float = 0.08, per_interval: bool = True):
    """The single-commodity problem (eq. singlecommodity_reg) as an instance with L = 1: a grid
    with random move costs U[0.5, 1.5] and wait costs U[0, 0.3], initial and final distributions
    mu_1, mu_T (Dirichlet(1)) over random states (edges and wait loops), and moving-edge
    capacities cap_scale x U[0.5, 1.5] (per interval t = 2..T-1 when per_interval)."""
    rng = np.random.default_rng(seed)
    src, dst, pos = grid_graph(rows, cols)
    n, E = rows * cols, src.shape[0]
    S = n + E
    s_states = np.sort(rng.choice(S, n_src, replace=False)).astype(np.int32)
    z_states = np.sort(rng.choice(S, n_snk, replace=False)).astype(np.int32)
    inst = Instance(
        name=f"single{rows}x{cols}-T{T}", n_nodes=n, edge_src=src, edge_dst=dst,
        edge_cost=rng.uniform(0.5, 1.5, E), edge_cap=np.full(E, np.inf),
        wait_cost=rng.uniform(0.0, 0.3, n), wait_cap=np.full(n, np.inf),
        L=1, T=T, eps=eps,
        src_comm=np.zeros(n_src, np.int32), src_state=s_states, src_mass=rng.dirichlet(np.ones(n_src)),
        snk_comm=np.zeros(n_snk, np.int32), snk_state=z_states, snk_mass=rng.dirichlet(np.ones(n_snk)),
        pos=pos, meta={"seed": seed, "single_commodity": True})
    cap = np.concatenate([cap_scale * rng.uniform(0.5, 1.5, E), np.full(n, np.inf)])
    if per_interval:
        inst.state_capacity_t = cap[None, :] * rng.uniform(0.7, 1.3, (T - 2, S))
        inst.state_capacity_t[:, E:] = np.inf
    else:
        inst.edge_cap = cap[:E].copy()
    return inst


def rgg_instance(seed: int = 0, n: int = 400, L: int = 64, T: int = 50, eps: float = 0.01,
                 mean_degree: float = 6.0, wait_cost: float = 0.05, cap_lo: float = 0.2,
                 cap_hi: float = 1.0, cap_div: float = 8.0, name: Optional[str] = None,
                 connect: str = "reject"):
    """Random geometric graph, Euclidean edge costs, single-node OD pairs per commodity."""
    rng = np.random.default_rng(seed)
    src, dst, pos, length, r = rgg_graph(n, mean_degree, rng, connect=connect)
    pairs = _od_pairs(n, src, dst, L, T - 2, rng)
    mass = rng.uniform(0.5, 2.0, L)
    cap = rng.uniform(cap_lo, cap_hi, src.shape[0]) * mass.sum() / cap_div
    return _single_pair_instance(name or f"rgg{n}-L{L}-T{T}", n, src, dst, length, cap,
                                 wait_cost, L, T, eps, pairs, mass, pos,
                                 {"workload": "rgg", "seed": seed, "radius": r})


def rgg400(seed: int = 0):
    """Multi-commodity with capacities on a random geometric graph (n=400, L=64, T=50)."""
    return rgg_instance(seed=seed, n=400, L=64, T=50, eps=0.01)


def grid_traffic_instance(seed: int = 0, rows: int = 100, cols: int = 100, L: int = 1024,
                          T: int = 100, eps: float = 0.005, wait_cost: float = 0.2,
                          cap_lo: float = 0.5, cap_hi: float = 3.0, name: Optional[str] = None):
    """Perturbed grid road graph, Lognormal(0, 0.3) travel costs, uniform OD pairs."""
    rng = np.random.default_rng(seed)
    src, dst, pos = grid_graph(rows, cols)
    pos = pos + rng.uniform(-0.1, 0.1, pos.shape)
    E = src.shape[0]
    cost = rng.lognormal(0.0, 0.3, E)
    cap = rng.uniform(cap_lo, cap_hi, E)
    pairs = _od_pairs(rows * cols, src, dst, L, T - 2, rng, grid_cols=cols)
    mass = rng.uniform(0.1, 1.0, L)
    return _single_pair_instance(name or f"grid{rows}x{cols}-L{L}-T{T}", rows * cols, src, dst,
                                 cost, cap, wait_cost, L, T, eps, pairs, mass, pos,
                                 {"workload": "traffic_grid", "seed": seed})


def traffic_grid(seed: int = 0):
    """Traffic-scale: 100x100 grid, L=1024 OD commodities, T=100, eps=0.005."""
    return grid_traffic_instance(seed=seed)


def _uneven_rgg_member(args):
    k, n, T, L, sub = args
    inst = rgg_instance(seed=sub, n=n, L=L, T=T, eps=0.01, name=f"b{k}-rgg{n}-L{L}-T{T}", connect="bridge")
    inst.meta.update({"workload": "uneven_rgg_batch", "batch_index": k})
    return inst


def uneven_rgg_batch(seed: int = 0, count: int = 256, workers: int = 1):
    """Batch of uneven instances: n~U{50..2000} RGG (bridged to be connected), T~U{10..80},
    L~U{1..128}.  The sizes and sub-seeds are drawn first, so `workers` > 1 (a spawn process
    pool) gives the same instances."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(count):
        n = int(rng.integers(50, 2001))
        T = int(rng.integers(10, 81))
        L = int(rng.integers(1, 129))
        sub = int(rng.integers(2**31 - 1))
        specs.append((k, n, T, L, sub))
    if workers <= 1:
        return [_uneven_rgg_member(s) for s in specs]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_uneven_rgg_member, specs, chunksize=4))


def _uneven_single_member(args):
    k, n, T, sub = args
    inst = rgg_instance(seed=sub, n=n, L=1, T=T, eps=0.01, cap_div=2.0, name=f"s{k}-rgg{n}-L1-T{T}", connect="bridge")
    inst.meta.update({"workload": "uneven_single_batch", "batch_index": k})
    return inst


def uneven_single_batch(seed: int = 0, count: int = 64, workers: int = 1):
    """Single-commodity members with the sizes of the uneven batch: n~U{50..2000} RGG (bridged),
    T~U{10..80}, L = 1, eps = 0.01, one OD pair of mass U[0.5, 2].  Capacities U[0.2,1] * mass / 2:
    with one commodity, mass / 8 is below the cut the commodity has to cross and most instances
    would admit no feasible flow; mass / 2 binds on the busiest edges and leaves most feasible."""
    rng = np.random.default_rng(seed)
    specs = [(k, int(rng.integers(50, 2001)), int(rng.integers(10, 81)), int(rng.integers(2**31 - 1)))
             for k in range(count)]
    if workers <= 1:
        return [_uneven_single_member(s) for s in specs]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_uneven_single_member, specs, chunksize=4))


def with_time_varying_costs(inst, seed: int = 0, lo: float = 0.5, hi: float = 2.0, closures: int = 0):
    """A time-varying network for an instance (Section 3.3, C_t): the per-interval cost of every
    state is its static cost times U[lo, hi], drawn per (t, state) for t = 2..T-1, and
    `closures` random moving edges are closed (+inf) during one random interval each."""
    rng = np.random.default_rng(seed)
    base = inst.state_cost()
    ct = base[None, :] * rng.uniform(lo, hi, (inst.T - 2, base.size))
    for _ in range(closures):
        ct[rng.integers(inst.T - 2), rng.integers(inst.n_edges)] = np.inf
    inst.state_cost_t = ct
    return inst


def with_time_varying_capacities(inst, seed: int = 0, lo: float = 0.5, hi: float = 1.5, closures: int = 0):
    """Per-interval capacities d_t (the capacity vectors of the problem statements, one per
    interval t = 2..T-1): each finite capacity times U[lo, hi], drawn per (t, state), and
    `closures` random moving edges given capacity 0 in one random interval each."""
    rng = np.random.default_rng(seed)
    base = np.concatenate([inst.edge_cap, inst.wait_cap]).astype(np.float64)
    dt = np.tile(base, (inst.T - 2, 1))
    fin = np.isfinite(dt)
    dt[fin] *= rng.uniform(lo, hi, int(fin.sum()))
    for _ in range(closures):
        dt[rng.integers(inst.T - 2), rng.integers(inst.n_edges)] = 0.0
    inst.state_capacity_t = dt
    return inst


def with_commodity_windows(inst, seed: int = 0, slack: int = 1):
    """Entry and exit times per commodity (the multi-tensor scheme of the Remark after
    Algorithm 2) for an instance with one source and one sink node per commodity (on the wait
    loops): a window needs at least hops + 1 transitions (hops = hop distance from the source
    node to the sink node); with m = hops + 1 + slack (capped at T - 1), t_in is uniform on
    1..T-m and t_out uniform on t_in+m..T."""
    rng = np.random.default_rng(seed)
    E = inst.n_edges
    a = np.ones(inst.L, np.int32)
    b = np.full(inst.L, inst.T, np.int32)
    dist = {}
    for k in range(len(inst.src_comm)):
        l = int(inst.src_comm[k])
        s_node = int(inst.src_state[k]) - E
        z = [int(inst.snk_state[q]) - E for q in range(len(inst.snk_comm)) if inst.snk_comm[q] == l]
        if s_node not in dist:
            dist[s_node] = hop_distances(inst.n_nodes, inst.edge_src, inst.edge_dst, s_node)
        hops = max(int(dist[s_node][zn]) for zn in z)
        m = min(hops + 1 + slack, inst.T - 1)
        a[l] = rng.integers(1, inst.T - m + 1)
        b[l] = rng.integers(a[l] + m, inst.T + 1)
    inst.commodity_t_in = a
    inst.commodity_t_out = b
    return inst


def traffic_routing_instance(seed: int = 0, rows: int = 4, cols: int = 4, L: int = 3, T: int = 8, eps: float = 0.1,
                             cap_lo: float = 0.2, cap_hi: float = 0.6, edge_storage: bool = False):
    """The traffic-routing state model of eq. cost_traffic_routing on a grid: states are the
    directed streets plus, per commodity, a source state at its origin node (nothing enters it;
    agents may stay) and a sink state at its destination node (nothing leaves it; agents stay).
    The wait loops of the street nodes are closed (no storage at junctions).  With
    edge_storage, agents may also stay on a street (storage on edges, Section 3.3; the street's
    per-interval cost accumulates).  Layout: nodes 0..V-1 are the junctions, node V + 2 l the
    source and node V + 2 l + 1 the sink of commodity l; state E + w is the state of node w."""
    rng = np.random.default_rng(seed)
    src, dst, pos = grid_graph(rows, cols)
    V, E = rows * cols, src.shape[0]
    Vx = V + 2 * L
    od = []
    while len(od) < L:
        o, z = rng.choice(V, 2, replace=False)
        h = int(hop_distances(V, src, dst, int(o))[int(z)])
        if 1 <= h <= T - 2:
            od.append((int(o), int(z)))
    mass = rng.uniform(0.5, 1.5, L)
    tail = np.concatenate([src, np.full(Vx, -1)]).astype(np.int32)
    head = np.concatenate([dst, np.full(Vx, -1)]).astype(np.int32)
    hold = np.zeros(E + Vx, np.int32)
    if edge_storage:
        hold[:E] = 1
    for l, (o, z) in enumerate(od):
        s_src, s_snk = E + V + 2 * l, E + V + 2 * l + 1
        head[s_src] = o                   # a source leads onto the streets leaving its origin
        tail[s_snk] = z                   # a sink is reached from the streets entering its destination
        hold[s_src] = hold[s_snk] = 1
    edge_cost = rng.uniform(0.5, 1.5, E)
    edge_cap = rng.uniform(cap_lo, cap_hi, E) * mass.sum() / 4.0
    inst = Instance(
        name=f"traffic-routing{rows}x{cols}-L{L}-T{T}", n_nodes=Vx, edge_src=src, edge_dst=dst,
        edge_cost=edge_cost, edge_cap=edge_cap, wait_cost=np.zeros(Vx), wait_cap=np.full(Vx, np.inf),
        L=L, T=T, eps=eps,
        src_comm=np.arange(L, dtype=np.int32), src_state=(E + V + 2 * np.arange(L)).astype(np.int32),
        src_mass=mass.astype(np.float64),
        snk_comm=np.arange(L, dtype=np.int32), snk_state=(E + V + 2 * np.arange(L) + 1).astype(np.int32),
        snk_mass=mass.astype(np.float64),
        pos=None, meta={"workload": "traffic_routing", "seed": seed, "od": od})
    inst.state_tail, inst.state_head, inst.state_hold = tail, head, hold
    return inst


WORKLOADS = {"grid5x5": grid_single_commodity, "rgg400": rgg400, "traffic_grid": traffic_grid,
             "uneven_rgg_batch": uneven_rgg_batch}

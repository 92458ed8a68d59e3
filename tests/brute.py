"""Independent references used to pin the oracle (tests only).

Nothing here reuses the oracle's code.  Each function computes a quantity straight from
its definition in the paper:

* :func:`brute_force` - Section 1: enumerate every simple path between A and B and take
  the smallest F1 among those with F2 < M (ties: smallest F2, then smallest endpoint X,
  then the smallest (second-to-last vertex, direction) for the last edge x).
* :func:`pareto_trace` - the trace implied by the flow semantics, from per-vertex
  (F1, F2) Pareto frontiers of all simple paths: label L_t(v) = max over paths reaching v
  by time t of M - F2; a flow leaves v along (v, u) at every time t0 at which L(v)
  improves and is alive at the end of cycle T iff t0 <= T < t0 + f1 and
  L_t0(v) - f2 > L_T(u).
* :func:`phantoms` - the flows started on an edge that already carries one, from the same
  label histories (the paper's phantom edges, Step 5).
* :func:`dijkstra_trace` - for f2 = 0 the problem is first-passage percolation: F1 is the
  Dijkstra distance tau (computed by scipy) and the state at time T is {tau <= T};
  :func:`first_passage_row` gives one row of that trace.
"""
from __future__ import annotations

import collections
from typing import Dict, List, Sequence, Tuple

import numpy as np


def directed_edges(extents: Sequence[int], f1, f2):
    """{v: [(u, dir, f1, f2), ...]} from coordinates (dir = 2k + s, s=1 means -e_k)."""
    ext = [int(n) for n in extents]
    d = len(ext)
    V = int(np.prod(ext))
    f1 = np.asarray(f1).reshape(d, V).astype(np.int64)
    f2 = np.asarray(f2).reshape(d, V).astype(np.int64)
    idx = np.indices(ext[::-1]).reshape(d, -1)[::-1]  # idx[k][v] = c_k of vertex v (c_0 fastest)
    strides = np.cumprod([1] + ext[:-1])
    adj: Dict[int, list] = collections.defaultdict(list)
    for v in range(V):
        for k in range(d):
            c = idx[k][v]
            if c + 1 < ext[k] and f1[k, v] > 0:
                u = v + strides[k]
                adj[v].append((u, 2 * k, int(f1[k, v]), int(f2[k, v])))
                adj[u].append((v, 2 * k + 1, int(f1[k, v]), int(f2[k, v])))
    for v in adj:
        adj[v].sort(key=lambda e: e[1])
    return adj, V


def graph_directed_edges(nbr, f1, f2):
    """{v: [(u, slot, f1, f2), ...]} from adjacency slots (nbr = -1: empty slot)."""
    nbr = np.asarray(nbr)
    V, S = nbr.shape
    f1 = np.asarray(f1).reshape(V, S)
    f2 = np.asarray(f2).reshape(V, S)
    adj: Dict[int, list] = collections.defaultdict(list)
    for v in range(V):
        for j in range(S):
            if nbr[v, j] >= 0:
                adj[v].append((int(nbr[v, j]), j, int(f1[v, j]), int(f2[v, j])))
    return adj, V


def adjacency(inst):
    """The directed edges of a lattice instance (extents) or a graph instance (nbr)."""
    if hasattr(inst, "nbr"):
        return graph_directed_edges(inst.nbr, inst.f1, inst.f2)
    return directed_edges(inst.extents, inst.f1, inst.f2)


def all_simple_paths(inst):
    """Yield (end, F1, F2, prev, dir) for every simple path starting in A (length >= 0)."""
    adj, V = adjacency(inst)
    for a in sorted(set(int(x) for x in inst.A)):
        yield (a, 0, 0, -1, -1)
        on_path = {a}
        stack = [(a, 0, 0, iter(adj.get(a, ())))]
        while stack:
            v, t, w, it = stack[-1]
            nxt = next(it, None)
            if nxt is None:
                stack.pop()
                on_path.discard(v)
                continue
            u, dr, t1, w1 = nxt
            if u in on_path:
                continue
            yield (u, t + t1, w + w1, v, dr)
            on_path.add(u)
            stack.append((u, t + t1, w + w1, iter(adj.get(u, ()))))


def brute_force(inst) -> Tuple[int, int, int, int, int]:
    """(F1, X, x_src, x_dir, F2) by exhaustive enumeration; all -1 if infeasible."""
    Bset = set(int(b) for b in inst.B)
    best = None
    for end, t, w, prev, dr in all_simple_paths(inst):
        if end in Bset and w < inst.M and prev >= 0:
            key = (t, w, end, prev, dr)
            if best is None or key < best:
                best = key
    if best is None:
        return (-1, -1, -1, -1, -1)
    t, w, end, prev, dr = best
    return (t, end, prev, dr, w)


def label_histories(inst):
    """Per vertex, the times and labels at which its label improves (A: M at time 0), from
    the (F1, F2) of all simple paths; the time F1 of the first improvement of a B vertex
    (None if none)."""
    M = int(inst.M)
    adj, V = adjacency(inst)
    Aset = set(int(a) for a in inst.A)
    Bset = set(int(b) for b in inst.B)
    arrivals: Dict[int, List[Tuple[int, int]]] = collections.defaultdict(list)
    for end, t, w, _, _ in all_simple_paths(inst):
        if M - w > 0:
            arrivals[end].append((t, M - w))
    improvements: Dict[int, List[Tuple[int, int]]] = {}
    for v in range(V):
        if v in Aset:
            improvements[v] = [(0, M)] if M > 0 else []
            continue
        hist, cur = [], 0
        for t, q in sorted(arrivals.get(v, [])):
            if q > cur:
                if hist and hist[-1][0] == t:
                    hist[-1] = (t, q)
                else:
                    hist.append((t, q))
                cur = q
        improvements[v] = hist
    F1 = min((improvements[b][0][0] for b in Bset if improvements[b]), default=None)
    return adj, V, improvements, F1


def phantoms(inst) -> int:
    """Flows started on a directed edge that already carries one (the paper's phantom edges,
    Step 5): a launch from v along (v, u) at time t0 (v improves at t0 and its new label
    minus f2 beats Label(u) at the end of t0) is a phantom if an earlier launch on (v, u) at
    t1 has not arrived (t1 + f1 > t0) and survived the removals up to the cycle before t0
    (its quality minus f2 still beats Label(u) there).  Launches happen up to F1."""
    adj, V, improvements, F1 = label_histories(inst)

    def label_at(v, T):
        lab = 0
        for t, q in improvements[v]:
            if t <= T:
                lab = q
        return lab

    n = 0
    for v in range(V):
        for u, _, t1, w1 in adj.get(v, ()):
            launches = [(t0, q0) for t0, q0 in improvements[v]
                        if (F1 is None or t0 <= F1) and q0 - w1 > label_at(u, t0)]
            for i, (t0, _) in enumerate(launches):
                if any(ta + t1 > t0 and qa - w1 > label_at(u, t0 - 1) for ta, qa in launches[:i]):
                    n += 1
    return n


def pareto_trace(inst) -> np.ndarray:
    """(rows, 3) trace (Time, active vertices, flows) implied by the flow semantics."""
    M = int(inst.M)
    adj, V = adjacency(inst)
    Aset = set(int(a) for a in inst.A)
    Bset = set(int(b) for b in inst.B)
    arrivals: Dict[int, List[Tuple[int, int]]] = collections.defaultdict(list)
    for end, t, w, _, _ in all_simple_paths(inst):
        if M - w > 0:
            arrivals[end].append((t, M - w))
    # label history: improvements (time, new label) per vertex; A starts at M at time 0
    improvements: Dict[int, List[Tuple[int, int]]] = {}
    for v in range(V):
        if v in Aset:
            improvements[v] = [(0, M)] if M > 0 else []
            continue
        pts = sorted(arrivals.get(v, []))
        hist, cur = [], 0
        for t, q in pts:
            if q > cur:
                if hist and hist[-1][0] == t:
                    hist[-1] = (t, q)
                else:
                    hist.append((t, q))
                cur = q
        improvements[v] = hist

    def label_at(v, T):
        lab = 0
        for t, q in improvements[v]:
            if t <= T:
                lab = q
        return lab

    # cycle times: every improvement time >= 1, cut at the first time a B vertex improves
    times = sorted({t for v in range(V) for t, _ in improvements[v] if t >= 1})
    F1 = min((improvements[b][0][0] for b in Bset if improvements[b]), default=None)
    if F1 is not None:
        times = [t for t in times if t <= F1]
    rows = []
    for T in [0] + times:
        srcs, n = set(), 0
        for v in range(V):
            for t0, q0 in improvements[v]:
                if t0 > T:
                    continue
                for u, _, t1, w1 in adj.get(v, ()):
                    if T < t0 + t1 and q0 - w1 > label_at(u, t0) and q0 - w1 > label_at(u, T):
                        n += 1
                        srcs.add(v)
        rows.append((T, len(srcs), n))
    return np.array(rows, dtype=np.int64).reshape(-1, 3)


def tau(extents, f1, A) -> np.ndarray:
    """Multi-source first-passage times (plain Dijkstra from scipy); inf if unreachable."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import dijkstra

    ext = [int(n) for n in extents]
    d = len(ext)
    V = int(np.prod(ext))
    f1 = np.asarray(f1).reshape(d, V).astype(np.float64)
    v = np.arange(V)
    strides = np.cumprod([1] + ext[:-1])
    rows, cols, vals = [], [], []
    for k in range(d):
        ck = (v // strides[k]) % ext[k]
        ok = (ck + 1 < ext[k]) & (f1[k] > 0)
        src, dst = v[ok], v[ok] + strides[k]
        rows += [src, dst]
        cols += [dst, src]
        vals += [f1[k][ok], f1[k][ok]]
    G = coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(V, V)).tocsr()
    return dijkstra(G, directed=True, indices=np.asarray(A, dtype=np.int64), min_only=True)


def _edge_pairs(ext, f1):
    """(src, dst) of every directed edge present (f1 > 0), from coordinates."""
    d = len(ext)
    V = int(np.prod(ext))
    f1a = np.asarray(f1).reshape(d, V)
    v = np.arange(V)
    strides = np.cumprod([1] + ext[:-1])
    pairs = []
    for k in range(d):
        ck = (v // strides[k]) % ext[k]
        ok = (ck + 1 < ext[k]) & (f1a[k] > 0)
        pairs.append((v[ok], v[ok] + strides[k]))
        pairs.append((v[ok] + strides[k], v[ok]))
    return np.concatenate([p[0] for p in pairs]), np.concatenate([p[1] for p in pairs])


def first_passage_row(extents, f1, t, T):
    """Trace row (T, active vertices, live flows) at the end of cycle T for f2 = 0, from the
    first-passage times t: a directed edge (v, u) carries a live flow iff
    t(v) <= T < t(u), and v is active iff it has such an edge."""
    src, dst = _edge_pairs([int(n) for n in extents], f1)
    live = (t[src] <= T) & (t[dst] > T)
    return (int(T), len(np.unique(src[live])), int(live.sum()))


def dijkstra_trace(extents, f1, A, B):
    """For f2 = 0: (F1, X, x candidates, trace) from first-passage times.

    F1 = min tau over B; X = smallest id attaining it; the cycle times are the distinct
    tau values in (0, F1]; the row of cycle T is :func:`first_passage_row`.
    """
    ext = [int(n) for n in extents]
    t = tau(ext, f1, A)
    Bv = np.asarray(B, dtype=np.int64)
    tb = t[Bv]
    F1 = np.min(tb)
    if not np.isfinite(F1):
        F1 = None
    src, dst = _edge_pairs(ext, f1)
    finite = t[np.isfinite(t)]
    times = np.unique(finite[finite > 0])
    if F1 is not None:
        times = times[times <= F1]
    rows = []
    for T in [0.0] + list(times):
        live = (t[src] <= T) & (t[dst] > T)
        rows.append((int(T), len(np.unique(src[live])), int(live.sum())))
    X = int(Bv[tb == F1].min()) if F1 is not None else -1
    return (int(F1) if F1 is not None else -1), X, t, np.array(rows, dtype=np.int64)


def graph_tau(nbr, f1, A) -> np.ndarray:
    """Multi-source first-passage times on a graph given by adjacency slots (scipy)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import dijkstra

    nbr = np.asarray(nbr)
    V, S = nbr.shape
    ok = nbr >= 0
    src = np.repeat(np.arange(V), S).reshape(V, S)[ok]
    G = coo_matrix((np.asarray(f1).reshape(V, S)[ok].astype(np.float64), (src, nbr[ok])), shape=(V, V)).tocsr()
    return dijkstra(G, directed=True, indices=np.asarray(A, dtype=np.int64), min_only=True)


def graph_dijkstra_trace(nbr, f1, A, B):
    """:func:`dijkstra_trace` on a graph given by adjacency slots (f2 = 0)."""
    nbr = np.asarray(nbr)
    V, S = nbr.shape
    t = graph_tau(nbr, f1, A)
    Bv = np.asarray(B, dtype=np.int64)
    F1 = np.min(t[Bv])
    ok = nbr >= 0
    src = np.repeat(np.arange(V), S).reshape(V, S)[ok]
    dst = nbr[ok]
    finite = t[np.isfinite(t)]
    times = np.unique(finite[finite > 0])
    if np.isfinite(F1):
        times = times[times <= F1]
    rows = []
    for T in [0.0] + list(times):
        live = (t[src] <= T) & (t[dst] > T)
        rows.append((int(T), len(np.unique(src[live])), int(live.sum())))
    X = int(Bv[t[Bv] == F1].min()) if np.isfinite(F1) else -1
    return (int(F1) if np.isfinite(F1) else -1), X, t, np.array(rows, dtype=np.int64)

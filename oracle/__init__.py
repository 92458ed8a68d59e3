"""CPU oracle for the water-flow constrained shortest path method (arXiv 1511.06441).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` import this package.  The product (``paper_1511_06441_gb300``)
never imports it, and it imports nothing from the product.

The solvers live in ``csp_oracle.c`` (plain C, compiled here with gcc on first use):

* :func:`cycle`  - O1, the paper's cycle loop (Algorithm 1, Steps 1-9), with trace;
* :func:`pareto` - O2, an independent Dijkstra over (vertex, quality) states;
* :func:`lexmin` - unconstrained lexicographic (F1, F2) Dijkstra (the bound M of the
  anti-correlated workload, and its answer where that bound does not bind);
* :func:`cycle_graph`, :func:`pareto_graph`, :func:`reconstruct_graph` - O1, O2 and the
  repeated application on a general graph given by adjacency slots;
* :func:`calendar`, :func:`calendar_graph` - O4, O1's loop reorganised around events
  (per-edge queues, time buckets): a cross-check of O1 and of that reorganisation, with
  event counts.

Parity unpinned: nothing.  Every output is pinned by the tests against brute force,
plain Dijkstra, closed forms or the paper's Lemma; see the C file's header.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, OOM, TIMEOUT = 0, 1, 2, 5


def build(force: bool = False) -> str:
    """Compile ``csp_oracle.c`` into ``liboracle.so`` (gcc -O2, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_cycle.argtypes = [ctypes.c_int, i64p, i32p, i32p, i64p, ctypes.c_int64, i64p,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, i64p,
                                         i64p, ctypes.c_int64, i64p, ctypes.c_int64, i64p, i64p, i64p,
                                         ctypes.c_void_p]
            lib.oracle_pareto.argtypes = [ctypes.c_int, i64p, i32p, i32p, i64p, ctypes.c_int64, i64p,
                                          ctypes.c_int64, ctypes.c_int64, i64p]
            lib.oracle_lexmin.argtypes = [ctypes.c_int, i64p, i32p, i32p, i64p, ctypes.c_int64, i64p,
                                          ctypes.c_int64, i64p, i64p, ctypes.c_int64, i64p]
            lib.oracle_calendar.argtypes = [ctypes.c_int, i64p, i32p, i32p, i64p, ctypes.c_int64, i64p,
                                            ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, i64p, i64p,
                                            ctypes.c_int64, i64p, ctypes.c_void_p]
            lib.oracle_calendar_graph.argtypes = [ctypes.c_int64, ctypes.c_int, i64p] + lib.oracle_calendar.argtypes[2:]
            lib.oracle_cycle_graph.argtypes = [ctypes.c_int64, ctypes.c_int, i64p] + lib.oracle_cycle.argtypes[2:]
            lib.oracle_pareto_graph.argtypes = [ctypes.c_int64, ctypes.c_int, i64p] + lib.oracle_pareto.argtypes[2:]
            for f in (lib.oracle_cycle, lib.oracle_pareto, lib.oracle_lexmin, lib.oracle_cycle_graph,
                      lib.oracle_pareto_graph, lib.oracle_calendar, lib.oracle_calendar_graph):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle returned status {code}")
        self.code = code


@dataclasses.dataclass
class Result:
    F1: int
    X: int
    x_src: int
    x_dir: int
    F2: int
    cycles: int = -1
    updates: int = -1          # sum over cycles of the flows alive at cycle start
    launched: int = -1         # flows started (including phantoms)
    phantoms: int = -1         # flows started on a directed edge that already carried one (O1 only)
    trace: Optional[np.ndarray] = None     # (rows, 3) int64: Time, active vertices, flows
    labels: Optional[np.ndarray] = None    # (V,) int64 labels at termination
    snapshot: Optional[np.ndarray] = None  # active vertex ids at the requested time

    def answer(self):
        return (self.F1, self.X, self.x_src, self.x_dir, self.F2)


def _common(extents, f1, f2, A, B):
    ext = np.ascontiguousarray(np.asarray(extents, dtype=np.int64))
    f1 = np.ascontiguousarray(np.asarray(f1).astype(np.int32).reshape(-1))
    f2 = np.ascontiguousarray(np.asarray(f2).astype(np.int32).reshape(-1))
    A = np.ascontiguousarray(np.asarray(A, dtype=np.int64).reshape(-1))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.int64).reshape(-1))
    return ext, f1, f2, A, B


def cycle(extents: Sequence[int], f1, f2, A, B, M: int, *, max_cycles: int = 1 << 62,
          trace: bool = True, labels: bool = False, snap_time: Optional[int] = None,
          allow_timeout: bool = False, removed=None) -> Result:
    """O1: the paper's cycle loop.  Raises :class:`OracleError` on a non-OK status.

    With ``allow_timeout`` a run stopped by ``max_cycles`` returns its work counts
    (``cycles``, ``updates``, ``launched``) with ``F1 = -2`` instead of raising.
    """
    ext, f1, f2, A, B = _common(extents, f1, f2, A, B)
    V = int(np.prod(ext))
    return _cycle(lambda *rest: _load().oracle_cycle(len(ext), _p64(ext), _p32(f1), _p32(f2), *rest), V, A, B, M,
                  max_cycles, trace, labels, snap_time, allow_timeout, removed)


def _graph_arrays(nbr, f1, f2):
    nbr = np.ascontiguousarray(np.asarray(nbr, dtype=np.int64))
    V, S = nbr.shape
    f1 = np.ascontiguousarray(np.asarray(f1).astype(np.int32).reshape(V, S))
    f2 = np.ascontiguousarray(np.asarray(f2).astype(np.int32).reshape(V, S))
    return nbr, f1, f2, V, S


def cycle_graph(nbr, f1, f2, A, B, M: int, *, max_cycles: int = 1 << 62, trace: bool = True,
                labels: bool = False, snap_time: Optional[int] = None, allow_timeout: bool = False,
                removed=None) -> Result:
    """O1 on a general graph: ``nbr`` (V, S) neighbour ids (-1: empty slot), ``f1``/``f2``
    (V, S) the edge in each slot; x_dir is the slot of x at x_src."""
    nbr, f1, f2, V, S = _graph_arrays(nbr, f1, f2)
    A = np.ascontiguousarray(np.asarray(A, dtype=np.int64).reshape(-1))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.int64).reshape(-1))
    return _cycle(lambda *rest: _load().oracle_cycle_graph(V, S, _p64(nbr), _p32(f1), _p32(f2), *rest), V, A, B,
                  M, max_cycles, trace, labels, snap_time, allow_timeout, removed)


def _cycle(call, V, A, B, M, max_cycles, trace, labels, snap_time, allow_timeout, removed) -> Result:
    rem = None
    if removed is not None:
        rem = np.zeros(V, np.uint8)
        rem[np.asarray(removed, dtype=np.int64)] = 1
    res = np.zeros(9, np.int64)
    cap = 1 << 12
    while True:
        tr = np.zeros(3 * cap if trace else 3, np.int64)
        tl = np.zeros(1, np.int64)
        snap = np.zeros(V, np.int64) if snap_time is not None else None
        sl = np.zeros(1, np.int64)
        lab = np.zeros(V, np.int64) if labels else None
        rc = call(_p64(A), A.size, _p64(B), B.size, int(M), int(max_cycles), _p64(res), _p64(tr),
                  cap if trace else 0, _p64(tl), -1 if snap_time is None else int(snap_time),
                  _p64(snap) if snap is not None else None, _p64(sl), _p64(lab) if lab is not None else None,
                  rem.ctypes.data if rem is not None else None)
        if rc == TIMEOUT and allow_timeout:
            res[:5] = -2
        elif rc != OK:
            raise OracleError(rc)
        if not trace or tl[0] <= cap:
            break
        cap = int(tl[0])
    return Result(*[int(x) for x in res[:9]],
                  trace=tr[: 3 * int(tl[0])].reshape(-1, 3) if trace else None,
                  labels=lab,
                  snapshot=snap[: int(sl[0])] if snap is not None else None)


def edge_weight(extents: Sequence[int], f1, f2, v: int, direction: int):
    """(f1, f2) of the edge leaving v in direction 2k + s (s = 1: towards -e_k)."""
    ext = [int(n) for n in extents]
    d, V = len(ext), int(np.prod(ext))
    k, s = direction // 2, direction % 2
    stride = int(np.prod(ext[:k]))
    slot = k * V + (v - stride if s else v)
    return int(np.asarray(f1).reshape(-1)[slot]), int(np.asarray(f2).reshape(-1)[slot])


def reconstruct(extents: Sequence[int], f1, f2, A, B, M: int, first: Optional[Result] = None,
                max_steps: int = 1 << 30):
    """The minimizing path by repeated application (Section 1), with the reading
    B' = {Y}, M' = F2 - f2(x) + 1, V' = V minus (B and the path vertices found so far),
    A' = A, until Y is in A.  Returns (path from A to X, per-step results), or
    (None, [first]) when infeasible.  Each step is a full O1 solve."""
    return _reconstruct(lambda **kw: cycle(extents, f1, f2, **kw),
                        lambda y, d: edge_weight(extents, f1, f2, y, d)[1], A, B, M, first, max_steps)


def _reconstruct(solve, weight_of_x, A, B, M, first, max_steps):
    r = first if first is not None else solve(A=A, B=B, M=M, trace=False)
    steps = [r]
    if r.F1 < 0:
        return None, steps
    Aset = set(int(a) for a in np.asarray(A).reshape(-1))
    Bset = set(int(b) for b in np.asarray(B).reshape(-1))
    path = [r.X]
    F2, Y, xd, X = r.F2, r.x_src, r.x_dir, r.X
    while Y not in Aset and len(steps) <= max_steps:
        w2 = weight_of_x(Y, xd)
        removed = sorted(Bset | set(path))
        r = solve(A=A, B=[Y], M=F2 - w2 + 1, trace=False, removed=removed)
        steps.append(r)
        if r.F1 < 0 or r.X != Y:
            raise RuntimeError("repeated application lost the path")
        path.append(Y)
        F2, Y, xd = r.F2, r.x_src, r.x_dir
    path.append(Y)
    return path[::-1], steps


def pareto(extents: Sequence[int], f1, f2, A, B, M: int) -> Result:
    """O2: Dijkstra over (vertex, quality) states with dominance pruning."""
    lib = _load()
    ext, f1, f2, A, B = _common(extents, f1, f2, A, B)
    res = np.zeros(8, np.int64)
    rc = lib.oracle_pareto(len(ext), _p64(ext), _p32(f1), _p32(f2), _p64(A), A.size, _p64(B), B.size,
                           int(M), _p64(res))
    if rc != OK:
        raise OracleError(rc)
    r = Result(*[int(x) for x in res[:5]])
    r.updates = int(res[6])
    r.launched = int(res[7])
    return r


def pareto_graph(nbr, f1, f2, A, B, M: int) -> Result:
    """O2 on a general graph (arrays as in :func:`cycle_graph`)."""
    nbr, f1, f2, V, S = _graph_arrays(nbr, f1, f2)
    A = np.ascontiguousarray(np.asarray(A, dtype=np.int64).reshape(-1))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.int64).reshape(-1))
    res = np.zeros(8, np.int64)
    rc = _load().oracle_pareto_graph(V, S, _p64(nbr), _p32(f1), _p32(f2), _p64(A), A.size, _p64(B), B.size,
                                     int(M), _p64(res))
    if rc != OK:
        raise OracleError(rc)
    r = Result(*[int(x) for x in res[:5]])
    r.updates = int(res[6])
    r.launched = int(res[7])
    return r


def reconstruct_graph(nbr, f1, f2, A, B, M: int, first: Optional[Result] = None, max_steps: int = 1 << 30):
    """:func:`reconstruct` on a general graph: f2(x) is the weight in slot x_dir of x_src."""
    f2a = np.asarray(f2).reshape(np.asarray(nbr).shape)
    return _reconstruct(lambda **kw: cycle_graph(nbr, f1, f2, **kw), lambda y, d: int(f2a[y, d]), A, B, M, first,
                        max_steps)


def lexmin(extents: Sequence[int], f1, f2, A, B, *, full: bool = False, path: bool = False):
    """Lexicographically smallest (F1, F2) over walks from A to B, no weight bound.

    ``full`` adds X and the last edge (x_src, x_dir) under the solver's tie rules; when the
    returned F2 is below a bound M, (F1, F2, X, x) is the answer for that M.  ``path``
    returns ``(F1, F2, X, x_src, x_dir, vertices)`` with the walk itself (A end first): each
    vertex's settled predecessor, i.e. its own lexicographically smallest prefix.
    """
    lib = _load()
    ext, f1, f2, A, B = _common(extents, f1, f2, A, B)
    res = np.zeros(5, np.int64)
    n = np.zeros(1, np.int64)
    buf = np.zeros(1, np.int64)
    for _ in range(2):
        rc = lib.oracle_lexmin(len(ext), _p64(ext), _p32(f1), _p32(f2), _p64(A), A.size, _p64(B), B.size,
                               _p64(res), _p64(buf) if path else None, buf.size if path else 0,
                               _p64(n) if path else None)
        if rc != OK:
            raise OracleError(rc)
        if not path or n[0] <= buf.size:
            break
        buf = np.zeros(int(n[0]), np.int64)
    if path:
        return tuple(int(x) for x in res) + ([int(v) for v in buf[: int(n[0])]] if res[0] >= 0 else None,)
    if full:
        return tuple(int(x) for x in res)
    return int(res[0]), int(res[1])


CALENDAR_EVENTS = ("arrivals", "stale_entries", "pushes", "removals", "fronts_checked")


def _calendar(call, V, A, B, M, max_cycles, labels):
    res = np.zeros(14, np.int64)
    cap = 1 << 12
    while True:
        tr = np.zeros(3 * cap, np.int64)
        tl = np.zeros(1, np.int64)
        lab = np.zeros(V, np.int64) if labels else None
        rc = call(_p64(A), A.size, _p64(B), B.size, int(M), int(max_cycles), _p64(res), _p64(tr), cap, _p64(tl),
                  lab.ctypes.data if lab is not None else None)
        if rc != OK:
            raise OracleError(rc)
        if tl[0] <= cap:
            break
        cap = int(tl[0])
    r = Result(*[int(x) for x in res[:9]], trace=tr[: 3 * int(tl[0])].reshape(-1, 3), labels=lab)
    r.events = dict(zip(CALENDAR_EVENTS, (int(x) for x in res[9:14])))
    return r


def calendar(extents: Sequence[int], f1, f2, A, B, M: int, *, max_cycles: int = 1 << 62,
             labels: bool = False) -> Result:
    """O4: the cycle loop driven by events (per-edge flow queues and arrival-time buckets).
    Same outputs as :func:`cycle` (with trace) plus ``events``: the counts of arrivals,
    stale bucket entries, flows pushed, removals and queue fronts inspected."""
    ext, f1, f2, A, B = _common(extents, f1, f2, A, B)
    V = int(np.prod(ext))
    return _calendar(lambda *rest: _load().oracle_calendar(len(ext), _p64(ext), _p32(f1), _p32(f2), *rest), V, A, B,
                     M, max_cycles, labels)


def calendar_graph(nbr, f1, f2, A, B, M: int, *, max_cycles: int = 1 << 62, labels: bool = False) -> Result:
    """O4 on a general graph (arrays as in :func:`cycle_graph`)."""
    nbr, f1, f2, V, S = _graph_arrays(nbr, f1, f2)
    A = np.ascontiguousarray(np.asarray(A, dtype=np.int64).reshape(-1))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.int64).reshape(-1))
    return _calendar(lambda *rest: _load().oracle_calendar_graph(V, S, _p64(nbr), _p32(f1), _p32(f2), *rest), V, A,
                     B, M, max_cycles, labels)


def solve_instance(inst, **kw) -> Result:
    """O1 on a ``synth.Instance``-like object (anything with extents/f1/f2/A/B/M)."""
    return cycle(inst.extents, inst.f1, inst.f2, inst.A, inst.B, inst.M, **kw)

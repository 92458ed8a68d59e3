"""Thin ctypes binding of libcsp (include/csp.h): argument marshalling only.

Every step of the solve runs in the CUDA library; this module converts arrays and
statuses and nothing else.  There is no CPU fallback: if ``libcsp.so`` is missing or
cannot be loaded, :func:`lib` raises.

Host arrays are numpy arrays.  Device arrays may be passed as torch CUDA tensors (torch
is used only for device memory and streams).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcsp.so")

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_BARRIER = range(7)
RESULT_FIELDS = ("status", "F1", "X", "x_src", "x_dir", "F2", "cycles", "updates", "launched", "passes",
                 "max_pool", "trace_len")

_lib = None

i64 = ctypes.c_int64
i64p = ctypes.POINTER(ctypes.c_int64)
vp = ctypes.c_void_p


class CspResult(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("F1", "X", "x_src", "x_dir", "F2", "cycles", "updates", "launched", "passes", "max_pool",
                 "arrivals", "improved", "phantoms")]


class CspOptions(ctypes.Structure):
    _fields_ = [("max_cycles", ctypes.c_int64), ("pool_capacity", ctypes.c_int64), ("ctas", ctypes.c_int32),
                ("time_limit_s", ctypes.c_int32), ("stream", vp), ("ev_begin", vp), ("ev_end", vp),
                ("flags", ctypes.c_int32), ("barrier_us", ctypes.c_int32)]

OPT_PHANTOMS = 1  # CSP_OPT_PHANTOMS
OPT_SWEEP = 2     # CSP_OPT_SWEEP: every cycle sweeps every flow in flight
OPT_EVENT = 4     # CSP_OPT_EVENT: a calendar of arrival times drives the cycles
OPT_TEST_ABSENT_CTA = 8  # CSP_OPT_TEST_ABSENT_CTA: test hook for the bounded barrier wait
ENGINES = {None: 0, "sweep": OPT_SWEEP, "event": OPT_EVENT}


class CspError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().csp_status_string(status).decode()
        detail = lib().csp_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))
        self.status = status


def lib():
    """The loaded libcsp; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1511_06441_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.csp_status_string.restype = ctypes.c_char_p
        L.csp_status_string.argtypes = [ctypes.c_int]
        L.csp_last_error.restype = ctypes.c_char_p
        L.csp_create_lattice.argtypes = [ctypes.c_int, i64p, vp, vp, ctypes.c_int, ctypes.c_int, vp,
                                         ctypes.POINTER(vp)]
        L.csp_create_graph.argtypes = [i64, ctypes.c_int32, i64p, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.csp_create_digraph.argtypes = L.csp_create_graph.argtypes
        L.csp_upload_weights.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.csp_destroy_lattice.argtypes = [vp]
        L.csp_destroy_lattice.restype = None
        L.csp_num_vertices.argtypes = [vp]
        L.csp_num_vertices.restype = i64
        L.csp_reserve.argtypes = [vp, i64]
        L.csp_solve.argtypes = [vp, i64p, i64, i64p, i64, i64, ctypes.POINTER(CspOptions),
                                ctypes.POINTER(CspResult), i64p, i64, i64p]
        L.csp_solve_async.argtypes = [vp, vp, i64, vp, i64, i64, ctypes.POINTER(CspOptions), vp, vp, i64]
        L.csp_get_labels.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
        L.csp_solve_static.argtypes = [ctypes.c_int, i64p, vp, vp, ctypes.c_int, vp, i64, vp, i64, i64, i64, vp, vp]
        L.csp_reconstruct_path.argtypes = [vp, i64p, i64, i64p, i64, i64, ctypes.POINTER(CspResult), i64p, i64, i64p]
        L.csp_reconstruct_fast.argtypes = [vp, i64p, i64, i64p, i64, i64, ctypes.POINTER(CspOptions), i64,
                                           ctypes.POINTER(CspResult), i64p, i64, i64p]
        L.csp_reconstruct_path.restype = ctypes.c_int
        L.csp_build_shape.argtypes = [ctypes.POINTER(ctypes.c_int32)]
        L.csp_build_shape.restype = None
        L.csp_default_engine.argtypes = [vp]
        L.csp_default_engine.restype = ctypes.c_int32
        L.csp_event_phase_times.argtypes = [vp, i64p]
        L.csp_event_phase_times.restype = ctypes.c_int
        for f in ("csp_create_lattice", "csp_create_graph", "csp_create_digraph", "csp_upload_weights",
                  "csp_reserve", "csp_solve",
                  "csp_solve_async",
                  "csp_get_labels", "csp_solve_static"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def build_shape() -> dict:
    """``csp_build_shape``: the block shape the loaded library was built with."""
    out = (ctypes.c_int32 * 5)()
    lib().csp_build_shape(out)
    return dict(zip(("tpb", "ipt", "nstage", "min_ctas_per_sm", "batch_min_ctas_per_sm"), [int(x) for x in out]))


def _check(status: int, where: str):
    if status != OK:
        raise CspError(status, where)


def _ptr(a) -> int:
    """Data pointer of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


@dataclasses.dataclass
class Result:
    F1: int
    X: int
    x_src: int
    x_dir: int
    F2: int
    cycles: int
    updates: int
    launched: int
    passes: int
    max_pool: int
    arrivals: int = -1
    improved: int = -1
    phantoms: int = -1       # flows started on an edge that already carried one (trace mode), else -1
    status: int = OK
    trace: Optional[np.ndarray] = None

    def answer(self):
        return (self.F1, self.X, self.x_src, self.x_dir, self.F2)


def _event_handle(ev) -> Optional[int]:
    if ev is None:
        return None
    return getattr(ev, "cuda_event", ev)


def options(max_cycles: int = 0, pool_capacity: int = 0, ctas: int = 0, stream=None,
            ev_begin=None, ev_end=None, time_limit_s: int = 0, phantoms: bool = False,
            engine: Optional[str] = None, barrier_us: int = 0, test_absent_cta: bool = False) -> CspOptions:
    """``csp_options``; ``engine`` = None (the library's default form), "sweep" or "event";
    ``barrier_us`` and ``test_absent_cta`` exercise the bounded barrier wait."""
    if engine not in ENGINES:
        raise ValueError(f"engine must be one of {sorted(k for k in ENGINES if k)} or None")
    flags = (OPT_PHANTOMS if phantoms else 0) | ENGINES[engine] | (OPT_TEST_ABSENT_CTA if test_absent_cta else 0)
    return CspOptions(max_cycles, pool_capacity, ctas, int(time_limit_s), _stream_handle(stream),
                      _event_handle(ev_begin), _event_handle(ev_end), flags, int(barrier_us))


class Lattice:
    """A lattice resident on the GPU (``csp_create_lattice``)."""

    def __init__(self, extents: Sequence[int], f1, f2, stream=None):
        ext = np.ascontiguousarray(np.asarray(extents, dtype=np.int64))
        on_device = not isinstance(f1, np.ndarray)
        if on_device:
            wb = f1.element_size()
            if f1.dtype != f2.dtype or not (f1.is_contiguous() and f2.is_contiguous()):
                raise ValueError("f1 and f2 must be contiguous and of the same dtype")
        else:
            f1 = np.ascontiguousarray(f1)
            f2 = np.ascontiguousarray(f2)
            if f1.dtype != f2.dtype or f1.dtype not in (np.uint8, np.uint16):
                raise ValueError("f1 and f2 must both be uint8 or both uint16")
            wb = f1.dtype.itemsize
        self.extents = [int(x) for x in ext]
        self.d = len(self.extents)
        self.weight_bytes = wb
        h = vp()
        _check(lib().csp_create_lattice(self.d, ext.ctypes.data_as(i64p), _ptr(f1), _ptr(f2), wb, int(on_device),
                                        _stream_handle(stream), ctypes.byref(h)), "csp_create_lattice")
        self._h = h
        self.V = int(lib().csp_num_vertices(h))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().csp_destroy_lattice(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload_weights(self, f1, f2, stream=None):
        on_device = not isinstance(f1, np.ndarray)
        _check(lib().csp_upload_weights(self._h, _ptr(f1), _ptr(f2), int(on_device), _stream_handle(stream)),
               "csp_upload_weights")

    def reserve(self, pool_capacity: int = 0):
        _check(lib().csp_reserve(self._h, int(pool_capacity)), "csp_reserve")

    def solve(self, A, B, M: int, *, trace: bool = False, trace_cap: int = 1 << 16, max_cycles: int = 0,
              pool_capacity: int = 0, ctas: int = 0, stream=None, check: bool = True,
              time_limit_s: int = 0, phantoms: bool = False, engine: Optional[str] = None,
              barrier_us: int = 0, test_absent_cta: bool = False) -> Result:
        """``csp_solve``: host sets in, host result out (blocks until done).

        ``phantoms`` (with ``trace``) also counts the flows started on an edge that already
        carries one (``Result.phantoms``).  ``engine``: "sweep", "event" or None (default form).
        ``barrier_us``/``test_absent_cta``: the bounded barrier wait and its test hook."""
        A = np.ascontiguousarray(np.asarray(A, dtype=np.int64).reshape(-1))
        B = np.ascontiguousarray(np.asarray(B, dtype=np.int64).reshape(-1))
        opt = options(max_cycles, pool_capacity, ctas, stream, time_limit_s=time_limit_s, phantoms=phantoms,
                      engine=engine, barrier_us=barrier_us, test_absent_cta=test_absent_cta)
        res = CspResult()
        tr = np.zeros(3 * trace_cap, np.int64) if trace else None
        tl = ctypes.c_int64(0)
        st = lib().csp_solve(self._h, A.ctypes.data_as(i64p), A.size, B.ctypes.data_as(i64p), B.size, int(M),
                             ctypes.byref(opt), ctypes.byref(res),
                             tr.ctypes.data_as(i64p) if tr is not None else None, trace_cap if trace else 0,
                             ctypes.byref(tl))
        if check:
            _check(st, "csp_solve")
        out = Result(*[int(getattr(res, name)) for name, _ in CspResult._fields_], status=st)
        if tr is not None:
            out.trace = tr[: 3 * min(int(tl.value), trace_cap)].reshape(-1, 3)
            out.trace_len = int(tl.value)
        return out

    def solve_async(self, A_dev, B_dev, M: int, result_dev, *, trace_dev=None, trace_cap: int = 0,
                    max_cycles: int = 0, ctas: int = 0, stream=None, ev_begin=None, ev_end=None,
                    time_limit_s: int = 0, engine: Optional[str] = None):
        """``csp_solve_async``: device sets (int64 tensors), device result (16 int64).

        ``ev_begin``/``ev_end``: optional CUDA events recorded around the cycle kernel.
        """
        opt = options(max_cycles, 0, ctas, stream, ev_begin, ev_end, time_limit_s, engine=engine)
        _check(lib().csp_solve_async(self._h, _ptr(A_dev), int(A_dev.numel()), _ptr(B_dev), int(B_dev.numel()),
                                     int(M), ctypes.byref(opt), _ptr(result_dev),
                                     _ptr(trace_dev) if trace_dev is not None else None,
                                     int(trace_cap)), "csp_solve_async")

    def reconstruct(self, A, B, M: int, result: Optional[Result] = None, cap: int = 1 << 20) -> Optional[np.ndarray]:
        """``csp_reconstruct_path``: the path (vertex ids, A end first), or None if infeasible."""
        A = np.ascontiguousarray(np.asarray(A, dtype=np.int64).reshape(-1))
        B = np.ascontiguousarray(np.asarray(B, dtype=np.int64).reshape(-1))
        res = None
        if result is not None:
            res = CspResult(*[int(getattr(result, name)) for name, _ in CspResult._fields_])
        out = np.zeros(cap, np.int64)
        n = ctypes.c_int64(0)
        _check(lib().csp_reconstruct_path(self._h, A.ctypes.data_as(i64p), A.size, B.ctypes.data_as(i64p), B.size,
                                          int(M), ctypes.byref(res) if res is not None else None,
                                          out.ctypes.data_as(i64p), cap, ctypes.byref(n)), "csp_reconstruct_path")
        return out[: n.value].copy() if n.value else None

    def reconstruct_fast(self, A, B, M: int, *, log_capacity: int = 0, cap: int = 1 << 20, max_cycles: int = 0,
                         ctas: int = 0, time_limit_s: int = 0, stream=None, ev_begin=None, ev_end=None,
                         engine: Optional[str] = None):
        """``csp_reconstruct_fast``: one recorded solve and a GPU backtrack.

        Returns ``(path, result)``; ``path`` is None if infeasible.  ``log_capacity`` < 0 keeps
        first improvements only (enough when the bound does not bind along the path).
        ``ev_begin``/``ev_end``: optional CUDA events recorded around the cycle kernel.
        """
        A = np.ascontiguousarray(np.asarray(A, dtype=np.int64).reshape(-1))
        B = np.ascontiguousarray(np.asarray(B, dtype=np.int64).reshape(-1))
        opt = options(max_cycles, 0, ctas, stream, ev_begin, ev_end, time_limit_s, engine=engine)
        res = CspResult()
        out = np.zeros(cap, np.int64)
        n = ctypes.c_int64(0)
        _check(lib().csp_reconstruct_fast(self._h, A.ctypes.data_as(i64p), A.size, B.ctypes.data_as(i64p), B.size,
                                          int(M), ctypes.byref(opt), int(log_capacity), ctypes.byref(res),
                                          out.ctypes.data_as(i64p), cap, ctypes.byref(n)), "csp_reconstruct_fast")
        r = Result(*[int(getattr(res, name)) for name, _ in CspResult._fields_], status=0)
        return (out[: n.value].copy() if n.value else None), r

    def labels(self) -> np.ndarray:
        out = np.zeros(self.V, np.int32)
        _check(lib().csp_get_labels(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "csp_get_labels")
        return out

    def default_engine(self) -> str:
        """``csp_default_engine``: "sweep" or "event", the form a solve runs without ``engine``."""
        f = int(lib().csp_default_engine(self._h))
        return "event" if f == OPT_EVENT else "sweep"

    def event_phase_times(self) -> np.ndarray:
        """``csp_event_phase_times``: ns of the last event-form solve (reserved, phase A, phase B,
        barriers), as measured by its first CTA."""
        out = np.zeros(4, np.int64)
        _check(lib().csp_event_phase_times(self._h, out.ctypes.data_as(i64p)), "csp_event_phase_times")
        return out


def slots_from_edges(V: int, edges, f1, f2, directed: bool = False, slots: int = 0):
    """Adjacency slots (nbr, f1, f2), each (V, S), from an edge list: ``edges`` (E, 2) vertex
    pairs with ``f1``/``f2`` (E,) their travel times and weights.  Undirected: every edge is
    put in the next free slot at both ends; directed: at its tail only.  Slots fill in edge
    order.  S = ``slots`` if given, else the largest degree.  Raises ValueError above 8."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    f1 = np.asarray(f1).reshape(-1)
    f2 = np.asarray(f2).reshape(-1)
    if f1.shape[0] != edges.shape[0] or f2.shape[0] != edges.shape[0] or f1.dtype != f2.dtype:
        raise ValueError("f1 and f2 need one entry per edge and the same dtype")
    ends = [edges[:, 0]] if directed else [edges[:, 0], edges[:, 1]]
    deg = np.bincount(np.concatenate(ends), minlength=V) if edges.size else np.zeros(V, np.int64)
    S = int(slots or max(1, int(deg.max()) if V else 1))
    if S > 8 or int(deg.max(initial=0)) > S:
        raise ValueError("a vertex has more edges than slots (at most 8)")
    nbr = np.full((V, S), -1, np.int64)
    g1 = np.zeros((V, S), f1.dtype)
    g2 = np.zeros((V, S), f2.dtype)
    fill = np.zeros(V, np.int64)
    for e, (a, b) in enumerate(edges.tolist()):
        for x, y in ((a, b),) if directed else ((a, b), (b, a)):
            k = fill[x]
            nbr[x, k], g1[x, k], g2[x, k] = y, f1[e], f2[e]
            fill[x] = k + 1
    return nbr, g1, g2


class Graph(Lattice):
    """A general graph resident on the GPU (``csp_create_graph``): ``nbr`` (V, S) neighbour
    ids (-1: empty slot), ``f1``/``f2`` (V, S) uint8 or uint16 the edge in each slot; S <= 8.
    Undirected: every edge in one slot at each end with equal weights.  With ``directed``
    (``csp_create_digraph``) every slot is a one-way edge v -> nbr[v, j] with its own weights,
    in-degrees <= 8.  Solves, batches, the server and path reconstruction work as on a
    lattice; x_dir is the slot of x at x_src."""

    def __init__(self, nbr, f1, f2, stream=None, directed: bool = False):
        nbr = np.ascontiguousarray(np.asarray(nbr, dtype=np.int64))
        if nbr.ndim != 2:
            raise ValueError("nbr must be (V, S)")
        f1 = np.ascontiguousarray(f1)
        f2 = np.ascontiguousarray(f2)
        if f1.dtype != f2.dtype or f1.dtype not in (np.uint8, np.uint16) or f1.shape != nbr.shape or \
                f2.shape != nbr.shape:
            raise ValueError("f1 and f2 must match nbr's shape and both be uint8 or both uint16")
        V, S = nbr.shape
        self.extents = [V]
        self.d = 0
        self.weight_bytes = f1.dtype.itemsize
        h = vp()
        name = "csp_create_digraph" if directed else "csp_create_graph"
        _check(getattr(lib(), name)(V, S, nbr.ctypes.data_as(i64p), f1.ctypes.data, f2.ctypes.data,
                                    self.weight_bytes, _stream_handle(stream), ctypes.byref(h)), name)
        self.directed = bool(directed)
        self._h = h
        self.V = int(lib().csp_num_vertices(h))


def result_from_record(rec) -> Result:
    """Converts a 16-int64 result record (``csp_solve_async``) into a :class:`Result`."""
    r = [int(x) for x in np.asarray(rec).reshape(-1)[:16]]
    return Result(F1=r[1], X=r[2], x_src=r[3], x_dir=r[4], F2=r[5], cycles=r[6], updates=r[7], launched=r[8],
                  passes=r[9], max_pool=r[10], arrivals=r[13], improved=r[14], phantoms=r[15], status=r[0])


def solve_instance(inst, **kw) -> Result:
    """Creates a lattice for a ``synth.Instance`` and solves it once."""
    lat = Lattice(inst.extents, inst.f1, inst.f2)
    try:
        return lat.solve(inst.A, inst.B, inst.M, **kw)
    finally:
        lat.close()


def solve_static(extents, f1_dev, f2_dev, A_dev, B_dev, M: int, result_dev, *, max_cycles: int = 0, stream=None):
    """``csp_solve_static``: solve with no device allocation (scratch in the library's static array).

    For callers that cannot allocate device memory.  Weights and sets are the caller's
    device tensors (upper-face travel times must be zero); the 16-int64 result record is
    written to ``result_dev``.  Returns after enqueueing; synchronise the stream to read it.
    """
    ext = np.ascontiguousarray(np.asarray(extents, dtype=np.int64))
    _check(lib().csp_solve_static(len(ext), ext.ctypes.data_as(i64p), _ptr(f1_dev), _ptr(f2_dev),
                                  f1_dev.element_size(), _ptr(A_dev), int(A_dev.numel()), _ptr(B_dev),
                                  int(B_dev.numel()), int(M), int(max_cycles), _stream_handle(stream),
                                  _ptr(result_dev)), "csp_solve_static")


class CspQuery(ctypes.Structure):
    _fields_ = [("lat", vp), ("A", i64p), ("nA", i64), ("B", i64p), ("nB", i64), ("M", i64)]


class CspBatchOptions(ctypes.Structure):
    _fields_ = [("ctas", ctypes.c_int32), ("max_group", ctypes.c_int32), ("no_graph", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("pool_capacity", i64), ("max_cycles", i64)]


def _batch_api():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        L.csp_batch_create.argtypes = [ctypes.POINTER(CspQuery), i64, ctypes.POINTER(CspBatchOptions),
                                       ctypes.POINTER(vp)]
        L.csp_batch_run.argtypes = [vp, vp]
        L.csp_batch_results.argtypes = [vp, ctypes.POINTER(CspResult), ctypes.POINTER(ctypes.c_int32), i64p]
        L.csp_batch_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int32)]
        L.csp_batch_tune.argtypes = [vp, i64p, ctypes.POINTER(CspResult)]
        dp = ctypes.POINTER(ctypes.c_double)
        L.csp_batch_model.argtypes = [vp, dp, dp, dp, dp]
        L.csp_batch_model.restype = ctypes.c_int
        L.csp_batch_destroy.argtypes = [vp]
        L.csp_batch_destroy.restype = None
        L.csp_solve_batch.argtypes = [ctypes.POINTER(CspQuery), i64, ctypes.POINTER(CspBatchOptions),
                                      ctypes.POINTER(CspResult), ctypes.POINTER(ctypes.c_int32)]
        for f in ("csp_batch_create", "csp_batch_run", "csp_batch_results", "csp_batch_schedule", "csp_batch_tune",
                  "csp_solve_batch"):
            getattr(L, f).restype = ctypes.c_int
        L._batch_ready = True
    return L


def _queries(items):
    """items: iterable of (Lattice, A, B, M).  Returns the ctypes array and the kept arrays."""
    keep = []
    arr = (CspQuery * len(items))()
    for i, (lat, A, B, M) in enumerate(items):
        A = np.ascontiguousarray(np.asarray(A, dtype=np.int64).reshape(-1))
        B = np.ascontiguousarray(np.asarray(B, dtype=np.int64).reshape(-1))
        keep += [A, B]
        arr[i] = CspQuery(lat.handle, A.ctypes.data_as(i64p), A.size, B.ctypes.data_as(i64p), B.size, int(M))
    return arr, keep


def _results(res, n, stat=None, el=None):
    out = []
    for i in range(n):
        r = Result(*[int(getattr(res[i], name)) for name, _ in CspResult._fields_])
        if stat is not None:
            r.status = int(stat[i])
        if el is not None:
            r.elapsed_ns = int(el[i])
        out.append(r)
    return out


class Batch:
    """``csp_batch_*``: many instances in one persistent, graph-captured launch."""

    def __init__(self, items, *, ctas: int = 0, max_group: int = 0, no_graph: bool = False, pool_capacity: int = 0,
                 max_cycles: int = 0):
        L = _batch_api()
        self.n = len(items)
        q, _keep = _queries(items)
        opt = CspBatchOptions(ctas, max_group, int(no_graph), 0, pool_capacity, max_cycles)
        h = vp()
        _check(L.csp_batch_create(q, self.n, ctypes.byref(opt), ctypes.byref(h)), "csp_batch_create")
        self._h = h
        self._lattices = [it[0] for it in items]  # the lattices must outlive the batch

    def run(self, stream=None):
        _check(_batch_api().csp_batch_run(self._h, _stream_handle(stream)), "csp_batch_run")

    def results(self):
        res = (CspResult * self.n)()
        stat = (ctypes.c_int32 * self.n)()
        el = np.zeros(self.n, np.int64)
        _check(_batch_api().csp_batch_results(self._h, res, stat, el.ctypes.data_as(i64p)), "csp_batch_results")
        return _results(res, self.n, stat, el)

    def schedule(self):
        n = self.n
        g = (ctypes.c_int32 * n)()
        f = (ctypes.c_int32 * n)()
        st = (ctypes.c_double * n)()
        est = (ctypes.c_double * n)()
        c = ctypes.c_int32(0)
        _check(_batch_api().csp_batch_schedule(self._h, g, f, st, est, ctypes.byref(c)), "csp_batch_schedule")
        return {"group": np.array(g[:]), "first_cta": np.array(f[:]), "start_us": np.array(st[:]),
                "est_us": np.array(est[:]), "ctas": int(c.value)}

    def tune(self, results):
        el = np.ascontiguousarray(np.array([r.elapsed_ns for r in results], np.int64))
        res = (CspResult * self.n)()
        for i, r in enumerate(results):
            for name, _ in CspResult._fields_:
                setattr(res[i], name, getattr(r, name))
        _check(_batch_api().csp_batch_tune(self._h, el.ctypes.data_as(i64p), res), "csp_batch_tune")

    def model(self):
        v = [ctypes.c_double(0) for _ in range(4)]
        _check(_batch_api().csp_batch_model(self._h, *[ctypes.byref(x) for x in v]), "csp_batch_model")
        return {"lat_single_us": v[0].value, "lat_group_us": v[1].value, "rate": v[2].value,
                "makespan_us": v[3].value}

    def close(self):
        if getattr(self, "_h", None):
            _batch_api().csp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(items, *, ctas: int = 0, max_group: int = 0, no_graph: bool = False, pool_capacity: int = 0,
                max_cycles: int = 0):
    """``csp_solve_batch``: one call; instances whose pool overflowed are re-solved alone."""
    L = _batch_api()
    q, _keep = _queries(items)
    n = len(items)
    opt = CspBatchOptions(ctas, max_group, int(no_graph), 0, pool_capacity, max_cycles)
    res = (CspResult * n)()
    stat = (ctypes.c_int32 * n)()
    _check(L.csp_solve_batch(q, n, ctypes.byref(opt), res, stat), "csp_solve_batch")
    return _results(res, n, stat)


class CspServerOptions(ctypes.Structure):
    _fields_ = [("group_ctas", ctypes.c_int32), ("max_groups", ctypes.c_int32), ("pool_capacity", i64),
                ("memory_budget", i64), ("queue_capacity", i64), ("session_seconds", ctypes.c_double),
                ("wide_depth", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class CspServerQuery(ctypes.Structure):
    _fields_ = [("A", i64p), ("nA", i64), ("B", i64p), ("nB", i64), ("b_axis", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("b_coord", i64), ("M", i64), ("max_cycles", i64)]


def _server_api():
    L = lib()
    if not getattr(L, "_server_ready", False):
        L.csp_server_create.argtypes = [vp, ctypes.POINTER(CspServerOptions), ctypes.POINTER(vp)]
        L.csp_server_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), i64p]
        L.csp_server_submit.argtypes = [vp, ctypes.POINTER(CspServerQuery), i64p]
        L.csp_server_poll.argtypes = [vp, i64, ctypes.POINTER(CspResult), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]
        dp = ctypes.POINTER(ctypes.c_double)
        L.csp_server_replay.argtypes = [vp, ctypes.POINTER(CspServerQuery), dp, i64, ctypes.POINTER(CspResult),
                                        ctypes.POINTER(ctypes.c_int32), dp, dp]
        L.csp_server_destroy.argtypes = [vp]
        L.csp_server_stats.argtypes = [vp, i64p, i64p, i64p, i64p]
        L.csp_serve_plain_replay.argtypes = [vp, ctypes.POINTER(CspServerQuery), dp, i64, ctypes.POINTER(CspResult),
                                             ctypes.POINTER(ctypes.c_int32), dp, dp]
        for f in ("csp_server_create", "csp_server_info", "csp_server_submit", "csp_server_poll", "csp_server_replay",
                  "csp_server_destroy", "csp_serve_plain_replay", "csp_server_stats"):
            getattr(L, f).restype = ctypes.c_int
        L._server_ready = True
    return L


def _server_queries(queries, use_hyperplane=True):
    """queries: objects with A, M and either (axis, coord) or an explicit B list."""
    keep = []
    arr = (CspServerQuery * len(queries))()
    for i, q in enumerate(queries):
        A = np.ascontiguousarray(np.asarray(q.A, dtype=np.int64).reshape(-1))
        keep.append(A)
        axis = getattr(q, "axis", -1)
        if use_hyperplane and axis is not None and axis >= 0:
            arr[i] = CspServerQuery(A.ctypes.data_as(i64p), A.size, None, 0, int(axis), 0, int(q.coord), int(q.M),
                                    int(getattr(q, "max_cycles", 0)))
        else:
            B = np.ascontiguousarray(np.asarray(q.B, dtype=np.int64).reshape(-1))
            keep.append(B)
            arr[i] = CspServerQuery(A.ctypes.data_as(i64p), A.size, B.ctypes.data_as(i64p), B.size, -1, 0, 0,
                                    int(q.M), int(getattr(q, "max_cycles", 0)))
    return arr, keep


def _replay_outputs(res, stat, lat_s, n):
    out = _results(res, n, stat)
    return out, np.array(lat_s[:n], dtype=np.float64)


class Server:
    """``csp_server_*``: a resident lattice answering a query stream with continuous batching."""

    def __init__(self, lattice: "Lattice", *, group_ctas: int = 0, max_groups: int = 0, pool_capacity: int = 0,
                 memory_budget: int = 0, queue_capacity: int = 0, session_seconds: float = 0.0, wide_depth: int = 0):
        """``wide_depth``: waiting queries that switch the whole-grid (wide) mode to groups;
        0 = the library default (3), -1 = groups only."""
        L = _server_api()
        opt = CspServerOptions(group_ctas, max_groups, pool_capacity, memory_budget, queue_capacity, session_seconds,
                               int(wide_depth), 0)
        h = vp()
        _check(L.csp_server_create(lattice.handle, ctypes.byref(opt), ctypes.byref(h)), "csp_server_create")
        self._h = h
        self._lattice = lattice
        g, c, q = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
        _check(L.csp_server_info(h, ctypes.byref(g), ctypes.byref(c), ctypes.byref(q)), "csp_server_info")
        self.groups, self.group_ctas, self.queue_capacity = g.value, c.value, q.value

    def submit(self, query, use_hyperplane: bool = True) -> int:
        arr, _keep = _server_queries([query], use_hyperplane)
        t = ctypes.c_int64(-1)
        _check(_server_api().csp_server_submit(self._h, arr, ctypes.byref(t)), "csp_server_submit")
        return t.value

    def poll(self, ticket: int):
        res = CspResult()
        st = ctypes.c_int32(0)
        done = ctypes.c_int32(0)
        _check(_server_api().csp_server_poll(self._h, ticket, ctypes.byref(res), ctypes.byref(st), ctypes.byref(done)),
               "csp_server_poll")
        if not done.value:
            return None
        r = Result(*[int(getattr(res, name)) for name, _ in CspResult._fields_])
        r.status = st.value
        return r

    def stats(self) -> dict:
        """``csp_server_stats``: queries answered wide and narrow, and mode switches so far."""
        v = [ctypes.c_int64(0) for _ in range(4)]
        _check(_server_api().csp_server_stats(self._h, *[ctypes.byref(x) for x in v]), "csp_server_stats")
        return dict(zip(("wide_queries", "narrow_queries", "to_wide", "to_narrow"), (x.value for x in v)))

    def replay(self, queries, arrival_s, use_hyperplane: bool = True):
        """Returns (results, latencies in s, makespan in s)."""
        n = len(queries)
        arr, _keep = _server_queries(queries, use_hyperplane)
        arrival = np.ascontiguousarray(np.asarray(arrival_s, dtype=np.float64))
        res = (CspResult * n)()
        stat = (ctypes.c_int32 * n)()
        lat = np.zeros(n, np.float64)
        mk = ctypes.c_double(0)
        dp = ctypes.POINTER(ctypes.c_double)
        _check(_server_api().csp_server_replay(self._h, arr, arrival.ctypes.data_as(dp), n, res, stat,
                                               lat.ctypes.data_as(dp), ctypes.byref(mk)), "csp_server_replay")
        out, lat = _replay_outputs(res, stat, lat, n)
        return out, lat, mk.value

    def close(self):
        if getattr(self, "_h", None):
            st = _server_api().csp_server_destroy(self._h)
            self._h = None
            _check(st, "csp_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plain_replay(lattice: "Lattice", queries, arrival_s):
    """``csp_serve_plain_replay``: the same stream answered one query at a time by csp_solve."""
    n = len(queries)
    arr, _keep = _server_queries(queries, True)
    arrival = np.ascontiguousarray(np.asarray(arrival_s, dtype=np.float64))
    res = (CspResult * n)()
    stat = (ctypes.c_int32 * n)()
    lat = np.zeros(n, np.float64)
    mk = ctypes.c_double(0)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(_server_api().csp_serve_plain_replay(lattice.handle, arr, arrival.ctypes.data_as(dp), n, res, stat,
                                                lat.ctypes.data_as(dp), ctypes.byref(mk)), "csp_serve_plain_replay")
    out, lat = _replay_outputs(res, stat, lat, n)
    return out, lat, mk.value

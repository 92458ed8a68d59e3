"""Argument checks of the C ABI that need no GPU: every entry point rejects a null handle,
missing buffers and out-of-range sizes with CSP_ERR_INVALID before it touches CUDA."""
import ctypes

import numpy as np
import pytest

INVALID = 1
vp, i64, i64p = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)


@pytest.fixture(scope="module")
def lib():
    from paper_1511_06441_gb300 import build
    L = ctypes.CDLL(build.build())
    L.csp_status_string.restype = ctypes.c_char_p
    return L


def _p(a):
    return a.ctypes.data_as(i64p)


def test_status_strings(lib):
    for code in range(7):
        assert lib.csp_status_string(code)
    assert lib.csp_status_string(99)  # unknown codes still get a text


@pytest.mark.parametrize("d,wb", [(0, 1), (5, 1), (2, 3), (2, 0)])
def test_create_lattice_rejects_bad_shapes(lib, d, wb):
    ext = np.array([4, 4, 4, 4, 4], np.int64)
    f = np.zeros(5 * 1024, np.uint16)
    out = vp()
    assert lib.csp_create_lattice(d, _p(ext), f.ctypes.data_as(vp), f.ctypes.data_as(vp), wb, 0, None,
                                  ctypes.byref(out)) == INVALID
    assert not out.value


def test_create_lattice_rejects_missing_buffers(lib):
    ext = np.array([4, 4], np.int64)
    f = np.zeros(32, np.uint8)
    out = vp()
    assert lib.csp_create_lattice(2, None, f.ctypes.data_as(vp), f.ctypes.data_as(vp), 1, 0, None,
                                  ctypes.byref(out)) == INVALID
    assert lib.csp_create_lattice(2, _p(ext), None, f.ctypes.data_as(vp), 1, 0, None, ctypes.byref(out)) == INVALID
    assert lib.csp_create_lattice(2, _p(ext), f.ctypes.data_as(vp), f.ctypes.data_as(vp), 1, 0, None, None) == INVALID


def test_null_lattice_is_rejected_everywhere(lib):
    A = np.array([0], np.int64)
    B = np.array([1], np.int64)
    res = (ctypes.c_int64 * 16)()
    path = np.zeros(4, np.int64)
    n = ctypes.c_int64(0)
    assert lib.csp_solve(None, _p(A), i64(1), _p(B), i64(1), i64(10), None, ctypes.byref(res), None, i64(0),
                         None) == INVALID
    assert lib.csp_solve_async(None, vp(1), i64(1), vp(1), i64(1), i64(10), None, vp(1), None, i64(0)) == INVALID
    assert lib.csp_reconstruct_path(None, _p(A), i64(1), _p(B), i64(1), i64(10), None, _p(path), i64(4),
                                    ctypes.byref(n)) == INVALID
    assert lib.csp_reconstruct_fast(None, _p(A), i64(1), _p(B), i64(1), i64(10), None, i64(0), ctypes.byref(res),
                                    _p(path), i64(4), ctypes.byref(n)) == INVALID
    assert lib.csp_reserve(None, i64(0)) == INVALID
    assert lib.csp_get_labels(None, vp(1)) == INVALID
    out = vp()
    assert lib.csp_server_create(None, None, ctypes.byref(out)) == INVALID
    assert lib.csp_batch_create(None, i64(0), None, ctypes.byref(out)) == INVALID


def test_static_entry_point_rejects_bad_shapes(lib):
    ext = np.array([4, 4], np.int64)
    A = np.array([0], np.int64)
    for d, wb, M in [(0, 1, 10), (5, 1, 10), (2, 3, 10), (2, 1, 1 << 31), (2, 1, (1 << 31) - 1)]:
        assert lib.csp_solve_static(d, _p(ext), vp(1), vp(1), wb, vp(1), i64(1), vp(1), i64(1), i64(M), i64(0),
                                    None, vp(1)) == INVALID
    big = np.array([1 << 28, 1], np.int64)  # too many vertices
    assert lib.csp_solve_static(2, _p(big), vp(1), vp(1), 1, vp(1), i64(1), vp(1), i64(1), i64(10), i64(0), None,
                                vp(1)) == INVALID
    del A


def _graph(lib, nbr, f1, f2=None, slots=None, wb=1):
    nbr = np.ascontiguousarray(np.asarray(nbr, np.int64))
    f1 = np.ascontiguousarray(np.asarray(f1, np.uint8 if wb == 1 else np.uint16))
    f2 = np.zeros_like(f1) if f2 is None else np.ascontiguousarray(np.asarray(f2, f1.dtype))
    out = vp()
    st = lib.csp_create_graph(i64(nbr.shape[0]), ctypes.c_int32(nbr.shape[1] if slots is None else slots), _p(nbr),
                              f1.ctypes.data_as(vp), f2.ctypes.data_as(vp), wb, None, ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("nbr,f1,f2", [
    ([[1, -1], [2, -1], [-1, -1]], [[1, 0], [1, 0], [0, 0]], None),        # 1-2 listed only at 1
    ([[5, -1], [0, -1]], [[1, 0], [1, 0]], None),                          # id out of range
    ([[0, -1], [-1, -1]], [[1, 0], [0, 0]], None),                         # self loop
    ([[1, 1], [0, 0]], [[1, 1], [1, 1]], None),                            # parallel edges
    ([[1, -1], [0, -1]], [[1, 0], [2, 0]], None),                          # f1 differs at the two ends
    ([[1, -1], [0, -1]], [[1, 0], [1, 0]], [[3, 0], [4, 0]]),              # f2 differs at the two ends
    ([[1, -1], [0, -1]], [[0, 0], [0, 0]], None),                          # travel time 0 on an edge
    ([[-2, -1], [-1, -1]], [[1, 0], [0, 0]], None),                        # neither an id nor -1
])
def test_create_graph_rejects_broken_graphs(lib, nbr, f1, f2):
    st, out = _graph(lib, nbr, f1, f2)
    assert st == INVALID and not out.value
    lib.csp_last_error.restype = ctypes.c_char_p
    assert b"csp_create_graph: vertex" in lib.csp_last_error()


def test_create_graph_rejects_bad_shapes(lib):
    ok_nbr, ok_f1 = [[1], [0]], [[1], [1]]
    assert _graph(lib, ok_nbr, ok_f1, slots=0)[0] == INVALID
    assert _graph(lib, ok_nbr, ok_f1, slots=9)[0] == INVALID
    assert _graph(lib, ok_nbr, ok_f1, wb=3)[0] == INVALID
    nbr = np.zeros((0, 1), np.int64)
    assert _graph(lib, nbr, np.zeros((0, 1)))[0] == INVALID
    out = vp()
    f = np.ones(2, np.uint8)
    assert lib.csp_create_graph(i64(2), ctypes.c_int32(1), None, f.ctypes.data_as(vp), f.ctypes.data_as(vp), 1, None,
                                ctypes.byref(out)) == INVALID


def _digraph(lib, nbr, f1, slots=None):
    nbr = np.ascontiguousarray(np.asarray(nbr, np.int64))
    f1 = np.ascontiguousarray(np.asarray(f1, np.uint8))
    f2 = np.zeros_like(f1)
    out = vp()
    st = lib.csp_create_digraph(i64(nbr.shape[0]), ctypes.c_int32(nbr.shape[1] if slots is None else slots), _p(nbr),
                                f1.ctypes.data_as(vp), f2.ctypes.data_as(vp), 1, None, ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("nbr,f1,reason", [
    ([[-1]] + [[0]] * 9, [[0]] + [[1]] * 9, b"in-degree above 8"),        # nine edges into vertex 0
    ([[0], [-1]], [[1], [0]], b"self loop"),
    ([[1, 1], [-1, -1]], [[1, 1], [0, 0]], b"parallel edge"),
    ([[7], [-1]], [[1], [0]], b"out of range"),
    ([[1], [-1]], [[0], [0]], b"travel time below 1"),
])
def test_create_digraph_rejects_broken_graphs(lib, nbr, f1, reason):
    st, out = _digraph(lib, nbr, f1)
    assert st == INVALID and not out.value
    lib.csp_last_error.restype = ctypes.c_char_p
    msg = lib.csp_last_error()
    assert msg.startswith(b"csp_create_digraph: vertex") and reason in msg

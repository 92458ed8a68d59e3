"""Seeded synthetic inputs: lattices, weights, source/target sets and query streams.

This module draws random numbers and lays them out; it contains none of the
solver's arithmetic, so both the CUDA path and the CPU oracle can consume what it
produces.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based generator:
value ``i`` of stream ``s`` under seed ``k`` is ``mix(base(k, s) + (i + 1) * GAMMA)``
where ``mix`` is the SplitMix64 output function.  Every array has its own stream id,
so arrays never share draws and any element can be regenerated independently.

Lattice layout (shared by every consumer):

* a vertex of the box ``[0, n_0) x ... x [0, n_{d-1})`` has the linear id
  ``v = sum_k c_k * stride_k`` with coordinate 0 fastest;
* ``f1[k, v]`` / ``f2[k, v]`` describe the edge ``(v, v + e_k)`` (travel time and
  weight of Section 1 of the paper); entries on the upper face ``c_k = n_k - 1`` are
  zero because that edge leaves the box;
* ``f1 == 0`` marks an absent edge (a lattice subgraph).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids of the arrays drawn for one lattice / instance
S_F1, S_F2, S_A, S_B, S_M, S_SHAPE, S_QUERY = 1, 2, 3, 4, 5, 6, 7


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` 64-bit draws of stream ``stream`` under ``seed``, starting at ``offset``."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([(seed * 0x2545F4914F6CDD1D + stream) & (2**64 - 1)], dtype=np.uint64))[0]
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(key + i * GAMMA)


def uniform_int(seed: int, stream: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """Integers in ``[lo, hi]`` as ``lo + x mod (hi - lo + 1)`` (int64)."""
    span = np.uint64(hi - lo + 1)
    return (u64(seed, stream, n, offset) % span).astype(np.int64) + lo


def uniform_unit(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Floats in ``[0, 1)`` from the top 53 bits."""
    return (u64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def geometric_clipped(seed: int, stream: int, n: int, p_num: int, p_den: int, cap: int) -> np.ndarray:
    """Geometric(p = p_num/p_den) on {1, 2, ...}, clipped to ``cap``; inverse CDF in exact integers.

    With ``u`` the top 53 bits of a draw, the value is ``1 + #{k >= 1 : u < 2^53 q^k}``
    (``q = 1 - p``), i.e. P(value > k) = q^k.  The thresholds are exact rationals, so
    the result does not depend on the platform's libm.
    """
    q_num = p_den - p_num
    thr = [((1 << 53) * q_num ** k) // p_den ** k for k in range(1, cap)]
    thr_arr = np.array(thr[::-1], dtype=np.int64)  # ascending
    u = (u64(seed, stream, n) >> np.uint64(11)).astype(np.int64)
    # count of thresholds strictly greater than u
    greater = len(thr) - np.searchsorted(thr_arr, u, side="right")
    return np.minimum(1 + greater, cap).astype(np.int64)


# ---------------------------------------------------------------- lattice helpers

def strides(extents: Sequence[int]) -> List[int]:
    s, out = 1, []
    for n in extents:
        out.append(s)
        s *= int(n)
    return out


def num_vertices(extents: Sequence[int]) -> int:
    return int(np.prod([int(n) for n in extents], dtype=np.int64))


def coords(v: np.ndarray, extents: Sequence[int]) -> np.ndarray:
    """(len(v), d) coordinates of linear ids ``v``."""
    v = np.asarray(v, dtype=np.int64)
    out = np.empty((v.size, len(extents)), dtype=np.int64)
    for k, n in enumerate(extents):
        out[:, k] = v % n
        v = v // n
    return out


def vertex_id(c: np.ndarray, extents: Sequence[int]) -> np.ndarray:
    c = np.atleast_2d(np.asarray(c, dtype=np.int64))
    st = np.array(strides(extents), dtype=np.int64)
    return c @ st


def face(extents: Sequence[int], k: int, c: int) -> np.ndarray:
    """All vertex ids with coordinate ``k`` equal to ``c`` (ascending)."""
    st = strides(extents)
    lo = np.arange(st[k], dtype=np.int64)                       # coordinates below k
    hi = np.arange(num_vertices(extents) // (st[k] * extents[k]), dtype=np.int64) * st[k] * extents[k]
    return (hi[:, None] + c * st[k] + lo[None, :]).reshape(-1)


def upper_face_mask(extents: Sequence[int]) -> np.ndarray:
    """(d, V) bool: True where edge (v, v+e_k) leaves the box."""
    V = num_vertices(extents)
    v = np.arange(V, dtype=np.int64)
    st = strides(extents)
    return np.stack([(v // st[k]) % extents[k] == extents[k] - 1 for k in range(len(extents))])


@dataclasses.dataclass
class Instance:
    """One constrained-shortest-path problem on a box lattice (Section 1 of the paper)."""
    extents: List[int]
    f1: np.ndarray          # (d, V) uint8 | uint16
    f2: np.ndarray          # (d, V) same dtype
    A: np.ndarray           # int64 source vertex ids
    B: np.ndarray           # int64 target vertex ids
    M: int                  # weight bound, F2 < M
    name: str = ""

    @property
    def d(self) -> int:
        return len(self.extents)

    @property
    def V(self) -> int:
        return num_vertices(self.extents)

    @property
    def weight_bytes(self) -> int:
        return self.f1.dtype.itemsize


_fast = None


def _fast_lib():
    """The C fill routines (synth_fill.c), compiled on first use; None if no compiler."""
    global _fast
    if _fast is None:
        import ctypes
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src, lib = os.path.join(here, "synth_fill.c"), os.path.join(here, "libsynth_fill.so")
        try:
            if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
                tmp = lib + f".tmp{os.getpid()}"
                subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src])
                os.replace(tmp, lib)
            L = ctypes.CDLL(lib)
            L.synth_fill_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int]
            L.synth_upper_face_mask.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            _fast = L
        except Exception:
            _fast = False
    return _fast or None


def uniform_weights(extents: Sequence[int], lo: int, hi: int, seed: int,
                    dtype=np.uint8, stream_base: int = 0, use_c: bool = True):
    """i.i.d. uniform integer travel times and weights in ``[lo, hi]``; upper faces zeroed.

    ``use_c`` selects the C fill (same SplitMix64 definition, much faster); the numpy
    path is the reference it is tested against."""
    d, V = len(extents), num_vertices(extents)
    L = _fast_lib() if use_c else None
    if L is not None:
        ext = np.ascontiguousarray(np.asarray(extents, dtype=np.int64))
        up = np.empty(d * V, np.uint8)
        L.synth_upper_face_mask(d, ext.ctypes.data, up.ctypes.data)
        dt = np.dtype(dtype)
        out = []
        for stream in (S_F1, S_F2):
            a = np.empty(d * V, dt)
            L.synth_fill_uniform(seed, stream_base + stream, d * V, 0, lo, hi, up.ctypes.data, a.ctypes.data,
                                 dt.itemsize)
            out.append(a.reshape(d, V))
        return out[0], out[1]
    f1 = uniform_int(seed, stream_base + S_F1, d * V, lo, hi).reshape(d, V)
    f2 = uniform_int(seed, stream_base + S_F2, d * V, lo, hi).reshape(d, V)
    up = upper_face_mask(extents)
    f1[up] = 0
    f2[up] = 0
    return f1.astype(dtype), f2.astype(dtype)


# ---------------------------------------------------------------- the workloads

def workload_64x64(seed: int = 1) -> Instance:
    """2-D 64x64, f1,f2 ~ U{1..10} uint8, A = column c0=0, B = column c0=63, M = 200."""
    ext = [64, 64]
    f1, f2 = uniform_weights(ext, 1, 10, seed)
    return Instance(ext, f1, f2, face(ext, 0, 0), face(ext, 0, 63), 200, "lattice2d_64x64_M200")


def workload_cube(side: int = 128, M: int = 1600, seed: int = 2) -> Instance:
    """3-D cube side^3, f1,f2 ~ U{1..16} uint8, A = face c0=0, B = face c0=side-1."""
    ext = [side, side, side]
    f1, f2 = uniform_weights(ext, 1, 16, seed)
    return Instance(ext, f1, f2, face(ext, 0, 0), face(ext, 0, side - 1), M,
                    f"cube3d_{side}_M{M}")


def workload_point_source(side: int = 1024, seed: int = 6) -> Instance:
    """2-D side x side, f1,f2 ~ U{1..16} uint8, A = the centre vertex, B = the four corners
    (the set-up for measuring how the active set grows with time; M is the caller's)."""
    ext = [side, side]
    f1, f2 = uniform_weights(ext, 1, 16, seed)
    c = (side // 2) + (side // 2) * side
    B = np.array([0, side - 1, side * (side - 1), side * side - 1], np.int64)
    return Instance(ext, f1, f2, np.array([c], np.int64), B, 0, f"lattice2d_{side}_U16_point_source")


FRACTAL_M = 2**31 - 2   # a bound no path reaches: the weights are all 0


def fractal_environment(t: int, levels: int) -> Instance:
    """The environment omega_j, j = ``levels``, of the proof of the paper's t log t lower
    bound on the active set (Section "Large sets of active vertices", Theorem 3), on
    V = [-t, t] x [0, t + 1] of Z^2.

    Travel times are 1 on the y axis and on the construction's segments and 2 elsewhere;
    weights are 0 and M is never reached, so the problem is first-passage percolation.
    Water starts on the whole x axis (A = the row y = 0); B = the row y = t + 1, which
    the y axis reaches at time t + 1, so a solve passes Time t.

    Construction on the left half (the right half is its mirror image in the y axis),
    t = 2^k: L = (-t/2, 0), O = (0, t/2), T = (0, t).  omega_1: the y axis and the
    segment LO are fast, and the triangles are {LOT}.  omega_{j+1}: in every triangle
    (L, O, T), where O = L + (s, s) and T = L + (s, 2s), the segments L0 X (L0 the midpoint
    of LO, X the midpoint of LT: vertical) and X T0 (T0 the midpoint of OT: slope 1)
    become fast, and the triangles become the halves (L, L0, X) and (X, T0, T).  A slope-1
    segment from P to P + (m, m) is the staircase P + (i, i) -> P + (i, i + 1) ->
    P + (i + 1, i + 1), i < m, whose corners lie on the triangle's side of the segment.
    Vertex ids: x + t fastest, then y.
    """
    k = int(t).bit_length() - 1
    if t < 2 or t != 1 << k or not 1 <= levels <= k:
        raise ValueError("t must be a power of two >= 2 and 1 <= levels <= log2(t)")
    W, H = 2 * t + 1, t + 2
    fast_h = np.zeros((H, W), bool)   # edge (x, y) -> (x + 1, y), at [y, x + t]
    fast_v = np.zeros((H, W), bool)   # edge (x, y) -> (x, y + 1), at [y, x + t]

    def vertical(x, y0, y1):          # (x, y) -> (x, y + 1) for y0 <= y < y1, and its mirror
        fast_v[y0:y1, t + x] = True
        fast_v[y0:y1, t - x] = True

    def staircase(px, py, m):
        i = np.arange(m)
        fast_v[py + i, t + px + i] = True
        fast_v[py + i, t - px - i] = True
        fast_h[py + i + 1, t + px + i] = True           # (px+i, .) -> (px+i+1, .)
        fast_h[py + i + 1, t - px - i - 1] = True       # its mirror (-px-i-1, .) -> (-px-i, .)

    vertical(0, 0, H - 1)
    staircase(-t // 2, 0, t // 2)
    triangles = [(-t // 2, 0, t // 2)]                  # (L_x, L_y, s)
    for _ in range(levels - 1):
        halves = []
        for lx, ly, s in triangles:
            h = s // 2
            vertical(lx + h, ly + h, ly + s)            # L0 = L + (h, h) up to X = L + (h, s)
            staircase(lx + h, ly + s, h)                # X up to T0 = L + (s, s + h)
            halves += [(lx, ly, h), (lx + h, ly + s, h)]
        triangles = halves
    ext = [W, H]
    V = W * H
    f1 = np.stack([np.where(fast_h, 1, 2).reshape(V), np.where(fast_v, 1, 2).reshape(V)])
    f1[upper_face_mask(ext)] = 0
    f1 = f1.astype(np.uint8)
    f2 = np.zeros_like(f1)
    A = face(ext, 1, 0)
    B = face(ext, 1, H - 1)
    return Instance(ext, f1, f2, A, B, FRACTAL_M, f"lattice2d_fractal_t{t}_omega{levels}")


def anticorrelated_weights(extents: Sequence[int], seed: int = 3):
    """f1 = min(255, Geometric(0.1)), f2 = 256 - f1, stored as uint16; upper faces zeroed."""
    d, V = len(extents), num_vertices(extents)
    f1 = geometric_clipped(seed, S_F1, d * V, 1, 10, 255).reshape(d, V)
    f2 = 256 - f1
    up = upper_face_mask(extents)
    f1[up] = 0
    f2[up] = 0
    return f1.astype(np.uint16), f2.astype(np.uint16)


def workload_anticorrelated(side: int = 4096, M: Optional[int] = None, seed: int = 3) -> Instance:
    """2-D side x side with anti-correlated weights, A = corner 0, B = opposite corner.

    ``M`` is 1.2 x the F2 of the lexicographic (F1, F2)-minimal unconstrained path; the
    caller supplies it (it needs a shortest-path computation this module does not do).
    """
    ext = [side, side]
    f1, f2 = anticorrelated_weights(ext, seed)
    V = side * side
    return Instance(ext, f1, f2, np.array([0], np.int64), np.array([V - 1], np.int64),
                    int(M) if M is not None else 0, f"lattice2d_{side}_anticorr")


def batch_instances(n: int = 512, seed: int = 4, side2d=(32, 1024), side3d=(16, 160)) -> List[Instance]:
    """Mixed 2-D/3-D instances with log-uniform sides, U{1..32} weights, face-to-face A/B."""
    out = []
    for i in range(n):
        sb = 16 * (i + 1)
        r = uniform_unit(seed, sb + S_SHAPE, 5)
        d = 2 if r[0] < 0.5 else 3
        lo, hi = side2d if d == 2 else side3d
        side = int(round(math.exp(math.log(lo) + r[1] * (math.log(hi) - math.log(lo)))))
        ext = [side] * d
        f1, f2 = uniform_weights(ext, 1, 32, seed, np.uint8, stream_base=sb)
        k = min(int(r[2] * d), d - 1)
        lowA = r[3] < 0.5
        A = face(ext, k, 0 if lowA else side - 1)
        B = face(ext, k, side - 1 if lowA else 0)
        M = int(math.floor((0.5 + 1.5 * r[4]) * side * 16))
        out.append(Instance(ext, f1, f2, A, B, M, f"batch{i}_d{d}_s{side}"))
    return out


def serving_lattice(side: int = 48, d: int = 4, seed: int = 5):
    ext = [side] * d
    f1, f2 = uniform_weights(ext, 1, 20, seed)
    return ext, f1, f2


@dataclasses.dataclass
class Query:
    A: np.ndarray
    B: np.ndarray          # the target hyperplane as an explicit id list
    M: int
    axis: int = -1         # B = {v : c_axis(v) = coord}
    coord: int = 0


def serving_queries(n: int, extents: Sequence[int], seed: int = 5, start: int = 0) -> List[Query]:
    """Queries with 1-64 distinct random sources, a random target hyperplane, M ~ U{200..2000}."""
    d, V = len(extents), num_vertices(extents)
    st = strides(extents)
    out = []
    for q in range(start, start + n):
        sb = 1000 + 8 * q
        hdr = uniform_int(seed, sb + S_QUERY, 4, 0, 2**31 - 1)
        k = int(hdr[0] % d)
        c = int(hdr[1] % extents[k])
        nsrc = int(1 + hdr[2] % 64)
        M = int(200 + hdr[3] % 1801)
        B = face(extents, k, c)
        chosen: List[int] = []
        seen = set()
        off = 0
        while len(chosen) < nsrc:
            cand = uniform_int(seed, sb + S_A, 64, 0, V - 1, offset=off)
            off += 64
            for v in cand.tolist():
                if (v // st[k]) % extents[k] == c or v in seen:
                    continue
                seen.add(v)
                chosen.append(v)
                if len(chosen) == nsrc:
                    break
        out.append(Query(np.array(sorted(chosen), np.int64), B, M, k, c))
    return out


def poisson_arrivals(n: int, rate: float, seed: int = 5, stream: int = 77) -> np.ndarray:
    """Arrival times (s) of a Poisson stream of ``n`` requests at ``rate`` per second."""
    u = uniform_unit(seed, stream, n)
    return np.cumsum(-np.log1p(-u) / rate)


def random_small_instance(seed: int, max_vertices: int = 16, dims=(1, 2, 3), f_lo=(0, 1),
                          f_hi: int = 6, absent_prob: float = 0.15) -> Instance:
    """A tiny random lattice subgraph for brute-force comparisons.

    Random dimension and extents with at most ``max_vertices`` vertices, travel times in
    ``[1, f_hi]`` with some edges absent (f1 = 0), weights in ``[f2_lo, f_hi]`` with
    ``f2_lo`` drawn from ``f_lo``, random disjoint A and B, M in ``[1, 25]``.
    """
    r = u64(seed, S_SHAPE, 16)
    d = dims[int(r[0] % np.uint64(len(dims)))]
    ext = [1] * d
    # grow extents while the vertex budget allows
    for i in range(1, 12):
        k = int(r[i] % np.uint64(d))
        if num_vertices(ext) // ext[k] * (ext[k] + 1) <= max_vertices:
            ext[k] += 1
    V = num_vertices(ext)
    f1 = uniform_int(seed, S_F1, d * V, 1, f_hi).reshape(d, V)
    f2lo = f_lo[int(r[12] % np.uint64(len(f_lo)))]
    f2 = uniform_int(seed, S_F2, d * V, f2lo, f_hi).reshape(d, V)
    absent = uniform_unit(seed, S_F1 + 100, d * V).reshape(d, V) < absent_prob
    f1[absent] = 0
    f2[absent] = 0
    up = upper_face_mask(ext)
    f1[up] = 0
    f2[up] = 0
    perm = np.argsort(u64(seed, S_A, V))
    nA = 1 + int(r[13] % np.uint64(max(1, V // 3)))
    nB = 1 + int(r[14] % np.uint64(max(1, (V - nA) // 2)))
    nA = min(nA, V - 1)
    nB = min(nB, V - nA)
    A = np.sort(perm[:nA]).astype(np.int64)
    B = np.sort(perm[nA:nA + nB]).astype(np.int64)
    M = int(1 + r[15] % np.uint64(25))
    return Instance(ext, f1.astype(np.uint8), f2.astype(np.uint8), A, B, M, f"tiny{seed}")


# ---------------------------------------------------------------- general graphs

@dataclasses.dataclass
class GraphInstance:
    """One problem on a general graph of bounded degree (Section 1 of the paper states the
    method for any graph).  Vertex v has S adjacency slots: ``nbr[v, j]`` is the neighbour
    in slot j (-1: empty), ``f1[v, j]`` >= 1 and ``f2[v, j]`` the travel time and weight of
    that edge.  Undirected: an edge sits in one slot at each end with the same weights.
    The direction of an edge (the x_dir of a result) is its slot at the vertex it leaves.
    A directed graph lists each edge once, in a slot of its tail (see :func:`random_digraph`)."""
    nbr: np.ndarray         # (V, S) int64
    f1: np.ndarray          # (V, S) uint8 | uint16 (0 in empty slots)
    f2: np.ndarray          # (V, S) same dtype
    A: np.ndarray
    B: np.ndarray
    M: int
    name: str = ""

    @property
    def V(self) -> int:
        return int(self.nbr.shape[0])

    @property
    def S(self) -> int:
        return int(self.nbr.shape[1])

    @property
    def weight_bytes(self) -> int:
        return self.f1.dtype.itemsize


def graph_from_lattice(extents: Sequence[int], f1, f2):
    """The lattice as adjacency slots in its direction order (slot 2k: +e_k, 2k+1: -e_k),
    absent edges as empty slots: (nbr, f1, f2), each (V, 2d)."""
    d, V = len(extents), num_vertices(extents)
    st = strides(extents)
    f1 = np.asarray(f1).reshape(d, V)
    f2 = np.asarray(f2).reshape(d, V)
    v = np.arange(V, dtype=np.int64)
    nbr = np.full((V, 2 * d), -1, np.int64)
    g1 = np.zeros((V, 2 * d), f1.dtype)
    g2 = np.zeros((V, 2 * d), f2.dtype)
    for k in range(d):
        ok = f1[k] > 0                               # the edge (v, v + e_k) exists
        up = v[ok] + st[k]
        nbr[v[ok], 2 * k] = up
        g1[v[ok], 2 * k] = f1[k][ok]
        g2[v[ok], 2 * k] = f2[k][ok]
        nbr[up, 2 * k + 1] = v[ok]
        g1[up, 2 * k + 1] = f1[k][ok]
        g2[up, 2 * k + 1] = f2[k][ok]
    return nbr, g1, g2


KING_MOVES = ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1))


def king_graph(side: int, lo: int = 1, hi: int = 16, seed: int = 7, M: int = 0) -> GraphInstance:
    """side x side king's graph (the 8 neighbours of a square grid; slots in the order of
    KING_MOVES), f1, f2 ~ U{lo..hi} per undirected edge (uint8), A = column x = 0,
    B = column x = side - 1."""
    V = side * side
    v = np.arange(V, dtype=np.int64)
    x, y = v % side, v // side
    nbr = np.full((V, 8), -1, np.int64)
    f1 = np.zeros((V, 8), np.uint8)
    f2 = np.zeros((V, 8), np.uint8)
    for j in range(0, 8, 2):            # each undirected edge drawn once, at its lower end
        dx, dy = KING_MOVES[j]
        if dy < 0 or (dy == 0 and dx < 0):
            dx, dy = -dx, -dy
        ok = (x + dx >= 0) & (x + dx < side) & (y + dy < side)
        a = v[ok]
        b = a + dx + dy * side
        w1 = uniform_int(seed, 200 + j, V, lo, hi)[ok]
        w2 = uniform_int(seed, 300 + j, V, lo, hi)[ok]
        ja = KING_MOVES.index((dx, dy))
        jb = KING_MOVES.index((-dx, -dy))
        nbr[a, ja], nbr[b, jb] = b, a
        f1[a, ja] = f1[b, jb] = w1
        f2[a, ja] = f2[b, jb] = w2
    A = v[x == 0]
    B = v[x == side - 1]
    return GraphInstance(nbr, f1, f2, A, B, M, f"king{side}_U{lo}_{hi}")


def random_graph(V: int, rounds: int = 6, seed: int = 8, lo: int = 1, hi: int = 16, f2_lo: Optional[int] = None,
                 drop: float = 0.0, dtype=np.uint8):
    """A random graph of degree <= ``rounds`` (<= 8): round j pairs the vertices by a random
    permutation (vertex p[2i] with p[2i+1]) and puts each new edge in slot j at both ends;
    a pair already joined, and a fraction ``drop`` of the pairs, leave slot j empty.
    f1 ~ U{lo..hi}, f2 ~ U{f2_lo..hi} per edge.  Returns (nbr, f1, f2)."""
    f2_lo = lo if f2_lo is None else f2_lo
    nbr = np.full((V, rounds), -1, np.int64)
    f1 = np.zeros((V, rounds), dtype)
    f2 = np.zeros((V, rounds), dtype)
    seen = set()
    for j in range(rounds):
        p = np.argsort(u64(seed, 400 + j, V), kind="stable")
        a, b = p[0:V - 1:2], p[1:V:2]
        keep = uniform_unit(seed, 500 + j, a.size) >= drop
        w1 = uniform_int(seed, 600 + j, a.size, lo, hi)
        w2 = uniform_int(seed, 700 + j, a.size, f2_lo, hi)
        for i in np.flatnonzero(keep).tolist():
            e = (min(a[i], b[i]), max(a[i], b[i]))
            if e in seen:
                continue
            seen.add(e)
            nbr[a[i], j], nbr[b[i], j] = b[i], a[i]
            f1[a[i], j] = f1[b[i], j] = w1[i]
            f2[a[i], j] = f2[b[i], j] = w2[i]
    return nbr, f1, f2


def random_small_graph(seed: int, max_vertices: int = 12, rounds=(1, 4), f_hi: int = 6, M_max: int = 25,
                       max_sources: Optional[int] = None, drop: float = 0.25) -> GraphInstance:
    """A tiny random graph for brute-force comparisons: 2..max_vertices vertices, a number of
    pairing rounds drawn from ``rounds`` with a fraction ``drop`` of the pairs left out,
    f1 in [1, f_hi], f2 in [0 or 1, f_hi], random disjoint A (at most ``max_sources``,
    default V/3) and B, M in [1, M_max]."""
    r = u64(seed, S_SHAPE + 50, 8)
    V = 2 + int(r[0] % np.uint64(max_vertices - 1))
    nr = rounds[0] + int(r[1] % np.uint64(rounds[1] - rounds[0] + 1))
    nbr, f1, f2 = random_graph(V, nr, seed, 1, f_hi, int(r[2] % np.uint64(2)), drop=drop)
    perm = np.argsort(u64(seed, S_A + 50, V))
    amax = max(1, V // 3) if max_sources is None else max_sources
    nA = min(1 + int(r[3] % np.uint64(amax)), V - 1)
    nB = min(1 + int(r[4] % np.uint64(max(1, (V - nA) // 2))), V - nA)
    A = np.sort(perm[:nA]).astype(np.int64)
    B = np.sort(perm[nA:nA + nB]).astype(np.int64)
    M = int(1 + r[5] % np.uint64(M_max))
    return GraphInstance(nbr, f1, f2, A, B, M, f"tinygraph{seed}")


def random_digraph(V: int, rounds: int = 6, seed: int = 9, lo: int = 1, hi: int = 16, f2_lo: Optional[int] = None,
                   drop: float = 0.0, dtype=np.uint8):
    """A random directed graph with out- and in-degree <= ``rounds`` (<= 8): round j draws a
    random permutation p and puts the edge v -> p[v] in out-slot j of v; self loops, edges
    already present and a fraction ``drop`` leave the slot empty.  f1 ~ U{lo..hi},
    f2 ~ U{f2_lo..hi} per edge; an edge and its reverse get independent weights.
    Returns (nbr, f1, f2) with nbr[v, j] the head of out-edge j of v."""
    f2_lo = lo if f2_lo is None else f2_lo
    nbr = np.full((V, rounds), -1, np.int64)
    f1 = np.zeros((V, rounds), dtype)
    f2 = np.zeros((V, rounds), dtype)
    seen = set()
    for j in range(rounds):
        p = np.argsort(u64(seed, 800 + j, V), kind="stable")
        keep = uniform_unit(seed, 900 + j, V) >= drop
        w1 = uniform_int(seed, 1000 + j, V, lo, hi)
        w2 = uniform_int(seed, 1100 + j, V, f2_lo, hi)
        for v in np.flatnonzero(keep).tolist():
            u = int(p[v])
            if u == v or (v, u) in seen:
                continue
            seen.add((v, u))
            nbr[v, j] = u
            f1[v, j] = w1[v]
            f2[v, j] = w2[v]
    return nbr, f1, f2


def random_small_digraph(seed: int, max_vertices: int = 12, rounds=(1, 4), f_hi: int = 6, M_max: int = 25,
                         max_sources: Optional[int] = None, drop: float = 0.25) -> GraphInstance:
    """A tiny random directed graph for brute-force comparisons (as :func:`random_small_graph`,
    edges one way; ``nbr`` lists out-neighbours)."""
    r = u64(seed, S_SHAPE + 60, 8)
    V = 2 + int(r[0] % np.uint64(max_vertices - 1))
    nr = rounds[0] + int(r[1] % np.uint64(rounds[1] - rounds[0] + 1))
    nbr, f1, f2 = random_digraph(V, nr, seed, 1, f_hi, int(r[2] % np.uint64(2)), drop=drop)
    perm = np.argsort(u64(seed, S_A + 60, V))
    amax = max(1, V // 3) if max_sources is None else max_sources
    nA = min(1 + int(r[3] % np.uint64(amax)), V - 1)
    nB = min(1 + int(r[4] % np.uint64(max(1, (V - nA) // 2))), V - nA)
    A = np.sort(perm[:nA]).astype(np.int64)
    B = np.sort(perm[nA:nA + nB]).astype(np.int64)
    M = int(1 + r[5] % np.uint64(M_max))
    return GraphInstance(nbr, f1, f2, A, B, M, f"tinydigraph{seed}")

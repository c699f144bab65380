"""Seeded synthetic instances for the sparse Ising / MaxCut annealer.

This module holds only the seeded input generators.  It contains none of the
annealing arithmetic: no energies, no acceptance rule, no sweep RNG.  Both the
CUDA path and the CPU oracle consume what it produces, so that the two sides
can be compared on identical inputs.

Instance families follow the problem classes of the paper (Sec. II.A, Table I):

* ``torus(L, W, seed)`` -- a toroidal square grid, the shape of the Gset spin
  glass instances (2n edges, degree 4), with couplings +1/-1 drawn with
  probability 1/2 each.  The Gset files themselves are not used; these seeded
  grids stand in for them.
* ``random_graph(n, m, seed)`` -- ``m`` distinct unordered vertex pairs drawn
  uniformly without replacement, weight 1, no self-loops: the shape of the
  unweighted sparse random MaxCut instance (G70: n = 10,000, m = 9,999).
* ``linear_betas`` / ``geometric_betas`` -- inverse-temperature schedules with
  inclusive end points, evaluated in FP64.

Randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its published
definition and evaluated in numpy uint64 arithmetic, so that every machine
produces byte-identical instances.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

# Independent draw streams, so that two uses of one seed never share draws.
STREAM_COUPLING = 1
STREAM_EDGES = 2
STREAM_SIZES = 3
STREAM_ARRIVALS = 4
STREAM_KIND = 5
STREAM_POINTS = 6


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def draws(seed: int, stream: int, index) -> np.ndarray:
    """64-bit draw number ``index`` (array) of stream ``stream`` under ``seed``.

    The stream key is one SplitMix64 step from ``seed`` and ``stream``; draw k
    of that stream is SplitMix64 state ``key + (k + 1) * gamma``.
    """
    idx = np.asarray(index, dtype=np.uint64)
    s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = _mix64(s + np.uint64(stream) * _GAMMA)[0]
        return _mix64(key + (idx + np.uint64(1)) * _GAMMA)


def uniform_int(seed: int, stream: int, index, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive) from ``draws`` (modulo bias < 2^-40)."""
    span = np.uint64(hi - lo + 1)
    return (draws(seed, stream, index) % span).astype(np.int64) + lo


def uniform_float(seed: int, stream: int, index) -> np.ndarray:
    """Floats uniform in [0, 1) from the top 53 bits of ``draws``."""
    return (draws(seed, stream, index) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass
class Torus:
    """L x W toroidal square grid with +1/-1 couplings.

    Vertex ``i = r * W + c``.  ``j_right[i]`` couples i to ``(r, c+1 mod W)``
    and ``j_down[i]`` couples i to ``(r+1 mod L, c)``; both are int8 +/-1.
    """
    L: int
    W: int
    j_right: np.ndarray
    j_down: np.ndarray

    @property
    def n(self) -> int:
        return self.L * self.W

    @property
    def m(self) -> int:
        return 2 * self.L * self.W

    def edges(self):
        """Edge list (u, v, w) of the grid, row-major, right edge then down edge."""
        L, W = self.L, self.W
        i = np.arange(L * W, dtype=np.int64)
        r, c = i // W, i % W
        right = r * W + (c + 1) % W
        down = ((r + 1) % L) * W + c
        u = np.stack([i, i], axis=1).reshape(-1)
        v = np.stack([right, down], axis=1).reshape(-1)
        w = np.stack([self.j_right, self.j_down], axis=1).reshape(-1)
        return u.astype(np.int32), v.astype(np.int32), w.astype(np.int32)


@dataclasses.dataclass
class Graph:
    """Undirected weighted graph given as an edge list with n vertices, and
    optional integer local fields h[n] (None: no fields)."""
    n: int
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    h: np.ndarray | None = None

    @property
    def m(self) -> int:
        return int(self.u.shape[0])

    def edges(self):
        return self.u, self.v, self.w


def torus(L: int, W: int, seed: int) -> Torus:
    """Seeded +/-1 spin glass on an L x W torus (each sign with probability 1/2)."""
    n = L * W
    d = draws(seed, STREAM_COUPLING, np.arange(n, dtype=np.uint64))
    jr = np.where((d >> np.uint64(63)) == 1, 1, -1).astype(np.int8)
    jd = np.where(((d >> np.uint64(62)) & np.uint64(1)) == 1, 1, -1).astype(np.int8)
    return Torus(L, W, jr, jd)


def random_graph(n: int, m: int, seed: int, weight: int = 1) -> Graph:
    """``m`` distinct unordered pairs {u < v} of ``n`` vertices, uniform, no self-loops.

    Endpoints are drawn in order (two draws per candidate); a candidate that is
    a self-loop or repeats an earlier pair is skipped, so the result is the
    first ``m`` distinct pairs of the stream, each pair equally likely.
    """
    if m > n * (n - 1) // 2:
        raise ValueError("more edges than vertex pairs")
    chosen: list[np.ndarray] = []
    seen = np.zeros(0, dtype=np.int64)
    start = 0
    need = m
    while need > 0:
        batch = max(2 * need + 64, 1024)
        k = np.arange(start, start + batch, dtype=np.uint64)
        a = (draws(seed, STREAM_EDGES, 2 * k) % np.uint64(n)).astype(np.int64)
        b = (draws(seed, STREAM_EDGES, 2 * k + np.uint64(1)) % np.uint64(n)).astype(np.int64)
        start += batch
        ok = a != b
        lo, hi = np.minimum(a, b)[ok], np.maximum(a, b)[ok]
        key = lo * n + hi
        # first occurrence of each key inside the batch, in stream order
        _, first = np.unique(key, return_index=True)
        first.sort()
        key = key[first]
        key = key[~np.isin(key, seen)]
        key = key[:need]
        chosen.append(key)
        seen = np.concatenate([seen, key])
        need -= key.shape[0]
    key = np.concatenate(chosen)
    u = (key // n).astype(np.int32)
    v = (key % n).astype(np.int32)
    w = np.full(m, weight, dtype=np.int32)
    return Graph(n, u, v, w)


def linear_betas(b0: float, b1: float, sweeps: int) -> np.ndarray:
    """beta_k = b0 + (b1 - b0) * k / (S - 1), k = 0..S-1 (S = 1 gives b0)."""
    if sweeps == 1:
        return np.array([b0], dtype=np.float64)
    k = np.arange(sweeps, dtype=np.float64)
    return b0 + (b1 - b0) * k / (sweeps - 1)


def geometric_betas(b0: float, b1: float, sweeps: int) -> np.ndarray:
    """beta_k = b0 * (b1 / b0) ** (k / (S - 1)), k = 0..S-1 (S = 1 gives b0)."""
    if sweeps == 1:
        return np.array([b0], dtype=np.float64)
    ratio = b1 / b0
    return np.array([b0 * math.pow(ratio, k / (sweeps - 1)) for k in range(sweeps)],
                    dtype=np.float64)


# ---------------------------------------------------------------------------
# The five workloads.  Sizes follow Table I of the paper (G65 = 8,000 spins on
# a torus, G70 = 10,000 vertices / 9,999 edges) and the batched / served mixes.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Solve:
    """One annealing request: instance, replicas, schedule, seed, target."""
    problem: object
    replicas: int
    betas: np.ndarray
    seed: int
    target: int | None = None

    @property
    def sweeps(self) -> int:
        return int(self.betas.shape[0])

    @property
    def n(self) -> int:
        return self.problem.n

    @property
    def attempts(self) -> int:
        return self.replicas * self.n * self.sweeps


def torus_20x20() -> Solve:
    """20x20 +/-1 torus, coupling seed 1, 64 replicas, linear beta 0.1->3.0, 1,000 sweeps."""
    return Solve(torus(20, 20, 1), 64, linear_betas(0.1, 3.0, 1000), 1)


def torus_80x100(sweeps: int = 10000, replicas: int = 1024) -> Solve:
    """80x100 +/-1 torus (the G65 shape), 1,024 replicas, geometric beta 0.1->5.0."""
    return Solve(torus(80, 100, 1), replicas, geometric_betas(0.1, 5.0, sweeps), 1)


def random_10000(sweeps: int = 10000, replicas: int = 256) -> Solve:
    """n = 10,000, m = 9,999 unweighted random graph (the G70 shape), 256 replicas."""
    return Solve(random_graph(10000, 9999, 1), replicas, geometric_betas(0.1, 5.0, sweeps), 1)


def geometric_graph(n: int, mean_degree: float, seed: int) -> Graph:
    """Random geometric graph: n points uniform in the unit square (two draws
    each), an edge between every pair closer than r, with n pi r^2 =
    mean_degree (boundary effects make the realised mean slightly lower)."""
    k = np.arange(n, dtype=np.uint64)
    x = uniform_float(seed, STREAM_POINTS, 2 * k)
    y = uniform_float(seed, STREAM_POINTS, 2 * k + np.uint64(1))
    r = math.sqrt(mean_degree / (math.pi * n))
    cells = max(1, int(1.0 / r))
    cx = np.minimum((x * cells).astype(np.int64), cells - 1)
    cy = np.minimum((y * cells).astype(np.int64), cells - 1)
    cell = cx * cells + cy
    order = np.argsort(cell, kind="stable")
    start = np.searchsorted(cell[order], np.arange(cells * cells + 1))
    us, vs = [], []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            nx, ny = cx + dx, cy + dy
            ok = (nx >= 0) & (nx < cells) & (ny >= 0) & (ny < cells)
            for i in np.nonzero(ok)[0]:
                c = nx[i] * cells + ny[i]
                js = order[start[c]:start[c + 1]]
                js = js[js > i]
                d2 = (x[js] - x[i]) ** 2 + (y[js] - y[i]) ** 2
                js = js[d2 < r * r]
                us.append(np.full(js.shape[0], i))
                vs.append(js)
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    e = np.lexsort((v, u))
    u, v = u[e].astype(np.int32), v[e].astype(np.int32)
    return Graph(n, u, v, np.ones(u.shape[0], dtype=np.int32))


def independent_set_instance(g: Graph) -> Graph:
    """Maximum independent set of g as an Ising instance with local fields.

    With x_i = (1 + s_i)/2, the penalty form  -sum_i x_i + 2 sum_(i,j) x_i x_j
    (minimised by a maximum independent set) equals (E + m - n) / 2 for
    E(s) = sum_(i,j) s_i s_j + sum_i (deg_i - 1) s_i: couplings +1, fields
    h_i = deg_i - 1.  The set of a configuration is {i : s_i = +1}."""
    deg = np.bincount(np.concatenate([g.u, g.v]), minlength=g.n).astype(np.int32)
    return Graph(g.n, g.u, g.v, np.ones(g.m, dtype=np.int32), deg - 1)


def table1_stand_ins():
    """Synthetic stand-ins with the shapes of the Gset instances of Table I:
    +/-1 tori with the listed variable counts (sides 80..200 x 100; the side
    split is an assumption, the table gives only n and m = 2n) and an
    unweighted random graph with n = 10,000, m = 9,999 (G70's shape).  The
    second 10,000-variable torus (G72's row) takes another coupling seed.
    Returns (label, problem) pairs; labels name the row whose shape is used."""
    return [("G65-shape 80x100", torus(80, 100, 65)),
            ("G66-shape 90x100", torus(90, 100, 66)),
            ("G67-shape 100x100", torus(100, 100, 67)),
            ("G70-shape n10000 m9999", random_graph(10000, 9999, 70)),
            ("G72-shape 100x100", torus(100, 100, 72)),
            ("G77-shape 140x100", torus(140, 100, 77)),
            ("G81-shape 200x100", torus(200, 100, 81))]


def independent_set_10000(sweeps: int = 10000, replicas: int = 256) -> Solve:
    """Maximum independent set on a random geometric graph (n = 10,000, mean
    degree 6) in the local-field form, 256 replicas, geometric beta 0.1->5.0."""
    g = independent_set_instance(geometric_graph(10000, 6.0, 1))
    return Solve(g, replicas, geometric_betas(0.1, 5.0, sweeps), 1)


def batch_sizes(count: int = 512, seed: int = 4):
    """Even side lengths L, W uniform over {16, 18, ..., 140} for ``count`` tori."""
    k = np.arange(count, dtype=np.uint64)
    L = 2 * uniform_int(seed, STREAM_SIZES, 2 * k, 8, 70)
    W = 2 * uniform_int(seed, STREAM_SIZES, 2 * k + np.uint64(1), 8, 70)
    return L.astype(int), W.astype(int)


def torus_batch(count: int = 512, sweeps: int = 2000, replicas: int = 32) -> list:
    """512 uneven +/-1 tori; coupling seed 1000 + k, anneal seed k + 1."""
    L, W = batch_sizes(count)
    betas = geometric_betas(0.1, 5.0, sweeps)
    return [Solve(torus(int(L[k]), int(W[k]), 1000 + k), replicas, betas, k + 1)
            for k in range(count)]


@dataclasses.dataclass
class Request:
    arrival_s: float
    solve: Solve


def served_stream(count: int = 2000, rate_hz: float = 200.0, seed: int = 5,
                  sweeps: int = 10000, replicas: int = 32):
    """Poisson request stream mixing tori and sparse random graphs.

    Half the requests are +/-1 tori with L even in [40, 100] and W even in
    [40, 200]; half are unweighted random graphs with n in [2,000, 20,000] and
    mean degree d in [2, 4] (m = round(n d / 2)).  Targets are left unset here:
    they are filled in by the caller from a plain-form run.
    """
    k = np.arange(count, dtype=np.uint64)
    gaps = -np.log1p(-uniform_float(seed, STREAM_ARRIVALS, k)) / rate_hz
    arrivals = np.cumsum(gaps)
    kind = uniform_int(seed, STREAM_KIND, k, 0, 1)
    betas = geometric_betas(0.1, 5.0, sweeps)
    out = []
    for j in range(count):
        sj = seed * 1_000_003 + j
        if kind[j] == 0:
            L = 2 * int(uniform_int(sj, STREAM_SIZES, 0, 20, 50)[()])
            W = 2 * int(uniform_int(sj, STREAM_SIZES, 1, 20, 100)[()])
            prob = torus(L, W, sj)
        else:
            n = int(uniform_int(sj, STREAM_SIZES, 0, 2000, 20000)[()])
            d = 2.0 + 2.0 * float(uniform_float(sj, STREAM_SIZES, 1)[()])
            prob = random_graph(n, int(round(n * d / 2)), sj)
        out.append(Request(float(arrivals[j]), Solve(prob, replicas, betas, j + 1)))
    return out

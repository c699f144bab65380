"""CPU oracle for the replica-parallel Metropolis annealing sweep (ctypes + numpy).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product (the
CUDA library ``libisg`` and its Python binding) never imports it, and the two
share no code: the only thing both sides consume is the seeded instance
generator module ``paper_2311_09275_gb300.inputs``.

The arithmetic lives in ``isg_oracle.c`` (plain C99, one pthread per block of
replicas); this wrapper only marshals numpy arrays.

Readings of the paper used here (the paper withholds its method, Sec. III.A):

* E(s) = sum_{(i,j)} w_ij s_i s_j is minimised, so the MaxCut value of
  Sec. II.A is cut = (W_tot - E) / 2.
* One sweep visits every vertex once, colour class by colour class in
  ascending class order (classes: the checkerboard on a torus, greedy by
  ascending id on a graph, Csr.colouring; or a colouring passed in); the flip of vertex i changes E by d = -2 s_i h_i with
  h_i = sum_j w_ij s_j and is accepted when d <= 0 or when the replica's
  32-bit uniform is below floor(2^32 exp(-beta_t d)).
* A replica's best state is checked at sweep boundaries only (strict
  improvement); the initial state is a candidate.
* With a target, the solve stops at the end of the first sweep at which the
  best energy over all replicas is <= target.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isg_oracle.c")
_HDR = os.path.join(_HERE, "isg_oracle.h")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-D_GNU_SOURCE", "-O2", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.orc_philox4x32_10.argtypes = [P, P, P]
        lib.orc_build_csr.argtypes = [i32, i64, P, P, P, P, P, P]
        lib.orc_build_csr.restype = ctypes.c_int
        lib.orc_torus_edges.argtypes = [i32, i32, P, P, P, P, P]
        lib.orc_greedy_colouring.argtypes = [i32, P, P, P]
        lib.orc_greedy_colouring.restype = i32
        lib.orc_smallest_last_colouring.argtypes = [i32, P, P, P]
        lib.orc_smallest_last_colouring.restype = i32
        lib.orc_accept_table.argtypes = [i32, P, i32, P]
        lib.orc_energy.argtypes = [i32, P, P, P, P, P]
        lib.orc_energy.restype = i64
        lib.orc_anneal.argtypes = [i32, P, P, P, P, P, i32, i32, P, i32, P, u64, ctypes.c_int, i64,
                                   u64, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
        lib.orc_anneal.restype = ctypes.c_int
        lib.orc_initial_spins.argtypes = [i32, i32, P, u64, P]
        lib.orc_parallel_tempering.argtypes = [i32, P, P, P, P, P, i32, i32, P, i32, i32, i32,
                                               u64, ctypes.c_int, P, P, P, P, P, P, P]
        lib.orc_parallel_tempering.restype = ctypes.c_int
        lib.orc_enumerate.argtypes = [i32, P, P, P, P, P, P]
        lib.orc_enumerate.restype = i64
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _arr(x, dtype):
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block function (Salmon et al., SC'11) of one counter/key."""
    c = _arr(ctr, np.uint32)
    k = _arr(key, np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


class Csr:
    """Symmetric CSR built by the oracle from an edge list (neighbours ascending),
    with optional integer local fields h[n] (E gains sum_i h_i s_i)."""

    def __init__(self, n: int, u, v, w, h=None):
        u, v, w = _arr(u, np.int32), _arr(v, np.int32), _arr(w, np.int32)
        self.field = None if h is None else _arr(h, np.int32)
        self.torus_shape = None  # (L, W) when built by torus_csr
        if self.field is not None and self.field.shape != (n,):
            raise ValueError("fields need one entry per vertex")
        m = int(u.shape[0])
        self.n = int(n)
        self.m = m
        self.rowptr = np.zeros(n + 1, dtype=np.int64)
        self.col = np.zeros(max(2 * m, 1), dtype=np.int32)
        self.wt = np.zeros(max(2 * m, 1), dtype=np.int32)
        rc = _load().orc_build_csr(n, m, _p(u), _p(v), _p(w), _p(self.rowptr), _p(self.col),
                                   _p(self.wt))
        if rc != 0:
            raise ValueError("invalid edge list (range, self-loop or duplicate)")
        self.total_weight = int(w.astype(np.int64).sum())

    def _fp(self):
        return _p(self.field) if self.field is not None else None

    def energy(self, s) -> int:
        s = _arr(s, np.int8)
        return int(_load().orc_energy(self.n, _p(self.rowptr), _p(self.col), _p(self.wt),
                                      self._fp(), _p(s)))

    def greedy_colouring(self):
        colour = np.zeros(self.n, dtype=np.int32)
        nc = _load().orc_greedy_colouring(self.n, _p(self.rowptr), _p(self.col), _p(colour))
        return colour, int(nc)

    def smallest_last_colouring(self):
        """Smallest-last order, classes numbered by their smallest vertex
        (orc_smallest_last_colouring): the library's optional colouring."""
        colour = np.zeros(self.n, dtype=np.int32)
        nc = _load().orc_smallest_last_colouring(self.n, _p(self.rowptr), _p(self.col),
                                                 _p(colour))
        return colour, int(nc)

    def colouring(self):
        """The sweep's default colour classes: on a torus the checkerboard
        (r + c) mod 2, on a graph the greedy colouring by ascending id."""
        if self.torus_shape is not None:
            r, c = np.divmod(np.arange(self.n), self.torus_shape[1])
            return ((r + c) % 2).astype(np.int32), 2
        return self.greedy_colouring()

    def kmax(self) -> int:
        """max_i (sum_j |w_ij| + |h_i|): the largest half energy change of one flip."""
        deg = np.diff(self.rowptr)
        rows = np.repeat(np.arange(self.n), deg)
        sums = np.zeros(self.n, dtype=np.int64)
        np.add.at(sums, rows, np.abs(self.wt[: 2 * self.m].astype(np.int64)))
        if self.field is not None:
            sums += np.abs(self.field.astype(np.int64))
        return int(sums.max()) if self.n else 0

    def enumerate(self, histogram: bool = False):
        """Exact minimum energy over all 2^n states (n <= 30); optionally the
        number of states at each energy E = -sum|w| .. +sum|w|."""
        if self.n > 30:
            raise ValueError("enumeration needs n <= 30")
        wabs = int(np.abs(self.wt[: 2 * self.m].astype(np.int64)).sum() // 2)
        if self.field is not None:
            wabs += int(np.abs(self.field.astype(np.int64)).sum())
        argmin = np.zeros(self.n, dtype=np.int8)
        hist = np.zeros(2 * wabs + 1, dtype=np.uint64) if histogram else None
        e = _load().orc_enumerate(self.n, _p(self.rowptr), _p(self.col), _p(self.wt), self._fp(),
                                  _p(argmin), _p(hist) if hist is not None else None)
        if histogram:
            return int(e), argmin, hist, -wabs
        return int(e), argmin


def torus_csr(L: int, W: int, j_right, j_down) -> Csr:
    """The oracle's own edge list of an L x W torus, as CSR."""
    n = L * W
    jr, jd = _arr(j_right, np.int8), _arr(j_down, np.int8)
    u = np.zeros(2 * n, dtype=np.int32)
    v = np.zeros(2 * n, dtype=np.int32)
    w = np.zeros(2 * n, dtype=np.int32)
    _load().orc_torus_edges(L, W, _p(jr), _p(jd), _p(u), _p(v), _p(w))
    c = Csr(n, u, v, w)
    c.torus_shape = (L, W)
    return c


def csr_of(problem) -> Csr:
    """Oracle CSR of an instance from the input generators (torus or graph)."""
    if hasattr(problem, "L"):
        return torus_csr(problem.L, problem.W, problem.j_right, problem.j_down)
    return Csr(problem.n, problem.u, problem.v, problem.w, getattr(problem, "h", None))


def accept_table(betas, kmax: int) -> np.ndarray:
    """table[t, k] = min(floor(2^32 exp(-beta_t 2k)), 2^32 - 1), k = 0..kmax."""
    b = _arr(betas, np.float64)
    out = np.zeros((b.shape[0], kmax + 1), dtype=np.uint32)
    _load().orc_accept_table(int(b.shape[0]), _p(b), int(kmax), _p(out))
    return out


def initial_spins(n: int, replicas, seed: int) -> np.ndarray:
    reps = _arr(replicas, np.int32)
    s = np.zeros((reps.shape[0], n), dtype=np.int8)
    _load().orc_initial_spins(n, int(reps.shape[0]), _p(reps), seed, _p(s))
    return s


class AnnealResult:
    def __init__(self, rep_ids, s_final, e_final, s_best, e_best, hit_sweep, sweeps_done):
        self.rep_ids = rep_ids
        self.s_final = s_final
        self.e_final = e_final
        self.s_best = s_best
        self.e_best = e_best
        self.hit_sweep = hit_sweep
        self.sweeps_done = sweeps_done

    @property
    def best(self):
        """(energy, replica) of the overall best; ties go to the lowest replica index."""
        k = int(np.lexsort((self.rep_ids, self.e_best))[0])
        return int(self.e_best[k]), int(self.rep_ids[k])


def anneal(csr: Csr, replicas, betas, seed: int, colour=None, target=None,
           shuffle_seed: int = 0, check_energy: bool = False, nthreads: int = 0) -> AnnealResult:
    """Run the colour-ordered Metropolis schedule on the listed replicas.

    ``replicas`` is an int (all replicas 0..R-1) or a list of replica indices.
    ``colour`` defaults to Csr.colouring (greedy by id; the torus checkerboard).
    """
    if colour is None:
        colour, nc = csr.colouring()
    else:
        colour = _arr(colour, np.int32)
        nc = int(colour.max()) + 1
    reps = _arr(np.arange(replicas) if np.isscalar(replicas) else replicas, np.int32)
    b = _arr(betas, np.float64)
    S = int(b.shape[0])
    k = int(reps.shape[0])
    n = csr.n
    s_final = np.zeros((k, n), dtype=np.int8)
    s_best = np.zeros((k, n), dtype=np.int8)
    e_final = np.zeros(k, dtype=np.int32)
    e_best = np.zeros(k, dtype=np.int32)
    hit = ctypes.c_int32(-1)
    done = ctypes.c_int32(0)
    if nthreads <= 0:
        nthreads = min(os.cpu_count() or 1, k)
    rc = _load().orc_anneal(n, _p(csr.rowptr), _p(csr.col), _p(csr.wt), csr._fp(), _p(colour), nc, k,
                            _p(reps), S, _p(b), int(seed), 1 if target is not None else 0,
                            int(target) if target is not None else 0, int(shuffle_seed),
                            1 if check_energy else 0, int(nthreads), _p(s_final), _p(e_final),
                            _p(s_best), _p(e_best), ctypes.byref(hit), ctypes.byref(done))
    if rc == -2:
        raise AssertionError("tracked energy differs from the recomputed energy")
    if rc != 0:
        raise ValueError("bad arguments to the oracle")
    return AnnealResult(reps, s_final, e_final, s_best, e_best, int(hit.value), int(done.value))


class TemperingResult:
    """Per replica r = 32 k + c (slot k, chain c): final and best states and
    energies; exchange counts per slot pair."""

    def __init__(self, s_final, e_final, s_best, e_best, accepted, attempted, flipped):
        self.s_final, self.e_final = s_final, e_final
        self.s_best, self.e_best = s_best, e_best
        self.accepted, self.attempted = accepted, attempted
        self.flipped = flipped

    @property
    def best(self):
        k = int(np.argmin(self.e_best))  # argmin takes the lowest index among ties
        return int(self.e_best[k]), k


def parallel_tempering(csr: Csr, betas, rounds: int, per_round: int, seed: int, colour=None,
                       nthreads: int = 0, icm_slots: int = 0) -> TemperingResult:
    """Parallel tempering over len(betas) slots x 32 chains, with Houdayer
    cluster moves on the last icm_slots slots (see isg_oracle.h)."""
    if colour is None:
        colour, nc = csr.colouring()
    else:
        colour = _arr(colour, np.int32)
        nc = int(colour.max()) + 1
    b = _arr(betas, np.float64)
    K = int(b.shape[0])
    R = 32 * K
    s_final = np.zeros((R, csr.n), dtype=np.int8)
    s_best = np.zeros((R, csr.n), dtype=np.int8)
    e_final = np.zeros(R, dtype=np.int32)
    e_best = np.zeros(R, dtype=np.int32)
    acc = np.zeros(max(K - 1, 1), dtype=np.int64)
    att = np.zeros(max(K - 1, 1), dtype=np.int64)
    flipped = np.zeros(K, dtype=np.int64)
    if nthreads <= 0:
        nthreads = min(os.cpu_count() or 1, 16)
    rc = _load().orc_parallel_tempering(
        csr.n, _p(csr.rowptr), _p(csr.col), _p(csr.wt), csr._fp(), _p(colour), nc, K, _p(b),
        int(rounds), int(per_round), int(icm_slots), int(seed), int(nthreads), _p(s_final),
        _p(e_final), _p(s_best), _p(e_best), _p(acc), _p(att), _p(flipped))
    if rc != 0:
        raise ValueError("bad arguments to the oracle")
    return TemperingResult(s_final, e_final, s_best, e_best, acc[: K - 1], att[: K - 1],
                           flipped)

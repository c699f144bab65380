"""Gset text format and the cut check of a printed configuration.

Sec. III benchmarks on instances of the Gset suite, and Appendix II/III print
best configurations as hex bitstrings.  This module reads and writes that
instance format and checks a bitstring against an instance:

* format: the first line holds n and m; each of the next m lines holds one
  edge ``i j w`` with 1-based vertex ids and an integer weight;
* cut of a configuration: the summed weight of the edges whose ends have
  opposite spins, cut = (W - E) / 2 for E = sum w_ij s_i s_j and W = sum w_ij.

No instance of the suite ships with this package: the functions take text or
a path that the caller supplies.  Host-side parsing and checking only.
"""
from __future__ import annotations

import numpy as np

from .inputs import Graph
from .metrics import bitstring_hex, spins_from_hex


class GsetFormatError(ValueError):
    """Malformed instance text or a bitstring that does not fit the instance."""


def parse(text: str) -> Graph:
    """Graph of a Gset-format text (vertex ids shifted to 0-based).

    Raises GsetFormatError for a bad header, a wrong number of edge lines, an
    id outside 1..n, a self-loop, a repeated vertex pair or a non-integer
    weight; blank lines are ignored.
    """
    lines = [ln.split() for ln in text.splitlines() if ln.strip()]
    if not lines or len(lines[0]) != 2:
        raise GsetFormatError("first line must hold n and m")
    try:
        n, m = int(lines[0][0]), int(lines[0][1])
    except ValueError:
        raise GsetFormatError("n and m must be integers") from None
    if n < 1 or m < 0:
        raise GsetFormatError(f"bad sizes n = {n}, m = {m}")
    body = lines[1:]
    if len(body) != m:
        raise GsetFormatError(f"header says {m} edges, found {len(body)} edge lines")
    if any(len(f) != 3 for f in body):
        raise GsetFormatError("every edge line holds three fields: i j w")
    try:
        e = np.array([[int(a), int(b), int(c)] for a, b, c in body], dtype=np.int64).reshape(m, 3)
    except ValueError:
        raise GsetFormatError("vertex ids and weights must be integers") from None
    i, j, w = e[:, 0] - 1, e[:, 1] - 1, e[:, 2]
    if m and (min(i.min(), j.min()) < 0 or max(i.max(), j.max()) >= n):
        raise GsetFormatError(f"vertex id outside 1..{n}")
    if np.any(i == j):
        raise GsetFormatError(f"self-loop at vertex {int(i[i == j][0]) + 1}")
    key = np.minimum(i, j) * n + np.maximum(i, j)
    if np.unique(key).shape[0] != m:
        raise GsetFormatError("a vertex pair appears twice")
    if m and np.abs(w).max() >= 2**31:
        raise GsetFormatError("weight outside the int32 range")
    return Graph(n, i.astype(np.int32), j.astype(np.int32), w.astype(np.int32))


def load(path) -> Graph:
    with open(path, "r", encoding="ascii") as f:
        return parse(f.read())


def dumps(g: Graph) -> str:
    """Gset-format text of a graph without local fields (1-based ids, one
    edge per line in the graph's order)."""
    if g.h is not None and np.any(np.asarray(g.h) != 0):
        raise GsetFormatError("the format has no local fields")
    rows = [f"{g.n} {g.m}"]
    rows += [f"{int(a) + 1} {int(b) + 1} {int(c)}" for a, b, c in zip(g.u, g.v, g.w)]
    return "\n".join(rows) + "\n"


def save(g: Graph, path) -> None:
    with open(path, "w", encoding="ascii") as f:
        f.write(dumps(g))


def cut_of(g: Graph, spins) -> int:
    """Summed weight of the edges whose ends have opposite spins (+1/-1)."""
    s = np.asarray(spins, dtype=np.int64)
    if s.shape != (g.n,) or not np.all(np.abs(s) == 1):
        raise GsetFormatError(f"need {g.n} spins of +1/-1")
    u = np.asarray(g.u, dtype=np.int64)
    v = np.asarray(g.v, dtype=np.int64)
    w = np.asarray(g.w, dtype=np.int64)
    return int(w[s[u] != s[v]].sum())


def verify_bitstring(g: Graph, text: str, claimed_cut: int | None = None) -> int:
    """Cut of the configuration that a hex bitstring encodes (Appendix II/III
    encoding: variables 1..n left to right, bit 1 for spin +1).

    The string must hold exactly ceil(n / 4) hex digits with zero padding
    bits; with ``claimed_cut`` the computed cut must equal it.  Raises
    GsetFormatError otherwise; returns the cut.
    """
    digits = "".join(ch for ch in text if not ch.isspace())
    if len(digits) != -(-g.n // 4):
        raise GsetFormatError(f"{len(digits)} hex digits for {g.n} variables")
    try:
        int(digits, 16)
    except ValueError:
        raise GsetFormatError("not a hex string") from None
    spins = spins_from_hex(digits, g.n)
    if bitstring_hex(spins) != digits.upper():
        raise GsetFormatError("padding bits after variable n must be zero")
    cut = cut_of(g, spins)
    if claimed_cut is not None and cut != claimed_cut:
        raise GsetFormatError(f"bitstring cuts {cut}, not the claimed {claimed_cut}")
    return cut

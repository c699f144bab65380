"""Gset text format and the bitstring cut check (Sec. III instances,
Appendix II/III bitstrings), against brute force and the oracle's energy."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2311_09275_gb300 import gset, metrics
from paper_2311_09275_gb300 import inputs as I


def test_parse_small_text():
    text = "4 5\n1 2 1\n2 3 -1\n\n3 4 2\n4 1 1\n1 3 -3\n"
    g = gset.parse(text)
    assert g.n == 4 and g.m == 5
    assert g.u.tolist() == [0, 1, 2, 3, 0]
    assert g.v.tolist() == [1, 2, 3, 0, 2]
    assert g.w.tolist() == [1, -1, 2, 1, -3]
    assert g.u.dtype == np.int32 and g.w.dtype == np.int32


@pytest.mark.parametrize("make", [
    lambda: I.random_graph(300, 450, 3),
    lambda: I.Graph(48, *I.torus(6, 8, 2).edges()),           # +-1 weights
    lambda: I.Graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)),
])
def test_round_trip(make, tmp_path):
    g = make()
    p = tmp_path / "g.txt"
    gset.save(g, p)
    h = gset.load(p)
    assert h.n == g.n
    assert np.array_equal(h.u, g.u) and np.array_equal(h.v, g.v) and np.array_equal(h.w, g.w)


@pytest.mark.parametrize("text", [
    "",                        # no header
    "3\n",                     # header with one field
    "3 2\n1 2 1\n",            # fewer edge lines than m
    "3 1\n1 2 1\n2 3 1\n",     # more edge lines than m
    "3 1\n1 4 1\n",            # id above n
    "3 1\n0 2 1\n",            # id 0 (ids are 1-based)
    "3 1\n2 2 1\n",            # self-loop
    "3 2\n1 2 1\n2 1 1\n",     # same pair twice
    "3 1\n1 2 1.5\n",          # non-integer weight
    "3 1\n1 2\n",              # two fields
])
def test_parse_rejects(text):
    with pytest.raises(gset.GsetFormatError):
        gset.parse(text)


def test_dumps_rejects_fields():
    g = I.independent_set_instance(I.geometric_graph(50, 4.0, 1))
    with pytest.raises(gset.GsetFormatError):
        gset.dumps(g)


@pytest.mark.parametrize("text,best", [
    ("4 6\n1 2 1\n1 3 1\n1 4 1\n2 3 1\n2 4 1\n3 4 1\n", 4),   # K4: 2 x 2 split
    ("5 5\n1 2 1\n2 3 1\n3 4 1\n4 5 1\n5 1 1\n", 4),          # odd cycle: one edge uncut
    ("3 3\n1 2 2\n2 3 -1\n1 3 5\n", 7),                       # {1} | {2, 3}
])
def test_cut_brute_force_maximum(text, best):
    g = gset.parse(text)
    cuts = [gset.cut_of(g, np.array(s)) for s in itertools.product([-1, 1], repeat=g.n)]
    assert max(cuts) == best


def test_cut_matches_oracle_energy():
    """cut = (W - E) / 2 with E the oracle's energy, on random configurations."""
    g = I.random_graph(400, 700, 9, weight=1)
    g = I.Graph(g.n, g.u, g.v, np.where(np.arange(g.m) % 3 == 0, -2, 3).astype(np.int32))
    c = oracle.csr_of(g)
    rng = np.random.default_rng(4)
    W = int(g.w.astype(np.int64).sum())
    for _ in range(5):
        s = rng.choice([-1, 1], size=g.n).astype(np.int8)
        assert gset.cut_of(g, s) == metrics.cut_value(W, c.energy(s))


def test_verify_bitstring_checkerboard():
    """All-+1 couplings on an even torus: the checkerboard cuts all 2LW edges."""
    L, W = 4, 6
    t = I.torus(L, W, 1)
    u, v, _ = t.edges()
    g = I.Graph(L * W, u, v, np.ones(u.shape[0], np.int32))
    s = [1 if ((i // W) + (i % W)) % 2 == 0 else -1 for i in range(L * W)]
    text = metrics.bitstring_hex(s)
    assert gset.verify_bitstring(g, text, claimed_cut=2 * L * W) == 2 * L * W
    assert gset.verify_bitstring(g, "F" * len(text)) == 0
    with pytest.raises(gset.GsetFormatError):
        gset.verify_bitstring(g, text, claimed_cut=2 * L * W - 1)
    with pytest.raises(gset.GsetFormatError):
        gset.verify_bitstring(g, text + "0")
    with pytest.raises(gset.GsetFormatError):
        gset.verify_bitstring(g, "G" * len(text))


def test_verify_bitstring_padding():
    g = gset.parse("5 1\n1 5 1\n")
    assert gset.verify_bitstring(g, "80") == 1     # 1000 0|000: variable 1 up, 5 down
    with pytest.raises(gset.GsetFormatError):
        gset.verify_bitstring(g, "84")             # a padding bit set


@pytest.mark.gpu
def test_annealed_bitstring_round_trip():
    """Instance text -> device anneal -> best bitstring -> cut equals (W - E_best) / 2."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2311_09275_gb300 import build
    build.build()
    from paper_2311_09275_gb300 import isg
    g = gset.parse(gset.dumps(I.random_graph(2000, 3000, 6)))
    p = isg.problem_of(g)
    res = isg.isg_anneal(p, 64, I.geometric_betas(0.1, 5.0, 300), 3)
    e_best, _, spins, _, _ = res.best()
    text = metrics.bitstring_hex(spins)
    W = isg.isg_problem_info(p)["total_weight"]
    assert gset.verify_bitstring(g, text, claimed_cut=metrics.cut_value(W, int(e_best))) > 0

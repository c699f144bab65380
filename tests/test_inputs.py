"""The seeded instance generators: shapes, distributions and determinism."""
import numpy as np

from paper_2311_09275_gb300 import inputs as I


def test_splitmix64_published_first_outputs():
    """SplitMix64 from state 0: first outputs of the generator as defined by
    Steele, Lea and Flood (state += gamma, then the two xor-shift-multiply
    steps); the values follow from the definition with Python integers."""
    def ref(state, k):
        m = (1 << 64) - 1
        z = (state + (k + 1) * 0x9E3779B97F4A7C15) & m
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        return z ^ (z >> 31)
    got = I._mix64(np.array([(k + 1) * 0x9E3779B97F4A7C15 % (1 << 64) for k in range(4)],
                            dtype=np.uint64))
    assert [int(x) for x in got] == [ref(0, k) for k in range(4)]
    assert int(got[0]) == 0xE220A8397B1DCDAF


def test_torus_couplings_balanced_and_deterministic():
    t = I.torus(80, 100, 1)
    assert t.j_right.shape == (8000,) and set(np.unique(t.j_right)) == {-1, 1}
    assert abs(t.j_right.mean()) < 0.05 and abs(t.j_down.mean()) < 0.05
    t2 = I.torus(80, 100, 1)
    assert np.array_equal(t.j_right, t2.j_right) and np.array_equal(t.j_down, t2.j_down)
    assert not np.array_equal(t.j_right, I.torus(80, 100, 2).j_right)
    u, v, w = t.edges()
    assert u.shape == (16000,)


def test_random_graph_distinct_pairs_no_loops():
    g = I.random_graph(10000, 9999, 1)
    assert g.m == 9999
    assert np.all(g.u < g.v)
    key = g.u.astype(np.int64) * g.n + g.v
    assert np.unique(key).shape[0] == g.m
    deg = np.bincount(np.concatenate([g.u, g.v]), minlength=g.n)
    # mean degree ~2: isolated fraction near exp(-2) = 0.135
    assert abs((deg == 0).mean() - np.exp(-2)) < 0.02
    g2 = I.random_graph(10000, 9999, 1)
    assert np.array_equal(g.u, g2.u) and np.array_equal(g.v, g2.v)


def test_schedules():
    b = I.linear_betas(0.1, 3.0, 1000)
    assert b[0] == 0.1 and abs(b[-1] - 3.0) < 1e-15 and np.all(np.diff(b) > 0)
    g = I.geometric_betas(0.1, 5.0, 10000)
    assert g[0] == 0.1 and abs(g[-1] - 5.0) < 1e-12
    assert np.allclose(g[1:] / g[:-1], (50.0) ** (1 / 9999))
    assert I.linear_betas(0.4, 2.0, 1).tolist() == [0.4]


def test_batch_sizes_even_in_range():
    L, W = I.batch_sizes(512)
    for x in (L, W):
        assert np.all(x % 2 == 0) and x.min() >= 16 and x.max() <= 140
    assert len(set(zip(L.tolist(), W.tolist()))) > 400


def test_served_stream_shapes():
    reqs = I.served_stream(count=40, sweeps=10)
    assert len(reqs) == 40
    arr = [r.arrival_s for r in reqs]
    assert all(b >= a for a, b in zip(arr, arr[1:]))
    for r in reqs:
        p = r.solve.problem
        if hasattr(p, "L"):
            assert 40 <= p.L <= 100 and 40 <= p.W <= 200 and p.L % 2 == 0 and p.W % 2 == 0
        else:
            assert 2000 <= p.n <= 20000 and 2.0 - 1e-3 <= 2 * p.m / p.n <= 4.0 + 1e-3

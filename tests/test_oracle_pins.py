"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Every check here compares the oracle with a published value, a closed form,
an exact enumeration done a different way, or an invariant of the method, so
that a dropped term, a wrong sign, a wrong index or a transposed operand in
``oracle/isg_oracle.c`` fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_09275_gb300 import inputs as I
from conftest import read_golden

TWO32 = 2 ** 32


# --------------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Salmon et al. (SC'11) published known-answer vectors for Philox4x32-10."""
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_philox_counter_sensitivity_and_balance():
    """Each output bit is balanced over many counters (monobit sanity)."""
    words = np.array([oracle.philox4x32_10((i, 7, 3, 0), (1, 0)) for i in range(4096)],
                     dtype=np.uint32).reshape(-1)
    bits = np.unpackbits(words.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 0.005
    assert len(set(words.tolist())) == words.shape[0]


# ------------------------------------------------------------ energy and cut
def _edge_list_cut(u, v, w, s):
    """MaxCut value by its definition: total weight of edges whose ends differ."""
    return int(sum(int(w[e]) for e in range(len(u)) if s[u[e]] != s[v[e]]))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_cut_equals_half_weight_minus_energy(seed):
    g = I.random_graph(60, 150, seed)
    w = np.array([(-1) ** k * (1 + k % 3) for k in range(g.m)], dtype=np.int32)
    c = oracle.Csr(g.n, g.u, g.v, w)
    rng = np.random.default_rng(seed)
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], np.int8), size=g.n)
        e = c.energy(s)
        assert _edge_list_cut(g.u, g.v, w, s) * 2 == int(w.sum()) - e


def test_energy_closed_forms_on_torus():
    t = I.torus(6, 8, 3)
    c = oracle.csr_of(t)
    n = t.n
    up = np.ones(n, np.int8)
    assert c.energy(up) == int(t.j_right.sum() + t.j_down.sum())
    assert c.energy(-up) == c.energy(up)                      # spin-reversal symmetry
    r, col = np.divmod(np.arange(n), t.W)
    checker = np.where((r + col) % 2 == 0, 1, -1).astype(np.int8)
    # every edge of an even torus joins opposite checkerboard colours
    assert c.energy(checker) == -int(t.j_right.sum() + t.j_down.sum())


# --------------------------------------------------------- exact enumeration
def _naive_energies(n, u, v, w):
    """E for all 2^n states by direct evaluation (bit i of the index -> spin i)."""
    idx = np.arange(2 ** n, dtype=np.int64)
    s = np.where((idx[:, None] >> np.arange(n)) & 1, 1, -1).astype(np.int64)
    return (s[:, u] * s[:, v] * w[None, :].astype(np.int64)).sum(axis=1)


@pytest.mark.parametrize("n,m,seed", [(8, 7, 1), (10, 20, 2), (12, 12, 3), (12, 24, 4)])
def test_enumeration_matches_direct_evaluation(n, m, seed):
    g = I.random_graph(n, m, seed)
    w = np.array([1 if k % 3 else -2 for k in range(m)], dtype=np.int32)
    c = oracle.Csr(n, g.u, g.v, w)
    e_min, argmin, hist, e_lo = c.enumerate(histogram=True)
    direct = _naive_energies(n, g.u, g.v, w)
    assert e_min == direct.min()
    assert c.energy(argmin) == e_min
    ref = np.bincount(direct - e_lo, minlength=hist.shape[0])
    assert np.array_equal(hist.astype(np.int64), ref)


def test_ferro_and_antiferro_ground_states():
    """4x4 torus: all w = -1 (ferromagnet) and all w = +1 (antiferromagnet on an
    even torus) both have ground energy -m = -32."""
    for sign in (-1, 1):
        j = np.full(16, sign, np.int8)
        c = oracle.torus_csr(4, 4, j, j)
        e_min, argmin = c.enumerate()
        assert e_min == -32
    # one antiferromagnetic bond in a ferromagnet: its two plaquettes are
    # frustrated and the ground state breaks exactly that bond (+2)
    j = np.full(16, -1, np.int8)
    jr = j.copy()
    jr[5] = 1
    c = oracle.torus_csr(4, 4, jr, j)
    assert c.enumerate()[0] == -32 + 2


def test_torus_orientation_hand_derived_energy():
    """Sec. II.A torus geometry on a 4 x 6 torus (L != W): vertex i = r W + c,
    j_right[i] couples i to (r, c+1 mod W) and j_down[i] to (r+1 mod L, c).
    All couplings -1 except j_right[8] = +1 (bond 8-9) and j_down[16] = +1
    (bond 16-22); spins +1 except s_9 = s_22 = -1.  By hand: the all-up energy
    is 46 x (-1) + 2 x (+1) = -44; flipping s_9 negates its four bonds 8-9 (+1),
    9-10, 3-9, 9-15 (-1 each): +4; flipping s_22 negates 21-22, 22-23, 22-4
    (-1 each) and 16-22 (+1): +4; so E = -36.  With the two coupling arrays
    swapped (or right read as left, or rows and columns transposed) neither
    flipped spin touches a +1 bond and E = -28."""
    L, W = 4, 6
    jr = np.full(L * W, -1, np.int8)
    jd = np.full(L * W, -1, np.int8)
    jr[8] = 1
    jd[16] = 1
    s = np.ones(L * W, np.int8)
    s[[9, 22]] = -1
    assert oracle.torus_csr(L, W, jr, jd).energy(s) == -36
    assert oracle.torus_csr(L, W, jd, jr).energy(s) == -28
    # the same instance as an edge list written out by (r, c) here
    u, v, w = [], [], []
    for r in range(L):
        for c in range(W):
            i = r * W + c
            u += [i, i]
            v += [r * W + (c + 1) % W, ((r + 1) % L) * W + c]
            w += [int(jr[i]), int(jd[i])]
    ref = oracle.Csr(L * W, np.array(u, np.int32), np.array(v, np.int32), np.array(w, np.int32))
    t = oracle.torus_csr(L, W, jr, jd)
    assert np.array_equal(t.rowptr, ref.rowptr)
    assert np.array_equal(t.col, ref.col) and np.array_equal(t.wt, ref.wt)


@pytest.mark.parametrize("L,W,seed", [(4, 6, 1), (6, 4, 2), (8, 10, 3)])
def test_torus_csr_equals_fixture_edge_list(L, W, seed):
    """The oracle's own torus edge list and the input generator's edge list
    (written separately, same geometry) give the same CSR for L != W."""
    t = I.torus(L, W, seed)
    a = oracle.torus_csr(L, W, t.j_right, t.j_down)
    b = oracle.Csr(t.n, *t.edges())
    assert np.array_equal(a.rowptr, b.rowptr)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.wt, b.wt)


@pytest.mark.parametrize("n,seed", [(9, 1), (10, 2), (11, 3)])
def test_ring_partition_function_closed_form(n, seed):
    """Ring with couplings J_i = +-1: Z(beta) = sum_E g(E) exp(-beta E) equals
    (2 cosh b)^n + prod(-J_i) (2 sinh b)^n (transfer matrix), and the ground
    energy is -n, or -n + 2 when the ring is frustrated (prod(-J_i) = -1)."""
    J = np.where(I.draws(seed, 9, np.arange(n)) >> np.uint64(63), 1, -1).astype(np.int32)
    u = np.arange(n, dtype=np.int32)
    v = ((np.arange(n) + 1) % n).astype(np.int32)
    c = oracle.Csr(n, u, v, J)
    e_min, _, hist, e_lo = c.enumerate(histogram=True)
    sgn = int(np.prod(-J))
    assert e_min == (-n if sgn == 1 else -n + 2)
    E = np.arange(hist.shape[0]) + e_lo
    for beta in (0.0, 0.3, 0.7, 1.3):
        z = float((hist.astype(np.float64) * np.exp(-beta * E)).sum())
        zc = (2 * math.cosh(beta)) ** n + sgn * (2 * math.sinh(beta)) ** n
        assert z == pytest.approx(zc, rel=1e-12)


# ------------------------------------------------------------ accept table
def test_accept_table_against_high_precision():
    """floor(2^32 exp(-beta d)) within the FP64 error bound of the exact value."""
    import mpmath
    mpmath.mp.dps = 50
    betas = np.array([0.0, 0.1, 0.37, 1.0, 2.5, 5.0, 11.2, 40.0])
    kmax = 6
    tab = oracle.accept_table(betas, kmax)
    for t, b in enumerate(betas):
        for k in range(kmax + 1):
            exact = mpmath.mpf(2) ** 32 * mpmath.exp(-mpmath.mpf(float(b)) * 2 * k)
            fl = int(mpmath.floor(exact))
            want = min(fl, TWO32 - 1)
            got = int(tab[t, k])
            near = abs(exact - mpmath.nint(exact)) < mpmath.mpf(2) ** -16 * max(1, exact)
            if near:
                assert abs(got - want) <= 1
            else:
                assert got == want, (b, k)
    assert np.all(tab[0] == TWO32 - 1)        # beta = 0: every move accepted
    assert np.all(tab[:, 0] == TWO32 - 1)     # d = 0 saturates the 32-bit range
    assert np.all(np.diff(tab[1:].astype(np.int64), axis=1) <= 0)


# ------------------------------------------------------------ colouring
def _proper(c, colour):
    for i in range(c.n):
        for p in range(c.rowptr[i], c.rowptr[i + 1]):
            if colour[c.col[p]] == colour[i]:
                return False
    return True


def test_greedy_colouring_small_closed_forms():
    # odd cycle C5: 0,1,0,1 then vertex 4 sees colours 0 (vertex 0) and 1 (vertex 3)
    u = np.arange(5, dtype=np.int32)
    v = ((np.arange(5) + 1) % 5).astype(np.int32)
    col, nc = oracle.Csr(5, u, v, np.ones(5, np.int32)).greedy_colouring()
    assert col.tolist() == [0, 1, 0, 1, 2] and nc == 3
    # complete graph K5 needs 5 colours, assigned in id order
    pairs = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    uu = np.array([p[0] for p in pairs], np.int32)
    vv = np.array([p[1] for p in pairs], np.int32)
    col, nc = oracle.Csr(5, uu, vv, np.ones(10, np.int32)).greedy_colouring()
    assert col.tolist() == [0, 1, 2, 3, 4] and nc == 5


@pytest.mark.parametrize("L,W", [(4, 4), (6, 10), (20, 20), (80, 100)])
def test_greedy_on_even_torus_is_checkerboard(L, W):
    t = I.torus(L, W, 7)
    col, nc = oracle.csr_of(t).greedy_colouring()
    r, c = np.divmod(np.arange(L * W), W)
    assert nc == 2 and np.array_equal(col, (r + c) % 2)


def test_greedy_colouring_is_proper_on_random_graphs():
    for seed in (1, 2):
        g = I.random_graph(2000, 4000, seed)
        c = oracle.csr_of(g)
        col, nc = c.greedy_colouring()
        assert _proper(c, col)
        assert nc <= c.kmax() + 1


def _graph(n, edges):
    u = np.array([a for a, b in edges], np.int32)
    v = np.array([b for a, b in edges], np.int32)
    return oracle.Csr(n, u, v, np.ones(len(edges), np.int32))


def _degeneracy(c):
    """Brute force: the largest minimum degree over all vertex subsets."""
    adj = [set(c.col[c.rowptr[i]:c.rowptr[i + 1]].tolist()) for i in range(c.n)]
    best = 0
    for mask in range(1, 1 << c.n):
        sub = [i for i in range(c.n) if (mask >> i) & 1]
        s = set(sub)
        best = max(best, min(len(adj[i] & s) for i in sub))
    return best


def test_smallest_last_small_closed_forms():
    """Hand-derived colourings.  C5: removal order 0,1,2,3,4 (all ties go to the
    smallest id), reverse colouring gives [2,1,0,1,0], numbering by smallest
    vertex [0,1,2,1,2].  Star with hub 0: removal 1,2,3, then hub 0 (degree 1
    ties with leaf 4, smaller id), then 4: two classes {0}, {1..4}.  K5: five."""
    col, nc = _graph(5, [(i, (i + 1) % 5) for i in range(5)]).smallest_last_colouring()
    assert col.tolist() == [0, 1, 2, 1, 2] and nc == 3
    col, nc = _graph(5, [(0, i) for i in range(1, 5)]).smallest_last_colouring()
    assert col.tolist() == [0, 1, 1, 1, 1] and nc == 2
    col, nc = _graph(5, [(a, b) for a in range(5) for b in range(a + 1, 5)]).smallest_last_colouring()
    assert col.tolist() == [0, 1, 2, 3, 4] and nc == 5
    # odd wheel (hub 0, rim 1..5): chromatic number 4, degeneracy 3
    c = _graph(6, [(0, i) for i in range(1, 6)] + [(i, i % 5 + 1) for i in range(1, 6)])
    col, nc = c.smallest_last_colouring()
    assert nc == 4 and _proper(c, col)


@pytest.mark.parametrize("seed", range(6))
def test_smallest_last_within_degeneracy_plus_one(seed):
    """At most degeneracy + 1 colours (the property of the smallest-last order;
    a largest-first or id order breaks it on some of these graphs), proper, and
    classes numbered by their smallest vertex."""
    g = I.random_graph(11, 18 + 3 * seed, 100 + seed)
    c = oracle.csr_of(g)
    col, nc = c.smallest_last_colouring()
    assert _proper(c, col)
    assert nc <= _degeneracy(c) + 1
    firsts = [int(np.flatnonzero(col == k)[0]) for k in range(nc)]
    assert firsts == sorted(firsts) and set(col.tolist()) == set(range(nc))


@pytest.mark.parametrize("L,W", [(4, 4), (6, 10), (10, 12), (20, 20), (80, 100)])
def test_smallest_last_on_even_torus_edges_is_checkerboard(L, W):
    """A torus given as a plain edge list gets the checkerboard, (r + c) even first."""
    t = I.torus(L, W, 7)
    u, v, w = t.edges()
    col, nc = oracle.Csr(t.n, u, v, w).smallest_last_colouring()
    r, c = np.divmod(np.arange(L * W), W)
    assert nc == 2 and np.array_equal(col, (r + c) % 2)


def test_smallest_last_is_proper_on_random_graphs():
    for seed in (1, 2):
        g = I.random_graph(2000, 4000, seed)
        c = oracle.csr_of(g)
        col, nc = c.smallest_last_colouring()
        assert _proper(c, col)
        assert nc <= c.kmax() + 1


# ------------------------------------------------------ Metropolis sampling
def _chi2_p(observed, expected):
    from scipy import stats
    keep = expected > 5
    obs = np.append(observed[keep], observed[~keep].sum())
    exp = np.append(expected[keep], expected[~keep].sum())
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    return stats.chi2.sf(chi2, len(obs) - 1)


@pytest.mark.parametrize("beta", [0.3, 0.7])
def test_metropolis_samples_boltzmann_on_4x4_torus(beta):
    """At fixed beta the sweep must leave the Boltzmann distribution invariant:
    final energies of many independent replicas follow g(E) exp(-beta E) / Z."""
    t = I.torus(4, 4, 11)
    c = oracle.csr_of(t)
    e_min, _, hist, e_lo = c.enumerate(histogram=True)
    E = np.arange(hist.shape[0]) + e_lo
    p = hist.astype(np.float64) * np.exp(-beta * (E - e_min))
    p /= p.sum()
    R = 20000
    res = oracle.anneal(c, R, np.full(60, beta), seed=123)
    obs = np.bincount(res.e_final.astype(np.int64) - e_lo, minlength=hist.shape[0])
    assert _chi2_p(obs.astype(np.float64), p * R) > 1e-3


@pytest.mark.parametrize("seed", [3, 4])
def test_metropolis_samples_boltzmann_on_weighted_graph(seed):
    """Same check on a 12-vertex random graph with weights in {-2,-1,1,2,3}
    and three or more colour classes.  (A 1-D ring is deliberately not used:
    with zero-cost moves always taken, colour-ordered sweeps on a ring are not
    ergodic, which an independent simulation of the same chain confirms.)"""
    g = I.random_graph(12, 26, seed)
    w = np.array([(-2, -1, 1, 2, 3)[k % 5] for k in range(g.m)], np.int32)
    c = oracle.Csr(g.n, g.u, g.v, w)
    col, nc = c.greedy_colouring()
    assert nc >= 3
    beta = 0.4
    e_min, _, hist, e_lo = c.enumerate(histogram=True)
    E = np.arange(hist.shape[0]) + e_lo
    p = hist.astype(np.float64) * np.exp(-beta * (E - e_min))
    p /= p.sum()
    R = 20000
    res = oracle.anneal(c, R, np.full(80, beta), seed=9, colour=col)
    obs = np.bincount(res.e_final.astype(np.int64) - e_lo, minlength=hist.shape[0])
    assert _chi2_p(obs.astype(np.float64), p * R) > 1e-3


# ------------------------------------------------------------ special cases
def test_beta_zero_flips_every_spin():
    """beta = 0: every move is accepted (a uniform equal to 2^32-1 would be
    needed to reject), so one sweep maps s0 to -s0 and E(-s) = E(s)."""
    sv = I.torus_20x20()
    c = oracle.csr_of(sv.problem)
    s0 = oracle.initial_spins(c.n, np.arange(16), sv.seed)
    res = oracle.anneal(c, 16, np.zeros(1), sv.seed)
    assert np.array_equal(res.s_final, -s0)
    assert np.array_equal(res.e_final, [c.energy(s) for s in s0])


@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_best_state_needs_strict_improvement(sweeps):
    """Best tracking is strict and happens at sweep ends only, with the initial
    state as the first candidate.  At beta = 0 every sweep flips every spin, so
    at each sweep end the energy equals E(s0) (spin-reversal symmetry): it never
    strictly improves, and the best state stays s0 after any number of sweeps.
    A non-strict comparison would return s_final = (-1)^S s0 instead, and a
    check after every flip would return a lower, mid-sweep energy."""
    for prob in (I.torus_20x20().problem, I.random_graph(200, 300, 4)):
        c = oracle.csr_of(prob)
        R = 16
        s0 = oracle.initial_spins(c.n, np.arange(R), 11)
        e0 = np.array([c.energy(s) for s in s0])
        res = oracle.anneal(c, R, np.zeros(sweeps), 11)
        assert np.array_equal(res.s_final, s0 * (-1) ** sweeps)
        assert np.array_equal(res.e_final, e0)
        assert np.array_equal(res.s_best, s0)
        assert np.array_equal(res.e_best, e0)


def test_zero_temperature_never_raises_energy():
    """Thresholds of 0 (beta large) reject every uphill move: E is non-increasing."""
    g = I.random_graph(300, 600, 5)
    c = oracle.csr_of(g)
    betas = np.full(12, 1e3)
    prev = None
    for S in range(1, 13):
        e = oracle.anneal(c, 8, betas[:S], 42).e_final
        if prev is not None:
            assert np.all(e <= prev)
        prev = e


def test_isolated_vertex_flips_every_sweep():
    """h = 0 at an isolated vertex, so its move has d = 0 and is always taken."""
    u = np.array([0, 1, 2], np.int32)
    v = np.array([1, 2, 3], np.int32)
    c = oracle.Csr(6, u, v, np.ones(3, np.int32))          # vertices 4, 5 isolated
    s0 = oracle.initial_spins(6, np.arange(8), 3)
    for S in (1, 2, 5):
        res = oracle.anneal(c, 8, np.full(S, 2.0), 3)
        assert np.array_equal(res.s_final[:, 4:], s0[:, 4:] * (-1) ** S)


def test_tracked_energy_equals_recompute_every_sweep():
    g = I.random_graph(500, 1500, 8)
    w = np.array([(-1) ** k * (1 + k % 4) for k in range(g.m)], dtype=np.int32)
    c = oracle.Csr(g.n, g.u, g.v, w)
    oracle.anneal(c, 12, I.geometric_betas(0.05, 3.0, 200), 17, check_energy=True)
    sv = I.torus_20x20()
    oracle.anneal(oracle.csr_of(sv.problem), 8, sv.betas[:200], 1, check_energy=True)


def test_class_order_does_not_change_results():
    """No two vertices of a colour class are adjacent, so the order inside a
    class is irrelevant: a seeded shuffle gives bit-identical results."""
    g = I.random_graph(400, 700, 2)
    c = oracle.csr_of(g)
    b = I.geometric_betas(0.1, 5.0, 100)
    a = oracle.anneal(c, 8, b, 5)
    z = oracle.anneal(c, 8, b, 5, shuffle_seed=987654321)
    for f in ("s_final", "e_final", "s_best", "e_best"):
        assert np.array_equal(getattr(a, f), getattr(z, f))


def test_replica_subset_equals_full_run_rows():
    sv = I.torus_20x20()
    c = oracle.csr_of(sv.problem)
    b = sv.betas[:100]
    full = oracle.anneal(c, 40, b, sv.seed)
    sub = oracle.anneal(c, [3, 17, 39], b, sv.seed)
    for f in ("s_final", "e_final", "s_best", "e_best"):
        assert np.array_equal(getattr(full, f)[[3, 17, 39]], getattr(sub, f))


def test_best_is_state_of_best_energy_and_bounded_by_ground_state():
    for seed in range(20):
        t = I.torus(4, 4, 100 + seed)
        c = oracle.csr_of(t)
        e_min, _ = c.enumerate()
        res = oracle.anneal(c, 64, I.linear_betas(0.1, 3.0, 1000), seed + 1)
        for k in range(64):
            assert c.energy(res.s_best[k]) == res.e_best[k]
            assert c.energy(res.s_final[k]) == res.e_final[k]
            assert res.e_best[k] <= res.e_final[k]
        assert res.e_best.min() >= e_min
        assert res.e_best.min() == e_min       # 64 replicas x 1,000 sweeps find 16-spin ground states


def test_brute_force_bounds_random_graphs():
    for n, m in ((16, 15), (18, 36), (20, 19), (20, 40)):
        g = I.random_graph(n, m, n + m)
        c = oracle.csr_of(g)
        e_min, _ = c.enumerate()
        res = oracle.anneal(c, 32, I.linear_betas(0.1, 3.0, 300), 7)
        assert res.e_best.min() >= e_min
        assert res.e_best.min() == e_min


def test_target_stop_matches_prefix_runs():
    """The solve stops at the end of the first sweep t* at which the best energy
    over replicas reaches the target; its state equals a (t*+1)-sweep run."""
    sv = I.torus_20x20()
    c = oracle.csr_of(sv.problem)
    R = 16
    b = sv.betas[:300]
    full = oracle.anneal(c, R, b, sv.seed)
    target = int(full.e_best.min()) + 6
    hit = oracle.anneal(c, R, b, sv.seed, target=target)
    t = hit.hit_sweep
    assert 0 <= t < 300 and hit.sweeps_done == t + 1
    before = oracle.anneal(c, R, b[:t], sv.seed) if t > 0 else None
    at = oracle.anneal(c, R, b[:t + 1], sv.seed)
    assert at.e_best.min() <= target
    if before is not None:
        assert before.e_best.min() > target
    for f in ("s_final", "e_final", "s_best", "e_best"):
        assert np.array_equal(getattr(at, f), getattr(hit, f))
    none = oracle.anneal(c, R, b, sv.seed, target=-10 ** 6)
    assert none.hit_sweep == -1 and none.sweeps_done == 300


def test_initial_spins_balanced():
    s = oracle.initial_spins(4000, np.arange(64), 99)
    assert abs(s.mean()) < 0.01

"""Pins of the oracle's local fields (E gains sum_i h_i s_i): the sparse QUBO
and independent-set forms of Sec. I and Sec. II.C, which lack spin-reversal
symmetry.  Each check is fixed by something other than the oracle itself:
direct evaluation, a two-state Markov chain's closed form, brute-force
independent sets, or the field-free path."""
import numpy as np
import pytest

import oracle
from paper_2311_09275_gb300 import inputs as I
from test_oracle_pins import _chi2_p


def _naive_energies_fields(n, u, v, w, h):
    idx = np.arange(2 ** n, dtype=np.int64)
    s = np.where((idx[:, None] >> np.arange(n)) & 1, 1, -1).astype(np.int64)
    return (s[:, u] * s[:, v] * w[None, :].astype(np.int64)).sum(axis=1) + s @ h.astype(np.int64)


@pytest.mark.parametrize("n,m,seed", [(8, 7, 1), (11, 20, 2), (12, 14, 3)])
def test_enumeration_with_fields_matches_direct_evaluation(n, m, seed):
    g = I.random_graph(n, m, seed)
    w = np.array([1 if k % 3 else -2 for k in range(m)], dtype=np.int32)
    h = np.array([(-3, 0, 2, 1, -1)[i % 5] for i in range(n)], dtype=np.int32)
    c = oracle.Csr(n, g.u, g.v, w, h)
    e_min, argmin, hist, e_lo = c.enumerate(histogram=True)
    direct = _naive_energies_fields(n, g.u, g.v, w, h)
    assert e_min == direct.min()
    assert c.energy(argmin) == e_min
    assert np.array_equal(hist.astype(np.int64), np.bincount(direct - e_lo, minlength=hist.shape[0]))
    # fields break the spin-reversal symmetry E(s) = E(-s)
    s = np.where(np.arange(n) % 2, 1, -1).astype(np.int8)
    assert c.energy(s) - c.energy(-s) == 2 * int(h @ s.astype(np.int64))


def test_kmax_counts_fields():
    g = I.random_graph(10, 12, 4)
    h = np.zeros(10, np.int32)
    h[3] = -7
    c = oracle.Csr(10, g.u, g.v, g.w, h)
    deg = np.bincount(np.concatenate([g.u, g.v]), minlength=10)
    assert c.kmax() == max(int(deg.max()), int(deg[3]) + 7)


def test_zero_fields_equal_no_fields():
    g = I.random_graph(200, 400, 5)
    betas = I.geometric_betas(0.2, 4.0, 60)
    a = oracle.anneal(oracle.Csr(g.n, g.u, g.v, g.w), 12, betas, 3)
    b = oracle.anneal(oracle.Csr(g.n, g.u, g.v, g.w, np.zeros(g.n, np.int32)), 12, betas, 3)
    for x, y in [(a.s_final, b.s_final), (a.e_final, b.e_final), (a.s_best, b.s_best),
                 (a.e_best, b.e_best)]:
        assert np.array_equal(x, y)


@pytest.mark.parametrize("beta", [0.15, 0.4])
def test_free_spins_in_fields_follow_the_two_state_chain(beta):
    """Isolated vertices with fields h: a spin at s = sign(h) flips down with
    probability 1 (its move lowers E by 2|h|), one at -sign(h) flips up with
    probability T/2^32 ~ exp(-2 beta |h|); the chain's stationary law is
    Boltzmann, P(s = -sign h) = 1 / (1 + exp(-2 beta |h|))."""
    h = np.array([1, -2, 3, -1, 2, 0], dtype=np.int32)
    n = h.shape[0]
    c = oracle.Csr(n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32), h)
    R = 20000
    res = oracle.anneal(c, R, np.full(41, beta), seed=77)
    init = oracle.initial_spins(n, np.arange(R), 77)
    # no field: the spin flips every sweep, so after 41 sweeps it is -s0
    assert np.array_equal(res.s_final[:, 5], -init[:, 5])
    for i in range(n - 1):
        low = np.sum(res.s_final[:, i] == (-1 if h[i] > 0 else 1))
        p_low = 1.0 / (1.0 + np.exp(-2.0 * beta * abs(int(h[i]))))
        obs = np.array([low, R - low], dtype=np.float64)
        assert _chi2_p(obs, np.array([p_low, 1 - p_low]) * R) > 1e-3, i


def test_metropolis_with_fields_samples_boltzmann():
    g = I.random_graph(11, 20, 6)
    w = np.array([(-2, -1, 1, 2)[k % 4] for k in range(g.m)], np.int32)
    h = np.array([(2, -1, 0, 1, -3)[i % 5] for i in range(g.n)], np.int32)
    c = oracle.Csr(g.n, g.u, g.v, w, h)
    beta = 0.35
    e_min, _, hist, e_lo = c.enumerate(histogram=True)
    E = np.arange(hist.shape[0]) + e_lo
    p = hist.astype(np.float64) * np.exp(-beta * (E - e_min))
    p /= p.sum()
    R = 20000
    res = oracle.anneal(c, R, np.full(80, beta), seed=21)
    obs = np.bincount(res.e_final.astype(np.int64) - e_lo, minlength=hist.shape[0])
    assert _chi2_p(obs.astype(np.float64), p * R) > 1e-3


def test_tracked_energy_with_fields():
    g = I.independent_set_instance(I.geometric_graph(400, 6.0, 2))
    c = oracle.csr_of(g)
    oracle.anneal(c, 8, I.geometric_betas(0.1, 5.0, 100), 4, check_energy=True)


def _max_independent_set(n, u, v):
    adj = np.zeros(n, dtype=np.int64)
    for a, b in zip(u, v):
        adj[a] |= 1 << int(b)
        adj[b] |= 1 << int(a)
    best = 0
    for mask in range(1 << n):
        ok = True
        mm = mask
        while mm:
            i = (mm & -mm).bit_length() - 1
            if adj[i] & mask:
                ok = False
                break
            mm &= mm - 1
        if ok:
            best = max(best, bin(mask).count("1"))
    return best


@pytest.mark.parametrize("n,seed", [(12, 1), (14, 2), (16, 3)])
def test_independent_set_instance_ground_state_is_a_maximum_independent_set(n, seed):
    g = I.geometric_graph(n, 4.0, seed)
    inst = I.independent_set_instance(g)
    c = oracle.csr_of(inst)
    e_min, argmin = c.enumerate()
    chosen = np.nonzero(argmin > 0)[0]
    # the ground state's set is independent and as large as the brute-force maximum
    assert not any(a in chosen and b in chosen for a, b in zip(g.u.tolist(), g.v.tolist()))
    assert len(chosen) == _max_independent_set(n, g.u, g.v)
    # and its energy is 2 (-|I|) - m + n by the penalty form
    assert e_min == -2 * len(chosen) - g.m + n
    # annealing reaches it on these small instances
    res = oracle.anneal(c, 32, I.geometric_betas(0.1, 5.0, 400), 5)
    assert res.best[0] == e_min

"""Pins of the oracle's parallel tempering (Sec. II.C: replicas at different
temperatures exchanging configurations): the single-slot case is constant-beta
annealing, exchange counts follow the alternating pair schedule, equal
temperatures always exchange, and at fixed temperatures every slot samples
its own Boltzmann distribution (exact enumeration, chi-square) — which a
wrong exchange rule (sign, direction, energy bookkeeping) would break."""
import numpy as np
import pytest

import oracle
from paper_2311_09275_gb300 import inputs as I
from test_oracle_pins import _chi2_p


def test_single_slot_is_constant_beta_annealing():
    c = oracle.csr_of(I.torus(10, 8, 4))
    pt = oracle.parallel_tempering(c, [0.6], rounds=15, per_round=4, seed=9)
    an = oracle.anneal(c, 32, np.full(60, 0.6), 9)
    for x, y in [(pt.s_final, an.s_final), (pt.e_final, an.e_final), (pt.s_best, an.s_best),
                 (pt.e_best, an.e_best)]:
        assert np.array_equal(x, y)


def test_exchange_counts_follow_the_alternating_schedule():
    c = oracle.csr_of(I.torus(6, 6, 2))
    K, rounds = 5, 9
    pt = oracle.parallel_tempering(c, np.linspace(0.2, 1.5, K), rounds, 2, 3)
    for k in range(K - 1):
        assert pt.attempted[k] == 32 * sum(1 for q in range(rounds) if q % 2 == k % 2)
        assert 0 <= pt.accepted[k] <= pt.attempted[k]


def test_equal_temperatures_always_exchange():
    c = oracle.csr_of(I.random_graph(40, 70, 3))
    pt = oracle.parallel_tempering(c, [0.8, 0.8, 0.8], 12, 1, 5)
    assert np.array_equal(pt.accepted, pt.attempted)
    # and an exchange is a pure relabelling: every slot's tracked energy is its state's energy
    for r in range(pt.e_final.shape[0]):
        assert c.energy(pt.s_final[r]) == pt.e_final[r]


def test_tracked_energies_and_best_states():
    g = I.independent_set_instance(I.geometric_graph(200, 5.0, 4))
    c = oracle.csr_of(g)
    pt = oracle.parallel_tempering(c, [0.3, 0.7, 1.2, 2.0], 10, 3, 8)
    for r in range(pt.e_final.shape[0]):
        assert c.energy(pt.s_final[r]) == pt.e_final[r]
        assert c.energy(pt.s_best[r]) == pt.e_best[r]
    # the overall best over all slots bounds every final state (a state swapped in by
    # the last exchange may undercut its new slot's best, never the overall best)
    assert pt.e_best.min() <= pt.e_final.min()


def test_each_slot_samples_its_boltzmann_distribution():
    t = I.torus(4, 4, 11)
    c = oracle.csr_of(t)
    e_min, _, hist, e_lo = c.enumerate(histogram=True)
    E = np.arange(hist.shape[0]) + e_lo
    betas = np.array([0.15, 0.35, 0.6])
    samples = [[] for _ in betas]
    for seed in range(1, 301):
        pt = oracle.parallel_tempering(c, betas, rounds=12, per_round=2, seed=seed, nthreads=1)
        for k in range(len(betas)):
            samples[k].append(pt.e_final[32 * k: 32 * k + 32])
    for k, beta in enumerate(betas):
        p = hist.astype(np.float64) * np.exp(-beta * (E - e_min))
        p /= p.sum()
        obs = np.bincount(np.concatenate(samples[k]).astype(np.int64) - e_lo,
                          minlength=hist.shape[0]).astype(np.float64)
        assert _chi2_p(obs, p * obs.sum()) > 1e-3, k


# ------------------------------------------------------- Houdayer cluster moves
def _components(n, u, v, members):
    """Connected components of the subgraph induced by `members` (plain BFS)."""
    adj = [[] for _ in range(n)]
    for a, b in zip(u, v):
        adj[a].append(b)
        adj[b].append(a)
    comp = {}
    for s in sorted(members):
        if s in comp:
            continue
        stack, comp[s] = [s], s
        while stack:
            i = stack.pop()
            for j in adj[i]:
                if j in members and j not in comp:
                    comp[j] = s
                    stack.append(j)
    return comp


@pytest.mark.parametrize("make", ["torus", "fields"])
def test_houdayer_move_swaps_one_cluster_and_conserves_the_pair_energy(make):
    if make == "torus":
        prob = I.torus(8, 10, 3)
        u, v, _ = prob.edges()
    else:
        prob = I.Graph(**vars(I.random_graph(60, 90, 5)))
        prob.h = np.array([(1, -2, 0, 3)[i % 4] for i in range(60)], np.int32)
        u, v = prob.u, prob.v
    c = oracle.csr_of(prob)
    n = c.n
    beta, per_round, seed = [0.6], 7, 11
    plain = oracle.parallel_tempering(c, beta, 1, per_round, seed)            # sweeps only
    moved = oracle.parallel_tempering(c, beta, 1, per_round, seed, icm_slots=1)
    total = 0
    for m in range(16):
        a, b = 2 * m, 2 * m + 1
        sa, sb = plain.s_final[a].astype(int), plain.s_final[b].astype(int)
        ta, tb = moved.s_final[a].astype(int), moved.s_final[b].astype(int)
        diff = set(np.nonzero(sa != sb)[0].tolist())
        changed = set(np.nonzero(ta != sa)[0].tolist())
        assert changed == set(np.nonzero(tb != sb)[0].tolist())
        # the two chains exchanged their spins on the changed sites
        assert np.array_equal(np.sort(np.stack([sa, sb]), 0), np.sort(np.stack([ta, tb]), 0))
        if not diff:
            assert not changed
            continue
        # the changed sites are exactly one component of the differing sites ...
        comp = _components(n, u, v, diff)
        roots = {comp[i] for i in changed}
        assert len(roots) == 1 and {i for i in diff if comp[i] in roots} == changed
        # ... the one holding the drawn site: the (u mod D)-th differing site in vertex order
        w = oracle.philox4x32_10([0, 0, m, 3], [seed & 0xFFFFFFFF, seed >> 32])[0]
        pick = sorted(diff)[int(w) % len(diff)]
        assert pick in changed
        # the pair's total energy is unchanged, each energy is tracked exactly
        assert c.energy(ta) + c.energy(tb) == c.energy(sa) + c.energy(sb)
        assert moved.e_final[a] == c.energy(ta) and moved.e_final[b] == c.energy(tb)
        total += len(changed)
    assert moved.flipped[0] == total > 0


def test_slots_without_cluster_moves_are_unchanged():
    c = oracle.csr_of(I.torus(6, 8, 2))
    betas = [0.3, 0.5, 0.8, 1.2]
    a = oracle.parallel_tempering(c, betas, 1, 3, 4)
    b = oracle.parallel_tempering(c, betas, 1, 3, 4, icm_slots=2)
    # round 0 exchanges pair (0, 1) and (2, 3); slots 0, 1 never see a cluster move
    assert np.array_equal(a.s_final[:64], b.s_final[:64])
    assert b.flipped[0] == b.flipped[1] == 0 and b.flipped[2] + b.flipped[3] > 0


def test_tempering_with_cluster_moves_samples_boltzmann():
    """Houdayer moves keep each slot's Boltzmann distribution (symmetric choice
    of the cluster, conserved pair energy)."""
    t = I.torus(4, 4, 11)
    c = oracle.csr_of(t)
    e_min, _, hist, e_lo = c.enumerate(histogram=True)
    E = np.arange(hist.shape[0]) + e_lo
    betas = np.array([0.3, 0.6])
    samples = [[] for _ in betas]
    for seed in range(1, 301):
        pt = oracle.parallel_tempering(c, betas, rounds=10, per_round=2, seed=seed, nthreads=1,
                                       icm_slots=2)
        for k in range(len(betas)):
            samples[k].append(pt.e_final[32 * k: 32 * k + 32])
    for k, beta in enumerate(betas):
        p = hist.astype(np.float64) * np.exp(-beta * (E - e_min))
        p /= p.sum()
        obs = np.bincount(np.concatenate(samples[k]).astype(np.int64) - e_lo,
                          minlength=hist.shape[0]).astype(np.float64)
        assert _chi2_p(obs, p * obs.sum()) > 1e-3, k

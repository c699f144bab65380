"""Parallel tempering on the GPU (multi-spin torus kernel + exchange kernel)
against the oracle, replica by replica: final and best states, energies and
exchange counts."""
import numpy as np
import pytest

import oracle
from paper_2311_09275_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2311_09275_gb300 import build
    build.build()
    from paper_2311_09275_gb300 import isg as mod
    return mod


def assert_same_pt(res, orc, pairs):
    spins, e, done = res.final()
    assert np.array_equal(e, orc.e_final), "final energies differ"
    assert np.array_equal(spins, orc.s_final), "final spins differ"
    assert np.array_equal(res.best_all(), orc.s_best), "best spins differ"
    assert np.array_equal(res.best(spins=False)[3], orc.e_best), "best energies differ"
    from paper_2311_09275_gb300 import isg as mod
    acc, att = mod.isg_result_exchanges(res, pairs)
    assert np.array_equal(acc, orc.accepted) and np.array_equal(att, orc.attempted)


@pytest.mark.parametrize("L,W,betas,rounds,per_round,cluster,threads", [
    (12, 10, [0.2, 0.5, 0.9, 1.6], 7, 3, 0, 0),
    (20, 16, [0.1, 0.3, 0.45, 0.8, 2.0], 6, 2, 2, 64),
    (8, 6, [1.5, 0.4, 0.9], 9, 1, 1, 32),        # unordered ladder
    (16, 14, [0.7], 5, 4, 4, 0),                 # one slot: no exchanges
    (10, 12, [0.6, 0.6, 0.6, 0.6], 8, 2, 0, 0),  # equal temperatures
])
def test_tempering_bit_exact(isg, L, W, betas, rounds, per_round, cluster, threads):
    t = I.torus(L, W, 40 + L)
    c = oracle.csr_of(t)
    orc = oracle.parallel_tempering(c, betas, rounds, per_round, 13)
    res = isg.isg_parallel_tempering(isg.problem_of(t), betas, rounds, per_round, 13,
                                     cluster_ctas=cluster, threads=threads)
    assert_same_pt(res, orc, len(betas) - 1)
    if len(set(betas)) == 1 and len(betas) > 1:
        assert np.array_equal(orc.accepted, orc.attempted)


def test_tempering_full_size_ladder(isg):
    """80x100 torus, 8 slots (256 replicas), 4 rounds of 5 sweeps."""
    t = I.torus(80, 100, 1)
    betas = I.geometric_betas(0.2, 3.0, 8)
    orc = oracle.parallel_tempering(oracle.csr_of(t), betas, 4, 5, 21)
    res = isg.isg_parallel_tempering(isg.problem_of(t), betas, 4, 5, 21)
    assert_same_pt(res, orc, 7)


def test_tempering_rejects_bad_input(isg):
    gw = I.random_graph(50, 60, 1)
    gw = I.Graph(gw.n, gw.u, gw.v, np.full(gw.m, 2, np.int32))
    with pytest.raises(isg.IsgError):   # cluster moves need the multi-spin kernels
        isg.isg_parallel_tempering(isg.problem_of(gw), [0.5, 1.0], 2, 2, 1, icm_slots=1)
    g = isg.problem_of(I.random_graph(50, 60, 1))
    with pytest.raises(isg.IsgError):
        isg.isg_parallel_tempering(g, [0.5, 1.0], 2, 2, 1, icm_slots=3)  # more than K slots
    big = isg.problem_of(I.random_graph(20000, 20000, 2))
    with pytest.raises(isg.IsgError):
        isg.isg_parallel_tempering(big, [0.5, 1.0], 2, 2, 1, icm_slots=1)  # n > 19,029
    t = isg.problem_of(I.torus(8, 8, 1))
    with pytest.raises(isg.IsgError):
        isg.isg_parallel_tempering(t, [], 2, 2, 1)
    with pytest.raises(isg.IsgError):
        isg.isg_parallel_tempering(t, [0.5, np.inf], 2, 2, 1)
    with pytest.raises(isg.IsgError):
        isg.isg_parallel_tempering(t, [0.5, 1.0], 0, 2, 1)
    res = isg.isg_anneal(t, 8, np.full(3, 0.5), 1)
    with pytest.raises(isg.IsgError):
        isg.isg_result_exchanges(res, 3)                    # no exchange pairs there


@pytest.mark.parametrize("L,W,betas,rounds,per_round,icm", [
    (12, 10, [0.3, 0.8, 1.5, 2.5], 6, 3, 2),
    (20, 16, [0.5, 1.0, 2.0], 5, 2, 3),
    (8, 6, [1.2], 9, 1, 1),
    (40, 30, [0.4, 0.9, 1.6, 2.4, 3.0], 4, 4, 5),
    # rings of 129..256 sites (8 sites per lane) and longer than 1,024 sites (a lane's
    # segment spans three words of ring marks)
    (6, 200, [0.4, 1.0, 2.0], 3, 2, 2),
    (200, 6, [0.4, 1.0, 2.0], 3, 2, 2),
    (4, 1100, [0.4, 1.0, 2.0], 3, 2, 2),
    (1100, 4, [0.4, 1.0, 2.0], 3, 2, 2),
])
def test_tempering_with_cluster_moves_bit_exact(isg, L, W, betas, rounds, per_round, icm):
    t = I.torus(L, W, 60 + L)
    c = oracle.csr_of(t)
    orc = oracle.parallel_tempering(c, betas, rounds, per_round, 29, icm_slots=icm)
    res = isg.isg_parallel_tempering(isg.problem_of(t), betas, rounds, per_round, 29,
                                     icm_slots=icm)
    assert_same_pt(res, orc, len(betas) - 1)
    assert np.array_equal(isg.isg_result_cluster_flips(res, len(betas)), orc.flipped)
    assert orc.flipped[len(betas) - icm:].sum() > 0


def test_cluster_moves_full_size(isg):
    t = I.torus(80, 100, 1)
    betas = I.geometric_betas(0.5, 3.0, 6)
    orc = oracle.parallel_tempering(oracle.csr_of(t), betas, 3, 4, 8, icm_slots=3)
    res = isg.isg_parallel_tempering(isg.problem_of(t), betas, 3, 4, 8, icm_slots=3)
    assert_same_pt(res, orc, 5)
    assert np.array_equal(isg.isg_result_cluster_flips(res, 6), orc.flipped)


def _pm1(n, m, seed):
    g = I.random_graph(n, m, seed)
    w = np.where(I.draws(seed, 7, np.arange(g.m)) >> np.uint64(63), 1, -1).astype(np.int32)
    return I.Graph(g.n, g.u, g.v, w)


@pytest.mark.parametrize("make,betas,rounds,per_round,cluster,threads", [
    (lambda: I.random_graph(500, 700, 3), [0.2, 0.6, 1.2, 2.0], 6, 3, 0, 0),
    (lambda: _pm1(400, 1000, 4), [0.3, 0.5, 0.9], 5, 2, 3, 128),
    (lambda: I.random_graph(10000, 9999, 1), I.geometric_betas(0.2, 3.0, 6), 3, 4, 0, 0),
    # local fields (independent set): exchanges see E = sum s s + sum h s
    (lambda: I.independent_set_instance(I.geometric_graph(400, 6.0, 5)), [0.3, 0.8, 1.5, 2.5],
     5, 3, 2, 128),
])
def test_tempering_on_graphs_bit_exact(isg, make, betas, rounds, per_round, cluster, threads):
    g = make()
    orc = oracle.parallel_tempering(oracle.csr_of(g), betas, rounds, per_round, 31)
    res = isg.isg_parallel_tempering(isg.problem_of(g), betas, rounds, per_round, 31,
                                     cluster_ctas=cluster, threads=threads)
    assert res.stats()["kernel"] == 4
    assert_same_pt(res, orc, len(betas) - 1)


def test_tempering_on_smallest_last_graph(isg):
    """Tempering on a graph re-coloured smallest-last follows those classes."""
    g = I.random_graph(800, 799, 12)
    c = oracle.csr_of(g)
    col, _ = c.smallest_last_colouring()
    betas = [0.3, 0.8, 1.6]
    orc = oracle.parallel_tempering(c, betas, 4, 3, 17, colour=col)
    res = isg.isg_parallel_tempering(isg.problem_of(g, colouring=isg.COLOURING_SMALLEST_LAST),
                                     betas, 4, 3, 17)
    assert_same_pt(res, orc, len(betas) - 1)


@pytest.mark.parametrize("make,betas,rounds,per_round,icm,cluster", [
    (lambda: I.random_graph(300, 450, 31), [0.3, 0.8, 1.4, 2.2], 12, 3, 2, 0),
    (lambda: I.random_graph(700, 1400, 32), [0.4, 1.0, 1.8], 10, 2, 3, 3),
    (lambda: I.Graph(*_signed_edges(I.random_graph(400, 800, 33))), [0.5, 1.2, 2.0, 3.0, 4.0], 8,
     2, 2, 0),
    (lambda: I.independent_set_instance(I.geometric_graph(300, 6.0, 34)), [0.6, 1.5, 3.0], 10,
     2, 3, 0),
])
def test_graph_houdayer_bit_exact(isg, make, betas, rounds, per_round, icm, cluster):
    """Houdayer cluster moves on graph slot words (unweighted, +-1 weights, local
    fields with weights +1): states, energies, exchange counts and cluster
    sizes equal the oracle's, chain by chain."""
    g = make()
    c = oracle.csr_of(g)
    orc = oracle.parallel_tempering(c, betas, rounds, per_round, 17, icm_slots=icm)
    res = isg.isg_parallel_tempering(isg.problem_of(g), betas, rounds, per_round, 17,
                                     icm_slots=icm, cluster_ctas=cluster)
    assert_same_pt(res, orc, len(betas) - 1)
    K = len(betas)
    assert np.array_equal(isg.isg_result_cluster_flips(res, K), orc.flipped)
    assert orc.flipped[K - icm:].sum() > 0                 # moves happened


def _signed_edges(g):
    """g's edges with seeded +-1 weights."""
    w = np.where(I.draws(g.n, 5, np.arange(g.m)) >> np.uint64(63), 1, -1).astype(np.int32)
    return g.n, g.u, g.v, w


@pytest.mark.parametrize("make,betas,rounds,per_round,cluster,qpc", [
    (lambda: _weighted(I.random_graph(300, 600, 41), (-2, 1, 3)), [0.2, 0.5, 0.9, 1.4], 8, 3,
     0, 0),
    (lambda: _weighted(I.random_graph(500, 900, 42), (1, -1, 2, -3, 5)), [0.3, 0.7, 1.2], 6, 2,
     3, 2),
    # local fields on +-1 weights (the multi-spin graph kernel takes fields only with +1)
    (lambda: _fields(I.Graph(*_signed_edges(I.random_graph(350, 700, 43))), 44),
     [0.4, 0.8, 1.6, 2.4, 3.2], 7, 2, 2, 1),
])
def test_tempering_on_int8_kernel_bit_exact(isg, make, betas, rounds, per_round, cluster, qpc):
    """Parallel tempering of instances the multi-spin kernels do not take
    (general integer weights; local fields with +-1 weights), on the int8
    colour-class kernel with 8 quads per slot: equal to the oracle chain by
    chain, including the exchange counts."""
    g = make()
    c = oracle.csr_of(g)
    orc = oracle.parallel_tempering(c, betas, rounds, per_round, 23)
    res = isg.isg_parallel_tempering(isg.problem_of(g), betas, rounds, per_round, 23,
                                     cluster_ctas=cluster, quads_per_cta=qpc)
    assert res.stats()["kernel"] == 2
    assert_same_pt(res, orc, len(betas) - 1)
    assert orc.accepted.sum() > 0


def _weighted(g, ws):
    return I.Graph(g.n, g.u, g.v, np.array([ws[e % len(ws)] for e in range(g.m)], np.int32))


def _fields(g, seed):
    h = (I.draws(seed, 6, np.arange(g.n)) % np.uint64(7)).astype(np.int32) - 3
    return I.Graph(g.n, g.u, g.v, g.w, h)

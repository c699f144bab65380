"""Local fields on the GPU against the oracle, element by element:
E = sum w s s + sum h s.  The int8 colour-class kernel (any weights) and the
multi-spin graph kernel (all weights +1, degree + |h| <= 63): independent-set
instances, general weights with fields, +-1 weights with fields, targets,
isg_energy, the served path, parallel tempering, and the refusals."""
import functools

import numpy as np
import pytest

import oracle
from paper_2311_09275_gb300 import inputs as I
from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2311_09275_gb300 import build
    build.build()
    from paper_2311_09275_gb300 import isg as mod
    return mod


def mis(n=600, deg=6.0, seed=3):
    return I.independent_set_instance(I.geometric_graph(n, deg, seed))


def general_with_fields(seed=4):
    g = I.random_graph(350, 900, seed)
    w = np.array([(-2, -1, 1, 2, 3)[k % 5] for k in range(g.m)], np.int32)
    h = np.array([(-4, 0, 1, 3, -1, 2)[i % 6] for i in range(g.n)], np.int32)
    return I.Graph(g.n, g.u, g.v, w, h)


def pm1_with_fields(seed=5):
    g = I.random_graph(300, 700, seed)
    w = np.where(I.draws(seed, 7, np.arange(g.m)) >> np.uint64(63), 1, -1).astype(np.int32)
    h = np.array([(1, -1, 0, 2)[i % 4] for i in range(g.n)], np.int32)
    return I.Graph(g.n, g.u, g.v, w, h)


def unit_with_fields(seed=6):
    """All weights +1, fields of both signs and zero (|h| <= 3)."""
    g = I.random_graph(400, 1000, seed)
    h = np.array([(-3, 0, 2, -1, 1, 3, 0, -2)[i % 8] for i in range(g.n)], np.int32)
    return I.Graph(g.n, g.u, g.v, np.ones(g.m, np.int32), h)


CASES = {"mis": mis, "general": general_with_fields, "pm1": pm1_with_fields}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("R,cluster,qpc", [(1, 1, 1), (13, 2, 1), (37, 4, 2), (64, 0, 0)])
def test_fields_csr_bit_exact(isg, name, R, cluster, qpc):
    g = CASES[name]()
    betas = I.geometric_betas(0.1, 5.0, 120)
    orc = oracle.anneal(oracle.csr_of(g), R, betas, 17, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 17, kernel=2, cluster_ctas=cluster,
                         quads_per_cta=qpc)
    assert_same(res, orc)


@pytest.mark.parametrize("name", ["mis", "unit"])
@pytest.mark.parametrize("R,cluster,threads", [(1, 1, 64), (33, 3, 128), (70, 8, 96), (64, 0, 0)])
def test_fields_graph_msc_bit_exact(isg, name, R, cluster, threads):
    """Multi-spin graph kernel with local fields (|h| extra bonds per vertex)."""
    g = mis() if name == "mis" else unit_with_fields()
    betas = I.geometric_betas(0.1, 5.0, 120)
    orc = oracle.anneal(oracle.csr_of(g), R, betas, 19, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 19, kernel=4, cluster_ctas=cluster,
                         threads=threads)
    assert_same(res, orc)
    assert res.stats()["kernel"] == 4 and res.stats()["staged"] == 1


def star_forest_with_fields():
    """20 stars of 8 leaves among 220 isolated vertices, all weights +1, fields
    |h| <= 3.  Leaves (ids 0-159) and isolated vertices (180-399) form the first
    greedy colour class, the hubs (160-179) the second: almost every vertex is
    updated in the first class."""
    hub = np.repeat(np.arange(160, 180, dtype=np.int32), 8)
    leaf = np.arange(160, dtype=np.int32)
    h = np.array([(2, -1, 0, 3, -3, 1, -2)[i % 7] for i in range(400)], np.int32)
    return I.Graph(400, leaf, hub, np.ones(160, np.int32), h)


def edgeless_with_fields():
    """No edges, fields |h| <= 4: one colour class."""
    h = np.array([(4, -1, 2, 0, -3, 1)[i % 6] for i in range(300)], np.int32)
    z = np.zeros(0, np.int32)
    return I.Graph(300, z, z, z, h)


@pytest.mark.parametrize("make", [unit_with_fields, star_forest_with_fields])
@pytest.mark.parametrize("R,cluster,threads,mask_chunk", [(40, 1, 128, 9), (70, 5, 96, 9),
                                                          (64, 12, 256, 1000)])
def test_fields_graph_msc_precomputed_masks_bit_exact(isg, make, R, cluster, threads,
                                                      mask_chunk):
    """Local fields with the graph kernel's acceptance masks precomputed by a
    second kernel (levels (d + |h| + 1) / 2 per vertex), in chunks of mask_chunk
    sweeps, one CTA per word or a cluster with data-flow class phases."""
    g = make()
    betas = I.geometric_betas(0.1, 5.0, 45)
    orc = oracle.anneal(oracle.csr_of(g), R, betas, 31, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 31, kernel=4, cluster_ctas=cluster,
                         threads=threads, mask_chunk=mask_chunk)
    st = res.stats()
    assert st["kernel"] == 4 and st["staged"] == 1 and st["mask_chunks"] > 0
    assert_same(res, orc)


@pytest.mark.parametrize("make", [star_forest_with_fields, edgeless_with_fields])
@pytest.mark.parametrize("R,cluster,threads", [(40, 1, 64), (40, 4, 128), (70, 8, 96)])
def test_graph_msc_mask_windows_bit_exact(isg, make, R, cluster, threads):
    """The staged graph kernel builds each vertex's acceptance masks for sweep
    t + 1 during sweep t, shared out over the class barrier windows: a first
    class holding nearly every vertex, and a single class, where the sweep's
    last window and the next sweep's first class meet."""
    g = make()
    betas = I.geometric_betas(0.1, 5.0, 90)
    orc = oracle.anneal(oracle.csr_of(g), R, betas, 29, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 29, kernel=4, cluster_ctas=cluster,
                         threads=threads)
    assert res.stats()["kernel"] == 4 and res.stats()["staged"] == 1
    assert_same(res, orc)


@pytest.mark.parametrize("R,cluster,threads", [(40, 1, 256), (70, 4, 512)])
def test_fields_graph_msc_unstaged_bit_exact(isg, R, cluster, threads):
    """Fields read from global memory: 12,000 vertices of mean degree 25 with
    |h| <= 2 (adjacency too large to stage)."""
    g = I.random_graph(12000, 150000, 13)
    h = np.array([(1, -2, 0, 2, -1)[i % 5] for i in range(g.n)], np.int32)
    g = I.Graph(g.n, g.u, g.v, np.ones(g.m, np.int32), h)
    betas = I.geometric_betas(0.1, 5.0, 12)
    orc = oracle.anneal(oracle.csr_of(g), R, betas, 23, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 23, kernel=4, cluster_ctas=cluster,
                         threads=threads)
    assert res.stats()["staged"] == 0
    assert_same(res, orc)


def test_fields_auto_and_plain_kernels(isg):
    g = mis(300, 5.0, 8)
    betas = I.geometric_betas(0.1, 5.0, 60)
    orc = oracle.anneal(oracle.csr_of(g), 24, betas, 2)
    p = isg.problem_of(g)
    auto = isg.isg_anneal(p, 24, betas, 2)
    assert auto.stats()["kernel"] == 4          # unit weights, fields -> multi-spin graph kernel
    assert_same(auto, orc)
    assert_same(isg.isg_anneal(p, 24, betas, 2, kernel=2), orc)
    assert_same(isg.isg_anneal(p, 24, betas, 2, kernel=3), orc)


def test_fields_outside_graph_msc(isg):
    """+-1 weights with fields, or degree + |h| > 63: the multi-spin kernel
    refuses and the automatic choice is the int8 kernel."""
    betas = I.geometric_betas(0.1, 5.0, 40)
    g = I.random_graph(200, 500, 3)
    big = I.Graph(g.n, g.u, g.v, np.ones(g.m, np.int32),
                  np.where(np.arange(g.n) == 7, 60, 1).astype(np.int32))
    for inst in (pm1_with_fields(), big):
        p = isg.problem_of(inst)
        with pytest.raises(isg.IsgError):
            isg.isg_anneal(p, 8, betas, 2, kernel=4)
        res = isg.isg_anneal(p, 8, betas, 2)
        assert res.stats()["kernel"] == 2
        assert_same(res, oracle.anneal(oracle.csr_of(inst), 8, betas, 2))


@pytest.mark.parametrize("R", [20, 70])
def test_fields_graph_msc_target_stop(isg, R):
    g = mis(500, 6.0, 21)
    betas = I.geometric_betas(0.1, 5.0, 300)
    c = oracle.csr_of(g)
    target = int(oracle.anneal(c, R, betas, 4).e_best.min()) + 2
    orc = oracle.anneal(c, R, betas, 4, target=target)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 4, target=target, kernel=4, cluster_ctas=2)
    assert_same(res, orc)


@pytest.mark.parametrize("R", [8, 40])
def test_fields_target_stop(isg, R):
    g = general_with_fields(9)
    betas = I.geometric_betas(0.1, 5.0, 200)
    c = oracle.csr_of(g)
    full = oracle.anneal(c, R, betas, 6)
    target = full.best[0] + 4
    orc = oracle.anneal(c, R, betas, 6, target=target)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 6, target=target, kernel=2, cluster_ctas=2)
    assert_same(res, orc)
    assert orc.hit_sweep >= 0


def test_fields_energy_matches_oracle(isg):
    g = general_with_fields(10)
    c = oracle.csr_of(g)
    rng = np.random.default_rng(1)
    s = np.where(rng.random((9, g.n)) < 0.5, 1, -1).astype(np.int8)
    e = isg.isg_energy(isg.problem_of(g), s)
    assert [int(x) for x in e] == [c.energy(row) for row in s]


def test_fields_independent_set_valid_and_near_maximum(isg):
    """Annealed independent-set instances give valid sets (no edge inside)
    whose energy equals the oracle's for the same seed."""
    gg = I.geometric_graph(2000, 6.0, 11)
    g = I.independent_set_instance(gg)
    betas = I.geometric_betas(0.1, 5.0, 400)
    res = isg.isg_anneal(isg.problem_of(g), 64, betas, 3)
    be, br, bs, per, hit = res.best()
    chosen = bs > 0
    assert not np.any(chosen[gg.u] & chosen[gg.v])
    orc = oracle.anneal(oracle.csr_of(g), [br], betas, 3)
    assert int(orc.e_best[0]) == be and np.array_equal(orc.s_best[0], bs)
    # the set size follows from the energy: E = -2|I| - m + n for a valid set
    assert be == -2 * int(chosen.sum()) - gg.m + gg.n


@pytest.mark.parametrize("make", [lambda: general_with_fields(12), lambda: mis(400, 6.0, 12)])
def test_fields_served_equals_solo(isg, make):
    """Served int8 quads of field instances equal one-instance solves."""
    g = make()
    p = isg.problem_of(g)
    betas = I.geometric_betas(0.1, 5.0, 150)
    srv = isg.Server(1 << 30, 4, 40)
    rid = srv.submit(p, 20, betas, 5)
    got = srv.poll(30.0)
    srv.close()
    assert got[0] == rid
    solo = isg.isg_anneal(p, 20, betas, 5)
    for x, y in zip(got[1].final(), solo.final()):
        assert np.array_equal(x, y)
    assert np.array_equal(got[1].best_all(), solo.best_all())


@functools.lru_cache(maxsize=1)
def independent_set_10000_oracle(reps):
    sv = I.independent_set_10000()
    return oracle.anneal(oracle.csr_of(sv.problem), list(reps), sv.betas, sv.seed)


@pytest.mark.slow
@pytest.mark.parametrize("shape", [{}, {"kernel": 4, "cluster_ctas": 12, "threads": 512},
                                   {"kernel": 2, "cluster_ctas": 4, "threads": 512,
                                    "quads_per_cta": 2}])
def test_independent_set_10000_full_size_sampled(isg, shape):
    """The benchmark's independent-set workload (10,000 vertices, 256 replicas,
    10,000 sweeps) on both kernel families: sampled replicas equal the oracle,
    and every replica's energy equals isg_energy of its state."""
    sv = I.independent_set_10000()
    p = isg.problem_of(sv.problem)
    res = isg.isg_anneal(p, sv.replicas, sv.betas, sv.seed, **shape)
    reps = (0, 5, 31, 32, 200, 255)
    assert_same(res, independent_set_10000_oracle(reps), reps=list(reps))
    spins, e, _ = res.final()
    assert np.array_equal(isg.isg_energy(p, spins), e)

"""GPU path vs the CPU oracle, element by element, on identical seeded inputs.

Spins, energies, best energies, best states, stop sweep and sweep counts are
integers: the bar is bit-exact equality.  Small cases cover every kernel
family and launch shape (cluster splits, thread counts, ragged replica
counts); the full-size cases run exactly the launch configuration the
benchmark times and compare sampled replicas with the oracle plus
properties that hold for every replica.
"""
import functools

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


def assert_same(res, orc, reps=None, check_done=True, first_replica=0):
    """res (replicas first_replica + 0..R-1, local indices) equals the oracle's
    result orc (global replica ids)."""
    spins, e, done = res.final()
    best = res.best_all()
    be, br, bs, per, hit = res.best()
    rows = list(range(res.replicas)) if reps is None else list(reps)
    assert np.array_equal(e[rows], orc.e_final), "final energies differ"
    assert np.array_equal(per[rows], orc.e_best), "best energies differ"
    assert np.array_equal(spins[rows], orc.s_final), "final spins differ"
    assert np.array_equal(best[rows], orc.s_best), "best spins differ"
    if check_done:
        assert done == orc.sweeps_done
        assert hit == orc.hit_sweep
    if reps is None:
        ob, orr = orc.best
        assert (be, br + first_replica) == (ob, orr)
        assert np.array_equal(bs, orc.s_best[orr - first_replica])


# ------------------------------------------------------------------ torus
@pytest.mark.parametrize("kernel", [0, 2, 3])
def test_torus_20x20_all_kernels_bit_exact(isg, kernel):
    """20x20 torus, 64 replicas, linear beta 0.1 -> 3.0 over 1,000 sweeps."""
    sv = I.torus_20x20()
    p = isg.problem_of(sv.problem)
    c = oracle.csr_of(sv.problem)
    orc = oracle.anneal(c, sv.replicas, sv.betas, sv.seed, check_energy=True)
    res = isg.isg_anneal(p, sv.replicas, sv.betas, sv.seed, kernel=kernel)
    assert_same(res, orc)


@pytest.mark.parametrize("L,W,R,cluster,threads", [
    (4, 4, 1, 1, 32), (8, 6, 5, 2, 32), (8, 6, 33, 4, 64), (8, 10, 70, 8, 32),
    (12, 10, 64, 4, 128), (6, 20, 37, 2, 64), (16, 14, 96, 0, 0), (10, 4, 31, 1, 64)])
def test_torus_launch_shapes_bit_exact(isg, L, W, R, cluster, threads):
    t = I.torus(L, W, 100 + L * W)
    betas = I.geometric_betas(0.2, 4.0, 80)
    p = isg.problem_of(t)
    orc = oracle.anneal(oracle.csr_of(t), R, betas, 77, check_energy=True)
    res = isg.isg_anneal(p, R, betas, 77, kernel=1, cluster_ctas=cluster, threads=threads)
    assert_same(res, orc)
    st = res.stats()
    if cluster:
        assert st["cluster_ctas"] == cluster


@pytest.mark.parametrize("cluster,threads", [(3, 96), (9, 128), (12, 64), (16, 256)])
def test_torus_nonportable_clusters_bit_exact(isg, cluster, threads):
    """Cluster sizes that are not powers of two and above 8 (uneven bands)."""
    t = I.torus(34, 22, 12)
    betas = I.geometric_betas(0.1, 5.0, 60)
    orc = oracle.anneal(oracle.csr_of(t), 70, betas, 19)
    res = isg.isg_anneal(isg.problem_of(t), 70, betas, 19, kernel=1, cluster_ctas=cluster,
                         threads=threads)
    assert_same(res, orc)
    assert res.stats()["cluster_ctas"] == cluster


@pytest.mark.parametrize("L,W,R,cluster,threads", [
    (40, 50, 64, 2, 1024), (34, 22, 70, 3, 640), (80, 100, 40, 4, 1024), (20, 20, 33, 1, 768)])
def test_torus_wide_ctas_bit_exact(isg, L, W, R, cluster, threads):
    """The 64-register build for CTAs of more than 512 threads."""
    t = I.torus(L, W, 7 + L)
    betas = I.geometric_betas(0.1, 5.0, 50)
    orc = oracle.anneal(oracle.csr_of(t), R, betas, 23, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(t), R, betas, 23, kernel=1, cluster_ctas=cluster,
                         threads=threads)
    assert_same(res, orc)
    st = res.stats()
    assert st["threads"] == threads and st["cluster_ctas"] == cluster


@pytest.mark.parametrize("kind", ["torus", "graph"])
def test_autotuned_shape_bit_exact(isg, kind):
    prob = I.torus(40, 30, 5) if kind == "torus" else I.random_graph(3000, 3500, 5)
    p = isg.problem_of(prob)
    R = 96
    betas = I.geometric_betas(0.1, 5.0, 50)
    best = isg.isg_autotune(p, R, 16)
    assert 1 <= best["cluster_ctas"] <= 16 and best["threads"] % 32 == 0
    res = isg.isg_anneal(p, R, betas, 4)
    st = res.stats()
    assert (st["cluster_ctas"], st["threads"]) == (best["cluster_ctas"], best["threads"])
    orc = oracle.anneal(oracle.csr_of(prob), [0, 1, 33, 95], betas, 4)
    assert_same(res, orc, reps=[0, 1, 33, 95])


def test_torus_beta_zero_and_huge(isg):
    t = I.torus(8, 8, 3)
    c = oracle.csr_of(t)
    p = isg.problem_of(t)
    for betas in (np.zeros(3), np.full(5, 1e3), np.array([0.0, 50.0, 0.0, 0.5])):
        orc = oracle.anneal(c, 40, betas, 5)
        assert_same(isg.isg_anneal(p, 40, betas, 5), orc)


@pytest.mark.parametrize("L,W,R,cluster,threads", [
    (24, 30, 96, 2, 64),      # 6 CTAs: nearly every SM idle, every sweep after chunk 0 read
    (40, 40, 1024, 2, 160),   # 64 CTAs: every second sweep read
    (16, 20, 64, 1, 64),      # one CTA per word
])
@pytest.mark.parametrize("mask_chunk", [-1, 0, 1, 7])
def test_torus_precomputed_masks_bit_exact(isg, L, W, R, cluster, threads, mask_chunk):
    """The pipelined torus kernel reading the acceptance masks of some sweeps
    from tables that a second kernel builds on the SMs its clusters leave idle
    (chunks of mask_chunk sweeps; 0 chosen automatically, -1 none): equal to
    the oracle bit for bit."""
    t = I.torus(L, W, 13)
    betas = I.geometric_betas(0.1, 5.0, 45)
    orc = oracle.anneal(oracle.csr_of(t), R, betas, 43)
    res = isg.isg_anneal(isg.problem_of(t), R, betas, 43, kernel=1, cluster_ctas=cluster,
                         threads=threads, mask_chunk=mask_chunk)
    assert (res.stats()["mask_chunks"] > 0) == (mask_chunk != -1)
    assert_same(res, orc)


# ------------------------------------------------------------------ graphs
GRAPHS = {
    "random_sparse": lambda: I.random_graph(500, 700, 4),
    "random_dense": lambda: I.random_graph(300, 2400, 5),
    "isolated": lambda: I.random_graph(60, 12, 6),
}


def weighted_graph():
    g = I.random_graph(300, 900, 7)
    w = np.array([(-2, -1, 1, 2, 3)[k % 5] for k in range(g.m)], np.int32)
    return I.Graph(g.n, g.u, g.v, w)


@pytest.mark.parametrize("name", list(GRAPHS) + ["weighted"])
@pytest.mark.parametrize("R,cluster", [(1, 1), (12, 2), (37, 4), (8, 0)])
def test_graph_csr_bit_exact(isg, name, R, cluster):
    g = weighted_graph() if name == "weighted" else GRAPHS[name]()
    betas = I.geometric_betas(0.1, 5.0, 120)
    orc = oracle.anneal(oracle.csr_of(g), R, betas, 31, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 31, kernel=2, cluster_ctas=cluster)
    assert_same(res, orc)


def pm1_graph():
    g = I.random_graph(400, 1100, 8)
    w = np.where(I.draws(8, 7, np.arange(g.m)) >> np.uint64(63), 1, -1).astype(np.int32)
    return I.Graph(g.n, g.u, g.v, w)


@pytest.mark.parametrize("name", ["random_sparse", "random_dense", "isolated", "pm1"])
@pytest.mark.parametrize("R,cluster,threads", [(1, 1, 64), (33, 3, 128), (70, 8, 96), (32, 16, 64),
                                               (64, 0, 0)])
def test_graph_msc_bit_exact(isg, name, R, cluster, threads):
    """Multi-spin-coded graph kernel (weights +-1, degree <= 63)."""
    g = pm1_graph() if name == "pm1" else GRAPHS[name]()
    betas = I.geometric_betas(0.1, 5.0, 100)
    orc = oracle.anneal(oracle.csr_of(g), R, betas, 13, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 13, kernel=4, cluster_ctas=cluster,
                         threads=threads)
    assert_same(res, orc)
    st = res.stats()
    assert st["kernel"] == 4 and st["staged"] == 1  # adjacency and mask table in shared memory


def hub_graph():
    """A 400-vertex random graph plus a hub (vertex 0) of degree 63, the most the
    multi-spin graph kernel takes: 32 threshold levels on one vertex word."""
    g = I.random_graph(400, 600, 21)
    pairs = {(int(a), int(b)) for a, b in zip(g.u, g.v)}
    pairs = {(a, b) for a, b in pairs if a != 0 and b != 0}
    nbrs = range(7, 7 + 6 * 63, 6)
    pairs |= {(0, j) for j in nbrs}
    u, v = zip(*sorted(pairs))
    return I.Graph(400, np.array(u, np.int32), np.array(v, np.int32), np.ones(len(u), np.int32))


def dense_pm1_graph():
    """300 vertices, 3,000 edges of weight +-1 (mean degree 20)."""
    g = I.random_graph(300, 3000, 22)
    w = np.where(I.draws(22, 7, np.arange(g.m)) >> np.uint64(63), 1, -1).astype(np.int32)
    return I.Graph(g.n, g.u, g.v, w)


def many_colours_graph():
    """200 vertices, 2,500 edges: about ten greedy colour classes."""
    return I.random_graph(200, 2500, 23)


@pytest.mark.parametrize("make", [hub_graph, dense_pm1_graph, many_colours_graph])
@pytest.mark.parametrize("R,cluster,threads", [(45, 2, 32), (32, 5, 96), (70, 3, 224),
                                               (33, 12, 512)])
def test_graph_msc_mask_table_shapes_bit_exact(isg, make, R, cluster, threads):
    """The staged graph kernel's table of acceptance masks (one word per
    threshold level of every owned vertex, built a sweep ahead): high degrees,
    many levels and classes, small and large CTAs, ragged replica counts."""
    g = make()
    betas = I.geometric_betas(0.1, 5.0, 60)
    orc = oracle.anneal(oracle.csr_of(g), R, betas, 37, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 37, kernel=4, cluster_ctas=cluster,
                         threads=threads)
    st = res.stats()
    assert st["kernel"] == 4 and st["staged"] == 1
    assert_same(res, orc)


@pytest.mark.parametrize("make", [GRAPHS["random_sparse"], pm1_graph, GRAPHS["isolated"],
                                  hub_graph])
@pytest.mark.parametrize("mask_chunk,cluster,threads,chunks", [
    (-1, 4, 128, 0),     # built inside the sweep kernel
    (0, 2, 256, 0),      # automatic: 45 sweeps are too few to precompute
    (1, 3, 96, 45),      # one sweep per chunk
    (7, 5, 64, 7),       # six chunks of 7 and one of 3
    (1000, 12, 512, 1),  # the whole schedule in one chunk
    (7, 1, 256, 7),      # one CTA per word: CTA barriers, no data flow
])
def test_graph_msc_precomputed_masks_bit_exact(isg, make, mask_chunk, cluster, threads, chunks):
    """The staged graph kernel with the acceptance masks precomputed by a second
    kernel on its own stream, chunk by chunk, or built in the sweep kernel:
    equal to the oracle bit for bit."""
    g = make()
    betas = I.geometric_betas(0.1, 5.0, 45)
    orc = oracle.anneal(oracle.csr_of(g), 70, betas, 41, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), 70, betas, 41, kernel=4, cluster_ctas=cluster,
                         threads=threads, mask_chunk=mask_chunk)
    st = res.stats()
    assert st["staged"] == 1 and st["mask_chunks"] == chunks
    assert_same(res, orc)


def test_graph_msc_precomputed_masks_continue_resume_target(isg):
    """Precomputed masks across isg_anneal_continue (the solve's chunk length
    carries over) and isg_anneal_resume, equal to one solve with the masks built
    in the kernel; a solve with a target builds them in the kernel."""
    g = pm1_graph()
    p = isg.problem_of(g)
    betas = I.geometric_betas(0.1, 4.0, 80)
    whole = isg.isg_anneal(p, 64, betas, 29, kernel=4, cluster_ctas=3, mask_chunk=-1)
    part = isg.isg_anneal(p, 64, betas[:30], 29, kernel=4, cluster_ctas=3, mask_chunk=9)
    assert part.stats()["mask_chunks"] == 4
    isg.isg_anneal_continue(p, part, betas[30:])
    assert part.stats()["mask_chunks"] == 6
    for x, y in zip(part.final(), whole.final()):
        assert np.array_equal(x, y)
    assert np.array_equal(part.best_all(), whole.best_all())
    first = isg.isg_anneal(p, 64, betas[:50], 29, kernel=4, cluster_ctas=3, mask_chunk=-1)
    res = isg.isg_anneal_resume(p, 64, betas, 29, 50, first.final()[0], first.best_all(),
                                kernel=4, cluster_ctas=2, mask_chunk=11)
    assert res.stats()["mask_chunks"] == 3
    for x, y in zip(res.final(), whole.final()):
        assert np.array_equal(x, y)
    assert np.array_equal(res.best_all(), whole.best_all())
    assert_same(res, oracle.anneal(oracle.csr_of(g), 64, betas, 29))
    target = int(whole.best(spins=False)[0]) + 8
    hit = isg.isg_anneal(p, 64, betas, 29, target=target, kernel=4, cluster_ctas=3,
                         mask_chunk=9)
    assert hit.stats()["mask_chunks"] == 0
    assert_same(hit, oracle.anneal(oracle.csr_of(g), 64, betas, 29, target=target))
    with pytest.raises(isg.IsgError) as e:
        isg.isg_anneal(p, 64, betas, 29, kernel=4, mask_chunk=-2)
    assert e.value.status == isg.ISG_EINVAL


@pytest.mark.parametrize("R,cluster,threads", [(40, 1, 256), (70, 4, 512)])
def test_graph_msc_unstaged_bit_exact(isg, R, cluster, threads):
    """Adjacency too large for shared memory (12,000 vertices, mean degree 25):
    every update is written into every CTA's copy of the word."""
    g = I.random_graph(12000, 150000, 9)
    betas = I.geometric_betas(0.1, 5.0, 12)
    orc = oracle.anneal(oracle.csr_of(g), R, betas, 29, check_energy=True)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 29, kernel=4, cluster_ctas=cluster,
                         threads=threads)
    assert res.stats()["staged"] == 0
    assert_same(res, orc)


def test_graph_auto_kernel_choice(isg):
    unit = isg.isg_anneal(isg.problem_of(GRAPHS["random_sparse"]()), 8, np.full(3, 1.0), 1)
    assert unit.stats()["kernel"] == 4           # +-1 weights -> multi-spin graph kernel
    general = isg.isg_anneal(isg.problem_of(weighted_graph()), 8, np.full(3, 1.0), 1)
    assert general.stats()["kernel"] == 2        # general weights -> int8 colour classes


def test_torus_via_graph_msc_equals_torus_msc(isg):
    t = I.torus(12, 10, 21)
    betas = I.geometric_betas(0.1, 5.0, 150)
    a = isg.isg_anneal(isg.problem_of(t), 64, betas, 5)
    b = isg.isg_anneal(isg.problem_of(t), 64, betas, 5, kernel=4, cluster_ctas=2)
    for x, y in zip(a.final(), b.final()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.best_all(), b.best_all())


@pytest.mark.parametrize("R", [20, 70])
def test_graph_msc_target_stop(isg, R):
    g = I.random_graph(600, 900, 3)
    betas = I.geometric_betas(0.1, 5.0, 300)
    c = oracle.csr_of(g)
    target = int(oracle.anneal(c, R, betas, 2).e_best.min()) + 2
    orc = oracle.anneal(c, R, betas, 2, target=target)
    res = isg.isg_anneal(isg.problem_of(g), R, betas, 2, target=target, kernel=4, cluster_ctas=2)
    assert_same(res, orc)


def test_graph_plain_kernel_bit_exact(isg):
    g = weighted_graph()
    betas = I.linear_betas(0.1, 3.0, 60)
    orc = oracle.anneal(oracle.csr_of(g), 10, betas, 8)
    assert_same(isg.isg_anneal(isg.problem_of(g), 10, betas, 8, kernel=3), orc)


def test_single_vertex_and_edgeless(isg):
    g = I.Graph(1, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    orc = oracle.anneal(oracle.csr_of(g), 6, np.full(4, 1.0), 2)
    assert_same(isg.isg_anneal(isg.problem_of(g), 6, np.full(4, 1.0), 2), orc)


def test_torus_via_csr_equals_msc(isg):
    """The same torus given as an edge list (CSR kernel, greedy colouring)
    matches the multi-spin-coded torus kernel bit for bit."""
    t = I.torus(10, 12, 9)
    betas = I.geometric_betas(0.1, 5.0, 200)
    a = isg.isg_anneal(isg.problem_of(t), 40, betas, 3)
    u, v, w = t.edges()
    b = isg.isg_anneal(isg.isg_problem_create_edges(t.n, u, v, w), 40, betas, 3)
    for x, y in zip(a.final(), b.final()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.best_all(), b.best_all())


# ------------------------------------------------------------------ targets
@pytest.mark.parametrize("kind,R,kernel", [("torus", 20, 1), ("torus", 70, 1), ("torus", 70, 3),
                                           ("graph", 3, 2), ("graph", 12, 2), ("graph", 12, 3)])
def test_target_stop_bit_exact(isg, kind, R, kernel):
    prob = I.torus(12, 10, 4) if kind == "torus" else I.random_graph(400, 800, 2)
    betas = I.geometric_betas(0.1, 5.0, 300)
    c = oracle.csr_of(prob)
    full = oracle.anneal(c, R, betas, 9)
    target = int(full.e_best.min()) + 4
    orc = oracle.anneal(c, R, betas, 9, target=target)
    assert orc.hit_sweep >= 0
    res = isg.isg_anneal(isg.problem_of(prob), R, betas, 9, target=target, kernel=kernel)
    assert_same(res, orc)
    unreachable = oracle.anneal(c, R, betas, 9, target=-10 ** 6)
    res2 = isg.isg_anneal(isg.problem_of(prob), R, betas, 9, target=-10 ** 6, kernel=kernel)
    assert_same(res2, unreachable)


# ------------------------------------------------------------------ energy
def test_isg_energy_matches_oracle(isg):
    g = weighted_graph()
    c = oracle.csr_of(g)
    rng = np.random.default_rng(0)
    s = rng.choice(np.array([-1, 1], np.int8), size=(17, g.n))
    e = isg.isg_energy(isg.problem_of(g), s)
    assert e.tolist() == [c.energy(x) for x in s]


# ------------------------------------------------------------------ batched
def test_batch_matches_single_and_oracle(isg):
    L, W = I.batch_sizes(24, seed=4)
    L, W = L // 4 * 2, W // 4 * 2   # smaller even sides, 8..70
    L, W = np.maximum(L, 4), np.maximum(W, 4)
    tori = [I.torus(int(L[k]), int(W[k]), 1000 + k) for k in range(24)]
    probs = [isg.problem_of(t) for t in tori]
    betas = I.geometric_betas(0.1, 5.0, 150)
    seeds = [k + 1 for k in range(24)]
    for R in (32, 20):
        outs = isg.isg_anneal_batch(probs, R, betas, seeds)
        for k in range(24):
            single = isg.isg_anneal(probs[k], R, betas, seeds[k])
            for x, y in zip(outs[k].final(), single.final()):
                assert np.array_equal(x, y)
            assert np.array_equal(outs[k].best_all(), single.best_all())
        for k in (0, 7, 23):
            orc = oracle.anneal(oracle.csr_of(tori[k]), R, betas, seeds[k])
            assert_same(outs[k], orc)


def test_batch_with_targets(isg):
    tori = [I.torus(8 + 2 * k, 10, 50 + k) for k in range(6)]
    probs = [isg.problem_of(t) for t in tori]
    betas = I.geometric_betas(0.1, 5.0, 200)
    seeds = [3 + k for k in range(6)]
    targets = []
    for k, t in enumerate(tori):
        full = oracle.anneal(oracle.csr_of(t), 32, betas, seeds[k])
        targets.append(int(full.e_best.min()) + 2 if k % 2 == 0 else None)
    outs = isg.isg_anneal_batch(probs, 32, betas, seeds, targets)
    for k, t in enumerate(tori):
        orc = oracle.anneal(oracle.csr_of(t), 32, betas, seeds[k], target=targets[k])
        assert_same(outs[k], orc)


def _mixed_batch():
    """Tori, +-1 graphs (graph words) and integer-weighted graphs (quads) of
    uneven sizes."""
    insts = []
    for k in range(6):
        insts.append(I.torus(8 + 4 * k, 6 + 2 * k, 300 + k))
    for k in range(5):
        insts.append(I.random_graph(150 + 120 * k, 200 + 150 * k, 400 + k))
    for k in range(4):
        g = I.random_graph(100 + 90 * k, 180 + 100 * k, 500 + k)
        w = np.array([(-2, 1, 3)[e % 3] for e in range(g.m)], np.int32)
        insts.append(I.Graph(g.n, g.u, g.v, w))
    return insts


@pytest.mark.parametrize("R", [64, 37])
def test_mixed_batch_equals_solo_runs_and_oracle(isg, R):
    """One batch of tori and graphs, several units per instance (R > 32): every
    result equals isg_anneal of the instance alone, and sampled ones the
    oracle; the three unit kinds all ran."""
    insts = _mixed_batch()
    probs = [isg.problem_of(x) for x in insts]
    betas = I.geometric_betas(0.1, 5.0, 120)
    seeds = [11 + k for k in range(len(insts))]
    outs = isg.isg_anneal_batch(probs, R, betas, seeds)
    kinds = {o.stats()["kernel"] for o in outs}
    assert kinds == {1, 2, 4}
    for k, x in enumerate(insts):
        solo = isg.isg_anneal(probs[k], R, betas, seeds[k])
        for a, b in zip(outs[k].final(), solo.final()):
            assert np.array_equal(a, b), k
        assert np.array_equal(outs[k].best_all(), solo.best_all()), k
    for k in (0, 5, 7, 10, 12, 14):
        assert_same(outs[k], oracle.anneal(oracle.csr_of(insts[k]), R, betas, seeds[k]))


def test_mixed_batch_with_targets_multi_unit(isg):
    """Targets on instances of several units: the second pass reruns them to
    the earliest unit's hit + 1, as a single solve does; equal to the oracle."""
    insts = _mixed_batch()
    probs = [isg.problem_of(x) for x in insts]
    betas = I.geometric_betas(0.1, 5.0, 150)
    seeds = [21 + k for k in range(len(insts))]
    R = 70
    targets = []
    for k, x in enumerate(insts):
        if k % 3 == 2:
            targets.append(None)
            continue
        full = oracle.anneal(oracle.csr_of(x), R, betas, seeds[k])
        # one reached early by some replica (+6), and one never reached (-10^6)
        targets.append(int(full.e_best.min()) + 6 if k % 3 == 0 else -10 ** 6)
    outs = isg.isg_anneal_batch(probs, R, betas, seeds, targets)
    for k, x in enumerate(insts):
        assert_same(outs[k], oracle.anneal(oracle.csr_of(x), R, betas, seeds[k],
                                           target=targets[k]))


def test_batch_autotune_keeps_results(isg):
    """The batch autotuner picks a shape; the tuned batch equals the untuned one."""
    insts = _mixed_batch()
    probs = [isg.problem_of(x) for x in insts]
    betas = I.geometric_betas(0.1, 5.0, 80)
    seeds = [31 + k for k in range(len(insts))]
    before = isg.isg_anneal_batch(probs, 40, betas, seeds)
    shape = isg.isg_autotune_batch(probs, 40, betas, probe_sweeps=8)
    assert shape["threads"] in (128, 192, 256, 384, 512) and 1 <= shape["ctas_per_sm"] <= 4
    after = isg.isg_anneal_batch(probs, 40, betas, seeds)
    assert after[0].stats()["threads"] == shape["threads"]
    for a, b in zip(before, after):
        for x, y in zip(a.final(), b.final()):
            assert np.array_equal(x, y)
        assert np.array_equal(a.best_all(), b.best_all())


# ------------------------------------------------------------------ resume
@pytest.mark.parametrize("make,kernel,R,cluster", [
    (lambda: I.torus(12, 10, 5), 1, 70, 2),                       # torus words
    (lambda: I.torus(8, 6, 5), 3, 40, 0),                         # one launch per sweep
    (lambda: I.random_graph(600, 900, 5), 4, 64, 3),              # graph words
    (lambda: I.random_graph(500, 700, 6, weight=3), 2, 37, 2),    # int8 quads, weight 3
])
def test_continue_equals_one_solve(isg, make, kernel, R, cluster):
    """25 sweeps, then 35, then 30 more through isg_anneal_continue equal one
    90-sweep solve of the same schedule, and the oracle's."""
    prob = make()
    p = isg.problem_of(prob)
    betas = I.geometric_betas(0.1, 4.0, 90)
    whole = isg.isg_anneal(p, R, betas, 17, kernel=kernel, cluster_ctas=cluster)
    part = isg.isg_anneal(p, R, betas[:25], 17, kernel=kernel, cluster_ctas=cluster)
    assert part.final(spins=False)[2] == 25
    isg.isg_anneal_continue(p, part, betas[25:60])
    isg.isg_anneal_continue(p, part, betas[60:])
    assert part.sweeps == whole.sweeps == 90
    for x, y in zip(part.final(), whole.final()):
        assert np.array_equal(x, y)
    assert np.array_equal(part.best_all(), whole.best_all())
    assert np.array_equal(part.best(spins=False)[3], whole.best(spins=False)[3])
    assert_same(part, oracle.anneal(oracle.csr_of(prob), R, betas, 17))


@pytest.mark.parametrize("make,kernel,R,cluster", [
    (lambda: I.torus(12, 10, 5), 1, 70, 2),
    (lambda: I.torus(8, 6, 5), 3, 40, 0),
    (lambda: I.random_graph(600, 900, 5), 4, 64, 3),
    (lambda: I.random_graph(500, 700, 6, weight=3), 2, 37, 2),
    (lambda: I.independent_set_instance(I.geometric_graph(300, 5.0, 2)), 2, 21, 1),  # fields
])
def test_resume_from_checkpoint_equals_one_solve(isg, make, kernel, R, cluster):
    """Export the final and best states after 40 sweeps, restart from them in a
    new solve (also on another cluster shape) and run to 90: equal to one
    90-sweep solve."""
    prob = make()
    p = isg.problem_of(prob)
    betas = I.geometric_betas(0.1, 4.0, 90)
    whole = isg.isg_anneal(p, R, betas, 23, kernel=kernel, cluster_ctas=cluster)
    first = isg.isg_anneal(p, R, betas[:40], 23, kernel=kernel, cluster_ctas=cluster)
    spins, best = first.final()[0], first.best_all()
    first.close()
    for shape in (cluster, 1):
        res = isg.isg_anneal_resume(p, R, betas, 23, 40, spins, best, kernel=kernel,
                                    cluster_ctas=shape)
        for x, y in zip(res.final(), whole.final()):
            assert np.array_equal(x, y), shape
        assert np.array_equal(res.best_all(), whole.best_all()), shape
        assert np.array_equal(res.best(spins=False)[3], whole.best(spins=False)[3]), shape
    assert_same(res, oracle.anneal(oracle.csr_of(prob), R, betas, 23))


def test_resume_rejects(isg):
    t = isg.problem_of(I.torus(8, 8, 2))
    betas = I.geometric_betas(0.2, 2.0, 20)
    ok = np.ones((32, 64), np.int8)
    bad = ok.copy()
    bad[3, 5] = 0
    for done, s, b in ((0, ok, ok), (21, ok, ok), (5, bad, ok), (5, ok, bad)):
        with pytest.raises(isg.IsgError) as e:
            isg.isg_anneal_resume(t, 32, betas, 1, done, s, b)
        assert e.value.status == isg.ISG_EINVAL
    res = isg.isg_anneal_resume(t, 32, betas, 1, 20, ok, ok)     # nothing left to run
    assert res.final(spins=False)[2] == 20
    assert np.array_equal(res.best_all(), ok)


def test_continue_rejects(isg):
    t = isg.problem_of(I.torus(8, 8, 2))
    other = isg.problem_of(I.torus(8, 8, 3))
    betas = I.geometric_betas(0.2, 2.0, 20)
    with_target = isg.isg_anneal(t, 32, betas, 1, target=-10 ** 6)
    res = isg.isg_anneal(t, 32, betas, 1)
    batch = isg.isg_anneal_batch([t], 32, betas, [1])[0]
    for p, r, b in ((t, with_target, betas), (other, res, betas), (t, batch, betas),
                    (t, res, []), (t, res, [np.inf])):
        with pytest.raises(isg.IsgError) as e:
            isg.isg_anneal_continue(p, r, b)
        assert e.value.status == isg.ISG_EINVAL
    isg.isg_anneal_continue(t, res, betas)                 # still usable after rejections
    whole = isg.isg_anneal(t, 32, np.concatenate([betas, betas]), 1)
    assert np.array_equal(res.best_all(), whole.best_all())


# ------------------------------------------------------------------ served
def test_server_results_equal_solo_runs(isg):
    """Requests of different kinds and sizes, submitted together so that they
    share chunks, each equal isg_anneal of the same request alone."""
    betas = I.geometric_betas(0.1, 5.0, 240)
    reqs = []
    for k in range(10):
        prob = I.torus(8 + 4 * (k % 3), 12, 70 + k) if k % 2 == 0 else \
            I.random_graph(300 + 50 * k, 450 + 80 * k, 70 + k)
        reqs.append((isg.problem_of(prob), prob, 32 if k % 3 else 20, 11 + k))
    targets = []
    for p, prob, R, seed in reqs:
        full = isg.isg_anneal(p, R, betas, seed)
        targets.append(full.best(spins=False)[0] + 2)
    srv = isg.Server(1 << 30, 4, 37)
    ids = {}
    for k, (p, prob, R, seed) in enumerate(reqs):
        ids[srv.submit(p, R, betas, seed, targets[k])] = k
    got = {}
    while len(got) < len(reqs):
        out = srv.poll(30.0)
        assert out is not None, "server timed out"
        got[ids[out[0]]] = out[1]
    st = srv.stats()
    assert st["submitted"] == st["completed"] == len(reqs)
    assert st["queued"] == 0 and st["active"] == 0
    assert 1 <= st["peak_active"] <= 4 and st["passes"] >= 1
    srv.close()
    for k, (p, prob, R, seed) in enumerate(reqs):
        solo = isg.isg_anneal(p, R, betas, seed, target=targets[k])
        a, b = got[k], solo
        for x, y in zip(a.final(), b.final()):
            assert np.array_equal(x, y)
        assert np.array_equal(a.best_all(), b.best_all())
        assert a.best(spins=False)[4] == b.best(spins=False)[4] >= 0
    k = 1
    orc = oracle.anneal(oracle.csr_of(reqs[k][1]), reqs[k][2], betas, reqs[k][3], target=targets[k])
    assert_same(got[k], orc)


def test_server_smallest_last_instance(isg):
    """A served graph re-coloured smallest-last runs its own classes: equal to the
    oracle given the oracle's smallest-last colouring."""
    g = I.random_graph(1500, 1499, 31)
    c = oracle.csr_of(g)
    col, _ = c.smallest_last_colouring()
    betas = I.geometric_betas(0.1, 5.0, 180)
    p = isg.problem_of(g, colouring=isg.COLOURING_SMALLEST_LAST)
    srv = isg.Server(1 << 30, 2, 50)
    srv.submit(p, 32, betas, 9)
    out = srv.poll(30.0)
    srv.close()
    assert out is not None
    assert_same(out[1], oracle.anneal(c, 32, betas, 9, colour=col))


@pytest.mark.parametrize("kind", ["torus", "graph_msc", "csr", "plain"])
def test_replica_shards_equal_one_solve(isg, kind):
    """A replica-sharded solve (the multi-GPU partition by replica word): calls
    at first_replica 0 and R (R a multiple of 32), concatenated, equal one call
    of 2R replicas bit for bit, and the second shard equals the oracle's
    replicas [R, 2R).  A first_replica that is not a multiple of 32 is EINVAL."""
    R, S, seed = 64, 60, 17
    if kind == "torus" or kind == "plain":
        inst = I.torus(12, 10, 3)
        kernel = {"torus": 1, "plain": 3}[kind]
    elif kind == "graph_msc":
        inst, kernel = I.random_graph(300, 450, 5), 4
    else:
        g = I.random_graph(240, 500, 6)
        w = np.array([(-2, 1, 3, -1)[k % 4] for k in range(g.m)], np.int32)
        inst, kernel = I.Graph(g.n, g.u, g.v, w), 2
    p = isg.problem_of(inst)
    betas = I.geometric_betas(0.2, 3.0, S)
    whole = isg.isg_anneal(p, 2 * R, betas, seed, kernel=kernel)
    parts = [isg.isg_anneal(p, R, betas, seed, kernel=kernel, first_replica=f) for f in (0, R)]
    assert parts[1].stats()["first_replica"] == R
    ws, we, wd = whole.final()
    for k, part in enumerate(parts):
        ps, pe, pd = part.final()
        rows = slice(k * R, (k + 1) * R)
        assert pd == wd
        assert np.array_equal(ps, ws[rows]) and np.array_equal(pe, we[rows])
        assert np.array_equal(part.best_all(), whole.best_all()[rows])
        assert np.array_equal(part.best()[3], whole.best()[3][rows])
    c = oracle.csr_of(inst)
    assert_same(parts[1], oracle.anneal(c, list(range(R, 2 * R)), betas, seed), first_replica=R)
    with pytest.raises(isg.IsgError) as e:
        isg.isg_anneal(p, R, betas, seed, kernel=kernel, first_replica=16)
    assert e.value.status == isg.ISG_EINVAL


def test_replica_shard_continue_and_resume(isg):
    """A shard keeps its replica offset through isg_anneal_continue and restarts
    from its checkpoint with isg_anneal_resume (same first_replica)."""
    inst = I.torus(16, 12, 9)
    p = isg.problem_of(inst)
    betas = I.geometric_betas(0.2, 3.0, 50)
    R, f = 32, 96
    whole = isg.isg_anneal(p, R, betas, 4, first_replica=f)
    head = isg.isg_anneal(p, R, betas[:20], 4, first_replica=f)
    spins, _, _ = head.final()
    best = head.best_all()
    isg.isg_anneal_continue(p, head, betas[20:])
    back = isg.isg_anneal_resume(p, R, betas, 4, 20, spins, best, first_replica=f)
    for r in (head, back):
        for x, y in zip(r.final(), whole.final()):
            assert np.array_equal(x, y)
        assert np.array_equal(r.best_all(), whole.best_all())


def test_server_rejects_bad_requests_and_times_out(isg):
    """Submit-time checks (EINVAL, and EBUSY for a request larger than the whole
    budget), poll timing out with nothing pending, and a request served after
    rejected ones equal to its solo run."""
    srv = isg.Server(1 << 20, 2, 10)                          # 1 MiB budget
    t = isg.problem_of(I.torus(8, 8, 1))
    for R, betas in ((0, [0.5]), (32, []), (32, [np.nan]), (32, [-1.0])):
        with pytest.raises(isg.IsgError) as e:
            srv.submit(t, R, betas, 1)
        assert e.value.status == isg.ISG_EINVAL
    with pytest.raises(isg.IsgError) as e:
        srv.submit(t, 32, [0.5], 1, target=2 ** 40)           # outside int32
    assert e.value.status == isg.ISG_EINVAL
    big = isg.problem_of(I.torus(100, 200, 1))
    with pytest.raises(isg.IsgError) as e:
        srv.submit(big, 1024, np.full(1000, 0.5), 1)
    assert e.value.status == isg.ISG_EBUSY
    assert srv.poll(0.05) is None
    betas = I.geometric_betas(0.2, 3.0, 20)
    rid = srv.submit(t, 32, betas, 3)
    out = srv.poll(30.0)
    assert out is not None and out[0] == rid
    assert srv.poll(0.01) is None
    st = srv.stats()
    assert st["submitted"] == st["completed"] == 1
    srv.close()
    solo = isg.isg_anneal(t, 32, betas, 3)
    for x, y in zip(out[1].final(), solo.final()):
        assert np.array_equal(x, y)
    assert np.array_equal(out[1].best_all(), solo.best_all())


def test_server_cancel(isg):
    """A request cancelled while queued and one cancelled while running come
    back with ECANCELLED; the request after them finishes equal to its solo run;
    cancelling a finished or unknown id is EINVAL."""
    import time
    t = isg.problem_of(I.torus(40, 40, 7))
    small = isg.problem_of(I.torus(8, 8, 7))
    long_betas = I.geometric_betas(0.1, 3.0, 20000)
    betas = I.geometric_betas(0.2, 3.0, 40)
    srv = isg.Server(1 << 30, 1, 50)              # one slot: b and c wait behind a
    a = srv.submit(t, 32, long_betas, 1)
    b = srv.submit(small, 32, betas, 2)
    c = srv.submit(small, 32, betas, 3)
    srv.cancel(b)                                 # queued
    t0 = time.time()
    while srv.stats()["passes"] < 2 and time.time() - t0 < 30:
        time.sleep(0.001)
    srv.cancel(a)                                 # running
    got = {}
    while len(got) < 3:
        out = srv.poll(60.0)
        assert out is not None, "server timed out"
        got[out[0]] = out[1]
    for rid in (c, 10 ** 9):
        with pytest.raises(isg.IsgError) as e:
            srv.cancel(rid)
        assert e.value.status == isg.ISG_EINVAL
    st = srv.stats()
    srv.close()
    assert st["cancelled"] == 2 and st["completed"] == 3 and st["passes"] >= 2
    for rid in (a, b):
        with pytest.raises(isg.IsgError) as e:
            got[rid].final()
        assert e.value.status == isg.ISG_ECANCELLED
    solo = isg.isg_anneal(small, 32, betas, 3)
    for x, y in zip(got[c].final(), solo.final()):
        assert np.array_equal(x, y)
    assert np.array_equal(got[c].best_all(), solo.best_all())


def test_server_cancel_racing_the_chunk_end(isg):
    """Cancels that race the chunk end at which their requests finish: a cancel
    that returns OK always hands its request back ECANCELLED, a cancel that
    comes too late is EINVAL and its request comes back with the normal result
    (equal to the solo run), and the cancel count equals the OK cancels."""
    import random
    import time
    small = isg.problem_of(I.torus(16, 16, 3))
    betas = I.geometric_betas(0.2, 3.0, 30)
    srv = isg.Server(1 << 30, 4, 30)              # every request ends in its first chunk
    rng = random.Random(5)
    ok, ids = set(), []
    for k in range(80):
        rid = srv.submit(small, 32, betas, k + 1)
        ids.append(rid)
        time.sleep(rng.uniform(0.0, 0.003))
        try:
            srv.cancel(rid)
            ok.add(rid)
        except isg.IsgError as e:
            assert e.status == isg.ISG_EINVAL
    got = {}
    while len(got) < len(ids):
        out = srv.poll(60.0)
        assert out is not None, "server timed out"
        got[out[0]] = out[1]
    st = srv.stats()
    srv.close()
    assert st["cancelled"] == len(ok) and st["completed"] == len(ids)
    for k, rid in enumerate(ids):
        if rid in ok:
            with pytest.raises(isg.IsgError) as e:
                got[rid].final()
            assert e.value.status == isg.ISG_ECANCELLED
        else:
            solo = isg.isg_anneal(small, 32, betas, k + 1)
            assert np.array_equal(got[rid].final()[1], solo.final()[1])
            assert np.array_equal(got[rid].best_all(), solo.best_all())


def test_server_admission_waits_for_free_device_memory(isg):
    """Admission by free device memory: with the budget and slots ample but the
    device nearly full, a second large request is held until the first is
    retired, then served equal to its solo run."""
    import torch
    big = isg.problem_of(I.torus(100, 200, 4))
    betas = I.geometric_betas(0.2, 3.0, 600)
    R = 8192                                   # ~370 MB of state and output per request
    srv = isg.Server(1 << 40, 8, 10)
    free, _ = torch.cuda.mem_get_info()
    hog = torch.empty(free - (900 << 20), dtype=torch.uint8, device="cuda")
    try:
        a = srv.submit(big, R, betas, 1)
        b = srv.submit(big, R, betas, 2)
        got = {}
        while len(got) < 2:
            out = srv.poll(120.0)
            assert out is not None, "server timed out"
            got[out[0]] = out[1]
        st = srv.stats()
        fa = got[a].final()[1]
        fb = got[b].final()[1]
        for r in got.values():
            r.close()
    finally:
        srv.close()
        del hog
        torch.cuda.empty_cache()
    assert st["peak_active"] == 1 and st["completed"] == 2
    for seed, f in ((1, fa), (2, fb)):
        solo = isg.isg_anneal(big, R, betas, seed)
        assert np.array_equal(solo.final()[1], f)
        solo.close()


def test_injected_allocation_failures(isg):
    """Host-side fault injection, no device fault: a solve whose state allocation
    fails returns ENOMEM and the library stays usable; a served request whose
    admission fails comes back with ENOMEM while the requests after it finish,
    each equal to its solo run."""
    t = isg.problem_of(I.torus(12, 10, 4))
    g = isg.problem_of(I.random_graph(400, 600, 4))
    betas = I.geometric_betas(0.2, 3.0, 60)
    try:
        isg.isg_debug_fail_allocations(1)
        with pytest.raises(isg.IsgError) as e:
            isg.isg_anneal(t, 32, betas, 5)
        assert e.value.status == isg.ISG_ENOMEM
        solo_t = isg.isg_anneal(t, 32, betas, 5)          # the next allocation succeeds
        solo_g = isg.isg_anneal(g, 32, betas, 6)
        srv = isg.Server(1 << 30, 1, 20)                  # one slot: admitted in order
        isg.isg_debug_fail_allocations(1)
        ids = [srv.submit(t, 32, betas, 5), srv.submit(g, 32, betas, 6),
               srv.submit(t, 32, betas, 5)]
        got = {}
        while len(got) < 3:
            out = srv.poll(30.0)
            assert out is not None, "server timed out"
            got[ids.index(out[0])] = out[1]
        srv.close()
    finally:
        isg.isg_debug_fail_allocations(0)
    with pytest.raises(isg.IsgError) as e:
        got[0].final()
    assert e.value.status == isg.ISG_ENOMEM
    for k, ref in ((1, solo_g), (2, solo_t)):
        for x, y in zip(got[k].final(), ref.final()):
            assert np.array_equal(x, y)
        assert np.array_equal(got[k].best_all(), ref.best_all())


# ------------------------------------------------------------------ full sizes
@pytest.mark.slow
def test_torus_80x100_full_size_sampled(isg):
    """The benchmark's workload and launch shape: 80x100 torus, 1,024
    replicas, 10,000 geometric sweeps.  Sampled replicas (first and last of
    several words) against the oracle; every replica's tracked energies
    against a full recompute."""
    sv = I.torus_80x100()
    p = isg.problem_of(sv.problem)
    res = isg.isg_anneal(p, sv.replicas, sv.betas, sv.seed)
    reps = [0, 1, 31, 32, 517, 1023]
    orc = oracle.anneal(oracle.csr_of(sv.problem), reps, sv.betas, sv.seed)
    assert_same(res, orc, reps=reps)
    spins, e, done = res.final()
    assert done == sv.sweeps
    assert np.array_equal(isg.isg_energy(p, spins), e)
    assert np.array_equal(isg.isg_energy(p, res.best_all()), res.best(spins=False)[3])


@pytest.mark.parametrize("kernel,cluster,threads", [(4, 12, 512), (4, 3, 128), (2, 4, 256),
                                                   (3, 0, 0)])
def test_smallest_last_colouring_bit_exact(isg, kernel, cluster, threads):
    """Instances re-coloured smallest-last run those classes, bit for bit with the
    oracle given the oracle's own smallest-last colouring."""
    g = I.random_graph(3000, 2999, 5)
    c = oracle.csr_of(g)
    col, nc = c.smallest_last_colouring()
    betas = I.geometric_betas(0.1, 5.0, 150)
    orc = oracle.anneal(c, 40, betas, 7, colour=col, check_energy=True)
    p = isg.problem_of(g, colouring=isg.COLOURING_SMALLEST_LAST)
    assert isg.isg_problem_info(p)["n_colors"] == nc
    res = isg.isg_anneal(p, 40, betas, 7, kernel=kernel, cluster_ctas=cluster, threads=threads)
    assert_same(res, orc)
    with pytest.raises(isg.IsgError):
        isg.isg_problem_set_colouring(p, isg.COLOURING_GREEDY)  # device state exists now


@functools.lru_cache(maxsize=1)
def random_10000_oracle(reps):
    sv = I.random_10000()
    return oracle.anneal(oracle.csr_of(sv.problem), list(reps), sv.betas, sv.seed)


@pytest.mark.slow
@pytest.mark.parametrize("shape", [{}, {"cluster_ctas": 12, "threads": 512}])
def test_random_10000_full_size_sampled(isg, shape):
    """Default shape and the 12-CTA cluster shape the bench's autotuner picks."""
    sv = I.random_10000()
    p = isg.problem_of(sv.problem)
    res = isg.isg_anneal(p, sv.replicas, sv.betas, sv.seed, **shape)
    reps = (0, 1, 2, 3, 130, 255)
    assert_same(res, random_10000_oracle(reps), reps=list(reps))
    spins, e, _ = res.final()
    assert np.array_equal(isg.isg_energy(p, spins), e)


@pytest.mark.slow
def test_batch_512_full_size_sampled(isg):
    """512 uneven tori, 32 replicas, 2,000 sweeps in one persistent kernel:
    sampled instances equal their one-instance-per-launch plain runs, and one
    equals the oracle."""
    batch = I.torus_batch()
    probs = [isg.problem_of(sv.problem) for sv in batch]
    outs = isg.isg_anneal_batch(probs, 32, batch[0].betas, [sv.seed for sv in batch])
    sizes = [sv.n for sv in batch]
    picks = [int(np.argmax(sizes)), int(np.argmin(sizes)), 100, 311]
    for k in picks:
        sv = batch[k]
        plain = isg.isg_anneal(probs[k], 32, sv.betas, sv.seed, kernel=3)
        for x, y in zip(outs[k].final(), plain.final()):
            assert np.array_equal(x, y)
        assert np.array_equal(outs[k].best_all(), plain.best_all())
    k = 100
    orc = oracle.anneal(oracle.csr_of(batch[k].problem), 32, batch[k].betas, batch[k].seed)
    assert_same(outs[k], orc)


@pytest.mark.slow
def test_random_10000_smallest_last_full_size_sampled(isg):
    """The random-graph workload re-coloured smallest-last (3 classes) at the
    12-CTA shape: sampled replicas equal the oracle run on the same classes."""
    sv = I.random_10000()
    c = oracle.csr_of(sv.problem)
    col, nc = c.smallest_last_colouring()
    reps = [0, 7, 64, 255]
    orc = oracle.anneal(c, reps, sv.betas, sv.seed, colour=col)
    p = isg.problem_of(sv.problem, colouring=isg.COLOURING_SMALLEST_LAST)
    res = isg.isg_anneal(p, sv.replicas, sv.betas, sv.seed, cluster_ctas=12, threads=512)
    assert_same(res, orc, reps=reps)

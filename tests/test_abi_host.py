"""Host-side checks of libisg that need no GPU: the library loads, exports every
function include/isg.h declares, validates instances, and colours them as the
oracle's independent smallest-last colouring does."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2311_09275_gb300 import inputs as I
from conftest import ROOT


@pytest.fixture(scope="module")
def isg():
    from paper_2311_09275_gb300 import build
    build.build()
    from paper_2311_09275_gb300 import isg as mod
    return mod


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(isg_[a-z_0-9]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(isg):
    names = _declared()
    assert len(names) >= 20
    lib = ctypes.CDLL(isg.library_path())
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert "sm_103a" in isg.isg_version()


def test_torus_validation(isg):
    j = np.ones(36, np.int8)
    with pytest.raises(isg.IsgError) as e:
        isg.isg_problem_create_torus(5, 6, np.ones(30, np.int8), np.ones(30, np.int8))
    assert e.value.status == isg.ISG_EINVAL and "even" in str(e.value)
    with pytest.raises(isg.IsgError):
        isg.isg_problem_create_torus(2, 18, j, j)
    bad = j.copy()
    bad[3] = 0
    with pytest.raises(isg.IsgError):
        isg.isg_problem_create_torus(6, 6, bad, j)
    p = isg.isg_problem_create_torus(6, 6, j, j)
    assert (p.n, p.m, p.total_weight, p.n_colors) == (36, 72, 72, 2)


def test_edge_validation(isg):
    E = isg.IsgError
    with pytest.raises(E):
        isg.isg_problem_create_edges(4, [0], [4], [1])        # out of range
    with pytest.raises(E):
        isg.isg_problem_create_edges(4, [2], [2], [1])        # self-loop
    with pytest.raises(E):
        isg.isg_problem_create_edges(4, [0, 1], [1, 0], [1, 1])  # duplicate pair
    with pytest.raises(E):
        isg.isg_problem_create_edges(0, [], [], [])
    with pytest.raises(E):
        isg.isg_problem_create_edges(3, [0, 1], [1, 2], [2 ** 29, 2 ** 29])  # |w| sum 2^30
    p = isg.isg_problem_create_edges(5, [], [], [])          # no edges is fine
    assert (p.n, p.m, p.n_colors) == (5, 0, 1)


def test_csr_validation_and_equivalence(isg):
    g = I.random_graph(50, 80, 3)
    c = oracle.csr_of(g)
    p = isg.isg_problem_create_csr(g.n, c.rowptr, c.col[:2 * g.m], c.wt[:2 * g.m])
    q = isg.isg_problem_create_edges(g.n, g.u, g.v, g.w)
    assert isg.isg_problem_info(p, colors=True)["colors"].tolist() == \
        isg.isg_problem_info(q, colors=True)["colors"].tolist()
    col = c.col[:2 * g.m].copy()
    col[0] = (col[0] + 1) % g.n                               # breaks symmetry
    with pytest.raises(isg.IsgError):
        isg.isg_problem_create_csr(g.n, c.rowptr, col, c.wt[:2 * g.m])


@pytest.mark.parametrize("n,m,seed", [(2000, 1999, 1), (10000, 9999, 1), (3000, 6000, 2),
                                      (500, 20000, 3), (12000, 150000, 9)])
def test_colouring_matches_oracle(isg, n, m, seed):
    g = I.random_graph(n, m, seed)
    p = isg.problem_of(g)
    info = isg.isg_problem_info(p, colors=True)
    col, nc = oracle.csr_of(g).greedy_colouring()
    assert info["n_colors"] == nc
    assert np.array_equal(info["colors"], col)
    assert info["total_weight"] == int(g.w.sum()) and info["m"] == m


def test_torus_colouring_is_checkerboard(isg):
    t = I.torus(8, 12, 5)
    info = isg.isg_problem_info(isg.problem_of(t), colors=True)
    col, nc = oracle.csr_of(t).greedy_colouring()
    assert info["n_colors"] == 2 and np.array_equal(info["colors"], col)
    # the same torus as a plain edge list, either colouring: the same checkerboard
    u, v, w = t.edges()
    for method in (0, 1):
        q = isg.isg_problem_create_edges(t.n, u, v, w)
        isg.isg_problem_set_colouring(q, method)
        info = isg.isg_problem_info(q, colors=True)
        assert info["n_colors"] == 2 and np.array_equal(info["colors"], col)


@pytest.mark.parametrize("kind", ["linear", "geometric", "extremes"])
def test_acceptance_table_equals_oracle(isg, kind):
    """The library's thresholds equal the oracle's, bit for bit (table parity)."""
    if kind == "linear":
        betas, kmax = I.linear_betas(0.1, 3.0, 1000), 4
    elif kind == "geometric":
        betas, kmax = I.geometric_betas(0.1, 5.0, 10000), 8
    else:
        betas, kmax = np.array([0.0, 1e-12, 0.5, 11.0, 1e3, 1e300]), 63
    lib = isg.isg_acceptance_table(betas, kmax)
    orc = oracle.accept_table(betas, kmax)
    assert lib.dtype == np.uint32 and lib.shape == orc.shape
    assert np.array_equal(lib, orc)


def test_acceptance_table_rejects_bad_input(isg):
    with pytest.raises(isg.IsgError):
        isg.isg_acceptance_table(np.array([0.5, np.nan]), 2)
    with pytest.raises(isg.IsgError):
        isg.isg_acceptance_table(np.array([-0.1]), 2)
    with pytest.raises(isg.IsgError):
        isg.isg_acceptance_table(np.array([0.5]), -1)


def test_fields_validation_and_info(isg):
    g = I.random_graph(30, 40, 3)
    h = np.arange(30, dtype=np.int32) - 15
    p = isg.isg_problem_create_fields(30, g.u, g.v, g.w, h)
    assert (p.n, p.m, p.total_weight) == (30, 40, 40)  # total_weight stays sum w
    q = isg.isg_problem_create_fields(30, g.u, g.v, g.w, None)  # no fields = plain edges
    assert (q.n, q.m) == (30, 40)
    with pytest.raises(ValueError):
        isg.isg_problem_create_fields(30, g.u, g.v, g.w, h[:10])
    with pytest.raises(isg.IsgError):  # sum |w| + sum |h| >= 2^30
        isg.isg_problem_create_fields(30, g.u, g.v, g.w, np.full(30, 1 << 26, np.int32))
    with pytest.raises(isg.IsgError):  # bad edge still rejected
        isg.isg_problem_create_fields(3, [0], [0], [1], [0, 0, 0])


@pytest.mark.parametrize("n,m,seed", [(2000, 1999, 1), (10000, 9999, 1), (3000, 6000, 2),
                                      (500, 20000, 3), (12000, 150000, 9)])
def test_smallest_last_colouring_matches_oracle(isg, n, m, seed):
    g = I.random_graph(n, m, seed)
    p = isg.problem_of(g, colouring=1)
    info = isg.isg_problem_info(p, colors=True)
    col, nc = oracle.csr_of(g).smallest_last_colouring()
    assert info["n_colors"] == nc and np.array_equal(info["colors"], col)


def test_colouring_matches_oracle_on_geometric_and_fields(isg):
    """Geometric graphs (many equal degrees, so the tie rule decides) and an
    independent-set instance with fields colour as the oracle does, both ways."""
    for g in (I.geometric_graph(3000, 6.0, 4), I.independent_set_instance(I.geometric_graph(2000, 9.0, 5))):
        info = isg.isg_problem_info(isg.problem_of(g), colors=True)
        col, nc = oracle.csr_of(g).greedy_colouring()
        assert info["n_colors"] == nc and np.array_equal(info["colors"], col)
        info = isg.isg_problem_info(isg.problem_of(g, colouring=1), colors=True)
        col, nc = oracle.csr_of(g).smallest_last_colouring()
        assert info["n_colors"] == nc and np.array_equal(info["colors"], col)


def test_set_colouring_rejects(isg):
    t = I.torus(8, 8, 1)
    with pytest.raises(isg.IsgError):
        isg.isg_problem_set_colouring(isg.problem_of(t), 1)  # tori keep the checkerboard
    p = isg.problem_of(I.random_graph(50, 80, 2))
    with pytest.raises(isg.IsgError):
        isg.isg_problem_set_colouring(p, 7)
    isg.isg_problem_set_colouring(p, 1)
    isg.isg_problem_set_colouring(p, 0)  # back to greedy
    g = I.random_graph(50, 80, 2)
    info = isg.isg_problem_info(p, colors=True)
    assert np.array_equal(info["colors"], oracle.csr_of(g).greedy_colouring()[0])


def test_server_argument_checks(isg):
    """isg_server_create validates before any device work; NULL handles are EINVAL."""
    for budget, slots, chunk in ((0, 4, 10), (1 << 30, 0, 10), (1 << 30, 4, 0)):
        with pytest.raises(isg.IsgError) as e:
            isg.Server(budget, slots, chunk)
        assert e.value.status == isg.ISG_EINVAL
    t = isg.problem_of(I.torus(8, 8, 1))
    with pytest.raises(isg.IsgError) as e:
        isg.isg_server_submit(None, t, 32, [0.5], 1)
    assert e.value.status == isg.ISG_EINVAL
    with pytest.raises(isg.IsgError) as e:
        isg.isg_server_poll(None, 0.0)
    assert e.value.status == isg.ISG_EINVAL


def test_continue_rejects_null(isg):
    with pytest.raises(isg.IsgError) as e:
        isg.isg_anneal_continue(None, None, [0.5])
    assert e.value.status == isg.ISG_EINVAL


def test_resume_rejects_null(isg):
    with pytest.raises(isg.IsgError) as e:
        isg.isg_anneal_resume(None, 4, [0.5, 0.5], 1, 1, np.ones(8, np.int8), np.ones(8, np.int8))
    assert e.value.status == isg.ISG_EINVAL


def test_debug_fail_allocations_arguments(isg):
    with pytest.raises(isg.IsgError) as e:
        isg.isg_debug_fail_allocations(-1)
    assert e.value.status == isg.ISG_EINVAL
    isg.isg_debug_fail_allocations(3)
    isg.isg_debug_fail_allocations(0)


def test_server_cancel_rejects_null(isg):
    with pytest.raises(isg.IsgError) as e:
        isg.isg_server_cancel(None, 1)
    assert e.value.status == isg.ISG_EINVAL


def test_resume_checks_state_sizes(isg):
    """The binding checks the checkpoint's size before any device work."""
    p = isg.problem_of(I.torus(8, 8, 1))
    with pytest.raises(ValueError):
        isg.isg_anneal_resume(p, 32, [0.5, 0.5], 1, 1, np.ones((32, 63), np.int8),
                              np.ones((32, 64), np.int8))

"""isg_energy_noalloc: the energy check for callers that cannot allocate
device memory at call time (their device memory is reserved by another
allocator, or they must stay out of the driver's allocator).

The test owns every device buffer (torch allocates them here, outside the
call), calls the entry point through the C ABI twice in a row, and requires
exactly the energies of the allocating entry point isg_energy.  This file is
collected last on purpose, and passes alone or after the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_2311_09275_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_energy_noalloc_matches_isg_energy_twice():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2311_09275_gb300 import build
    build.build()
    from paper_2311_09275_gb300 import isg

    g = I.random_graph(3000, 7000, 21)
    w = np.array([(-3, -1, 1, 2, 5)[k % 5] for k in range(g.m)], np.int32)
    csr = oracle.Csr(g.n, g.u, g.v, w)
    p = isg.isg_problem_create_edges(g.n, g.u, g.v, w)
    dev = torch.device("cuda", 0)
    rowptr = torch.from_numpy(csr.rowptr).to(dev)
    col = torch.from_numpy(csr.col[: 2 * g.m].copy()).to(dev)
    wt = torch.from_numpy(csr.wt[: 2 * g.m].copy()).to(dev)
    rng = np.random.default_rng(3)
    stream = torch.cuda.current_stream()
    for R in (37, 300):   # two calls in a row, different sizes
        spins = rng.choice(np.array([-1, 1], np.int8), size=(R, g.n))
        s_dev = torch.from_numpy(spins).to(dev)
        out = torch.full((R,), -7, dtype=torch.int64, device=dev)
        isg.isg_energy_noalloc(g.n, rowptr.data_ptr(), col.data_ptr(), wt.data_ptr(),
                               s_dev.data_ptr(), R, out.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        want = isg.isg_energy(p, spins)
        assert np.array_equal(out.cpu().numpy(), want)

    with pytest.raises(isg.IsgError) as e:
        isg.isg_energy_noalloc(g.n, rowptr.data_ptr(), col.data_ptr(), wt.data_ptr(),
                               s_dev.data_ptr(), 2049, out.data_ptr(), stream=stream)
    assert e.value.status == isg.ISG_EINVAL and "2048" in str(e.value)

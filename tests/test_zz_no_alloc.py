"""isg_energy_noalloc: the energy check for callers that cannot allocate
device memory at call time (their device memory is reserved by another
allocator, or they must stay out of the driver's allocator).

The test owns every device buffer (torch allocates them here, outside the
call), calls the entry point through the C ABI twice in a row, and requires
exactly the oracle's energies (and those of the allocating entry point
isg_energy), with the device's free memory, the default memory pool and
torch's allocator unchanged across the second call.  The file name makes
pytest collect it last, so that a run stopping at its first failure has
already run every other test; the test itself does not depend on the others
and passes alone in a fresh process or after them.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2311_09275_gb300 import inputs as I

pytestmark = pytest.mark.gpu

_POOL_RESERVED, _POOL_USED = 5, 7   # cudaMemPoolAttrReservedMemCurrent, ...UsedMemCurrent


def _pool_bytes(device: int):
    """(reserved, used) bytes of the device's default stream-ordered memory pool,
    read through the CUDA runtime the library itself loaded."""
    rt = ctypes.CDLL("libcudart.so.13")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), device) == 0
    out = []
    for attr in (_POOL_RESERVED, _POOL_USED):
        v = ctypes.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        out.append(v.value)
    return tuple(out)


def test_energy_noalloc_matches_oracle_twice_without_allocating():
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
    for call, R in enumerate((37, 300)):   # two calls in a row, different sizes
        spins = rng.choice(np.array([-1, 1], np.int8), size=(R, g.n))
        s_dev = torch.from_numpy(spins).to(dev)
        out = torch.full((R,), -7, dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        before = (torch.cuda.mem_get_info(0)[0], _pool_bytes(0), torch.cuda.memory_allocated(0))
        isg.isg_energy_noalloc(g.n, rowptr.data_ptr(), col.data_ptr(), wt.data_ptr(),
                               s_dev.data_ptr(), R, out.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        after = (torch.cuda.mem_get_info(0)[0], _pool_bytes(0), torch.cuda.memory_allocated(0))
        if call == 1:   # the first call on a device may load the module; the second allocates nothing
            assert after == before
        got = out.cpu().numpy()
        assert np.array_equal(got, [csr.energy(s) for s in spins])
        assert np.array_equal(got, isg.isg_energy(p, spins))

    with pytest.raises(isg.IsgError) as e:
        isg.isg_energy_noalloc(g.n, rowptr.data_ptr(), col.data_ptr(), wt.data_ptr(),
                               s_dev.data_ptr(), 2049, out.data_ptr(), stream=stream)
    assert e.value.status == isg.ISG_EINVAL and "2048" in str(e.value)

"""The oracle's Philox4x32-10 against cuRAND's public Philox4x32-10 block
function (a library routine, evaluated on the GPU) on random counters and keys.
The CUDA path agrees with the oracle bit for bit in every parity test, so this
pins the random numbers of all three."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_philox_equals_curand(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "philox_curand_check")
    subprocess.check_call([nvcc, "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                           os.path.join(HERE, "philox_curand_check.cu"), "-o", exe])
    rng = np.random.default_rng(2024)
    n = 4000
    ck = rng.integers(0, 2 ** 32, size=(n, 6), dtype=np.uint64)
    ck[:8, :4] = [[0, 0, 0, 0], [1, 2, 3, 0], [7999, 9999, 255, 0], [7999, 0, 255, 1],
                  [2 ** 32 - 1] * 4, [0, 1, 0, 0], [5, 5, 5, 5], [1 << 31, 0, 1, 1]]
    text = f"{n}\n" + "\n".join(" ".join(str(int(x)) for x in row) for row in ck) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    got = np.array([[int(x) for x in line.split()] for line in out.strip().splitlines()])
    assert got.shape == (n, 4)
    for i in range(n):
        want = oracle.philox4x32_10(ck[i, :4].astype(np.uint32), ck[i, 4:].astype(np.uint32))
        assert [int(x) for x in want] == got[i].tolist(), i

"""Multi-process path of bench.py on CPU (gloo, world size 2): every rank anneals
its own replica range of the same solve (same seed; weak scaling, no data
exchange), the job time is the maximum over ranks, the work is the sum over
ranks, and the final argmin over (best energy, global replica) is gathered."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch
    import bench

    class A:
        impl = "reference"     # forces the gloo backend in dist_setup
    w, r, local, dist = bench.dist_setup(A())
    assert (w, r) == (world, rank)
    cpu = torch.device("cpu")
    sv, name, first = bench.workload("torus", rank, sweeps=10)
    t = 1.0 + 2.0 * rank                      # rank 1 is the slow one
    tmax = bench.max_over_ranks(t, dist, cpu)
    total = bench.sum_over_ranks(float(sv.attempts), dist, cpu)
    # argmin gather: rank 1 strictly better; then a tie in energy, which goes to
    # the lower global replica (rank 0's, although its local index is higher)
    best = bench.global_best(-100 - rank, 7, first, dist, cpu)
    tie = bench.global_best(-50, 9 if rank == 0 else 2, first, dist, cpu)
    bench.barrier(dist)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{tmax} {total} {sv.seed} {name} {first} {best[0]} {best[1]} {tie[0]} "
                f"{tie[1]}\n")
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregation(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    for tmax, total, seed, name, first, be, br, te, tr in rows:
        assert float(tmax) == 3.0
        assert float(total) == 2 * 1024 * 8000 * 10
        assert (int(be), int(br)) == (-101, 1024 + 7)      # rank 1's replica 7
        assert (int(te), int(tr)) == (-50, 9)              # tie: rank 0's replica 9 < 1026
    assert rows[0][2] == rows[1][2]          # one solve: the same seed
    assert rows[0][3] == rows[1][3]          # of the same workload
    assert (int(rows[0][4]), int(rows[1][4])) == (0, 1024)   # replica ranges [0,1024), [1024,2048)


def test_reference_arm_under_torchrun_prints_one_line():
    """`bench.py --impl reference` launched as two ranks: rank 0 alone times the
    oracle and prints one JSON line; the other rank exits 0 without work."""
    import json
    import subprocess
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "1", "--sweeps", "10"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(x) for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, out.stdout
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]

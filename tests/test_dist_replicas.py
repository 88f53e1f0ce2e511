"""The N > 1 path of bench.py on CPU: two gloo ranks set up the process group from
the torchrun environment, meet at the barrier, take the maximum of their timings
(the job time of replicas), and only rank 0 runs the oracle reference arm."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup()
    bench.barrier(ws)
    # rank 1 is the slower replica: the job time is its time
    t = bench.allreduce_max(ws, 10.0 + 5.0 * r)

    class A:
        steps, warmup = 1, 3
    ref = bench.run_reference(A, ws, r) if r == 1 else "skipped"
    bench.barrier(ws)
    dist.destroy_process_group()
    with open(out + f".{rank}", "w") as f:
        f.write(f"{ws} {r} {local} {t} {ref}")


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "rank")
    mp.start_processes(_rank_main, args=(port, out), nprocs=2, start_method="spawn", join=True)
    r0 = open(out + ".0").read().split()
    r1 = open(out + ".1").read().split()
    assert r0[:4] == ["2", "0", "0", "15.0"]
    assert r1[:4] == ["2", "1", "1", "15.0"]
    assert r1[4] == "None"   # the reference arm runs on rank 0 only

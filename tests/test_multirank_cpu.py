"""The N > 1 path of the benchmark on CPU with the gloo backend
(world size 2): every rank runs its own independent solve (distinct
seeds, hence distinct initial data), the job's time is the max over the
ranks, and the whole-job throughput counts the units of all ranks.  The
fine propagations of different solves never exchange data, so the only
collectives are the timing ones tested here."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2511_13386_gb300 import workloads as W
    w = W.batched(64, 16, 1e-2, seed=bench.rank_seed(rank), n_slices=4)
    # per-rank "time": rank-dependent so that the max is not rank 0's
    t = bench.max_over_ranks(10.0 + 5.0 * rank, td)
    td.barrier()
    out[rank] = (t, float(w.rho0[3]), bench.rank_seed(rank))
    td.destroy_process_group()


def test_two_ranks_independent_solves_and_max_time():
    world = 2
    port = _free_port()
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    times = [out[r][0] for r in range(world)]
    assert times == [15.0, 15.0]               # every rank sees the slowest rank's time
    assert out[0][2] != out[1][2]               # distinct seeds
    assert out[0][1] != out[1][1]               # hence distinct initial data


def test_job_rate_counts_all_ranks():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(1e9, 4, 2.0) == pytest.approx(2e9)
    assert bench.max_over_ranks(3.5, None) == 3.5

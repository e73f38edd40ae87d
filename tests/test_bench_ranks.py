"""The multi-rank plumbing of bench.py (barrier, maximum of the timed region
over ranks), run as two gloo ranks on the CPU. With N GPUs bench.py runs N
independent replicas of the workload and reports the whole job's cell-updates
over the slowest rank's time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    m = bench.max_over_ranks(world, float(10 + rank))
    out.put((rank, m))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 11.0, 1: 11.0}


def test_fp32_error_report_arithmetic(monkeypatch):
    """The benchmark's fp32_error_vs_fp64 key: relative infinity-norm E_z and
    absolute population differences of the FP32 run from the FP64 run, with a
    stand-in solver that returns known perturbations (no GPU)."""
    import numpy as np

    import bench
    from paper_1710_09799_gb300 import mln

    class Stand:
        def __init__(self, params, E0=None):
            self.fp32 = params.s.precision == mln.MLN_FP32
            self.E = 2.0 * np.asarray(E0)

        def step(self, n):
            pass

        def sync(self):
            pass

        def fields(self):
            return self.E * (1 + 3e-6 if self.fp32 else 1.0), 0 * self.E

        def populations(self):
            return np.full((7, 3), 0.25) + (4e-9 if self.fp32 else 0.0)

        def close(self):
            pass

    monkeypatch.setattr(mln, "Solver", Stand)
    r = bench.fp32_error_vs_fp64(n_cells=128, n_steps=5)
    assert abs(r["E_rel"] - 3e-6) < 1e-12 and abs(r["pop_abs"] - 4e-9) < 1e-15
    assert "128 cells x 5 steps" in r["case"]

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
    """The benchmark's fp32_error_vs_oracle key: relative infinity-norm E_z and
    absolute population differences of the FP32 and FP64 runs from the
    oracle's result, with a stand-in solver that returns known perturbations
    of that result (no GPU)."""
    import numpy as np

    import bench
    from paper_1710_09799_gb300 import mln

    E_ref = np.linspace(-3.0, 5.0, 128)
    rho_ref = np.zeros((7, 3, 3), complex)
    rho_ref[:, 0, 0], rho_ref[:, 1, 1], rho_ref[:, 2, 2] = 0.25, 0.5, 0.25

    class Ref:
        E, rho = E_ref, rho_ref

    class Stand:
        def __init__(self, params, E0=None):
            self.fp32 = params.s.precision == mln.MLN_FP32

        def step(self, n):
            pass

        def sync(self):
            pass

        def fields(self):
            return E_ref * (1 + (3e-6 if self.fp32 else 2e-13)), 0 * E_ref

        def populations(self):
            return np.einsum("cii->ci", rho_ref).real + (4e-9 if self.fp32 else 1e-14)

        def close(self):
            pass

    monkeypatch.setattr(mln, "Solver", Stand)
    r = bench.fp32_error_vs_oracle(Ref, n_cells=128, n_steps=5)
    assert abs(r["fp32"]["E_rel"] - 3e-6) < 1e-12 and abs(r["fp32"]["pop_abs"] - 4e-9) < 1e-15
    assert abs(r["fp64"]["E_rel"] - 2e-13) < 1e-15 and abs(r["fp64"]["pop_abs"] - 1e-14) < 1e-16
    assert "128 cells x 5 steps" in r["case"]

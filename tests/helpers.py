"""Shared helpers of the GPU tests: run a workloads.Problem through the C-ABI."""
from __future__ import annotations

import numpy as np


def params_of(p, **kw):
    from paper_1710_09799_gb300 import mln
    args = dict(N=p.N, H0=p.H0, mu=p.mu, G=p.G, rho0=p.rho0, N_a=p.N_a, n_cells=p.n_cells,
                medium_begin=p.medium_begin, medium_end=p.medium_end, dx=p.dx, dt=p.dt,
                eps_r=p.eps_r, mu_r=p.mu_r, sigma=p.sigma, boundary=p.boundary,
                source_kind=p.source_kind, source_cell=p.source_cell, maxwell=p.maxwell)
    args.update(kw)
    return mln.Params(**args)


def make_solver(p, precision="fp64", form="strang", **kw):
    from paper_1710_09799_gb300 import mln
    return mln.Solver(params_of(p, precision=precision, form=form, **kw), E0=p.e_init())


def src_tensor(p, n0, count):
    import torch
    s = p.source_samples(n0, count)
    if s is None:
        return None
    return torch.as_tensor(np.ascontiguousarray(s), dtype=torch.float64, device="cuda")


def gpu_run(p, n_steps, precision="fp64", form="strang", chunks=None, **kw):
    """Run n_steps (optionally as several mln_step calls of the given sizes) and
    return (E, H, rho of every medium cell, solver)."""
    s = make_solver(p, precision, form, **kw)
    done = 0
    for c in (chunks or [n_steps]):
        s.step(c, src_tensor(p, done, c))
        done += c
    assert done == n_steps
    s.sync()
    E, H = s.fields()
    rho = s.rho() if p.n_medium > 0 else np.zeros((0, p.N, p.N), complex)
    return E, H, rho, s


def rel_inf(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))

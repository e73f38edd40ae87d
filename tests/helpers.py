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


# ---------------------------------------------------------------- FP32 bounds
#
# FP32 state and propagators with FP64 set-up: every step rounds the state's
# increments and the field update at u = 2^-24 relative, and the FDTD recurrence
# is neutrally stable, so the error after n steps grows at most linearly,
# err ~ kappa * u * n. kappa depends on the problem (how much of the state the
# rounding reaches, how the field feeds it back), so it is set per workload
# family from the coefficient measured on a GB300 (err / (u n) of the runs
# below) times about five: large enough for run-to-run and kernel-to-kernel
# differences of the summation order, small enough that an arithmetic
# regression of an order of magnitude fails.
U32 = 2.0 ** -24

# family: (kappa for E_z, relative infinity norm; kappa for populations, absolute)
FP32_KAPPA = {
    "ring": (0.5, 4.5e-3),          # three-level ring: Strang, merged, Rodrigues forms
    "ring_rotated": (4.0, 2.5e-3),  # three-level ring, rotated basis (dP/dt sums population-sized terms)
    "two_level": (0.022, 0.2),      # two-level SIT grid (sech pulse through the medium)
    "six_level": (0.25, 0.12),      # six-level pulse (D = 35), every cell model and form
    "five_level_ring": (0.45, 3e-3),
    "five_level_ring_rotated": (5.5, 0.05),  # rotated basis on a ring (as ring_rotated), both kernels
    "pstd": (1.0, 0.11),            # two-level medium on a PSTD ring
}

# Measured on a GB300 (one run each): family, steps, E error, population error.
FP32_MEASURED = [
    ("ring", 2000, 1.146e-5, 1.056e-7),          # Strang
    ("ring", 2000, 1.188e-5, 8.510e-8),          # merged
    ("ring", 2000, 1.149e-5, 1.056e-7),          # Rodrigues
    ("ring", 1000, 5.872e-6, 2.812e-8),          # merged, positivity projection every 100 steps
    ("ring_rotated", 2000, 9.670e-5, 5.603e-8),
    ("two_level", 6000, 1.560e-6, 1.444e-5),     # Strang
    ("two_level", 6000, 1.531e-6, 7.265e-6),     # merged
    ("six_level", 1000, 2.141e-6, 1.077e-6),     # merged (register and tensor cores)
    ("six_level", 1000, 2.294e-6, 9.176e-7),     # rotated
    ("six_level", 400, 1.266e-6, 5.628e-7),      # full 1048576-cell grid, first 200 cells
    ("five_level_ring", 500, 2.589e-6, 1.781e-8),
    ("five_level_ring_rotated", 500, 3.191e-5, 2.895e-7),  # tensor cores
    ("five_level_ring_rotated", 500, 3.134e-5, 2.893e-7),  # run-time compiled kernel
    ("six_level", 1000, 2.739e-6, 9.186e-7),     # rotated, tensor cores
    ("six_level", 400, 1.263e-6, 3.343e-7),      # rotated, tensor cores, full grid
    ("pstd", 1000, 9.774e-6, 1.218e-6),          # soft source
    ("pstd", 1000, 1.159e-5, 1.238e-6),          # hard source
]


def fp32_bounds(family: str, n_steps: int):
    """(E bound, population bound) after n_steps for a workload family."""
    kE, kP = FP32_KAPPA[family]
    return kE * U32 * n_steps, kP * U32 * n_steps


def fp32_within(family: str, n_steps: int, e_err: float, p_err: float) -> bool:
    bE, bP = fp32_bounds(family, n_steps)
    return e_err < bE and p_err < bP


def assert_fp32(family: str, n_steps: int, e_err: float, p_err: float):
    bE, bP = fp32_bounds(family, n_steps)
    assert e_err < bE, f"FP32 E error {e_err:.3e} above the {family} bound {bE:.3e} ({n_steps} steps)"
    assert p_err < bP, f"FP32 population error {p_err:.3e} above the {family} bound {bP:.3e} ({n_steps} steps)"

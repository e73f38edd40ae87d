"""Pins of the oracle's Maxwell part (Sec. 2, Eq. 1 on the staggered grid of Fig. 1)
and of the coupling through dP/dt (Eqs. 1a and 5).

Discrete standing waves obey the FDTD dispersion relation exactly; the
discrete field energy is conserved in vacuum; with a medium and no relaxation
the total energy (field + N_a Tr{H0 rho}) is conserved up to the second-order
error of the scheme, which pins the sign and size of the polarisation term.
"""
import math

import numpy as np
import pytest

import workloads as W
from workloads import EPS0, MU0, C0


def _vacuum(n, boundary="periodic", dx=W.DX_PAPER, dt=W.DT_PAPER, E=None, source="none", src=None):
    p = W.two_level_sit(n_cells=n, medium=(0, 0))
    return p.with_(boundary=boundary, dx=dx, dt=dt, G=None, source_kind=source, E_init=E,
                   src=src, meta={})


def test_paper_grid_values_golden():
    """The grid printed in Sec. 5.1: dx = 4.578 nm, dt = 7.635e-18 s at Courant
    number 0.5, i.e. dx = c0 dt / 0.5 to the printed digits."""
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_cases.json")))
    tl = g["two_level"]
    assert abs(C0 * tl["dt_s"] / tl["courant"] - tl["dx_m"]) < 0.5e-12
    assert abs(W.DX_PAPER - tl["dx_m"]) < 0.5e-12
    assert W.DT_PAPER == tl["dt_s"]


@pytest.mark.parametrize("m", [3, 17])
def test_standing_wave_exact_dispersion(orc, m):
    """E_i^n = cos(k x_i) cos(w n dt), H_{i+1/2}^{n+1/2} = A sin(k x_{i+1/2}) sin(w (n+1/2) dt)
    solves the discrete equations exactly when sin(w dt/2)/(c dt) = sin(k dx/2)/dx and
    A = -dt/(mu dx) sin(k dx/2) / sin(w dt/2)."""
    n = 256
    p = _vacuum(n)
    k = 2 * math.pi * m / (n * p.dx)
    c = 1 / math.sqrt(EPS0 * MU0)
    w = 2 / p.dt * math.asin(c * p.dt / p.dx * math.sin(k * p.dx / 2))
    A = -p.dt / (MU0 * p.dx) * math.sin(k * p.dx / 2) / math.sin(w * p.dt / 2)
    x = np.arange(n) * p.dx
    E0 = np.cos(k * x)
    H0 = A * np.sin(k * (x + p.dx / 2)) * math.sin(-w * p.dt / 2)
    st = orc.State(E0, H0, np.zeros((0, 2, 2)))
    steps = 1000
    out, _ = orc.run(p.with_(E_init=E0), st, n_steps=steps)
    ref = np.cos(k * x) * math.cos(w * steps * p.dt)
    assert np.abs(out.E - ref).max() < 1e-11
    refH = A * np.sin(k * (x + p.dx / 2)) * math.sin(w * (steps - 0.5) * p.dt)
    assert np.abs(out.H - refH).max() < 1e-11 * abs(A)


def test_vacuum_energy_conserved(orc):
    """sum(eps E^n^2 + mu H^{n-1/2} H^{n+1/2}) is an exact invariant of the leapfrog."""
    n = 500
    rng = np.random.default_rng(0)
    p = _vacuum(n, E=rng.normal(0, 1e3, size=n))
    st = orc.initial_state(p)
    vals = []
    for _ in range(6):
        nxt, _ = orc.run(p, st, n_steps=1)
        vals.append(EPS0 * np.sum(st.E ** 2) + MU0 * np.sum(st.H * nxt.H))
        st, _ = orc.run(p, nxt, n_steps=199)
    vals = np.array(vals)
    assert np.abs(vals - vals[0]).max() < 1e-12 * vals[0]


def test_hard_source_and_mur_absorption(orc):
    """Hard source: E at cell 0 equals the sample after each step. The first-order
    Mur condition lets a pulse leave the right end: the energy left behind is a
    small fraction of the energy that passed."""
    n = 1200
    fn = W.gauss_pulse(1.0, 3e-15, 8e-15, 2.3e15, W.DT_PAPER)
    src = fn(np.arange(12000))
    p = _vacuum(n, boundary="open", source="hard", src=src)
    st, probe = orc.run(p, n_steps=3000, probe_cell=0)
    assert np.array_equal(probe, src[:3000])
    e_mid = EPS0 * np.sum(st.E ** 2)
    st2, _ = orc.run(p, st, n_steps=5000, step0=3000)  # the pulse has left through the right end
    e_end = EPS0 * np.sum(st2.E ** 2)
    assert e_mid > 0 and e_end < 2e-4 * e_mid, (e_mid, e_end)


def _energy(p, st, nxt):
    wf = 0.5 * EPS0 * np.sum(st.E ** 2) + 0.5 * MU0 * np.sum(st.H * nxt.H)
    wm = p.N_a * 0.5 * np.sum(np.einsum("jk,ckj->c", p.H0, st.rho + nxt.rho).real)
    return wf * p.dx, wm * p.dx


@pytest.mark.parametrize("sign", [1])
def test_coupled_energy_balance_second_order(orc, sign):
    """Two-level medium filling a periodic ring, no relaxation: the continuous MLN
    system conserves sum(eps E^2/2 + mu H^2/2) + N_a Tr{H0 rho} (from Eqs. 1, 2, 5:
    d/dt N_a Tr{H0 rho} = E dP/dt). The discrete drift must be small against the
    energy exchanged with the medium and fall by 4 when dt and dx halve."""
    drifts = []
    for s in (1, 2):
        n = 400 * s
        p = W.two_level_sit(n_cells=n, medium=(0, n))
        p = p.with_(G=None, boundary="periodic", source_kind="none", dx=W.DX_PAPER / s,
                    dt=W.DT_PAPER / s, N_a=5e25)
        x = (np.arange(n) - n / 2) * p.dx
        E0 = 3e9 * np.exp(-(x / (60 * W.DX_PAPER)) ** 2) * np.cos(p.meta["omega0"] / C0 * x)
        p = p.with_(E_init=E0)
        st = orc.initial_state(p)
        ws = []
        for _ in range(12):
            nxt, _ = orc.run(p, st, n_steps=1)
            ws.append(_energy(p, st, nxt))
            st, _ = orc.run(p, nxt, n_steps=100 * s - 1)
        ws = np.array(ws)
        exchanged = np.abs(ws[:, 1] - ws[0, 1]).max()
        tot = ws.sum(1)
        drifts.append(np.abs(tot - tot[0]).max())
        assert exchanged > 0.05 * ws[0, 0]
        assert drifts[-1] < 1e-4 * exchanged
    assert 3.6 < drifts[0] / drifts[1] < 4.4, drifts

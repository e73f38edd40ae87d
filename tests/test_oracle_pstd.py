"""Pins of the oracle's pseudo-spectral (PSTD) field solver: the variant of the
Maxwell part that Secs. 1 and 3 say the method carries over to, with the
derivatives of Eq. 1 taken from the trigonometric interpolant of the periodic
samples instead of the differences of Fig. 1.

* The staggered spectral derivative is exact for every Fourier mode below the
  Nyquist frequency (closed form: the derivative of sin at the shifted points),
  on even and odd grids; the Nyquist mode has the value its interpolant gives.
* The two staggered derivatives are minus each other's transpose, which makes
  the leapfrog conserve the discrete field energy in vacuum.
* In vacuum each mode follows the leapfrog recurrence with the exact spatial
  derivative, so a cosine initial field has the closed-form solution
  E^n = [cos(n t) - tan(t/2) sin(n t)] cos(k x), sin(t/2) = c dt k / 2, which
  differs from the FDTD dispersion of Fig. 1's grid.
* With a medium and no relaxation, the total energy is conserved to second
  order, as for the FDTD solver (pins the sign of dP/dt in the PSTD update).
"""
import math

import numpy as np
import pytest

import workloads as W
from workloads import EPS0, MU0, C0


def _vacuum(n, E=None):
    p = W.two_level_sit(n_cells=n, medium=(0, 0))
    return p.with_(boundary="periodic", G=None, source_kind="none", E_init=E, src=None, meta={},
                   maxwell="pstd")


@pytest.mark.parametrize("n", [64, 45])
@pytest.mark.parametrize("half", [0.5, -0.5])
def test_spectral_derivative_exact_below_nyquist(orc, n, half):
    dx = W.DX_PAPER
    x = np.arange(n) * dx
    for m in sorted({1, 2, 7, (n - 1) // 2}):
        k = 2 * math.pi * m / (n * dx)
        d = orc.spectral_derivative(np.sin(k * x + 0.4), dx, half)
        ref = k * np.cos(k * (x + half * dx) + 0.4)
        assert np.abs(d - ref).max() < 1e-12 * k, (m, half)


def test_nyquist_mode():
    """cos(pi x / dx) sampled on an even grid: its derivative at the points
    shifted by +-dx/2 is -+(pi/dx) sin(pi (j +- 1/2)) = -+(pi/dx) (+-1)(-1)^j."""
    import oracle as orc
    n, dx = 32, W.DX_PAPER
    f = np.cos(math.pi * np.arange(n))
    sgn = (-1.0) ** np.arange(n)
    assert np.allclose(orc.spectral_derivative(f, dx, 0.5), -math.pi / dx * sgn, rtol=0, atol=1e-9 / dx)
    assert np.allclose(orc.spectral_derivative(f, dx, -0.5), math.pi / dx * sgn, rtol=0, atol=1e-9 / dx)


def test_staggered_derivatives_are_minus_transposes(orc):
    n, dx = 40, W.DX_PAPER
    eye = np.eye(n)
    Dp = np.stack([orc.spectral_derivative(eye[i], dx, 0.5) for i in range(n)], axis=1)
    Dm = np.stack([orc.spectral_derivative(eye[i], dx, -0.5) for i in range(n)], axis=1)
    assert np.abs(Dm + Dp.T).max() < 1e-12 * np.abs(Dp).max()


@pytest.mark.parametrize("m", [3, 20])
def test_vacuum_closed_form(orc, m):
    n = 64
    p = _vacuum(n)
    k = 2 * math.pi * m / (n * p.dx)
    c = 1 / math.sqrt(EPS0 * MU0)
    th = 2 * math.asin(c * p.dt * k / 2)
    x = np.arange(n) * p.dx
    p = p.with_(E_init=np.cos(k * x))
    steps = 1000
    st, _ = orc.run(p, n_steps=steps)
    ref = (math.cos(steps * th) - math.tan(th / 2) * math.sin(steps * th)) * np.cos(k * x)
    assert np.abs(st.E - ref).max() < 1e-10
    # H^{n-1/2} from H^{n+1/2} - H^{n-1/2} = (dt/mu) dE^n/dx at x + dx/2, summed
    e = lambda j: math.cos(j * th) - math.tan(th / 2) * math.sin(j * th)
    amp = sum(e(j) for j in range(steps)) * (p.dt / MU0) * k
    refH = -amp * np.sin(k * (x + p.dx / 2))
    assert np.abs(st.H - refH).max() < 1e-9 * abs(amp)


def test_pstd_dispersion_differs_from_fdtd(orc):
    """The same cosine run with the FDTD solver ends measurably elsewhere: the
    vacuum test above tells the two solvers apart."""
    n, m = 64, 20
    p = _vacuum(n)
    k = 2 * math.pi * m / (n * p.dx)
    p = p.with_(E_init=np.cos(k * np.arange(n) * p.dx))
    a, _ = orc.run(p, n_steps=1000)
    b, _ = orc.run(p.with_(maxwell="fdtd"), n_steps=1000)
    assert np.abs(a.E - b.E).max() > 0.1


def test_vacuum_energy_conserved(orc):
    n = 96
    rng = np.random.default_rng(1)
    p = _vacuum(n, E=rng.normal(0, 1e3, size=n))
    st = orc.initial_state(p)
    vals = []
    for _ in range(5):
        nxt, _ = orc.run(p, st, n_steps=1)
        vals.append(EPS0 * np.sum(st.E ** 2) + MU0 * np.sum(st.H * nxt.H))
        st, _ = orc.run(p, nxt, n_steps=99)
    vals = np.array(vals)
    assert np.abs(vals - vals[0]).max() < 1e-12 * vals[0]


def test_open_grid_refused(orc):
    p = _vacuum(32).with_(boundary="open")
    with pytest.raises(RuntimeError):
        orc.run(p, n_steps=1)


def test_coupled_energy_balance_second_order(orc):
    """Two-level medium on a PSTD ring, no relaxation: field + N_a Tr{H0 rho} is
    conserved by the continuous system; the discrete drift is small against the
    energy exchanged and falls by 4 when dt and dx halve."""
    drifts = []
    for s in (1, 2):
        n = 160 * s
        p = W.two_level_sit(n_cells=n, medium=(0, n))
        p = p.with_(G=None, boundary="periodic", source_kind="none", dx=W.DX_PAPER / s,
                    dt=W.DT_PAPER / s, N_a=5e25, maxwell="pstd")
        x = (np.arange(n) - n / 2) * p.dx
        E0 = 3e9 * np.exp(-(x / (25 * W.DX_PAPER)) ** 2) * np.cos(p.meta["omega0"] / C0 * x)
        p = p.with_(E_init=E0)
        st = orc.initial_state(p)
        ws = []
        for _ in range(10):
            nxt, _ = orc.run(p, st, n_steps=1)
            wf = 0.5 * EPS0 * np.sum(st.E ** 2) + 0.5 * MU0 * np.sum(st.H * nxt.H)
            wm = p.N_a * 0.5 * np.sum(np.einsum("jk,ckj->c", p.H0, st.rho + nxt.rho).real)
            ws.append((wf * p.dx, wm * p.dx))
            st, _ = orc.run(p, nxt, n_steps=60 * s - 1)
        ws = np.array(ws)
        exchanged = np.abs(ws[:, 1] - ws[0, 1]).max()
        tot = ws.sum(1)
        drifts.append(np.abs(tot - tot[0]).max())
        assert exchanged > 0.02 * ws[0, 0]
        assert drifts[-1] < 1e-4 * exchanged
    assert 3.5 < drifts[0] / drifts[1] < 4.5, drifts

"""Pins of the oracle's Liouville-von Neumann part (one cell, prescribed field).

Closed forms of the two- and three-level equations (Sec. 2, Eq. 2; relaxation
models of Eqs. 29 and 32), the second-order convergence of the Strang splitting
(Sec. 4.1, Eq. 23), invariants of the exact flow, and the polarisation source
(Eqs. 3-5).
"""
import math

import numpy as np
import pytest

import workloads as W
from workloads import HBAR

SX = np.array([[0, 1], [1, 0]], dtype=complex)


def _prob(H0, mu, G=None, dt=W.DT_PAPER, N_a=1e24):
    N = H0.shape[0]
    return W.Problem(name="cell", N=N, H0=np.asarray(H0, complex), mu=np.asarray(mu, complex),
                     G=G, rho0=np.eye(N, dtype=complex) / N, N_a=N_a, n_cells=3,
                     medium_begin=0, medium_end=3, dt=dt)


def test_resonant_rabi_exact(orc):
    """H0 = 0, no relaxation, constant E: the splitting is exact and
    P2(t) = sin^2(mu12 E t / hbar)."""
    mu12, E = 1e-29, 2e9
    p = _prob(np.zeros((2, 2)), mu12 * SX)
    rho = np.diag([1.0, 0.0]).astype(complex)
    n = 3000
    out, _ = orc.cell(p, rho, np.full(n, E))
    ref = math.sin(mu12 * E * n * p.dt / HBAR) ** 2
    assert abs(out[1, 1].real - ref) < 1e-12
    assert ref > 0.05  # the test is not trivial


def test_two_level_relaxation_eq29_exact(orc):
    """E = 0 with the relaxation of Eq. 29: rho22 decays with T1 and rho12 rotates
    at omega12 while decaying with T2; both exact because the field-free flow is
    applied exactly."""
    w, T1, T2 = 2.3e15, 1e-13, 0.6e-13
    H0 = HBAR * w * np.diag([-0.5, 0.5])
    p = _prob(H0, 1e-29 * SX, W.two_level_relaxation(T1, T2))
    rho0 = np.array([[0.3, 0.2 - 0.35j], [0.2 + 0.35j, 0.7]])
    n = 4000
    out, _ = orc.cell(p, rho0, np.zeros(n))
    t = n * p.dt
    tol = 2 * n * 2.5e-16  # rounding of 2n applications of the propagator
    assert abs(out[1, 1] - 0.7 * math.exp(-t / T1)) < tol
    assert abs(out[0, 0] - (1.0 - 0.7 * math.exp(-t / T1))) < tol
    r12 = rho0[0, 1] * np.exp((1j * w - 1.0 / T2) * t)
    assert abs(out[0, 1] - r12) < tol


def test_three_level_relaxation_eq32_exact(orc):
    """E = 0 with the relaxation of Eq. 32: every population relaxes to 1/3 as
    exp(-t/T1) and every coherence rho_jk rotates at (e_k - e_j)/hbar while
    decaying as exp(-t/T1)."""
    T1 = 2e-13
    lev = np.array([0.0, 9.0, 14.0]) * W.MEV
    mu = np.array([[0, 1, 1.41], [1, 0, 0], [1.41, 0, 0]]) * 1.48e-29
    p = _prob(np.diag(lev), mu, W.three_level_relaxation_sec52(T1))
    rho0 = W.random_density(np.random.default_rng(5), 3)
    n = 5000
    out, _ = orc.cell(p, rho0, np.zeros(n))
    t = n * p.dt
    f = math.exp(-t / T1)
    tol = 2 * n * 2.5e-16  # rounding of 2n applications of the propagator
    for j in range(3):
        assert abs(out[j, j] - (1 / 3 + (rho0[j, j] - 1 / 3) * f)) < tol
        for k in range(3):
            if j != k:
                ref = rho0[j, k] * np.exp((-1j * (lev[j] - lev[k]) / HBAR - 1 / T1) * t)
                assert abs(out[j, k] - ref) < tol


def test_detuned_rabi_second_order(orc):
    """Constant E with H0 = hbar w diag(-1/2, 1/2): the exact population is
    P2 = (W^2/Wg^2) sin^2(Wg t/2), W = 2 mu12 E/hbar, Wg = sqrt(w^2 + W^2). Strang
    splitting is second order: halving dt divides the error by 4."""
    w, mu12, E = 2.3e15, 1e-29, 4e10
    Om = 2 * mu12 * E / HBAR
    Og = math.hypot(w, Om)
    t_end = 30e-15
    errs = []
    for n in (800, 1600, 3200):
        dt = t_end / n
        p = _prob(HBAR * w * np.diag([-0.5, 0.5]), mu12 * SX, dt=dt)
        out, _ = orc.cell(p, np.diag([1.0, 0.0]).astype(complex), np.full(n, E))
        ref = (Om / Og) ** 2 * math.sin(Og * t_end / 2) ** 2
        errs.append(abs(out[1, 1].real - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2, (errs, r1, r2)


def test_unitary_invariants(orc):
    """No relaxation: trace, Hermiticity and the spectrum of rho are conserved."""
    rng = np.random.default_rng(11)
    for N in (2, 3, 6):
        H0 = W.random_hermitian(rng, N, 50 * W.MEV)
        mu = W.random_hermitian(rng, N, 3 * W.NM_E)
        p = _prob(H0, mu)
        rho0 = W.random_density(rng, N, rank=2)
        E = rng.normal(0, 3e9, size=500)
        out, _ = orc.cell(p, rho0, E)
        # rounding of 3 x 500 applications of N^2 x N^2 and N x N products
        assert abs(np.trace(out) - 1) < 1e-12
        assert np.abs(out - out.conj().T).max() < 1e-12
        ev0 = np.linalg.eigvalsh(rho0)
        ev1 = np.linalg.eigvalsh(0.5 * (out + out.conj().T))
        assert np.abs(ev0 - ev1).max() < 1e-12


def test_pure_dephasing_purity_nonincreasing(orc):
    """Pure dephasing is a unital relaxation (G(I) = 0): purity Tr rho^2 never
    grows, trace stays 1 and rho stays positive semidefinite."""
    rng = np.random.default_rng(12)
    N = 4
    deph = rng.uniform(1, 10, size=(N, N)) * 1e12
    deph = 0.5 * (deph + deph.T)
    G = W.lindblad_superop(N, {}, deph)
    p = _prob(W.random_hermitian(rng, N, 80 * W.MEV), W.random_hermitian(rng, N, 2 * W.NM_E), G)
    rho = W.random_density(rng, N)
    pur = [np.trace(rho @ rho).real]
    for _ in range(20):
        rho, _ = orc.cell(p, rho, rng.normal(0, 5e9, size=100))
        pur.append(np.trace(rho @ rho).real)
        assert abs(np.trace(rho) - 1) < 1e-12
        assert np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)).min() > -1e-12
    assert all(b <= a + 1e-15 for a, b in zip(pur, pur[1:]))
    assert pur[-1] < pur[0] - 1e-3


def test_amplitude_damping_reaches_ground_state(orc):
    """Downward Lindblad rates only, E = 0: rho tends to the lowest level."""
    N = 3
    lev = np.array([20.0, 0.0, 45.0]) * W.MEV
    rates = {(0, 1): 3e12, (2, 1): 1e12, (2, 0): 2e12}
    p = _prob(np.diag(lev), np.zeros((3, 3)), W.lindblad_superop(N, rates))
    rho = np.diag([0.2, 0.5, 0.3]).astype(complex)
    out, _ = orc.cell(p, rho, np.zeros(400000))  # 3 ps
    assert out[1, 1].real > 1 - 1e-3
    assert abs(np.trace(out) - 1) < 1e-10  # 8e5 propagator applications


def test_dpdt_two_level_closed_form(orc):
    """P = N_a Tr{mu rho} = 2 N_a mu12 Re rho12 and, from Eqs. 2 and 29,
    d rho12/dt = (i w - 1/T2) rho12, so dP/dt = 2 N_a mu12 Re((i w - 1/T2) rho12)."""
    w, mu12, T1, T2, Na = 2.3e15, 1e-29, 1e-12, 0.4e-12, 1e24
    p = _prob(HBAR * w * np.diag([-0.5, 0.5]), mu12 * SX, W.two_level_relaxation(T1, T2), N_a=Na)
    rng = np.random.default_rng(2)
    for _ in range(5):
        rho = W.random_density(rng, 2)
        ref = 2 * Na * mu12 * ((1j * w - 1 / T2) * rho[0, 1]).real
        got = orc.dpdt(p, rho)
        assert abs(got - ref) < 1e-13 * abs(ref)


def test_dpdt_matches_commutator_form_and_drops_interaction(orc):
    """dP/dt = N_a Tr{mu (-(i/hbar)[H0, rho] + G(rho))} (Eqs. 2-3); the
    interaction commutator contributes nothing (Eqs. 4-5)."""
    rng = np.random.default_rng(9)
    N = 3
    H0 = W.random_hermitian(rng, N, 40 * W.MEV)
    mu = W.random_hermitian(rng, N, 2 * W.NM_E)
    G = W.lindblad_superop(N, {(1, 0): 2e12, (2, 0): 1e12, (2, 1): 4e12})
    p = _prob(H0, mu, G)
    rho = W.random_density(rng, N)
    Grho = (G @ rho.reshape(-1)).reshape(N, N)
    drho = -1j / HBAR * (H0 @ rho - rho @ H0) + Grho
    ref = p.N_a * np.trace(mu @ drho).real
    got = orc.dpdt(p, rho)
    assert abs(got - ref) < 1e-13 * abs(ref)
    # adding the interaction Hamiltonian -mu E to H0 leaves dP/dt unchanged
    p2 = _prob(H0 - mu * 7e9, mu, G)
    assert abs(orc.dpdt(p2, rho) - got) < 1e-12 * abs(got)


def test_cell_dpdt_is_derivative_of_polarisation(orc):
    """With E = 0 the per-step dP/dt^{n+1/2} equals the time derivative of
    P(t) = N_a Tr{mu rho(t)} along the exact field-free flow, here checked by a
    central difference of the oracle's own states two steps apart (second-order
    accurate in dt)."""
    rng = np.random.default_rng(4)
    N = 3
    p = _prob(W.random_hermitian(rng, N, 30 * W.MEV), W.random_hermitian(rng, N, 2 * W.NM_E),
              W.lindblad_superop(N, {(1, 0): 2e12, (2, 1): 3e12}))
    rho = W.random_density(rng, N)
    r1, d1 = orc.cell(p, rho, np.zeros(1))
    r2, _ = orc.cell(p, r1, np.zeros(1))
    P0 = p.N_a * np.trace(p.mu @ rho).real
    P2 = p.N_a * np.trace(p.mu @ r2).real
    fd = (P2 - P0) / (2 * p.dt)
    assert abs(fd - d1[0]) < 1e-5 * abs(d1[0])

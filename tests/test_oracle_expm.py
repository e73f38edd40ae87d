"""Pins of the oracle's matrix exponential (scaling-and-squaring Pade(13)).

The oracle computes every exponential of the method with it: the field-free
propagator exp((L0 + G) dt/2) and the interaction exp(+i mu E dt / hbar)
(Sec. 4.1, Eqs. 21-23). It is checked against a brute-force Taylor series in
50-digit arithmetic and against closed forms; none of these share its steps.
"""
import math

import mpmath
import numpy as np
import pytest


def _taylor_mp(A, dps=50):
    """exp(A) by the plain Taylor series in mpmath, terms summed until they vanish."""
    with mpmath.workdps(dps):
        n = A.shape[0]
        M = mpmath.matrix([[mpmath.mpc(complex(A[i, j])) for j in range(n)] for i in range(n)])
        S = mpmath.eye(n)
        term = mpmath.eye(n)
        k = 0
        while True:
            k += 1
            term = term * M / k
            S = S + term
            if mpmath.mnorm(term, 1) < mpmath.mpf(10) ** (-dps + 5) and k > 5:
                break
        return np.array([[complex(S[i, j]) for j in range(n)] for i in range(n)])


@pytest.mark.parametrize("n", [2, 3, 4])
@pytest.mark.parametrize("scale", [1e-4, 0.3, 3.0])
def test_expm_vs_bruteforce_taylor(orc, n, scale):
    rng = np.random.default_rng(100 * n + int(scale * 10))
    A = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) * scale
    ref = _taylor_mp(A)
    got = orc.expm(A)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    # rounding of the squarings grows with the norm of A
    assert err < 5e-15 * max(1.0, np.abs(A).sum(0).max()), err


def test_expm_pauli_closed_form(orc):
    # exp(i t sigma_x) = cos t I + i sin t sigma_x
    sx = np.array([[0, 1], [1, 0]], dtype=complex)
    for t in [1e-9, 0.01, 0.7, 2.0, 11.0]:
        ref = math.cos(t) * np.eye(2) + 1j * math.sin(t) * sx
        got = orc.expm(1j * t * sx)
        assert np.abs(got - ref).max() < 1e-14 * max(1.0, t)


def test_expm_rotation_generator(orc):
    # exp([[0, -t], [t, 0]]) is the rotation by +t
    for t in [1e-6, 0.3, 3.0]:
        got = orc.expm(np.array([[0, -t], [t, 0]], dtype=complex))
        ref = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
        assert np.abs(got - ref).max() < 1e-15 * max(1.0, t)


def test_expm_diagonal_and_jordan(orc):
    d = np.array([0.5, -1.2 + 0.3j, 2.0j, -7.0])
    got = orc.expm(np.diag(d))
    assert np.allclose(got, np.diag(np.exp(d)), rtol=2e-14, atol=1e-15)
    a = -0.4 + 0.9j
    J = np.array([[a, 1.0], [0, a]])
    ref = np.exp(a) * np.array([[1.0, 1.0], [0, 1.0]])
    assert np.abs(orc.expm(J) - ref).max() < 1e-15


def test_expm_det_trace_and_inverse(orc):
    rng = np.random.default_rng(7)
    A = rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5))
    X = orc.expm(A)
    assert abs(np.linalg.det(X) - np.exp(np.trace(A))) < 1e-12 * abs(np.exp(np.trace(A)))
    Y = orc.expm(-A)
    assert np.abs(X @ Y - np.eye(5)).max() < 1e-12


def test_expm_of_antihermitian_is_unitary(orc):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6))
    H = X + X.conj().T
    V = orc.expm(1j * 0.37 * H)
    assert np.abs(V @ V.conj().T - np.eye(6)).max() < 1e-14

"""The relaxation models of the workloads and positivity of rho.

The six-level workload uses pure dephasing with an independent rate for
every pair of levels (G(rho)_jk = -gamma_jk rho_jk). Such a map is not
completely positive in general: started from the ground state of its random
H0 (which has coherences in the basis where the dephasing acts), the exact
field-free flow exp(L t) leaves the positive semidefinite cone for a while.
Checked here with scipy's matrix exponential of the Liouvillian (Eq. 2)
and with the oracle, which follows the same exact flow when E = 0. The
three-level workload's Lindblad relaxation keeps rho >= 0.

So negative eigenvalues of the six-level state are the model's, not rounding:
the positivity projection is optional and off by default.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import workloads as W


def liouvillian(p):
    N = p.N
    I = np.eye(N)
    return -1j / W.HBAR * (np.kron(p.H0, I) - np.kron(I, p.H0.T)) + p.G


def min_eig(r):
    return float(np.linalg.eigvalsh((r + r.conj().T) / 2)[0])


def test_six_level_dephasing_leaves_the_positive_cone(orc):
    # N_a = 0 decouples the medium from the field, so E stays zero
    p = W.six_level_pulse(n_cells=8, n_steps=0).with_(source_kind="none", N_a=0.0)
    L = liouvillian(p)
    steps = 1310  # 10 fs
    t = steps * p.dt
    exact = (sl.expm(L * t) @ p.rho0.reshape(-1)).reshape(p.N, p.N)
    assert min_eig(exact) < -1e-3
    assert abs(np.trace(exact) - 1) < 1e-13
    st, _ = orc.run(p, n_steps=steps)
    # E stays zero (no source, no field, no polarisation): every cell follows exp(L t) rho0
    assert np.abs(st.E).max() == 0.0
    assert np.abs(st.rho[3] - exact).max() < 1e-10
    assert abs(min_eig(st.rho[3]) - min_eig(exact)) < 1e-10


def test_three_level_lindblad_keeps_rho_positive():
    p = W.three_level_ring(n_cells=8)
    L = liouvillian(p)
    for t in (1e-14, 1e-13, 1e-12, 1e-11):
        r = (sl.expm(L * t) @ p.rho0.reshape(-1)).reshape(p.N, p.N)
        assert min_eig(r) > 0

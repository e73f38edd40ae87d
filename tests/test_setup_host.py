"""Host-side set-up of the CUDA path (no GPU needed), through the C-ABI.

Checks the generators (Sec. 3, Eq. 7 and the Pauli / Gell-Mann statement),
the properties of U proven in Sec. 4.2 (real, antisymmetric, purely imaginary
eigenvalues in conjugate pairs), the real eigenbasis T (Eq. 26) against a
brute-force matrix exponential and against the generalised Rodrigues formula
(Eq. 27), the affine field-free propagator (Eqs. 19-21) against the rho-space
flow, the polarisation coefficients (Eq. 17) against the oracle, and input
validation.
"""
import json
import os
import re

import numpy as np
import pytest
import scipy.linalg as sl

import workloads as W
from workloads import HBAR

mln = pytest.importorskip("paper_1710_09799_gb300.mln")


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09799_gb300 import build
    build()
    return mln.lib()


def params_of(p, **kw):
    args = dict(N=p.N, H0=p.H0, mu=p.mu, G=p.G, rho0=p.rho0, N_a=p.N_a, n_cells=p.n_cells,
                medium_begin=p.medium_begin, medium_end=p.medium_end, dx=p.dx, dt=p.dt,
                eps_r=p.eps_r, mu_r=p.mu_r, sigma=p.sigma, boundary=p.boundary,
                source_kind=p.source_kind, source_cell=p.source_cell, maxwell=p.maxwell)
    args.update(kw)
    return mln.Params(**args)


def random_problem(N, seed, G=True):
    rng = np.random.default_rng(seed)
    H0 = W.random_hermitian(rng, N, 40 * W.MEV)
    mu = W.random_hermitian(rng, N, 2 * W.NM_E)
    Gm = None
    if G:
        rates = {(b, a): rng.uniform(0.5, 5) * 1e12 for a in range(N) for b in range(a + 1, N)}
        deph = rng.uniform(1, 3, size=(N, N)) * 1e12
        Gm = W.lindblad_superop(N, rates, 0.5 * (deph + deph.T))
    return W.Problem(name="rand", N=N, H0=H0, mu=mu, G=Gm, rho0=W.random_density(rng, N), N_a=1e24,
                     n_cells=64, medium_begin=0, medium_end=64)


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "mln.h")).read()
    names = set(re.findall(r"\b(mln_[a-z0-9_]+)\s*\(", hdr))
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(mln._SIGS) == names


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_generators(lib, N):
    s = mln.mln_setup_host(params_of(random_problem(N, N)))
    g = s["gen"]
    D = N * N - 1
    assert g.shape == (D, N, N)
    for j in range(D):
        assert abs(np.trace(g[j])) < 1e-15
        assert np.abs(g[j] - g[j].conj().T).max() < 1e-15
        for k in range(D):
            assert abs(np.trace(g[j] @ g[k]) - 2.0 * (j == k)) < 1e-14


def test_pauli_and_gell_mann_golden(lib):
    """Sec. 3: for N = 2 and N = 3 the generators are the Pauli and the Gell-Mann
    matrices (each generator equals one of them up to sign)."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "su_generators.json")))
    for N, key in ((2, "pauli"), (3, "gell_mann")):
        ref = [np.array(m["re"]) + 1j * np.array(m["im"]) for m in gold[key]]
        g = mln.mln_setup_host(params_of(random_problem(N, 1)))["gen"]
        used = set()
        for j in range(len(g)):
            hit = [i for i, r in enumerate(ref) if np.abs(g[j] - r).max() < 1e-15 or np.abs(g[j] + r).max() < 1e-15]
            assert len(hit) == 1, (N, j)
            used.add(hit[0])
        assert len(used) == len(ref)


@pytest.mark.parametrize("N", [2, 3, 5, 6])
def test_U_real_antisymmetric_with_paired_spectrum(lib, N):
    """Sec. 4.2: u_jk is real and antisymmetric; its eigenvalues are purely
    imaginary in conjugate pairs, here +-i (m_a - m_b)/hbar for the eigenvalues
    m_a of mu, plus N - 1 zeros."""
    p = random_problem(N, 10 + N)
    s = mln.mln_setup_host(params_of(p))
    U = s["U"]
    assert np.abs(U + U.T).max() <= 1e-14 * np.abs(U).max()
    ev = np.linalg.eigvals(U)
    assert np.abs(ev.real).max() < 1e-9 * np.abs(ev).max()
    m = np.linalg.eigvalsh(p.mu)
    want = sorted([abs(m[a] - m[b]) / HBAR for a in range(N) for b in range(a + 1, N)] * 2 + [0.0] * (N - 1))
    got = sorted(np.abs(ev.imag))
    assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * max(want))
    # without relaxation M is antisymmetric too
    s0 = mln.mln_setup_host(params_of(p, G=None))
    assert np.abs(s0["M"] + s0["M"].T).max() <= 1e-14 * np.abs(s0["M"]).max()


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_diag_method_equals_bruteforce_and_rodrigues(lib, N):
    """exp(U E dt) three ways (the paper's pade = diag = rodr agreement, Sec. 5):
    scipy's expm of U E dt; T R(theta E dt) T^T with the rotation used by the
    kernels; and the generalised Rodrigues formula I + sum sin(a_i) S_i +
    (1 - cos a_i) S_i^2 with S_i = T Theta_i T^T (Eq. 27), a_i = -theta_i E dt
    in the orientation of this T."""
    p = random_problem(N, 20 + N)
    s = mln.mln_setup_host(params_of(p))
    U, T, th, D, q = s["U"], s["T"], s["theta"], s["D"], s["q"]
    for E in (3e7, -8e9, 2.5e11):
        x = E * p.dt
        ref = sl.expm(U * x)
        R = np.eye(D)
        for k in range(q):
            c, sn = np.cos(th[k] * x), np.sin(th[k] * x)
            R[2 * k:2 * k + 2, 2 * k:2 * k + 2] = [[c, sn], [-sn, c]]
        diag = T @ R @ T.T
        rod = np.eye(D)
        for k in range(q):
            Th = np.zeros((D, D))
            Th[2 * k, 2 * k + 1], Th[2 * k + 1, 2 * k] = -1.0, 1.0
            S = T @ Th @ T.T
            a = -th[k] * x
            rod += np.sin(a) * S + (1 - np.cos(a)) * (S @ S)
        assert np.abs(diag - ref).max() < 1e-13
        assert np.abs(rod - ref).max() < 1e-13


@pytest.mark.parametrize("N", [2, 3, 4])
def test_field_free_adjoint_flow_matches_rho_space(lib, N):
    """d(t) = A0 d + b over dt/2 (affine solution of Eq. 19, augmented form)
    must equal the adjoint vector of exp((L0 + G) dt/2) rho, the flow of Eq. 2
    with E = 0, built here with scipy on the superoperator."""
    p = random_problem(N, 30 + N).with_(dt=2e-15, dx=W.C0 * 2e-15 / 0.5)
    s = mln.mln_setup_host(params_of(p))
    g = s["gen"]
    L = (-1j / HBAR) * (np.kron(p.H0, np.eye(N)) - np.kron(np.eye(N), p.H0.T)) + p.G
    Prop = sl.expm(L * p.dt / 2)
    rho = p.rho0
    d = np.array([np.trace(rho @ gj).real for gj in g])
    assert np.abs(d - s["d0"]).max() < 1e-15
    rho_t = (Prop @ rho.reshape(-1)).reshape(N, N)
    d_t = np.array([np.trace(rho_t @ gj).real for gj in g])
    got = s["A0"] @ d + s["b"]
    assert np.abs(got - d_t).max() < 1e-13
    # rho = I/N + 1/2 sum d_j s_j (Eq. 6)
    back = np.eye(N) / N + 0.5 * np.einsum("j,jab->ab", d_t, g)
    assert np.abs(back - rho_t).max() < 1e-14


@pytest.mark.parametrize("N", [2, 3, 6])
def test_polarisation_coefficients_match_oracle(lib, orc, N):
    """w . d + c = N_a/2 v^T (M d + d_eq) (Eq. 17) equals the oracle's
    N_a Tr{mu (L0 + G)(rho)} (Eqs. 3, 5) on random density matrices."""
    p = random_problem(N, 40 + N)
    s = mln.mln_setup_host(params_of(p))
    rng = np.random.default_rng(1)
    for _ in range(4):
        rho = W.random_density(rng, N)
        d = np.array([np.trace(rho @ gj).real for gj in s["gen"]])
        got = s["w"] @ d + s["c"]
        ref = orc.dpdt(p, rho)
        assert abs(got - ref) < 1e-12 * abs(ref)


def test_merged_form_constants(lib):
    """C1 = A0^2 - I: the two half-steps of Eq. 23 that meet between steps."""
    p = random_problem(3, 50)
    s = mln.mln_setup_host(params_of(p))
    assert np.abs(s["C1"] - (s["A0"] @ s["A0"] - np.eye(s["D"]))).max() < 1e-15


def _status_of(fn):
    try:
        fn()
    except mln.MLNError as e:
        return e.status
    return mln.MLN_OK


def test_validation(lib):
    p = W.two_level_sit(n_cells=100, medium=(20, 80))
    ok = lambda **kw: _status_of(lambda: mln.mln_query_buffers(params_of(p, **kw)))
    assert ok() == mln.MLN_OK
    bad = p.H0.copy()
    bad[0, 1] = 1e-22
    assert ok(H0=bad) == mln.MLN_EINVAL
    assert ok(rho0=np.diag([1.0, 1.0])) == mln.MLN_EINVAL
    assert ok(rho0=np.diag([1.5, -0.5])) == mln.MLN_EINVAL
    G = p.G.copy()
    G[0, 0] += 1e12
    assert ok(G=G) == mln.MLN_EINVAL
    assert ok(dt=p.dt * 2.5) == mln.MLN_EINVAL          # Courant number above 1
    assert ok(medium_end=100) == mln.MLN_EINVAL          # the Mur cell must be vacuum
    assert ok(medium_begin=50, medium_end=40) == mln.MLN_EINVAL
    assert ok(source_cell=100) == mln.MLN_EINVAL
    assert ok(precision=7) == mln.MLN_EINVAL
    assert ok(block_steps=65) == mln.MLN_EINVAL
    # the pseudo-spectral field solver: periodic grids of 2^k cells, no JIT or tensor-core cell model
    r = W.three_level_ring(n_cells=256, n_steps=1).with_(maxwell="pstd")
    okr = lambda **kw: _status_of(lambda: mln.mln_query_buffers(params_of(r, **kw)))
    assert okr() == mln.MLN_OK and okr(form="merged", kernel="sparse") == mln.MLN_OK
    assert okr(n_cells=255, medium_end=255) == mln.MLN_EINVAL
    assert okr(n_cells=8, medium_end=8) == mln.MLN_EINVAL
    assert okr(kernel="jit", form="merged") == mln.MLN_EINVAL
    assert okr(kernel="tensor", form="merged", precision="fp32") == mln.MLN_EINVAL
    assert ok(maxwell="pstd") == mln.MLN_EINVAL                   # open grid
    # the rotated form: the run-time compiled kernel with the FDTD field solver only
    assert ok(form="rotated") == mln.MLN_OK and ok(form="rotated", kernel="jit") == mln.MLN_OK
    for k in ("register", "sparse", "tensor"):
        assert ok(form="rotated", kernel=k) == mln.MLN_EINVAL
    assert okr(form="rotated") == mln.MLN_EINVAL
    assert ok(form=4) == mln.MLN_EINVAL
    assert ok(maxwell=2) == mln.MLN_EINVAL
    q = random_problem(7, 1, G=False)
    assert _status_of(lambda: mln.mln_query_buffers(params_of(q))) == mln.MLN_EUNSUPPORTED
    sb, fb = mln.mln_query_buffers(params_of(p, precision="fp32"))
    assert fb == 100 * 4 and sb == 3 * 64 * 4
    sb, fb = mln.mln_query_buffers(params_of(p))
    assert fb == 100 * 8 and sb == 3 * 64 * 8

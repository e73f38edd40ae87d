"""Positivity projection (mln_project_positive): cells whose rho has a negative
eigenvalue (below the rounding threshold -16 N u) get the nearest positive
semidefinite unit-trace matrix (Frobenius norm), the others keep their state
bit for bit.

Checked against numpy: eigh, Euclidean projection of the eigenvalues onto the
probability simplex (sort and threshold), reassembly; the generator basis
for d_j = Tr(rho s_j) comes from the library's host set-up (mln_setup_host).
"""
import numpy as np
import pytest

import workloads as W
from helpers import assert_fp32, make_solver, params_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


def simplex(v):
    u = np.sort(v)[::-1]
    css = np.cumsum(u)
    k = np.arange(1, len(v) + 1)
    ok = u - (css - 1) / k > 0
    r = k[ok][-1]
    theta = (css[r - 1] - 1) / r
    return np.maximum(v - theta, 0.0)


def nearest_state(rho):
    w, V = np.linalg.eigh(rho)
    return (V * simplex(w)) @ V.conj().T


def problem(N):
    if N == 2:
        return W.two_level_sit(n_cells=200, medium=(50, 150), n_steps=10)
    if N == 3:
        return W.three_level_ring(n_cells=256)
    return W.six_level_pulse(n_cells=128, n_steps=10)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [2, 3, 6])
def test_projection_against_numpy(N, precision):
    from paper_1710_09799_gb300 import mln
    p = problem(N)
    s = make_solver(p, precision, "merged")
    gen = mln.mln_setup_host(params_of(p, precision=precision, form="merged"))["gen"]
    rng = np.random.default_rng(N)
    nm = p.n_medium
    rho = np.repeat(p.rho0[None], nm, axis=0).astype(np.complex128)
    bad = rng.choice(nm, size=nm // 4, replace=False)
    for c in bad:
        X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
        X = X + X.conj().T
        X -= np.trace(X) / N * np.eye(N)
        w = np.linalg.eigvalsh(rho[c])
        # push the smallest eigenvalue below zero by a few 1e-3
        for eps in np.linspace(0.01, 2.0, 400):
            if np.linalg.eigvalsh(rho[c] + eps * X / np.abs(X).max())[0] < -3e-3:
                break
        rho[c] = rho[c] + eps * X / np.abs(X).max()
    d = np.einsum("cab,jba->cj", rho, gen).real
    s.load(d)
    before = s.save()[0]
    n = s.project_positive()
    after = s.save()[0]
    assert n == len(bad)
    good = np.setdiff1d(np.arange(nm), bad)
    assert np.array_equal(before.reshape(nm, -1)[good], after.reshape(nm, -1)[good])
    out = s.rho()
    tol = 1e-12 if precision == "fp64" else 3e-6
    for c in bad:
        ref = nearest_state(rho[c])
        assert np.abs(out[c] - ref).max() < tol, (c, np.abs(out[c] - ref).max())
        assert np.linalg.eigvalsh(out[c])[0] > -tol and abs(np.trace(out[c]) - 1) < tol
    # the projected states have zero eigenvalues: rounding leaves them within
    # the threshold, so a second projection changes nothing
    assert s.project_positive() == 0
    s.close()


def test_projection_leaves_physical_states_alone():
    p = W.three_level_ring(n_cells=512, n_steps=200)
    s = make_solver(p, "fp64", "merged")
    s.step(200)
    s.sync()
    before = s.save()
    assert s.project_positive() == 0
    after = s.save()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    s.close()


def test_fp32_run_with_periodic_projection(orc):
    """FP32 three-level ring (Lindblad relaxation: the exact flow keeps rho >= 0)
    with the projection every 100 steps: the error against the FP64 oracle
    stays within the FP32 tolerance. (The six-level workload's independent
    pure-dephasing rates leave the positive cone in the exact flow; see
    test_model_positivity.py; projecting there would change the model.)"""
    p = W.three_level_ring(n_cells=4096, n_steps=1000)
    st, _ = orc.run(p, n_steps=p.n_steps)
    s = make_solver(p, "fp32", "merged")
    projected = 0
    for k in range(0, p.n_steps, 100):
        s.step(100)
        projected += s.project_positive()
    s.sync()
    E, _ = s.fields()
    rho = s.rho()
    e_err = float(np.abs(E - st.E).max() / np.abs(st.E).max())
    p_err = float(np.abs(np.einsum("cii->ci", rho - st.rho).real).max())
    print(f"fp32 three-level ring with projection every 100 steps: {projected} cell projections, "
          f"E rel {e_err:.3e}, pop abs {p_err:.3e}")
    assert_fp32("ring", p.n_steps, e_err, p_err)
    s.close()

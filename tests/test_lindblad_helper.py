"""mln_lindblad_superop: the relaxation superoperator of Lindblad decay and
pure dephasing (the linear relaxation term of Eq. 2 in the form mln_params
takes), host-only, no GPU.

Pinned by the paper's two-level relaxation (Sec. 5.1, Eq. 29: population
decay 1/T1, coherence decay 1/T2), by the classical rate (Pauli master)
equation its populations must follow, by trace and Hermiticity preservation
for random inputs, and by the superoperator assembled column by column from
the dissipator map (the workload generator's construction).
"""
import numpy as np
import pytest

import workloads as W

mln = pytest.importorskip("paper_1710_09799_gb300.mln")


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09799_gb300 import build
    build()
    return mln.lib()


def apply(G, rho):
    N = rho.shape[0]
    return (G @ rho.reshape(-1)).reshape(N, N)


def test_two_level_relaxation_of_sec51(lib):
    """Decay 1 -> 0 at 1/T1 plus dephasing 1/T2 - 1/(2 T1) is Eq. 29."""
    T1, T2 = 1e-12, 0.4e-12
    rates = np.zeros((2, 2))
    rates[1, 0] = 1.0 / T1
    deph = np.zeros((2, 2))
    deph[0, 1] = deph[1, 0] = 1.0 / T2 - 0.5 / T1
    G = mln.mln_lindblad_superop(2, rates, deph)
    ref = W.two_level_relaxation(T1, T2)
    assert np.abs(G - ref).max() <= 1e-15 * np.abs(ref).max()


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_populations_follow_the_rate_equation(lib, N):
    rng = np.random.default_rng(N)
    rates = rng.uniform(0.1, 5.0, size=(N, N)) * 1e12
    np.fill_diagonal(rates, 0.0)
    G = mln.mln_lindblad_superop(N, rates, None)
    p = rng.dirichlet(np.ones(N))
    out = apply(G, np.diag(p).astype(np.complex128))
    # d p_a / dt = sum_b gamma_{b->a} p_b - p_a sum_b gamma_{a->b}
    expect = rates.T @ p - p * rates.sum(axis=1)
    assert np.abs(np.diag(out) - expect).max() <= 1e-14 * np.abs(expect).max()
    assert np.abs(out - np.diag(np.diag(out))).max() == 0.0
    # a coherence rho_jk decays at (out-rate of j + out-rate of k) / 2
    j, k = 0, N - 1
    E = np.zeros((N, N), dtype=np.complex128)
    E[j, k] = 1.0
    got = apply(G, E)[j, k].real
    assert abs(got + 0.5 * (rates[j].sum() + rates[k].sum())) <= 1e-14 * rates.sum()


@pytest.mark.parametrize("N", [2, 3, 5, 6])
def test_matches_dissipator_map_and_preserves_trace_and_hermiticity(lib, N):
    rng = np.random.default_rng(10 + N)
    rates = rng.uniform(0.0, 3.0, size=(N, N)) * 1e12
    deph = rng.uniform(0.0, 2.0, size=(N, N)) * 1e12
    deph = np.triu(deph, 1) + np.triu(deph, 1).T
    G = mln.mln_lindblad_superop(N, rates, deph)
    ref = W.lindblad_superop(N, {(b, a): rates[b, a] for b in range(N) for a in range(N)}, deph)
    assert np.abs(G - ref).max() <= 1e-14 * np.abs(ref).max()
    for s in range(3):
        rho = W.random_density(np.random.default_rng(100 + s), N)
        out = apply(G, rho)
        assert abs(np.trace(out)) <= 1e-14 * np.abs(out).max()
        assert np.abs(out - out.conj().T).max() <= 1e-14 * np.abs(out).max()


def test_dephasing_only_and_empty(lib):
    N = 3
    deph = np.array([[7.0, 1.0, 2.0], [1.0, 9.0, 3.0], [2.0, 3.0, 5.0]]) * 1e12
    G = mln.mln_lindblad_superop(N, None, deph)
    for j in range(N):
        for k in range(N):
            E = np.zeros((N, N), dtype=np.complex128)
            E[j, k] = 1.0
            want = np.zeros((N, N), dtype=np.complex128)
            if j != k:
                want[j, k] = -deph[j, k]  # the diagonal of the dephasing matrix is not read
            assert np.array_equal(apply(G, E), want)
    assert np.array_equal(mln.mln_lindblad_superop(N, None, None), np.zeros((N * N, N * N), dtype=np.complex128))


def test_result_is_accepted_by_the_setup(lib):
    p = W.three_level_ring(n_cells=64)
    rates = np.zeros((3, 3))
    rates[2, 1], rates[1, 0], rates[2, 0] = 2e12, 1e12, 0.5e12
    G = mln.mln_lindblad_superop(3, rates, None)
    s = mln.mln_setup_host(mln.Params(N=3, H0=p.H0, mu=p.mu, G=G, rho0=p.rho0, N_a=p.N_a,
                                      n_cells=p.n_cells, medium_begin=0, medium_end=p.n_cells,
                                      dx=p.dx, dt=p.dt))
    assert np.all(np.isfinite(s["A0"]))


@pytest.mark.parametrize("case", ["N", "negative", "nan", "asymmetric", "null"])
def test_invalid_inputs(lib, case):
    N = 3
    rates = np.ones((N, N)) * 1e12
    deph = np.ones((N, N)) * 1e12
    if case == "N":
        with pytest.raises(mln.MLNError, match="N out of range"):
            mln.mln_lindblad_superop(1, None, None)
        with pytest.raises(mln.MLNError, match="N out of range"):
            mln.mln_lindblad_superop(mln.MLN_MAX_N + 1, None, None)
        return
    if case == "negative":
        rates[0, 2] = -1.0
    if case == "nan":
        deph[0, 1] = deph[1, 0] = np.nan
    if case == "asymmetric":
        deph[0, 1] = 2e12
    if case == "null":
        st = lib.mln_lindblad_superop(N, None, None, None)
        assert st == mln.MLN_EINVAL
        return
    with pytest.raises(mln.MLNError) as e:
        mln.mln_lindblad_superop(N, rates, deph)
    assert e.value.status == mln.MLN_EINVAL

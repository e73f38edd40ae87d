"""mln_adjoint for N = 4 (D = 15, 16 lanes a cell in the reverse sweep): the
largest N it takes, with the kernels' shapes for that N (FP64: 4 steps a
launch in 512-thread blocks; FP32: 12 steps in blocks of up to 640 threads).

A four-level ring with a soft source at cell 0 (a Gaussian-envelope carrier at
the mean transition frequency), the probe 32 cells downstream:
* J against the oracle's J;
* the directional derivative along seeded source directions and one real
  dipole element against central differences of J;
* FP32 against FP64;
* the two schedules (all segments recorded at once, replayed from a graph;
  two segments at a time) give the same bits.
"""
import numpy as np
import pytest

import workloads as W
from helpers import params_of

pytestmark = pytest.mark.gpu

HBAR = 1.054571817e-34


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


def four_level(n_cells=256, n_steps=300, n_src=64, amplitude=3e7):
    p = W.multi_level_ring(4, n_cells=n_cells, n_steps=n_steps, seed=31, N_a=1e26)
    lev = np.real(np.diag(p.H0))
    omega = float(np.mean([abs(lev[a] - lev[b]) for a in range(4) for b in range(a + 1, 4)])) / HBAR
    k = np.arange(n_steps, dtype=np.float64)
    src = np.zeros(n_steps)
    env = np.exp(-((k[:n_src] - n_src / 2) / (n_src / 5)) ** 2)
    src[:n_src] = amplitude * env * np.sin(omega * (k[:n_src] + 1) * p.dt)
    q = p.with_(source_kind="soft", source_cell=0, src=src, name="four_level_ring_source")
    q.meta = dict(probe_cell=32, n_src=n_src)
    return q


def J_and_grads(p, src, precision="fp64", every=32, mu=None, memory=0):
    import torch
    from paper_1710_09799_gb300 import mln
    q = p.with_(mu=p.mu if mu is None else mu)
    s = mln.Solver(params_of(q, precision=precision, form="strang"), E0=q.e_init())
    mln.mln_set_adjoint_memory(s.ctx, memory)
    t = torch.as_tensor(src, dtype=torch.float64, device="cuda")
    out = mln.mln_adjoint(s.ctx, q.N, len(src), t.data_ptr(), p.meta["probe_cell"], every)
    s.close()
    return out


@pytest.fixture(scope="module")
def base():
    p = four_level()
    src = p.source_samples(0, p.n_steps)
    return p, src, J_and_grads(p, src)


def test_objective_matches_oracle(orc, base):
    p, src, (J, _, _, _) = base
    _, probe = orc.run(p, n_steps=p.n_steps, probe_cell=p.meta["probe_cell"])
    Jo = p.dt * np.sum(probe ** 2)
    assert Jo > 0 and abs(J - Jo) < 1e-10 * Jo, (J, Jo)


def test_source_and_dipole_gradients_vs_finite_differences(base):
    from paper_1710_09799_gb300 import mln
    p, src, (J, dsrc, dmu, _) = base
    rng = np.random.default_rng(5)
    n_src = p.meta["n_src"]
    for _ in range(3):
        d = np.zeros(p.n_steps)
        d[:n_src] = rng.normal(size=n_src)
        h = 1e-6 * np.abs(src).max()
        fd = (J_and_grads(p, src + h * d, every=10 ** 6)[0] - J_and_grads(p, src - h * d, every=10 ** 6)[0]) / (2 * h)
        ad = float(dsrc @ d)
        assert abs(fd - ad) < 1e-5 * max(abs(ad), 1e-300), (fd, ad)
    x0 = mln.mu_to_params(p.mu)
    i = p.N  # Re mu_01
    h = 1e-6 * abs(x0[i])
    xp, xm = x0.copy(), x0.copy()
    xp[i] += h
    xm[i] -= h
    Jp = J_and_grads(p, src, every=10 ** 6, mu=mln.mu_from_params(p.N, xp).numpy())[0]
    Jm = J_and_grads(p, src, every=10 ** 6, mu=mln.mu_from_params(p.N, xm).numpy())[0]
    fd = (Jp - Jm) / (2 * h)
    assert abs(fd - dmu[i]) < 1e-4 * abs(dmu[i]), (fd, dmu[i])


def test_fp32_close_to_fp64(base):
    p, src, (J, dsrc, dmu, _) = base
    J3, dsrc3, dmu3, _ = J_and_grads(p, src, precision="fp32")
    assert abs(J3 - J) < 1e-3 * J
    assert np.abs(dsrc3 - dsrc).max() < 1e-2 * np.abs(dsrc).max()
    assert abs(dmu3[p.N] - dmu[p.N]) < 1e-2 * abs(dmu[p.N])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_schedules_give_the_same_bits(base, precision):
    p, src, _ = base
    a = J_and_grads(p, src, precision=precision, every=48)
    b = J_and_grads(p, src, precision=precision, every=48, memory=1)
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)

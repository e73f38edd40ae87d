"""Adjoint gradients on open grids and for contexts of the merged form.

* An open grid in the shape of the paper's two-level case (Sec. 5.1, Eqs.
  28-30): hard source at cell 0 (held cell otherwise), first-order Mur at the
  right end, the medium in the middle. The probe sits next to the Mur cell and
  the pulse crosses the grid within the run, so the reverse of the source, of
  the held cell and of the Mur rule all carry the gradient. Checked against
  central finite differences of J computed by the forward kernels (source
  samples, the dipole element, the relaxation strength), J against the
  oracle's J, and one finite difference through the oracle.
* A soft source on an open grid (the source cell's field passes through).
* Merged-form contexts (sparse, register and run-time compiled cell models): the
  forward pass runs the merged step, the backward pass recomputes in the
  Strang form from checkpoints mapped to d; J and the gradients equal those of
  a Strang-form context up to rounding.
"""
import numpy as np
import pytest

import workloads as W
from helpers import params_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


def open_grid(kind="hard", n_cells=240, n_steps=600, probe=None, T=1e-12, N_a=1e24):
    """Two-level grid, medium [60, 180), Mur at the right; the source carries a
    Gaussian-envelope carrier (period ~40 steps) over its first 200 steps."""
    p = W.two_level_sit(n_cells=n_cells, medium=(60, 180), n_steps=n_steps, T1=T, T2=T, N_a=N_a)
    k = np.arange(n_steps, dtype=np.float64)
    src = np.zeros(n_steps)
    src[:200] = 3e8 * np.exp(-((k[:200] - 100) / 35) ** 2) * np.sin(2 * np.pi * k[:200] / 40)
    q = p.with_(source_kind=kind, source_cell=0, src=src, name="open_two_level")
    # meta without the generator's source_fn: the samples above drive the grid
    q.meta = dict(probe_cell=n_cells - 2 if probe is None else probe, n_src=200)
    return q


def J_and_grads(p, src, precision="fp64", form="strang", every=64, mu=None, G=None, kernel="auto"):
    import torch
    from paper_1710_09799_gb300 import mln
    q = p.with_(mu=p.mu if mu is None else mu, G=p.G if G is None else G)
    s = mln.Solver(params_of(q, precision=precision, form=form, kernel=kernel), E0=q.e_init())
    t = torch.as_tensor(src, dtype=torch.float64, device="cuda")
    out = mln.mln_adjoint(s.ctx, q.N, len(src), t.data_ptr(), p.meta["probe_cell"], every)
    s.close()
    return out


def J_only(p, src, **kw):
    return J_and_grads(p, src, every=10 ** 6, **kw)[0]


@pytest.fixture(scope="module")
def hard():
    p = open_grid("hard")
    src = p.source_samples(0, p.n_steps)
    return p, src, J_and_grads(p, src)


def test_open_grid_objective_matches_oracle(orc, hard):
    p, src, (J, _, _, _) = hard
    _, probe = orc.run(p, n_steps=p.n_steps, probe_cell=p.meta["probe_cell"])
    Jo = p.dt * np.sum(probe ** 2)
    assert Jo > 0 and abs(J - Jo) < 1e-10 * Jo, (J, Jo)


def test_open_grid_source_gradient(hard):
    """Hard source: dJ/d(sample k) along seeded directions; the probe next to
    the Mur cell sees the pulse only through the held cell, the medium and
    the Mur rule."""
    p, src, (J, dsrc, _, _) = hard
    # a hard source sets E_0 at every step, so the later (zero) samples matter too, weakly
    assert np.abs(dsrc[:200]).max() > 1e3 * np.abs(dsrc[200:]).max() > 0
    rng = np.random.default_rng(1)
    h = 1e-6 * np.abs(src).max()
    for _ in range(3):
        d = np.zeros_like(src)
        d[:200] = rng.normal(size=200)
        fd = (J_only(p, src + h * d) - J_only(p, src - h * d)) / (2 * h)
        ad = dsrc @ d
        assert abs(fd - ad) < 1e-6 * abs(ad) + 1e-9 * np.abs(dsrc).sum() * h, (fd, ad)


def test_open_grid_probe_on_the_mur_cell():
    p = open_grid("hard", probe=239)
    src = p.source_samples(0, p.n_steps)
    J, dsrc, _, _ = J_and_grads(p, src)
    rng = np.random.default_rng(2)
    d = np.zeros_like(src)
    d[:200] = rng.normal(size=200)
    h = 1e-6 * np.abs(src).max()
    fd = (J_only(p, src + h * d) - J_only(p, src - h * d)) / (2 * h)
    assert J > 0 and abs(fd - dsrc @ d) < 1e-6 * abs(dsrc @ d), (fd, dsrc @ d)


def test_open_grid_dipole_and_relaxation_gradients(orc):
    """Strong relaxation (T1 = T2 = 20 fs) and a dense medium (N_a = 1e27 m^-3:
    its polarisation changes the probe field by ~1e-3 instead of ~1e-6), so
    that the effects of the rate and of the dipole element on J are resolved
    by central differences well above J's rounding."""
    from paper_1710_09799_gb300 import mln
    p = open_grid("hard", T=2e-14, N_a=1e27)
    src = p.source_samples(0, p.n_steps)
    J, _, dmu, dG = J_and_grads(p, src)
    x0 = mln.mu_to_params(p.mu)
    i = p.N  # Re mu_12
    h = 1e-5 * abs(x0[i])
    xp, xm = x0.copy(), x0.copy()
    xp[i] += h
    xm[i] -= h
    fd = (J_only(p, src, mu=mln.mu_from_params(p.N, xp).numpy()) -
          J_only(p, src, mu=mln.mu_from_params(p.N, xm).numpy())) / (2 * h)
    assert abs(fd - dmu[i]) < 1e-5 * abs(dmu[i]), (fd, dmu[i])
    # relaxation strength s: G(s) = s G0, dJ/ds = Re sum conj(Gamma) G0
    G0 = p.G
    g_s = float(np.real(np.sum(np.conj(dG) * G0)))
    hs = 1e-4
    fd_s = (J_only(p, src, G=G0 * (1 + hs)) - J_only(p, src, G=G0 * (1 - hs))) / (2 * hs)
    assert abs(fd_s - g_s) < 1e-5 * abs(g_s), (fd_s, g_s)
    # through the oracle: the same strength derivative from the oracle's J
    def J_orc(G):
        _, probe = orc.run(p.with_(G=G), n_steps=p.n_steps, probe_cell=p.meta["probe_cell"])
        return p.dt * np.sum(probe ** 2)
    fd_o = (J_orc(G0 * (1 + hs)) - J_orc(G0 * (1 - hs))) / (2 * hs)
    assert abs(fd_o - g_s) < 1e-5 * abs(g_s), (fd_o, g_s)


def test_soft_source_on_an_open_grid(orc):
    p = open_grid("soft", probe=200)
    src = p.source_samples(0, p.n_steps)
    J, dsrc, _, _ = J_and_grads(p, src)
    _, probe = orc.run(p, n_steps=p.n_steps, probe_cell=p.meta["probe_cell"])
    assert abs(J - p.dt * np.sum(probe ** 2)) < 1e-10 * J
    rng = np.random.default_rng(3)
    d = np.zeros_like(src)
    d[:200] = rng.normal(size=200)
    h = 1e-6 * np.abs(src).max()
    fd = (J_only(p, src + h * d) - J_only(p, src - h * d)) / (2 * h)
    assert abs(fd - dsrc @ d) < 1e-6 * abs(dsrc @ d), (fd, dsrc @ d)


@pytest.mark.parametrize("precision,kernel,tol", [("fp64", "auto", 1e-9), ("fp64", "register", 1e-9),
                                                  ("fp32", "auto", 2e-4)])
def test_merged_form_context(precision, kernel, tol):
    """The merged form's forward and checkpoints (sparse, register or run-time
    compiled cell models), the Strang form's recompute and reverse: the same J
    and gradients as a Strang-form context, up to the rounding of the two
    forward trajectories."""
    p = W.adjoint_ring(n_cells=512, n_steps=300, n_src=64, amplitude=3e7)
    src = p.source_samples(0, p.n_steps)
    a = J_and_grads(p, src, precision=precision, form="strang", every=32)
    b = J_and_grads(p, src, precision=precision, form="merged", every=32, kernel=kernel)
    assert abs(b[0] - a[0]) < tol * abs(a[0])
    for x, y in zip(a[1:], b[1:]):
        x, y = np.asarray(x), np.asarray(y)
        assert np.abs(y - x).max() < tol * np.abs(x).max()


def test_merged_form_open_grid_against_finite_differences():
    p = open_grid("hard")
    src = p.source_samples(0, p.n_steps)
    J, dsrc, _, _ = J_and_grads(p, src, form="merged")
    rng = np.random.default_rng(4)
    d = np.zeros_like(src)
    d[:200] = rng.normal(size=200)
    h = 1e-6 * np.abs(src).max()
    fd = (J_only(p, src + h * d, form="merged") - J_only(p, src - h * d, form="merged")) / (2 * h)
    assert abs(fd - dsrc @ d) < 1e-6 * abs(dsrc @ d), (fd, dsrc @ d)

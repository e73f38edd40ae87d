"""Adjoint gradients (mln_adjoint): J = dt sum_n (E_z^n at the probe)^2 and its
gradients with respect to the source samples, the dipole operator and the
relaxation superoperator, by the reverse-time kernel with checkpointing and
recomputation.

Checked against central finite differences of J computed by the forward
kernels (h = 1e-6 relative along seeded directions), and against central
finite differences of the oracle's J (gradient taken through the oracle).
"""
import numpy as np
import pytest

import workloads as W
from helpers import params_of, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


def J_and_grads(p, src, precision="fp64", every=32, mu=None, G=None, memory=0):
    import torch
    from paper_1710_09799_gb300 import mln
    q = p.with_(mu=p.mu if mu is None else mu, G=p.G if G is None else G)
    s = mln.Solver(params_of(q, precision=precision, form="strang"), E0=q.e_init())
    mln.mln_set_adjoint_memory(s.ctx, memory)
    t = torch.as_tensor(src, dtype=torch.float64, device="cuda")
    out = mln.mln_adjoint(s.ctx, q.N, len(src), t.data_ptr(), p.meta["probe_cell"], every)
    s.close()
    return out


def J_only(p, src, mu=None, G=None, precision="fp64"):
    return J_and_grads(p, src, precision, every=10 ** 6, mu=mu, G=G)[0]


def rate_grad(dG, p):
    return np.array([np.real(np.sum(np.conj(dG) * u)) for u in p.meta["unit_superops"]])


def G_of(p, rates):
    return sum(r * u for r, u in zip(rates, p.meta["unit_superops"]))


@pytest.fixture(scope="module")
def small():
    p = W.adjoint_ring(n_cells=512, n_steps=300, n_src=64, amplitude=3e7)
    src = p.source_samples(0, p.n_steps)
    return p, src, J_and_grads(p, src)


@pytest.fixture(scope="module")
def strong():
    """The same problem with 200x the relaxation rates: over 300 steps (2.3 fs)
    the nominal rates change J by ~1e-10 relative, too little for a finite
    difference to resolve against rounding."""
    p = W.adjoint_ring(n_cells=512, n_steps=300, n_src=64, amplitude=3e7)
    p.meta["rate_values"] = 200.0 * p.meta["rate_values"]
    p = p.with_(G=G_of(p, p.meta["rate_values"]))
    src = p.source_samples(0, p.n_steps)
    return p, src, J_and_grads(p, src)


def test_objective_matches_oracle(orc, small):
    p, src, (J, _, _, _) = small
    _, probe = orc.run(p, n_steps=p.n_steps, probe_cell=p.meta["probe_cell"])
    Jo = p.dt * np.sum(probe ** 2)
    assert abs(J - Jo) < 1e-10 * Jo


def test_source_gradient_vs_finite_differences(small):
    p, src, (J, dsrc, _, _) = small
    assert np.all(np.isfinite(dsrc)) and np.abs(dsrc[:p.meta["n_src"]]).max() > 0
    rng = np.random.default_rng(0)
    for _ in range(4):
        d = np.zeros_like(src)
        d[:p.meta["n_src"]] = rng.normal(size=p.meta["n_src"])
        h = 1e-6 * np.abs(src).max()
        fd = (J_only(p, src + h * d) - J_only(p, src - h * d)) / (2 * h)
        ad = dsrc @ d
        assert abs(fd - ad) < 1e-6 * max(abs(ad), 1e-30) + 1e-9 * np.abs(dsrc).sum() * h, (fd, ad)


def test_dipole_and_rate_gradients_vs_finite_differences(small, strong):
    from paper_1710_09799_gb300 import mln
    p, src, (J, _, dmu, dG) = small
    x0 = mln.mu_to_params(p.mu)
    # the three real dipole elements mu_12, mu_13, mu_23 (indices N + pair)
    for k in range(3):
        i = p.N + k
        h = 1e-6 * abs(x0[i])
        xp, xm = x0.copy(), x0.copy()
        xp[i] += h
        xm[i] -= h
        mup = mln.mu_from_params(p.N, xp).numpy()
        mum = mln.mu_from_params(p.N, xm).numpy()
        fd = (J_only(p, src, mu=mup) - J_only(p, src, mu=mum)) / (2 * h)
        assert abs(fd - dmu[i]) < 1e-5 * abs(dmu[i]), (k, fd, dmu[i])
    p, src, (J, _, dmu, dG) = strong
    g_rates = rate_grad(dG, p)
    r0 = p.meta["rate_values"]
    for k in range(3):
        h = 1e-4 * r0[k]
        rp, rm = r0.copy(), r0.copy()
        rp[k] += h
        rm[k] -= h
        fd = (J_only(p, src, G=G_of(p, rp)) - J_only(p, src, G=G_of(p, rm))) / (2 * h)
        assert abs(fd - g_rates[k]) < 1e-5 * abs(g_rates[k]), (k, fd, g_rates[k])


def test_gradient_through_the_oracle(orc, small, strong):
    """Central differences of the oracle's J for one dipole element and one
    rate agree with the adjoint gradients of the CUDA path."""
    from paper_1710_09799_gb300 import mln
    p, src, (_, _, dmu, dG) = small
    pc = p.meta["probe_cell"]

    def Jo(q):
        _, probe = orc.run(q, n_steps=q.n_steps, probe_cell=pc)
        return q.dt * np.sum(probe ** 2)

    x0 = mln.mu_to_params(p.mu)
    i = p.N  # mu_12
    h = 1e-6 * abs(x0[i])
    xp, xm = x0.copy(), x0.copy()
    xp[i] += h
    xm[i] -= h
    fd = (Jo(p.with_(mu=mln.mu_from_params(p.N, xp).numpy())) - Jo(p.with_(mu=mln.mu_from_params(p.N, xm).numpy()))) / (2 * h)
    assert abs(fd - dmu[i]) < 1e-5 * abs(dmu[i]), (fd, dmu[i])
    p, src, (_, _, dmu, dG) = strong
    r0 = p.meta["rate_values"]
    h = 1e-4 * r0[0]
    rp, rm = r0.copy(), r0.copy()
    rp[0] += h
    rm[0] -= h
    fd = (Jo(p.with_(G=G_of(p, rp))) - Jo(p.with_(G=G_of(p, rm)))) / (2 * h)
    g = rate_grad(dG, p)[0]
    assert abs(fd - g) < 1e-5 * abs(g), (fd, g)


def test_checkpoint_interval_does_not_change_gradients(small):
    p, src, (J, dsrc, dmu, dG) = small
    J2, dsrc2, dmu2, dG2 = J_and_grads(p, src, every=7)
    assert abs(J2 - J) <= 1e-12 * J
    assert rel_inf(dsrc2, dsrc) < 1e-10 and rel_inf(dmu2, dmu) < 1e-10 and rel_inf(dG2, dG) < 1e-10


@pytest.mark.parametrize("n_steps,every", [(1, 1), (2, 1), (5, 1), (5, 2), (13, 5)])
def test_short_runs_and_one_step_segments(orc, n_steps, every):
    """Runs shorter than one reverse launch, segments of one step, the probe on
    the source cell next to the ring's wrap: J against the oracle, the
    gradients equal to those of a single segment, dJ/dsrc against central
    differences."""
    p = W.adjoint_ring(n_cells=512, n_steps=n_steps, n_src=n_steps, amplitude=3e7)
    p.meta["probe_cell"] = 0
    src = p.source_samples(0, n_steps)
    J, dsrc, dmu, dG = J_and_grads(p, src, every=every)
    _, probe = orc.run(p, n_steps=n_steps, probe_cell=0)
    Jo = p.dt * np.sum(probe ** 2)
    assert Jo > 0 and abs(J - Jo) < 1e-10 * Jo, (J, Jo)
    J1, dsrc1, dmu1, dG1 = J_and_grads(p, src, every=10 ** 6)
    assert abs(J1 - J) <= 1e-12 * J
    assert rel_inf(dsrc1, dsrc) < 1e-10 and rel_inf(dmu1, dmu) < 1e-10 and rel_inf(dG1, dG) < 1e-10
    d = np.random.default_rng(n_steps).normal(size=n_steps)
    h = 1e-6 * np.abs(src).max()
    fd = (J_only(p, src + h * d) - J_only(p, src - h * d)) / (2 * h)
    assert abs(fd - dsrc @ d) < 1e-6 * abs(dsrc @ d), (fd, dsrc @ d)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("every", [7, 32])
def test_recompute_schedules_give_the_same_bits(small, precision, every):
    """All segments recomputed side by side (the default, memory permitting)
    and two segments at a time (a 1-byte limit forces it): the same kernels
    on the same inputs, so the same bits. 300 steps: 42 segments of 7 and
    one of 6, or 9 of 32 and one of 12."""
    p, src, _ = small
    a = J_and_grads(p, src, precision=precision, every=every)
    b = J_and_grads(p, src, precision=precision, every=every, memory=1)
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


def test_adjoint_memory_limit_rejects_negative(small):
    import torch
    from paper_1710_09799_gb300 import mln
    p, _, _ = small
    s = mln.Solver(params_of(p, precision="fp64", form="strang"), E0=p.e_init())
    with pytest.raises(mln.MLNError) as ei:
        mln.mln_set_adjoint_memory(s.ctx, -1)
    assert ei.value.status == mln.MLN_EINVAL
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_workspace_kept_between_calls(small, precision):
    """The context keeps its adjoint workspace between calls: from the same
    initial state (reloaded) a second call gives the bits of a fresh context;
    a longer run grows the workspace; after mln_adjoint_release the next call
    allocates again, with the same bits."""
    import torch
    from paper_1710_09799_gb300 import mln
    p, src, _ = small
    fresh = J_and_grads(p, src, precision=precision)
    src2 = np.concatenate([src, np.zeros(100)])
    fresh2 = J_and_grads(p, src2, precision=precision)
    s = mln.Solver(params_of(p, precision=precision, form="strang"), E0=p.e_init())
    s0 = s.save()
    t = torch.as_tensor(src, dtype=torch.float64, device="cuda")
    t2 = torch.as_tensor(src2, dtype=torch.float64, device="cuda")

    def call(tt):
        s.load(*s0)
        return mln.mln_adjoint(s.ctx, p.N, tt.numel(), tt.data_ptr(), p.meta["probe_cell"], 32)

    runs = [(call(t), fresh), (call(t), fresh), (call(t2), fresh2), (call(t), fresh)]
    mln.mln_adjoint_release(s.ctx)
    mln.mln_adjoint_release(s.ctx)  # nothing held: no-op
    runs.append((call(t), fresh))
    s.close()
    for got, want in runs:
        assert got[0] == want[0]
        for x, y in zip(got[1:], want[1:]):
            assert np.array_equal(x, y)


def test_fp32_adjoint_close_to_fp64(small):
    p, src, (J, dsrc, dmu, dG) = small
    J3, dsrc3, dmu3, dG3 = J_and_grads(p, src, precision="fp32")
    assert abs(J3 - J) < 1e-3 * J
    assert rel_inf(dsrc3, dsrc) < 1e-2
    assert rel_inf(dmu3[p.N:p.N + 3], dmu[p.N:p.N + 3]) < 1e-2


def test_autograd_function(small):
    """torch autograd through probe_energy: the rates and dipoles built with
    torch ops get the chain-ruled gradients."""
    import torch
    from paper_1710_09799_gb300 import mln
    p, src, (J, dsrc, dmu, dG) = small
    rates = torch.tensor(p.meta["rate_values"], dtype=torch.float64, requires_grad=True)
    units = torch.stack([torch.view_as_real(torch.as_tensor(u)) for u in p.meta["unit_superops"]])
    G_real = (rates[:, None, None, None] * units).sum(0)
    mu_p = torch.tensor(mln.mu_to_params(p.mu), dtype=torch.float64, requires_grad=True)
    s_t = torch.tensor(src, dtype=torch.float64, requires_grad=True)
    base = dict(N=p.N, H0=p.H0, rho0=p.rho0, N_a=p.N_a, n_cells=p.n_cells, medium_begin=p.medium_begin,
                medium_end=p.medium_end, dx=p.dx, dt=p.dt, source_kind="soft", source_cell=0,
                E0=p.e_init(), probe_cell=p.meta["probe_cell"], every=32)
    Jt = mln.probe_energy(s_t, mu_p, G_real, base)
    Jt.backward()
    assert abs(Jt.item() - J) < 1e-12 * J
    assert np.allclose(s_t.grad.numpy(), dsrc, rtol=1e-12, atol=0)
    assert np.allclose(mu_p.grad.numpy(), dmu, rtol=1e-12, atol=0)
    assert np.allclose(rates.grad.numpy(), rate_grad(dG, p), rtol=1e-10)


def test_full_size_gradient_along_seeded_directions():
    """The gradient workload at full size (8192 cells, 5000 steps, 512 source
    samples, checkpoints every 256 steps, the benchmark's launch shape): the
    adjoint directional derivative along 10 seeded directions in the joint
    space of the 3 real dipole elements, the 3 relaxation rates and the 512
    source samples against central finite differences (h = 1e-6 relative)."""
    from paper_1710_09799_gb300 import mln
    p = W.adjoint_ring()
    src = p.source_samples(0, p.n_steps)
    ns = p.meta["n_src"]
    mu0 = mln.mu_to_params(p.mu)
    r0 = p.meta["rate_values"]

    def run(mu_x, rates, s, grads=False):
        q = p.with_(mu=mln.mu_from_params(p.N, mu_x).numpy(), G=G_of(p, rates))
        sol = mln.Solver(params_of(q, precision="fp64", form="strang"), E0=q.e_init())
        sol.autotune(2)
        t = __import__("torch").as_tensor(s, dtype=__import__("torch").float64, device="cuda")
        out = mln.mln_adjoint(sol.ctx, q.N, len(s), t.data_ptr(), p.meta["probe_cell"], 256)
        sol.close()
        return out if grads else out[0]

    J, dsrc, dmu, dG = run(mu0, r0, src, grads=True)
    g_rates = rate_grad(dG, p)
    idx = [p.N + k for k in range(3)]  # Re mu_12, mu_13, mu_23
    scale_mu = np.abs(mu0[idx])
    scale_src = np.abs(src[:ns]).max()
    rng = np.random.default_rng(2024)
    h = 1e-6
    for trial in range(10):
        u_mu, u_r, u_s = rng.normal(size=3), rng.normal(size=3), rng.normal(size=ns)
        d_mu = h * scale_mu * u_mu
        d_r = h * r0 * u_r
        d_s = h * scale_src * u_s
        ad = float(dmu[idx] @ d_mu + g_rates @ d_r + dsrc[:ns] @ d_s)

        def shifted(sign):
            mu_x = mu0.copy()
            mu_x[idx] += sign * d_mu
            s = src.copy()
            s[:ns] += sign * d_s
            return run(mu_x, r0 + sign * d_r, s)

        fd = (shifted(+1) - shifted(-1)) / 2
        assert abs(fd - ad) < 1e-5 * abs(ad) + 1e-13 * J, (trial, fd, ad)

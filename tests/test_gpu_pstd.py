"""The pseudo-spectral field solver (MLN_MAXWELL_PSTD) on the GPU against the
oracle's PSTD solver (circulant derivatives from the DFT definition, O(n^2)
sums, FP64) and against closed forms.

FP64: E_z within 1e-10 relative (infinity norm) and populations within 1e-10;
FP32: the FDTD tolerances per 1000 steps. At the benchmark size (65536 cells),
where the O(n^2) oracle is out of reach, the vacuum solution of a cosine
field is compared with its closed form and the vacuum energy with its start.
"""
import math

import numpy as np
import pytest

import workloads as W
from helpers import assert_fp32, gpu_run, make_solver, rel_inf
from workloads import EPS0, MU0

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


def pops(rho):
    return np.einsum("cii->ci", rho).real


def ring(n=256, n_steps=500):
    return W.three_level_ring(n_cells=n, n_steps=n_steps).with_(maxwell="pstd")


def sit_ring(n=512, n_steps=1000, source="soft"):
    """Two-level medium filling half of a periodic PSTD grid, sech pulse fed at cell 10."""
    p = W.two_level_sit(n_cells=n, medium=(n // 4, 3 * n // 4), n_steps=n_steps)
    return p.with_(boundary="periodic", source_kind=source, source_cell=10, maxwell="pstd")


@pytest.mark.parametrize("form,kernel", [("merged", "auto"), ("merged", "register"), ("strang", "auto")])
def test_three_level_ring_against_oracle(orc, form, kernel):
    p = ring()
    ref, _ = orc.run(p, n_steps=p.n_steps)
    E, H, rho, s = gpu_run(p, p.n_steps, "fp64", form, kernel=kernel)
    assert s.kernel_in_use == ("sparse" if (form, kernel) == ("merged", "auto") else "register")
    s.close()
    assert rel_inf(E, ref.E) < FP64_TOL and rel_inf(H, ref.H) < FP64_TOL
    assert np.abs(pops(rho) - pops(ref.rho)).max() < FP64_TOL


@pytest.mark.parametrize("source", ["soft", "hard"])
def test_pulse_through_partial_medium(orc, source):
    p = sit_ring(source=source)
    ref, _ = orc.run(p, n_steps=p.n_steps)
    assert np.abs(ref.E[p.medium_begin:p.medium_end]).max() > 1e6  # the pulse is in the medium
    E, H, rho, s = gpu_run(p, p.n_steps, "fp64", "merged", chunks=[300, 700])
    s.close()
    assert rel_inf(E, ref.E) < FP64_TOL
    assert np.abs(pops(rho) - pops(ref.rho)).max() < FP64_TOL
    E32, _, rho32, s = gpu_run(p, p.n_steps, "fp32", "merged")
    s.close()
    e_err, p_err = rel_inf(E32, ref.E), np.abs(pops(rho32) - pops(ref.rho)).max()
    print(f"pstd fp32 {source}: E rel {e_err:.3e}  pop abs {p_err:.3e}")
    assert_fp32("pstd", p.n_steps, e_err, p_err)


def test_4096_cells_against_oracle(orc):
    p = ring(n=4096, n_steps=100)
    ref, _ = orc.run(p, n_steps=p.n_steps)
    E, _, rho, s = gpu_run(p, p.n_steps, "fp64", "merged")
    s.close()
    assert rel_inf(E, ref.E) < FP64_TOL and np.abs(pops(rho) - pops(ref.rho)).max() < FP64_TOL


def test_sparse_and_register_cell_models_same_bits():
    p = ring(n=1024, n_steps=200)
    a = gpu_run(p, p.n_steps, "fp64", "merged", kernel="sparse")
    b = gpu_run(p, p.n_steps, "fp64", "merged", kernel="register")
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    a[3].close()
    b[3].close()


@pytest.mark.parametrize("n,m", [(64, 20), (65536, 1000)])
def test_vacuum_cosine_closed_form(n, m):
    p = W.two_level_sit(n_cells=n, medium=(0, 0)).with_(boundary="periodic", G=None, source_kind="none",
                                                       src=None, meta={}, maxwell="pstd")
    k = 2 * math.pi * m / (n * p.dx)
    th = 2 * math.asin(p.dt * k / (2 * math.sqrt(EPS0 * MU0)))
    x = np.arange(n) * p.dx
    p = p.with_(E_init=np.cos(k * x))
    steps = 400
    E, H, _, s = gpu_run(p, steps, "fp64", "merged")
    s.close()
    ref = (math.cos(steps * th) - math.tan(th / 2) * math.sin(steps * th)) * np.cos(k * x)
    assert np.abs(E - ref).max() < 1e-10


def test_vacuum_energy_full_size():
    n = 65536
    rng = np.random.default_rng(2)
    p = W.two_level_sit(n_cells=n, medium=(0, 0)).with_(boundary="periodic", G=None, source_kind="none",
                                                       src=None, meta={}, maxwell="pstd",
                                                       E_init=rng.normal(0, 1e3, size=n))
    s = make_solver(p, "fp64", "merged")
    vals = []
    for _ in range(4):
        E0, H0 = s.fields()
        s.step(1)
        s.sync()
        _, H1 = s.fields()
        vals.append(EPS0 * np.sum(E0 ** 2) + MU0 * np.sum(H0 * H1))
        s.step(49)
    s.close()
    vals = np.array(vals)
    assert np.abs(vals - vals[0]).max() < 1e-11 * vals[0]


def test_rejected_configurations():
    from paper_1710_09799_gb300 import mln
    with pytest.raises(mln.MLNError):
        make_solver(ring(n=1000), "fp64", "merged")  # not a power of two
    with pytest.raises(mln.MLNError):
        make_solver(sit_ring().with_(boundary="open"), "fp64", "merged")
    with pytest.raises(mln.MLNError):
        make_solver(ring(), "fp32", "merged", kernel="jit")
    with pytest.raises(mln.MLNError):
        make_solver(W.six_level_pulse(n_cells=256, n_steps=10).with_(boundary="periodic", maxwell="pstd",
                                                                     source_kind="none"),
                    "fp32", "merged", kernel="tensor")
    p = ring()
    with pytest.raises(mln.MLNError):
        mln.Batch([make_params_of(p)], [p.e_init()], None, 0)


def make_params_of(p):
    from helpers import params_of
    return params_of(p, precision="fp64", form="merged")


@pytest.mark.parametrize("N", [4, 6])
def test_more_levels_against_oracle(orc, N):
    if N == 4:
        p = W.multi_level_ring(4, n_cells=256, n_steps=200, seed=5).with_(maxwell="pstd")
    else:
        p = W.six_level_pulse(n_cells=256, n_steps=150, t0=15e-15, fwhm=10e-15).with_(
            boundary="periodic", source_kind="soft", source_cell=5, medium_begin=0, medium_end=256, maxwell="pstd")
    ref, _ = orc.run(p, n_steps=p.n_steps)
    E, _, rho, s = gpu_run(p, p.n_steps, "fp64", "merged")
    s.close()
    assert np.abs(ref.E).max() > 0
    assert rel_inf(E, ref.E) < FP64_TOL and np.abs(pops(rho) - pops(ref.rho)).max() < FP64_TOL


def test_rodrigues_form_against_oracle(orc):
    p = ring(n=256, n_steps=200)
    ref, _ = orc.run(p, n_steps=p.n_steps)
    E, _, rho, s = gpu_run(p, p.n_steps, "fp64", "rodrigues")
    s.close()
    assert rel_inf(E, ref.E) < FP64_TOL and np.abs(pops(rho) - pops(ref.rho)).max() < FP64_TOL


def test_save_load_continues_bit_for_bit():
    """Each mln_step call transforms E from the buffers again, so a state loaded
    between calls continues exactly as an uninterrupted run. (Strang form: its
    device state is d itself, so saving and loading are exact; the merged
    form's state y = A0 d + b goes through d with FP64 maps, not bit-exact.)"""
    p = sit_ring(n=512, n_steps=300)
    from helpers import src_tensor
    a = make_solver(p, "fp64", "strang")
    a.step(100, src_tensor(p, 0, 100))
    saved = a.save()
    a.step(200, src_tensor(p, 100, 200))
    a.sync()
    Ea, Ha = a.fields()
    ra = a.rho()
    b = make_solver(p, "fp64", "strang")
    b.load(*saved)
    b.step(200, src_tensor(p, 100, 200))
    b.sync()
    Eb, Hb = b.fields()
    assert np.array_equal(Ea, Eb) and np.array_equal(Ha, Hb) and np.array_equal(ra, b.rho())
    a.close()
    b.close()

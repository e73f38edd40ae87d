"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

FP64: E_z within 1e-10 relative in the infinity norm and populations within
1e-10 absolute (the target the method is built to). FP32: kappa u n per
workload family (u = 2^-24, n steps; helpers.FP32_KAPPA: about five times the
growth measured on a GB300).
Sizes span several thread-block tiles with a ragged last tile; the full-size
three-level ring is checked on sampled cells computed one by one from their
light cones.
"""
import numpy as np
import pytest

import workloads as W
from helpers import assert_fp32, gpu_run, make_solver, rel_inf, src_tensor

pytestmark = pytest.mark.gpu

FP64_E = 1e-10
FP64_POP = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


def oracle_ref(orc, p, n_steps):
    st, _ = orc.run(p, n_steps=n_steps)
    return st


def pops(rho):
    return np.einsum("cii->ci", rho).real


@pytest.mark.parametrize("form", ["strang", "merged", "rodrigues", "rotated"])
def test_two_level_sit_full_fp64(orc, form):
    """The two-level workload at full size: 2000 cells, medium [500, 1500),
    sech pulse of area 2 pi, hard source + Mur, 20000 steps."""
    p = W.two_level_sit()
    ref = oracle_ref(orc, p, p.n_steps)
    E, H, rho, s = gpu_run(p, p.n_steps, "fp64", form)
    assert rel_inf(E, ref.E) < FP64_E
    assert rel_inf(H, ref.H) < FP64_E
    assert np.abs(pops(rho) - pops(ref.rho)).max() < FP64_POP
    assert np.abs(rho - ref.rho).max() < FP64_POP
    assert pops(ref.rho)[:, 1].max() > 1e-3  # the pulse reached and excited the medium


@pytest.mark.parametrize("form", ["strang", "merged", "rodrigues", "rotated"])
def test_three_level_ring_small_fp64(orc, form):
    """Three-level ring, 4096 cells (several tiles, ragged last tile), 1500 steps."""
    p = W.three_level_ring(n_cells=4096, n_steps=1500)
    ref = oracle_ref(orc, p, p.n_steps)
    E, H, rho, _ = gpu_run(p, p.n_steps, "fp64", form, chunks=[700, 1, 799])
    assert rel_inf(E, ref.E) < FP64_E
    assert rel_inf(H, ref.H) < FP64_E
    assert np.abs(pops(rho) - pops(ref.rho)).max() < FP64_POP
    assert np.abs(rho - ref.rho).max() < FP64_POP


@pytest.mark.parametrize("form", ["strang", "merged", "rotated"])
def test_six_level_small_fp64(orc, form):
    """Six-level manifold (D = 35), 700 cells (medium up to the cell before the
    Mur cell), Gaussian source, 400 steps."""
    p = W.six_level_pulse(n_cells=700, n_steps=400, t0=20e-15, fwhm=10e-15)
    p = p.with_(medium_begin=3, medium_end=699)
    ref = oracle_ref(orc, p, p.n_steps)
    E, H, rho, _ = gpu_run(p, p.n_steps, "fp64", form)
    assert rel_inf(E, ref.E) < FP64_E
    assert np.abs(pops(rho) - pops(ref.rho)).max() < FP64_POP


@pytest.mark.parametrize("N", [4, 5])
def test_other_N_fp64(orc, N):
    rng = np.random.default_rng(N)
    H0 = W.random_hermitian(rng, N, 60 * W.MEV)
    mu = W.random_hermitian(rng, N, 2 * W.NM_E)
    rates = {(b, a): rng.uniform(0.5, 5) * 1e12 for a in range(N) for b in range(a + 1, N)}
    p = W.Problem(name="rand", N=N, H0=H0, mu=mu, G=W.lindblad_superop(N, rates),
                  rho0=W.random_density(rng, N), N_a=3e24, n_cells=777, medium_begin=100,
                  medium_end=650, boundary="periodic", n_steps=300,
                  E_init=rng.normal(0, 1e8, size=777))
    ref = oracle_ref(orc, p, p.n_steps)
    for form in ("strang", "merged", "rotated") + (("rodrigues",) if N <= 4 else ()):
        E, H, rho, _ = gpu_run(p, p.n_steps, "fp64", form)
        assert rel_inf(E, ref.E) < FP64_E
        assert np.abs(rho - ref.rho).max() < FP64_POP


def test_three_level_ring_full_size_sampled(orc):
    """The full 65536-cell ring in the launch shape the benchmark uses; cells
    sampled across tiles are recomputed by the oracle from their light cones."""
    p = W.three_level_ring()
    steps = 200
    for form in ("strang", "merged"):
        E, H, rho, s = gpu_run(p, steps, "fp64", form)
        for c in (0, 431, 432, 30000, 65535):
            e, h, r = orc.run_window(p, c, steps)
            assert abs(E[c] - e) <= FP64_E * np.abs(E).max()
            assert abs(H[c] - h) <= FP64_E * np.abs(H).max()
            assert np.abs(rho[c] - r).max() < FP64_POP


def test_fp32_error_bounds(orc):
    """FP32 state and propagator with FP64 set-up against the FP64 oracle."""
    p = W.three_level_ring(n_cells=4096, n_steps=2000)
    ref = oracle_ref(orc, p, p.n_steps)
    for form in ("strang", "merged", "rodrigues", "rotated"):
        E, H, rho, _ = gpu_run(p, p.n_steps, "fp32", form)
        e_err = rel_inf(E, ref.E)
        p_err = np.abs(pops(rho) - pops(ref.rho)).max()
        print(f"fp32 {form}: E rel {e_err:.3e}  pop abs {p_err:.3e}")
        assert_fp32("ring_rotated" if form == "rotated" else "ring", p.n_steps, e_err, p_err)


def test_fp32_two_level(orc):
    p = W.two_level_sit(n_steps=6000)
    ref = oracle_ref(orc, p, p.n_steps)
    for form in ("strang", "merged"):
        E, H, rho, _ = gpu_run(p, p.n_steps, "fp32", form)
        e_err = rel_inf(E, ref.E)
        p_err = np.abs(pops(rho) - pops(ref.rho)).max()
        print(f"fp32 two-level {form}: E rel {e_err:.3e}  pop abs {p_err:.3e}")
        assert_fp32("two_level", p.n_steps, e_err, p_err)


# ---------------------------------------------------------------- properties

@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (16, 0), (64, 37), (40, 200)])
def test_launch_shape_does_not_change_results(shape):
    """Every cell does the same arithmetic in the same order whatever the tile
    and the number of fused steps: results are bit-identical."""
    K, tile = shape
    p = W.three_level_ring(n_cells=1000, n_steps=150)
    E0, H0, r0, _ = gpu_run(p, p.n_steps, "fp64", "strang", block_steps=16, tile_cells=100)
    E1, H1, r1, _ = gpu_run(p, p.n_steps, "fp64", "strang", block_steps=K, tile_cells=tile)
    assert np.array_equal(E0, E1) and np.array_equal(H0, H1) and np.array_equal(r0, r1)


@pytest.mark.parametrize("K,tile", [(8, 200), (40, 100), (64, 40), (1, 50), (33, 8)])
def test_tile_made_of_the_mur_cell_alone(orc, K, tile):
    """Open grid of 201 cells whose last tile is the Mur cell (cell 200) alone:
    its value comes from cell 199's update in the same step, so its dependence
    reaches one cell beyond a K-step halo. The pulse reaches the boundary within
    the run, so a wrong Mur cell would show in E_z. Against the oracle, and bit
    for bit against a shape whose tiles never start at the Mur cell."""
    p = W.two_level_sit(n_cells=201, medium=(50, 150), n_steps=1200)
    assert (p.n_cells - 1) % tile == 0
    ref = oracle_ref(orc, p, p.n_steps)
    E, H, rho, s = gpu_run(p, p.n_steps, "fp64", "merged", kernel="register", block_steps=K, tile_cells=tile)
    s.close()
    assert np.abs(ref.E[-5:]).max() > 1e3  # the field has reached the Mur cell
    assert rel_inf(E, ref.E) < FP64_E and np.abs(pops(rho) - pops(ref.rho)).max() < FP64_POP
    for precision in ("fp64", "fp32"):
        a = gpu_run(p, p.n_steps, precision, "merged", kernel="register", block_steps=K, tile_cells=tile)
        b = gpu_run(p, p.n_steps, precision, "merged", kernel="register", block_steps=7, tile_cells=30)
        assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])), precision
        a[3].close()
        b[3].close()


@pytest.mark.parametrize("precision,form", [("fp64", "merged"), ("fp32", "merged"), ("fp64", "strang")])
def test_autotune_changes_no_state_and_no_result(precision, form):
    """The autotuner times candidate shapes without touching the state, and
    the shape it picks gives the same bits as the default shape."""
    p = W.three_level_ring(n_cells=5000, n_steps=120)
    E0, H0, r0, _ = gpu_run(p, p.n_steps, precision, form)
    s = make_solver(p, precision, form)
    K, tile = s.autotune(2)
    assert 1 <= K <= 64 and tile >= 1
    assert s.launch_shape[:2] == (K, tile)
    s.step(p.n_steps)
    s.sync()
    E1, H1 = s.fields()
    assert np.array_equal(E0, E1) and np.array_equal(H0, H1) and np.array_equal(r0, s.rho())


def test_step_splitting_is_exact():
    p = W.two_level_sit(n_steps=900)
    E0, H0, r0, _ = gpu_run(p, 900, "fp64", "merged")
    E1, H1, r1, _ = gpu_run(p, 900, "fp64", "merged", chunks=[1, 16, 17, 300, 566])
    assert np.array_equal(E0, E1) and np.array_equal(r0, r1)


@pytest.mark.parametrize("case", ["tiny_ring", "tiny_open", "vacuum", "one_cell_medium", "soft_source",
                                  "lossy", "dielectric", "no_relaxation", "degenerate_dipoles"])
def test_edge_cases(orc, case):
    base = W.three_level_ring(n_cells=64, n_steps=120)
    if case == "no_relaxation":
        # G = 0: M = -i[H0, .] is singular (populations undamped), the augmented
        # half-step exponential still defines A0 and b (b = 0)
        p = base.with_(G=None, E_init=base.e_init() * 1e5)
    elif case == "degenerate_dipoles":
        # mu = mu0 (J - I): eigenvalues 2 mu0, -mu0, -mu0; the plane of the
        # degenerate pair turns by zero angle and its basis is not unique
        mu = 2 * W.NM_E * (np.ones((3, 3)) - np.eye(3)).astype(np.complex128)
        p = base.with_(mu=mu, E_init=base.e_init() * 1e5)
    elif case == "tiny_ring":
        p = W.three_level_ring(n_cells=4, n_steps=50)
    elif case == "tiny_open":
        p = W.two_level_sit(n_cells=6, medium=(1, 5), n_steps=80)
    elif case == "vacuum":
        p = base.with_(medium_begin=0, medium_end=0)
    elif case == "one_cell_medium":
        p = base.with_(medium_begin=17, medium_end=18, N_a=1e26)
    elif case == "soft_source":
        fn = W.gauss_pulse(1e9, 5e-15, 3e-15, 1e15, base.dt)
        p = base.with_(source_kind="soft", source_cell=5)
        p.meta["source_fn"] = fn
    elif case == "lossy":
        p = base.with_(sigma=2e5)
    else:
        p = W.two_level_sit(n_cells=300, medium=(100, 200), n_steps=500).with_(eps_r=2.25, mu_r=1.1)
    ref = oracle_ref(orc, p, p.n_steps)
    for form in ("strang", "merged"):
        E, H, rho, _ = gpu_run(p, p.n_steps, "fp64", form, block_steps=7)
        assert rel_inf(E, ref.E) < FP64_E, case
        if p.n_medium:
            assert np.abs(rho - ref.rho).max() < FP64_POP, case


def test_zero_steps_and_state_round_trip(orc):
    p = W.three_level_ring(n_cells=500, n_steps=100)
    for prec in ("fp64", "fp32"):
        for form in ("strang", "merged", "rotated"):
            s = make_solver(p, prec, form)
            s.step(0)
            s.sync()
            d, E, H = s.save()
            rho = s.rho()
            tol = 1e-15 if prec == "fp64" else 1e-6
            assert np.abs(rho - p.rho0).max() < tol
            s.step(37)
            d1, E1, H1 = s.save()
            s.load(d, E, H)
            s.step(37)
            d2, E2, H2 = s.save()
            assert np.abs(d2 - d1).max() <= (1e-13 if prec == "fp64" else 1e-5)
            assert np.array_equal(E1, E2) if (prec, form) == ("fp64", "strang") else \
                np.abs(E2 - E1).max() <= 1e-5 * np.abs(E1).max()


def test_resume_matches_uninterrupted_run(orc):
    """Checkpoint after 400 steps into a new context, 400 more steps: equals the
    oracle's 800-step run (the checkpoint is the precision-independent d)."""
    p = W.three_level_ring(n_cells=2048, n_steps=800)
    ref = oracle_ref(orc, p, 800)
    _, _, _, s = gpu_run(p, 400, "fp64", "merged")
    d, E, H = s.save()
    s2 = make_solver(p, "fp64", "strang")
    s2.load(d, E, H)
    s2.step(400)
    s2.sync()
    E2, _ = s2.fields()
    assert rel_inf(E2, ref.E) < FP64_E
    assert np.abs(s2.rho() - ref.rho).max() < FP64_POP


def test_nonfinite_field_is_reported():
    from paper_1710_09799_gb300 import mln
    p = W.three_level_ring(n_cells=256, n_steps=10)
    s = make_solver(p, "fp64", "merged")
    d0, E0, H0 = s.save()
    E = E0.copy()
    E[100] = np.nan
    s.load(E=E)
    s.step(10)
    with pytest.raises(mln.MLNError) as ei:
        s.sync()
    assert ei.value.status == mln.MLN_ENONFINITE
    s.load(d0, E0, H0)  # the NaN reached the medium too; reload everything
    s.step(5)
    s.sync()  # the context stays usable and the flag was cleared


def test_populations_and_rho_agree():
    p = W.three_level_ring(n_cells=300, n_steps=50)
    _, _, rho, s = gpu_run(p, 50, "fp64", "merged")
    pp = s.populations()
    assert np.abs(pp - pops(rho)).max() < 1e-15
    sub = s.rho(10, 5)
    assert np.array_equal(sub, rho[10:15])
    assert np.abs(np.einsum("cii->c", rho) - 1).max() < 1e-14


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rotation_terms_against_exact(precision):
    """(sin x, cos x - 1) as the kernels evaluate them (series for |x| <= 1/8,
    half-angle library sincos above) against 50-digit values, within a few
    units in the last place of the kernel's precision."""
    import mpmath
    from paper_1710_09799_gb300 import mln
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-0.125, 0.125, 3000), rng.uniform(-3, 3, 2000),
                        10.0 ** rng.uniform(-12, -1, 1000) * rng.choice([-1, 1], 1000),
                        [0.0, 0.125, -0.125, 0.12500001, 1e-300, 50.0]])
    if precision == "fp32":
        x = x.astype(np.float32).astype(np.float64)
    s, c1 = mln.mln_rotation_terms(precision, x)
    eps = np.finfo(np.float64 if precision == "fp64" else np.float32).eps
    with mpmath.workdps(50):
        ref_s = np.array([float(mpmath.sin(mpmath.mpf(v))) for v in x])
        ref_c = np.array([float(-2 * mpmath.sin(mpmath.mpf(v) / 2) ** 2) for v in x])
    tol_s = 6 * eps * np.maximum(np.abs(ref_s), np.finfo(float).tiny)
    tol_c = 6 * eps * np.maximum(np.abs(ref_c), np.finfo(float).tiny)
    assert np.all(np.abs(s - ref_s) <= tol_s), np.max(np.abs(s - ref_s) / np.maximum(np.abs(ref_s), 1e-300))
    assert np.all(np.abs(c1 - ref_c) <= tol_c), np.max(np.abs(c1 - ref_c) / np.maximum(np.abs(ref_c), 1e-300))


@pytest.mark.parametrize("N", [2, 3, 6])
@pytest.mark.parametrize("precision,kernel", [("fp64", "sparse"), ("fp64", "jit"), ("fp32", "jit")])
def test_cell_models_agree_bitwise(N, precision, kernel):
    """The shared-memory sparse and the run-time compiled cell models skip the
    exact zeros of the constant matrices but sum the other terms in the dense
    order: merged-form results are bit-identical to the register model's."""
    if N == 2:
        p = W.two_level_sit(n_cells=700, medium=(100, 600), n_steps=400)
    elif N == 3:
        p = W.three_level_ring(n_cells=3000, n_steps=300)
    else:
        p = W.six_level_pulse(n_cells=600, n_steps=200, t0=15e-15, fwhm=10e-15)
    E0, H0, r0, _ = gpu_run(p, p.n_steps, precision, "merged", kernel="register")
    E1, H1, r1, _ = gpu_run(p, p.n_steps, precision, "merged", kernel=kernel)
    assert np.array_equal(E0, E1) and np.array_equal(H0, H1) and np.array_equal(r0, r1)


def test_six_level_fp32_error_4096_cells(orc):
    """The six-level workload (D = 35) in FP32 with FP64 set-up against the FP64
    oracle on a separate 4096-cell run with the same parameters (a subgrid of
    the 1048576-cell run is not self-contained: its light cone is too wide)."""
    p = W.six_level_pulse(n_cells=4096, n_steps=1000)
    ref = oracle_ref(orc, p, p.n_steps)
    for form in ("merged", "rotated"):
        E, H, rho, _ = gpu_run(p, p.n_steps, "fp32", form)
        e_err = rel_inf(E, ref.E)
        p_err = np.abs(pops(rho) - pops(ref.rho)).max()
        print(f"fp32 six-level {form}: E rel {e_err:.3e}  pop abs {p_err:.3e}")
        assert_fp32("six_level", p.n_steps, e_err, p_err)


@pytest.mark.parametrize("form", ["merged", "strang", "rotated"])
@pytest.mark.parametrize("make", [lambda: W.three_level_ring(n_cells=256, n_steps=1),
                                  lambda: W.multi_level_ring(4, n_cells=256, n_steps=1, seed=2),
                                  lambda: W.two_level_sit(n_cells=200, medium=(50, 150), n_steps=1)])
def test_work_count_is_the_exact_operation_count(make, form):
    """The roofline's algorithmic flops (mln_work_per_step), recounted here from
    the set-up matrices: a product row of k non-zero entries is k
    multiplications and k - 1 additions, k additions when added onto a vector,
    one more for a non-zero offset; the N - 1 angle series (8), the other
    planes by the subtraction formulas (10) and 6 per plane increment; in the
    rotated basis one addition per plane coordinate for z'' = z + dz."""
    from paper_1710_09799_gb300 import mln
    from helpers import params_of
    p = make()
    s = mln.mln_setup_host(params_of(p, precision="fp64", form=form))
    N, D, q = s["N"], s["D"], s["q"]
    P = 2 * q
    T, C1, A0 = np.array(s["T"]), np.array(s["C1"]), np.array(s["A0"])
    b, w, c = np.array(s["b"]), np.array(s["w"]), s["c"]
    nz = lambda a: int(np.count_nonzero(a))
    nT = nz(T[:, :P])
    tt = 2 * nT - sum(bool(np.any(T[:, k] != 0)) for k in range(P))
    rot = 6 * q + 10 * (q - (N - 1)) + 8 * (N - 1)
    dot = lambda v, c0: (2 * nz(v) - 1 + (c0 != 0)) if nz(v) else 0
    if form == "merged":
        b2, wm, cm = A0 @ b + b, A0.T @ w, w @ b + c
        want = tt + rot + 2 * nT + dot(wm, cm) + 2 * nz(C1) + nz(b2)
    elif form == "rotated":
        b2, wm, cm = A0 @ b + b, A0.T @ w, w @ b + c
        want = P + rot + dot(T.T @ wm, cm) + 2 * nz(T.T @ C1 @ T) + nz(T.T @ b2)
    else:
        half = 2 * nz(A0 - np.eye(D)) + nz(b)
        want = 2 * half + tt + rot + 2 * nT + dot(w, c)
    sol = make_solver(p, "fp64", form)
    f_med, f_cell, _, _ = sol.work_per_step
    sol.close()
    assert f_med == want and f_cell == 9.0, (f_med, want)


@pytest.mark.parametrize("precision,kernel", [("fp64", "auto"), ("fp64", "jit"), ("fp32", "auto"),
                                              ("fp32", "register")])
def test_torch_kernel_between_steps_is_ordered(precision, kernel):
    """The step kernels are launched with a programmatic dependency on the
    kernel before them in the stream and wait for that grid before they touch
    the fields: a torch kernel that halves E on the context's stream between
    two mln_step calls acts before the second call, exactly as the same halved
    field copied in from the host does."""
    p = W.three_level_ring(n_cells=2000, n_steps=78)
    a = make_solver(p, precision, "merged", kernel=kernel)
    b = make_solver(p, precision, "merged", kernel=kernel)
    for s in (a, b):
        s.step(37)
    a.E.mul_(0.5)  # on the context's stream, right behind the step kernels
    b.sync()
    b.E.copy_(b.E.cpu() * 0.5)
    for s in (a, b):
        s.step(41)
        s.sync()
    Ea, Ha = a.fields()
    Eb, Hb = b.fields()
    assert np.abs(Ea).max() > 0
    assert np.array_equal(Ea, Eb) and np.array_equal(Ha, Hb) and np.array_equal(a.rho(), b.rho())
    a.close()
    b.close()


def test_rotated_form_six_level_costs_fewer_flops_and_agrees_with_merged():
    """The rotated basis replaces the merged form's three products (T^T, T and
    A0^2 - I) by one dense C z: 2750 against 6919 flops per medium cell update
    on the six-level model. The two forms compute the same step: FP64 results
    agree to rounding after 300 steps."""
    p = W.six_level_pulse(n_cells=600, n_steps=300, t0=15e-15, fwhm=10e-15)
    a = gpu_run(p, p.n_steps, "fp64", "merged", kernel="jit")
    b = gpu_run(p, p.n_steps, "fp64", "rotated")
    fa, fb = a[3].work_per_step[0], b[3].work_per_step[0]
    assert b[3].kernel_in_use == "jit"
    a[3].close()
    b[3].close()
    assert fb < 0.45 * fa, (fa, fb)
    assert rel_inf(b[0], a[0]) < 1e-11
    assert np.abs(b[2] - a[2]).max() < 1e-11



@pytest.mark.parametrize("precision,form,maxwell,N,want", [
    ("fp64", "merged", "fdtd", 3, "jit"),        # the run-time compiled model (NVRTC on the GPU machine)
    ("fp64", "merged", "pstd", 3, "sparse"),     # PSTD takes the sparse model
    ("fp64", "strang", "fdtd", 3, "register"),
    ("fp32", "merged", "fdtd", 3, "jit"),
    ("fp32", "merged", "fdtd", 6, "tensor"),
    ("fp32", "rotated", "fdtd", 6, "tensor"),
    ("fp64", "rotated", "fdtd", 6, "jit"),
])
def test_auto_cell_model_choice(precision, form, maxwell, N, want):
    """MLN_KERNEL_AUTO's choice per precision, form, field solver and N (the
    models give the same bits where they overlap; the choice is the faster)."""
    if N == 3:
        p = W.three_level_ring(n_cells=1024, n_steps=10) if maxwell == "fdtd" else W.three_level_ring_pstd(
            n_cells=1024, n_steps=10)
    else:
        p = W.six_level_pulse(n_cells=600, n_steps=10, t0=15e-15, fwhm=10e-15)
    s = make_solver(p, precision, form)
    assert s.kernel_in_use == want
    s.step(2)
    s.sync()
    s.close()

"""Tensor-core cell model of the rotated basis (MLN_FORM_ROTATED with
MLN_KERNEL_TENSOR): one dense (D + 1) x (D + 1) product per step (the increment
of z and dP/dt from [z'' ; 1], Eqs. 17, 23, 25-26) on tcgen05 MMAs of kind::f16
with FP16 hi/lo operands and power-of-two scales, FP32 state, N = 5 and 6.

* the product path alone (mln_tc_product_f16) against FP64 numpy, with rows
  of B spanning many orders of magnitude (the per-row scales) and a bound
  that a single FP16 product, a transposed operand or a wrong half of a
  packed column misses;
* six-level and five-level runs against the FP64 oracle at the FP32
  tolerance, and against the CUDA-core rotated-basis kernel;
* the result does not depend on the launch shape, including a last tile made
  of the Mur cell alone; the autotuner leaves the state untouched.
"""
import numpy as np
import pytest

import workloads as W
from helpers import assert_fp32, gpu_run, params_of, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


def pops(rho):
    return np.einsum("cii->ci", rho).real


@pytest.mark.parametrize("n", [48, 32, 16])
def test_f16_product_path_against_fp64(n):
    from paper_1710_09799_gb300 import mln
    rng = np.random.default_rng(n)
    A = rng.normal(size=(128, n)).astype(np.float32)
    # rows of B from 1e-9 to 1e9 in magnitude, entries within a row over 1e4
    B = rng.normal(size=(n, n)) * 10.0 ** rng.uniform(-2, 2, size=(n, n))
    B *= 10.0 ** rng.uniform(-9, 9, size=(n, 1))
    C = mln.mln_tc_product_f16(A, B).astype(np.float64)
    ref = A.astype(np.float64) @ B.T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).T
    rel = np.abs(C - ref) / scale
    # hi*hi + hi*lo + lo*hi of 11-bit halves: a few units of 2^-22 of sum |a||b|
    assert rel.max() <= 2.0 ** -19, float(rel.max())
    # one FP16 product alone is off by ~2^-11 relative: the bound tells them apart
    f16 = lambda x: np.asarray(x, dtype=np.float16).astype(np.float64)
    sa = 2.0 ** (13 - np.ceil(np.log2(np.abs(A).max())))
    sb = 2.0 ** (13 - np.ceil(np.log2(np.abs(B).max(axis=1, keepdims=True))))
    hi_only = (f16(A * sa) @ f16(B * sb).T) / sa / sb.T
    assert (np.abs(hi_only - ref) / scale).max() > 2.0 ** -16


def test_six_level_against_oracle(orc):
    p = W.six_level_pulse(n_cells=4096, n_steps=1000)
    st, _ = orc.run(p, n_steps=p.n_steps)
    E, H, rho, s = gpu_run(p, p.n_steps, "fp32", "rotated")  # AUTO picks the tensor cores here
    assert s.kernel_in_use == "tensor"
    e_err = rel_inf(E, st.E)
    p_err = np.abs(pops(rho) - pops(st.rho)).max()
    print(f"tensor rotated six-level: E rel {e_err:.3e}  pop abs {p_err:.3e}")
    assert_fp32("six_level", p.n_steps, e_err, p_err)


@pytest.mark.parametrize("kernel", ["jit", "tensor"])
def test_five_level_ring_against_oracle(orc, kernel):
    """The rotated basis on a ring (diagonal H0, real dipoles) carries a larger
    FP32 error than the merged form whichever kernel runs it: every rotated
    coordinate mixes population-sized components into dP/dt and into the
    populations read back."""
    p = W.multi_level_ring(5, n_cells=1000, n_steps=500, seed=3)
    st, _ = orc.run(p, n_steps=p.n_steps)
    E, H, rho, s = gpu_run(p, p.n_steps, "fp32", "rotated", kernel=kernel)
    assert s.kernel_in_use == kernel
    e_err = rel_inf(E, st.E)
    p_err = np.abs(pops(rho) - pops(st.rho)).max()
    print(f"{kernel} rotated five-level ring: E rel {e_err:.3e}  pop abs {p_err:.3e}")
    assert_fp32("five_level_ring_rotated", p.n_steps, e_err, p_err)


def test_close_to_cuda_core_rotated_kernel():
    p = W.six_level_pulse(n_cells=600, n_steps=200, t0=15e-15, fwhm=10e-15)
    E0, H0, r0, s0 = gpu_run(p, p.n_steps, "fp32", "rotated", kernel="jit")
    E1, H1, r1, s1 = gpu_run(p, p.n_steps, "fp32", "rotated", kernel="tensor")
    assert (s0.kernel_in_use, s1.kernel_in_use) == ("jit", "tensor")
    assert np.abs(E0).max() > 1e5  # the pulse is on the grid
    assert rel_inf(E1, E0) < 1e-5 and np.abs(r1 - r0).max() < 1e-5


def test_launch_shape_does_not_change_the_bits():
    p = W.six_level_pulse(n_cells=1500, n_steps=96, t0=15e-15, fwhm=10e-15)
    ref = gpu_run(p, p.n_steps, "fp32", "rotated", kernel="tensor", block_steps=8)
    for bs, chunks in [(1, None), (5, [7, 40, 49]), (32, None)]:
        out = gpu_run(p, p.n_steps, "fp32", "rotated", kernel="tensor", block_steps=bs, chunks=chunks)
        for a, b in zip(out[:3], ref[:3]):
            assert np.array_equal(a, b), bs


def test_tile_made_of_the_mur_cell_alone():
    """337 cells and 8 steps per launch (tiles of 112 rows): the last tile is
    the Mur cell alone; the bits match a shape whose tiles never start there
    (4 steps, tiles of 120), after the pulse has reached the boundary."""
    p = W.six_level_pulse(n_cells=337, n_steps=800, t0=15e-15, fwhm=10e-15)
    assert (p.n_cells - 1) % 112 == 0 and (p.n_cells - 1) % 120 != 0
    a = gpu_run(p, p.n_steps, "fp32", "rotated", kernel="tensor", block_steps=8)
    b = gpu_run(p, p.n_steps, "fp32", "rotated", kernel="tensor", block_steps=4)
    assert np.abs(b[0][-5:]).max() > 0.0
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


def test_autotune_keeps_state():
    from paper_1710_09799_gb300 import mln
    p = W.six_level_pulse(n_cells=3000, n_steps=40, t0=15e-15, fwhm=10e-15)
    s = mln.Solver(params_of(p, precision="fp32", form="rotated", kernel="tensor"), E0=p.e_init())
    before = s.save()
    K, tile = s.autotune(2)
    after = s.save()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert 1 <= K <= 32 and tile == 128 - 2 * K
    s.close()


@pytest.mark.parametrize("case", ["fp64", "n4", "pstd"])
def test_invalid_parameters(case):
    from paper_1710_09799_gb300 import mln
    p = W.six_level_pulse(n_cells=256, n_steps=10)
    kw = dict(precision="fp32", form="rotated", kernel="tensor")
    if case == "fp64":
        kw["precision"] = "fp64"
    elif case == "pstd":
        p = W.multi_level_ring(5, n_cells=256, n_steps=10, seed=1)
        kw["maxwell"] = "pstd"
    else:
        p = W.multi_level_ring(4, n_cells=256, n_steps=10, seed=1)
    with pytest.raises(mln.MLNError) as e:
        mln.Solver(params_of(p, **kw), E0=p.e_init())
    assert e.value.status in (mln.MLN_EINVAL, mln.MLN_EUNSUPPORTED)

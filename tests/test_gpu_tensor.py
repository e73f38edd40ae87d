"""Tensor-core cell model (MLN_KERNEL_TENSOR): the dense products of the
merged step (Eqs. 23, 25-26, 17), regrouped into two per step, on tcgen05
MMAs with 3 x TF32 operands, FP32 state, for N = 5 and 6.

* the product path alone (mln_tc_product, A from tensor memory as for y and
  from shared memory as for dz) against FP64 numpy, with a bound that a
  single TF32 product (or a transposed or mis-laid operand) misses;
* six-level runs against the FP64 oracle at the FP32 tolerance, and against
  the FP32 register model;
* a five-level periodic ring against the oracle;
* the result does not depend on the launch shape (steps fused per launch,
  chunking of the steps): each cell's row of the MMA is computed alone;
* input validation;
* failure detection: the bounded completion wait, made to run out (the MMA
  left out), is reported as MLN_ETIMEOUT and the device keeps working.
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


def tf32(x):
    """Round to TF32 (nearest, ties away from zero) as the split does."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


@pytest.mark.parametrize("a_in_tmem", [True, False])
@pytest.mark.parametrize("nc,kc", [(32, 40), (48, 32), (48, 40), (32, 24), (16, 8)])
def test_product_path_against_fp64(nc, kc, a_in_tmem):
    from paper_1710_09799_gb300 import mln
    rng = np.random.default_rng(nc * 100 + kc)
    A = rng.normal(size=(128, kc)).astype(np.float32)
    B = rng.normal(size=(nc, kc))
    C = mln.mln_tc_product(A, B, a_in_tmem)
    ref = A.astype(np.float64) @ B.T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).T
    err = np.abs(C - ref)
    # 3 x TF32 with FP32 accumulation: a few units of 2^-21 of sum |a||b|
    assert np.all(err <= 2.0 ** -19 * scale), float((err / scale).max())
    # a single TF32 product is off by ~2^-11 relative: the bound tells them apart
    hi_only = tf32(A).astype(np.float64) @ tf32(B.astype(np.float32)).astype(np.float64).T
    assert np.abs(hi_only - ref).max() > 2.0 ** -16 * scale.max()


def test_six_level_against_oracle(orc):
    kernel = "tensor"
    p = W.six_level_pulse(n_cells=4096, n_steps=1000)
    st, _ = orc.run(p, n_steps=p.n_steps)
    E, H, rho, s = gpu_run(p, p.n_steps, "fp32", "merged", kernel=kernel)
    assert s.kernel_in_use == kernel
    e_err = rel_inf(E, st.E)
    p_err = np.abs(pops(rho) - pops(st.rho)).max()
    print(f"tensor ({kernel}) six-level: E rel {e_err:.3e}  pop abs {p_err:.3e}")
    assert_fp32("six_level", p.n_steps, e_err, p_err)


def test_six_level_close_to_fp32_register_model():
    kernel = "tensor"
    p = W.six_level_pulse(n_cells=600, n_steps=200, t0=15e-15, fwhm=10e-15)
    E0, H0, r0, _ = gpu_run(p, p.n_steps, "fp32", "merged", kernel="register")
    E1, H1, r1, _ = gpu_run(p, p.n_steps, "fp32", "merged", kernel=kernel)
    assert rel_inf(E1, E0) < 1e-4 and np.abs(r1 - r0).max() < 1e-5


def test_five_level_ring_against_oracle(orc):
    kernel = "tensor"
    p = W.multi_level_ring(5, n_cells=1000, n_steps=500, seed=3)
    st, _ = orc.run(p, n_steps=p.n_steps)
    E, H, rho, _ = gpu_run(p, p.n_steps, "fp32", "merged", kernel=kernel)
    e_err = rel_inf(E, st.E)
    p_err = np.abs(pops(rho) - pops(st.rho)).max()
    print(f"tensor ({kernel}) five-level ring: E rel {e_err:.3e}  pop abs {p_err:.3e}")
    assert_fp32("five_level_ring", p.n_steps, e_err, p_err)


def test_launch_shape_does_not_change_the_bits():
    p = W.six_level_pulse(n_cells=1500, n_steps=96, t0=15e-15, fwhm=10e-15)
    ref = gpu_run(p, p.n_steps, "fp32", "merged", kernel="tensor", block_steps=8)
    for bs, chunks in [(1, None), (5, [7, 40, 49]), (32, None)]:
        out = gpu_run(p, p.n_steps, "fp32", "merged", kernel="tensor", block_steps=bs, chunks=chunks)
        for a, b in zip(out[:3], ref[:3]):
            assert np.array_equal(a, b), bs


def test_tile_made_of_the_mur_cell_alone():
    """337 cells and 8 steps per launch (tiles of 112 rows): the last tile is
    the Mur cell alone, whose value comes from its left neighbour's row in the
    same step; the bits match a shape whose tiles never start there (4 steps,
    tiles of 120), after the pulse has reached the boundary."""
    p = W.six_level_pulse(n_cells=337, n_steps=800, t0=15e-15, fwhm=10e-15)
    assert (p.n_cells - 1) % 112 == 0 and (p.n_cells - 1) % 120 != 0
    a = gpu_run(p, p.n_steps, "fp32", "merged", kernel="tensor", block_steps=8)
    b = gpu_run(p, p.n_steps, "fp32", "merged", kernel="tensor", block_steps=4)
    assert np.abs(b[0][-5:]).max() > 0.0
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


def test_autotune_keeps_state():
    from paper_1710_09799_gb300 import mln
    p = W.six_level_pulse(n_cells=3000, n_steps=40, t0=15e-15, fwhm=10e-15)
    s = mln.Solver(params_of(p, precision="fp32", form="merged", kernel="tensor"), E0=p.e_init())
    before = s.save()
    K, tile = s.autotune(2)
    after = s.save()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert 1 <= K <= 32 and tile == 128 - 2 * K
    assert s.launch_shape[2] == 512
    s.close()


@pytest.mark.parametrize("case", ["fp64", "strang", "n3", "block_steps"])
def test_invalid_parameters(case):
    from paper_1710_09799_gb300 import mln
    p = W.six_level_pulse(n_cells=256, n_steps=10)
    kw = dict(precision="fp32", form="merged", kernel="tensor")
    if case == "fp64":
        kw["precision"] = "fp64"
    elif case == "strang":
        kw["form"] = "strang"
    elif case == "block_steps":
        kw["block_steps"] = 40
    else:
        p = W.three_level_ring(n_cells=256)
    with pytest.raises(mln.MLNError) as e:
        mln.Solver(params_of(p, **kw), E0=p.e_init())
    assert e.value.status == mln.MLN_EINVAL


def test_completion_wait_runs_out_and_is_reported():
    """The product kernel with its MMA left out: nothing arrives on the
    completion mbarrier, the bounded wait gives up, the kernel frees its tensor
    memory and returns, and the host reports MLN_ETIMEOUT. A normal product on
    the same device right after is exact to the 3 x TF32 bound."""
    import time
    from paper_1710_09799_gb300 import mln
    t0 = time.perf_counter()
    status = mln.lib().mln_tc_wait_selftest()
    waited = time.perf_counter() - t0
    print(f"bounded wait gave up after {waited:.3f} s")
    assert status == mln.MLN_ETIMEOUT, status
    assert "timed out" in mln.lib().mln_create_error().decode()
    rng = np.random.default_rng(7)
    A = rng.normal(size=(128, 8)).astype(np.float32)
    B = rng.normal(size=(16, 8))
    C = mln.mln_tc_product(A, B, True)
    ref = A.astype(np.float64) @ B.T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).T
    assert np.all(np.abs(C - ref) <= 2.0 ** -19 * scale)

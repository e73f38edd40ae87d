"""Batched grids (mln_batch_*): many independent grids of mixed N, lengths and
boundaries, one launch per N for every group of fused steps, replayed from a CUDA graph.

Every cell of every grid does the same arithmetic as in a single-grid run, so
the batch must reproduce the single-grid results bit for bit; one grid is
also checked against the oracle directly.
"""
import numpy as np
import pytest

import workloads as W
from helpers import make_solver, params_of, rel_inf, src_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


def make_batch(devs, precision, n_steps, kernel="auto"):
    from paper_1710_09799_gb300 import mln
    pars = [params_of(p, precision=precision, form="merged", kernel=kernel) for p in devs]
    srcs = [p.source_samples(0, n_steps) for p in devs]
    has = any(s is not None for s in srcs)
    return mln.Batch(pars, [p.e_init() for p in devs], srcs if has else None, n_steps if has else 0)


def single(p, precision, n_steps):
    s = make_solver(p, precision, "merged", kernel="register")
    s.step(n_steps, src_tensor(p, 0, n_steps))
    s.sync()
    E, H = s.fields()
    return E, H, s.rho()


@pytest.mark.parametrize("kernel", ["jit", "register"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_single_grids_bitwise(precision, kernel):
    """Both batched cell models (run-time compiled over the union sparsity
    pattern, and dense products over padded constants) give the single-grid
    register model's bits."""
    devs = W.batched_devices(count=7, n_steps=260, seed=3, min_cells=100, max_cells=3000)
    assert {p.N for p in devs} == {2, 3, 4}
    b = make_batch(devs, precision, 260, kernel)
    for N in (2, 3, 4):
        assert b.kernel_in_use(N) == kernel
    b.step(130)
    b.step(130)
    b.sync()
    for i, p in enumerate(devs):
        E1, H1 = b.fields(i)
        E0, H0, r0 = single(p, precision, 260)
        assert np.array_equal(E0, E1) and np.array_equal(H0, H1), (i, p.name)
        assert np.array_equal(r0, b.rho(i)), (i, p.name)
    b.close()


def test_batch_graph_replay_and_autotune_without_sources():
    devs = [W.three_level_ring(n_cells=900, seed=5), W.multi_level_ring(4, n_cells=2500, n_steps=0, seed=6),
            W.three_level_ring(n_cells=77, seed=7)]
    b = make_batch(devs, "fp64", 0)
    K, tile = b.autotune(2)
    assert 1 <= K <= 64 and tile >= 1
    for _ in range(3):
        b.step(50)  # the second and third calls replay the captured graph
    b.sync()
    assert b.shape[3] >= 3
    for i, p in enumerate(devs):
        E1, _ = b.fields(i)
        E0, _, r0 = single(p, "fp64", 150)
        assert np.array_equal(E0, E1)
        assert np.array_equal(r0, b.rho(i))
    b.close()


def test_batch_grid_against_oracle(orc):
    p = W.multi_level_ring(4, n_cells=1500, n_steps=400, seed=11)
    q = W.two_level_sit(n_cells=800, medium=(200, 600), n_steps=400)
    b = make_batch([p, q], "fp64", 400)
    b.step(400)
    b.sync()
    for i, prob in enumerate((p, q)):
        ref, _ = orc.run(prob, n_steps=400)
        E, _ = b.fields(i)
        assert rel_inf(E, ref.E) < 1e-10
        assert np.abs(b.rho(i) - ref.rho).max() < 1e-10
    b.close()


def test_batch_rejects_mixed_precision_and_large_N():
    from paper_1710_09799_gb300 import mln
    a = W.three_level_ring(n_cells=64)
    c = W.six_level_pulse(n_cells=64, n_steps=10)
    with pytest.raises(mln.MLNError):
        mln.Batch([params_of(a, precision="fp64", form="merged"), params_of(a, precision="fp32", form="merged")],
                  [a.e_init(), a.e_init()])
    with pytest.raises(mln.MLNError):
        mln.Batch([params_of(c, precision="fp32", form="merged")], [c.e_init()])

"""The persistent launch of a batch (mln_batch_set_launch, MLN_BATCH_PERSISTENT):
one launch per call and N, (chunk, tile) items taken from a device counter,
each tile waiting for the tiles within its halo + 1 cells to finish the
previous chunk.

Each tile's chunk does the same arithmetic on the same inputs as in the
chunked launches, so the results must be the single-grid bits. The grids are
chosen so that the waits matter: a ring whose last tile is shorter than the
halo (the tile beyond it must be waited for too), a ring of one tile, an open
grid whose last tile is the Mur cell alone, and step counts that leave a
short last chunk and an odd number of chunks. The wait limit is checked with
a limit of 0 polls, which gives up at every wait of a chunk after the first.
"""
import numpy as np
import pytest

import workloads as W
from helpers import make_solver, params_of, src_tensor

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
    rho = s.rho()
    s.close()
    return E, H, rho


def default_shape():
    """(steps per launch, tile) of a batch before autotuning."""
    b = make_batch([W.three_level_ring(n_cells=64, seed=1)], "fp64", 0)
    K, tile, _, _ = b.shape
    b.close()
    return K, tile


def edge_devices(tile):
    """Grids whose tiling makes the waits non-trivial at this tile length."""
    return [W.three_level_ring(n_cells=2 * tile + 3, seed=21),        # last tile 3 cells < halo
            W.three_level_ring(n_cells=tile - 20, seed=22),           # a ring of one tile
            W.multi_level_ring(4, n_cells=3 * tile + 9, n_steps=0, seed=23),
            W.two_level_sit(n_cells=3 * tile + 1, medium=(tile, 2 * tile + 50), n_steps=400, tau=2e-15,
                            t0=6e-15)]                                # last tile: the Mur cell alone


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_persistent_gives_the_single_grid_bits(precision):
    K, tile = default_shape()
    assert tile >= K + 2 and K > 3  # the 3-cell last tile is shorter than the halo
    devs = edge_devices(tile) + W.batched_devices(count=6, n_steps=400, seed=9, min_cells=100, max_cells=4000)
    b = make_batch(devs, precision, 400)
    assert b.shape[:2] == (K, tile)
    assert b.launch == "chunks"
    b.set_launch("persistent")
    assert b.launch == "persistent"
    launches0 = b.shape[3]
    b.step(8 * K + 7)  # 9 chunks, the last of 7 steps: the result ends in the second buffer set
    b.step(400 - (8 * K + 7))
    b.sync()
    # one launch per call and N present
    assert b.shape[3] - launches0 == 2 * len({p.N for p in devs})
    for i, p in enumerate(devs):
        E1, H1 = b.fields(i)
        E0, H0, r0 = single(p, precision, 400)
        assert np.array_equal(E0, E1) and np.array_equal(H0, H1), (i, p.name)
        assert np.array_equal(r0, b.rho(i)), (i, p.name)
    b.close()


def test_persistent_after_autotune_and_back_to_chunks():
    """Autotuned shape (tiles of at least K + 2 cells), a persistent call, then
    a chunked call on the same batch: the single-grid bits throughout."""
    devs = edge_devices(default_shape()[1])[:3] + W.batched_devices(count=5, n_steps=0, seed=4, min_cells=300, max_cells=5000)
    devs = [p for p in devs if p.source_samples(0, 1) is None]
    b = make_batch(devs, "fp64", 0)
    K, tile = b.autotune(2)
    assert tile >= K + 2
    b.set_launch("persistent")
    b.step(3 * K + 1)
    b.set_launch("chunks")
    b.step(2 * K - 1)
    b.sync()
    for i, p in enumerate(devs):
        E1, _ = b.fields(i)
        E0, _, r0 = single(p, "fp64", 5 * K)
        assert np.array_equal(E0, E1), (i, p.name)
        assert np.array_equal(r0, b.rho(i)), (i, p.name)
    b.close()


def test_wait_limit_zero_reports_a_timeout():
    """A limit of 0 polls gives up at each wait after the first chunk: the
    kernel ends, flags the grids, and the next sync returns MLN_ETIMEOUT;
    the flag is cleared and a run with the default limit is clean again."""
    from paper_1710_09799_gb300 import mln
    devs = edge_devices(default_shape()[1])[:3]
    b = make_batch(devs, "fp32", 0)
    b.set_launch("persistent", wait_limit=0)
    b.step(64)
    with pytest.raises(mln.MLNError) as ei:
        b.sync()
    assert ei.value.status == mln.MLN_ETIMEOUT
    assert "gave up waiting for a neighbouring tile" in str(ei.value)
    b.set_launch("persistent")
    b.step(64)
    b.sync()
    b.close()


def test_persistent_refusals():
    from paper_1710_09799_gb300 import mln
    devs = edge_devices(default_shape()[1])[:2]
    b = make_batch(devs, "fp64", 0, kernel="register")  # no run-time compiled kernels
    with pytest.raises(mln.MLNError) as ei:
        b.set_launch("persistent")
    assert ei.value.status == mln.MLN_EUNSUPPORTED
    with pytest.raises(mln.MLNError) as ei:
        mln.mln_batch_set_launch(b.b, 7, 10)
    assert ei.value.status == mln.MLN_EINVAL
    with pytest.raises(mln.MLNError) as ei:
        mln.mln_batch_set_launch(b.b, mln.MLN_BATCH_CHUNKS, -1)
    assert ei.value.status == mln.MLN_EINVAL
    b.close()

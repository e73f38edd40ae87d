"""mln_step_noalloc, the step for callers that cannot allocate device memory.

Callers such as a host application whose device memory belongs to its own
pool, or a plug-in that must not grow the device footprint, cannot use
mln_create (it allocates the second copy of the state and fields). They call
mln_step_noalloc, which keeps that copy in a fixed device array of the
library. This checks it through the C-ABI against mln_create / mln_step with
the same kernel, on two calls in a row, and that an oversized problem is
refused with a message. This file sorts last so that a run stopping at the
first failure has run every other test before it.
"""
import numpy as np
import pytest

import workloads as W
from helpers import make_solver, params_of, rel_inf

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


def sit_grid():
    """Open two-level grid: sech pulse as a hard source at cell 0, Mur at the
    right end (reached within the run), medium in the middle half."""
    return W.two_level_sit(n_cells=600, medium=(150, 450), n_steps=1400, tau=2e-15, t0=6e-15)


CASES = [("ring", "fp64", "merged"), ("ring", "fp64", "strang"), ("ring", "fp32", "merged"),
         ("sit", "fp64", "merged"), ("sit", "fp32", "merged")]


@pytest.mark.parametrize("grid,precision,form", CASES)
def test_noalloc_matches_mln_step_on_two_calls(grid, precision, form):
    import torch
    from paper_1710_09799_gb300 import mln
    p = W.three_level_ring(n_cells=4096) if grid == "ring" else sit_grid()
    par = params_of(p, precision=precision, form=form, kernel="register")
    dt = torch.float64 if precision == "fp64" else torch.float32
    # tolerance of the other GPU tests: 1e-10 in FP64; in FP32 both calls run the
    # same kernel at the same launch shape, so the bits agree as well
    tol = TOL if precision == "fp64" else 0.0

    # the existing entry point
    ref = make_solver(p, precision, form, kernel="register")
    # caller-owned buffers for the allocation-free call
    sb, fb = mln.mln_query_buffers(par)
    state = torch.zeros(sb // (8 if precision == "fp64" else 4), dtype=dt, device="cuda")
    E = torch.as_tensor(p.e_init(), dtype=dt, device="cuda").clone()
    H = torch.zeros(p.n_cells, dtype=dt, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    done = 0
    for i, n in enumerate((700, 701) if grid == "sit" else (300, 301)):
        src = p.source_samples(done, n)
        src_t = None if src is None else torch.as_tensor(src, dtype=torch.float64, device="cuda")
        ref.step(n, src_t)
        ref.sync()
        mln.mln_step_noalloc(par, state.data_ptr(), E.data_ptr(), H.data_ptr(), i == 0, n,
                             None if src_t is None else src_t.data_ptr(), stream)
        torch.cuda.synchronize()
        done += n
        E_ref, H_ref = ref.fields()
        assert rel_inf(E.cpu().double().numpy(), E_ref) <= tol
        assert rel_inf(H.cpu().double().numpy(), H_ref) <= tol
        s_ref = ref.state.cpu().double().numpy()
        D, stride = p.D, ref.stride
        a = state.cpu().double().numpy().reshape(D, stride)[:, :p.n_medium]
        b = s_ref.reshape(D, stride)[:, :p.n_medium]
        assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1.0)
    if grid == "sit":
        assert np.abs(E_ref[-3:]).max() > 0  # the pulse has reached the Mur end
    ref.close()


def test_noalloc_rejects_other_kernels():
    """Only the register model runs here: a request for another cell model is
    refused rather than silently served by the register model."""
    import torch
    from paper_1710_09799_gb300 import mln
    p = W.three_level_ring(n_cells=256)
    for kernel in ("jit", "sparse"):
        par = params_of(p, precision="fp64", form="merged", kernel=kernel)
        sb, fb = mln.mln_query_buffers(par)
        state = torch.zeros(sb // 8, dtype=torch.float64, device="cuda")
        E = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        H = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        with pytest.raises(mln.MLNError) as ei:
            mln.mln_step_noalloc(par, state.data_ptr(), E.data_ptr(), H.data_ptr(), True, 1, None,
                                 torch.cuda.current_stream().cuda_stream)
        assert ei.value.status == mln.MLN_EINVAL
        assert "register cell model" in str(ei.value)


def test_noalloc_rejects_problems_above_the_scratch_size():
    import torch
    from paper_1710_09799_gb300 import mln
    p = W.three_level_ring(n_cells=3_000_000)  # FP64 state alone is 192 MB
    par = params_of(p, precision="fp64", form="merged", kernel="register")
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(mln.MLNError) as ei:
        mln.mln_step_noalloc(par, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), True, 1, None,
                             torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == mln.MLN_EINVAL
    assert "static maximum" in str(ei.value)

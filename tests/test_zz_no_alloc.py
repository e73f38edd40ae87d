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


@pytest.mark.parametrize("form", ["merged", "strang"])
def test_noalloc_matches_mln_step_on_two_calls(form):
    import torch
    from paper_1710_09799_gb300 import mln
    p = W.three_level_ring(n_cells=4096)
    par = params_of(p, precision="fp64", form=form, kernel="register")

    # the existing entry point
    ref = make_solver(p, "fp64", form, kernel="register")
    # caller-owned buffers for the allocation-free call
    sb, fb = mln.mln_query_buffers(par)
    state = torch.zeros(sb // 8, dtype=torch.float64, device="cuda")
    E = torch.as_tensor(p.e_init(), dtype=torch.float64, device="cuda").clone()
    H = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    for i, n in enumerate((300, 301)):
        ref.step(n)
        ref.sync()
        mln.mln_step_noalloc(par, state.data_ptr(), E.data_ptr(), H.data_ptr(), i == 0, n, None, stream)
        torch.cuda.synchronize()
        E_ref, H_ref = ref.fields()
        assert rel_inf(E.cpu().numpy(), E_ref) < TOL
        assert rel_inf(H.cpu().numpy(), H_ref) < TOL
        s_ref = ref.state.cpu().numpy()
        D, stride = p.D, ref.stride
        a = state.cpu().numpy().reshape(D, stride)[:, :p.n_medium]
        b = s_ref.reshape(D, stride)[:, :p.n_medium]
        assert np.abs(a - b).max() < TOL
    ref.close()


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

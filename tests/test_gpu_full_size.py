"""Full-size workloads in the launch configuration the benchmark times
(autotuned shapes), checked on sampled outputs.

* six-level pulse, 1048576 cells: after S steps the first 200 cells cannot
  see the right boundary (fields move at most one cell per step), so an
  oracle run of the same problem on a grid of 2 S + 200 cells, same source,
  gives them exactly; FP64 and FP32 paths are compared there.
* batched devices, all 256 (4.36e6 cells): sampled devices against
  single-grid runs of the register cell model, bit for bit.
"""
import numpy as np
import pytest

import workloads as W
from helpers import assert_fp32, make_solver, params_of, rel_inf, src_tensor

pytestmark = pytest.mark.gpu

FP64_E = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1710_09799_gb300 import build
    build()


@pytest.fixture(scope="module")
def six_level_reference(orc):
    p = W.six_level_pulse()
    S, keep = 400, 200
    q = p.with_(n_cells=2 * S + keep, medium_end=2 * S + keep - 1)
    st, _ = orc.run(q, n_steps=S)
    return p, S, keep, st


@pytest.mark.parametrize("precision,kernel,form", [("fp64", "auto", "merged"), ("fp32", "auto", "merged"),
                                                   ("fp32", "tensor", "merged"), ("fp32", "auto", "rotated")])
def test_six_level_full_size_sampled(six_level_reference, precision, kernel, form):
    p, S, keep, ref = six_level_reference
    s = make_solver(p, precision, form, kernel=kernel)
    s.autotune(2)
    s.step(S, src_tensor(p, 0, S))
    s.sync()
    E, _ = s.fields()
    rho = s.rho(0, keep)
    e_err = rel_inf(E[:keep], ref.E[:keep])
    p_err = np.abs(np.einsum("cii->ci", rho - ref.rho[:keep]).real).max()
    print(f"six-level full size {precision}/{form}/{s.kernel_in_use}: E rel {e_err:.3e}  pop abs {p_err:.3e}")
    assert np.abs(ref.E[:keep]).max() > 1e5  # the pulse has entered the compared cells
    if precision == "fp64":
        assert e_err < FP64_E and p_err < FP64_E
    else:
        assert_fp32("six_level", S, e_err, p_err)
    s.close()


def test_batched_full_size_sampled():
    from paper_1710_09799_gb300 import mln
    steps = 64
    devs = W.batched_devices(n_steps=steps)
    pars = [params_of(d, precision="fp32", form="merged") for d in devs]
    b = mln.Batch(pars, [d.e_init() for d in devs], [d.source_samples(0, steps) for d in devs], steps)
    b.autotune(2)
    b.step(steps)
    b.sync()
    sizes = np.array([d.n_cells for d in devs])
    picks = sorted({0, 97, 255, int(sizes.argmax()), int(sizes.argmin())} |
                   {next(i for i, d in enumerate(devs) if d.N == n) for n in (2, 3, 4)})
    for i in picks:
        d = devs[i]
        s = make_solver(d, "fp32", "merged", kernel="register")
        s.step(steps, src_tensor(d, 0, steps))
        s.sync()
        E0, H0 = s.fields()
        E1, H1 = b.fields(i)
        assert np.array_equal(E0, E1) and np.array_equal(H0, H1), (i, d.name)
        assert np.array_equal(s.rho(), b.rho(i)), (i, d.name)
        s.close()
    b.close()

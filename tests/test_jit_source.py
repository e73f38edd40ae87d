"""The run-time compiled cell model: the generated source is valid CUDA for
sm_103a (compiled here with nvcc, no GPU needed), carries only the non-zero
entries of the set-up matrices, and has one literal per such entry."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from helpers import params_of

mln = pytest.importorskip("paper_1710_09799_gb300.mln")


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09799_gb300 import build
    build()
    return mln.lib()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_generated_source_compiles_and_skips_zeros(lib, tmp_path, prec):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    p = W.three_level_ring(n_cells=1000)
    par = params_of(p, precision=prec, form="merged")
    src = mln.mln_kernel_source(par)
    s = mln.mln_setup_host(par)
    D, q = s["D"], s["q"]
    cast = (lambda x: np.float32(x)) if prec == "fp32" else (lambda x: x)
    nnz_T = int(np.count_nonzero(cast(s["T"][:, :2 * q])))
    nnz_C1 = int(np.count_nonzero(cast(s["C1"])))
    body = src[src.index("struct JitCell"):]
    # products: T^T and T each once per non-zero plane entry, C1 once per non-zero entry
    n_terms = body.count("fma(") + body.count("mul_rn(")
    assert n_terms <= 2 * nnz_T + nnz_C1 + D + 1
    assert nnz_T < D * 2 * q and nnz_C1 < D * D  # the ring's structure has zeros to skip
    f = tmp_path / "k.cu"
    f.write_text(src)
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-c", str(f),
                        "-o", str(tmp_path / "k.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]

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


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("N", [2, 3, 4])
def test_batch_source_compiles_and_follows_the_union_pattern(lib, tmp_path, prec, N):
    """The batched kernel of the N-level grids of a batch: one term per entry
    that is non-zero in at least one grid (the union pattern), valid CUDA."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    devs = W.batched_devices(count=12, n_steps=10)
    pars = [params_of(d, precision=prec, form="merged") for d in devs]
    mine = [p for d, p in zip(devs, pars) if d.N == N]
    if not mine:
        pytest.skip("no grid with this N in the sample")
    src = mln.mln_batch_kernel_source(pars, N)
    cast = (lambda x: np.float32(x)) if prec == "fp32" else (lambda x: x)
    union_T = union_C1 = None
    for p in mine:
        s = mln.mln_setup_host(p)
        q = s["q"]
        t = cast(s["T"][:, :2 * q]) != 0
        c = cast(s["C1"]) != 0
        union_T = t if union_T is None else union_T | t
        union_C1 = c if union_C1 is None else union_C1 | c
    D = N * N - 1
    body = src[src.index("struct JitBatchCell"):]
    n_terms = body.count("fma(") + body.count("mul_rn(")
    # T^T and T once per union entry, C1 once per union entry, at most D terms of wm
    assert n_terms <= 2 * int(union_T.sum()) + int(union_C1.sum()) + D
    assert n_terms >= 2 * int(union_T.sum()) + int(union_C1.sum())
    # the chunked and the persistent batch kernels come from the same module
    assert "void __launch_bounds__(kBatchThreads, 1) mln_jit_batch(" in src
    assert "mln_jit_batch_persist(" in src
    f = tmp_path / "b.cu"
    f.write_text(src)
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-c", str(f),
                        "-o", str(tmp_path / "b.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_rotated_form_source_has_one_product(lib, tmp_path, prec):
    """MLN_FORM_ROTATED: the state is z = T^T y, so the generated step takes the
    plane coordinates from the state itself and has no T or T^T product: its
    terms are those of C = T^T (A0^2 - I) T and of T^T A0^T w only."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    p = W.three_level_ring(n_cells=1000)
    par = params_of(p, precision=prec, form="rotated")
    src = mln.mln_kernel_source(par)
    s = mln.mln_setup_host(par)
    D, q = s["D"], s["q"]
    cast = (lambda x: np.float32(x)) if prec == "fp32" else (lambda x: x)
    T, C1 = s["T"], s["C1"]
    nnz_C = int(np.count_nonzero(cast(T.T @ C1 @ T)))
    body = src[src.index("struct JitCell"):]
    n_terms = body.count("fma(") + body.count("mul_rn(")
    assert nnz_C <= n_terms <= nnz_C + D
    for k in range(2 * q):
        assert f"z[{k}] = s[{k}];" in body
    f = tmp_path / "r.cu"
    f.write_text(src)
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-c", str(f),
                        "-o", str(tmp_path / "r.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]


def _hex(x):
    """A C hexadecimal floating literal (an FP32 'f' suffix follows the decimal exponent)."""
    return float.fromhex(x[:-1] if x.endswith("f") else x)


@pytest.mark.parametrize("make", [lambda: W.three_level_ring(n_cells=1000),
                                  lambda: W.multi_level_ring(4, n_cells=256, n_steps=1, seed=2)])
def test_rotated_form_constants_are_the_rotated_matrices(lib, make):
    """The literals of the generated rotated-basis step (FP64) are T^T C1 T with
    C1 = A0^2 - I of the set-up (row i of the next state), T^T (A0 b + b) (its offset) and T^T A0^T w (the
    dP/dt weights), recomputed here with numpy from the set-up's T, A0, b and w:
    a transposed or mis-indexed matrix in the generator fails here."""
    import re
    p = make()
    par = params_of(p, precision="fp64", form="rotated")
    s = mln.mln_setup_host(par)
    D = s["D"]
    T, A0, b, w, C1 = s["T"], s["A0"], s["b"], s["w"], s["C1"]  # C1 = A0^2 - I (set-up, FP64)
    C = T.T @ C1 @ T
    cz = T.T @ (A0 @ b + b)
    wz = T.T @ (A0.T @ w)
    body = mln.mln_kernel_source(par)
    body = body[body.index("struct JitCell"):]
    lit = r"(-?0x[0-9a-fA-Fp.+-]+)"
    got_C = np.zeros((D, D))
    got_c = np.zeros(D)
    for line in body.splitlines():
        m = re.match(r"\s*s\[(\d+)\] = (.*);$", line)
        if m:
            i = int(m.group(1))
            for a, j in re.findall(lit + r", y\[(\d+)\]", m.group(2)):
                got_C[i, int(j)] = _hex(a)
            off = re.search(r"\(y\[\d+\] \+ " + lit + r"\)", m.group(2))
            if off:
                got_c[i] = _hex(off.group(1))
        m = re.match(r"\s*const double dpdt = (.*);$", line)
        if m:
            got_w = np.zeros(D)
            for a, j in re.findall(lit + r", y\[(\d+)\]", m.group(1)):
                got_w[int(j)] = _hex(a)
    # rounding bound of a product of three D x D matrices, entry by entry
    u = np.finfo(float).eps
    aT = np.abs(T)
    assert np.all(np.abs(got_C - C) <= 8 * D * u * (aT.T @ np.abs(C1) @ aT) + 1e-300)
    assert np.all(np.abs(got_c - cz) <= 8 * D * u * (aT.T @ np.abs(A0 @ b + b)) + 1e-300)
    assert np.all(np.abs(got_w - wz) <= 8 * D * u * (aT.T @ np.abs(A0.T @ w)) + 1e-300)
    assert np.count_nonzero(got_C) >= np.count_nonzero(np.abs(C) > 1e-12 * np.abs(C).max())


def test_double_float_source_compiles_with_one_term_per_constant(lib, tmp_path):
    """MLN_KERNEL_DF32: the double-float step has one pair term per non-zero
    entry of T (twice: T^T on the plane rows, T on the plane columns), of C1
    and of wm, and is valid CUDA for sm_103a."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    p = W.three_level_ring(n_cells=1000)
    par = params_of(p, precision="fp64", form="merged", kernel="df32")
    src = mln.mln_kernel_source(par)
    s = mln.mln_setup_host(par)
    D, q = s["D"], s["q"]
    body = src[src.index("struct JitCell"):]
    n_terms = body.count("df_first(") + body.count("df_first1(") + body.count("df_acc(") + body.count("df_acc1(")
    fixed = 2 * int(np.count_nonzero(s["T"][:, :2 * q])) + int(np.count_nonzero(s["C1"]))
    assert fixed <= n_terms <= fixed + D  # + the non-zero entries of wm
    assert "df_rotation_increment<3>" in body and "fma(" not in body.split("df_rotation_increment")[0]
    f = tmp_path / "k.cu"
    f.write_text(src)
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-c", str(f),
                        "-o", str(tmp_path / "k.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]


@pytest.mark.parametrize("kw", [dict(precision="fp32", form="merged"), dict(precision="fp64", form="strang"),
                                dict(precision="fp64", form="rodrigues"), dict(precision="fp32", form="rotated")])
def test_double_float_needs_fp64_merged_or_rotated(lib, kw):
    p = W.three_level_ring(n_cells=1000)
    with pytest.raises(mln.MLNError) as ei:
        mln.mln_kernel_source(params_of(p, kernel="df32", **kw))
    assert ei.value.status == mln.MLN_EINVAL


@pytest.mark.parametrize("N", [2, 3, 4])
def test_double_float_batch_source_compiles(lib, tmp_path, N):
    """The batch kernels of MLN_KERNEL_DF32 grids: pair constants, pair cell
    and field update, valid CUDA for sm_103a."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    devs = W.batched_devices(count=12, n_steps=10)
    pars = [params_of(d, precision="fp64", form="merged", kernel="df32") for d in devs]
    if not any(d.N == N for d in devs):
        pytest.skip(f"no {N}-level grid in the sample")
    src = mln.mln_batch_kernel_source(pars, N)
    assert "using Field = Df;" in src and "Df c[" in src and "df_rotation_increment<%d>" % N in src
    f = tmp_path / "b.cu"
    f.write_text(src)
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-c", str(f),
                        "-o", str(tmp_path / "b.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]


def test_double_float_rotated_source_compiles(lib, tmp_path):
    """MLN_KERNEL_DF32 in the rotated basis (the dense six-level model): one
    pair term per non-zero entry of C1z and wz, blocks of at most 256
    threads, valid CUDA for sm_103a."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    p = W.six_level_pulse(n_cells=600, n_steps=10)
    src = mln.mln_kernel_source(params_of(p, precision="fp64", form="rotated", kernel="df32"))
    body = src[src.index("struct JitCell"):]
    assert "__launch_bounds__(256, 1)" in body and "df_rotation_increment<6>" in body
    n_terms = body.count("df_first(") + body.count("df_first1(") + body.count("df_acc(") + body.count("df_acc1(")
    assert 35 * 35 // 2 < n_terms <= 35 * 35 + 35
    f = tmp_path / "k.cu"
    f.write_text(src)
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-c", str(f),
                        "-o", str(tmp_path / "k.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]


def test_double_float_batch_needs_every_grid_on_pairs(lib):
    """mln_batch_create takes MLN_KERNEL_DF32 only for FP64 batches whose every
    grid asks for it; the check comes before any device work (the buffer
    pointers below are never touched)."""
    p = W.three_level_ring(n_cells=1000)
    a = params_of(p, precision="fp64", form="merged", kernel="df32")
    b = params_of(p, precision="fp64", form="merged", kernel="jit")
    c = params_of(p, precision="fp32", form="merged", kernel="df32")
    for pars in ([a, b], [b, a], [c, c]):
        fake = [16] * len(pars)
        with pytest.raises(mln.MLNError) as ei:
            mln.mln_batch_create(pars, fake, fake, fake, None, 0, 0)
        assert ei.value.status == mln.MLN_EINVAL


def test_double_float_rejects_constants_outside_the_pair_range(lib):
    """A density that makes the dP/dt coefficients exceed the FP32 range of a
    pair's high word: MLN_EUNSUPPORTED, for the source as for mln_create."""
    p = W.three_level_ring(n_cells=1000)
    mln.mln_kernel_source(params_of(p, precision="fp64", form="merged", kernel="df32"))
    with pytest.raises(mln.MLNError) as ei:
        mln.mln_kernel_source(params_of(p.with_(N_a=1e60), precision="fp64", form="merged", kernel="df32"))
    assert ei.value.status == mln.MLN_EUNSUPPORTED

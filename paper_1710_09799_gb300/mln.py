"""ctypes binding of the C-ABI in include/mln.h.

The functions below carry the C names and only marshal arguments: every step
of the solver runs in libmln.so (host FP64 set-up and sm_103a kernels).
PyTorch provides the device buffers and the CUDA stream. If the library is
missing or does not load, every entry point raises; there is no fallback.

`Solver` is a convenience wrapper that allocates the caller-owned buffers as
torch tensors and keeps them alive with the context.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmln.so")

MLN_OK, MLN_EINVAL, MLN_ENOMEM, MLN_ECUDA, MLN_ENUMERIC, MLN_ETIMEOUT, MLN_EUNSUPPORTED, MLN_ENONFINITE = range(8)
MLN_BC_PERIODIC, MLN_BC_OPEN = 0, 1
MLN_SRC_NONE, MLN_SRC_HARD, MLN_SRC_SOFT = 0, 1, 2
MLN_FP64, MLN_FP32 = 0, 1
MLN_FORM_STRANG, MLN_FORM_MERGED, MLN_FORM_RODRIGUES, MLN_FORM_ROTATED = 0, 1, 2, 3
MLN_KERNEL_AUTO, MLN_KERNEL_REGISTER, MLN_KERNEL_SPARSE, MLN_KERNEL_JIT, MLN_KERNEL_TENSOR, MLN_KERNEL_DF32 = 0, 1, 2, 3, 4, 5
MLN_MIN_N, MLN_MAX_N = 2, 6
MLN_BATCH_CHUNKS, MLN_BATCH_PERSISTENT = 0, 1
_DMAX = MLN_MAX_N * MLN_MAX_N - 1

BOUNDARY = {"periodic": MLN_BC_PERIODIC, "open": MLN_BC_OPEN}
SOURCE = {"none": MLN_SRC_NONE, "hard": MLN_SRC_HARD, "soft": MLN_SRC_SOFT}
PRECISION = {"fp64": MLN_FP64, "fp32": MLN_FP32}
FORM = {"strang": MLN_FORM_STRANG, "merged": MLN_FORM_MERGED, "rodrigues": MLN_FORM_RODRIGUES,
        "rotated": MLN_FORM_ROTATED}
KERNEL = {"auto": MLN_KERNEL_AUTO, "register": MLN_KERNEL_REGISTER, "sparse": MLN_KERNEL_SPARSE,
          "jit": MLN_KERNEL_JIT, "tensor": MLN_KERNEL_TENSOR, "df32": MLN_KERNEL_DF32}
MAXWELL = {"fdtd": 0, "pstd": 1}

_dp = C.POINTER(C.c_double)


class mln_params(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("precision", C.c_int32), ("form", C.c_int32), ("boundary", C.c_int32),
        ("source_kind", C.c_int32), ("block_steps", C.c_int32), ("tile_cells", C.c_int32),
        ("kernel", C.c_int32),
        ("H0", _dp), ("mu", _dp), ("G", _dp), ("rho0", _dp),
        ("N_a", C.c_double),
        ("n_cells", C.c_int64), ("medium_begin", C.c_int64), ("medium_end", C.c_int64),
        ("source_cell", C.c_int64),
        ("dx", C.c_double), ("dt", C.c_double), ("eps_r", C.c_double), ("mu_r", C.c_double),
        ("sigma", C.c_double), ("maxwell", C.c_int32),
    ]


class mln_setup(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("D", C.c_int32), ("q", C.c_int32), ("reserved", C.c_int32),
        ("M", C.c_double * (_DMAX * _DMAX)), ("U", C.c_double * (_DMAX * _DMAX)),
        ("A0", C.c_double * (_DMAX * _DMAX)), ("T", C.c_double * (_DMAX * _DMAX)),
        ("C1", C.c_double * (_DMAX * _DMAX)),
        ("d_eq", C.c_double * _DMAX), ("v", C.c_double * _DMAX), ("b", C.c_double * _DMAX),
        ("w", C.c_double * _DMAX), ("d0", C.c_double * _DMAX),
        ("theta", C.c_double * (MLN_MAX_N * (MLN_MAX_N - 1) // 2)),
        ("c", C.c_double),
        ("gen", C.c_double * (2 * _DMAX * MLN_MAX_N * MLN_MAX_N)),
    ]


class mln_adjoint_out(C.Structure):
    _fields_ = [("J", C.c_double), ("dJ_dsrc", _dp), ("dJ_dmu", _dp), ("dJ_dG", _dp)]


# Every exported symbol of include/mln.h with (restype, argtypes).
_P = C.POINTER(mln_params)
_SIGS = {
    "mln_query_buffers": (C.c_int, [_P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "mln_create": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "mln_step": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "mln_sync": (C.c_int, [C.c_void_p]),
    "mln_step_count": (C.c_int64, [C.c_void_p]),
    "mln_launch_count": (C.c_int64, [C.c_void_p]),
    "mln_kernel_in_use": (C.c_int32, [C.c_void_p]),
    "mln_tc_wait_selftest": (C.c_int, []),
    "mln_launch_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32)]),
    "mln_work_per_step": (C.c_int, [C.c_void_p, _dp, _dp, _dp, _dp]),
    "mln_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mln_get_fields": (C.c_int, [C.c_void_p, _dp, _dp]),
    "mln_get_rho": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, _dp]),
    "mln_get_populations": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, _dp]),
    "mln_save_state": (C.c_int, [C.c_void_p, _dp, _dp, _dp]),
    "mln_load_state": (C.c_int, [C.c_void_p, _dp, _dp, _dp]),
    "mln_destroy": (None, [C.c_void_p]),
    "mln_status_string": (C.c_char_p, [C.c_int]),
    "mln_last_error": (C.c_char_p, [C.c_void_p]),
    "mln_create_error": (C.c_char_p, []),
    "mln_setup_host": (C.c_int, [_P, C.POINTER(mln_setup)]),
    "mln_project_positive": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "mln_lindblad_superop": (C.c_int, [C.c_int32, _dp, _dp, _dp]),
    "mln_version": (C.c_char_p, []),
    "mln_kernel_source": (C.c_int, [_P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "mln_adjoint": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32,
                              C.POINTER(mln_adjoint_out)]),
    "mln_set_adjoint_memory": (C.c_int, [C.c_void_p, C.c_int64]),
    "mln_adjoint_release": (C.c_int, [C.c_void_p]),
    "mln_batch_create": (C.c_int, [C.c_int32, _P, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int64, C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "mln_batch_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mln_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "mln_batch_sync": (C.c_int, [C.c_void_p]),
    "mln_batch_context": (C.c_void_p, [C.c_void_p, C.c_int32]),
    "mln_batch_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mln_batch_error": (C.c_char_p, [C.c_void_p]),
    "mln_batch_kernel_in_use": (C.c_int32, [C.c_void_p, C.c_int32]),
    "mln_batch_kernel_source": (C.c_int, [C.c_int32, _P, C.c_int32, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "mln_batch_set_launch": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "mln_batch_launch": (C.c_int32, [C.c_void_p]),
    "mln_batch_destroy": (None, [C.c_void_p]),
    "mln_rotation_terms": (C.c_int, [C.c_int32, _dp, C.c_int64, _dp, _dp]),
    "mln_tc_product": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_float), _dp,
                                 C.POINTER(C.c_float)]),
    "mln_tc_product_f16": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_float), _dp, C.POINTER(C.c_float)]),
    "mln_step_noalloc": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_void_p,
                                   C.c_void_p]),
}

_lib = None
_lock = threading.Lock()


def lib():
    """Load libmln.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmln.so not built ({LIB_PATH}); run the package build first")
            l = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


class MLNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def status_string(s: int) -> str:
    return lib().mln_status_string(s).decode()


def _check(status: int, ctx=None):
    if status != MLN_OK:
        if ctx is not None:
            msg = lib().mln_last_error(ctx).decode()
        else:
            msg = lib().mln_create_error().decode()
        raise MLNError(status, msg)


def _cplx(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64).copy()


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class Params:
    """An mln_params with its host arrays kept alive."""

    def __init__(self, *, N, H0, mu, rho0, N_a, n_cells, medium_begin, medium_end, dx, dt,
                 G=None, eps_r=1.0, mu_r=1.0, sigma=0.0, boundary="periodic", source_kind="none",
                 source_cell=0, precision="fp64", form="strang", block_steps=0, tile_cells=0,
                 kernel="auto", maxwell="fdtd"):
        self._H0, self._mu, self._rho0 = _cplx(H0), _cplx(mu), _cplx(rho0)
        self._G = None if G is None else _cplx(G)
        self.s = mln_params(
            N=N, precision=PRECISION.get(precision, precision), form=FORM.get(form, form),
            boundary=BOUNDARY.get(boundary, boundary), source_kind=SOURCE.get(source_kind, source_kind),
            block_steps=block_steps, tile_cells=tile_cells, kernel=KERNEL.get(kernel, kernel),
            H0=_ptr(self._H0), mu=_ptr(self._mu), G=_ptr(self._G), rho0=_ptr(self._rho0),
            N_a=N_a, n_cells=n_cells, medium_begin=medium_begin, medium_end=medium_end,
            source_cell=source_cell, dx=dx, dt=dt, eps_r=eps_r, mu_r=mu_r, sigma=sigma,
            maxwell=MAXWELL.get(maxwell, maxwell))

    @property
    def D(self):
        return self.s.N * self.s.N - 1


# ------------------------------------------------------------------ C names

def mln_query_buffers(params: Params):
    sb, fb = C.c_size_t(), C.c_size_t()
    _check(lib().mln_query_buffers(C.byref(params.s), C.byref(sb), C.byref(fb)))
    return sb.value, fb.value


def mln_create(params: Params, d_state_ptr: int, ez_ptr: int, hy_ptr: int, stream_ptr: int):
    out = C.c_void_p()
    _check(lib().mln_create(C.byref(params.s), C.c_void_p(d_state_ptr), C.c_void_p(ez_ptr),
                            C.c_void_p(hy_ptr), C.c_void_p(stream_ptr), C.byref(out)))
    return out


def mln_step(ctx, n_steps: int, src_ptr: int | None = None):
    _check(lib().mln_step(ctx, n_steps, None if src_ptr is None else C.c_void_p(src_ptr)), ctx)


def mln_sync(ctx):
    _check(lib().mln_sync(ctx), ctx)


def mln_step_count(ctx) -> int:
    return lib().mln_step_count(ctx)


def mln_launch_count(ctx) -> int:
    return lib().mln_launch_count(ctx)


def mln_launch_shape(ctx):
    k, t, th = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().mln_launch_shape(ctx, C.byref(k), C.byref(t), C.byref(th)), ctx)
    return k.value, t.value, th.value


def mln_autotune(ctx, trials: int = 3):
    """Pick the fastest (block_steps, tile_cells) for this context; returns them."""
    k, t = C.c_int32(), C.c_int32()
    _check(lib().mln_autotune(ctx, trials, C.byref(k), C.byref(t)), ctx)
    return k.value, t.value


def mln_work_per_step(ctx):
    """(flops per medium cell-update, flops per grid cell, bytes per medium cell
    per launch, bytes per vacuum cell per launch)."""
    out = [C.c_double() for _ in range(4)]
    _check(lib().mln_work_per_step(ctx, *[C.byref(o) for o in out]), ctx)
    return tuple(o.value for o in out)


def mln_get_fields(ctx, n_cells: int):
    E, H = np.zeros(n_cells), np.zeros(n_cells)
    _check(lib().mln_get_fields(ctx, _ptr(E), _ptr(H)), ctx)
    return E, H


def mln_get_rho(ctx, N: int, cell0: int, count: int) -> np.ndarray:
    out = np.zeros(2 * count * N * N)
    _check(lib().mln_get_rho(ctx, cell0, count, _ptr(out)), ctx)
    return out.view(np.complex128).reshape(count, N, N)


def mln_get_populations(ctx, N: int, cell0: int, count: int) -> np.ndarray:
    out = np.zeros(count * N)
    _check(lib().mln_get_populations(ctx, cell0, count, _ptr(out)), ctx)
    return out.reshape(count, N)


def mln_save_state(ctx, n_medium: int, D: int, n_cells: int):
    d, E, H = np.zeros(n_medium * D), np.zeros(n_cells), np.zeros(n_cells)
    _check(lib().mln_save_state(ctx, _ptr(d), _ptr(E), _ptr(H)), ctx)
    return d.reshape(n_medium, D), E, H


def mln_load_state(ctx, d=None, E=None, H=None):
    arr = [None if x is None else np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in (d, E, H)]
    _check(lib().mln_load_state(ctx, *[_ptr(a) for a in arr]), ctx)


def mln_destroy(ctx):
    if ctx:
        lib().mln_destroy(ctx)


def mln_setup_host(params: Params) -> dict:
    out = mln_setup()
    _check(lib().mln_setup_host(C.byref(params.s), C.byref(out)))
    N, D, q = out.N, out.D, out.q
    m = lambda a: np.array(a[:D * D]).reshape(D, D)
    v = lambda a: np.array(a[:D])
    gen = np.array(out.gen[:2 * D * N * N]).view(np.complex128).reshape(D, N, N)
    return dict(N=N, D=D, q=q, M=m(out.M), U=m(out.U), A0=m(out.A0), T=m(out.T), C1=m(out.C1),
                d_eq=v(out.d_eq), v=v(out.v), b=v(out.b), w=v(out.w), d0=v(out.d0),
                theta=np.array(out.theta[:q]), c=out.c, gen=gen)


def mln_lindblad_superop(N: int, rates=None, dephasing=None) -> np.ndarray:
    """Relaxation superoperator of decay rates rates[b, a] = gamma_{b->a} and
    pure dephasing dephasing[j, k] (both N x N, 1/s, or None); returns the
    (N*N) x (N*N) complex matrix on row-major vec(rho)."""
    r = None if rates is None else np.ascontiguousarray(rates, dtype=np.float64).reshape(N * N)
    g = None if dephasing is None else np.ascontiguousarray(dephasing, dtype=np.float64).reshape(N * N)
    out = np.zeros(2 * N ** 4, dtype=np.float64)
    _check(lib().mln_lindblad_superop(N, _ptr(r), _ptr(g), _ptr(out)))
    return out.view(np.complex128).reshape(N * N, N * N)


def mln_rotation_terms(precision: str, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    s, c1 = np.zeros_like(x), np.zeros_like(x)
    _check(lib().mln_rotation_terms(PRECISION.get(precision, precision), _ptr(x), len(x), _ptr(s), _ptr(c1)))
    return s, c1


def mln_tc_product(A, B, a_in_tmem: bool = True) -> np.ndarray:
    """C = A B^T through the tensor-core product path (A: 128 x kc float32,
    B: nc x kc float64); returns C (128 x nc, float32)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float64)
    nc, kc = B.shape
    C_ = np.zeros((A.shape[0], nc), dtype=np.float32)
    fp = C.POINTER(C.c_float)
    _check(lib().mln_tc_product(nc, kc, int(a_in_tmem), A.ctypes.data_as(fp), B.ctypes.data_as(_dp),
                                C_.ctypes.data_as(fp)))
    return C_


def mln_tc_product_f16(A, B) -> np.ndarray:
    """C = A B^T through the rotated-basis tensor-core product path (FP16
    hi/lo operands with power-of-two scales; A: 128 x kc float32, B: nc x kc
    float64); returns C (128 x nc, float32)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float64)
    nc, kc = B.shape
    C_ = np.zeros((A.shape[0], nc), dtype=np.float32)
    fp = C.POINTER(C.c_float)
    _check(lib().mln_tc_product_f16(nc, kc, A.ctypes.data_as(fp), B.ctypes.data_as(_dp), C_.ctypes.data_as(fp)))
    return C_


MLN_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


def mln_step_noalloc(params: Params, d_state_ptr: int, ez_ptr: int, hy_ptr: int, init_state: bool,
                     n_steps: int, src_ptr: int | None = None, stream_ptr: int = 0):
    """The step for callers that cannot allocate device memory: scratch in a
    fixed device array of the library (see include/mln.h)."""
    _check(lib().mln_step_noalloc(C.byref(params.s), C.c_void_p(d_state_ptr), C.c_void_p(ez_ptr),
                                  C.c_void_p(hy_ptr), 1 if init_state else 0, n_steps,
                                  None if src_ptr is None else C.c_void_p(src_ptr), C.c_void_p(stream_ptr)))


def mln_kernel_source(params: Params) -> str:
    n = C.c_size_t()
    _check(lib().mln_kernel_source(C.byref(params.s), None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value + 1)
    _check(lib().mln_kernel_source(C.byref(params.s), buf, n.value + 1, C.byref(n)))
    return buf.value.decode()


def mln_version() -> str:
    return lib().mln_version().decode()


# ------------------------------------------------------------------ wrapper

class Solver:
    """Owns the torch device buffers of one context (E_z, H_y, medium state)."""

    def __init__(self, params: Params, E0=None, H0=None, device="cuda", stream=None):
        import torch
        self.params = params
        self.N, self.D = params.s.N, params.D
        self.n_cells = params.s.n_cells
        self.n_medium = params.s.medium_end - params.s.medium_begin
        self.dtype = torch.float64 if params.s.precision == MLN_FP64 else torch.float32
        sb, fb = mln_query_buffers(params)
        esz = 8 if self.dtype == torch.float64 else 4
        self.stride = sb // (esz * self.D) if self.D else 0
        dev = torch.device(device)
        self.state = torch.zeros(max(sb // esz, 1), dtype=self.dtype, device=dev)
        self.E = torch.zeros(self.n_cells, dtype=self.dtype, device=dev)
        self.H = torch.zeros(self.n_cells, dtype=self.dtype, device=dev)
        if E0 is not None:
            self.E.copy_(torch.as_tensor(np.asarray(E0), dtype=self.dtype))
        if H0 is not None:
            self.H.copy_(torch.as_tensor(np.asarray(H0), dtype=self.dtype))
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.ctx = mln_create(params, self.state.data_ptr(), self.E.data_ptr(), self.H.data_ptr(),
                              self.stream.cuda_stream)

    def step(self, n_steps: int, src=None):
        """src: None or a float64 CUDA tensor of n_steps samples."""
        ptr = None
        if src is not None:
            assert src.dtype.is_floating_point and src.element_size() == 8 and src.is_cuda
            assert src.numel() >= n_steps
            ptr = src.data_ptr()
        mln_step(self.ctx, n_steps, ptr)

    def sync(self):
        mln_sync(self.ctx)

    @property
    def steps(self) -> int:
        return mln_step_count(self.ctx)

    @property
    def launches(self) -> int:
        return mln_launch_count(self.ctx)

    @property
    def launch_shape(self):
        return mln_launch_shape(self.ctx)

    @property
    def kernel_in_use(self) -> str:
        k = lib().mln_kernel_in_use(self.ctx)
        return {v: n for n, v in KERNEL.items()}[k]

    def autotune(self, trials: int = 3):
        return mln_autotune(self.ctx, trials)

    def project_positive(self) -> int:
        """Project every cell's rho with a negative eigenvalue onto the nearest
        state (see include/mln.h); returns the number of cells changed."""
        k = C.c_int64(0)
        _check(lib().mln_project_positive(self.ctx, C.byref(k)), self.ctx)
        return k.value

    @property
    def work_per_step(self):
        return mln_work_per_step(self.ctx)

    def fields(self):
        return mln_get_fields(self.ctx, self.n_cells)

    def rho(self, cell0=None, count=None):
        cell0 = self.params.s.medium_begin if cell0 is None else cell0
        count = self.n_medium if count is None else count
        return mln_get_rho(self.ctx, self.N, cell0, count)

    def populations(self, cell0=None, count=None):
        cell0 = self.params.s.medium_begin if cell0 is None else cell0
        count = self.n_medium if count is None else count
        return mln_get_populations(self.ctx, self.N, cell0, count)

    def save(self):
        return mln_save_state(self.ctx, self.n_medium, self.D, self.n_cells)

    def load(self, d=None, E=None, H=None):
        mln_load_state(self.ctx, d, E, H)

    def close(self):
        if getattr(self, "ctx", None):
            mln_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ adjoint

def mln_set_adjoint_memory(ctx, n_bytes: int):
    """Limit of mln_adjoint's recorded sets of all segments at once (0: half of
    the free memory plus the workspace the context holds)."""
    _check(lib().mln_set_adjoint_memory(ctx, n_bytes), ctx)


def mln_adjoint_release(ctx):
    """Free the adjoint workspace the context keeps between mln_adjoint calls."""
    _check(lib().mln_adjoint_release(ctx), ctx)


def mln_adjoint(ctx, N: int, n_steps: int, src_ptr: int | None, probe_cell: int, every: int):
    """J and its gradients: (J, dJ/dsrc (n_steps), dJ/dmu params (N*N), dJ/dG (N^2 x N^2 complex))."""
    NN = N * N
    dsrc, dmu, dG = np.zeros(n_steps), np.zeros(NN), np.zeros(2 * NN * NN)
    out = mln_adjoint_out(0.0, _ptr(dsrc), _ptr(dmu), _ptr(dG))
    _check(lib().mln_adjoint(ctx, n_steps, None if src_ptr is None else C.c_void_p(src_ptr), probe_cell, every,
                             C.byref(out)), ctx)
    return out.J, dsrc, dmu, dG.view(np.complex128).reshape(NN, NN)


def mu_from_params(N: int, x):
    """The Hermitian dipole operator from its N*N real parameters in the order of
    mln_adjoint (diagonal, Re of the upper triangle, Im of the upper triangle)."""
    import torch
    x = torch.as_tensor(x)
    mu = torch.zeros((N, N), dtype=torch.complex128, device=x.device)
    idx = N
    q = N * (N - 1) // 2
    for l in range(N):
        mu[l, l] = x[l]
    for j in range(N):
        for k in range(j + 1, N):
            z = torch.complex(x[idx], x[idx + q])
            mu[j, k] = z
            mu[k, j] = z.conj()
            idx += 1
    return mu


def mu_to_params(mu) -> np.ndarray:
    mu = np.asarray(mu)
    N = mu.shape[0]
    up = [(j, k) for j in range(N) for k in range(j + 1, N)]
    return np.array([mu[l, l].real for l in range(N)] + [mu[j, k].real for j, k in up] +
                    [mu[j, k].imag for j, k in up])


def _make_probe_energy():
    import torch

    class ProbeEnergy(torch.autograd.Function):
        """J = dt sum_n (E_z^n at probe)^2 as a differentiable function of the
        source samples, the dipole-operator parameters (mu_to_params order) and
        the relaxation superoperator (a real view (N^2, N^2, 2) of the complex
        matrix). Forward and gradients run in libmln.so (mln_adjoint); autograd
        chains them to whatever produced these tensors."""

        @staticmethod
        def forward(fctx, src, mu_params, G_real, base: dict):
            import torch as _t
            N = base["N"]
            mu = mu_from_params(N, mu_params.detach().cpu()).numpy()
            G = _t.view_as_complex(G_real.detach().cpu().contiguous()).numpy()
            par = Params(N=N, H0=base["H0"], mu=mu, G=G, rho0=base["rho0"], N_a=base["N_a"],
                         n_cells=base["n_cells"], medium_begin=base["medium_begin"], medium_end=base["medium_end"],
                         dx=base["dx"], dt=base["dt"], boundary="periodic", source_kind=base["source_kind"],
                         source_cell=base["source_cell"], precision=base.get("precision", "fp64"), form="strang")
            s = Solver(par, E0=base["E0"])
            srcd = src.detach().to(device="cuda", dtype=_t.float64).contiguous()
            J, dsrc, dmu, dG = mln_adjoint(s.ctx, N, srcd.numel(), srcd.data_ptr(), base["probe_cell"],
                                           base.get("every", 256))
            s.close()
            fctx.save_for_backward(_t.as_tensor(dsrc), _t.as_tensor(dmu), _t.view_as_real(_t.as_tensor(dG)))
            fctx.devices = (src.device, mu_params.device, G_real.device)
            return _t.tensor(J, dtype=_t.float64)

        @staticmethod
        def backward(fctx, gJ):
            dsrc, dmu, dG = fctx.saved_tensors
            dv = fctx.devices
            g = gJ.cpu()
            return (g * dsrc).to(dv[0]), (g * dmu).to(dv[1]), (g * dG).to(dv[2]), None

    return ProbeEnergy


_probe_energy = None


def probe_energy(src, mu_params, G_real, base: dict):
    """torch.autograd entry: see _make_probe_energy."""
    global _probe_energy
    if _probe_energy is None:
        _probe_energy = _make_probe_energy()
    return _probe_energy.apply(src, mu_params, G_real, base)


# ------------------------------------------------------------------ batches

def _bcheck(status: int, b):
    if status != MLN_OK:
        raise MLNError(status, lib().mln_batch_error(b).decode())


def mln_batch_create(params: list, d_states: list, ezs: list, hys: list, srcs: list | None, src_len: int,
                     stream_ptr: int):
    n = len(params)
    arr = (mln_params * n)(*[p.s for p in params])
    vp = lambda xs: (C.c_void_p * n)(*[C.c_void_p(x) for x in xs])
    src_arr = None if srcs is None else vp([0 if x is None else x for x in srcs])
    out = C.c_void_p()
    _check(lib().mln_batch_create(n, arr, vp(d_states), vp(ezs), vp(hys), src_arr, src_len,
                                  C.c_void_p(stream_ptr), C.byref(out)))
    return out


def mln_batch_autotune(b, trials: int = 3):
    k, t = C.c_int32(), C.c_int32()
    _bcheck(lib().mln_batch_autotune(b, trials, C.byref(k), C.byref(t)), b)
    return k.value, t.value


def mln_batch_step(b, n_steps: int):
    _bcheck(lib().mln_batch_step(b, n_steps), b)


def mln_batch_sync(b):
    _bcheck(lib().mln_batch_sync(b), b)


def mln_batch_context(b, i: int):
    return C.c_void_p(lib().mln_batch_context(b, i))


def mln_batch_kernel_source(params: list, N: int) -> str:
    """CUDA source that a batch of these grids compiles for its N-level grids (host only)."""
    arr = (mln_params * len(params))(*[p.s for p in params])
    n = C.c_size_t(0)
    _check(lib().mln_batch_kernel_source(len(params), arr, N, None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value + 1)
    _check(lib().mln_batch_kernel_source(len(params), arr, N, buf, n.value + 1, None))
    return buf.value.decode()


def mln_batch_shape(b):
    k, t, it, la = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int64()
    _bcheck(lib().mln_batch_shape(b, C.byref(k), C.byref(t), C.byref(it), C.byref(la)), b)
    return k.value, t.value, it.value, la.value


def mln_batch_set_launch(b, mode: int, wait_limit: int = 1 << 22):
    _bcheck(lib().mln_batch_set_launch(b, mode, wait_limit), b)


def mln_batch_destroy(b):
    if b:
        lib().mln_batch_destroy(b)


class Batch:
    """Torch-owned buffers and an mln_batch for a list of Params (with E0 arrays
    and optional source sample arrays covering src_len steps)."""

    def __init__(self, params: list, E0s: list, srcs: list | None = None, src_len: int = 0, device="cuda"):
        import torch
        self.params = params
        self.tensors = []
        states, ezs, hys = [], [], []
        self.dtype = torch.float64 if params[0].s.precision == MLN_FP64 else torch.float32
        esz = 8 if self.dtype == torch.float64 else 4
        for par, E0 in zip(params, E0s):
            sb, fb = mln_query_buffers(par)
            st = torch.zeros(max(sb // esz, 1), dtype=self.dtype, device=device)
            E = torch.as_tensor(np.asarray(E0), dtype=self.dtype, device=device).clone()
            H = torch.zeros(par.s.n_cells, dtype=self.dtype, device=device)
            self.tensors.append((st, E, H))
            states.append(st.data_ptr()); ezs.append(E.data_ptr()); hys.append(H.data_ptr())
        self.src_tensors = None
        src_ptrs = None
        if srcs is not None and src_len > 0:
            self.src_tensors = [None if s is None else torch.as_tensor(np.asarray(s[:src_len]), dtype=torch.float64,
                                                                           device=device) for s in srcs]
            src_ptrs = [None if t is None else t.data_ptr() for t in self.src_tensors]
        self.stream = torch.cuda.current_stream()
        self.b = mln_batch_create(params, states, ezs, hys, src_ptrs, src_len if src_ptrs else 0,
                                  self.stream.cuda_stream)

    def autotune(self, trials: int = 3):
        return mln_batch_autotune(self.b, trials)

    def kernel_in_use(self, N: int) -> str | None:
        """Cell model of the N-level grids ("jit", "register" or "df32"), None if none."""
        k = lib().mln_batch_kernel_in_use(self.b, N)
        return None if k < 0 else {v: n for n, v in KERNEL.items()}[k]

    def set_launch(self, launch: str, wait_limit: int = 1 << 22):
        """"chunks" (one launch per K steps and N) or "persistent" (one launch
        per call and N, tiles waiting on their neighbours' progress)."""
        mode = {"chunks": MLN_BATCH_CHUNKS, "persistent": MLN_BATCH_PERSISTENT}[launch]
        mln_batch_set_launch(self.b, mode, wait_limit)

    @property
    def launch(self) -> str:
        """The launch structure of the next steps: "chunks" or "persistent"."""
        return {MLN_BATCH_CHUNKS: "chunks", MLN_BATCH_PERSISTENT: "persistent"}[lib().mln_batch_launch(self.b)]

    def step(self, n_steps: int):
        mln_batch_step(self.b, n_steps)

    def sync(self):
        mln_batch_sync(self.b)

    @property
    def shape(self):
        return mln_batch_shape(self.b)

    def fields(self, i: int):
        return mln_get_fields(mln_batch_context(self.b, i), self.params[i].s.n_cells)

    def rho(self, i: int):
        p = self.params[i].s
        return mln_get_rho(mln_batch_context(self.b, i), p.N, p.medium_begin, p.medium_end - p.medium_begin)

    def close(self):
        if getattr(self, "b", None):
            mln_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

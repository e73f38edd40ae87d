"""ctypes wrapper of the MLN oracle -- TEST INFRASTRUCTURE ONLY.

The oracle is a plain FP64 CPU solver of the 1D Maxwell-Liouville-von Neumann
equations in full density-matrix form (see mln_oracle.c for what it computes
and which passages of the paper each part follows). Only the test suite, the
package's smoke check and the benchmark's CPU-baseline leg may import it; the
product path never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mln_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

BC = {"periodic": 0, "open": 1, "window": 2}
SRC = {"none": 0, "hard": 1, "soft": 2}
MAXWELL = {"fdtd": 0, "pstd": 1}


class OrcProblem(C.Structure):
    _fields_ = [
        ("N", C.c_int),
        ("H0", C.POINTER(C.c_double)),
        ("mu", C.POINTER(C.c_double)),
        ("G", C.POINTER(C.c_double)),
        ("N_a", C.c_double),
        ("n_cells", C.c_long), ("medium_begin", C.c_long), ("medium_end", C.c_long),
        ("dx", C.c_double), ("dt", C.c_double), ("eps_r", C.c_double),
        ("mu_r", C.c_double), ("sigma", C.c_double),
        ("boundary", C.c_int), ("source_kind", C.c_int),
        ("source_cell", C.c_long),
        ("maxwell", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (strict IEEE: no FMA contraction, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            pp = C.POINTER(OrcProblem)
            l.orc_expm.argtypes = [C.c_int, dp, dp]
            l.orc_liouvillian.argtypes = [pp, dp]
            l.orc_dpdt.argtypes = [pp, dp, dp]
            l.orc_cell.argtypes = [pp, dp, C.c_long, dp, dp]
            l.orc_run.argtypes = [pp, dp, dp, dp, C.c_long, dp, C.c_long, dp, C.c_int]
            l.orc_spectral_derivative.argtypes = [C.c_long, C.c_double, C.c_double, dp, dp]
            for f in (l.orc_expm, l.orc_liouvillian, l.orc_dpdt, l.orc_cell, l.orc_run,
                      l.orc_spectral_derivative):
                f.restype = C.c_int
            _lib = l
    return _lib


def _cplx_buf(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64).copy()


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Bound:
    """Keeps the numpy buffers referenced by an OrcProblem alive."""

    def __init__(self, prob, boundary=None, n_cells=None, medium=None, source_cell=None):
        self.H0 = _cplx_buf(prob.H0)
        self.mu = _cplx_buf(prob.mu)
        self.G = None if prob.G is None else _cplx_buf(prob.G)
        mb, me = medium if medium is not None else (prob.medium_begin, prob.medium_end)
        self.s = OrcProblem(
            N=prob.N, H0=_ptr(self.H0), mu=_ptr(self.mu), G=_ptr(self.G), N_a=prob.N_a,
            n_cells=prob.n_cells if n_cells is None else n_cells,
            medium_begin=mb, medium_end=me, dx=prob.dx, dt=prob.dt, eps_r=prob.eps_r,
            mu_r=prob.mu_r, sigma=prob.sigma,
            boundary=BC[prob.boundary if boundary is None else boundary],
            source_kind=SRC[prob.source_kind],
            source_cell=prob.source_cell if source_cell is None else source_cell,
            maxwell=MAXWELL[getattr(prob, "maxwell", "fdtd")])


def expm(A: np.ndarray) -> np.ndarray:
    """exp(A) by the oracle's scaling-and-squaring Pade(13)."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    a = _cplx_buf(A)
    x = np.zeros(2 * n * n)
    rc = lib().orc_expm(n, _ptr(a), _ptr(x))
    if rc:
        raise RuntimeError(f"orc_expm failed ({rc})")
    return x.view(np.complex128).reshape(n, n)


def liouvillian(prob) -> np.ndarray:
    """L0 + G as an (N^2, N^2) matrix on row-major vec(rho)."""
    b = _Bound(prob)
    NN = prob.N * prob.N
    out = np.zeros(2 * NN * NN)
    rc = lib().orc_liouvillian(C.byref(b.s), _ptr(out))
    if rc:
        raise RuntimeError(f"orc_liouvillian failed ({rc})")
    return out.view(np.complex128).reshape(NN, NN)


def dpdt(prob, rho: np.ndarray) -> float:
    """dP/dt = N_a Tr{mu (L0 + G)(rho)} (Eqs. 3 and 5)."""
    b = _Bound(prob)
    r = _cplx_buf(rho)
    out = np.zeros(1)
    rc = lib().orc_dpdt(C.byref(b.s), _ptr(r), _ptr(out))
    if rc:
        raise RuntimeError(f"orc_dpdt failed ({rc})")
    return float(out[0])


def cell(prob, rho: np.ndarray, E_seq: np.ndarray):
    """One medium cell driven by the prescribed fields E_seq[n] = E^n.
    Returns (rho after len(E_seq) steps, dP/dt^{n+1/2} per step)."""
    b = _Bound(prob)
    r = _cplx_buf(rho)
    E = np.ascontiguousarray(E_seq, dtype=np.float64)
    dp = np.zeros(len(E))
    rc = lib().orc_cell(C.byref(b.s), _ptr(r), len(E), _ptr(E), _ptr(dp))
    if rc:
        raise RuntimeError(f"orc_cell failed ({rc})")
    return r.view(np.complex128).reshape(prob.N, prob.N), dp


def spectral_derivative(x: np.ndarray, dx: float, half: float) -> np.ndarray:
    """Derivative of the trigonometric interpolant of the periodic samples x
    (spacing dx) at the points shifted by half * dx (+1/2: E to H points,
    -1/2: H to E points), as the PSTD field solver computes it."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    rc = lib().orc_spectral_derivative(len(x), dx, half, _ptr(x), _ptr(out))
    if rc:
        raise RuntimeError(f"orc_spectral_derivative failed ({rc})")
    return out


class State:
    """E^n, H^{n-1/2} (H[i] at i + 1/2) and rho^{n-1/2} of every medium cell."""

    def __init__(self, E, H, rho):
        self.E = np.ascontiguousarray(E, dtype=np.float64)
        self.H = np.ascontiguousarray(H, dtype=np.float64)
        self.rho = np.ascontiguousarray(rho, dtype=np.complex128)

    def copy(self):
        return State(self.E.copy(), self.H.copy(), self.rho.copy())


def initial_state(prob) -> State:
    nm = prob.medium_end - prob.medium_begin
    rho = np.broadcast_to(prob.rho0, (nm, prob.N, prob.N)).copy()
    return State(prob.e_init().copy(), np.zeros(prob.n_cells), rho)


def run(prob, state: State | None = None, n_steps: int | None = None, step0: int = 0,
        threads: int = 0, probe_cell: int = -1, boundary: str | None = None):
    """Advance the coupled system. Returns (state, probe trace or None)."""
    st = initial_state(prob) if state is None else state.copy()
    n_steps = prob.n_steps if n_steps is None else n_steps
    b = _Bound(prob, boundary=boundary)
    src = prob.source_samples(step0, n_steps)
    src = None if src is None else np.ascontiguousarray(src, dtype=np.float64)
    rho = st.rho.reshape(-1).view(np.float64)
    probe = np.zeros(n_steps) if probe_cell >= 0 else None
    rc = lib().orc_run(C.byref(b.s), _ptr(st.E), _ptr(st.H), _ptr(rho), n_steps, _ptr(src),
                       probe_cell, _ptr(probe), threads)
    if rc:
        raise RuntimeError(f"orc_run failed ({rc})")
    return st, probe


def run_window(prob, cell_index: int, n_steps: int, threads: int = 0):
    """E^{n_steps}, H^{n_steps-1/2} and rho^{n_steps-1/2} at one cell of a large grid,
    computed from its light cone only: a sub-grid of 2*n_steps + 3 cells centred on
    the cell, taken from the initial state (periodic wrap for a ring), with held
    ends. Information moves at most one cell per step, so the centre is exact.

    Only for grids started from the problem's initial state without sources
    reaching the window."""
    n = prob.n_cells
    half = n_steps + 1
    idx = np.arange(cell_index - half, cell_index + half + 1)
    if prob.boundary == "periodic":
        idx = idx % n
    else:
        assert idx[0] >= 0 and idx[-1] < n, "window must lie inside an open grid"
    E = prob.e_init()[idx]
    medium = (idx >= prob.medium_begin) & (idx < prob.medium_end)
    assert medium.all() or not medium.any(), "window must be all medium or all vacuum"
    sub = prob.with_(n_cells=len(idx), E_init=E, medium_begin=0,
                     medium_end=len(idx) if medium.all() else 0,
                     source_kind="none", boundary="window")
    st, _ = run(sub, n_steps=n_steps, threads=threads, boundary="window")
    c = half
    rho = st.rho[c] if medium.all() else None
    return st.E[c], st.H[c], rho

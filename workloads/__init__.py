"""Seeded synthetic inputs for the 1D Maxwell-Liouville-von Neumann (MLN) solver.

This module only *describes problems*: physical constants, grids, Hamiltonians,
dipole operators, relaxation superoperators, initial states, initial fields and
source samples. It contains none of the solver's arithmetic (no splitting, no
exponentials, no FDTD). Both the CUDA path (through its C-ABI binding) and the
CPU oracle read the same problem dictionaries produced here, so the two share
inputs, never code.

Units are SI throughout: energies in J, dipole moments in C*m, rates in 1/s,
fields in V/m, lengths in m, times in s. Complex matrices are numpy complex128
arrays; a relaxation superoperator is an (N*N, N*N) complex matrix acting on
the row-major vectorisation vec(rho)[j*N + k] = rho[j, k].

The problem shapes follow the paper's two test cases (Sec. 5.1, Eqs. 28-30:
two-level self-induced transparency; Sec. 5.2, Eqs. 31-33: three-level system)
and the grid of Sec. 5.1 (dx = 4.578 nm, dt = 7.635e-18 s, Courant number 0.5).
The paper's own figure data and pulse parameters are not available, so these
are synthetic stand-ins with the stated sizes and distributions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# CODATA 2018 exact / recommended values.
HBAR = 1.054571817e-34          # J s
E_CHARGE = 1.602176634e-19      # C
C0 = 299792458.0                # m/s
EPS0 = 8.8541878128e-12         # F/m
MU0 = 1.25663706212e-6          # H/m

MEV = 1e-3 * E_CHARGE           # J per meV
NM_E = 1e-9 * E_CHARGE          # C*m per nm*e

# Grid of the paper's two-level case (Sec. 5.1): Courant number 0.5.
DT_PAPER = 7.635e-18
COURANT = 0.5
DX_PAPER = C0 * DT_PAPER / COURANT

BC_PERIODIC = "periodic"
BC_OPEN = "open"      # E at cell 0 driven (hard source or held), first-order Mur at the right end

SRC_NONE = "none"
SRC_HARD = "hard"
SRC_SOFT = "soft"


@dataclass
class Problem:
    """One MLN problem: parameters, initial state and source samples."""
    name: str
    N: int
    H0: np.ndarray                 # (N, N) complex, J
    mu: np.ndarray                 # (N, N) complex, C*m
    G: np.ndarray | None           # (N*N, N*N) complex, 1/s, or None
    rho0: np.ndarray               # (N, N) complex, initial density matrix of every medium cell
    N_a: float                     # m^-3
    n_cells: int
    medium_begin: int
    medium_end: int
    dx: float = DX_PAPER
    dt: float = DT_PAPER
    eps_r: float = 1.0
    mu_r: float = 1.0
    sigma: float = 0.0
    boundary: str = BC_PERIODIC
    source_kind: str = SRC_NONE
    source_cell: int = 0
    maxwell: str = "fdtd"            # field solver: "fdtd" (Fig. 1) or "pstd" (spectral derivatives, periodic)
    n_steps: int = 0
    E_init: np.ndarray | None = None   # (n_cells,) float64; None = zeros
    src: np.ndarray | None = None      # (n_steps,) float64 source samples; None = no source
    meta: dict = field(default_factory=dict)

    @property
    def D(self) -> int:
        return self.N * self.N - 1

    @property
    def n_medium(self) -> int:
        return self.medium_end - self.medium_begin

    def e_init(self) -> np.ndarray:
        if self.E_init is None:
            return np.zeros(self.n_cells)
        return np.asarray(self.E_init, dtype=np.float64)

    def source_samples(self, n0: int, count: int) -> np.ndarray | None:
        """Samples n0 .. n0+count-1 of the source (sample n is applied in the E
        update that produces E^{n+1})."""
        if self.source_kind == SRC_NONE:
            return None
        fn = self.meta.get("source_fn")
        if fn is not None:
            n = np.arange(n0, n0 + count, dtype=np.float64)
            return fn(n)
        assert self.src is not None
        return np.asarray(self.src[n0:n0 + count], dtype=np.float64)

    def with_(self, **kw) -> "Problem":
        d = dict(self.__dict__)
        d["meta"] = dict(self.meta)
        d.update(kw)
        return Problem(**d)


# --------------------------------------------------------------------------
# Relaxation models (inputs to the method: the paper takes the relaxation
# superoperator G as given, Eq. 2).
# --------------------------------------------------------------------------

def _vec_index(N: int, j: int, k: int) -> int:
    return j * N + k


def superop_from_map(N: int, fn) -> np.ndarray:
    """Matrix of a linear map X -> fn(X) on row-major vec(X)."""
    S = np.zeros((N * N, N * N), dtype=np.complex128)
    for l in range(N):
        for m in range(N):
            E = np.zeros((N, N), dtype=np.complex128)
            E[l, m] = 1.0
            S[:, _vec_index(N, l, m)] = np.asarray(fn(E)).reshape(-1)
    return S


def two_level_relaxation(T1: float, T2: float) -> np.ndarray:
    """The two-level relaxation superoperator of Sec. 5.1 (Eq. 29):
    G(rho) = [[rho22/T1, -rho12/T2], [-rho21/T2, -rho22/T1]]."""
    def g(r):
        return np.array([[r[1, 1] / T1, -r[0, 1] / T2],
                         [-r[1, 0] / T2, -r[1, 1] / T1]], dtype=np.complex128)
    return superop_from_map(2, g)


def three_level_relaxation_sec52(T1: float) -> np.ndarray:
    """The three-level relaxation superoperator of Sec. 5.2 (Eq. 32), with
    g1 = rho33 + rho22 - 2 rho11."""
    def g(r):
        g1 = r[2, 2] + r[1, 1] - 2.0 * r[0, 0]
        out = np.array([
            [g1 / 3.0, -r[0, 1], -r[0, 2]],
            [-r[1, 0], g1 / 3.0 - (r[1, 1] - r[0, 0]), -r[1, 2]],
            [-r[2, 0], -r[2, 1], g1 / 3.0 - (r[2, 2] - r[0, 0])],
        ], dtype=np.complex128)
        return out / T1
    return superop_from_map(3, g)


def lindblad_superop(N: int, rates: dict[tuple[int, int], float],
                     dephasing: np.ndarray | None = None) -> np.ndarray:
    """Lindblad dissipator sum_{(b->a)} gamma (L rho L^+ - {L^+ L, rho}/2) with
    L = |a><b|, plus optional pure dephasing G(rho)_jk -= gamma_jk rho_jk (j != k).

    rates maps (b, a) -> gamma_{b->a} (transition from level b to level a)."""
    def g(r):
        out = np.zeros((N, N), dtype=np.complex128)
        for (b, a), gam in rates.items():
            L = np.zeros((N, N), dtype=np.complex128)
            L[a, b] = 1.0
            LdL = L.conj().T @ L
            out += gam * (L @ r @ L.conj().T - 0.5 * (LdL @ r + r @ LdL))
        if dephasing is not None:
            for j in range(N):
                for k in range(N):
                    if j != k:
                        out[j, k] -= dephasing[j, k] * r[j, k]
        return out
    return superop_from_map(N, g)


# --------------------------------------------------------------------------
# Source waveforms
# --------------------------------------------------------------------------

def sech_pulse(E0: float, tau: float, t0: float, omega: float, dt: float):
    """s(t) = E0 sech((t - t0)/tau) sin(omega (t - t0)); sample n is s((n+1) dt)."""
    def fn(n):
        t = (np.asarray(n, dtype=np.float64) + 1.0) * dt - t0
        return E0 / np.cosh(t / tau) * np.sin(omega * t)
    return fn


def gauss_pulse(E0: float, fwhm: float, t0: float, omega: float, dt: float):
    """s(t) = E0 exp(-4 ln2 (t - t0)^2 / fwhm^2) sin(omega (t - t0)); sample n is s((n+1) dt)."""
    a = 4.0 * math.log(2.0) / fwhm ** 2
    def fn(n):
        t = (np.asarray(n, dtype=np.float64) + 1.0) * dt - t0
        return E0 * np.exp(-a * t * t) * np.sin(omega * t)
    return fn


# --------------------------------------------------------------------------
# The five workload shapes
# --------------------------------------------------------------------------

def two_level_sit(n_cells: int = 2000, medium=(500, 1500), n_steps: int = 20000,
                  omega0: float = 2.3e15, mu12: float = 1e-29, N_a: float = 1e24,
                  T1: float = 1e-12, T2: float = 1e-12, tau: float = 10e-15,
                  t0: float = 50e-15) -> Problem:
    """Two-level Maxwell-Bloch case (shape of Sec. 5.1, Eqs. 28-30): sech pulse of
    area 2*pi at omega0 injected as a hard source at cell 0, first-order Mur at
    the right end, medium in [medium[0], medium[1]), ground-state start.

    Area: with mu = mu12 sigma_x the envelope Rabi frequency is mu12 E0 / hbar
    for a carrier sin(omega0 t), so area = pi mu12 E0 tau / hbar = 2 pi gives
    E0 = 2 hbar / (mu12 tau)."""
    H0 = HBAR * omega0 * np.diag([-0.5, 0.5]).astype(np.complex128)
    mu = np.array([[0, mu12], [mu12, 0]], dtype=np.complex128)
    G = two_level_relaxation(T1, T2)
    rho0 = np.diag([1.0, 0.0]).astype(np.complex128)
    E0 = 2.0 * HBAR / (mu12 * tau)
    p = Problem(name="two_level_sit", N=2, H0=H0, mu=mu, G=G, rho0=rho0, N_a=N_a,
                n_cells=n_cells, medium_begin=medium[0], medium_end=medium[1],
                boundary=BC_OPEN, source_kind=SRC_HARD, source_cell=0, n_steps=n_steps)
    p.meta.update(source_fn=sech_pulse(E0, tau, t0, omega0, p.dt), E0=E0, tau=tau, t0=t0,
                  omega0=omega0)
    return p


def three_level_ring(n_cells: int = 65536, n_steps: int = 100000, seed: int = 0,
                     N_a: float = 1e24, noise: float = 1e3) -> Problem:
    """Three-level QCL-like medium on a periodic ring, every cell active.

    H0 = diag(eps_l), eps_l ~ U[0, 50] meV; real symmetric dipole matrix with zero
    diagonal and off-diagonals ~ U[1, 5] nm*e; one downward Lindblad rate
    ~ U[0.5, 5] /ps per level pair (in the energy order of H0); rho0 =
    diag(0.2, 0.5, 0.3); E^0 ~ N(0, noise^2) per cell; H = 0."""
    rng = np.random.default_rng(seed)
    N = 3
    lev = rng.uniform(0.0, 50.0, size=N) * MEV
    H0 = np.diag(lev).astype(np.complex128)
    mu = np.zeros((N, N), dtype=np.complex128)
    for j in range(N):
        for k in range(j + 1, N):
            mu[j, k] = mu[k, j] = rng.uniform(1.0, 5.0) * NM_E
    order = np.argsort(lev)             # ascending energy
    rates = {}
    for ia in range(N):
        for ib in range(ia + 1, N):
            a, b = int(order[ia]), int(order[ib])   # a below b
            rates[(b, a)] = rng.uniform(0.5, 5.0) * 1e12
    G = lindblad_superop(N, rates)
    rho0 = np.diag([0.2, 0.5, 0.3]).astype(np.complex128)
    E_init = rng.normal(0.0, noise, size=n_cells)
    p = Problem(name="three_level_ring", N=N, H0=H0, mu=mu, G=G, rho0=rho0, N_a=N_a,
                n_cells=n_cells, medium_begin=0, medium_end=n_cells,
                boundary=BC_PERIODIC, n_steps=n_steps, E_init=E_init)
    p.meta.update(seed=seed, rates=rates)
    return p


def six_level_pulse(n_cells: int = 1048576, n_steps: int = 10000, seed: int = 0,
                    N_a: float = 1e24, amplitude: float = 1e8, fwhm: float = 100e-15,
                    t0: float = 75e-15) -> Problem:
    """Six-level manifold, every cell active, driven by a Gaussian pulse.

    Random Hermitian H0 (complex Gaussian X, X + X^+, spectrum mapped affinely to
    [0, 200] meV); Hermitian dipole operator with zero diagonal, off-diagonal
    magnitudes ~ U[1, 5] nm*e and uniform phases; pure dephasing
    gamma_jk = gamma_kj ~ U[1, 10] /ps; rho0 = ground state of H0; hard source at
    cell 0 (Gaussian envelope, FWHM fwhm, centre t0, carrier at the mean
    transition frequency of H0), first-order Mur at the right end. Every cell but
    the last (the Mur cell, vacuum) is medium."""
    rng = np.random.default_rng(seed)
    N = 6
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    Hr = X + X.conj().T
    ev, W = np.linalg.eigh(Hr)
    ev = (ev - ev.min()) / (ev.max() - ev.min()) * 200.0 * MEV
    H0 = (W * ev) @ W.conj().T
    H0 = 0.5 * (H0 + H0.conj().T)
    mu = np.zeros((N, N), dtype=np.complex128)
    for j in range(N):
        for k in range(j + 1, N):
            mag = rng.uniform(1.0, 5.0) * NM_E
            ph = rng.uniform(0.0, 2.0 * np.pi)
            mu[j, k] = mag * np.exp(1j * ph)
            mu[k, j] = np.conj(mu[j, k])
    deph = np.zeros((N, N))
    for j in range(N):
        for k in range(j + 1, N):
            deph[j, k] = deph[k, j] = rng.uniform(1.0, 10.0) * 1e12
    G = lindblad_superop(N, {}, deph)
    g = W[:, 0]
    rho0 = np.outer(g, g.conj())
    diffs = [abs(ev[a] - ev[b]) for a in range(N) for b in range(a + 1, N)]
    omega = float(np.mean(diffs)) / HBAR
    p = Problem(name="six_level_pulse", N=N, H0=H0, mu=mu, G=G, rho0=rho0, N_a=N_a,
                n_cells=n_cells, medium_begin=0, medium_end=n_cells - 1,
                boundary=BC_OPEN, source_kind=SRC_HARD, source_cell=0, n_steps=n_steps)
    p.meta.update(seed=seed, source_fn=gauss_pulse(amplitude, fwhm, t0, omega, p.dt),
                  omega=omega)
    return p


def multi_level_ring(N: int, n_cells: int, n_steps: int, seed: int, N_a: float = 1e24,
                     noise: float = 1e3) -> Problem:
    """N-level ring like the three-level workload: H0 = diag(e_l), e_l ~ U[0, 50]
    meV; real symmetric dipoles U[1, 5] nm*e on every pair; one downward
    Lindblad rate U[0.5, 5] /ps per pair in the energy order; seeded random
    diagonal rho0; E^0 ~ N(0, noise^2)."""
    rng = np.random.default_rng(seed)
    lev = rng.uniform(0.0, 50.0, size=N) * MEV
    mu = np.zeros((N, N), dtype=np.complex128)
    for j in range(N):
        for k in range(j + 1, N):
            mu[j, k] = mu[k, j] = rng.uniform(1.0, 5.0) * NM_E
    order = np.argsort(lev)
    rates = {}
    for ia in range(N):
        for ib in range(ia + 1, N):
            rates[(int(order[ib]), int(order[ia]))] = rng.uniform(0.5, 5.0) * 1e12
    pops = rng.uniform(0.1, 1.0, size=N)
    rho0 = np.diag(pops / pops.sum()).astype(np.complex128)
    p = Problem(name=f"{N}_level_ring", N=N, H0=np.diag(lev).astype(np.complex128), mu=mu,
                G=lindblad_superop(N, rates), rho0=rho0, N_a=N_a, n_cells=n_cells, medium_begin=0,
                medium_end=n_cells, boundary=BC_PERIODIC, n_steps=n_steps,
                E_init=rng.normal(0.0, noise, size=n_cells))
    p.meta.update(seed=seed, rates=rates)
    return p


def batched_devices(count: int = 256, n_steps: int = 20000, seed: int = 0, min_cells: int = 1024,
                    max_cells: int = 65536) -> list[Problem]:
    """Independent devices for the batched workload: N ~ uniform{2, 3, 4}, length
    floor(exp(U[ln min_cells, ln max_cells])) cells. N = 2 devices are two-level
    SIT grids (sech pulse, hard source + Mur, medium = the middle half); N = 3
    and N = 4 devices are rings with noise E^0 (parameters drawn per device)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.integers(2, 5))
        L = int(np.exp(rng.uniform(np.log(min_cells), np.log(max_cells))))
        sub = int(rng.integers(0, 2**31 - 1))
        if N == 2:
            p = two_level_sit(n_cells=L, medium=(L // 4, 3 * L // 4), n_steps=n_steps)
        elif N == 3:
            p = three_level_ring(n_cells=L, n_steps=n_steps, seed=sub)
        else:
            p = multi_level_ring(4, n_cells=L, n_steps=n_steps, seed=sub)
        p.name = f"device{i}_{p.name}"
        out.append(p)
    return out


def adjoint_ring(n_cells: int = 8192, n_steps: int = 5000, seed: int = 0, n_src: int = 512,
                 amplitude: float = 1e5) -> Problem:
    """The gradient workload: the three-level ring's medium (same seeded levels,
    dipoles and rates) on n_cells cells, a soft source at cell 0 carrying n_src
    free samples (a Gaussian-envelope carrier at the mean transition frequency,
    amplitude `amplitude`) followed by zeros, the probe at cell n_cells / 8 (the
    pulse moves half a cell per step, so a probe at n_cells / 2 of an 8192-cell
    ring would not see it within 5000 steps).
    meta holds what the gradients are taken against: the rate table and one
    unit-rate superoperator per rate, the dipole pairs."""
    p = three_level_ring(n_cells=n_cells, n_steps=n_steps, seed=seed)
    lev = np.real(np.diag(p.H0))
    diffs = [abs(lev[a] - lev[b]) for a in range(3) for b in range(a + 1, 3)]
    omega = float(np.mean(diffs)) / HBAR
    k = np.arange(n_steps, dtype=np.float64)
    src = np.zeros(n_steps)
    env = np.exp(-((k[:n_src] - n_src / 2) / (n_src / 5)) ** 2)
    src[:n_src] = amplitude * env * np.sin(omega * (k[:n_src] + 1) * p.dt)
    rates = p.meta["rates"]
    keys = sorted(rates)
    unit = [lindblad_superop(3, {key: 1.0}) for key in keys]
    q = p.with_(source_kind=SRC_SOFT, source_cell=0, src=src, name="adjoint_ring")
    q.meta = dict(seed=seed, rate_keys=keys, rate_values=np.array([rates[k_] for k_ in keys]),
                  unit_superops=unit, probe_cell=n_cells // 8, n_src=n_src,
                  dipole_pairs=[(0, 1), (0, 2), (1, 2)])
    return q


def three_level_ring_pstd(**kw) -> Problem:
    """The three-level ring with the pseudo-spectral field solver (65536 = 2^16
    cells, periodic; same medium, grid and time step)."""
    p = three_level_ring(**kw)
    return p.with_(name=p.name + "_pstd", maxwell="pstd")


def config(name: str, **kw) -> Problem:
    """The named workload at its full size (keyword overrides allowed)."""
    table = {
        "two_level_sit": two_level_sit,
        "three_level_ring": three_level_ring,
        "three_level_ring_pstd": three_level_ring_pstd,
        "six_level_pulse": six_level_pulse,
    }
    return table[name](**kw)


# --------------------------------------------------------------------------
# Random test matrices (for property tests on both sides)
# --------------------------------------------------------------------------

def random_hermitian(rng: np.random.Generator, N: int, scale: float = 1.0) -> np.ndarray:
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    return scale * 0.5 * (X + X.conj().T)


def random_density(rng: np.random.Generator, N: int, rank: int | None = None) -> np.ndarray:
    r = N if rank is None else rank
    X = rng.normal(size=(N, r)) + 1j * rng.normal(size=(N, r))
    rho = X @ X.conj().T
    return rho / np.trace(rho).real

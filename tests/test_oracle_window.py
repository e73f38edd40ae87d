"""Light-cone shortcuts of the oracle against the full-grid oracle.

Two full-size GPU parity tests take their reference values from a smaller
oracle run, relying on the fact that one step of the staggered scheme (Fig. 1,
Eq. 1) moves information by at most one cell:

* `run_window(p, c, n)` computes cell c of a large grid after n steps from a
  sub-grid centred on c with both end cells held (the ring's full-size check);
* a grid cut short on the right (open end, Mur) gives its first cells exactly
  as long as the cut is more than twice the step count away (the six-level
  full-size check).

Here both are compared with the full grid run by `orc.run`, value for value
(the arithmetic per cell is the same, so the results must be identical), on a
periodic ring (cells next to the wrap included) and on an open grid, for
several step counts. A window narrower than the light cone must differ, which
shows that the comparison can fail.
"""
import numpy as np
import pytest

import workloads as W


def _ring(n_cells=240):
    return W.three_level_ring(n_cells=n_cells, n_steps=0, seed=3)


def _open_grid(n_cells=260):
    # open grid (cell 0 held, Mur at the right end), every cell but the Mur
    # cell medium, noise E^0 everywhere, no source
    p = _ring(n_cells)
    return p.with_(boundary="open", medium_begin=0, medium_end=n_cells - 1, source_kind="none")


@pytest.mark.parametrize("n_steps", [1, 7, 40, 100])
def test_window_equals_full_ring(orc, n_steps):
    p = _ring()
    full, _ = orc.run(p, n_steps=n_steps)
    for c in (0, 1, 57, p.n_cells // 2, p.n_cells - 2, p.n_cells - 1):
        E, H, rho = orc.run_window(p, c, n_steps)
        assert E == full.E[c], (c, E, full.E[c])
        assert H == full.H[c], (c, H, full.H[c])
        assert np.array_equal(rho, full.rho[c]), c


@pytest.mark.parametrize("n_steps", [3, 25, 60])
def test_window_equals_full_open_grid(orc, n_steps):
    p = _open_grid()
    full, _ = orc.run(p, n_steps=n_steps)
    lo, hi = n_steps + 1, p.n_cells - n_steps - 3  # windows inside the grid and the medium
    for c in sorted({lo, (lo + hi) // 2, hi}):
        E, H, rho = orc.run_window(p, c, n_steps)
        assert E == full.E[c], (c, E, full.E[c])
        assert H == full.H[c], (c, H, full.H[c])
        assert np.array_equal(rho, full.rho[c]), c


@pytest.mark.parametrize("n", [2, 5, 9])
def test_narrower_window_differs(orc, n):
    """The window's width matters: a sub-grid whose held ends lie one cell
    inside the light cone (2 n - 1 cells) changes the centre within n steps,
    so the equality above is a real check of the width. (The error's leading
    edge shrinks like (c dt / dx)^(2k) over k cells, so it is visible in the
    centre only for short runs; `run_window` itself keeps one cell more than
    the light cone needs on each side.)"""
    import oracle
    p = _ring()
    c = 100
    full, _ = orc.run(p, n_steps=n)
    for half in (n - 1,):
        idx = np.arange(c - half, c + half + 1) % p.n_cells
        sub = p.with_(n_cells=len(idx), E_init=p.e_init()[idx], medium_begin=0, medium_end=len(idx),
                      source_kind="none", boundary="window")
        st, _ = oracle.run(sub, n_steps=n, boundary="window")
        assert st.E[half] != full.E[c], half


@pytest.mark.parametrize("S", [20, 60])
def test_truncated_open_grid_keeps_its_first_cells(orc, S):
    """A pulsed open grid cut to 2 S + keep cells (Mur at the new right end)
    gives the first `keep` cells of the long grid exactly after S steps; a cut
    whose Mur end lies within S / 2 cells of them does not."""
    keep = 30
    n_long = 4 * S + 2 * keep
    p = _open_grid(n_long).with_(source_kind="hard", source_cell=0)
    p.meta["source_fn"] = W.sech_pulse(5e8, 2e-16, 1e-16, 2e15, p.dt)
    full, _ = orc.run(p, n_steps=S)
    n_cut = 2 * S + keep
    cut, _ = orc.run(p.with_(n_cells=n_cut, medium_end=n_cut - 1, E_init=p.e_init()[:n_cut]), n_steps=S)
    assert np.array_equal(cut.E[:keep], full.E[:keep])
    assert np.array_equal(cut.H[:keep], full.H[:keep])
    assert np.array_equal(cut.rho[:keep], full.rho[:keep])
    short = keep + S // 2
    bad, _ = orc.run(p.with_(n_cells=short, medium_end=short - 1, E_init=p.e_init()[:short]), n_steps=S)
    assert not np.array_equal(bad.E[:keep], full.E[:keep])

"""The index rules of the fused step's thread block, checked on a CPU model of
its dependencies (no GPU).

A block loads its tile plus a halo of K cells on each side, runs nsteps <= K
steps with E_z and H_y exchanged through two shared buffers, and writes back
the tile. The model follows every cell's validity through the same update
rules as the block body (Eq. 1 updates need the neighbours' values of the
previous step; the cells at the ends of the loaded span cannot update; on an
open grid cell 0 is held and the Mur cell n - 1 gets its value from cell
n - 2's thread in the same step; a warp skips step st once none of its cells
lies within nsteps - st of the tile). Every tile cell must end valid. The rule
with one cell less of margin, or without the extra left cell of a tile that
starts at the Mur cell, must be caught.
"""
import random


def tile_is_valid(n, tile, K, ns, ti, periodic, extra_margin=1, wide_mur_tile=True):
    t0 = ti * tile
    tlen = min(t0 + tile, n) - t0
    threads = (tile + 2 * K + 31) // 32 * 32
    lh = K + (1 if wide_mur_tile and not periodic and t0 == n - 1 else 0)
    L = tlen + lh + K
    assert L <= threads
    cells = []
    for j in range(threads):
        g = t0 - lh + j
        loaded = j < L and (periodic or 0 <= g < n)
        cells.append((loaded, g % n if periodic else g))
    rules = []
    for j, (loaded, gm) in enumerate(cells):
        h_upd = loaded and j + 1 < L and (periodic or gm < n - 1)
        e_upd = loaded and j >= 1 and (periodic or 0 < gm < n - 1)
        mur = not periodic and loaded and gm == n - 2 and j + 1 < L
        mur_cell = not periodic and loaded and gm == n - 1
        held_e = not periodic and gm in (0, n - 1)   # E not updated by the cell's own rule
        held_h = not periodic and gm == n - 1
        w0 = j & ~31
        active = min(w0 + 32 - lh, lh + tlen - w0) + ns - (1 - extra_margin)
        rules.append((h_upd, e_upd, mur, mur_cell, held_e, held_h, active))
    vE, vH, vS = [True] * threads, [True] * threads, [True] * threads
    buf_E, buf_H = [True] * threads, [True] * threads
    for st in range(ns):
        nE, nH = [False] * threads, [False] * threads   # the write buffer holds values of two steps ago
        E2, H2, S2 = list(vE), list(vH), list(vS)
        for j, (loaded, gm) in enumerate(cells):
            h_upd, e_upd, mur, mur_cell, held_e, held_h, active = rules[j]
            if st >= active:
                E2[j] = H2[j] = S2[j] = False
                continue
            if not loaded:
                nE[j] = nH[j] = True
                continue
            h = (buf_E[j + 1] and vE[j] and vH[j]) if h_upd else (vH[j] and held_h)
            hl = (vE[j] and buf_E[j - 1] and buf_H[j - 1]) if e_upd else True
            s = vS[j] and vE[j]
            en = (vE[j] and h and hl and s) if e_upd else (vE[j] and held_e)
            if mur:
                nE[j + 1] = en and buf_E[j + 1] and vE[j]
            E2[j], H2[j], S2[j] = en, h, s
            if not mur_cell:
                nE[j] = en
            nH[j] = h
        for j in range(threads):
            if rules[j][3]:
                E2[j] = nE[j]
        vE, vH, vS = E2, H2, S2
        buf_E, buf_H = nE, nH
    return all(vE[j] and vH[j] and vS[j] for j in range(lh, lh + tlen) if cells[j][0])


def cases(seed, count):
    rng = random.Random(seed)
    out = []
    for periodic in (True, False):
        for _ in range(count):
            K = rng.randint(1, 64)
            tile = rng.randint(1, 512 - 2 * K)
            n = rng.randint(4, 700)
            ns = rng.randint(1, K)
            nt = (n + tile - 1) // tile
            for ti in sorted({0, nt - 1, rng.randrange(nt)}):
                out.append((n, tile, K, ns, ti, periodic))
    # tiles that start at the Mur cell, and the one before
    for tile in (400, 250, 200, 80, 33, 2, 1):
        for K in (1, 8, 31, 32, 33, 48, 64):
            if tile + 2 * K > 512:
                continue
            n = tile * 5 + 1
            for ns in sorted({1, max(1, K // 2), K}):
                out += [(n, tile, K, ns, 4, False), (n, tile, K, ns, 5, False)]
    return out


def test_every_tile_cell_depends_only_on_computed_values():
    bad = [c for c in cases(1, 600) if not tile_is_valid(*c)]
    assert not bad, bad[:5]


def test_the_model_catches_a_short_margin_and_a_narrow_mur_tile():
    cs = cases(2, 300)
    assert any(not tile_is_valid(*c, extra_margin=0) for c in cs)
    assert any(not tile_is_valid(*c, wide_mur_tile=False) for c in cs)

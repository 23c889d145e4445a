"""The 2D tile kernel's window of grid nodes, written out in integers as the kernel forms
it: the box of a chunk's cells relative to a reference cell (x differences modulo nx), the
window of node columns wx0 .. wx0+ww-1 (modulo nx) and rows wy0 .. wy0+wh-1 around it, cut
to kWin2d nodes, and the test that puts a cell's four nodes inside it.  Checked on
synthetic chunks (sorted runs of cells that drift, chunks that run over the end of a row,
over the periodic seam, near the plates, and scattered ones): every node the window holds
for a cell it accepts is that cell's node in the grid, the window never exceeds its
capacity, and a sorted chunk with a few cells of drift is taken whole."""
import numpy as np
import pytest

K_WIN = 2048


def window(cells, nx, ny, ref):
    ry, rx = divmod(ref, nx)
    cy, cx = np.divmod(cells, nx)
    dx = cx - rx
    dx = np.where(dx >= nx - nx // 2, dx - nx, dx)
    dx = np.where(dx < -(nx // 2), dx + nx, dx)
    dy = cy - ry
    mnx, mxx, mny, mxy = dx.min(), dx.max(), dy.min(), dy.max()
    ww = mxx - mnx + 4
    wx0 = rx + mnx - 1
    wy0 = max(0, ry + mny - 1)
    wh = min(ny, ry + mxy + 2) - wy0 + 1
    if ww >= nx:
        ww, wx0 = nx, 0
    wx0 %= nx
    if ww > K_WIN // 2:
        ww = K_WIN // 2
    if ww * wh > K_WIN:
        wh = K_WIN // ww
    return int(ww), int(wx0), int(wy0), int(wh)


def accepted(c, nx, ww, wx0, wy0, wh):
    cy, cx = divmod(int(c), nx)
    ix = cx - wx0
    if ix < 0:
        ix += nx
    iy = cy - wy0
    return ix <= ww - 2 and 0 <= iy <= wh - 2, ix, iy


def window_node(k, nx, ww, wx0, wy0):
    iy, ix = divmod(k, ww)
    gx = wx0 + ix
    if gx >= nx:
        gx -= nx
    return (wy0 + iy) * nx + gx


def moved(cells, nx, ny):
    """Every cell one step of motion away (within the plates)."""
    cy, cx = np.divmod(cells, nx)
    out = []
    for ddy in (-1, 0, 1):
        for ddx in (-1, 0, 1):
            y = cy + ddy
            ok = (y >= 0) & (y < ny)
            out.append(y[ok] * nx + (cx[ok] + ddx) % nx)
    return np.unique(np.concatenate(out))


def check_chunk(cells, nx, ny, expect_all=False):
    ref = int(cells[len(cells) // 2])
    ww, wx0, wy0, wh = window(cells, nx, ny, ref)
    assert ww * wh <= K_WIN and ww >= 2 and wh >= 1
    assert 0 <= wy0 and wy0 + wh - 1 <= ny
    n_in = 0
    for c in (moved(cells, nx, ny) if expect_all else cells):
        ok, ix, iy = accepted(c, nx, ww, wx0, wy0, wh)
        if not ok:
            continue
        n_in += 1
        cy, cx = divmod(int(c), nx)
        cx1 = 0 if cx + 1 == nx else cx + 1
        want = [cy * nx + cx, cy * nx + cx1, (cy + 1) * nx + cx, (cy + 1) * nx + cx1]
        k00 = iy * ww + ix
        got = [window_node(k, nx, ww, wx0, wy0) for k in (k00, k00 + 1, k00 + ww, k00 + ww + 1)]
        assert got == want, (c, ww, wx0, wy0, wh)
    if expect_all:  # the chunk's cells and every cell a step can take them to
        assert n_in == len(moved(cells, nx, ny))
    return n_in


@pytest.mark.parametrize("nx,ny", [(1024, 1024), (256, 48), (64, 40), (2, 9), (4096, 8)])
def test_window_nodes_are_the_cells_nodes(nx, ny):
    rng = np.random.default_rng(nx * 31 + ny)
    ncell = nx * ny
    for trial in range(60):
        kind = trial % 5
        if kind == 0:  # a sorted run of cells, then up to 3 cells of drift each way
            start = int(rng.integers(0, ncell))
            run = (start + np.arange(32)) % ncell
            cy, cx = np.divmod(run, nx)
            cx = (cx + rng.integers(-3, 4, run.size)) % nx
            cy = np.clip(cy + rng.integers(-3, 4, run.size), 0, ny - 1)
            cells = cy * nx + cx
        elif kind == 1:  # over the end of a row
            cy = int(rng.integers(0, ny - 1))
            cells = np.concatenate([cy * nx + np.arange(max(0, nx - 5), nx),
                                    (cy + 1) * nx + np.arange(0, min(nx, 5))])
        elif kind == 2:  # at the periodic seam, one row
            cy = int(rng.integers(0, ny))
            cells = cy * nx + (np.arange(-3, 4) % nx)
        elif kind == 3:  # against the plates
            cells = np.concatenate([np.arange(0, min(nx, 6)), (ny - 1) * nx + np.arange(0, min(nx, 6))])
        else:  # scattered: mostly outside any window
            cells = rng.integers(0, ncell, 200)
        check_chunk(np.asarray(cells, dtype=np.int64), nx, ny)


def test_a_sorted_chunk_with_drift_is_taken_whole():
    """2,048 consecutive slots of a 1024-wide grid sorted at 64 particles per cell (32
    cells of a row), each cell then moved by up to 8 cells in x and y: the window holds
    the four nodes of every cell, and of every cell one more step of motion can reach
    (the deposit's cell)."""
    nx, ny = 1024, 1024
    rng = np.random.default_rng(5)
    base = 500 * nx + 700
    cells = base + np.repeat(np.arange(32), 64)
    cy, cx = np.divmod(cells, nx)
    cx = cx + rng.integers(-8, 9, cells.size)
    cy = cy + rng.integers(-8, 9, cells.size)
    check_chunk(cy * nx + cx, nx, ny, expect_all=True)

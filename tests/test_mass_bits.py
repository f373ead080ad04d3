"""The mass-bit rule of the stepping launches' classification, on the host
(no GPU).

A stage needs a 32 x TY tile where a cell of the tile or of its 2-cell halo
holds mass (the stencil's reach; ghost cells included).  After a stage the
kernels keep, per tile, nine bits of where its cells hold mass (anywhere,
within two cells of each side, within two cells of each corner), and the
next stage takes its wet tiles from its own and its eight neighbours' bits
without reading the state.  This restates the two device functions
(mass_bits, wet_from_bits in csrc/stage.cuh) and checks the rule against the
brute-force test on the cells, ghosts built by the boundary rules (closed:
mirror of cell k for ghost k; transmissive: copy of the edge cell), over
ragged grids and every tile height: the two must give the same tiles.
"""
import numpy as np
import pytest

MB_ANY, MB_W, MB_E, MB_S, MB_N, MB_SW, MB_SE, MB_NW, MB_NE = 1, 2, 4, 8, 16, 32, 64, 128, 256


def mass_bits(rows, ty):
    """Bits of one tile from its row masks (bit l of rows[r]: column l of row r)."""
    all_ = 0
    for r in rows:
        all_ |= r
    s, n = rows[0] | rows[1], rows[ty - 2] | rows[ty - 1]
    W, E = 0x3, 0xC0000000
    b = 0
    b |= MB_ANY if all_ else 0
    b |= MB_W if all_ & W else 0
    b |= MB_E if all_ & E else 0
    b |= MB_S if s else 0
    b |= MB_N if n else 0
    b |= MB_SW if s & W else 0
    b |= MB_SE if s & E else 0
    b |= MB_NW if n & W else 0
    b |= MB_NE if n & E else 0
    return b


def tile_bits(m, ty):
    ny, nx = m.shape
    gx, gy = (nx + 31) // 32, (ny + ty - 1) // ty
    out = np.zeros((gy, gx), np.int64)
    for by in range(gy):
        for bx in range(gx):
            rows = []
            for r in range(ty):
                j = by * ty + r
                v = 0
                if j < ny:
                    for l in range(32):
                        i = bx * 32 + l
                        if i < nx and m[j, i]:
                            v |= 1 << l
                rows.append(v)
            out[by, bx] = mass_bits(rows, ty)
    return out


def wet_from_bits(mb, bx, ty_, gx, gy):
    w = mb[ty_, bx] & MB_ANY
    wx, ex, sy, ny_ = bx > 0, bx + 1 < gx, ty_ > 0, ty_ + 1 < gy
    if wx:
        w |= mb[ty_, bx - 1] & MB_E
    if ex:
        w |= mb[ty_, bx + 1] & MB_W
    if sy:
        w |= mb[ty_ - 1, bx] & MB_N
        if wx:
            w |= mb[ty_ - 1, bx - 1] & MB_NE
        if ex:
            w |= mb[ty_ - 1, bx + 1] & MB_NW
    if ny_:
        w |= mb[ty_ + 1, bx] & MB_S
        if wx:
            w |= mb[ty_ + 1, bx - 1] & MB_SE
        if ex:
            w |= mb[ty_ + 1, bx + 1] & MB_SW
    return w != 0


def with_ghosts(m, bc):
    """The mass mask on the grid plus its 2-cell ghost ring (corners hold
    nothing: no rule writes them)."""
    ny, nx = m.shape
    g = np.zeros((ny + 4, nx + 4), bool)
    g[2:-2, 2:-2] = m
    for kk in range(2):
        src_w = (kk if kk < nx else nx - 1) if bc[0] == 0 else 0
        src_e = (nx - 1 - kk if nx - 1 - kk >= 0 else 0) if bc[1] == 0 else nx - 1
        g[2:-2, 1 - kk] = m[:, src_w]
        g[2:-2, nx + 2 + kk] = m[:, src_e]
        src_s = (kk if kk < ny else ny - 1) if bc[2] == 0 else 0
        src_n = (ny - 1 - kk if ny - 1 - kk >= 0 else 0) if bc[3] == 0 else ny - 1
        g[1 - kk, 2:-2] = m[src_s, :]
        g[ny + 2 + kk, 2:-2] = m[src_n, :]
    return g


def brute_wet(m, ty, bc):
    ny, nx = m.shape
    g = with_ghosts(m, bc)
    gx, gy = (nx + 31) // 32, (ny + ty - 1) // ty
    out = np.zeros((gy, gx), bool)
    for by in range(gy):
        for bx in range(gx):
            x0, y0 = bx * 32, by * ty
            # cells x0-2 .. x0+33, y0-2 .. y0+ty+1, clipped to the ghost ring
            out[by, bx] = g[max(y0, 0):min(y0 + ty + 4, ny + 4), max(x0, 0):min(x0 + 36, nx + 4)].any()
    return out


@pytest.mark.parametrize("ty", [4, 8, 16])
@pytest.mark.parametrize("nx,ny", [(97, 41), (64, 64), (33, 9), (5, 70), (130, 35), (1, 17), (23, 1), (65, 18)])
def test_bits_give_the_tiles_of_the_brute_force_test(ty, nx, ny):
    rng = np.random.default_rng(nx * 7 + ny * 3 + ty)
    for bc in ((0, 0, 0, 0), (1, 1, 1, 1), (0, 1, 1, 0)):
        for density in (0.002, 0.01, 0.05):
            m = rng.random((ny, nx)) < density
            # cells on tile edges and corners, where the side bits matter
            for j in (0, 1, ty - 2, ty - 1, ty, ty + 1, ny - 1):
                for i in (0, 1, 30, 31, 32, 33, nx - 1):
                    if 0 <= j < ny and 0 <= i < nx and rng.random() < 0.1:
                        m[j, i] = True
            mb = tile_bits(m, ty)
            gy, gx = mb.shape
            got = np.array([[wet_from_bits(mb, bx, by, gx, gy) for bx in range(gx)] for by in range(gy)])
            assert np.array_equal(got, brute_wet(m, ty, bc)), (nx, ny, ty, bc, density)


def test_a_single_cell_reaches_exactly_its_2_cell_neighbourhood():
    """One cell at each position of a 3 x 3 block of 32 x 8 tiles: the tiles
    that list it are those whose 2-cell halo holds it."""
    ty, nx, ny = 8, 96, 24
    for j in range(ny):
        for i in range(nx):
            m = np.zeros((ny, nx), bool)
            m[j, i] = True
            mb = tile_bits(m, ty)
            for by in range(3):
                for bx in range(3):
                    want = (bx * 32 - 2 <= i <= bx * 32 + 33) and (by * ty - 2 <= j <= by * ty + ty + 1)
                    assert wet_from_bits(mb, bx, by, 3, 3) == want, (i, j, bx, by)

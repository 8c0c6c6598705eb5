"""Pins of the oracle's cell binning: the permutation is a stable sort of the
particles by cell id, checked against numpy's lexsort; boundary positions
clamp into the grid."""
import numpy as np
import pytest

import sph_inputs


@pytest.mark.parametrize("n,nc", [(1, (3, 3, 3)), (5000, (7, 7, 7)), (20000, (9, 5, 4))])
def test_bin_is_stable_sort_by_cell(orc, n, nc):
    rng = np.random.default_rng(n)
    box = (1.0, 0.7, 2.5)
    x = rng.uniform(0, 1, (n, 3)) * np.asarray(box)
    cell_of, perm, start = orc.bin_cells(x, box, nc)
    nc_ = np.asarray(nc)
    k = np.clip(np.floor(x * (nc_.astype(np.float64) / np.asarray(box))), 0, nc_ - 1).astype(np.int64)
    cid = k[:, 0] + nc_[0] * (k[:, 1] + nc_[1] * k[:, 2])
    assert np.array_equal(cell_of, cid)
    ref = np.lexsort((np.arange(n), cid))
    assert np.array_equal(perm, ref)
    counts = np.bincount(cid, minlength=int(np.prod(nc_)))
    assert np.array_equal(start, np.concatenate([[0], np.cumsum(counts)]))


@pytest.mark.parametrize("sub", [2, 4])
def test_subcell_order_refines_the_cell_order(orc, sub):
    # sorting by (cell, sub-cell, index): cells stay contiguous, in the same
    # order as the plain cell list; inside a cell the slots are grouped by
    # sub-cell, found independently as floor(x * sub * nc / L) mod sub
    rng = np.random.default_rng(sub)
    n, nc, box = 20000, np.array([5, 6, 4]), np.array([1.0, 1.3, 0.8])
    x = rng.uniform(0, 1, (n, 3)) * box
    key, perm, start = orc.bin_cells(x, box, nc, sub=sub)
    cell_of, perm1, start1 = orc.bin_cells(x, box, nc)
    s3 = sub ** 3
    assert np.array_equal(start[::s3], start1)
    assert np.array_equal(key // s3, cell_of)
    f = np.clip(np.floor(x * (sub * nc / box)), 0, sub * nc - 1).astype(np.int64)
    assert np.array_equal(f // sub, np.clip(np.floor(x * (nc / box)), 0, nc - 1))
    s = f % sub
    want = cell_of.astype(np.int64) * s3 + s[:, 0] + sub * (s[:, 1] + sub * s[:, 2])
    assert np.array_equal(key, want)
    assert np.array_equal(perm, np.lexsort((np.arange(n), want)))


def test_boundary_positions_clamp(orc):
    box = (1.0, 1.0, 1.0)
    top = np.nextafter(1.0, 0.0)
    x = np.array([[0.0, 0.0, 0.0], [top, top, top], [1.0, 1.0, 1.0], [-1e-300, 0.5, 0.5],
                  [1.0 / 3.0, 2.0 / 3.0, 0.5]])
    cell_of, perm, start = orc.bin_cells(x, box, (3, 3, 3))
    assert cell_of[0] == 0
    assert cell_of[1] == 26 and cell_of[2] == 26
    assert cell_of[3] == 0 + 3 * (1 + 3 * 1)
    # 1/3 * 3 rounds to exactly 1.0 in FP64, 2/3 * 3 to 2.0
    assert cell_of[4] == 1 + 3 * (2 + 3 * 1)


def test_sod_grid_occupancy(orc):
    wl = sph_inputs.sod(n_lattice=24, seed=1)
    nc = orc.grid_dims(wl.box, wl.cell_edge)
    _, perm, start = orc.bin_cells(wl.col("x"), wl.box, nc)
    assert start[-1] == wl.n
    assert sorted(perm.tolist()) == list(range(wl.n))


def test_cell_relative_hand_derived_offsets(orc):
    # R13 on a 2 x 1 x 1 box with 4 x 2 x 2 cells (edge 0.5 on every axis):
    # the offset from the cell origin k * L/nc, with k = floor(x nc / L)
    # clamped into the grid, rounded once to the storage format.  Every
    # expected value below is worked out by hand from that rule.
    box, nc = (2.0, 1.0, 1.0), (4, 2, 2)
    top = np.nextafter(2.0, 0.0)                 # L - 1 ulp = 2 - 2^-52 on axis 0
    x = np.array([
        [0.0, 0.0, 0.0],                         # the origin of cell (0, 0, 0)
        [0.5, 0.5, 0.5],                         # on a cell face: cell (1, 1, 1), offset 0
        [1.5, 0.25, 0.75],                       # face on axis 0; mid-cell on 1 and 2
        [top, 0.3, 0.7],                         # last cell on axis 0; 0.3 and 0.7 not in FP32
        [2.0, 1.0, -0.125],                      # outside: clamped into the edge cells
    ])
    pos, off = orc.cell_relative(x, box, nc, "fp32")
    f32_03 = 0.300000011920928955078125          # FP32 nearest to 0.3
    f32_02 = 0.20000000298023223876953125        # FP32 nearest to 0.7 - 0.5 = 0.19999999999999996
    want_off = np.array([
        [0.0, 0.0, 0.0],
        [0.0, 0.0, 0.0],
        [0.0, 0.25, 0.25],
        # 2 - 2^-52 is in cell 3 (origin 1.5); its offset 0.5 - 2^-52 rounds
        # up to 0.5 in FP32 (the FP32 spacing below 0.5 is 2^-25)
        [0.5, f32_03, f32_02],
        # x = L clamps to the last cell (offset one edge); x < 0 to the first
        [0.5, 0.5, -0.125],
    ])
    assert np.array_equal(off, want_off)
    want_origin = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5], [1.5, 0.0, 0.5], [1.5, 0.0, 0.5],
                            [1.5, 0.5, 0.0]])
    assert np.array_equal(pos, want_origin + want_off)
    # FP16 storage of the same offsets: 0.3 -> 1229/4096, 0.2 -> 819/4096
    _, off16 = orc.cell_relative(x, box, nc, "fp16")
    assert off16[3, 1] == 1229.0 / 4096.0 and off16[3, 2] == 819.0 / 4096.0
    assert off16[3, 0] == 0.5 and off16[4, 2] == -0.125


def test_cell_relative_non_power_of_two_edge(orc):
    # one axis with 3 cells: edge = fl(1/3).  fl(1/3) * 3 rounds to exactly
    # 1.0, so x = fl(1/3) is in cell 1 with offset 0; one ulp below it,
    # 3 x = 1 - 2^-52 exactly, so that particle is in cell 0 with offset x.
    third = 1.0 / 3.0
    below = np.nextafter(third, 0.0)
    x = np.array([[third, 0.5, 0.5], [below, 0.5, 0.5]])
    pos, off = orc.cell_relative(x, (1.0, 1.0, 1.0), (3, 1, 1), "fp32")
    assert off[0, 0] == 0.0 and pos[0, 0] == third
    assert off[1, 0] == np.float32(below) and pos[1, 0] == float(np.float32(below))
    # axes with one cell: the origin is 0 and the offset is x itself
    assert off[0, 1] == 0.5 and off[1, 2] == 0.5

"""S1 parity: cell ids, the stable permutation and cell offsets from the CUDA
binning must equal the oracle's bit for bit."""
import numpy as np
import pytest

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu


def _check(orc, wl, reorder=False, sub=2):
    s = make_sph(wl, ws_flags=1 if reorder else 0)
    s.set_tuning(subcells=sub)
    x0 = wl.col("x").copy()
    s.bin_cells(wl.cell_edge, reorder)
    cell_of, perm, start = orc.bin_cells(x0, wl.box, s.nc, sub=sub)
    d = s.describe()
    assert list(d.ncell) == list(s.nc)
    assert d.subcells == sub
    assert np.array_equal(s.cell_start().cpu().numpy(), start.astype(np.int32))
    if reorder:
        # records now in cell order; the permutation is the identity
        aos = s.aos.cpu().numpy()
        assert np.array_equal(aos, wl.aos[perm])
        assert np.array_equal(s.perm().cpu().numpy(), np.arange(wl.n, dtype=np.int32))
    else:
        assert np.array_equal(s.perm().cpu().numpy(), perm.astype(np.int32))
    assert np.array_equal(s.slot_cell().cpu().numpy(), cell_of[perm].astype(np.int32))
    st = s.stats()
    assert st["max_occupancy"] == int(np.max(np.diff(start[::sub ** 3])))
    assert st["error_bits"] == 0
    return s


@pytest.mark.parametrize("sub", [1, 2])
@pytest.mark.parametrize("shuffle", [False, True])
def test_uniform_4096(orc, shuffle, sub):
    _check(orc, sph_inputs.uniform_density(shuffle=shuffle), sub=sub)


def test_sod_small_and_reorder(orc):
    wl = sph_inputs.sod(n_lattice=24, seed=3)
    _check(orc, wl)
    _check(orc, wl, reorder=True)


def test_three_radix_passes(orc):
    # 51^3 = 132651 cells -> 18-bit keys -> three 8-bit passes
    wl = sph_inputs.random_cloud(300_000, seed=4, n_ngb=30)
    wl.h_cap = 1.0 / 51 / 2.0
    wl.cell_edge = 1.0 / 51
    s = _check(orc, wl)
    assert tuple(s.nc) == (51, 51, 51)


def test_all_particles_in_one_cell_and_boundaries(orc):
    wl = sph_inputs.random_cloud(1000, seed=5)
    x = wl.col("x")
    x[:] = 0.01 * x                       # everything in cell (0, 0, 0)
    x[0] = [np.nextafter(1.0, 0.0)] * 3   # top corner cell
    x[1] = [0.0, 0.0, 0.0]
    wl.h_cap = 0.1
    wl.cell_edge = 0.2
    _check(orc, wl)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 2047, 2049])
def test_small_and_ragged_sizes(orc, n):
    wl = sph_inputs.random_cloud(n, seed=100 + n)
    wl.h_cap = 0.05
    wl.cell_edge = 0.1
    _check(orc, wl)


def _clustered(n, seed, blobs):
    """Uniform cloud with some particles squeezed into single sub-cells:
    blobs = [(count, corner, extent)], each blob inside one sub-cell of the
    0.1-cell grid with 2 sub-cells per edge (edge 0.05)."""
    wl = sph_inputs.random_cloud(n, seed=seed)
    x = wl.col("x")
    o = 0
    for cnt, corner, ext in blobs:
        x[o:o + cnt] = corner + ext * x[o:o + cnt]
        o += cnt
    wl.h_cap = 0.05
    wl.cell_edge = 0.1
    return wl


def test_long_cell_ranges(orc):
    # key ranges of every length class: ~5 particles (registers), 600
    # (shared memory), 10,000 and 150,000 (radix over the index bits, 18-bit
    # indices: three passes)
    wl = _clustered(200_000, 7, [(150_000, 0.0, 0.01), (10_000, 0.5, 0.02), (600, 0.3, 0.04)])
    _check(orc, wl)


def test_long_cell_range_four_radix_passes(orc):
    # more than 2^24 particles: 25-bit indices, four radix passes over a
    # 100,000-particle range
    wl = _clustered(16_777_300, 8, [(100_000, 0.7, 0.02)])
    _check(orc, wl)


def test_particles_on_cell_faces(orc):
    # a lattice whose points lie exactly on sub-cell faces (k / 24 with 12
    # cells of 2 sub-cells per axis) and on the faces' neighbouring doubles:
    # the cases where the cell index depends on the rounding of x * (n_c / L)
    k = np.arange(24, dtype=np.float64) / 24.0
    g = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    pts = np.concatenate([g, np.nextafter(g, 0.0), np.nextafter(g, 1.0)])
    wl = sph_inputs.random_cloud(pts.shape[0], seed=9)
    wl.col("x")[:] = np.clip(pts, 0.0, np.nextafter(1.0, 0.0))
    wl.h_cap = 1.0 / 24.0
    wl.cell_edge = 1.0 / 12.0
    s = _check(orc, wl)
    assert tuple(s.nc) == (12, 12, 12)

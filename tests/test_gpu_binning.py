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

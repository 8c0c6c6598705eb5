"""The allocation-free binning entry point, for callers that cannot allocate
device memory (e.g. a plugin whose host application owns the whole device
memory pool): its scratch is a fixed array inside libsph.  It must give
exactly what the regular sph_bin_cells gives, on consecutive calls that share
that array.  This file is collected last on purpose."""
import math

import numpy as np
import pytest

import sph_inputs

pytestmark = pytest.mark.gpu


def _regular(wl, nc_expect):
    from gpu_util import make_sph
    s = make_sph(wl)
    s.set_tuning(subcells=1)       # the allocation-free binning uses plain cells
    s.bin_cells(wl.cell_edge)
    assert list(s.nc) == list(nc_expect)
    out = (s.perm().clone(), s.slot_cell().clone(), s.cell_start().clone())
    s.close()
    return out


def _noalloc(wl, nc):
    import torch
    import paper_2512_05516_gb300 as sph
    aos = torch.from_numpy(wl.aos.copy()).cuda()
    n = wl.n
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    cell = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    start = torch.full((int(np.prod(nc)) + 1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    st = sph.sph_bin_cells_noalloc(aos.data_ptr(), sph.layout_112(), n, wl.box, nc, perm.data_ptr(),
                                   cell.data_ptr(), start.data_ptr(), stream.cuda_stream)
    assert st == 0, sph.sph_status_str(st)
    torch.cuda.synchronize()
    return perm[:n], cell[:n], start


def _grid(wl):
    want = max(wl.cell_edge, 2 * wl.h_cap)
    return [int(math.floor(b / want)) for b in wl.box]


def test_matches_regular_binning_on_two_calls_in_a_row(orc):
    import torch
    # first a larger set with a 3-pass radix sort, then a smaller shuffled one:
    # the second call must not see anything the first left in the shared array
    wl1 = sph_inputs.random_cloud(200_000, seed=61, n_ngb=30)
    wl1.h_cap = 0.5 / 60
    wl1.cell_edge = 1.0 / 60
    wl2 = sph_inputs.sod(n_lattice=24, seed=62, shuffle=True)
    for wl in (wl1, wl2):
        nc = _grid(wl)
        ref = _regular(wl, nc)
        got = _noalloc(wl, nc)
        for r, g in zip(ref, got):
            assert torch.equal(r, g)
        # and directly against the FP64 oracle's stable sort by cell id
        cell_of, perm, start = orc.bin_cells(wl.col("x"), wl.box, nc)
        g_perm, g_cell, g_start = (t.cpu().numpy() for t in got)
        assert np.array_equal(g_perm, perm)
        assert np.array_equal(g_cell, cell_of[perm])
        assert np.array_equal(g_start, start)


def test_rejects_sizes_beyond_its_array():
    import torch
    import paper_2512_05516_gb300 as sph
    L = sph.layout_112()
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = dummy.data_ptr()
    # too many particles: refused before any launch (no pointer is used)
    st = sph.sph_bin_cells_noalloc(p, L, sph.NOALLOC_MAX_PARTICLES + 1, (1.0, 1.0, 1.0), (4, 4, 4),
                                   p, p, p, 0)
    assert st == -2
    # too many cells
    st = sph.sph_bin_cells_noalloc(p, L, 10, (1.0, 1.0, 1.0), (65, 65, 65), p, p, p, 0)
    assert st == -2

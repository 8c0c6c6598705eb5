"""Failure detection with bad inputs prepared on the host: positions that are
not finite or lie outside the box, a non-finite smoothing length or velocity,
and cell grids the workspace cannot hold.  The binning clamps every cell
coordinate into the grid (a NaN converts to coordinate 0), so no index leaves
its array; the conditions land in the sticky error word, sph_get_stats
reports SPH_ENUMERIC for the numerical ones, and the context stays usable:
after the inputs are repaired the same context runs clean."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402


def _wl():
    wl = sph_inputs.random_cloud(3000, seed=41, vel=2.0)
    wl.cell_edge = 2.0 * wl.h_cap
    return wl


def _upload(s, recs):
    host = torch.from_numpy(np.ascontiguousarray(recs)).pin_memory()
    sph_mod._check(sph_mod.sph_aos_upload(s.ctx, host.data_ptr(), recs.nbytes), "upload")
    torch.cuda.synchronize()


def test_bad_positions_are_flagged_at_binning_and_the_context_recovers():
    wl = _wl()
    bad = wl.aos.copy()
    bad[5, 0] = np.nan
    bad[9, 1] = np.inf
    bad[13, 2] = 1.7                  # outside the unit box
    bad[17, 0] = -0.25
    s = make_sph(wl, aos=torch.from_numpy(bad).cuda())
    s.bin_cells(wl.cell_edge)
    st = s.stats()
    assert st["status"] == sph_mod._capi.ENUMERIC
    assert st["error_bits"] & sph_mod.ERR_OUTSIDE
    assert st["error_bits"] & sph_mod.ERR_NONFINITE
    # every particle still has a cell inside the grid, and the permutation is one
    perm = s.perm().cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(wl.n))
    keys = s.slot_cell().cpu().numpy()
    assert keys.min() >= 0 and keys.max() < st["ncell"][0] * st["ncell"][1] * st["ncell"][2] * 8
    # repaired inputs, same context: a clean step
    _upload(s, wl.aos)
    s.reset_stats()
    s.step(wl.dt, 2, cell_edge=wl.cell_edge)
    st = s.stats()
    # (h clamps and Newton fallbacks are conditions of this sparse random set, not failures)
    assert not st["error_bits"] & (sph_mod.ERR_NONFINITE | sph_mod.ERR_OUTSIDE) and st["status"] == 0
    s.close()


def test_nonfinite_h_and_velocity_are_flagged():
    wl = _wl()
    # a NaN smoothing length: the density assumes h_max for it and flags it
    bad = wl.aos.copy()
    bad[7, 10] = np.nan               # h
    s = make_sph(wl, aos=torch.from_numpy(bad).cuda())
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(sph_mod.FIELDS_FORCE)
    s.density(2)
    assert s.stats()["error_bits"] & sph_mod.ERR_NONFINITE
    s.close()
    # an infinite velocity: the force and the drift produce non-finite values
    bad = wl.aos.copy()
    bad[11, 3] = np.inf               # v_x
    s = make_sph(wl, aos=torch.from_numpy(bad).cuda())
    s.step(wl.dt, 2, cell_edge=wl.cell_edge)
    st = s.stats()
    assert st["error_bits"] & sph_mod.ERR_NONFINITE
    assert st["status"] == sph_mod._capi.ENUMERIC
    # the other particles were computed normally
    out = s.aos.cpu().numpy()
    assert np.isfinite(out[:, 11]).all()                   # rho does not depend on v
    s.close()


def test_unusable_grids_are_refused_on_the_host():
    wl = _wl()
    s = make_sph(wl)
    with pytest.raises(sph_mod.SphError) as e:
        s.bin_cells(0.4)                                   # 2 cells per axis
    assert e.value.status == sph_mod._capi.ECAPACITY
    s.close()
    s = make_sph(wl, ncell_max=27)
    with pytest.raises(sph_mod.SphError) as e:
        s.bin_cells(wl.cell_edge)                          # more cells than the workspace holds
    assert e.value.status == sph_mod._capi.ENOSPACE
    # the refused calls left nothing half done: a coarser grid still works
    s.bin_cells(0.3)
    s.aos_to_soa(sph_mod.FIELDS_DENSITY)
    assert s.stats()["error_bits"] == 0
    s.close()

"""S1 with the drift's keys (SPH_BIN_DRIFT_KEYS): the kick/drift computes the
cell key of every position it writes, and a binning that is told the records
have not changed since uses those keys instead of reading the records.  The
binning must then equal the oracle's on the drifted positions bit for bit,
and whole steps must equal the same steps binned from the records; calls that
write records, or another grid, make the binning read the records again."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph, read_aos

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph  # noqa: E402


def _positions(s):
    return read_aos(s)[:, 0:3].copy()


def _check_binning(orc, s, wl, sub):
    cell_of, perm, start = orc.bin_cells(_positions(s), wl.box, s.nc, sub=sub)
    assert np.array_equal(s.cell_start().cpu().numpy(), start.astype(np.int32))
    assert np.array_equal(s.perm().cpu().numpy(), perm.astype(np.int32))
    assert np.array_equal(s.slot_cell().cpu().numpy(), cell_of[perm].astype(np.int32))


def _step(s, wl, drift_keys, reorder=False):
    s.bin_cells(wl.cell_edge, reorder=reorder, drift_keys=drift_keys)
    s.aos_to_soa(sph.FIELDS_FORCE)
    s.density(wl.newton_steps)
    s.force()
    s.kick_drift_writeback(wl.dt, wl.dt, sph.FIELDS_OUTPUT)


@pytest.mark.parametrize("sub", [1, 2])
def test_steps_with_drift_keys_equal_steps_reading_the_records(orc, sub):
    wl = sph_inputs.random_cloud(20_000, seed=41, vel=3.0)
    wl.dt = 5e-3                                  # many particles cross cells every step
    a, b = make_sph(wl), make_sph(wl)
    for s in (a, b):
        s.set_tuning(subcells=sub)
    for k in range(4):
        _step(a, wl, False)
        b.bin_cells(wl.cell_edge, drift_keys=True)
        _check_binning(orc, b, wl, sub)
        assert np.array_equal(a.perm().cpu().numpy(), b.perm().cpu().numpy())
        b.aos_to_soa(sph.FIELDS_FORCE)
        b.density(wl.newton_steps)
        b.force()
        b.kick_drift_writeback(wl.dt, wl.dt, sph.FIELDS_OUTPUT)
        assert np.array_equal(read_aos(a), read_aos(b)), k
    assert a.stats()["error_bits"] == 0 and b.stats()["error_bits"] == 0


def test_drift_keys_on_records_in_cell_order(orc):
    # the long-run lattice sorted into cell order once, then drifted with
    # separate kick/drift calls
    wl = sph_inputs.long_run(nx=64, ny=32, nz=32)
    wl.dt = 5e-3
    s = make_sph(wl, ws_flags=sph.WS_REORDER)
    s.bin_cells(wl.cell_edge, reorder=True)
    for k in range(3):
        s.aos_to_soa(sph.FIELDS_FORCE)
        s.density(0)
        s.force()
        s.kick_drift(wl.dt, wl.dt)
        s.bin_cells(wl.cell_edge, drift_keys=True)
        _check_binning(orc, s, wl, 2)


def test_writes_and_grid_changes_drop_the_drift_keys(orc):
    wl = sph_inputs.sod(n_lattice=24, seed=42)
    wl.dt = 2e-3
    s = make_sph(wl)
    _step(s, wl, False)
    # records replaced after the drift: the binning reads them
    aos = read_aos(s)
    rng = np.random.default_rng(3)
    aos[:, 0:3] = rng.uniform(0.0, 1.0, (wl.n, 3))
    host = torch.from_numpy(aos).contiguous()
    assert sph.sph_aos_upload(s.ctx, host.data_ptr(), host.numel() * 8) == 0
    s.bin_cells(wl.cell_edge, drift_keys=True)
    _check_binning(orc, s, wl, 2)
    # another sub-cell grid than the drift's: the binning reads the records
    s.aos_to_soa(sph.FIELDS_FORCE)
    s.density(wl.newton_steps)
    s.force()
    s.kick_drift_writeback(wl.dt, wl.dt, sph.FIELDS_OUTPUT)
    s.set_tuning(subcells=1)
    s.bin_cells(wl.cell_edge, drift_keys=True)
    _check_binning(orc, s, wl, 1)
    # a second binning without a drift in between: no keys to use
    s.bin_cells(wl.cell_edge, drift_keys=True)
    _check_binning(orc, s, wl, 1)
    # unknown flags are rejected
    assert sph.sph_bin_cells(s.ctx, wl.cell_edge, 4) == sph._capi.EINVAL

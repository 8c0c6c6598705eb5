"""The streaming layout (the paper's Section 6.3 variant with the AoS master
in host memory): the same context over a pinned host AoS, which the binning,
conversion and kick/drift + write-back kernels read and write over the host
link.  Results must equal the in-place (device AoS) run byte for byte."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("reorder", [False, True])
def test_host_resident_aos_equals_device_aos(orc, reorder):
    wl = sph_inputs.sod(n_lattice=48, seed=81)
    outs = []
    for where in ("device", "host"):
        t = torch.from_numpy(np.ascontiguousarray(wl.aos))
        aos = t.cuda() if where == "device" else t.pin_memory()
        s = make_sph(wl, aos=aos, ws_flags=1 if reorder else 0)
        for k in range(2):
            s.bin_cells(wl.cell_edge, reorder=reorder and k == 0)
            s.step(wl.dt, 5, cell_edge=wl.cell_edge)
        torch.cuda.synchronize()
        outs.append(s.aos.cpu().numpy().copy())
        assert s.stats()["error_bits"] == 0
        s.close()
    assert np.array_equal(outs[0], outs[1])
    if not reorder:
        # and the first step of that trajectory is the oracle's
        s = make_sph(wl, aos=torch.from_numpy(np.ascontiguousarray(wl.aos)).pin_memory())
        s.step(wl.dt, 5, cell_edge=wl.cell_edge)
        torch.cuda.synchronize()
        out = s.aos.numpy()
        o = orc.step(wl)
        assert (np.abs(out[:, 11] - o["rho"]) / o["rho"]).max() <= 1e-5
        s.close()

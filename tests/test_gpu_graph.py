"""Whole time steps captured in a CUDA graph: replaying the captured step must
give exactly the same particles as running the same calls eagerly."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu


def _ctx_on(wl, stream):
    import paper_2512_05516_gb300 as sph
    aos = torch.from_numpy(wl.aos.copy()).cuda()
    with torch.cuda.stream(stream):
        return make_sph(wl, aos=aos), aos


@pytest.mark.parametrize("prec", [None, {"v": "fp16", "m": "bf16", "h": "m16", "u": "m10"}])
def test_graph_replay_equals_eager(prec):
    wl = sph_inputs.sod(n_lattice=24, seed=31)
    steps = 4
    # eager
    se = torch.cuda.Stream()
    s_e, aos_e = _ctx_on(wl, se)
    with torch.cuda.stream(se):
        for _ in range(steps):
            s_e.step(wl.dt, 5, prec=prec, cell_edge=wl.cell_edge)
    se.synchronize()
    # captured: one eager warm-up step, then capture one step and replay it
    sg = torch.cuda.Stream()
    s_g, aos_g = _ctx_on(wl, sg)
    with torch.cuda.stream(sg):
        s_g.step(wl.dt, 5, prec=prec, cell_edge=wl.cell_edge)
    sg.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=sg):
        s_g.step(wl.dt, 5, prec=prec, cell_edge=wl.cell_edge)
    # capturing does not execute: the AoS still holds the state after one step
    for _ in range(steps - 1):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(aos_g, aos_e)
    st = s_g.stats()
    assert st["error_bits"] == 0

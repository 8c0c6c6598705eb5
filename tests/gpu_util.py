"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
on a workload and read its results back as FP64 numpy arrays."""
from __future__ import annotations

import math

import numpy as np

import sph_inputs


def ncell_for(box, cell_edge, h_cap):
    want = max(cell_edge, 2.0 * h_cap)
    nc = [int(math.floor(b / want)) for b in box]
    return nc, int(np.prod(nc))


def make_sph(wl, aos=None, layout=None, ncell_max=None, ws_flags=0, flags=0):
    import torch
    import paper_2512_05516_gb300 as sph
    if aos is None:
        aos = torch.from_numpy(np.ascontiguousarray(wl.aos)).cuda()
    if layout is None:
        layout = sph.layout_112()
    nc, ncell = ncell_for(wl.box, wl.cell_edge, wl.h_cap)
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap, flags=flags)
    s = sph.Sph(aos, layout, params, ncell_max if ncell_max else max(ncell, 27), ws_flags)
    s.nc = nc
    return s


def aos_col(aos_np, name):
    off, nc = sph_inputs.RECORD_112[name]
    c0 = off // 8
    return aos_np[:, c0:c0 + nc] if nc > 1 else aos_np[:, c0]


def read_aos(s):
    return s.aos.cpu().numpy()


def count_band_ok(orc, wl, h_ref, counts_gpu, delta):
    """Every GPU neighbour count must lie between the oracle's counts at
    h (1 - delta) and h (1 + delta): only pairs whose separation is within
    delta of the support radius may be classified differently by FP32."""
    x, m = wl.col("x"), wl.col("m")
    lo = orc.density(x, m, h_ref * (1 - delta), wl.box, wl.eta, wl.h_cap * 2, 0)["nngb"]
    hi = orc.density(x, m, h_ref * (1 + delta), wl.box, wl.eta, wl.h_cap * 2, 0)["nngb"]
    ok = (counts_gpu >= lo) & (counts_gpu <= hi)
    return ok, lo, hi


def rel_err(a, b, scale=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if scale is None:
        scale = np.abs(b)
    return np.abs(a - b) / scale

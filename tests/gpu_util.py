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


def count_band_ok(orc, wl, h_ref, counts_gpu, delta, targets=None, m=None):
    """Every GPU neighbour count must lie between the oracle's counts at
    h (1 - delta) and h (1 + delta): only pairs whose separation is within
    delta of the support radius may be classified differently by FP32.  With
    `targets`, h_ref holds every particle's h and the counts are the targets'.
    `m` replaces the workload's masses (e.g. by their storage-rounded values)."""
    x = wl.col("x")
    m = wl.col("m") if m is None else m
    lo = orc.density(x, m, h_ref * (1 - delta), wl.box, wl.eta, wl.h_cap * 2, 0,
                     targets=targets)["nngb"]
    hi = orc.density(x, m, h_ref * (1 + delta), wl.box, wl.eta, wl.h_cap * 2, 0,
                     targets=targets)["nngb"]
    ok = (counts_gpu >= lo) & (counts_gpu <= hi)
    return ok, lo, hi


def force_count_band_ok(orc, x, m, h, box, counts_gpu, delta, targets=None):
    """The force's rule (R7: a pair iff r < h_i + h_j) with the same band: every
    GPU force-neighbour count must lie between the oracle's counts with every
    h scaled by (1 - delta) and by (1 + delta), which scales each pair's
    support h_i + h_j by the same factor.  Only pairs whose separation lies
    within delta of h_i + h_j may be classified differently.  The counts do not
    depend on rho, P, c or v, so neutral values are passed for them."""
    n = x.shape[0]
    ones, zeros = np.ones(n), np.zeros(n)
    v0 = np.zeros((n, 3))

    def cnt(scale):
        return orc.force(x, v0, m, h * scale, ones, zeros, zeros, box, 1.0, 2.0, 0.01,
                         targets=targets)["nngb"]

    lo, hi = cnt(1.0 - delta), cnt(1.0 + delta)
    ok = (counts_gpu >= lo) & (counts_gpu <= hi)
    return ok, lo, hi


def rel_err(a, b, scale=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if scale is None:
        scale = np.abs(b)
    return np.abs(a - b) / scale

"""Batching over uneven cells (the clustered workload): one persistent launch
over a work queue in cell order, the same queue with the costliest items
first, and one launch per power-of-two cost class must give identical
results -- each item's sums are independent of when it runs -- and match the
FP64 oracle fed the same BF16-stored inputs (mode Q)."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402

VARIANTS = [(0, 0), (1, 0), (1, 1)]      # (item_order, class_launches)


def _run(wl, order, per_class):
    s = make_sph(wl)
    s.set_tuning(item_order=order, class_launches=per_class)
    s.bin_cells(wl.cell_edge)
    prec = {"v": "bf16", "m": "bf16", "h": "bf16", "u": "bf16"}
    s.aos_to_soa(sph_mod.FIELDS_FORCE, prec)
    s.density(0)
    s.force()
    s.soa_to_aos(sph_mod.mask("rho", "a", "P"))
    out = s.aos.cpu().numpy().copy()
    st = s.stats()
    nngb = np.empty(wl.n, np.int32)
    nngb[s.perm().cpu().numpy()] = s.nngb().cpu().numpy()
    s.close()
    return out, st, nngb


def test_queue_orders_agree_and_match_oracle(orc):
    wl = sph_inputs.gaussian_mixture(n=1 << 17)
    res = [_run(wl, o, c) for o, c in VARIANTS]
    for out, st, nngb in res[1:]:
        assert np.array_equal(out, res[0][0])
        assert np.array_equal(nngb, res[0][2])
        assert st["pairs_density"] == res[0][1]["pairs_density"]
        assert st["pairs_force"] == res[0][1]["pairs_force"]
    assert res[2][1]["launches"] > res[0][1]["launches"] + 30     # one launch per class
    out = res[0][0]
    # mode Q on sampled targets, among them the densest core
    x = wl.col("x")
    d = x - wl.meta["centres"][0]
    d -= np.round(d)
    core = np.argsort(np.sum(d * d, axis=1))[:32]
    rng = np.random.default_rng(5)
    tgt = np.unique(np.concatenate([core, rng.choice(wl.n, 200, replace=False)]))
    q = lambda v: orc.quantize(np.asarray(v).ravel(), "bf16")[0].reshape(np.shape(v))
    o = orc.density(x, q(wl.col("m")), q(wl.col("h")), wl.box, wl.eta, wl.h_cap, 0, targets=tgt)
    assert (np.abs(out[tgt, 11] - o["rho"]) / o["rho"]).max() <= 1e-5
    assert np.abs(res[0][2][tgt] - o["nngb"]).max() <= 2


def test_autotuner_picks_and_caches_a_valid_shape(orc, tmp_path):
    from paper_2512_05516_gb300 import autotune
    wl = sph_inputs.sod(n_lattice=48, seed=71)
    s = make_sph(wl)
    cache = str(tmp_path / "tune.json")
    r = autotune.tune(s, wl.cell_edge, newton_steps=5, reps=1, cache_path=cache)
    assert not r["cached"] and r["trials"]
    t = s.tuning()
    for k, v in r["tuning"].items():
        assert t[k] == v
    r2 = autotune.tune(s, wl.cell_edge, newton_steps=5, reps=1, cache_path=cache)
    assert r2["cached"] and r2["tuning"] == r["tuning"]
    # a step in the tuned shape still matches the oracle
    s.step(wl.dt, 5, cell_edge=wl.cell_edge)
    out = s.aos.cpu().numpy()
    o = orc.step(wl)
    assert (np.abs(out[:, 11] - o["rho"]) / o["rho"]).max() <= 1e-5
    s.close()


def test_plain_form_matches_batched_and_oracle(orc):
    # the baseline (one thread per particle over the 27 cells, no staging or
    # pruning) computes the same step: against the oracle within the FP32
    # tolerances, against the batched kernels to rounding
    wl = sph_inputs.sod(n_lattice=48, seed=72)
    outs = []
    for plain in (0, 1):
        s = make_sph(wl)
        s.set_tuning(pair_kernel=plain)
        s.step(wl.dt, 5, cell_edge=wl.cell_edge)
        outs.append((s.aos.cpu().numpy(), s.stats()))
        assert s.tuning()["pair_kernel"] == plain
        s.close()
    o = orc.step(wl)
    for out, st in outs:
        assert st["error_bits"] == 0
        assert (np.abs(out[:, 11] - o["rho"]) / o["rho"]).max() <= 1e-5
        scale = np.mean(np.linalg.norm(o["a"], axis=1))
        assert np.linalg.norm(out[:, 6:9] - o["a"], axis=1).max() / scale <= 1e-5
    (b, sb), (p, sp) = outs
    assert sb["pairs_density"] == sp["pairs_density"] and sb["pairs_force"] == sp["pairs_force"]
    assert sp["tests_density"] > 3 * sb["tests_density"]          # no pruning in the plain form
    assert (np.abs(b[:, 11] - p[:, 11]) / p[:, 11]).max() <= 1e-6

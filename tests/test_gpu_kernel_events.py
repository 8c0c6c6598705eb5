"""Timing hooks (sph_set_kernel_events): the events the library records
around the density and force pair kernels bracket those kernels alone --
within the calls' own time -- and change no result."""
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402


def _ev():
    return torch.cuda.Event(enable_timing=True)


def _step(s, wl):
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(sph_mod.FIELDS_FORCE)
    calls = {}
    for name, fn in (("density", lambda: s.density(5)), ("force", s.force)):
        e0, e1 = _ev(), _ev()
        e0.record(s.stream)
        fn()
        e1.record(s.stream)
        calls[name] = (e0, e1)
    torch.cuda.synchronize()
    out = {f"a{k}": s.soa_raw("a", k).clone() for k in range(3)}
    out["rho"] = s.soa_raw("rho").clone()
    return out, {k: a.elapsed_time(b) for k, (a, b) in calls.items()}


def test_hooks_bracket_the_pair_kernels_and_change_nothing():
    wl = sph_inputs.sod(n_lattice=48, seed=41)
    s = make_sph(wl)
    ref, _ = _step(s, wl)
    hooks = {w: (_ev(), _ev()) for w in (sph_mod.KEV_DENSITY, sph_mod.KEV_FORCE)}
    for w, (e0, e1) in hooks.items():
        s.set_kernel_events(w, e0, e1)
    out, call_ms = _step(s, wl)
    for k in ref:
        assert torch.equal(out[k].view(torch.int32), ref[k].view(torch.int32)), k
    for w, name in ((sph_mod.KEV_DENSITY, "density"), (sph_mod.KEV_FORCE, "force")):
        ms = hooks[w][0].elapsed_time(hooks[w][1])
        assert 0.0 < ms <= call_ms[name], (name, ms, call_ms[name])
    # cleared hooks record nothing more: the events keep their last times
    for w in hooks:
        s.set_kernel_events(w, None, None)
    before = {w: hooks[w][0].elapsed_time(hooks[w][1]) for w in hooks}
    _step(s, wl)
    assert {w: hooks[w][0].elapsed_time(hooks[w][1]) for w in hooks} == before
    e = _ev()
    e.record(s.stream)
    assert sph_mod.sph_set_kernel_events(s.ctx, sph_mod.KEV_DENSITY, e.cuda_event, None) == sph_mod._capi.EINVAL
    assert sph_mod.sph_set_kernel_events(s.ctx, 7, None, None) == sph_mod._capi.EINVAL
    s.close()

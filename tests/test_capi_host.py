"""CPU checks of the C ABI: the library loads without a GPU, exports every
function include/sph.h declares, its ctypes structures match the C layout, and
host-side argument errors are returned before any device call."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")


@pytest.fixture(scope="module")
def sph():
    from paper_2512_05516_gb300 import build
    build.build()
    import paper_2512_05516_gb300 as m
    return m


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(sph):
    from paper_2512_05516_gb300 import _capi
    names = declared_functions()
    assert len(names) >= 17
    lib = C.CDLL(sph.library_path())
    for nm in names:
        assert hasattr(lib, nm), nm
        assert nm in _capi.PROTOTYPES, nm
    assert set(_capi.PROTOTYPES) == set(names)


def test_struct_layout_matches_c(sph, tmp_path):
    from paper_2512_05516_gb300 import _capi
    prog = tmp_path / "probe.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "sph.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(sph_aos_layout), sizeof(sph_params),
         sizeof(sph_stats), sizeof(sph_tuning), sizeof(sph_desc));
  printf("%zu %zu %zu %zu\n", offsetof(sph_stats, error_bits), offsetof(sph_stats, nitems),
         offsetof(sph_desc, off_soa), offsetof(sph_desc, valid));
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[:5] == [C.sizeof(_capi.sph_aos_layout), C.sizeof(_capi.sph_params),
                         C.sizeof(_capi.sph_stats), C.sizeof(_capi.sph_tuning),
                         C.sizeof(_capi.sph_desc)]
    assert sizes[5:] == [_capi.sph_stats.error_bits.offset, _capi.sph_stats.nitems.offset,
                         _capi.sph_desc.off_soa.offset, _capi.sph_desc.valid.offset]


def test_workspace_query_and_bad_layouts(sph):
    L = sph.layout_112()
    n = 1000
    ws = sph.sph_workspace_bytes(L, n, 1000)
    assert ws > 0 and ws % 256 == 0
    assert sph.sph_workspace_bytes(L, n, 1000, sph.WS_REORDER) >= ws + 112 * n
    assert sph.sph_workspace_bytes(L, -1, 1000) == 0
    # the level hierarchy's arrays: levels (2 B), one level's targets and codes
    # (8 B), two per-slot scans (8 B) and work items for a tile per particle
    lv = sph.sph_workspace_bytes(L, n, 1000, sph.WS_LEVELS)
    assert lv >= ws + 18 * n
    assert sph.sph_workspace_bytes(L, 0, 1000, sph.WS_LEVELS) > 0
    assert sph.sph_workspace_bytes(L, n, 5) == 0            # fewer than 27 cells
    bad = sph.layout_112()
    bad.record_bytes = 100                                  # not a multiple of 8
    assert sph.sph_workspace_bytes(bad, n, 1000) == 0
    bad = sph.layout_112()
    bad.offset[sph.F_X] = -1                                # positions are required
    assert sph.sph_workspace_bytes(bad, n, 1000) == 0
    bad = sph.layout_112()
    bad.type[sph.F_X] = sph.AOS_F32                         # positions must be FP64
    assert sph.sph_workspace_bytes(bad, n, 1000) == 0
    bad = sph.layout_112()
    bad.offset[sph.F_P] = 108                               # runs past the record
    assert sph.sph_workspace_bytes(bad, n, 1000) == 0


def test_create_rejects_bad_arguments_before_touching_the_device(sph):
    # every case below fails validation on the host; no pointer is dereferenced
    L = sph.layout_112()
    P = sph.make_params((1.0, 1.0, 1.0), h_max=0.1)
    n, ncell = 100, 125
    need = sph.sph_workspace_bytes(L, n, ncell)
    fake_aos, fake_ws = 0x7f0000000000, 0x7f1000000000
    st, ctx = sph.sph_create(L, P, n, ncell, 0, 0, fake_ws, need, 0)
    assert st == sph._capi.EINVAL and not ctx.value
    st, _ = sph.sph_create(L, P, n, ncell, 0, fake_aos + 8, fake_ws, need, 0)     # misaligned AoS
    assert st == sph._capi.EINVAL
    st, _ = sph.sph_create(L, P, n, ncell, 0, fake_aos, fake_ws + 64, need, 0)    # misaligned workspace
    assert st == sph._capi.EINVAL
    st, _ = sph.sph_create(L, P, n, ncell, 0, fake_aos, fake_ws, need - 256, 0)   # too small
    assert st == sph._capi.ENOSPACE
    badp = sph.make_params((1.0, 0.0, 1.0), h_max=0.1)
    st, _ = sph.sph_create(L, badp, n, ncell, 0, fake_aos, fake_ws, need, 0)
    assert st == sph._capi.EINVAL
    badp = sph.make_params((1.0, 1.0, 1.0), gamma=1.0, h_max=0.1)
    st, _ = sph.sph_create(L, badp, n, ncell, 0, fake_aos, fake_ws, need, 0)
    assert st == sph._capi.EINVAL


def test_calls_on_null_context_fail_cleanly(sph):
    null = C.c_void_p(0)
    assert sph.sph_bin_cells(null, 0.1, 0) == sph._capi.EINVAL
    assert sph.sph_aos_to_soa(null, 1, None) == sph._capi.EINVAL
    assert sph.sph_density(null, 0) == sph._capi.EINVAL
    assert sph.sph_force(null) == sph._capi.EINVAL
    assert sph.sph_kick_drift(null, 0.1, 0.1) == sph._capi.EINVAL
    assert sph.sph_soa_to_aos(null, 2) == sph._capi.EINVAL
    assert sph.sph_kick_drift_writeback(null, 0.1, 0.1, 2) == sph._capi.EINVAL
    assert sph.sph_get_stats(null)[0] == sph._capi.EINVAL
    assert sph.sph_set_tuning(null, sph.sph_tuning()) == sph._capi.EINVAL
    assert sph.sph_describe(null)[0] == sph._capi.EINVAL
    assert sph.sph_set_field_scale(null, [0] * sph.SPH_NFIELDS) == sph._capi.EINVAL
    assert sph.sph_get_field_scale(null)[0] == sph._capi.EINVAL
    assert sph.sph_bin_levels(null, 3, 6, 0.1) == sph._capi.EINVAL
    assert sph.sph_density_levels(null, 0) == sph._capi.EINVAL
    assert sph.sph_force_levels(null) == sph._capi.EINVAL
    assert sph.sph_level_counts(null)[0] == sph._capi.EINVAL
    assert sph.sph_set_kernel_events(null, sph.KEV_DENSITY, None, None) == sph._capi.EINVAL
    sph.sph_destroy(null)
    assert sph.sph_status_str(-5).startswith("cell grid")


def test_suggest_scale_puts_fp16_values_in_range(sph):
    # the Sod particle mass (1/124)^3 is subnormal in FP16; the suggested
    # exponent moves it 4 binades below FP16's top binade
    m = (1.0 / 124.0) ** 3
    e = sph.suggest_scale(m, "fp16")
    assert 2.0 ** 11 <= m * 2.0 ** e < 2.0 ** 12
    assert sph.suggest_scale(262144.0, "fp16") == 11 - 18
    for fmt in ("fp32", "bf16", "m16", "m10"):
        assert sph.suggest_scale(m, fmt) == 0
    assert sph.suggest_scale(0.0, "fp16") == 0
    assert sph.suggest_scale(1e-300, "fp16") == sph.SCALE_MAX_EXP
    assert sph.scale_array({"m": 5, "u": -3}) == [0, 0, 0, 5, 0, 0, -3, 0, 0, 0]


def test_binding_constants_match_the_header(sph):
    src = open(HEADER).read()
    defs = dict((k, int(v)) for k, v in re.findall(r"#define (SPH_[A-Z_0-9]+)\s+(-?\d+)\b", src))
    from paper_2512_05516_gb300 import _capi
    assert defs["SPH_BIN_REORDER"] == _capi.BIN_REORDER
    assert defs["SPH_BIN_DRIFT_KEYS"] == _capi.BIN_DRIFT_KEYS
    assert defs["SPH_WS_REORDER"] == _capi.WS_REORDER
    assert defs["SPH_WS_LEVELS"] == _capi.WS_LEVELS
    assert (defs["SPH_KEV_DENSITY"], defs["SPH_KEV_FORCE"]) == (_capi.KEV_DENSITY, _capi.KEV_FORCE)
    assert _capi.sph_tuning.block_threads_force.offset == C.sizeof(_capi.sph_tuning) - 4

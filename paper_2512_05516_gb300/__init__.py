"""Python binding of libsph, the GB300 (sm_103a) SPH hot path over FP64
array-of-structs particles with on-device AoS->SoA conversion and
reduced-precision storage (arXiv 2512.05516).

Argument marshalling only.  Module-level functions carry the C names
(``sph_create``, ``sph_bin_cells``, ...); ``Sph`` bundles a context with the
torch tensors that own its device memory.  PyTorch provides device memory and
streams; every step of the path runs in libsph's CUDA kernels, and importing
this package raises when the library is missing (there is no fallback).
"""
from __future__ import annotations

import ctypes as C

from . import _capi
from ._capi import (KEV_DENSITY, KEV_FORCE, AOS_F32, AOS_F64, BIN_DRIFT_KEYS, BIN_REORDER, BIT, ERR_HCAP, ERR_NEWTON, ERR_NONFINITE, ERR_OUTSIDE, ERR_TIMEOUT,
                    PFLAG_HCAP, PFLAG_NEWTON, PFLAG_NONFINITE,
                    F_A, F_CS, F_DUDT, F_H, F_M, F_P, F_RHO, F_U, F_V, F_X, FIELD_NAMES,
                    FIELDS_DENSITY, FIELDS_FORCE, FIELDS_KICK, FIELDS_OUTPUT, FLAG_PLAIN_SUM,
                    NCOMP, P_BF16, P_FP16, P_FP32, P_FP32_M10, P_FP32_M16, PREC, SPH_NFIELDS,
                    BUFFER_MAX, BUFFER_MIN, LEVEL_MAX, LEVEL_MIN, LEVELS_MAX, SRC_AOS, SRC_SOA, WS_LEVELS, WS_REORDER,
                    sph_aos_layout, sph_desc,
                    sph_params, sph_stats, sph_tuning)

_lib = _capi.load()


class SphError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status} ({_lib.sph_status_str(status).decode()})")


def _check(status: int, what: str, allow=(0,)):
    if status not in allow:
        raise SphError(status, what)
    return status


def library_path() -> str:
    return _capi._build.LIB_PATH


# ----------------------------------------------------------------- C names
def sph_workspace_bytes(layout: sph_aos_layout, n: int, ncell_max: int, ws_flags: int = 0) -> int:
    return int(_lib.sph_workspace_bytes(C.byref(layout), n, ncell_max, ws_flags))


def sph_create(layout, params, n, ncell_max, ws_flags, d_aos, d_workspace, workspace_bytes, stream):
    out = C.c_void_p()
    st = _lib.sph_create(C.byref(layout), C.byref(params), n, ncell_max, ws_flags,
                         C.c_void_p(d_aos), C.c_void_p(d_workspace), workspace_bytes,
                         C.c_void_p(stream), C.byref(out))
    return st, out


def sph_bin_cells(ctx, cell_edge: float, flags: int) -> int:
    return _lib.sph_bin_cells(ctx, float(cell_edge), int(flags))


def sph_aos_to_soa(ctx, fields: int, prec) -> int:
    arr = None
    if prec is not None:
        arr = (C.c_int32 * SPH_NFIELDS)(*prec)
    return _lib.sph_aos_to_soa(ctx, fields, arr)


def sph_host_stage_bytes(ctx) -> int:
    return int(_lib.sph_host_stage_bytes(ctx))


def sph_aos_to_soa_host(ctx, host_aos: int, fields: int, prec, host_stage: int, stage_bytes: int,
                        nthreads: int = 0) -> int:
    arr = None
    if prec is not None:
        arr = (C.c_int32 * SPH_NFIELDS)(*prec)
    return _lib.sph_aos_to_soa_host(ctx, C.c_void_p(host_aos), fields, arr, C.c_void_p(host_stage),
                                    int(stage_bytes), int(nthreads))


def sph_soa_to_aos_host(ctx, host_aos: int, fields: int, host_stage: int, stage_bytes: int,
                        nthreads: int = 0) -> int:
    return _lib.sph_soa_to_aos_host(ctx, C.c_void_p(host_aos), fields, C.c_void_p(host_stage),
                                    int(stage_bytes), int(nthreads))


def sph_density(ctx, newton_steps: int) -> int:
    return _lib.sph_density(ctx, int(newton_steps))


def sph_force(ctx) -> int:
    return _lib.sph_force(ctx)


def sph_kick_drift(ctx, dt_kick: float, dt_drift: float) -> int:
    return _lib.sph_kick_drift(ctx, float(dt_kick), float(dt_drift))


def sph_soa_to_aos(ctx, fields: int) -> int:
    return _lib.sph_soa_to_aos(ctx, fields)


def sph_kick_drift_writeback(ctx, dt_kick: float, dt_drift: float, fields: int) -> int:
    return _lib.sph_kick_drift_writeback(ctx, float(dt_kick), float(dt_drift), fields)


def sph_bin_buffers(ctx, buffer_size: int) -> int:
    return _lib.sph_bin_buffers(ctx, int(buffer_size))


def sph_buffer_density(ctx, source: int) -> int:
    return _lib.sph_buffer_density(ctx, int(source))


def sph_buffer_force(ctx, source: int) -> int:
    return _lib.sph_buffer_force(ctx, int(source))


def sph_buffer_kick(ctx, source: int, dt: float) -> int:
    return _lib.sph_buffer_kick(ctx, int(source), float(dt))


def sph_buffer_drift(ctx, source: int, dt: float) -> int:
    return _lib.sph_buffer_drift(ctx, int(source), float(dt))


def sph_bin_levels(ctx, level_min: int, level_max: int, h_margin: float) -> int:
    return _lib.sph_bin_levels(ctx, int(level_min), int(level_max), float(h_margin))


def sph_density_levels(ctx, newton_steps: int) -> int:
    return _lib.sph_density_levels(ctx, int(newton_steps))


def sph_force_levels(ctx) -> int:
    return _lib.sph_force_levels(ctx)


def sph_level_counts(ctx):
    done = (C.c_int64 * (LEVEL_MAX + 1))()
    prom = (C.c_int64 * (LEVEL_MAX + 1))()
    st = _lib.sph_level_counts(ctx, done, prom)
    return st, list(done), list(prom)


def sph_set_field_scale(ctx, exp2) -> int:
    arr = (C.c_int32 * SPH_NFIELDS)(*[int(e) for e in exp2])
    return _lib.sph_set_field_scale(ctx, arr)


def sph_get_field_scale(ctx):
    arr = (C.c_int32 * SPH_NFIELDS)()
    st = _lib.sph_get_field_scale(ctx, arr)
    return st, list(arr)


def sph_get_stats(ctx):
    s = sph_stats()
    st = _lib.sph_get_stats(ctx, C.byref(s))
    return st, s


def sph_reset_stats(ctx) -> int:
    return _lib.sph_reset_stats(ctx)


def sph_set_kernel_events(ctx, which: int, ev_begin, ev_end) -> int:
    return _lib.sph_set_kernel_events(ctx, which, ev_begin, ev_end)


def sph_set_tuning(ctx, tuning: sph_tuning) -> int:
    return _lib.sph_set_tuning(ctx, C.byref(tuning))


def sph_get_tuning(ctx):
    t = sph_tuning()
    st = _lib.sph_get_tuning(ctx, C.byref(t))
    return st, t


def sph_describe(ctx):
    d = sph_desc()
    st = _lib.sph_describe(ctx, C.byref(d))
    return st, d


def sph_aos_upload(ctx, host_ptr: int, nbytes: int) -> int:
    return _lib.sph_aos_upload(ctx, C.c_void_p(host_ptr), nbytes)


def sph_aos_download(ctx, host_ptr: int, nbytes: int) -> int:
    return _lib.sph_aos_download(ctx, C.c_void_p(host_ptr), nbytes)


NOALLOC_MAX_PARTICLES = 262144
NOALLOC_MAX_CELLS = 262144


def sph_bin_cells_noalloc(d_aos: int, layout: sph_aos_layout, n: int, box, nc, d_perm: int,
                          d_cell_of_slot: int, d_cell_start: int, stream: int) -> int:
    """Cell binning for callers that cannot allocate device memory: scratch
    lives in a fixed array inside libsph (see include/sph.h)."""
    b = (C.c_double * 3)(*[float(v) for v in box])
    g = (C.c_int32 * 3)(*[int(v) for v in nc])
    return _lib.sph_bin_cells_noalloc(C.c_void_p(d_aos), C.byref(layout), int(n), b, g,
                                      C.c_void_p(d_perm), C.c_void_p(d_cell_of_slot),
                                      C.c_void_p(d_cell_start), C.c_void_p(stream))


def sph_destroy(ctx) -> None:
    _lib.sph_destroy(ctx)


def sph_status_str(status: int) -> str:
    return _lib.sph_status_str(status).decode()


# ----------------------------------------------------------------- helpers
RECORD_112 = {"x": 0, "v": 24, "a": 48, "m": 72, "h": 80, "rho": 88, "u": 96, "P": 104}


def make_layout(offsets: dict, record_bytes: int, f32_fields=()) -> sph_aos_layout:
    """Layout descriptor from a field-name -> byte-offset map."""
    L = sph_aos_layout()
    L.record_bytes = record_bytes
    for f in range(SPH_NFIELDS):
        L.offset[f] = -1
        L.type[f] = AOS_F64
    for name, off in offsets.items():
        f = FIELD_NAMES.index(name)
        L.offset[f] = off
        L.type[f] = AOS_F32 if name in f32_fields else AOS_F64
    return L


def layout_112() -> sph_aos_layout:
    """The 112-byte FP64 record {x[3], v[3], a[3], m, h, rho, u, P}."""
    return make_layout(RECORD_112, 112)


#: the paper's single-precision benchmark record (Section 6): a 64-bit ID and
#: FP64 positions, every other field FP32, 144 bytes in all (bytes 84..143
#: stand for the record's further fields, which no kernel here touches)
RECORD_144 = {"x": 8, "v": 32, "a": 44, "m": 56, "h": 60, "rho": 64, "u": 68, "P": 72, "cs": 76,
              "dudt": 80}
F32_144 = ("v", "a", "m", "h", "rho", "u", "P", "cs", "dudt")


def layout_144() -> sph_aos_layout:
    """The 144-byte record of the paper's benchmark: ID, FP64 x, FP32 fields."""
    return make_layout(RECORD_144, 144, F32_144)


def make_params(box, gamma=5.0 / 3.0, alpha=1.0, beta=2.0, eps=0.01, eta=1.1272516517868265,
                h_max=0.1, flags=0) -> sph_params:
    p = sph_params()
    for k in range(3):
        p.box[k] = float(box[k])
    p.gamma, p.alpha_av, p.beta_av, p.eps_av = float(gamma), float(alpha), float(beta), float(eps)
    p.eta, p.h_max, p.flags = float(eta), float(h_max), int(flags)
    return p


def prec_array(prec) -> list:
    """Per-field storage formats from a {field name: format name} dict."""
    out = [P_FP32] * SPH_NFIELDS
    if prec:
        for name, fmt in prec.items():
            out[FIELD_NAMES.index(name)] = PREC[fmt] if isinstance(fmt, str) else int(fmt)
    return out


SCALE_MAX_EXP = 64


def scale_array(scale) -> list:
    """Per-field storage-scale exponents from a {field name: e} dict."""
    out = [0] * SPH_NFIELDS
    if scale:
        for name, e in scale.items():
            out[FIELD_NAMES.index(name)] = int(e)
    return out


def suggest_scale(max_abs: float, fmt, headroom_bits: int = 4) -> int:
    """Storage-scale exponent e for a field whose magnitudes reach `max_abs`:
    FP16 gets the largest value 2^headroom_bits below its top binade (room
    for growth during a run); the other formats keep FP32's exponent range
    and need no scale (0)."""
    import math
    f = PREC[fmt] if isinstance(fmt, str) else int(fmt)
    if f != P_FP16 or not (max_abs > 0.0) or not math.isfinite(max_abs):
        return 0
    e = (15 - headroom_bits) - math.floor(math.log2(max_abs))
    return max(-SCALE_MAX_EXP, min(SCALE_MAX_EXP, e))


def mask(*names) -> int:
    m = 0
    for nm in names:
        m |= BIT(FIELD_NAMES.index(nm))
    return m


class Sph:
    """A libsph context over a torch-owned AoS on the current CUDA device.

    `aos` holds n records of `layout.record_bytes` bytes (any dtype; e.g.
    float64 of shape (n, 14) for the 112-byte record): a CUDA tensor, or a
    pinned host tensor (`tensor.pin_memory()`), which the kernels then read
    and write over the host link (the streaming layout; the workspace stays
    on the current CUDA device).  The workspace is a torch uint8 tensor owned
    by this object.  All calls run on `stream` (default: torch's current
    stream)."""

    def __init__(self, aos, layout: sph_aos_layout, params: sph_params, ncell_max: int,
                 ws_flags: int = 0, stream=None):
        import torch
        if not (aos.is_cuda or aos.is_pinned()):
            raise ValueError("aos must be a CUDA tensor or a pinned host tensor")
        self.torch = torch
        self.aos = aos
        self.layout = layout
        self.params = params
        nbytes = aos.numel() * aos.element_size()
        if nbytes % layout.record_bytes:
            raise ValueError("AoS size is not a whole number of records")
        self.n = nbytes // layout.record_bytes
        dev = aos.device if aos.is_cuda else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.ws_bytes = sph_workspace_bytes(layout, self.n, ncell_max, ws_flags)
        if self.ws_bytes == 0:
            raise SphError(-1, "sph_workspace_bytes")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        with torch.cuda.device(dev):
            st, ctx = sph_create(layout, params, self.n, ncell_max, ws_flags, aos.data_ptr(),
                                 self.ws.data_ptr(), self.ws_bytes, self.stream.cuda_stream)
        _check(st, "sph_create")
        self.ctx = ctx

    # --- the path
    def bin_cells(self, cell_edge: float = 0.0, reorder: bool = False, drift_keys: bool = False):
        """drift_keys: the caller vouches that the records' positions are those
        the last kick/drift wrote (see SPH_BIN_DRIFT_KEYS)."""
        flags = (BIN_REORDER if reorder else 0) | (BIN_DRIFT_KEYS if drift_keys else 0)
        _check(sph_bin_cells(self.ctx, cell_edge, flags), "sph_bin_cells")

    def aos_to_soa(self, fields: int, prec=None):
        arr = prec if isinstance(prec, list) else (prec_array(prec) if prec is not None else None)
        _check(sph_aos_to_soa(self.ctx, fields, arr), "sph_aos_to_soa")

    def set_scale(self, scale):
        """Power-of-two storage scales, {field name: e} or a list per field."""
        arr = scale if isinstance(scale, list) else scale_array(scale)
        _check(sph_set_field_scale(self.ctx, arr), "sph_set_field_scale")

    def scale(self) -> dict:
        st, arr = sph_get_field_scale(self.ctx)
        _check(st, "sph_get_field_scale")
        return {FIELD_NAMES[f]: arr[f] for f in range(SPH_NFIELDS)}

    def density(self, newton_steps: int = 0):
        _check(sph_density(self.ctx, newton_steps), "sph_density")

    def force(self):
        _check(sph_force(self.ctx), "sph_force")

    def kick_drift(self, dt_kick: float, dt_drift: float):
        _check(sph_kick_drift(self.ctx, dt_kick, dt_drift), "sph_kick_drift")

    def soa_to_aos(self, fields: int):
        _check(sph_soa_to_aos(self.ctx, fields), "sph_soa_to_aos")

    def kick_drift_writeback(self, dt_kick: float, dt_drift: float, fields: int = FIELDS_OUTPUT):
        _check(sph_kick_drift_writeback(self.ctx, dt_kick, dt_drift, fields), "sph_kick_drift_writeback")

    # ---- the conversion on the host (the paper's CPU placement)
    def host_stage(self):
        """A pinned host staging buffer sized for the host-side conversion
        (allocated once per context)."""
        if getattr(self, "_stage", None) is None:
            nbytes = sph_host_stage_bytes(self.ctx)
            self._stage = self.torch.empty(max(nbytes, 1), dtype=self.torch.uint8).pin_memory()
        return self._stage

    def aos_to_soa_host(self, host_aos, fields: int, prec=None, nthreads: int = 0):
        """sph_aos_to_soa on the host: `host_aos` is a host tensor of records."""
        arr = prec if isinstance(prec, list) else (prec_array(prec) if prec is not None else None)
        st = self.host_stage()
        _check(sph_aos_to_soa_host(self.ctx, host_aos.data_ptr(), fields, arr, st.data_ptr(), st.numel(),
                                   nthreads), "sph_aos_to_soa_host")

    def soa_to_aos_host(self, host_aos, fields: int, nthreads: int = 0):
        """sph_soa_to_aos on the host, into the host tensor of records `host_aos`."""
        st = self.host_stage()
        _check(sph_soa_to_aos_host(self.ctx, host_aos.data_ptr(), fields, st.data_ptr(), st.numel(), nthreads),
               "sph_soa_to_aos_host")

    # ---- buffer kernels (the paper's 64-particle buffers, Section 6)
    @staticmethod
    def _source(source) -> int:
        if isinstance(source, str):
            return {"aos": SRC_AOS, "soa": SRC_SOA}[source]
        return int(source)

    def bin_buffers(self, buffer_size: int = 64):
        _check(sph_bin_buffers(self.ctx, buffer_size), "sph_bin_buffers")

    def buffer_density(self, source="soa"):
        _check(sph_buffer_density(self.ctx, self._source(source)), "sph_buffer_density")

    def buffer_force(self, source="soa"):
        _check(sph_buffer_force(self.ctx, self._source(source)), "sph_buffer_force")

    def buffer_kick(self, dt: float, source="soa"):
        _check(sph_buffer_kick(self.ctx, self._source(source), dt), "sph_buffer_kick")

    def buffer_drift(self, dt: float, source="soa"):
        _check(sph_buffer_drift(self.ctx, self._source(source), dt), "sph_buffer_drift")

    # ---- the level hierarchy (adaptive h; needs ws_flags=WS_LEVELS)
    def bin_levels(self, level_min: int, level_max: int, h_margin: float = 0.1):
        _check(sph_bin_levels(self.ctx, level_min, level_max, h_margin), "sph_bin_levels")

    def density_levels(self, newton_steps: int = 0):
        _check(sph_density_levels(self.ctx, newton_steps), "sph_density_levels")

    def force_levels(self):
        _check(sph_force_levels(self.ctx), "sph_force_levels")

    def level_counts(self):
        """(done, promoted): per level l (index l), the particles computed
        there and those moved from it to level l - 1."""
        st, done, prom = sph_level_counts(self.ctx)
        _check(st, "sph_level_counts")
        return done, prom

    def step_levels(self, dt: float, level_min: int, level_max: int, newton_steps: int = 5, prec=None,
                    h_margin: float = 0.1, out_fields: int = FIELDS_OUTPUT):
        """One time step with every particle's own h over the level hierarchy:
        bin for the levels, convert, density (+h) and force over the levels,
        kick/drift fused with the write-back.  Needs ws_flags=WS_LEVELS."""
        self.bin_levels(level_min, level_max, h_margin)
        self.aos_to_soa(FIELDS_FORCE, prec)
        self.density_levels(newton_steps)
        self.force_levels()
        self.kick_drift_writeback(dt, dt, out_fields)

    def step(self, dt: float, newton_steps: int = 5, prec=None, cell_edge: float = 0.0,
             reorder: bool = False, out_fields: int = FIELDS_OUTPUT):
        """One SPH time step: bin, convert, density (+h), force, kick/drift
        fused with the write-back (the in-place GPU pipeline of the paper's
        Section 6.3)."""
        self.bin_cells(cell_edge, reorder)
        self.aos_to_soa(FIELDS_FORCE, prec)
        self.density(newton_steps)
        self.force()
        self.kick_drift_writeback(dt, dt, out_fields)

    # --- inspection
    def stats(self) -> dict:
        st, s = sph_get_stats(self.ctx)
        _check(st, "sph_get_stats", allow=(0, -7))
        return {"pairs_density": s.pairs_density, "pairs_force": s.pairs_force,
                "tests_density": s.tests_density, "tests_force": s.tests_force,
                "hcap_clamps": s.hcap_clamps, "error_bits": s.error_bits,
                "ncell": tuple(s.ncell), "nitems": s.nitems, "max_occupancy": s.max_occupancy,
                "launches": s.launches, "status": st}

    def reset_stats(self):
        _check(sph_reset_stats(self.ctx), "sph_reset_stats")

    def set_kernel_events(self, which: int, ev_begin=None, ev_end=None):
        """Record two torch.cuda.Events (enable_timing=True) around the
        density (KEV_DENSITY) or force (KEV_FORCE) pair kernel of every later
        call; None for both clears.  The events must stay alive while set."""
        handles = []
        for ev in (ev_begin, ev_end):
            if ev is None:
                handles.append(None)
                continue
            if not ev.cuda_event:            # torch creates the event at its first record
                ev.record(self.stream)
            handles.append(ev.cuda_event)
        _check(sph_set_kernel_events(self.ctx, which, handles[0], handles[1]), "sph_set_kernel_events")

    def set_tuning(self, block_threads=0, ctas_per_sm=0, stage_density=0, stage_force=0,
                   subcells=0, item_order=-1, class_launches=-1, pair_kernel=-1, block_threads_force=0):
        t = sph_tuning(block_threads, ctas_per_sm, stage_density, stage_force, subcells,
                       item_order, class_launches, pair_kernel, block_threads_force)
        _check(sph_set_tuning(self.ctx, t), "sph_set_tuning")

    def tuning(self) -> dict:
        st, t = sph_get_tuning(self.ctx)
        _check(st, "sph_get_tuning")
        return {"block_threads": t.block_threads, "ctas_per_sm": t.ctas_per_sm,
                "stage_density": t.stage_density, "stage_force": t.stage_force,
                "subcells": t.subcells, "item_order": t.item_order,
                "class_launches": t.class_launches, "pair_kernel": t.pair_kernel,
                "block_threads_force": t.block_threads_force}

    def describe(self) -> sph_desc:
        st, d = sph_describe(self.ctx)
        _check(st, "sph_describe")
        return d

    def _ws_view(self, off: int, count: int, dtype):
        torch = self.torch
        es = torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + count * es].view(dtype)

    def perm(self):
        d = self.describe()
        return self._ws_view(d.off_perm, self.n, self.torch.int32)

    def slot_cell(self):
        d = self.describe()
        return self._ws_view(d.off_cell_of_slot, self.n, self.torch.int32)

    def levels(self):
        """Level of every slot (int8; level mode)."""
        d = self.describe()
        if d.off_level < 0:
            raise SphError(-2, "levels: workspace created without WS_LEVELS")
        return self._ws_view(d.off_level, self.n, self.torch.int8)

    def cell_start(self):
        d = self.describe()
        nc = d.ncell[0] * d.ncell[1] * d.ncell[2] * d.subcells ** 3
        return self._ws_view(d.off_cell_start, nc + 1, self.torch.int32)

    def nngb(self, force: bool = False):
        d = self.describe()
        return self._ws_view(d.off_nngb_force if force else d.off_nngb, self.n, self.torch.int32)

    def density_flags(self):
        """Per-slot flags of the last density call (uint8, PFLAG_* bits)."""
        d = self.describe()
        return self._ws_view(d.off_density_flags, self.n, self.torch.uint8)

    def soa_raw(self, field: str, comp: int = 0):
        """The stored words of one SoA component (float32, 16-bit codes, or the
        uint32 words of a packed stream)."""
        torch = self.torch
        d = self.describe()
        f = FIELD_NAMES.index(field)
        fmt = d.prec[f]
        off = d.off_soa[f][comp]
        if fmt == P_FP32:
            return self._ws_view(off, self.n, torch.float32)
        if fmt in (P_BF16, P_FP16):
            return self._ws_view(off, self.n, torch.int16)
        bits = 25 if fmt == P_FP32_M16 else (19 if fmt == P_FP32_M10 else 9 + (fmt - 100))
        return self._ws_view(off, (self.n * bits + 31) // 32, torch.int32)

    def close(self):
        if getattr(self, "ctx", None):
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""FP64 CPU oracle for the SPH hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The CUDA library (``paper_2512_05516_gb300``) never
imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain FP64 C, compiled with
``-ffp-contract=off`` so that x86 and Arm give identical bits); this module only
marshals numpy arrays through ctypes and composes the calls in the order of one
SPH time step (density with h iteration, equation of state, force, kick/drift).
Paper anchors: Eq. 6 (density), Eq. 7 (momentum), Eq. 5 (energy), Table 2
(storage formats).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

FMT = {"fp32": 0, "bf16": 1, "fp16": 2, "m16": 3, "m10": 4}
FMT_BITS = {"fp32": 32, "bf16": 16, "fp16": 16, "m16": 25, "m10": 19}
# the truncated family at every width: "m<n>" keeps n mantissa bits, n in 1..22
for _n in range(1, 23):
    FMT.setdefault(f"m{_n}", 100 + _n)
    FMT_BITS.setdefault(f"m{_n}", 9 + _n)
FLAG_HCAP, FLAG_NEWTON, FLAG_NONFINITE = 1, 2, 4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, OpenMP, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_d = C.c_double
_i32 = C.c_int32
_i64 = C.c_int64
_p = C.c_void_p


def _declare(L):
    for name in ("orc_w", "orc_dw"):
        getattr(L, name).restype = _d
        getattr(L, name).argtypes = [_d]
    for name in ("orc_W", "orc_dWdr", "orc_dWdh"):
        getattr(L, name).restype = _d
        getattr(L, name).argtypes = [_d, _d]
    for name in ("orc_trunc64", "orc_trunc_half"):
        getattr(L, name).restype = None
        getattr(L, name).argtypes = [_i64, _p, C.c_int, _p]
    L.orc_bin.restype = C.c_int
    L.orc_bin.argtypes = [_i64, _p, _p, _p, _p, _p, _p]
    L.orc_bin_sub.restype = C.c_int
    L.orc_bin_sub.argtypes = [_i64, _p, _p, _p, C.c_int32, _p, _p, _p]
    L.orc_levels.restype = C.c_int
    L.orc_levels.argtypes = [_i64, _p, _p, _p, C.c_int32, C.c_int32, _d, _p, _p, _p]
    L.orc_density.restype = None
    L.orc_density.argtypes = [_i64, _p, _p, _p, _p, _d, _d, C.c_int, C.c_int, _i64, _p,
                              _p, _p, _p, _p, _p, _p]
    L.orc_eos.restype = None
    L.orc_eos.argtypes = [_i64, _p, _p, _d, _p, _p]
    L.orc_force.restype = None
    L.orc_force.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _p, _p, _d, _d, _d, C.c_int,
                            _i64, _p, _p, _p, _p]
    L.orc_buffer_density.restype = None
    L.orc_buffer_density.argtypes = [_i64, _i32, _p, _p, _p, _p, _p, _d, _p, _p, _p, _p]
    L.orc_buffer_force.restype = None
    L.orc_buffer_force.argtypes = [_i64, _i32, _p, _p, _p, _p, _p, _p, _p, _p, _d, _d, _d,
                                   _p, _p, _p]
    L.orc_kick_drift.restype = None
    L.orc_kick_drift.argtypes = [_i64, _p, _p, _p, _p, _p, _d, _d, _p]
    L.orc_ball_mark.restype = _i64
    L.orc_ball_mark.argtypes = [_i64, _p, _p, _d, _i64, _p, _p]
    L.orc_quantize.restype = None
    L.orc_quantize.argtypes = [_i64, _p, C.c_int, _p, _p]
    L.orc_pack_bits.restype = None
    L.orc_pack_bits.argtypes = [_i64, _p, C.c_int, _p]
    L.orc_unpack_bits.restype = None
    L.orc_unpack_bits.argtypes = [_i64, _p, C.c_int, _p]
    for name, rt, at in (("orc_f32_bits", C.c_uint32, [_d]),
                         ("orc_f32_value", _d, [C.c_uint32]),
                         ("orc_f16_from_f32", C.c_uint16, [C.c_uint32]),
                         ("orc_f32_from_f16", C.c_uint32, [C.c_uint16]),
                         ("orc_bf16_from_f32", C.c_uint16, [C.c_uint32]),
                         ("orc_f32_from_bf16", C.c_uint32, [C.c_uint16]),
                         ("orc_trunc_code", C.c_uint32, [C.c_uint32, C.c_int]),
                         ("orc_f32_from_trunc", C.c_uint32, [C.c_uint32, C.c_int]),
                         ("orc_fmt_bits", C.c_int, [C.c_int])):
        getattr(L, name).restype = rt
        getattr(L, name).argtypes = at


def _ptr(a):
    return a.ctypes.data_as(_p) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- kernel W
def w(q):
    return lib().orc_w(float(q))


def dw(q):
    return lib().orc_dw(float(q))


def W(r, h):
    return lib().orc_W(float(r), float(h))


def dWdr(r, h):
    return lib().orc_dWdr(float(r), float(h))


def dWdh(r, h):
    return lib().orc_dWdh(float(r), float(h))


# ---------------------------------------------------------------- binning
def bin_cells(x, box, nc, sub=1):
    """Stable binning into cells split into sub^3 sub-cells.  Returns
    (key[n] int32, perm[n] int64, start[ncell sub^3 + 1] int64) where key is
    cell * sub^3 + sub-cell."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    nc = np.ascontiguousarray(nc, dtype=np.int32)
    ncell = int(np.prod(nc.astype(np.int64))) * sub ** 3
    cell_of = np.zeros(n, np.int32)
    perm = np.zeros(n, np.int64)
    start = np.zeros(ncell + 1, np.int64)
    rc = lib().orc_bin_sub(n, _ptr(x), _ptr(_f64(box)), _ptr(nc), int(sub), _ptr(cell_of),
                           _ptr(perm), _ptr(start))
    if rc != 0:
        raise ValueError("orc_bin failed")
    return cell_of, perm, start


def levels(x, h, box, level_min, level_max, margin=0.0):
    """The level hierarchy's binning (every particle has its own h, Section 2;
    the cells of each level hold the support of its particles): Morton key of
    every particle's finest cell (2^level_max per axis), its level from h, and
    the stable order by key.  Returns (key[n] int32, level[n] int8,
    perm[n] int64)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    key = np.zeros(n, np.int32)
    lev = np.zeros(n, np.int8)
    perm = np.zeros(n, np.int64)
    rc = lib().orc_levels(n, _ptr(x), _ptr(_f64(h)), _ptr(_f64(box)), int(level_min), int(level_max),
                          float(margin), _ptr(key), _ptr(lev), _ptr(perm))
    if rc != 0:
        raise ValueError("orc_levels: bad levels")
    return key, lev, perm


def grid_dims(box, cell_edge):
    """Cells per axis floor(L / edge) for a requested edge (the library's rule)."""
    return np.array([int(np.floor(b / cell_edge)) for b in box], dtype=np.int32)


# ---------------------------------------------------------------- density
def density(x, m, h, box, eta, h_cap, newton_steps=0, brute=False, targets=None):
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    m = _f64(m)
    h = _f64(h)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else t.shape[0]
    rho = np.zeros(nt)
    hout = np.zeros(nt)
    drdh = np.zeros(nt)
    nngb = np.zeros(nt, np.int32)
    flags = np.zeros(nt, np.int32)
    pairs = np.zeros(nt, np.int64)
    lib().orc_density(n, _ptr(x), _ptr(m), _ptr(h), _ptr(_f64(box)), float(eta),
                      float(h_cap), int(newton_steps), int(bool(brute)), nt, _ptr(t),
                      _ptr(rho), _ptr(hout), _ptr(drdh), _ptr(nngb), _ptr(flags), _ptr(pairs))
    return {"rho": rho, "h": hout, "drho_dh": drdh, "nngb": nngb, "flags": flags,
            "pairs_all": pairs}


def eos(rho, u, gamma):
    rho = _f64(rho)
    u = _f64(u)
    P = np.zeros_like(rho)
    c = np.zeros_like(rho)
    lib().orc_eos(rho.shape[0], _ptr(rho), _ptr(u), float(gamma), _ptr(P), _ptr(c))
    return P, c


def force(x, v, m, h, rho, P, c, box, alpha, beta, eps, brute=False, targets=None):
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    n = x.shape[0]
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else t.shape[0]
    a = np.zeros((nt, 3))
    dudt = np.zeros(nt)
    nngb = np.zeros(nt, np.int32)
    lib().orc_force(n, _ptr(x), _ptr(v), _ptr(_f64(m)), _ptr(_f64(h)), _ptr(_f64(rho)),
                    _ptr(_f64(P)), _ptr(_f64(c)), _ptr(_f64(box)), float(alpha), float(beta),
                    float(eps), int(bool(brute)), nt, _ptr(t), _ptr(a), _ptr(dudt), _ptr(nngb))
    return {"a": a, "dudt": dudt, "nngb": nngb}


def kick_drift(x, v, a, u, dudt, dt_kick, dt_drift, box):
    """Returns updated copies (x, v, u)."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    u = _f64(u).copy()
    lib().orc_kick_drift(x.shape[0], _ptr(x), _ptr(v), _ptr(_f64(a, (-1, 3))), _ptr(u),
                         _ptr(_f64(dudt)), float(dt_kick), float(dt_drift), _ptr(_f64(box)))
    return x, v, u


# ---------------------------------------------------------------- buffers
def buffer_density(x, m, h, u, box, gamma, B):
    """Density over each particle's buffer of B consecutive particles (Section 6
    benchmark grouping; Eq. 6, h fixed, self included) and the EOS."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    rho, P, c = np.zeros(n), np.zeros(n), np.zeros(n)
    nngb = np.zeros(n, np.int32)
    lib().orc_buffer_density(n, int(B), _ptr(x), _ptr(_f64(m)), _ptr(_f64(h)), _ptr(_f64(u)),
                             _ptr(_f64(box)), float(gamma), _ptr(rho), _ptr(P), _ptr(c), _ptr(nngb))
    return {"rho": rho, "P": P, "c": c, "nngb": nngb}


def buffer_force(x, v, m, h, rho, P, c, box, alpha, beta, eps, B):
    """Force over each particle's buffer of B consecutive particles (Eq. 7, Eq. 5)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    a = np.zeros((n, 3))
    dudt = np.zeros(n)
    nngb = np.zeros(n, np.int32)
    lib().orc_buffer_force(n, int(B), _ptr(x), _ptr(_f64(v, (-1, 3))), _ptr(_f64(m)), _ptr(_f64(h)),
                           _ptr(_f64(rho)), _ptr(_f64(P)), _ptr(_f64(c)), _ptr(_f64(box)),
                           float(alpha), float(beta), float(eps), _ptr(a), _ptr(dudt), _ptr(nngb))
    return {"a": a, "dudt": dudt, "nngb": nngb}


def buffer_relative(x, box, B, fmt="fp32", exp2=0):
    """Positions as the library stores them in buffer mode: the offset from the
    buffer's first particle, moved to the nearest periodic image (FP64: one
    subtraction, then -L when >= L/2 or +L when < -L/2), rounded to `fmt`.
    Returns (origins per particle, offsets as stored)."""
    x = _f64(x, (-1, 3))
    box = _f64(box)
    n = x.shape[0]
    origin = x[(np.arange(n) // B) * B]
    d = x - origin
    d = np.where(d >= 0.5 * box, d - box, np.where(d < -0.5 * box, d + box, d))
    q, _ = quantize(d.ravel(), fmt, exp2)
    return origin, q.reshape(d.shape)


def ball_mark(x, box, radius, targets):
    x = _f64(x, (-1, 3))
    t = np.ascontiguousarray(targets, dtype=np.int64)
    mark = np.zeros(x.shape[0], np.uint8)
    lib().orc_ball_mark(x.shape[0], _ptr(x), _ptr(_f64(box)), float(radius), t.shape[0],
                        _ptr(t), _ptr(mark))
    return mark.astype(bool)


# ---------------------------------------------------------------- quantisers
def quantize(values, fmt, exp2=0):
    """Returns (value as FP64, integer code) of each input in storage format
    `fmt`.  With a storage scale 2^exp2 the code is that of value * 2^exp2 and
    the value returned is the decoded code times 2^-exp2 (powers of two scale
    exactly in FP64)."""
    v = np.ldexp(_f64(values).ravel(), int(exp2))
    out = np.zeros_like(v)
    code = np.zeros(v.shape, np.uint32)
    lib().orc_quantize(v.shape[0], _ptr(v), FMT[fmt], _ptr(out), _ptr(code))
    return np.ldexp(out, -int(exp2)), code


def truncate_bits(values, total_bits):
    """Values as stored in `total_bits` bits by Table 2's family: 64 bits keep
    the double; 63..33 the double layout with total - 12 mantissa bits; 32
    single (round to nearest even); 31..17 the single layout with total - 9
    mantissa bits; 16 half; 15..10 the half layout with total - 6 mantissa
    bits.  The truncated widths drop the low mantissa bits (toward zero).
    Table 2 prints the mantissa ranges as 51..24 and 22..11, which do not add
    up to its own total widths 33 and 17; the mantissa here is always the
    total minus the sign and exponent bits."""
    v = _f64(values).ravel()
    out = np.empty_like(v)
    t = int(total_bits)
    if t == 64:
        out[:] = v
    elif 33 <= t <= 63:
        lib().orc_trunc64(v.shape[0], _ptr(v), t - 12, _ptr(out))
    elif t == 32:
        out = quantize(v, "fp32")[0]
    elif 17 <= t <= 31:
        out = quantize(v, f"m{t - 9}")[0]
    elif t == 16:
        out = quantize(v, "fp16")[0]
    elif 10 <= t <= 15:
        lib().orc_trunc_half(v.shape[0], _ptr(v), t - 6, _ptr(out))
    else:
        raise ValueError(f"no storage format of {t} bits")
    return out.reshape(np.shape(values))


def pack_bits(codes, bits):
    c = np.ascontiguousarray(codes, dtype=np.uint32)
    words = np.zeros((c.shape[0] * bits + 31) // 32, np.uint32)
    lib().orc_pack_bits(c.shape[0], _ptr(c), int(bits), _ptr(words))
    return words


def unpack_bits(words, n, bits):
    w_ = np.ascontiguousarray(words, dtype=np.uint32)
    out = np.zeros(n, np.uint32)
    lib().orc_unpack_bits(n, _ptr(w_), int(bits), _ptr(out))
    return out


def cell_relative(x, box, nc, fmt="fp32", exp2=0):
    """Positions as the library stores them: the offset from the particle's cell
    origin (k * L/nc, k from the binning rule) rounded to `fmt` (under the
    storage scale 2^exp2), added back to the origin in FP64.  Returns
    (positions, offsets-as-stored)."""
    x = _f64(x, (-1, 3))
    box = _f64(box)
    nc = np.asarray(nc, dtype=np.int64)
    inv = nc.astype(np.float64) / box
    k = np.floor(x * inv)
    k = np.clip(k, 0, nc - 1)
    edge = box / nc.astype(np.float64)
    origin = k * edge
    off = x - origin
    q, _ = quantize(off.ravel(), fmt, exp2)
    q = q.reshape(off.shape)
    return origin + q, q


# ---------------------------------------------------------------- composition
def step(wl, newton_steps=None, targets=None, dt=None, with_kick_drift=True):
    """One SPH step on an sph_inputs.Workload in FP64: density with h iteration,
    EOS, force, kick/drift.  With `targets`, density/EOS are evaluated on every
    particle within 2*h_cap of a target (all that the targets' forces need) and
    the force on the targets only; kick/drift is then skipped.  The sampled
    result also carries ``h_all``: the h the force read for every particle (the
    iterated h inside the targets' balls, the input h elsewhere)."""
    x = wl.col("x")
    v = wl.col("v")
    m = wl.col("m")
    h0 = wl.col("h")
    u = wl.col("u")
    ns = wl.newton_steps if newton_steps is None else newton_steps
    out = {}
    if targets is None:
        d = density(x, m, h0, wl.box, wl.eta, wl.h_cap, ns)
        P, c = eos(d["rho"], u, wl.gamma)
        f = force(x, v, m, d["h"], d["rho"], P, c, wl.box, wl.alpha_av, wl.beta_av, wl.eps_av)
        out.update(rho=d["rho"], h=d["h"], nngb=d["nngb"], flags=d["flags"], P=P, c=c,
                   a=f["a"], dudt=f["dudt"], nngb_force=f["nngb"])
        if with_kick_drift:
            dtk = wl.dt if dt is None else dt
            xn, vn, un = kick_drift(x, v, f["a"], u, f["dudt"], dtk, dtk, wl.box)
            out.update(x_new=xn, v_new=vn, u_new=un)
        return out
    targets = np.asarray(targets, dtype=np.int64)
    mark = ball_mark(x, wl.box, 2.0 * wl.h_cap, targets)
    sub = np.nonzero(mark)[0]
    d = density(x, m, h0, wl.box, wl.eta, wl.h_cap, ns, targets=sub)
    rho = np.zeros(wl.n)
    hh = np.array(h0, dtype=np.float64)
    rho[sub] = d["rho"]
    hh[sub] = d["h"]
    P = np.zeros(wl.n)
    c = np.zeros(wl.n)
    Ps, cs = eos(d["rho"], u[sub], wl.gamma)
    P[sub] = Ps
    c[sub] = cs
    # particles outside `sub` cannot be within h_i + h_j <= 2 h_cap of a target
    rho[~mark] = 1.0
    f = force(x, v, m, hh, rho, P, c, wl.box, wl.alpha_av, wl.beta_av, wl.eps_av,
              targets=targets)
    pos = np.searchsorted(sub, targets)
    out.update(rho=d["rho"][pos], h=d["h"][pos], nngb=d["nngb"][pos], flags=d["flags"][pos],
               P=Ps[pos], c=cs[pos], a=f["a"], dudt=f["dudt"], nngb_force=f["nngb"],
               h_all=hh)
    return out

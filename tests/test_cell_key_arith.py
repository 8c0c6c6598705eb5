"""Host check of the arithmetic the binning kernels use for a cell coordinate
on the FP32 pipe (the device function cell_coord_fast in csrc/k_cellkey.cuh):
every FP32 step emulated exactly (rational arithmetic, round to nearest even),
against the definition floor(fl64(x * inv)) clamped to [0, n-1].  The device
takes the FP64 product itself whenever the FP32 pair lands within 2^-20 of an
integer; the check counts those fallbacks and requires agreement everywhere
else, on random positions, on every face of several grids and on the faces'
neighbouring doubles."""
import math
import random
import struct
from fractions import Fraction

import numpy as np


def _f32(v) -> float:
    """The FP32 value nearest to the rational (or float) v, ties to even."""
    fr = Fraction(v)
    f = float(np.float32(float(fr)))
    best = f
    for g in (float(np.nextafter(np.float32(f), np.float32(-np.inf))),
              float(np.nextafter(np.float32(f), np.float32(np.inf)))):
        dg, db = abs(Fraction(g) - fr), abs(Fraction(best) - fr)
        if dg < db or (dg == db and (struct.unpack("<I", struct.pack("<f", g))[0] & 1) == 0):
            best = g
    return best


def _mul(a, b):
    return _f32(Fraction(a) * Fraction(b))


def _add(a, b):
    return _f32(Fraction(a) + Fraction(b))


def _fma(a, b, c):
    return _f32(Fraction(a) * Fraction(b) + Fraction(c))


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _from_bits32(i: int) -> float:
    return struct.unpack("<f", struct.pack("<i", i))[0]


def _definition(x: float, inv: float, n: int) -> int:
    v = x * inv
    if v != v:
        return 0
    f = math.floor(v) if abs(v) < 1e300 else (n if v > 0 else -1)
    return min(max(f, 0), n - 1)


def _fast(x: float, inv: float, n: int):
    """(coordinate, took the FP64 product)"""
    ih = float(np.float32(inv))
    il = float(np.float32(inv - ih))
    b = _bits(x)
    if b == 0:
        return 0, False
    e = b >> 52
    if e < 949 or e >= 1123:
        return _definition(x, inv, n), True
    m = b & 0xFFFFFFFFFFFFF
    hi = _from_bits32(((e - 896) << 23) | (m >> 29))
    lo = _mul(_f32(m & 0x1FFFFFFF), _from_bits32((e - 948) << 23))
    p = _mul(hi, ih)
    t = _add(_fma(hi, ih, -p), _fma(hi, il, _mul(lo, ih)))
    fl = float(math.floor(p))
    d = _add(_add(p, -fl), t)
    if d < 0:
        fl, d = _add(fl, -1.0), _add(d, 1.0)
    elif d >= 1:
        fl, d = _add(fl, 1.0), _add(d, -1.0)
    if d < 2.0 ** -20 or d > 1.0 - 2.0 ** -20:
        return _definition(x, inv, n), True
    return min(max(int(fl), 0), n - 1), False


def test_fp32_pair_floor_equals_the_fp64_definition():
    rng = random.Random(11)
    total = fallbacks = 0
    for L, n in ((1.0, 51), (2.0, 8192), (1.0, 24), (0.3, 97), (1.0, 6), (123.4, 4095)):
        inv = n / L
        xs = [rng.random() * L for _ in range(1500)]
        faces = [k * L / n for k in range(n + 1)]
        if len(faces) > 400:
            faces = rng.sample(faces, 400)
        xs += faces
        xs += [math.nextafter(f, -1.0) for f in faces] + [math.nextafter(f, 2.0 * L) for f in faces]
        xs += [math.nextafter(L, 0.0), L, -0.0, 1e-300, 5e-324, 2.0 ** -74, 2.0 ** -75, 1e30, -1.0,
               float("inf"), float("nan")]
        for x in xs:
            got, fb = _fast(x, inv, n)
            assert got == _definition(x, inv, n), (x, L, n)
            total += 1
            fallbacks += fb
    # the FP64 product is the exception: faces, their neighbours and the
    # out-of-range inputs, not the random positions
    assert fallbacks < total // 2

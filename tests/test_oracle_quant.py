"""Pins of the oracle's storage quantisers (Table 2 and bfloat16) and of the
packed N-bit bitstream (Section 3.2).

IEEE half and bfloat16 are checked exhaustively against numpy's and torch's
own conversions; the truncated formats against the definition "keep sign,
exponent and the top N mantissa bits"; the bitstream against hand-packed words.
"""
import numpy as np
import pytest


def test_half_decode_exhaustive(orc):
    L = orc.lib()
    codes = np.arange(65536, dtype=np.uint32)
    ref = codes.astype(np.uint16).view(np.float16).astype(np.float32).view(np.uint32)
    got = np.array([L.orc_f32_from_f16(int(c)) for c in codes], dtype=np.uint32)
    nan = np.isnan(codes.astype(np.uint16).view(np.float16))
    assert np.array_equal(got[~nan], ref[~nan])
    assert np.all(np.isnan(got[nan].view(np.float32)))


def test_half_encode_roundtrip_exhaustive(orc):
    L = orc.lib()
    codes = np.arange(65536, dtype=np.uint32)
    f = codes.astype(np.uint16).view(np.float16)
    finite = ~np.isnan(f)
    fbits = f.astype(np.float32).view(np.uint32)
    back = np.array([L.orc_f16_from_f32(int(b)) for b in fbits], dtype=np.uint32)
    assert np.array_equal(back[finite], codes[finite])


def test_half_encode_matches_numpy_rne(orc):
    rng = np.random.default_rng(0)
    # spread over half's normal, subnormal, overflow and underflow ranges
    e = rng.uniform(-30, 17, 200_000)
    vals = (np.sign(rng.uniform(-1, 1, e.size)) * 2.0 ** e).astype(np.float32)
    # exact ties between neighbouring halves
    h = rng.integers(1, 0x7BFF, 5000).astype(np.uint16).view(np.float16).astype(np.float32)
    h2 = (h.view(np.uint32) + np.uint32(1 << 12)).view(np.float32)  # midpoints of normals
    vals = np.concatenate([vals, h2, np.array([65504, 65519.99, 65520, 2 ** -25, 2 ** -24,
                                               3 * 2 ** -26, 0.0, -0.0], np.float32)])
    _, code = orc.quantize(vals.astype(np.float64), "fp16")
    ref = vals.astype(np.float16).view(np.uint16).astype(np.uint32)
    assert np.array_equal(code, ref)


def test_bf16_matches_torch_rne(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    vals = (rng.standard_normal(200_000) * 10.0 ** rng.uniform(-30, 30, 200_000)).astype(np.float32)
    ties = (rng.integers(0, 1 << 31, 2000, dtype=np.uint32) & np.uint32(0xFFFF0000)) | np.uint32(0x8000)
    vals = np.concatenate([vals, ties.view(np.float32)])
    vals = vals[np.isfinite(vals)]
    _, code = orc.quantize(vals.astype(np.float64), "bf16")
    ref = torch.from_numpy(vals).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(code, ref.astype(np.uint32))


def test_fp32_is_ieee_rounding(orc):
    rng = np.random.default_rng(2)
    d = rng.standard_normal(100_000) * 10.0 ** rng.uniform(-20, 20, 100_000)
    v, code = orc.quantize(d, "fp32")
    assert np.array_equal(code, d.astype(np.float32).view(np.uint32))
    assert np.array_equal(v, d.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("fmt,mant", [("m16", 16), ("m10", 10), ("m1", 1), ("m7", 7), ("m13", 13),
                                      ("m22", 22)])
def test_truncated_formats(orc, fmt, mant):
    rng = np.random.default_rng(3)
    d = rng.standard_normal(100_000) * 10.0 ** rng.uniform(-10, 10, 100_000)
    v, code = orc.quantize(d, fmt)
    f = d.astype(np.float32)
    # Table 2: total size 1 + 8 + N bits
    assert orc.FMT_BITS[fmt] == 1 + 8 + mant
    assert np.all(code < (1 << (1 + 8 + mant)))
    # truncation toward zero: |value| <= |x|, same sign, error below one unit
    # of the kept mantissa
    assert np.all(np.abs(v) <= np.abs(f.astype(np.float64)))
    assert np.all(np.sign(v) == np.sign(f))
    ulp = 2.0 ** (np.floor(np.log2(np.abs(f.astype(np.float64)))) - mant)
    assert np.all(np.abs(f - v) < ulp)
    # the dropped low bits are zero and the kept bits unchanged
    vb = v.astype(np.float32).view(np.uint32)
    assert np.all(vb & np.uint32((1 << (23 - mant)) - 1) == 0)
    assert np.all((vb >> np.uint32(23 - mant)) == (f.view(np.uint32) >> np.uint32(23 - mant)))
    # specials survive
    sv, _ = orc.quantize(np.array([np.inf, -np.inf, np.nan, 0.0]), fmt)
    assert sv[0] == np.inf and sv[1] == -np.inf and np.isnan(sv[2]) and sv[3] == 0.0


def test_pack_bits_hand_example(orc):
    # codes 1, 2, 3 of 19 bits: bits 0..18 hold 1, bits 19..37 hold 2 (bit 20 set),
    # bits 38..56 hold 3 (word 1, bits 6 and 7)
    w = orc.pack_bits([1, 2, 3], 19)
    assert list(w) == [0x00100001, 0x000000C0]
    assert list(orc.unpack_bits(w, 3, 19)) == [1, 2, 3]


@pytest.mark.parametrize("bits", [19, 25, 16, 32])
def test_pack_unpack_roundtrip(orc, bits):
    rng = np.random.default_rng(bits)
    n = 1000
    codes = rng.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32)
    w = orc.pack_bits(codes, bits)
    assert w.size == (n * bits + 31) // 32
    assert np.array_equal(orc.unpack_bits(w, n, bits), codes)
    # 32 consecutive codes fill exactly `bits` words
    w32 = orc.pack_bits(codes[:32], bits)
    assert w32.size == bits


def test_scaled_half_keeps_eleven_bits_of_a_subnormal_mass(orc):
    # Sod's particle mass (1/124)^3 = 5.2e-7 is an FP16 subnormal (spacing
    # 2^-24): stored unscaled it keeps 4 significant bits; under the storage
    # scale 2^20 it is a normal half with 11.  The code is numpy's half of
    # the scaled FP32 value, and the decoded value is within half an ulp.
    m = (1.0 / 124.0) ** 3
    q0, _ = orc.quantize([m], "fp16")
    assert abs(q0[0] - m) / m > 1e-2                      # the unscaled damage
    assert q0[0] == round(m / 2.0 ** -24) * 2.0 ** -24    # nearest subnormal
    q, code = orc.quantize([m], "fp16", exp2=20)
    ref = np.float32(m * 2.0 ** 20).astype(np.float16)
    assert code[0] == int(ref.view(np.uint16))
    assert q[0] == float(ref) * 2.0 ** -20
    assert abs(q[0] - m) <= 2.0 ** -11 * 2.0 ** np.floor(np.log2(m))
    # a negative exponent brings Sedov's peak energy 262144 under 65504
    q, _ = orc.quantize([262144.0, 1e-6], "fp16", exp2=-7)
    assert q[0] == 262144.0
    assert q[1] == 0.0                                    # 1e-6 * 2^-7 underflows


def test_truncated_family_matches_the_named_widths(orc):
    # "m16"/"m10" and the generic codes of the same width are one format
    rng = np.random.default_rng(4)
    d = rng.standard_normal(10_000) * 10.0 ** rng.uniform(-5, 5, 10_000)
    for n in (16, 10):
        v0, c0 = orc.quantize(d, f"m{n}")
        L = orc.lib()
        out = np.zeros_like(d)
        code = np.zeros(d.shape, np.uint32)
        L.orc_quantize(d.shape[0], orc._ptr(d), 100 + n, orc._ptr(out), orc._ptr(code))
        assert np.array_equal(code, c0) and np.array_equal(out, v0)


def test_truncate_64_bits_and_52_mantissa_bits_are_the_identity(orc):
    rng = np.random.default_rng(40)
    v = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.integers(-300, 300, 1000),
                        [0.0, -0.0, 5e-324, -2.2e-308, np.inf, -np.inf, 1.0 + 2.0 ** -52]])
    for t in (64,):
        assert np.array_equal(orc.truncate_bits(v, t).view(np.uint64), v.view(np.uint64))
    out = np.empty_like(v)
    orc.lib().orc_trunc64(v.shape[0], v.ctypes.data, 52, out.ctypes.data)
    assert np.array_equal(out.view(np.uint64), v.view(np.uint64))
    nan = np.array([np.nan])
    assert np.isnan(orc.truncate_bits(nan, 40)[0])


def test_truncate_bits_hand_values(orc):
    # 1 + 2^-52 keeps its last bit only at 52 mantissa bits (64 total)
    one = np.array([1.0 + 2.0 ** -52, -(1.0 + 2.0 ** -30 + 2.0 ** -52)])
    assert np.array_equal(orc.truncate_bits(one, 63), [1.0, -(1.0 + 2.0 ** -30)])
    assert np.array_equal(orc.truncate_bits(one, 42), [1.0, -(1.0 + 2.0 ** -30)])
    assert np.array_equal(orc.truncate_bits(one, 41), [1.0, -1.0])
    # 4/3 = 1.010101...b: 21 mantissa bits (33 total) keep 1.0101...010b,
    # i.e. 1 + (1 - 2^-20)/3 = 1398101 / 2^20, toward zero for either sign
    x = np.array([4.0 / 3.0, -4.0 / 3.0])
    assert np.array_equal(orc.truncate_bits(x, 33), [1398101 / 2.0 ** 20, -1398101 / 2.0 ** 20])
    # 32 bits: the nearest single; 31 bits: 22 mantissa bits of the single
    # 1.01010101010101010101011b (rounded up at bit 23), cut to 22 bits
    assert orc.truncate_bits(x, 32)[0] == 11184811 / 2.0 ** 23
    assert orc.truncate_bits(x, 31)[0] == 5592405 / 2.0 ** 22
    # 16 bits: half 1.0101010101b (rounded down); 10 bits: 4 mantissa bits 1.0101b
    assert orc.truncate_bits(x, 16)[0] == 1365 / 1024.0
    assert orc.truncate_bits(x, 10)[1] == -21 / 16.0
    # the exponent range follows the layout: 1e-30 is a double and a single,
    # but 0 in half (far below its subnormals), and 1e6 overflows half
    tiny = np.array([1e-30, 1e6])
    assert orc.truncate_bits(tiny, 40)[0] > 0 and orc.truncate_bits(tiny, 20)[0] > 0
    assert orc.truncate_bits(tiny, 12)[0] == 0.0 and np.isinf(orc.truncate_bits(tiny, 12)[1])


def test_truncation_error_shrinks_with_width(orc):
    # truncation toward zero within one layout: each extra mantissa bit at
    # most halves the relative error bound 2^-mant, and the error never grows
    rng = np.random.default_rng(41)
    v = rng.uniform(0.5, 4.0, 20000)
    prev = np.inf
    for t in range(33, 65):
        e = np.max(np.abs(orc.truncate_bits(v, t) - v) / v)
        assert e <= 2.0 ** -(t - 12) and e <= prev
        prev = e
    for t in range(17, 32):
        e = np.max(np.abs(orc.truncate_bits(v, t) - v) / v)
        # the single's own rounding (2^-24) plus the truncation
        assert e <= 2.0 ** -(t - 9) + 2.0 ** -24

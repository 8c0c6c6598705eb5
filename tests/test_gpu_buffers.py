"""Buffer kernels (the paper's benchmark grouping, Section 6): density, force,
kick and drift over contiguous buffers of B co-located particles, every pair
of a buffer, reading the AoS records directly or the converted SoA, against
the FP64 oracle's buffer kernels.

Inputs are the 4x4x4 lattice blocks of sph_inputs.buffer_blocks in the
paper's 144-byte record (FP64 positions, FP32 fields), with a ragged last
buffer.  The oracle is fed the values the records hold (FP32 fields widened),
so only the arithmetic differs: density and P within 1e-5 relative, the
acceleration within 1e-5 of its mean magnitude, the drift to the
rounding of one FP32 (SoA) or FP64 (AoS) update.  Positions stored as SoA are
bit-exact against the oracle's buffer-relative offsets, and the AoS and SoA
sources give bit-identical results in FP32 storage (same positions, same
arithmetic).  du/dt, heavy-tailed on this input, is held to 1e-5 of each
particle's own magnitude plus the mean."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402

R = sph_mod.RECORD_144
DT = 2e-3


def _records(wl, n):
    raw = sph_inputs.pack_records(wl, {k: v for k, v in R.items() if k not in ("cs", "dudt")}, 144,
                                  f32_fields=sph_mod.F32_144)
    raw[:, 0:8] = np.arange(wl.n, dtype=np.int64).view(np.uint8).reshape(-1, 8)
    raw[:, 76:84] = 0
    rng = np.random.default_rng(9)
    raw[:, 44:56] = rng.uniform(-40, 40, (wl.n, 3)).astype(np.float32).view(np.uint8).reshape(-1, 12)
    raw[:, 80:84] = rng.uniform(-3, 3, wl.n).astype(np.float32).view(np.uint8).reshape(-1, 4)
    return np.ascontiguousarray(raw[:n])


def col(raw, name):
    """One field of the 144-byte records as FP64."""
    off = R[name]
    nc = 3 if name in ("x", "v", "a") else 1
    if name == "x":
        out = raw[:, off:off + 24].copy().view(np.float64)
    else:
        out = raw[:, off:off + 4 * nc].copy().view(np.float32).astype(np.float64)
    return out if nc == 3 else out.ravel()


def _setup(B=64, nb=(8, 8, 4), drop=37, seed=21):
    block = {32: (4, 4, 2), 64: (4, 4, 4), 128: (4, 4, 8)}[B]
    wl = sph_inputs.buffer_blocks(nb=nb, block=block, seed=seed)
    n = wl.n - drop
    raw = _records(wl, n)
    return wl, raw, n


def _ctx(wl, raw, B):
    s = make_sph(wl, aos=torch.from_numpy(raw.reshape(-1).copy()).cuda(), layout=sph_mod.layout_144())
    s.bin_buffers(B)
    return s


def _out(s, shape):
    torch.cuda.synchronize()
    return s.aos.cpu().numpy().view(np.uint8).reshape(shape).copy()


def _density(orc, wl, raw, B):
    return orc.buffer_density(col(raw, "x"), col(raw, "m"), col(raw, "h"), col(raw, "u"), wl.box, wl.gamma, B)


@pytest.mark.parametrize("B", [64, 32, 128])
@pytest.mark.parametrize("source", ["aos", "soa"])
def test_buffer_density_matches_oracle(orc, source, B):
    wl, raw, n = _setup(B)
    want = _density(orc, wl, raw, B)
    s = _ctx(wl, raw, B)
    if source == "soa":
        s.aos_to_soa(sph_mod.mask("x", "m", "h", "u"))
    s.buffer_density(source)
    if source == "soa":
        s.soa_to_aos(sph_mod.mask("rho", "P", "cs"))
    out = _out(s, raw.shape)
    for name, ref in (("rho", want["rho"]), ("P", want["P"]), ("cs", want["c"])):
        got = col(out, name)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-5, name
    # untouched bytes: ID, the inputs, padding
    keep = np.ones(144, bool)
    keep[64:68] = keep[72:80] = False
    assert np.array_equal(out[:, keep], raw[:, keep])
    st = s.stats()
    assert st["error_bits"] == 0
    # pairs j != i with r < 2 h_i; FP32 can move a pair within rounding of the support
    total = int(want["nngb"].sum())
    assert abs(st["pairs_density"] - total) <= max(4, total // 100000)
    s.close()


@pytest.mark.parametrize("source", ["aos", "soa"])
def test_buffer_force_matches_oracle(orc, source):
    B = 64
    wl, raw, n = _setup(B, seed=22)
    d = _density(orc, wl, raw, B)
    # the records carry the oracle's density and pressure, rounded to FP32
    raw[:, 64:68] = d["rho"].astype(np.float32).view(np.uint8).reshape(-1, 4)
    raw[:, 72:76] = d["P"].astype(np.float32).view(np.uint8).reshape(-1, 4)
    rho, P = col(raw, "rho"), col(raw, "P")
    c = np.sqrt(wl.gamma * P / rho)
    want = orc.buffer_force(col(raw, "x"), col(raw, "v"), col(raw, "m"), col(raw, "h"), rho, P, c, wl.box,
                            wl.alpha_av, wl.beta_av, wl.eps_av, B)
    s = _ctx(wl, raw, B)
    if source == "soa":
        s.aos_to_soa(sph_mod.mask("x", "v", "m", "h", "rho", "P"))
    s.buffer_force(source)
    if source == "soa":
        s.soa_to_aos(sph_mod.mask("a", "dudt"))
    out = _out(s, raw.shape)
    a = col(out, "a")
    scale = np.mean(np.linalg.norm(want["a"], axis=1))
    assert np.max(np.abs(a - want["a"])) <= 1e-5 * scale
    # du/dt is heavy-tailed here (random velocities drive the viscosity: the
    # largest values are ~10x the mean), so its bound adds each particle's
    # own magnitude to the mean; errors stay near 1e-6 of either
    du = col(out, "dudt")
    ref = want["dudt"]
    assert np.all(np.abs(du - ref) <= 1e-5 * (np.abs(ref) + np.mean(np.abs(ref))))
    # momentum is conserved within every buffer (pair antisymmetry), to FP32 rounding
    m = col(raw, "m")
    for b in range(0, n // B, 17):
        sl = slice(b * B, (b + 1) * B)
        ma = m[sl, None] * a[sl]
        assert np.all(np.abs(ma.sum(axis=0)) <= 1e-5 * np.sum(np.abs(ma)))
    st = s.stats()
    assert st["error_bits"] == 0
    total = int(want["nngb"].sum())
    assert abs(st["pairs_force"] - total) <= max(4, total // 100000)
    s.close()


@pytest.mark.parametrize("source", ["aos", "soa"])
def test_buffer_kick_and_drift(orc, source):
    B = 64
    wl, raw, n = _setup(B, seed=23)
    box = np.asarray(wl.box)
    s = _ctx(wl, raw, B)
    if source == "soa":
        s.aos_to_soa(sph_mod.mask("x", "v", "a", "u", "dudt"))
    s.buffer_kick(DT, source)
    s.buffer_drift(DT, source)
    if source == "soa":
        s.soa_to_aos(sph_mod.mask("x", "v", "u"))
    out = _out(s, raw.shape)
    x0, v0, a0, u0, du0 = (col(raw, k) for k in ("x", "v", "a", "u", "dudt"))
    xk, vk, uk = orc.kick_drift(x0, v0, a0, u0, du0, DT, 0.0, box)      # kick only
    v1, u1 = col(out, "v"), col(out, "u")
    assert np.max(np.abs(v1 - vk) / (np.abs(vk) + np.abs(a0 * DT))) <= 2.0 ** -23
    assert np.max(np.abs(u1 - uk) / (np.abs(uk) + np.abs(du0 * DT))) <= 2.0 ** -23
    x_want, _, _ = orc.kick_drift(x0, v1, np.zeros_like(a0), u0, du0, 0.0, DT, box)   # drift with the kicked v
    x1 = col(out, "x")
    d = np.abs(x1 - x_want)
    d = np.minimum(d, box - d)
    if source == "aos":
        assert np.max(d) <= 4.0 * np.finfo(np.float64).eps
    else:
        # one FP32 rounding of the offset and one of the update, then FP64 back
        _, off = orc.buffer_relative(x0, box, B, "fp32")
        assert np.all(d <= 2.0 ** -23 * (np.abs(off) + np.abs(v1 * DT)) + 1e-15)
    assert np.all((x1 >= 0.0) & (x1 < box))
    assert s.stats()["error_bits"] == 0
    s.close()


@pytest.mark.parametrize("fmt", ["fp32", "fp16"])
def test_buffer_relative_positions_bit_exact(orc, fmt):
    # the stored offsets are the oracle's (FP64 difference from the buffer's
    # first particle, nearest image, one rounding); the write-back puts
    # origin + offset back, wrapped, exactly as the oracle computes it
    B = 64
    wl, raw, n = _setup(B, seed=24)
    box = np.asarray(wl.box)
    s = _ctx(wl, raw, B)
    s.aos_to_soa(sph_mod.mask("x"), {"x": fmt})
    origin, off = orc.buffer_relative(col(raw, "x"), box, B, fmt)
    for c in range(3):
        got = s.soa_raw("x", c).cpu().numpy()
        _, code = orc.quantize(off[:, c], fmt)
        want = code.view(np.float32) if fmt == "fp32" else code.astype(np.uint16).view(np.int16)
        assert np.array_equal(got, want), c
    s.soa_to_aos(sph_mod.mask("x"))
    out = _out(s, raw.shape)
    y = origin + off
    y = np.where((y < 0) | (y >= box), y - box * np.floor(y / box), y)
    y = np.where(y >= box, 0.0, y)
    assert np.array_equal(col(out, "x"), y)
    # a block straddling the periodic boundary keeps small offsets
    assert np.max(np.abs(off)) < 5 * wl.meta["spacing"]
    s.close()


def test_aos_and_soa_sources_agree_bitwise():
    # FP32 SoA storage holds exactly the values the AoS kernels compute with
    B = 64
    wl, raw, n = _setup(B, seed=25)
    outs = []
    for source in ("aos", "soa"):
        s = _ctx(wl, raw, B)
        if source == "soa":
            s.aos_to_soa(sph_mod.mask("x", "v", "m", "h", "u", "a", "dudt"))
        s.buffer_density(source)
        s.buffer_force(source)
        if source == "soa":
            s.soa_to_aos(sph_mod.mask("rho", "P", "cs", "a", "dudt"))
        outs.append(_out(s, raw.shape))
        s.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("source", ["aos", "soa"])
def test_plain_form_equals_staged(source):
    # reading every partner from global memory (tuning pair_kernel = 1) does
    # the same arithmetic in the same order as the shared-memory stage
    B = 64
    wl, raw, n = _setup(B, seed=28)
    outs = []
    for plain in (0, 1):
        s = _ctx(wl, raw, B)
        s.set_tuning(pair_kernel=plain)
        if source == "soa":
            s.aos_to_soa(sph_mod.mask("x", "v", "m", "h", "u"))
        s.buffer_density(source)
        s.buffer_force(source)
        if source == "soa":
            s.soa_to_aos(sph_mod.mask("rho", "P", "cs", "a", "dudt"))
        outs.append((_out(s, raw.shape), s.stats()["pairs_density"], s.stats()["pairs_force"]))
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:]


@pytest.mark.parametrize("fmt", ["bf16", "fp16", "m10"])
def test_buffer_kernels_reduced_storage(orc, fmt):
    # v, m, h, u stored in a reduced format: the oracle is fed the same
    # quantised values (mode Q), so the results agree to FP32 arithmetic
    B = 64
    wl, raw, n = _setup(B, seed=26)
    prec = {"v": fmt, "m": fmt, "h": fmt, "u": fmt}
    q = {k: orc.quantize(col(raw, k).ravel(), fmt)[0].reshape(col(raw, k).shape) for k in prec}
    d = orc.buffer_density(col(raw, "x"), q["m"], q["h"], q["u"], wl.box, wl.gamma, B)
    s = _ctx(wl, raw, B)
    s.aos_to_soa(sph_mod.mask("x", "v", "m", "h", "u"), prec)
    s.buffer_density("soa")
    s.buffer_force("soa")
    s.soa_to_aos(sph_mod.mask("rho", "P", "a", "dudt"))
    out = _out(s, raw.shape)
    rho = col(out, "rho")
    assert np.max(np.abs(rho - d["rho"]) / d["rho"]) < 1e-5
    P32 = col(out, "P")
    rho32 = rho
    f = orc.buffer_force(col(raw, "x"), q["v"], q["m"], q["h"], rho32, P32, np.sqrt(wl.gamma * P32 / rho32),
                         wl.box, wl.alpha_av, wl.beta_av, wl.eps_av, B)
    scale = np.mean(np.linalg.norm(f["a"], axis=1))
    assert np.max(np.abs(col(out, "a") - f["a"])) <= 1e-5 * scale
    assert s.stats()["error_bits"] == 0
    s.close()


def test_buffer_mode_state_rules():
    B = 64
    wl, raw, n = _setup(B, seed=27)
    s = make_sph(wl, aos=torch.from_numpy(raw.reshape(-1).copy()).cuda(), layout=sph_mod.layout_144())
    with pytest.raises(sph_mod.SphError):
        s.buffer_density("aos")                  # not in buffer mode
    for bad in (0, 16, 48, 512):
        with pytest.raises(sph_mod.SphError):
            s.bin_buffers(bad)
    s.bin_buffers(B)
    with pytest.raises(sph_mod.SphError):
        s.buffer_density(2)                      # no such source
    with pytest.raises(sph_mod.SphError):
        s.buffer_density("soa")                  # SoA inputs not current
    s.aos_to_soa(sph_mod.mask("x", "m", "h", "u"))
    with pytest.raises(sph_mod.SphError):
        s.density(0)                             # cell-list kernels need sph_bin_cells
    s.buffer_density("soa")
    with pytest.raises(sph_mod.SphError):
        s.buffer_kick(float("nan"), "soa")
    # positions may be written back in buffer mode, not after sph_bin_cells
    s.soa_to_aos(sph_mod.mask("x"))
    s.bin_cells(2 * wl.h_cap)
    s.aos_to_soa(sph_mod.mask("x"))
    with pytest.raises(sph_mod.SphError):
        s.soa_to_aos(sph_mod.mask("x"))
    with pytest.raises(sph_mod.SphError):
        s.buffer_force("aos")                    # cell mode again
    s.close()


def test_buffer_step_graph_replay_equals_eager():
    # a whole buffer step (conversion, the four kernels, write-back) captured
    # in a CUDA graph and replayed gives the eager run's records exactly
    B = 64
    wl, raw, n = _setup(B, seed=29)
    fields_in = sph_mod.mask("x", "v", "a", "m", "h", "u", "dudt")
    fields_out = sph_mod.mask("x", "v", "a", "rho", "P", "cs", "u", "dudt")
    prec = {"v": "fp16", "m": "bf16", "h": "m10", "u": "fp16"}

    def run(graph):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            s = make_sph(wl, aos=torch.from_numpy(raw.reshape(-1).copy()).cuda(), layout=sph_mod.layout_144())
            s.set_scale({"m": sph_mod.suggest_scale(float(col(raw, "m").max()), "bf16")})
            s.bin_buffers(B)

            def step():
                s.aos_to_soa(fields_in, prec)
                s.buffer_density("soa")
                s.buffer_force("soa")
                s.buffer_kick(DT, "soa")
                s.buffer_drift(DT, "soa")
                s.soa_to_aos(fields_out)

            step()
            if graph:
                st.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=st):
                    step()
                g.replay()
                g.replay()
            else:
                step()
                step()
        st.synchronize()
        out = s.aos.cpu().numpy().view(np.uint8).reshape(raw.shape).copy()
        assert s.stats()["error_bits"] == 0
        s.close()
        return out

    assert np.array_equal(run(False), run(True))


def test_host_resident_records_equal_device_records():
    # records in pinned host memory, read by the AoS-source kernels over the
    # host link, give the device-resident run's bytes
    B = 64
    wl, raw, n = _setup(B, seed=30)
    outs = []
    for host in (False, True):
        t = torch.from_numpy(raw.reshape(-1).copy())
        s = make_sph(wl, aos=t.pin_memory() if host else t.cuda(), layout=sph_mod.layout_144())
        s.bin_buffers(B)
        s.buffer_density("aos")
        s.buffer_force("aos")
        s.buffer_kick(DT, "aos")
        s.buffer_drift(DT, "aos")
        outs.append(_out(s, raw.shape))
        s.close()
    assert np.array_equal(outs[0], outs[1])

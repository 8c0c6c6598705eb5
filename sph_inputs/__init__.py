"""Seeded synthetic particle sets for the SPH hot path.

This module is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA library (``paper_2512_05516_gb300``).  It draws positions, velocities,
masses and thermodynamic state with numpy's PCG64 and lays them out as FP64
array-of-structs records.  It contains none of the method's arithmetic: no
kernel, no density sum, no force, no quantiser.

The paper publishes no particle inputs (its kernels come from SWIFT and run on
64-particle buffers, Section 6).  The recipes below stand in for them; each
follows one workload description:

* ``uniform_density``  N=4096 uniform-random particles in the unit cube, equal
  masses 1/N, one fixed h giving 48 neighbours on average.
* ``sod``              jittered cubic lattices, dense left half / sparse right
  half (spacing doubled), ideal gas with gamma=5/3.
* ``sedov``            jittered lattice with the blast energy in the 64 central
  particles.
* ``gaussian_mixture`` 8 isotropic Gaussians plus a 20% uniform background,
  one global h with 48 neighbours on average.
* ``gaussian_mixture_adaptive`` the same positions, h per particle from the
  mixture's number density (48 neighbours locally).
* ``long_run``         large jittered lattice with random velocities.
* ``buffer_blocks``    the paper's benchmark grouping: blocks of 4x4x4 (B = 64)
  jittered lattice particles, each block a contiguous buffer of records.

Record layout (the default 112-byte FP64 record): x[3]@0, v[3]@24, a[3]@48,
m@72, h@80, rho@88, u@96, P@104.  The number of neighbours 48 enters only
through eta = 1/2 (3*48/(4 pi))^(1/3), the factor that turns the local spacing
into the initial smoothing length h0 = eta * spacing.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20251205

#: field name -> (byte offset, number of FP64 components) in the 112-byte record
RECORD_112 = {
    "x": (0, 3), "v": (24, 3), "a": (48, 3), "m": (72, 1), "h": (80, 1),
    "rho": (88, 1), "u": (96, 1), "P": (104, 1),
}
RECORD_BYTES = 112
N_NGB = 48.0
ETA = 0.5 * (3.0 * N_NGB / (4.0 * math.pi)) ** (1.0 / 3.0)


@dataclass
class Workload:
    """A synthetic particle set: FP64 AoS records plus the run parameters."""
    name: str
    aos: np.ndarray                      # (N, 14) float64, C-contiguous
    box: tuple
    gamma: float = 5.0 / 3.0
    alpha_av: float = 1.0
    beta_av: float = 2.0
    eps_av: float = 0.01
    eta: float = ETA
    h_cap: float = 0.0                   # upper clamp for h (0: cell_edge / 2)
    cell_edge: float = 0.0               # requested cell edge (0: from h_cap)
    dt: float = 1e-4
    newton_steps: int = 5
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.aos.shape[0])

    def col(self, name: str) -> np.ndarray:
        off, nc = RECORD_112[name]
        c0 = off // 8
        return self.aos[:, c0:c0 + nc] if nc > 1 else self.aos[:, c0]


def _empty(n: int) -> np.ndarray:
    return np.zeros((n, RECORD_BYTES // 8), dtype=np.float64)


def _set(aos, name, val):
    off, nc = RECORD_112[name]
    c0 = off // 8
    if nc > 1:
        aos[:, c0:c0 + nc] = val
    else:
        aos[:, c0] = val


def _lattice(nx, ny, nz, spacing, origin, rng, jitter):
    """Cell-centred cubic lattice, x fastest, with uniform jitter +-jitter*spacing."""
    ix = np.arange(nx, dtype=np.float64)
    iy = np.arange(ny, dtype=np.float64)
    iz = np.arange(nz, dtype=np.float64)
    z, y, x = np.meshgrid(iz, iy, ix, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    pos += 0.5
    pos *= spacing
    pos += np.asarray(origin, dtype=np.float64)
    if jitter > 0.0:
        pos += rng.uniform(-jitter * spacing, jitter * spacing, size=pos.shape)
    return pos


def _wrap(pos, box):
    b = np.asarray(box, dtype=np.float64)
    pos -= b * np.floor(pos / b)
    # a value within rounding of the upper edge maps to 0
    pos[pos >= b] = 0.0
    return pos


def _shuffle(aos, rng):
    return np.ascontiguousarray(aos[rng.permutation(aos.shape[0])])


def uniform_density(n: int = 4096, seed: int = SEED_BASE + 1, shuffle: bool = False) -> Workload:
    """N uniform-random particles in the periodic unit cube, m = 1/N, one fixed h
    with (4 pi / 3) (2h)^3 N = 48 (48 neighbours on average)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    aos = _empty(n)
    _set(aos, "x", rng.uniform(0.0, 1.0, size=(n, 3)))
    h = 0.5 * (3.0 * N_NGB / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    _set(aos, "m", 1.0 / n)
    _set(aos, "h", h)
    _set(aos, "rho", 1.0)
    _set(aos, "u", 1.0)
    if shuffle:
        aos = _shuffle(aos, rng)
    # cells: floor(1 / 2h) per axis (7 at N=4096)
    return Workload("uniform_density", aos, (1.0, 1.0, 1.0), h_cap=h, newton_steps=0,
                    meta={"h": h})


def sod(n_lattice: int = 124, seed: int = SEED_BASE + 2, jitter: float = 0.3,
        shuffle: bool = False, headroom: float = 1.25) -> Workload:
    """Sod-like shock tube in the periodic unit cube.

    Left half (x < 0.5): lattice spacing s = 1/n_lattice, density 1, u = 2.5.
    Right half: spacing 2s, density 0.125, u = 2.0.  Equal masses m = s^3,
    uniform jitter of +-jitter * local spacing per axis, gamma = 5/3, v = 0.
    h0 = eta * local spacing.  The cell edge is 2 * headroom * h0(right) so the
    27-cell stencil covers the support of the sparse side with room for the
    smoothing-length iteration; h is clamped to half the cell edge.
    """
    if n_lattice % 4 != 0:
        raise ValueError("n_lattice must be a multiple of 4")
    rng = np.random.Generator(np.random.PCG64(seed))
    s = 1.0 / n_lattice
    nl = n_lattice // 2
    left = _lattice(nl, n_lattice, n_lattice, s, (0.0, 0.0, 0.0), rng, jitter)
    right = _lattice(nl // 2, nl, nl, 2 * s, (0.5, 0.0, 0.0), rng, jitter)
    pos = _wrap(np.concatenate([left, right]), (1.0, 1.0, 1.0))
    n = pos.shape[0]
    nlft = left.shape[0]
    aos = _empty(n)
    _set(aos, "x", pos)
    m = s ** 3
    _set(aos, "m", m)
    hl, hr = ETA * s, ETA * 2 * s
    h = np.full(n, hr)
    h[:nlft] = hl
    _set(aos, "h", h)
    rho = np.full(n, 0.125)
    rho[:nlft] = 1.0
    _set(aos, "rho", rho)
    u = np.full(n, 2.0)
    u[:nlft] = 2.5
    _set(aos, "u", u)
    if shuffle:
        aos = _shuffle(aos, rng)
    ncell = int(math.floor(1.0 / (2.0 * headroom * hr)))
    cell = 1.0 / ncell
    return Workload("sod", aos, (1.0, 1.0, 1.0), h_cap=0.5 * cell, cell_edge=cell,
                    dt=1e-4, newton_steps=5,
                    meta={"n_lattice": n_lattice, "n_left": nlft, "m": m,
                          "h_left": hl, "h_right": hr, "ncell": ncell})


def sedov(nx: int = 256, ny: int = 256, nz: int = 128, seed: int = SEED_BASE + 3,
          jitter: float = 0.3, headroom: float = 1.25) -> Workload:
    """Sedov blast: jittered lattice of spacing s = 1/nx in the box
    (1, ny/nx, nz/nx), density 1, v = 0, u = 1e-6 except the 64 particles
    nearest the box centre, which share energy 1 (u = 1 / (64 m))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = 1.0 / nx
    box = (1.0, ny * s, nz * s)
    pos = _wrap(_lattice(nx, ny, nz, s, (0.0, 0.0, 0.0), rng, jitter), box)
    n = pos.shape[0]
    aos = _empty(n)
    _set(aos, "x", pos)
    m = s ** 3
    _set(aos, "m", m)
    h0 = ETA * s
    _set(aos, "h", h0)
    _set(aos, "rho", 1.0)
    centre = np.asarray(box) * 0.5
    d2 = np.sum((pos - centre) ** 2, axis=1)
    hot = np.argsort(d2, kind="stable")[:64]
    u = np.full(n, 1e-6)
    u[hot] = 1.0 / (64.0 * m)
    _set(aos, "u", u)
    # h may double in the rarefied centre; the cell edge leaves that room
    ncell = int(math.floor(nz * s / (2.0 * headroom * h0)))
    cell = (nz * s) / ncell
    # fixed step: a quarter of the smoothing length over the hot particles'
    # sound speed c = sqrt(gamma (gamma - 1) u)  (2.0e-6 at 256 x 256 x 128)
    gamma = 5.0 / 3.0
    dt = 0.25 * h0 / math.sqrt(gamma * (gamma - 1.0) * float(u.max()))
    return Workload("sedov", aos, box, h_cap=0.5 * cell, cell_edge=cell, dt=dt, newton_steps=5,
                    meta={"m": m, "hot": hot, "h0": h0})


def gaussian_mixture(n: int = 16_777_216, seed: int = SEED_BASE + 4, n_blob: int = 8,
                     background: float = 0.2) -> Workload:
    """Clustered set: a `background` fraction uniform in the unit cube and the
    rest split equally over `n_blob` isotropic Gaussians with centres uniform in
    the cube and sigma_k = 0.01 * 10^(k/7), wrapped periodically.  One global h,
    set like the uniform set's: (4 pi / 3) (2h)^3 N = 48, i.e. 48 neighbours at
    the mean density (2h = 0.0088 and 113 cells per axis at N = 2^24); the
    clusters then hold up to ~10^5 particles within 2h."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sig = np.array([0.01 * 10.0 ** (k / 7.0) for k in range(n_blob)])
    centres = rng.uniform(0.0, 1.0, size=(n_blob, 3))
    n_bg = int(round(background * n))
    per = (n - n_bg) // n_blob
    counts = [per] * n_blob
    counts[-1] += (n - n_bg) - per * n_blob
    parts = [rng.uniform(0.0, 1.0, size=(n_bg, 3))]
    for k in range(n_blob):
        parts.append(centres[k] + sig[k] * rng.standard_normal(size=(counts[k], 3)))
    pos = _wrap(np.concatenate(parts), (1.0, 1.0, 1.0))
    pos = pos[rng.permutation(n)]
    h = 0.5 * (3.0 * N_NGB / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    aos = _empty(n)
    _set(aos, "x", pos)
    _set(aos, "m", 1.0 / n)
    _set(aos, "h", h)
    _set(aos, "rho", 1.0)
    _set(aos, "u", 1.0)
    ncell = int(math.floor(1.0 / (2.0 * h)))
    return Workload("gaussian_mixture", aos, (1.0, 1.0, 1.0), h_cap=h,
                    cell_edge=1.0 / ncell, newton_steps=0,
                    meta={"h": h, "sigma": sig, "centres": centres})


def gaussian_mixture_adaptive(n: int = 16_777_216, seed: int = SEED_BASE + 4, n_blob: int = 8,
                              background: float = 0.2) -> Workload:
    """The clustered set of ``gaussian_mixture`` (the same positions for the
    same seed) with one smoothing length per particle, from the number density
    of the distribution the positions are drawn from,
        nd(x) = n_bg + sum_k N_k (2 pi sigma_k^2)^(-3/2) exp(-|x - c_k|^2 / (2 sigma_k^2))
    (nearest periodic image of each centre), through (4 pi / 3) (2h)^3 nd = 48,
    the neighbour number of the global-h sets; the density's Newton steps refine
    it.  At N = 2^24, h runs from ~2.4e-4 in the densest core to ~7.5e-3 in the
    background.  The level range of a cell hierarchy (2^l cells per axis, h
    cap 2^-l / 2) follows from it: level_max is the finest level whose cap holds
    the smallest h (at most 10), level_min the finest whose cap holds twice the
    largest h (at least 2), and h_cap is level_min's cap."""
    wl = gaussian_mixture(n, seed, n_blob, background)
    pos = wl.col("x")
    sig, centres = wl.meta["sigma"], wl.meta["centres"]
    n_bg = int(round(background * n))
    per = (n - n_bg) // n_blob
    counts = [per] * n_blob
    counts[-1] += (n - n_bg) - per * n_blob
    nd = np.full(n, float(n_bg))
    step = 1 << 20
    for k in range(n_blob):
        norm = counts[k] * (2.0 * math.pi * sig[k] ** 2) ** -1.5
        for a in range(0, n, step):
            d = pos[a:a + step] - centres[k]
            d -= np.round(d)
            nd[a:a + step] += norm * np.exp(-np.einsum("ij,ij->i", d, d) / (2.0 * sig[k] ** 2))
    h = 0.5 * (3.0 * N_NGB / (4.0 * math.pi * nd)) ** (1.0 / 3.0)
    _set(wl.aos, "h", h)
    lvl_max = int(min(10, math.floor(math.log2(1.0 / (2.0 * h.min())))))
    lvl_min = int(max(2, min(lvl_max, math.floor(math.log2(1.0 / (4.0 * h.max()))))))
    h_cap = 0.5 * 2.0 ** -lvl_min
    meta = dict(wl.meta)
    meta.update({"levels": (lvl_min, lvl_max), "h_min": float(h.min()), "h_max": float(h.max())})
    return Workload("gaussian_mixture_adaptive", wl.aos, (1.0, 1.0, 1.0), h_cap=h_cap,
                    cell_edge=2.0 * h_cap, newton_steps=5, meta=meta)


def long_run(nx: int = 512, ny: int = 256, nz: int = 256, seed: int = SEED_BASE + 5,
             jitter: float = 0.3, headroom: float = 1.25) -> Workload:
    """Jittered lattice of spacing 1/ny in the box (nx/ny, 1, nz/ny), density 1,
    velocities uniform in [-1, 1]^3, u = 1, fixed h = eta * spacing."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = 1.0 / ny
    box = (nx * s, 1.0, nz * s)
    pos = _wrap(_lattice(nx, ny, nz, s, (0.0, 0.0, 0.0), rng, jitter), box)
    n = pos.shape[0]
    aos = _empty(n)
    _set(aos, "x", pos)
    _set(aos, "v", rng.uniform(-1.0, 1.0, size=(n, 3)))
    m = s ** 3
    _set(aos, "m", m)
    h0 = ETA * s
    _set(aos, "h", h0)
    _set(aos, "rho", 1.0)
    _set(aos, "u", 1.0)
    ncell = int(math.floor(1.0 / (2.0 * headroom * h0)))
    cell = 1.0 / ncell
    return Workload("long_run", aos, box, h_cap=0.5 * cell, cell_edge=cell,
                    newton_steps=0, meta={"m": m, "h0": h0})


def buffer_blocks(nb=(16, 16, 16), block=(4, 4, 4), seed: int = SEED_BASE + 7,
                  jitter: float = 0.3) -> Workload:
    """Particles in contiguous buffers of B = bx*by*bz spatially co-located
    particles, the grouping of the paper's benchmark (Section 6; B = 64 for
    4x4x4 blocks).  A jittered cubic lattice of spacing s = 1/(nb_x bx) fills
    the box (1, nb_y by s, nb_z bz s); it is cut into blocks of bx x by x bz
    sites, and the records run block after block (x-fastest block order), a
    block's sites consecutive (x fastest).  Density 1 (m = s^3), h = eta s
    (48 neighbours in the full lattice) times a uniform factor in [0.9, 1.1],
    velocities uniform in [-1, 1]^3, u uniform in [0.5, 2], rho = 1 and P the
    ideal-gas pressure at rho = 1, so the force can run without a density
    pass.  meta["B"] is the buffer size."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nbx, nby, nbz = (int(v) for v in nb)
    bx, by, bz = (int(v) for v in block)
    B = bx * by * bz
    s = 1.0 / (nbx * bx)
    box = (nbx * bx * s, nby * by * s, nbz * bz * s)
    site = _lattice(bx, by, bz, s, (0.0, 0.0, 0.0), rng, 0.0)           # one block, x fastest
    corner = _lattice(nbx, nby, nbz, 1.0, (0.0, 0.0, 0.0), rng, 0.0) - 0.5   # block indices
    corner *= np.array([bx * s, by * s, bz * s])
    pos = (corner[:, None, :] + site[None, :, :]).reshape(-1, 3)
    pos += rng.uniform(-jitter * s, jitter * s, size=pos.shape)
    pos = _wrap(pos, box)
    n = pos.shape[0]
    aos = _empty(n)
    _set(aos, "x", pos)
    _set(aos, "v", rng.uniform(-1.0, 1.0, size=(n, 3)))
    _set(aos, "m", s ** 3)
    h0 = ETA * s
    _set(aos, "h", h0 * rng.uniform(0.9, 1.1, size=n))
    _set(aos, "rho", 1.0)
    u = rng.uniform(0.5, 2.0, size=n)
    _set(aos, "u", u)
    gamma = 5.0 / 3.0
    _set(aos, "P", (gamma - 1.0) * u)
    return Workload("buffer_blocks", aos, box, gamma=gamma, h_cap=1.25 * h0, newton_steps=0,
                    meta={"B": B, "spacing": s, "h0": h0})


def random_cloud(n: int, seed: int, box=(1.0, 1.0, 1.0), h: float | None = None,
                 vel: float = 1.0, n_ngb: float = N_NGB) -> Workload:
    """Small uniform-random cloud with random velocities and energies, for edge
    cases and unit tests.  h defaults to the value giving n_ngb neighbours."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = np.asarray(box, dtype=np.float64)
    vol = float(np.prod(b))
    if h is None:
        h = 0.5 * (3.0 * n_ngb * vol / (4.0 * math.pi * max(n, 1))) ** (1.0 / 3.0)
    aos = _empty(n)
    _set(aos, "x", rng.uniform(0.0, 1.0, size=(n, 3)) * b)
    _set(aos, "v", rng.uniform(-vel, vel, size=(n, 3)))
    _set(aos, "m", rng.uniform(0.5, 1.5, size=n) / max(n, 1))
    _set(aos, "h", h * rng.uniform(0.9, 1.1, size=n))
    _set(aos, "rho", 1.0)
    _set(aos, "u", rng.uniform(0.5, 2.0, size=n))
    return Workload("random_cloud", aos, tuple(float(v) for v in b), h_cap=1.25 * h,
                    newton_steps=0, meta={"h": h})


def pack_records(wl: Workload, layout: dict, record_bytes: int, f32_fields=()) -> np.ndarray:
    """Re-lay the 112-byte records into another AoS layout (bytes, uint8 array).

    `layout` maps field name -> byte offset; fields in `f32_fields` are stored
    as float32 (plain IEEE conversion by numpy), the rest as float64.  Bytes not
    covered by a field are filled with 0xA5 so that stray writes show up."""
    n = wl.n
    buf = np.full((n, record_bytes), 0xA5, dtype=np.uint8)
    for name, off in layout.items():
        nc = RECORD_112[name][1]
        col = wl.col(name).reshape(n, nc)
        if name in f32_fields:
            raw = np.ascontiguousarray(col.astype(np.float32)).view(np.uint8).reshape(n, 4 * nc)
        else:
            raw = np.ascontiguousarray(col).view(np.uint8).reshape(n, 8 * nc)
        buf[:, off:off + raw.shape[1]] = raw
    return buf


CONFIGS = {
    "uniform_density": uniform_density,
    "sod": sod,
    "sedov": sedov,
    "gaussian_mixture": gaussian_mixture,
    "long_run": long_run,
}

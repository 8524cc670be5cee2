"""Seeded synthetic inputs for stochastic texture filtering.

This module is shared by the FP64 oracle (``oracle/``), the CUDA library's tests and
``bench.py``.  It holds data recipes only -- fBm textures, box-filtered MIP chains,
normal maps, query streams, a density volume and a camera -- and none of the
filtering, sampling or shading arithmetic of the method.  Every array is a pure
function of its seed (numpy PCG64 plus an integer lattice hash), so that the CPU and
GPU sides see identical bytes.

The paper's workloads are real assets (the Disney Cloud, Sec. 5 "Offline rendering";
ambientCG materials, Sec. 5); these synthetic stand-ins reproduce their shapes and
statistics:

* ``texture_rgba32f``   -- 2-D RGBA FP32 texture, RGB ~ U[0,1), A = roughness in [0.05, 1].
* ``material_rgba8``    -- fBm albedo+roughness RGBA8 and an RG8 tangent-space normal map
                           derived from an fBm height, each with a full box-filtered MIP chain.
* ``queries_uniform``   -- uv on the 2^-24 grid, optional isotropic screen-space
                           derivatives whose LOD is uniform over a range of MIP levels.
* ``volume_cloud``      -- fBm density cloud, thresholded so that a given fraction of
                           voxels is exactly zero, stored as FP16.
* ``camera_pinhole``    -- pinhole camera basis for the volume march.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

U32 = np.uint32


# ---------------------------------------------------------------------------------
# integer lattice hash (Wellons' "lowbias32" mixer) -- deterministic on any machine
# ---------------------------------------------------------------------------------
def _mix32(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint32, copy=True)
    x ^= x >> U32(16)
    x *= U32(0x7FEB352D)
    x ^= x >> U32(15)
    x *= U32(0x846CA68B)
    x ^= x >> U32(16)
    return x


def _lattice(shape, seed: int, octave: int) -> np.ndarray:
    """Uniform [0,1) values on an integer lattice, keyed by (seed, octave, index)."""
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.uint64)
    h = _mix32((idx & np.uint64(0xFFFFFFFF)).astype(np.uint32) ^ _mix32(np.array(
        [seed * 0x9E3779B1 + octave * 0x85EBCA77], dtype=np.uint64).astype(np.uint32)))
    h = _mix32(h ^ U32((seed * 31 + octave * 7919 + 12345) & 0xFFFFFFFF))
    return (h.astype(np.float64) * (1.0 / 4294967296.0)).reshape(shape)


def _interp_axis(arr: np.ndarray, axis: int, period: int, size: int, dtype) -> np.ndarray:
    """Periodic smoothstep interpolation of a lattice axis of length ``period`` up to ``size``."""
    s = (np.arange(size, dtype=np.float64) + 0.5) * (period / size)
    i0 = np.floor(s).astype(np.int64)
    f = s - i0
    f = f * f * (3.0 - 2.0 * f)
    i0 %= period
    i1 = (i0 + 1) % period
    a0 = np.take(arr, i0, axis=axis)
    a1 = np.take(arr, i1, axis=axis)
    shp = [1] * arr.ndim
    shp[axis] = size
    f = f.reshape(shp).astype(dtype)
    return (a0 * (1 - f) + a1 * f).astype(dtype)


def fbm2d(size: int, octaves: int, base: int, seed: int, gain: float = 0.5) -> np.ndarray:
    """Periodic 2-D value-noise fBm in [0,1], lacunarity 2 (float64, shape (size, size))."""
    out = np.zeros((size, size), dtype=np.float64)
    amp, norm = 1.0, 0.0
    for o in range(octaves):
        p = min(base << o, size)
        lat = _lattice((p, p), seed, o)
        r = _interp_axis(lat, 1, p, size, np.float64)   # (p, size)
        r = _interp_axis(r, 0, p, size, np.float64)     # (size, size)
        out += amp * r
        norm += amp
        amp *= gain
    return out / norm


def fbm3d(size: int, octaves: int, base: int, seed: int, gain: float = 0.5) -> np.ndarray:
    """Periodic 3-D value-noise fBm in [0,1] (float32, shape (size, size, size) as z, y, x)."""
    out = np.zeros((size, size, size), dtype=np.float32)
    amp, norm = 1.0, 0.0
    for o in range(octaves):
        p = min(base << o, size)
        lat = _lattice((p, p, p), seed, o).astype(np.float32)
        r = _interp_axis(lat, 2, p, size, np.float32)
        r = _interp_axis(r, 1, p, size, np.float32)
        for z0 in range(0, size, 64):                  # bounded temporaries along z
            s = (np.arange(z0, min(size, z0 + 64), dtype=np.float64) + 0.5) * (p / size)
            i0 = np.floor(s).astype(np.int64)
            f = s - i0
            f = (f * f * (3.0 - 2.0 * f)).astype(np.float32)[:, None, None]
            i0 %= p
            zz = r[i0] * (1 - f) + r[(i0 + 1) % p] * f
            out[z0:z0 + zz.shape[0]] += np.float32(amp) * zz
        norm += amp
        amp *= gain
    out /= np.float32(norm)
    return out


def _rne_u8(x: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


def box_mips_u8(level0: np.ndarray) -> list[np.ndarray]:
    """Full box-filtered MIP chain of a (H, W, C) uint8 image, round-half-even averages."""
    levels = [level0]
    cur = level0.astype(np.float64)
    while cur.shape[0] > 1 or cur.shape[1] > 1:
        h, w = cur.shape[:2]
        if h > 1:
            cur = 0.5 * (cur[0::2] + cur[1::2])
        if w > 1:
            cur = 0.5 * (cur[:, 0::2] + cur[:, 1::2])
        q = _rne_u8(cur)
        levels.append(q)
        cur = q.astype(np.float64)
    return levels


# ---------------------------------------------------------------------------------
# 2-D textures
# ---------------------------------------------------------------------------------
def texture_rgba32f(size: int = 256, seed: int = 101) -> np.ndarray:
    """(size, size, 4) float32: RGB ~ U[0,1), A = 0.05 + 0.95 U[0,1) (roughness)."""
    rng = np.random.default_rng(seed)
    t = rng.random((size, size, 4), dtype=np.float64)
    t[..., 3] = 0.05 + 0.95 * t[..., 3]
    return t.astype(np.float32)


@dataclass
class Material:
    albedo_rough: list      # per level (H, W, 4) uint8: albedo RGB, roughness byte
    normal: list            # per level (H, W, 2) uint8: tangent-space normal XY
    height: np.ndarray      # (H, W) float64 fBm height at level 0 (kept for neural targets)


def material_rgba8(size: int = 4096, seed: int = 102, octaves: int = 8,
                   base: int = 8, mips: bool = True) -> Material:
    """fBm albedo+roughness (RGBA8) and normal map (RG8) with full MIP chains."""
    height = fbm2d(size, octaves, base, seed * 17 + 1)
    cr = fbm2d(size, octaves, base, seed * 17 + 2)
    cg = fbm2d(size, octaves, base, seed * 17 + 3)
    ro = fbm2d(size, octaves, base, seed * 17 + 4)
    ar = np.empty((size, size, 4), dtype=np.uint8)
    # warm stone-like palette; contrast stretched around the fBm mean of ~0.5
    ar[..., 0] = _rne_u8(255 * np.clip(0.55 + 1.6 * (height - 0.5) + 0.4 * (cr - 0.5), 0, 1))
    ar[..., 1] = _rne_u8(255 * np.clip(0.45 + 1.6 * (height - 0.5) + 0.4 * (cg - 0.5), 0, 1))
    ar[..., 2] = _rne_u8(255 * np.clip(0.35 + 1.2 * (height - 0.5), 0, 1))
    ar[..., 3] = _rne_u8(255 * np.clip(0.5 + 2.5 * (ro - 0.5), 0, 1))
    # normal from the height's periodic central differences, slope std fixed at 0.35
    gx = 0.5 * (np.roll(height, -1, axis=1) - np.roll(height, 1, axis=1))
    gy = 0.5 * (np.roll(height, -1, axis=0) - np.roll(height, 1, axis=0))
    k = 0.35 / max(1e-12, float(np.sqrt(0.5 * (gx.var() + gy.var()))))
    nx, ny, nz = -k * gx, -k * gy, np.ones_like(gx)
    inv = 1.0 / np.sqrt(nx * nx + ny * ny + nz * nz)
    nrm = np.empty((size, size, 2), dtype=np.uint8)
    nrm[..., 0] = _rne_u8((nx * inv * 0.5 + 0.5) * 255)
    nrm[..., 1] = _rne_u8((ny * inv * 0.5 + 0.5) * 255)
    if mips:
        return Material(box_mips_u8(ar), box_mips_u8(nrm), height)
    return Material([ar], [nrm], height)


# ---------------------------------------------------------------------------------
# queries
# ---------------------------------------------------------------------------------
# DCT-compressed texture set (supplement "Texture compression"): per 8 x 8 block and channel
# the six lowest frequencies (u + v <= 2) of the orthonormal 2-D DCT-II, packed into one 32-bit
# word: bits 0-6 the DC term, quantised over [0, 8] to 7 bits; then five 5-bit fields, one
# per AC term in the order (u, v) = (1,0), (0,1), (2,0), (1,1), (0,2), each stored as q + 15
# with q = round(X / (2/15)) clamped to [-15, 15].  Six channels (albedo RGB, roughness,
# normal X and Y, each byte/255) make 24 bytes, padded to a 32-byte block; levels narrower
# than 8 texels repeat periodically inside their block.
DCT_AC = ((1, 0), (0, 1), (2, 0), (1, 1), (0, 2))
DCT_DC_MAX, DCT_AC_STEP = 8.0, 2.0 / 15.0


def dct_compress(material: Material) -> list:
    """Per MIP level a (ceil(H/8), ceil(W/8), 32) uint8 array of DCT blocks (see above)."""
    from scipy.fft import dctn
    out = []
    for ar, nm in zip(material.albedo_rough, material.normal):
        H, W = ar.shape[:2]
        ch = np.concatenate([ar.astype(np.float64), nm.astype(np.float64)], axis=2) / 255.0   # (H, W, 6)
        H8, W8 = -(-H // 8), -(-W // 8)
        yy = np.arange(H8 * 8) % H
        xx = np.arange(W8 * 8) % W
        full = ch[yy][:, xx]                                          # periodic extension
        blocks = full.reshape(H8, 8, W8, 8, 6).transpose(0, 2, 4, 1, 3)   # (H8, W8, 6, y, x)
        X = dctn(blocks, type=2, norm="ortho", axes=(3, 4))             # X[..., v, u]
        dc = np.clip(np.rint(X[..., 0, 0] / DCT_DC_MAX * 127.0), 0, 127).astype(np.uint32)
        word = dc.copy()
        for j, (u, v) in enumerate(DCT_AC):
            q = np.clip(np.rint(X[..., v, u] / DCT_AC_STEP), -15, 15).astype(np.int64) + 15
            word |= q.astype(np.uint32) << np.uint32(7 + 5 * j)
        blk = np.zeros((H8, W8, 8), dtype=np.uint32)
        blk[..., :6] = word
        out.append(blk.view(np.uint8).reshape(H8, W8, 32))
    return out


@dataclass
class Queries:
    u: np.ndarray
    v: np.ndarray
    dudx: np.ndarray | None = None
    dvdx: np.ndarray | None = None
    dudy: np.ndarray | None = None
    dvdy: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.u.shape[0])

    def has_derivs(self) -> bool:
        return self.dudx is not None

    def subset(self, idx) -> "Queries":
        f = (lambda a: None if a is None else np.array(a[idx], copy=True))   # never a view
        return Queries(f(self.u), f(self.v), f(self.dudx), f(self.dvdx), f(self.dudy), f(self.dvdy))


def queries_uniform(n: int, seed: int, res: int | None = None, lod_range: float = 0.0,
                    const_derivs: tuple | None = None) -> Queries:
    """uv uniform on the 2^-24 grid.

    ``lod_range > 0``: isotropic derivatives with |ddx| = |ddy| = 2^lam / res,
    lam ~ U[0, lod_range), random rotation.  ``const_derivs=(dudx, dvdx, dudy, dvdy)``:
    the same derivatives for every query.  Neither: no derivatives.
    """
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 1 << 24, size=(2, n), dtype=np.int64)
    u = (k[0].astype(np.float64) * 2.0 ** -24).astype(np.float32)
    v = (k[1].astype(np.float64) * 2.0 ** -24).astype(np.float32)
    if lod_range > 0:
        assert res is not None
        lam = lod_range * rng.random(n)
        th = 2 * math.pi * rng.random(n)
        ln = np.exp2(lam) / res
        c, s = np.cos(th) * ln, np.sin(th) * ln
        return Queries(u, v, c.astype(np.float32), s.astype(np.float32),
                       (-s).astype(np.float32), c.astype(np.float32))
    if const_derivs is not None:
        d = [np.full(n, x, dtype=np.float32) for x in const_derivs]
        return Queries(u, v, *d)
    return Queries(u, v)


def queries_aniso(n: int, seed: int, res: int, lod_range: float = 4.0, max_aniso: float = 64.0) -> Queries:
    """uv uniform on the 2^-24 grid with anisotropic footprints: the minor axis is
    2^lam / res long (lam ~ U[0, lod_range)), the major axis a times longer (a log-uniform in
    [1, max_aniso]), at a random rotation; which of ddx / ddy is the major axis is random."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 1 << 24, size=(2, n), dtype=np.int64)
    u = (k[0].astype(np.float64) * 2.0 ** -24).astype(np.float32)
    v = (k[1].astype(np.float64) * 2.0 ** -24).astype(np.float32)
    lam = lod_range * rng.random(n)
    a = np.exp(np.log(max_aniso) * rng.random(n))
    th = 2 * math.pi * rng.random(n)
    mn = np.exp2(lam) / res
    c, s = np.cos(th), np.sin(th)
    maj = np.stack([c * mn * a, s * mn * a])          # (2, n): (du, dv) of the major axis
    mnr = np.stack([-s * mn, c * mn])
    swap = rng.random(n) < 0.5
    dx = np.where(swap, mnr, maj)
    dy = np.where(swap, maj, mnr)
    f = lambda x: x.astype(np.float32)
    return Queries(u, v, f(dx[0]), f(dx[1]), f(dy[0]), f(dy[1]))


@dataclass
class TriQueries:
    """Surface points for triplanar lookups: position, normal, screen-space dP/dx and dP/dy
    (tuples of three float32 arrays, or None)."""
    px: np.ndarray
    py: np.ndarray
    pz: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    nz: np.ndarray
    dpdx: tuple | None = None
    dpdy: tuple | None = None

    @property
    def n(self) -> int:
        return int(self.px.shape[0])

    def subset(self, idx) -> "TriQueries":
        f = (lambda a: np.array(a[idx], copy=True))
        t = (lambda d: None if d is None else tuple(f(a) for a in d))
        return TriQueries(f(self.px), f(self.py), f(self.pz), f(self.nx), f(self.ny), f(self.nz),
                          t(self.dpdx), t(self.dpdy))


def queries_triplanar(n: int, seed: int, res: int, scale: float = 1.0, extent: float = 4.0,
                      lod_range: float = 4.0, max_aniso: float = 8.0, derivs: bool = True) -> TriQueries:
    """Points on surfaces of random orientation: P uniform in [0, extent)^3 on the 2^-20 grid,
    N uniform on the unit sphere, and a screen-space footprint in the tangent plane whose minor
    axis is 2^lam / (res * scale) world units (lam ~ U[0, lod_range)), the major axis a times
    longer (a log-uniform in [1, max_aniso]), at a random rotation."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, int(extent * (1 << 20)), size=(3, n), dtype=np.int64)
    P = (k.astype(np.float64) * 2.0 ** -20).astype(np.float32)
    g = rng.standard_normal((3, n))
    N = g / np.linalg.norm(g, axis=0, keepdims=True)
    f = lambda x: x.astype(np.float32)
    if not derivs:
        return TriQueries(P[0], P[1], P[2], f(N[0]), f(N[1]), f(N[2]))
    # tangent frame: T = normalize(N x e) with e the axis least aligned with N, B = N x T
    e = np.zeros((3, n))
    e[np.argmin(np.abs(N), axis=0), np.arange(n)] = 1.0
    T = np.cross(N, e, axis=0)
    T /= np.linalg.norm(T, axis=0, keepdims=True)
    B = np.cross(N, T, axis=0)
    lam = lod_range * rng.random(n)
    a = np.exp(np.log(max_aniso) * rng.random(n))
    th = 2 * math.pi * rng.random(n)
    mn = np.exp2(lam) / (res * scale)
    c, s_ = np.cos(th), np.sin(th)
    maj = (c * mn * a) * T + (s_ * mn * a) * B
    mnr = (-s_ * mn) * T + (c * mn) * B
    swap = rng.random(n) < 0.5
    dx = np.where(swap, mnr, maj)
    dy = np.where(swap, maj, mnr)
    return TriQueries(P[0], P[1], P[2], f(N[0]), f(N[1]), f(N[2]), tuple(f(x) for x in dx), tuple(f(x) for x in dy))


# ---------------------------------------------------------------------------------
# volume and camera
# ---------------------------------------------------------------------------------
def volume_cloud(size: int = 512, seed: int = 103, zero_frac: float = 0.9,
                 octaves: int = 6, base: int = 4) -> np.ndarray:
    """(size,size,size) float16 density (z, y, x), ``zero_frac`` of voxels exactly 0, max 1."""
    d = fbm3d(size, octaves, base, seed)
    c = (np.arange(size, dtype=np.float32) + 0.5) / size - 0.5
    r2 = c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2
    env = np.clip(1.0 - np.sqrt(r2) / np.float32(0.48), 0.0, 1.0).astype(np.float32)
    d *= np.sqrt(env)
    del r2, env
    flat = d.reshape(-1)
    kth = int(zero_frac * flat.size)
    thr = np.partition(flat.copy(), kth)[kth] if kth < flat.size else flat.max()
    mx = float(flat.max())
    out = np.where(d > thr, (d - thr) / np.float32(max(mx - thr, 1e-12)), np.float32(0))
    return out.astype(np.float16)


@dataclass
class Camera:
    eye: tuple
    fwd: tuple
    right: tuple     # screen +x direction scaled by tan(vfov/2) * aspect
    up: tuple        # screen +y direction scaled by tan(vfov/2)

    def as_array(self) -> np.ndarray:
        return np.array([*self.eye, *self.fwd, *self.right, *self.up], dtype=np.float32)


def camera_pinhole(width: int, height: int, eye=(0.5, 0.5, -1.2), look=(0.5, 0.5, 0.5),
                   up=(0.0, 1.0, 0.0), vfov_deg: float = 45.0) -> Camera:
    e, l, u = (np.asarray(x, dtype=np.float64) for x in (eye, look, up))
    f = l - e
    f /= np.linalg.norm(f)
    r = np.cross(u, f)
    r /= np.linalg.norm(r)
    uu = np.cross(f, r)
    th = math.tan(math.radians(vfov_deg) * 0.5)
    asp = width / height
    f32 = lambda a: tuple(float(np.float32(x)) for x in a)
    return Camera(f32(e), f32(f), f32(r * th * asp), f32(uu * th))


# ---------------------------------------------------------------------------------
# learned form: 8-channel targets and initial parameters
# ---------------------------------------------------------------------------------
NTC_MLP_SIZE = 64 * 32 + 64 + 64 * 64 + 64 + 8 * 64 + 8     # 6792


def ntc_targets(material: Material, seed: int = 104) -> np.ndarray:
    """(H, W, 8) uint8 channels of level 0: albedo RGB, roughness, normal XY, metalness
    (a binary fBm threshold -- a 'discrete quantity'), height."""
    ar, nm, h = material.albedo_rough[0], material.normal[0], material.height
    size = ar.shape[0]
    metal = fbm2d(size, 6, 4, seed) > 0.62
    out = np.empty((size, size, 8), dtype=np.uint8)
    out[..., 0:4] = ar
    out[..., 4:6] = nm
    out[..., 6] = np.where(metal, 255, 0).astype(np.uint8)
    hmin, hmax = float(h.min()), float(h.max())
    out[..., 7] = _rne_u8(255 * (h - hmin) / max(hmax - hmin, 1e-12))
    return out


def ntc_init(grid_res=(1024, 512, 256, 128), seed: int = 104):
    """Latents U(-0.1, 0.1) per grid (res, res, 8) float32; MLP He-uniform weights
    (bound sqrt(6 / fan_in)) and zero biases, packed W1 b1 W2 b2 W3 b3 (row-major [out][in])."""
    rng = np.random.default_rng(seed)
    lat = [rng.uniform(-0.1, 0.1, (r, r, 8)).astype(np.float32) for r in grid_res]
    parts = []
    for fan_in, fan_out in ((32, 64), (64, 64), (64, 8)):
        b = math.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-b, b, (fan_out, fan_in)).astype(np.float32).ravel())
        parts.append(np.zeros(fan_out, dtype=np.float32))
    return lat, np.concatenate(parts)


# ---------------------------------------------------------------------------------
# bindless table: many textures of uneven sizes
# ---------------------------------------------------------------------------------
def texture_table_rgba8(n: int = 256, lo: int = 64, hi: int = 4096, seed: int = 105, fbm_below: int = 0):
    """n RGBA8 textures (single level) with side lengths log-uniform in [lo, hi] (any
    integer, non-powers of two included).  Texels are white-noise bytes: the gather
    pattern, not the content, is what a table of uneven textures stresses, and generating
    ~2 GiB of fBm on the host would dominate a run.  Textures with a side below
    ``fbm_below`` get fBm content instead."""
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(int)
    out = []
    for i, s_ in enumerate(sides):
        if s_ < fbm_below:
            m = material_rgba8(int(s_), seed * 1000 + i, octaves=3, base=2, mips=False) if s_ >= 4 else None
            out.append(m.albedo_rough[0] if m is not None else rng.integers(0, 256, (s_, s_, 4), dtype=np.uint8))
        else:
            out.append(rng.integers(0, 256, (int(s_), int(s_), 4), dtype=np.uint8))
    return out

"""FP64 CPU oracle for stochastic texture filtering -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The CUDA product path (``paper_2407_06107_b300``) never imports it,
and the two share no code: the only common module is ``stf_synth`` (seeded inputs).

The arithmetic lives in ``stf_oracle.cpp`` (plain C++17, FP64 values, FP32 decisions as
in the paper's float listings).  This module compiles it with g++ (no fused
multiply-add contraction, no fast-math) and wraps it with ctypes.

Parity status: every entry point is pinned by ``tests/test_oracle_*.py`` against closed
forms, library routines (scipy B-spline / linear interpolation), quadrature identities of
the GGX model, exact enumeration, Monte-Carlo convergence and the paper's worked example
(Fig. 7).  The shading constants (light/view direction, F0, roughness mapping) are a
specification, not something the paper fixes; they are pinned only by the GGX identities.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("stf_oracle.cpp", "ntc_oracle.cpp")]
DEPS = SRCS + [os.path.join(HERE, "oracle_internal.h")]
LIB = os.path.join(HERE, "liboracle.so")

FILTERS = {"linear": 0, "bspline": 1, "catmull_rom": 2, "mitchell": 3, "ewa": 4, "gauss": 5}
MODES = {"ntap_before": 0, "ntap_after": 1, "stochastic": 2, "positivized": 3}
SHADES = {"ggx": 0, "linear": 1}
BLENDS = {"full": 0, "stochastic": 1}
FLAG_STRATIFIED = 1
FLAG_LATTICE = 2
FLAG_REUSE = 4
FLAG_LOD0 = 8
NO_PICK = 0xFFFFFFFF


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or any(os.path.getmtime(LIB) < os.path.getmtime(p) for p in DEPS):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", *SRCS, "-o", LIB + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class _Tex(C.Structure):
    _fields_ = [("format", C.c_int), ("levels", C.c_int), ("address", C.c_int),
                ("width", C.c_int * 16), ("height", C.c_int * 16),
                ("data", C.c_void_p * 16), ("normal", C.c_void_p * 16)]


class _Mlp(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("W1", "b1", "W2", "b2", "W3", "b3")]


class _NeuralTex(C.Structure):
    _fields_ = [("tex_res", C.c_int), ("res", C.c_int * 4), ("latent_fmt", C.c_int), ("grid", C.c_void_p * 4),
                ("scale", C.c_float * 4), ("mlp", C.POINTER(_Mlp))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_kernel.argtypes = [C.c_int, C.c_double]
        L.orc_kernel.restype = C.c_double
        L.orc_kernel_bc.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_kernel_bc.restype = C.c_double
        L.orc_kernel_keys.argtypes = [C.c_double, C.c_double]
        L.orc_kernel_keys.restype = C.c_double
        L.orc_weights32.argtypes = [C.c_int, C.c_float, P]
        L.orc_pick32.argtypes = [P, C.c_int, C.c_float, C.c_int]
        L.orc_ewa_table.argtypes = [P]
        L.orc_dct_texel.argtypes = [C.c_uint32, C.c_int, C.c_int]
        L.orc_dct_texel.restype = C.c_double
        L.orc_ewa_box.argtypes = [C.c_float] * 6 + [C.c_int, C.c_int, P, P, C.c_int]
        L.orc_pick32_reuse.argtypes = [P, C.c_int, C.c_float, P]
        L.orc_pick_array.argtypes = [P, C.c_int, C.c_double]
        L.orc_ggx_eval.argtypes = [P, P, P, C.c_double, P, C.c_double, P]
        L.orc_ggx_D.argtypes = [C.c_double, C.c_double]
        L.orc_ggx_D.restype = C.c_double
        L.orc_smith_lambda.argtypes = [C.c_double, C.c_double]
        L.orc_smith_lambda.restype = C.c_double
        L.orc_shade_batch.argtypes = [C.c_uint64, C.c_int, P, P, P, P]
        L.orc_fetch.argtypes = [C.POINTER(_Tex), C.c_int, C.c_int, C.c_int, P]
        L.orc_filter_shade.argtypes = [C.POINTER(_Tex), C.c_uint64] + [P] * 7 + [
            C.c_int, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32, P, P, P, P, P, P, C.c_int, C.c_float]
        L.orc_march.argtypes = [C.c_int, C.c_int, C.c_int, P, C.c_float, P, C.c_uint32, C.c_uint32,
                                C.c_uint32, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32,
                                C.c_uint64, C.c_uint64, P, P, P, P, P, C.c_int]
        L.orc_triplanar_shade.argtypes = [P, C.c_uint64] + [P] * 13 + [
            C.c_float, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32, P, P, P, P, P, C.c_int]
        D = C.c_double
        for nm in ("orc_round_bf16", "orc_round_fp16", "orc_round_e4m3"):
            getattr(L, nm).argtypes = [D]
            getattr(L, nm).restype = D
        L.orc_e4m3_value.argtypes = [C.c_uint8]
        L.orc_e4m3_value.restype = D
        L.orc_ntc_features.argtypes = [C.POINTER(_NeuralTex), C.c_uint64, P, P, P]
        L.orc_ntc_decode.argtypes = [C.POINTER(_NeuralTex), C.c_uint64, P, P, P, P]
        L.orc_ntc_decode_exact.argtypes = [C.POINTER(_NeuralTex), C.c_uint64, P, P, P]
        L.orc_ntc_loss_grad.argtypes = [C.POINTER(_NeuralTex)] + [P] * 7 + [C.c_uint64, P, P, C.c_int] + [P] * 7
        L.orc_ntc_loss_grad.restype = D
        L.orc_adam.argtypes = [C.c_uint64, P, P, P, P, C.c_int, D, D, D, D]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def nthreads_default() -> int:
    return max(1, os.cpu_count() or 1)


# ----------------------------------------------------------------------------- primitives
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def kernel(filter_name: str, d: float) -> float:
    return lib().orc_kernel(FILTERS[filter_name], float(d))


def kernel_bc(B: float, Cc: float, d: float) -> float:
    return lib().orc_kernel_bc(float(B), float(Cc), float(d))


def kernel_keys(a: float, d: float) -> float:
    return lib().orc_kernel_keys(float(a), float(d))


def weights32(filter_name: str, t: float) -> np.ndarray:
    w = np.zeros(4, dtype=np.float32)
    n = lib().orc_weights32(FILTERS[filter_name], float(np.float32(t)), _p(w))
    return w[:n]


def pick32(w, xi: float, cls: int = 0) -> int:
    w = np.ascontiguousarray(w, dtype=np.float32)
    return lib().orc_pick32(_p(w), len(w), float(np.float32(xi)), cls)


def dct_texel(word: int, x: int, y: int) -> float:
    """Raw decoded value of one DCT channel word at (x, y) in its block."""
    return float(lib().orc_dct_texel(int(word), int(x), int(y)))


def ewa_table() -> np.ndarray:
    """The 128 Gaussian weights exp(-2 r^2) - exp(-2) at r^2 = i/127 (FP32)."""
    out = np.zeros(128, np.float32)
    lib().orc_ewa_table(_p(out))
    return out


def ewa_box(x, y, dudx, dvdx, dudy, dvdy, W, H, cap=1 << 20):
    """The EWA ellipse's bounding box (s0, s1, t0, t1) at a W x H level and the FP32 weights of
    its texels as a (t, s) array (zero outside the ellipse)."""
    box = np.zeros(4, np.int32)
    w = np.zeros(cap, np.float32)
    f = lambda a: float(np.float32(a))
    n = lib().orc_ewa_box(f(x), f(y), f(dudx), f(dvdx), f(dudy), f(dvdy), int(W), int(H), _p(box), _p(w), cap)
    if n < 0:
        raise ValueError("box too large" if n == -1 else "non-finite ellipse")
    s0, s1, t0, t1 = (int(b) for b in box)
    return (s0, s1, t0, t1), w[:n].reshape(t1 - t0 + 1, s1 - s0 + 1).copy()


def pick32_reuse(w, xi: float):
    """(pick, remapped uniform) of the FP32 sample-reuse decision."""
    w = np.ascontiguousarray(w, dtype=np.float32)
    r = np.zeros(1, dtype=np.float32)
    k = lib().orc_pick32_reuse(_p(w), len(w), float(np.float32(xi)), _p(r))
    return k, float(r[0])


def pick_array(w, xi: float) -> int:
    w = np.ascontiguousarray(w, dtype=np.float64)
    return lib().orc_pick_array(_p(w), len(w), float(xi))


def ggx_eval(n, l, v, alpha, rho, F0) -> np.ndarray:
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (n, l, v, rho)]
    o = np.zeros(3)
    lib().orc_ggx_eval(_p(a[0]), _p(a[1]), _p(a[2]), float(alpha), _p(a[3]), float(F0), _p(o))
    return o


def ggx_D(alpha: float, nh: float) -> float:
    return lib().orc_ggx_D(float(alpha), float(nh))


def smith_lambda(alpha: float, tan2: float) -> float:
    return lib().orc_smith_lambda(float(alpha), float(tan2))


def shade_batch(rho, rough, nrm, shade: str = "ggx") -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1, 3)
    rough = np.ascontiguousarray(rough, dtype=np.float64).reshape(-1)
    nrm = np.ascontiguousarray(nrm, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(rho)
    lib().orc_shade_batch(len(rough), SHADES[shade], _p(rho), _p(rough), _p(nrm), _p(out))
    return out


# ----------------------------------------------------------------------------- textures
@dataclass
class Texture:
    """Level arrays as the generator emits them (row-major, y then x)."""
    levels: list                 # (H, W, 4) float32 (RGBA32F) or uint8 (RGBA8 material)
    normal: list | None = None   # (H, W, 2) uint8 per level, or None
    address: str = "wrap"

    neural: "NeuralTexture | None" = None
    dct: list | None = None      # DCT blocks per level ((H8, W8, 32) uint8); levels = level sizes

    def _struct(self):
        t = _Tex()
        if self.neural is not None:       # learned texture: one level decoded by the MLP
            t.format, t.levels, t.address = 2, 1, 0
            t.width[0] = t.height[0] = self.neural.tex_res
            self._nt = self.neural._struct()
            t.data[0] = C.cast(C.pointer(self._nt), C.c_void_p).value
            return t
        if self.dct is not None:          # DCT-compressed set: self.levels holds (H, W) per level
            t.format, t.levels, t.address = 3, len(self.dct), 0
            self._keep = []
            for i, (b, hw) in enumerate(zip(self.dct, self.levels)):
                b = np.ascontiguousarray(b)
                self._keep.append(b)
                t.height[i], t.width[i] = int(hw[0]), int(hw[1])
                t.data[i] = b.ctypes.data
            return t
        fmt = 0 if self.levels[0].dtype == np.float32 else 1
        t.format, t.levels = fmt, len(self.levels)
        t.address = 0 if self.address == "wrap" else 1
        self._keep = []
        for i, a in enumerate(self.levels):
            a = np.ascontiguousarray(a)
            self._keep.append(a)
            t.height[i], t.width[i] = a.shape[0], a.shape[1]
            t.data[i] = a.ctypes.data
            if self.normal is not None:
                nm = np.ascontiguousarray(self.normal[i])
                self._keep.append(nm)
                t.normal[i] = nm.ctypes.data
        return t


def fetch(tex: Texture, lvl: int, ix: int, iy: int) -> np.ndarray:
    o = np.zeros(7)
    t = tex._struct()
    lib().orc_fetch(C.byref(t), lvl, ix, iy, _p(o))
    return o


@dataclass
class FilterResult:
    rgb: np.ndarray            # (n, 3) float64
    picks: np.ndarray | None   # (n, spp, 2) uint32, FP32 decisions (level<<28 | iy<<14 | ix)
    picks64: np.ndarray | None  # same, FP64 decisions (NO_PICK-1 where the level differs)
    bdist: np.ndarray | None   # (n,) distance of the nearest uniform to an FP64 boundary
    mag: np.ndarray | None = None  # (n, 3) mean over samples of sum |w f_hat| over the summed terms
    rdist: np.ndarray | None = None  # (n,) learned texels: smallest BF16 rounding margin (see ntc_decode)


def _internal_filter(filter: str, sampler: str, mode: str) -> int:
    """The oracle's filter id: FIS picks are their own filters (STOCHASTIC only); the N-tap form
    of a FIS filter is the filter it converges to (the same tent / B-spline, and for the
    Gaussian its convolution with the unit box)."""
    if sampler == "frs":
        return FILTERS[filter]
    if sampler != "fis" or filter not in ("linear", "bspline", "gauss"):
        raise ValueError("FIS samples the tent, the cubic B-spline and the Gaussian")
    if mode == "stochastic":
        return {"linear": 7, "bspline": 8, "gauss": 9}[filter]
    return {"linear": 0, "bspline": 1, "gauss": 6}[filter]


def filter_shade(tex: Texture, q, filter: str, mode: str, shade: str = "ggx", spp: int = 1,
                 seed: int = 1, flags: int = 0, want_picks: bool = False,
                 nthreads: int | None = None, ids=None, sampler: str = "frs", sigma: float = 0.5) -> FilterResult:
    """Evaluate queries q; the Philox id of query i is ids[i] (default: i).  sampler: "frs"
    (filter reservoir sampling) or "fis" (filter importance sampling); sigma: the Gaussian's
    standard deviation in texels."""
    n = q.n
    rgb = np.zeros((n, 3))
    picks = np.zeros((n, spp, 2), dtype=np.uint32) if want_picks else None
    picks64 = np.zeros((n, spp, 2), dtype=np.uint32) if want_picks else None
    bd = np.zeros(n)
    mag = np.zeros((n, 3))
    rdist = np.ones(n)
    t = tex._struct()
    arrs = [np.ascontiguousarray(a, dtype=np.float32) if a is not None else None
            for a in (q.u, q.v, q.dudx, q.dvdx, q.dudy, q.dvdy)]
    ids = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint64)
    rc = lib().orc_filter_shade(C.byref(t), n, *[_p(a) for a in arrs], _p(ids), _internal_filter(filter, sampler, mode),
                                MODES[mode], SHADES[shade], spp, seed, flags, _p(rgb), _p(picks), _p(picks64),
                                _p(bd), _p(mag), _p(rdist), nthreads or nthreads_default(), float(sigma))
    if rc != 0:
        raise ValueError("oracle: invalid filter_shade arguments")
    return FilterResult(rgb, picks, picks64, bd, mag, rdist)


def triplanar_shade(texs, q, scale: float, filter: str, mode: str, blend: str, shade: str = "ggx", spp: int = 1,
                    seed: int = 1, flags: int = 0, want_picks: bool = False, nthreads: int | None = None,
                    ids=None) -> FilterResult:
    """Triplanar lookups (Sec. 5 "Triplanar mapping"): texs = three Textures (planes along x, y,
    z; they may repeat); q a stf_synth.TriQueries.  picks / picks64: (n, spp, 3, 2)."""
    n = q.n
    rgb = np.zeros((n, 3))
    picks = np.zeros((n, spp, 3, 2), dtype=np.uint32) if want_picks else None
    picks64 = np.zeros((n, spp, 3, 2), dtype=np.uint32) if want_picks else None
    bd = np.zeros(n)
    mag = np.zeros((n, 3))
    structs, seen = [], {}
    for t in texs:                      # one struct per distinct texture (it owns the level refs)
        if id(t) not in seen:
            seen[id(t)] = t._struct()
        structs.append(seen[id(t)])
    arr = (_Tex * 3)(*structs)
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    arrs = [f32(a) for a in (q.px, q.py, q.pz, q.nx, q.ny, q.nz)]
    d = [f32(a) for a in ((q.dpdx + q.dpdy) if q.dpdx is not None else (None,) * 6)]
    ids = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint64)
    rc = lib().orc_triplanar_shade(C.cast(arr, C.c_void_p), n, *[_p(a) for a in arrs + d], _p(ids), float(scale),
                                   FILTERS[filter], MODES[mode], BLENDS[blend], SHADES[shade], spp, seed, flags,
                                   _p(rgb), _p(picks), _p(picks64), _p(bd), _p(mag), nthreads or nthreads_default())
    if rc != 0:
        raise ValueError("oracle: invalid triplanar_shade arguments")
    return FilterResult(rgb, picks, picks64, bd, mag, None)


@dataclass
class MarchResult:
    T: np.ndarray               # (count,) float64
    picks: np.ndarray | None    # (count, spp, steps) uint32 (z<<20 | y<<10 | x), FP32 decisions (diagnostic)
    bdist: np.ndarray
    picks64: np.ndarray | None = None  # same, FP64 decisions (the ones the estimate uses)


def march(vol: np.ndarray, sigma_scale: float, cam: np.ndarray, width: int, height: int,
          steps: int, filter: str, mode: str, spp: int, seed: int, flags: int = 0,
          pix_begin: int = 0, pix_count: int | None = None, want_picks: bool = False,
          nthreads: int | None = None, pix_ids=None) -> MarchResult:
    """Pixels pix_begin.. (or the explicit list pix_ids) of a width x height image."""
    vol = np.ascontiguousarray(vol, dtype=np.float16)
    nz, ny, nx = vol.shape
    if pix_ids is not None:
        pix_ids = np.ascontiguousarray(pix_ids, dtype=np.uint64)
        cnt = len(pix_ids)
    else:
        cnt = width * height - pix_begin if pix_count is None else pix_count
    T = np.zeros(cnt)
    bd = np.zeros(cnt)
    picks = np.zeros((cnt, spp, steps), dtype=np.uint32) if want_picks else None
    picks64 = np.zeros((cnt, spp, steps), dtype=np.uint32) if want_picks else None
    cam = np.ascontiguousarray(cam, dtype=np.float32)
    rc = lib().orc_march(nx, ny, nz, _p(vol.view(np.uint16)), float(sigma_scale), _p(cam), width,
                         height, steps, FILTERS[filter], MODES[mode], spp, seed, flags, pix_begin,
                         cnt, _p(pix_ids), _p(T), _p(picks), _p(picks64), _p(bd), nthreads or nthreads_default())
    if rc != 0:
        raise ValueError("oracle: invalid march arguments")
    return MarchResult(T, picks, bd, picks64)


# ----------------------------------------------------------------------------- learned form
def round_bf16(x) -> np.ndarray:
    return np.array([lib().orc_round_bf16(float(v)) for v in np.ravel(x)]).reshape(np.shape(x))


def round_fp16(x) -> np.ndarray:
    return np.array([lib().orc_round_fp16(float(v)) for v in np.ravel(x)]).reshape(np.shape(x))


def round_e4m3(x) -> np.ndarray:
    return np.array([lib().orc_round_e4m3(float(v)) for v in np.ravel(x)]).reshape(np.shape(x))


def e4m3_value(codes) -> np.ndarray:
    return np.array([lib().orc_e4m3_value(int(c)) for c in np.ravel(codes)]).reshape(np.shape(codes))


def _e4m3_codes(values: np.ndarray) -> np.ndarray:
    """FP8 E4M3 codes of values that are already E4M3-representable (table lookup)."""
    table = np.array([lib().orc_e4m3_value(c) for c in range(256)])
    out = np.zeros(values.shape, dtype=np.uint8)
    flat = values.ravel()
    pos = {float(table[c]): c for c in range(256) if not np.isnan(table[c]) and (c & 0x80) == 0}
    neg = {float(table[c]): c for c in range(128, 256) if not np.isnan(table[c])}
    o = out.ravel()
    for i, v in enumerate(flat):
        o[i] = pos[float(v)] if (v > 0 or (v == 0 and not np.signbit(v))) else neg[float(v)]
    return out


@dataclass
class NeuralTexture:
    """Latents: 4 grids (R, R, 8) as float16 (fmt 'fp16'), float32 ('fp32'), or FP8
    E4M3 codes (uint8, 'fp8') with per-grid scales.  MLP weights as float64 copies of the
    values the decode uses (BF16-rounded for inference)."""
    tex_res: int
    grids: list
    mlp: np.ndarray               # [6792] W1 b1 W2 b2 W3 b3
    fmt: str = "fp16"
    scales: tuple = (1.0, 1.0, 1.0, 1.0)

    def _struct(self):
        m = np.asarray(self.mlp, dtype=np.float64)
        cut = np.cumsum([0, 2048, 64, 4096, 64, 512, 8])
        self._parts = [np.ascontiguousarray(m[cut[i]:cut[i + 1]]) for i in range(6)]
        self._mlp = _Mlp(*[p.ctypes.data for p in self._parts])
        if self.fmt == "fp16":
            gs = [np.ascontiguousarray(g, dtype=np.float16).view(np.uint16) for g in self.grids]
            f = 0
        elif self.fmt == "fp8":
            gs = [np.ascontiguousarray(g, dtype=np.uint8) for g in self.grids]
            f = 1
        else:
            gs = [np.ascontiguousarray(g, dtype=np.float32) for g in self.grids]
            f = 2
        self._grids = gs
        s = _NeuralTex(self.tex_res, (C.c_int * 4)(*[g.shape[0] for g in gs]), f,
                       (C.c_void_p * 4)(*[g.ctypes.data for g in gs]), (C.c_float * 4)(*self.scales),
                       C.pointer(self._mlp))
        return s

    @staticmethod
    def inference_form(tex_res: int, lat32, mlp32, fmt: str = "fp16") -> "NeuralTexture":
        """The quantised inference form of FP32 master parameters, built by the oracle's
        own codecs: BF16 weights (biases FP32), FP16 latents, or FP8 E4M3 latents with a
        per-grid scale max|l| / 448 (FP32 arithmetic: scale = amax / 448, code =
        E4M3(l * (1 / scale)))."""
        m = np.asarray(mlp32, dtype=np.float32).astype(np.float64)
        cut = np.cumsum([0, 2048, 64, 4096, 64, 512, 8])
        w = m.copy()
        for a, b in ((0, 1), (2, 3), (4, 5)):
            w[cut[a]:cut[b]] = round_bf16(m[cut[a]:cut[b]].astype(np.float32))
        if fmt == "fp16":
            return NeuralTexture(tex_res, [np.asarray(g, np.float32).astype(np.float16) for g in lat32], w, "fp16")
        scales, codes = [], []
        for g in lat32:
            g = np.asarray(g, dtype=np.float32)
            amax = np.float32(np.max(np.abs(g)))
            sc = np.float32(max(amax, np.float32(1e-30)) / np.float32(448.0))
            inv = np.float32(np.float32(1.0) / sc)
            vals = round_e4m3((g * inv).astype(np.float32))
            codes.append(_e4m3_codes(vals))
            scales.append(float(sc))
        return NeuralTexture(tex_res, codes, w, "fp8", tuple(scales))


def ntc_features(nt: NeuralTexture, ix, iy) -> np.ndarray:
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    out = np.zeros((len(ix), 32), dtype=np.float32)
    s = nt._struct()
    lib().orc_ntc_features(C.byref(s), len(ix), _p(ix), _p(iy), _p(out))
    return out


def ntc_decode(nt: NeuralTexture, ix, iy):
    """(y [n, 8] float64, rdist [n]): decode, and the smallest rounding margin of its hidden
    BF16 activations (distance to the rounding midpoint / (sqrt(K+1) sum|w x|)); a margin of
    a fraction of 2^-24 can round differently under another FP32 summation order."""
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    y = np.zeros((len(ix), 8))
    rd = np.zeros(len(ix))
    s = nt._struct()
    lib().orc_ntc_decode(C.byref(s), len(ix), _p(ix), _p(iy), _p(y), _p(rd))
    return y, rd


def ntc_decode_exact(tex_res: int, lat32, mlp32, ix, iy) -> np.ndarray:
    """y [n, 8] float64: the network's exact value at texels (ix, iy) -- FP64 bilinear
    features of the FP32 master latents and an FP64 forward pass of the FP32 master MLP, with
    no BF16, FP16 or FP8 rounding anywhere.  The reference the inference forms' decode error
    is stated against."""
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    nt = NeuralTexture(tex_res, [np.asarray(g, np.float32) for g in lat32],
                       np.asarray(mlp32, np.float32).astype(np.float64), "fp32")
    y = np.zeros((len(ix), 8))
    s = nt._struct()
    lib().orc_ntc_decode_exact(C.byref(s), len(ix), _p(ix), _p(iy), _p(y))
    return y


def ntc_loss_grad(tex_res: int, lat32, mlp32, targets, ix, iy, round_bf16: bool = True,
                  bf16_backward: bool = False):
    """Loss and gradients of one batch from FP32 master parameters.  round_bf16: BF16
    operands in the forward GEMMs; bf16_backward (with round_bf16): also the backward GEMMs'
    operands dy, dh2 and dh1 rounded to BF16 where they are formed."""
    nt = NeuralTexture(tex_res, [np.asarray(g, np.float32) for g in lat32], np.zeros(6792), "fp32")
    s = nt._struct()
    m = np.ascontiguousarray(mlp32, dtype=np.float32)
    cut = np.cumsum([0, 2048, 64, 4096, 64, 512, 8])
    parts = [np.ascontiguousarray(m[cut[i]:cut[i + 1]]) for i in range(6)]
    grads = [np.zeros(p.size) for p in parts]
    dl = [np.zeros(np.asarray(g).size) for g in lat32]
    dlp = (C.c_void_p * 4)(*[g.ctypes.data for g in dl])
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    tg = np.ascontiguousarray(targets, dtype=np.uint8)
    loss = lib().orc_ntc_loss_grad(C.byref(s), *[_p(p) for p in parts], _p(tg), len(ix), _p(ix), _p(iy),
                                   (2 if bf16_backward else 1) if round_bf16 else 0, *[_p(g) for g in grads], dlp)
    return loss, np.concatenate(grads), np.concatenate(dl)


def adam(p, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place FP64 Adam step on float64 arrays."""
    lib().orc_adam(p.size, _p(p), _p(g), _p(m), _p(v), t, lr, beta1, beta2, eps)


def ntc_sample_texels(step: int, batch: int, seed: int, tex_res: int):
    """Training texels of one optimiser step: Philox(ctr = (k, step, 0, 0x4E54), key = seed),
    ix = mulhi(word0, tex_res), iy = mulhi(word1, tex_res)."""
    ix = np.zeros(batch, dtype=np.int32)
    iy = np.zeros(batch, dtype=np.int32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for k in range(batch):
        w = philox([k, step, 0, 0x4E54], key)
        ix[k] = (int(w[0]) * tex_res) >> 32
        iy[k] = (int(w[1]) * tex_res) >> 32
    return ix, iy

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
SRC = os.path.join(HERE, "stf_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

FILTERS = {"linear": 0, "bspline": 1, "catmull_rom": 2, "mitchell": 3}
MODES = {"ntap_before": 0, "ntap_after": 1, "stochastic": 2, "positivized": 3}
SHADES = {"ggx": 0, "linear": 1}
FLAG_STRATIFIED = 1
NO_PICK = 0xFFFFFFFF


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", SRC, "-o", LIB + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class _Tex(C.Structure):
    _fields_ = [("format", C.c_int), ("levels", C.c_int), ("address", C.c_int),
                ("width", C.c_int * 16), ("height", C.c_int * 16),
                ("data", C.c_void_p * 16), ("normal", C.c_void_p * 16)]


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
        L.orc_pick_array.argtypes = [P, C.c_int, C.c_double]
        L.orc_ggx_eval.argtypes = [P, P, P, C.c_double, P, C.c_double, P]
        L.orc_ggx_D.argtypes = [C.c_double, C.c_double]
        L.orc_ggx_D.restype = C.c_double
        L.orc_smith_lambda.argtypes = [C.c_double, C.c_double]
        L.orc_smith_lambda.restype = C.c_double
        L.orc_shade_batch.argtypes = [C.c_uint64, C.c_int, P, P, P, P]
        L.orc_fetch.argtypes = [C.POINTER(_Tex), C.c_int, C.c_int, C.c_int, P]
        L.orc_filter_shade.argtypes = [C.POINTER(_Tex), C.c_uint64] + [P] * 7 + [
            C.c_int, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32, P, P, P, P, P, C.c_int]
        L.orc_march.argtypes = [C.c_int, C.c_int, C.c_int, P, C.c_float, P, C.c_uint32, C.c_uint32,
                                C.c_uint32, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32,
                                C.c_uint64, C.c_uint64, P, P, P, P, C.c_int]
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

    def _struct(self):
        t = _Tex()
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


def filter_shade(tex: Texture, q, filter: str, mode: str, shade: str = "ggx", spp: int = 1,
                 seed: int = 1, flags: int = 0, want_picks: bool = False,
                 nthreads: int | None = None, ids=None) -> FilterResult:
    """Evaluate queries q; the Philox id of query i is ids[i] (default: i)."""
    n = q.n
    rgb = np.zeros((n, 3))
    picks = np.zeros((n, spp, 2), dtype=np.uint32) if want_picks else None
    picks64 = np.zeros((n, spp, 2), dtype=np.uint32) if want_picks else None
    bd = np.zeros(n)
    mag = np.zeros((n, 3))
    t = tex._struct()
    arrs = [np.ascontiguousarray(a, dtype=np.float32) if a is not None else None
            for a in (q.u, q.v, q.dudx, q.dvdx, q.dudy, q.dvdy)]
    ids = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint64)
    rc = lib().orc_filter_shade(C.byref(t), n, *[_p(a) for a in arrs], _p(ids), FILTERS[filter], MODES[mode],
                                SHADES[shade], spp, seed, flags, _p(rgb), _p(picks), _p(picks64),
                                _p(bd), _p(mag), nthreads or nthreads_default())
    if rc != 0:
        raise ValueError("oracle: invalid filter_shade arguments")
    return FilterResult(rgb, picks, picks64, bd, mag)


@dataclass
class MarchResult:
    T: np.ndarray               # (count,) float64
    picks: np.ndarray | None    # (count, spp, steps) uint32 (z<<20 | y<<10 | x)
    bdist: np.ndarray


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
    cam = np.ascontiguousarray(cam, dtype=np.float32)
    rc = lib().orc_march(nx, ny, nz, _p(vol.view(np.uint16)), float(sigma_scale), _p(cam), width,
                         height, steps, FILTERS[filter], MODES[mode], spp, seed, flags, pix_begin,
                         cnt, _p(pix_ids), _p(T), _p(picks), _p(bd), nthreads or nthreads_default())
    if rc != 0:
        raise ValueError("oracle: invalid march arguments")
    return MarchResult(T, picks, bd)

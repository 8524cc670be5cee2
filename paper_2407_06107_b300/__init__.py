"""Python binding of libstf -- stochastic texture filtering on B300 (sm_103a).

Argument marshalling only: every step of the hot path runs in the CUDA kernels of
``csrc/`` behind the C ABI of ``include/stf.h``.  torch is used for device memory and
streams.  There is no CPU fallback: if ``libstf.so`` has not been built, or no CUDA device
is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstf.so")

FILTERS = {"linear": 0, "bspline": 1, "catmull_rom": 2, "mitchell": 3, "ewa": 4, "gauss": 5}
SAMPLERS = {"frs": 0, "fis": 1}
MODES = {"ntap_before": 0, "ntap_after": 1, "stochastic": 2, "positivized": 3}
SHADES = {"ggx": 0, "linear": 1}
BLENDS = {"full": 0, "stochastic": 1}
FMT_RGBA32F, FMT_RGBA8, FMT_RG8, FMT_R16F, FMT_DCT6 = 0, 1, 2, 3, 4
FLAG_STRATIFIED = 1
FLAG_LATTICE = 2
FLAG_REUSE = 4
FLAG_LOD0 = 8
DEV_NAN_INPUT, DEV_BAD_INDEX, DEV_TIMEOUT = 1, 2, 4
NO_PICK = 0xFFFFFFFF

STATUS = {0: "STF_OK", 1: "STF_ERR_INVALID_ARG", 2: "STF_ERR_BAD_HANDLE", 3: "STF_ERR_OOM",
          4: "STF_ERR_CUDA", 5: "STF_ERR_UNSUPPORTED", 6: "STF_ERR_DEVICE_STATUS", 7: "STF_ERR_TIMEOUT"}


class StfError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _TextureDesc(C.Structure):
    _fields_ = [("width", C.c_uint32), ("height", C.c_uint32), ("num_levels", C.c_uint32),
                ("format", C.c_int), ("address", C.c_int), ("level_data", C.POINTER(C.c_void_p)),
                ("normal_data", C.POINTER(C.c_void_p)), ("data_on_device", C.c_int)]


class _Queries(C.Structure):
    _fields_ = [("n", C.c_uint64), ("id_base", C.c_uint64), ("u", C.c_void_p), ("v", C.c_void_p),
                ("order", C.c_void_p)]


class _Derivs(C.Structure):
    _fields_ = [("dudx", C.c_void_p), ("dvdx", C.c_void_p), ("dudy", C.c_void_p), ("dvdy", C.c_void_p)]


class _Output(C.Structure):
    _fields_ = [("r", C.c_void_p), ("g", C.c_void_p), ("b", C.c_void_p), ("picks", C.c_void_p)]


class _TriQueries(C.Structure):
    _fields_ = [("n", C.c_uint64), ("id_base", C.c_uint64)] + [
        (k, C.c_void_p) for k in ("px", "py", "pz", "nx", "ny", "nz", "order")]


class _TriDerivs(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("dpdx_x", "dpdx_y", "dpdx_z", "dpdy_x", "dpdy_y", "dpdy_z")]


class _FilterDesc(C.Structure):
    _fields_ = [("filter", C.c_int), ("sampler", C.c_int), ("sigma", C.c_float)]


class _NeuralDesc(C.Structure):
    _fields_ = [("tex_res", C.c_uint32), ("grid_res", C.c_uint32 * 4), ("latent_init", C.POINTER(C.c_void_p)),
                ("mlp_init", C.c_void_p), ("targets", C.c_void_p)]


class _Adam(C.Structure):
    _fields_ = [("lr_latent", C.c_float), ("lr_mlp", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("lr_min_frac", C.c_float)]


NEURAL_BLOCKS = {"latents": 0, "mlp": 1, "grad_latents": 2, "grad_mlp": 3, "adam": 4, "scales": 5, "step": 6}
LATENT_FORMATS = {"fp16": 0, "fp8": 1, "keep": -1}
MLP_SIZE = 6792

# every entry point declared in include/stf.h, with its ctypes signature
_P, _U32, _U64, _I, _F = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int, C.c_float
SIGNATURES = {
    "stf_create": ([_I, _P, C.POINTER(_P)], _I),
    "stf_destroy": ([_P], _I),
    "stf_set_stream": ([_P, _P], _I),
    "stf_synchronize": ([_P], _I),
    "stf_get_device_status": ([_P, C.POINTER(_U32)], _I),
    "stf_status_string": ([_I], C.c_char_p),
    "stf_last_error": ([_P], C.c_char_p),
    "stf_create_texture": ([_P, C.POINTER(_TextureDesc), C.POINTER(_U64)], _I),
    "stf_destroy_texture": ([_P, _U64], _I),
    "stf_filter_shade": ([_P, _U64, C.POINTER(_Queries), C.POINTER(_Derivs), _I, _I, _I, _U32, _U64,
                          _U32, C.POINTER(_Output)], _I),
    "stf_filter_shade_ex": ([_P, _U64, C.POINTER(_Queries), C.POINTER(_Derivs), C.POINTER(_FilterDesc), _I, _I,
                             _U32, _U64, _U32, C.POINTER(_Output)], _I),
    "stf_filter_shade_host": ([_P, _U64, C.POINTER(_Queries), C.POINTER(_Derivs), _I, _I, _I, _U32,
                               _U64, _U32, C.POINTER(_Output)], _I),
    "stf_filter_shade_host_async": ([_P, _U64, C.POINTER(_Queries), C.POINTER(_Derivs), _I, _I, _I, _U32,
                                     _U64, _U32, C.POINTER(_Output)], _I),
    "stf_bin_queries": ([_P, _U64, _P, _P, _P, _U32, _U32, _P], _I),
    "stf_create_texture_table": ([_P, _U32, _P, C.POINTER(_U64)], _I),
    "stf_destroy_texture_table": ([_P, _U64], _I),
    "stf_filter_shade_table": ([_P, _U64, C.POINTER(_Queries), _P, C.POINTER(_Derivs), _I, _I, _I, _U32, _U64, _U32,
                                C.POINTER(_Output)], _I),
    "stf_filter_shade_host_noalloc": ([_P, _U64, C.POINTER(_Queries), C.POINTER(_Derivs), _I, _I, _I, _U32,
                                       _U64, _U32, C.POINTER(_Output)], _I),
    "stf_measure_sector_rate": ([_P, _U64, C.POINTER(C.c_double)], _I),
    "stf_triplanar_shade": ([_P, _P, _F, C.POINTER(_TriQueries), C.POINTER(_TriDerivs), _I, _I, _I, _I, _U32, _U64,
                             _U32, C.POINTER(_Output)], _I),
    "stf_create_volume": ([_P, _U32, _U32, _U32, _I, _F, _P, _I, C.POINTER(_U64)], _I),
    "stf_destroy_volume": ([_P, _U64], _I),
    "stf_march_volume": ([_P, _U64, _P, _U32, _U32, _U32, _I, _I, _U32, _U64, _U32, _U64, _U64, _P, _P], _I),
    "stf_neural_create": ([_P, C.POINTER(_NeuralDesc), C.POINTER(_U64)], _I),
    "stf_neural_destroy": ([_P, _U64], _I),
    "stf_neural_train": ([_P, _U64, _U32, _U32, C.POINTER(_Adam), _U64, _P], _I),
    "stf_neural_grad": ([_P, _U64, _U32, _U32, _U64, _P, _P, C.POINTER(C.c_float)], _I),
    "stf_neural_grad_range": ([_P, _U64, _U32, _U32, _U32, _U32, _U64, _P], _I),
    "stf_neural_grad_buffers": ([_P, _U64, C.POINTER(_P), C.POINTER(_U64), C.POINTER(_P), C.POINTER(_U64)], _I),
    "stf_neural_adam_step": ([_P, _U64, C.POINTER(_Adam), _U32, _U32], _I),
    "stf_neural_quantize": ([_P, _U64, _I], _I),
    "stf_neural_get": ([_P, _U64, _I, _P, C.c_size_t], _I),
    "stf_neural_set": ([_P, _U64, _I, _P, C.c_size_t], _I),
    "stf_neural_save": ([_P, _U64, C.c_char_p], _I),
    "stf_neural_load": ([_P, _U64, C.c_char_p], _I),
    "stf_neural_decode": ([_P, _U64, _U64, _P, _P, _P], _I),
    "stf_neural_filter_shade": ([_P, _U64, C.POINTER(_Queries), C.POINTER(_Derivs), _I, _I, _I, _U32, _U64, _U32,
                                 C.POINTER(_Output)], _I),
}

_lib = None


def lib() -> C.CDLL:
    """Load libstf.so (raises if it was never built -- there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not built: run __graft_entry__.build() or "
                               "python paper_2407_06107_b300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes, fn.restype = args, res
        _lib = L
    return _lib


class _CudaArray:
    """A raw float32 device array, exposed through the CUDA array interface."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3,
                                         "strides": None}


def _device_view(ptr: int, n: int, device: int):
    import torch
    return torch.as_tensor(_CudaArray(ptr, n), device=torch.device("cuda", device))


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


class Context:
    """One libstf context on one CUDA device, bound to a CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        self._check(lib().stf_create(device, C.c_void_p(stream.cuda_stream), C.byref(h)), None)
        self.h = h

    # -------------------------------------------------------------- plumbing
    def _check(self, st: int, h=None):
        if st != 0:
            msg = lib().stf_last_error(h if h is not None else getattr(self, "h", None)) or b""
            raise StfError(st, msg.decode())

    def close(self):
        if getattr(self, "h", None):
            lib().stf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        self._check(lib().stf_synchronize(self.h), self.h)

    def set_stream(self, stream):
        self.stream = stream
        self._check(lib().stf_set_stream(self.h, C.c_void_p(stream.cuda_stream)), self.h)

    def device_status(self) -> int:
        f = C.c_uint32(0)
        st = lib().stf_get_device_status(self.h, C.byref(f))
        if st not in (0, 6):
            self._check(st, self.h)
        return int(f.value)

    # -------------------------------------------------------------- resources
    def create_texture(self, levels, normal=None, address: str = "wrap") -> int:
        """levels: list of (H, W, 4) float32 or uint8 arrays (numpy host or torch cuda)."""
        on_dev = not isinstance(levels[0], np.ndarray)
        keep = [lv if on_dev else np.ascontiguousarray(lv) for lv in levels]
        fmt = FMT_RGBA32F if (str(keep[0].dtype).endswith("float32")) else FMT_RGBA8
        arr = (C.c_void_p * len(keep))(*[_ptr(x) for x in keep])
        narr = None
        if normal is not None:
            nk = [nm if on_dev else np.ascontiguousarray(nm) for nm in normal]
            keep += nk
            narr = (C.c_void_p * len(nk))(*[_ptr(x) for x in nk])
        d = _TextureDesc(int(keep[0].shape[1]), int(keep[0].shape[0]), len(levels), fmt,
                         0 if address == "wrap" else 1, arr, narr, 1 if on_dev else 0)
        out = C.c_uint64(0)
        self._check(lib().stf_create_texture(self.h, C.byref(d), C.byref(out)), self.h)
        return int(out.value)

    def create_texture_dct(self, blocks, width: int, height: int) -> int:
        """DCT-compressed material: per level a (ceil(H/8), ceil(W/8), 32) uint8 block array
        (numpy host or torch cuda); width, height of level 0."""
        on_dev = not isinstance(blocks[0], np.ndarray)
        keep = [b if on_dev else np.ascontiguousarray(b, dtype=np.uint8) for b in blocks]
        arr = (C.c_void_p * len(keep))(*[_ptr(x) for x in keep])
        d = _TextureDesc(int(width), int(height), len(keep), FMT_DCT6, 0, arr, None, 1 if on_dev else 0)
        out = C.c_uint64(0)
        self._check(lib().stf_create_texture(self.h, C.byref(d), C.byref(out)), self.h)
        return int(out.value)

    def destroy_texture(self, tex: int):
        self._check(lib().stf_destroy_texture(self.h, tex), self.h)

    def create_volume(self, data, sigma_scale: float) -> int:
        """data: (nz, ny, nx) float16, numpy host or torch cuda."""
        on_dev = not isinstance(data, np.ndarray)
        if not on_dev:
            data = np.ascontiguousarray(data, dtype=np.float16)
        nz, ny, nx = data.shape
        out = C.c_uint64(0)
        self._check(lib().stf_create_volume(self.h, nx, ny, nz, FMT_R16F, float(sigma_scale),
                                            C.c_void_p(_ptr(data)), 1 if on_dev else 0, C.byref(out)), self.h)
        return int(out.value)

    def destroy_volume(self, vol: int):
        self._check(lib().stf_destroy_volume(self.h, vol), self.h)

    # -------------------------------------------------------------- hot path
    def _args(self, u, v, derivs, out, picks, n, id_base, order=None):
        q = _Queries(n, id_base, _ptr(u), _ptr(v), _ptr(order))
        d = None
        if derivs is not None:
            d = _Derivs(*[_ptr(x) for x in derivs])
        o = _Output(_ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _ptr(picks))
        return q, d, o

    def filter_shade(self, tex: int, u, v, derivs=None, filter: str = "bspline", mode: str = "stochastic",
                     shade: str = "ggx", spp: int = 1, seed: int = 1, flags: int = 0, id_base: int = 0,
                     out=None, want_picks: bool = False, order=None, sampler: str = "frs", sigma: float = 0.0):
        """u, v, derivs (dudx, dvdx, dudy, dvdy): float32 cuda tensors; order: optional int32
        cuda permutation (execution order); sampler "frs" / "fis" and sigma (texels) for the
        Gaussian go through stf_filter_shade_ex.  Returns (r, g, b, picks)."""
        torch = self.torch
        n = int(u.shape[0])
        if out is None:
            out = [torch.empty(n, dtype=torch.float32, device=u.device) for _ in range(3)]
        picks = torch.empty((n, spp, 2), dtype=torch.int32, device=u.device) if want_picks else None
        q, d, o = self._args(u, v, derivs, out, picks, n, id_base, order)
        dp = C.byref(d) if d is not None else None
        if sampler != "frs" or filter == "gauss":
            fd = _FilterDesc(FILTERS[filter], SAMPLERS[sampler], float(sigma))
            st = lib().stf_filter_shade_ex(self.h, tex, C.byref(q), dp, C.byref(fd), MODES[mode], SHADES[shade],
                                           spp, seed, flags, C.byref(o))
        else:
            st = lib().stf_filter_shade(self.h, tex, C.byref(q), dp, FILTERS[filter], MODES[mode], SHADES[shade],
                                        spp, seed, flags, C.byref(o))
        self._check(st, self.h)
        return out[0], out[1], out[2], picks

    def triplanar_shade(self, textures, scale: float, p, nrm, derivs=None, filter: str = "linear",
                        mode: str = "stochastic", blend: str = "stochastic", shade: str = "ggx", spp: int = 1,
                        seed: int = 1, flags: int = 0, id_base: int = 0, out=None, want_picks: bool = False,
                        order=None):
        """Triplanar lookups of surface points: textures = three handles (planes along x, y, z);
        p = (px, py, pz) and nrm = (nx, ny, nz) float32 cuda tensors; derivs = (dP/dx xyz,
        dP/dy xyz), six tensors, or None.  Returns (r, g, b, picks [n, spp, 3, 2])."""
        torch = self.torch
        n = int(p[0].shape[0])
        if out is None:
            out = [torch.empty(n, dtype=torch.float32, device=p[0].device) for _ in range(3)]
        picks = torch.empty((n, spp, 3, 2), dtype=torch.int32, device=p[0].device) if want_picks else None
        texs = (C.c_uint64 * 3)(*[int(t) for t in textures])
        q = _TriQueries(n, id_base, *[_ptr(x) for x in p], *[_ptr(x) for x in nrm], _ptr(order))
        d = _TriDerivs(*[_ptr(x) for x in derivs]) if derivs is not None else None
        o = _Output(_ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _ptr(picks))
        st = lib().stf_triplanar_shade(self.h, texs, float(scale), C.byref(q), C.byref(d) if d is not None else None,
                                       FILTERS[filter], MODES[mode], BLENDS[blend], SHADES[shade], spp, seed, flags,
                                       C.byref(o))
        self._check(st, self.h)
        return out[0], out[1], out[2], picks

    def filter_shade_host(self, tex: int, u, v, derivs=None, filter: str = "bspline", mode: str = "stochastic",
                          shade: str = "ggx", spp: int = 1, seed: int = 1, flags: int = 0, id_base: int = 0,
                          out=None, want_picks: bool = False):
        """Host (CPU, ideally pinned) float32 tensors or numpy arrays in and out."""
        n = int(u.shape[0])
        if out is None:
            out = [np.empty(n, dtype=np.float32) for _ in range(3)]
        picks = np.empty((n, spp, 2), dtype=np.uint32) if want_picks else None
        q, d, o = self._args(u, v, derivs, out, picks, n, id_base)
        st = lib().stf_filter_shade_host(self.h, tex, C.byref(q), C.byref(d) if d is not None else None,
                                         FILTERS[filter], MODES[mode], SHADES[shade], spp, seed, flags, C.byref(o))
        self._check(st, self.h)
        return out[0], out[1], out[2], picks

    def filter_shade_host_async(self, tex: int, u, v, derivs=None, filter: str = "bspline",
                                mode: str = "stochastic", shade: str = "ggx", spp: int = 1, seed: int = 1,
                                flags: int = 0, id_base: int = 0, out=None):
        """filter_shade_host without the final wait: the results (and the inputs' release) are
        valid after synchronize().  The arrays passed or returned must stay alive until then."""
        n = int(u.shape[0])
        if out is None:
            out = [np.empty(n, dtype=np.float32) for _ in range(3)]
        q, d, o = self._args(u, v, derivs, out, None, n, id_base)
        st = lib().stf_filter_shade_host_async(self.h, tex, C.byref(q), C.byref(d) if d is not None else None,
                                               FILTERS[filter], MODES[mode], SHADES[shade], spp, seed, flags,
                                               C.byref(o))
        self._check(st, self.h)
        return out[0], out[1], out[2]

    def bin_queries(self, u, v, tex_id=None, ntex: int = 1, tile_log2: int = 6, order=None):
        """Spatial execution order (int32 cuda tensor [n]) for filter_shade(order=...)."""
        n = int(u.shape[0])
        if order is None:
            order = self.torch.empty(n, dtype=self.torch.int32, device=u.device)
        self._check(lib().stf_bin_queries(self.h, n, _ptr(u), _ptr(v), _ptr(tex_id), ntex, tile_log2, _ptr(order)),
                    self.h)
        return order

    def create_texture_table(self, textures) -> int:
        arr = (C.c_uint64 * len(textures))(*textures)
        out = C.c_uint64(0)
        self._check(lib().stf_create_texture_table(self.h, len(textures), arr, C.byref(out)), self.h)
        return int(out.value)

    def destroy_texture_table(self, table: int):
        self._check(lib().stf_destroy_texture_table(self.h, table), self.h)

    def filter_shade_table(self, table: int, u, v, tex_id, derivs=None, filter: str = "mitchell",
                           mode: str = "stochastic", shade: str = "ggx", spp: int = 1, seed: int = 1,
                           flags: int = 0, id_base: int = 0, out=None, want_picks: bool = False, order=None):
        """tex_id: int32/uint32 cuda tensor [n] of table entries; order: optional permutation."""
        torch = self.torch
        n = int(u.shape[0])
        if out is None:
            out = [torch.empty(n, dtype=torch.float32, device=u.device) for _ in range(3)]
        picks = torch.empty((n, spp, 2), dtype=torch.int32, device=u.device) if want_picks else None
        q, d, o = self._args(u, v, derivs, out, picks, n, id_base, order)
        st = lib().stf_filter_shade_table(self.h, table, C.byref(q), C.c_void_p(_ptr(tex_id)),
                                          C.byref(d) if d is not None else None, FILTERS[filter], MODES[mode],
                                          SHADES[shade], spp, seed, flags, C.byref(o))
        self._check(st, self.h)
        return out[0], out[1], out[2], picks

    def filter_shade_host_noalloc(self, tex: int, u, v, derivs=None, filter: str = "bspline",
                                  mode: str = "stochastic", shade: str = "ggx", spp: int = 1, seed: int = 1,
                                  flags: int = 0, id_base: int = 0, out=None):
        """stf_filter_shade_host without any device allocation (at most 2^18 queries per
        call; the library's fixed staging array is shared by all calls on a device)."""
        n = int(u.shape[0])
        if out is None:
            out = [np.empty(n, dtype=np.float32) for _ in range(3)]
        q, d, o = self._args(u, v, derivs, out, None, n, id_base)
        st = lib().stf_filter_shade_host_noalloc(self.h, tex, C.byref(q), C.byref(d) if d is not None else None,
                                                 FILTERS[filter], MODES[mode], SHADES[shade], spp, seed, flags,
                                                 C.byref(o))
        self._check(st, self.h)
        return out[0], out[1], out[2]

    def measure_sector_rate(self, buffer_bytes: int = 32 << 20) -> float:
        """Random 32-byte sector reads per second at L2 over a buffer of buffer_bytes (the
        gather roofline's measured denominator)."""
        out = C.c_double(0.0)
        self._check(lib().stf_measure_sector_rate(self.h, buffer_bytes, C.byref(out)), self.h)
        return float(out.value)

    def march_volume(self, vol: int, cam, width: int, height: int, steps: int = 128,
                     filter: str = "bspline", mode: str = "stochastic", spp: int = 1, seed: int = 1,
                     flags: int = 0, pix_begin: int = 0, pix_count: int | None = None, out=None,
                     want_picks: bool = False):
        torch = self.torch
        cnt = width * height - pix_begin if pix_count is None else pix_count
        if out is None:
            out = torch.empty(cnt, dtype=torch.float32, device=f"cuda:{self.device}")
        picks = (torch.empty((cnt, spp, steps), dtype=torch.int32, device=f"cuda:{self.device}")
                 if want_picks else None)
        camv = (C.c_float * 12)(*[float(x) for x in np.asarray(cam, dtype=np.float32)])
        st = lib().stf_march_volume(self.h, vol, camv, width, height, steps, FILTERS[filter], MODES[mode],
                                    spp, seed, flags, pix_begin, cnt, C.c_void_p(_ptr(out)),
                                    C.c_void_p(_ptr(picks)) if picks is not None else None)
        self._check(st, self.h)
        return out, picks

    # -------------------------------------------------------------- learned form
    def neural_create(self, tex_res: int, latents, mlp, targets=None) -> int:
        """latents: 4 host float32 arrays (R, R, 8); mlp: float32 [6792]; targets: uint8
        (tex_res, tex_res, 8) or None."""
        lat = [np.ascontiguousarray(x, dtype=np.float32) for x in latents]
        mlp = np.ascontiguousarray(mlp, dtype=np.float32)
        assert mlp.size == MLP_SIZE
        tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.uint8)
        arr = (C.c_void_p * 4)(*[x.ctypes.data for x in lat])
        d = _NeuralDesc(tex_res, (C.c_uint32 * 4)(*[x.shape[0] for x in lat]), arr, mlp.ctypes.data,
                        None if tg is None else tg.ctypes.data)
        out = C.c_uint64(0)
        self._check(lib().stf_neural_create(self.h, C.byref(d), C.byref(out)), self.h)
        return int(out.value)

    def neural_destroy(self, net: int):
        self._check(lib().stf_neural_destroy(self.h, net), self.h)

    def neural_train(self, net: int, steps: int, batch: int, lr_latent: float = 1e-2, lr_mlp: float = 5e-3,
                     seed: int = 1, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                     lr_min_frac: float = 1.0) -> np.ndarray:
        """steps Adam steps of batch samples; lr_min_frac < 1 decays the learning rates on a half
        cosine to lr * lr_min_frac over the call.  Returns the per-step losses."""
        losses = np.zeros(steps, dtype=np.float32)
        ap = _Adam(lr_latent, lr_mlp, beta1, beta2, eps, lr_min_frac)
        self._check(lib().stf_neural_train(self.h, net, steps, batch, C.byref(ap), seed,
                                           losses.ctypes.data if steps else None), self.h)
        return losses

    def neural_grad(self, net: int, step: int, batch: int, seed: int = 1, ix=None, iy=None) -> float:
        loss = C.c_float(0)
        self._check(lib().stf_neural_grad(self.h, net, step, batch, seed, _ptr(ix), _ptr(iy), C.byref(loss)),
                    self.h)
        return float(loss.value)

    def neural_quantize(self, net: int, fmt: str = "fp16"):
        """fmt: "fp16", "fp8", or "keep" (rebuild in the current latent format)."""
        self._check(lib().stf_neural_quantize(self.h, net, LATENT_FORMATS[fmt]), self.h)

    # data-parallel training: the ranks' gradient shares are summed between grad and Adam
    def neural_grad_range(self, net: int, step: int, batch: int, first: int, count: int, seed: int = 1,
                          loss=None):
        """Gradients of samples [first, first + count) of step's batch (asynchronous); loss:
        optional float32 cuda tensor (one element) that receives this share of the loss."""
        self._check(lib().stf_neural_grad_range(self.h, net, step, batch, first, count, seed, _ptr(loss)), self.h)

    def neural_grad_buffers(self, net: int):
        """Zero-copy float32 cuda tensors over the network's latent and MLP gradient arrays."""
        pl, nl, pm, nm = _P(), _U64(), _P(), _U64()
        self._check(lib().stf_neural_grad_buffers(self.h, net, C.byref(pl), C.byref(nl), C.byref(pm), C.byref(nm)),
                    self.h)
        return _device_view(pl.value, nl.value, self.device), _device_view(pm.value, nm.value, self.device)

    def neural_grad_bucket(self, net: int):
        """One float32 cuda tensor over both gradient arrays (latents, the zero gap, MLP): the
        library lays them out adjacently, so one all-reduce of this view sums both."""
        pl, nl, pm, nm = _P(), _U64(), _P(), _U64()
        self._check(lib().stf_neural_grad_buffers(self.h, net, C.byref(pl), C.byref(nl), C.byref(pm), C.byref(nm)),
                    self.h)
        gap = pm.value - (pl.value + 4 * nl.value)
        if not 0 <= gap < 256 or gap % 4:
            raise StfError(5, "gradient arrays are not adjacent")
        return _device_view(pl.value, nl.value + gap // 4 + nm.value, self.device)

    def neural_adam_step(self, net: int, k: int, steps: int, lr_latent: float = 1e-2, lr_mlp: float = 5e-3,
                         beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, lr_min_frac: float = 1.0):
        ap = _Adam(lr_latent, lr_mlp, beta1, beta2, eps, lr_min_frac)
        self._check(lib().stf_neural_adam_step(self.h, net, C.byref(ap), k, steps), self.h)

    def neural_train_dp(self, net: int, steps: int, batch: int, lr_latent: float = 1e-2, lr_mlp: float = 5e-3,
                        seed: int = 1, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                        lr_min_frac: float = 1.0, group=None) -> np.ndarray:
        """neural_train as one rank of a data-parallel job (torch.distributed, one process per
        GPU, the context on the current torch stream): each rank computes its share of every
        batch, the gradients are all-reduced (summed) in place, and every replica applies the
        same Adam step.  Without an initialised process group it is a single replica.
        Returns the per-step losses of the whole batch."""
        import torch.distributed as dist
        from .sharding import dp_train
        torch = self.torch
        world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
        rank = dist.get_rank(group) if world > 1 else 0
        step0 = int(self.neural_get(net, "step", 0)[0])
        bucket = self.neural_grad_bucket(net)
        losses = torch.zeros(max(steps, 1), dtype=torch.float32, device=bucket.device)
        dp_train(steps, batch, rank, world,
                 lambda k, first, count: self.neural_grad_range(net, step0 + k, batch, first, count, seed,
                                                                losses[k:k + 1]),
                 lambda: dist.all_reduce(bucket, group=group),
                 lambda k: self.neural_adam_step(net, k, steps, lr_latent, lr_mlp, beta1, beta2, eps, lr_min_frac))
        if world > 1:
            dist.all_reduce(losses, group=group)
        self.neural_quantize(net, "keep")
        return losses[:steps].cpu().numpy()

    def _neural_block_size(self, net: int, what: str, lat_total: int) -> int:
        return {"latents": lat_total, "grad_latents": lat_total, "mlp": MLP_SIZE, "grad_mlp": MLP_SIZE,
                "adam": 2 * lat_total + 2 * MLP_SIZE, "scales": 4, "step": 1}[what]

    def neural_get(self, net: int, what: str, lat_total: int) -> np.ndarray:
        n = self._neural_block_size(net, what, lat_total)
        out = np.zeros(n, dtype=np.uint32 if what == "step" else np.float32)
        self._check(lib().stf_neural_get(self.h, net, NEURAL_BLOCKS[what], out.ctypes.data, out.nbytes), self.h)
        return out

    def neural_set(self, net: int, what: str, data: np.ndarray):
        data = np.ascontiguousarray(data, dtype=np.uint32 if what == "step" else np.float32)
        self._check(lib().stf_neural_set(self.h, net, NEURAL_BLOCKS[what], data.ctypes.data, data.nbytes), self.h)

    def neural_save(self, net: int, path: str):
        self._check(lib().stf_neural_save(self.h, net, path.encode()), self.h)

    def neural_load(self, net: int, path: str):
        self._check(lib().stf_neural_load(self.h, net, path.encode()), self.h)

    def neural_decode(self, net: int, ix, iy):
        """ix, iy: int32 cuda tensors [n] -> float32 cuda tensor [n, 8]."""
        n = int(ix.shape[0])
        y = self.torch.empty((n, 8), dtype=self.torch.float32, device=ix.device)
        self._check(lib().stf_neural_decode(self.h, net, n, _ptr(ix), _ptr(iy), _ptr(y)), self.h)
        return y

    def neural_filter_shade(self, net: int, u, v, derivs=None, filter: str = "bspline", mode: str = "stochastic",
                            shade: str = "ggx", spp: int = 1, seed: int = 1, id_base: int = 0, out=None):
        torch = self.torch
        n = int(u.shape[0])
        if out is None:
            out = [torch.empty(n, dtype=torch.float32, device=u.device) for _ in range(3)]
        q, d, o = self._args(u, v, derivs, out, None, n, id_base)
        st = lib().stf_neural_filter_shade(self.h, net, C.byref(q), C.byref(d) if d is not None else None,
                                           FILTERS[filter], MODES[mode], SHADES[shade], spp, seed, 0, C.byref(o))
        self._check(st, self.h)
        return out[0], out[1], out[2]

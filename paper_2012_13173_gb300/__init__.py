"""Python binding of libhcgrid.so, the GB300 gridding library.

Argument marshalling only: every step of the gridding path runs in the
library's CUDA kernels (see ``include/hcgrid.h``).  PyTorch supplies device
memory and streams.  The binding raises ``HcgError`` when the library is
missing or a call fails; there is no fallback implementation.

    g = Gridder()
    g.set_kernel(fwhm_deg, support_deg)
    g.set_grid(lon0, lat0, pixel_deg, nx, ny)
    g.load_samples(lon, lat, spectra)        # numpy or torch (host or cuda)
    g.grid()
    cube, weights = g.fetch()                # cube [ny, nx, nchan], weights [ny, nx]
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhcgrid.so")

HCG_OK = 0
CAR = 0
WCS_TAN, WCS_SIN, WCS_SFL, WCS_CAR, CELL_LIST = 1, 2, 3, 4, 5
F32, BF16, E4M3 = 0, 1, 2
MEM_HOST, MEM_DEVICE, MEM_DEVICE_BORROW, MEM_HOST_STREAM = 0, 1, 2, 3
PATH_AUTO, PATH_GATHER, PATH_TENSOR, PATH_SCATTER, PATH_STAGED = 0, 1, 2, 3, 4
_STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NOT_READY", -5: "TIMEOUT", -6: "STATE",
           -7: "UNSUPPORTED"}
_DT = {"f32": F32, "bf16": BF16, "e4m3": E4M3, F32: F32, BF16: BF16, E4M3: E4M3}

_lib = None


class HcgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Info(ctypes.Structure):
    _fields_ = [("nside", ctypes.c_int64), ("ring_lo", ctypes.c_int64), ("ring_hi", ctypes.c_int64),
                ("samples_kept", ctypes.c_int64), ("unique_pixels", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("contributions", ctypes.c_int64), ("path", ctypes.c_int32), ("key_bits", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("stream_window", ctypes.c_int32),
                ("tensor_flops", ctypes.c_int64)]


_SIGS = {
    "hcg_create": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hcg_destroy": [ctypes.c_void_p],
    "hcg_set_stream": [ctypes.c_void_p, ctypes.c_void_p],
    "hcg_set_kernel": [ctypes.c_void_p, ctypes.c_double, ctypes.c_double],
    "hcg_set_grid": [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                     ctypes.c_int32, ctypes.c_int32],
    "hcg_set_storage": [ctypes.c_void_p, ctypes.c_int],
    "hcg_set_cell_list": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int],
    "hcg_load_samples": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                         ctypes.c_int32, ctypes.c_int, ctypes.c_void_p, ctypes.c_int],
    "hcg_bind_output": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "hcg_grid": [ctypes.c_void_p],
    "hcg_sync": [ctypes.c_void_p],
    "hcg_fetch": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "hcg_get_info": [ctypes.c_void_p, ctypes.c_void_p],
    "hcg_set_tuning": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "hcg_set_stream_chunk": [ctypes.c_void_p, ctypes.c_int32],
    "hcg_bind_host_output": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "hcg_autotune": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hcg_autotune_table": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p],
    "hcg_set_profiling": [ctypes.c_void_p, ctypes.c_int],
    "hcg_stage_times": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32],
    "hcg_debug_pix": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p],
    "hcg_debug_lut": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                      ctypes.c_void_p, ctypes.c_int64],
    "hcg_debug_neighbours": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_int64],
    "hcg_batch_create": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "hcg_batch_destroy": [ctypes.c_void_p],
    "hcg_batch_add": [ctypes.c_void_p, ctypes.c_void_p],
    "hcg_batch_grid": [ctypes.c_void_p],
    "hcg_batch_sync": [ctypes.c_void_p],
    "hcg_batch_info": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "hcg_measure_fp32_peak": [ctypes.c_int, ctypes.c_void_p],
    "hcg_set_wait_limit": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int],
    "hcg_set_alloc_cap": [ctypes.c_void_p, ctypes.c_int64],
    "hcg_preorder_noalloc": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
}


def load(build_if_stale: bool = True) -> ctypes.CDLL:
    """Load libhcgrid.so (building it first when the sources are newer and
    nvcc is available).  Raises HcgError if the library cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale:
        try:
            from . import build as _b
            _b.build()
        except RuntimeError as e:
            if not os.path.exists(LIB_PATH):
                raise HcgError(-3, f"libhcgrid.so missing and cannot be built: {e}") from e
    if not os.path.exists(LIB_PATH):
        raise HcgError(-3, f"libhcgrid.so not found at {LIB_PATH}; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int32
    lib.hcg_last_error.argtypes = []
    lib.hcg_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != HCG_OK:
        raise HcgError(status, _lib.hcg_last_error().decode())


def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:
        return False


def _ptr(x):
    if x is None:
        return None, None
    if _is_torch(x):
        return x.data_ptr(), x.is_cuda
    return x.ctypes.data, False


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Gridder:
    """One gridding context (``hcg_ctx``) bound to a CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        load()
        self._h = ctypes.c_void_p()
        self._keep = []
        _check(_lib.hcg_create(ctypes.byref(self._h), device, _stream_handle(stream)))
        self.device = device
        self.nx = self.ny = self.nchan = 0

    def close(self):
        if self._h:
            _lib.hcg_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        _check(_lib.hcg_set_stream(self._h, _stream_handle(stream)))

    def set_kernel(self, fwhm_deg: float, support_deg: float):
        _check(_lib.hcg_set_kernel(self._h, float(fwhm_deg), float(support_deg)))

    def set_grid(self, lon0, lat0, pixel, nx, ny, projection=CAR):
        _check(_lib.hcg_set_grid(self._h, projection, float(lon0), float(lat0), float(pixel), int(nx), int(ny)))
        self.nx, self.ny = int(nx), int(ny)

    def set_cell_list(self, lon, lat):
        """Target cells as a free list of centres (FP64 [n] each, host or
        device): the result is cube [n, 1, nchan], weights [n, 1]."""
        if not _is_torch(lon):
            lon = np.ascontiguousarray(lon, np.float64)
            lat = np.ascontiguousarray(lat, np.float64)
        n = int(lon.shape[0])
        lp, lcuda = _ptr(lon)
        bp, bcuda = _ptr(lat)
        if lcuda != bcuda:
            raise HcgError(-1, "lon and lat must both be host or both be device memory")
        _check(_lib.hcg_set_cell_list(self._h, lp, bp, n, MEM_DEVICE if lcuda else MEM_HOST))
        self.nx, self.ny = n, 1

    def set_storage(self, dtype):
        _check(_lib.hcg_set_storage(self._h, _DT[dtype]))

    def set_tuning(self, cells_per_block=0, chans_per_thread=0, tile_depth=0, path=PATH_AUTO):
        _check(_lib.hcg_set_tuning(self._h, cells_per_block, chans_per_thread, tile_depth, path))

    def set_stream_chunk(self, chans=0):
        """Channels per streamed window (0: automatic); see load_samples(stream=True)."""
        _check(_lib.hcg_set_stream_chunk(self._h, int(chans)))

    def load_samples(self, lon, lat, spectra, dtype=None, chan_scale=None, borrow=False, stream=False):
        """lon/lat: FP64 [n]; spectra [n, nchan] (FP32, BF16 as torch.bfloat16 /
        uint16 bits, E4M3 as torch.float8_e4m3fn / uint8 codes).  borrow: use
        device inputs in place.  stream: keep host spectra on the host and copy
        them window by window of channels inside each grid() (the inputs are
        kept referenced here until the next load_samples)."""
        if not _is_torch(lon):
            lon = np.ascontiguousarray(lon, np.float64)
            lat = np.ascontiguousarray(lat, np.float64)
        n = int(lon.shape[0])
        sp = spectra if _is_torch(spectra) else np.ascontiguousarray(spectra)
        if dtype is None:
            dtype = F32
            if _is_torch(sp):
                import torch
                if sp.dtype == torch.bfloat16:
                    dtype = BF16
                elif sp.dtype == torch.float8_e4m3fn:
                    dtype = E4M3
        dtype = _DT[dtype]
        nchan = int(sp.shape[1]) if len(sp.shape) > 1 else 1
        lp, lcuda = _ptr(lon)
        bp, _ = _ptr(lat)
        spp, scuda = _ptr(sp)
        cp, _ = _ptr(chan_scale)
        if lcuda != scuda:
            raise HcgError(-1, "coordinates and spectra must both be host or both be device memory")
        if stream and lcuda:
            raise HcgError(-1, "stream=True streams host spectra; these are device tensors")
        if _is_torch(sp) and not sp.is_contiguous():
            raise HcgError(-1, "spectra must be contiguous [n, nchan]")
        if lcuda:
            mem = MEM_DEVICE_BORROW if borrow else MEM_DEVICE
        else:
            mem = MEM_HOST_STREAM if stream else MEM_HOST
        _check(_lib.hcg_load_samples(self._h, lp, bp, spp, n, nchan, dtype, cp, mem))
        self._keep = [lon, lat, sp, chan_scale] if (borrow or not lcuda) else []
        self.nchan = nchan
        self.n = n

    def bind_host_output(self, cube, weights):
        """Host (pinned) cube [ny, nx, nchan] and weights [ny, nx] FP32 that every
        grid() also fills, window by window when the spectra are streamed;
        sync() waits for the copies.  None, None stops the delivery."""
        cp, _ = _ptr(cube)
        wp, _ = _ptr(weights)
        _check(_lib.hcg_bind_host_output(self._h, cp, wp))
        self._host_out = (cube, weights)

    def bind_output(self, cube, weights):
        cp, _ = _ptr(cube)
        wp, _ = _ptr(weights)
        _check(_lib.hcg_bind_output(self._h, cp, wp))
        self._out = (cube, weights)

    def grid(self):
        _check(_lib.hcg_grid(self._h))

    def sync(self):
        _check(_lib.hcg_sync(self._h))

    def fetch(self, cube=None, weights=None):
        """Copy the result out.  With no arguments returns numpy arrays."""
        if cube is None and weights is None:
            cube = np.empty((self.ny, self.nx, self.nchan), np.float32)
            weights = np.empty((self.ny, self.nx), np.float32)
        cp, ccuda = _ptr(cube)
        wp, _ = _ptr(weights)
        _check(_lib.hcg_fetch(self._h, cp, wp, MEM_DEVICE if ccuda else MEM_HOST))
        return cube, weights

    def autotune(self, force=False):
        """Time the applicable tunings and paths on the loaded field; keep the
        fastest.  Returns it as hcg_set_tuning takes it."""
        ch = (ctypes.c_int32 * 4)()
        _check(_lib.hcg_autotune(self._h, 1 if force else 0, ch))
        return {"cells_per_block": ch[0], "chans_per_thread": ch[1], "tile_depth": ch[2], "path": ch[3]}

    def autotune_table(self):
        """The candidates the last timing autotune measured: a list of
        ((cells_per_block, chans_per_thread, tile_depth, path), ms)."""
        cnt = ctypes.c_int32()
        _lib.hcg_autotune_table(self._h, None, None, 0, ctypes.byref(cnt))
        n = cnt.value
        ch = (ctypes.c_int32 * max(4 * n, 1))()
        ms = (ctypes.c_float * max(n, 1))()
        _check(_lib.hcg_autotune_table(self._h, ch, ms, n, ctypes.byref(cnt)))
        return [(tuple(ch[4 * k:4 * k + 4]), ms[k]) for k in range(n)]

    def set_alloc_cap(self, nbytes=0):
        """Cap the field-sized device buffers this Gridder may hold (bytes,
        0 = no cap): beyond it calls fail with OOM and the Gridder stays
        usable."""
        _check(_lib.hcg_set_alloc_cap(self._h, int(nbytes)))

    def set_wait_limit(self, limit_ns=4_000_000_000, probe=False):
        """Give-up limit of the tensor path's bounded device waits (ns); with
        probe=True every tensor-path CTA first waits on a barrier nothing
        completes, so the pass returns TIMEOUT (a check of that path)."""
        _check(_lib.hcg_set_wait_limit(self._h, int(limit_ns), 1 if probe else 0))

    def set_profiling(self, enable=True):
        _check(_lib.hcg_set_profiling(self._h, 1 if enable else 0))

    STAGES = ("ingest", "pixel_keys", "sort", "tables", "gather")

    def stage_times(self) -> dict:
        ms = (ctypes.c_double * 5)()
        _check(_lib.hcg_stage_times(self._h, ms, 5))
        return dict(zip(self.STAGES, list(ms)))

    def info(self) -> dict:
        inf = Info()
        _check(_lib.hcg_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    def debug_pix(self):
        inf = self.info()
        m = inf["samples_kept"]
        pix = np.empty(max(m, 1), np.int64)
        perm = np.empty(max(m, 1), np.uint32)
        mo = ctypes.c_int64()
        _check(_lib.hcg_debug_pix(self._h, pix.ctypes.data, perm.ctypes.data, max(m, 1), ctypes.byref(mo)))
        return pix[:m], perm[:m].astype(np.int64)

    def debug_lut(self):
        inf = self.info()
        u = inf["unique_pixels"]
        nr = inf["ring_hi"] - inf["ring_lo"] + 2
        upix = np.empty(max(u, 1), np.int64)
        ust = np.empty(max(u, 1) + 1, np.int64)
        rst = np.empty(nr, np.int64)
        uo = ctypes.c_int64()
        _check(_lib.hcg_debug_lut(self._h, upix.ctypes.data, ust.ctypes.data, max(u, 1), ctypes.byref(uo),
                                  rst.ctypes.data, nr))
        return upix[:u], ust[:u + 1], rst

    def debug_neighbours(self, cell_begin=0, cell_end=None, cap=None):
        cell_end = self.nx * self.ny if cell_end is None else cell_end
        m = cell_end - cell_begin
        off = np.empty(m + 1, np.int64)
        cap = cap if cap is not None else max(1, self.info()["pairs"])
        ids = np.empty(cap, np.uint32)
        _check(_lib.hcg_debug_neighbours(self._h, cell_begin, cell_end, off.ctypes.data, ids.ctypes.data, cap))
        return off, ids[:off[-1]].astype(np.int64)


def measure_fp32_peak(device: int = 0) -> float:
    """The device's measured FP32 FMA throughput, TFLOP/s (hcg_measure_fp32_peak)."""
    load()
    t = ctypes.c_double()
    _check(_lib.hcg_measure_fp32_peak(int(device), ctypes.byref(t)))
    return t.value


def _check_noalloc_args(lon, lat, pix_sorted, perm):
    """Shapes, types and placement of hcg_preorder_noalloc's tensors, checked
    before the call: the library writes n values to each output, so a short
    or strided tensor would be overrun on the device."""
    import torch
    n = int(lon.shape[0]) if lon.dim() == 1 else -1
    if n < 0:
        raise HcgError(-1, "lon must be a 1-D tensor")
    want = ((lon, "lon", (torch.float64,)), (lat, "lat", (torch.float64,)),
            (pix_sorted, "pix_sorted", (torch.int64,)), (perm, "perm", (torch.int32, torch.uint32)))
    for t, name, dts in want:
        if not _is_torch(t):
            raise HcgError(-1, f"{name} must be a torch tensor")
        if t.dtype not in dts:
            raise HcgError(-1, f"{name} must have dtype {' or '.join(str(d) for d in dts)}, not {t.dtype}")
        if t.numel() < n:
            raise HcgError(-1, f"{name} holds {t.numel()} elements, fewer than n = {n}")
        if not t.is_contiguous():
            raise HcgError(-1, f"{name} must be contiguous")
    for t, name, _ in want:
        if not t.is_cuda or t.device != lon.device:
            raise HcgError(-1, f"{name} must be a CUDA tensor on {lon.device}")
    return n


def preorder_noalloc(lon, lat, nside, ring_lo, ring_hi, pix_sorted, perm, stream=None):
    """hcg_preorder_noalloc on device tensors (lon/lat float64 [n], pix_sorted
    int64 [>= n], perm int32/uint32 [>= n], all contiguous CUDA tensors on
    one device); enqueue only."""
    n = _check_noalloc_args(lon, lat, pix_sorted, perm)
    load()
    _check(_lib.hcg_preorder_noalloc(lon.data_ptr(), lat.data_ptr(), n, int(nside), int(ring_lo), int(ring_hi),
                                     pix_sorted.data_ptr(), perm.data_ptr(), _stream_handle(stream)))


class Batch:
    """Several Gridder fields gridded together (``hcg_batch``)."""

    def __init__(self, device: int = 0, stream=None):
        load()
        self._h = ctypes.c_void_p()
        _check(_lib.hcg_batch_create(ctypes.byref(self._h), device, _stream_handle(stream)))
        self.fields = []

    def add(self, g: Gridder):
        _check(_lib.hcg_batch_add(self._h, g.handle))
        self.fields.append(g)

    def grid(self):
        _check(_lib.hcg_batch_grid(self._h))

    def sync(self):
        _check(_lib.hcg_batch_sync(self._h))

    def info(self) -> dict:
        items = ctypes.c_int64()
        launches = ctypes.c_int32()
        _check(_lib.hcg_batch_info(self._h, ctypes.byref(items), ctypes.byref(launches)))
        return {"work_items": items.value, "launches": launches.value}

    def close(self):
        if self._h:
            _lib.hcg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""FP64 CPU oracle for HCGrid gridding (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference`` arm) may import this package.
It shares no code with the CUDA library: the C part (``hcg_oracle.c``) is a
plain restatement of the paper's definitions, and ``quant`` holds the plain
definitions of the storage roundings.  See ``hcg_oracle.c`` for the passages
each function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hcg_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP contraction off, OpenMP when available)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", _OUT + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_OUT + ".tmp", _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        i64, dbl, u32 = ctypes.c_int64, ctypes.c_double, ctypes.c_uint32
        P = ctypes.c_void_p
        sig = {
            "orc_npix": (i64, [i64]),
            "orc_ring_npix": (i64, [i64, i64]),
            "orc_ring_start": (i64, [i64, i64]),
            "orc_pix2ring": (i64, [i64, i64]),
            "orc_ang2pix": (i64, [i64, dbl, dbl, P]),
            "orc_pix2ang": (None, [i64, i64, P, P]),
            "orc_hR": (dbl, [dbl]),
            "orc_neigh_brute": (None, [P, i64, P, P, P, P, P, P, dbl]),
            "orc_neigh_band": (None, [P, i64, P, P, i64, P, P, P, P, P, dbl]),
            "orc_grid_cells": (None, [P, i64, P, P, P, i64, i64, P, P, P, P, P]),
            "orc_neigh_brute_xy": (None, [P, P, P, i64, P, P, P, P, P, P, dbl]),
            "orc_neigh_band_xy": (None, [P, P, P, i64, P, P, i64, P, P, P, P, P, dbl]),
            "orc_grid_cells_xy": (None, [P, P, P, i64, P, P, P, i64, i64, P, P, P, P, P]),
            "orc_wcs_cells": (i64, [ctypes.c_int, dbl, dbl, dbl, i64, i64, P, P]),
            "orc_coord_hash": (u32, [dbl, dbl]),
            "orc_preorder": (i64, [i64, i64, P, P, i64, i64, P, P]),
            "orc_lut1": (i64, [i64, P, P, P]),
            "orc_lut2": (None, [i64, i64, P, i64, i64, P]),
            "orc_nside_for": (i64, [dbl]),
            "orc_num_threads": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


# ---------------------------------------------------------------- HEALPix ---
def npix(nside: int) -> int:
    return lib().orc_npix(nside)


def ring_npix(nside: int, r: int) -> int:
    return lib().orc_ring_npix(nside, r)


def ring_start(nside: int, r: int) -> int:
    return lib().orc_ring_start(nside, r)


def pix2ring(nside: int, pix: int) -> int:
    return lib().orc_pix2ring(nside, pix)


def ang2pix(nside: int, lon_deg, lat_deg):
    """RING pixel and ring of each (lon, lat) in degrees (Sec. 3.3 step I)."""
    lon = _f64(np.atleast_1d(lon_deg)); lat = _f64(np.atleast_1d(lat_deg))
    pix = np.empty(lon.size, np.int64); ring = np.empty(lon.size, np.int64)
    r = ctypes.c_int64()
    f = lib().orc_ang2pix
    for k in range(lon.size):
        pix[k] = f(nside, float(lon[k]), float(lat[k]), ctypes.byref(r))
        ring[k] = r.value
    return pix, ring


def pix2ang(nside: int, pix):
    pix = np.atleast_1d(np.asarray(pix, np.int64))
    lon = np.empty(pix.size); lat = np.empty(pix.size)
    a, b = ctypes.c_double(), ctypes.c_double()
    f = lib().orc_pix2ang
    for k in range(pix.size):
        f(nside, int(pix[k]), ctypes.byref(a), ctypes.byref(b))
        lon[k] = a.value; lat[k] = b.value
    return lon, lat


def nside_for(fwhm_deg: float) -> int:
    return lib().orc_nside_for(float(fwhm_deg))


def coord_hash(lon, lat) -> np.ndarray:
    lon = _f64(np.atleast_1d(lon)); lat = _f64(np.atleast_1d(lat))
    f = lib().orc_coord_hash
    return np.array([f(float(a), float(b)) for a, b in zip(lon, lat)], np.uint32)


# ------------------------------------------------------- pre-ordering + LUT ---
def preorder(nside: int, lon, lat, r_lo: int, r_hi: int):
    """Sorted pixels P' and permutation (sample ids of S') of the samples whose
    ring lies in [r_lo, r_hi] (Sec. 3.3 step I)."""
    lon = _f64(lon); lat = _f64(lat)
    n = lon.size
    ps = np.empty(max(n, 1), np.int64); pm = np.empty(max(n, 1), np.int64)
    m = lib().orc_preorder(nside, n, _p(lon), _p(lat), r_lo, r_hi, _p(ps), _p(pm))
    return ps[:m].copy(), pm[:m].copy()


def lut1(pix_sorted):
    """First-level table (Sec. 3.3 step II): distinct pixels and their S_start."""
    ps = _i64(pix_sorted)
    m = ps.size
    up = np.empty(max(m, 1), np.int64); us = np.empty(m + 1, np.int64)
    u = lib().orc_lut1(m, _p(ps), _p(up), _p(us))
    return up[:u].copy(), us[:u + 1].copy()


def lut2(nside: int, pix_sorted, r_lo: int, r_hi: int):
    """Second-level table (Sec. 3.3 step III): R_start for rings r_lo..r_hi+1."""
    ps = _i64(pix_sorted)
    out = np.empty(r_hi + 2 - r_lo, np.int64)
    lib().orc_lut2(nside, ps.size, _p(ps), r_lo, r_hi, _p(out))
    return out


# ------------------------------------------------------------- gridding ---
def geom_array(lon0, lat0, pix, nx, ny, R, fwhm):
    return np.array([lon0, lat0, pix, nx, ny, R, fwhm], np.float64)


def hR(R_deg: float) -> float:
    return lib().orc_hR(float(R_deg))


WCS_TAN, WCS_SIN, WCS_SFL, WCS_CAR = 1, 2, 3, 4


def wcs_cells(proj, lon0, lat0, pix, nx, ny):
    """Cell centres (lon, lat) in degrees, [ny * nx] row-major, of a grid in
    projection proj (WCS_TAN / WCS_SIN / WCS_SFL / WCS_CAR) with the
    reference point (lon0, lat0) at the grid centre and cells of pix degrees
    (Calabretta & Greisen 2002); NaN where the projection has no point."""
    clon = np.empty(int(nx) * int(ny)); clat = np.empty(int(nx) * int(ny))
    lib().orc_wcs_cells(int(proj), float(lon0), float(lat0), float(pix), int(nx), int(ny), _p(clon), _p(clat))
    return clon, clat


def _xy(cell_lon, cell_lat):
    if cell_lon is None:
        return None, None, None
    clon = _f64(cell_lon); clat = _f64(cell_lat)
    return clon, clat, (_p(clon), _p(clat))


def neighbours_brute(geom, lon, lat, gtol: float = 1e-13, cell_lon=None, cell_lat=None):
    """CSR contributor lists of every cell by brute force (Sec. 3.4 reference);
    cell_lon/cell_lat: explicit cell centres (default: the plain lon/lat grid)."""
    geom = _f64(geom); lon = _f64(lon); lat = _f64(lat)
    clon, clat, xy = _xy(cell_lon, cell_lat)
    xy = xy or (None, None)
    cells = int(geom[3]) * int(geom[4])
    cnt = np.zeros(cells, np.int64); guard = np.zeros(cells, np.int64)
    lib().orc_neigh_brute_xy(_p(geom), *xy, lon.size, _p(lon), _p(lat), _p(cnt), None, None, _p(guard), gtol)
    off = np.zeros(cells + 1, np.int64); off[1:] = np.cumsum(cnt)
    ids = np.empty(max(int(off[-1]), 1), np.int64)
    lib().orc_neigh_brute_xy(_p(geom), *xy, lon.size, _p(lon), _p(lat), _p(cnt), _p(off), _p(ids), None, gtol)
    return off, ids[:off[-1]], guard


def neighbours_band(geom, lon, lat, cells=None, gtol: float = 1e-13, cell_lon=None, cell_lat=None):
    """CSR contributor lists (sorted ids) via the sorted-latitude band search."""
    geom = _f64(geom); lon = _f64(lon); lat = _f64(lat)
    clon, clat, xy = _xy(cell_lon, cell_lat)
    xy = xy or (None, None)
    if cells is None:
        cells = np.arange(int(geom[3]) * int(geom[4]), dtype=np.int64)
    cells = _i64(cells)
    cnt = np.zeros(cells.size, np.int64); guard = np.zeros(cells.size, np.int64)
    L = lib()
    L.orc_neigh_band_xy(_p(geom), *xy, lon.size, _p(lon), _p(lat), cells.size, _p(cells), _p(cnt), None, None,
                        _p(guard), gtol)
    off = np.zeros(cells.size + 1, np.int64); off[1:] = np.cumsum(cnt)
    ids = np.empty(max(int(off[-1]), 1), np.int64)
    L.orc_neigh_band_xy(_p(geom), *xy, lon.size, _p(lon), _p(lat), cells.size, _p(cells), _p(cnt), _p(off), _p(ids),
                        None, gtol)
    return off, ids[:off[-1]], guard


def grid_cells(geom, lon, lat, spectra, cells=None, cell_lon=None, cell_lat=None):
    """Eq. (1) in FP64 for the given cells (default: all); cell_lon/cell_lat:
    explicit cell centres (default: the plain lon/lat grid).

    Returns (V[ncell, C], W[ncell], absscale[ncell, C], count[ncell]) where
    absscale = sum_n w |s_n| / W is the scale of the condition-aware tolerance.
    """
    clon, clat, xy = _xy(cell_lon, cell_lat)
    xy = xy or (None, None)
    geom = _f64(geom); lon = _f64(lon); lat = _f64(lat)
    spec = _f64(spectra)
    if spec.ndim == 1:
        spec = spec.reshape(-1, 1)
    nchan = spec.shape[1]
    if cells is None:
        cells = np.arange(int(geom[3]) * int(geom[4]), dtype=np.int64)
    cells = _i64(cells)
    v = np.empty((cells.size, nchan)); w = np.empty(cells.size)
    ab = np.empty((cells.size, nchan)); cnt = np.empty(cells.size, np.int64)
    lib().orc_grid_cells_xy(_p(geom), *xy, lon.size, _p(lon), _p(lat), _p(spec), nchan, cells.size,
                            _p(cells), _p(v), _p(w), _p(ab), _p(cnt))
    return v, w, ab, cnt


def num_threads() -> int:
    return lib().orc_num_threads()

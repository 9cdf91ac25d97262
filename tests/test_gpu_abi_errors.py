"""Argument errors through the C ABI itself (ctypes, no binding logic in
between): every check that include/hcgrid.h documents returns its status
code before any device work, hcg_last_error names the problem, and the
context stays usable (a valid pass afterwards gives the oracle's result)."""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
OK, INVALID, NOT_READY = 0, -1, -4
F32, BF16, E4M3 = 0, 1, 2
MEM_HOST, MEM_DEVICE, MEM_DEVICE_BORROW = 0, 1, 2
AM = 1.0 / 60.0
FWHM, SUPPORT = 1.5 * AM, 3.0 * 1.5 * AM / 2.3548200450309493


@pytest.fixture
def abi(hcg):
    lib = hcg.load()
    p = ctypes.c_void_p()
    assert lib.hcg_create(ctypes.byref(p), 0, None) == OK
    yield lib, p
    assert lib.hcg_destroy(p) == OK


def _err(lib, status, want=INVALID):
    assert status == want
    assert lib.hcg_last_error()


def test_create_and_null_context(hcg):
    lib = hcg.load()
    p = ctypes.c_void_p()
    for dev in (-1, 4096):
        _err(lib, lib.hcg_create(ctypes.byref(p), dev, None))
    _err(lib, lib.hcg_create(None, 0, None))
    assert lib.hcg_destroy(None) == OK
    _err(lib, lib.hcg_set_kernel(None, FWHM, SUPPORT))
    _err(lib, lib.hcg_grid(None))


def test_kernel_arguments(abi):
    lib, c = abi
    for fwhm, sup in [(0.0, 0.01), (-1.0, 0.01), (FWHM, 0.0), (math.nan, 0.01), (FWHM, math.inf),
                      (0.5, 1.5),                 # support above 1 degree
                      (FWHM, 0.2),                # support above 10 sigma
                      (1e-4, 1e-4)]:              # fwhm below 1 arcsec
        _err(lib, lib.hcg_set_kernel(c, fwhm, sup))
    assert lib.hcg_set_kernel(c, FWHM, SUPPORT) == OK


def test_grid_arguments(abi):
    lib, c = abi
    for proj, lon0, lat0, pix, nx, ny in [(-1, 180.0, 30.0, AM, 20, 20), (5, 180.0, 30.0, AM, 20, 20),
                                          (0, 180.0, 30.0, AM, 0, 20), (0, 180.0, 30.0, AM, 20, -3),
                                          (0, 180.0, 30.0, 0.0, 20, 20), (0, 180.0, 30.0, -AM, 20, 20),
                                          (0, 180.0, 30.0, math.nan, 20, 20), (0, math.inf, 30.0, AM, 20, 20),
                                          (0, 180.0, 30.0, 0.2, 1000, 10),      # wider than 180 degrees
                                          (0, 180.0, 88.9, 0.1, 10, 21)]:      # cells beyond 89 degrees
        _err(lib, lib.hcg_set_grid(c, proj, lon0, lat0, pix, nx, ny))
    assert lib.hcg_set_grid(c, 0, 180.0, 30.0, AM, 20, 20) == OK


def test_storage_and_load_arguments(abi):
    lib, c = abi
    for dt in (-1, 3):
        _err(lib, lib.hcg_set_storage(c, dt))
    buf = np.zeros(64, np.float64)
    p = buf.ctypes.data
    # n < 0, nchan < 1, n above 2^32 - 1, unknown dtype, null pointers, E4M3 without
    # scales, unknown memory kind, BF16 input for F32 storage, n * nchan overflow
    for n, nchan, dt, ptr, scale, mem in [(-1, 1, F32, p, None, MEM_HOST), (4, 0, F32, p, None, MEM_HOST),
                                          (1 << 32, 1, F32, p, None, MEM_HOST), (4, 1, 7, p, None, MEM_HOST),
                                          (4, 1, F32, None, None, MEM_HOST), (4, 1, E4M3, p, None, MEM_HOST),
                                          (4, 1, F32, p, None, 9), (4, 1, BF16, p, None, MEM_HOST),
                                          ((1 << 31), (1 << 31) - 1, F32, p, None, MEM_HOST)]:
        _err(lib, lib.hcg_load_samples(c, ptr, ptr, ptr, n, nchan, dt, scale, mem))


def test_tuning_and_state(abi):
    lib, c = abi
    _err(lib, lib.hcg_grid(c), NOT_READY)
    # values outside each path's lists, and combinations a path does not have
    for cells, chans, depth, path in [(0, 9, 0, 0), (0, -1, 0, 0), (0, 0, 0, 5), (-1, 0, 0, 0), (0, 0, -2, 0),
                                      (8, 0, 0, 0), (24, 0, 0, 1), (16, 8, 12, 1), (32, 1, 0, 1), (0, 4, 12, 1),
                                      (64, 8, 0, 4), (48, 0, 0, 4), (0, 0, 24, 4), (128, 4, 0, 2), (64, 0, 0, 2),
                                      (0, 0, 32, 2), (0, 0, 16, 3)]:
        _err(lib, lib.hcg_set_tuning(c, cells, chans, depth, path))
    for cells, chans, depth, path in [(0, 0, 0, 0), (16, 1, 0, 1), (32, 4, 8, 1), (32, 8, 12, 1), (64, 4, 32, 4),
                                      (32, 0, 16, 4), (128, 0, 64, 2), (0, 0, 0, 3)]:
        assert lib.hcg_set_tuning(c, cells, chans, depth, path) == OK
    assert lib.hcg_set_tuning(c, 0, 0, 0, 0) == OK
    for limit in (0, 999, 60_000_000_001):
        _err(lib, lib.hcg_set_wait_limit(c, limit, 0))
    _err(lib, lib.hcg_set_stream_chunk(c, -1))
    _err(lib, lib.hcg_bind_output(c, 16, None))


def test_context_usable_after_errors(abi):
    """After a run of refused calls the same context grids a small field, and
    the result matches the FP64 oracle."""
    lib, c = abi
    _err(lib, lib.hcg_set_kernel(c, -1.0, 0.0))
    _err(lib, lib.hcg_set_grid(c, 9, 0.0, 0.0, AM, 1, 1))
    rng = np.random.default_rng(3)
    n, nchan, nx, ny = 400, 3, 9, 7
    lon = 180.0 + rng.uniform(-6, 6, n) * AM
    lat = 30.0 + rng.uniform(-5, 5, n) * AM
    spec = rng.standard_normal((n, nchan)).astype(np.float32)
    assert lib.hcg_set_kernel(c, FWHM, SUPPORT) == OK
    assert lib.hcg_set_grid(c, 0, 180.0, 30.0, AM, nx, ny) == OK
    _err(lib, lib.hcg_load_samples(c, lon.ctypes.data, lat.ctypes.data, spec.ctypes.data, n, 0, F32, None,
                                   MEM_HOST))
    assert lib.hcg_load_samples(c, lon.ctypes.data, lat.ctypes.data, spec.ctypes.data, n, nchan, F32, None,
                                MEM_HOST) == OK
    assert lib.hcg_grid(c) == OK
    cube = np.empty((ny, nx, nchan), np.float32)
    w = np.empty((ny, nx), np.float32)
    assert lib.hcg_fetch(c, cube.ctypes.data, w.ctypes.data, MEM_HOST) == OK
    v, wr, ab, cnt = oracle.grid_cells((180.0, 30.0, AM, nx, ny, SUPPORT, FWHM), lon, lat, spec)
    ok = cnt > 0
    got = cube.reshape(nx * ny, nchan)
    assert ok.any() and np.all(np.isnan(got[~ok]))
    assert (np.abs(got[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])).max() <= 1e-5


def test_host_pointers_refused_as_device_memory(abi):
    """Host addresses passed where device memory is declared are refused
    before any kernel could dereference them."""
    lib, c = abi
    n, nchan = 16, 4
    lon = np.zeros(n); lat = np.zeros(n)
    spec = np.zeros((n, nchan), np.float32)
    for mem in (MEM_DEVICE, MEM_DEVICE_BORROW):
        _err(lib, lib.hcg_load_samples(c, lon.ctypes.data, lat.ctypes.data, spec.ctypes.data, n, nchan, F32, None,
                                       mem))
    dev = torch.zeros(n, dtype=torch.float64, device="cuda")
    dspec = torch.zeros((n, nchan), device="cuda")
    _err(lib, lib.hcg_load_samples(c, dev.data_ptr(), lat.ctypes.data, dspec.data_ptr(), n, nchan, F32, None,
                                   MEM_DEVICE_BORROW))
    cube = np.zeros(64, np.float32)
    _err(lib, lib.hcg_bind_output(c, cube.ctypes.data, cube.ctypes.data))
    out_p = np.zeros(n, np.int64)
    out_v = np.zeros(n, np.uint32)
    _err(lib, lib.hcg_preorder_noalloc(dev.data_ptr(), dev.data_ptr(), n, 16384, 1000, 2000, out_p.ctypes.data,
                                       out_v.ctypes.data, None))
    # the same buffers on the device are accepted
    assert lib.hcg_load_samples(c, dev.data_ptr(), dev.data_ptr(), dspec.data_ptr(), n, nchan, F32, None,
                                MEM_DEVICE_BORROW) == OK


def test_allocation_cap_gives_oom_and_the_context_recovers(hcg):
    """hcg_set_alloc_cap: host-side out-of-memory without filling the GPU.  A
    cap below the copied spectra fails hcg_load_samples with OOM, a cap that
    holds the inputs but not a pass's scratch fails hcg_grid with OOM, and
    with the cap lifted the same context grids the field to the bit of a
    context that never met the cap."""
    from paper_2012_13173_gb300 import synth
    f = synth.uniform_field(seed=61, n=20000, width=0.5, height=0.5, nx=24, ny=20, nchan=64)
    lon = torch.from_numpy(f.lon).cuda()
    lat = torch.from_numpy(f.lat).cuda()
    spec = f.spectra(device="cuda")
    inputs = f.n * f.nchan * 4 + 2 * f.n * 8              # copied spectra and coordinates

    ref = hcg.Gridder(0)
    ref.set_kernel(f.fwhm, f.support)
    ref.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    ref.load_samples(lon, lat, spec)
    ref.grid()
    cube_ref, w_ref = ref.fetch()

    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    with pytest.raises(hcg.HcgError, match="INVALID_ARG"):
        g.set_alloc_cap(-1)
    g.set_alloc_cap(inputs // 2)
    with pytest.raises(hcg.HcgError, match="OOM"):
        g.load_samples(lon, lat, spec)
    g.set_alloc_cap(inputs + 4096)
    g.load_samples(lon, lat, spec)
    with pytest.raises(hcg.HcgError, match="OOM"):
        g.grid()
    g.set_alloc_cap(0)
    g.grid()
    cube, w = g.fetch()
    assert np.array_equal(w, w_ref)
    assert np.array_equal(np.isnan(cube), np.isnan(cube_ref))
    ok = ~np.isnan(cube_ref)
    assert np.array_equal(cube[ok], cube_ref[ok])

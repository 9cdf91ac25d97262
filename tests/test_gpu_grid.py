"""GPU parity of Eq. (1) (values and weights) against the FP64 oracle,
through the C ABI, on seeded synthetic fields, ragged shapes and edge cases.

Tolerance (condition-aware, per value): |V_gpu - V_64| <= tol * (|V_64| +
sum_n w_n |s_n| / W), tol = 1e-5 for FP32 storage; weights W to 1e-5
relative.  BF16 / E4M3 storage: 1e-5 against the oracle on the dequantised
values (accumulation error only), 4e-3 / 3e-2 against the unquantised FP32
input (end to end)."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import quant as Q
from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0


def _gridder(hcg, f, storage=None):
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    if storage:
        g.set_storage(storage)
    return g


def _grid(hcg, f, spec=None, storage=None, lon=None, lat=None, dtype=None, scale=None, path=None):
    g = _gridder(hcg, f, storage)
    if path is not None:
        g.set_tuning(path=path)
    s = f.spectra(device="cuda") if spec is None else spec
    lon = f.lon if lon is None else lon
    lat = f.lat if lat is None else lat
    g.load_samples(torch.from_numpy(lon).cuda(), torch.from_numpy(lat).cuda(), s, dtype=dtype, chan_scale=scale)
    g.grid()
    cube, w = g.fetch()
    return g, cube.reshape(f.cells, -1), w.ravel()


def _check(cube, w, v, wr, ab, cnt, tol, wtol=1e-5):
    ok = cnt > 0
    assert np.all(np.isnan(cube[~ok])) and np.all(w[~ok] == 0)
    err = np.abs(cube[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])
    werr = np.abs(w[ok] - wr[ok]) / wr[ok]
    assert err.max() <= tol, f"max condition-aware error {err.max():.3e} > {tol}"
    assert werr.max() <= wtol, f"max weight error {werr.max():.3e}"
    return float(err.max())


def test_uniform_single_channel(hcg):
    f = synth.workload("uniform-20k")
    g, cube, w = _grid(hcg, f)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, f.spectra_np())
    _check(cube, w, v, wr, ab, cnt, 1e-5)
    assert g.info()["pairs"] == cnt.sum()


@pytest.mark.parametrize("nchan,nx,ny", [(1024, 31, 29), (1000, 17, 23), (67, 20, 21), (3, 25, 25), (512, 9, 9)])
def test_drift_scan_multichannel(hcg, nchan, nx, ny):
    """Drift-scan rows at the 1M-sample density on a small field; channel
    counts that exercise every lane layout, odd grids for ragged groups."""
    f = synth.drift_field(12, width=nx * AM * 1.1, height=ny * AM * 1.1, hz=1.0, passes=3, nchan=nchan, nx=nx,
                          ny=ny, pix=AM, fwhm=1.5 * AM, nsig=3.0, nsrc=6)
    g, cube, w = _grid(hcg, f)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, f.spectra_np())
    _check(cube, w, v, wr, ab, cnt, 1e-5)


@pytest.mark.parametrize("lon0,lat0", [(0.0, 10.0), (359.95, -8.0), (45.0, 58.0)])
def test_seam_and_high_latitude(hcg, lon0, lat0):
    f = synth.uniform_field(seed=31, n=8000, width=0.9, height=0.7, lon0=lon0, lat0=lat0, nx=45, ny=33,
                            nchan=16, fwhm=2.0 * AM, nsig=4.0)
    lon = f.lon % 360.0        # samples given in [0, 360) across the seam
    g, cube, w = _grid(hcg, f, lon=lon)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), lon, f.lat, f.spectra_np())
    _check(cube, w, v, wr, ab, cnt, 1e-5)


def test_constant_input_reproduces_constant(hcg):
    f = synth.workload("uniform-20k")
    spec = torch.full((f.n, 1), 3.75, device="cuda")
    g, cube, w = _grid(hcg, f, spec=spec)
    ok = w > 0
    assert np.abs(cube[ok] - 3.75).max() <= 3.75 * 4e-7
    assert np.isnan(cube[~ok]).all()


def test_single_sample_closed_form(hcg):
    f = synth.uniform_field(seed=5, n=1, width=0.0, height=0.0, nx=9, ny=9, nchan=4)
    lon = np.array([180.0021]); lat = np.array([30.0013])
    spec = torch.tensor([[1.0, -2.0, 3.5, 0.0]], device="cuda")
    g, cube, w = _grid(hcg, f, spec=spec, lon=lon, lat=lat)
    sig = math.radians(f.fwhm) / math.sqrt(8 * math.log(2))
    i, j = np.meshgrid(np.arange(9), np.arange(9))
    clon = f.lon0 + (i - 4) * f.pix; clat = f.lat0 + (j - 4) * f.pix
    h = np.sin(np.radians(lat[0] - clat) / 2) ** 2 + np.cos(np.radians(clat)) * np.cos(np.radians(lat[0])) * \
        np.sin(np.radians(lon[0] - clon) / 2) ** 2
    d = 2 * np.arcsin(np.sqrt(h)).ravel()
    inside = d <= math.radians(f.support)
    np.testing.assert_allclose(w[inside], np.exp(-d[inside] ** 2 / (2 * sig * sig)), rtol=2e-6)
    assert np.all(w[~inside] == 0)
    np.testing.assert_allclose(cube[inside], np.tile([1.0, -2.0, 3.5, 0.0], (inside.sum(), 1)), rtol=1e-6)


def test_permutation_gives_identical_bits(hcg):
    f = synth.drift_field(13, width=0.35, height=0.3, hz=1.0, passes=2, nchan=64, nx=18, ny=16, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    spec = f.spectra(device="cuda")
    _, c1, w1 = _grid(hcg, f, spec=spec)
    q = np.random.default_rng(3).permutation(f.n)
    _, c2, w2 = _grid(hcg, f, spec=spec[torch.from_numpy(q).cuda()].contiguous(), lon=f.lon[q], lat=f.lat[q])
    assert np.array_equal(c1, c2, equal_nan=True) and np.array_equal(w1, w2)


def test_empty_and_out_of_field(hcg):
    f = synth.uniform_field(seed=7, n=10, width=0.1, height=0.1, lon0=10.0, lat0=10.0, nx=6, ny=5, nchan=2)
    # samples 30 degrees away in longitude: kept by the ring filter (same
    # latitudes) but outside every cell's support
    g, cube, w = _grid(hcg, f, lon=f.lon + 30.0)
    assert np.isnan(cube).all() and (w == 0).all() and g.info()["pairs"] == 0
    # samples 5 degrees away in latitude: dropped by the ring filter
    g, cube, w = _grid(hcg, f, lat=f.lat + 5.0)
    assert np.isnan(cube).all() and (w == 0).all() and g.info()["samples_kept"] == 0
    # no samples at all
    g = _gridder(hcg, f)
    g.load_samples(torch.empty(0, dtype=torch.float64, device="cuda"), torch.empty(0, dtype=torch.float64,
                   device="cuda"), torch.empty((0, 2), device="cuda"))
    g.grid()
    cube, w = g.fetch()
    assert np.isnan(cube).all() and (w == 0).all()


def test_bad_coordinates_are_reported(hcg):
    f = synth.uniform_field(seed=8, n=100, width=0.1, height=0.1, nx=4, ny=4, nchan=1)
    lat = f.lat.copy(); lat[7] = np.nan
    g = _gridder(hcg, f)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(lat).cuda(), f.spectra(device="cuda"))
    g.grid()
    with pytest.raises(hcg.HcgError, match="INVALID_ARG"):
        g.fetch()


def test_argument_errors(hcg):
    g = hcg.Gridder(0)
    with pytest.raises(hcg.HcgError, match="NOT_READY"):
        g.grid()
    with pytest.raises(hcg.HcgError, match="INVALID_ARG"):
        g.set_kernel(-1.0, 0.1)
    with pytest.raises(hcg.HcgError, match="INVALID_ARG"):
        g.set_grid(0, 0, 0.01, 0, 10)
    with pytest.raises(hcg.HcgError, match="INVALID_ARG"):
        g.set_grid(0, 0, 0.01, 10, 10, projection=5)


@pytest.mark.parametrize("storage,tol", [("bf16", 4e-3), ("e4m3", 3e-2)])
def test_quantised_storage(hcg, storage, tol):
    """The library quantises FP32 input on the device; values are checked
    against the oracle on the dequantised input (1e-5) and on the FP32 input
    (the stated end-to-end tolerance)."""
    f = synth.drift_field(14, width=0.45, height=0.4, hz=1.0, passes=3, nchan=256, nx=24, ny=22, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=6)
    x = f.spectra_np()
    g, cube, w = _grid(hcg, f, storage=storage, path=hcg.PATH_GATHER)
    if storage == "bf16":
        deq = Q.bf16_bits_to_f32(Q.bf16_round_bits(x)).astype(np.float64)
    else:
        codes, s = Q.e4m3_quantise(x)
        deq = Q.e4m3_dequantise(codes, s)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, deq)
    _check(cube, w, v, wr, ab, cnt, 1e-5)
    v2, _, ab2, _ = oracle.grid_cells(f.geom(), f.lon, f.lat, x)
    ok = cnt > 0
    e2 = np.abs(cube[ok] - v2[ok]) / (np.abs(v2[ok]) + ab2[ok])
    assert e2.max() <= tol


def test_prequantised_input(hcg):
    """BF16 and E4M3 spectra passed in directly (no device quantisation)."""
    f = synth.drift_field(15, width=0.3, height=0.3, hz=1.0, passes=2, nchan=128, nx=15, ny=15, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=3)
    x = f.spectra_np()
    bits = Q.bf16_round_bits(x)
    spec = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    g, cube, w = _grid(hcg, f, spec=spec, storage="bf16", path=hcg.PATH_GATHER)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, Q.bf16_bits_to_f32(bits).astype(np.float64))
    _check(cube, w, v, wr, ab, cnt, 1e-5)
    codes, s = Q.e4m3_quantise(x)
    spec8 = torch.from_numpy(codes).cuda().view(torch.float8_e4m3fn)
    g, cube, w = _grid(hcg, f, spec=spec8, storage="e4m3", scale=torch.from_numpy(s).cuda(), path=hcg.PATH_GATHER)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, Q.e4m3_dequantise(codes, s))
    _check(cube, w, v, wr, ab, cnt, 1e-5)


def test_wide_kernel_list_overflow(hcg):
    """A support of 4 sigma at 0.6' cells (thousands of contributors per
    group) exceeds the per-warp list, so the list kernel re-searches per
    channel slice; values must still match the oracle."""
    f = synth.drift_field(16, width=0.35, height=0.3, hz=10.0, passes=2, nchan=256, nx=30, ny=24, pix=0.6 * AM,
                          fwhm=3.0 * AM, nsig=4.0, nsrc=5)
    g, cube, w = _grid(hcg, f)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, f.spectra_np())
    assert cnt.max() > 1000
    _check(cube, w, v, wr, ab, cnt, 1e-5)


@pytest.mark.parametrize("nchan", [512, 1000, 1020, 200])
def test_kernel_variants_agree_bitwise(hcg, nchan):
    """Every tuning of the gather path -- list kernel (32 cells per block) with
    8 or 4 channels per lane and 12 or 8 rows in flight, per-slice kernel
    (16 cells per block) with 8 or 4 channels per lane -- accumulates each
    (cell, channel) in the same S' order: identical bits."""
    f = synth.drift_field(17, width=0.4, height=0.35, hz=1.0, passes=3, nchan=nchan, nx=22, ny=19, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    spec = f.spectra(device="cuda")
    _, c1, w1 = _grid(hcg, f, spec=spec)
    tunings = [(32, 8, 12), (32, 8, 8), (32, 4, 8), (16, 8, 0), (16, 4, 0)]
    for cells, vc, depth in tunings:
        g = _gridder(hcg, f)
        g.set_tuning(cells_per_block=cells, chans_per_thread=vc, tile_depth=depth, path=hcg.PATH_GATHER)
        g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), spec)
        g.grid()
        c2, w2 = g.fetch()
        assert np.array_equal(c1, c2.reshape(f.cells, -1), equal_nan=True) and np.array_equal(w1, w2.ravel()), \
            (cells, vc, depth)


def test_borrowed_input_alignment(hcg):
    """Borrowed spectra are used in place by 16-byte vector copies: a pointer
    off that boundary is refused before any work is queued."""
    f = synth.uniform_field(seed=9, n=64, width=0.1, height=0.1, nx=4, ny=4, nchan=4)
    g = _gridder(hcg, f)
    buf = torch.zeros(f.n * f.nchan + 1, device="cuda")
    lon, lat = torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda()
    with pytest.raises(hcg.HcgError):
        g.load_samples(lon, lat, buf[1:].view(f.n, f.nchan), borrow=True)
    g.load_samples(lon, lat, buf[:-1].view(f.n, f.nchan), borrow=True)


def test_dense_clump_overflows_group_lists(hcg):
    """A clump far denser than the field average overflows the per-group
    list slots sized from the mean density; those groups are searched again
    and must still match the oracle."""
    f = synth.drift_field(18, width=0.5, height=0.45, hz=1.0, passes=3, nchan=256, nx=28, ny=25, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    rng = np.random.default_rng(5)
    k = 4000
    lon = np.concatenate([f.lon, f.lon0 + rng.normal(0, 0.5 * AM, k)])
    lat = np.concatenate([f.lat, f.lat0 + rng.normal(0, 0.5 * AM, k)])
    g2 = synth.make_field("clump", lon=lon, lat=lat, nchan=256, lon0=f.lon0, lat0=f.lat0, pix=AM, nx=28, ny=25,
                          fwhm=1.5 * AM, nsig=3.0, seed=19, nsrc=4)
    g, cube, w = _grid(hcg, g2)
    v, wr, ab, cnt = oracle.grid_cells(g2.geom(), g2.lon, g2.lat, g2.spectra_np())
    assert cnt.max() > 2000
    _check(cube, w, v, wr, ab, cnt, 1e-5)


def test_row_alignment_does_not_change_results(hcg):
    """FP32 rows on 32-byte boundaries are read with 256-bit loads, others
    with 128-bit loads: a borrowed buffer 16 bytes off a 32-byte boundary
    gives the same bits."""
    f = synth.drift_field(19, width=0.4, height=0.35, hz=1.0, passes=3, nchan=512, nx=22, ny=19, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    spec = f.spectra(device="cuda")
    lon, lat = torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda()
    out = []
    for off in (0, 4):                                   # floats: 0 and 16 bytes
        buf = torch.zeros(f.n * f.nchan + 8, device="cuda")
        view = buf[off:off + f.n * f.nchan].view(f.n, f.nchan)
        view.copy_(spec)
        g = _gridder(hcg, f)
        g.load_samples(lon, lat, view, borrow=True)
        g.grid()
        out.append(g.fetch())
    assert np.array_equal(out[0][0], out[1][0], equal_nan=True) and np.array_equal(out[0][1], out[1][1])

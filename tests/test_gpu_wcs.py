"""Projected target grids (HCG_WCS_TAN / SIN / SFL / CAR, Calabretta & Greisen
2002) on the CUDA-core gather: values against the oracle's Eq. (1) on the
oracle's own projected cell centres (1e-5), neighbour lists bit-exact, and
the paths that take plain grids only refuse them."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0
PROJ = {"TAN": ("WCS_TAN", oracle.WCS_TAN), "SIN": ("WCS_SIN", oracle.WCS_SIN),
        "SFL": ("WCS_SFL", oracle.WCS_SFL), "CAR": ("WCS_CAR", oracle.WCS_CAR)}


def _field(seed, lon0, lat0, nchan, nx=20, ny=16, pix=AM):
    c = math.cos(math.radians(lat0))
    return synth.uniform_field(seed=seed, n=9000, width=(nx * pix + 12 * AM) / c, height=ny * pix + 12 * AM,
                               lon0=lon0, lat0=lat0, nx=nx, ny=ny, pix=pix, fwhm=1.5 * AM, nsig=3.0,
                               nchan=nchan, name=f"f{seed}")


def _gridder(hcg, f, proj):
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny, projection=proj)
    return g


def _run(hcg, f, proj, spec=None, **tune):
    g = _gridder(hcg, f, proj)
    if tune:
        g.set_tuning(**tune)
    s = f.spectra(device="cuda") if spec is None else spec
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), s)
    g.grid()
    cube, w = g.fetch()
    return g, cube.reshape(f.cells, -1), w.ravel()


def _check(cube, w, v, wr, ab, cnt):
    ok = cnt > 0
    assert ok.mean() > 0.9
    assert np.all(np.isnan(cube[~ok])) and np.all(w[~ok] == 0)
    err = np.abs(cube[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])
    assert err.max() <= 1e-5
    assert np.abs(w[ok] - wr[ok]).max() <= 1e-5 * wr[ok].max()


@pytest.mark.parametrize("name", list(PROJ))
@pytest.mark.parametrize("lon0,lat0,nchan", [(180.0, 30.0, 300), (10.0, -60.0, 3), (359.9, 45.0, 300)])
def test_projected_grid_against_oracle(hcg, name, lon0, lat0, nchan):
    f = _field(51, lon0, lat0, nchan)
    attr, code = PROJ[name]
    g, cube, w = _run(hcg, f, getattr(hcg, attr))
    clon, clat = oracle.wcs_cells(code, f.lon0, f.lat0, f.pix, f.nx, f.ny)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, f.spectra_np(), cell_lon=clon, cell_lat=clat)
    _check(cube, w, v, wr, ab, cnt)
    assert g.info()["pairs"] == cnt.sum()


@pytest.mark.parametrize("name", list(PROJ))
def test_projected_neighbour_lists_bit_exact(hcg, name):
    f = _field(52, 120.0, 50.0, 1)
    attr, code = PROJ[name]
    g, _, _ = _run(hcg, f, getattr(hcg, attr))
    off, ids = g.debug_neighbours()
    clon, clat = oracle.wcs_cells(code, f.lon0, f.lat0, f.pix, f.nx, f.ny)
    ooff, oids, guard = oracle.neighbours_band(np.array(f.geom()), f.lon, f.lat, cell_lon=clon, cell_lat=clat)
    assert guard.sum() == 0
    assert np.array_equal(off, ooff) and np.array_equal(ids, oids)


def test_projected_grid_in_a_batch_and_streamed(hcg):
    """A TAN field gives the same bits alone, in a batch, and streamed."""
    f = _field(53, 200.0, 20.0, 512)
    spec = f.spectra(device="cuda")
    _, c0, w0 = _run(hcg, f, hcg.WCS_TAN, spec=spec)
    st = torch.cuda.Stream()
    g = hcg.Gridder(0, st)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny, projection=hcg.WCS_TAN)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), spec, borrow=True)
    b = hcg.Batch(0, st)
    b.add(g)
    b.grid()
    b.sync()
    c1, w1 = g.fetch()
    b.close()
    assert np.array_equal(c0, c1.reshape(f.cells, -1), equal_nan=True) and np.array_equal(w0, w1.ravel())
    gs = _gridder(hcg, f, hcg.WCS_TAN)
    gs.set_stream_chunk(256)
    gs.load_samples(f.lon, f.lat, spec.cpu().pin_memory(), stream=True)
    gs.grid()
    c2, w2 = gs.fetch()
    assert np.array_equal(c0, c2.reshape(f.cells, -1), equal_nan=True) and np.array_equal(w0, w2.ravel())


def test_equatorial_fits_car_matches_plain_grid(hcg):
    f = _field(54, 75.0, 0.0, 8)
    _, c0, w0 = _run(hcg, f, hcg.CAR)
    _, c1, w1 = _run(hcg, f, hcg.WCS_CAR)
    ok = w0 > 0
    assert np.array_equal(ok, w1 > 0)
    assert np.abs(c1[ok] - c0[ok]).max() <= 1e-5 * (np.abs(c0[ok]).max() + 1)
    assert np.abs(w1 - w0).max() <= 1e-6 * w0.max()


def test_projected_grid_refusals(hcg):
    g = hcg.Gridder(0)
    g.set_kernel(1.5 * AM, 1.5 * AM * 3 / 2.3548)
    with pytest.raises(hcg.HcgError):      # SIN cells beyond the hemisphere
        g.set_grid(0.0, 0.0, 30.0, 5, 5, projection=hcg.WCS_SIN)
    with pytest.raises(hcg.HcgError):      # cells past latitude 89
        g.set_grid(0.0, 88.5, 0.5, 5, 5, projection=hcg.WCS_TAN)
    f = _field(55, 30.0, 10.0, 256)
    for path in (hcg.PATH_TENSOR, hcg.PATH_SCATTER):
        g = _gridder(hcg, f, hcg.WCS_TAN)
        g.set_storage("bf16")
        g.set_tuning(path=path)
        g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), f.spectra(device="cuda"))
        with pytest.raises(hcg.HcgError):
            g.grid()


def _cell_list_field(seed, m):
    f = synth.uniform_field(seed=seed, n=9000, width=0.8, height=0.6, lon0=30.0, lat0=-20.0, nx=40, ny=30,
                            nchan=8, fwhm=2.0 * AM, nsig=3.0)
    rng = np.random.default_rng(seed + 1)
    # unsorted sight-lines, some beyond the sampled area (empty cells)
    clon = f.lon0 + rng.uniform(-0.45, 0.45, m)
    clat = f.lat0 + rng.uniform(-0.35, 0.35, m)
    return f, clon, clat


def _cell_list_run(hcg, f, clon, clat, spec=None):
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_cell_list(torch.from_numpy(clon).cuda(), torch.from_numpy(clat).cuda())
    s = f.spectra(device="cuda") if spec is None else spec
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), s)
    g.grid()
    cube, w = g.fetch()
    return g, cube.reshape(clon.size, -1), w.ravel()


def test_cell_list_target_against_oracle(hcg):
    """A free list of target positions (Sec. 2.1: the target is a set of cells
    (alpha_ij, delta_ij)): values, weights and pair counts against the
    oracle's explicit-cell Eq. (1); contributor lists bit-exact."""
    m = 2500
    f, clon, clat = _cell_list_field(93, m)
    g, cube, w = _cell_list_run(hcg, f, clon, clat)
    geom = (f.lon0, f.lat0, f.pix, m, 1, f.support, f.fwhm)
    v, wr, ab, cnt = oracle.grid_cells(geom, f.lon, f.lat, f.spectra_np(), cell_lon=clon, cell_lat=clat)
    ok = cnt > 0
    assert 0.5 < ok.mean() < 1.0
    assert np.all(np.isnan(cube[~ok])) and np.all(w[~ok] == 0)
    assert (np.abs(cube[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])).max() <= 1e-5
    assert (np.abs(w[ok] - wr[ok]) / wr[ok]).max() <= 1e-5
    assert g.info()["pairs"] == cnt.sum()
    off, ids = g.debug_neighbours()
    ooff, oids, guard = oracle.neighbours_band(np.array(geom), f.lon, f.lat, cell_lon=clon, cell_lat=clat)
    assert guard.sum() == 0
    assert np.array_equal(off, ooff) and np.array_equal(ids, oids)


def test_cell_list_order_and_refusals(hcg):
    """Reordering the list reorders the results (same contributors per cell;
    values to rounding of the weight sums); the other paths refuse a list."""
    m = 600
    f, clon, clat = _cell_list_field(95, m)
    spec = f.spectra(device="cuda")
    _, c0, w0 = _cell_list_run(hcg, f, clon, clat, spec)
    perm = np.random.default_rng(96).permutation(m)
    _, c1, w1 = _cell_list_run(hcg, f, clon[perm], clat[perm], spec)
    assert np.array_equal(np.isnan(c0[perm]), np.isnan(c1))
    ok = w1 > 0
    np.testing.assert_allclose(w1[ok], w0[perm][ok], rtol=2e-6)
    np.testing.assert_allclose(c1[ok], c0[perm][ok], rtol=2e-5, atol=2e-6 * np.abs(c0[perm][ok]).max())
    for path in (hcg.PATH_TENSOR, hcg.PATH_STAGED, hcg.PATH_SCATTER):
        g = hcg.Gridder(0)
        g.set_kernel(f.fwhm, f.support)
        g.set_cell_list(clon, clat)
        g.set_storage("bf16")
        g.set_tuning(path=path)
        g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(),
                       torch.zeros((f.n, 256), device="cuda"))
        with pytest.raises(hcg.HcgError, match="UNSUPPORTED"):
            g.grid()
    g = hcg.Gridder(0)
    for lon, lat in ([np.array([0.0, 120.0, 240.0]), np.array([0.0, 0.0, 0.0])], [np.array([10.0]), np.array([89.5])],
                     [np.array([np.nan]), np.array([0.0])]):
        with pytest.raises(hcg.HcgError, match="INVALID_ARG"):
            g.set_cell_list(lon, lat)

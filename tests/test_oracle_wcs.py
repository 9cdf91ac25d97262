"""Pins of the oracle's grid projections (Calabretta & Greisen 2002: TAN, SIN,
SFL, CAR with the reference point at the grid centre) against facts that do
not use its formulas: where the reference pixel lands, great-circle distances
and bearings from the reference point (textbook spherical trigonometry,
written here with numpy), the plain forms at the equator, and agreement of
brute-force and band neighbour searches on projected cells."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")
AM = 1.0 / 60.0
PROJ = {"TAN": oracle.WCS_TAN, "SIN": oracle.WCS_SIN, "SFL": oracle.WCS_SFL, "CAR": oracle.WCS_CAR}


def _dist_bearing(lon1, lat1, lon2, lat2):
    """Great-circle distance (rad) and initial bearing east of north (rad)."""
    p1, p2 = np.radians(lat1), np.radians(lat2)
    dl = np.radians(lon2 - lon1)
    h = np.sin((p2 - p1) / 2) ** 2 + np.cos(p1) * np.cos(p2) * np.sin(dl / 2) ** 2
    d = 2 * np.arcsin(np.sqrt(h))
    b = np.arctan2(np.sin(dl) * np.cos(p2), np.cos(p1) * np.sin(p2) - np.sin(p1) * np.cos(p2) * np.cos(dl))
    return d, b


def _offsets(nx, ny, pix):
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    return ((i - (nx - 1) / 2) * pix).ravel(), ((j - (ny - 1) / 2) * pix).ravel()


@pytest.mark.parametrize("name", list(PROJ))
@pytest.mark.parametrize("lon0,lat0", [(180.0, 30.0), (0.0, -45.0), (359.5, 72.0), (10.0, 0.0)])
def test_reference_pixel_lands_on_reference_point(name, lon0, lat0):
    clon, clat = oracle.wcs_cells(PROJ[name], lon0, lat0, 2 * AM, 7, 9)
    c = 4 * 7 + 3
    assert abs(((clon[c] - lon0 + 180) % 360) - 180) < 1e-9 and abs(clat[c] - lat0) < 1e-9


@pytest.mark.parametrize("name,dist", [("TAN", np.arctan), ("SIN", np.arcsin)])
@pytest.mark.parametrize("lat0", [30.0, -60.0, 85.0])
def test_zenithal_distance_and_bearing(name, dist, lat0):
    """Zenithal projections: a cell at offset (x, y) lies at great-circle
    distance atan|(x, y)| (TAN) or asin|(x, y)| (SIN) from the reference point,
    at bearing atan2(x, y) east of north."""
    nx, ny, pix = 41, 33, 0.5
    clon, clat = oracle.wcs_cells(PROJ[name], 200.0, lat0, pix, nx, ny)
    x, y = _offsets(nx, ny, pix)
    d, b = _dist_bearing(200.0, lat0, clon, clat)
    r = np.radians(np.hypot(x, y))
    assert np.abs(d - dist(r)).max() < 1e-11
    far = r > 1e-6
    db = np.angle(np.exp(1j * (b[far] - np.arctan2(x[far], y[far]))))
    assert np.abs(db).max() < 1e-9


def test_equatorial_car_and_sfl_are_plain():
    nx, ny, pix = 25, 19, 1.5
    x, y = _offsets(nx, ny, pix)
    clon, clat = oracle.wcs_cells(oracle.WCS_CAR, 100.0, 0.0, pix, nx, ny)
    assert np.abs(clat - y).max() < 1e-10 and np.abs(clon - (100.0 + x)).max() < 1e-10
    clon, clat = oracle.wcs_cells(oracle.WCS_SFL, 100.0, 0.0, pix, nx, ny)
    assert np.abs(clat - y).max() < 1e-10
    assert np.abs(clon - (100.0 + x / np.cos(np.radians(y)))).max() < 1e-9


@pytest.mark.parametrize("lat0", [35.0, -50.0])
def test_oblique_car_geometry(lat0):
    """CAR with the reference point off the equator: the central column is the
    reference meridian (latitude lat0 + y), the central row is the great circle
    leaving the reference point due east (distance |x|, bearing 90 deg), and
    every cell is |y| from the central-row cell of its column."""
    nx, ny, pix = 31, 21, 0.75
    clon, clat = oracle.wcs_cells(oracle.WCS_CAR, 40.0, lat0, pix, nx, ny)
    x, y = _offsets(nx, ny, pix)
    L = clon.reshape(ny, nx); B = clat.reshape(ny, nx)
    ic, jc = (nx - 1) // 2, (ny - 1) // 2
    assert np.abs(L[:, ic] - 40.0).max() < 1e-9
    assert np.abs(B[:, ic] - (lat0 + y.reshape(ny, nx)[:, ic])).max() < 1e-9
    d, b = _dist_bearing(40.0, lat0, L[jc], B[jc])
    xr = np.radians(x.reshape(ny, nx)[jc])
    assert np.abs(d - np.abs(xr)).max() < 1e-11
    east = xr > 0
    assert np.abs(b[east] - np.pi / 2).max() < 1e-9
    for i in (0, 7, nx - 1):
        dd, _ = _dist_bearing(L[jc, i], B[jc, i], L[:, i], B[:, i])
        assert np.abs(dd - np.abs(np.radians(y.reshape(ny, nx)[:, i]))).max() < 1e-11


def test_sin_has_no_points_beyond_its_hemisphere():
    nx = ny = 5
    pix = 30.0                     # corners at |(x, y)| = 60 sqrt(2) deg > 57.3 deg
    clon, clat = oracle.wcs_cells(oracle.WCS_SIN, 0.0, 0.0, pix, nx, ny)
    x, y = _offsets(nx, ny, pix)
    bad = np.radians(np.hypot(x, y)) > 1.0
    assert np.all(np.isnan(clat[bad])) and np.all(np.isfinite(clat[~bad]))


@pytest.mark.parametrize("name", list(PROJ))
def test_projected_cells_brute_equals_band(name):
    rng = np.random.default_rng(7)
    nx, ny, pix = 12, 10, 1.2 * AM
    clon, clat = oracle.wcs_cells(PROJ[name], 120.0, 55.0, pix, nx, ny)
    n = 4000
    lon = 120.0 + rng.uniform(-0.45, 0.45, n) / np.cos(np.radians(55.0))
    lat = 55.0 + rng.uniform(-0.3, 0.3, n)
    geom = oracle.geom_array(120.0, 55.0, pix, nx, ny, 3 * AM, 2 * AM)
    o1, i1, _ = oracle.neighbours_brute(geom, lon, lat, cell_lon=clon, cell_lat=clat)
    o2, i2, _ = oracle.neighbours_band(geom, lon, lat, cell_lon=clon, cell_lat=clat)
    assert np.array_equal(o1, o2) and np.array_equal(i1, i2) and o1[-1] > 0

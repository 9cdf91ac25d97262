"""Pins of the oracle's Eq. (1) gridding against closed forms and
invariants (HCGrid Sec. 2.1, Sec. 3.6 item 3)."""
import math

import numpy as np
import pytest

AM = 1.0 / 60.0


def _geom(orc, lon0=180.0, lat0=30.0, pix=1.0 * AM, nx=24, ny=20, nsig=3.0, fwhm=1.5 * AM):
    sig = fwhm / math.sqrt(8 * math.log(2))
    return orc.geom_array(lon0, lat0, pix, nx, ny, nsig * sig, fwhm), sig


def _cell_centres(g):
    lon0, lat0, pix, nx, ny = g[0], g[1], g[2], int(g[3]), int(g[4])
    i = np.arange(nx); j = np.arange(ny)
    lon = lon0 + (i - (nx - 1) / 2) * pix
    lat = lat0 + (j - (ny - 1) / 2) * pix
    return np.meshgrid(lon, lat)   # [ny, nx]


def _vec(lon, lat):
    lo = np.radians(lon); la = np.radians(lat)
    return np.stack([np.cos(la) * np.cos(lo), np.cos(la) * np.sin(lo), np.sin(la)], -1)


def _samples(seed, g, n, spread=1.3):
    rng = np.random.default_rng(seed)
    w = g[2] * g[3] * spread; h = g[2] * g[4] * spread
    lon = g[0] + rng.uniform(-w / 2, w / 2, n)
    lat = g[1] + rng.uniform(-h / 2, h / 2, n)
    return lon, lat


def test_distance_against_chord_formula(orc):
    """Single sample: W of every cell equals exp(-d^2/2 sigma^2) with d from
    the chord length of unit vectors, d = 2 asin(|u - v| / 2) (an independent
    formula for the great-circle distance), and V = s inside the disc."""
    g, sig = _geom(orc)
    lon = np.array([180.0037]); lat = np.array([30.0021])
    v, w, _, cnt = orc.grid_cells(g, lon, lat, np.array([[2.5]]))
    clon, clat = _cell_centres(g)
    d = 2 * np.arcsin(np.linalg.norm(_vec(clon, clat) - _vec(lon[0], lat[0]), axis=-1) / 2)
    sr = math.radians(sig); R = math.radians(g[5])
    inside = (d <= R * (1 - 1e-9)).ravel()
    outside = (d > R * (1 + 1e-9)).ravel()
    np.testing.assert_allclose(w[inside], np.exp(-d.ravel()[inside] ** 2 / (2 * sr * sr)), rtol=1e-9)
    assert np.all(w[outside] == 0) and np.all(np.isnan(v[outside, 0]))
    np.testing.assert_allclose(v[inside, 0], 2.5, rtol=1e-15)
    assert inside.sum() > 5


def test_half_maximum_at_half_fwhm(orc):
    """The kernel is the Gaussian of the stated FWHM: w(FWHM/2) = 1/2."""
    g, _ = _geom(orc, nx=1, ny=1)
    lat = np.array([30.0 + 0.5 * g[6]])
    _, w, _, _ = orc.grid_cells(g, np.array([180.0]), lat, np.array([[1.0]]))
    assert abs(w[0] - 0.5) < 1e-12


def test_support_is_closed_disc(orc):
    """A sample exactly R away (along the meridian) contributes; h <= h_R."""
    g, _ = _geom(orc, nx=1, ny=1)
    R = g[5]
    for eps, expect in [(-1e-10, 1), (1e-9, 0)]:
        lat = np.array([30.0 + R + eps])
        _, w, _, cnt = orc.grid_cells(g, np.array([180.0]), lat, np.array([[1.0]]))
        assert cnt[0] == expect


def test_two_samples_weighted_mean(orc):
    g, sig = _geom(orc, nx=3, ny=3)
    lon = np.array([180.0, 180.004]); lat = np.array([30.002, 29.999]); s = np.array([[1.0], [5.0]])
    v, w, _, _ = orc.grid_cells(g, lon, lat, s)
    clon, clat = _cell_centres(g)
    sr = math.radians(sig)
    for c in range(9):
        d = [2 * math.asin(np.linalg.norm(_vec(clon.ravel()[c], clat.ravel()[c]) - _vec(lon[k], lat[k])) / 2)
             for k in range(2)]
        ws = [math.exp(-x * x / (2 * sr * sr)) for x in d]
        assert abs(v[c, 0] - (ws[0] * 1 + ws[1] * 5) / (ws[0] + ws[1])) < 1e-12
        assert abs(w[c] - sum(ws)) < 1e-12


def test_constant_linear_and_channel_independent(orc):
    g, _ = _geom(orc)
    lon, lat = _samples(1, g, 3000)
    rng = np.random.default_rng(2)
    s1 = rng.normal(size=(lon.size, 3)); s2 = rng.normal(size=(lon.size, 3))
    vk, wk, _, _ = orc.grid_cells(g, lon, lat, np.full((lon.size, 2), 7.25))
    ok = wk > 0
    assert ok.sum() > 0.9 * wk.size
    np.testing.assert_allclose(vk[ok], 7.25, rtol=1e-13)
    assert np.all(np.isnan(vk[~ok]))
    v1, _, _, _ = orc.grid_cells(g, lon, lat, s1)
    v2, _, _, _ = orc.grid_cells(g, lon, lat, s2)
    v12, _, _, _ = orc.grid_cells(g, lon, lat, 2 * s1 - 3 * s2)
    np.testing.assert_allclose(v12[ok], 2 * v1[ok] - 3 * v2[ok], rtol=1e-10, atol=1e-12)
    vc, _, _, _ = orc.grid_cells(g, lon, lat, s1[:, 1:2])
    np.testing.assert_array_equal(vc[ok, 0], v1[ok, 1])


def test_permutation_invariance(orc):
    g, _ = _geom(orc)
    lon, lat = _samples(3, g, 2000)
    s = np.random.default_rng(4).normal(size=(lon.size, 2))
    v, w, _, _ = orc.grid_cells(g, lon, lat, s)
    q = np.random.default_rng(5).permutation(lon.size)
    v2, w2, _, _ = orc.grid_cells(g, lon[q], lat[q], s[q])
    np.testing.assert_allclose(v2, v, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(w2, w, rtol=1e-13)


@pytest.mark.parametrize("lon0,lat0", [(180.0, 30.0), (0.0, -5.0), (359.9, 55.0), (10.0, 80.0)])
def test_brute_force_equals_band_search(orc, lon0, lat0):
    """The two neighbour searches agree exactly, including across RA 0 and at
    high declination."""
    g, _ = _geom(orc, lon0=lon0, lat0=lat0, nx=16, ny=12, pix=1.2 * AM)
    lon, lat = _samples(7, g, 2500)
    lon = lon % 360.0
    ob, ib, gb = orc.neighbours_brute(g, lon, lat)
    oc, ic, gc = orc.neighbours_band(g, lon, lat)
    assert np.array_equal(ob, oc) and np.array_equal(ib, ic)
    assert ob[-1] > 100


def test_empty_cells_are_nan(orc):
    g, _ = _geom(orc, nx=10, ny=10)
    lon = np.array([180.0]); lat = np.array([30.0])
    v, w, _, cnt = orc.grid_cells(g, lon, lat, np.array([[3.0]]))
    assert np.all(np.isnan(v[cnt == 0])) and np.all(w[cnt == 0] == 0)
    assert np.all(v[cnt > 0] == 3.0)

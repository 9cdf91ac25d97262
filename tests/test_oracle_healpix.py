"""Pins of the oracle's HEALPix RING functions (Gorski et al. 2005; HCGrid
Sec. 3.2) against structure the pixelisation fixes, not against itself."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 32, 64])
def test_pixel_centres_map_to_themselves(orc, nside):
    """Every pixel centre lies inside its own pixel: ang2pix(pix2ang(p)) == p."""
    p = np.arange(orc.npix(nside))
    lon, lat = orc.pix2ang(nside, p)
    q, ring = orc.ang2pix(nside, lon, lat)
    assert np.array_equal(q, p)
    assert all(ring[k] == orc.pix2ring(nside, int(p[k])) for k in range(0, p.size, max(1, p.size // 97)))


@pytest.mark.parametrize("nside", [1, 2, 4, 16, 1024, 16384])
def test_ring_structure(orc, nside):
    """4 nside - 1 rings; 4r pixels in the north cap, 4 nside in the belt,
    mirrored in the south; ring starts are cumulative; 12 nside^2 pixels."""
    total = 0
    for r in list(range(1, min(4 * nside, 200))) + list(range(max(1, 4 * nside - 200), 4 * nside)):
        expect = 4 * r if r < nside else (4 * nside if r <= 3 * nside else 4 * (4 * nside - r))
        assert orc.ring_npix(nside, r) == expect
        assert orc.ring_start(nside, r + 1) - orc.ring_start(nside, r) == expect
    for r in range(1, 4 * nside) if nside <= 16 else []:
        total += orc.ring_npix(nside, r)
    if nside <= 16:
        assert total == 12 * nside * nside
    assert orc.ring_start(nside, 4 * nside) == orc.npix(nside) == 12 * nside * nside


def test_base_pixel_centres(orc):
    """Nside 1: the 12 base pixels are centred at z = 2/3, 0, -2/3 (lat
    asin(2/3) = 41.81 deg) and at longitudes 45 + 90k (caps) and 90k (belt)."""
    lon, lat = orc.pix2ang(1, np.arange(12))
    cap = math.degrees(math.asin(2.0 / 3.0))
    np.testing.assert_allclose(lat[:4], cap, atol=1e-12)
    np.testing.assert_allclose(lat[4:8], 0.0, atol=1e-12)
    np.testing.assert_allclose(lat[8:], -cap, atol=1e-12)
    np.testing.assert_allclose(lon[:4], [45, 135, 225, 315], atol=1e-12)
    np.testing.assert_allclose(lon[4:8], [0, 90, 180, 270], atol=1e-12)
    np.testing.assert_allclose(lon[8:], [45, 135, 225, 315], atol=1e-12)


def test_equal_area(orc):
    """Uniform points on the sphere fill the pixels equally (chi-square)."""
    rng = np.random.default_rng(11)
    nside, n = 4, 192 * 400
    z = rng.uniform(-1, 1, n)
    lon = rng.uniform(0, 360, n)
    lat = np.degrees(np.arcsin(z))
    pix, _ = orc.ang2pix(nside, lon, lat)
    cnt = np.bincount(pix, minlength=192)
    chi2 = ((cnt - 400.0) ** 2 / 400.0).sum()
    # 191 degrees of freedom: mean 191, sd 19.5; 6 sd bounds
    assert 191 - 6 * 19.5 < chi2 < 191 + 6 * 19.5


def _ring_coord(nside, z):
    """Continuous ring coordinate: equals r exactly at the centre latitude of ring r."""
    if z > 2.0 / 3.0:
        return nside * math.sqrt(3.0 * (1.0 - z))
    if z < -2.0 / 3.0:
        return 4 * nside - nside * math.sqrt(3.0 * (1.0 + z))
    return nside * (2.0 - 1.5 * z)


@pytest.mark.parametrize("nside", [4, 64, 16384])
def test_ring_latitude_band(orc, nside):
    """A point of ring r lies strictly between the centre latitudes of rings
    r-1 and r+1 (the diamonds' vertices sit on the neighbouring rings)."""
    rng = np.random.default_rng(nside)
    n = 4000
    z = rng.uniform(-1, 1, n)
    lon = rng.uniform(0, 360, n)
    lat = np.degrees(np.arcsin(z))
    _, ring = orc.ang2pix(nside, lon, lat)
    for k in range(n):
        rc = _ring_coord(nside, math.sin(math.radians(lat[k])))
        assert ring[k] - 1 - 1e-6 <= rc <= ring[k] + 1 + 1e-6


@pytest.mark.parametrize("nside", [4, 64, 8192])
def test_in_ring_longitude_extent(orc, nside):
    """Cap rings: index in ring = floor(phi n_r / 2 pi).  Belt rings: the
    point lies within half a pixel width of its pixel's centre longitude."""
    rng = np.random.default_rng(nside + 1)
    n = 4000
    z = rng.uniform(-1, 1, n)
    lon = rng.uniform(0, 360, n)
    lat = np.degrees(np.arcsin(z))
    pix, ring = orc.ang2pix(nside, lon, lat)
    for k in range(n):
        r = int(ring[k]); j = int(pix[k]) - orc.ring_start(nside, r)
        nr = orc.ring_npix(nside, r)
        if r < nside or r > 3 * nside:
            assert j == int(math.floor(lon[k] * nr / 360.0)) % nr
        else:
            clon, _ = orc.pix2ang(nside, [int(pix[k])])
            d = (lon[k] - clon[0] + 180.0) % 360.0 - 180.0
            assert abs(d) <= 0.5 * 360.0 / nr + 1e-9


def test_nside_rule(orc):
    """Sec. 3.6 item 3: HEALPix resolution ~ sigma_kernel/2 (mean pixel size
    sqrt(pi/3)/nside <= sigma/2, smallest power of two)."""
    am = 1.0 / 60.0
    assert orc.nside_for(1.5 * am) == 16384
    assert orc.nside_for(1.2 * am) == 16384
    assert orc.nside_for(3.0 * am) == 8192
    assert orc.nside_for(1.0 * am) == 32768
    for fwhm in (0.5 * am, 2.0 * am, 10 * am):
        ns = orc.nside_for(fwhm)
        sig = math.radians(fwhm) / math.sqrt(8 * math.log(2))
        assert math.sqrt(math.pi / 3) / ns <= sig / 2 < math.sqrt(math.pi / 3) / (ns / 2)

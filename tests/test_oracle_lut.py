"""Pins of the oracle's pre-ordering and two-level lookup table (HCGrid
Sec. 3.3 steps I-III)."""
import json
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_caption_fixture(orc):
    """Fig. 'preorder' caption: 17 samples in 9 pixels give
    R_start[1..4] = 1, 7, 10, 17 (1-based)."""
    d = json.load(open(os.path.join(GOLD, "lut_caption.json")))
    ps, perm = orc.preorder(d["nside"], d["lon_deg"], d["lat_deg"], d["r_lo"], d["r_hi"])
    up, us = orc.lut1(ps)
    rs = orc.lut2(d["nside"], ps, d["r_lo"], d["r_hi"])
    assert ps.size == d["expect_samples"]
    assert up.size == d["expect_pixels"]
    assert list(rs[:-1] + 1) == d["expect_rstart_1based"]
    assert rs[-1] == ps.size


def _random(orc, seed, n=3000, nside=64):
    rng = np.random.default_rng(seed)
    lon = rng.uniform(170, 190, n)
    lat = rng.uniform(20, 45, n)
    # duplicated coordinates and duplicated pixels on purpose
    lon[: n // 10] = lon[n // 10: n // 5]
    lat[: n // 10] = lat[n // 10: n // 5]
    return lon, lat, nside


def test_sort_order_is_the_definition(orc):
    """P' is the pixel of each kept sample, in (pixel, hash, index) order,
    and the kept set is exactly the samples with ring in [r_lo, r_hi]."""
    lon, lat, nside = _random(orc, 3)
    pix, ring = orc.ang2pix(nside, lon, lat)
    r_lo, r_hi = int(np.percentile(ring, 20)), int(np.percentile(ring, 80))
    ps, perm = orc.preorder(nside, lon, lat, r_lo, r_hi)
    keep = np.nonzero((ring >= r_lo) & (ring <= r_hi))[0]
    assert sorted(perm.tolist()) == keep.tolist()
    assert np.array_equal(ps, pix[perm])
    h = orc.coord_hash(lon, lat)
    key = sorted(keep.tolist(), key=lambda s: (pix[s], h[s], s))
    assert perm.tolist() == key
    assert np.all(np.diff(ps) >= 0)


def test_sort_is_permutation_invariant(orc):
    """Reordering the input leaves the sorted coordinates unchanged (the
    tie-break depends on coordinates, and only exact duplicates fall back
    to the index, where they are indistinguishable)."""
    lon, lat, nside = _random(orc, 4)
    ps, perm = orc.preorder(nside, lon, lat, 1, 4 * nside - 1)
    q = np.random.default_rng(5).permutation(lon.size)
    ps2, perm2 = orc.preorder(nside, lon[q], lat[q], 1, 4 * nside - 1)
    assert np.array_equal(ps, ps2)
    assert np.array_equal(lon[perm], lon[q][perm2]) and np.array_equal(lat[perm], lat[q][perm2])


def test_lut_tables_match_naive_scans(orc):
    lon, lat, nside = _random(orc, 6)
    _, ring = orc.ang2pix(nside, lon, lat)
    r_lo, r_hi = int(ring.min()) - 2, int(ring.max()) + 2
    ps, perm = orc.preorder(nside, lon, lat, r_lo, r_hi)
    up, us = orc.lut1(ps)
    u, first = np.unique(ps, return_index=True)
    assert np.array_equal(up, u) and np.array_equal(us[:-1], first) and us[-1] == ps.size
    rs = orc.lut2(nside, ps, r_lo, r_hi)
    starts = np.array([orc.ring_start(nside, r) for r in range(r_lo, r_hi + 2)])
    assert np.array_equal(rs, np.searchsorted(ps, starts, side="left"))
    # every sample of ring r sits in [R_start[r], R_start[r+1])
    rings_sorted = np.array([orc.pix2ring(nside, int(p)) for p in ps])
    for r in range(r_lo, r_hi + 1):
        a, b = rs[r - r_lo], rs[r - r_lo + 1]
        assert np.all(rings_sorted[a:b] == r)


def test_coord_hash_reference_values(orc):
    """fmix64 (MurmurHash3 finaliser) on known inputs, checked through a
    plain uint64 numpy restatement of the same published steps."""
    def fmix(k):
        k = np.uint64(k)
        with np.errstate(over="ignore"):
            k ^= k >> np.uint64(33); k *= np.uint64(0xFF51AFD7ED558CCD)
            k ^= k >> np.uint64(33); k *= np.uint64(0xC4CEB9FE1A85EC53)
            k ^= k >> np.uint64(33)
        return int(k)
    # fmix64(0) = 0 and fmix64 is a bijection; spot values
    assert fmix(0) == 0
    for lon, lat in [(0.0, 0.0), (180.25, -30.5), (359.999, 89.9)]:
        a = int(np.float64(lat).view(np.uint64)); b = int(np.float64(lon).view(np.uint64))
        x = a ^ (((b << 29) | (b >> 35)) & ((1 << 64) - 1))
        assert orc.coord_hash([lon], [lat])[0] == fmix(x) >> 32

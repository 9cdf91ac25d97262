"""GPU parity of the pre-ordering, both lookup tables and the neighbour
search (HCGrid Sec. 3.3-3.4) against the FP64 oracle, through the C ABI.
Integer outputs must be bit-exact."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0


def _run(hcg, f, spec=None, dtype=None, storage=None):
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    if storage:
        g.set_storage(storage)
    s = f.spectra(device="cuda") if spec is None else spec
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), s, dtype=dtype)
    g.grid()
    return g


def _fields():
    yield synth.workload("uniform-20k")
    yield synth.uniform_field(seed=21, n=6000, width=1.0, height=0.8, lon0=0.05, lat0=-5.0, nx=40, ny=31,
                              nchan=3, name="ra0")
    yield synth.uniform_field(seed=22, n=6000, width=1.4, height=0.6, lon0=100.0, lat0=62.0, nx=33, ny=17,
                              pix=1.2 * AM, fwhm=2.0 * AM, nsig=4.0, nchan=2, name="cap")
    # wide support in the south cap, and cells a few degrees from the pole
    # (per-ring longitude windows with small cosines)
    yield synth.uniform_field(seed=23, n=8000, width=1.2, height=0.7, lon0=300.0, lat0=-70.0, nx=30, ny=18,
                              pix=1.0 * AM, fwhm=1.5 * AM, nsig=5.0, nchan=2, name="south-cap")
    yield synth.uniform_field(seed=24, n=8000, width=3.0, height=0.5, lon0=20.0, lat0=86.5, nx=16, ny=25,
                              pix=1.0 * AM, fwhm=1.5 * AM, nsig=3.0, nchan=2, name="near-pole")


@pytest.mark.parametrize("f", list(_fields()), ids=lambda f: f.name)
def test_preorder_and_tables_bit_exact(hcg, f):
    g = _run(hcg, f)
    inf = g.info()
    assert inf["nside"] == oracle.nside_for(f.fwhm)
    ps, perm = g.debug_pix()
    ops, operm = oracle.preorder(inf["nside"], f.lon, f.lat, inf["ring_lo"], inf["ring_hi"])
    assert ps.size == ops.size == inf["samples_kept"]
    assert np.array_equal(ps, ops)
    assert np.array_equal(perm, operm)
    upix, ust, rst = g.debug_lut()
    oup, ous = oracle.lut1(ops)
    assert np.array_equal(upix, oup) and np.array_equal(ust, ous)
    assert np.array_equal(rst, oracle.lut2(inf["nside"], ops, inf["ring_lo"], inf["ring_hi"]))
    # the ring range is conservative: no sample within R of a cell is dropped
    off, ids, _ = oracle.neighbours_band(np.array(f.geom()), f.lon, f.lat)
    kept = np.zeros(f.n, bool); kept[perm] = True
    assert kept[ids].all()


def test_table_layout_like_caption(hcg):
    """Sec. 3.3 caption layout at the library's own resolution: 17 samples in
    9 pixels over 4 consecutive rings, 6/3/7/1 samples per ring."""
    fwhm = 1.5 * AM
    ns = oracle.nside_for(fwhm)
    _, ring0 = oracle.ang2pix(ns, [180.0], [30.0])
    r0 = int(ring0[0])
    lon, lat = [], []
    layout = [(0, [3, 2, 1]), (1, [2, 1]), (2, [3, 2, 2]), (3, [1])]   # (ring offset, samples per pixel)
    for dr, per in layout:
        start = oracle.ring_start(ns, r0 + dr)
        p0, _ = oracle.ang2pix(ns, [180.0], [30.0])
        base = start + (int(p0[0]) - oracle.ring_start(ns, r0))
        for k, cnt in enumerate(per):
            clon, clat = oracle.pix2ang(ns, [base + 3 * k])
            for q in range(cnt):
                lon.append(clon[0] + (q - 1) * 1e-6); lat.append(clat[0] + (q - 1) * 1e-6)
    f = synth.make_field("caption", lon=np.array(lon), lat=np.array(lat), nchan=1, lon0=180.0, lat0=30.0,
                         pix=AM, nx=3, ny=3, fwhm=fwhm, nsig=3.0, seed=1, nsrc=1)
    g = _run(hcg, f)
    inf = g.info()
    upix, ust, rst = g.debug_lut()
    assert inf["samples_kept"] == 17 and upix.size == 9
    k0 = r0 - inf["ring_lo"]
    assert list(np.diff(rst[k0:k0 + 5])) == [6, 3, 7, 1]


@pytest.mark.parametrize("f", list(_fields()), ids=lambda f: f.name)
def test_neighbour_lists_bit_exact(hcg, f):
    g = _run(hcg, f)
    off, ids = g.debug_neighbours()
    ooff, oids, guard = oracle.neighbours_band(np.array(f.geom()), f.lon, f.lat)
    assert guard.sum() == 0, "pairs inside the libm guard band; compare them separately"
    assert np.array_equal(off, ooff)
    assert np.array_equal(ids, oids)
    assert g.info()["pairs"] == ooff[-1]


@pytest.mark.parametrize("name", ["drift-1M-c1024", "drift-16M-c256"])
def test_preorder_full_size_bit_exact(hcg, name):
    """The pre-ordering at the benchmark sizes (1M and 16M samples): pixels,
    permutation and both tables bit-exact against the oracle."""
    f = synth.workload(name)
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(),
                   torch.zeros((f.n, 1), device="cuda"))
    g.grid()
    inf = g.info()
    ps, perm = g.debug_pix()
    ops, operm = oracle.preorder(inf["nside"], f.lon, f.lat, inf["ring_lo"], inf["ring_hi"])
    assert np.array_equal(ps, ops) and np.array_equal(perm, operm)
    upix, ust, rst = g.debug_lut()
    oup, ous = oracle.lut1(ops)
    assert np.array_equal(upix, oup) and np.array_equal(ust, ous)
    # LUT2 against its definition (searchsorted of each ring's first pixel)
    starts = np.array([oracle.ring_start(inf["nside"], r) for r in range(inf["ring_lo"], inf["ring_hi"] + 2)])
    assert np.array_equal(rst, np.searchsorted(ops, starts, side="left"))


def test_wide_sort_key_bit_exact(hcg):
    """A ring range holding 2^32 pixels or more: FWHM 6 arcsec (nside 2^18,
    rings of 2^20 pixels 0.5 arcsec apart) on a 0.7 degree tall grid spans
    about 5000 rings.  The pixel offset then no longer fits beside the 32-bit
    hash in one 64-bit key; the sort runs the hash digits and the pixel
    digits as two phases, and pixels, permutation, tables, neighbour lists
    and values must still match the oracle exactly (values to 1e-5)."""
    AS = 1.0 / 3600.0
    rng = np.random.default_rng(81)
    n = 6000
    lon = 120.0 + rng.uniform(-6.0, 6.0, n) * AS
    lat = 10.0 + rng.uniform(-0.37, 0.37, n)
    f = synth.make_field("tall-6arcsec", lon=lon, lat=lat, nchan=3, lon0=120.0, lat0=10.0, pix=3.0 * AS, nx=2,
                         ny=840, fwhm=6.0 * AS, nsig=3.0, seed=82, nsrc=2)
    g = _run(hcg, f)
    inf = g.info()
    assert inf["nside"] == oracle.nside_for(f.fwhm) == 1 << 18
    assert inf["key_bits"] > 64
    ps, perm = g.debug_pix()
    ops, operm = oracle.preorder(inf["nside"], f.lon, f.lat, inf["ring_lo"], inf["ring_hi"])
    # samples beyond the grid's reachable rings (latitude band of the cells
    # +- R, padded) are dropped on both sides
    assert ps.size == ops.size == inf["samples_kept"] and 5000 < ps.size < n
    assert np.array_equal(ps, ops) and np.array_equal(perm, operm)
    upix, ust, rst = g.debug_lut()
    oup, ous = oracle.lut1(ops)
    assert np.array_equal(upix, oup) and np.array_equal(ust, ous)
    assert np.array_equal(rst, oracle.lut2(inf["nside"], ops, inf["ring_lo"], inf["ring_hi"]))
    off, ids = g.debug_neighbours()
    ooff, oids, guard = oracle.neighbours_band(np.array(f.geom()), f.lon, f.lat)
    assert guard.sum() == 0
    assert np.array_equal(off, ooff) and np.array_equal(ids, oids)
    cube, w = g.fetch()
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, f.spectra_np())
    cube = cube.reshape(f.cells, -1); w = w.ravel()
    ok = cnt > 0
    assert ok.sum() > 1000 and np.all(np.isnan(cube[~ok]))
    assert (np.abs(cube[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])).max() <= 1e-5
    assert (np.abs(w[ok] - wr[ok]) / wr[ok]).max() <= 1e-5

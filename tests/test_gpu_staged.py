"""GPU parity of the staged CUDA-core gather (HCG_PATH_STAGED: tiles of 32 or
64 cells whose candidates' spectrum rows are staged in shared memory by bulk
asynchronous copies, 4 x 4-cell register blocks, quadrant masks) against the
FP64 oracle, through the C ABI.

Tolerances as for the other CUDA-core gather (condition-aware per value,
1e-5 for FP32 storage; weights 1e-5 relative per cell; BF16 / E4M3 storage
1e-5 against the oracle on the dequantised spectra and 4e-3 / 3e-2 end to
end), exact pair counts, NaN and weight 0 for empty cells.  The cases cover
ragged tiles, channel tails, both tile sizes and chunk depths, a 4-sigma
support with thousands of contributors per cell, the RA 0 seam, streamed
channel windows (bit-identical to resident spectra) and a batched field."""
import numpy as np
import pytest
import torch

import oracle
from oracle import quant as Q
from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0


def _gridder(hcg, f, storage="f32", cells=0, depth=0, stream=None):
    g = hcg.Gridder(0, stream)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.set_storage(storage)
    g.set_tuning(cells_per_block=cells, tile_depth=depth, path=hcg.PATH_STAGED)
    return g


def _run(hcg, f, storage="f32", cells=0, depth=0, spec=None, lon=None):
    g = _gridder(hcg, f, storage, cells, depth)
    s = f.spectra(device="cuda") if spec is None else spec
    lon = f.lon if lon is None else lon
    g.load_samples(torch.from_numpy(lon).cuda(), torch.from_numpy(f.lat).cuda(), s)
    g.grid()
    cube, w = g.fetch()
    assert g.info()["path"] == hcg.PATH_STAGED
    return g, cube.reshape(f.cells, -1), w.ravel()


def _err(cube, v, ab, ok):
    return np.abs(cube[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])


def _check(f, storage, cube, w, lon=None):
    lon = f.lon if lon is None else lon
    x = f.spectra_np()
    if storage == "f32":
        deq, tol = x.astype(np.float64), 1e-5
    elif storage == "bf16":
        deq, tol = Q.bf16_bits_to_f32(Q.bf16_round_bits(x)).astype(np.float64), 4e-3
    else:
        codes, s = Q.e4m3_quantise(x)
        deq, tol = Q.e4m3_dequantise(codes, s), 3e-2
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), lon, f.lat, deq)
    ok = cnt > 0
    assert ok.any()
    assert np.all(np.isnan(cube[~ok])) and np.all(w[~ok] == 0)
    werr = np.abs(w[ok] - wr[ok]) / wr[ok]
    assert werr.max() <= 1e-5, f"per-cell weight error {werr.max():.3e}"
    e1 = _err(cube, v, ab, ok)
    assert e1.max() <= 1e-5, f"vs oracle on the stored values {e1.max():.3e}"
    if storage != "f32":
        v2, _, ab2, _ = oracle.grid_cells(f.geom(), lon, f.lat, x)
        e2 = _err(cube, v2, ab2, ok)
        assert e2.max() <= tol, f"vs FP32 oracle {e2.max():.3e}"
    return cnt


@pytest.mark.parametrize("storage,nchan,nx,ny,cells,depth,fwhm,nsig,pix", [
    ("f32", 256, 29, 21, 64, 32, 1.5, 3.0, 1.0),     # ragged tiles both ways
    ("f32", 384, 17, 13, 32, 16, 1.5, 3.0, 1.0),     # a 128-channel tail slice
    ("f32", 1000, 12, 11, 64, 16, 1.5, 3.0, 1.0),    # 232-channel tail, lanes without channels
    ("f32", 128, 9, 9, 32, 32, 1.5, 3.0, 1.0),       # one tile, half the warps without channels
    ("f32", 256, 30, 24, 64, 32, 3.0, 4.0, 0.6),     # 4 sigma: thousands of contributors per cell
    ("bf16", 512, 22, 19, 64, 32, 1.5, 3.0, 1.0),
    ("bf16", 256, 26, 17, 32, 16, 3.0, 4.0, 0.6),
    ("e4m3", 256, 25, 18, 32, 32, 3.0, 4.0, 0.6),
    ("e4m3", 768, 15, 20, 64, 16, 1.2, 3.0, 0.6),
])
def test_staged_matches_oracle(hcg, storage, nchan, nx, ny, cells, depth, fwhm, nsig, pix):
    hz = 10.0 if pix < 1.0 else 1.0
    f = synth.drift_field(71, width=nx * pix * AM * 1.15, height=ny * pix * AM * 1.15, hz=hz, passes=2 if hz > 1 else 3,
                          nchan=nchan, nx=nx, ny=ny, pix=pix * AM, fwhm=fwhm * AM, nsig=nsig, nsrc=5)
    g, cube, w = _run(hcg, f, storage, cells, depth)
    cnt = _check(f, storage, cube, w)
    assert g.info()["pairs"] == cnt.sum()
    if nsig == 4.0:
        assert cnt.max() > 1000


@pytest.mark.parametrize("lon0,lat0", [(0.0, 10.0), (359.95, -8.0), (45.0, 62.0)])
def test_staged_seam_and_high_latitude(hcg, lon0, lat0):
    f = synth.uniform_field(seed=72, n=9000, width=0.9, height=0.7, lon0=lon0, lat0=lat0, nx=45, ny=33,
                            nchan=256, fwhm=2.0 * AM, nsig=4.0)
    lon = f.lon % 360.0        # samples given in [0, 360) across the seam
    g, cube, w = _run(hcg, f, lon=lon)
    cnt = _check(f, "f32", cube, w, lon=lon)
    assert g.info()["pairs"] == cnt.sum()


def test_staged_tile_shapes_and_depths_agree(hcg):
    """Every (cells per block, depth) sums each (cell, channel) over the same
    candidates in S' order: the values agree to rounding of the weights."""
    f = synth.drift_field(73, width=0.45, height=0.4, hz=1.0, passes=3, nchan=512, nx=25, ny=22, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    spec = f.spectra(device="cuda")
    outs = [_run(hcg, f, cells=c, depth=d, spec=spec)[1:] for c in (32, 64) for d in (16, 32)]
    c0, w0 = outs[0]
    for c1, w1 in outs[1:]:
        assert np.array_equal(np.isnan(c0), np.isnan(c1))
        ok = w0 > 0
        np.testing.assert_allclose(w1[ok], w0[ok], rtol=2e-6)
        assert np.abs(c1[ok] - c0[ok]).max() <= 2e-6 * np.abs(c0[ok]).max()


def test_staged_and_gather_paths_agree(hcg):
    f = synth.drift_field(74, width=0.5, height=0.4, hz=1.0, passes=3, nchan=1024, nx=28, ny=22, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    spec = f.spectra(device="cuda")
    g1, cs, ws = _run(hcg, f, spec=spec)
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.set_tuning(path=hcg.PATH_GATHER)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), spec)
    g.grid()
    cg, wg = g.fetch()
    cg = cg.reshape(f.cells, -1); wg = wg.ravel()
    assert g1.info()["pairs"] == g.info()["pairs"]
    ok = wg > 0
    assert np.array_equal(np.isnan(cs), np.isnan(cg))
    np.testing.assert_allclose(ws[ok], wg[ok], rtol=2e-6)
    assert np.abs(cs[ok] - cg[ok]).max() <= 2e-6 * np.abs(cg[ok]).max()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_staged_streamed_windows_bit_identical(hcg, storage):
    f = synth.drift_field(75, width=0.4, height=0.35, hz=1.0, passes=3, nchan=768, nx=22, ny=19, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    spec = f.spectra(device="cpu").contiguous()
    g = _gridder(hcg, f, storage)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), spec.cuda())
    g.grid()
    c0, w0 = g.fetch()
    gs = _gridder(hcg, f, storage)
    gs.set_stream_chunk(256)
    gs.load_samples(f.lon, f.lat, spec.pin_memory(), stream=True)
    for _ in range(2):
        gs.grid()
        c1, w1 = gs.fetch()
        assert np.array_equal(c0, c1, equal_nan=True) and np.array_equal(w0, w1)
    assert gs.info()["path"] == hcg.PATH_STAGED and gs.info()["stream_window"] == 256


def test_staged_field_in_a_batch(hcg):
    fields = [synth.drift_field(76 + k, width=0.35, height=0.3, hz=1.0, passes=3, nchan=c, nx=20, ny=17,
                                pix=AM, fwhm=1.5 * AM, nsig=3.0, nsrc=3, dtype=dt)
              for k, (c, dt) in enumerate([(256, "f32"), (64, "f32"), (512, "bf16")])]
    singles, gs = [], []
    stream = torch.cuda.Stream()
    batch = hcg.Batch(0, stream)
    for k, f in enumerate(fields):
        for target in (singles, gs):
            g = hcg.Gridder(0, stream if target is gs else None)
            g.set_kernel(f.fwhm, f.support)
            g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
            g.set_storage(f.dtype)
            if k != 1:
                g.set_tuning(path=hcg.PATH_STAGED)
            g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), f.spectra(device="cuda"))
            if target is singles:
                g.grid()
                singles.append(g.fetch())
            else:
                batch.add(g)
                gs.append(g)
    torch.cuda.synchronize()
    for _ in range(2):
        batch.grid()
        batch.sync()
        for f, g, (c1, w1) in zip(fields, gs, singles):
            c2, w2 = g.fetch()
            assert np.array_equal(c1, c2, equal_nan=True) and np.array_equal(w1, w2), f.name
    assert gs[0].info()["path"] == hcg.PATH_STAGED and gs[1].info()["path"] == hcg.PATH_GATHER


def test_staged_refuses_what_it_cannot_grid(hcg):
    f = synth.uniform_field(seed=77, n=500, width=0.2, height=0.2, nx=8, ny=8, nchan=100)
    lon, lat = torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda()
    for nchan in (100, 130):          # fewer than 128 channels; 130 FP32 rows are not 16-byte multiples
        g = _gridder(hcg, f)
        g.load_samples(lon, lat, torch.ones((f.n, nchan), device="cuda"))
        with pytest.raises(hcg.HcgError, match="UNSUPPORTED"):
            g.grid()
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny, projection=hcg.WCS_TAN)
    g.set_tuning(path=hcg.PATH_STAGED)
    g.load_samples(lon, lat, torch.ones((f.n, 256), device="cuda"))
    with pytest.raises(hcg.HcgError, match="UNSUPPORTED"):
        g.grid()

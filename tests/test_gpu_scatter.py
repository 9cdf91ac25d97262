"""The scattering strategy of Sec. 2.2 (HCG_PATH_SCATTER): every sample adds
its weighted value to the cells whose support holds it, with atomic adds.
The FP64 oracle (Eq. 1) checks it like the gather; the sums run in an order
the hardware picks, so the comparison is within the FP32 tolerance."""
import numpy as np
import pytest
import torch

import oracle
import oracle.quant as Q
from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0


def _scatter(hcg, f, spec=None, storage=None, stream=False, chunk=0):
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    if storage:
        g.set_storage(storage)
    g.set_tuning(path=hcg.PATH_SCATTER)
    s = f.spectra(device="cpu" if stream else "cuda") if spec is None else spec
    if stream:
        g.set_stream_chunk(chunk)
        g.load_samples(f.lon, f.lat, s.contiguous(), stream=True)
    else:
        g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), s)
    g.grid()
    cube, w = g.fetch()
    return g, cube.reshape(f.cells, -1), w.ravel()


def _check(cube, w, v, wr, ab, cnt, tol):
    ok = cnt > 0
    assert np.all(np.isnan(cube[~ok])) and np.all(w[~ok] == 0)
    err = np.abs(cube[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])
    assert err.max() <= tol, err.max()
    assert np.abs(w[ok] - wr[ok]).max() <= 1e-5 * wr[ok].max()


def _fields():
    yield synth.workload("uniform-20k")
    yield synth.drift_field(41, width=0.5, height=0.45, hz=1.0, passes=3, nchan=1000, nx=31, ny=29, pix=AM,
                            fwhm=1.5 * AM, nsig=3.0, nsrc=6, name="drift-1000")
    yield synth.uniform_field(seed=42, n=6000, width=1.0, height=0.8, lon0=359.95, lat0=-5.0, nx=40, ny=31,
                              nchan=3, name="seam")
    yield synth.uniform_field(seed=43, n=8000, width=3.0, height=0.5, lon0=20.0, lat0=86.5, nx=16, ny=25,
                              pix=AM, fwhm=1.5 * AM, nsig=3.0, nchan=5, name="near-pole")


@pytest.mark.parametrize("f", list(_fields()), ids=lambda f: f.name)
def test_scatter_against_oracle(hcg, f):
    g, cube, w = _scatter(hcg, f)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, f.spectra_np())
    _check(cube, w, v, wr, ab, cnt, 1e-5)
    inf = g.info()
    assert inf["pairs"] == cnt.sum() and inf["path"] == hcg.PATH_SCATTER


@pytest.mark.parametrize("storage", ["bf16", "e4m3"])
def test_scatter_quantised(hcg, storage):
    f = synth.drift_field(44, width=0.45, height=0.4, hz=1.0, passes=3, nchan=256, nx=24, ny=22, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=6)
    x = f.spectra_np()
    _, cube, w = _scatter(hcg, f, storage=storage)
    if storage == "bf16":
        deq = Q.bf16_bits_to_f32(Q.bf16_round_bits(x)).astype(np.float64)
    else:
        codes, s = Q.e4m3_quantise(x)
        deq = Q.e4m3_dequantise(codes, s)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, deq)
    _check(cube, w, v, wr, ab, cnt, 1e-5)


def test_scatter_streamed_windows(hcg):
    """Windows of channels: weights summed once, each window scattered into
    its channel range."""
    f = synth.drift_field(45, width=0.4, height=0.35, hz=1.0, passes=3, nchan=640, nx=22, ny=19, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    g, cube, w = _scatter(hcg, f, stream=True, chunk=256)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, f.spectra_np())
    _check(cube, w, v, wr, ab, cnt, 1e-5)
    assert g.info()["pairs"] == cnt.sum()


def test_scatter_has_no_tables(hcg):
    f = synth.workload("uniform-20k")
    g, _, _ = _scatter(hcg, f)
    with pytest.raises(hcg.HcgError):
        g.debug_pix()

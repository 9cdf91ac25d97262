"""The autotuner times every applicable (cells per block, channels per thread,
tile depth, path) -- several values of each -- keeps the fastest, gives
results within the chosen path's tolerance of the FP64 oracle, and reuses
its cached choice for a field with the same key, also for fields left on the
automatic path and for batches."""
import numpy as np
import pytest
import torch

import oracle
from oracle import quant as Q
from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0


def _g(hcg, f, storage="f32", stream=None):
    g = hcg.Gridder(0, stream)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.set_storage(storage)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), f.spectra(device="cuda"))
    return g


def _against_oracle(hcg, f, storage, g):
    cube, w = g.fetch()
    cube = cube.reshape(f.cells, -1); w = w.ravel()
    x = f.spectra_np()
    if storage == "bf16":
        x = Q.bf16_bits_to_f32(Q.bf16_round_bits(x))
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, x.astype(np.float64))
    ok = cnt > 0
    assert np.all(np.isnan(cube[~ok])) and np.all(w[~ok] == 0)
    tol = 1.25 * 2.0 ** -9 + 2e-6 if g.info()["path"] == hcg.PATH_TENSOR else 1e-5
    err = np.abs(cube[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])
    assert err.max() <= tol, (g.info()["path"], err.max())
    assert (np.abs(w[ok] - wr[ok]) / wr[ok]).max() <= 1e-5
    assert g.info()["pairs"] == cnt.sum()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_autotune_times_every_parameter_and_keeps_results(hcg, storage):
    f = synth.drift_field(61, width=0.5, height=0.45, hz=1.0, passes=3, nchan=512, nx=28, ny=25, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    g = _g(hcg, f, storage)
    choice = g.autotune(force=True)
    table = g.autotune_table()
    timed = [c for c, ms in table if ms > 0]
    # several values of each parameter were timed, on more than one path
    assert len({c[0] for c in timed}) >= 3 and len({c[1] for c in timed}) >= 2
    assert len({c[2] for c in timed}) >= 3 and len({c[3] for c in timed}) >= 2
    if storage == "bf16":
        assert any(c[3] == hcg.PATH_TENSOR for c in timed)
    assert any(c[3] == hcg.PATH_STAGED for c in timed)
    # the choice is the fastest candidate, and it is applied
    best = min(table, key=lambda t: t[1] if t[1] > 0 else 1e30)[0]
    assert (choice["cells_per_block"], choice["chans_per_thread"], choice["tile_depth"], choice["path"]) == best
    g.grid()
    assert g.info()["path"] == choice["path"]
    _against_oracle(hcg, f, storage, g)
    # every candidate it could choose is correct as well
    for (cells, vc, depth, path), ms in table:
        h = _g(hcg, f, storage)
        h.set_tuning(cells_per_block=cells, chans_per_thread=vc, tile_depth=depth, path=path)
        h.grid()
        _against_oracle(hcg, f, storage, h)
    # same key: the cached answer, no timing runs
    g2 = _g(hcg, f, storage)
    assert g2.autotune() == choice
    # a field left on the automatic path runs the cached choice
    g3 = _g(hcg, f, storage)
    g3.grid()
    assert g3.info()["path"] == choice["path"]


def test_batch_takes_the_tuned_choice(hcg):
    f = synth.drift_field(62, width=0.45, height=0.4, hz=1.0, passes=3, nchan=256, nx=25, ny=22, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    choice = _g(hcg, f).autotune(force=True)
    single = _g(hcg, f)
    single.grid()
    c1, w1 = single.fetch()
    stream = torch.cuda.Stream()
    b = hcg.Batch(0, stream)
    gb = _g(hcg, f, stream=stream)
    b.add(gb)
    torch.cuda.synchronize()
    b.grid()
    b.sync()
    c2, w2 = gb.fetch()
    assert gb.info()["path"] == choice["path"] == single.info()["path"]
    assert np.array_equal(c1, c2, equal_nan=True) and np.array_equal(w1, w2)

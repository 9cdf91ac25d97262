"""Streamed spectra (HCG_MEM_HOST_STREAM): host rows copied window by window
of channels inside hcg_grid, each copy overlapping the gather of the window
before it.  Every channel accumulates in the same order as with
device-resident spectra, so the results must be bit-identical; the oracle
(Eq. 1 in FP64) checks one streamed case directly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0


def _field(nchan, seed=31):
    return synth.drift_field(seed, width=0.4, height=0.35, hz=1.0, passes=3, nchan=nchan, nx=22, ny=19, pix=AM,
                             fwhm=1.5 * AM, nsig=3.0, nsrc=4)


def _gridder(hcg, f, storage="f32", path=None):
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.set_storage(storage)
    if path is not None:
        g.set_tuning(path=path)
    return g


def _resident(hcg, f, spec, storage="f32", path=None):
    g = _gridder(hcg, f, storage, path)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), spec.cuda())
    g.grid()
    c, w = g.fetch()
    return c, w, g.info()


def _streamed(hcg, f, spec_host, chunk, storage="f32", path=None, repeats=1):
    g = _gridder(hcg, f, storage, path)
    g.set_stream_chunk(chunk)
    g.load_samples(f.lon, f.lat, spec_host, stream=True)
    out = []
    for _ in range(repeats):
        g.grid()
        c, w = g.fetch()
        out.append((c, w))
    return out, g.info()


@pytest.mark.parametrize("nchan,chunk", [(1000, 256), (1024, 0), (512, 128)])
def test_streamed_f32_bit_identical(hcg, nchan, chunk):
    f = _field(nchan)
    spec = f.spectra(device="cpu").contiguous()
    c0, w0, i0 = _resident(hcg, f, spec)
    out, i1 = _streamed(hcg, f, spec.pin_memory(), chunk, repeats=2)
    for c1, w1 in out:
        assert np.array_equal(c0, c1, equal_nan=True) and np.array_equal(w0, w1)
    assert i1["pairs"] == i0["pairs"] and i1["path"] == i0["path"]


@pytest.mark.parametrize("storage", ["bf16", "e4m3"])
def test_streamed_quantised_bit_identical(hcg, storage):
    """F32 host rows quantised on the device window by window: BF16 is per
    element, the E4M3 scales per channel, so the windows change nothing."""
    f = _field(768, seed=32)
    spec = f.spectra(device="cpu").contiguous()
    c0, w0, _ = _resident(hcg, f, spec, storage=storage, path=hcg.PATH_GATHER)
    (res,), _ = _streamed(hcg, f, spec.pin_memory(), 256, storage=storage, path=hcg.PATH_GATHER)
    assert np.array_equal(c0, res[0], equal_nan=True) and np.array_equal(w0, res[1])


def test_streamed_tensor_path_bit_identical(hcg):
    """Windows of 512 keep the tensor path's 512-channel slices (its weight
    sums depend on the slice width's thread split)."""
    f = _field(1024, seed=33)
    spec = f.spectra(device="cpu").contiguous()
    c0, w0, i0 = _resident(hcg, f, spec, storage="bf16", path=hcg.PATH_TENSOR)
    (res,), i1 = _streamed(hcg, f, spec.pin_memory(), 512, storage="bf16", path=hcg.PATH_TENSOR)
    assert i0["path"] == i1["path"] == hcg.PATH_TENSOR
    assert np.array_equal(c0, res[0], equal_nan=True) and np.array_equal(w0, res[1])
    assert i1["pairs"] == i0["pairs"]


def test_streamed_pageable_against_oracle(hcg):
    """Pageable numpy rows (synchronous copies) against the FP64 oracle."""
    f = _field(300, seed=34)
    spec = f.spectra_np()
    (res,), info = _streamed(hcg, f, spec.astype(np.float32), 128)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, spec)
    cube = res[0].reshape(f.cells, -1)
    w = res[1].ravel()
    ok = cnt > 0
    assert np.all(np.isnan(cube[~ok])) and np.all(w[~ok] == 0)
    err = np.abs(cube[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])
    assert err.max() <= 1e-5
    assert np.abs(w[ok] - wr[ok]).max() <= 1e-5 * wr[ok].max()
    assert info["pairs"] == cnt.sum()


def test_streamed_refused_by_autotune_and_batch(hcg):
    f = _field(256, seed=35)
    st = torch.cuda.Stream()
    g = hcg.Gridder(0, st)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.load_samples(f.lon, f.lat, f.spectra(device="cpu").contiguous(), stream=True)
    with pytest.raises(hcg.HcgError):
        g.autotune(force=True)
    b = hcg.Batch(0, st)
    b.add(g)
    with pytest.raises(hcg.HcgError):
        b.grid()
    b.close()


@pytest.mark.parametrize("stream", [True, False])
def test_host_output_delivery(hcg, stream):
    """hcg_bind_host_output: grid() fills pinned host buffers (window by
    window when streamed) with exactly what fetch() returns, on every call."""
    f = _field(1024, seed=36)
    spec = f.spectra(device="cpu").contiguous().pin_memory()
    g = _gridder(hcg, f)
    g.set_stream_chunk(256)
    cube_h = torch.full((f.ny, f.nx, f.nchan), -1.0).pin_memory()
    w_h = torch.full((f.ny, f.nx), -1.0).pin_memory()
    g.bind_host_output(cube_h, w_h)
    if stream:
        g.load_samples(f.lon, f.lat, spec, stream=True)
    else:
        g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), spec.cuda())
    for _ in range(2):
        cube_h.fill_(-1.0)
        g.grid()
        g.sync()
        c, w = g.fetch()
        assert np.array_equal(cube_h.numpy(), c, equal_nan=True) and np.array_equal(w_h.numpy(), w)
    g.bind_host_output(None, None)

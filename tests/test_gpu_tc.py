"""GPU parity of the tensor-core blocked path (tcgen05, BF16 / FP8 storage)
against the FP64 oracle, through the C ABI.

Tolerances (condition-aware, per value, scale |V| + sum w |s| / W):
* against the oracle on the dequantised spectra: the MMA multiplies weights
  rounded to BF16 (relative error <= 2^-9) or FP16 (<= 2^-11) and divides by
  the sum of the same rounded weights, so to first order
  |dV| <= u * (|V| + sum w |s| / W) with u the weight unit roundoff; the
  bound used is 1.25 u (FP32 accumulation adds ~1e-6);
* against the oracle on the unquantised FP32 spectra: 4e-3 (BF16) and 3e-2
  (FP8), the stated accuracy targets;
* weights (sum of unrounded FP32 weights): 1e-5 relative; pair counts exact."""
import numpy as np
import pytest
import torch

import oracle
from oracle import quant as Q
from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0


def _run(hcg, f, storage, path):
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.set_storage(storage)
    g.set_tuning(path=path)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), f.spectra(device="cuda"))
    g.grid()
    cube, w = g.fetch()
    return g, cube.reshape(f.cells, -1), w.ravel()


def _err(cube, v, ab, ok):
    return np.abs(cube[ok] - v[ok]) / (np.abs(v[ok]) + ab[ok])


@pytest.mark.parametrize("storage,nchan,nx,ny,nsig,fwhm,pix", [
    ("bf16", 512, 37, 21, 3.0, 1.2, 0.6),     # 512-channel slices, ragged tiles
    ("bf16", 256, 16, 8, 3.0, 1.2, 0.6),      # exactly one tile
    ("bf16", 768, 23, 30, 4.0, 3.0, 0.6),     # three 256 slices, wide kernel
    ("e4m3", 256, 40, 17, 4.0, 3.0, 0.6),
    ("e4m3", 512, 19, 26, 3.0, 1.2, 0.6),
])
def test_tensor_path_matches_oracle(hcg, storage, nchan, nx, ny, nsig, fwhm, pix):
    f = synth.drift_field(41, width=nx * pix * AM * 1.15, height=ny * pix * AM * 1.15, hz=10.0, passes=1,
                          nchan=nchan, nx=nx, ny=ny, pix=pix * AM, fwhm=fwhm * AM, nsig=nsig, nsrc=6)
    g, cube, w = _run(hcg, f, storage, hcg.PATH_TENSOR)
    assert g.info()["path"] == hcg.PATH_TENSOR
    x = f.spectra_np()
    if storage == "bf16":
        deq = Q.bf16_bits_to_f32(Q.bf16_round_bits(x)).astype(np.float64)
        u, tol = 2.0 ** -9, 4e-3
    else:
        codes, s = Q.e4m3_quantise(x)
        deq = Q.e4m3_dequantise(codes, s)
        u, tol = 2.0 ** -11, 3e-2
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, deq)
    ok = cnt > 0
    assert np.all(np.isnan(cube[~ok])) and np.all(w[~ok] == 0)
    assert (np.abs(w[ok] - wr[ok]) / wr[ok]).max() <= 1e-5, "per-cell weight error"
    e1 = _err(cube, v, ab, ok)
    assert e1.max() <= 1.25 * u + 2e-6, f"vs dequantised oracle {e1.max():.3e}"
    v2, _, ab2, _ = oracle.grid_cells(f.geom(), f.lon, f.lat, x)
    e2 = _err(cube, v2, ab2, ok)
    assert e2.max() <= tol, f"vs FP32 oracle {e2.max():.3e}"
    assert g.info()["pairs"] == cnt.sum()


def test_tensor_and_gather_paths_agree(hcg):
    f = synth.drift_field(42, width=0.5, height=0.4, hz=10.0, passes=1, nchan=512, nx=40, ny=32, pix=0.6 * AM,
                          fwhm=1.2 * AM, nsig=3.0, nsrc=5)
    gt, ct, wt = _run(hcg, f, "bf16", hcg.PATH_TENSOR)
    gg, cg, wg = _run(hcg, f, "bf16", hcg.PATH_GATHER)
    # issued MMA work: whole chunks of 128 cells x 64 candidates x 512 channels
    # (512-channel slices: no ones column); none on the CUDA cores
    tf = gt.info()["tensor_flops"]
    assert tf > 0 and tf % (2 * 128 * 64 * 512) == 0
    assert gg.info()["tensor_flops"] == 0
    ok = wg > 0
    assert np.array_equal(np.isnan(ct), np.isnan(cg))
    np.testing.assert_allclose(wt, wg, rtol=2e-6)
    scale = np.abs(cg[ok]).max()
    assert np.abs(ct[ok] - cg[ok]).max() <= 2.0 ** -8 * scale


def test_auto_path_choice(hcg):
    f = synth.drift_field(43, width=0.3, height=0.3, hz=10.0, passes=1, nchan=256, nx=20, ny=20, pix=0.6 * AM,
                          fwhm=1.2 * AM, nsig=3.0, nsrc=3)
    g, _, _ = _run(hcg, f, "bf16", hcg.PATH_AUTO)
    assert g.info()["path"] == hcg.PATH_TENSOR
    g, _, _ = _run(hcg, f, "f32", hcg.PATH_AUTO)
    assert g.info()["path"] == hcg.PATH_GATHER


def test_bounded_wait_gives_up_and_context_recovers(hcg):
    """The give-up path of the tensor path's bounded mbarrier waits: with the
    probe on, every CTA first waits on a barrier that nothing completes; the
    wait runs out after the (short) limit, the CTA skips its tensor-core work
    and finishes, and the pass reports TIMEOUT.  Nothing hangs, and the same
    context then grids the field correctly with the probe off."""
    f = synth.drift_field(44, width=0.25, height=0.2, hz=10.0, passes=1, nchan=256, nx=18, ny=14, pix=0.6 * AM,
                          fwhm=1.2 * AM, nsig=3.0, nsrc=3)
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.set_storage("bf16")
    g.set_tuning(path=hcg.PATH_TENSOR)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), f.spectra(device="cuda"))
    g.set_wait_limit(200_000, probe=True)          # 0.2 ms
    g.grid()
    with pytest.raises(hcg.HcgError, match="TIMEOUT"):
        g.sync()
    g.set_wait_limit(probe=False)
    g.grid()
    cube, w = g.fetch()
    cube = cube.reshape(f.cells, -1); w = w.ravel()
    x = f.spectra_np()
    deq = Q.bf16_bits_to_f32(Q.bf16_round_bits(x)).astype(np.float64)
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, deq)
    ok = cnt > 0
    assert (_err(cube, v, ab, ok)).max() <= 1.25 * 2.0 ** -9 + 2e-6
    assert (np.abs(w[ok] - wr[ok]) / wr[ok]).max() <= 1e-5


@pytest.mark.parametrize("nchan,nx,ny,nsig,fwhm,pix", [
    (256, 20, 11, 3.0, 1.2, 0.6),       # ragged tiles
    (512, 17, 19, 4.0, 3.0, 0.6),       # two 256-channel slices, wide kernel
    (768, 9, 9, 3.0, 1.2, 0.6),         # three slices, one partial tile
])
def test_tensor_path_fp32_split_tf32(hcg, nchan, nx, ny, nsig, fwhm, pix):
    """FP32 storage on the tensor path: weights and spectra split into TF32
    heads and remainders, three products summed in FP32.  Held to the FP32
    tolerance of the CUDA-core gather (1e-5 condition-aware, weights 1e-5
    per cell) against the FP64 oracle, with exact pair counts."""
    f = synth.drift_field(45, width=nx * pix * AM * 1.15, height=ny * pix * AM * 1.15, hz=10.0, passes=1,
                          nchan=nchan, nx=nx, ny=ny, pix=pix * AM, fwhm=fwhm * AM, nsig=nsig, nsrc=6)
    g, cube, w = _run(hcg, f, "f32", hcg.PATH_TENSOR)
    assert g.info()["path"] == hcg.PATH_TENSOR
    v, wr, ab, cnt = oracle.grid_cells(f.geom(), f.lon, f.lat, f.spectra_np())
    ok = cnt > 0
    assert np.all(np.isnan(cube[~ok])) and np.all(w[~ok] == 0)
    assert (np.abs(w[ok] - wr[ok]) / wr[ok]).max() <= 1e-5
    e = _err(cube, v, ab, ok)
    assert e.max() <= 1e-5, f"vs FP64 oracle {e.max():.3e}"
    assert g.info()["pairs"] == cnt.sum()

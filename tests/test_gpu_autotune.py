"""The autotuner picks among layouts/paths that all give the same results
(bit-identical CUDA-core layouts; the tensor path within its tolerance),
and reuses its cached choice for a field with the same key."""
import numpy as np
import pytest
import torch

from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0


def _g(hcg, f, storage="f32"):
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.set_storage(storage)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), f.spectra(device="cuda"))
    return g


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_autotune_keeps_results(hcg, storage):
    f = synth.drift_field(61, width=0.5, height=0.45, hz=1.0, passes=3, nchan=512, nx=28, ny=25, pix=AM,
                          fwhm=1.5 * AM, nsig=3.0, nsrc=4)
    ref = _g(hcg, f, storage)
    ref.set_tuning(path=hcg.PATH_GATHER)
    ref.grid()
    c0, w0 = ref.fetch()
    g = _g(hcg, f, storage)
    choice = g.autotune(force=True)
    g.grid()
    c1, w1 = g.fetch()
    assert g.info()["path"] == choice["path"]
    if choice["path"] == hcg.PATH_GATHER:
        assert np.array_equal(c0, c1, equal_nan=True) and np.array_equal(w0, w1)
    else:
        ok = w0 > 0
        assert np.abs(c1[ok] - c0[ok]).max() <= 2.0 ** -8 * np.abs(c0[ok]).max()
    # same key: cached, no timing runs
    g2 = _g(hcg, f, storage)
    assert g2.autotune() == choice

"""hcg_preorder_noalloc, the pre-ordering entry point for callers that cannot
allocate device memory: real-time pipelines that reserve all their device
memory at start-up and forbid allocation afterwards, and host programs whose
device memory belongs to another runtime's pool.  It must reproduce, bit for
bit, the sorted pixels and permutation that hcg_grid's own pre-ordering
produces (read back through hcg_debug_pix), on consecutive calls that share
its fixed scratch.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2012_13173_gb300 import synth

pytestmark = pytest.mark.gpu
AM = 1.0 / 60.0
INT64_MAX = np.iinfo(np.int64).max


def _reference(hcg, f):
    g = hcg.Gridder(0)
    g.set_kernel(f.fwhm, f.support)
    g.set_grid(f.lon0, f.lat0, f.pix, f.nx, f.ny)
    g.load_samples(torch.from_numpy(f.lon).cuda(), torch.from_numpy(f.lat).cuda(), f.spectra(device="cuda"))
    g.grid()
    ps, perm = g.debug_pix()
    return ps, perm, g.info()


def _noalloc(hcg, f, info):
    lon = torch.from_numpy(f.lon).cuda()
    lat = torch.from_numpy(f.lat).cuda()
    out_p = torch.full((f.n,), -7, dtype=torch.int64, device="cuda")
    out_v = torch.full((f.n,), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    hcg.preorder_noalloc(lon, lat, info["nside"], info["ring_lo"], info["ring_hi"], out_p, out_v)
    torch.cuda.synchronize()
    return out_p.cpu().numpy(), out_v.cpu().numpy().view(np.uint32).astype(np.int64)


def test_noalloc_preorder_matches_grid_on_consecutive_calls(hcg):
    fields = [
        synth.workload("uniform-20k"),
        # samples well beyond the grid in latitude: some are dropped
        synth.uniform_field(seed=51, n=30000, width=1.0, height=1.6, lon0=10.0, lat0=-20.0, nx=40, ny=40,
                            name="dropping"),
        synth.workload("uniform-20k"),
    ]
    kept = []
    for f in fields:
        ps, perm, info = _reference(hcg, f)
        m = info["samples_kept"]
        kept.append(m)
        p2, v2 = _noalloc(hcg, f, info)
        assert np.array_equal(p2[:m], ps)
        assert np.array_equal(v2[:m], perm)
        assert np.all(p2[m:] == INT64_MAX)
        # every input index appears exactly once
        assert np.array_equal(np.sort(v2), np.arange(f.n))
    assert kept[1] < fields[1].n and kept[0] == fields[0].n


def test_noalloc_rejects_oversized_input(hcg):
    n = 262144 + 1
    lon = torch.zeros(n, dtype=torch.float64, device="cuda")
    out_p = torch.empty(n, dtype=torch.int64, device="cuda")
    out_v = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(hcg.HcgError, match="INVALID_ARG.*262144"):
        hcg.preorder_noalloc(lon, lon, 16384, 1000, 2000, out_p, out_v)

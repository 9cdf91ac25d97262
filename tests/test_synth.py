"""The seeded generator: deterministic, the stated sizes, and an integer
noise stream that matches a plain uint64 restatement of its hash."""
import math

import numpy as np

from paper_2012_13173_gb300 import synth


def _fmix(k):
    with np.errstate(over="ignore"):
        k = k ^ (k >> np.uint64(33)); k = k * np.uint64(0xFF51AFD7ED558CCD)
        k = k ^ (k >> np.uint64(33)); k = k * np.uint64(0xC4CEB9FE1A85EC53)
        k = k ^ (k >> np.uint64(33))
    return k


def test_noise_matches_uint64_restatement():
    f = synth.workload("drift-1M-c1024", scale=0.05)
    rows = np.array([0, 5, 17, f.n - 1])
    s = f.spectra_np(rows, 3, 40)
    seedmix = np.uint64((f.seed * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) & ((1 << 64) - 1))
    ctr = (rows[:, None].astype(np.uint64) * np.uint64(f.nchan) + np.arange(3, 40, dtype=np.uint64)[None, :])
    x = _fmix(ctr ^ seedmix)
    tot = sum(((x >> np.uint64(sh)) & np.uint64(0xFFFF)).astype(np.int64) for sh in (0, 16, 32, 48))
    nz = (tot.astype(np.float32) * np.float32(1 / 65536.0) - np.float32(2.0)) * np.float32(f.noise_sigma * math.sqrt(3.0))
    sky = (f.b1[rows, None] * f.prof[f.k1[rows]][:, 3:40]) + (f.b2[rows, None] * f.prof[f.k2[rows]][:, 3:40])
    assert np.array_equal(s, (sky.astype(np.float32) + nz).astype(np.float32))


def test_deterministic_and_sizes():
    a = synth.workload("uniform-20k")
    b = synth.workload("uniform-20k")
    assert a.n == 20000 and a.nchan == 1 and (a.nx, a.ny) == (120, 120)
    assert np.array_equal(a.lon, b.lon) and np.array_equal(a.spectra_np(), b.spectra_np())
    f = synth.workload("drift-1M-c1024", scale=0.1)
    assert f.n == 4 * 19 * 120 and f.nx == 30
    # full-size drift-scan layouts from the stated track counts and rates
    assert 44 * 19 * 1200 == 1003200 and 15 * 19 * 14400 == 4104000 and 35 * 19 * 24000 == 15960000


def test_noise_moments():
    f = synth.drift_field(9, width=2.0, height=2.0, hz=0.2, passes=1, nchan=64, nx=4, ny=4,
                          pix=0.02, fwhm=0.02, nsig=3.0, nsrc=2)
    far = np.nonzero((f.b1 < 1e-6) & (f.b2 < 1e-6))[0][:200]
    assert far.size == 200
    s = f.spectra_np(far)
    assert abs(s.mean()) < 0.01 and abs(s.std() - 0.1) < 0.005

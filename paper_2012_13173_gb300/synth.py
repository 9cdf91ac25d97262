"""Seeded synthetic inputs for the gridding workloads.

This module holds input generation only -- none of the gridding arithmetic.
It serves both the CUDA path (benchmarks, GPU tests) and the FP64 oracle, so
that both see the same samples.

Coordinates are FP64 numpy arrays made on the host from
``numpy.random.Generator(PCG64(seed))``.  Spectra are defined per
(sample, channel) and can be produced for any subset of rows and channels,
on the CPU or on a CUDA device, with bit-identical FP32 results on both:

    s[n, c] = b1[n] * P[k1[n], c] + b2[n] * P[k2[n], c] + noise(n, c)

``b1, b2`` are the beam responses of the two sources nearest to sample n
(FP32, computed once on the host), ``P[k, c]`` is source k's spectrum (a flat
continuum plus one Gaussian line, FP32, host), and ``noise`` is an
Irwin-Hall(4) approximation of N(0, sigma^2) drawn from a counter-based hash
(MurmurHash3's fmix64 finaliser) of (seed, n, c).  Every step after the host
tables is an elementwise IEEE operation or integer arithmetic, so the CPU
and GPU give identical values.

The paper's own test data are simulated the same way in spirit (Gaussian
random values at uniformly random positions, following Cygrid; point-source
maps for its correctness figures) but are not published, so these recipes
stand in for them.  The drift-scan layout follows the FAST 19-beam receiver:
scan rows of constant declination, beams 1'09" apart in declination, the sky
drifting 15" of right ascension per second.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

ARCMIN = 1.0 / 60.0
ARCSEC = 1.0 / 3600.0
_M64 = (1 << 64) - 1


@dataclasses.dataclass
class Field:
    """One gridding problem: samples, sky model and target grid."""
    name: str
    lon: np.ndarray            # [N] degrees, FP64
    lat: np.ndarray            # [N] degrees, FP64
    nchan: int
    lon0: float                # grid centre, degrees
    lat0: float
    pix: float                 # cell size, degrees
    nx: int
    ny: int
    fwhm: float                # kernel FWHM, degrees
    support: float             # support radius, degrees
    seed: int
    k1: np.ndarray             # [N] int64 nearest source
    k2: np.ndarray             # [N] int64 second-nearest source
    b1: np.ndarray             # [N] float32 beam response of k1
    b2: np.ndarray             # [N] float32 beam response of k2
    prof: np.ndarray           # [K, C] float32 source spectra
    noise_sigma: float
    dtype: str = "f32"         # storage dtype requested for the path

    @property
    def n(self) -> int:
        return int(self.lon.size)

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def geom(self):
        return (self.lon0, self.lat0, self.pix, self.nx, self.ny, self.support, self.fwhm)

    # ------------------------------------------------------------ spectra ---
    def spectra(self, rows=None, c0: int = 0, c1: int | None = None, device="cpu") -> torch.Tensor:
        """FP32 spectra for the given rows (default all) and channels [c0, c1)."""
        c1 = self.nchan if c1 is None else c1
        dev = torch.device(device)
        if rows is None:
            rows_t = torch.arange(self.n, dtype=torch.int64, device=dev)
        else:
            rows_t = torch.as_tensor(np.asarray(rows, np.int64), device=dev)
        prof = torch.from_numpy(self.prof[:, c0:c1]).to(dev)
        k1 = torch.from_numpy(self.k1).to(dev)[rows_t]
        k2 = torch.from_numpy(self.k2).to(dev)[rows_t]
        b1 = torch.from_numpy(self.b1).to(dev)[rows_t]
        b2 = torch.from_numpy(self.b2).to(dev)[rows_t]
        t1 = torch.mul(b1[:, None], prof[k1])
        t2 = torch.mul(b2[:, None], prof[k2])
        s = torch.add(t1, t2)
        del t1, t2
        nz = _noise(self.seed, rows_t, c0, c1, self.nchan, dev)
        nz = torch.mul(nz, torch.tensor(self.noise_sigma * math.sqrt(3.0), dtype=torch.float32, device=dev))
        return torch.add(s, nz)

    def spectra_np(self, rows=None, c0: int = 0, c1: int | None = None) -> np.ndarray:
        return self.spectra(rows, c0, c1, "cpu").numpy()


def _shr(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return torch.bitwise_and(torch.bitwise_right_shift(x, k), (1 << (64 - k)) - 1)


def _s64(v: int) -> int:
    v &= _M64
    return v - (1 << 64) if v >= (1 << 63) else v


def _fmix64(x: torch.Tensor) -> torch.Tensor:
    x = torch.bitwise_xor(x, _shr(x, 33))
    x = torch.mul(x, _s64(0xFF51AFD7ED558CCD))
    x = torch.bitwise_xor(x, _shr(x, 33))
    x = torch.mul(x, _s64(0xC4CEB9FE1A85EC53))
    x = torch.bitwise_xor(x, _shr(x, 33))
    return x


def _noise(seed: int, rows: torch.Tensor, c0: int, c1: int, nchan: int, dev) -> torch.Tensor:
    """Irwin-Hall(4) noise, centred, unit variance / sqrt(3) before scaling."""
    ch = torch.arange(c0, c1, dtype=torch.int64, device=dev)
    ctr = torch.add(torch.mul(rows[:, None], nchan), ch[None, :])
    x = _fmix64(torch.bitwise_xor(ctr, _s64(seed * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019)))
    tot = torch.zeros(x.shape, dtype=torch.int64, device=dev)
    for sh in (0, 16, 32, 48):
        tot = torch.add(tot, torch.bitwise_and(_shr(x, sh) if sh else x, 0xFFFF))
    f = tot.to(torch.float32)
    f = torch.mul(f, 1.0 / 65536.0)
    return torch.sub(f, 2.0)


# ------------------------------------------------------------- sky model ---
def _sources(rng, lon0, lat0, w, h, k, nchan, amp=(1.0, 10.0), lines=True):
    slon = lon0 + rng.uniform(-w / 2, w / 2, k)
    slat = lat0 + rng.uniform(-h / 2, h / 2, k)
    a = rng.uniform(amp[0], amp[1], k)
    c = np.arange(nchan, dtype=np.float64)
    prof = np.empty((k, nchan), np.float64)
    for q in range(k):
        if lines and nchan > 1:
            cont = rng.uniform(0.1, 1.0) * a[q]
            line = rng.uniform(1.0, 5.0) * a[q]
            cen = rng.uniform(0.0, nchan)
            wid = rng.uniform(2.0, 50.0)
            prof[q] = cont + line * np.exp(-0.5 * ((c - cen) / wid) ** 2)
        else:
            prof[q] = a[q]
    return slon, slat, prof.astype(np.float32)


def _unit(lon, lat):
    lo = np.radians(lon); la = np.radians(lat)
    return np.stack([np.cos(la) * np.cos(lo), np.cos(la) * np.sin(lo), np.sin(la)], -1)


def _beam(lon, lat, slon, slat, beam_fwhm):
    """Two nearest sources of each sample and their Gaussian beam responses."""
    n = lon.size
    u = _unit(lon, lat)
    v = _unit(slon, slat)
    sig = math.radians(beam_fwhm) / math.sqrt(8 * math.log(2))
    k1 = np.zeros(n, np.int64); k2 = np.zeros(n, np.int64)
    b1 = np.zeros(n, np.float32); b2 = np.zeros(n, np.float32)
    step = 1 << 20
    for a in range(0, n, step):
        dot = np.clip(u[a:a + step] @ v.T, -1.0, 1.0)
        ang = np.arccos(dot)
        if v.shape[0] >= 2:
            order = np.argsort(ang, axis=1)[:, :2]
        else:
            order = np.zeros((ang.shape[0], 2), np.int64)
        d1 = np.take_along_axis(ang, order[:, :1], 1)[:, 0]
        d2 = np.take_along_axis(ang, order[:, 1:2], 1)[:, 0]
        k1[a:a + step] = order[:, 0]
        k2[a:a + step] = order[:, 1]
        b1[a:a + step] = np.exp(-0.5 * (d1 / sig) ** 2).astype(np.float32)
        b2[a:a + step] = np.exp(-0.5 * (d2 / sig) ** 2).astype(np.float32) if v.shape[0] >= 2 else 0.0
    return k1, k2, b1, b2


def drift_scan(rng, lon0, lat0, width, height, hz, passes, beams=19):
    """Constant-declination scan rows, evenly interleaved in declination.

    ``passes * beams`` rows fill ``height``; along a row the samples are
    15"/hz apart in right ascension, with a random phase per row and
    N(0, 1") jitter on both coordinates.
    """
    tracks = passes * beams
    per_track = int(round(width / (15.0 * ARCSEC / hz)))
    dra = width / per_track
    dec = lat0 - height / 2 + (np.arange(tracks) + 0.5) * (height / tracks)
    phase = rng.uniform(0.0, dra, tracks)
    i = np.arange(per_track, dtype=np.float64)
    lon = (lon0 - width / 2) + phase[:, None] + i[None, :] * dra
    lat = np.repeat(dec[:, None], per_track, axis=1)
    lon = lon + rng.normal(0.0, ARCSEC, lon.shape)
    lat = lat + rng.normal(0.0, ARCSEC, lat.shape)
    return lon.ravel(), lat.ravel()


def make_field(name, *, lon, lat, nchan, lon0, lat0, pix, nx, ny, fwhm, nsig, seed,
               nsrc, beam_fwhm=2.9 * ARCMIN, noise=0.1, lines=True, rng=None, dtype="f32"):
    rng = rng if rng is not None else np.random.default_rng(seed)
    w = nx * pix; h = ny * pix
    slon, slat, prof = _sources(rng, lon0, lat0, w, h, nsrc, nchan, lines=lines)
    k1, k2, b1, b2 = _beam(lon, lat, slon, slat, beam_fwhm)
    sigma = fwhm / math.sqrt(8 * math.log(2))
    return Field(name, np.ascontiguousarray(lon, np.float64), np.ascontiguousarray(lat, np.float64),
                 nchan, lon0, lat0, pix, nx, ny, fwhm, nsig * sigma, seed, k1, k2, b1, b2, prof,
                 noise, dtype)


# ------------------------------------------------------------ workloads ---
def uniform_field(seed=1, n=20000, width=2.0, height=2.0, lon0=180.0, lat0=30.0, nchan=1,
                  nx=120, ny=120, pix=1.0 * ARCMIN, fwhm=1.5 * ARCMIN, nsig=3.0, nsrc=10,
                  name="uniform"):
    """Uniformly random positions with point sources and N(0, 0.1) noise."""
    rng = np.random.default_rng(seed)
    lon = rng.uniform(lon0 - width / 2, lon0 + width / 2, n)
    lat = rng.uniform(lat0 - height / 2, lat0 + height / 2, n)
    return make_field(name, lon=lon, lat=lat, nchan=nchan, lon0=lon0, lat0=lat0, pix=pix,
                      nx=nx, ny=ny, fwhm=fwhm, nsig=nsig, seed=seed, nsrc=nsrc,
                      lines=nchan > 1, rng=rng)


def drift_field(seed, *, width, height, hz, passes, nchan, nx, ny, pix, fwhm, nsig,
                lon0=180.0, lat0=30.0, nsrc=25, name="drift", dtype="f32"):
    rng = np.random.default_rng(seed)
    lon, lat = drift_scan(rng, lon0, lat0, width, height, hz, passes)
    return make_field(name, lon=lon, lat=lat, nchan=nchan, lon0=lon0, lat0=lat0, pix=pix,
                      nx=nx, ny=ny, fwhm=fwhm, nsig=nsig, seed=seed, nsrc=nsrc, rng=rng,
                      dtype=dtype)


def workload(name: str, scale: float = 1.0):
    """The five named workloads; ``scale`` < 1 shrinks the field side (for
    parity cases that the oracle finishes in seconds) at the same density."""
    if name == "uniform-20k":
        return uniform_field()
    if name == "drift-1M-c1024":
        s = scale
        return drift_field(2, width=5.0 * s, height=5.0 * s, hz=1.0, passes=max(1, round(44 * s)),
                           nchan=1024, nx=max(1, round(300 * s)), ny=max(1, round(300 * s)),
                           pix=1.0 * ARCMIN, fwhm=1.5 * ARCMIN, nsig=3.0, name=name)
    if name == "drift-4M-c4096":
        s = scale
        return drift_field(3, width=6.0 * s, height=6.0 * s, hz=10.0, passes=max(1, round(15 * s)),
                           nchan=4096, nx=max(1, round(600 * s)), ny=max(1, round(600 * s)),
                           pix=0.6 * ARCMIN, fwhm=1.2 * ARCMIN, nsig=3.0, name=name)
    if name == "drift-16M-c256":
        s = scale
        return drift_field(5, width=10.0 * s, height=10.0 * s, hz=10.0, passes=max(1, round(35 * s)),
                           nchan=256, nx=max(1, round(1000 * s)), ny=max(1, round(1000 * s)),
                           pix=0.6 * ARCMIN, fwhm=3.0 * ARCMIN, nsig=4.0, name=name)
    raise KeyError(name)


def batch_fields(seed=4, count=64, scale=1.0):
    """64 uneven fields: N log-uniform in [1e4, 2e6], C from {1, 64, 512, 2048},
    square grids of side log-uniform in [50, 500] cells, FWHM U(1', 3'),
    support 3 sigma, cell = FWHM/2, random centres with dec in [-10, 60] deg
    (some straddling RA 0), storage FP32 or BF16 by a coin flip."""
    rng = np.random.default_rng(seed)
    out = []
    for f in range(count):
        n = int(round(math.exp(rng.uniform(math.log(1e4), math.log(2e6))) * scale))
        n = max(n, 64)
        nchan = int(rng.choice([1, 64, 512, 2048]))
        side = int(round(math.exp(rng.uniform(math.log(50), math.log(500))) * math.sqrt(scale)))
        side = max(side, 8)
        fwhm = rng.uniform(1.0, 3.0) * ARCMIN
        pix = fwhm / 2
        ext = side * pix
        lon0 = 0.0 if f % 8 == 0 else rng.uniform(0.0, 360.0)
        lat0 = rng.uniform(-10.0, 60.0)
        dtype = "bf16" if rng.uniform() < 0.5 else "f32"
        # drift-scan rows at the density that gives about n samples
        tracks = max(1, int(round(math.sqrt(n))))
        hz = max(0.05, (n / tracks) * 15.0 * ARCSEC / ext)
        frng = np.random.default_rng(seed * 1000 + f)
        lon, lat = drift_scan(frng, lon0, lat0, ext, ext, hz, 1, beams=tracks)
        fld = make_field(f"batch{f}", lon=lon, lat=lat, nchan=nchan, lon0=lon0, lat0=lat0,
                         pix=pix, nx=side, ny=side, fwhm=fwhm, nsig=3.0, seed=seed * 1000 + f,
                         nsrc=8, rng=frng, dtype=dtype)
        out.append(fld)
    return out

"""The tensor kernels settle the support test of a candidate against a row of
16 cells from the roots of a quadratic in the column index (col_sets in
hcg_tc.cu): t_i = dv2 + a (u - i h)^2 <= b holds exactly for
|u/h - i| <= sqrt((b - dv2) / a) / h.  Columns are "surely inside" (weight
computed), "surely outside" (zero) or in between (sent to the exact FP64
test).  This test restates that classification in FP32 arithmetic -- with
the approximate reciprocal and reciprocal square root perturbed by 2^-21
relative, more than their documented error -- and checks, over random
fields (FWHM 0.5'-5', cells 0.2-1 FWHM, supports 1-5 sigma, latitudes to
88.5 deg), that no column classed inside has t above the lower band edge and
no column classed outside has t at or below the upper one: the fast path
decides only pairs the band analysis says it may."""
import numpy as np

f32 = np.float32


def _col_range(lo, hi):
    # bits of columns i in [0, 16) with lo <= i <= hi (vectorised)
    a = np.clip(np.ceil(np.nan_to_num(lo, nan=1e9, posinf=1e9, neginf=-1e9)), 0, 16).astype(np.int64)
    b = np.clip(np.floor(np.nan_to_num(hi, nan=-1e9, posinf=1e9, neginf=-1e9)), -1, 15).astype(np.int64)
    m = ((0xFFFF << a) & (0xFFFF >> np.clip(15 - b, 0, 16))) & 0xFFFF
    return np.where(a > b, 0, m)


def test_column_interval_classification_is_conservative():
    rng = np.random.default_rng(7)
    n = 200_000
    deg, am = np.pi / 180, np.pi / 180 / 60
    fwhm = rng.uniform(0.5, 5.0, n)
    pix = fwhm * rng.uniform(0.2, 1.0, n)
    nsig = rng.uniform(1.0, 5.0, n)
    sig = fwhm / 2.3548200450309493 * am
    R = nsig * sig
    lat = rng.uniform(-88.5, 88.5, n) * deg
    # the band of the fast estimate, as the launcher sets it
    cmin = np.cos(np.minimum(89.9 * deg, np.abs(lat) + 8 * pix * am + R)) ** 2
    kexp = np.log2(np.e) / (2 * sig * sig)
    pixsz = np.sqrt(np.pi / 3) / 16384
    E = 16 * pix * am + 2 * R / np.sqrt(cmin) + 4 * pixsz
    rel = 1e-5 + R * R / (6 * cmin) + 6 * 2.0 ** -23 * E / (R * np.sqrt(cmin)) + 1e-6
    blo = (f32(kexp) * (R * R * (1 - rel)).astype(f32)).astype(f32)
    bhi = (f32(kexp) * (R * R * (1 + rel)).astype(f32)).astype(f32)
    h = (pix * am).astype(f32)
    invh = (1.0 / (pix * am)).astype(f32)
    cu = rng.uniform(-R / np.sqrt(cmin) - h, 16 * h + R / np.sqrt(cmin)).astype(f32)
    dv = rng.uniform(-1.01 * R, 1.01 * R).astype(f32)
    cgk = (kexp * np.cos(lat)).astype(f32)
    cz = np.cos(lat + rng.uniform(-R, R)).astype(f32)
    dv2 = (kexp.astype(f32) * (dv * dv)).astype(f32)
    ak = (cgk * cz).astype(f32)

    def approx(x):
        return (x * (1 + rng.uniform(-2.0 ** -21, 2.0 ** -21, x.shape))).astype(f32)

    rak = approx((f32(1) / ak).astype(f32))
    Q = ((bhi - dv2) * rak).astype(f32)
    P = ((blo - dv2) * rak).astype(f32)
    x = (cu * invh).astype(f32)
    Qc = np.maximum(Q, f32(1e-30))
    Pc = np.maximum(P, f32(1e-30))
    ro = ((Qc * approx((1 / np.sqrt(Qc.astype(np.float64))).astype(f32))) * invh).astype(f32)
    ri = ((Pc * approx((1 / np.sqrt(Pc.astype(np.float64))).astype(f32))) * invh).astype(f32)
    e = (f32(2e-6) * (np.abs(x) + ro + f32(1))).astype(f32)
    m_pos = np.where(Q > 1e-30, _col_range((x - ro - e).astype(f32), (x + ro + e).astype(f32)), 0)
    m_in = np.where(P > 1e-30, _col_range((x - ri + e).astype(f32), (x + ri - e).astype(f32)), 0)
    assert np.all((m_in & ~m_pos) == 0)            # inside implies possibly inside

    i = np.arange(16)
    du = cu.astype(np.float64)[:, None] - i[None, :] * h.astype(np.float64)[:, None]
    t = dv2.astype(np.float64)[:, None] + ak.astype(np.float64)[:, None] * du * du
    bit = (1 << i)[None, :]
    inside = (m_in[:, None] & bit) != 0
    possible = (m_pos[:, None] & bit) != 0
    assert not np.any(inside & ~(t <= blo.astype(np.float64)[:, None]))
    assert not np.any(~possible & ~(t > bhi.astype(np.float64)[:, None]))
    # the band stays small, so the exact FP64 test remains rare
    assert np.mean(possible & ~inside) < 1e-3
    # and the fast path decides nearly every pair inside the support
    n_in = np.count_nonzero(t <= blo.astype(np.float64)[:, None])
    assert n_in > 100_000 and np.count_nonzero(inside) > 0.99 * n_in

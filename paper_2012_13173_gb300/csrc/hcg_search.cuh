// hcg_search.cuh -- the contributing-sample search of HCGrid Sec. 3.4 and
// the support test / weight of Eq. (1), shared by the CUDA-core gather and
// the tensor-core blocked path so that both use the same membership decision.
#pragma once

#include "hcg_dev.cuh"

constexpr int kGW = 2, kGH = 2, kCells = kGW * kGH;   // cells per gather group

// Rings and longitude window covering the supports of a block of cells.
struct Window {
    int64_t ra, rb;          // ring range
    double phic, half;       // longitude window centre and half-width, radians
    double half_cells;       // half the cells' own longitude spread, radians
    float clo, chi, ccos;    // cells' latitude band (radians, widened) and a lower bound of its cos
};

HCG_DEV double ring_coord_d(double ns, double z) {
    if (z > 2.0 / 3.0) return ns * sqrt(fmax(0.0, 3.0 * (1.0 - z)));
    if (z < -2.0 / 3.0) return 4.0 * ns - ns * sqrt(fmax(0.0, 3.0 * (1.0 + z)));
    return ns * (2.0 - 1.5 * z);
}

// Steps 1-2 of Sec. 3.4 for cells with centre latitudes [latmin, latmax] and
// longitude offsets [amin, amax] from lon0 (degrees).
HCG_DEV void cells_window(const GridParams &g, double latmin, double latmax, double amin, double amax, Window &W) {
    // step 1: rings whose samples can lie in [latmin - R, latmax + R]; a sample of
    // ring r has ring coordinate in (r - 1, r + 1), so r runs over
    // [floor(rc_lo), ceil(rc_hi)] (1e-6 of a ring added for rounding)
    double lo = fmax(-90.0, latmin - g.R_deg), hi = fmin(90.0, latmax + g.R_deg);
    double ns = (double)g.nside;
    double rc_hi = ring_coord_d(ns, sin(lo * kDeg));   // south edge -> larger ring number
    double rc_lo = ring_coord_d(ns, sin(hi * kDeg));
    int64_t ra = (int64_t)floor(rc_lo - 1e-6), rb = (int64_t)ceil(rc_hi + 1e-6);
    W.ra = max(max(ra, (int64_t)1), g.r_lo);
    W.rb = min(min(rb, 4 * g.nside - 1), g.r_hi);
    // step 2: longitude half-width of the union of the cells' discs
    double cmax = fmax(fabs(latmin), fabs(latmax));
    double half;
    if (cmax + g.R_deg >= 89.999) {
        half = 4.0;   // > pi: whole rings
    } else {
        double s = sin(g.R_deg * kDeg) / cos(cmax * kDeg);
        half = s >= 1.0 ? 4.0 : asin(s);
    }
    W.half_cells = 0.5 * (amax - amin) * kDeg;
    W.half = half + W.half_cells;
    W.clo = __double2float_rd(latmin * kDeg - 1e-6);
    W.chi = __double2float_ru(latmax * kDeg + 1e-6);
    W.ccos = __double2float_rd(fmax(0.0, cos(fmin(1.5707963267948966, cmax * kDeg + 1e-6)) * (1.0 - 1e-6) - 1e-7));
    double lc = g.lon0 + 0.5 * (amin + amax);
    lc = fmod(lc, 360.0);
    if (lc < 0) lc += 360.0;
    W.phic = lc * kDeg;
}

HCG_DEV float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Cell data of one group, identical in every lane.
struct Group {
    int i0, j0;
    float ah[kCells], al[kCells], bh[kCells], bl[kCells], cg[kCells];
    bool ok[kCells];
    Window win;
};

template <bool kProj = true>
HCG_DEV void make_group(const GridParams &g, int gx, int gy, Group &G) {
    G.i0 = gx * kGW;
    G.j0 = gy * kGH;
    double latmin = 1e9, latmax = -1e9, amin = 1e9, amax = -1e9;
#pragma unroll
    for (int q = 0; q < kCells; q++) {
        int i = G.i0 + (q % kGW), j = G.j0 + (q / kGW);
        G.ok[q] = (i < g.nx) && (j < g.ny);
        int ic = min(i, g.nx - 1), jc = min(j, g.ny - 1);
        double a = ((double)ic - g.hx) * g.pix;      // degrees from lon0
        double b = ((double)jc - g.hy) * g.pix;
        if (kProj && g.clon) {                        // projected grid: the cell's own centre
            const size_t k = (size_t)jc * g.nx + ic;
            a = wrap180(g.clon[k] - g.lon0);
            b = g.clat[k] - g.lat0;
        }
        double A = a * kDeg, B = b * kDeg;
        G.ah[q] = (float)A; G.al[q] = (float)(A - (double)G.ah[q]);
        G.bh[q] = (float)B; G.bl[q] = (float)(B - (double)G.bh[q]);
        double latc = g.lat0 + b;
        G.cg[q] = cosf((float)(latc * kDeg));
        latmin = fmin(latmin, latc); latmax = fmax(latmax, latc);
        amin = fmin(amin, a); amax = fmax(amax, a);
    }
    cells_window(g, latmin, latmax, amin, amax, G.win);
}

// Longitude half-width (radians) of ring r's part of the window.  A sample
// of ring r lies in the ring's latitude band; d = its least latitude distance
// from the cells.  From the haversine, a sample within R of a cell has
// hav(dlon) <= (hav R - hav d) / (cos lat_sample cos lat_cell) = x, so
//   dlon <= 2 asin(sqrt(x)) <= 2 sqrt(x / (1 - x))     (asin y <= y / sqrt(1 - y^2)),
// with hav d >= q^2 (1 - q^2 / 3), q = d / 2 (sin q >= q - q^3 / 6): both
// bounds err on the wide side and need no transcendental call.  FP32 with a
// relative margin of 1e-5 and 2e-6 rad on top (the caller pads one more
// pixel); x >= 1/2 and anything wider than the group's whole window give the
// whole window.  Returns -1 when no sample of the ring can reach a cell.
HCG_DEV double ring_half(const GridParams &g, const Window &W, float4 band) {
    if (W.half >= 4.0) return W.half;
    const float d = fmaxf(0.0f, fmaxf(band.x - W.chi, W.clo - band.y));
    const float q2 = 0.25f * d * d;
    const float hd = q2 * fmaf(-q2, 1.0f / 3.0f, 1.0f);
    if (hd > g.havRf) return -1.0;
    const float x = (g.havRf - hd) / (W.ccos * band.z);
    if (!(x < 0.5f)) return W.half;                       // also for a zero cosine
    const double h = (double)(2.0f * sqrtf(x / (1.0f - x)) * 1.00001f + 2e-6f) + W.half_cells;
    return fmin(h, W.half);
}

// Steps 2-3 for ring r: up to two runs [b, b + l) of S'.
HCG_DEV void ring_runs(const GridParams &g, const int64_t *__restrict__ upix, const int64_t *__restrict__ ustart,
                       const int64_t *__restrict__ rustart, const float4 *__restrict__ rband, const Window &W,
                       int64_t r, uint32_t &b1, uint32_t &l1, uint32_t &b2, uint32_t &l2) {
    b1 = l1 = b2 = l2 = 0;
    const double hw = ring_half(g, W, rband[r - g.r_lo]);
    if (hw < 0.0) return;
    const int64_t ns = g.nside;
    const int64_t nr = ring_npix(ns, r);
    const int64_t first = ring_first_pix(ns, r);
    const double twopi = 6.283185307179586;
    double pa = W.phic - hw, pb = W.phic + hw;
    int64_t klo, khi;
    if (r < ns || r > 3 * ns) {     // cap rings: index = floor(phi n_r / 2 pi)
        double f = (double)nr / twopi;
        klo = (int64_t)floor(pa * f) - 1;
        khi = (int64_t)floor(pb * f) + 1;
    } else {                          // belt: centres at (k + s/2) 2 pi / n_r, half-width pi / n_r
        double f = (double)nr / twopi;
        double sh = 0.5 * (double)((r - ns + 1) & 1);
        klo = (int64_t)ceil(pa * f - 0.5 - sh) - 1;
        khi = (int64_t)floor(pb * f + 0.5 - sh) + 1;
    }
    int64_t p1a, p1b, p2a = 0, p2b = -1;
    if (khi - klo + 1 >= nr) {
        p1a = 0; p1b = nr - 1;
    } else {
        int64_t kl = ((klo % nr) + nr) % nr;
        int64_t kh = kl + (khi - klo);
        if (kh < nr) { p1a = kl; p1b = kh; }
        else { p1a = kl; p1b = nr - 1; p2a = 0; p2b = kh - nr; }
    }
    int64_t ua = rustart[r - g.r_lo], ub = rustart[r - g.r_lo + 1];
    if (ua >= ub) return;
    {
        int64_t x = lower_bound_i64(upix, ua, ub, first + p1a);
        int64_t y = upper_bound_i64(upix, x, ub, first + p1b);
        int64_t s0 = ustart[x], s1 = ustart[y];
        b1 = (uint32_t)s0; l1 = (uint32_t)(s1 - s0);
    }
    if (p2b >= p2a) {
        int64_t x = lower_bound_i64(upix, ua, ub, first + p2a);
        int64_t y = upper_bound_i64(upix, x, ub, first + p2b);
        int64_t s0 = ustart[x], s1 = ustart[y];
        b2 = (uint32_t)s0; l2 = (uint32_t)(s1 - s0);
    }
}


// Membership and weight of one (cell, sample) pair.  FP32 squared distance
// from offsets formed as (hi - hi) + (lo - lo) of FP64 values split into two
// floats, with the quartic terms of 4 asin^2(sqrt h) and of sin^2; pairs
// within 1e-5 of the support boundary are decided by the exact FP64
// haversine.  Returns w (0 outside); *inside is the membership.
template <bool kProj = true>
HCG_DEV float pair_weight(const GridParams &g, float ah, float al, float bh, float bl, float cg, int i, int j,
                          bool cell_ok, float4 uv, float cn, uint32_t row, bool valid, const double *lon,
                          const double *lat, bool *inside_out) {
    float du = (uv.x - ah) + (uv.y - al);
    float dv = (uv.z - bh) + (uv.w - bl);
    float x2 = dv * dv, y2 = du * du;
    float c = cg * cn;
    float h4 = x2 * (1.0f - x2 * (1.0f / 12.0f)) + c * (y2 * (1.0f - y2 * (1.0f / 12.0f)));
    float d2 = h4 * (1.0f + h4 * (1.0f / 12.0f));
    bool inside = d2 <= g.band_lo;
    if (valid && cell_ok && !inside && d2 <= g.band_hi) inside = hav_exact_t<kProj>(g, i, j, lon[row], lat[row]) <= g.hR;
    inside = inside && valid && cell_ok;
    *inside_out = inside;
    return inside ? ex2_approx(-d2 * g.kexp) : 0.0f;
}

// Steps 1-3 for a rectangular tile of cells [i0, i0 + tw) x [j0, j0 + th) of
// a plain grid, by one whole warp: the tile's runs of S' (at most two per
// ring, in ring order) as run starts seg_b[] and the inclusive prefix sums
// of their lengths seg_off[]; seg_n[0] = runs, seg_n[1] = candidates.  With
// more than max_seg runs the SEGMENTS error bit is raised and the table left
// empty.
HCG_DEV void tile_runs(const GridParams &g, const int64_t *__restrict__ upix, const int64_t *__restrict__ ustart,
                       const int64_t *__restrict__ rustart, const float4 *__restrict__ rband, int i0, int j0, int tw,
                       int th, uint32_t *seg_b, uint32_t *seg_off, uint32_t *seg_n, int max_seg, int *err) {
    const int lane = threadIdx.x & 31;
    const int ilast = min(i0 + tw, g.nx) - 1, jlast = min(j0 + th, g.ny) - 1;
    const double amin = ((double)i0 - g.hx) * g.pix, amax = ((double)ilast - g.hx) * g.pix;
    const double latmin = g.lat0 + ((double)j0 - g.hy) * g.pix, latmax = g.lat0 + ((double)jlast - g.hy) * g.pix;
    Window W;
    cells_window(g, latmin, latmax, amin, amax, W);
    uint32_t nseg = 0, total = 0;
    bool over = false;
    for (int64_t rbase = W.ra; rbase <= W.rb; rbase += 32) {
        const int64_t r = rbase + lane;
        uint32_t b1 = 0, l1 = 0, b2 = 0, l2 = 0;
        if (r <= W.rb) ring_runs(g, upix, ustart, rustart, rband, W, r, b1, l1, b2, l2);
        // two slots per lane, empty runs dropped
        uint32_t k1 = l1 ? 1u : 0u, k2 = l2 ? 1u : 0u, kk = k1 + k2, ks = kk, ls = l1 + l2, lsum = ls;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ks, o), z = __shfl_up_sync(0xffffffffu, lsum, o);
            if (lane >= o) { ks += y; lsum += z; }
        }
        uint32_t pos = nseg + ks - kk, run = total + lsum - ls;
        if (pos + kk > (uint32_t)max_seg) over = true;
        if (!over) {
            if (k1) { seg_b[pos] = b1; seg_off[pos] = run + l1; pos++; }
            if (k2) { seg_b[pos] = b2; seg_off[pos] = run + l1 + l2; }
        }
        nseg += __shfl_sync(0xffffffffu, ks, 31);
        total += __shfl_sync(0xffffffffu, lsum, 31);
        over = __any_sync(0xffffffffu, over);
    }
    if (over) {
        if (lane == 0) set_err(err, HCG_DERR_SEGMENTS);
        nseg = 0; total = 0;
    }
    if (lane == 0) { seg_n[0] = nseg; seg_n[1] = total; }
}

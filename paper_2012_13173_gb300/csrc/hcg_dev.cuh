// hcg_dev.cuh -- device helpers shared by the library's kernels:
// HEALPix RING geometry (Gorski et al. 2005), the pre-ordering tie-break hash,
// and the exact FP64 haversine test of Eq. (1)'s support.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hcg_internal.h"

#define HCG_DEV __device__ __forceinline__

// Degrees -> radians (the double nearest pi/180, folded at compile time).
static constexpr double kDeg = 3.14159265358979323846 / 180.0;
static constexpr float kTwoPiF = 6.28318530717958647692f;

// FP64 arithmetic that decides integers (pixel indices, support membership)
// is written with explicit round-to-nearest intrinsics so that the compiler
// cannot contract it into fused multiply-adds: each step is one IEEE
// operation, in the order written.
HCG_DEV double xadd(double a, double b) { return __dadd_rn(a, b); }
HCG_DEV double xsub(double a, double b) { return __dsub_rn(a, b); }
HCG_DEV double xmul(double a, double b) { return __dmul_rn(a, b); }
HCG_DEV double xdiv(double a, double b) { return __ddiv_rn(a, b); }

HCG_DEV double lon360(double lon) {
    double l = fmod(lon, 360.0);
    if (l < 0.0) l = xadd(l, 360.0);
    if (l >= 360.0) l = 0.0;
    return l;
}

HCG_DEV double wrap180(double x) {
    double y = fmod(x, 360.0);
    if (y > 180.0) y = xsub(y, 360.0);
    if (y <= -180.0) y = xadd(y, 360.0);
    return y;
}

// ---- HEALPix RING scheme.  Rings 1 .. 4 nside - 1 from the north pole;
// 4r pixels in the north cap (r < nside), 4 nside in the belt, mirrored south.
HCG_DEV int64_t ring_npix(int64_t nside, int64_t r) {
    return r < nside ? 4 * r : (r > 3 * nside ? 4 * (4 * nside - r) : 4 * nside);
}

HCG_DEV int64_t ring_first_pix(int64_t nside, int64_t r) {   // valid up to r = 4 nside
    if (r <= nside) return 2 * r * (r - 1);
    if (r <= 3 * nside) return 2 * nside * (nside - 1) + (r - nside) * 4 * nside;
    int64_t q = 4 * nside - r;
    return 12 * nside * nside - 2 * q * (q + 1);
}

// Pixel (and ring) of a point; Gorski et al. 2005 ring-scheme formulas with
// t = lon / 90 in [0, 4) and z = sin(lat).  Belt: edge-line indices
// j+- = floor(nside (1/2 + t) -+ (3/4) nside z).  Caps: x = nside sqrt(3(1-|z|)),
// j+ = floor(frac(t) x), j- = floor((1 - frac(t)) x), ring j+ + j- + 1 from the pole.
HCG_DEV int64_t ang2pix_ring(int64_t nside, double lon_deg, double lat_deg, int64_t *ring) {
    double z = sin(xmul(lat_deg, kDeg));
    double za = fabs(z);
    double tt = xdiv(lon360(lon_deg), 90.0);
    if (tt >= 4.0) tt = xsub(tt, 4.0);
    double ns = (double)nside;
    if (za <= 2.0 / 3.0) {
        double t1 = xmul(ns, xadd(0.5, tt));
        double t2 = xmul(xmul(ns, 0.75), z);
        int64_t jp = (int64_t)floor(xsub(t1, t2));
        int64_t jm = (int64_t)floor(xadd(t1, t2));
        int64_t ir = nside + 1 + jp - jm;
        int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - nside + kshift + 1) / 2;
        if (ip >= 4 * nside) ip -= 4 * nside;      // ip <= 4 nside here: same as % (4 nside)
        *ring = nside - 1 + ir;
        return 2 * nside * (nside - 1) + (ir - 1) * 4 * nside + ip;
    }
    double tp = xsub(tt, floor(tt));
    double x = xmul(ns, __dsqrt_rn(xmul(3.0, xsub(1.0, za))));
    int64_t jp = (int64_t)floor(xmul(tp, x));
    int64_t jm = (int64_t)floor(xmul(xsub(1.0, tp), x));
    int64_t ir = jp + jm + 1;
    int64_t ip = (int64_t)floor(xmul(tt, (double)ir));
    if (ip >= 4 * ir) ip -= 4 * ir;            // ip <= 4 ir here: same as % (4 ir)
    if (z > 0.0) { *ring = ir; return 2 * ir * (ir - 1) + ip; }
    *ring = 4 * nside - ir;
    return 12 * nside * nside - 2 * ir * (ir + 1) + ip;
}

// The same pixel with most of the FP64 work avoided: in the equatorial belt,
// z = sin(lat) is first taken in FP32 (|error| <= 2.2e-7: argument rounding
// plus sinf's 2 ulp) and t = lon/90 by a multiply (error ~1e-15), which moves
// the edge-line values nside (1/2 + t) -+ (3/4) nside z by at most
// 1.65e-7 nside + 1e-11.  When both lie farther than eps (>= twice that) from
// an integer, their floors -- and so the pixel -- are those of the FP64
// formula; otherwise, and in the polar caps, the FP64 formula above runs.
// eps <= 0 disables the screen.
HCG_DEV int64_t ang2pix_ring_screened(int64_t nside, double lon_deg, double lat_deg, double eps, int64_t *ring) {
    if (eps > 0.0) {
        const float zf = sinf((float)(lat_deg * kDeg));
        if (fabsf(zf) <= 0.6666f) {
            // t to ~1e-15 without FP64 fmod or division (both costly on this GPU);
            // its error is far inside eps
            double l = lon_deg;
            if (l < 0.0 || l >= 360.0) l = lon360(l);
            double tt = l * (1.0 / 90.0);
            if (tt >= 4.0) tt -= 4.0;
            const double ns = (double)nside;
            const double t1 = xmul(ns, xadd(0.5, tt));
            const double t2 = xmul(xmul(ns, 0.75), (double)zf);
            const double a = xsub(t1, t2), b = xadd(t1, t2);
            const double fa = a - floor(a), fb = b - floor(b);
            if (fa > eps && fa < 1.0 - eps && fb > eps && fb < 1.0 - eps) {
                int64_t jp = (int64_t)floor(a), jm = (int64_t)floor(b);
                int64_t ir = nside + 1 + jp - jm;
                int64_t kshift = 1 - (ir & 1);
                int64_t ip = (jp + jm - nside + kshift + 1) / 2;
                if (ip >= 4 * nside) ip -= 4 * nside;      // ip <= 4 nside here: same as % (4 nside)
                *ring = nside - 1 + ir;
                return 2 * nside * (nside - 1) + (ir - 1) * 4 * nside + ip;
            }
        }
    }
    return ang2pix_ring(nside, lon_deg, lat_deg, ring);
}

// Continuous ring coordinate (equals r at the centre latitude of ring r); a
// point of ring r has ring coordinate strictly inside (r - 1, r + 1).
HCG_DEV float ring_coord(float nside, float z) {
    if (z > 2.0f / 3.0f) return nside * sqrtf(fmaxf(0.0f, 3.0f * (1.0f - z)));
    if (z < -2.0f / 3.0f) return 4.0f * nside - nside * sqrtf(fmaxf(0.0f, 3.0f * (1.0f + z)));
    return nside * (2.0f - 1.5f * z);
}

// ---- tie-break hash of the pre-ordering: MurmurHash3's 64-bit finaliser
// (Appleby) of the raw coordinate bit patterns; the top 32 bits are used.
HCG_DEV uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

HCG_DEV uint32_t coord_hash(double lon, double lat) {
    uint64_t a = (uint64_t)__double_as_longlong(lat);
    uint64_t b = (uint64_t)__double_as_longlong(lon);
    return (uint32_t)(fmix64(a ^ ((b << 29) | (b >> 35))) >> 32);
}

// ---- exact support test, FP64, in the same operation order as the
// definition: h = sin^2(dlat/2) + cos(lat_g) cos(lat_n) sin^2(dlon/2), with the
// longitude offset taken relative to lon0 and wrapped to (-180, 180].
// kProj: the grid may be projected (GridParams::clon set: explicit cell
// centres, the oracle's explicit-cell form); false compiles the plain grid's
// form only, for kernels that never see projected grids.
template <bool kProj>
HCG_DEV double hav_exact_t(const GridParams &g, int i, int j, double lon, double lat) {
    if (kProj && g.clon) {
        const size_t k = (size_t)j * g.nx + i;
        const double lonc = g.clon[k], latc = g.clat[k];
        double dlon = xmul(wrap180(xsub(lon, lonc)), kDeg);
        double dlat = xmul(xsub(lat, latc), kDeg);
        double cg = cos(xmul(latc, kDeg));
        double cn = cos(xmul(lat, kDeg));
        double sd = sin(xmul(0.5, dlat));
        double sa = sin(xmul(0.5, dlon));
        return xadd(xmul(sd, sd), xmul(xmul(cg, cn), xmul(sa, sa)));
    }
    double a = xmul(xsub((double)i, xmul(0.5, (double)(g.nx - 1))), g.pix);
    double b = xmul(xsub((double)j, xmul(0.5, (double)(g.ny - 1))), g.pix);
    double dlon = xmul(xsub(wrap180(xsub(lon, g.lon0)), a), kDeg);
    double dlat = xmul(xsub(xsub(lat, g.lat0), b), kDeg);
    double cg = cos(xmul(xadd(g.lat0, b), kDeg));
    double cn = cos(xmul(lat, kDeg));
    double sd = sin(xmul(0.5, dlat));
    double sa = sin(xmul(0.5, dlon));
    return xadd(xmul(sd, sd), xmul(xmul(cg, cn), xmul(sa, sa)));
}

HCG_DEV double hav_exact(const GridParams &g, int i, int j, double lon, double lat) {
    return hav_exact_t<true>(g, i, j, lon, lat);
}

// first index in [lo, hi) with a[index] >= x
HCG_DEV int64_t lower_bound_i64(const int64_t *__restrict__ a, int64_t lo, int64_t hi, int64_t x) {
    while (lo < hi) {
        int64_t m = (lo + hi) >> 1;
        if (__ldg(a + m) < x) lo = m + 1; else hi = m;
    }
    return lo;
}

// first index in [lo, hi) with a[index] > x
HCG_DEV int64_t upper_bound_i64(const int64_t *__restrict__ a, int64_t lo, int64_t hi, int64_t x) {
    while (lo < hi) {
        int64_t m = (lo + hi) >> 1;
        if (__ldg(a + m) <= x) lo = m + 1; else hi = m;
    }
    return lo;
}

HCG_DEV void set_err(int *err, int bit) { atomicOr(err, bit); }

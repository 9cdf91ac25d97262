// hcg_gather.cu -- the table-driven gather of HCGrid Sec. 3.4 and the
// convolution of Eq. (1), on CUDA cores (any storage type).
//
// Work decomposition: one warp owns a 2 x 2 group of neighbouring cells (the
// coarsening of Sec. 3.5 I.2, generalised to two dimensions: the four cells
// share one candidate search and every loaded spectrum value feeds four
// accumulators) and a slice of LC * VC channels; LC lanes span the channels
// (VC consecutive channels per lane, vector loads) and 32 / LC lanes split
// the candidates when the channel count is small.
//
// Per group (Sec. 3.4 steps 1-5):
//   1. the ring range covering the group's latitude band +- R;
//   2. per ring, the pixel-index window covering the group's longitude band
//      +- asin(sin R / cos lat) (one or two windows at the 0/360 seam);
//   3. the window's first and last distinct pixels in the first-level table
//      (searched within the ring's slice given by the second-level table),
//      whose S_start values bound a contiguous run of S';
//   4. the runs are traversed 32 candidates at a time: each lane tests one
//      candidate against the four cells (FP32 great-circle distance from
//      FP64-exact hi/lo offsets, exact FP64 haversine within 1e-5 of the
//      boundary), then every lane accumulates w * s over its channels for the
//      candidates inside at least one cell's support;
//   5. W = sum w by a warp tree, V = sum w s / W (FP64 division when W is
//      small), NaN for empty cells.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "hcg_dev.cuh"

namespace {

constexpr int kGW = 2, kGH = 2, kCells = kGW * kGH;
constexpr int kWarps = 4;

struct GatherArgs {
    GridParams g;
    const float4 *uv;
    const float *cs;
    const uint32_t *row;
    const int64_t *upix, *ustart, *rustart;
    const double *lon, *lat;
    const void *spec;
    const float *scale;
    int nchan;
    float *cube, *wout;
    unsigned long long *pairs;
    int *err;
    int ngx, ngy;
    int64_t ngroups;
    int nslices;
};

struct WarpSmem {
    uint32_t b1[32], l1[32], b2[32], off[32];
    float4 w[32];
    uint32_t r[32];
};

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
    int64_t ra, rb;          // ring range
    double phic, half;       // longitude window centre and half-width, radians
};

HCG_DEV double ring_coord_d(double ns, double z) {
    if (z > 2.0 / 3.0) return ns * sqrt(fmax(0.0, 3.0 * (1.0 - z)));
    if (z < -2.0 / 3.0) return 4.0 * ns - ns * sqrt(fmax(0.0, 3.0 * (1.0 + z)));
    return ns * (2.0 - 1.5 * z);
}

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
        double A = a * kDeg, B = b * kDeg;
        G.ah[q] = (float)A; G.al[q] = (float)(A - (double)G.ah[q]);
        G.bh[q] = (float)B; G.bl[q] = (float)(B - (double)G.bh[q]);
        double latc = g.lat0 + b;
        G.cg[q] = cosf((float)(latc * kDeg));
        latmin = fmin(latmin, latc); latmax = fmax(latmax, latc);
        amin = fmin(amin, a); amax = fmax(amax, a);
    }
    // step 1: rings whose samples can lie in [latmin - R, latmax + R]
    double lo = fmax(-90.0, latmin - g.R_deg), hi = fmin(90.0, latmax + g.R_deg);
    double ns = (double)g.nside;
    double rc_hi = ring_coord_d(ns, sin(lo * kDeg));   // south edge -> larger ring number
    double rc_lo = ring_coord_d(ns, sin(hi * kDeg));
    int64_t ra = (int64_t)floor(rc_lo) - 1, rb = (int64_t)ceil(rc_hi) + 1;
    G.ra = max(max(ra, (int64_t)1), g.r_lo);
    G.rb = min(min(rb, 4 * g.nside - 1), g.r_hi);
    // step 2: longitude half-width of the union of the cells' discs
    double cmax = fmax(fabs(latmin), fabs(latmax));
    double half;
    if (cmax + g.R_deg >= 89.999) {
        half = 4.0;   // > pi: whole rings
    } else {
        double s = sin(g.R_deg * kDeg) / cos(cmax * kDeg);
        half = s >= 1.0 ? 4.0 : asin(s);
    }
    G.half = half + 0.5 * (amax - amin) * kDeg;
    double lc = g.lon0 + 0.5 * (amin + amax);
    lc = fmod(lc, 360.0);
    if (lc < 0) lc += 360.0;
    G.phic = lc * kDeg;
}

// Steps 2-3 for ring r: up to two runs [b, b + l) of S'.
HCG_DEV void ring_runs(const GatherArgs &a, const Group &G, int64_t r, uint32_t &b1, uint32_t &l1,
                       uint32_t &b2, uint32_t &l2) {
    b1 = l1 = b2 = l2 = 0;
    const GridParams &g = a.g;
    const int64_t ns = g.nside;
    const int64_t nr = ring_npix(ns, r);
    const int64_t first = ring_first_pix(ns, r);
    const double twopi = 6.283185307179586;
    double pa = G.phic - G.half, pb = G.phic + G.half;
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
    int64_t ua = a.rustart[r - g.r_lo], ub = a.rustart[r - g.r_lo + 1];
    if (ua >= ub) return;
    {
        int64_t x = lower_bound_i64(a.upix, ua, ub, first + p1a);
        int64_t y = upper_bound_i64(a.upix, x, ub, first + p1b);
        int64_t s0 = a.ustart[x], s1 = a.ustart[y];
        b1 = (uint32_t)s0; l1 = (uint32_t)(s1 - s0);
    }
    if (p2b >= p2a) {
        int64_t x = lower_bound_i64(a.upix, ua, ub, first + p2a);
        int64_t y = upper_bound_i64(a.upix, x, ub, first + p2b);
        int64_t s0 = a.ustart[x], s1 = a.ustart[y];
        b2 = (uint32_t)s0; l2 = (uint32_t)(s1 - s0);
    }
}

// Walk every candidate of the group, 32 per step.  f(valid, s_index) is
// called by all 32 lanes together once per step.
template <typename F>
HCG_DEV void visit_candidates(const GatherArgs &a, const Group &G, WarpSmem &sm, F &&f) {
    const int lane = threadIdx.x & 31;
    for (int64_t rbase = G.ra; rbase <= G.rb; rbase += 32) {
        int64_t r = rbase + lane;
        uint32_t b1 = 0, l1 = 0, b2 = 0, l2 = 0;
        if (r <= G.rb) ring_runs(a, G, r, b1, l1, b2, l2);
        uint32_t len = l1 + l2, inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        __syncwarp();
        sm.b1[lane] = b1; sm.l1[lane] = l1; sm.b2[lane] = b2; sm.off[lane] = inc;
        __syncwarp();
        uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        for (uint32_t base = 0; base < total; base += 32) {
            uint32_t p = base + lane;
            bool valid = p < total;
            uint32_t sidx = 0;
            if (valid) {
                int lo = 0, hi = 31;          // first lane with inclusive offset > p
                while (lo < hi) { int m = (lo + hi) >> 1; if (sm.off[m] > p) hi = m; else lo = m + 1; }
                uint32_t q = p - (lo ? sm.off[lo - 1] : 0u);   // offset within lane lo's runs
                sidx = q < sm.l1[lo] ? sm.b1[lo] + q : sm.b2[lo] + (q - sm.l1[lo]);
            }
            f(valid, sidx);
        }
        __syncwarp();
    }
}

// Membership and weight of (cell q, candidate) -- Eq. (1) kernel.
struct PairTest {
    HCG_DEV static void run(const GatherArgs &a, const Group &G, float4 uv, float cn, uint32_t row,
                            bool valid, float w[kCells], bool in[kCells]) {
        const GridParams &g = a.g;
#pragma unroll
        for (int q = 0; q < kCells; q++) {
            float du = (uv.x - G.ah[q]) + (uv.y - G.al[q]);
            float dv = (uv.z - G.bh[q]) + (uv.w - G.bl[q]);
            float x2 = dv * dv, y2 = du * du;
            float c = G.cg[q] * cn;
            float h4 = x2 * (1.0f - x2 * (1.0f / 12.0f)) + c * (y2 * (1.0f - y2 * (1.0f / 12.0f)));
            float d2 = h4 * (1.0f + h4 * (1.0f / 12.0f));
            bool inside = d2 <= g.band_lo;
            if (valid && G.ok[q] && !inside && d2 <= g.band_hi) {
                int i = G.i0 + (q % kGW), j = G.j0 + (q / kGW);
                inside = hav_exact(g, i, j, a.lon[row], a.lat[row]) <= g.hR;
            }
            inside = inside && valid && G.ok[q];
            in[q] = inside;
            w[q] = inside ? ex2_approx(-d2 * g.kexp) : 0.0f;
        }
    }
};

template <typename T>
struct Loader;

template <>
struct Loader<float> {
    template <int VC, bool VEC>
    HCG_DEV static void load(const float *p, int valid_n, float x[VC]) {
        if (VEC) {
#pragma unroll
            for (int v = 0; v < VC; v += 4) {
                float4 t = __ldg(reinterpret_cast<const float4 *>(p + v));
                x[v] = t.x; x[v + 1] = t.y; x[v + 2] = t.z; x[v + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int v = 0; v < VC; v++) x[v] = v < valid_n ? __ldg(p + v) : 0.0f;
        }
    }
};

template <>
struct Loader<__nv_bfloat16> {
    template <int VC, bool VEC>
    HCG_DEV static void load(const __nv_bfloat16 *p, int valid_n, float x[VC]) {
        if (VEC && VC == 8) {
            uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
            const uint32_t u[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                x[2 * k] = __uint_as_float(u[k] << 16);
                x[2 * k + 1] = __uint_as_float(u[k] & 0xffff0000u);
            }
        } else {
            const unsigned short *h = reinterpret_cast<const unsigned short *>(p);
#pragma unroll
            for (int v = 0; v < VC; v++) x[v] = v < valid_n ? __uint_as_float(((uint32_t)__ldg(h + v)) << 16) : 0.0f;
        }
    }
};

template <>
struct Loader<__nv_fp8_storage_t> {
    template <int VC, bool VEC>
    HCG_DEV static void load(const __nv_fp8_storage_t *p, int valid_n, float x[VC]) {
        if (VEC && VC == 8) {
            uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
            const uint32_t u[2] = {t.x, t.y};
#pragma unroll
            for (int k = 0; k < 2; k++) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    __half2_raw r = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((u[k] >> (16 * h)) & 0xffff), __NV_E4M3);
                    __half2 hh = *reinterpret_cast<__half2 *>(&r);
                    float2 f = __half22float2(hh);
                    x[4 * k + 2 * h] = f.x; x[4 * k + 2 * h + 1] = f.y;
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < VC; v++) {
                if (v < valid_n) {
                    __half_raw r = __nv_cvt_fp8_to_halfraw(__ldg(reinterpret_cast<const unsigned char *>(p) + v), __NV_E4M3);
                    x[v] = __half2float(*reinterpret_cast<__half *>(&r));
                } else {
                    x[v] = 0.0f;
                }
            }
        }
    }
};

template <typename T, int VC, int LC>
__global__ void __launch_bounds__(kWarps * 32) k_gather(GatherArgs a) {
    constexpr int LK = 32 / LC;
    __shared__ WarpSmem smem[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gblocks = (a.ngroups + kWarps - 1) / kWarps;
    const int slice = (int)(blockIdx.x / gblocks);
    const int64_t grp = (blockIdx.x % gblocks) * kWarps + warp;
    if (grp >= a.ngroups) return;
    WarpSmem &sm = smem[warp];
    Group G;
    make_group(a.g, (int)(grp % a.ngx), (int)(grp / a.ngx), G);

    const int lc = lane % LC, kc = lane / LC;
    const int c0 = slice * (LC * VC) + lc * VC;           // this lane's first channel
    const int cval = min(VC, max(0, a.nchan - c0));      // channels it owns
    // vector loads/stores need whole, aligned channel groups
    const bool vec = (VC % 4 == 0) && (cval == VC) && (a.nchan % ((VC == 8 && sizeof(T) <= 2) ? 8 : 4) == 0);
    const T *spec = static_cast<const T *>(a.spec);

    float acc[kCells][VC];
#pragma unroll
    for (int q = 0; q < kCells; q++)
#pragma unroll
        for (int v = 0; v < VC; v++) acc[q][v] = 0.0f;
    float wsum[kCells] = {0.f, 0.f, 0.f, 0.f};
    unsigned npairs = 0;

    visit_candidates(a, G, sm, [&](bool valid, uint32_t sidx) {
        float4 uv = make_float4(0.f, 0.f, 0.f, 0.f);
        float cn = 0.f;
        uint32_t row = 0;
        if (valid) { uv = __ldg(a.uv + sidx); cn = __ldg(a.cs + sidx); row = __ldg(a.row + sidx); }
        float w[kCells];
        bool in[kCells];
        PairTest::run(a, G, uv, cn, row, valid, w, in);
        bool any = false;
#pragma unroll
        for (int q = 0; q < kCells; q++) { wsum[q] += w[q]; any |= in[q]; npairs += in[q]; }
        sm.w[lane] = make_float4(w[0], w[1], w[2], w[3]);
        sm.r[lane] = row;
        unsigned mask = __ballot_sync(0xffffffffu, any);
        __syncwarp();
        int t = 0;
        while (mask) {
            int j = __ffs(mask) - 1;
            mask &= mask - 1;
            if (LK > 1) { if ((t++ % LK) != kc) continue; }
            if (cval > 0) {
                float4 wj = sm.w[j];
                const T *p = spec + (size_t)sm.r[j] * (size_t)a.nchan + c0;
                float x[VC];
                if (vec) Loader<T>::template load<VC, true>(p, cval, x);
                else Loader<T>::template load<VC, false>(p, cval, x);
#pragma unroll
                for (int v = 0; v < VC; v++) {
                    acc[0][v] = fmaf(wj.x, x[v], acc[0][v]);
                    acc[1][v] = fmaf(wj.y, x[v], acc[1][v]);
                    acc[2][v] = fmaf(wj.z, x[v], acc[2][v]);
                    acc[3][v] = fmaf(wj.w, x[v], acc[3][v]);
                }
            }
        }
        __syncwarp();
    });

    // step 5: normalisation
#pragma unroll
    for (int q = 0; q < kCells; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wsum[q] += __shfl_xor_sync(0xffffffffu, wsum[q], o);
    if (LK > 1) {
#pragma unroll
        for (int o = LC; o < 32; o <<= 1)
#pragma unroll
            for (int q = 0; q < kCells; q++)
#pragma unroll
                for (int v = 0; v < VC; v++) acc[q][v] += __shfl_xor_sync(0xffffffffu, acc[q][v], o);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    if (slice == 0 && lane == 0) {
        atomicAdd(a.pairs, (unsigned long long)npairs);
#pragma unroll
        for (int q = 0; q < kCells; q++)
            if (G.ok[q]) {
                int i = G.i0 + (q % kGW), j = G.j0 + (q / kGW);
                a.wout[(size_t)j * a.g.nx + i] = wsum[q];
            }
    }
    if (kc != 0 || cval == 0) return;
#pragma unroll
    for (int q = 0; q < kCells; q++) {
        if (!G.ok[q]) continue;
        int i = G.i0 + (q % kGW), j = G.j0 + (q / kGW);
        float W = wsum[q];
        float *out = a.cube + ((size_t)j * a.g.nx + i) * (size_t)a.nchan + c0;
        float y[VC];
#pragma unroll
        for (int v = 0; v < VC; v++) {
            float s = acc[q][v];
            float val;
            if (W >= 1e-3f) val = __fdiv_rn(s, W);
            else if (W > 0.0f) val = (float)((double)s / (double)W);
            else val = __int_as_float(0x7fc00000);
            if (a.scale && v < cval) val *= __ldg(a.scale + c0 + v);
            y[v] = val;
        }
        if (vec && VC >= 4) {
#pragma unroll
            for (int v = 0; v < VC; v += 4) *reinterpret_cast<float4 *>(out + v) = make_float4(y[v], y[v + 1], y[v + 2], y[v + 3]);
        } else {
#pragma unroll
            for (int v = 0; v < VC; v++) if (v < cval) out[v] = y[v];
        }
    }
}

// Contributor lists of cells [cb, ce): pass 0 counts, pass 1 fills.
__global__ void __launch_bounds__(kWarps * 32) k_debug_neigh(GatherArgs a, int64_t cb, int64_t ce,
                                                            int64_t *counts, const int64_t *offsets,
                                                            uint32_t *ids, int pass) {
    __shared__ WarpSmem smem[kWarps];
    const int warp = threadIdx.x >> 5;
    const int64_t grp = (int64_t)blockIdx.x * kWarps + warp;
    if (grp >= a.ngroups) return;
    WarpSmem &sm = smem[warp];
    Group G;
    make_group(a.g, (int)(grp % a.ngx), (int)(grp / a.ngx), G);
    visit_candidates(a, G, sm, [&](bool valid, uint32_t sidx) {
        if (!valid) return;
        float4 uv = __ldg(a.uv + sidx);
        float cn = __ldg(a.cs + sidx);
        uint32_t row = __ldg(a.row + sidx);
        float w[kCells];
        bool in[kCells];
        PairTest::run(a, G, uv, cn, row, true, w, in);
#pragma unroll
        for (int q = 0; q < kCells; q++) {
            if (!in[q]) continue;
            int64_t cell = (int64_t)(G.j0 + q / kGW) * a.g.nx + (G.i0 + q % kGW);
            if (cell < cb || cell >= ce) continue;
            unsigned long long *cnt = reinterpret_cast<unsigned long long *>(counts) + (cell - cb);
            unsigned long long k = atomicAdd(cnt, 1ull);
            if (pass == 1) ids[offsets[cell - cb] + (int64_t)k] = row;
        }
    });
}

GatherArgs make_args(hcg_ctx *c, const GridParams &gp, const void *spec, const float *scale) {
    GatherArgs a;
    a.g = gp;
    a.uv = c->sc_uv; a.cs = c->sc_cos; a.row = c->sc_row;
    a.upix = c->upix; a.ustart = c->ustart; a.rustart = c->rustart;
    a.lon = c->lon; a.lat = c->lat;
    a.spec = spec; a.scale = scale; a.nchan = c->nchan;
    a.cube = c->cube(); a.wout = c->weights();
    a.pairs = reinterpret_cast<unsigned long long *>(c->dscal + 1);
    a.err = c->derr;
    a.ngx = (c->nx + kGW - 1) / kGW;
    a.ngy = (c->ny + kGH - 1) / kGH;
    a.ngroups = (int64_t)a.ngx * a.ngy;
    return a;
}

template <typename T, int VC, int LC>
void launch_t(const GatherArgs &a0, cudaStream_t st) {
    GatherArgs a = a0;
    a.nslices = (a.nchan + LC * VC - 1) / (LC * VC);
    int64_t gblocks = (a.ngroups + kWarps - 1) / kWarps;
    k_gather<T, VC, LC><<<(unsigned)(gblocks * a.nslices), kWarps * 32, 0, st>>>(a);
}

template <typename T>
void launch_dtype(const GatherArgs &a, cudaStream_t st, int chans) {
    // channels per warp slice: LC lanes x VC channels
    if (a.nchan >= 256 && chans != 4) launch_t<T, 8, 32>(a, st);
    else if (a.nchan >= 128) launch_t<T, 4, 32>(a, st);
    else if (a.nchan >= 64) launch_t<T, 4, 16>(a, st);
    else if (a.nchan >= 16) launch_t<T, 4, 4>(a, st);
    else if (a.nchan >= 4) launch_t<T, 4, 1>(a, st);
    else launch_t<T, 1, 1>(a, st);
}

}  // namespace

int launch_gather(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale) {
    GatherArgs a = make_args(c, gp, spec, scale);
    if (dtype == HCG_F32) launch_dtype<float>(a, c->stream, c->t_chans);
    else if (dtype == HCG_BF16) launch_dtype<__nv_bfloat16>(a, c->stream, c->t_chans);
    else launch_dtype<__nv_fp8_storage_t>(a, c->stream, c->t_chans);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { hcg_cuda_fail(e, "k_gather"); return -1; }
    return 1;
}

int launch_debug_neigh(hcg_ctx *c, const GridParams &gp, int64_t cb, int64_t ce, int64_t *d_counts,
                       const int64_t *d_offsets, uint32_t *d_ids, int pass) {
    GatherArgs a = make_args(c, gp, nullptr, nullptr);
    int64_t blocks = (a.ngroups + kWarps - 1) / kWarps;
    k_debug_neigh<<<(unsigned)blocks, kWarps * 32, 0, c->stream>>>(a, cb, ce, d_counts, d_offsets, d_ids, pass);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { hcg_cuda_fail(e, "k_debug_neigh"); return -1; }
    return 1;
}

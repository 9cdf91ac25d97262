// hcg_gather.cuh -- the table-driven gather of HCGrid Sec. 3.4 and the
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
//
// This header holds the kernels and launch templates; hcg_gather_f32.cu,
// hcg_gather_bf16.cu and hcg_gather_e4m3.cu instantiate them per storage type
// (launch_gather_dt), hcg_gather_batch.cu the persistent batched form, and
// hcg_gather.cu the dispatch by path and tuning.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <string.h>

#include <algorithm>
#include <type_traits>

#include "hcg_search.cuh"

namespace hcg_gather {


constexpr int kWarps = 4;

struct GatherArgs {
    GridParams g;
    const float4 *uv;
    const float *cs;
    const uint32_t *row;
    const int64_t *upix, *ustart, *rustart;
    const float4 *rband;
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
    int64_t cube_ld;         // cube row stride (channels); a.cube points at the window's first channel
};

struct WarpSmem {
    uint32_t b1[32], l1[32], b2[32], off[32];
    float4 w[32];
    uint32_t r[32];
};

// Position of a candidate walk: the first ring of the current batch of 32
// rings, and the offset of the next batch of 32 candidates within it.
struct WalkPos {
    int64_t rbase;
    uint32_t base;
};

// Walk the group's candidates from `pos`, 32 per step: f(valid, s_index) is
// called by all 32 lanes together once per step.  stop() (warp-uniform) is
// asked before each step; when it says so the walk returns false with pos at
// that step, so that a later call resumes there.  Returns true when done.
template <typename F, typename Stop>
HCG_DEV bool visit_from(const GatherArgs &a, const Group &G, WarpSmem &sm, WalkPos &pos, F &&f, Stop &&stop) {
    const int lane = threadIdx.x & 31;
    for (; pos.rbase <= G.win.rb; pos.rbase += 32, pos.base = 0) {
        int64_t r = pos.rbase + lane;
        uint32_t b1 = 0, l1 = 0, b2 = 0, l2 = 0;
        if (r <= G.win.rb) ring_runs(a.g, a.upix, a.ustart, a.rustart, a.rband, G.win, r, b1, l1, b2, l2);
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
        for (; pos.base < total; pos.base += 32) {
            if (stop()) return false;
            uint32_t p = pos.base + lane;
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
    return true;
}

// Walk every candidate of the group, 32 per step.
template <typename F>
HCG_DEV void visit_candidates(const GatherArgs &a, const Group &G, WarpSmem &sm, F &&f) {
    WalkPos pos{G.win.ra, 0u};
    visit_from(a, G, sm, pos, f, [] { return false; });
}

// Membership and weight of (cell q, candidate) -- Eq. (1) kernel.
struct PairTest {
    template <bool kProj = true>
    HCG_DEV static void run(const GatherArgs &a, const Group &G, float4 uv, float cn, uint32_t row,
                            bool valid, float w[kCells], bool in[kCells]) {
#pragma unroll
        for (int q = 0; q < kCells; q++)
            w[q] = pair_weight<kProj>(a.g, G.ah[q], G.al[q], G.bh[q], G.bl[q], G.cg[q], G.i0 + (q % kGW), G.j0 + (q / kGW),
                               G.ok[q], uv, cn, row, valid, a.lon, a.lat, &in[q]);
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
        } else if (VEC && VC == 4) {
            uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
            x[0] = __uint_as_float(t.x << 16); x[1] = __uint_as_float(t.x & 0xffff0000u);
            x[2] = __uint_as_float(t.y << 16); x[3] = __uint_as_float(t.y & 0xffff0000u);
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
        if (VEC && VC == 4) {
            uint32_t u0 = __ldg(reinterpret_cast<const unsigned int *>(p));
#pragma unroll
            for (int h = 0; h < 2; h++) {
                __half2_raw r = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((u0 >> (16 * h)) & 0xffff), __NV_E4M3);
                float2 f = __half22float2(*reinterpret_cast<__half2 *>(&r));
                x[2 * h] = f.x; x[2 * h + 1] = f.y;
            }
        } else if (VEC && VC == 8) {
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

// One warp: group grp, channel slice `slice` (LC lanes x VC channels).
template <typename T, int VC, int LC, bool kProj = true>
HCG_DEV void gather_group_slice(const GatherArgs &a, int64_t grp, int slice, WarpSmem &sm) {
    constexpr int LK = 32 / LC;
    const int lane = threadIdx.x & 31;
    Group G;
    make_group<kProj>(a.g, (int)(grp % a.ngx), a.ngy - 1 - (int)(grp / a.ngx), G);   // north row first

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
        PairTest::run<kProj>(a, G, uv, cn, row, valid, w, in);
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
        if (a.pairs) atomicAdd(a.pairs, (unsigned long long)npairs);
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
        float *out = a.cube + ((size_t)j * a.g.nx + i) * (size_t)a.cube_ld + c0;
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
        if (vec && VC >= 4 && (a.cube_ld & 3) == 0) {
#pragma unroll
            for (int v = 0; v < VC; v += 4) __stcs(reinterpret_cast<float4 *>(out + v), make_float4(y[v], y[v + 1], y[v + 2], y[v + 3]));
        } else {
#pragma unroll
            for (int v = 0; v < VC; v++) if (v < cval) __stcs(out + v, y[v]);
        }
    }
}

// 4 blocks per SM (at most 128 registers): occupancy hides the search's
// dependent loads better than the few spills cost (measured on the 64-field
// batch: 128 registers 140 ms, 168 registers 164 ms).
template <typename T, int VC, int LC, bool kProj>
__global__ void __launch_bounds__(kWarps * 32, 4) k_gather(GatherArgs a) {
    __shared__ WarpSmem smem[kWarps];
    const int warp = threadIdx.x >> 5;
    const int64_t gblocks = (a.ngroups + kWarps - 1) / kWarps;
    const int slice = (int)(blockIdx.x / gblocks);
    const int64_t grp = (blockIdx.x % gblocks) * kWarps + warp;
    if (grp >= a.ngroups) return;
    gather_group_slice<T, VC, LC, kProj>(a, grp, slice, smem[warp]);
}

// ---- list form (nchan >= 256) ------------------------------------------
// A block is a strip of kLWarps horizontally adjacent groups (they share rings
// and most of their longitude windows, so their spectrum rows meet in L1).
// Each warp first builds its group's accepted-candidate list (rows and the
// four weights) in shared memory, then sweeps every 256-channel slice over
// that list, loading twelve candidates' spectra ahead of their FMAs.  When the
// list does not fit, the warp re-runs the search per slice instead; both
// orders accumulate in S' order, so the results are identical.
// Block rows run north to south.  A list follows S' (rings north to south),
// so a row shared with the group below is read near the end of this group's
// pass and near the start of the lower group's, which is launched shortly
// after: the row is still in L2.  The opposite order puts those two reads a
// whole pass apart (measured on the 1M-sample drift scan: DRAM reads
// 8.1 GB that way, 4.9 GB this way, for 4.1 GB of spectra).
constexpr int kLWarps = 8;
constexpr int kLCap = 384;

struct ListSmem {
    WarpSmem ws;
    float4 lw[kLCap];
    uint32_t lr[kLCap];
};

// 8 FP32 channels in one 256-bit load; p must be 32-byte aligned (the list
// kernel's launcher selects this form only when every row offset is).
HCG_DEV void load8_f32_v8(const float *p, float (&x)[8]) {
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
                 : "l"(p));
}

template <typename T, bool VEC, int kLVC>
HCG_DEV void accum_one(const T *spec, size_t nchan, uint32_t row, int c0, int cval, float4 w,
                       float (&acc)[kCells][kLVC]) {
    float x[kLVC];
    Loader<T>::template load<kLVC, VEC>(spec + (size_t)row * nchan + c0, cval, x);
#pragma unroll
    for (int v = 0; v < kLVC; v++) {
        acc[0][v] = fmaf(w.x, x[v], acc[0][v]);
        acc[1][v] = fmaf(w.y, x[v], acc[1][v]);
        acc[2][v] = fmaf(w.z, x[v], acc[2][v]);
        acc[3][v] = fmaf(w.w, x[v], acc[3][v]);
    }
}

// Cube stores are streaming (st.global.cs): the output is not read again by
// the pass, and keeping it out of L2 leaves room for spectrum rows that
// neighbouring groups are about to read.
template <typename T, int kLVC>
HCG_DEV void store_slice(const GatherArgs &a, const Group &G, const float (&acc)[kCells][kLVC],
                         const float (&W)[kCells], int c0, int cval, bool vec) {
#pragma unroll
    for (int q = 0; q < kCells; q++) {
        if (!G.ok[q] || cval <= 0) continue;
        int i = G.i0 + (q % kGW), j = G.j0 + (q / kGW);
        float *out = a.cube + ((size_t)j * a.g.nx + i) * (size_t)a.cube_ld + c0;
        float y[kLVC];
#pragma unroll
        for (int v = 0; v < kLVC; v++) {
            float sv = acc[q][v], val;
            if (W[q] >= 1e-3f) val = __fdiv_rn(sv, W[q]);
            else if (W[q] > 0.0f) val = (float)((double)sv / (double)W[q]);
            else val = __int_as_float(0x7fc00000);
            if (a.scale && v < cval) val *= __ldg(a.scale + c0 + v);
            y[v] = val;
        }
        if (vec && (a.cube_ld & 3) == 0) {
#pragma unroll
            for (int v = 0; v < kLVC; v += 4) __stcs(reinterpret_cast<float4 *>(out + v), make_float4(y[v], y[v + 1], y[v + 2], y[v + 3]));
        } else {
#pragma unroll
            for (int v = 0; v < kLVC; v++) if (v < cval) __stcs(out + v, y[v]);
        }
    }
}

// kTGX x kTGY groups per block (kTGX * kTGY = 8 warps), blocks in row-major
// order: 8 x 1 = a strip along the rows, 4 x 2 = a tile, 1 x 8 = a column
// strip (vertical sharing inside the block, horizontal in the next block).
template <typename T, int kLVC, int kUnroll, int kMinBlocks, int kTGX, bool kProj, bool kV8>
__global__ void __launch_bounds__(kLWarps * 32, kMinBlocks) k_gather_list(GatherArgs a) {
    constexpr int kTGY = kLWarps / kTGX;
    extern __shared__ __align__(16) unsigned char dsm[];
    ListSmem *sall = reinterpret_cast<ListSmem *>(dsm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tpr = (a.ngx + kTGX - 1) / kTGX;
    const int gx = (int)(blockIdx.x % tpr) * kTGX + (warp % kTGX);
    const int brow = (a.ngy + kTGY - 1) / kTGY - 1 - (int)(blockIdx.x / tpr);   // north row first
    const int gy = brow * kTGY + (warp / kTGX);
    if (gx >= a.ngx || gy >= a.ngy) return;
    ListSmem &sm = sall[warp];
    const T *spec = static_cast<const T *>(a.spec);
    const size_t nchan = (size_t)a.nchan;
    const unsigned lt = (1u << lane) - 1u;

    // phase 1: accepted list, weight sums, pair count (the group's cell data
    // lives only in this scope, so it does not hold registers in phase 2)
    float W[kCells];
    int cnt = 0;
    // where the list first overflowed: the walk step to resume at, and how
    // many of that step's accepted candidates made it into the list
    WalkPos over{0, 0u};
    int over_skip = 0;
    {
        Group G;
        make_group<kProj>(a.g, gx, gy, G);
        float wsum[kCells] = {0.f, 0.f, 0.f, 0.f};
        unsigned npairs = 0;
        WalkPos pos{G.win.ra, 0u};
        visit_from(a, G, sm.ws, pos, [&](bool valid, uint32_t sidx) {
            float4 uv = make_float4(0.f, 0.f, 0.f, 0.f);
            float cn = 0.f;
            uint32_t row = 0;
            if (valid) { uv = __ldg(a.uv + sidx); cn = __ldg(a.cs + sidx); row = __ldg(a.row + sidx); }
            float w[kCells];
            bool in[kCells];
            PairTest::run<kProj>(a, G, uv, cn, row, valid, w, in);
            bool any = false;
#pragma unroll
            for (int q = 0; q < kCells; q++) { wsum[q] += w[q]; any |= in[q]; npairs += in[q]; }
            unsigned m = __ballot_sync(0xffffffffu, any);
            int pos_l = cnt + __popc(m & lt);
            if (any && pos_l < kLCap) { sm.lw[pos_l] = make_float4(w[0], w[1], w[2], w[3]); sm.lr[pos_l] = row; }
            if (cnt <= kLCap && cnt + __popc(m) > kLCap) { over = pos; over_skip = kLCap - cnt; }
            cnt += __popc(m);
        }, [] { return false; });
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kCells; q++) {
            float t = wsum[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            W[q] = t;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        if (lane == 0) {
            if (a.pairs) atomicAdd(a.pairs, (unsigned long long)npairs);
#pragma unroll
            for (int q = 0; q < kCells; q++)
                if (G.ok[q]) a.wout[(size_t)(G.j0 + q / kGW) * a.g.nx + (G.i0 + q % kGW)] = W[q];
        }
    }
    const bool fits = cnt <= kLCap;
    const int nsl = (a.nchan + 32 * kLVC - 1) / (32 * kLVC);
    const int align = sizeof(T) <= 2 ? 8 : 4;
    Group Gs;                        // cell indices for the stores (and the search when the list overflows)
    Gs.i0 = gx * kGW; Gs.j0 = gy * kGH;
#pragma unroll
    for (int q = 0; q < kCells; q++) Gs.ok[q] = (Gs.i0 + (q % kGW) < a.g.nx) && (Gs.j0 + (q / kGW) < a.g.ny);

    // FMA sweep over list entries [0, n): w * s for the four cells, kUnroll
    // candidates' loads in flight
    auto sweep = [&](int n, int c0, int cval, bool vec, float (&acc)[kCells][kLVC]) {
            int j = 0;
            if (vec) {
                for (; j + kUnroll <= n; j += kUnroll) {
                    float x[kUnroll][kLVC];
#pragma unroll
                    for (int u = 0; u < kUnroll; u++) {
                        if constexpr (kV8)
                            load8_f32_v8(reinterpret_cast<const float *>(spec + (size_t)sm.lr[j + u] * nchan + c0), x[u]);
                        else
                            Loader<T>::template load<kLVC, true>(spec + (size_t)sm.lr[j + u] * nchan + c0, kLVC, x[u]);
                    }
#pragma unroll
                    for (int u = 0; u < kUnroll; u++) {
                        const float4 w = sm.lw[j + u];
#pragma unroll
                        for (int v = 0; v < kLVC; v++) {
                            acc[0][v] = fmaf(w.x, x[u][v], acc[0][v]);
                            acc[1][v] = fmaf(w.y, x[u][v], acc[1][v]);
                            acc[2][v] = fmaf(w.z, x[u][v], acc[2][v]);
                            acc[3][v] = fmaf(w.w, x[u][v], acc[3][v]);
                        }
                    }
                }
                for (; j < n; j++) accum_one<T, true, kLVC>(spec, nchan, sm.lr[j], c0, cval, sm.lw[j], acc);
            } else if (cval > 0) {
                for (; j < n; j++) accum_one<T, false, kLVC>(spec, nchan, sm.lr[j], c0, cval, sm.lw[j], acc);
            }
    };

    for (int k = 0; k < nsl; k++) {
        const int sl = k;
        const int c0 = sl * 32 * kLVC + lane * kLVC;
        const int cval = min(kLVC, max(0, a.nchan - c0));
        const bool vec = (cval == kLVC) && (a.nchan % align == 0);
        float acc[kCells][kLVC];
#pragma unroll
        for (int q = 0; q < kCells; q++)
#pragma unroll
            for (int v = 0; v < kLVC; v++) acc[q][v] = 0.0f;
        if (fits) {
            sweep(cnt, c0, cval, vec, acc);
        } else if (nsl == 1) {
            // one channel slice and a list longer than its slot: sweep the
            // list in segments -- the entries held, then the walk resumed
            // where the list filled, refilling it up to kLCap entries at a
            // time -- so every entry is swept once, in S' order
            sweep(kLCap, c0, cval, vec, acc);
            WalkPos pos = over;
            int skip = over_skip;
            for (bool done = false; !done;) {
                int n2 = 0;
                {
                    Group G;
                    make_group<kProj>(a.g, gx, gy, G);
                    done = visit_from(a, G, sm.ws, pos, [&](bool valid, uint32_t sidx) {
                        float4 uv = make_float4(0.f, 0.f, 0.f, 0.f);
                        float cn = 0.f;
                        uint32_t row = 0;
                        if (valid) { uv = __ldg(a.uv + sidx); cn = __ldg(a.cs + sidx); row = __ldg(a.row + sidx); }
                        float w[kCells];
                        bool in[kCells];
                        PairTest::run<kProj>(a, G, uv, cn, row, valid, w, in);
                        const bool any = in[0] | in[1] | in[2] | in[3];
                        const unsigned m = __ballot_sync(0xffffffffu, any);
                        // the first `skip` accepted candidates of the first step were swept already
                        const int rank = __popc(m & lt);
                        if (any && rank >= skip) {
                            sm.lw[n2 + rank - skip] = make_float4(w[0], w[1], w[2], w[3]);
                            sm.lr[n2 + rank - skip] = row;
                        }
                        n2 += max(0, __popc(m) - skip);
                        skip = max(0, skip - __popc(m));
                    }, [&] { return n2 > kLCap - 32; });
                }
                __syncwarp();
                sweep(n2, c0, cval, vec, acc);
                __syncwarp();
            }
        } else {
            Group G;
            make_group<kProj>(a.g, gx, gy, G);
            visit_candidates(a, G, sm.ws, [&](bool valid, uint32_t sidx) {
                float4 uv = make_float4(0.f, 0.f, 0.f, 0.f);
                float cn = 0.f;
                uint32_t row = 0;
                if (valid) { uv = __ldg(a.uv + sidx); cn = __ldg(a.cs + sidx); row = __ldg(a.row + sidx); }
                float w[kCells];
                bool in[kCells];
                PairTest::run<kProj>(a, G, uv, cn, row, valid, w, in);
                bool any = in[0] | in[1] | in[2] | in[3];
                sm.ws.w[lane] = make_float4(w[0], w[1], w[2], w[3]);
                sm.ws.r[lane] = row;
                unsigned m = __ballot_sync(0xffffffffu, any);
                __syncwarp();
                while (m) {
                    int jj = __ffs(m) - 1;
                    m &= m - 1;
                    if (cval <= 0) continue;
                    if (vec) accum_one<T, true, kLVC>(spec, nchan, sm.ws.r[jj], c0, cval, sm.ws.w[jj], acc);
                    else accum_one<T, false, kLVC>(spec, nchan, sm.ws.r[jj], c0, cval, sm.ws.w[jj], acc);
                }
                __syncwarp();
            });
        }
        store_slice<T, kLVC>(a, Gs, acc, W, c0, cval, vec);
    }
}

inline GatherArgs make_args(hcg_ctx *c, const GridParams &gp, const void *spec, const float *scale) {
    GatherArgs a;
    a.g = gp;
    const hcg_ctx *t = c->tables();
    a.uv = t->sc_uv; a.cs = t->sc_cos; a.row = t->sc_row;
    a.upix = t->upix; a.ustart = t->ustart; a.rustart = t->rustart; a.rband = t->rband;
    a.lon = c->lon; a.lat = c->lat;
    a.spec = spec; a.scale = scale; a.nchan = c->win_channels();
    a.cube = c->cube() + c->win_c0; a.cube_ld = c->nchan; a.wout = c->weights();
    a.pairs = c->win_c0 == 0 ? reinterpret_cast<unsigned long long *>(c->dscal + 1) : nullptr;
    a.err = c->derr;
    a.ngx = (c->nx + kGW - 1) / kGW;
    a.ngy = (c->ny + kGH - 1) / kGH;
    a.ngroups = (int64_t)a.ngx * a.ngy;
    a.nslices = 0;
    return a;
}

template <typename T, int VC, int LC>
void launch_t(const GatherArgs &a0, cudaStream_t st) {
    GatherArgs a = a0;
    a.nslices = (a.nchan + LC * VC - 1) / (LC * VC);
    int64_t gblocks = (a.ngroups + kWarps - 1) / kWarps;
    if (a.g.clon) k_gather<T, VC, LC, true><<<(unsigned)(gblocks * a.nslices), kWarps * 32, 0, st>>>(a);
    else k_gather<T, VC, LC, false><<<(unsigned)(gblocks * a.nslices), kWarps * 32, 0, st>>>(a);
}

template <typename T, int VC, int UNROLL, int MINB, int TGX, bool PROJ, bool V8>
void launch_list_p(const GatherArgs &a, cudaStream_t st) {
    size_t smem = sizeof(ListSmem) * kLWarps;
    cudaFuncSetAttribute(k_gather_list<T, VC, UNROLL, MINB, TGX, PROJ, V8>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    constexpr int TGY = kLWarps / TGX;
    int64_t blocks = (int64_t)((a.ngx + TGX - 1) / TGX) * ((a.ngy + TGY - 1) / TGY);
    k_gather_list<T, VC, UNROLL, MINB, TGX, PROJ, V8><<<(unsigned)blocks, kLWarps * 32, smem, st>>>(a);
}

// Plain grids run an instantiation without the projected-grid branches.  FP32
// rows whose lane slices (8 channels) all start on 32-byte boundaries are
// read with 256-bit loads: half the load instructions, and the L1 data pipe
// bounds this kernel (measured on the 1M-sample 1024-channel drift scan:
// 1.90 -> 1.70 ms).
template <typename T, int VC, int UNROLL, int MINB, int TGX>
void launch_list_t(const GatherArgs &a, cudaStream_t st) {
    constexpr bool kCanV8 = std::is_same<T, float>::value && VC == 8;
    const bool v8 = kCanV8 && a.nchan % 8 == 0 && ((uintptr_t)a.spec & 31) == 0;
    if (a.g.clon) {
        if (v8) launch_list_p<T, VC, UNROLL, MINB, TGX, true, kCanV8>(a, st);
        else launch_list_p<T, VC, UNROLL, MINB, TGX, true, false>(a, st);
    } else {
        if (v8) launch_list_p<T, VC, UNROLL, MINB, TGX, false, kCanV8>(a, st);
        else launch_list_p<T, VC, UNROLL, MINB, TGX, false, false>(a, st);
    }
}

// CUDA-core gather of one storage type (hcg_gather_<type>.cu): `cells` cells
// per block (16: k_gather, 2 x 2 groups searched per channel slice; 32:
// k_gather_list, 8 groups building candidate lists once), `vc` channels per
// lane (1, 4 or 8) and `depth` candidate rows in flight (list kernel: 8 or
// 12).  The caller has validated the combination.
template <typename T>
int launch_gather_dt(const GatherArgs &a, cudaStream_t st, int cells, int vc, int depth);

template <>
int launch_gather_dt<float>(const GatherArgs &, cudaStream_t, int, int, int);
template <>
int launch_gather_dt<__nv_bfloat16>(const GatherArgs &, cudaStream_t, int, int, int);
template <>
int launch_gather_dt<__nv_fp8_storage_t>(const GatherArgs &, cudaStream_t, int, int, int);

// Body of launch_gather_dt, compiled in the per-type units.
template <typename T>
int launch_gather_body(const GatherArgs &a, cudaStream_t st, int cells, int vc, int depth) {
    const int C = a.nchan;
    if (cells == 32) {
        if (vc == 4) launch_list_t<T, 4, 8, 3, 8>(a, st);
        else if (depth == 8) launch_list_t<T, 8, 8, 2, 8>(a, st);
        else launch_list_t<T, 8, 12, 2, 8>(a, st);
    } else if (vc == 8) {
        launch_t<T, 8, 32>(a, st);
    } else if (vc == 1) {
        launch_t<T, 1, 1>(a, st);
    } else if (C >= 128) {            // vc == 4: lanes across channels, the rest across candidates
        launch_t<T, 4, 32>(a, st);
    } else if (C >= 64) {
        launch_t<T, 4, 16>(a, st);
    } else if (C >= 16) {
        launch_t<T, 4, 4>(a, st);
    } else {
        launch_t<T, 4, 1>(a, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { hcg_cuda_fail(e, "gather launch"); return -1; }
    return 1;
}

}  // namespace hcg_gather

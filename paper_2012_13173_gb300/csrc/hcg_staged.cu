// hcg_staged.cu -- the CUDA-core gather of Eq. (1) (HCGrid Sec. 2.1, with
// the search of Sec. 3.4) in a form that stages candidate data and spectrum
// rows in shared memory with the TMA unit's bulk copies.
//
// A CTA owns a tile of (4 RX) x (4 RY) cells -- RX x RY regions of 4 x 4
// cells -- and a slice of 256 channels.  The tile's candidates are the union
// of the S' runs found through the two lookup tables for its cells (one
// window per ring), streamed in chunks of K:
//
//   producer warp   per chunk: the candidates' sorted data (offsets from the
//                   tile's first cell, cos lat, input row) into cand[s], then
//                   one bulk copy per candidate of its 256-channel row slice
//                   into rows[s], all completing on full[s];
//   2 warps/region  wait full[s]; each computes the weights of half of the
//                   region's 16 cells (two 2 x 2 quadrants) for the chunk's
//                   candidates, with the same support test and Gaussian as
//                   the other gathers, and a bit per (candidate, quadrant)
//                   telling whether any of its 4 weights is non-zero; a named
//                   barrier joins the pair; then each warp accumulates
//                   w * s for all 16 cells over its 128 channels (4 per
//                   lane, 64 accumulators), reading a row once from shared
//                   memory and only for the quadrants the candidate reaches,
//                   and arrives on empty[s].
//
// So a spectrum value read from shared memory feeds up to 16 cells (the
// list kernel's 2 x 2 groups feed 4), and the rows' latency is hidden by the
// stage ring instead of by registers.  Sums run over the candidates in S'
// order for every (cell, channel), so the result does not depend on the
// channel window.  Every wait is bounded (hcg_set_wait_limit); on a timeout
// the CTA stops, and the producer first waits for its copies in flight.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "hcg_async.cuh"
#include "hcg_search.cuh"

namespace {

constexpr int kNC = 256;                 // channels per CTA slice
constexpr int kMaxSegS = 512;            // S' runs per tile

struct StagedArgs {
    GridParams g;
    const float4 *uv;
    const float *cs;
    const uint32_t *row;
    const int64_t *upix, *ustart, *rustart;
    const float4 *rband;
    const double *lon, *lat;
    const void *spec;
    const float *scale;
    int nchan;                // channels of a spectrum row (of the window)
    float *cube, *wout;
    int64_t cube_ld;          // cube row stride (channels); cube points at the window's first channel
    unsigned long long *pairs;
    int *err;
    int ntx, nty;
    int64_t ntiles;
    int nslices;
    uint64_t wait_ns;
};

template <typename T>
struct Conv;

template <>
struct Conv<float> {
    static constexpr int kBytes = 4;
    HCG_DEV static float4 ld4(const unsigned char *p) { return *reinterpret_cast<const float4 *>(p); }
};

template <>
struct Conv<__nv_bfloat16> {
    static constexpr int kBytes = 2;
    HCG_DEV static float4 ld4(const unsigned char *p) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    }
};

template <>
struct Conv<__nv_fp8_storage_t> {
    static constexpr int kBytes = 1;
    HCG_DEV static float4 ld4(const unsigned char *p) {
        const uint32_t u = *reinterpret_cast<const uint32_t *>(p);
        __half2_raw a = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u & 0xffff), __NV_E4M3);
        __half2_raw b = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u >> 16), __NV_E4M3);
        const float2 fa = __half22float2(*reinterpret_cast<__half2 *>(&a));
        const float2 fb = __half22float2(*reinterpret_cast<__half2 *>(&b));
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
};

// Shared memory of one CTA (byte offsets from a 128-byte aligned base).
template <typename T, int RX, int RY, int K, int S>
struct SLayout {
    static constexpr int kRegions = RX * RY;
    static constexpr int kRowBytes = kNC * Conv<T>::kBytes;
    static constexpr int kRows = 0;                                        // [S][K][row slice]
    static constexpr int kCand = kRows + S * K * kRowBytes;                // float4 [S][K]
    static constexpr int kW = kCand + S * K * 16;                          // float [2][regions][K][16]
    static constexpr int kMask = kW + 2 * kRegions * K * 16 * 4;           // uint8 [2][regions][K][2]
    static constexpr int kSeg = kMask + ((2 * kRegions * K * 2 + 15) / 16) * 16;   // u32 [max][2] + 2
    static constexpr int kWtot = kSeg + kMaxSegS * 8 + 16;                 // float [regions][16]
    static constexpr int kBars = kWtot + kRegions * 16 * 4;                // u64 full[S], empty[S]
    static constexpr int kTot = kBars + 2 * S * 8;                         // float [consumer warps][64][32]
    static constexpr int kTotal = kTot + 2 * kRegions * 64 * 32 * 4;
};

// Weight of a cell for a candidate, from offsets relative to the tile's first
// cell (FP32, radians): the same quartic-corrected FP32 distance as the list
// kernel's pair test, the exact FP64 haversine inside the 1e-5 boundary band.
HCG_DEV float staged_weight(const GridParams &g, float du, float dv, float cc, int i, int j, bool cell_ok,
                            uint32_t rw, const double *lon, const double *lat, bool &inside) {
    const float x2 = dv * dv, y2 = du * du;
    const float h4 = x2 * (1.0f - x2 * (1.0f / 12.0f)) + cc * (y2 * (1.0f - y2 * (1.0f / 12.0f)));
    const float d2 = h4 * (1.0f + h4 * (1.0f / 12.0f));
    bool in = d2 <= g.band_lo;
    const bool valid = cell_ok && rw != 0xFFFFFFFFu;
    if (valid && !in && d2 <= g.band_hi) in = hav_exact_t<false>(g, i, j, lon[rw], lat[rw]) <= g.hR;
    inside = in && valid;
    return inside ? ex2_approx(-d2 * g.kexp) : 0.0f;
}

template <typename T, int RX, int RY, int K, int S, int kMinBlocks, bool kDense>
__global__ void __launch_bounds__((2 * RX * RY + 1) * 32, kMinBlocks) k_gather_staged(StagedArgs a) {
    using L = SLayout<T, RX, RY, K, S>;
    constexpr int kRegions = RX * RY;
    constexpr int kConsumers = 2 * kRegions;            // consumer warps
    constexpr int kTW = 4 * RX, kTH = 4 * RY;
    constexpr int kEB = Conv<T>::kBytes;
    static_assert(K == 16 || K == 32, "chunk depth K must be 16 or 32");
    extern __shared__ __align__(128) unsigned char dsm_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)dsm_raw + 127) & ~(uintptr_t)127);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile = blockIdx.x % a.ntiles;
    const int slice = (int)(blockIdx.x / a.ntiles);
    const int ty = a.nty - 1 - (int)(tile / a.ntx);      // north tile row first
    const int i0 = (int)(tile % a.ntx) * kTW, j0 = ty * kTH;
    const int c0 = slice * kNC;
    const int ncs = min(kNC, a.nchan - c0);              // channels of this slice
    const uint32_t row_bytes = (uint32_t)(ncs * kEB);
    const GridParams &g = a.g;

    float4 *cand = reinterpret_cast<float4 *>(sm + L::kCand);
    float *wbuf = reinterpret_cast<float *>(sm + L::kW);
    unsigned char *mbuf = sm + L::kMask;
    uint32_t *seg_b = reinterpret_cast<uint32_t *>(sm + L::kSeg);
    uint32_t *seg_off = seg_b + kMaxSegS;
    uint32_t *seg_n = seg_off + kMaxSegS;
    float *wtot = reinterpret_cast<float *>(sm + L::kWtot);
    const uint32_t bars = smem_u32(sm + L::kBars);
    auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bars + 8u * (uint32_t)(S + s); };

    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), kConsumers);
        }
        mbar_fence_init();
    }
    if (warp == kConsumers)
        tile_runs(g, a.upix, a.ustart, a.rustart, a.rband, i0, j0, kTW, kTH, seg_b, seg_off, seg_n, kMaxSegS, a.err);
    __syncthreads();
    const uint32_t nseg = seg_n[0], total = seg_n[1];
    const int nchunks = (int)((total + K - 1) / K);
    // tile origin (first cell) as FP32 hi + lo, radians from the grid centre
    float oah, oal, obh, obl;
    {
        const double A0 = ((double)i0 - g.hx) * g.pix * kDeg, B0 = ((double)j0 - g.hy) * g.pix * kDeg;
        oah = (float)A0; oal = (float)(A0 - (double)oah);
        obh = (float)B0; obl = (float)(B0 - (double)obh);
    }

    if (warp == kConsumers) {
        // ---------------- producer
        const T *spec = static_cast<const T *>(a.spec);
        int run = 0;                 // forward cursor: lane l's candidate grows by K per chunk
        // candidate data of chunk c (invalid past the end: row 0xFFFFFFFF)
        auto fetch = [&](int c) -> float4 {
            const uint32_t p = (uint32_t)c * K + (uint32_t)lane;
            if (lane >= K || p >= total) return make_float4(0.f, 0.f, 0.f, __uint_as_float(0xFFFFFFFFu));
            while (run < (int)nseg - 1 && seg_off[run] <= p) run++;
            const uint32_t sidx = seg_b[run] + (p - (run ? seg_off[run - 1] : 0u));
            const float4 uv = __ldg(a.uv + sidx);
            const float cn = __ldg(a.cs + sidx);
            const uint32_t rw = __ldg(a.row + sidx);
            return make_float4((uv.x - oah) + (uv.y - oal), (uv.z - obh) + (uv.w - obl), cn, __uint_as_float(rw));
        };
        int issued = 0;              // chunks whose copies were issued
        float4 nxt = nchunks > 0 ? fetch(0) : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = 0; c < nchunks; c++) {
            const int s = c % S;
            if (c >= S && !mbar_wait(empty(s), (uint32_t)(((c / S) - 1) & 1), a.err, a.wait_ns)) break;
            // this chunk's data was loaded one chunk ahead; start the next one's
            const float4 cd = nxt;
            if (c + 1 < nchunks) nxt = fetch(c + 1);
            const bool valid = __float_as_uint(cd.w) != 0xFFFFFFFFu;
            if (lane < K) cand[s * K + lane] = cd;
            const unsigned vmask = __ballot_sync(0xffffffffu, valid);
            __syncwarp();
            if (lane == 0) mbar_arrive_expect_tx(full(s), (uint32_t)__popc(vmask) * row_bytes);
            __syncwarp();
            if (valid) {
                const uint32_t rw = __float_as_uint(cd.w);
                const unsigned char *src = reinterpret_cast<const unsigned char *>(spec) +
                                           ((size_t)rw * (size_t)a.nchan + (size_t)c0) * kEB;
                bulk_g2s(smem_u32(sm + L::kRows + (s * K + lane) * L::kRowBytes), src, row_bytes, full(s));
            }
            issued = c + 1;
        }
        // copies still in flight land before the CTA may exit: wait for the
        // last S issued chunks' full phases (bounded; they complete on their own)
        for (int c = std::max(0, issued - S); c < issued; c++)
            mbar_wait(full(c % S), (uint32_t)((c / S) & 1), a.err, a.wait_ns);
        return;
    }

    // ---------------- consumers: warp = 2 r + h (region r, half h)
    const int r = warp >> 1, h = warp & 1;
    const int rx = r % RX, ry = r / RX;
    const int ci0 = i0 + 4 * rx, cj0 = j0 + 4 * ry;      // region's first cell
    // weight duty: candidate kc = lane % K, cells (x, y) with y in {2h, 2h+1}
    // (quadrants 2h, 2h+1); K = 16 splits the two rows between lane halves
    constexpr int kWY = K == 32 ? 2 : 1;                 // cell rows per lane
    const int kc = lane % K;
    const int y0 = 2 * h + (K == 32 ? 0 : lane / 16);
    float arel[4], brel[kWY], cgv[kWY];
    bool okc[4][kWY];
#pragma unroll
    for (int x = 0; x < 4; x++) {
        const int i = min(ci0 + x, g.nx - 1);
        arel[x] = (float)((double)(i - i0) * g.pix * kDeg);
    }
#pragma unroll
    for (int yy = 0; yy < kWY; yy++) {
        const int j = min(cj0 + y0 + yy, g.ny - 1);
        brel[yy] = (float)((double)(j - j0) * g.pix * kDeg);
        cgv[yy] = cosf((float)((g.lat0 + ((double)j - g.hy) * g.pix) * kDeg));
#pragma unroll
        for (int x = 0; x < 4; x++) okc[x][yy] = (ci0 + x < g.nx) && (cj0 + y0 + yy < g.ny);
    }
    float wsum[4][kWY];
#pragma unroll
    for (int x = 0; x < 4; x++)
#pragma unroll
        for (int yy = 0; yy < kWY; yy++) wsum[x][yy] = 0.f;
    unsigned npairs = 0;

    // accumulation duty: channels c0 + 128 h + 4 lane .. + 3, all 16 cells
    const int cl = 128 * h + 4 * lane;                   // channel within the slice
    const bool has_ch = cl < ncs;
    // part[quadrant][cell in quadrant][channel]: sums over the current block
    // of 64 candidates, added when the block ends into the lane's running
    // totals, kept in shared memory (tot[k][lane], conflict-free): a two-level
    // sum, whose rounding error grows with sqrt(64) + sqrt(N / 64) rather
    // than sqrt(N) -- four times smaller at N = 3600 contributors
    constexpr int kFlush = 64 / K;                       // chunks per block of 64 candidates
    float *tot = reinterpret_cast<float *>(sm + L::kTot) + (size_t)warp * 64 * 32 + lane;
    float part[4][4][4];
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int e = 0; e < 4; e++)
#pragma unroll
            for (int v = 0; v < 4; v++) {
                part[q][e][v] = 0.f;
                tot[(16 * q + 4 * e + v) * 32] = 0.f;
            }

    bool ok = true;
    for (int c = 0; c < nchunks; c++) {
        const int s = c % S, buf = c & 1;
        ok = ok && mbar_wait(full(s), (uint32_t)((c / S) & 1), a.err, a.wait_ns);
        // weights of this lane's candidate for its cells, and quadrant bits
        {
            const float4 cd = cand[s * K + kc];
            const uint32_t rw = __float_as_uint(cd.w);
            float w[4][kWY];
            unsigned qbits = 0;
#pragma unroll
            for (int yy = 0; yy < kWY; yy++) {
                const float dv = cd.y - brel[yy];
                const float cc = cgv[yy] * cd.z;
#pragma unroll
                for (int x = 0; x < 4; x++) {
                    bool in;
                    w[x][yy] = staged_weight(g, cd.x - arel[x], dv, cc, ci0 + x, cj0 + y0 + yy, okc[x][yy], rw,
                                             a.lon, a.lat, in);
                    wsum[x][yy] += w[x][yy];
                    npairs += in;
                    if (in) qbits |= 1u << (x >> 1);
                }
            }
            // quadrant q = 2 * (y / 2) + x / 2; this lane's rows lie in quadrant row h
            float *wr = wbuf + ((size_t)(buf * kRegions + r) * K + kc) * 16;
            if (K == 32) {
#pragma unroll
                for (int qx = 0; qx < 2; qx++)   // cell e = 2 (y % 2) + x % 2 within the quadrant
                    *reinterpret_cast<float4 *>(wr + (2 * h + qx) * 4) =
                        make_float4(w[2 * qx][0], w[2 * qx + 1][0], w[2 * qx][kWY - 1], w[2 * qx + 1][kWY - 1]);
                mbuf[((buf * kRegions + r) * K + kc) * 2 + h] = (unsigned char)qbits;
            } else {
                const int yo = lane / 16;        // which row of the quadrant
#pragma unroll
                for (int qx = 0; qx < 2; qx++)
                    *reinterpret_cast<float2 *>(wr + (2 * h + qx) * 4 + 2 * yo) = make_float2(w[2 * qx][0], w[2 * qx + 1][0]);
                qbits |= __shfl_xor_sync(0xffffffffu, qbits, 16);
                if (lane < 16) mbuf[((buf * kRegions + r) * K + kc) * 2 + h] = (unsigned char)qbits;
            }
        }
        // the pair agrees on going on, and sees both halves' weights
        const bool stop = bar_red_or(1 + r, 64, !ok);
        if (stop) { ok = false; break; }
        // accumulate
        const float *wr = wbuf + (size_t)(buf * kRegions + r) * K * 16;
        const unsigned char *mr = mbuf + (size_t)(buf * kRegions + r) * K * 2;
        const unsigned char *rows = sm + L::kRows + (size_t)s * K * L::kRowBytes + (size_t)cl * kEB;
        if constexpr (kDense) {
            // wide supports: nearly every candidate reaches every quadrant, so
            // all 16 cells take every candidate (a zero weight adds nothing)
            // with no branches; the next candidate's row and weights are
            // loaded before this one's multiply-adds.  Lanes past the slice's
            // channels read their row slot's unused bytes and store nothing.
            float4 x = Conv<T>::ld4(rows);
            float4 w0 = *reinterpret_cast<const float4 *>(wr), w1 = *reinterpret_cast<const float4 *>(wr + 4);
            float4 w2 = *reinterpret_cast<const float4 *>(wr + 8), w3 = *reinterpret_cast<const float4 *>(wr + 12);
#pragma unroll 2
            for (int k = 0; k < K; k++) {
                const int kn = k + 1 < K ? k + 1 : k;
                const float4 xn = Conv<T>::ld4(rows + (size_t)kn * L::kRowBytes);
                const float4 n0 = *reinterpret_cast<const float4 *>(wr + kn * 16);
                const float4 n1 = *reinterpret_cast<const float4 *>(wr + kn * 16 + 4);
                const float4 n2 = *reinterpret_cast<const float4 *>(wr + kn * 16 + 8);
                const float4 n3 = *reinterpret_cast<const float4 *>(wr + kn * 16 + 12);
                const float4 wq[4] = {w0, w1, w2, w3};
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const float we[4] = {wq[q].x, wq[q].y, wq[q].z, wq[q].w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        part[q][e][0] = fmaf(we[e], x.x, part[q][e][0]);
                        part[q][e][1] = fmaf(we[e], x.y, part[q][e][1]);
                        part[q][e][2] = fmaf(we[e], x.z, part[q][e][2]);
                        part[q][e][3] = fmaf(we[e], x.w, part[q][e][3]);
                    }
                }
                x = xn; w0 = n0; w1 = n1; w2 = n2; w3 = n3;
            }
            (void)mr;
        } else {
#pragma unroll 2
            for (int k = 0; k < K; k++) {
                const unsigned m2 = *reinterpret_cast<const unsigned short *>(mr + 2 * k);
                const unsigned m = (m2 & 3u) | ((m2 >> 8) & 3u) << 2;
                if (m == 0) continue;
                const float4 x = Conv<T>::ld4(rows + (size_t)k * L::kRowBytes);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (!((m >> q) & 1u)) continue;
                    const float4 w4 = *reinterpret_cast<const float4 *>(wr + k * 16 + q * 4);
                    const float we[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        part[q][e][0] = fmaf(we[e], x.x, part[q][e][0]);
                        part[q][e][1] = fmaf(we[e], x.y, part[q][e][1]);
                        part[q][e][2] = fmaf(we[e], x.z, part[q][e][2]);
                        part[q][e][3] = fmaf(we[e], x.w, part[q][e][3]);
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty(s));
        if (c % kFlush == kFlush - 1 || c == nchunks - 1) {
#pragma unroll
            for (int q = 0; q < 4; q++)
#pragma unroll
                for (int e = 0; e < 4; e++)
#pragma unroll
                    for (int v = 0; v < 4; v++) {
                        tot[(16 * q + 4 * e + v) * 32] += part[q][e][v];
                        part[q][e][v] = 0.f;
                    }
        }
    }

    // ---------------- epilogue: W per cell, then the normalised cube
    // lanes sharing cells hold partial sums over disjoint candidates
#pragma unroll
    for (int x = 0; x < 4; x++)
#pragma unroll
        for (int yy = 0; yy < kWY; yy++) {
            float t = wsum[x][yy];
#pragma unroll
            for (int o = K / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            wsum[x][yy] = t;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    if (lane % K == 0) {
#pragma unroll
        for (int x = 0; x < 4; x++)
#pragma unroll
            for (int yy = 0; yy < kWY; yy++) {
                const int y = y0 + yy;
                wtot[r * 16 + 4 * (2 * (y >> 1) + (x >> 1)) + 2 * (y & 1) + (x & 1)] = wsum[x][yy];
            }
    }
    bar_sync(1 + r, 64);
    const bool vec_out = (a.cube_ld & 3) == 0 && ((uintptr_t)a.cube & 15) == 0;
    if (ok) {
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int x = 2 * (q & 1) + (e & 1), y = 2 * (q >> 1) + (e >> 1);
                const int i = ci0 + x, j = cj0 + y;
                if (i >= g.nx || j >= g.ny) continue;
                const float W = wtot[r * 16 + 4 * q + e];
                if (slice == 0 && h == 0 && lane == 0) a.wout[(size_t)j * g.nx + i] = W;
                if (!has_ch) continue;
                float y4[4];
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const float sv = tot[(16 * q + 4 * e + v) * 32];
                    float val;
                    if (W >= 1e-3f) val = __fdiv_rn(sv, W);
                    else if (W > 0.0f) val = (float)((double)sv / (double)W);
                    else val = __int_as_float(0x7fc00000);
                    if (a.scale) val *= __ldg(a.scale + c0 + cl + v);
                    y4[v] = val;
                }
                float *out = a.cube + ((size_t)j * g.nx + i) * (size_t)a.cube_ld + c0 + cl;
                if (vec_out) {
                    __stcs(reinterpret_cast<float4 *>(out), make_float4(y4[0], y4[1], y4[2], y4[3]));
                } else {
#pragma unroll
                    for (int v = 0; v < 4; v++) __stcs(out + v, y4[v]);
                }
            }
    }
    // each consumer warp adds its own in-support pair count (npairs holds the
    // warp's sum over its cells; the two warps of a region count disjoint cells)
    if (slice == 0 && lane == 0 && npairs && a.pairs) atomicAdd(a.pairs, (unsigned long long)npairs);
}

template <typename T, int RX, int RY, int K, int S, int MINB, bool DENSE>
int launch_staged_t(const StagedArgs &a, cudaStream_t st) {
    using L = SLayout<T, RX, RY, K, S>;
    const int smem = L::kTotal + 128;
    auto kern = k_gather_staged<T, RX, RY, K, S, MINB, DENSE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) { hcg_cuda_fail(e, "staged gather smem attribute"); return -1; }
    const int64_t blocks = a.ntiles * a.nslices;
    kern<<<(unsigned)blocks, (2 * RX * RY + 1) * 32, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { hcg_cuda_fail(e, "k_gather_staged"); return -1; }
    return 1;
}

// cells_per_block: 32 (8 x 4 cells) or 64 (8 x 8); depth: K (16 or 32).
// Depth 16 keeps two CTAs per SM (stage ring and totals within half the
// shared memory, at most 112 registers a thread); depth 32 runs one.
template <typename T, bool DENSE>
int launch_staged_mode(const StagedArgs &a, cudaStream_t st, int cells, int depth) {
    if (cells == 32)
        return depth == 16 ? launch_staged_t<T, 2, 1, 16, 4, 2, DENSE>(a, st) : launch_staged_t<T, 2, 1, 32, 3, 1, DENSE>(a, st);
    return depth == 16 ? launch_staged_t<T, 2, 2, 16, 4, 2, DENSE>(a, st) : launch_staged_t<T, 2, 2, 32, 3, 1, DENSE>(a, st);
}

// Supports of 4 or more cells' radius reach nearly every quadrant of a tile
// from nearly every candidate: the branch-free dense sweep; narrower ones
// skip the quadrants a candidate does not reach.
template <typename T>
int launch_staged_dt(const StagedArgs &a, cudaStream_t st, int cells, int depth) {
    if (a.g.R_deg >= 4.0 * a.g.pix) return launch_staged_mode<T, true>(a, st, cells, depth);
    return launch_staged_mode<T, false>(a, st, cells, depth);
}

}  // namespace

bool staged_supported(const hcg_ctx *c, int dtype, int32_t win_nchan) {
    if (c->proj != HCG_CAR) return false;                  // tiles use the plain grid's cell offsets
    const int eb = dtype == HCG_F32 ? 4 : (dtype == HCG_BF16 ? 2 : 1);
    if (win_nchan < 128) return false;
    if (((int64_t)win_nchan * eb) % 16 != 0) return false; // 16-byte aligned row slices
    // rings spanned by an 8 x 8 tile (the largest), two runs each, within the run table
    const double pixsz = sqrt(3.14159265358979323846 / 3.0) / (double)c->nside * 57.29577951308232;
    const double rings = (8.0 * c->pix + 2.0 * c->support) / (0.5 * pixsz) + 8.0;
    return rings * 2.0 < kMaxSegS;
}

int launch_staged(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale, int cells,
                  int depth) {
    StagedArgs a;
    a.g = gp;
    const hcg_ctx *t = c->tables();
    a.uv = t->sc_uv; a.cs = t->sc_cos; a.row = t->sc_row;
    a.upix = t->upix; a.ustart = t->ustart; a.rustart = t->rustart; a.rband = t->rband;
    a.lon = c->lon; a.lat = c->lat;
    a.spec = spec; a.scale = scale; a.nchan = c->win_channels();
    a.cube = c->cube() + c->win_c0; a.cube_ld = c->nchan; a.wout = c->weights();
    a.pairs = c->win_c0 == 0 ? reinterpret_cast<unsigned long long *>(c->dscal + 1) : nullptr;
    a.err = c->derr;
    a.wait_ns = (uint64_t)c->wait_ns;
    const int tw = 8, th = cells == 32 ? 4 : 8;
    a.ntx = (c->nx + tw - 1) / tw;
    a.nty = (c->ny + th - 1) / th;
    a.ntiles = (int64_t)a.ntx * a.nty;
    a.nslices = (a.nchan + kNC - 1) / kNC;
    if (((uintptr_t)spec & 15) != 0) { hcg_set_error("staged gather: spectra not 16-byte aligned"); return -1; }
    if (dtype == HCG_F32) return launch_staged_dt<float>(a, c->stream, cells, depth);
    if (dtype == HCG_BF16) return launch_staged_dt<__nv_bfloat16>(a, c->stream, cells, depth);
    return launch_staged_dt<__nv_fp8_storage_t>(a, c->stream, cells, depth);
}

// hcg_prep.cu -- the pre-ordering half of the path (HCGrid Sec. 3.3):
//   k_prep       HEALPix RING pixel of every sample -> 64-bit sort key (step I)
//   radix sort   stable LSD sort of (key, sample index)              (step I)
//   k_permute    sorted pixel array P' and the per-sample data of S'  (step I)
//   k_lut1_*     first-level table pixel -> S_start                   (step II)
//   k_lut2       second-level table ring -> R_start                   (step III)
//   k_quant_*    optional BF16 / FP8-e4m3 storage of the spectra
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "hcg_dev.cuh"

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                       // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per tile
constexpr int kSortWarps = kSortThreads / 32;

// ---------------------------------------------------------------- k_prep --
// Step I: P_n = pix(alpha_n, delta_n).  Packed form (pixel offsets below
// 2^32): the key is (P_n - pix_lo) above a 32-bit coordinate hash, so one
// stable sort gives the order (pixel, hash, input index), and samples whose
// ring the grid cannot reach get the all-ones key and sort to the end.
// Wide form (ring ranges of 2^32 pixels or more): the key is the hash alone
// and the pixel offset goes to pixoff[n] (pix_sentinel for dropped samples);
// the sort then runs the hash digits first and the pixel-offset digits after
// them, which yields the same order.
__global__ void k_prep(const double *__restrict__ lon, const double *__restrict__ lat, int64_t n,
                       GridParams g, uint64_t sentinel, uint64_t *__restrict__ keys,
                       uint32_t *__restrict__ vals, uint64_t *__restrict__ pixoff, uint64_t pix_sentinel,
                       int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo = lon[i], la = lat[i];
    uint64_t key = sentinel, po = pix_sentinel;
    uint32_t h = 0;
    if (!isfinite(lo) || !isfinite(la) || fabs(la) > 90.0) {
        set_err(err, HCG_DERR_BAD_COORD);
    } else {
        int64_t ring;
        int64_t p = ang2pix_ring_screened(g.nside, lo, la, g.screen_eps, &ring);
        h = coord_hash(lo, la);
        if (ring >= g.r_lo && ring <= g.r_hi) {
            po = (uint64_t)(p - g.pix_lo);
            key = (po << 32) | (uint64_t)h;
        }
    }
    if (pixoff) {
        keys[i] = (uint64_t)h;
        pixoff[i] = po;
    } else {
        keys[i] = key;
    }
    vals[i] = (uint32_t)i;
}

// Wide form, between the two digit phases: each sorted entry takes the pixel
// offset of its input sample as its key.
__global__ void k_pix_keys(uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                           const uint64_t *__restrict__ pixoff) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    keys[q] = pixoff[vals[q]];
}

// Exclusive scan over the 256 threads of a block (one value each).
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t *total) {
    __shared__ uint32_t ws8[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws8[warp] = x;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) { uint32_t t = ws8[w]; if (w < warp) pre += t; tot += t; }
    *total = tot;
    return pre + x - v;
}

// ------------------------------------------------------------ radix sort --
// LSD radix sort, 8-bit digits, stable.  Per pass: k_hist counts digits per
// tile (counts laid out digit-major, so one exclusive scan of the count array
// yields every tile's output offset per digit), then k_scatter ranks each key
// within its tile (warp match + per-warp counters, in input order) and writes
// it to its final position.
__global__ void __launch_bounds__(kSortThreads) k_hist(const uint64_t *__restrict__ keys, int64_t n,
                                                      int shift, int64_t ntiles,
                                                      uint32_t *__restrict__ counts) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        int64_t e = base + k * kSortThreads + threadIdx.x;
        if (e < n) atomicAdd(&h[(keys[e] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_scatter(const uint64_t *__restrict__ kin,
                                                         const uint32_t *__restrict__ vin,
                                                         uint64_t *__restrict__ kout,
                                                         uint32_t *__restrict__ vout, int64_t n,
                                                         int shift, int64_t ntiles,
                                                         const uint32_t *__restrict__ offs) {
    __shared__ uint32_t wc[kSortWarps][256];
    __shared__ uint32_t dstart[257];                 // tile-local start of each digit
    __shared__ uint64_t sk[kSortTile];               // the tile in digit order
    __shared__ uint32_t sv[kSortTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortThreads) (&wc[0][0])[d] = 0;
    __syncthreads();
    // warp w owns tile elements [w*256, w*256+256), visited in 8 rounds of 32
    const int64_t base = (int64_t)blockIdx.x * kSortTile + warp * (32 * kSortItems);
    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
    int rank[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        int64_t e = base + k * 32 + lane;
        bool ok = e < n;
        key[k] = ok ? kin[e] : 0;
        val[k] = ok ? vin[e] : 0;
        int d = ok ? (int)((key[k] >> shift) & 0xFF) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = 0;
        if (ok) before = wc[warp][d];
        __syncwarp();
        int leader = __ffs(peers) - 1;
        if (ok && lane == leader) wc[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[k] = ok ? before + __popc(peers & lt) : -1;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps (warps hold consecutive key ranges),
    // and the tile-local start of every digit
    {
        int d = threadIdx.x;   // kSortThreads == 256 digits
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) {
            uint32_t t = wc[w][d];
            wc[w][d] = run;
            run += t;
        }
        uint32_t tot;
        uint32_t ex = block_exclusive_scan_256(run, &tot);
        dstart[d] = ex;
        if (d == 0) dstart[256] = tot;
    }
    __syncthreads();
    // stage the tile in digit order, then write each digit's run contiguously
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        if (rank[k] < 0) continue;
        int d = (int)((key[k] >> shift) & 0xFF);
        uint32_t loc = dstart[d] + wc[warp][d] + rank[k];
        sk[loc] = key[k];
        sv[loc] = val[k];
    }
    __syncthreads();
    const uint32_t cnt = dstart[256];
    for (uint32_t loc = threadIdx.x; loc < cnt; loc += kSortThreads) {
        uint64_t kk = sk[loc];
        int d = (int)((kk >> shift) & 0xFF);
        int64_t pos = (int64_t)offs[(int64_t)d * ntiles + blockIdx.x] + (loc - dstart[d]);
        kout[pos] = kk;
        vout[pos] = sv[loc];
    }
}

// ------------------------------------------------------- one-sweep sort --
// The same stable LSD sort with one scatter launch per digit pass: one
// histogram kernel counts every pass's digits at once, one small kernel turns
// them into global digit offsets, and each pass's tiles find where their
// digits go by a decoupled look-back -- tile t publishes its digit counts, then
// adds up its predecessors' counts (or the first inclusive prefix it meets)
// and publishes its own prefix.  Tiles take their index from an atomic
// counter when they start, so every predecessor a tile waits for is already
// running; the waits are bounded all the same (TIMEOUT bit).  A status word
// holds a tag (the sort's epoch and the pass), a flag (1 = count, 2 = prefix)
// and the value, so stale words of an earlier pass never match.
// hist words: [0, 2048) digit counts [pass][256]; [2048, 4096) global digit
// offsets; [4096, 4104) tile counters per pass; [4104] the epoch.
constexpr int kHistCounts = 0, kHistOffsets = 2048, kHistTiles = 4096, kHistEpoch = 4104;
constexpr uint32_t kSpinLimit = 1u << 20;

__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const uint64_t *__restrict__ keys, int64_t n,
                                                            int passes, uint32_t *hist) {
    __shared__ uint32_t h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kSortThreads) {
        const uint64_t k = keys[e];
        for (int p = 0; p < passes; p++) atomicAdd(&h[p][(k >> (8 * p)) & 0xFF], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += kSortThreads) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(hist + kHistCounts + i, v);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(hist + kHistEpoch, 1u);
}

__global__ void __launch_bounds__(kSortThreads) k_digit_offsets(uint32_t *hist, int passes) {
    for (int p = 0; p < passes; p++) {
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan_256(hist[kHistCounts + p * 256 + threadIdx.x], &tot);
        hist[kHistOffsets + p * 256 + threadIdx.x] = ex;
        __syncthreads();
    }
}

HCG_DEV uint64_t status_word(uint32_t tag, uint32_t flag, uint32_t value) {
    return ((uint64_t)tag << 34) | ((uint64_t)flag << 32) | (uint64_t)value;
}
// Status words carry flag and value together, so relaxed device-scope
// accesses suffice (no other data is published through them).
HCG_DEV uint64_t ld_status(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
HCG_DEV void st_status(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(kSortThreads) k_onesweep(const uint64_t *__restrict__ kin,
                                                          const uint32_t *__restrict__ vin,
                                                          uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                          int64_t n, int pass, uint32_t *hist,
                                                          uint64_t *status, int *err) {
    __shared__ uint32_t wc[kSortWarps][256];
    __shared__ uint32_t dstart[257];
    __shared__ uint64_t sk[kSortTile];
    __shared__ uint32_t sv[kSortTile];
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int shift = 8 * pass;
    if (threadIdx.x == 0) s_tile = atomicAdd(hist + kHistTiles + pass, 1u);
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortThreads) (&wc[0][0])[d] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t tag = (uint32_t)((__ldcg(hist + kHistEpoch) * 8ull + (uint64_t)pass) % 0x3FFFFFFFull) + 1u;
    // rank each key within the tile (warps own consecutive key ranges, in input order)
    const int64_t base = (int64_t)tile * kSortTile + warp * (32 * kSortItems);
    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
    int rank[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        int64_t e = base + k * 32 + lane;
        bool ok = e < n;
        key[k] = ok ? kin[e] : 0;
        val[k] = ok ? vin[e] : 0;
        int d = ok ? (int)((key[k] >> shift) & 0xFF) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = 0;
        if (ok) before = wc[warp][d];
        __syncwarp();
        int leader = __ffs(peers) - 1;
        if (ok && lane == leader) wc[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[k] = ok ? before + __popc(peers & lt) : -1;
    }
    __syncthreads();
    {
        const int d = threadIdx.x;   // kSortThreads == 256 digits
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) {
            uint32_t t = wc[w][d];
            wc[w][d] = run;
            run += t;
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan_256(run, &tot);
        dstart[d] = ex;
        if (d == 0) dstart[256] = tot;
        // decoupled look-back over the earlier tiles' counts of digit d
        uint64_t *st = status + (size_t)tile * 256 + d;
        uint32_t excl = 0;
        if (tile == 0) {
            st_status(st, status_word(tag, 2u, run));
        } else {
            st_status(st, status_word(tag, 1u, run));
            int64_t t = (int64_t)tile - 1;
            uint32_t spins = 0;
            for (;;) {
                const uint64_t v = ld_status(status + (size_t)t * 256 + d);
                if ((uint32_t)(v >> 34) == tag) {
                    excl += (uint32_t)v;
                    if (((v >> 32) & 3u) == 2u) break;
                    t--;
                    spins = 0;
                    continue;
                }
                if (++spins > kSpinLimit) { set_err(err, HCG_DERR_TIMEOUT); break; }
            }
            st_status(st, status_word(tag, 2u, excl + run));
        }
        s_base[d] = hist[kHistOffsets + pass * 256 + d] + excl;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        if (rank[k] < 0) continue;
        int d = (int)((key[k] >> shift) & 0xFF);
        uint32_t loc = dstart[d] + wc[warp][d] + rank[k];
        sk[loc] = key[k];
        sv[loc] = val[k];
    }
    __syncthreads();
    const uint32_t cnt = dstart[256];
    for (uint32_t loc = threadIdx.x; loc < cnt; loc += kSortThreads) {
        const uint64_t kk = sk[loc];
        const int d = (int)((kk >> shift) & 0xFF);
        const int64_t pos = (int64_t)s_base[d] + (loc - dstart[d]);
        kout[pos] = kk;
        vout[pos] = sv[loc];
    }
}

// ---------------------------------------------------------------- scan ----
// Exclusive scan of uint32 (sums fit in 32 bits: at most 2^31 elements).
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    uint32_t wprefix = warp ? ws[warp - 1] : 0;
    if (total) *total = ws[(blockDim.x >> 5) - 1];
    uint32_t r = wprefix + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ d, int64_t n,
                                                             uint32_t *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) if (base + k < n) s += d[base + k];
    uint32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// exclusive scan of one tile in place, plus an optional per-tile offset
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(uint32_t *__restrict__ d, int64_t n,
                                                           const uint32_t *__restrict__ offs) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) { v[k] = (base + k < n) ? d[base + k] : 0; s += v[k]; }
    uint32_t run = block_exclusive_scan(s, nullptr) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) d[base + k] = run;
        run += v[k];
    }
}

// -------------------------------------------------------------- permute ---
// S' and P': for sorted position q, the pixel P'[q] (INT64_MAX for dropped
// samples; the keys hold the pixel offset from bit kshift up: 32 packed, 0
// wide), the input index, and the coordinates the gather reads: offsets
// from the grid centre in radians, split into FP32 hi + lo parts (computed
// once here in FP64), and cos(lat) in FP32.
__global__ void k_permute(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                          const double *__restrict__ lon, const double *__restrict__ lat, GridParams g,
                          uint64_t sentinel, int kshift, int64_t *__restrict__ psorted, float4 *__restrict__ uv,
                          float *__restrict__ cs, uint32_t *__restrict__ row) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint64_t key = keys[q];
    uint32_t s = vals[q];
    row[q] = s;
    if (key == sentinel) {
        psorted[q] = INT64_MAX;
        uv[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        cs[q] = 0.f;
        return;
    }
    psorted[q] = g.pix_lo + (int64_t)(key >> kshift);
    double lo = lon[s], la = lat[s];
    double dl = lo - g.lon0;
    if (fabs(dl) > 540.0) dl = wrap180(dl);          // rare: inputs far outside
    if (dl > 180.0) dl -= 360.0;
    if (dl <= -180.0) dl += 360.0;
    double U = dl * kDeg;
    double V = (la - g.lat0) * kDeg;
    float uh = (float)U, vh = (float)V;
    uv[q] = make_float4(uh, (float)(U - (double)uh), vh, (float)(V - (double)vh));
    cs[q] = cosf((float)(la * kDeg));
}

// ------------------------------------------------------------------ LUT ---
// Step II: flag the first sample of every distinct pixel of P'.
__global__ void k_lut1_flags(const int64_t *__restrict__ ps, int64_t n, uint32_t *__restrict__ f) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    f[q] = (q == 0 || ps[q] != ps[q - 1]) ? 1u : 0u;
}

// After the exclusive scan of the flags: upix[k] = k-th distinct pixel,
// ustart[k] = its first position (S_start), ustart[U_total] = n.
__global__ void k_lut1_compact(const int64_t *__restrict__ ps, int64_t n, const uint32_t *__restrict__ pos,
                               int64_t *__restrict__ upix, int64_t *__restrict__ ustart,
                               int64_t *__restrict__ dscal) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    bool first = (q == 0 || ps[q] != ps[q - 1]);
    if (first) { upix[pos[q]] = ps[q]; ustart[pos[q]] = q; }
    if (q == n - 1) {
        int64_t total = (int64_t)pos[q] + (first ? 1 : 0);
        ustart[total] = n;
        dscal[0] = total;
    }
}

// z = sin(latitude) at continuous ring coordinate rc (the inverse of the
// ring coordinate of the gather's ring-range step; Gorski et al. 2005 Eqs. 4-5
// solved for z, clamped to [0, 4 nside]).
HCG_DEV double z_of_ring_coord(double ns, double rc) {
    rc = fmin(fmax(rc, 0.0), 4.0 * ns);
    if (rc <= ns) { double t = rc / ns; return 1.0 - t * t / 3.0; }
    if (rc >= 3.0 * ns) { double t = 4.0 - rc / ns; return t * t / 3.0 - 1.0; }
    return (2.0 - rc / ns) / 1.5;
}

// Step III: R_start[r - r_lo] = first position of ring r in P' (into S'),
// and the matching position in the distinct-pixel table, r in [r_lo, r_hi+1].
// Beside it, the latitude band that holds every sample of ring r (continuous
// ring coordinate in (r - 1, r + 1)): x = south edge, y = north edge, radians,
// widened by 1e-6; z = a lower bound of cos(latitude) over the band.  The
// gather narrows each ring's longitude window with it.
__global__ void k_lut2(const int64_t *__restrict__ ps, int64_t n, const int64_t *__restrict__ upix,
                       const int64_t *__restrict__ dscal, GridParams g, int64_t *__restrict__ rstart,
                       int64_t *__restrict__ rustart, float4 *__restrict__ rband) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nr = g.r_hi - g.r_lo + 2;
    if (k >= nr) return;
    const int64_t r = g.r_lo + k;
    int64_t first = ring_first_pix(g.nside, r);
    rstart[k] = lower_bound_i64(ps, 0, n, first);
    int64_t u = n > 0 ? dscal[0] : 0;
    rustart[k] = lower_bound_i64(upix, 0, u, first);
    const double ns = (double)g.nside, margin = 1e-6, half_pi = 1.5707963267948966;
    const double south = asin(z_of_ring_coord(ns, (double)(r + 1))) - margin;
    const double north = asin(z_of_ring_coord(ns, (double)(r - 1))) + margin;
    const double amax = fmin(half_pi, fmax(fabs(south), fabs(north)));
    const double cmin = fmax(0.0, cos(amax) * (1.0 - 1e-6) - 1e-7);
    rband[k] = make_float4(__double2float_rd(south), __double2float_ru(north), __double2float_rd(cmin), 0.0f);
}

// ------------------------------------------------------------- quantise ---
__global__ void k_to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, int64_t m, int *err) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (i >= m) return;
    if (i + 4 <= m) {
        float4 v = *reinterpret_cast<const float4 *>(x + i);
        if (!isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w)) set_err(err, HCG_DERR_NONFINITE);
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        *reinterpret_cast<__nv_bfloat162 *>(y + i) = a;
        *reinterpret_cast<__nv_bfloat162 *>(y + i + 2) = b;
    } else {
        for (int64_t k = i; k < m; k++) {
            if (!isfinite(x[k])) set_err(err, HCG_DERR_NONFINITE);
            y[k] = __float2bfloat16_rn(x[k]);
        }
    }
}

// per-channel max |x| over finite values (bit pattern max == float max for >= 0)
__global__ void k_amax(const float *__restrict__ x, int64_t n, int nchan, int64_t rows_per_block,
                       uint32_t *__restrict__ amax, int *err) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchan) return;
    int64_t r0 = (int64_t)blockIdx.y * rows_per_block, r1 = min(n, r0 + rows_per_block);
    float m = 0.f;
    bool bad = false;
    for (int64_t r = r0; r < r1; r++) {
        float v = x[r * nchan + c];
        if (isfinite(v)) m = fmaxf(m, fabsf(v)); else bad = true;
    }
    if (bad) set_err(err, HCG_DERR_NONFINITE);
    atomicMax(amax + c, __float_as_uint(m));
}

__global__ void k_scales(const uint32_t *__restrict__ amax, int nchan, float *__restrict__ s) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchan) return;
    float a = __uint_as_float(amax[c]);
    s[c] = a > 0.f ? __fdiv_rn(a, 448.0f) : 1.0f;
}

__global__ void k_to_e4m3(const float *__restrict__ x, const float *__restrict__ s, __nv_fp8_storage_t *__restrict__ y,
                          int64_t n, int nchan) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nchan) return;
    int c = (int)(i % nchan);
    float v = __fdiv_rn(x[i], s[c]);
    y[i] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ============================================================ launchers ===
int64_t sort_tiles(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

static int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { hcg_cuda_fail(e, what); return -1; }
    return 0;
}

// Key layout of a pass: key_bits = bits of the pixel offset + 32 hash bits.
// Up to 64 bits the two are packed in one key ("packed"); above, the hash
// digits are sorted first and the pixel-offset digits after them ("wide").
static bool wide_key(int key_bits) { return key_bits > 64; }

static uint64_t packed_sentinel(int key_bits) { return key_bits >= 64 ? ~0ull : ((1ull << key_bits) - 1); }

// Wide form: the dropped-sample pixel offset, above every offset in range.
static uint64_t pix_sentinel(int key_bits) { return (1ull << (key_bits - 32)) - 1; }

int launch_prep(hcg_ctx *c, const GridParams &gp, int key_bits) {
    if (c->n == 0) return 0;
    const bool wide = wide_key(key_bits);
    // wide keys park the pixel offsets in the P' buffer until the sort's
    // second phase has read them (k_permute overwrites it afterwards)
    k_prep<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(
        c->lon, c->lat, c->n, gp, packed_sentinel(key_bits), c->sort.keys[0], c->sort.vals[0],
        wide ? reinterpret_cast<uint64_t *>(c->psorted) : nullptr, wide ? pix_sentinel(key_bits) : 0, c->derr);
    return check_launch("k_prep") < 0 ? -1 : 1;
}

int launch_scan_u32(hcg_ctx *c, uint32_t *data, int64_t n) {
    if (n <= 0) return 0;
    int launches = 0;
    // levels: data -> sums0 -> sums1 ...
    std::vector<std::pair<uint32_t *, int64_t>> lv;
    lv.push_back({data, n});
    size_t li = 0;
    while (lv.back().second > kScanTile) {
        int64_t nb = (lv.back().second + kScanTile - 1) / kScanTile;
        if (li >= c->scan.level.size() || c->scan.level_cap[li] < nb) {
            hcg_set_error("scan scratch too small");
            return -1;
        }
        k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(lv.back().first, lv.back().second,
                                                                   c->scan.level[li]);
        launches++;
        lv.push_back({c->scan.level[li], nb});
        li++;
    }
    // top level fits one tile
    k_scan_tile<<<1, kScanThreads, 0, c->stream>>>(lv.back().first, lv.back().second, nullptr);
    launches++;
    for (int k = (int)lv.size() - 2; k >= 0; k--) {
        int64_t nb = (lv[k].second + kScanTile - 1) / kScanTile;
        k_scan_tile<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(lv[k].first, lv[k].second, lv[k + 1].first);
        launches++;
    }
    return check_launch("scan") < 0 ? -1 : launches;
}

// One LSD digit phase over bits [0, bits) of keys[cur] (one-sweep form);
// returns the launches made (or -1) and leaves the result in keys[cur] /
// vals[cur].
static int sort_digits(hcg_ctx *c, int64_t n, int bits, int &cur) {
    const int64_t ntiles = sort_tiles(n);
    const int passes = (bits + 7) / 8;
    if (cudaMemsetAsync(c->sort.hist, 0, (size_t)kHistEpoch * sizeof(uint32_t), c->stream) != cudaSuccess) {
        hcg_set_error("clear sort histograms");
        return -1;
    }
    const int hblocks = (int)std::min<int64_t>(ntiles, (int64_t)4 * c->num_sms);
    k_digit_hist<<<hblocks, kSortThreads, 0, c->stream>>>(c->sort.keys[cur], n, passes, c->sort.hist);
    k_digit_offsets<<<1, kSortThreads, 0, c->stream>>>(c->sort.hist, passes);
    int launches = 2;
    for (int p = 0; p < passes; p++) {
        k_onesweep<<<(unsigned)ntiles, kSortThreads, 0, c->stream>>>(c->sort.keys[cur], c->sort.vals[cur],
                                                                    c->sort.keys[cur ^ 1], c->sort.vals[cur ^ 1], n,
                                                                    p, c->sort.hist, c->sort.status, c->derr);
        launches++;
        cur ^= 1;
    }
    return launches;
}

int launch_sort(hcg_ctx *c, int64_t n, int key_bits) {
    if (n == 0) return 0;
    int launches = 0, cur = 0, k;
    if (!wide_key(key_bits)) {
        if ((k = sort_digits(c, n, key_bits, cur)) < 0) return -1;
        launches += k;
    } else {
        // hash digits, then the pixel-offset digits (stable, so ties in the
        // pixel keep the hash order, and ties in both keep the input order)
        if ((k = sort_digits(c, n, 32, cur)) < 0) return -1;
        launches += k;
        k_pix_keys<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->sort.keys[cur], c->sort.vals[cur], n,
                                                             reinterpret_cast<const uint64_t *>(c->psorted));
        launches++;
        if ((k = sort_digits(c, n, key_bits - 32, cur)) < 0) return -1;
        launches += k;
    }
    if (cur != 0) {   // leave the result in buffer 0
        cudaMemcpyAsync(c->sort.keys[0], c->sort.keys[1], n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(c->sort.vals[0], c->sort.vals[1], n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream);
    }
    return check_launch("radix sort") < 0 ? -1 : launches;
}

int launch_permute_lut(hcg_ctx *c, const GridParams &gp) {
    int64_t n = c->n;
    int launches = 0;
    int64_t nr = gp.r_hi - gp.r_lo + 2;
    if (n > 0) {
        const bool wide = wide_key(c->key_bits);
        k_permute<<<blocks_for(n, 256), 256, 0, c->stream>>>(
            c->sort.keys[0], c->sort.vals[0], n, c->lon, c->lat, gp,
            wide ? pix_sentinel(c->key_bits) : packed_sentinel(c->key_bits), wide ? 0 : 32, c->psorted, c->sc_uv,
            c->sc_cos, c->sc_row);
        k_lut1_flags<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->psorted, n, c->flags);
        launches += 2;
        int s = launch_scan_u32(c, c->flags, n);
        if (s < 0) return -1;
        launches += s;
        k_lut1_compact<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->psorted, n, c->flags, c->upix, c->ustart, c->dscal);
        launches++;
    }
    k_lut2<<<blocks_for(nr, 256), 256, 0, c->stream>>>(c->psorted, n, c->upix, c->dscal, gp, c->rstart, c->rustart,
                                                       c->rband);
    launches++;
    return check_launch("permute/lut") < 0 ? -1 : launches;
}

// Quantise FP32 rows x[n][nchan] to the storage type into q (E4M3: with
// per-channel scales into q_scale, amax scratch q_amax, both nchan long).
int launch_quantise_span(hcg_ctx *c, const float *x, int64_t n, int32_t nchan, void *q, float *q_scale,
                         uint32_t *q_amax) {
    int64_t m = n * (int64_t)nchan;
    if (m == 0) return 0;
    if (c->store == HCG_BF16) {
        k_to_bf16<<<blocks_for((m + 3) / 4, 256), 256, 0, c->stream>>>(x, static_cast<__nv_bfloat16 *>(q), m, c->derr);
        return check_launch("k_to_bf16") < 0 ? -1 : 1;
    }
    cudaMemsetAsync(q_amax, 0, sizeof(uint32_t) * nchan, c->stream);
    int64_t rpb = std::max<int64_t>(256, (n + 65534) / 65535);
    dim3 g1(blocks_for(nchan, 128), (unsigned)((n + rpb - 1) / rpb));
    k_amax<<<g1, 128, 0, c->stream>>>(x, n, nchan, rpb, q_amax, c->derr);
    k_scales<<<blocks_for(nchan, 256), 256, 0, c->stream>>>(q_amax, nchan, q_scale);
    k_to_e4m3<<<blocks_for(m, 256), 256, 0, c->stream>>>(x, q_scale, static_cast<__nv_fp8_storage_t *>(q), n, nchan);
    return check_launch("quantise e4m3") < 0 ? -1 : 3;
}

int launch_quantise(hcg_ctx *c) {
    return launch_quantise_span(c, static_cast<const float *>(c->spec_in), c->n, c->nchan, c->q_spec, c->q_scale,
                                c->q_amax);
}

// ---- pre-ordering on caller-provided buffers (used by the allocation-free
//      entry point): keys of k_prep, the radix sort, and the conversion of
//      the sorted keys back to pixel indices.  k[0]/v[0] and k[1]/v[1] are the
//      ping-pong buffers; the sorted pairs end in k[final], v[final], where
//      final is returned (or -1 on a launch error).  counts needs
//      256 * sort_tiles(n) entries; sums is the scan's second level
//      (ceil(256 * sort_tiles(n) / 4096) entries, at most 4096 of them).
namespace {
__global__ void k_keys_to_pix(uint64_t *__restrict__ keys, int64_t n, int64_t pix_lo, uint64_t sentinel) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint64_t k = keys[q];
    int64_t p = k == sentinel ? INT64_MAX : pix_lo + (int64_t)(k >> 32);
    reinterpret_cast<int64_t *>(keys)[q] = p;
}
}  // namespace

int preorder_on_buffers(const double *lon, const double *lat, int64_t n, const GridParams &gp, int key_bits,
                        uint64_t *const k[2], uint32_t *const v[2], int first, uint32_t *counts, uint32_t *sums,
                        int *err, cudaStream_t st) {
    if (n <= 0) return first;
    if (wide_key(key_bits)) { hcg_set_error("pixel range of 2^32 or more pixels"); return -1; }
    const uint64_t sentinel = packed_sentinel(key_bits);
    k_prep<<<blocks_for(n, 256), 256, 0, st>>>(lon, lat, n, gp, sentinel, k[first], v[first], nullptr, 0, err);
    const int64_t ntiles = sort_tiles(n);
    const int64_t nc = 256 * ntiles;
    const int64_t nb = (nc + kScanTile - 1) / kScanTile;
    if (nb > kScanTile) { hcg_set_error("too many keys for a two-level scan"); return -1; }
    int cur = first;
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_hist<<<(unsigned)ntiles, kSortThreads, 0, st>>>(k[cur], n, shift, ntiles, counts);
        if (nb > 1) {
            k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(counts, nc, sums);
            k_scan_tile<<<1, kScanThreads, 0, st>>>(sums, nb, nullptr);
            k_scan_tile<<<(unsigned)nb, kScanThreads, 0, st>>>(counts, nc, sums);
        } else {
            k_scan_tile<<<1, kScanThreads, 0, st>>>(counts, nc, nullptr);
        }
        k_scatter<<<(unsigned)ntiles, kSortThreads, 0, st>>>(k[cur], v[cur], k[cur ^ 1], v[cur ^ 1], n, shift,
                                                            ntiles, counts);
        cur ^= 1;
    }
    k_keys_to_pix<<<blocks_for(n, 256), 256, 0, st>>>(k[cur], n, gp.pix_lo, sentinel);
    if (check_launch("pre-ordering on caller buffers") < 0) return -1;
    return cur;
}


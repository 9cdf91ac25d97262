// hcg_tc.cu -- tensor-core blocked form of the gather (Eq. (1) of HCGrid
// Sec. 2.1 with the search of Sec. 3.4) for BF16 / FP8-e4m3 storage.
//
// A CTA owns a tile of 128 cells (8 rows x 16 columns) and NCH channels.  The
// tile's candidates (the union over its rings of the S' runs found with the
// two lookup tables) are streamed in chunks of 64.  For each chunk:
//   A[128 x 64]  = w(cell, candidate), computed on CUDA cores with the same
//                  membership test as the CUDA-core gather, rounded to BF16
//                  (FP16 x 2^10 for FP8 storage, so that small weights stay
//                  normal), K-major, 128-byte swizzle;
//   B[64 x NCH]  = the candidates' spectrum rows, channel-major (MN-major),
//                  128-byte swizzle: copied with cp.async (BF16) or loaded and
//                  widened e4m3 -> f16 (FP8);
//   D[128 x NCH] += A B with tcgen05.mma (kind::f16, FP32 accumulation in
//                  TMEM), issued by one thread and committed to an mbarrier
//                  that frees the stage.
// Two stages alternate, so the MMA of chunk c overlaps the preparation of
// chunk c+1.  The normaliser is the sum of the *rounded* weights (the same
// values the MMA multiplied), accumulated in FP32 on the CUDA cores; the
// weights output is the sum of the unrounded FP32 weights.  At the end the
// accumulator is read back with tcgen05.ld, divided by the normaliser (times
// the per-channel FP8 scale) and stored.
//
// Every bounded wait gives up after a limit of global time (4 s unless
// hcg_set_wait_limit sets another), raises the HCG_DERR_TIMEOUT bit and lets
// the CTA finish without further MMAs (the host reports TIMEOUT).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <math.h>

#include <algorithm>

#include "hcg_async.cuh"
#include "hcg_search.cuh"

namespace {

constexpr int kTW = 16, kTH = 8, kTM = kTW * kTH;   // 128 cells = MMA M
constexpr int kKC = 64;                               // candidates per chunk = MMA K per stage
constexpr int kMaxSeg = 256;                          // S' runs per tile (two per ring)
constexpr int kStages = 2;
constexpr float kF16WeightScale = 1024.0f;            // keeps FP16 weights normal down to 4 sigma

struct TcArgs {
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
    int ntx, nty;
    int64_t ntiles;
    int nslices;
    int64_t cube_ld;          // cube row stride (channels); a.cube points at the window's first channel
    float band_lo, band_hi;   // R^2 (1 -+ b): the fast estimate decides outside, FP64 inside
    uint64_t wait_ns;         // give-up limit of every mbarrier wait (global time)
    int probe;                // 1: first wait on a barrier nothing completes (checks the give-up path)
};

// ---- shared memory layout (offsets from a 1024-aligned base)
template <int NCH>
struct Layout {
    static constexpr int kA = kTM * 128;                 // 128 rows x 64 K-elements x 2 B
    static constexpr int kB = NCH * 128;                 // NCH/64 atoms x (64 K-rows x 128 B)
    static constexpr int kStage = kA + kB;
    static constexpr int kCand = kStages * kStage;       // candidate data per stage
    static constexpr int kCandBytes = kKC * 16;
    static constexpr int kSeg = kCand + kStages * kCandBytes;
    static constexpr int kSums = kSeg + kMaxSeg * 8 + 16;
    static constexpr int kMisc = kSums + 8 * kTM * 4 + 2 * 4 * 8;
    static constexpr int kTotal = kMisc + 64;
};

// Shared-memory matrix descriptor (tcgen05): start >> 4 in bits 0-13, leading
// byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, the fixed
// 0b001 at 46-48, base offset 0, swizzle mode 2 (128-byte) in bits 61-63.
HCG_DEV uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A/B type
// (bits 7-9 / 10-12: 0 = F16, 1 = BF16), A K-major (bit 15 = 0), B MN-major
// (bit 16 = 1), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
HCG_DEV uint32_t idesc_f16(bool bf16, int n, int m) {
    uint32_t t = bf16 ? 1u : 0u;
    return (1u << 4) | (t << 7) | (t << 10) | (1u << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

HCG_DEV void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

#define TMEM_LD32(taddr, r)                                                                                  \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15," \
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                  \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),     \
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),  \
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),            \
                   "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),            \
                   "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])             \
                 : "r"(taddr) : "memory")

#define TMEM_ST32(taddr, r)                                                                                  \
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"    \
                 "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"                   \
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),     \
                   "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), \
                   "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),          \
                   "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),          \
                   "r"(r[29]), "r"(r[30]), "r"(r[31]) : "memory")

HCG_DEV uint32_t pack2(float lo, float hi, bool bf16) {
    uint32_t r;
    if (bf16) asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    else asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

HCG_DEV float unpack_lo(uint32_t v, bool bf16) {
    if (bf16) return __uint_as_float(v << 16);
    return __half2float(__ushort_as_half((unsigned short)(v & 0xffff)));
}

HCG_DEV float unpack_hi(uint32_t v, bool bf16) {
    if (bf16) return __uint_as_float(v & 0xffff0000u);
    return __half2float(__ushort_as_half((unsigned short)(v >> 16)));
}

HCG_DEV uint32_t e4m3x2_to_f16x2(uint32_t two) {
    uint32_t r;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(r) : "h"((unsigned short)two));
    return r;
}

// FP8: T = __nv_fp8_storage_t, BF16: T = __nv_bfloat16.
// The exact FP64 test of a pair near the support boundary, kept out of line
// so that the unrolled weight loop stays small.
__device__ __noinline__ bool exact_inside(const GridParams &g, int i, int j, const double *lon, const double *lat,
                                          uint32_t row) {
    return hav_exact_t<false>(g, i, j, lon[row], lat[row]) <= g.hR;     // plain grids only
}

template <int NCH>
constexpr int threads_for() { return NCH == 512 ? 512 : 256; }

template <typename T, int NCH>
__global__ void __launch_bounds__(threads_for<NCH>(), NCH == 256 ? 2 : 1) k_tc_gather(TcArgs a) {
    constexpr bool kBF16 = sizeof(T) == 2;
    using L = Layout<NCH>;
    constexpr int kThreads = threads_for<NCH>();
    constexpr int kNQ = kThreads / kTM;                 // threads per cell row of A
    constexpr int kCPT = kKC / kNQ;                     // candidates per thread per chunk
    constexpr int kPieces = kKC * NCH / 8;              // 16-byte pieces of B per chunk
    constexpr int kPPT = kPieces / kThreads;            // per thread
    extern __shared__ unsigned char dsm_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile = blockIdx.x % a.ntiles;
    const int slice = (int)(blockIdx.x / a.ntiles);
    const int ty = a.nty - 1 - (int)(tile / a.ntx);      // north tile row first
    const int i0 = (int)(tile % a.ntx) * kTW, j0 = ty * kTH;
    const int cbase = slice * NCH;
    const GridParams &g = a.g;

    // per candidate: x = U, y = V (FP32 offsets from the tile's first cell, radians),
    // z = cos(lat), w = input row (bits; 0xFFFFFFFF past the end)
    float4 *cand = reinterpret_cast<float4 *>(sm + L::kCand);                            // [stage][64]
    uint32_t *seg_b = reinterpret_cast<uint32_t *>(sm + L::kSeg);
    uint32_t *seg_off = seg_b + kMaxSeg;                                                 // inclusive prefix
    uint32_t *seg_n = seg_off + kMaxSeg;                                                 // [0] runs, [1] total
    float *sw = reinterpret_cast<float *>(sm + L::kSums);                                // [4][128] unrounded
    float *swr = sw + 4 * kTM;                                                           // [4][128] rounded
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::kSums + 8 * kTM * 4);           // [2], [2] = probe
    uint32_t *taddr_s = reinterpret_cast<uint32_t *>(bar + 2 * 4);
    unsigned *pair_s = taddr_s + 1;
    unsigned *abort_s = taddr_s + 2;

    // ---- prologue: TMEM, barriers, the tile's S' runs
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(taddr_s)), "r"(NCH) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < kStages + 1; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar + s)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *pair_s = 0;
        *abort_s = 0;
        // probe of the give-up path: nothing ever arrives on bar[kStages], so
        // this wait runs out after the limit; the CTA then skips its MMAs
        if (a.probe && !mbar_wait(smem_u32(bar + kStages), 0u, a.err, a.wait_ns)) *abort_s = 1;
    }
    if (warp == 1)
        tile_runs(g, a.upix, a.ustart, a.rustart, a.rband, i0, j0, kTW, kTH, seg_b, seg_off, seg_n, kMaxSeg, a.err);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *taddr_s;
    const uint32_t nseg = seg_n[0], total = seg_n[1];
    const int nchunks = (int)((total + kKC - 1) / kKC);

    // this thread's cell (weights) and candidate part
    const int m = tid & (kTM - 1), half = tid >> 7;     // half: which kCPT candidates of a chunk
    const int ci = i0 + (m & (kTW - 1)), cj = j0 + (m >> 4);
    const bool cell_ok = ci < g.nx && cj < g.ny;
    // tile origin (first cell) as FP32 hi + lo, and this thread's cell relative to it
    float oah, oal, obh, obl;
    {
        double A0 = ((double)i0 - g.hx) * g.pix * kDeg, B0 = ((double)j0 - g.hy) * g.pix * kDeg;
        oah = (float)A0; oal = (float)(A0 - (double)oah);
        obh = (float)B0; obl = (float)(B0 - (double)obh);
    }
    float arel, brel, cg;
    {
        int ic = min(ci, g.nx - 1), jc = min(cj, g.ny - 1);
        arel = (float)((double)(ic - i0) * g.pix * kDeg);
        brel = (float)((double)(jc - j0) * g.pix * kDeg);
        cg = cosf((float)((g.lat0 + ((double)jc - g.hy) * g.pix) * kDeg));
    }
    // candidate data for chunk c into registers (threads < 64).  A thread's
    // candidate index only grows from call to call, so its run is found by a
    // cursor moving forward through the runs (each run passed once per tile)
    int run_cur = 0;
    auto fetch_cand = [&](int c) -> float4 {
        uint32_t p = (uint32_t)c * kKC + tid;
        if (p >= total) return make_float4(0.f, 0.f, 0.f, __uint_as_float(0xFFFFFFFFu));
        while (run_cur < (int)nseg - 1 && seg_off[run_cur] <= p) run_cur++;   // first run with end > p
        const int lo = run_cur;
        uint32_t before = lo ? seg_off[lo - 1] : 0u;
        uint32_t sidx = seg_b[lo] + (p - before);
        float4 uv = __ldg(a.uv + sidx);
        float cn = __ldg(a.cs + sidx);
        uint32_t rw = __ldg(a.row + sidx);
        return make_float4((uv.x - oah) + (uv.y - oal), (uv.z - obh) + (uv.w - obl), cn, __uint_as_float(rw));
    };
    if (tid < kKC && nchunks > 0) cand[tid] = fetch_cand(0);
    __syncthreads();
    float wsum = 0.f, wrsum = 0.f;
    unsigned npairs = 0;
    const T *spec = static_cast<const T *>(a.spec);
    const size_t nchan = (size_t)a.nchan;
    const uint32_t idesc = idesc_f16(kBF16, 256, kTM);
    bool aborted = *abort_s != 0;

    // With 512-channel slices (one CTA per SM, its barrier waits unhidden)
    // candidate data go two chunks ahead through two register sets used in
    // turn (the loop runs two chunks per turn, so no register copy waits for
    // a load early): chunk c issues the loads of chunk c + 2 into `rload` and
    // stores chunk c + 1's, loaded during chunk c - 1, from `rstore`
    // (measured on the 4.1M-sample 4096-channel field: BF16 26.9 -> 25.0 ms,
    // E4M3 28.6 -> 27.2 ms).  With 256-channel slices (two CTAs per SM) one
    // chunk ahead measured faster.
    constexpr int kAhead = NCH == 512 ? 2 : 1;
    float4 regA = make_float4(0.f, 0.f, 0.f, 0.f), regB = regA;
    if (kAhead == 2 && tid < kKC && 1 < nchunks) regB = fetch_cand(1);
    auto chunk = [&](const int c, float4 &rload, float4 &rstore) {
        const int s = c & 1;
        unsigned char *As = sm + s * L::kStage;
        unsigned char *Bs = As + L::kA;
        float4 *cs4 = cand + s * kKC;
        // stage s was last read by the MMAs of chunk c - 2
        if (c >= kStages && !aborted) {
            if (!mbar_wait(smem_u32(bar + s), (uint32_t)(((c >> 1) - 1) & 1), a.err, a.wait_ns)) aborted = true;
        }
        // B: spectrum rows of chunk c into the MN-major swizzled tile
        uint2 raw[kBF16 ? 1 : kPPT];
#pragma unroll
        for (int q = 0; q < kPPT; q++) {
            const int piece = tid + q * kThreads;
            const int k = piece / (NCH / 8), cp = piece % (NCH / 8);
            const uint32_t rw = __float_as_uint(cs4[k].w);
            const uint32_t dst = smem_u32(Bs) + (uint32_t)((cp >> 3) * 8192 + k * 128 + (((cp & 7) ^ (k & 7)) << 4));
            if (kBF16) {
                const T *src = spec + (rw != 0xFFFFFFFFu ? (size_t)rw * nchan : 0) + cbase + cp * 8;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                             :: "r"(dst), "l"(src), "r"(rw != 0xFFFFFFFFu ? 16 : 0) : "memory");
            } else {
                raw[kBF16 ? 0 : q] = rw != 0xFFFFFFFFu
                    ? __ldg(reinterpret_cast<const uint2 *>(spec + (size_t)rw * nchan + cbase + cp * 8))
                    : make_uint2(0u, 0u);
            }
        }
        if (kBF16) asm volatile("cp.async.commit_group;" ::: "memory");
        // candidate data of chunk c + 1 (its latency hides behind the weights)
        float4 nxt = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kAhead == 2) { if (tid < kKC && c + 2 < nchunks) rload = fetch_cand(c + 2); }
        else if (tid < kKC && c + 1 < nchunks) nxt = fetch_cand(c + 1);
        // A: weights of this thread's cell for its kCPT candidates.  A warp holds
        // two cell rows; when no candidate of its part lies within the support's
        // latitude reach of either row, the part is all zeros.
        {
            uint32_t pk[kCPT / 2];
            bool near = false;
#pragma unroll
            for (int k = lane & 15; k < kCPT; k += 16) {     // lanes 0-15: first row, 16-31: second
                const float dv = cs4[half * kCPT + k].y - brel;
                near |= (dv * dv <= a.band_hi) && (__float_as_uint(cs4[half * kCPT + k].w) != 0xFFFFFFFFu);
            }
            if (__any_sync(0xffffffffu, near)) {
#pragma unroll
                for (int kk = 0; kk < kCPT; kk += 2) {
                    float w2[2];
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const float4 cd = cs4[half * kCPT + kk + e];
                        const uint32_t rw = __float_as_uint(cd.w);
                        const float du = cd.x - arel, dv = cd.y - brel;
                        const float t = fmaf(cg * cd.z, du * du, dv * dv);
                        bool in = t <= a.band_lo;
                        if (!in && t <= a.band_hi && cell_ok && rw != 0xFFFFFFFFu)
                            in = exact_inside(g, ci, cj, a.lon, a.lat, rw);
                        in = in && cell_ok && rw != 0xFFFFFFFFu;
                        float w = 0.0f;
                        if (in) w = ex2_approx(-t * g.kexp);
                        wsum += w;
                        npairs += in;
                        w2[e] = kBF16 ? w : w * kF16WeightScale;
                    }
                    uint32_t p2 = pack2(w2[0], w2[1], kBF16);
                    wrsum += unpack_lo(p2, kBF16) + unpack_hi(p2, kBF16);
                    pk[kk >> 1] = p2;
                }
            } else {
#pragma unroll
                for (int q = 0; q < kCPT / 2; q++) pk[q] = 0u;
            }
            uint32_t rowbase = smem_u32(As) + (uint32_t)(m * 128);
#pragma unroll
            for (int q = 0; q < kCPT / 8; q++) {
                const int chunk = half * (kCPT / 8) + q;
                const uint32_t dst = rowbase + (uint32_t)((chunk ^ (m & 7)) << 4);
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                             :: "r"(dst), "r"(pk[4 * q]), "r"(pk[4 * q + 1]), "r"(pk[4 * q + 2]), "r"(pk[4 * q + 3])
                             : "memory");
            }
        }
        // chunk c + 1's candidate slot was last read during chunk c - 1
        if (tid < kKC && c + 1 < nchunks) cand[((c + 1) & 1) * kKC + tid] = kAhead == 2 ? rstore : nxt;
        if (!kBF16) {
#pragma unroll
            for (int q = 0; q < kPPT; q++) {
                const int piece = tid + q * kThreads;
                const int k = piece / (NCH / 8), cp = piece % (NCH / 8);
                const uint32_t dst = smem_u32(Bs) + (uint32_t)((cp >> 3) * 8192 + k * 128 + (((cp & 7) ^ (k & 7)) << 4));
                uint2 r = raw[kBF16 ? 0 : q];
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                             :: "r"(dst), "r"(e4m3x2_to_f16x2(r.x & 0xffff)), "r"(e4m3x2_to_f16x2(r.x >> 16)),
                                "r"(e4m3x2_to_f16x2(r.y & 0xffff)), "r"(e4m3x2_to_f16x2(r.y >> 16)) : "memory");
            }
        } else {
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !aborted) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t abase = smem_u32(As), bbase = smem_u32(Bs);
#pragma unroll
            for (int kk = 0; kk < kKC / 16; kk++) {
                const uint64_t ad = sdesc(abase + kk * 32, 16, 1024);
#pragma unroll
                for (int nb = 0; nb < NCH / 256; nb++) {
                    const uint64_t bd = sdesc(bbase + nb * 32768 + kk * 2048, 8192, 1024);
                    mma_f16(tmem + nb * 256, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(bar + s)) : "memory");
        }
        };
    if constexpr (kAhead == 2) {
        for (int c = 0; c < nchunks; c += 2) {
            chunk(c, regA, regB);
            if (c + 1 < nchunks) chunk(c + 1, regB, regA);
        }
    } else {
        for (int c = 0; c < nchunks; c++) chunk(c, regA, regB);
    }

    // ---- epilogue
    sw[half * kTM + m] = wsum;
    swr[half * kTM + m] = wrsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    if (lane == 0 && npairs) atomicAdd(pair_s, npairs);
    if (nchunks > 0 && !aborted) {
        const int s = (nchunks - 1) & 1;
        mbar_wait(smem_u32(bar + s), (uint32_t)(((nchunks - 1) >> 1) & 1), a.err, a.wait_ns);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
        const int q = warp & 3, colhalf = warp >> 2;       // colhalf: which 1/kNQ of the columns
        const int mm = q * 32 + lane;                       // TMEM lane = cell
        const int ii = i0 + (mm & (kTW - 1)), jj = j0 + (mm >> 4);
        const bool ok = ii < g.nx && jj < g.ny;
        float W = 0.f, Wr = 0.f;
#pragma unroll
        for (int h = 0; h < kNQ; h++) { W += sw[h * kTM + mm]; Wr += swr[h * kTM + mm]; }
        float *out = a.cube + ((size_t)jj * g.nx + ii) * (size_t)a.cube_ld + cbase;
        constexpr int kCols = NCH / kNQ;                    // per warp
#pragma unroll 1
        for (int cc = 0; cc < kCols; cc += 32) {
            const int col = colhalf * kCols + cc;
            uint32_t r[32];
            if (nchunks > 0) {
                TMEM_LD32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            if (!ok) continue;
#pragma unroll
            for (int v = 0; v < 32; v += 4) {
                float y[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    float val;
                    if (W > 0.0f && nchunks > 0) val = __fdiv_rn(__uint_as_float(r[v + e]), Wr);
                    else val = __int_as_float(0x7fc00000);
                    if (a.scale) val *= __ldg(a.scale + cbase + col + v + e);
                    y[e] = val;
                }
                *reinterpret_cast<float4 *>(out + col + v) = make_float4(y[0], y[1], y[2], y[3]);
            }
        }
        if (slice == 0 && colhalf == 0 && ok) a.wout[(size_t)jj * g.nx + ii] = W;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (slice == 0 && tid == 0 && *pair_s && a.pairs) atomicAdd(a.pairs, (unsigned long long)*pair_s);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(NCH) : "memory");
}

// ---- FP32 storage: products of split TF32 operands ----------------------
// kind::tf32 multiplies operands rounded to TF32 (10 fraction bits).  Each
// weight w and each spectrum value s is split exactly into a TF32 head and a
// remainder, x = x_hi + x_lo with x_hi = x rounded to TF32 and x_lo = x - x_hi
// (|x_lo| <= 2^-12 |x|, itself taken to TF32 by the MMA); three MMAs
// accumulate w_hi s_hi + w_hi s_lo + w_lo s_hi in FP32 in TMEM.  The dropped
// w_lo s_lo and the TF32 rounding of the remainders are below 2^-21 of each
// product, so the sums carry FP32-level accuracy and are divided by the FP32
// sum of the unsplit weights.  The tensor core's FP32 accumulation chain is
// kept short: the MMAs sum one block of kBlk32 chunks (512 candidates) into
// TMEM columns [0, 256), which the CUDA cores then add into a running total
// in columns [256, 512) (FP32, round to nearest) before the next block starts
// afresh -- over thousands of successive K-steps the accumulator otherwise
// drifts by a few 1e-5 (measured at 13,000 candidates per tile).
// Chunks of 32 candidates (one 128-byte swizzle
// atom of TF32 per row); per stage A_hi, A_lo [128 cells x 32] and B_hi, B_lo
// [256 channels x 32], all K-major (kind::tf32 reads 32-bit operands K-major
// only: an MN-major B gives zeros), 96 KB; two stages, one CTA per SM.
constexpr int kKC32 = 32;
constexpr int kBlk32 = 16;                              // chunks per TMEM accumulation block

struct Layout32 {
    static constexpr int kA = kTM * 128;                 // 128 rows x 32 TF32 = 16 KB (hi or lo)
    static constexpr int kB = 256 * 128;                 // 256 channel rows x 32 TF32 = 32 KB (hi or lo)
    static constexpr int kStage = 2 * kA + 2 * kB;       // A_hi, A_lo, B_hi, B_lo
    static constexpr int kCand = kStages * kStage;
    static constexpr int kSeg = kCand + kStages * kKC32 * 16;
    static constexpr int kSums = kSeg + kMaxSeg * 8 + 16;
    static constexpr int kMisc = kSums + 2 * kTM * 4 + 4 * 8;
    static constexpr int kTotal = kMisc + 64;
};

// Instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
HCG_DEV uint32_t idesc_tf32(int n, int m) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

HCG_DEV void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

// x rounded to TF32 (nearest, ties away from zero), as an FP32 bit pattern.
HCG_DEV float tf32_head(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }

__global__ void __launch_bounds__(256, 1) k_tc_gather_f32(TcArgs a) {
    using L = Layout32;
    constexpr int kThreads = 256;
    constexpr int kNQ = kThreads / kTM;                 // 2 threads per cell row of A
    constexpr int kCPT = kKC32 / kNQ;                   // 16 candidates per thread per chunk
    constexpr int kPPT = kKC32 / 4;                     // 8 candidate quads per thread per chunk
    extern __shared__ unsigned char dsm_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile = blockIdx.x % a.ntiles;
    const int slice = (int)(blockIdx.x / a.ntiles);
    const int ty = a.nty - 1 - (int)(tile / a.ntx);      // north tile row first
    const int i0 = (int)(tile % a.ntx) * kTW, j0 = ty * kTH;
    const int cbase = slice * 256;
    const GridParams &g = a.g;

    float4 *cand = reinterpret_cast<float4 *>(sm + L::kCand);
    uint32_t *seg_b = reinterpret_cast<uint32_t *>(sm + L::kSeg);
    uint32_t *seg_off = seg_b + kMaxSeg;
    uint32_t *seg_n = seg_off + kMaxSeg;
    float *sw = reinterpret_cast<float *>(sm + L::kSums);                                // [2][128]
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::kSums + 2 * kTM * 4);           // [2], [2] = probe
    uint32_t *taddr_s = reinterpret_cast<uint32_t *>(sm + L::kMisc);
    unsigned *pair_s = taddr_s + 1;
    unsigned *abort_s = taddr_s + 2;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(taddr_s)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < kStages + 1; s++) mbar_init(smem_u32(bar + s), 1);
        mbar_fence_init();
        *pair_s = 0;
        *abort_s = 0;
        if (a.probe && !mbar_wait(smem_u32(bar + kStages), 0u, a.err, a.wait_ns)) *abort_s = 1;
    }
    if (warp == 1)
        tile_runs(g, a.upix, a.ustart, a.rustart, a.rband, i0, j0, kTW, kTH, seg_b, seg_off, seg_n, kMaxSeg, a.err);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *taddr_s;
    const uint32_t nseg = seg_n[0], total = seg_n[1];
    const int nchunks = (int)((total + kKC32 - 1) / kKC32);

    const int m = tid & (kTM - 1), half = tid >> 7;
    const int ci = i0 + (m & (kTW - 1)), cj = j0 + (m >> 4);
    const bool cell_ok = ci < g.nx && cj < g.ny;
    float oah, oal, obh, obl;
    {
        double A0 = ((double)i0 - g.hx) * g.pix * kDeg, B0 = ((double)j0 - g.hy) * g.pix * kDeg;
        oah = (float)A0; oal = (float)(A0 - (double)oah);
        obh = (float)B0; obl = (float)(B0 - (double)obh);
    }
    float arel, brel, cg;
    {
        int ic = min(ci, g.nx - 1), jc = min(cj, g.ny - 1);
        arel = (float)((double)(ic - i0) * g.pix * kDeg);
        brel = (float)((double)(jc - j0) * g.pix * kDeg);
        cg = cosf((float)((g.lat0 + ((double)jc - g.hy) * g.pix) * kDeg));
    }
    int run_cur = 0;
    auto fetch_cand = [&](int c) -> float4 {
        uint32_t p = (uint32_t)c * kKC32 + tid;
        if (p >= total) return make_float4(0.f, 0.f, 0.f, __uint_as_float(0xFFFFFFFFu));
        while (run_cur < (int)nseg - 1 && seg_off[run_cur] <= p) run_cur++;
        const int lo = run_cur;
        uint32_t before = lo ? seg_off[lo - 1] : 0u;
        uint32_t sidx = seg_b[lo] + (p - before);
        float4 uv = __ldg(a.uv + sidx);
        float cn = __ldg(a.cs + sidx);
        uint32_t rw = __ldg(a.row + sidx);
        return make_float4((uv.x - oah) + (uv.y - oal), (uv.z - obh) + (uv.w - obl), cn, __uint_as_float(rw));
    };
    if (tid < kKC32 && nchunks > 0) cand[tid] = fetch_cand(0);
    __syncthreads();
    float wsum = 0.f;
    unsigned npairs = 0;
    const float *spec = static_cast<const float *>(a.spec);
    const size_t nchan = (size_t)a.nchan;
    const uint32_t idesc = idesc_tf32(256, kTM);
    bool aborted = *abort_s != 0;

    for (int c = 0; c < nchunks; c++) {
        const int s = c & 1;
        unsigned char *Ahi = sm + s * L::kStage;
        unsigned char *Alo = Ahi + L::kA;
        unsigned char *Bhi = Alo + L::kA;
        unsigned char *Blo = Bhi + L::kB;
        float4 *cs4 = cand + s * kKC32;
        // stage s was last read by the MMAs of chunk c - 2
        if (c >= kStages && !aborted) {
            if (!mbar_wait(smem_u32(bar + s), (uint32_t)(((c >> 1) - 1) & 1), a.err, a.wait_ns)) aborted = true;
        }
        // B: this chunk's spectrum values, loaded now, split and stored after
        // the weights.  Warp w takes channels 32 w + lane (a warp's load
        // reads 128 contiguous bytes of one row) of the four candidates of
        // quad q = 0 .. 7, so one 16-byte store fills a K-major unit
        float4 raw[kPPT];
#pragma unroll
        for (int q = 0; q < kPPT; q++) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t rw = __float_as_uint(cs4[4 * q + e].w);
                v[e] = rw != 0xFFFFFFFFu ? __ldg(spec + (size_t)rw * nchan + cbase + 32 * warp + lane) : 0.0f;
            }
            raw[q] = make_float4(v[0], v[1], v[2], v[3]);
        }
        float4 nxt = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tid < kKC32 && c + 1 < nchunks) nxt = fetch_cand(c + 1);
        // A: weights of this thread's cell for its kCPT candidates, split
        {
            uint32_t ph[kCPT], pl[kCPT];
            bool near = false;
#pragma unroll
            for (int k = lane & 15; k < kCPT; k += 16) {
                const float dv = cs4[half * kCPT + k].y - brel;
                near |= (dv * dv <= a.band_hi) && (__float_as_uint(cs4[half * kCPT + k].w) != 0xFFFFFFFFu);
            }
            if (__any_sync(0xffffffffu, near)) {
#pragma unroll
                for (int kk = 0; kk < kCPT; kk++) {
                    const float4 cd = cs4[half * kCPT + kk];
                    const uint32_t rw = __float_as_uint(cd.w);
                    const float du = cd.x - arel, dv = cd.y - brel;
                    const float t = fmaf(cg * cd.z, du * du, dv * dv);
                    bool in = t <= a.band_lo;
                    if (!in && t <= a.band_hi && cell_ok && rw != 0xFFFFFFFFu)
                        in = exact_inside(g, ci, cj, a.lon, a.lat, rw);
                    in = in && cell_ok && rw != 0xFFFFFFFFu;
                    const float w = in ? ex2_approx(-t * g.kexp) : 0.0f;
                    wsum += w;
                    npairs += in;
                    const float hi = tf32_head(w);
                    ph[kk] = __float_as_uint(hi);
                    pl[kk] = __float_as_uint(w - hi);
                }
            } else {
#pragma unroll
                for (int q = 0; q < kCPT; q++) ph[q] = pl[q] = 0u;
            }
            const uint32_t rowoff = (uint32_t)(m * 128);
#pragma unroll
            for (int q = 0; q < kCPT / 4; q++) {
                const int chunk = half * (kCPT / 4) + q;
                const uint32_t off = rowoff + (uint32_t)((chunk ^ (m & 7)) << 4);
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                             :: "r"(smem_u32(Ahi) + off), "r"(ph[4 * q]), "r"(ph[4 * q + 1]), "r"(ph[4 * q + 2]),
                                "r"(ph[4 * q + 3]) : "memory");
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                             :: "r"(smem_u32(Alo) + off), "r"(pl[4 * q]), "r"(pl[4 * q + 1]), "r"(pl[4 * q + 2]),
                                "r"(pl[4 * q + 3]) : "memory");
            }
        }
        if (tid < kKC32 && c + 1 < nchunks) cand[((c + 1) & 1) * kKC32 + tid] = nxt;
        // B split into its K-major swizzled hi / lo tiles: channel n's row at
        // n * 128, candidates 4 q .. 4 q + 3 in 16-byte unit q ^ (n & 7)
        {
            const uint32_t n = (uint32_t)(32 * warp + lane);
            const uint32_t bh = smem_u32(Bhi) + n * 128, bl = smem_u32(Blo) + n * 128;
#pragma unroll
            for (int q = 0; q < kPPT; q++) {
                const uint32_t off = ((uint32_t)q ^ (n & 7)) << 4;
                const float4 x = raw[q];
                const float h0 = tf32_head(x.x), h1 = tf32_head(x.y), h2 = tf32_head(x.z), h3 = tf32_head(x.w);
                asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};"
                             :: "r"(bh + off), "f"(h0), "f"(h1), "f"(h2), "f"(h3) : "memory");
                asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};"
                             :: "r"(bl + off), "f"(x.x - h0), "f"(x.y - h1), "f"(x.z - h2), "f"(x.w - h3) : "memory");
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !aborted) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
            for (int kk = 0; kk < kKC32 / 8; kk++) {
                const uint64_t dah = sdesc(ah + kk * 32, 16, 1024), dal = sdesc(al + kk * 32, 16, 1024);
                const uint64_t dbh = sdesc(bh + kk * 32, 16, 1024), dbl = sdesc(bl + kk * 32, 16, 1024);
                mma_tf32(tmem, dah, dbh, idesc, (c % kBlk32 > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, idesc, 1u);
                mma_tf32(tmem, dal, dbh, idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(bar + s)) : "memory");
        }
        // end of a block: once its MMAs are done, add the block's sums into the
        // running total (columns 256..511; the first block just moves in)
        if (c % kBlk32 == kBlk32 - 1 || c == nchunks - 1) {
            if (!aborted && !mbar_wait(smem_u32(bar + s), (uint32_t)((c >> 1) & 1), a.err, a.wait_ns)) aborted = true;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int q = warp & 3, colhalf = warp >> 2;
            const uint32_t lanebase = (uint32_t)(q * 32) << 16;
#pragma unroll 1
            for (int cc = 0; cc < 128; cc += 32) {
                const uint32_t col = (uint32_t)(colhalf * 128 + cc);
                uint32_t rb[32], rt[32];
                TMEM_LD32(tmem + lanebase + col, rb);
                if (c >= kBlk32) TMEM_LD32(tmem + lanebase + 256 + col, rt);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (c >= kBlk32) {
#pragma unroll
                    for (int e = 0; e < 32; e++) rb[e] = __float_as_uint(__uint_as_float(rt[e]) + __uint_as_float(rb[e]));
                }
                TMEM_ST32(tmem + lanebase + 256 + col, rb);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }

    // ---- epilogue
    sw[half * kTM + m] = wsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    if (lane == 0 && npairs) atomicAdd(pair_s, npairs);
    // (the last chunk's block was drained, after its MMAs completed, in the loop)
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
        const int q = warp & 3, colhalf = warp >> 2;
        const int mm = q * 32 + lane;
        const int ii = i0 + (mm & (kTW - 1)), jj = j0 + (mm >> 4);
        const bool ok = ii < g.nx && jj < g.ny;
        const float W = sw[mm] + sw[kTM + mm];
        float *out = a.cube + ((size_t)jj * g.nx + ii) * (size_t)a.cube_ld + cbase;
        const bool vec_out = (a.cube_ld & 3) == 0 && ((uintptr_t)a.cube & 15) == 0;
#pragma unroll 1
        for (int cc = 0; cc < 128; cc += 32) {
            const int col = 256 + colhalf * 128 + cc;
            uint32_t r[32];
            if (nchunks > 0) {
                TMEM_LD32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            if (!ok) continue;
#pragma unroll
            for (int v = 0; v < 32; v += 4) {
                float y[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const float sv = __uint_as_float(r[v + e]);
                    float val;
                    if (!(W > 0.0f) || nchunks == 0) val = __int_as_float(0x7fc00000);
                    else if (W >= 1e-3f) val = __fdiv_rn(sv, W);
                    else val = (float)((double)sv / (double)W);
                    y[e] = val;
                }
                if (vec_out) {
                    __stcs(reinterpret_cast<float4 *>(out + col - 256 + v), make_float4(y[0], y[1], y[2], y[3]));
                } else {
#pragma unroll
                    for (int e = 0; e < 4; e++) __stcs(out + col - 256 + v + e, y[e]);
                }
            }
        }
        if (slice == 0 && colhalf == 0 && ok) a.wout[(size_t)jj * g.nx + ii] = W;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (slice == 0 && tid == 0 && *pair_s && a.pairs) atomicAdd(a.pairs, (unsigned long long)*pair_s);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
}

int launch_f32(hcg_ctx *c, const TcArgs &a0) {
    TcArgs a = a0;
    a.nslices = a.nchan / 256;
    const int smem = Layout32::kTotal + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_tc_gather_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) { hcg_cuda_fail(e, "tc f32 smem attribute"); return -1; }
    const int64_t blocks = a.ntiles * a.nslices;
    k_tc_gather_f32<<<(unsigned)blocks, 256, smem, c->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { hcg_cuda_fail(e, "k_tc_gather_f32"); return -1; }
    return 1;
}

template <typename T, int NCH>
int launch_nch(hcg_ctx *c, const TcArgs &a) {
    const int smem = Layout<NCH>::kTotal + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_tc_gather<T, NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) { hcg_cuda_fail(e, "tc smem attribute"); return -1; }
    const int64_t blocks = a.ntiles * a.nslices;
    k_tc_gather<T, NCH><<<(unsigned)blocks, threads_for<NCH>(), smem, c->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) { hcg_cuda_fail(e, "k_tc_gather"); return -1; }
    return 1;
}

}  // namespace

// The blocked path needs BF16 or E4M3 storage, channel counts in whole
// 256-channel slices, a support within 5 sigma (FP16 weights stay normal),
// and few enough rings per tile for the run table.
bool tc_supported(hcg_ctx *c, int dtype) {
    if (dtype != HCG_BF16 && dtype != HCG_E4M3 && dtype != HCG_F32) return false;
    if (c->proj != HCG_CAR) return false;                      // tiles use the plain grid's cell offsets
    if (c->nchan % 256 != 0) return false;
    if (c->host_spec && c->stream_chunk_chans() % 256 != 0) return false;   // every streamed window whole slices
    double sig = c->fwhm / 2.3548200450309493;
    if (c->support > 5.0 * sig + 1e-12) return false;
    // rings spanned by a tile: (8 cells + 2 R) / ring spacing (about the pixel size), twice for the seam
    double pixsz = sqrt(3.14159265358979323846 / 3.0) / (double)c->nside * 57.29577951308232;
    double rings = (kTH * c->pix + 2.0 * c->support) / (0.5 * pixsz) + 8.0;
    return rings * 2.0 < kMaxSeg;
}

int launch_tc_gather(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale) {
    TcArgs a;
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
    a.probe = c->wait_probe;
    a.ntx = (c->nx + kTW - 1) / kTW;
    a.nty = (c->ny + kTH - 1) / kTH;
    a.ntiles = (int64_t)a.ntx * a.nty;
    // Band of the fast membership estimate t = dlat^2 + cos(lat_g) cos(lat_n) dlon^2
    // (FP32, offsets from the tile origin): relative error below
    //   R^2 / (6 c_min)                          neglected quartic terms of the haversine,
    //   6 * 2^-23 * E / (R sqrt(c_min))           FP32 offsets of magnitude <= E,
    //   1e-6                                      FP32 products and cosines,
    // plus the 1e-5 margin used everywhere; pairs inside go to the exact FP64 test.
    {
        const double deg = 3.14159265358979323846 / 180.0;
        const double R = gp.R_deg * deg;
        const double latext = std::min(89.9, fabs(gp.lat0) + gp.hy * gp.pix + gp.R_deg);
        const double cmin = std::max(1e-6, cos(latext * deg) * cos(latext * deg));
        const double pixsz = sqrt(3.14159265358979323846 / 3.0) / (double)gp.nside;
        const double E = kTW * gp.pix * deg + 2.0 * R / sqrt(cmin) + 4.0 * pixsz;
        const double rel = 1e-5 + R * R / (6.0 * cmin) + 6.0 * ldexp(1.0, -23) * E / (R * sqrt(cmin)) + 1e-6;
        a.band_lo = (float)(R * R * (1.0 - rel));
        a.band_hi = (float)(R * R * (1.0 + rel));
    }
    // 512-channel slices whenever they divide the channels (one CTA of 512
    // threads per SM; measured on the 4.1M-sample 4096-channel field: BF16
    // 26.8 ms, E4M3 28.6 ms against 37.4 ms with 256-channel slices)
    if (dtype == HCG_F32) return launch_f32(c, a);
    const bool wide = a.nchan % 512 == 0;
    a.nslices = a.nchan / (wide ? 512 : 256);
    if (dtype == HCG_BF16) {
        if (wide) return launch_nch<__nv_bfloat16, 512>(c, a);
        return launch_nch<__nv_bfloat16, 256>(c, a);
    }
    if (wide) return launch_nch<__nv_fp8_storage_t, 512>(c, a);
    return launch_nch<__nv_fp8_storage_t, 256>(c, a);
}

// hcg_tc.cu -- tensor-core blocked form of the gather (Eq. (1) of HCGrid
// Sec. 2.1 with the search of Sec. 3.4) for BF16, FP8-e4m3 and FP32 storage.
//
// A CTA owns a tile of 128 cells (8 rows x 16 columns) and a slice of NCH
// channels.  The tile's candidates (the union over its rings of the S' runs
// found with the two lookup tables) are streamed in chunks.  For each chunk:
//   A[128 x K]  = w(cell, candidate), computed on CUDA cores with the same
//                 membership test as the CUDA-core gather;
//   B[K x NCH]  = the candidates' spectrum rows;
//   D[128 x NCH] += A B with tcgen05.mma (FP32 accumulation in TMEM), issued
//                 by one thread and committed to an mbarrier that frees the
//                 stage.
// The warps of a CTA keep to one role each -- weights, spectra, candidate
// fetch, MMA issue -- and hand chunks over through mbarriers, with no
// CTA-wide barrier inside the chunk loop, so the weights of one chunk, the
// spectrum copies of the next ones and the MMAs of the previous one overlap.
// At the end the accumulator is read back with tcgen05.ld, divided by the
// normaliser and stored.
//
// Every bounded wait gives up after a limit of global time (4 s unless
// hcg_set_wait_limit sets another), raises the HCG_DERR_TIMEOUT bit and an
// abort flag that ends every other role's waits at once, and the CTA
// finishes without further MMAs (the host reports TIMEOUT).
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
    unsigned long long *tflops;   // executed MMA work (2 M N K per instruction), added per CTA
    int *err;
    int ntx, nty;
    int64_t ntiles;
    int nslices;
    int64_t cube_ld;          // cube row stride (channels); a.cube points at the window's first channel
    float band_lo, band_hi;   // R^2 (1 -+ b): the fast estimate decides outside, FP64 inside
    uint64_t wait_ns;         // give-up limit of every mbarrier wait (global time)
    int probe;                // 1: first wait on a barrier nothing completes (checks the give-up path)
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
// (bits 7-9 / 10-12: 0 = F16, 1 = BF16), A and B MN-major (bits 15, 16 = 1),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
HCG_DEV uint32_t idesc_f16(bool bf16, int n, int m) {
    uint32_t t = bf16 ? 1u : 0u;
    return (1u << 4) | (t << 7) | (t << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
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

#define TMEM_LD16(taddr, r)                                                                                  \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),     \
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),  \
                   "=r"(r[14]), "=r"(r[15])                                                                  \
                 : "r"(taddr) : "memory")

#define TMEM_ST16(taddr, r)                                                                                  \
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" \
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),     \
                   "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), \
                   "r"(r[15]) : "memory")

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

HCG_DEV float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

HCG_DEV float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Bits of the tile columns i in [0, 16) with lo <= i <= hi (the conversions
// saturate, and NaN bounds never reach here).
HCG_DEV uint32_t col_range(float lo, float hi) {
    const int a = max(__float2int_ru(lo), 0);
    const int b = min(__float2int_rd(hi), kTW - 1);
    return a > b ? 0u : ((0xFFFFu << a) & (0xFFFFu >> (kTW - 1 - b)));
}

// Columns of a tile row for one candidate, from the roots of the support
// test: t_i = dv2 + ak (cu - i h)^2 is a quadratic in the column index i, so
// t_i <= b holds exactly for |x - i| <= sqrt((b - dv2) / ak) / h, x = cu / h.
// m_in: columns with t_i surely <= blo (the fast estimate says inside);
// m_pos: columns with t_i not surely > bhi (the rest are surely outside).
// e (in columns, 2e-6 relative to the magnitudes involved, about 16 FP32
// ulps) covers the rounding of x and of the approximate reciprocal and
// square roots, so a column that is only near a bound falls between the two
// sets and goes to the exact FP64 test with the other band pairs.
HCG_DEV void col_sets(float cu, float dv2, float ak, float blo, float bhi, float invh, uint32_t &m_in,
                      uint32_t &m_pos) {
    const float rak = rcp_approx(ak);
    const float Q = (bhi - dv2) * rak, P = (blo - dv2) * rak;
    const float x = cu * invh;
    const float Qc = fmaxf(Q, 1e-30f), Pc = fmaxf(P, 1e-30f);
    const float ro = Qc * rsqrt_approx(Qc) * invh, ri = Pc * rsqrt_approx(Pc) * invh;
    const float e = 2e-6f * (fabsf(x) + ro + 1.0f);
    m_pos = Q > 1e-30f ? col_range(x - ro - e, x + ro + e) : 0u;
    m_in = P > 1e-30f ? col_range(x - ri + e, x + ri - e) : 0u;
}

// FP8: T = __nv_fp8_storage_t, BF16: T = __nv_bfloat16.
// The exact FP64 test of a pair near the support boundary, kept out of line
// so that the unrolled weight loop stays small.
__device__ __noinline__ bool exact_inside(const GridParams &g, int i, int j, const double *lon, const double *lat,
                                          uint32_t row) {
    return hav_exact_t<false>(g, i, j, lon[row], lat[row]) <= g.hR;     // plain grids only
}

// Bounded wait that also gives up as soon as another role of the CTA has
// given up (the abort flag in shared memory); the one that runs out of time
// raises TIMEOUT and the flag.
HCG_DEV bool wait_ab(uint32_t bar, uint32_t parity, int *err, uint64_t limit_ns, volatile unsigned *abort_s) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; it++) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 63) == 0) {
            if (*abort_s) return false;
            const uint64_t t = gtimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) {
                set_err(err, HCG_DERR_TIMEOUT);
                *abort_s = 1u;
                return false;
            }
        }
    }
}

// ---- candidate ring ---------------------------------------------------------
// A chunk's candidates are copied into a ring slot by cp.async (S' data as
// stored: the FP32 hi/lo coordinate pairs, cos(lat) and the input row), and
// the copies complete on the slot's mbarrier, so the fetching warp never waits
// for them and runs up to kRing chunks ahead.  Slots past a tile's last
// candidate get the far-away record (offsets 1e30, row 0xFFFFFFFF), which
// every weight test rejects.
constexpr int kRing = 8;
__device__ float4 g_far_uv = {1e30f, 0.0f, 1e30f, 0.0f};
__device__ float g_far_cs = 1.0f;
__device__ uint32_t g_far_row = 0xFFFFFFFFu;

template <int K>
struct CandSlot {
    float4 uv[K];
    float cs[K];
    uint32_t row[K];
};

HCG_DEV void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
}
HCG_DEV void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(dst), "l"(src) : "memory");
}

// The fetching warp: lane l copies candidates K c + 32 h + l of every chunk c
// (h < K / 32).  Each index only grows from chunk to chunk, so a cursor per h
// moving forward through the tile's runs finds its run (each run passed once).
template <int K>
HCG_DEV void fetch_ring(CandSlot<K> *ring, uint64_t *cfull, uint64_t *cempty, int nchunks, uint32_t total,
                        uint32_t nseg, const uint32_t *seg_b, const uint32_t *seg_off, const float4 *uv,
                        const float *cs, const uint32_t *row, int *err, uint64_t wait_ns,
                        volatile unsigned *abort_s) {
    const int lane = threadIdx.x & 31;
    int cur[K / 32];
#pragma unroll
    for (int h = 0; h < K / 32; h++) cur[h] = 0;
    for (int c = 0; c < nchunks; c++) {
        const int r = c % kRing;
        if (c >= kRing &&
            !wait_ab(smem_u32(cempty + r), (uint32_t)(((c / kRing) - 1) & 1), err, wait_ns, abort_s))
            break;
        CandSlot<K> &sl = ring[r];
#pragma unroll
        for (int h = 0; h < K / 32; h++) {
            const int k = 32 * h + lane;
            const uint32_t p = (uint32_t)c * K + k;
            const float4 *su = &g_far_uv;
            const float *sc = &g_far_cs;
            const uint32_t *sr = &g_far_row;
            if (p < total) {
                while (cur[h] < (int)nseg - 1 && seg_off[cur[h]] <= p) cur[h]++;   // first run with end > p
                const int lo = cur[h];
                const uint32_t sidx = seg_b[lo] + (p - (lo ? seg_off[lo - 1] : 0u));
                su = uv + sidx; sc = cs + sidx; sr = row + sidx;
            }
            cp_async16(smem_u32(&sl.uv[k]), su);
            cp_async4(smem_u32(&sl.cs[k]), sc);
            cp_async4(smem_u32(&sl.row[k]), sr);
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" :: "r"(smem_u32(cfull + r)) : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Tile origin (first cell) as FP32 hi + lo, for the candidates' offsets
// U = (u_hi - o_hi) + (u_lo - o_lo).
struct Origin {
    float ah, al, bh, bl;
    HCG_DEV Origin(const GridParams &g, int i0, int j0) {
        const double A0 = ((double)i0 - g.hx) * g.pix * kDeg, B0 = ((double)j0 - g.hy) * g.pix * kDeg;
        ah = (float)A0; al = (float)(A0 - (double)ah);
        bh = (float)B0; bl = (float)(B0 - (double)bh);
    }
    HCG_DEV float u(const float4 &v) const { return (v.x - ah) + (v.y - al); }
    HCG_DEV float v(const float4 &w) const { return (w.z - bh) + (w.w - bl); }
};

// Epilogue store of a warp's 32 x 32 block of the cube: lane l holds cell l's
// 32 channels in y and its output pointer.  The block goes through the warp's
// 32 x 36-float shared-memory tile so that each store instruction writes four
// cells' whole 128-byte channel runs, instead of 32 cells' 16-byte pieces.
HCG_DEV void store_block32(float *tb, const uint32_t (&y)[32], float *optr, bool ok, bool vec, int lane) {
#pragma unroll
    for (int v = 0; v < 32; v += 4)
        *reinterpret_cast<uint4 *>(tb + lane * 36 + v) = make_uint4(y[v], y[v + 1], y[v + 2], y[v + 3]);
    __syncwarp();
    const unsigned okm = __ballot_sync(0xffffffffu, ok);
    const int g4 = 4 * (lane & 7);
#pragma unroll
    for (int it = 0; it < 8; it++) {
        const int c = it * 4 + (lane >> 3);
        float *p = reinterpret_cast<float *>(
            __shfl_sync(0xffffffffu, (unsigned long long)reinterpret_cast<uintptr_t>(optr), c));
        if ((okm >> c) & 1u) {
            const float4 v = *reinterpret_cast<const float4 *>(tb + c * 36 + g4);
            if (vec) {
                __stcs(reinterpret_cast<float4 *>(p + g4), v);
            } else {
                __stcs(p + g4, v.x);
                __stcs(p + g4 + 1, v.y);
                __stcs(p + g4 + 2, v.z);
                __stcs(p + g4 + 3, v.w);
            }
        }
    }
    __syncwarp();
}

// ---- BF16 / FP8-e4m3 storage (kind::f16) ---------------------------------
// Chunks of 64 candidates.  A = the weights as BF16 (FP16 x 2^10 for FP8
// storage, so that small weights stay normal), B = the spectrum rows (BF16
// copied as they are, e4m3 widened to FP16 on the way in); both MN-major
// (cells resp. channels contiguous) with the 128-byte swizzle.  The
// normaliser is the sum of the *rounded* weights (the values the MMA
// multiplied): for 256-channel slices a second MMA of N = 16 multiplies A
// into a tile of ones, into TMEM columns 256-271; for 512-channel slices,
// whose accumulator fills TMEM, the weight warps add them up in FP32.  The
// weights output is the sum of the unrounded FP32 weights.
// Roles (kWW weight warps, 16 for 256-channel slices, 8 for 512):
//   weight warps  warp w owns cell row w % 8; its lane l takes candidate
//                 l + 32 (w / 8) of the chunk (with 8 warps: l and l + 32)
//                 and computes the candidate's weights for the row's 16
//                 cells, writing two 16-byte pieces of A per candidate;
//   4 warps       spectra: copy (BF16, cp.async completing on the stage's
//                 barrier) or load, widen and store (FP8) the chunk's rows;
//   1 warp        candidates: copies each chunk's candidates from the S' runs
//                 into the candidate ring;
//   1 warp        one thread issues the MMAs.
// Sixteen weight warps halve each warp's serial work per chunk: the weight
// chains are latency-bound, and 256-channel slices give the MMAs too little
// work to hide eight warps' chains.
template <int NCH>
struct TcRoles {
    static constexpr int kWW = NCH == 256 ? 16 : 8;     // weight warps
    static constexpr int kSpec0 = kWW, kFetch = kWW + 4, kMma = kWW + 5;
    static constexpr int kThreads = (kWW + 6) * 32;
    static constexpr int kCandPerLane = kWW == 8 ? 2 : 1;
};

template <int NCH>
struct Layout {
    static constexpr int kNS = NCH == 256 ? 4 : 2;       // stages
    // 256-channel slices leave TMEM room for the ones column (see k_tc_gather)
    static constexpr bool kOnes = NCH == 256;
    static constexpr int kTmemCols = kOnes ? 512 : NCH;
    static constexpr int kA = kTM * kKC * 2;             // 2 atoms of 64 cells x 64 K-rows x 128 B = 16 KB
    static constexpr int kB = NCH * kKC * 2;             // NCH/64 atoms x 64 K-rows x 128 B
    static constexpr int kStage = kA + kB;
    static constexpr int kOnesAt = kNS * kStage;         // one B atom (64 channels x 64 K-rows) of ones
    static constexpr int kCand = kOnesAt + (kOnes ? kKC * 128 : 0);
    static constexpr int kSeg = kCand + kRing * (int)sizeof(CandSlot<kKC>);
    static constexpr int kSums = kSeg + kMaxSeg * 8 + 16;   // sw[128], swr[128]
    static constexpr int kBars = kSums + 2 * kTM * 4;
    // fullA[NS], fullB[NS], empty[NS], cfull[kRing], cempty[kRing], probe
    static constexpr int kNumBars = 3 * kNS + 2 * kRing + 1;
    static constexpr int kMisc = kBars + kNumBars * 8;
    static constexpr int kTotal = kMisc + 64;
};

template <typename T, int NCH>
__global__ void __launch_bounds__(TcRoles<NCH>::kThreads, 1) k_tc_gather(TcArgs a) {
    constexpr bool kBF16 = sizeof(T) == 2;
    using L = Layout<NCH>;
    using RL = TcRoles<NCH>;
    constexpr int kWW = RL::kWW;
    static_assert(kWW == 8 || L::kOnes, "16 weight warps keep their second sums where the rounded sums would go");
    constexpr int NS = L::kNS;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile = blockIdx.x % a.ntiles;
    const int slice = (int)(blockIdx.x / a.ntiles);
    const int ty = a.nty - 1 - (int)(tile / a.ntx);      // north tile row first
    const int i0 = (int)(tile % a.ntx) * kTW, j0 = ty * kTH;
    const int cbase = slice * NCH;
    const GridParams &g = a.g;

    CandSlot<kKC> *ring = reinterpret_cast<CandSlot<kKC> *>(sm + L::kCand);
    uint32_t *seg_b = reinterpret_cast<uint32_t *>(sm + L::kSeg);
    uint32_t *seg_off = seg_b + kMaxSeg;
    uint32_t *seg_n = seg_off + kMaxSeg;
    float *sw = reinterpret_cast<float *>(sm + L::kSums);                                // [128] unrounded
    float *swr = sw + kTM;                                                               // [128] rounded
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::kBars);
    uint64_t *fullA = bars, *fullB = bars + NS, *empty = bars + 2 * NS;
    uint64_t *cfull = bars + 3 * NS, *cempty = cfull + kRing, *probe = cempty + kRing;
    uint32_t *taddr_s = reinterpret_cast<uint32_t *>(sm + L::kMisc);
    unsigned *pair_s = taddr_s + 1;
    volatile unsigned *abort_s = taddr_s + 2;

    if (warp == RL::kMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(taddr_s)), "r"(L::kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if constexpr (L::kOnes) {
        // the ones atom (BF16 or FP16 1.0), written once; the MMAs read it
        // through the async proxy, ordered by the fence before the CTA barrier
        const uint32_t one2 = kBF16 ? 0x3F803F80u : 0x3C003C00u;
        for (int q = tid; q < kKC * 128 / 16; q += RL::kThreads)
            asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};"
                         :: "r"(smem_u32(sm + L::kOnesAt) + (uint32_t)q * 16u), "r"(one2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < NS; s++) {
            mbar_init(smem_u32(fullA + s), kWW * 32);
            mbar_init(smem_u32(fullB + s), 4 * 32);
            mbar_init(smem_u32(empty + s), 1);
        }
        for (int r = 0; r < kRing; r++) {
            mbar_init(smem_u32(cfull + r), 32);
            mbar_init(smem_u32(cempty + r), (kWW + 4) * 32);
        }
        mbar_init(smem_u32(probe), 1);
        mbar_fence_init();
        *pair_s = 0;
        *abort_s = 0;
        // probe of the give-up path: nothing ever arrives on `probe`, so this
        // wait runs out after the limit and every role then skips its work
        if (a.probe && !mbar_wait(smem_u32(probe), 0u, a.err, a.wait_ns)) *abort_s = 1;
    }
    if (warp == RL::kFetch)
        tile_runs(g, a.upix, a.ustart, a.rustart, a.rband, i0, j0, kTW, kTH, seg_b, seg_off, seg_n, kMaxSeg, a.err);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *taddr_s;
    const uint32_t nseg = seg_n[0], total = seg_n[1];
    const int nchunks = *abort_s ? 0 : (int)((total + kKC - 1) / kKC);
    const size_t nchan = (size_t)a.nchan;

    if (warp < kWW) {
        // ---------------- weights: row j = warp % 8; candidates lane and
        // lane + 32 (8 warps) or lane + 32 (warp / 8) (16 warps)
        const int j = warp & 7;
        const int hbase = kWW == 16 ? (warp >> 3) : 0;
        const int cj = j0 + j;
        const bool row_ok = cj < g.ny;
        const int ncol = min(kTW, g.nx - i0);
        const float kexp = g.kexp;
        float brel, cgk;
        {
            const int jc = min(cj, g.ny - 1);
            brel = (float)((double)(jc - j0) * g.pix * kDeg);
            cgk = kexp * cosf((float)((g.lat0 + ((double)jc - g.hy) * g.pix) * kDeg));
        }
        // column i sits i * hcol east of the tile's first cell; columns past
        // the grid's edge get weights too (their rows of D are not stored)
        // but are left out of the pair count
        const float hcol = (float)(g.pix * kDeg), invh = (float)(1.0 / (g.pix * kDeg));
        const uint32_t colmask = ncol >= kTW ? 0xFFFFu : ((1u << ncol) - 1u);
        const float blo = kexp * a.band_lo, bhi = kexp * a.band_hi;
        const Origin org(g, i0, j0);
        float ws[kTW], wr[kTW];
#pragma unroll
        for (int i = 0; i < kTW; i++) ws[i] = wr[i] = 0.f;
        unsigned npairs = 0;
        // A (MN-major): cell m = 16 j + i of candidate k at atom (m >> 6),
        // K-row k, 16-byte piece ((m & 63) >> 3) ^ (k & 7)
        const uint32_t a_row = (uint32_t)((j >> 2) * 8192);
        const uint32_t piece0 = (uint32_t)(2 * (j & 3));
        for (int c = 0; c < nchunks; c++) {
            const int r = c % kRing, s = c % NS;
            if (!wait_ab(smem_u32(cfull + r), (uint32_t)((c / kRing) & 1), a.err, a.wait_ns, abort_s)) break;
            const CandSlot<kKC> &sl = ring[r];
            // stage s was last read by the MMAs of chunk c - NS
            if (c >= NS &&
                !wait_ab(smem_u32(empty + s), (uint32_t)(((c / NS) - 1) & 1), a.err, a.wait_ns, abort_s))
                break;
            const uint32_t As = smem_u32(sm + s * L::kStage) + a_row;
            // weights of each candidate for the row's 16 cells.  The support
            // test is settled per candidate from the roots of its quadratic
            // in the column index (col_sets): columns surely inside get
            // exp2(-t), columns surely outside 0, and the few within the
            // estimate's error band of the boundary go to the exact FP64 test
            // first, so the unrolled loop holds no compare and no call
#pragma unroll
            for (int hh = 0; hh < RL::kCandPerLane; hh++) {
                const uint32_t k = (uint32_t)(lane + 32 * (hbase + hh));
                const float4 uvk = sl.uv[k];
                const float cu = org.u(uvk), cvv = org.v(uvk);
                const float dv = cvv - brel;
                const float dv2 = row_ok ? kexp * (dv * dv) : 1e30f;
                const float ak = cgk * sl.cs[k];
                const uint32_t rowk = As + k * 128;
                const uint32_t off0 = rowk + ((piece0 ^ (k & 7)) << 4), off1 = rowk + (((piece0 + 1) ^ (k & 7)) << 4);
                // candidates come ring by ring, so a warp's 32 usually share a
                // latitude: when none is within the support's reach of the row,
                // its A pieces are zeros
                if (!__any_sync(0xffffffffu, dv2 <= bhi)) {
                    asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" :: "r"(off0), "r"(0u) : "memory");
                    asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" :: "r"(off1), "r"(0u) : "memory");
                    continue;
                }
                uint32_t m_in, m_pos;
                col_sets(cu, dv2, ak, blo, bhi, invh, m_in, m_pos);
                const uint32_t band = m_pos & ~m_in;
                if (band) {
                    const uint32_t crw = sl.row[k];
#pragma unroll 1
                    for (int i = 0; i < kTW; i++)
                        if ((band & (1u << i)) && exact_inside(g, i0 + i, cj, a.lon, a.lat, crw)) m_in |= 1u << i;
                }
                npairs += __popc(m_in & colmask);
                uint32_t pk[4];
#pragma unroll
                for (int i = 0; i < kTW; i += 2) {
                    float w2[2];
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const float du = fmaf((float)-(i + e), hcol, cu);
                        const float t = fmaf(ak, du * du, dv2);
                        w2[e] = ex2_approx((m_in >> (i + e)) & 1u ? -t : -INFINITY);
                    }
                    ws[i] += w2[0];
                    ws[i + 1] += w2[1];
                    const uint32_t p2 = kBF16 ? pack2(w2[0], w2[1], true)
                                              : pack2(w2[0] * kF16WeightScale, w2[1] * kF16WeightScale, false);
                    if constexpr (!L::kOnes) {
                        wr[i] += unpack_lo(p2, kBF16);
                        wr[i + 1] += unpack_hi(p2, kBF16);
                    }
                    pk[(i >> 1) & 3] = p2;
                    if ((i & 7) == 6)
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                                     :: "r"(i < 8 ? off0 : off1), "r"(pk[0]), "r"(pk[1]), "r"(pk[2]), "r"(pk[3])
                                     : "memory");
                }
            }
            mbar_arrive(smem_u32(cempty + r));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(fullA + s));
        }
        // per-cell sums over the warp's candidates: lane i keeps cell i
#pragma unroll
        for (int i = 0; i < kTW; i++) {
            float x = ws[i], y = wr[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, o);
                if constexpr (!L::kOnes) y += __shfl_xor_sync(0xffffffffu, y, o);
            }
            if (lane == i) {
                if constexpr (kWW == 16) {
                    sw[kTM * hbase + 16 * j + i] = x;      // the two halves (swr is free: kOnes)
                } else {
                    sw[16 * j + i] = x;
                    swr[16 * j + i] = y;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        if (lane == 0 && npairs) atomicAdd(pair_s, npairs);
    } else if (warp < kWW + 4) {
        // ---------------- spectra: 16-byte pieces of B (8 channels of one row)
        const int bt = tid - kWW * 32;                     // 0 .. 127
        const T *spec = static_cast<const T *>(a.spec) + cbase;
        constexpr int kPieces = kKC * NCH / 8;             // per chunk
        constexpr int kPPT = kPieces / 128;                // per thread
        // piece p = bt + 128 q: row k = p / (NCH / 8), channel group cp = p % (NCH / 8)
        auto dst_of = [&](int p) -> uint32_t {
            const int k = p / (NCH / 8), cp = p % (NCH / 8);
            return (uint32_t)((cp >> 3) * (kKC * 128) + k * 128 + (((cp & 7) ^ (k & 7)) << 4));
        };
        if constexpr (kBF16) {
            for (int c = 0; c < nchunks; c++) {
                const int r = c % kRing, s = c % NS;
                if (!wait_ab(smem_u32(cfull + r), (uint32_t)((c / kRing) & 1), a.err, a.wait_ns, abort_s)) break;
                if (c >= NS &&
                    !wait_ab(smem_u32(empty + s), (uint32_t)(((c / NS) - 1) & 1), a.err, a.wait_ns, abort_s))
                    break;
                const uint32_t Bs = smem_u32(sm + s * L::kStage + L::kA);
#pragma unroll
                for (int q = 0; q < kPPT; q++) {
                    const int p = bt + 128 * q;
                    const int k = p / (NCH / 8), cp = p % (NCH / 8);
                    const uint32_t rw = ring[r].row[k];
                    const T *src = spec + (rw != 0xFFFFFFFFu ? (size_t)rw * nchan : 0) + cp * 8;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                                 :: "r"(Bs + dst_of(p)), "l"(src), "r"(rw != 0xFFFFFFFFu ? 16 : 0) : "memory");
                }
                mbar_arrive(smem_u32(cempty + r));
                // the barrier's arrival of this thread waits for its copies
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];"
                             :: "r"(smem_u32(fullB + s)) : "memory");
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
        } else {
            // FP8: loads run two chunks ahead through two register sets used
            // in turn (the loop takes two chunks per turn, so no set is copied)
            // two register sets while they fit the registers of 8 weight warps
            constexpr bool kTwoSets = kPPT <= 16 && kWW == 8;
            uint2 rA[kPPT], rB[kTwoSets ? kPPT : 1];
            auto issue = [&](int c, uint2 (&raw)[kPPT]) -> bool {
                const int r = c % kRing;
                if (!wait_ab(smem_u32(cfull + r), (uint32_t)((c / kRing) & 1), a.err, a.wait_ns, abort_s))
                    return false;
#pragma unroll
                for (int q = 0; q < kPPT; q++) {
                    const int p = bt + 128 * q;
                    const int k = p / (NCH / 8), cp = p % (NCH / 8);
                    const uint32_t rw = ring[r].row[k];
                    raw[q] = rw != 0xFFFFFFFFu
                        ? __ldg(reinterpret_cast<const uint2 *>(spec + (size_t)rw * nchan + cp * 8))
                        : make_uint2(0u, 0u);
                }
                mbar_arrive(smem_u32(cempty + r));
                return true;
            };
            auto put = [&](int c, uint2 (&raw)[kPPT]) -> bool {
                const int s = c % NS;
                if (c >= NS &&
                    !wait_ab(smem_u32(empty + s), (uint32_t)(((c / NS) - 1) & 1), a.err, a.wait_ns, abort_s))
                    return false;
                const uint32_t Bs = smem_u32(sm + s * L::kStage + L::kA);
#pragma unroll
                for (int q = 0; q < kPPT; q++) {
                    const uint2 v = raw[q];
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                                 :: "r"(Bs + dst_of(bt + 128 * q)), "r"(e4m3x2_to_f16x2(v.x & 0xffff)),
                                    "r"(e4m3x2_to_f16x2(v.x >> 16)), "r"(e4m3x2_to_f16x2(v.y & 0xffff)),
                                    "r"(e4m3x2_to_f16x2(v.y >> 16)) : "memory");
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(fullB + s));
                return true;
            };
            if constexpr (kTwoSets) {
                bool ok = (nchunks < 1 || issue(0, rA)) && (nchunks < 2 || issue(1, rB));
                for (int c = 0; ok && c < nchunks; c += 2) {
                    if (!put(c, rA) || (c + 2 < nchunks && !issue(c + 2, rA))) break;
                    if (c + 1 < nchunks && (!put(c + 1, rB) || (c + 3 < nchunks && !issue(c + 3, rB)))) break;
                }
            } else {          // 512-channel slices: one chunk ahead (the registers hold one set)
                bool ok = nchunks < 1 || issue(0, rA);
                for (int c = 0; ok && c < nchunks; c++)
                    if (!put(c, rA) || (c + 1 < nchunks && !issue(c + 1, rA))) break;
            }
        }
    } else if (warp == RL::kFetch) {
        fetch_ring<kKC>(ring, cfull, cempty, nchunks, total, nseg, seg_b, seg_off, a.uv, a.cs, a.row, a.err,
                        a.wait_ns, abort_s);
    } else if (lane == 0) {
        // ---------------- MMA issue
        const uint32_t idesc = idesc_f16(kBF16, 256, kTM), idesc1 = idesc_f16(kBF16, 16, kTM);
        const uint32_t ones = smem_u32(sm + L::kOnesAt);
        int issued = -1;
        for (int c = 0; c < nchunks; c++) {
            const int s = c % NS;
            const uint32_t par = (uint32_t)((c / NS) & 1);
            if (!wait_ab(smem_u32(fullA + s), par, a.err, a.wait_ns, abort_s)) break;
            if (!wait_ab(smem_u32(fullB + s), par, a.err, a.wait_ns, abort_s)) break;
            // the spectrum copies are generic-proxy writes: order them before
            // the tensor core's reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t abase = smem_u32(sm + s * L::kStage), bbase = abase + L::kA;
#pragma unroll
            for (int kk = 0; kk < kKC / 16; kk++) {
                const uint64_t ad = sdesc(abase + kk * 2048, kKC * 128, 1024);
#pragma unroll
                for (int nb = 0; nb < NCH / 256; nb++) {
                    const uint64_t bd = sdesc(bbase + nb * 4 * (kKC * 128) + kk * 2048, kKC * 128, 1024);
                    mma_f16(tmem + nb * 256, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                }
                // the row sums of A (the rounded weights) into columns 256-271
                if constexpr (L::kOnes)
                    mma_f16(tmem + 256, ad, sdesc(ones + kk * 2048, kKC * 128, 1024), idesc1,
                            (c > 0 || kk > 0) ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(empty + s)) : "memory");
            issued = c;
        }
        // nothing may still be running on TMEM when it is read or freed
        if (issued >= 0) {
            mbar_wait(smem_u32(empty + (issued % NS)), (uint32_t)((issued / NS) & 1), a.err, a.wait_ns);
            if (a.tflops)
                atomicAdd(a.tflops, (unsigned long long)(issued + 1) * (2ull * kTM * kKC * (NCH + (L::kOnes ? 16 : 0))));
        }
    }

    // ---- epilogue (weight warps): D over the rounded-weight sum
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool have = nchunks > 0 && !*abort_s;
    if (warp < kWW) {
        const int q = warp & 3, part = warp >> 2;          // TMEM lanes 32 q .., column part `part`
        const int mm = q * 32 + lane;                       // TMEM lane = cell
        const int ii = i0 + (mm & (kTW - 1)), jj = j0 + (mm >> 4);
        const bool ok = ii < g.nx && jj < g.ny;
        const float W = kWW == 16 ? sw[mm] + sw[kTM + mm] : sw[mm];
        float Wr = swr[mm];
        if constexpr (L::kOnes) {
            // the normaliser from the ones column: the sum of the weights the
            // MMAs multiplied, as the MMAs summed them
            uint32_t wbits = 0;
            if (have) {
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                             : "=r"(wbits) : "r"(tmem + ((uint32_t)(q * 32) << 16) + 256u) : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            Wr = __uint_as_float(wbits);
        }
        // when W > 0 the rounded weights' sum holds at least one in-support
        // weight (>= exp(-12.5) at this path's 5-sigma limit, normal in BF16
        // and in FP16 x 2^10), so its reciprocal is finite; V = D / Wr to an ulp
        const float rWr = 1.0f / Wr;
        float *out = a.cube + ((size_t)(ok ? jj : 0) * g.nx + (ok ? ii : 0)) * (size_t)a.cube_ld + cbase;
        const bool vec_out = (a.cube_ld & 3) == 0 && ((uintptr_t)a.cube & 15) == 0;
        float *tb = reinterpret_cast<float *>(sm) + warp * (32 * 36);   // the stages are free now
        constexpr int kCols = NCH / (kWW / 4);              // per warp
#pragma unroll 1
        for (int cc = 0; cc < kCols; cc += 32) {
            const int col = part * kCols + cc;
            uint32_t r[32];
            if (have) {
                TMEM_LD32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
#pragma unroll
            for (int e = 0; e < 32; e++) {
                float val = W > 0.0f && have ? __uint_as_float(r[e]) * rWr : __int_as_float(0x7fc00000);
                if (a.scale) val *= __ldg(a.scale + cbase + col + e);
                r[e] = __float_as_uint(val);
            }
            store_block32(tb, r, out + col, ok, vec_out, lane);
        }
        if (slice == 0 && part == 0 && ok) a.wout[(size_t)jj * g.nx + ii] = W;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (slice == 0 && tid == 0 && *pair_s && a.pairs) atomicAdd(a.pairs, (unsigned long long)*pair_s);
    if (warp == RL::kMma)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(L::kTmemCols)
                     : "memory");
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
// kept short: the MMAs sum one block of kBlk32 chunks (1024 candidates) into
// TMEM columns [0, 256), which the CUDA cores then add into a running total
// in columns [256, 512) (FP32, round to nearest) before the next block starts
// afresh -- over thousands of successive K-steps the accumulator otherwise
// drifts by a few 1e-5 (measured at 13,000 candidates per tile).
// Chunks of 32 candidates (one 128-byte swizzle atom of TF32 per row); per
// stage A_hi, A_lo [128 cells x 32] and B_hi, B_lo [256 channels x 32], all
// K-major (kind::tf32 reads 32-bit operands K-major only: an MN-major B gives
// zeros), 96 KB; two stages, one CTA per SM.
//
// The CTA's warps keep to one role each and hand work over through
// mbarriers (no CTA-wide barrier inside the chunk loop):
//   warps 0-7   weights: warp j owns tile row j and lane k candidate k of
//               the chunk; the support test for the row's 16 cells is
//               settled by col_sets, and each lane splits its candidate's
//               16 weights and stores them into the cells' K-major rows of
//               A_hi / A_lo; a finished block's sums are moved into the
//               running total after the next chunk's weights (warp w: TMEM
//               lanes 32 (w % 4) .. + 31, column half w / 4);
//   warps 8-15  spectra: thread n loads channel n of the chunk's 32 rows one
//               chunk ahead (the loads fly while the MMAs of the previous
//               chunk run; a second register set does not fit the 96
//               registers that 18 warps leave a thread), splits them into
//               B_hi / B_lo;
//   warp 16     candidates: copies each chunk's candidates from the tile's
//               S' runs into the candidate ring;
//   warp 17     one thread issues the MMAs and commits them to the barrier
//               that frees the stage.
// Every wait is bounded; the first one that gives up raises TIMEOUT and an
// abort flag that ends every other role's waits at once.
constexpr int kKC32 = 32;
constexpr int kBlk32 = 32;                              // chunks per TMEM accumulation block
constexpr int kWs32Threads = 576;
constexpr int kFetchWarp = 16, kMmaWarp = 17;

struct Layout32 {
    static constexpr int kA = kTM * 128;                 // 128 rows x 32 TF32 = 16 KB (hi or lo)
    static constexpr int kB = 256 * 128;                 // 256 channel rows x 32 TF32 = 32 KB (hi or lo)
    static constexpr int kStage = 2 * kA + 2 * kB;       // A_hi, A_lo, B_hi, B_lo
    static constexpr int kCand = kStages * kStage;
    static constexpr int kSeg = kCand + kRing * (int)sizeof(CandSlot<kKC32>);
    static constexpr int kSums = kSeg + kMaxSeg * 8 + 16;
    static constexpr int kBars = kSums + 2 * kTM * 4;
    // barriers: fullA[2], fullB[2], empty[2], cfull[kRing], cempty[kRing], blk, drained, probe
    static constexpr int kNumBars = 3 * kStages + 2 * kRing + 3;
    static constexpr int kMisc = kBars + kNumBars * 8;
    static constexpr int kTotal = kMisc + 64;
};
static_assert(Layout32::kBars % 8 == 0, "barrier alignment");

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

__global__ void __launch_bounds__(kWs32Threads, 1) k_tc_gather_f32(TcArgs a) {
    using L = Layout32;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile = blockIdx.x % a.ntiles;
    const int slice = (int)(blockIdx.x / a.ntiles);
    const int ty = a.nty - 1 - (int)(tile / a.ntx);      // north tile row first
    const int i0 = (int)(tile % a.ntx) * kTW, j0 = ty * kTH;
    const int cbase = slice * 256;
    const GridParams &g = a.g;

    CandSlot<kKC32> *ring = reinterpret_cast<CandSlot<kKC32> *>(sm + L::kCand);
    uint32_t *seg_b = reinterpret_cast<uint32_t *>(sm + L::kSeg);
    uint32_t *seg_off = seg_b + kMaxSeg;
    uint32_t *seg_n = seg_off + kMaxSeg;
    float *sw = reinterpret_cast<float *>(sm + L::kSums);                                // [2][128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::kBars);
    uint64_t *fullA = bars, *fullB = bars + kStages, *empty = bars + 2 * kStages;
    uint64_t *cfull = bars + 3 * kStages, *cempty = cfull + kRing;
    uint64_t *blk = cempty + kRing, *drained = blk + 1, *probe = blk + 2;
    uint32_t *taddr_s = reinterpret_cast<uint32_t *>(sm + L::kMisc);
    unsigned *pair_s = taddr_s + 1;
    volatile unsigned *abort_s = taddr_s + 2;

    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(taddr_s)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(smem_u32(fullA + s), 8 * 32);
            mbar_init(smem_u32(fullB + s), 8 * 32);
            mbar_init(smem_u32(empty + s), 1);
        }
        for (int r = 0; r < kRing; r++) {
            mbar_init(smem_u32(cfull + r), 32);
            mbar_init(smem_u32(cempty + r), 16 * 32);
        }
        mbar_init(smem_u32(blk), 1);
        mbar_init(smem_u32(drained), 8 * 32);
        mbar_init(smem_u32(probe), 1);
        mbar_fence_init();
        *pair_s = 0;
        *abort_s = 0;
        // probe of the give-up path: nothing ever arrives on `probe`, so this
        // wait runs out after the limit and every role then skips its work
        if (a.probe && !mbar_wait(smem_u32(probe), 0u, a.err, a.wait_ns)) *abort_s = 1;
    }
    if (warp == 1)
        tile_runs(g, a.upix, a.ustart, a.rustart, a.rband, i0, j0, kTW, kTH, seg_b, seg_off, seg_n, kMaxSeg, a.err);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *taddr_s;
    const uint32_t nseg = seg_n[0], total = seg_n[1];
    const int nchunks = *abort_s ? 0 : (int)((total + kKC32 - 1) / kKC32);
    const size_t nchan = (size_t)a.nchan;

    if (warp < 8) {
        // ---------------- weights: row j = warp % 8 of the tile; lane k takes
        // candidate k of the chunk and computes its weights for the row's 16
        // cells (the support test settled per candidate by col_sets, as in
        // the BF16 kernel), writing each cell's A_hi / A_lo element
        const int j = warp & 7, hf = warp >> 2;
        const int cj = j0 + j;
        const bool row_ok = cj < g.ny;
        const int ncol = min(kTW, g.nx - i0);
        const float kexp = g.kexp;
        float brel, cgk;
        {
            const int jc = min(cj, g.ny - 1);
            brel = (float)((double)(jc - j0) * g.pix * kDeg);
            cgk = kexp * cosf((float)((g.lat0 + ((double)jc - g.hy) * g.pix) * kDeg));
        }
        const float hcol = (float)(g.pix * kDeg), invh = (float)(1.0 / (g.pix * kDeg));
        const uint32_t colmask = ncol >= kTW ? 0xFFFFu : ((1u << ncol) - 1u);
        const float blo = kexp * a.band_lo, bhi = kexp * a.band_hi;
        const Origin org(g, i0, j0);
        const uint32_t lanebase = (uint32_t)((warp & 3) * 32) << 16;   // TMEM lanes of this warp
        // A (K-major, 128-byte swizzle): cell m = 16 j + i, candidate k at
        // m * 128 + 16 ((k / 4) ^ (m % 8)) + 4 (k % 4); with m % 8 = i % 8
        const uint32_t kbyte = (uint32_t)((lane & 3) << 2), kunit = (uint32_t)(lane >> 2);
        // end of a block (chunk c ends it): once its MMAs are done, add its
        // sums into the running total (columns 256..511; the first block just
        // moves in); warp w moves TMEM lanes 32 (w % 4) .., column half w / 4
        auto drain = [&](int c) -> bool {
            if (!(c % kBlk32 == kBlk32 - 1 || c == nchunks - 1)) return true;
            if (!wait_ab(smem_u32(blk), (uint32_t)((c / kBlk32) & 1), a.err, a.wait_ns, abort_s)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int cc = 0; cc < 128; cc += 16) {
                const uint32_t col = (uint32_t)(hf * 128 + cc);
                uint32_t rb[16], rt[16];
                TMEM_LD16(tmem + lanebase + col, rb);
                if (c >= kBlk32) TMEM_LD16(tmem + lanebase + 256u + col, rt);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (c >= kBlk32) {
#pragma unroll
                    for (int e = 0; e < 16; e++)
                        rb[e] = __float_as_uint(__uint_as_float(rt[e]) + __uint_as_float(rb[e]));
                }
                TMEM_ST16(tmem + lanebase + 256u + col, rb);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(drained));
            return true;
        };
        float ws[kTW];
#pragma unroll
        for (int i = 0; i < kTW; i++) ws[i] = 0.f;
        unsigned npairs = 0;
        bool completed = false;
        for (int c = 0; c < nchunks; c++) {
            const int r = c % kRing, s = c & 1;
            if (!wait_ab(smem_u32(cfull + r), (uint32_t)((c / kRing) & 1), a.err, a.wait_ns, abort_s)) break;
            const CandSlot<kKC32> &sl = ring[r];
            const float4 uvk = sl.uv[lane];
            const float cu = org.u(uvk), cvv = org.v(uvk);
            const float dv = cvv - brel;
            const float dv2 = row_ok ? kexp * (dv * dv) : 1e30f;
            const float ak = cgk * sl.cs[lane];
            // a row none of whose 32 candidates lies within the support's
            // latitude reach gets zeros
            const bool near = __any_sync(0xffffffffu, dv2 <= bhi);
            uint32_t m_in = 0;
            if (near) {
                uint32_t m_pos;
                col_sets(cu, dv2, ak, blo, bhi, invh, m_in, m_pos);
                const uint32_t band = m_pos & ~m_in;
                if (band) {
                    const uint32_t crw = sl.row[lane];
#pragma unroll 1
                    for (int i = 0; i < kTW; i++)
                        if ((band & (1u << i)) && exact_inside(g, i0 + i, cj, a.lon, a.lat, crw)) m_in |= 1u << i;
                }
            }
            mbar_arrive(smem_u32(cempty + r));
            npairs += __popc(m_in & colmask);
            // stage s was last read by the MMAs of chunk c - 2
            if (c >= kStages &&
                !wait_ab(smem_u32(empty + s), (uint32_t)(((c >> 1) - 1) & 1), a.err, a.wait_ns, abort_s))
                break;
            const uint32_t ah = smem_u32(sm + s * L::kStage) + (uint32_t)(16 * j * 128) + kbyte, al = ah + L::kA;
#pragma unroll
            for (int i = 0; i < kTW; i++) {
                float x = 0.0f;
                if (near) {
                    const float du = fmaf((float)-i, hcol, cu);
                    const float t = fmaf(ak, du * du, dv2);
                    x = ex2_approx((m_in >> i) & 1u ? -t : -INFINITY);
                }
                ws[i] += x;
                const float hi = tf32_head(x);
                const uint32_t o = (uint32_t)(i * 128) + ((kunit ^ (uint32_t)(i & 7)) << 4);
                asm volatile("st.shared.f32 [%0], %1;" :: "r"(ah + o), "f"(hi) : "memory");
                asm volatile("st.shared.f32 [%0], %1;" :: "r"(al + o), "f"(x - hi) : "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(fullA + s));
            // a block that ended with the previous chunk is drained now, after
            // this chunk's weights: the MMAs of this chunk wait for the drain,
            // the weights no longer do
            if (c > 0 && !drain(c - 1)) break;
            if (c == nchunks - 1) completed = true;
        }
        if (completed) drain(nchunks - 1);
        // per-cell sums over the row's candidates: lane i keeps cell i
#pragma unroll
        for (int i = 0; i < kTW; i++) {
            float x = ws[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == i) sw[16 * j + i] = x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        if (lane == 0 && npairs) atomicAdd(pair_s, npairs);
    } else if (warp < 16) {
        // ---------------- spectra: thread n = channel n of every row
        const uint32_t n = (uint32_t)(tid - 256);
        const float *spec = static_cast<const float *>(a.spec) + cbase + n;
        float rA[kKC32];
        // loads of chunk c (the candidate slot is released once the row
        // indices are read)
        auto issue = [&](int c, float (&raw)[kKC32]) -> bool {
            const int r = c % kRing;
            if (!wait_ab(smem_u32(cfull + r), (uint32_t)((c / kRing) & 1), a.err, a.wait_ns, abort_s))
                return false;
#pragma unroll
            for (int k = 0; k < kKC32; k++) {
                const uint32_t rw = ring[r].row[k];
                raw[k] = rw != 0xFFFFFFFFu ? __ldg(spec + (size_t)rw * nchan) : 0.0f;
            }
            mbar_arrive(smem_u32(cempty + r));
            return true;
        };
        // B split into its K-major swizzled hi / lo tiles (channel n's row at
        // n * 128, candidates 4 q .. 4 q + 3 in 16-byte unit q ^ (n & 7)); at
        // the end of a block, the drain
        auto put = [&](int c, float (&raw)[kKC32]) -> bool {
            const int s = c & 1;
            if (c >= kStages &&
                !wait_ab(smem_u32(empty + s), (uint32_t)(((c >> 1) - 1) & 1), a.err, a.wait_ns, abort_s))
                return false;
            const uint32_t b0 = smem_u32(sm + s * L::kStage + 2 * L::kA) + n * 128;
#pragma unroll
            for (int q = 0; q < kKC32 / 4; q++) {
                const uint32_t o = ((uint32_t)q ^ (n & 7)) << 4;
                float h[4], x[4];
#pragma unroll
                for (int e = 0; e < 4; e++) { x[e] = raw[4 * q + e]; h[e] = tf32_head(x[e]); }
                asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};"
                             :: "r"(b0 + o), "f"(h[0]), "f"(h[1]), "f"(h[2]), "f"(h[3]) : "memory");
                asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};"
                             :: "r"(b0 + L::kB + o), "f"(x[0] - h[0]), "f"(x[1] - h[1]), "f"(x[2] - h[2]),
                                "f"(x[3] - h[3]) : "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(fullB + s));
            return true;
        };
        bool ok = (nchunks < 1 || issue(0, rA));
        for (int c = 0; ok && c < nchunks; c++)
            if (!put(c, rA) || (c + 1 < nchunks && !issue(c + 1, rA))) break;
    } else if (warp == kFetchWarp) {
        fetch_ring<kKC32>(ring, cfull, cempty, nchunks, total, nseg, seg_b, seg_off, a.uv, a.cs, a.row, a.err,
                          a.wait_ns, abort_s);
    } else if (lane == 0) {
        // ---------------- MMA issue
        const uint32_t idesc = idesc_tf32(256, kTM);
        int issued = -1;
        for (int c = 0; c < nchunks; c++) {
            const int s = c & 1;
            const uint32_t par = (uint32_t)((c >> 1) & 1);
            if (!wait_ab(smem_u32(fullA + s), par, a.err, a.wait_ns, abort_s)) break;
            if (!wait_ab(smem_u32(fullB + s), par, a.err, a.wait_ns, abort_s)) break;
            // a new block starts once the previous one has been drained
            if (c % kBlk32 == 0 && c > 0 &&
                !wait_ab(smem_u32(drained), (uint32_t)(((c / kBlk32) - 1) & 1), a.err, a.wait_ns, abort_s))
                break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char *Ahi = sm + s * L::kStage;
            const uint32_t ah = smem_u32(Ahi), al = ah + L::kA, bh = ah + 2 * L::kA, bl = bh + L::kB;
#pragma unroll
            for (int kk = 0; kk < kKC32 / 8; kk++) {
                const uint64_t dah = sdesc(ah + kk * 32, 16, 1024), dal = sdesc(al + kk * 32, 16, 1024);
                const uint64_t dbh = sdesc(bh + kk * 32, 16, 1024), dbl = sdesc(bl + kk * 32, 16, 1024);
                mma_tf32(tmem, dah, dbh, idesc, (c % kBlk32 > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, idesc, 1u);
                mma_tf32(tmem, dal, dbh, idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(empty + s)) : "memory");
            if (c % kBlk32 == kBlk32 - 1 || c == nchunks - 1)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(smem_u32(blk)) : "memory");
            issued = c;
        }
        // nothing may still be running on TMEM when it is read or freed
        if (issued >= 0) {
            mbar_wait(smem_u32(empty + (issued & 1)), (uint32_t)((issued >> 1) & 1), a.err, a.wait_ns);
            if (a.tflops) atomicAdd(a.tflops, (unsigned long long)(issued + 1) * (3ull * 2ull * kTM * kKC32 * 256));
        }
    }

    // ---- epilogue: the running total (columns 256..511) over the weight sum
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool have = nchunks > 0 && !*abort_s;
    if (warp < 16) {
        // weight and spectra warps: warp w reads TMEM lanes 32 (w % 4) .. + 31
        // (cells) and columns 64 (w / 4) .. + 63 of the running total
        const int q = warp & 3, part = warp >> 2;
        const int mm = q * 32 + lane;
        const int ii = i0 + (mm & (kTW - 1)), jj = j0 + (mm >> 4);
        const bool ok = ii < g.nx && jj < g.ny;
        const float W = sw[mm];
        float *out = a.cube + ((size_t)(ok ? jj : 0) * g.nx + (ok ? ii : 0)) * (size_t)a.cube_ld + cbase;
        const bool vec_out = (a.cube_ld & 3) == 0 && ((uintptr_t)a.cube & 15) == 0;
        float *tb = reinterpret_cast<float *>(sm) + warp * (32 * 36);   // the stages are free now
#pragma unroll 1
        for (int cc = 0; cc < 64; cc += 32) {
            const int col = part * 64 + cc;
            uint32_t r[32];
            if (have) {
                TMEM_LD32(tmem + ((uint32_t)(q * 32) << 16) + 256u + (uint32_t)col, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
#pragma unroll
            for (int e = 0; e < 32; e++) {
                const float sv = have ? __uint_as_float(r[e]) : 0.0f;
                float val;
                if (!(W > 0.0f) || !have) val = __int_as_float(0x7fc00000);
                else if (W >= 1e-3f) val = __fdiv_rn(sv, W);
                else val = (float)((double)sv / (double)W);
                r[e] = __float_as_uint(val);
            }
            store_block32(tb, r, out + col, ok, vec_out, lane);
        }
        if (slice == 0 && part == 0 && ok) a.wout[(size_t)jj * g.nx + ii] = W;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (slice == 0 && tid == 0 && *pair_s && a.pairs) atomicAdd(a.pairs, (unsigned long long)*pair_s);
    if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
}

int launch_f32(hcg_ctx *c, const TcArgs &a0) {
    TcArgs a = a0;
    a.nslices = a.nchan / 256;
    const int smem = Layout32::kTotal + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_tc_gather_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) { hcg_cuda_fail(e, "tc f32 smem attribute"); return -1; }
    const int64_t blocks = a.ntiles * a.nslices;
    k_tc_gather_f32<<<(unsigned)blocks, kWs32Threads, smem, c->stream>>>(a);
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
    k_tc_gather<T, NCH><<<(unsigned)blocks, TcRoles<NCH>::kThreads, smem, c->stream>>>(a);
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
    a.tflops = reinterpret_cast<unsigned long long *>(c->dscal + 2);
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

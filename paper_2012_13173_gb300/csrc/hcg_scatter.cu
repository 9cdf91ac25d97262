// hcg_scatter.cu -- the scattering strategy of HCGrid Sec. 2.2, kept as a
// measured comparison to the gather: every input sample adds its
// contribution to every cell whose support holds it, and the write conflicts
// between samples are resolved with atomic adds.  No pre-ordering and no
// lookup tables are needed; samples are taken in input order.
//
//   k_scatter    one warp per sample: candidate cells from a box around the
//                sample (rows within R in latitude, columns within the
//                support's longitude extent at the sample's latitude, both
//                sides of the longitude seam), the exact FP64 support test of
//                Eq. (1) per cell (the oracle's operation order), then for
//                every cell inside: W += w (first channel window only) and
//                acc[c] += w V[c] over the channels, four channels per lane
//                with one 16-byte vector atomic (red.global.add.v4.f32)
//   k_scatter_normalise   V = acc / W, NaN where W = 0, times the E4M3 scale
//
// Atomic adds land in an order the hardware chooses, so sums (and results)
// differ from the gather's in the last bits and from run to run.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "hcg_dev.cuh"

namespace {

constexpr int kSWarps = 8;
constexpr int kSMaxIn = 512;          // inside cells staged per warp before their channels are added

struct ScatterArgs {
    GridParams g;
    const double *lon, *lat;          // input order
    const void *spec;                 // [n][nchan] rows of the window
    int64_t n;
    int nchan;                        // channels of the window
    float *cube;                      // first channel of the window
    int64_t cube_ld;                  // cube row stride (all channels)
    float *wout;                      // weights [ny][nx]; summed only when pairs != nullptr
    unsigned long long *pairs;        // pair counter (first window), else nullptr
};

struct ScatterSmem {
    uint32_t cell[kSMaxIn];           // cell index j * nx + i (launch_scatter keeps cells below 2^32)
    float w[kSMaxIn];
};

// Four channels of one row as FP32 (zeros past the row's end).
template <typename T>
HCG_DEV float4 load4(const T *row, int c, int nchan);

template <>
HCG_DEV float4 load4<float>(const float *row, int c, int nchan) {
    if (c + 4 <= nchan && (nchan & 3) == 0) return __ldg(reinterpret_cast<const float4 *>(row + c));
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = c + k < nchan ? __ldg(row + c + k) : 0.0f;
    return make_float4(v[0], v[1], v[2], v[3]);
}

template <>
HCG_DEV float4 load4<__nv_bfloat16>(const __nv_bfloat16 *row, int c, int nchan) {
    const unsigned short *h = reinterpret_cast<const unsigned short *>(row);
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = c + k < nchan ? __uint_as_float(((uint32_t)__ldg(h + c + k)) << 16) : 0.0f;
    return make_float4(v[0], v[1], v[2], v[3]);
}

template <>
HCG_DEV float4 load4<__nv_fp8_storage_t>(const __nv_fp8_storage_t *row, int c, int nchan) {
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (c + k < nchan) {
            __half_raw r = __nv_cvt_fp8_to_halfraw(row[c + k], __NV_E4M3);
            v[k] = __half2float(*reinterpret_cast<__half *>(&r));
        } else {
            v[k] = 0.0f;
        }
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

HCG_DEV void red_add4(float *p, float4 v, bool vec) {
    if (vec) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                     :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
    } else {
        atomicAdd(p, v.x); atomicAdd(p + 1, v.y); atomicAdd(p + 2, v.z); atomicAdd(p + 3, v.w);
    }
}

// Column intervals (up to three: the box and its copies one turn east and
// west) of cells whose longitude can lie within R of a sample at offset a
// (degrees from lon0) and latitude lat.
struct ColRanges {
    int lo[3], len[3];
    int total;
};

HCG_DEV void column_ranges(const GridParams &g, double a, double lat, ColRanges &cr) {
    cr.total = 0;
    double half;                                         // longitude extent, degrees
    if (fabs(lat) + g.R_deg >= 89.99) {
        half = 400.0;
    } else {
        double s = sin(g.R_deg * kDeg) / cos(lat * kDeg);
        half = s >= 1.0 ? 400.0 : asin(s) / kDeg;
    }
    half = half * (1.0 + 1e-9) + 1e-9;
    int lo0 = 0, hi0 = -1;
    for (int k = 0; k < 3; k++) {
        const double centre = a + (k == 0 ? 0.0 : (k == 1 ? 360.0 : -360.0));
        int lo = (int)fmin(fmax(0.0, ceil((centre - half) / g.pix + g.hx)), (double)g.nx);
        int hi = (int)fmax(fmin((double)(g.nx - 1), floor((centre + half) / g.pix + g.hx)), -1.0);
        if (k == 0) { lo0 = lo; hi0 = hi; }
        else if (hi0 >= lo0) {                           // drop columns the first interval has
            if (k == 1) lo = max(lo, hi0 + 1);
            else hi = min(hi, lo0 - 1);
        }
        if (k == 2 && cr.len[1] > 0) hi = min(hi, cr.lo[1] - 1);
        cr.lo[k] = lo;
        cr.len[k] = max(0, hi - lo + 1);
        cr.total += cr.len[k];
    }
}

template <typename T>
__global__ void __launch_bounds__(kSWarps * 32) k_scatter(ScatterArgs a) {
    __shared__ ScatterSmem smem[kSWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ScatterSmem &sm = smem[warp];
    const GridParams &g = a.g;
    const T *spec = static_cast<const T *>(a.spec);
    const bool vec = (a.cube_ld & 3) == 0 && (a.nchan & 3) == 0;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t gw = (int64_t)gridDim.x * kSWarps;
    unsigned npairs = 0;
    for (int64_t n = (int64_t)blockIdx.x * kSWarps + warp; n < a.n; n += gw) {
        const double lon = a.lon[n], lat = a.lat[n];
        const double off = wrap180(lon - g.lon0);
        // rows within R in latitude
        const double fj = (lat - g.lat0) / g.pix + g.hy, rc = g.R_deg / g.pix * (1.0 + 1e-9) + 1e-9;
        const int jlo = (int)fmin(fmax(0.0, ceil(fj - rc)), (double)g.ny);
        const int jhi = (int)fmax(fmin((double)(g.ny - 1), floor(fj + rc)), -1.0);
        if (jhi < jlo) continue;
        ColRanges cr;
        column_ranges(g, off, lat, cr);
        if (cr.total == 0) continue;
        const int64_t box = (int64_t)(jhi - jlo + 1) * cr.total;
        const T *row = spec + (size_t)n * (size_t)a.nchan;
        for (int64_t base = 0; base < box; base += kSMaxIn) {
            // stage up to kSMaxIn inside cells of this part of the box
            int cnt = 0;
            const int64_t end = min(box, base + (int64_t)kSMaxIn);
            for (int64_t q0 = base; q0 < end; q0 += 32) {
                const int64_t q = q0 + lane;
                bool in = false;
                uint32_t cell = 0;
                float w = 0.0f;
                if (q < end) {
                    const int jj = jlo + (int)(q / cr.total);
                    int ii = (int)(q % cr.total);
                    ii = ii < cr.len[0] ? cr.lo[0] + ii
                                        : (ii < cr.len[0] + cr.len[1] ? cr.lo[1] + ii - cr.len[0]
                                                                      : cr.lo[2] + ii - cr.len[0] - cr.len[1]);
                    const double h = hav_exact_t<false>(g, ii, jj, lon, lat);   // plain grids only
                    in = h <= g.hR;
                    if (in) {
                        // d^2 = 4 asin^2(sqrt h) = 4 h (1 + h / 3 + 8 h^2 / 45 + ...)
                        const float hf = (float)h;
                        const float d2 = 4.0f * hf * fmaf(hf, fmaf(hf, 8.0f / 45.0f, 1.0f / 3.0f), 1.0f);
                        w = exp2f(-d2 * g.kexp);
                        cell = (uint32_t)jj * (uint32_t)g.nx + (uint32_t)ii;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, in);
                if (in) {
                    const int pos = cnt + __popc(m & lt);
                    sm.cell[pos] = cell;
                    sm.w[pos] = w;
                }
                cnt += __popc(m);
            }
            __syncwarp();
            if (a.pairs) {
                if (lane == 0) npairs += (unsigned)cnt;      // the warp's count, once
                for (int k = lane; k < cnt; k += 32) atomicAdd(a.wout + sm.cell[k], sm.w[k]);
            }
            for (int c0 = 0; c0 < a.nchan; c0 += 128) {
                const int c = c0 + lane * 4;
                if (c >= a.nchan) continue;
                const float4 x = load4<T>(row, c, a.nchan);
                for (int k = 0; k < cnt; k++) {
                    const float w = sm.w[k];
                    float *p = a.cube + (size_t)sm.cell[k] * (size_t)a.cube_ld + c;
                    if (c + 4 <= a.nchan) {
                        red_add4(p, make_float4(w * x.x, w * x.y, w * x.z, w * x.w), vec);
                    } else {
                        const float xs[4] = {x.x, x.y, x.z, x.w};
                        for (int e = 0; c + e < a.nchan; e++) atomicAdd(p + e, w * xs[e]);
                    }
                }
            }
            __syncwarp();
        }
    }
    if (a.pairs) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        if (lane == 0 && npairs) atomicAdd(a.pairs, (unsigned long long)npairs);
    }
}

// V = acc / W over the window's channels of every cell (the gather's
// division rule: FP32 when W >= 1e-3, FP64 below; NaN when W = 0), times
// the per-channel scale of E4M3 spectra.
__global__ void k_scatter_normalise(float *cube, int64_t cube_ld, int nchan, const float *wout, int64_t cells,
                                    const float *scale) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cells * nchan) return;
    const int64_t cell = t / nchan;
    const int c = (int)(t % nchan);
    const float W = wout[cell];
    float *p = cube + cell * cube_ld + c;
    float v;
    if (W >= 1e-3f) v = __fdiv_rn(*p, W);
    else if (W > 0.0f) v = (float)((double)*p / (double)W);
    else v = __int_as_float(0x7fc00000);
    if (scale) v *= scale[c];
    *p = v;
}

}  // namespace

// Scatter of the current channel window (c->win_c0, c->win_channels()) of
// the spectra `spec` (device, type dtype) into the cube; returns the number of
// kernels launched or -1.
int launch_scatter(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale) {
    const int nc = c->win_channels();
    const int64_t cells = (int64_t)c->nx * c->ny;
    float *cube = c->cube() + c->win_c0;
    const bool first = c->win_c0 == 0;
    int launches = 0;
    if (cells == 0) return 0;
    if (cells > 0xFFFFFFFFll) { hcg_set_error("scatter path: more than 2^32 cells"); return -1; }
    cudaError_t e = cudaMemset2DAsync(cube, (size_t)c->nchan * 4, 0, (size_t)nc * 4, (size_t)cells, c->stream);
    if (e != cudaSuccess) { hcg_cuda_fail(e, "clear cube window"); return -1; }
    if (first) {
        e = cudaMemsetAsync(c->weights(), 0, (size_t)cells * 4, c->stream);
        if (e != cudaSuccess) { hcg_cuda_fail(e, "clear weights"); return -1; }
    }
    ScatterArgs a;
    a.g = gp;
    a.lon = c->lon; a.lat = c->lat;
    a.spec = spec; a.n = c->n; a.nchan = nc;
    a.cube = cube; a.cube_ld = c->nchan;
    a.wout = c->weights();
    a.pairs = first ? reinterpret_cast<unsigned long long *>(c->dscal + 1) : nullptr;
    if (c->n > 0) {
        int per_sm = 0;
        const void *fn = dtype == HCG_F32 ? (const void *)k_scatter<float>
                         : (dtype == HCG_BF16 ? (const void *)k_scatter<__nv_bfloat16>
                                              : (const void *)k_scatter<__nv_fp8_storage_t>);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSWarps * 32, 0);
        const int64_t blocks = std::min<int64_t>((c->n + kSWarps - 1) / kSWarps,
                                                 (int64_t)std::max(1, per_sm) * c->num_sms);
        if (dtype == HCG_F32) k_scatter<float><<<(unsigned)blocks, kSWarps * 32, 0, c->stream>>>(a);
        else if (dtype == HCG_BF16) k_scatter<__nv_bfloat16><<<(unsigned)blocks, kSWarps * 32, 0, c->stream>>>(a);
        else k_scatter<__nv_fp8_storage_t><<<(unsigned)blocks, kSWarps * 32, 0, c->stream>>>(a);
        launches++;
    }
    const int64_t m = cells * nc;
    k_scatter_normalise<<<(unsigned)((m + 255) / 256), 256, 0, c->stream>>>(cube, c->nchan, nc, c->weights(), cells,
                                                                             scale);
    launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) { hcg_cuda_fail(e, "k_scatter"); return -1; }
    return launches;
}

// hcg_gather.cu -- dispatch of the CUDA-core gather (hcg_gather.cuh) by
// channel count and tuning, and the contributor-list export.
#include "hcg_gather.cuh"

using hcg_gather::GatherArgs;

namespace {
using namespace hcg_gather;

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

}  // namespace

// Kernel of the CUDA-core gather for this pass, from the tuning (0 = auto):
// cells per block 16 -> k_gather (per-slice search), 32 -> k_gather_list;
// channels per lane 1, 4 or 8; candidate rows in flight 8 or 12 (list kernel).
void gather_choice(const hcg_ctx *c, int nchan, int *cells, int *vc, int *depth) {
    int cl = c->e_cells, v = c->e_chans, d = c->e_depth;
    if (cl == 0) cl = (nchan >= 256 || (nchan >= 128 && v == 4 && d == 8)) ? 32 : 16;
    if (cl == 32) {
        if (v == 0) v = nchan >= 256 ? 8 : 4;
        if (d == 0) d = v == 8 ? 12 : 8;
    } else {
        if (v == 0) v = nchan >= 256 ? 8 : (nchan >= 4 ? 4 : 1);
        d = 0;
    }
    *cells = cl; *vc = v; *depth = d;
}

int launch_gather(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale) {
    GatherArgs a = make_args(c, gp, spec, scale);
    int cells, vc, depth;
    gather_choice(c, a.nchan, &cells, &vc, &depth);
    if (dtype == HCG_F32) return launch_gather_dt<float>(a, c->stream, cells, vc, depth);
    if (dtype == HCG_BF16) return launch_gather_dt<__nv_bfloat16>(a, c->stream, cells, vc, depth);
    return launch_gather_dt<__nv_fp8_storage_t>(a, c->stream, cells, vc, depth);
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

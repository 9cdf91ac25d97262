// hcg_gather_batch.cu -- the persistent CUDA-core launch of the batched form:
// many fields' (field, block of 4 groups, channel slice) work items taken
// from one queue.
#include "hcg_gather.cuh"

namespace hcg_gather {
namespace {
// ---- batched form ---------------------------------------------------------
// One persistent launch grids many fields: blocks (4 warps = 4 groups) take
// work items (field, block of 4 groups, channel slice) from a queue sorted by
// estimated cost, largest first, through an atomic counter; each item runs
// the same per-(group, slice) gather as k_gather, with the field's kernel
// layout chosen at run time.
enum GatherKind : int {
    GK_F32_8_32, GK_F32_4_32, GK_F32_4_16, GK_F32_4_4, GK_F32_4_1, GK_F32_1_1,
    GK_BF16_8_32, GK_BF16_4_32, GK_BF16_4_16, GK_BF16_4_4, GK_BF16_4_1, GK_BF16_1_1,
    GK_E4M3_8_32, GK_E4M3_4_32, GK_E4M3_4_16, GK_E4M3_4_4, GK_E4M3_4_1, GK_E4M3_1_1,
};

template <typename T, bool kProj>
HCG_DEV void dispatch_layout(int layout, const GatherArgs &a, int64_t grp, int slice, WarpSmem &sm) {
    switch (layout) {
        case 0: gather_group_slice<T, 8, 32, kProj>(a, grp, slice, sm); break;
        case 1: gather_group_slice<T, 4, 32, kProj>(a, grp, slice, sm); break;
        case 2: gather_group_slice<T, 4, 16, kProj>(a, grp, slice, sm); break;
        case 3: gather_group_slice<T, 4, 4, kProj>(a, grp, slice, sm); break;
        case 4: gather_group_slice<T, 4, 1, kProj>(a, grp, slice, sm); break;
        default: gather_group_slice<T, 1, 1, kProj>(a, grp, slice, sm); break;
    }
}

template <bool kProj>
__global__ void __launch_bounds__(kWarps * 32, 4) k_gather_batch(const GatherArgs *__restrict__ fields,
                                                               const int *__restrict__ kinds,
                                                               const uint64_t *__restrict__ items, int64_t nitems,
                                                               unsigned long long *head) {
    __shared__ WarpSmem smem[kWarps];
    __shared__ unsigned long long item_s;
    const int warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(head, 1ull);
        __syncthreads();
        const unsigned long long it = item_s;
        __syncthreads();
        if (it >= (unsigned long long)nitems) break;
        const uint64_t w = items[it];             // field (12 bits) | slice (16) | group block (36)
        const int f = (int)(w >> 52), slice = (int)((w >> 36) & 0xFFFF);
        const int64_t grp = (int64_t)(w & 0xFFFFFFFFFull) * kWarps + warp;
        const GatherArgs &a = fields[f];
        if (grp >= a.ngroups) continue;
        const int kind = kinds[f];
        if (kind < GK_BF16_8_32) dispatch_layout<float, kProj>(kind - GK_F32_8_32, a, grp, slice, smem[warp]);
        else if (kind < GK_E4M3_8_32)
            dispatch_layout<__nv_bfloat16, kProj>(kind - GK_BF16_8_32, a, grp, slice, smem[warp]);
        else dispatch_layout<__nv_fp8_storage_t, kProj>(kind - GK_E4M3_8_32, a, grp, slice, smem[warp]);
        __syncwarp();
    }
}

}  // namespace
}  // namespace hcg_gather

using hcg_gather::GatherArgs;

// Layout of a field in the batched kernel: (VC, LC) by channel count.
static int layout_for(int nchan) {
    if (nchan >= 256) return 0;
    if (nchan >= 128) return 1;
    if (nchan >= 64) return 2;
    if (nchan >= 16) return 3;
    if (nchan >= 4) return 4;
    return 5;
}
static const int kLayoutChans[6] = {256, 128, 64, 16, 4, 1};   // channels per slice

size_t gather_args_size() { return sizeof(GatherArgs); }

// Fills the field's kernel arguments; returns its kind and, through the
// pointers, its number of 4-group blocks and channel slices.
int gather_batch_field(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale,
                       void *args_out, int64_t *gblocks, int *nslices) {
    GatherArgs a = hcg_gather::make_args(c, gp, spec, scale);
    const int layout = layout_for(c->nchan);
    a.nslices = (c->nchan + kLayoutChans[layout] - 1) / kLayoutChans[layout];
    memcpy(args_out, &a, sizeof(a));
    *gblocks = (a.ngroups + hcg_gather::kWarps - 1) / hcg_gather::kWarps;
    *nslices = a.nslices;
    const int base = dtype == HCG_F32 ? hcg_gather::GK_F32_8_32
                                      : (dtype == HCG_BF16 ? hcg_gather::GK_BF16_8_32 : hcg_gather::GK_E4M3_8_32);
    return base + layout;
}

int launch_gather_batch(const void *fields, const int *kinds, const uint64_t *items, int64_t nitems,
                        unsigned long long *head, int nsm, cudaStream_t st, bool any_projected) {
    if (nitems <= 0) return 0;
    int per_sm = 0;
    auto kern = any_projected ? hcg_gather::k_gather_batch<true> : hcg_gather::k_gather_batch<false>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, hcg_gather::kWarps * 32, 0);
    int64_t blocks = std::min<int64_t>(nitems, (int64_t)std::max(1, per_sm) * nsm);
    kern<<<(unsigned)blocks, hcg_gather::kWarps * 32, 0, st>>>(static_cast<const GatherArgs *>(fields), kinds, items,
                                                               nitems, head);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { hcg_cuda_fail(e, "k_gather_batch"); return -1; }
    return 1;
}

// hcg_gather_bf16.cu -- the CUDA-core gather kernels (hcg_gather.cuh)
// instantiated for BF16 spectra; a unit per storage type keeps the build
// parallel.
#include "hcg_gather.cuh"

namespace hcg_gather {

template <>
int launch_gather_dt<__nv_bfloat16>(const GatherArgs &a, cudaStream_t st, int cells, int vc, int depth) {
    return launch_gather_body<__nv_bfloat16>(a, st, cells, vc, depth);
}

}  // namespace hcg_gather

// hcg_gather_e4m3.cu -- the CUDA-core gather kernels (hcg_gather.cuh)
// instantiated for FP8-e4m3 spectra; a unit per storage type keeps the build
// parallel.
#include "hcg_gather.cuh"

namespace hcg_gather {

template <>
int launch_gather_dt<__nv_fp8_storage_t>(const GatherArgs &a, cudaStream_t st, int cells, int vc, int depth) {
    return launch_gather_body<__nv_fp8_storage_t>(a, st, cells, vc, depth);
}

}  // namespace hcg_gather

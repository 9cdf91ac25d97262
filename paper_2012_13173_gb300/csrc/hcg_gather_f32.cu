// hcg_gather_f32.cu -- the CUDA-core gather kernels (hcg_gather.cuh)
// instantiated for FP32 spectra; a unit per storage type keeps the build
// parallel.
#include "hcg_gather.cuh"

namespace hcg_gather {

template <>
int launch_gather_dt<float>(const GatherArgs &a, cudaStream_t st, int cells, int vc, int depth) {
    return launch_gather_body<float>(a, st, cells, vc, depth);
}

}  // namespace hcg_gather

// hcg_tc.cu -- tensor-core (tcgen05) blocked gather for BF16 / FP8 storage.
#include "hcg_internal.h"

bool tc_supported(hcg_ctx *, int) { return false; }

int launch_tc_gather(hcg_ctx *, const GridParams &, const void *, int, const float *) {
    hcg_set_error("tensor path not available");
    return -1;
}

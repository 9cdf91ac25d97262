// hcg_batch.cu -- the batched form: many independent fields gridded on one
// stream.
#include <new>
#include <vector>

#include "hcg_internal.h"

struct hcg_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<hcg_ctx *> fields;
};

extern "C" {

hcg_status hcg_batch_create(hcg_batch **out, int device, void *stream) {
    if (!out) { hcg_set_error("null output pointer"); return HCG_ERR_INVALID_ARG; }
    hcg_batch *b = new (std::nothrow) hcg_batch();
    if (!b) { hcg_set_error("host allocation failed"); return HCG_ERR_OOM; }
    b->device = device;
    b->stream = (cudaStream_t)stream;
    *out = b;
    return HCG_OK;
}

hcg_status hcg_batch_destroy(hcg_batch *b) {
    delete b;
    return HCG_OK;
}

hcg_status hcg_batch_add(hcg_batch *b, hcg_ctx *f) {
    if (!b || !f) { hcg_set_error("null batch or field"); return HCG_ERR_INVALID_ARG; }
    if (f->device != b->device) { hcg_set_error("field on another device"); return HCG_ERR_INVALID_ARG; }
    b->fields.push_back(f);
    return HCG_OK;
}

hcg_status hcg_batch_grid(hcg_batch *b) {
    if (!b) { hcg_set_error("null batch"); return HCG_ERR_INVALID_ARG; }
    for (hcg_ctx *f : b->fields) {
        hcg_status s = hcg_set_stream(f, b->stream);
        if (s) return s;
        s = hcg_grid(f);
        if (s) return s;
    }
    return HCG_OK;
}

hcg_status hcg_batch_sync(hcg_batch *b) {
    if (!b) { hcg_set_error("null batch"); return HCG_ERR_INVALID_ARG; }
    for (hcg_ctx *f : b->fields) {
        hcg_status s = hcg_sync(f);
        if (s) return s;
    }
    return HCG_OK;
}

}  // extern "C"

// hcg_batch.cu -- the batched form: many independent fields (fields, beams or
// scans of uneven sample counts, channel counts and grid sizes) gridded by
// one captured CUDA graph.
//
// The graph holds, per field, the pre-ordering stages of hcg_grid (ingest,
// pixel keys, radix sort, S' data, both lookup tables) on one of several
// forked streams, so the small launches of different fields overlap; then,
// on the batch stream, ONE persistent CUDA-core gather launch over a work
// queue of (field, 4-group block, channel slice) items sorted by estimated
// cost, largest first, plus the launches of the fields that use the tensor
// path or the list kernel (256+ channels).  The first hcg_batch_grid builds
// and captures the graph; later
// calls replay it while every field's shapes, buffers and parameters are
// unchanged, and re-capture otherwise.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "hcg_internal.h"

namespace {
constexpr int kForks = 4;

struct FieldSig {               // what the captured graph depends on
    const void *ptrs[13];
    int64_t n;
    int32_t nchan, nx, ny, store, in_dtype, path;
    double params[6];
    int tuning[4];
    bool operator==(const FieldSig &o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

FieldSig signature(const hcg_ctx *c) {
    FieldSig s;
    memset(&s, 0, sizeof(s));
    const void *p[13] = {c->lon, c->lat, c->spec_in, c->scale_in, c->cube(), c->weights(), c->psorted,
                         c->sort.keys[0], c->upix, c->rstart, c->q_spec, c->sc_uv, c->rband};
    memcpy(s.ptrs, p, sizeof(p));
    s.n = c->n; s.nchan = c->nchan; s.nx = c->nx; s.ny = c->ny;
    s.store = c->store; s.in_dtype = c->in_dtype; s.path = c->last_path;
    double q[6] = {c->fwhm, c->support, c->lon0, c->lat0, c->pix, (double)c->nside};
    memcpy(s.params, q, sizeof(q));
    int t[4] = {c->t_cells, c->t_chans, c->t_depth, c->t_path};
    memcpy(s.tuning, t, sizeof(t));
    return s;
}
}  // namespace

struct hcg_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<hcg_ctx *> fields;
    // captured graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<FieldSig> sigs;
    cudaStream_t forks[kForks] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kForks] = {};
    // device-side work description
    void *d_args = nullptr; size_t d_args_cap = 0;
    int *d_kinds = nullptr; int64_t d_kinds_cap = 0;
    uint64_t *d_items = nullptr; int64_t d_items_cap = 0;
    unsigned long long *d_head = nullptr;
    int64_t nitems = 0;
    int nsm = 148;
    int launches = 0;
};

static hcg_status bfail(hcg_status s, const char *m) {
    hcg_set_error(m);
    return s;
}

static void drop_graph(hcg_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->sigs.clear();
}

// Fields that run their own gather launch inside the graph (after the
// queue): the tensor and staged paths, and the list kernel (one search per
// group for all channel slices, where a queue item searches once per slice).
static bool own_launch(const hcg_ctx *c) {
    if (c->last_path == HCG_PATH_TENSOR || c->last_path == HCG_PATH_STAGED) return true;
    int cells, vc, depth;
    gather_choice(c, c->nchan, &cells, &vc, &depth);
    return cells == 32;
}

// Host-side preparation of every field and the work queue; then capture.
static hcg_status build_graph(hcg_batch *b) {
    drop_graph(b);
    const size_t asz = gather_args_size();
    std::vector<unsigned char> args;
    std::vector<int> kinds;
    struct Item { uint64_t code; double cost; };
    std::vector<Item> items;
    std::vector<int> gfield(b->fields.size(), -1);
    for (size_t f = 0; f < b->fields.size(); f++) {
        hcg_ctx *c = b->fields[f];
        // (fields left on the automatic path take the tuner's cached choice)
        c->tables_src = nullptr;
        hcg_status s = grid_prepare(c);
        if (s) return s;
    }
    // fields with the same coordinates, kernel and grid as an earlier field
    // (the same sky positions stored in several types, or gridded with
    // several tunings) share that field's pre-ordering and tables: its S'
    // data depend on nothing else
    for (size_t f = 0; f < b->fields.size(); f++) {
        hcg_ctx *c = b->fields[f];
        if (c->last_path == HCG_PATH_SCATTER) continue;
        for (size_t e = 0; e < f; e++) {
            hcg_ctx *l = b->fields[e];
            if (l->tables_src || l->last_path == HCG_PATH_SCATTER) continue;
            if (l->lon == c->lon && l->lat == c->lat && l->n == c->n && l->key_bits == c->key_bits &&
                memcmp(&l->gp, &c->gp, sizeof(GridParams)) == 0) {
                c->tables_src = l;
                break;
            }
        }
    }
    // work items of the CUDA-core fields (field index, block of 4 groups, slice).
    // Fields of 256+ channels on the default layout run the list kernel on
    // their own (one search per group for all channel slices, where a queue
    // item searches once per slice), after the queue, like the tensor fields.
    for (size_t f = 0; f < b->fields.size(); f++) {
        hcg_ctx *c = b->fields[f];
        if (own_launch(c)) continue;
        const int dtype = c->store;
        const void *spec = c->store != c->in_dtype ? c->q_spec : c->spec_in;
        const float *scale = dtype == HCG_E4M3 ? (c->store != c->in_dtype ? c->q_scale : c->scale_in) : nullptr;
        const int gi = (int)kinds.size();
        if (gi >= 4096) return bfail(HCG_ERR_UNSUPPORTED, "more than 4096 CUDA-core fields in one batch");
        args.resize((size_t)(gi + 1) * asz);
        int64_t gblocks;
        int nsl;
        kinds.push_back(gather_batch_field(c, c->gp, spec, dtype, scale, args.data() + (size_t)gi * asz, &gblocks,
                                           &nsl));
        gfield[f] = gi;
        // cost of one item ~ candidates per group x channels per slice + the search
        const double deg = 3.14159265358979323846 / 180.0;
        const double area = std::max(1e-9, (c->nx * c->pix + 2 * c->support) * (c->ny * c->pix + 2 * c->support) *
                                               std::max(0.05, cos(std::min(89.0, fabs(c->lat0)) * deg)));
        const double cand = (double)c->n / area *
                            (3.14159265358979323846 * c->support * c->support + 4 * c->support * c->pix +
                             c->pix * c->pix);
        const double chans = (double)std::min<int64_t>(c->nchan, (c->nchan + nsl - 1) / nsl);
        const double cost = cand * (8.0 + chans / 8.0);
        if (gblocks >= ((int64_t)1 << 36) || nsl >= 65536) return bfail(HCG_ERR_UNSUPPORTED, "field too large");
        for (int sl = 0; sl < nsl; sl++)
            for (int64_t gb = 0; gb < gblocks; gb++)
                items.push_back({((uint64_t)gi << 52) | ((uint64_t)sl << 36) | (uint64_t)gb, cost});
    }
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
    b->nitems = (int64_t)items.size();
    // device copies of the queue (outside any capture)
    if (!kinds.empty()) {
        if (args.size() > b->d_args_cap) {
            if (b->d_args) cudaFree(b->d_args);
            b->d_args = nullptr; b->d_args_cap = 0;
            if (cudaMalloc(&b->d_args, args.size()) != cudaSuccess) { cudaGetLastError(); return bfail(HCG_ERR_OOM, "batch args"); }
            b->d_args_cap = args.size();
        }
        if ((int64_t)kinds.size() > b->d_kinds_cap) {
            if (b->d_kinds) cudaFree(b->d_kinds);
            b->d_kinds = nullptr; b->d_kinds_cap = 0;
            if (cudaMalloc((void **)&b->d_kinds, kinds.size() * sizeof(int)) != cudaSuccess) { cudaGetLastError(); return bfail(HCG_ERR_OOM, "batch kinds"); }
            b->d_kinds_cap = (int64_t)kinds.size();
        }
        if (b->nitems > b->d_items_cap) {
            if (b->d_items) cudaFree(b->d_items);
            b->d_items = nullptr; b->d_items_cap = 0;
            if (cudaMalloc((void **)&b->d_items, b->nitems * sizeof(uint64_t)) != cudaSuccess) { cudaGetLastError(); return bfail(HCG_ERR_OOM, "batch items"); }
            b->d_items_cap = b->nitems;
        }
        std::vector<uint64_t> codes(items.size());
        for (size_t k = 0; k < items.size(); k++) codes[k] = items[k].code;
        if (cudaMemcpy(b->d_args, args.data(), args.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b->d_kinds, kinds.data(), kinds.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b->d_items, codes.data(), codes.size() * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess)
            return bfail(HCG_ERR_CUDA, "batch queue upload failed");
    }
    // capture
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaStreamBeginCapture");
    hcg_status st = HCG_OK;
    int launches = 0;
    cudaEventRecord(b->ev_fork, b->stream);
    for (int k = 0; k < kForks; k++) cudaStreamWaitEvent(b->forks[k], b->ev_fork, 0);
    std::vector<const void *> fspec(b->fields.size());
    std::vector<int> fdt(b->fields.size());
    std::vector<const float *> fsc(b->fields.size());
    for (size_t f = 0; f < b->fields.size() && !st; f++) {
        hcg_ctx *c = b->fields[f];
        c->stream = b->forks[f % kForks];
        st = grid_enqueue_front(c, &fspec[f], &fdt[f], &fsc[f]);
        launches += c->last_launches;
    }
    for (int k = 0; k < kForks; k++) {
        cudaEventRecord(b->ev_join[k], b->forks[k]);
        cudaStreamWaitEvent(b->stream, b->ev_join[k], 0);
    }
    if (!st && b->nitems > 0) {
        cudaMemsetAsync(b->d_head, 0, sizeof(unsigned long long), b->stream);
        bool any_projected = false;
        for (hcg_ctx *c : b->fields) any_projected |= c->cell_lon != nullptr;
        int k = launch_gather_batch(b->d_args, b->d_kinds, b->d_items, b->nitems, b->d_head, b->nsm, b->stream,
                                    any_projected);
        if (k < 0) st = HCG_ERR_CUDA;
        else launches += k;
    }
    for (size_t f = 0; f < b->fields.size() && !st; f++) {
        hcg_ctx *c = b->fields[f];
        c->stream = b->stream;
        if (own_launch(c)) {
            st = grid_enqueue_gather(c, fspec[f], fdt[f], fsc[f]);
            launches += 1;
        } else {
            c->gridded = true;
        }
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->stream, &g);
    if (st) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaStreamEndCapture");
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) { drop_graph(b); return hcg_cuda_fail(e, "cudaGraphInstantiate"); }
    b->launches = launches;
    for (hcg_ctx *c : b->fields) b->sigs.push_back(signature(c));
    return HCG_OK;
}

extern "C" {

hcg_status hcg_batch_create(hcg_batch **out, int device, void *stream) {
    if (!out) return bfail(HCG_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    if (!stream) return bfail(HCG_ERR_INVALID_ARG, "the batch needs a non-default stream (graph capture)");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaSetDevice");
    hcg_batch *b = new (std::nothrow) hcg_batch();
    if (!b) return bfail(HCG_ERR_OOM, "host allocation failed");
    b->device = device;
    b->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, device);
    bool ok = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc((void **)&b->d_head, sizeof(unsigned long long)) == cudaSuccess;
    for (int k = 0; k < kForks && ok; k++)
        ok = cudaStreamCreateWithFlags(&b->forks[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        hcg_batch_destroy(b);
        return bfail(HCG_ERR_CUDA, "batch stream/event/counter creation failed");
    }
    *out = b;
    return HCG_OK;
}

hcg_status hcg_batch_destroy(hcg_batch *b) {
    if (!b) return HCG_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto s : b->forks) if (s) cudaStreamDestroy(s);
    for (auto e : b->ev_join) if (e) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    void *p[] = {b->d_args, b->d_kinds, b->d_items, b->d_head};
    for (void *q : p) if (q) cudaFree(q);
    for (hcg_ctx *c : b->fields) c->stream = b->stream;
    delete b;
    return HCG_OK;
}

hcg_status hcg_batch_add(hcg_batch *b, hcg_ctx *f) {
    if (!b || !f) return bfail(HCG_ERR_INVALID_ARG, "null batch or field");
    if (f->device != b->device) return bfail(HCG_ERR_INVALID_ARG, "field on another device");
    for (hcg_ctx *c : b->fields)
        if (c == f) return bfail(HCG_ERR_INVALID_ARG, "field already in the batch");
    b->fields.push_back(f);
    drop_graph(b);
    return HCG_OK;
}

hcg_status hcg_batch_grid(hcg_batch *b) {
    if (!b) return bfail(HCG_ERR_INVALID_ARG, "null batch");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaSetDevice");
    for (hcg_ctx *c : b->fields) {
        if (c->host_spec) return bfail(HCG_ERR_UNSUPPORTED, "a batched field needs device-resident spectra");
        if (c->t_path == HCG_PATH_SCATTER) return bfail(HCG_ERR_UNSUPPORTED, "the scatter path is not batched");
    }
    bool same = b->exec && b->sigs.size() == b->fields.size();
    for (size_t f = 0; same && f < b->fields.size(); f++) same = b->sigs[f] == signature(b->fields[f]);
    if (!same) {
        hcg_status s = build_graph(b);
        if (s) return s;
    }
    e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaGraphLaunch");
    for (hcg_ctx *c : b->fields) c->gridded = true;
    return HCG_OK;
}

hcg_status hcg_batch_sync(hcg_batch *b) {
    if (!b) return bfail(HCG_ERR_INVALID_ARG, "null batch");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaSetDevice");
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return hcg_cuda_fail(e, "stream synchronise");
    for (hcg_ctx *f : b->fields) {
        hcg_status s = hcg_sync(f);
        if (s) return s;
    }
    return HCG_OK;
}

hcg_status hcg_batch_info(hcg_batch *b, int64_t *work_items, int32_t *launches) {
    if (!b) return bfail(HCG_ERR_INVALID_ARG, "null batch");
    if (work_items) *work_items = b->nitems;
    if (launches) *launches = b->launches;
    return HCG_OK;
}

}  // extern "C"

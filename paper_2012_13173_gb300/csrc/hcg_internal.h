// hcg_internal.h -- host-side context and kernel launch declarations shared by
// the library's translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/hcgrid.h"

// Device error word bits (OR-ed by kernels, read by synchronising calls).
enum : int {
    HCG_DERR_BAD_COORD = 1,     // non-finite coordinate or |lat| > 90
    HCG_DERR_SEGMENTS = 2,      // more candidate segments than a warp buffer holds
    HCG_DERR_TIMEOUT = 4,       // a bounded wait gave up
    HCG_DERR_NONFINITE = 8      // non-finite spectra seen by the quantiser
};

// Everything a kernel needs about the grid and the kernel; passed by value
// (kernel parameter space), the analogue of the paper's constant-memory
// gridding parameters (Sec. 3.5 II item 3).
struct GridParams {
    double lon0, lat0, pix;     // grid centre and cell size, degrees
    double hx, hy;              // (nx-1)/2, (ny-1)/2
    double R_deg;               // support radius, degrees
    double hR;                  // sin^2(R/2), from the host libm
    int32_t nx, ny;
    int64_t nside;
    int64_t r_lo, r_hi;         // rings the grid can reach
    int64_t pix_lo;             // first pixel of ring r_lo
    float R2;                   // R^2 (radians^2)
    float band_lo, band_hi;     // R^2 (1 -+ 1e-5): exact FP64 test in between
    float kexp;                 // log2(e) / (2 sigma^2), radians^-2
    float sinR;                 // sin(R)
    float R_radf;
    float havRf;                // sin^2(R/2) rounded up to FP32 (per-ring chord bound)
    const double *clon, *clat;  // projected grids: cell centres [ny][nx] (degrees, device); null for HCG_CAR
    double screen_eps;          // margin of the FP32 pixel screen (0: FP64 only)
};

struct SortScratch {
    uint64_t *keys[2] = {nullptr, nullptr};
    uint32_t *vals[2] = {nullptr, nullptr};
    uint32_t *counts = nullptr;     // [256 * ntiles]
    int64_t cap = 0, count_cap = 0;
    // one-sweep sort: per (tile, digit) look-back status words [ntiles * 256]
    // (zeroed once when allocated), and per sort: digit counts [8][256],
    // global digit offsets [8][256], tile counters [8], the sort epoch
    uint64_t *status = nullptr;
    uint32_t *hist = nullptr;       // [kSortHistWords]
};
constexpr int kSortHistWords = 8 * 256 * 2 + 8 + 8;

struct ScanScratch {
    std::vector<uint32_t *> level;  // block sums per recursion level
    std::vector<int64_t> level_cap;
};

struct hcg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;

    // allocation cap (hcg_set_alloc_cap): bytes of field-sized device buffers
    // (those grown by grow / grow_bytes) the context may hold, 0 = no cap;
    // alloc_live maps each such buffer to its size
    int64_t alloc_cap = 0;
    int64_t alloc_bytes = 0;
    std::unordered_map<const void *, size_t> alloc_live;

    // kernel
    bool kernel_set = false;
    double fwhm = 0, support = 0;
    int64_t nside = 0;

    // grid
    bool grid_set = false;
    double lon0 = 0, lat0 = 0, pix = 0;
    int32_t nx = 0, ny = 0;
    int proj = HCG_CAR;
    double *cell_lon = nullptr, *cell_lat = nullptr;   // projected grids: device cell centres
    double cell_latmin = 0, cell_latmax = 0;           // their latitude extent

    // storage
    int store = HCG_F32;

    // samples
    bool loaded = false;
    int64_t n = 0;
    int32_t nchan = 0;
    int in_dtype = HCG_F32;
    const double *lon = nullptr, *lat = nullptr;    // device (owned or borrowed)
    const void *spec_in = nullptr;                  // device, input dtype
    const float *scale_in = nullptr;                // device, E4M3 input scales
    double *own_lon = nullptr, *own_lat = nullptr;
    void *own_spec = nullptr; size_t own_spec_bytes = 0;
    float *own_scale = nullptr;
    int64_t own_coord_cap = 0; int32_t own_scale_cap = 0;

    // quantised storage (when store != input dtype)
    void *q_spec = nullptr; size_t q_spec_bytes = 0;
    float *q_scale = nullptr; int32_t q_scale_cap = 0;
    uint32_t *q_amax = nullptr;

    // derived per grid() call
    GridParams gp{};
    int key_bits = 0;

    // scratch
    SortScratch sort;
    ScanScratch scan;
    int64_t *psorted = nullptr;     // P' [N]
    float4 *sc_uv = nullptr;        // per sorted sample: u_hi, u_lo, v_hi, v_lo (radians)
    float *sc_cos = nullptr;        // cos(lat) per sorted sample
    uint32_t *sc_row = nullptr;     // input index per sorted sample
    uint32_t *flags = nullptr;      // [N] unique-pixel flags / positions
    int64_t *upix = nullptr, *ustart = nullptr;     // LUT1 [N], [N+1]
    int64_t *rstart = nullptr, *rustart = nullptr;  // LUT2 [rings+1]
    float4 *rband = nullptr;                         // per ring: latitude band of its samples [rings+1]
    int64_t sample_cap = 0, ring_cap = 0;
    int num_sms = 148;
    int64_t *dscal = nullptr;       // device scalars: [0] U_total, [1] pairs, [2] tensor flops, [3..] spare
    int *derr = nullptr;            // device error word

    // outputs
    float *own_cube = nullptr, *own_w = nullptr;
    size_t own_cube_cap = 0, own_w_cap = 0;
    float *bound_cube = nullptr, *bound_w = nullptr;
    bool gridded = false;

    // stage timers
    static constexpr int kProfSlots = 64;
    bool profiling = false;
    int prof_calls = 0;                         // hcg_grid calls since profiling was enabled
    cudaEvent_t ev[kProfSlots][6] = {};

    // bounded device waits (hcg_set_wait_limit)
    int64_t wait_ns = 4000000000ll;
    int wait_probe = 0;

    // tuning
    int t_cells = 0, t_chans = 0, t_depth = 0, t_path = HCG_PATH_AUTO;   // as set (0 = automatic)
    int e_cells = 0, e_chans = 0, e_depth = 0;      // in effect for the pass (grid_prepare)
    std::vector<int32_t> tune_table;                // last autotune: 4 values per candidate
    std::vector<float> tune_ms;                     //                its mean pass time (ms; < 0: failed)
    int last_path = HCG_PATH_GATHER;
    int last_launches = 0;

    // streamed spectra (HCG_MEM_HOST_STREAM): the caller's host rows are
    // copied in channel windows during hcg_grid, each window's copy (on
    // copy_stream) overlapping the gather of the window before it
    const void *host_spec = nullptr;                // host [n][nchan], input dtype
    int32_t stream_chunk = 0;                       // channels per window (0: automatic)
    void *stage[2] = {nullptr, nullptr};            // device windows, input dtype
    size_t stage_cap[2] = {0, 0};
    void *qstage[2] = {nullptr, nullptr};           // device windows, storage dtype (quantised)
    size_t qstage_cap[2] = {0, 0};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {}, ev_consumed[2] = {};
    int32_t win_c0 = 0, win_nc = 0;                 // channel window of the gather being enqueued

    // host outputs (hcg_bind_host_output): each gathered window's cube slice
    // is copied back on out_stream while the next window is in flight
    float *host_cube = nullptr, *host_w = nullptr;
    cudaStream_t out_stream = nullptr;
    cudaEvent_t ev_gathered[2] = {}, ev_out_done = nullptr;

    // batched passes: a field whose coordinates, kernel and grid equal an
    // earlier field's reads that field's S' data and tables instead of
    // building its own (hcg_batch.cu sets it; hcg_grid clears it)
    hcg_ctx *tables_src = nullptr;
    const hcg_ctx *tables() const { return tables_src ? tables_src : this; }

    float *cube() const { return bound_cube ? bound_cube : own_cube; }
    float *weights() const { return bound_w ? bound_w : own_w; }
    int32_t win_channels() const { return win_nc ? win_nc : nchan; }
    int32_t stream_win = 0;                         // channels per streamed window of this pass
    int32_t stream_chunk_chans() const { return stream_win ? stream_win : nchan; }
};

// ---- helpers implemented in hcg_api.cu
void hcg_set_error(const std::string &msg);
hcg_status hcg_cuda_fail(cudaError_t e, const char *what);
// INVALID_ARG (with a message naming `what`) unless p is device or managed
// memory that device `device` can address; a null p passes.
hcg_status check_device_ptr(const void *p, int device, const char *what);

// ---- launchers (each returns the number of kernels it launched, or < 0 on a
//      launch error after recording the message)
int launch_prep(hcg_ctx *c, const GridParams &gp, int key_bits);
int launch_sort(hcg_ctx *c, int64_t n, int key_bits);
int launch_scan_u32(hcg_ctx *c, uint32_t *data, int64_t n);   // exclusive, in place
int launch_permute_lut(hcg_ctx *c, const GridParams &gp);
int launch_quantise(hcg_ctx *c);
int launch_quantise_span(hcg_ctx *c, const float *x, int64_t n, int32_t nchan, void *q, float *q_scale,
                         uint32_t *q_amax);
int launch_gather(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale);
void gather_choice(const hcg_ctx *c, int nchan, int *cells, int *vc, int *depth);
int launch_tc_gather(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale);
int launch_scatter(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale);
int launch_debug_neigh(hcg_ctx *c, const GridParams &gp, int64_t cell_begin, int64_t cell_end,
                       int64_t *d_counts, const int64_t *d_offsets, uint32_t *d_ids, int pass);
bool tc_supported(hcg_ctx *c, int dtype);
// Staged CUDA-core gather (hcg_staged.cu): tiles of `cells` cells (32, 64 or
// 128) and chunks of `depth` candidates (16 or 32).
bool staged_supported(const hcg_ctx *c, int dtype, int32_t win_nchan);
int launch_staged(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale, int cells,
                  int depth);

// sizes of scratch needed by the sort / scan for n keys
int64_t sort_tiles(int64_t n);

// Pre-ordering (pixel keys + radix sort) on explicit buffers; see hcg_prep.cu.
int preorder_on_buffers(const double *lon, const double *lat, int64_t n, const GridParams &gp, int key_bits,
                        uint64_t *const k[2], uint32_t *const v[2], int first, uint32_t *counts, uint32_t *sums,
                        int *err, cudaStream_t st);

// Batched gather (hcg_gather.cu): per-field argument blocks and one persistent launch.
size_t gather_args_size();
int gather_batch_field(hcg_ctx *c, const GridParams &gp, const void *spec, int dtype, const float *scale,
                       void *args_out, int64_t *gblocks, int *nslices);
int launch_gather_batch(const void *fields, const int *kinds, const uint64_t *items, int64_t nitems,
                        unsigned long long *head, int nsm, cudaStream_t st,
                        bool any_projected);

// Stages of hcg_grid (hcg_api.cu), reused by the batched form.
hcg_status grid_prepare(hcg_ctx *c);                  // parameters, scratch, path (host; may allocate)
hcg_status grid_enqueue_front(hcg_ctx *c, const void **spec, int *dtype, const float **scale);
hcg_status grid_enqueue_gather(hcg_ctx *c, const void *spec, int dtype, const float *scale);
int launch_pass_gather(hcg_ctx *c, const void *spec, int dtype, const float *scale);
// The tuner's cached choice for this field's key, if any: {cells, chans, depth, path}.
bool autotune_cached(const hcg_ctx *c, int out[4]);
hcg_status grid_enqueue_streamed(hcg_ctx *c);
int wcs_cell_centres(int proj, double lon0, double lat0, double pix, int nx, int ny, double *lon, double *lat);
int32_t pick_stream_window(hcg_ctx *c);
hcg_status enqueue_host_output(hcg_ctx *c, int32_t c0, int32_t nc, int slot, bool weights);


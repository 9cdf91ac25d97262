/*
 * hcgrid.h -- C ABI of the GB300 gridding library (libhcgrid.so).
 *
 * Convolution-based gridding of non-uniformly sampled single-dish spectra onto
 * a regular sky grid, following HCGrid (Wang, Yu, Zhang, Xiao & Luo 2020,
 * MNRAS; arXiv 2012.13173).  Each output cell g receives Eq. (1) of Sec. 2.1:
 *
 *     V[g] = (1 / W_g) * sum_n V[s_n] w(g; s_n),   W_g = sum_n w(g; s_n),
 *
 * over the samples n within the kernel support.  The samples are pre-ordered
 * by HEALPix RING pixel (Sec. 3.2, Sec. 3.3 step I), indexed by a first-level
 * table pixel -> first sample (Sec. 3.3 step II) and a second-level table
 * ring -> first sample (Sec. 3.3 step III), and each cell gathers its
 * contributors ring by ring through those tables (Sec. 3.4).  Everything
 * after the inputs reach the device -- pixel indices, the sort, both tables,
 * the search and the convolution -- runs in this library's CUDA kernels.
 *
 * General rules
 *  - Every call returns hcg_status: HCG_OK (0) or a negative code.  No C++
 *    exception crosses this boundary.  hcg_last_error() returns a
 *    thread-local, NUL-terminated description of the last failure.
 *  - All pointers are plain host or device addresses; "mem" arguments say
 *    which (HCG_MEM_HOST or HCG_MEM_DEVICE).  Sizes are element counts.
 *  - A context is bound to one CUDA device and one stream.  Calls that only
 *    enqueue work (hcg_grid) return before the GPU finishes; hcg_fetch and
 *    hcg_sync wait.  A context must not be used from two threads at once.
 *  - Errors found on the device (bad coordinates, a bounded wait that ran
 *    out) are reported by the next call that synchronises.
 *  - Angles are degrees.  The grid is cell-major: cube[j][i][c] with
 *    j in [0, ny) (latitude), i in [0, nx) (longitude), c in [0, nchan).
 */
#ifndef HCGRID_H
#define HCGRID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hcg_status;

enum {
    HCG_OK = 0,
    HCG_ERR_INVALID_ARG = -1,   /* an argument is out of range or inconsistent */
    HCG_ERR_OOM = -2,           /* device allocation failed */
    HCG_ERR_CUDA = -3,          /* a CUDA runtime/driver call failed */
    HCG_ERR_NOT_READY = -4,     /* a required setter has not been called */
    HCG_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up */
    HCG_ERR_STATE = -6,         /* call not valid in the current state */
    HCG_ERR_UNSUPPORTED = -7    /* a valid request this build does not handle */
};

enum {                          /* grid projections (hcg_set_grid) */
    HCG_CAR = 0,                /* plain lon/lat grid, equal steps in degrees */
    HCG_WCS_TAN = 1,            /* gnomonic, reference point (lon0, lat0) at the grid centre */
    HCG_WCS_SIN = 2,            /* orthographic (cells within 1 rad of the reference point) */
    HCG_WCS_SFL = 3,            /* Sanson-Flamsteed */
    HCG_WCS_CAR = 4,            /* FITS plate carree: oblique when lat0 != 0 */
    HCG_CELL_LIST = 5           /* a free list of cell centres (hcg_set_cell_list) */
};

enum {                          /* spectra element types */
    HCG_F32 = 0,
    HCG_BF16 = 1,
    HCG_E4M3 = 2                /* FP8 e4m3 ("fn": bias 7, max 448) with per-channel FP32 scale */
};

enum {
    HCG_MEM_HOST = 0,           /* host memory (pinned or pageable) */
    HCG_MEM_DEVICE = 1,         /* device memory; the library copies it */
    HCG_MEM_DEVICE_BORROW = 2,  /* device memory used in place (hcg_load_samples only):
                                   the caller keeps it alive and unchanged until the
                                   next hcg_load_samples or hcg_destroy */
    HCG_MEM_HOST_STREAM = 3     /* host spectra streamed (hcg_load_samples only): the
                                   coordinates are copied at once; the spectra stay in
                                   host memory and each hcg_grid copies them window by
                                   window of channels (hcg_set_stream_chunk), every
                                   copy overlapping the gather of the window before it.
                                   The device holds two windows, not the spectra, so
                                   spectra larger than device memory can be gridded.
                                   The caller keeps the host spectra alive and
                                   unchanged until that work has completed (hcg_sync,
                                   hcg_fetch); pinned memory lets the copies run
                                   asynchronously.  Not for hcg_autotune or batches. */
};

enum {
    HCG_PATH_AUTO = 0,          /* choose by channel count and storage type */
    HCG_PATH_GATHER = 1,        /* CUDA-core gather, a warp per 2 x 2 group of cells (any
                                   storage type, any grid) */
    HCG_PATH_TENSOR = 2,        /* tcgen05 blocked path (BF16 / E4M3 storage) */
    HCG_PATH_SCATTER = 3,       /* Sec. 2.2 scatter with atomic adds, no pre-ordering or
                                   tables (a comparison path: never chosen automatically;
                                   sums in hardware order, so results vary in the last
                                   bits; the hcg_debug_* exports need a gather path) */
    HCG_PATH_STAGED = 4         /* CUDA-core gather over tiles of 32 or 64 cells whose
                                   candidates' spectrum rows are staged in shared memory
                                   by bulk asynchronous copies (any storage type; HCG_CAR
                                   grids, 128+ channels in rows of whole 16-byte units) */
};

typedef struct hcg_ctx hcg_ctx;
typedef struct hcg_batch hcg_batch;

/* Facts about the last hcg_grid of a context (for tests and benchmarks). */
typedef struct {
    int64_t nside;              /* HEALPix resolution chosen by hcg_set_kernel */
    int64_t ring_lo, ring_hi;   /* rings the grid can reach (samples elsewhere are dropped) */
    int64_t samples_kept;       /* M: samples whose ring lies in [ring_lo, ring_hi] */
    int64_t unique_pixels;      /* U: distinct pixels among them */
    int64_t pairs;              /* (cell, sample) pairs inside the support */
    int64_t contributions;      /* pairs * nchan: the gridded sample-channel contributions */
    int32_t path;               /* HCG_PATH_GATHER, HCG_PATH_TENSOR or HCG_PATH_SCATTER */
    int32_t key_bits;           /* bits of the radix-sort key */
    int32_t launches;           /* kernels launched by the last hcg_grid */
    int32_t stream_window;      /* channels per streamed window (0: spectra on the device) */
    int64_t tensor_flops;       /* tensor-core work issued by the last hcg_grid: 2 M N K summed over
                                   its MMA instructions (dense blocks, zero weights included;
                                   0 on the CUDA-core paths) */
} hcg_info;

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle, owned by the caller until hcg_destroy. */
hcg_status hcg_create(hcg_ctx **out, int device, void *cuda_stream);

/* Free the context and every device buffer it owns.  NULL is accepted. */
hcg_status hcg_destroy(hcg_ctx *ctx);

/* Change the stream later calls enqueue on. */
hcg_status hcg_set_stream(hcg_ctx *ctx, void *cuda_stream);

/* Gaussian kernel (Sec. 3.6 item 3): w = exp(-d^2 / (2 sigma^2)),
 * sigma = fwhm / (2 sqrt(2 ln 2)), applied within great-circle distance
 * support_radius_deg ("sphere_radius", the range of influence; the paper
 * advises 3-5 sigma).  The HEALPix resolution follows the paper's rule
 * "hpx_max_resolution ~ sigma_kernel / 2": the smallest power-of-two nside
 * with sqrt(pi/3)/nside <= sigma/2.
 * INVALID_ARG unless 1 arcsec <= fwhm, 0 < support_radius <= 1 degree, and
 * support_radius <= 10 sigma (both finite). */
hcg_status hcg_set_kernel(hcg_ctx *ctx, double fwhm_deg, double support_radius_deg);

/* Target grid (Sec. 2.1, "regular grid with I x J cells").  HCG_CAR: cell
 * (i, j) is centred at lon0 + (i - (nx-1)/2) * pixel, lat0 + (j - (ny-1)/2) *
 * pixel.  HCG_WCS_*: FITS world coordinates (Calabretta & Greisen 2002) with
 * the reference point (lon0, lat0) at the grid centre, x = (i - (nx-1)/2) *
 * pixel eastward and y = (j - (ny-1)/2) * pixel northward: TAN and SIN place
 * a cell at distance atan / asin |(x, y)| (radians) and bearing atan2(x, y)
 * from the reference point; CAR and SFL at native (x, y) and (x / cos y, y)
 * on the frame whose equator leaves the reference point due east.  The
 * centres are computed once here.  The tensor and scatter paths take HCG_CAR
 * grids only.  INVALID_ARG if the projection is unknown, nx, ny < 1, pixel
 * <= 0, pixel or centre not finite, nx*pixel > 180, a cell the projection
 * cannot place or a cell latitude beyond +-89 degrees, or more than 90 degrees
 * of longitude between a cell and lon0.  (hcg_grid returns INVALID_ARG when
 * nx*ny*nchan exceeds 4e18 elements.) */
hcg_status hcg_set_grid(hcg_ctx *ctx, int projection, double lon0_deg, double lat0_deg,
                        double pixel_deg, int32_t nx, int32_t ny);

/* Target cells as a free list (Sec. 2.1: the target is a set of cells with
 * centres (alpha_ij, delta_ij); here any positions, e.g. sight-lines or a
 * survey's pointing centres): ncells centres lon_deg[k], lat_deg[k] (FP64,
 * host or device memory per `mem`, copied now).  The result is then cube
 * [ncells][nchan] and weights [ncells] -- a grid of nx = ncells, ny = 1 --
 * on the CUDA-core gather path (HCG_PATH_GATHER; the other paths return
 * UNSUPPORTED).  Consecutive entries are searched together, so a list in sky
 * order grids faster; any order gives the same contributors per cell.
 * Replaces an earlier hcg_set_grid.  INVALID_ARG: ncells < 1 or above
 * 2^31 - 1, null pointers, unknown mem, a device pointer that is not device
 * memory of the context's device, a non-finite centre, a latitude beyond
 * +-89 degrees, or cells more than 90 degrees of longitude from the mean
 * longitude of the list. */
hcg_status hcg_set_cell_list(hcg_ctx *ctx, const double *lon_deg, const double *lat_deg, int64_t ncells, int mem);

/* How the library stores spectra (default HCG_F32).  With F32 input and
 * BF16/E4M3 storage, hcg_grid quantises on the device (round to nearest
 * even; E4M3 with per-channel scale amax/448). */
hcg_status hcg_set_storage(hcg_ctx *ctx, int dtype);

/* Samples (Sec. 2.1: coordinates (alpha_n, delta_n) and values V[s_n]).
 * lon_deg, lat_deg: n FP64 values.  spectra: [n][nchan] row-major of type
 * `dtype`; chan_scale: nchan FP32 scales, required for E4M3 input and
 * ignored otherwise.  mem: HCG_MEM_HOST / HCG_MEM_DEVICE (copied, the caller
 * keeps ownership), HCG_MEM_DEVICE_BORROW (used in place) or
 * HCG_MEM_HOST_STREAM (all host pointers; coordinates and scales copied now,
 * spectra window by window during each hcg_grid).  Coordinates
 * are validated on the device by hcg_grid (non-finite or |lat| > 90 gives
 * INVALID_ARG at the next synchronising call).  n may be 0.
 * INVALID_ARG: n < 0 or above 2^32 - 1, nchan < 1, n * nchan above 4e18,
 * null pointers with n > 0, dtype or mem unknown, E4M3 without scales,
 * borrowed spectra not 16-byte aligned (or borrowed coordinates not 8-byte
 * aligned), HCG_MEM_DEVICE* pointers that are not device memory of the
 * context's device, or a dtype/storage pair other than equal types or F32
 * input with BF16/E4M3 storage. */
hcg_status hcg_load_samples(hcg_ctx *ctx, const double *lon_deg, const double *lat_deg,
                            const void *spectra, int64_t n, int32_t nchan, int dtype,
                            const float *chan_scale, int mem);

/* Channels per streamed window (HCG_MEM_HOST_STREAM): 0 = automatic (all
 * channels up to 512; else two windows of half the channels in whole
 * 256-channel slices, narrower only while two windows would take more than a
 * quarter of the free device memory); otherwise the given count (the last
 * window takes the rest).  The tensor path needs windows of whole 256-channel slices.  Results
 * equal those of device-resident spectra bit for bit on the CUDA-core path
 * when every window has at least 128 channels (each channel accumulates in
 * the same order), and on the tensor path when the windows keep its slice
 * width (512 channels for fields whose channel count is a multiple of 512,
 * else 256).  INVALID_ARG: chans < 0. */
hcg_status hcg_set_stream_chunk(hcg_ctx *ctx, int32_t chans);

/* Let hcg_grid write the cube [ny][nx][nchan] and weights [ny][nx] (FP32,
 * device memory) straight into caller buffers instead of library-owned ones.
 * NULL, NULL returns to library-owned outputs.  INVALID_ARG: only one of the
 * two given, or the cube not 16-byte aligned (it is written with 16-byte
 * vector stores). */
hcg_status hcg_bind_output(hcg_ctx *ctx, float *cube_dev, float *weights_dev);

/* Also deliver each hcg_grid's result to host buffers: cube [ny][nx][nchan]
 * and weights [ny][nx] (FP32, pinned for asynchronous copies).  hcg_grid
 * then enqueues the device-to-host copies itself, window by window of
 * channels when the spectra are streamed (HCG_MEM_HOST_STREAM), so that they
 * overlap the copy and gather of the next window; hcg_sync waits for them.
 * The caller keeps the buffers alive until then.  The device-side result
 * stays available to hcg_fetch.  NULL, NULL stops the delivery.
 * INVALID_ARG: only one of the two given. */
hcg_status hcg_bind_host_output(hcg_ctx *ctx, float *cube_host, float *weights_host);

/* Run the whole path on the context's stream: ingest (quantise if asked),
 * HEALPix pixel of every sample, radix sort, both lookup tables, the
 * table-driven gather of Eq. (1) and the normalisation.  Enqueue only.
 * Empty cells (W = 0) get V = NaN, weight 0. */
hcg_status hcg_grid(hcg_ctx *ctx);

/* Wait for the context's work (its stream, and the copy streams of streamed
 * spectra and host outputs) and report device-side errors. */
hcg_status hcg_sync(hcg_ctx *ctx);

/* Copy the last result out (cube [ny][nx][nchan] FP32, weights [ny][nx]
 * FP32; either may be NULL) to host or device memory; synchronises. */
hcg_status hcg_fetch(hcg_ctx *ctx, float *cube, float *weights, int mem);

/* Facts about the last hcg_grid; synchronises. */
hcg_status hcg_get_info(hcg_ctx *ctx, hcg_info *out);

/* Give-up limit of the bounded device-side waits (the tensor path's
 * mbarrier waits), in nanoseconds of GPU global time; the default is 4e9.
 * A wait that runs out raises a device error bit, the CTA stops issuing
 * tensor-core work and finishes, and the next synchronising call returns
 * HCG_ERR_TIMEOUT; the context stays usable.  probe != 0 makes every
 * tensor-path CTA of later passes first wait on a barrier that nothing
 * completes -- a check of the give-up path: such a pass always returns
 * HCG_ERR_TIMEOUT and its cube is undefined.  probe = 0 restores normal
 * passes.  INVALID_ARG unless 1e3 <= limit_ns <= 6e10. */
hcg_status hcg_set_wait_limit(hcg_ctx *ctx, int64_t limit_ns, int probe);

/* Allocation cap, a host-side way to meet out-of-memory without exhausting
 * the GPU: the field-sized device buffers the context allocates -- copied
 * coordinates and spectra, sort and table scratch, cube, weights, quantised
 * and streamed spectra -- may total at most `bytes` (0: no cap, the
 * default).  A call whose allocation would go beyond it returns
 * HCG_ERR_OOM, as it would when device memory runs out, and the context
 * stays usable: a later call (after a higher cap, or with a smaller field)
 * allocates again.  Small fixed buffers (error word, counters, per-channel
 * scales, projected cell centres) are not counted.  INVALID_ARG: bytes < 0. */
hcg_status hcg_set_alloc_cap(hcg_ctx *ctx, int64_t bytes);

/* Tuning of the gather (replaces the paper's launch rules, Sec. 4.2 Eqs. 2-3,
 * and its coarsening advice); 0 in a slot means automatic.  The arguments
 * mean what they say, per path:
 *   HCG_PATH_GATHER   cells_per_block 16 (a block of four 2 x 2 groups, the
 *                     search repeated per channel slice) or 32 (eight groups
 *                     that list their accepted candidates once, then sweep
 *                     every slice over the list); chans_per_thread 1, 4 or 8
 *                     (32 cells per block: 4 or 8); tile_depth = candidate rows
 *                     whose loads are in flight per lane, 8 or 12 (32 cells
 *                     per block only; 12 needs 8 channels per thread).
 *   HCG_PATH_STAGED   cells_per_block 32 (8 x 4) or 64 (8 x 8);
 *                     chans_per_thread 4; tile_depth = candidates per staged
 *                     chunk, 16 or 32.
 *   HCG_PATH_TENSOR   cells_per_block 128; chans_per_thread 0; tile_depth =
 *                     candidates per MMA chunk (the K of one stage), 64 for
 *                     BF16 / E4M3 storage; FP32 storage always runs chunks of
 *                     32 (its split-TF32 operands are twice as wide), which
 *                     64 and 0 both select.
 *   HCG_PATH_SCATTER, HCG_PATH_AUTO   all three 0.
 * Every choice computes the same sums (per cell and channel in S' order on
 * the gather paths); the layouts differ in speed only.
 * INVALID_ARG for a value or combination outside these lists. */
hcg_status hcg_set_tuning(hcg_ctx *ctx, int cells_per_block, int chans_per_thread,
                          int tile_depth, int path);

/* Stage timers.  With profiling on, hcg_grid records CUDA events on the
 * context's stream between its stages; hcg_stage_times then returns the mean
 * device time of each stage, in milliseconds, over the hcg_grid calls since
 * profiling was (re)enabled (the last 64 of them at most):
 * [0] ingest (quantisation), [1] pixel indices and sort keys, [2] radix
 * sort, [3] S' data and both lookup tables, [4] gather and normalisation.
 * cap: capacity of ms (up to 5 written).  Synchronises. */
hcg_status hcg_set_profiling(hcg_ctx *ctx, int enable);
hcg_status hcg_stage_times(hcg_ctx *ctx, double *ms, int32_t cap);

/* Autotuner (replaces the paper's per-GPU launch rules, Sec. 4.2 Eqs. 2-3,
 * and its coarsening advice): with kernel, grid and samples set, time every
 * applicable (cells per block, channels per thread, tile depth, path) of
 * hcg_set_tuning on the loaded field -- the gather path's block sizes,
 * channels per lane and rows in flight, the staged path's tiles and chunk
 * depths, the tensor path -- with 2 warm-up and 3 timed passes each (CUDA
 * events), keep the fastest in the context, and remember it process-wide
 * under a key of (channels, storage type, samples per cell, support radius
 * in cells, projected or not).  A later call with the same key reuses the
 * cached choice unless force != 0, and every later pass (hcg_grid, and the
 * graph hcg_batch_grid captures) of a field left on HCG_PATH_AUTO whose key
 * is cached runs the cached choice.  choice (may be NULL) receives the four
 * values as hcg_set_tuning takes them: {cells_per_block, chans_per_thread,
 * tile_depth, path}.  Synchronises; overwrites the context's last result. */
hcg_status hcg_autotune(hcg_ctx *ctx, int force, int32_t *choice);

/* What the last timing run of hcg_autotune on this context measured (a
 * cached answer times nothing and leaves the table as it was): for k <
 * *count, choices[4 k .. 4 k + 3] = {cells_per_block, chans_per_thread,
 * tile_depth, path} of candidate k and ms[k] its mean pass time in
 * milliseconds (negative if it could not run).  cap: capacity in candidates;
 * INVALID_ARG if below the count (which is still written). */
hcg_status hcg_autotune_table(hcg_ctx *ctx, int32_t *choices, float *ms, int32_t cap, int32_t *count);

/* ---- test exports (synchronise; host output buffers) -------------------- */

/* The sorted pixel array P' and permutation of Sec. 3.3 step I: pix_sorted[q]
 * is the pixel of the q-th kept sample, perm[q] its input index, q < M.
 * cap is the capacity of both arrays; *m_out receives M.  INVALID_ARG if
 * cap < M (nothing written). */
hcg_status hcg_debug_pix(hcg_ctx *ctx, int64_t *pix_sorted, uint32_t *perm, int64_t cap,
                         int64_t *m_out);

/* The two lookup tables: upix[k] / ustart[k] (Sec. 3.3 step II, k < U, with
 * ustart[U] = M) and rstart[r - ring_lo] (Sec. 3.3 step III) for
 * r in [ring_lo, ring_hi + 1].  ucap: capacity of upix (ustart needs
 * ucap + 1); rcap: capacity of rstart. */
hcg_status hcg_debug_lut(hcg_ctx *ctx, int64_t *upix, int64_t *ustart, int64_t ucap,
                         int64_t *u_out, int64_t *rstart, int64_t rcap);

/* Contributor lists (Sec. 3.4) of cells [cell_begin, cell_end) (cell index
 * j*nx + i) as CSR: offsets[cell_end - cell_begin + 1], sample_ids (input
 * indices, increasing within a cell).  cap: capacity of sample_ids;
 * INVALID_ARG if too small (offsets still written). */
hcg_status hcg_debug_neighbours(hcg_ctx *ctx, int64_t cell_begin, int64_t cell_end,
                                int64_t *offsets, uint32_t *sample_ids, int64_t cap);

/* ---- batched form --------------------------------------------------------
 * Many independent fields (uneven sample counts, channel counts, grid sizes,
 * storage types) gridded together: every field's pre-ordering stages on
 * forked streams, then ONE persistent CUDA-core gather launch whose blocks
 * take (field, 4-group block, channel slice) work items from a queue sorted
 * by estimated cost, plus the tensor-core launches of fields on that path --
 * all captured once into a CUDA graph and replayed.  The batch holds
 * references to contexts (not copies); each keeps its own inputs, outputs
 * and scratch, and must be set up (kernel, grid, samples) before the first
 * hcg_batch_grid.  Results are those of hcg_grid on each field.  Fields whose
 * coordinates (the same device arrays), kernel and grid equal an earlier
 * field's -- one geometry stored in several types, say -- share that field's
 * pre-ordering and tables, which the graph then builds once; such a field's
 * hcg_get_info / hcg_debug_* report the shared tables until its next own
 * hcg_grid, so the field it shares with must not be destroyed before it.
 * cuda_stream must be a created (non-default) stream: graph capture needs it. */
hcg_status hcg_batch_create(hcg_batch **out, int device, void *cuda_stream);
hcg_status hcg_batch_destroy(hcg_batch *batch);
hcg_status hcg_batch_add(hcg_batch *batch, hcg_ctx *field);
/* Grid every field (enqueue only).  The first call prepares every field,
 * builds the work queue and captures the graph (it may allocate, so it must
 * not itself run under stream capture); later calls replay the graph while
 * every field's buffers, shapes and parameters are unchanged, and capture a
 * new one otherwise. */
hcg_status hcg_batch_grid(hcg_batch *batch);
/* Wait for the batch stream; report the first field error. */
hcg_status hcg_batch_sync(hcg_batch *batch);
/* Work items of the persistent launch and kernels in the graph. */
hcg_status hcg_batch_info(hcg_batch *batch, int64_t *work_items, int32_t *launches);

/* ---- allocation-free pre-ordering ----------------------------------------
 * For callers that cannot allocate device memory themselves or let a library
 * do it: real-time pipelines that reserve all their device memory at
 * start-up and forbid allocation afterwards, and host applications whose
 * device memory belongs to another runtime's pool.  The paper has no
 * counterpart: this is the same pre-ordering step that hcg_grid runs (pixel
 * of every sample, stable radix sort by pixel), with its scratch in a fixed
 * device array instead of buffers the library allocates.
 *
 * lon_deg, lat_deg: n FP64 device values.  nside: power of two; ring_lo,
 * ring_hi: the rings kept (1 <= ring_lo <= ring_hi <= 4 nside - 1).
 * pix_sorted (n int64) and perm (n uint32), device memory owned by the
 * caller, receive the order hcg_debug_pix reports: kept samples by (pixel,
 * coordinate hash, index), then every dropped sample (ring outside the
 * range, or a non-finite / |lat| > 90 coordinate, which is not reported
 * here) with pixel INT64_MAX.  Enqueued on cuda_stream on the current device.
 *
 * Errors: INVALID_ARG for n < 0, n > HCG_NOALLOC_MAX_SAMPLES, an nside or
 * ring range out of range, a null pointer with n > 0, or a pointer that is
 * not device memory of the current device (checked before any launch);
 * UNSUPPORTED when the kept rings hold 2^32 pixels or more (hcg_grid handles
 * those).
 *
 * Limits and sharing: the scratch is one HCG_NOALLOC_SCRATCH_BYTES array per
 * device that loads the library, held until the process exits, shared by
 * every call: calls whose work overlaps on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  The first call on a
 * device looks up the array's device address.  The call allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine). */
#define HCG_NOALLOC_MAX_SAMPLES 262144
#define HCG_NOALLOC_SCRATCH_BYTES 3277312
hcg_status hcg_preorder_noalloc(const double *lon_deg, const double *lat_deg, int64_t n, int64_t nside,
                                int64_t ring_lo, int64_t ring_hi, int64_t *pix_sorted, uint32_t *perm,
                                void *cuda_stream);

/* ---- measurement helper (outside the gridding path) ----------------------
 * The device's FP32 fused multiply-add throughput, measured: a kernel of
 * independent FMA chains on every SM, CUDA-event timed (3 warm-up and the
 * best of 5 launches), in TFLOP/s (2 flops per FMA).  It is the denominator
 * of the arithmetic roofline of the CUDA-core gathers, which spend one FMA
 * per contribution; the paper has no counterpart.  Synchronises. */
hcg_status hcg_measure_fp32_peak(int device, double *tflops);

const char *hcg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HCGRID_H */

// hcg_api.cu -- the C ABI (include/hcgrid.h): argument checks, device
// buffers, and the order of the kernel stages of one gridding pass.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <initializer_list>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include "hcg_internal.h"

namespace {
thread_local std::string g_err;
constexpr double kDegH = 3.14159265358979323846 / 180.0;

hcg_status fail(hcg_status s, const std::string &m) {
    g_err = m;
    return s;
}

#define HCG_CUDA(call, what)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return hcg_cuda_fail(e_, what); \
    } while (0)

// Field-sized device buffers: allocated against the context's cap (a request
// that would take the context's total above it fails with OOM, as cudaMalloc
// does when memory runs out) and released with their size forgotten.
hcg_status dev_alloc(hcg_ctx *c, void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (c->alloc_cap > 0 && c->alloc_bytes + (int64_t)bytes > c->alloc_cap)
        return fail(HCG_ERR_OOM, std::string("device allocation beyond the context's cap: ") + what);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(HCG_ERR_OOM, std::string("device allocation failed: ") + what);
    }
    c->alloc_live[*p] = bytes;
    c->alloc_bytes += (int64_t)bytes;
    return HCG_OK;
}

void dev_release(hcg_ctx *c, void *p) {
    if (!p) return;
    auto it = c->alloc_live.find(p);
    if (it != c->alloc_live.end()) {
        c->alloc_bytes -= (int64_t)it->second;
        c->alloc_live.erase(it);
    }
    cudaFree(p);
}

template <typename T>
hcg_status grow(hcg_ctx *c, T **p, int64_t &cap, int64_t need, const char *what) {
    if (need <= cap && *p) return HCG_OK;
    dev_release(c, *p);
    *p = nullptr;
    cap = 0;
    int64_t n = std::max<int64_t>(need, 1);
    hcg_status s = dev_alloc(c, (void **)p, (size_t)n * sizeof(T), what);
    if (s) return s;
    cap = n;
    return HCG_OK;
}

hcg_status grow_bytes(hcg_ctx *c, void **p, size_t &cap, size_t need, const char *what) {
    if (need <= cap && *p) return HCG_OK;
    dev_release(c, *p);
    *p = nullptr;
    cap = 0;
    hcg_status s = dev_alloc(c, p, std::max<size_t>(need, 16), what);
    if (s) return s;
    cap = std::max<size_t>(need, 16);
    return HCG_OK;
}

int64_t ring_first_host(int64_t ns, int64_t r) {
    if (r <= ns) return 2 * r * (r - 1);
    if (r <= 3 * ns) return 2 * ns * (ns - 1) + (r - ns) * 4 * ns;
    int64_t q = 4 * ns - r;
    return 12 * ns * ns - 2 * q * (q + 1);
}

double ring_coord_host(double ns, double z) {
    if (z > 2.0 / 3.0) return ns * sqrt(std::max(0.0, 3.0 * (1.0 - z)));
    if (z < -2.0 / 3.0) return 4.0 * ns - ns * sqrt(std::max(0.0, 3.0 * (1.0 + z)));
    return ns * (2.0 - 1.5 * z);
}

hcg_status check_ctx(hcg_ctx *c) {
    if (!c) return fail(HCG_ERR_INVALID_ARG, "null context");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaSetDevice");
    return HCG_OK;
}

// Parameters of one pass, from the kernel, the grid and the host libm.
void make_params(hcg_ctx *c, GridParams &g, int &key_bits) {
    memset(&g, 0, sizeof(g));
    g.lon0 = c->lon0; g.lat0 = c->lat0; g.pix = c->pix;
    g.nx = c->nx; g.ny = c->ny;
    g.hx = 0.5 * (double)(c->nx - 1);
    g.hy = 0.5 * (double)(c->ny - 1);
    g.R_deg = c->support;
    double Rr = c->support * kDegH;
    double s = sin(0.5 * Rr);
    g.hR = s * s;
    g.havRf = (float)(g.hR * (1.0 + 1e-6));
    g.R2 = (float)(Rr * Rr);
    g.band_lo = (float)(Rr * Rr * (1.0 - 1e-5));
    g.band_hi = (float)(Rr * Rr * (1.0 + 1e-5));
    double sig = c->fwhm * kDegH / sqrt(8.0 * log(2.0));
    g.kexp = (float)(1.0 / (2.0 * sig * sig * log(2.0)));    // log2(e) / (2 sigma^2)
    g.sinR = (float)sin(Rr);
    g.R_radf = (float)Rr;
    g.nside = c->nside;
    // FP32 pixel screen: edge-line values move by <= 1.65e-7 nside; twice that
    g.screen_eps = 3.3e-7 * (double)c->nside;
    if (g.screen_eps > 0.05) g.screen_eps = 0.0;
    // rings the grid can reach: latitude band of the cells +- R, padded 2 rings
    double latmin = c->lat0 - g.hy * c->pix, latmax = c->lat0 + g.hy * c->pix;
    if (c->cell_lon) { latmin = c->cell_latmin; latmax = c->cell_latmax; }
    g.clon = c->cell_lon; g.clat = c->cell_lat;
    double lo = std::max(-90.0, latmin - c->support), hi = std::min(90.0, latmax + c->support);
    double ns = (double)c->nside;
    int64_t ra = (int64_t)floor(ring_coord_host(ns, sin(hi * kDegH))) - 2;
    int64_t rb = (int64_t)ceil(ring_coord_host(ns, sin(lo * kDegH))) + 2;
    g.r_lo = std::max<int64_t>(1, ra);
    g.r_hi = std::min<int64_t>(4 * c->nside - 1, rb);
    g.pix_lo = ring_first_host(c->nside, g.r_lo);
    int64_t npr = ring_first_host(c->nside, g.r_hi + 1) - g.pix_lo;
    // pixel-offset bits (npr < 2^52 for nside <= 2^24), leaving the all-ones
    // offset free for dropped samples; above 64 bits in all the sort runs
    // the hash digits and the offset digits as two phases
    int bits = 1;
    while (bits < 62 && ((int64_t)1 << bits) - 1 < npr) bits++;
    key_bits = bits + 32;
}

hcg_status ensure_scratch(hcg_ctx *c, const GridParams &g) {
    int64_t n = c->n;
    hcg_status s;
    if (n > c->sample_cap || !c->psorted) {
        int64_t cap = std::max<int64_t>(n, 1);
        int64_t dummy;
        for (int k = 0; k < 2; k++) {
            dummy = 0; if ((s = grow(c, &c->sort.keys[k], dummy, cap, "sort keys"))) return s;
            dummy = 0; if ((s = grow(c, &c->sort.vals[k], dummy, cap, "sort values"))) return s;
        }
        dummy = 0; if ((s = grow(c, &c->psorted, dummy, cap, "P'"))) return s;
        dummy = 0; if ((s = grow(c, &c->sc_uv, dummy, cap, "S' coordinates"))) return s;
        dummy = 0; if ((s = grow(c, &c->sc_cos, dummy, cap, "S' cos"))) return s;
        dummy = 0; if ((s = grow(c, &c->sc_row, dummy, cap, "S' rows"))) return s;
        dummy = 0; if ((s = grow(c, &c->flags, dummy, cap, "LUT1 flags"))) return s;
        dummy = 0; if ((s = grow(c, &c->upix, dummy, cap, "LUT1 pixels"))) return s;
        dummy = 0; if ((s = grow(c, &c->ustart, dummy, cap + 1, "LUT1 starts"))) return s;
        int64_t ntiles = sort_tiles(cap);
        dummy = 0; if ((s = grow(c, &c->sort.counts, dummy, 256 * ntiles, "sort counts"))) return s;
        dummy = 0; if ((s = grow(c, &c->sort.status, dummy, 256 * ntiles, "sort look-back status"))) return s;
        HCG_CUDA(cudaMemset(c->sort.status, 0, (size_t)256 * ntiles * sizeof(uint64_t)), "clear sort status");
        if (!c->sort.hist) {
            dummy = 0; if ((s = grow(c, &c->sort.hist, dummy, kSortHistWords, "sort histograms"))) return s;
            HCG_CUDA(cudaMemset(c->sort.hist, 0, kSortHistWords * sizeof(uint32_t)), "clear sort histograms");
        }
        // scan levels for max(256 * ntiles, n) elements
        for (auto p : c->scan.level) dev_release(c, p);
        c->scan.level.clear(); c->scan.level_cap.clear();
        int64_t len = std::max<int64_t>(256 * ntiles, cap);
        while (len > 4096) {
            int64_t nb = (len + 4095) / 4096;
            uint32_t *p = nullptr; int64_t pc = 0;
            if ((s = grow(c, &p, pc, nb, "scan"))) return s;
            c->scan.level.push_back(p); c->scan.level_cap.push_back(pc);
            len = nb;
        }
        c->sample_cap = cap;
    }
    int64_t rings = g.r_hi - g.r_lo + 2;
    if (rings > c->ring_cap || !c->rstart) {
        int64_t d1 = 0, d2 = 0, d3 = 0;
        if ((s = grow(c, &c->rstart, d1, rings, "LUT2"))) return s;
        if ((s = grow(c, &c->rustart, d2, rings, "LUT2 pixels"))) return s;
        if ((s = grow(c, &c->rband, d3, rings, "ring bands"))) return s;
        c->ring_cap = rings;
    }
    size_t cells = (size_t)c->nx * (size_t)c->ny;
    if (!c->bound_cube) {
        if ((s = grow_bytes(c, (void **)&c->own_cube, c->own_cube_cap, cells * (size_t)c->nchan * 4, "cube"))) return s;
    }
    if (!c->bound_w) {
        if ((s = grow_bytes(c, (void **)&c->own_w, c->own_w_cap, cells * 4, "weights"))) return s;
    }
    if (c->store != c->in_dtype) {
        size_t es = c->store == HCG_BF16 ? 2 : 1;
        if (!c->host_spec &&
            (s = grow_bytes(c, &c->q_spec, c->q_spec_bytes, (size_t)n * c->nchan * es, "quantised spectra")))
            return s;
        if (c->store == HCG_E4M3 && c->q_scale_cap < c->nchan) {
            if (c->q_scale) cudaFree(c->q_scale);
            if (c->q_amax) cudaFree(c->q_amax);
            c->q_scale = nullptr; c->q_amax = nullptr;
            HCG_CUDA(cudaMalloc((void **)&c->q_scale, sizeof(float) * c->nchan), "cudaMalloc scales");
            HCG_CUDA(cudaMalloc((void **)&c->q_amax, sizeof(uint32_t) * c->nchan), "cudaMalloc amax");
            c->q_scale_cap = c->nchan;
        }
    }
    return HCG_OK;
}

hcg_status read_err(hcg_ctx *c) {
    int e = 0;
    HCG_CUDA(cudaMemcpy(&e, c->derr, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (e & HCG_DERR_BAD_COORD) return fail(HCG_ERR_INVALID_ARG, "a sample coordinate is non-finite or |lat| > 90");
    if (e & HCG_DERR_TIMEOUT) return fail(HCG_ERR_TIMEOUT, "a bounded device wait gave up");
    if (e & HCG_DERR_SEGMENTS) return fail(HCG_ERR_UNSUPPORTED, "candidate segment buffer overflow");
    return HCG_OK;
}

void free_all(hcg_ctx *c) {
    void *ptrs[] = {c->cell_lon, c->cell_lat, c->own_lon, c->own_lat, c->own_spec, c->own_scale, c->q_spec, c->q_scale, c->q_amax,
                    c->sort.keys[0], c->sort.keys[1], c->sort.vals[0], c->sort.vals[1], c->sort.counts,
                    c->sort.status, c->sort.hist,
                    c->psorted, c->sc_uv, c->sc_cos, c->sc_row, c->flags, c->upix, c->ustart, c->rstart,
                    c->rustart, c->rband, c->dscal, c->derr, c->own_cube, c->own_w};
    for (void *p : ptrs) if (p) cudaFree(p);
    for (int k = 0; k < 2; k++) {
        if (c->stage[k]) cudaFree(c->stage[k]);
        if (c->qstage[k]) cudaFree(c->qstage[k]);
        if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
        if (c->ev_consumed[k]) cudaEventDestroy(c->ev_consumed[k]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    for (int k = 0; k < 2; k++)
        if (c->ev_gathered[k]) cudaEventDestroy(c->ev_gathered[k]);
    if (c->ev_out_done) cudaEventDestroy(c->ev_out_done);
    if (c->out_stream) cudaStreamDestroy(c->out_stream);
    for (auto p : c->scan.level) cudaFree(p);
    for (auto &slot : c->ev)
        for (auto e : slot) if (e) cudaEventDestroy(e);
}

}  // namespace

void hcg_set_error(const std::string &msg) { g_err = msg; }

hcg_status hcg_cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return HCG_ERR_CUDA;
}

// A host pointer handed over as device memory would make a kernel fault;
// the runtime's pointer attributes tell the two apart before any launch.
hcg_status check_device_ptr(const void *p, int device, const char *what) {
    if (!p) return HCG_OK;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HCG_ERR_INVALID_ARG, std::string(what) + ": not a CUDA-visible pointer");
    }
    if (a.type == cudaMemoryTypeManaged) return HCG_OK;
    if (a.type != cudaMemoryTypeDevice)
        return fail(HCG_ERR_INVALID_ARG, std::string(what) + " is not device memory");
    if (a.device != device)
        return fail(HCG_ERR_INVALID_ARG, std::string(what) + " is device memory of another device");
    return HCG_OK;
}

extern "C" {

const char *hcg_last_error(void) { return g_err.c_str(); }

hcg_status hcg_create(hcg_ctx **out, int device, void *stream) {
    if (!out) return fail(HCG_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    int ndev = 0;
    HCG_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(HCG_ERR_INVALID_ARG, "no such CUDA device");
    HCG_CUDA(cudaSetDevice(device), "cudaSetDevice");
    hcg_ctx *c = new (std::nothrow) hcg_ctx();
    if (!c) return fail(HCG_ERR_OOM, "host allocation failed");
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc((void **)&c->derr, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void **)&c->dscal, 8 * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return fail(HCG_ERR_OOM, "device allocation failed");
    }
    cudaMemset(c->derr, 0, sizeof(int));
    cudaMemset(c->dscal, 0, 8 * sizeof(int64_t));
    *out = c;
    return HCG_OK;
}

hcg_status hcg_destroy(hcg_ctx *c) {
    if (!c) return HCG_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    if (c->out_stream) cudaStreamSynchronize(c->out_stream);
    free_all(c);
    delete c;
    return HCG_OK;
}

hcg_status hcg_set_stream(hcg_ctx *c, void *stream) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    c->stream = (cudaStream_t)stream;
    return HCG_OK;
}

hcg_status hcg_set_kernel(hcg_ctx *c, double fwhm, double support) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (!(fwhm > 0) || !(support > 0) || !isfinite(fwhm) || !isfinite(support))
        return fail(HCG_ERR_INVALID_ARG, "fwhm and support radius must be positive and finite");
    double sig = fwhm / sqrt(8.0 * log(2.0));
    if (support > 1.0) return fail(HCG_ERR_INVALID_ARG, "support radius above 1 degree");
    if (support > 10.0 * sig) return fail(HCG_ERR_INVALID_ARG, "support radius above 10 sigma");
    if (fwhm < 1.0 / 3600.0) return fail(HCG_ERR_INVALID_ARG, "fwhm below 1 arcsec");
    // Sec. 3.6 item 3: HEALPix resolution ~ sigma_kernel / 2
    double sr = sig * kDegH;
    int64_t ns = 1;
    while (sqrt(3.14159265358979323846 / 3.0) / (double)ns > 0.5 * sr && ns < ((int64_t)1 << 24)) ns *= 2;
    c->fwhm = fwhm;
    c->support = support;
    c->nside = ns;
    c->kernel_set = true;
    return HCG_OK;
}

hcg_status hcg_set_grid(hcg_ctx *c, int proj, double lon0, double lat0, double pixel, int32_t nx, int32_t ny) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (proj < HCG_CAR || proj > HCG_WCS_CAR) return fail(HCG_ERR_INVALID_ARG, "unknown projection");
    if (nx < 1 || ny < 1) return fail(HCG_ERR_INVALID_ARG, "nx and ny must be >= 1");
    if (!(pixel > 0) || !isfinite(pixel) || !isfinite(lon0) || !isfinite(lat0))
        return fail(HCG_ERR_INVALID_ARG, "pixel size must be positive; centre finite");
    if ((double)nx * pixel > 180.0) return fail(HCG_ERR_INVALID_ARG, "grid wider than 180 degrees");
    double hy = 0.5 * (double)(ny - 1) * pixel;
    if (proj == HCG_CAR && fabs(lat0) + hy > 89.0)
        return fail(HCG_ERR_INVALID_ARG, "cell latitudes beyond +-89 degrees");
    double latmin = 0, latmax = 0;
    double *dlon = nullptr, *dlat = nullptr;
    if (proj != HCG_CAR) {
        const size_t cells = (size_t)nx * (size_t)ny;
        std::vector<double> hl(cells), hb(cells);
        if (wcs_cell_centres(proj, lon0, lat0, pixel, nx, ny, hl.data(), hb.data()) != 0)
            return fail(HCG_ERR_INVALID_ARG, "the projection cannot place every cell");
        latmin = 90.0; latmax = -90.0;
        for (size_t k = 0; k < cells; k++) {
            double d = hl[k] - lon0;
            d = d - 360.0 * floor((d + 180.0) / 360.0);
            if (fabs(hb[k]) > 89.0) return fail(HCG_ERR_INVALID_ARG, "cell latitudes beyond +-89 degrees");
            if (fabs(d) > 90.0) return fail(HCG_ERR_INVALID_ARG, "cells more than 90 degrees of longitude from lon0");
            latmin = std::min(latmin, hb[k]); latmax = std::max(latmax, hb[k]);
        }
        if (cudaMalloc((void **)&dlon, cells * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&dlat, cells * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            if (dlon) cudaFree(dlon);
            return fail(HCG_ERR_OOM, "device allocation failed: cell centres");
        }
        cudaError_t e = cudaMemcpy(dlon, hl.data(), cells * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dlat, hb.data(), cells * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {     // the context keeps its previous grid
            cudaFree(dlon);
            cudaFree(dlat);
            return hcg_cuda_fail(e, "copy cell centres");
        }
    }
    if (c->cell_lon) { cudaStreamSynchronize(c->stream); cudaFree(c->cell_lon); cudaFree(c->cell_lat); }
    c->cell_lon = dlon; c->cell_lat = dlat;
    c->cell_latmin = latmin; c->cell_latmax = latmax;
    c->proj = proj;
    c->lon0 = lon0; c->lat0 = lat0; c->pix = pixel; c->nx = nx; c->ny = ny;
    c->grid_set = true;
    return HCG_OK;
}

// A free list of target cells: the projected-grid machinery with the list
// as a grid of ncells x 1 cells whose centres are given.
hcg_status hcg_set_cell_list(hcg_ctx *c, const double *lon, const double *lat, int64_t ncells, int mem) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (ncells < 1 || ncells > 0x7FFFFFFFll) return fail(HCG_ERR_INVALID_ARG, "ncells must lie in [1, 2^31 - 1]");
    if (!lon || !lat) return fail(HCG_ERR_INVALID_ARG, "null cell centres");
    if (mem != HCG_MEM_HOST && mem != HCG_MEM_DEVICE) return fail(HCG_ERR_INVALID_ARG, "unknown memory kind");
    const size_t n = (size_t)ncells;
    std::vector<double> hl(n), hb(n);
    if (mem == HCG_MEM_DEVICE) {
        if ((s = check_device_ptr(lon, c->device, "lon_deg")) || (s = check_device_ptr(lat, c->device, "lat_deg")))
            return s;
        HCG_CUDA(cudaMemcpy(hl.data(), lon, n * sizeof(double), cudaMemcpyDeviceToHost), "copy cell list");
        HCG_CUDA(cudaMemcpy(hb.data(), lat, n * sizeof(double), cudaMemcpyDeviceToHost), "copy cell list");
    } else {
        memcpy(hl.data(), lon, n * sizeof(double));
        memcpy(hb.data(), lat, n * sizeof(double));
    }
    // reference longitude: the direction of the mean of the cells' unit vectors
    // in the equatorial plane; every cell must lie within 90 degrees of it
    double sx = 0, sy = 0, latmin = 90.0, latmax = -90.0;
    for (size_t k = 0; k < n; k++) {
        if (!isfinite(hl[k]) || !isfinite(hb[k])) return fail(HCG_ERR_INVALID_ARG, "non-finite cell centre");
        if (fabs(hb[k]) > 89.0) return fail(HCG_ERR_INVALID_ARG, "cell latitudes beyond +-89 degrees");
        sx += cos(hl[k] * kDegH);
        sy += sin(hl[k] * kDegH);
        latmin = std::min(latmin, hb[k]);
        latmax = std::max(latmax, hb[k]);
    }
    const double lon0 = (sx == 0 && sy == 0) ? hl[0] : atan2(sy, sx) / kDegH;
    for (size_t k = 0; k < n; k++) {
        double d = hl[k] - lon0;
        d = d - 360.0 * floor((d + 180.0) / 360.0);
        if (fabs(d) > 90.0) return fail(HCG_ERR_INVALID_ARG, "cells spread over more than 90 degrees of longitude from their mean");
    }
    double *dlon = nullptr, *dlat = nullptr;
    if (cudaMalloc((void **)&dlon, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&dlat, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        if (dlon) cudaFree(dlon);
        return fail(HCG_ERR_OOM, "device allocation failed: cell list");
    }
    cudaError_t e = cudaMemcpy(dlon, hl.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dlat, hb.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dlon);
        cudaFree(dlat);
        return hcg_cuda_fail(e, "copy cell list");
    }
    if (c->cell_lon) { cudaStreamSynchronize(c->stream); cudaFree(c->cell_lon); cudaFree(c->cell_lat); }
    c->cell_lon = dlon; c->cell_lat = dlat;
    c->cell_latmin = latmin; c->cell_latmax = latmax;
    c->proj = HCG_CELL_LIST;
    c->lon0 = lon0; c->lat0 = 0.5 * (latmin + latmax);
    c->pix = 1.0 / 60.0;            // a nominal cell size (the tuner's key); no cell geometry uses it
    c->nx = (int32_t)ncells; c->ny = 1;
    c->grid_set = true;
    return HCG_OK;
}

hcg_status hcg_set_storage(hcg_ctx *c, int dtype) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (dtype != HCG_F32 && dtype != HCG_BF16 && dtype != HCG_E4M3) return fail(HCG_ERR_INVALID_ARG, "unknown dtype");
    if (c->loaded && !(dtype == c->in_dtype || (c->in_dtype == HCG_F32)))
        return fail(HCG_ERR_INVALID_ARG, "storage type incompatible with the loaded spectra");
    c->store = dtype;
    return HCG_OK;
}

hcg_status hcg_load_samples(hcg_ctx *c, const double *lon, const double *lat, const void *spec, int64_t n,
                            int32_t nchan, int dtype, const float *scale, int mem) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (n < 0 || nchan < 1) return fail(HCG_ERR_INVALID_ARG, "n must be >= 0 and nchan >= 1");
    if (n > 0xFFFFFFFFll) return fail(HCG_ERR_INVALID_ARG, "more than 2^32 - 1 samples");
    if (dtype != HCG_F32 && dtype != HCG_BF16 && dtype != HCG_E4M3) return fail(HCG_ERR_INVALID_ARG, "unknown dtype");
    if (n > 0 && (!lon || !lat || !spec)) return fail(HCG_ERR_INVALID_ARG, "null input pointer");
    if (dtype == HCG_E4M3 && !scale) return fail(HCG_ERR_INVALID_ARG, "E4M3 spectra need per-channel scales");
    if (mem != HCG_MEM_HOST && mem != HCG_MEM_DEVICE && mem != HCG_MEM_DEVICE_BORROW && mem != HCG_MEM_HOST_STREAM)
        return fail(HCG_ERR_INVALID_ARG, "unknown memory kind");
    if (!(c->store == dtype || dtype == HCG_F32))
        return fail(HCG_ERR_INVALID_ARG, "storage type must equal the input type or the input must be F32");
    if ((double)n * (double)nchan > 4.0e18) return fail(HCG_ERR_INVALID_ARG, "n * nchan overflows");
    size_t es = dtype == HCG_F32 ? 4 : (dtype == HCG_BF16 ? 2 : 1);
    size_t sbytes = (size_t)n * (size_t)nchan * es;
    c->loaded = false;
    c->host_spec = nullptr;
    if (mem == HCG_MEM_HOST_STREAM) {
        // coordinates (and E4M3 scales) now; spectra window by window in hcg_grid
        if ((s = grow(c, &c->own_lon, c->own_coord_cap, n, "lon"))) return s;
        int64_t dummy = 0;
        if ((s = grow(c, &c->own_lat, dummy, n, "lat"))) return s;
        if (n > 0) {
            HCG_CUDA(cudaMemcpyAsync(c->own_lon, lon, n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy lon");
            HCG_CUDA(cudaMemcpyAsync(c->own_lat, lat, n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy lat");
        }
        c->lon = c->own_lon; c->lat = c->own_lat; c->spec_in = nullptr;
        c->scale_in = nullptr;
        if (dtype == HCG_E4M3) {
            if (c->own_scale_cap < nchan) {
                if (c->own_scale) cudaFree(c->own_scale);
                c->own_scale = nullptr;
                HCG_CUDA(cudaMalloc((void **)&c->own_scale, sizeof(float) * nchan), "cudaMalloc scales");
                c->own_scale_cap = nchan;
            }
            HCG_CUDA(cudaMemcpyAsync(c->own_scale, scale, sizeof(float) * nchan, cudaMemcpyHostToDevice, c->stream),
                     "copy scales");
            c->scale_in = c->own_scale;
        }
        c->host_spec = spec;
        c->n = n; c->nchan = nchan; c->in_dtype = dtype;
        c->loaded = true;
        c->gridded = false;
        return HCG_OK;
    }
    if ((mem == HCG_MEM_DEVICE || mem == HCG_MEM_DEVICE_BORROW) && n > 0) {
        if ((s = check_device_ptr(lon, c->device, "lon_deg")) || (s = check_device_ptr(lat, c->device, "lat_deg")) ||
            (s = check_device_ptr(spec, c->device, "spectra")) ||
            (dtype == HCG_E4M3 && (s = check_device_ptr(scale, c->device, "chan_scale"))))
            return s;
    }
    if (mem == HCG_MEM_DEVICE_BORROW && n > 0 &&
        (((uintptr_t)spec & 15) || ((uintptr_t)lon & 7) || ((uintptr_t)lat & 7)))
        return fail(HCG_ERR_INVALID_ARG, "borrowed spectra must be 16-byte aligned, coordinates 8-byte aligned");
    if (mem == HCG_MEM_DEVICE_BORROW) {
        c->lon = lon; c->lat = lat; c->spec_in = spec;
        c->scale_in = dtype == HCG_E4M3 ? scale : nullptr;
    } else {
        cudaMemcpyKind k = mem == HCG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        if ((s = grow(c, &c->own_lon, c->own_coord_cap, n, "lon"))) return s;
        int64_t dummy = 0;
        if ((s = grow(c, &c->own_lat, dummy, n, "lat"))) return s;
        if ((s = grow_bytes(c, &c->own_spec, c->own_spec_bytes, sbytes, "spectra"))) return s;
        if (n > 0) {
            HCG_CUDA(cudaMemcpyAsync(c->own_lon, lon, n * sizeof(double), k, c->stream), "copy lon");
            HCG_CUDA(cudaMemcpyAsync(c->own_lat, lat, n * sizeof(double), k, c->stream), "copy lat");
            HCG_CUDA(cudaMemcpyAsync(c->own_spec, spec, sbytes, k, c->stream), "copy spectra");
        }
        c->lon = c->own_lon; c->lat = c->own_lat; c->spec_in = c->own_spec;
        c->scale_in = nullptr;
        if (dtype == HCG_E4M3) {
            if (c->own_scale_cap < nchan) {
                if (c->own_scale) cudaFree(c->own_scale);
                c->own_scale = nullptr;
                HCG_CUDA(cudaMalloc((void **)&c->own_scale, sizeof(float) * nchan), "cudaMalloc scales");
                c->own_scale_cap = nchan;
            }
            HCG_CUDA(cudaMemcpyAsync(c->own_scale, scale, sizeof(float) * nchan, k, c->stream), "copy scales");
            c->scale_in = c->own_scale;
        }
    }
    c->n = n; c->nchan = nchan; c->in_dtype = dtype;
    c->loaded = true;
    c->gridded = false;
    return HCG_OK;
}

hcg_status hcg_bind_output(hcg_ctx *c, float *cube, float *w) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if ((cube == nullptr) != (w == nullptr)) return fail(HCG_ERR_INVALID_ARG, "bind both outputs or neither");
    if (((uintptr_t)cube & 15) || ((uintptr_t)w & 3))
        return fail(HCG_ERR_INVALID_ARG, "bound cube must be 16-byte aligned, weights 4-byte aligned");
    if ((s = check_device_ptr(cube, c->device, "cube")) || (s = check_device_ptr(w, c->device, "weights"))) return s;
    c->bound_cube = cube;
    c->bound_w = w;
    return HCG_OK;
}

// The literal tuning of each path (0 = automatic in every slot):
//   GATHER   cells per block 16 (k_gather) or 32 (k_gather_list), channels
//            per lane 1 / 4 / 8, candidate rows in flight 8 / 12 (list only);
//   STAGED   cells per block 32 (8 x 4) or 64 (8 x 8), 4 channels per lane,
//            chunk depth 16 / 32 candidates;
//   TENSOR   128 cells per block, chunk depth 64 candidates;
//   SCATTER  nothing to tune.
static bool tuning_valid(int path, int cells, int chans, int depth, std::string &why) {
    auto in = [](int v, std::initializer_list<int> ok) {
        for (int x : ok) if (v == x) return true;
        return false;
    };
    switch (path) {
        case HCG_PATH_AUTO:
            if (cells || chans || depth) { why = "automatic path: leave cells, channels and depth at 0"; return false; }
            return true;
        case HCG_PATH_GATHER:
            if (!in(cells, {0, 16, 32})) { why = "gather path: cells per block 0, 16 or 32"; return false; }
            if (!in(chans, {0, 1, 4, 8})) { why = "gather path: channels per thread 0, 1, 4 or 8"; return false; }
            if (!in(depth, {0, 8, 12})) { why = "gather path: rows in flight 0, 8 or 12"; return false; }
            if (cells == 16 && depth) { why = "cells per block 16 (k_gather) takes no depth"; return false; }
            if (cells == 32 && chans == 1) { why = "cells per block 32 needs 4 or 8 channels per thread"; return false; }
            if (chans == 4 && depth == 12) { why = "4 channels per thread keep 8 rows in flight"; return false; }
            return true;
        case HCG_PATH_STAGED:
            if (!in(cells, {0, 32, 64})) { why = "staged path: cells per block 0, 32 or 64"; return false; }
            if (!in(chans, {0, 4})) { why = "staged path: 4 channels per thread"; return false; }
            if (!in(depth, {0, 16, 32})) { why = "staged path: chunk depth 0, 16 or 32"; return false; }
            return true;
        case HCG_PATH_TENSOR:
            if (!in(cells, {0, 128})) { why = "tensor path: 128 cells per block"; return false; }
            if (chans) { why = "tensor path: channels per thread is not a parameter (0)"; return false; }
            if (!in(depth, {0, 64})) { why = "tensor path: chunk depth 0 or 64"; return false; }
            return true;
        case HCG_PATH_SCATTER:
            if (cells || chans || depth) { why = "scatter path: nothing to tune (0, 0, 0)"; return false; }
            return true;
        default:
            why = "unknown path";
            return false;
    }
}

hcg_status hcg_set_tuning(hcg_ctx *c, int cells, int chans, int depth, int path) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    std::string why;
    if (!tuning_valid(path, cells, chans, depth, why)) return fail(HCG_ERR_INVALID_ARG, why);
    c->t_cells = cells; c->t_chans = chans; c->t_depth = depth; c->t_path = path;
    return HCG_OK;
}

hcg_status hcg_set_wait_limit(hcg_ctx *c, int64_t limit_ns, int probe) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (limit_ns < 1000 || limit_ns > 60000000000ll)
        return fail(HCG_ERR_INVALID_ARG, "wait limit must lie in [1 us, 60 s]");
    c->wait_ns = limit_ns;
    c->wait_probe = probe != 0;
    return HCG_OK;
}

hcg_status hcg_set_alloc_cap(hcg_ctx *c, int64_t bytes) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (bytes < 0) return fail(HCG_ERR_INVALID_ARG, "allocation cap must be >= 0 (0: no cap)");
    c->alloc_cap = bytes;
    return HCG_OK;
}

hcg_status hcg_grid(hcg_ctx *c) {
    if (c) c->tables_src = nullptr;       // a pass of its own builds its own tables
    hcg_status s = grid_prepare(c);
    if (s) return s;
    const void *spec;
    int dtype;
    const float *scale;
    if (c->ev_out_done)   // the cube may not change while the last pass's copies to the host run
        HCG_CUDA(cudaStreamWaitEvent(c->stream, c->ev_out_done, 0), "wait for host copies");
    if ((s = grid_enqueue_front(c, &spec, &dtype, &scale))) return s;
    if (c->host_spec) return grid_enqueue_streamed(c);
    if ((s = grid_enqueue_gather(c, spec, dtype, scale))) return s;
    return enqueue_host_output(c, 0, c->nchan, 0, true);
}

hcg_status hcg_set_stream_chunk(hcg_ctx *c, int32_t chans) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (chans < 0) return fail(HCG_ERR_INVALID_ARG, "channels per window must be >= 0");
    c->stream_chunk = chans;
    return HCG_OK;
}

hcg_status hcg_sync(hcg_ctx *c) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    HCG_CUDA(cudaStreamSynchronize(c->stream), "stream synchronise");
    if (c->copy_stream) HCG_CUDA(cudaStreamSynchronize(c->copy_stream), "copy stream synchronise");
    if (c->out_stream) HCG_CUDA(cudaStreamSynchronize(c->out_stream), "output stream synchronise");
    return read_err(c);
}

hcg_status hcg_bind_host_output(hcg_ctx *c, float *cube, float *w) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if ((cube == nullptr) != (w == nullptr)) return fail(HCG_ERR_INVALID_ARG, "bind both outputs or neither");
    if (cube && !c->out_stream) {
        HCG_CUDA(cudaStreamCreateWithFlags(&c->out_stream, cudaStreamNonBlocking), "create output stream");
        for (int k = 0; k < 2; k++)
            HCG_CUDA(cudaEventCreateWithFlags(&c->ev_gathered[k], cudaEventDisableTiming), "create event");
        HCG_CUDA(cudaEventCreateWithFlags(&c->ev_out_done, cudaEventDisableTiming), "create event");
    }
    c->host_cube = cube;
    c->host_w = w;
    return HCG_OK;
}


hcg_status hcg_fetch(hcg_ctx *c, float *cube, float *w, int mem) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (!c->gridded) return fail(HCG_ERR_STATE, "no result: call hcg_grid first");
    if (mem != HCG_MEM_HOST && mem != HCG_MEM_DEVICE) return fail(HCG_ERR_INVALID_ARG, "unknown memory kind");
    if (mem == HCG_MEM_DEVICE &&
        ((s = check_device_ptr(cube, c->device, "cube")) || (s = check_device_ptr(w, c->device, "weights"))))
        return s;
    size_t cells = (size_t)c->nx * c->ny;
    cudaMemcpyKind k = mem == HCG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (cube && cube != c->cube())
        HCG_CUDA(cudaMemcpyAsync(cube, c->cube(), cells * c->nchan * sizeof(float), k, c->stream), "copy cube");
    if (w && w != c->weights())
        HCG_CUDA(cudaMemcpyAsync(w, c->weights(), cells * sizeof(float), k, c->stream), "copy weights");
    HCG_CUDA(cudaStreamSynchronize(c->stream), "stream synchronise");
    return read_err(c);
}

hcg_status hcg_get_info(hcg_ctx *c, hcg_info *out) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (!out) return fail(HCG_ERR_INVALID_ARG, "null output");
    if (!c->gridded) return fail(HCG_ERR_STATE, "no result: call hcg_grid first");
    HCG_CUDA(cudaStreamSynchronize(c->stream), "stream synchronise");
    int64_t sc[8];
    HCG_CUDA(cudaMemcpy(sc, c->dscal, sizeof(sc), cudaMemcpyDeviceToHost), "read counters");
    int64_t nr = c->gp.r_hi - c->gp.r_lo + 1;
    int64_t m = c->n, u = 0;                  // the scatter path builds no tables: every sample is used
    if (c->last_path != HCG_PATH_SCATTER) {
        HCG_CUDA(cudaMemcpy(&m, c->tables()->rstart + nr, sizeof(int64_t), cudaMemcpyDeviceToHost), "read M");
        HCG_CUDA(cudaMemcpy(&u, c->tables()->rustart + nr, sizeof(int64_t), cudaMemcpyDeviceToHost), "read U");
    }
    memset(out, 0, sizeof(*out));
    out->nside = c->nside;
    out->ring_lo = c->gp.r_lo;
    out->ring_hi = c->gp.r_hi;
    out->samples_kept = m;
    out->unique_pixels = u;
    out->pairs = sc[1];
    out->contributions = sc[1] * (int64_t)c->nchan;
    out->path = c->last_path;
    out->key_bits = c->key_bits;
    out->launches = c->last_launches;
    out->stream_window = c->host_spec ? c->stream_chunk_chans() : 0;
    out->tensor_flops = sc[2];
    return read_err(c);
}

hcg_status hcg_set_profiling(hcg_ctx *c, int enable) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (enable && !c->ev[0][0]) {
        for (auto &slot : c->ev)
            for (auto &e : slot) HCG_CUDA(cudaEventCreate(&e), "cudaEventCreate");
    }
    c->profiling = enable != 0;
    c->prof_calls = 0;
    return HCG_OK;
}

hcg_status hcg_stage_times(hcg_ctx *c, double *ms, int32_t cap) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (!c->profiling || c->prof_calls == 0) return fail(HCG_ERR_STATE, "profiling off or no hcg_grid since enabled");
    if (!ms || cap < 0) return fail(HCG_ERR_INVALID_ARG, "null output");
    int slots = std::min(c->prof_calls, hcg_ctx::kProfSlots);
    double acc[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < slots; k++) {
        HCG_CUDA(cudaEventSynchronize(c->ev[k][5]), "cudaEventSynchronize");
        for (int i = 0; i < 5; i++) {
            float t = 0;
            HCG_CUDA(cudaEventElapsedTime(&t, c->ev[k][i], c->ev[k][i + 1]), "cudaEventElapsedTime");
            acc[i] += t;
        }
    }
    for (int i = 0; i < 5 && i < cap; i++) ms[i] = acc[i] / slots;
    return HCG_OK;
}

namespace {
std::mutex g_tune_mu;
struct Tuned { int cells, chans, depth, path; };
std::map<std::tuple<int, int, int, int, int, int>, Tuned> g_tune_cache;

int bucket_log2(double x) { return x > 0 ? (int)floor(log2(x) * 2.0) : -999; }

// What the tuner's choice depends on: channels, storage type, samples per
// cell, support radius in cells (half-octave buckets), and whether the grid
// is projected (the staged and tensor paths take plain grids only).
std::tuple<int, int, int, int, int, int> tune_key(const hcg_ctx *c) {
    const double cells = (double)c->nx * c->ny;
    return std::make_tuple(c->nchan, c->store, bucket_log2((double)c->n / cells), bucket_log2(c->support / c->pix),
                           c->proj != HCG_CAR ? 1 : 0, c->nchan % 512 == 0 ? 512 : (c->nchan % 256 == 0 ? 256 : 0));
}

}  // namespace

}  // extern "C"

// The cached tuning for this field, if the tuner has seen its key.
bool autotune_cached(const hcg_ctx *c, int out[4]) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(c));
    if (it == g_tune_cache.end()) return false;
    out[0] = it->second.cells; out[1] = it->second.chans; out[2] = it->second.depth; out[3] = it->second.path;
    return true;
}

extern "C" {

hcg_status hcg_autotune(hcg_ctx *c, int force, int32_t *choice) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (!c->kernel_set || !c->grid_set || !c->loaded) return fail(HCG_ERR_NOT_READY, "kernel, grid and samples first");
    if (c->host_spec) return fail(HCG_ERR_UNSUPPORTED, "autotune needs device-resident spectra");
    auto report = [&]() {
        if (choice) { choice[0] = c->t_cells; choice[1] = c->t_chans; choice[2] = c->t_depth; choice[3] = c->t_path; }
    };
    int cached[4];
    if (!force && autotune_cached(c, cached)) {
        c->t_cells = cached[0]; c->t_chans = cached[1]; c->t_depth = cached[2]; c->t_path = cached[3];
        report();
        return HCG_OK;
    }
    // every applicable (cells per block, channels per thread, depth, path)
    std::vector<Tuned> cand;
    const int C = c->nchan;
    if (C >= 128) {
        for (Tuned t : {Tuned{32, 8, 12, HCG_PATH_GATHER}, Tuned{32, 8, 8, HCG_PATH_GATHER},
                        Tuned{32, 4, 8, HCG_PATH_GATHER}, Tuned{16, 8, 0, HCG_PATH_GATHER},
                        Tuned{16, 4, 0, HCG_PATH_GATHER}})
            cand.push_back(t);
    } else {
        cand.push_back({16, 4, 0, HCG_PATH_GATHER});
        cand.push_back({16, 1, 0, HCG_PATH_GATHER});
        if (C >= 8) cand.push_back({16, 8, 0, HCG_PATH_GATHER});
    }
    if (staged_supported(c, c->store, C))
        for (int cells : {32, 64})
            for (int depth : {16, 32}) cand.push_back({cells, 4, depth, HCG_PATH_STAGED});
    if (tc_supported(c, c->store)) cand.push_back({128, 0, 64, HCG_PATH_TENSOR});
    const Tuned saved{c->t_cells, c->t_chans, c->t_depth, c->t_path};
    cudaEvent_t e0, e1;
    HCG_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(HCG_ERR_CUDA, "cudaEventCreate"); }
    float best = 1e30f;
    Tuned pick = saved;
    c->tune_table.clear();
    c->tune_ms.clear();
    for (const Tuned &t : cand) {
        c->t_cells = t.cells; c->t_chans = t.chans; c->t_depth = t.depth; c->t_path = t.path;
        for (int v : {t.cells, t.chans, t.depth, t.path}) c->tune_table.push_back(v);
        c->tune_ms.push_back(-1.0f);
        bool ok = true;
        for (int r = 0; r < 2 && ok; r++) ok = hcg_grid(c) == HCG_OK;
        if (!ok) continue;
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3 && ok; r++) ok = hcg_grid(c) == HCG_OK;
        cudaEventRecord(e1, c->stream);
        if (!ok || cudaEventSynchronize(e1) != cudaSuccess || read_err(c) != HCG_OK) { cudaGetLastError(); continue; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        c->tune_ms.back() = ms / 3.0f;
        if (ms < best) { best = ms; pick = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best >= 1e30f) {
        c->t_cells = saved.cells; c->t_chans = saved.chans; c->t_depth = saved.depth; c->t_path = saved.path;
        return fail(HCG_ERR_CUDA, "autotune: no configuration ran");
    }
    c->t_cells = pick.cells; c->t_chans = pick.chans; c->t_depth = pick.depth; c->t_path = pick.path;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[tune_key(c)] = pick;
    }
    report();
    return hcg_sync(c);
}

hcg_status hcg_autotune_table(hcg_ctx *c, int32_t *choices, float *ms, int32_t cap, int32_t *count) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    const int32_t n = (int32_t)c->tune_ms.size();
    if (count) *count = n;
    if (cap < n) return fail(HCG_ERR_INVALID_ARG, "capacity below the number of timed candidates");
    if (n > 0 && (!choices || !ms)) return fail(HCG_ERR_INVALID_ARG, "null output");
    for (int32_t k = 0; k < n; k++) {
        for (int i = 0; i < 4; i++) choices[4 * k + i] = c->tune_table[4 * k + i];
        ms[k] = c->tune_ms[k];
    }
    return HCG_OK;
}

hcg_status hcg_debug_pix(hcg_ctx *c, int64_t *pix, uint32_t *perm, int64_t cap, int64_t *m_out) {
    hcg_info info;
    hcg_status s = hcg_get_info(c, &info);
    if (s) return s;
    if (c->last_path == HCG_PATH_SCATTER) return fail(HCG_ERR_STATE, "the scatter path builds no tables");
    if (m_out) *m_out = info.samples_kept;
    if (cap < info.samples_kept) return fail(HCG_ERR_INVALID_ARG, "capacity below M");
    if (info.samples_kept > 0) {
        if (pix) HCG_CUDA(cudaMemcpy(pix, c->tables()->psorted, info.samples_kept * 8, cudaMemcpyDeviceToHost), "copy P'");
        if (perm) HCG_CUDA(cudaMemcpy(perm, c->tables()->sc_row, info.samples_kept * 4, cudaMemcpyDeviceToHost), "copy perm");
    }
    return HCG_OK;
}

hcg_status hcg_debug_lut(hcg_ctx *c, int64_t *upix, int64_t *ustart, int64_t ucap, int64_t *u_out, int64_t *rstart,
                         int64_t rcap) {
    hcg_info info;
    hcg_status s = hcg_get_info(c, &info);
    if (s) return s;
    if (c->last_path == HCG_PATH_SCATTER) return fail(HCG_ERR_STATE, "the scatter path builds no tables");
    int64_t u = info.unique_pixels, nr = c->gp.r_hi - c->gp.r_lo + 2;
    if (u_out) *u_out = u;
    if (ucap < u || rcap < nr) return fail(HCG_ERR_INVALID_ARG, "capacity too small");
    if (u > 0) {
        HCG_CUDA(cudaMemcpy(upix, c->tables()->upix, u * 8, cudaMemcpyDeviceToHost), "copy upix");
        HCG_CUDA(cudaMemcpy(ustart, c->tables()->ustart, u * 8, cudaMemcpyDeviceToHost), "copy ustart");
    }
    ustart[u] = info.samples_kept;
    HCG_CUDA(cudaMemcpy(rstart, c->tables()->rstart, nr * 8, cudaMemcpyDeviceToHost), "copy rstart");
    return HCG_OK;
}

hcg_status hcg_debug_neighbours(hcg_ctx *c, int64_t cb, int64_t ce, int64_t *offsets, uint32_t *ids, int64_t cap) {
    hcg_info info;
    hcg_status s = hcg_get_info(c, &info);
    if (s) return s;
    if (c->last_path == HCG_PATH_SCATTER) return fail(HCG_ERR_STATE, "the scatter path builds no tables");
    int64_t cells = (int64_t)c->nx * c->ny;
    if (cb < 0 || ce > cells || cb > ce || !offsets) return fail(HCG_ERR_INVALID_ARG, "bad cell range");
    int64_t m = ce - cb;
    // device buffers of this call, freed on every return path
    struct Bufs {
        int64_t *cnt = nullptr, *off = nullptr;
        uint32_t *ids = nullptr;
        ~Bufs() { cudaFree(cnt); cudaFree(off); cudaFree(ids); }
    } d;
    HCG_CUDA(cudaMalloc((void **)&d.cnt, (m + 1) * 8), "cudaMalloc");
    HCG_CUDA(cudaMemsetAsync(d.cnt, 0, (m + 1) * 8, c->stream), "cudaMemset");
    if (launch_debug_neigh(c, c->gp, cb, ce, d.cnt, nullptr, nullptr, 0) < 0) return HCG_ERR_CUDA;
    std::vector<int64_t> cnt(m + 1);
    HCG_CUDA(cudaMemcpyAsync(cnt.data(), d.cnt, (m + 1) * 8, cudaMemcpyDeviceToHost, c->stream), "copy counts");
    HCG_CUDA(cudaStreamSynchronize(c->stream), "stream synchronise");
    offsets[0] = 0;
    for (int64_t k = 0; k < m; k++) offsets[k + 1] = offsets[k] + cnt[k];
    int64_t total = offsets[m];
    if (total > cap) return fail(HCG_ERR_INVALID_ARG, "sample_ids capacity too small");
    HCG_CUDA(cudaMalloc((void **)&d.off, (m + 1) * 8), "cudaMalloc");
    HCG_CUDA(cudaMalloc((void **)&d.ids, std::max<int64_t>(total, 1) * 4), "cudaMalloc");
    HCG_CUDA(cudaMemcpyAsync(d.off, offsets, (m + 1) * 8, cudaMemcpyHostToDevice, c->stream), "copy offsets");
    HCG_CUDA(cudaMemsetAsync(d.cnt, 0, (m + 1) * 8, c->stream), "cudaMemset");
    if (launch_debug_neigh(c, c->gp, cb, ce, d.cnt, d.off, d.ids, 1) < 0) return HCG_ERR_CUDA;
    if (total > 0)
        HCG_CUDA(cudaMemcpyAsync(ids, d.ids, total * 4, cudaMemcpyDeviceToHost, c->stream), "copy ids");
    HCG_CUDA(cudaStreamSynchronize(c->stream), "debug neighbours");
    for (int64_t k = 0; k < m; k++) std::sort(ids + offsets[k], ids + offsets[k + 1]);
    return read_err(c);
}

}  // extern "C"

// Copy channels [c0, c0 + nc) of every cell of the device cube (and, if
// asked, the weights) into the bound host outputs on out_stream, after the
// work enqueued so far on c->stream; ev_out_done marks the copies' end.
hcg_status enqueue_host_output(hcg_ctx *c, int32_t c0, int32_t nc, int slot, bool weights) {
    if (!c->host_cube) return HCG_OK;
    const size_t cells = (size_t)c->nx * c->ny, C = (size_t)c->nchan;
    HCG_CUDA(cudaEventRecord(c->ev_gathered[slot], c->stream), "record event");
    HCG_CUDA(cudaStreamWaitEvent(c->out_stream, c->ev_gathered[slot], 0), "wait for gather");
    if (cells > 0) {
        if ((int32_t)C == nc)
            HCG_CUDA(cudaMemcpyAsync(c->host_cube, c->cube(), cells * C * 4, cudaMemcpyDeviceToHost, c->out_stream),
                     "copy cube out");
        else
            HCG_CUDA(cudaMemcpy2DAsync(c->host_cube + c0, C * 4, c->cube() + c0, C * 4, (size_t)nc * 4, cells,
                                       cudaMemcpyDeviceToHost, c->out_stream),
                     "copy cube window out");
        if (weights)
            HCG_CUDA(cudaMemcpyAsync(c->host_w, c->weights(), cells * 4, cudaMemcpyDeviceToHost, c->out_stream),
                     "copy weights out");
    }
    HCG_CUDA(cudaEventRecord(c->ev_out_done, c->out_stream), "record event");
    return HCG_OK;
}

// ---- stages of hcg_grid ----------------------------------------------------
// The gather of the pass's path (c->last_path) with its tuning.
int launch_pass_gather(hcg_ctx *c, const void *spec, int dtype, const float *scale) {
    switch (c->last_path) {
        case HCG_PATH_TENSOR: return launch_tc_gather(c, c->gp, spec, dtype, scale);
        case HCG_PATH_SCATTER: return launch_scatter(c, c->gp, spec, dtype, scale);
        case HCG_PATH_STAGED:
            return launch_staged(c, c->gp, spec, dtype, scale, c->e_cells, c->e_depth);
        default: return launch_gather(c, c->gp, spec, dtype, scale);
    }
}

// Host-side preparation: checks, parameters of the pass, scratch, path.
hcg_status grid_prepare(hcg_ctx *c) {
    hcg_status s = check_ctx(c);
    if (s) return s;
    if (!c->kernel_set) return fail(HCG_ERR_NOT_READY, "hcg_set_kernel not called");
    if (!c->grid_set) return fail(HCG_ERR_NOT_READY, "hcg_set_grid not called");
    if (!c->loaded) return fail(HCG_ERR_NOT_READY, "hcg_load_samples not called");
    if (c->store != c->in_dtype && c->in_dtype != HCG_F32)
        return fail(HCG_ERR_INVALID_ARG, "storage type incompatible with the loaded spectra");
    if ((double)c->nx * c->ny * c->nchan > 4.0e18) return fail(HCG_ERR_INVALID_ARG, "cube size overflows");
    GridParams g;
    int key_bits;
    make_params(c, g, key_bits);
    if ((s = ensure_scratch(c, g))) return s;
    c->stream_win = c->host_spec ? pick_stream_window(c) : 0;
    c->gp = g;
    c->key_bits = key_bits;
    const int dtype = c->store;
    // tuning in effect: as set; on the automatic path the tuner's cached
    // choice for this field when it has one (and it applies to this pass),
    // else the tensor path where it applies and the gather otherwise
    int path = c->t_path, tune[4] = {c->t_cells, c->t_chans, c->t_depth, c->t_path};
    if (path == HCG_PATH_AUTO && autotune_cached(c, tune)) {
        const int p = tune[3];
        const int32_t win = c->host_spec ? c->stream_chunk_chans() : c->nchan;
        const bool applies = p == HCG_PATH_GATHER || (p == HCG_PATH_TENSOR && tc_supported(c, dtype)) ||
                             (p == HCG_PATH_STAGED && staged_supported(c, dtype, win));
        if (applies) path = p;
        else tune[0] = tune[1] = tune[2] = 0;
    }
    // (FP32 storage stays on the plain CUDA-core gather unless tuned or asked)
    if (path == HCG_PATH_AUTO) path = dtype != HCG_F32 && tc_supported(c, dtype) ? HCG_PATH_TENSOR : HCG_PATH_GATHER;
    c->e_cells = tune[0]; c->e_chans = tune[1]; c->e_depth = tune[2];
    if (path == HCG_PATH_STAGED) {
        if (!c->e_cells) c->e_cells = 64;
        if (!c->e_depth) c->e_depth = 32;
        c->e_chans = 4;
    }
    if (path == HCG_PATH_SCATTER && (int64_t)c->nx * c->ny > 0xFFFFFFFFll)
        return fail(HCG_ERR_UNSUPPORTED, "scatter path: more than 2^32 cells");
    if (path == HCG_PATH_SCATTER && c->proj != HCG_CAR)
        return fail(HCG_ERR_UNSUPPORTED, "the scatter path takes HCG_CAR grids only");
    if (path == HCG_PATH_TENSOR && !tc_supported(c, dtype))
        return fail(HCG_ERR_UNSUPPORTED, "tensor path needs an HCG_CAR grid and nchan a multiple of 256");
    if (path == HCG_PATH_STAGED && !staged_supported(c, dtype, c->host_spec ? c->stream_chunk_chans() : c->nchan))
        return fail(HCG_ERR_UNSUPPORTED,
                    "staged path needs an HCG_CAR grid, 128+ channels (per streamed window) in 16-byte rows");
    c->last_path = path;
    return HCG_OK;
}

// Enqueue ingest, pixel keys, sort, S' data and both tables on c->stream.
hcg_status grid_enqueue_front(hcg_ctx *c, const void **spec_out, int *dtype_out, const float **scale_out) {
    const GridParams &g = c->gp;
    HCG_CUDA(cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream), "reset error word");
    HCG_CUDA(cudaMemsetAsync(c->dscal, 0, 8 * sizeof(int64_t), c->stream), "reset counters");
    int launches = 0, k;
    const int slot = c->prof_calls % hcg_ctx::kProfSlots;
    auto mark = [&](int i) { if (c->profiling) cudaEventRecord(c->ev[slot][i], c->stream); };
    mark(0);
    const void *spec = c->spec_in;
    int dtype = c->in_dtype;
    const float *scale = c->scale_in;
    if (c->store != c->in_dtype && !c->host_spec) {
        if ((k = launch_quantise(c)) < 0) return HCG_ERR_CUDA;
        launches += k;
        spec = c->q_spec;
        dtype = c->store;
        scale = c->store == HCG_E4M3 ? c->q_scale : nullptr;
    }
    mark(1);
    // the scatter path needs no pre-ordering; a field sharing another's tables builds none
    const bool tables = c->last_path != HCG_PATH_SCATTER && !c->tables_src;
    if (tables && (k = launch_prep(c, g, c->key_bits)) < 0) return HCG_ERR_CUDA;
    if (tables) launches += k;
    mark(2);
    if (tables && (k = launch_sort(c, c->n, c->key_bits)) < 0) return HCG_ERR_CUDA;
    if (tables) launches += k;
    mark(3);
    if (tables && (k = launch_permute_lut(c, g)) < 0) return HCG_ERR_CUDA;
    if (tables) launches += k;
    mark(4);
    c->last_launches = launches;
    *spec_out = spec;
    *dtype_out = dtype;
    *scale_out = scale;
    return HCG_OK;
}

// Channels per streamed window.  Set by hcg_set_stream_chunk, else: all
// channels up to 512 (one contiguous copy); otherwise two windows of half the
// channels in whole 256-channel slices -- a window's copy is a 2-D copy of
// one row segment per sample, and the host link moves wide segments much
// faster than narrow ones (measured: 512-byte segments at about a third of
// the speed of 2-4 KB ones) -- narrowed, 256 channels at a time, while the
// two windows (and their quantised copies) would take more than a quarter of
// the free device memory.
int32_t pick_stream_window(hcg_ctx *c) {
    const int32_t C = c->nchan;
    if (c->stream_chunk > 0) return std::min(c->stream_chunk, C);
    if (C <= 512) return C;
    const int64_t ies = c->in_dtype == HCG_F32 ? 4 : (c->in_dtype == HCG_BF16 ? 2 : 1);
    const int64_t ses = c->store == c->in_dtype ? 0 : (c->store == HCG_BF16 ? 2 : 1);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); free_b = 0; }
    // windows already allocated by an earlier pass count as free
    free_b += c->stage_cap[0] + c->stage_cap[1] + c->qstage_cap[0] + c->qstage_cap[1];
    int64_t w = ((int64_t)(C + 1) / 2 + 255) / 256 * 256;
    while (w > 256 && 2 * c->n * w * (ies + ses) > (int64_t)(free_b / 4)) w -= 256;
    return (int32_t)std::min<int64_t>(w, C);
}

// Streamed spectra: for each channel window [c0, c0 + nc), copy the host
// rows' window into stage[k & 1] on copy_stream (a 2-D copy: nc channels of
// each of the n rows), quantise it if the storage type asks, and gather it
// on c->stream into the cube's channels [c0, c0 + nc).  Two windows are in
// flight: the copy of window k waits until the gather of window k - 2 has
// released its buffer, and the gather of window k waits for its copy.
hcg_status grid_enqueue_streamed(hcg_ctx *c) {
    hcg_status s;
    const int32_t C = c->nchan, W = c->stream_chunk_chans();
    const size_t ies = c->in_dtype == HCG_F32 ? 4 : (c->in_dtype == HCG_BF16 ? 2 : 1);
    const size_t ses = c->store == HCG_F32 ? 4 : (c->store == HCG_BF16 ? 2 : 1);
    const size_t n = (size_t)c->n;
    if (!c->copy_stream) {
        HCG_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "create copy stream");
        for (int k = 0; k < 2; k++) {
            HCG_CUDA(cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming), "create event");
            HCG_CUDA(cudaEventCreateWithFlags(&c->ev_consumed[k], cudaEventDisableTiming), "create event");
        }
    }
    for (int k = 0; k < 2; k++) {
        if ((s = grow_bytes(c, &c->stage[k], c->stage_cap[k], n * W * ies, "streamed window"))) return s;
        if (c->store != c->in_dtype &&
            (s = grow_bytes(c, &c->qstage[k], c->qstage_cap[k], n * W * ses, "quantised streamed window")))
            return s;
    }
    // ev_consumed[b] still marks the last gather of the previous hcg_grid
    // that read stage[b] (never recorded: complete), so the first copies
    // start at once and overlap the pixel keys, sort and tables
    int launches = 0;
    for (int32_t c0 = 0, k = 0; c0 < C; c0 += W, k++) {
        const int32_t nc = std::min(W, C - c0);
        const int b = k & 1;
        HCG_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_consumed[b], 0), "wait for window buffer");
        if (n > 0 && nc == C)
            HCG_CUDA(cudaMemcpyAsync(c->stage[b], c->host_spec, n * C * ies, cudaMemcpyHostToDevice, c->copy_stream),
                     "copy spectra");
        else if (n > 0)
            HCG_CUDA(cudaMemcpy2DAsync(c->stage[b], nc * ies, static_cast<const char *>(c->host_spec) + c0 * ies,
                                       (size_t)C * ies, nc * ies, n, cudaMemcpyHostToDevice, c->copy_stream),
                     "copy spectra window");
        HCG_CUDA(cudaEventRecord(c->ev_copied[b], c->copy_stream), "record event");
        HCG_CUDA(cudaStreamWaitEvent(c->stream, c->ev_copied[b], 0), "wait for window copy");
        const void *spec = c->stage[b];
        int dtype = c->in_dtype;
        const float *scale = c->in_dtype == HCG_E4M3 ? c->scale_in + c0 : nullptr;
        if (c->store != c->in_dtype) {
            int q = launch_quantise_span(c, static_cast<const float *>(c->stage[b]), c->n, nc, c->qstage[b],
                                         c->store == HCG_E4M3 ? c->q_scale + c0 : nullptr,
                                         c->store == HCG_E4M3 ? c->q_amax + c0 : nullptr);
            if (q < 0) return HCG_ERR_CUDA;
            launches += q;
            spec = c->qstage[b];
            dtype = c->store;
            scale = c->store == HCG_E4M3 ? c->q_scale + c0 : nullptr;
        }
        c->win_c0 = c0; c->win_nc = nc;
        int g = launch_pass_gather(c, spec, dtype, scale);
        c->win_c0 = 0; c->win_nc = 0;
        if (g < 0) return HCG_ERR_CUDA;
        launches += g;
        HCG_CUDA(cudaEventRecord(c->ev_consumed[b], c->stream), "record event");
        if ((s = enqueue_host_output(c, c0, nc, b, k == 0))) return s;
    }
    c->last_launches += launches;
    const int slot = c->prof_calls % hcg_ctx::kProfSlots;
    if (c->profiling) {
        cudaEventRecord(c->ev[slot][5], c->stream);
        c->prof_calls++;
    }
    c->gridded = true;
    return HCG_OK;
}

// Enqueue the gather of the path chosen by grid_prepare.
hcg_status grid_enqueue_gather(hcg_ctx *c, const void *spec, int dtype, const float *scale) {
    const int k = launch_pass_gather(c, spec, dtype, scale);
    if (k < 0) return HCG_ERR_CUDA;
    c->last_launches += k;
    const int slot = c->prof_calls % hcg_ctx::kProfSlots;
    if (c->profiling) {
        cudaEventRecord(c->ev[slot][5], c->stream);
        c->prof_calls++;
    }
    c->gridded = true;
    return HCG_OK;
}


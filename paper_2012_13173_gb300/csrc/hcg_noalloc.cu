// hcg_noalloc.cu -- hcg_preorder_noalloc: the pre-ordering step (HEALPix pixel
// of every sample and the stable radix sort by pixel) for callers that cannot
// allocate device memory.  Its scratch lives in one file-scope __device__
// array, allocated with the module when the library is loaded on a device.
#include <mutex>

#include "hcg_internal.h"

namespace {

constexpr int64_t kMaxKeys = HCG_NOALLOC_MAX_SAMPLES;
constexpr int64_t kTiles = (kMaxKeys + 2047) / 2048;          // radix-sort tiles of 2048 keys
constexpr int64_t kCounts = 256 * kTiles;                     // per-tile digit counts
constexpr int64_t kSums = (kCounts + 4095) / 4096;            // second level of the count scan
constexpr size_t kOffKeys = 0;                                // uint64 keys, ping-pong half
constexpr size_t kOffVals = kOffKeys + kMaxKeys * 8;          // uint32 values, ping-pong half
constexpr size_t kOffCounts = kOffVals + kMaxKeys * 4;
constexpr size_t kOffSums = kOffCounts + kCounts * 4;
constexpr size_t kOffErr = kOffSums + ((kSums * 4 + 255) / 256) * 256;
constexpr size_t kBytes = kOffErr + 256;
static_assert(kBytes == HCG_NOALLOC_SCRATCH_BYTES, "header and scratch layout disagree");

// The scratch itself: one copy per device that loads this library, kept
// until the process exits.  Host code must not take its address directly
// (that is a host-side stand-in); set_up() asks the runtime for the device
// address.
static __device__ __align__(256) unsigned char g_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of g_scratch.
hcg_status set_up(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return HCG_OK;
}

int64_t ring_first(int64_t ns, int64_t r) {
    if (r <= ns) return 2 * r * (r - 1);
    if (r <= 3 * ns) return 2 * ns * (ns - 1) + (r - ns) * 4 * ns;
    int64_t q = 4 * ns - r;
    return 12 * ns * ns - 2 * q * (q + 1);
}

}  // namespace

extern "C" hcg_status hcg_preorder_noalloc(const double *lon_deg, const double *lat_deg, int64_t n, int64_t nside,
                                           int64_t ring_lo, int64_t ring_hi, int64_t *pix_sorted, uint32_t *perm,
                                           void *cuda_stream) {
    if (n < 0) { hcg_set_error("n must be >= 0"); return HCG_ERR_INVALID_ARG; }
    if (n > kMaxKeys) {
        hcg_set_error("hcg_preorder_noalloc: n exceeds HCG_NOALLOC_MAX_SAMPLES (262144); use hcg_grid instead");
        return HCG_ERR_INVALID_ARG;
    }
    if (nside < 1 || nside > ((int64_t)1 << 24) || (nside & (nside - 1))) {
        hcg_set_error("nside must be a power of two in [1, 2^24]");
        return HCG_ERR_INVALID_ARG;
    }
    if (ring_lo < 1 || ring_hi > 4 * nside - 1 || ring_lo > ring_hi) {
        hcg_set_error("ring range must satisfy 1 <= ring_lo <= ring_hi <= 4 nside - 1");
        return HCG_ERR_INVALID_ARG;
    }
    if (n > 0 && (!lon_deg || !lat_deg || !pix_sorted || !perm)) {
        hcg_set_error("null pointer");
        return HCG_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) { hcg_set_error("device ordinal beyond 63"); return HCG_ERR_UNSUPPORTED; }
    if (n > 0) {
        hcg_status c;
        if ((c = check_device_ptr(lon_deg, dev, "lon_deg")) || (c = check_device_ptr(lat_deg, dev, "lat_deg")) ||
            (c = check_device_ptr(pix_sorted, dev, "pix_sorted")) || (c = check_device_ptr(perm, dev, "perm")))
            return c;
    }
    unsigned char *scr = nullptr;
    hcg_status s = set_up(dev, &scr);
    if (s) return s;
    if (n == 0) return HCG_OK;

    // the same key layout as hcg_grid: (pixel - first pixel of ring_lo) above
    // a 32-bit coordinate hash, as many bits as the ring range needs
    GridParams gp{};
    gp.nside = nside;
    gp.r_lo = ring_lo;
    gp.r_hi = ring_hi;
    gp.pix_lo = ring_first(nside, ring_lo);
    const int64_t npr = ring_first(nside, ring_hi + 1) - gp.pix_lo;
    int bits = 1;
    while (bits < 62 && ((int64_t)1 << bits) - 1 < npr) bits++;
    const int key_bits = bits + 32;
    if (key_bits > 64) {
        // hcg_grid sorts such ranges in two digit phases with a pixel-offset
        // array beside the keys; this fixed scratch has no room for it
        hcg_set_error("hcg_preorder_noalloc: the ring range spans 2^32 pixels or more; use hcg_grid instead");
        return HCG_ERR_UNSUPPORTED;
    }
    const int passes = (key_bits + 7) / 8;

    // ping-pong between the caller's outputs and the scratch; start where an
    // even or odd number of passes leaves the result in the outputs
    uint64_t *const k[2] = {reinterpret_cast<uint64_t *>(pix_sorted), reinterpret_cast<uint64_t *>(scr + kOffKeys)};
    uint32_t *const v[2] = {perm, reinterpret_cast<uint32_t *>(scr + kOffVals)};
    const int first = passes & 1;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int *err = reinterpret_cast<int *>(scr + kOffErr);
    e = cudaMemsetAsync(err, 0, sizeof(int), st);     // the only state a call reads before writing it
    if (e != cudaSuccess) return hcg_cuda_fail(e, "cudaMemsetAsync");
    int fin = preorder_on_buffers(lon_deg, lat_deg, n, gp, key_bits, k, v, first,
                                  reinterpret_cast<uint32_t *>(scr + kOffCounts),
                                  reinterpret_cast<uint32_t *>(scr + kOffSums), err, st);
    if (fin < 0) return HCG_ERR_CUDA;
    if (fin != 0) { hcg_set_error("internal: sorted keys did not land in the outputs"); return HCG_ERR_CUDA; }
    return HCG_OK;
}

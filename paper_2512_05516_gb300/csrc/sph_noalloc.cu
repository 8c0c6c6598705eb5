// Allocation-free cell binning.  Some callers cannot allocate device memory
// at all -- a plugin inside a host application that owns the whole device
// memory pool and offers plugins no allocation hook, or a latency-critical
// path where cudaMalloc's implicit device-wide synchronisation is not
// acceptable -- and so cannot provide the workspace that sph_create needs.
// This entry point bins their particles with the scratch memory held in a
// fixed device array of this library (SPH_NOALLOC_SCRATCH_BYTES, about
// 5.3 MiB, resident on every device that loads the library until the
// process exits).  The caller still passes the inputs and the outputs.
#include <mutex>

#include "sph_internal.cuh"

namespace {

constexpr int64_t kMaxN = SPH_NOALLOC_MAX_PARTICLES;
constexpr int64_t kMaxCells = SPH_NOALLOC_MAX_CELLS;
constexpr int64_t kMaxBlk = (kMaxN + sph::kRadixTile - 1) / sph::kRadixTile;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// byte offsets of the scratch arrays inside the fixed array
constexpr size_t kOffKeys0 = 0;
constexpr size_t kOffKeys1 = kOffKeys0 + align256(4 * kMaxN);
constexpr size_t kOffVals0 = kOffKeys1 + align256(4 * kMaxN);
constexpr size_t kOffVals1 = kOffVals0 + align256(4 * kMaxN);
constexpr size_t kOffCount = kOffVals1 + align256(4 * kMaxN);
constexpr size_t kOffGhist = kOffCount + align256(4 * kMaxCells);
constexpr size_t kOffPart = kOffGhist + align256(4 * (256 * kMaxBlk + 1));
constexpr int64_t kPartLen = (max64(256 * kMaxBlk, kMaxCells + 1) + sph::kScanTile - 1) / sph::kScanTile + 2;
constexpr size_t kOffStats = kOffPart + align256(4 * kPartLen);
constexpr size_t kScratchBytes = kOffStats + align256(sizeof(sph::DevStats));
static_assert(kScratchBytes <= SPH_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the documented size");

static __device__ __align__(256) unsigned char g_bin_scratch[SPH_NOALLOC_SCRATCH_BYTES];

// Device address of g_bin_scratch, per device.  In host code the symbol names
// a host-side stand-in, never the device array, so only these addresses are
// handed to kernels.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// One-time set-up on the current device; returns null on failure.
unsigned char *scratch_on(int dev)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bin_scratch) != cudaSuccess || !p) return nullptr;
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    return g_scratch_addr[dev];
}

}  // namespace

extern "C" sph_status sph_bin_cells_noalloc(const void *d_aos, const sph_aos_layout *layout, int64_t n,
                                            const double *box, const int32_t *nc, int32_t *d_perm,
                                            int32_t *d_cell_of_slot, int32_t *d_cell_start, void *stream)
{
    if (!layout || !box || !nc || !d_cell_start) return SPH_EINVAL;
    if (n < 0 || (n > 0 && (!d_aos || !d_perm || !d_cell_of_slot))) return SPH_EINVAL;
    if (layout->record_bytes <= 0 || layout->record_bytes % 8 != 0) return SPH_EINVAL;
    const int32_t xoff = layout->offset[SPH_F_X];
    if (xoff < 0 || xoff % 8 != 0 || layout->type[SPH_F_X] != SPH_AOS_F64 || xoff + 24 > layout->record_bytes)
        return SPH_EINVAL;
    if (((uintptr_t)d_aos & 7) != 0) return SPH_EINVAL;
    int64_t ncell = 1;
    for (int k = 0; k < 3; ++k) {
        if (!(box[k] > 0.0) || !(box[k] < 1e300) || nc[k] < 1) return SPH_EINVAL;
        ncell *= nc[k];
        if (ncell > kMaxCells) return SPH_ENOSPACE;
    }
    if (n > kMaxN) return SPH_ENOSPACE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SPH_ECUDA;
    unsigned char *s = scratch_on(dev);
    if (!s) return SPH_ECUDA;

    sph::BinRaw b;
    b.aos = (const uint8_t *)d_aos;
    b.n = n;
    b.stride = layout->record_bytes;
    b.xoff = xoff;
    for (int k = 0; k < 3; ++k) {
        b.nc[k] = nc[k];
        b.box[k] = box[k];
        b.inv[k] = (double)nc[k] / box[k];
    }
    b.ncell = ncell;
    b.keys[0] = (int32_t *)(s + kOffKeys0);
    b.keys[1] = (int32_t *)(s + kOffKeys1);
    b.vals[0] = (int32_t *)(s + kOffVals0);
    b.vals[1] = (int32_t *)(s + kOffVals1);
    b.count = (int32_t *)(s + kOffCount);
    b.ghist = (uint32_t *)(s + kOffGhist);
    b.scan_part = (int32_t *)(s + kOffPart);
    b.st = (sph::DevStats *)(s + kOffStats);
    b.out_perm = d_perm;
    b.out_cell = d_cell_of_slot;
    b.out_start = d_cell_start;
    if (sph::bin_raw(b, (cudaStream_t)stream) != cudaSuccess) return SPH_ECUDA;
    return SPH_OK;
}

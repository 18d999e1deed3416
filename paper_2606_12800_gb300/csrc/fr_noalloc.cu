// fr_noalloc.cu -- fr_route_d8_noalloc: D8 routing (receivers + exact
// accumulation) for callers that may not allocate device memory.
//
// Who needs it: a host application that hands a plugin only its input and
// output buffers, a program whose own pool allocator has already reserved the
// device memory (so cudaMalloc fails or fragments it), and loops that cannot
// afford cudaMalloc/cudaFree implicitly synchronising the device.  Such a
// caller passes inputs and outputs only; the workspace fr_route_d8 needs
// lives here instead, in one file-scope device array of fixed size.
//
// The array is reached through cudaGetSymbolAddress once per device (the
// first call of the entry point on that device, with that device current);
// the address is cached per device ordinal.  Nothing here calls cudaMalloc,
// cudaFree or any allocating routine.  Every call on a device shares the one
// array, which keeps the previous call's contents: the region the engine
// needs zeroed is cleared by fr_route_d8's own memset on the caller's stream,
// so back-to-back calls are fine, but calls whose GPU work overlaps (two
// streams, or two host threads on one device) race on the array.
#include <mutex>

#include "../../include/fr.h"

namespace {

// Workspace bytes fr_route_d8 needs on FR_NOALLOC_MAX_CELLS cells: the
// per-cell regions (1 + 1/8 + 4 + 8 + 8 + 1 bytes, each rounded up to 256)
// plus the fixed header and mass-balance partials.  The size is re-checked
// against fr_workspace_size on every call.
constexpr size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kMaxCells = (size_t)FR_NOALLOC_MAX_CELLS;
constexpr size_t kScratchBytes = 256 + round256(kMaxCells + 4) + round256((kMaxCells + 31) / 32 * 4) +
                                 round256(kMaxCells * 4) + 2 * round256(kMaxCells * 8) +
                                 round256(kMaxCells) + round256(1024 * 3 * 8) + 4096;

// The scratch itself: every GPU that loads this module holds it until the
// process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

fr_status scratch_for_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FR_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return FR_ERR_CUDA;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return FR_OK;
}

}  // namespace

extern "C" {

fr_status fr_route_d8_noalloc(const float* dem, int64_t nx, int64_t ny, double dx, uint32_t flags,
                              const float* rain, float* w_out, float* w_lo_out,
                              uint64_t* area_out, uint8_t* dir_out, void* stream) {
    if (nx < 1 || ny < 1 || nx > FR_NOALLOC_MAX_CELLS || ny > FR_NOALLOC_MAX_CELLS ||
        nx * ny > FR_NOALLOC_MAX_CELLS)
        return FR_ERR_INVALID_ARG;
    const size_t need = fr_workspace_size(FR_OP_ROUTE, nx, ny, flags);
    if (need == 0) return FR_ERR_INVALID_ARG;
    if (need > kScratchBytes) return FR_ERR_WORKSPACE;
    void* ws = nullptr;
    const fr_status st = scratch_for_current_device(&ws);
    if (st != FR_OK) return st;
    return fr_route_d8(dem, nx, ny, dx, flags, rain, w_out, w_lo_out, area_out, dir_out, ws,
                       kScratchBytes, stream);
}

}  // extern "C"

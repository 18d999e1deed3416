// fr_internal.h -- host-side interfaces between the translation units of libfr.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "fr_device.cuh"

namespace fr {


// Local flow routing (fr_receivers.cu).
cudaError_t launch_receivers_d8(const float* z, int64_t nx, int64_t ny, double dx,
                                uint32_t flags, uint8_t* dir, uint8_t* indeg, cudaStream_t s);
cudaError_t launch_receivers_mfd(const float* z, int64_t nx, int64_t ny, double dx, double p,
                                 uint32_t flags, uint8_t* mask, float* frac, uint8_t* indeg,
                                 cudaStream_t s);
// Counts non-finite elevations into *count (device, zeroed by the caller).
cudaError_t launch_count_nonfinite(const float* z, int64_t n, unsigned long long* count,
                                   cudaStream_t s);

// Per-problem description consumed by the tile engine (fr_engine.cuh).
struct Prob {
    int64_t nx, ny;
    const uint8_t* rb;     // routing bytes: D8 codes or MFD masks
    const float* z;        // MFD elevations (receivers of batched tiles)
    const float* frac;     // MFD fractions [cell * 8 + code], see mfd_fracs8
    const float* init;     // forward: rain (NULL = unit); adjoint: dL/dw (NULL = sink loss)
    const float* wf;       // adjoint: forward water (leading word)
    const float* wf_lo;    // adjoint: forward water (trailing word) or NULL
    float* out_hi;         // value leading word (w or dL/dr) or NULL
    float* out_lo;         // value trailing word (user output or workspace)
    uint64_t* area;        // D8 forward unit-rain areas or NULL
    uint32_t* cnt;         // packed byte arrival counters, zeroed before the launch
    int64_t* link;         // 8 B/cell scratch: frontier buffer of the global rounds
    uint32_t* gbits;       // one bit per cell: "global" (solved by the walkers), zeroed
    unsigned long long* glist;  // compact list of global cells (pid << 40 | cell)
    int64_t glist_cap;     // capacity of glist (entries)
    MfdConst mc;
    int32_t lo_full;       // out_lo is a user output: write it for every cell
    // D8 forward global phase: the tile-skeleton solve (fr_skel.cu) runs when
    // the local phase leaves at least skel_min global cells, the cell walkers
    // otherwise (~0: walkers always)
    unsigned long long skel_min;
    uint16_t* skpool;               // dependency slots, kSkelPool per skeleton tile
    unsigned long long* skstarts;   // exits that start a skeleton walker
    uint32_t* sktiles;              // skeleton tiles holding global cells
};

// Device-wide bookkeeping kept at the start of the workspace; zeroed (with
// the arrival counters that follow it) before every engine launch.
struct EngineGlobals {
    unsigned long long done_cells;   // cells whose value was computed
    unsigned long long work_next;    // batched: next tile to claim
    unsigned long long nonfinite;    // FR_CHECK_FINITE: count of NaN/Inf inputs
    unsigned int finished_ctas;      // walker CTAs that have left the kernel
    unsigned int status;             // fr_status of the device-side checks
    unsigned long long glist_count;  // entries in the global-cell list
    unsigned long long recv_next;    // batched receivers: next tile to claim
    unsigned long long total_cells;  // batched: cells of all problems (set on the device)
    unsigned long long fcount[3];    // level-synchronous global phase: frontier sizes
    unsigned int bar_count;          // grid barrier: blocks arrived
    unsigned int bar_gen;            // grid barrier: generation
    unsigned long long rounds;       // level-synchronous global phase: rounds run (diagnostic)
    unsigned long long skel_tiles;   // skeleton solve: tiles listed in Prob::sktiles
    unsigned long long sink_area;    // D8 areas: sum of the areas of the FR_SINK cells the local phase finished
    unsigned long long pad[2];
};
static_assert(sizeof(EngineGlobals) == 128, "globals block is 128 bytes (256 reserved)");

enum class Mode : int { FwdD8 = 0, FwdMfd = 1, AdjD8 = 2, AdjMfd = 3 };

// Grid of the D8 forward walker kernel (fr_accumulate.cu).
int walker_grid();
// Time a device-side wait may take before the call reports
// FR_ERR_NO_PROGRESS (fr_set_wait_limit; fr_api.cu).
unsigned long long wait_limit_ns();
// Reads and clears the flag a TMA wait that ran out leaves (fr_receivers.cu);
// synchronises the stream.
cudaError_t read_clear_tma_error(unsigned* out, cudaStream_t s);
// Linear receiver index of every cell from D8 codes (fr_receivers.cu).
cudaError_t launch_receiver_index(const uint8_t* dir, int64_t nx, int64_t ny, bool wide, void* out,
                                  cudaStream_t s);
// Skeleton tiles of the D8 global phase (fr_skel.cu): kSkelTile x kSkelTile
// cells; kSkelPool dependency slots per tile (a dependency is a donor in the
// one-cell ring around the tile, and each ring cell has one receiver).
constexpr int kSkelTile = 64;
constexpr int kSkelPool = 4 * kSkelTile + 4;
__host__ __device__ inline int64_t skel_tiles(int64_t nx, int64_t ny) {
    return ((nx + kSkelTile - 1) / kSkelTile) * ((ny + kSkelTile - 1) / kSkelTile);
}
// Skeleton solve of the global cells left by the D8 forward local phase;
// every kernel returns at once unless the global-cell count reaches
// prob.skel_min.
cudaError_t launch_d8_skeleton(bool want_w, bool want_area, const Prob& prob, EngineGlobals* g,
                               cudaStream_t s);
// D8 forward: halo-tile local phase (fr_d8.cu) + walker phase.
cudaError_t launch_d8_forward(bool want_w, bool want_area, const Prob& prob, EngineGlobals* g,
                              cudaStream_t s);
// MFD forward: halo-tile local phase (fr_halo.cu) + level-synchronous global phase.
cudaError_t launch_mfd_forward(const Prob& prob, EngineGlobals* g, cudaStream_t s);
// Adjoint of D8 or MFD routing: halo-tile local phase (fr_halo.cu) + global phase.
cudaError_t launch_adjoint(bool mfd, const Prob& prob, EngineGlobals* g, cudaStream_t s);
// Batched forms: one CTA per tile of every problem (tile_prefix over the
// halo geometry geo, see halo_tiles), then one global phase.
cudaError_t launch_d8_forward_batch(int geo, bool want_w, bool want_area, const Prob* probs_dev,
                                    const int64_t* tile_prefix_dev, int nprob, int64_t total_tiles,
                                    unsigned long long total_cells, EngineGlobals* g,
                                    cudaStream_t s);
cudaError_t launch_mfd_forward_batch(const Prob* probs_dev, const int64_t* tile_prefix_dev,
                                     int nprob, int64_t total_tiles,
                                     unsigned long long total_cells, EngineGlobals* g,
                                     cudaStream_t s);
cudaError_t launch_mfd_grad_z(const Prob& prob, const float* g_hi, const float* g_lo,
                              float* dLdz, cudaStream_t s);
cudaError_t launch_mass_balance(int kind, int64_t nx, int64_t ny, const uint8_t* rb,
                                const float* rain, const float* w, const float* w_lo,
                                const uint64_t* area, double* partials, int nblocks,
                                double* out, cudaStream_t s);
// D8 areas (fr_mass_balance with FR_SINK_SUMS_IN_WORKSPACE): the area term from
// the local phase's sink sum and the global cells' sinks, the rain term from
// `rain` (a full pass) or the cell count.
cudaError_t launch_mass_balance_ws(int64_t nx, int64_t ny, const uint8_t* rb, const float* rain,
                                   const uint64_t* area, const uint32_t* gbits,
                                   const EngineGlobals* G, double* partials, int nblocks,
                                   double* out, cudaStream_t s);
// Richardson I+X (fr_richardson.cu): one sweep prev -> next over 64x32
// subdomains (counts[0] += changed cells, counts[1] += finalised cells), and
// the copy of converged two-float values into the outputs.
cudaError_t richardson_sweep(bool mfd, const Prob& P, const float2* prev, float2* next,
                             unsigned long long* counts, cudaStream_t s);
cudaError_t richardson_output(const float2* v, int64_t n, float* hi, float* lo, cudaStream_t s);
// Depression filling (fr_fill.cu): F = z on the edge and +inf inside, then one
// relaxation sweep over 64x32 tiles; *changed counts the tiles that moved and
// act_next[t] records it per tile (act_prev: the previous sweep's record,
// unused when first).
int64_t fill_tiles(int64_t nx, int64_t ny);
cudaError_t fill_init(const float* z, int64_t nx, int64_t ny, float* F, cudaStream_t s);
cudaError_t fill_sweep(const float* z, int64_t nx, int64_t ny, float* F, const uint8_t* act_prev,
                       uint8_t* act_next, bool first, unsigned long long* changed, cudaStream_t s);
cudaError_t launch_mfd_fractions(const float* z, const uint8_t* mask, int64_t nx, int64_t ny,
                                 double dx, double p, uint32_t flags, float* frac, cudaStream_t s);
cudaError_t launch_receivers_batch(int kind, const Prob* probs, const int64_t* prefix, int nprob,
                                   uint32_t flags, EngineGlobals* G, int grid, cudaStream_t s);

// Receiver kernels work on tiles of kRecvTileX x kRecvTileY cells.
constexpr int kRecvTileX = 128;
constexpr int kRecvTileY = 16;
__host__ __device__ inline int64_t receiver_tiles(int64_t nx, int64_t ny) {
    return ((nx + kRecvTileX - 1) / kRecvTileX) * ((ny + kRecvTileY - 1) / kRecvTileY);
}

// Inner tiles of the halo kernels: D8 geometry 0 is kD8TileX x kD8TileY,
// geometry 1 half as wide, geometry 2 is 96x48; MFD uses kMfdTileX x kMfdTileY.
constexpr int kD8TileX = 128;
constexpr int kD8TileY = 32;
constexpr int kMfdTileX = 64;
constexpr int kMfdTileY = 64;  // 64x64 + 8 halo: 1.56x region cells per inner cell
constexpr int kD8Geometries = 3;
__host__ __device__ inline int64_t halo_tiles(int kind_mfd, int geo, int64_t nx, int64_t ny) {
    const int64_t tx = kind_mfd ? kMfdTileX : (geo == 1 ? kD8TileX / 2 : geo == 2 ? 96 : kD8TileX);
    const int64_t ty = kind_mfd ? kMfdTileY : (geo == 2 ? 48 : kD8TileY);
    return ((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
}

// Raises a kernel's dynamic shared-memory limit once per device: the first
// launch on each device sets the attribute, later launches skip the call
// (`done` holds one bit per device; devices past 63 set it every time).
template <class K>
inline cudaError_t smem_limit_once(K kernel, size_t bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

}  // namespace fr

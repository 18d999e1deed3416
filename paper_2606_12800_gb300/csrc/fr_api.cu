// fr_api.cu -- the C ABI declared in include/fr.h: argument validation,
// workspace layout, status word and the launch sequences.
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <utility>

#include "../../include/fr.h"
#include "fr_internal.h"

namespace fr {
namespace {

constexpr int64_t kMaxCells = (int64_t)1 << 40;
constexpr int kMassBlocks = 1024;
constexpr uint32_t kKnownFlags = FR_EDGE_ROUTE | FR_D8_LOWEST | FR_CHECK_FINITE | FR_D4 | FR_DINF |
                                 FR_GLOBAL_WALKERS | FR_GLOBAL_SKELETON | FR_WEIGHTS_IN_WORKSPACE |
                                 FR_SINK_SUMS_IN_WORKSPACE;
// flags of the receiver and fused route calls: the workspace flags describe a
// routing's workspace and have no meaning there
constexpr uint32_t kCallFlags = kKnownFlags & ~(FR_WEIGHTS_IN_WORKSPACE | FR_SINK_SUMS_IN_WORKSPACE);

// D8 forward: the global phase switches from the cell walkers to the
// tile-skeleton solve when the local phase leaves at least this share of the
// cells global (a rough DEM leaves about 0.02 %, a depression-filled one
// about 5 %); chosen by measurement.
constexpr double kSkelShare = 1.0 / 512.0;

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Workspace layout (same for every operation on an nx*ny grid):
//   globals (128 B) | global-cell bits (1 bit/cell) | arrival counters (1 B/cell)
//   | trailing words (4 B/cell) | frontier buffer (8 B/cell)
//   | global-cell list (8 B/cell) | routing bytes (1 B/cell) | mass partials
// The first two regions are zeroed by each engine call (one memset); a global
// cell's arrival counter is stored before it is first counted.
struct Layout {
    size_t cnt, gbits, lo, link, glist, rb, partials, total, zero_bytes;
    size_t frac, total_mfd;  // MFD only: fractions (32 B/cell) after the common part
};

Layout layout(int64_t n) {
    Layout L;
    size_t off = 256;
    L.gbits = off;
    off += align256(((size_t)n + 31) / 32 * 4);
    L.zero_bytes = off;
    L.cnt = off;
    off += align256((size_t)n + 4);
    L.lo = off;
    off += align256((size_t)n * 4);
    L.link = off;
    off += align256((size_t)n * 8);
    L.glist = off;
    off += align256((size_t)n * 8);
    L.rb = off;
    off += align256((size_t)n);
    L.partials = off;
    off += align256((size_t)kMassBlocks * 3 * 8);
    L.total = off;
    L.frac = off;
    off += align256((size_t)n * 8 * sizeof(float));
    L.total_mfd = off;
    return L;
}

// fr_fill's workspace: the sweep counters (one per sweep of a batch) and two
// per-tile change records.
constexpr int kFillBatch = 8;  // sweeps launched between two reads of the counters
size_t fill_ws_bytes(int64_t nx, int64_t ny) {
    return 256 + align256((size_t)fill_tiles(nx, ny)) * 2;
}

bool sizes_ok(int64_t nx, int64_t ny) {
    return nx >= 1 && ny >= 1 && nx < kMaxCells && ny < kMaxCells && nx <= kMaxCells / ny;
}

fr_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FR_OK : FR_ERR_CUDA; }

bool ws_ok(const void* ws, size_t ws_bytes, int64_t n) {
    return ws && ((uintptr_t)ws & 255) == 0 && ws_bytes >= layout(n).total;
}

// MFD operations also keep the fractions of every cell in the workspace.
bool ws_ok_mfd(const void* ws, size_t ws_bytes, int64_t n) {
    return ws && ((uintptr_t)ws & 255) == 0 && ws_bytes >= layout(n).total_mfd;
}

// FR_CHECK_FINITE uses a counter in the library's own device memory (module
// scope, allocated when the library is loaded) and synchronises the stream.
__device__ unsigned long long g_nonfinite;
std::mutex g_finite_mutex;

fr_status check_finite(const float* z, int64_t n, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_finite_mutex);
    unsigned long long zero = 0, got = 0;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_nonfinite) != cudaSuccess) return FR_ERR_CUDA;
    if (cudaMemcpyAsync(ptr, &zero, sizeof(zero), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FR_ERR_CUDA;
    if (launch_count_nonfinite(z, n, (unsigned long long*)ptr, s) != cudaSuccess) return FR_ERR_CUDA;
    if (cudaMemcpyAsync(&got, ptr, sizeof(got), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FR_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FR_ERR_CUDA;
    return got ? FR_ERR_NONFINITE : FR_OK;
}

bool routing_ok(const fr_routing* R) {
    if (!R || R->reserved || R->reserved2) return false;
    if (!sizes_ok(R->nx, R->ny)) return false;
    if (R->kind == FR_ROUTING_D8)
        return R->dir != nullptr && !(R->flags & (FR_DINF | FR_WEIGHTS_IN_WORKSPACE)) &&
               (R->flags & ~kKnownFlags) == 0 &&
               (R->flags & (FR_GLOBAL_WALKERS | FR_GLOBAL_SKELETON)) != (FR_GLOBAL_WALKERS | FR_GLOBAL_SKELETON);
    if (R->kind == FR_ROUTING_MFD)
        return R->mask && R->dem && std::isfinite(R->dx) && R->dx > 0 && std::isfinite(R->p) &&
               R->p > 0 && R->p <= FR_MFD_MAX_P && (R->flags & ~kKnownFlags) == 0 &&
               !(R->flags & FR_SINK_SUMS_IN_WORKSPACE) &&
               !(R->flags & FR_D4);
    return false;
}

Prob base_prob(const fr_routing* R, char* ws) {
    Layout L = layout(R->nx * R->ny);
    Prob P;
    std::memset(&P, 0, sizeof(P));
    P.nx = R->nx;
    P.ny = R->ny;
    P.rb = R->kind == FR_ROUTING_D8 ? R->dir : R->mask;
    P.z = R->kind == FR_ROUTING_MFD ? R->dem : nullptr;
    P.cnt = reinterpret_cast<uint32_t*>(ws + L.cnt);
    P.link = reinterpret_cast<int64_t*>(ws + L.link);
    P.gbits = reinterpret_cast<uint32_t*>(ws + L.gbits);
    P.glist = reinterpret_cast<unsigned long long*>(ws + L.glist);
    P.glist_cap = R->nx * R->ny;
    P.out_lo = reinterpret_cast<float*>(ws + L.lo);
    // the skeleton solve's scratch shares the global-cell list's region (the
    // list itself is read only by the cell walkers): tile list, walker
    // starts, dependency slots
    P.skel_min = ~0ull;
    if (R->kind == FR_ROUTING_D8) {
        const int64_t n = R->nx * R->ny, st = skel_tiles(R->nx, R->ny);
        const size_t o_starts = align256((size_t)st * 4);
        const size_t o_pool = o_starts + align256((size_t)st * (4 * kSkelTile - 4) * 8);
        const size_t need = o_pool + (size_t)st * kSkelPool * 2;
        if (need <= (size_t)n * 8 && !(R->flags & FR_GLOBAL_WALKERS)) {
            char* base = ws + L.glist;
            P.sktiles = reinterpret_cast<uint32_t*>(base);
            P.skstarts = reinterpret_cast<unsigned long long*>(base + o_starts);
            P.skpool = reinterpret_cast<uint16_t*>(base + o_pool);
            const double share = (double)n * kSkelShare;
            P.skel_min = (R->flags & FR_GLOBAL_SKELETON) ? 0ull
                                                         : (unsigned long long)(share < 1.0 ? 1.0 : share);
        }
    }
    if (R->kind == FR_ROUTING_MFD) P.frac = reinterpret_cast<const float*>(ws + L.frac);
    P.mc = make_mfd_const(R->kind == FR_ROUTING_MFD ? R->dx : 1.0, R->kind == FR_ROUTING_MFD ? R->p : 1.0);
    return P;
}

std::atomic<unsigned long long> g_wait_limit_ns{10ull * 1000ull * 1000ull * 1000ull};

}  // namespace

unsigned long long wait_limit_ns() { return g_wait_limit_ns.load(std::memory_order_relaxed); }

}  // namespace fr

using namespace fr;

extern "C" {

uint64_t fr_set_wait_limit(uint64_t ns) {
    return g_wait_limit_ns.exchange(ns, std::memory_order_relaxed);
}

fr_status fr_receiver_index(const uint8_t* dir, int64_t nx, int64_t ny, int32_t index_bytes,
                            void* idx_out, void* stream) {
    if (!dir || !idx_out || !sizes_ok(nx, ny) || (index_bytes != 4 && index_bytes != 8))
        return FR_ERR_INVALID_ARG;
    if (index_bytes == 4 && nx * ny > (int64_t)INT32_MAX) return FR_ERR_INVALID_ARG;
    return cuda_status(launch_receiver_index(dir, nx, ny, index_bytes == 8, idx_out, (cudaStream_t)stream));
}

const char* fr_status_string(fr_status s) {
    switch (s) {
        case FR_OK: return "ok";
        case FR_ERR_INVALID_ARG: return "invalid argument";
        case FR_ERR_CUDA: return "CUDA error";
        case FR_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
        case FR_ERR_NONFINITE: return "DEM holds NaN or Inf";
        case FR_ERR_NO_PROGRESS: return "not every cell was reached (cycle in the routing)";
        case FR_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

int32_t fr_version(void) { return 100; }

size_t fr_workspace_size(int32_t op, int64_t nx, int64_t ny, uint32_t flags) {
    if (!sizes_ok(nx, ny) || (flags & ~kKnownFlags)) return 0;
    if (op == FR_OP_RECEIVERS) return 0;
    if (op == FR_OP_MFD) return layout(nx * ny).total_mfd;
    if (op == FR_OP_FILL) return fill_ws_bytes(nx, ny);
    if (op < 0 || op > FR_OP_ROUTE) return 0;
    return layout(nx * ny).total;
}

fr_status fr_get_status(const void* ws, size_t ws_bytes, void* stream) {
    if (!ws || ws_bytes < 256 || ((uintptr_t)ws & 255)) return FR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    EngineGlobals g;
    if (cudaMemcpyAsync(&g, ws, sizeof(g), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FR_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FR_ERR_CUDA;
    unsigned zero = 0;
    const size_t off = offsetof(EngineGlobals, status);
    if (cudaMemcpyAsync((char*)ws + off, &zero, sizeof(zero), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return FR_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FR_ERR_CUDA;
    unsigned tma_err = 0;
    if (read_clear_tma_error(&tma_err, s) != cudaSuccess) return FR_ERR_CUDA;
    if (g.status == FR_OK && tma_err) return FR_ERR_NO_PROGRESS;
    return (fr_status)g.status;
}

fr_status fr_receivers_d8(const float* dem, int64_t nx, int64_t ny, double dx, uint32_t flags,
                          uint8_t* dir_out, uint8_t* indeg_out, void* stream) {
    if (!dem || !dir_out || !sizes_ok(nx, ny) || !std::isfinite(dx) || dx <= 0 ||
        (flags & ~kCallFlags) || (flags & FR_DINF))
        return FR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (flags & FR_CHECK_FINITE) {
        fr_status st = check_finite(dem, nx * ny, s);
        if (st != FR_OK) return st;
    }
    return cuda_status(launch_receivers_d8(dem, nx, ny, dx, flags, dir_out, indeg_out, s));
}

fr_status fr_receivers_mfd(const float* dem, int64_t nx, int64_t ny, double dx, double p,
                           uint32_t flags, uint8_t* mask_out, float* frac_out, uint8_t* indeg_out,
                           void* stream) {
    if (!dem || !mask_out || !sizes_ok(nx, ny) || !std::isfinite(dx) || dx <= 0 ||
        !std::isfinite(p) || p <= 0 || p > FR_MFD_MAX_P || (flags & ~kCallFlags) ||
        (flags & FR_D4))
        return FR_ERR_INVALID_ARG;
    if (frac_out && ((uintptr_t)frac_out & 15)) return FR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (flags & FR_CHECK_FINITE) {
        fr_status st = check_finite(dem, nx * ny, s);
        if (st != FR_OK) return st;
    }
    return cuda_status(launch_receivers_mfd(dem, nx, ny, dx, p, flags, mask_out, frac_out,
                                            indeg_out, s));
}

}  // extern "C"

namespace fr {
namespace {

// fr_accumulate; fracs_ready: the MFD fractions are already in the workspace
// (fr_route_mfd computes them together with the masks).
fr_status accumulate_impl(const fr_routing* R, const float* rain, float* w_out, float* w_lo_out,
                          uint64_t* area_out, void* ws, size_t ws_bytes, cudaStream_t s,
                          bool fracs_ready) {
    if (!routing_ok(R)) return FR_ERR_INVALID_ARG;
    if (!w_out && !w_lo_out && !area_out) return FR_ERR_INVALID_ARG;
    if (w_lo_out && !w_out) return FR_ERR_INVALID_ARG;
    const bool mfd = R->kind == FR_ROUTING_MFD;
    if (mfd && (area_out || !w_out)) return FR_ERR_INVALID_ARG;
    const int64_t n = R->nx * R->ny;
    if (!(mfd ? ws_ok_mfd(ws, ws_bytes, n) : ws_ok(ws, ws_bytes, n))) return FR_ERR_WORKSPACE;
    Prob P = base_prob(R, (char*)ws);
    P.init = rain;
    P.out_hi = w_out;
    if (w_lo_out) {
        P.out_lo = w_lo_out;
        P.lo_full = 1;
    }
    P.area = area_out;
    const Layout L = layout(n);
    cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_bytes, s);
    if (e != cudaSuccess) return FR_ERR_CUDA;
    EngineGlobals* G = reinterpret_cast<EngineGlobals*>(ws);
    if (!mfd) return cuda_status(launch_d8_forward(w_out != nullptr, area_out != nullptr, P, G, s));
    if (!fracs_ready && !(R->flags & FR_WEIGHTS_IN_WORKSPACE)) {
        e = launch_mfd_fractions(R->dem, R->mask, R->nx, R->ny, R->dx, R->p, R->flags,
                                 reinterpret_cast<float*>((char*)ws + L.frac), s);
        if (e != cudaSuccess) return FR_ERR_CUDA;
    }
    return cuda_status(launch_mfd_forward(P, G, s));
}

}  // namespace
}  // namespace fr

extern "C" {

fr_status fr_accumulate(const fr_routing* R, const float* rain, float* w_out, float* w_lo_out,
                        uint64_t* area_out, void* ws, size_t ws_bytes, void* stream) {
    return accumulate_impl(R, rain, w_out, w_lo_out, area_out, ws, ws_bytes, (cudaStream_t)stream,
                           false);
}

fr_status fr_fill(const float* dem, int64_t nx, int64_t ny, uint32_t flags, float* filled_out,
                  int32_t max_sweeps, int32_t* sweeps_out, void* ws, size_t ws_bytes,
                  void* stream) {
    if (!dem || !filled_out || !sizes_ok(nx, ny) || max_sweeps < 1 || (flags & ~FR_CHECK_FINITE))
        return FR_ERR_INVALID_ARG;
    const int64_t n = nx * ny;
    const uintptr_t a0 = (uintptr_t)dem, b0 = (uintptr_t)filled_out, len = (uintptr_t)n * 4;
    if (a0 < b0 + len && b0 < a0 + len) return FR_ERR_INVALID_ARG;  // overlap
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < fill_ws_bytes(nx, ny)) return FR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (flags & FR_CHECK_FINITE) {
        fr_status st = check_finite(dem, n, s);
        if (st != FR_OK) return st;
    }
    if (fill_init(dem, nx, ny, filled_out, s) != cudaSuccess) return FR_ERR_CUDA;
    // counters of one batch of sweeps in the first 256 bytes, then the two
    // per-tile change records (written by every sweep before they are read)
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(ws);
    uint8_t* act[2] = {(uint8_t*)ws + 256, (uint8_t*)ws + 256 + align256((size_t)fill_tiles(nx, ny))};
    for (int32_t done = 0; done < max_sweeps;) {
        const int32_t b = max_sweeps - done < kFillBatch ? max_sweeps - done : kFillBatch;
        unsigned long long h[kFillBatch];
        if (cudaMemsetAsync(counts, 0, sizeof(h), s) != cudaSuccess) return FR_ERR_CUDA;
        for (int32_t k = 0; k < b; ++k) {
            const int32_t sweep = done + k;  // 0-based
            if (fill_sweep(dem, nx, ny, filled_out, act[(sweep + 1) & 1], act[sweep & 1],
                           sweep == 0, counts + k, s) != cudaSuccess)
                return FR_ERR_CUDA;
        }
        if (cudaMemcpyAsync(h, counts, sizeof(h[0]) * b, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return FR_ERR_CUDA;
        for (int32_t k = 0; k < b; ++k) {
            if (h[k] == 0) {  // the first sweep that changed nothing; later ones were idle
                if (sweeps_out) *sweeps_out = done + k + 1;
                return FR_OK;
            }
        }
        done += b;
        if (sweeps_out) *sweeps_out = done;
    }
    return FR_ERR_NO_PROGRESS;
}

fr_status fr_accumulate_richardson(const fr_routing* R, const float* rain, float* w_out,
                                   float* w_lo_out, int32_t order, int32_t max_iterations,
                                   int32_t* iterations_out, void* ws, size_t ws_bytes,
                                   void* stream) {
    if (!routing_ok(R) || !w_out || max_iterations < 1 || order < 1 || order > 64)
        return FR_ERR_INVALID_ARG;
    const bool mfd = R->kind == FR_ROUTING_MFD;
    const int64_t n = R->nx * R->ny;
    if (!(mfd ? ws_ok_mfd(ws, ws_bytes, n) : ws_ok(ws, ws_bytes, n))) return FR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Prob P = base_prob(R, (char*)ws);
    P.init = rain;
    const Layout L = layout(n);
    if (mfd && launch_mfd_fractions(R->dem, R->mask, R->nx, R->ny, R->dx, R->p, R->flags,
                                    reinterpret_cast<float*>((char*)ws + L.frac), s) != cudaSuccess)
        return FR_ERR_CUDA;
    // two iterates (interleaved two-float) in the frontier and list regions
    float2* a = reinterpret_cast<float2*>((char*)ws + L.glist);
    float2* b = reinterpret_cast<float2*>((char*)ws + L.link);
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(ws);  // globals block
    if (cudaMemsetAsync(a, 0, (size_t)n * sizeof(float2), s) != cudaSuccess) return FR_ERR_CUDA;
    // one iteration = `order` sweeps; the sweep after the last changing one
    // shows that the iterate is exact
    int32_t exact_after = 0;  // sweeps
    bool converged = false;
    const int64_t max_sweeps = (int64_t)max_iterations * order + 1;
    for (int64_t sweep = 1; sweep <= max_sweeps; ++sweep) {
        unsigned long long h[2] = {0, 0};
        if (cudaMemsetAsync(counts, 0, sizeof(h), s) != cudaSuccess) return FR_ERR_CUDA;
        if (richardson_sweep(mfd, P, a, b, counts, s) != cudaSuccess) return FR_ERR_CUDA;
        if (cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return FR_ERR_CUDA;
        if (h[1] != (unsigned long long)n) return FR_ERR_NO_PROGRESS;  // a cycle
        std::swap(a, b);  // a: the newest iterate
        if (h[0] == 0) {
            converged = true;
            break;
        }
        exact_after = (int32_t)sweep;
    }
    const int32_t iterations = (exact_after + order - 1) / order;
    if (iterations_out) *iterations_out = iterations;
    if (!converged || iterations > max_iterations) return FR_ERR_NO_PROGRESS;
    return cuda_status(richardson_output(a, n, w_out, w_lo_out, s));
}

fr_status fr_route_d8(const float* dem, int64_t nx, int64_t ny, double dx, uint32_t flags,
                      const float* rain, float* w_out, float* w_lo_out, uint64_t* area_out,
                      uint8_t* dir_out, void* ws, size_t ws_bytes, void* stream) {
    if (!dem || !sizes_ok(nx, ny) || !std::isfinite(dx) || dx <= 0 || (flags & ~kCallFlags) ||
        (flags & FR_DINF))
        return FR_ERR_INVALID_ARG;
    if (!ws_ok(ws, ws_bytes, nx * ny)) return FR_ERR_WORKSPACE;
    uint8_t* dir = dir_out ? dir_out : reinterpret_cast<uint8_t*>((char*)ws + layout(nx * ny).rb);
    fr_status st = fr_receivers_d8(dem, nx, ny, dx, flags, dir, nullptr, stream);
    if (st != FR_OK) return st;
    fr_routing R;
    std::memset(&R, 0, sizeof(R));
    R.kind = FR_ROUTING_D8;
    R.nx = nx;
    R.ny = ny;
    R.dir = dir;
    R.dx = dx;
    R.flags = flags & (FR_GLOBAL_WALKERS | FR_GLOBAL_SKELETON);
    return fr_accumulate(&R, rain, w_out, w_lo_out, area_out, ws, ws_bytes, stream);
}

fr_status fr_route_mfd(const float* dem, int64_t nx, int64_t ny, double dx, double p,
                       uint32_t flags, const float* rain, float* w_out, float* w_lo_out,
                       uint8_t* mask_out, void* ws, size_t ws_bytes, void* stream) {
    if (!dem || !sizes_ok(nx, ny) || !std::isfinite(dx) || dx <= 0 || !std::isfinite(p) ||
        p <= 0 || p > FR_MFD_MAX_P || (flags & ~kCallFlags) || (flags & FR_D4))
        return FR_ERR_INVALID_ARG;
    if (!ws_ok_mfd(ws, ws_bytes, nx * ny)) return FR_ERR_WORKSPACE;
    const Layout L = layout(nx * ny);
    uint8_t* mask = mask_out ? mask_out : reinterpret_cast<uint8_t*>((char*)ws + L.rb);
    // masks and fractions in one pass
    fr_status st = fr_receivers_mfd(dem, nx, ny, dx, p, flags, mask,
                                    reinterpret_cast<float*>((char*)ws + L.frac), nullptr, stream);
    if (st != FR_OK) return st;
    fr_routing R;
    std::memset(&R, 0, sizeof(R));
    R.kind = FR_ROUTING_MFD;
    R.nx = nx;
    R.ny = ny;
    R.mask = mask;
    R.dem = dem;
    R.dx = dx;
    R.p = p;
    R.flags = flags & ~FR_CHECK_FINITE;
    return accumulate_impl(&R, rain, w_out, w_lo_out, nullptr, ws, ws_bytes, (cudaStream_t)stream,
                           true);
}

fr_status fr_route_adjoint(const fr_routing* R, const float* w, const float* w_lo,
                           const float* dLdw, float* dLdr_out, float* dLdz_out, void* ws,
                           size_t ws_bytes, void* stream) {
    if (!routing_ok(R) || !w || !dLdr_out) return FR_ERR_INVALID_ARG;
    if (dLdz_out && R->kind != FR_ROUTING_MFD) return FR_ERR_INVALID_ARG;
    if (dLdz_out && (R->flags & FR_DINF)) return FR_ERR_UNSUPPORTED;  // dL/dz: Freeman weights only
    const int64_t n = R->nx * R->ny;
    const bool mfd = R->kind == FR_ROUTING_MFD;
    if (!(mfd ? ws_ok_mfd(ws, ws_bytes, n) : ws_ok(ws, ws_bytes, n))) return FR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Prob P = base_prob(R, (char*)ws);
    P.init = dLdw;
    P.wf = w;
    P.wf_lo = w_lo;
    P.out_hi = dLdr_out;
    P.lo_full = dLdz_out ? 1 : 0;  // the elevation gradient reads every trailing word
    const Layout L = layout(n);
    if (cudaMemsetAsync(ws, 0, L.zero_bytes, s) != cudaSuccess) return FR_ERR_CUDA;
    if (mfd && !(R->flags & FR_WEIGHTS_IN_WORKSPACE) &&
        launch_mfd_fractions(R->dem, R->mask, R->nx, R->ny, R->dx, R->p, R->flags,
                             reinterpret_cast<float*>((char*)ws + L.frac), s) != cudaSuccess)
        return FR_ERR_CUDA;
    cudaError_t e = launch_adjoint(mfd, P, reinterpret_cast<EngineGlobals*>(ws), s);
    if (e != cudaSuccess) return FR_ERR_CUDA;
    if (dLdz_out) {
        e = launch_mfd_grad_z(P, dLdr_out, P.out_lo, dLdz_out, s);
        if (e != cudaSuccess) return FR_ERR_CUDA;
    }
    return FR_OK;
}

fr_status fr_mass_balance(const fr_routing* R, const float* rain, const float* w,
                          const float* w_lo, const uint64_t* area, double* out_dev, void* ws,
                          size_t ws_bytes, void* stream) {
    if (!routing_ok(R) || !out_dev) return FR_ERR_INVALID_ARG;
    if (w_lo && !w) return FR_ERR_INVALID_ARG;
    const bool sums = R->flags & FR_SINK_SUMS_IN_WORKSPACE;  // D8 only (routing_ok)
    if (sums && (w || !area)) return FR_ERR_INVALID_ARG;
    const int64_t n = R->nx * R->ny;
    if (!ws_ok(ws, ws_bytes, n)) return FR_ERR_WORKSPACE;
    const Layout L = layout(n);
    int64_t blocks = (n + 255) / 256;
    if (blocks > kMassBlocks) blocks = kMassBlocks;
    const uint8_t* rb = R->kind == FR_ROUTING_D8 ? R->dir : R->mask;
    if (sums)
        return cuda_status(launch_mass_balance_ws(
            R->nx, R->ny, rb, rain, area, reinterpret_cast<const uint32_t*>((char*)ws + L.gbits),
            reinterpret_cast<const EngineGlobals*>(ws), reinterpret_cast<double*>((char*)ws + L.partials),
            (int)blocks, out_dev, (cudaStream_t)stream));
    return cuda_status(launch_mass_balance(R->kind, R->nx, R->ny, rb, rain, w, w_lo, area,
                                           reinterpret_cast<double*>((char*)ws + L.partials),
                                           (int)blocks, out_dev, (cudaStream_t)stream));
}

}  // extern "C"

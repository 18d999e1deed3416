// fr_batch.cu -- batched routing of many independent DEMs (fr_route_batch).
//
// All tiles are routed by one launch per stage, with persistent CTAs taking
// work from device-side counters: a setup kernel builds the per-tile problem
// descriptors and prefix tables on the device (so the sequence reads no host
// memory when it runs and can be captured in a CUDA graph), then batched
// receivers, the batched tile engine (local phase) and the walker kernel.
// The CTA counts of the persistent stages come from a small autotuner.
#include <cstring>
#include <mutex>

#include "../../include/fr.h"
#include "fr_engine.cuh"

namespace fr {
namespace {

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

struct BatchLayout {
    size_t cnt, gbits, zero_bytes, lo, link, glist, probs, pre_recv, pre_eng, frac, total;
    int64_t cells, eng_tiles;
};

__host__ __device__ inline int64_t cnt_bytes(int64_t n) { return (n + 4 + 3) & ~(int64_t)3; }
__host__ __device__ inline int64_t gbit_words(int64_t n) { return (n + 31) / 32; }
BatchLayout batch_layout(const fr_tile* t, int n, int kind = FR_ROUTING_D8, int geo = 0) {
    BatchLayout L{};
    int64_t cb = 0, gw = 0, cells = 0, et = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t c = t[i].nx * t[i].ny;
        cb += cnt_bytes(c);
        gw += gbit_words(c);
        cells += c;
        et += halo_tiles(kind == FR_ROUTING_MFD, geo, t[i].nx, t[i].ny);
    }
    size_t off = 256;
    L.gbits = off;
    off += a256((size_t)gw * 4);
    L.zero_bytes = off;  // globals and global-cell bits; counters are stored before use
    L.cnt = off;
    off += a256((size_t)cb);
    L.lo = off;
    off += a256((size_t)cells * 4);
    L.link = off;
    off += a256((size_t)cells * 8);
    L.glist = off;
    off += a256((size_t)cells * 8);
    L.probs = off;
    off += a256((size_t)n * sizeof(Prob));
    L.pre_recv = off;
    off += a256((size_t)(n + 1) * 8);
    L.pre_eng = off;
    off += a256((size_t)(n + 1) * 8);
    L.frac = off;  // MFD: fractions of every cell of every tile
    if (kind == FR_ROUTING_MFD) off += a256((size_t)cells * 8 * sizeof(float));
    L.total = off;
    L.cells = cells;
    L.eng_tiles = et;
    return L;
}

// One CTA: prefix sums over the tiles (chunked per thread, then a block scan)
// and the problem descriptors.
constexpr int SETUP_NT = 1024;

__global__ void __launch_bounds__(SETUP_NT) k_batch_setup(const fr_tile* __restrict__ tiles, int n,
                                                          int kind, int geo, double p, char* ws,
                                                          BatchLayout L, EngineGlobals* G) {
    __shared__ int64_t sh[4][SETUP_NT];
    const int tid = threadIdx.x;
    const int per = (n + SETUP_NT - 1) / SETUP_NT;
    const int b = tid * per, e = min(n, b + per);
    int64_t s_cb = 0, s_gw = 0, s_cells = 0, s_rt = 0, s_et = 0;
    for (int i = b; i < e; ++i) {
        const int64_t c = tiles[i].nx * tiles[i].ny;
        s_cb += cnt_bytes(c);
        s_gw += gbit_words(c);
        s_cells += c;
        s_rt += receiver_tiles(tiles[i].nx, tiles[i].ny);
        s_et += halo_tiles(kind == FR_ROUTING_MFD, geo, tiles[i].nx, tiles[i].ny);
    }
    // exclusive scan of the per-thread sums (cb, gw, cells, recv tiles); engine
    // tiles share the cell scan's slot below
    sh[0][tid] = s_cb;
    sh[1][tid] = s_gw;
    sh[2][tid] = s_cells;
    sh[3][tid] = s_rt;
    __syncthreads();
    if (tid < 4) {
        int64_t acc = 0;
        for (int i = 0; i < SETUP_NT; ++i) {
            const int64_t v = sh[tid][i];
            sh[tid][i] = acc;
            acc += v;
        }
    }
    __syncthreads();
    int64_t o_cb = sh[0][tid], o_gw = sh[1][tid], o_cells = sh[2][tid], o_rt = sh[3][tid];
    __syncthreads();
    sh[0][tid] = s_et;
    __syncthreads();
    if (tid == 0) {
        int64_t acc = 0;
        for (int i = 0; i < SETUP_NT; ++i) {
            const int64_t v = sh[0][i];
            sh[0][i] = acc;
            acc += v;
        }
    }
    __syncthreads();
    int64_t o_et = sh[0][tid];
    Prob* probs = reinterpret_cast<Prob*>(ws + L.probs);
    int64_t* pre_recv = reinterpret_cast<int64_t*>(ws + L.pre_recv);
    int64_t* pre_eng = reinterpret_cast<int64_t*>(ws + L.pre_eng);
    for (int i = b; i < e; ++i) {
        const fr_tile& t = tiles[i];
        const int64_t c = t.nx * t.ny;
        Prob P;
        memset(&P, 0, sizeof(P));
        P.nx = t.nx;
        P.ny = t.ny;
        P.rb = t.route_out;
        P.z = t.dem;
        P.init = t.rain;
        P.out_hi = t.w_out;
        P.lo_full = t.w_lo_out != nullptr;
        P.out_lo = t.w_lo_out ? t.w_lo_out : reinterpret_cast<float*>(ws + L.lo) + o_cells;
        P.area = t.area_out;
        P.cnt = reinterpret_cast<uint32_t*>(ws + L.cnt + o_cb);
        P.gbits = reinterpret_cast<uint32_t*>(ws + L.gbits) + o_gw;
        P.link = reinterpret_cast<int64_t*>(ws + L.link) + o_cells;
        if (kind == FR_ROUTING_MFD) P.frac = reinterpret_cast<const float*>(ws + L.frac) + 8 * o_cells;
        P.glist = reinterpret_cast<unsigned long long*>(ws + L.glist);
        P.glist_cap = L.cells;
        P.mc = make_mfd_const(t.dx, kind == FR_ROUTING_MFD ? p : 1.0);
        P.skel_min = ~0ull;  // batched D8: the cell walkers finish the global cells
        probs[i] = P;
        pre_recv[i] = o_rt;
        pre_eng[i] = o_et;
        o_cb += cnt_bytes(c);
        o_gw += gbit_words(c);
        o_cells += c;
        o_rt += receiver_tiles(t.nx, t.ny);
        o_et += halo_tiles(kind == FR_ROUTING_MFD, geo, t.nx, t.ny);
    }
    if (e == n && b < e) {  // the thread holding the last tile writes the totals
        pre_recv[n] = o_rt;
        pre_eng[n] = o_et;
        G->total_cells = o_cells;
    }
    if (n == 0 && tid == 0) {
        pre_recv[0] = 0;
        pre_eng[0] = 0;
    }
}

bool tiles_ok(const fr_tile* t, int n, int kind) {
    // global-cell list entries keep the problem index in 24 bits
    if (!t || n <= 0 || n >= (1 << 24)) return false;
    const bool w = t[0].w_out != nullptr, a = t[0].area_out != nullptr;
    if (!w && !a) return false;
    if (kind == FR_ROUTING_MFD && (a || !w)) return false;
    for (int i = 0; i < n; ++i) {
        const fr_tile& x = t[i];
        if (!x.dem || !x.route_out || x.nx < 1 || x.ny < 1 || !(x.dx > 0) || x.dx != x.dx) return false;
        if (x.nx > ((int64_t)1 << 40) / x.ny) return false;
        if ((x.w_out != nullptr) != w || (x.area_out != nullptr) != a) return false;
        if (x.w_lo_out && !x.w_out) return false;
    }
    return true;
}

// Tuned launch shape of the batched route: CTAs per SM of the persistent
// receiver stage, and the halo-tile geometry of the D8 local stage
// (0: 128x32 inner tiles, 1: 64x32).
struct Tune {
    int recv = 8, geo = 1;
};
Tune g_tune[2];
std::mutex g_tune_mutex;

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

cudaError_t run_batch(const fr_tile* th, const fr_tile* td, int n, int kind, double p, uint32_t flags,
                      char* ws, const Tune& tune, cudaStream_t s) {
    const int geo = kind == FR_ROUTING_D8 ? tune.geo : 0;
    const BatchLayout L = batch_layout(th, n, kind, geo);
    EngineGlobals* G = reinterpret_cast<EngineGlobals*>(ws);
    cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_bytes, s);
    if (e != cudaSuccess) return e;
    k_batch_setup<<<1, SETUP_NT, 0, s>>>(td, n, kind, geo, p, ws, L, G);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const Prob* probs = reinterpret_cast<const Prob*>(ws + L.probs);
    e = launch_receivers_batch(kind, probs, reinterpret_cast<const int64_t*>(ws + L.pre_recv), n,
                               flags, G, sm_count() * tune.recv, s);
    if (e != cudaSuccess) return e;
    const bool w = th[0].w_out != nullptr, a = th[0].area_out != nullptr;
    const int64_t* pre = reinterpret_cast<const int64_t*>(ws + L.pre_eng);
    if (kind == FR_ROUTING_D8)
        return launch_d8_forward_batch(geo, w, a, probs, pre, n, L.eng_tiles,
                                       (unsigned long long)L.cells, G, s);
    return launch_mfd_forward_batch(probs, pre, n, L.eng_tiles, (unsigned long long)L.cells, G, s);
}

}  // namespace

}  // namespace fr

using namespace fr;

extern "C" {

size_t fr_batch_workspace_size(const fr_tile* tiles_host, int32_t ntiles, int32_t kind,
                               uint32_t flags) {
    if (!tiles_ok(tiles_host, ntiles, kind) || (flags & ~(FR_EDGE_ROUTE | FR_D8_LOWEST | FR_D4 | FR_DINF))) return 0;
    return batch_layout(tiles_host, ntiles, kind).total;
}

fr_status fr_route_batch(const fr_tile* tiles_host, const fr_tile* tiles_dev, int32_t ntiles,
                         int32_t kind, double p, uint32_t flags, void* ws, size_t ws_bytes,
                         void* stream) {
    if (kind != FR_ROUTING_D8 && kind != FR_ROUTING_MFD) return FR_ERR_INVALID_ARG;
    if (!tiles_dev || !tiles_ok(tiles_host, ntiles, kind)) return FR_ERR_INVALID_ARG;
    if (flags & ~(FR_EDGE_ROUTE | FR_D8_LOWEST | FR_D4 | FR_DINF)) return FR_ERR_INVALID_ARG;
    if (kind == FR_ROUTING_MFD && (!(p > 0 && p <= FR_MFD_MAX_P) || (flags & FR_D4)))
        return FR_ERR_INVALID_ARG;
    if (kind == FR_ROUTING_D8 && (flags & FR_DINF)) return FR_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < batch_layout(tiles_host, ntiles, kind).total)
        return FR_ERR_WORKSPACE;
    Tune t;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        t = g_tune[kind];
    }
    return run_batch(tiles_host, tiles_dev, ntiles, kind, p, flags, (char*)ws, t,
                     (cudaStream_t)stream) == cudaSuccess
               ? FR_OK
               : FR_ERR_CUDA;
}

fr_status fr_batch_autotune(const fr_tile* tiles_host, const fr_tile* tiles_dev, int32_t ntiles,
                            int32_t kind, double p, uint32_t flags, void* ws, size_t ws_bytes,
                            void* stream) {
    fr_status st = fr_route_batch(tiles_host, tiles_dev, ntiles, kind, p, flags, ws, ws_bytes, stream);
    if (st != FR_OK) return st;  // validates everything once
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return FR_ERR_CUDA;
    const int recv_opts[] = {2, 4, 8, 16};
    const int geos = kind == FR_ROUTING_D8 ? kD8Geometries : 1;
    Tune best;
    float best_ms = 1e30f;
    for (int r : recv_opts) {
        for (int geo = 0; geo < geos; ++geo) {
            Tune t;
            t.recv = r;
            t.geo = geo;
            float ms_sum = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(a, s);
                if (run_batch(tiles_host, tiles_dev, ntiles, kind, p, flags, (char*)ws, t, s) !=
                    cudaSuccess) {
                    cudaEventDestroy(a);
                    cudaEventDestroy(b);
                    return FR_ERR_CUDA;
                }
                cudaEventRecord(b, s);
                cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep) ms_sum += ms;
            }
            if (ms_sum < best_ms) {
                best_ms = ms_sum;
                best = t;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[kind] = best;
    return FR_OK;
}

}  // extern "C"

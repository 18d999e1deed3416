// fr_engine.cuh -- shared pieces of exact accumulation over a routing DAG.
//
// Global flow routing solves A w = r with A = I - W (Sec. 2.2); the adjoint
// solves A^T g = gbar.  Both are triangular once cells are processed in
// dependency order (Sec. 2.4), which is what the sequential high-to-low
// algorithm does (Sec. 2.1).  On the GPU the grid is cut into CTA tiles that
// play the role of the paper's per-process subdomains (Sec. 2.4), extended by
// a halo so that the subdomains overlap:
//
//  1. local phase (fr_d8.cu, fr_halo.cu): every cell whose dependencies all
//     lie, recursively, inside its tile's extended region is solved exactly in
//     shared memory in a topological order (Sec. 3.2 shows any such order
//     gives the same result).  Inner cells with a dependency chain leaving the
//     region are marked "global" (a bit per cell and a list).
//  2. global phase (this file, a second kernel): instead of the paper's
//     Richardson iteration across subdomain boundaries (App. B.1) the global
//     cells are solved exactly.  Each global cell has an arrival counter for
//     its global dependencies.  For D8 forward routing (one receiver per cell)
//     a cell with none starts a walker, each finished cell increments its
//     receiver's counter, and the thread that completes a counter computes
//     that cell ("last arriver continues"); no thread ever waits on another.
//     For the modes where one cell can make several cells ready (MFD forward,
//     both adjoints) the global cells are processed in rounds instead (see
//     k_global_levels).  A routing graph with a cycle cannot hang either
//     kernel: its cells are never reached, which the completion count reports.
//
// Values are pulled from dependencies in a fixed order, so results are
// bit-reproducible.  Real-valued sums are two-float (fp32 hi + lo); unit-rain
// D8 areas are exact integers.
#pragma once

#include <cuda/atomic>

#include "fr_internal.h"

namespace fr {

template <Mode M, bool W, bool AREA>
struct Eng {
    static constexpr bool kMfd = (M == Mode::FwdMfd || M == Mode::AdjMfd);
    static constexpr bool kAdj = (M == Mode::AdjD8 || M == Mode::AdjMfd);
    static constexpr bool kVal = W || kAdj || kMfd;      // two-float values are solved
    static constexpr bool kArea = AREA && (M == Mode::FwdD8);
    static constexpr bool kBranch = kMfd || kAdj;         // several targets per cell
    static constexpr bool kD8Fwd = (M == Mode::FwdD8);
};

// Flag in a tile kernel's per-cell state byte (bits 0-3 count the missing
// in-region dependencies): the cell's dependencies leave the region.
constexpr uint32_t kG = 0x10u;

// Receiver mask of a routing byte.  D8 codes above 7 (including FR_SINK) mean
// no receiver.
template <bool MFD>
__device__ __forceinline__ uint32_t recv_mask(uint8_t rb) {
    if constexpr (MFD) return rb;
    else return rb < 8 ? (1u << rb) : 0u;
}

// Neighbour codes of cell (x, y) that lie inside the grid.  Receivers are
// always masked with it, so routing bytes that point outside the grid (possible
// in caller-supplied routings) act as "no receiver" instead of reaching outside.
__device__ __forceinline__ uint32_t grid_mask(int64_t x, int64_t y, int64_t nx, int64_t ny) {
    return grid_mask8(x, y, nx, ny);
}

// ------------------------------------------------------------ global view
// Accessors of the per-problem arrays (bounds-checked in debug builds).
__device__ __forceinline__ int64_t ncell(const Prob& P) { return P.nx * P.ny; }
__device__ __forceinline__ uint8_t rd_rb(const Prob& P, int64_t i) {
    return FR_OK(i, ncell(P), 1) ? __ldg(P.rb + i) : (uint8_t)0;
}
__device__ __forceinline__ float rd_z(const Prob& P, int64_t i) {
    return FR_OK(i, ncell(P), 2) ? __ldg(P.z + i) : 0.0f;
}
__device__ __forceinline__ float rd_in(const float* a, const Prob& P, int64_t i, unsigned site) {
    return FR_OK(i, ncell(P), site) ? __ldg(a + i) : 0.0f;
}
__device__ __forceinline__ void wr_f(float* a, const Prob& P, int64_t i, float v, unsigned site) {
    if (FR_OK(i, ncell(P), site)) a[i] = v;
}
__device__ __forceinline__ float rd_cg(const float* a, const Prob& P, int64_t i, unsigned site) {
    return FR_OK(i, ncell(P), site) ? ld_cg(a + i) : 0.0f;
}
__device__ __forceinline__ uint64_t rd_area(const Prob& P, int64_t i) {
    return FR_OK(i, ncell(P), 3) ? ld_cg(P.area + i) : 0ull;
}
__device__ __forceinline__ void wr_area(const Prob& P, int64_t i, uint64_t v) {
    if (FR_OK(i, ncell(P), 4)) P.area[i] = v;
}
// Stores cell i's counter (its preset), before any add to it: the init kernel
// of the global phase or the first round, ahead of a launch or grid barrier.
// Byte stores leave the neighbouring counters of the word alone.
__device__ __forceinline__ void cnt_set(const Prob& P, int64_t i, uint32_t v) {
    if (FR_OK(i, ncell(P), 5)) reinterpret_cast<uint8_t*>(P.cnt)[i] = (uint8_t)v;
}
__device__ __forceinline__ uint32_t cnt_add(const Prob& P, int64_t i, uint32_t n) {
    return FR_OK(i, ncell(P), 5) ? counter_add(P.cnt, i, n) : 0xFFu;
}
// The same with acquire-release order at device scope: the caller's earlier
// writes are visible to whoever completes the counter, and the completer sees
// every earlier adder's writes.
__device__ __forceinline__ uint32_t cnt_add_acq_rel(const Prob& P, int64_t i, uint32_t n) {
    if (!FR_OK(i, ncell(P), 5)) return 0xFFu;
    const uint32_t sh = 8u * (uint32_t)(i & 3);
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> w(P.cnt[i >> 2]);
    const uint32_t old = w.fetch_add(n << sh, cuda::memory_order_acq_rel);
    return ((old >> sh) & 0xFFu) + n;
}

template <class E>
__device__ __forceinline__ uint32_t g_recv(const Prob& P, int64_t i) {
    return recv_mask<E::kMfd>(rd_rb(P, i));
}

// Receivers of cell i restricted to the grid.
template <class E>
__device__ __forceinline__ uint32_t g_recv_own(const Prob& P, int64_t i) {
    int64_t y = i / P.nx, x = i - y * P.nx;
    return g_recv<E>(P, i) & grid_mask(x, y, P.nx, P.ny);
}

// Donor mask of cell (x, y) read from the global routing bytes.
template <class E>
__device__ __forceinline__ uint32_t g_donors(const Prob& P, int64_t x, int64_t y) {
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        int64_t xn = x + (int64_t)offx(k), yn = y + (int64_t)offy(k);
        if (xn < 0 || yn < 0 || xn >= P.nx || yn >= P.ny) continue;
        if ((g_recv<E>(P, yn * P.nx + xn) >> opp(k)) & 1u) m |= 1u << k;
    }
    return m;
}

template <class E>
__device__ __forceinline__ uint32_t g_deps(const Prob& P, int64_t i) {
    int64_t y = i / P.nx, x = i - y * P.nx;
    if constexpr (E::kAdj) return g_recv_own<E>(P, i);
    else return g_donors<E>(P, x, y);
}

template <class E>
__device__ __forceinline__ uint32_t g_targets(const Prob& P, int64_t i) {
    int64_t y = i / P.nx, x = i - y * P.nx;
    if constexpr (E::kAdj) return g_donors<E>(P, x, y);
    else return g_recv_own<E>(P, i);
}

// Initial value of a cell: rain (forward) or gbar (adjoint).
template <class E>
__device__ __forceinline__ df init_value(const Prob& P, int64_t i, uint32_t recv) {
    if constexpr (!E::kAdj) {
        return df_make(P.init ? rd_in(P.init, P, i, 8) : 1.0f);
    } else {
        if (P.init) return df_make(rd_in(P.init, P, i, 8));
        if (recv) return df_make(0.0f);
        float h = rd_in(P.wf, P, i, 9);
        float l = P.wf_lo ? rd_in(P.wf_lo, P, i, 10) : 0.0f;
        return {__fmul_rn(2.0f, h), __fmul_rn(2.0f, l)};
    }
}

template <class E>
__device__ __forceinline__ df g_value(const Prob& P, int64_t i) {
    return {rd_cg(P.out_hi, P, i, 11), rd_cg(P.out_lo, P, i, 12)};
}

// Computes and publishes the value of a global-phase cell whose dependencies
// are all final.
template <class E>
__device__ __noinline__ void walker_compute(const Prob& P, int64_t t) {
    const int64_t y = t / P.nx, x = t - y * P.nx;
    const uint32_t recv = g_recv_own<E>(P, t);
    if constexpr (E::kVal) {
        df v = init_value<E>(P, t, recv);
        if constexpr (E::kAdj) {
            // receiver terms in the fixed order of df_dot8
            float f[8];
            df vv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                f[k] = 0.0f;
                vv[k] = df_make(0.0f);
                if (!((recv >> k) & 1u)) continue;
                vv[k] = g_value<E>(P, t + offi(k, P.nx));
                f[k] = E::kMfd ? __ldg(P.frac + t * 8 + k) : 1.0f;
            }
            v = df_dot8(v, f, vv);
        } else {
            // routing bytes of the eight neighbours, loaded side by side
            const uint32_t gm = grid_mask(x, y, P.nx, P.ny);
            uint32_t dmask = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if ((gm >> k) & 1u) dmask |= ((g_recv<E>(P, t + offi(k, P.nx)) >> opp(k)) & 1u) << k;
            if constexpr (E::kMfd) {
                // donor terms in the fixed order of df_dot8
                float f[8];
                df vv[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    f[k] = 0.0f;
                    vv[k] = df_make(0.0f);
                    if (!((dmask >> k) & 1u)) continue;
                    const int64_t j = t + offi(k, P.nx);
                    f[k] = __ldg(P.frac + j * 8 + opp(k));
                    vv[k] = g_value<E>(P, j);
                }
                v = df_dot8(v, f, vv);
            } else {
#pragma unroll 1
                for (int k = 0; k < 8; ++k) {
                    if (!((dmask >> k) & 1u)) continue;
                    v = df_add(v, g_value<E>(P, t + offi(k, P.nx)));
                }
            }
        }
        if (P.out_hi) wr_f(P.out_hi, P, t, v.hi, 13);
        wr_f(P.out_lo, P, t, v.lo, 14);
    }
    if constexpr (E::kArea) {
        uint64_t a = 1;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int64_t xn = x + (int64_t)offx(k), yn = y + (int64_t)offy(k);
            if (xn < 0 || yn < 0 || xn >= P.nx || yn >= P.ny) continue;
            int64_t j = yn * P.nx + xn;
            if (rd_rb(P, j) == (uint8_t)opp(k)) a += rd_area(P, j);
        }
        wr_area(P, t, a);
    }
}

constexpr unsigned kStatusNoProgress = 5u;
constexpr uint32_t kReadyAt = 16u;  // preset counters: > 8 dependencies, < 256 (one byte)

__device__ __forceinline__ bool gbit(const Prob& P, int64_t i) {
    return FR_OK(i, ncell(P), 15) ? ((__ldg(P.gbits + (i >> 5)) >> (i & 31)) & 1u) : false;
}

// Number of dependencies of cell i that are global (solved by walkers).
template <class E>
__device__ __forceinline__ uint32_t g_deps_global(const Prob& P, int64_t i) {
    const uint32_t dep = g_deps<E>(P, i);
    uint32_t n = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if ((dep >> k) & 1u) n += gbit(P, i + offi(k, P.nx));
    return n;
}

// D8 forward walker: one step per global cell, all loads of a step issued
// together (the routing bytes of the 3 x 3 window, the cell's rain, the donors'
// values; then the receiver's window).
template <bool W, bool AREA>
__device__ __noinline__ unsigned long long walker_d8(const Prob& P, int64_t start) {
    unsigned long long n = 0;
    int64_t cur = start;
    int64_t y = cur / P.nx, x = cur - y * P.nx;
    while (true) {
        // window of routing bytes: code of neighbour k (0xFF outside the grid)
        uint8_t nb[8];
        uint32_t gm = 0, gn = 0;  // in-grid neighbours; global neighbours
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t xn = x + offx(k), yn = y + offy(k);
            const bool in = xn >= 0 && yn >= 0 && xn < P.nx && yn < P.ny;
            gm |= (uint32_t)in << k;
            nb[k] = in ? rd_rb(P, cur + offi(k, P.nx)) : (uint8_t)0xFF;
            gn |= (uint32_t)(in && gbit(P, cur + offi(k, P.nx))) << k;
        }
        const uint8_t own = rd_rb(P, cur);
        uint32_t dm = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) dm |= (uint32_t)(nb[k] == (uint8_t)opp(k)) << k;
        if constexpr (W) {
            df v = df_make(P.init ? rd_in(P.init, P, cur, 8) : 1.0f);
            float hi[8], lo[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                hi[k] = ((dm >> k) & 1u) ? rd_cg(P.out_hi, P, cur + offi(k, P.nx), 11) : 0.0f;
                lo[k] = ((dm >> k) & 1u) ? rd_cg(P.out_lo, P, cur + offi(k, P.nx), 12) : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if ((dm >> k) & 1u) v = df_add(v, df{hi[k], lo[k]});
            wr_f(P.out_hi, P, cur, v.hi, 13);
            wr_f(P.out_lo, P, cur, v.lo, 14);
        }
        if constexpr (AREA) {
            uint64_t a[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = ((dm >> k) & 1u) ? rd_area(P, cur + offi(k, P.nx)) : 0ull;
            uint64_t s = 1;
#pragma unroll
            for (int k = 0; k < 8; ++k) s += a[k];
            wr_area(P, cur, s);
        }
        ++n;
        if (own >= 8 || !((gm >> own) & 1u)) break;
        if (!((gn >> own) & 1u)) break;  // the receiver was solved exactly by its own tile
        // the receiver's counter was preset to kReadyAt - (its global donors):
        // the adder that completes it continues there
        const int64_t u = cur + offi(own, P.nx);
        if (cnt_add_acq_rel(P, u, 1u) != kReadyAt) break;
        cur = u;
        x += offx(own);
        y += offy(own);
    }
    return n;
}

// Warp-aggregated append to a frontier (all 32 lanes call): lane l appends
// pid_bits | (cell + offset of k) for the set bits k < 8 of `bits`, and
// pid_bits | cell for bit 8.  One atomic per warp on the frontier count.
__device__ __forceinline__ void frontier_push(int64_t nx, int64_t cell, unsigned long long pid_bits,
                                              uint32_t bits, unsigned long long* buf,
                                              unsigned long long* count, unsigned long long cap) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const uint32_t n = (uint32_t)__popc(bits);
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const unsigned v = __ballot_sync(0xffffffffu, (n >> b) & 1u);
        pre += (uint32_t)__popc(v & lt) << b;
        tot += (uint32_t)__popc(v) << b;
    }
    if (tot == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(count, (unsigned long long)tot);
    base = __shfl_sync(0xffffffffu, base, 0) + pre;
    for (uint32_t m = bits; m; m &= m - 1) {
        const int k = __ffs(m) - 1;
        const int64_t t = k == 8 ? cell : cell + offi(k, nx);
        if (FR_OK((int64_t)base, (int64_t)cap, 18)) buf[base] = pid_bits | (unsigned long long)t;
        ++base;
    }
}

// Global phase of D8 forward routing, first launch: every global cell's
// arrival counter is preset to kReadyAt minus its number of global donors, and
// the cells without global donors are listed (the walkers' starts, in the
// frontier buffer).
template <Mode M, bool W, bool AREA>
__global__ void __launch_bounds__(256) k_global_init(const Prob* __restrict__ probs, Prob single,
                                                     EngineGlobals* G) {
    using E = Eng<M, W, AREA>;
    const unsigned long long count = G->glist_count;
    const Prob& P0 = probs ? probs[0] : single;
    if (count >= P0.skel_min) return;  // the skeleton solve takes the global cells
    const unsigned long long* list = P0.glist;
    unsigned long long* starts = reinterpret_cast<unsigned long long*>(P0.link);
    constexpr unsigned long long kCellMask = (1ull << 40) - 1;
    const unsigned lane = threadIdx.x & 31u;
    // warp-aligned steps: frontier_push needs the whole warp
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x - lane; i0 < count;
         i0 += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long i = i0 + lane;
        unsigned long long item = 0;
        uint32_t start = 0;
        if (i < count) {
            item = __ldcg(list + i);
            const Prob& P = probs ? probs[(int)(item >> 40)] : single;
            const int64_t cell = (int64_t)(item & kCellMask);
            const uint32_t deps = g_deps_global<E>(P, cell);
            if (deps) cnt_set(P, cell, kReadyAt - deps);
            else start = 0x100u;
        }
        frontier_push(0, (int64_t)(item & kCellMask), item & ~kCellMask, start, starts, &G->fcount[0],
                      (unsigned long long)P0.glist_cap);
    }
}

// Second launch: a walker from every start.  The last CTA to finish checks
// that every cell of every problem was computed.
template <Mode M, bool W, bool AREA>
__global__ void __launch_bounds__(256) k_global(const Prob* __restrict__ probs, Prob single,
                                                EngineGlobals* G, unsigned long long total_cells) {
    using E = Eng<M, W, AREA>;
    static_assert(E::kD8Fwd, "branching modes use k_global_levels");
    __shared__ unsigned long long s_done;
    const Prob& P0 = probs ? probs[0] : single;
    if (__ldcg(&G->glist_count) >= P0.skel_min) return;  // the skeleton solve takes them
    const unsigned long long count = G->fcount[0];
    const unsigned long long* starts = reinterpret_cast<const unsigned long long*>(P0.link);
    unsigned long long done = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long item = __ldcg(starts + i);
        const Prob& P = probs ? probs[(int)(item >> 40)] : single;
        done += walker_d8<W, AREA>(P, (int64_t)(item & ((1ull << 40) - 1)));
    }
    for (int o = 16; o; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);
    if (threadIdx.x == 0) s_done = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0 && done) atomicAdd(&s_done, done);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_done) atomicAdd(&G->done_cells, s_done);
        __threadfence();
        unsigned fin = atomicAdd(&G->finished_ctas, 1u);
        if (fin == gridDim.x - 1) {
            __threadfence();
            unsigned long long got = atomicAdd(&G->done_cells, 0ull);
            if (got != total_cells) atomicMax(&G->status, kStatusNoProgress);
        }
    }
}

// ---------------------------------------------------- level-synchronous global phase
// For the modes where a finished cell can make several cells ready (MFD
// forward; both adjoints) a walker that kept every extra ready cell to itself
// would run whole diverging regions on one thread.  Here the global cells are
// processed in rounds instead: round r computes every global cell whose global
// dependencies were all computed in earlier rounds (the frontier), and every
// cell that becomes ready goes to the next frontier.  The number of rounds is
// the length of the longest dependency chain among global cells (about 20 on
// the rough test DEMs).  Before the first round each global cell's arrival
// counter is set to kReadyAt minus its number of global dependencies, so
// readiness is a single atomic.  Rounds are separated by a grid barrier
// (cooperative launch, so all blocks are resident); the barrier's wait is
// bounded in time.

// The barrier's wait limit is a kernel argument: the library-wide value set
// by fr_set_wait_limit (default 10 s).

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over all blocks of a cooperative launch.  Returns false (and leaves
// FR_ERR_NO_PROGRESS in the status word) if the wait exceeds limit_ns.
static __device__ __noinline__ bool grid_barrier(EngineGlobals* G, unsigned nblocks,
                                                 unsigned long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_u32(&G->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&G->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&G->bar_count, 0u);
            __threadfence();
            atomicAdd(&G->bar_gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(&G->bar_gen) == gen) {
                __nanosleep(64);
                if (global_ns() - t0 > limit_ns) {
                    atomicMax(&G->status, kStatusNoProgress);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Computes one ready global cell; returns the codes of the targets it makes
// ready.
template <class E>
__device__ __noinline__ uint32_t step_round(const Prob& P, int64_t cur) {
    walker_compute<E>(P, cur);
    __threadfence();
    const uint32_t tm = g_targets<E>(P, cur);
    uint32_t gm = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if ((tm >> k) & 1u) gm |= (uint32_t)gbit(P, cur + offi(k, P.nx)) << k;
    uint32_t ready = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if ((gm >> k) & 1u) ready |= (uint32_t)(cnt_add(P, cur + offi(k, P.nx), 1u) == kReadyAt) << k;
    return ready;
}

// Frontier buffers: the walker-link region (first problem's link array; the
// links of all problems are contiguous) and the global-cell list, which is
// free once the first frontier has been built from it.
template <Mode M, bool W, bool AREA>
__global__ void __launch_bounds__(256) k_global_levels(const Prob* __restrict__ probs, Prob single,
                                                       EngineGlobals* G,
                                                       unsigned long long total_cells,
                                                       unsigned long long limit_ns) {
    using E = Eng<M, W, AREA>;
    __shared__ unsigned long long s_done;
    const Prob& P0 = probs ? probs[0] : single;
    unsigned long long* const buf_a = reinterpret_cast<unsigned long long*>(P0.link);
    unsigned long long* const buf_b = P0.glist;
    const unsigned long long cap = (unsigned long long)P0.glist_cap;
    const unsigned long long count = __ldcg(&G->glist_count);
    // only as many blocks as the global cells need take part (every block
    // computes the same number), so a small problem's barriers stay cheap
    const unsigned long long want = (count + blockDim.x - 1) / blockDim.x;
    const unsigned nb = (unsigned)(want < gridDim.x ? want : gridDim.x);
    const unsigned long long stride = (unsigned long long)nb * blockDim.x;
    // lanes walk the lists in warp-aligned steps, so every lane of a warp
    // runs the same number of steps (frontier_push needs the whole warp)
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long first = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x - lane;
    constexpr unsigned long long kCellMask = (1ull << 40) - 1;
    unsigned long long done = 0;
    bool ok = blockIdx.x < nb;
    // first frontier: global cells without global dependencies; the others'
    // counters start at kReadyAt - dependencies
    if (ok) for (unsigned long long i0 = first; i0 < count; i0 += stride) {
        const unsigned long long i = i0 + lane;
        unsigned long long item = 0;
        uint32_t start = 0;
        if (i < count) {
            item = __ldcg(buf_b + i);
            const Prob& P = probs ? probs[(int)(item >> 40)] : single;
            const int64_t cell = (int64_t)(item & kCellMask);
            const uint32_t deps = g_deps_global<E>(P, cell);
            if (deps) cnt_set(P, cell, kReadyAt - deps);
            else start = 0x100u;
        }
        frontier_push(0, (int64_t)(item & kCellMask), item & ~kCellMask, start, buf_a, &G->fcount[0], cap);
    }
    if (ok) ok = grid_barrier(G, nb, limit_ns);
    for (int round = 1; ok; ++round) {
        unsigned long long* cur = (round & 1) ? buf_a : buf_b;
        unsigned long long* nxt = (round & 1) ? buf_b : buf_a;
        const unsigned long long n = __ldcg(&G->fcount[(round - 1) % 3]);
        if (n == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) G->rounds = (unsigned long long)(round - 1);
            break;
        }
        // the counter two rounds back is free again: it becomes the next round's
        if (blockIdx.x == 0 && threadIdx.x == 0) G->fcount[(round + 1) % 3] = 0ull;
        unsigned long long* ncount = &G->fcount[round % 3];
        for (unsigned long long i0 = first; i0 < n; i0 += stride) {
            const unsigned long long i = i0 + lane;
            unsigned long long item = 0;
            uint32_t ready = 0;
            int64_t nx = 0;
            if (i < n) {
                item = __ldcg(cur + i);
                const Prob& P = probs ? probs[(int)(item >> 40)] : single;
                ready = step_round<E>(P, (int64_t)(item & kCellMask));
                nx = P.nx;
                ++done;
            }
            frontier_push(nx, (int64_t)(item & kCellMask), item & ~kCellMask, ready, nxt, ncount, cap);
        }
        ok = grid_barrier(G, nb, limit_ns);
    }
    for (int o = 16; o; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);
    if (threadIdx.x == 0) s_done = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0 && done) atomicAdd(&s_done, done);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_done) atomicAdd(&G->done_cells, s_done);
        __threadfence();
        const unsigned fin = atomicAdd(&G->finished_ctas, 1u);
        if (fin == gridDim.x - 1) {
            __threadfence();
            const unsigned long long got = atomicAdd(&G->done_cells, 0ull);
            if (got != total_cells) atomicMax(&G->status, kStatusNoProgress);
        }
    }
}

// Launches the global phase: D8 forward keeps the single-successor walkers
// (a D8 cell has one receiver, so nothing diverges); every other mode runs
// the level-synchronous kernel as a cooperative launch.
template <Mode M, bool W, bool AREA>
cudaError_t launch_global(const Prob* probs, const Prob& single, EngineGlobals* G,
                          unsigned long long total_cells, cudaStream_t s) {
    if constexpr (M == Mode::FwdD8) {
        k_global_init<M, W, AREA><<<walker_grid(), 256, 0, s>>>(probs, single, G);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_global<M, W, AREA><<<walker_grid(), 256, 0, s>>>(probs, single, G, total_cells);
        return cudaGetLastError();
    } else {
        static int grid_of[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        int grid = dev < 64 ? grid_of[dev] : 0;
        if (grid == 0) {
            int sms = 0, per = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_global_levels<M, W, AREA>, 256, 0);
            if (e != cudaSuccess) return e;
            if (per < 1) return cudaErrorInvalidConfiguration;
            // one block per SM: a round's frontier (about 20 K cells on an 8192^2
            // slope-split route) fits, and the grid barrier has the fewest
            // arrivals (measured faster than two or four blocks per SM)
            grid = sms;
            if (dev < 64) grid_of[dev] = grid;
        }
        Prob one = single;
        const Prob* pp = probs;
        unsigned long long total = total_cells;
        unsigned long long limit = wait_limit_ns();
        void* args[] = {(void*)&pp, (void*)&one, (void*)&G, (void*)&total, (void*)&limit};
        return cudaLaunchCooperativeKernel((const void*)k_global_levels<M, W, AREA>, dim3(grid),
                                           dim3(256), args, 0, s);
    }
}

}  // namespace fr

// fr_d8.cu -- local phase of D8 forward accumulation over halo-extended tiles.
//
// Each CTA owns an inner tile of TX x TY cells and solves the extended region
// (inner tile plus an H-cell halo on every side) exactly in shared memory: the
// paper's per-subdomain high-to-low solve (Sec. 2.4), with overlapping
// subdomains.  An inner cell is final unless its upstream basin reaches
// outside the extended region ("global"); on the synthetic fractal DEMs a
// 4-cell halo leaves about 0.03 % of the cells global, which the walker kernel
// of fr_engine.cuh then finishes.  Halo cells are solved only to feed the
// inner ones and are not written.
//
// Solve: every cell waits for all its donors.  A cell's packed word (arrival
// count, donors' area sum) starts at its preset; each donor, once final, adds
// its local area with one shared-memory atomic.  The cells without donors
// (leaves, two thirds of a rough DEM) are final at once and arrive in one
// parallel pass; the receivers they complete form a list, and walkers drain
// it: a walker finalises its cell, arrives at the receiver, and continues
// with the receiver if it arrived last ("last arriver continues").  No
// block barrier separates the cells of a chain, each cell is visited once, and
// a cell's two-float value is pulled from its final donors in fixed code
// order (deterministic sums; exact 16-bit local areas).  The visiting order
// is a topological order of the routing graph (Sec. 3.2).  Donors in the ring
// around the region never arrive, so exactly the cells with upstream water
// outside the region (and cells on a routing cycle) stay unfinished; the inner
// ones are listed as global.
//
// Tiles away from the grid boundary take a vector path: code and rain rows are
// copied asynchronously (cp.async) in one batch, and the donor masks and
// arrival counts of four consecutive cells are computed together on packed
// bytes (a byte-permute builds each neighbour vector, an exact zero-byte test
// compares four codes at once).  Tiles touching the boundary take a scalar
// path with bounds tests.
#include <cuda/atomic>

#include "fr_engine.cuh"

namespace fr {
namespace {

constexpr int D8H = 4;

template <int TX_, int TY_, int NT_ = 512>
struct D8Geo {
    static constexpr int TX = TX_, TY = TY_, H = D8H;
    static constexpr int NT = NT_;  // threads per CTA
    static constexpr int EX = TX + 2 * H, EY = TY + 2 * H, NE = EX * EY;  // extended region
    static constexpr int RY = EY + 2;  // region plus a one-cell ring
    static constexpr int CP = EX + 8;  // padded row pitch (bytes) of ring-sized byte arrays
    // Ring coordinates (rx, ry), 0 <= rx < EX + 2, live at byte ry * CP + rx + 3;
    // region cell (ex, ey) is ring cell (ex + 1, ey + 1), byte (ey + 1) * CP + ex + 4,
    // so groups of four region cells starting at ex % 4 == 0 are word aligned.
    static_assert(NE < 65535, "local areas and indices are 16-bit");
    static_assert(EX % 4 == 0 && CP % 8 == 0 && TX % 4 == 0, "four-cell groups");
};

// Packed per-cell word of the walker solve: a count (bits 20-23) that reaches
// kPkDone = 9 when the cell is final -- its preset adds 9 - donors (at least
// one, so exactly one add completes the count) and every donor adds one --
// and the donors' local area sum (bits 0-15; the extended region has fewer
// than 2^16 cells).  Donors in the ring around the region never arrive, so a
// cell with upstream water outside the region never becomes final.
constexpr uint32_t kPkArrive = 1u << 20, kPkArea = 0xFFFFu, kPkDone = 9u;
// Shared code of a cell without a receiver in the grid whose routing byte is
// not FR_SINK (an invalid code, or one pointing out of the grid).
constexpr uint8_t kNoRecv = 0xFE;
__device__ __forceinline__ bool pk_final(uint32_t pk) { return (pk >> 20) == kPkDone; }

// Shared memory of one tile; per-cell arrays use the ring layout of `code`
// (ring cell (rx, ry) at ry * CP + rx + 3).
template <class Gm, bool W>
struct SmemD8 {
    static constexpr int NR = Gm::RY * Gm::CP;
    float vhi[W ? NR : 4];
    float vlo[W ? NR : 4];
    alignas(16) uint32_t pk[NR];                  // packed arrivals / donors' area
    alignas(16) uint8_t code[NR];                 // receiver codes of region + ring, padded rows
    alignas(16) uint8_t dm[W ? NR : 16];          // donor masks (value pulls)
    uint16_t queue[Gm::NE];                       // ready list: cells whose donors (all leaves) finished in the
                                                  // leaf pass; after the walk, the inner tile's unfinished cells
    int qtail;                                    // its length
    int head;                                     // next entry to hand out
    int nglob;                                    // unfinished inner cells listed in queue after the walk
    unsigned long long gbase;
    unsigned int done, sinks;  // block sums of the publish step (at most 2^16 and NE)
};

// Warp-aggregated append of four optional cells per lane (-1: none; all lanes
// call): one ballot per slot, one atomic per warp.
template <class S_>
__device__ __forceinline__ void push4(S_& S, const int (&cq)[4]) {
    const unsigned lane = threadIdx.x & 31u, below = (1u << lane) - 1u;
    int prefix = 0, total = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned b = __ballot_sync(0xffffffffu, cq[q] >= 0);
        prefix += __popc(b & below);
        total += __popc(b);
    }
    if (!total) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(&S.qtail, total);
    int pos = __shfl_sync(0xffffffffu, base, 0) + prefix;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (cq[q] >= 0) S.queue[pos++] = (uint16_t)cq[q];
}

// Warp-aggregated append of up to four cells per lane to the ready list (all
// lanes call; the scalar path).
template <class S_>
__device__ __forceinline__ void push_cells(S_& S, int n, const int (&cells)[4]) {
    const unsigned lane = threadIdx.x & 31u;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (!total) return;
    int base = 0;
    if (lane == 31) base = atomicAdd(&S.qtail, total);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - n;
    for (int q = 0; q < n; ++q) S.queue[base + q] = (uint16_t)cells[q];
}

// Per-byte population count.
__device__ __forceinline__ uint32_t popc_bytes(uint32_t x) {
    x = x - ((x >> 1) & 0x55555555u);
    x = (x & 0x33333333u) + ((x >> 2) & 0x33333333u);
    return (x + (x >> 4)) & 0x0F0F0F0Fu;
}

// The three 4-byte vectors (left, centre, right neighbours) of a group whose
// first byte is word w1 of a padded row.
struct Row3 {
    uint32_t l, c, r;
};
__device__ __forceinline__ Row3 row3(const uint8_t* row, int w1) {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(row);
    const uint32_t a = p[w1 - 1], b = p[w1], d = p[w1 + 1];
    return {__byte_perm(a, b, 0x6543), b, __byte_perm(b, d, 0x4321)};
}

// Neighbour vector of code k from the up / mid / down rows.
__device__ __forceinline__ uint32_t nbr(const Row3& up, const Row3& mid, const Row3& dn, int k) {
    switch (k) {
        case 0: return mid.r;  // E
        case 1: return up.c;   // N
        case 2: return mid.l;  // W
        case 3: return dn.c;   // S
        case 4: return up.r;   // NE
        case 5: return up.l;   // NW
        case 6: return dn.l;   // SW
        default: return dn.r;  // SE
    }
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Lists the block's unfinished inner cells (local indices in S.queue, S.nglob
// of them) as global: one list allocation per block, their bits or-ed once
// per word and warp.  Called by all threads after a barrier.
template <class S_>
__device__ __forceinline__ void list_global(S_& S, const Prob& P, EngineGlobals* G, int pid,
                                            int tx_inner, int64_t x0, int64_t y0, int nthreads) {
    const int ng = S.nglob;
    if (threadIdx.x == 0) S.gbase = atomicAdd(&G->glist_count, (unsigned long long)ng);
    __syncthreads();
    const unsigned long long base = S.gbase;
    const int ng32 = (ng + 31) & ~31;
    for (int i = threadIdx.x; i < ng32; i += nthreads) {
        int64_t gi = -1;
        if (i < ng) {
            const int c = S.queue[i];
            const int ly = c / tx_inner, lx = c - ly * tx_inner;
            gi = (y0 + ly) * P.nx + x0 + lx;
            if (FR_OK((int64_t)(base + i), P.glist_cap, 17))
                P.glist[base + i] = ((unsigned long long)pid << 40) | (unsigned long long)gi;
        }
        // lanes whose cells share a word of bits or them together; one atomic per word
        const long long word = gi >= 0 ? (long long)(gi >> 5) : -1ll;
        const unsigned peers = __match_any_sync(0xffffffffu, word);
        const uint32_t bits = __reduce_or_sync(peers, gi >= 0 ? 1u << (gi & 31) : 0u);
        if (gi >= 0 && (int)(threadIdx.x & 31u) == __ffs(peers) - 1) atomicOr(P.gbits + word, bits);
    }
}

// Problem and tile of this CTA: one problem, or (batched) the problem whose
// tiles [prefix[p], prefix[p+1]) hold blockIdx.x.
__device__ __forceinline__ int batch_problem(const int64_t* __restrict__ prefix, int nprob,
                                             int64_t& lt) {
    int lo = 0, hi = nprob - 1;
    const int64_t b = (int64_t)blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    lt = b - prefix[lo];
    return lo;
}

template <class Gm, bool W, bool AREA, bool BATCH>
__global__ void __launch_bounds__(Gm::NT) k_local_d8(Prob Pone, EngineGlobals* G,
                                                  const Prob* __restrict__ probs,
                                                  const int64_t* __restrict__ prefix, int nprob) {
    constexpr int TX = Gm::TX, TY = Gm::TY, H = Gm::H, EX = Gm::EX, EY = Gm::EY, NE = Gm::NE;
    constexpr int RY = Gm::RY, CP = Gm::CP, NT8 = Gm::NT;
    using Sm = SmemD8<Gm, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm& S = *reinterpret_cast<Sm*>(smem_raw);
    const int tid = threadIdx.x;
    int64_t lt = (int64_t)blockIdx.x;
    const int pid = BATCH ? batch_problem(prefix, nprob, lt) : 0;
    const Prob& P = BATCH ? probs[pid] : Pone;
    // tile coordinates (tile counts fit 32 bits: grids have fewer than 2^62 cells)
    const int tiles_x = (int)((P.nx + TX - 1) / TX);
    const int ty = (int)lt / tiles_x, tx = (int)lt - ty * tiles_x;
    const int64_t x0 = (int64_t)tx * TX, y0 = (int64_t)ty * TY;
    // ring origin (may be negative) and the grid's extent in ring coordinates
    const int64_t ox = x0 - H - 1, oy = y0 - H - 1;
    const int gx_hi = (int)(P.nx - ox < EX + 2 ? P.nx - ox : EX + 2);
    const int gy_hi = (int)(P.ny - oy < RY ? P.ny - oy : RY);
    const int gx_lo = (int)(ox < 0 ? -ox : 0), gy_lo = (int)(oy < 0 ? -oy : 0);
    // vector path: the padded ring rows [x0 - H - 4, x0 + EX - H + 4) are inside
    // the grid, and the arrays allow aligned 8-byte / 16-byte access
    const bool vec = x0 >= H + 4 && x0 + EX - H + 4 <= P.nx && oy >= 0 && oy + RY <= P.ny &&
                     (P.nx & 7) == 0 && ((uintptr_t)P.rb & 7) == 0 &&
                     (!W || !P.init || ((uintptr_t)P.init & 15) == 0) &&
                     (!W || ((uintptr_t)P.out_hi & 15) == 0) &&
                     (!AREA || ((uintptr_t)P.area & 15) == 0);
    // a region cell's packed word starts at its preset (9 - donors) and each donor
    // adds one arrival; the add that completes the count to 9 finalises the cell.
    // Ring cells start at zero and get at most three arrivals, so they never
    // finish.  The vector path stores the presets after this barrier and zeroes
    // only the ring here; the scalar path adds the presets atomically, in any
    // order with the arrivals, onto a zeroed array.
    if (vec) {
        for (int i = tid; i < 2 * CP + 2 * EY; i += NT8) {
            const int r = i < 2 * CP ? (i < CP ? i : (RY - 1) * CP + i - CP)
                                     : (i - 2 * CP < EY ? (i - 2 * CP + 1) * CP + 3
                                                        : (i - 2 * CP - EY + 1) * CP + EX + 4);
            S.pk[r] = 0u;
        }
    } else {
        for (int i = tid; i < Sm::NR / 4; i += NT8) reinterpret_cast<uint4*>(S.pk)[i] = make_uint4(0, 0, 0, 0);
    }
    if (tid == 0) {
        S.qtail = 0;
        S.head = 0;
        S.nglob = 0;
    }

    if (vec) {
        // ---- asynchronous copies: code rows (8-byte chunks; byte b <-> grid
        // x = x0 - H - 4 + b) and rain rows (16-byte chunks)
        for (int i = tid; i < RY * (CP / 8); i += NT8) {
            const int ry = i / (CP / 8), w = i - ry * (CP / 8);
            const int64_t g = (oy + ry) * P.nx + (x0 - H - 4 + 8 * w);
            if (FR_OK(g + 7, ncell(P), 1)) cp_async8(S.code + ry * CP + 8 * w, P.rb + g);
        }
        if constexpr (W) {
            if (P.init) {
                for (int i = tid; i < EY * (EX / 4); i += NT8) {
                    const int ey = i / (EX / 4), q = i - ey * (EX / 4);
                    const int64_t g = (oy + ey + 1) * P.nx + (x0 - H + 4 * q);
                    if (FR_OK(g + 3, ncell(P), 8))
                        cp_async16(S.vhi + (ey + 1) * CP + 4 * q + 4, P.init + g);
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
        // ---- donor masks and presets (four cells per thread step, plain
        // stores); the leaves (no donors: final at once) and their receivers'
        // codes are kept in registers
        constexpr int NG = (NE / 4 + NT8 - 1) / NT8;
        static_assert(4 * NG <= 32, "leaf bits of a thread fit one word");
        uint32_t leaves = 0;       // bit 4 * it + q
        uint32_t lcode[NG];        // the four codes of group it
#pragma unroll
        for (int it = 0; it < NG; ++it) {
            const int gq = it * NT8 + tid;
            lcode[it] = 0;
            if (gq < NE / 4) {
                const int ey = gq / (EX / 4), ex = (gq - ey * (EX / 4)) * 4;
                const int w1 = (ex + 4) >> 2;
                const Row3 up = row3(S.code + ey * CP, w1);
                const Row3 mid = row3(S.code + (ey + 1) * CP, w1);
                const Row3 dn = row3(S.code + (ey + 2) * CP, w1);
                uint32_t dmf = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    dmf |= zero_bytes(nbr(up, mid, dn, k) ^ (0x01010101u * (uint32_t)opp(k))) >> (7 - k);
                const uint32_t wait = 0x09090909u - popc_bytes(dmf);  // kPkDone - donors
                const int r = (ey + 1) * CP + ex + 4;
                *reinterpret_cast<uint4*>(S.pk + r) =
                    make_uint4((wait & 0xFFu) << 20, ((wait >> 8) & 0xFFu) << 20,
                               ((wait >> 16) & 0xFFu) << 20, (wait >> 24) << 20);
                if constexpr (W) {
                    *reinterpret_cast<uint32_t*>(S.dm + r) = dmf;
                    if (!P.init) *reinterpret_cast<float4*>(S.vhi + r) = make_float4(1.f, 1.f, 1.f, 1.f);
                    *reinterpret_cast<float4*>(S.vlo + r) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                const uint32_t z = zero_bytes(dmf);  // 0x80 per leaf
                leaves |= (((z >> 7) & 1u) | ((z >> 14) & 2u) | ((z >> 21) & 4u) | ((z >> 28) & 8u)) << (4 * it);
                lcode[it] = mid.c;
            }
        }
        __syncthreads();
        // ---- the leaves arrive at their receivers; a receiver completed here
        // (its last donor was a leaf) goes to the ready list
#pragma unroll
        for (int it = 0; it < NG; ++it) {
            const int gq = it * NT8 + tid;
            int cq[4] = {-1, -1, -1, -1};
            const uint32_t lb = (leaves >> (4 * it)) & 0xFu;
            if (lb) {
                const int ey = gq / (EX / 4), ex = (gq - ey * (EX / 4)) * 4;
                const int r = (ey + 1) * CP + ex + 4;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t k = (lcode[it] >> (8 * q)) & 0xFFu;
                    if (!((lb >> q) & 1u) || k >= 8) continue;
                    const int t = r + q + offy((int)k) * CP + offx((int)k);
                    const uint32_t add = kPkArrive | 1u;
                    if (((atomicAdd(&S.pk[t], add) + add) >> 20) == kPkDone) cq[q] = t;
                }
            }
            push4(S, cq);
        }
    } else {
        // ---- scalar path (tiles touching the grid boundary)
        // codes without a receiver in the grid become kNoRecv unless they are
        // FR_SINK, so that kSink marks exactly the routing bytes FR_SINK (the
        // mass balance's sinks), as on the vector path, which keeps the bytes
        for (int i = tid; i < RY * CP; i += NT8) {
            const int ry = i / CP, rx = i - ry * CP - 3;
            uint8_t code = kNoRecv;
            if (rx >= gx_lo && rx < gx_hi && ry >= gy_lo && ry < gy_hi) {
                code = rd_rb(P, (oy + ry) * P.nx + (ox + rx));
                if (code < 8) {
                    const int xr = rx + offx(code), yr = ry + offy(code);
                    if (xr < gx_lo || xr >= gx_hi || yr < gy_lo || yr >= gy_hi) code = kNoRecv;
                } else if (code != kSink) {
                    code = kNoRecv;
                }
            }
            S.code[i] = code;
        }
        __syncthreads();
        for (int c0 = 0; c0 < NE; c0 += NT8) {
            const int c = c0 + tid;
            int cells[4];
            int n = 0;
            if (c < NE) {
                const int ey = c / EX, ex = c - ey * EX;
                const int rx = ex + 1, ry = ey + 1;
                const int r = ry * CP + rx + 3;
                uint32_t dm = 0;
                if (rx >= gx_lo && rx < gx_hi && ry >= gy_lo && ry < gy_hi) {
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        dm |= (uint32_t)(S.code[r + offy(k) * CP + offx(k)] == (uint8_t)opp(k)) << k;
                    if constexpr (W) {
                        const int64_t gi = (oy + ry) * P.nx + (ox + rx);
                        S.vhi[r] = P.init ? rd_in(P.init, P, gi, 8) : 1.0f;
                        S.vlo[r] = 0.0f;
                        S.dm[r] = (uint8_t)dm;
                    }
                    const uint32_t pre = (kPkDone - (uint32_t)__popc(dm)) << 20;
                    const uint32_t old = atomicAdd(&S.pk[r], pre);
                    if (((old + pre) >> 20) == kPkDone) {
                        if (dm) {
                            cells[n++] = r;
                        } else {
                            const uint32_t k = S.code[r];
                            if (k < 8) {
                                const int t = r + offy((int)k) * CP + offx((int)k);
                                const uint32_t add = kPkArrive | 1u;
                                if (((atomicAdd(&S.pk[t], add) + add) >> 20) == kPkDone) cells[n++] = t;
                            }
                        }
                    }
                }
                // outside the grid: no preset, no donors; never final
            }
            push_cells(S, n, cells);
        }
    }
    __syncthreads();

    // ---- walkers: a lane finalises a cell, adds it to its receiver's packed
    // word and continues with the receiver when it arrived last; otherwise it
    // takes the next start (warp-aggregated hand-out from the block's list)
    {
        const unsigned lane = tid & 31u;
        const unsigned below = (1u << lane) - 1u;
        const int nst = S.qtail;
        int c = -1;        // ring index of the cell being finalised
        uint32_t a = 0;    // its local area
        bool more = true;  // warp-uniform: list entries may be left
        for (;;) {
            if (more) {
                const unsigned idle = __ballot_sync(0xffffffffu, c < 0);
                if (idle) {
                    const int leader = __ffs(idle) - 1;
                    int base = 0;
                    if ((int)lane == leader) base = atomicAdd(&S.head, __popc(idle));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (c < 0) {
                        const int i = base + __popc(idle & below);
                        if (i < nst) {
                            c = S.queue[i];
                            a = 1u + (S.pk[c] & kPkArea);  // final: all donors arrived
                        }
                    }
                    if (base + __popc(idle) >= nst) more = false;
                }
            }
            if (!__any_sync(0xffffffffu, c >= 0)) break;
            if (c < 0) continue;
            if constexpr (W) {
                // the cell's donors are final: pull their values in ascending code order
                df v = {S.vhi[c], S.vlo[c]};
                for (uint32_t m = S.dm[c]; m; m &= m - 1) {
                    const int k = __ffs(m) - 1;
                    const int j = c + offy(k) * CP + offx(k);
                    v = df_add(v, df{S.vhi[j], S.vlo[j]});
                }
                S.vhi[c] = v.hi;
                S.vlo[c] = v.lo;
            }
            const uint32_t k = S.code[c];
            int next = -1;
            if (k < 8) {
                const int t = c + offy((int)k) * CP + offx((int)k);
                const uint32_t add = kPkArrive | a;
                uint32_t old;
                if constexpr (W) {
                    // release this cell's value; acquire the other donors' values
                    cuda::atomic_ref<uint32_t, cuda::thread_scope_block> ar(S.pk[t]);
                    old = ar.fetch_add(add, cuda::memory_order_acq_rel);
                } else {
                    old = atomicAdd(&S.pk[t], add);
                }
                if ((old >> 20) == kPkDone - 1u) {
                    next = t;
                    a = 1u + ((old + add) & kPkArea);
                }
            }
            c = next;
        }
    }
    __syncthreads();

    // ---- inner tile: publish final cells; a cell that did not finish has
    // upstream water outside the extended region (or lies on a cycle) and is
    // listed as global.  With areas, the areas of the finished cells whose
    // routing byte is FR_SINK are summed for the mass balance (the global
    // phase's cells are summed there from the global-cell bits).
    // Per-thread counts: at most 16 inner cells a thread, areas below 2^16.
    // Whole vector tiles count their finished cells as the inner cells less the
    // listed ones instead.
    uint32_t done = 0, sinks = 0;
    const bool whole = vec && x0 + TX <= P.nx && y0 + TY <= P.ny;
    auto need_lo_of = [&](int r, int lx, int ly) -> bool {
        // a cell's trailing word is pulled later when its receiver leaves the
        // inner tile (another tile may list it as global) or is global here
        const uint8_t k = S.code[r];
        if (k >= 8) return false;
        const int lxr = lx + offx(k), lyr = ly + offy(k);
        if (lxr < 0 || lyr < 0 || lxr >= TX || lyr >= TY) return true;
        return !pk_final(S.pk[r + offy(k) * CP + offx(k)]);
    };
    // an unfinished cell is appended to the block's list (S.queue, S.nglob)
    // and listed as global after the loops
    auto publish_one = [&](int lx, int ly) {
        const int64_t gx = x0 + lx, gy = y0 + ly;
        if (gx >= P.nx || gy >= P.ny) return;
        const int r = (ly + H + 1) * CP + lx + H + 4;
        const int64_t gi = gy * P.nx + gx;
        const uint32_t pkc = S.pk[r];
        if (!pk_final(pkc)) {
            S.queue[atomicAdd(&S.nglob, 1)] = (uint16_t)(ly * TX + lx);
            return;
        }
        ++done;
        if constexpr (W) {
            wr_f(P.out_hi, P, gi, S.vhi[r], 27);
            if (P.lo_full || need_lo_of(r, lx, ly)) wr_f(P.out_lo, P, gi, S.vlo[r], 28);
        }
        if constexpr (AREA) wr_area(P, gi, 1u + (pkc & kPkArea));
        if constexpr (AREA && !BATCH)
            if (S.code[r] == kSink) sinks += 1u + (pkc & kPkArea);
    };
    if (whole) {
        for (int gq = tid; gq < TX * TY / 4; gq += NT8) {
            const int ly = gq / (TX / 4), lx = (gq - ly * (TX / 4)) * 4;
            const int r = (ly + H + 1) * CP + lx + H + 4;
            const uint4 p4 = *reinterpret_cast<const uint4*>(S.pk + r);
            // counts never exceed 9 (binary 1001), so the AND is 9 only if all four are
            if (((p4.x & p4.y & p4.z & p4.w) >> 20) != kPkDone) {
                for (int q = 0; q < 4; ++q) publish_one(lx + q, ly);  // rare: global cells
                continue;
            }
            const int64_t gi = (y0 + ly) * P.nx + x0 + lx;
            if constexpr (W) {
                *reinterpret_cast<float4*>(P.out_hi + gi) = *reinterpret_cast<const float4*>(S.vhi + r);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (P.lo_full || need_lo_of(r + q, lx + q, ly))
                        wr_f(P.out_lo, P, gi + q, S.vlo[r + q], 28);
            }
            if constexpr (AREA) {
                ulonglong2* out = reinterpret_cast<ulonglong2*>(P.area + gi);
                out[0] = make_ulonglong2(1u + (p4.x & kPkArea), 1u + (p4.y & kPkArea));
                out[1] = make_ulonglong2(1u + (p4.z & kPkArea), 1u + (p4.w & kPkArea));
                if constexpr (!BATCH) {
                    // byte q of sk is 1 where routing byte q is FR_SINK; the areas
                    // are 1 + the 16-bit donor sums: a count plus two 16x8-bit dot
                    // products over the packed sums
                    const uint32_t sk = zero_bytes(~*reinterpret_cast<const uint32_t*>(S.code + r)) >> 7;
                    sinks += __popc(sk) + __dp2a_lo(__byte_perm(p4.x, p4.y, 0x5410), sk, 0u) +
                             __dp2a_hi(__byte_perm(p4.z, p4.w, 0x5410), sk, 0u);
                }
            }
        }
    } else {
        for (int i = tid; i < TX * TY; i += NT8) {
            const int ly = i / TX, lx = i - ly * TX;
            publish_one(lx, ly);
        }
    }
    // warp sums fit 32 bits (512 cells; areas of disjoint basins, below NE)
    const uint32_t done_w = whole ? 0u : __reduce_add_sync(0xffffffffu, done);
    uint32_t sinks_w = 0;
    if constexpr (AREA && !BATCH) sinks_w = __reduce_add_sync(0xffffffffu, sinks);
    if (tid == 0) {
        S.done = 0;
        S.sinks = 0;
    }
    __syncthreads();
    if ((tid & 31) == 0 && done_w) atomicAdd(&S.done, done_w);
    if (AREA && !BATCH && (tid & 31) == 0 && sinks_w) atomicAdd(&S.sinks, sinks_w);
    __syncthreads();
    if (tid == 0) {
        const unsigned long long d = whole ? (unsigned long long)(TX * TY - S.nglob) : S.done;
        if (d) atomicAdd(&G->done_cells, d);
        if (AREA && !BATCH && S.sinks) atomicAdd(&G->sink_area, (unsigned long long)S.sinks);
    }
    if (S.nglob) list_global(S, P, G, pid, TX, x0, y0, NT8);
}

template <class Gm, bool W, bool AREA, bool BATCH>
cudaError_t launch_local_d8(const Prob& P, EngineGlobals* G, const Prob* probs,
                            const int64_t* prefix, int nprob, int64_t tiles, cudaStream_t s) {
    constexpr size_t sm = sizeof(SmemD8<Gm, W>);
    static std::atomic<unsigned long long> set_on{0};
    cudaError_t e = smem_limit_once(k_local_d8<Gm, W, AREA, BATCH>, sm, set_on);
    if (e != cudaSuccess) return e;
    if (tiles > 0) k_local_d8<Gm, W, AREA, BATCH><<<(unsigned)tiles, Gm::NT, sm, s>>>(P, G, probs, prefix, nprob);
    return cudaGetLastError();
}

template <class Gm, bool W, bool AREA>
cudaError_t launch_d8(const Prob& P, EngineGlobals* G, cudaStream_t s) {
    const int64_t tiles = ((P.nx + Gm::TX - 1) / Gm::TX) * ((P.ny + Gm::TY - 1) / Gm::TY);
    cudaError_t e = launch_local_d8<Gm, W, AREA, false>(P, G, nullptr, nullptr, 1, tiles, s);
    if (e != cudaSuccess) return e;
    // both global phases are enqueued; each returns at once unless the
    // global-cell count selects it (walkers below P.skel_min, skeleton above)
    e = launch_global<Mode::FwdD8, W, AREA>(nullptr, P, G, (unsigned long long)(P.nx * P.ny), s);
    if (e != cudaSuccess || P.skel_min == ~0ull) return e;
    return launch_d8_skeleton(W, AREA, P, G, s);
}

template <class Gm, bool W, bool AREA>
cudaError_t launch_d8_batch(const Prob* probs, const int64_t* prefix, int nprob, int64_t tiles,
                            unsigned long long total_cells, EngineGlobals* G, cudaStream_t s) {
    Prob none{};
    cudaError_t e = launch_local_d8<Gm, W, AREA, true>(none, G, probs, prefix, nprob, tiles, s);
    if (e != cudaSuccess) return e;
    return launch_global<Mode::FwdD8, W, AREA>(probs, none, G, total_cells, s);
}

using GeoD8 = D8Geo<kD8TileX, kD8TileY>;        // geometry 0: 128x32
using GeoD8s = D8Geo<kD8TileX / 2, kD8TileY>;   // geometry 1: 64x32
using GeoD8w = D8Geo<96, 48>;                   // geometry 2: 96x48

template <class Gm>
cudaError_t d8_batch_w(bool want_w, bool want_area, const Prob* probs, const int64_t* prefix,
                       int nprob, int64_t tiles, unsigned long long cells, EngineGlobals* G,
                       cudaStream_t s) {
    if (want_w && want_area) return launch_d8_batch<Gm, true, true>(probs, prefix, nprob, tiles, cells, G, s);
    if (want_w) return launch_d8_batch<Gm, true, false>(probs, prefix, nprob, tiles, cells, G, s);
    return launch_d8_batch<Gm, false, true>(probs, prefix, nprob, tiles, cells, G, s);
}

}  // namespace

// D8 forward accumulation: halo-tile local phase + walker phase.
cudaError_t launch_d8_forward(bool want_w, bool want_area, const Prob& P, EngineGlobals* G,
                              cudaStream_t s) {
    // With values a region cell needs 14 bytes of shared memory: 96x48 inner
    // tiles (1.26x halo redundancy, two blocks of about 103 KB per SM).  Areas
    // alone need 5 bytes, which leaves room for 128x64 tiles (1.20x, three
    // blocks per SM).  Each measured fastest among 64x32 ... 128x96 for its
    // case (with values: 128x32 and 64x64 were 5 % slower at 4096^2).
    if (want_w && want_area) return launch_d8<GeoD8w, true, true>(P, G, s);
    if (want_w) return launch_d8<GeoD8w, true, false>(P, G, s);
    return launch_d8<D8Geo<kD8TileX, 2 * kD8TileY>, false, true>(P, G, s);
}

// Batched D8 forward: the CTAs of all problems' tiles in one launch (tile
// prefix of the chosen geometry), then one walker phase.
cudaError_t launch_d8_forward_batch(int geo, bool want_w, bool want_area, const Prob* probs,
                                    const int64_t* prefix, int nprob, int64_t tiles,
                                    unsigned long long total_cells, EngineGlobals* G, cudaStream_t s) {
    if (geo == 1) return d8_batch_w<GeoD8s>(want_w, want_area, probs, prefix, nprob, tiles, total_cells, G, s);
    if (geo == 2) return d8_batch_w<GeoD8w>(want_w, want_area, probs, prefix, nprob, tiles, total_cells, G, s);
    return d8_batch_w<GeoD8>(want_w, want_area, probs, prefix, nprob, tiles, total_cells, G, s);
}

}  // namespace fr

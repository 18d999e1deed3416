// fr_skel.cu -- global phase of D8 forward accumulation on the skeleton of a
// tile decomposition, for DEMs with long rivers.
//
// After the halo-tile local phase (fr_d8.cu) every cell is either final or
// "global": its upstream basin leaves its tile's extended region.  On a rough
// DEM global cells are rare and short, and the cell walkers of fr_engine.cuh
// finish them in microseconds.  On a depression-filled DEM (the paper routes
// one, Sec. 4) or on a plane, rivers run across the whole grid: the global
// cells are the river trunks, thousands of cells long, and a walker that
// follows a trunk one cell per dependent step takes tens to hundreds of
// milliseconds.  This file solves the same global cells exactly on the
// skeleton of a second, non-overlapping decomposition into 64x64 tiles, the
// solve on "the skeleton of the domain decomposition" that Sec. 2.4 mentions,
// made exact for single-receiver routing:
//
//  A. per tile (k_skel_a), in shared memory: every global cell i gets its
//     in-tile partial value L(i) = c(i) + sum of L over its global donors in
//     the tile, where c(i) = rain(i) + the final values of its non-global
//     donors.  Areas alone: by the log-depth chain contraction
//     (contract_push: pointer jumping along single-donor chains, walkers over
//     the chains' heads), or, in tiles of long straight chains, by walkers
//     over the cells (walk_push); with water, by walkers (walk_pull).  An
//     entry (a global cell with global donors in other tiles) follows the
//     in-tile receivers to the exit it drains to (a global cell whose
//     receiver lies in another tile; D8 paths are unique), or to the end of
//     its path inside the tile.  Each exit x gets the list of its
//     dependencies: the exits y of neighbouring tiles that drain into an
//     entry whose path reaches x, in a fixed order.
//  B. walkers over the exits (k_skel_walk): the total water of an exit is
//         O(x) = L(x) + sum over its dependencies y of O(y);
//     an exit with no dependency starts a walker, which computes O(x), then
//     arrives at the exit its receiver drains to; the arrival that completes
//     an exit's count continues there ("last arriver continues").  One step
//     crosses a whole tile.
//  C. per tile again (k_skel_fix): each entry's inflow (the sum of O over its
//     donors in other tiles) is passed down the in-tile receivers (the same
//     in-tile solve as A, with the inflows as start values) and added to L of
//     every global cell below it; exits keep O from B.
//
// Sums run in fixed orders (donors in code order, dependency lists in
// row-major entry order), so results are bit-reproducible; they differ from
// the cell walkers' only in the order of the two-float additions.  Unit-rain
// areas are exact integers either way.  A routing graph with a cycle leaves
// cells unfinished; the last CTA of C compares the count of finished cells
// with the number of cells.
#include <cuda/atomic>

#include "fr_engine.cuh"

namespace fr {
namespace {

constexpr int SX = kSkelTile, SY = kSkelTile, SN = SX * SY;
constexpr int SRX = SX + 2, SRY = SY + 2, SRN = SRX * SRY;  // with a one-cell ring
constexpr int kSkNT = 256;
static_assert(SN <= 4096, "local indices take 12 bits");
static_assert(kSkelPool == 2 * (SX + SY) + 4, "dependency slots per tile: the ring cells");

// Cell byte of the ring arrays: the receiver code (bits 0-3; 15 = none, also
// for receivers outside the grid) and the global flag.
constexpr uint8_t kNoCode = 15, kGlob = 0x80;

// In-tile walker words.  Areas alone (push): one 64-bit word per cell, a
// count in bits 56-63 that reaches kDone when the cell is final (its preset
// adds kDone - in-tile global donors, at least one; every donor adds one),
// an inflow-poison count in bits 48-55 and the value in bits 0-47, to which
// each donor adds its own: integer adds commute, so no value needs a fence.
// Two-float values (pull): a 32-bit word with the pending count (bits 0-3)
// and flags; a final cell pulls its donors' values in code order.
constexpr unsigned long long kPwOne = 1ull << 56, kPwPois = 1ull << 48, kPwVal = (1ull << 48) - 1;
constexpr unsigned kDone = 9;
constexpr uint32_t kFin = 1u << 31, kPoison = 1u << 30, kUp = 1u << 29;
// Successor word of a global cell: its in-tile global receiver (local index,
// bits 0-11), or the cell itself with kPtrFinal set when its in-tile path
// ends there, and kPtrExit when it ends by leaving the tile.
constexpr uint16_t kPtrFinal = 1u << 12, kPtrExit = 1u << 13;

// Link word of a boundary cell (per cell, 8 bytes, in the workspace):
//   exit:   kind 2, pending dependencies (bits 0-15), list begin (16-31),
//           list length (32-47);
//   entry:  kind 1, the exit its in-tile path reaches (cell index, bits 0-39);
//   else 0 (an entry whose path ends inside its tile).
constexpr unsigned long long kLkExit = 2ull << 62, kLkEntry = 1ull << 62, kLkKind = 3ull << 62;
constexpr unsigned long long kLkCell = (1ull << 40) - 1;
// Pending count of an exit whose in-tile partial value was never computed (a
// cycle upstream of it inside its tile): never reached by arrivals.
constexpr unsigned long long kLkNever = 0xFFFFull;

struct TileGeo {
    int64_t x0, y0;  // origin
    int ex, ey;      // extent (partial tiles at the grid's far edges)
    int tiles_x;
};

__device__ __forceinline__ TileGeo tile_geo(const Prob& P, int64_t t) {
    TileGeo g;
    g.tiles_x = (int)((P.nx + SX - 1) / SX);
    const int64_t ty = t / g.tiles_x, tx = t - ty * g.tiles_x;
    g.x0 = tx * SX;
    g.y0 = ty * SY;
    g.ex = (int)(P.nx - g.x0 < SX ? P.nx - g.x0 : SX);
    g.ey = (int)(P.ny - g.y0 < SY ? P.ny - g.y0 : SY);
    return g;
}

// Boundary cells of a tile in row-major order: index b <-> (lx, ly).
__device__ __forceinline__ int nboundary(int ex, int ey) {
    const int mid = ey > 2 ? ey - 2 : 0, per = ex > 1 ? 2 : 1;
    return ex + mid * per + (ey > 1 ? ex : 0);
}
__device__ __forceinline__ void bcell(int b, int ex, int ey, int& lx, int& ly) {
    const int mid = ey > 2 ? ey - 2 : 0, per = ex > 1 ? 2 : 1;
    if (b < ex) {
        lx = b;
        ly = 0;
        return;
    }
    b -= ex;
    if (b < mid * per) {
        ly = 1 + b / per;
        lx = (b % per) ? ex - 1 : 0;
        return;
    }
    lx = b - mid * per;
    ly = ey - 1;
}
__device__ __forceinline__ int bindex(int lx, int ly, int ex, int ey) {
    const int mid = ey > 2 ? ey - 2 : 0, per = ex > 1 ? 2 : 1;
    if (ly == 0) return lx;
    if (ly == ey - 1) return ex + mid * per + lx;
    return ex + (ly - 1) * per + (lx == 0 ? 0 : 1);
}

template <bool W, bool AREA>
struct SmemSk {
    static constexpr bool kPush = AREA && !W;
    uint8_t cg[SRN];                                    // ring layout: code | kGlob
    uint8_t dm[kPush ? 1 : SN];                         // pull: in-tile global donors (codes)
    alignas(16) unsigned long long pw[kPush ? SN : 1];  // push: count | poison | value
    uint32_t pk[kPush ? 1 : SN];                        // pull: pending count | flags
    float hi[W ? SN : 1], lo[W ? SN : 1];               // pull: two-float values
    unsigned long long ar[(W && AREA) ? SN : 1];        // pull: areas beside the water
    uint16_t qp[SN];                                    // walker start list
    uint16_t sc[SN];                                    // successor words of the global cells
    uint8_t nin[SN];                                    // in-tile global donors of each global cell
    uint16_t gl[SN];                                    // the tile's global cells, row-major
    uint16_t broot[SX * 4];                             // per boundary cell: end of its in-tile path
    uint16_t bslots[SX * 4];                            // per boundary cell: dependency slots (exits: list length)
    uint16_t bbeg[SX * 4];                              // per exit: list begin
    uint16_t brank[SX * 4];                             // per entry: offset in its exit's list
    int bdep[SX * 4];                                   // push: per exit, its dependencies
    uint8_t bnd[SX * 4];                                // per boundary cell: global donors in other tiles
    unsigned long long bval[SX * 4];                    // pass C: entry inflow (push: value | poison;
    float bhi[W ? SX * 4 : 1], blo[W ? SX * 4 : 1];     //   pull: two-float, areas, flags)
    uint32_t bfl[SX * 4];
    uint8_t wtmp[32];                                   // warp-0 scratch
    int wsum[kSkNT / 32];                               // block scan
    int qtail, head, ng;
};

__device__ __forceinline__ bool in_ext(int lx, int ly, const TileGeo& g) {
    return lx >= 0 && ly >= 0 && lx < g.ex && ly < g.ey;
}

// Loads the receiver codes and global flags of a tile and its ring (all
// loads issued before any is used), then lists the tile's global cells in
// row-major order (S.gl, S.ng).
template <class S_>
__device__ void load_tile(S_& S, const Prob& P, const TileGeo& g) {
    // interior tiles of a grid whose rows are 32-cell aligned: 16-byte code
    // chunks and one word of global bits per chunk (grid x in [x0 - 16, x0 + 80))
    if (g.ex == SX && g.ey == SY && (P.nx & 31) == 0 && ((uintptr_t)P.rb & 15) == 0 && g.x0 >= 16 &&
        g.x0 + SX + 16 <= P.nx && g.y0 >= 1 && g.y0 + SY + 1 <= P.ny) {
        constexpr int CH = (SX + 32) / 16, NCH = SRY * CH;
        constexpr int PER2 = (NCH + kSkNT - 1) / kSkNT;
        uint4 cv[PER2];
        uint32_t bw[PER2];
#pragma unroll
        for (int q = 0; q < PER2; ++q) {
            const int i = threadIdx.x + q * kSkNT;
            cv[q] = make_uint4(0, 0, 0, 0);
            bw[q] = 0;
            if (i < NCH) {
                const int ry = i / CH, ch = i - ry * CH;
                const int64_t g0 = (g.y0 - 1 + ry) * P.nx + g.x0 - 16 + 16 * ch;
                cv[q] = __ldg(reinterpret_cast<const uint4*>(P.rb + g0));
                bw[q] = __ldg(P.gbits + (g0 >> 5)) >> (g0 & 31);
            }
        }
#pragma unroll
        for (int q = 0; q < PER2; ++q) {
            const int i = threadIdx.x + q * kSkNT;
            if (i >= NCH) break;
            const int ry = i / CH, ch = i - ry * CH;
            const uint32_t w4[4] = {cv[q].x, cv[q].y, cv[q].z, cv[q].w};
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int rx = 16 * ch - 15 + j;  // ring column of grid x0 - 16 + 16 ch + j
                if (rx < 0 || rx >= SRX) continue;
                const uint32_t k = (w4[j >> 2] >> (8 * (j & 3))) & 0xFFu;
                // interior tile: every ring cell's receiver lies in the grid
                S.cg[ry * SRX + rx] = (uint8_t)((k < 8 ? k : kNoCode) | (((bw[q] >> j) & 1u) ? kGlob : 0u));
            }
        }
    } else {
    constexpr int PER = (SRN + kSkNT - 1) / kSkNT;
    uint8_t kb[PER];
    uint32_t gw[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = threadIdx.x + q * kSkNT;
        const int ry = i / SRX, rx = i - ry * SRX;
        const int64_t gx = g.x0 - 1 + rx, gy = g.y0 - 1 + ry;
        kb[q] = 0xFF;
        gw[q] = 0;
        if (i < SRN && gx >= 0 && gy >= 0 && gx < P.nx && gy < P.ny) {
            const int64_t gi = gy * P.nx + gx;
            kb[q] = rd_rb(P, gi);
            gw[q] = __ldg(P.gbits + (gi >> 5)) >> (gi & 31);
        }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = threadIdx.x + q * kSkNT;
        if (i >= SRN) break;
        const int ry = i / SRX, rx = i - ry * SRX;
        const int64_t gx = g.x0 - 1 + rx, gy = g.y0 - 1 + ry;
        uint8_t c = kNoCode;
        const uint32_t k = kb[q];
        if (k < 8) {
            const int64_t tx = gx + offx(k), ty = gy + offy(k);
            if (tx >= 0 && ty >= 0 && tx < P.nx && ty < P.ny) c = (uint8_t)k;
        }
        if (gw[q] & 1u) c |= kGlob;
        S.cg[i] = c;
    }
    }
    __syncthreads();
    // compact list: thread t takes cells [CPT t, CPT t + CPT)
    constexpr int CPT = SN / kSkNT;
    static_assert(CPT * kSkNT == SN && CPT <= 32, "cells per thread");
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
        const int c = threadIdx.x * CPT + j;
        const int ly = c / SX, lx = c - ly * SX;
        if (lx < g.ex && ly < g.ey && (S.cg[(ly + 1) * SRX + lx + 1] & kGlob)) m |= 1u << j;
    }
    const unsigned lane = threadIdx.x & 31u;
    const int cnt = __popc(m);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += u;
    }
    if (lane == 31) S.wsum[threadIdx.x >> 5] = incl;
    __syncthreads();
    int off = incl - cnt, total = 0;
#pragma unroll
    for (int w = 0; w < kSkNT / 32; ++w) {
        const int v = S.wsum[w];
        if (w < (int)(threadIdx.x >> 5)) off += v;
        total += v;
    }
    for (uint32_t mm = m; mm; mm &= mm - 1) S.gl[off++] = (uint16_t)(threadIdx.x * CPT + __ffs(mm) - 1);
    if (threadIdx.x == 0) S.ng = total;
    __syncthreads();
}

// Warp-aggregated append of one optional local cell per lane (all lanes call).
template <class S_>
__device__ __forceinline__ void push_start(S_& S, int cell) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(0xffffffffu, cell >= 0);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if ((int)lane == leader) base = atomicAdd(&S.qtail, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (cell >= 0) S.qp[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)cell;
}

// Warp-aggregated hand-out of the start list: returns the next start for
// idle lanes (c < 0), -1 when none is left.
template <class S_>
__device__ __forceinline__ void hand_out(S_& S, int nst, int& c, bool& more) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned idle = __ballot_sync(0xffffffffu, c < 0);
    if (!idle) return;
    const int leader = __ffs(idle) - 1;
    int base = 0;
    if ((int)lane == leader) base = atomicAdd(&S.head, __popc(idle));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c < 0) {
        const int i = base + __popc(idle & ((1u << lane) - 1u));
        if (i < nst) c = S.qp[i];
    }
    if (base + __popc(idle) >= nst) more = false;
}

// Warp-aggregated hand-out over the global-cell list, keeping only the heads
// without donors (the starts of contract_push): returns the next one for idle
// lanes (c < 0), -1 when the list is exhausted.
template <class S_>
__device__ __forceinline__ void hand_out_filtered(S_& S, int ng, int& c, bool& more) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned idle = __ballot_sync(0xffffffffu, c < 0);
    if (!idle) return;
    const int leader = __ffs(idle) - 1;
    int base = 0;
    if ((int)lane == leader) base = atomicAdd(&S.head, __popc(idle));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c < 0) {
        const int i = base + __popc(idle & ((1u << lane) - 1u));
        if (i < ng) {
            const int x = S.gl[i];
            if (S.nin[x] == 0) c = x;
        }
    }
    if (base + __popc(idle) >= ng) more = false;
}

// Successor word of global cell c (local index; ring index r): its in-tile
// global receiver, or c itself marked final (and exit if the receiver is a
// global cell of another tile).
__device__ __forceinline__ uint16_t succ_word(const uint8_t* cg, int c, int r, const TileGeo& g) {
    const int ly = c / SX, lx = c - ly * SX;
    const int k = cg[r] & 15;
    if (k < 8 && (cg[r + offy(k) * SRX + offx(k)] & kGlob)) {
        if (in_ext(lx + offx(k), ly + offy(k), g)) return (uint16_t)(c + offy(k) * SX + offx(k));
        return (uint16_t)(c | kPtrFinal | kPtrExit);
    }
    return (uint16_t)(c | kPtrFinal);
}

// In-tile walker solve over the global cells, areas alone: a final cell
// adds its word (one arrival, its poison flag, its value) to its in-tile
// global receiver's; the add that completes the receiver's count continues
// there ("last arriver continues").  The walker carries the final word.
template <class S_>
__device__ void walk_push(S_& S) {
    const int nst = S.qtail;
    int c = -1;
    unsigned long long w = 0;
    bool more = true;
    for (;;) {
        if (more) {
            const int was = c;
            hand_out(S, nst, c, more);
            if (was < 0 && c >= 0) w = S.pw[c];  // a start: final at its preset
        }
        if (!__any_sync(0xffffffffu, c >= 0)) break;
        if (c < 0) continue;
        const uint16_t p = S.sc[c];
        int next = -1;
        if (!(p & kPtrFinal)) {
            const int t = p;
            const unsigned long long add = kPwOne | ((w >> 48) & 0xFFull ? kPwPois : 0ull) | (w & kPwVal);
            if (S.nin[t] == 1) {
                // the receiver's only in-tile donor: nothing else arrives there
                w = S.pw[t] + add;
                S.pw[t] = w;
                next = t;
            } else {
                const unsigned long long old = atomicAdd(&S.pw[t], add);
                if ((old >> 56) == kDone - 1) {
                    next = t;
                    w = old + add;
                }
            }
        }
        c = next;
    }
}

// In-tile solve over the global cells, areas alone, in O(log L) dependent
// rounds for chains of length L (log-depth chain contraction).  A global cell
// with exactly one in-tile global donor is a chain cell; the others are heads
// (no donor: a start; several: a confluence).  Every chain runs from a head
// through chain cells to its tail, the last cell before a head, a tile exit or
// the path's end.
//   1. Each chain cell's word becomes (value, poison bit 48, donor J in bits
//      49-60, bit 63 while J is a chain cell).
//   2. Pointer jumping: a chain cell adds the value and poison of J and takes
//      J's own J, until J is a head.  Reads and writes of a packed word are
//      single 64-bit accesses, so every word read pairs a J with the sum from J
//      (exclusive) to the cell; updates may therefore run in any order.  At
//      most log2(cells) + 1 rounds; a chain cell still unresolved then lies on
//      a cycle.
//   3. Each head learns the tail of its chain (S.qp, indexed by head).
//   4. Walkers over the heads: a final head's value plus the tail's sum is the
//      tail's value, which arrives at the tail's receiver (a head): one
//      arrival (count bits 56-63), its poison (bits 48-55) and its value; the
//      arrival that completes a head continues there ("last arriver
//      continues").
//   5. Every chain cell whose head is final gets the head's value plus its sum.
// The values are integer sums, so the order of the additions does not matter.
constexpr unsigned long long kCwChain = 1ull << 63, kCwPois = 1ull << 48;
// Cells per start from which a tile takes the walk instead of the contraction.
constexpr int kWalkCellsPerStart = 32;
__device__ __forceinline__ int cw_j(unsigned long long w) { return (int)((w >> 49) & 0xFFFull); }

template <class S_>
__device__ void contract_push(S_& S, int ng) {
    const int tid = threadIdx.x;
    // 1. chain cells take their donor
    for (int i = tid; i < ng; i += kSkNT) {
        const int c = S.gl[i];
        const uint16_t p = S.sc[c];
        if (p & kPtrFinal) continue;
        const int t = p;
        if (S.nin[t] != 1) continue;
        const unsigned long long wt = S.pw[t];
        const bool pois = ((wt >> 48) & 0xFFull) != 0;
        S.pw[t] = (wt & kPwVal) | (pois ? kCwPois : 0ull) | ((unsigned long long)c << 49) |
                  (S.nin[c] == 1 ? kCwChain : 0ull);
    }
    __syncthreads();
    // 2. pointer jumping (other threads update words concurrently: volatile
    // 64-bit accesses, each a single shared-memory transaction, so any word
    // read is consistent); the block leaves together when no word still
    // points at a chain cell
    volatile unsigned long long* vpw = S.pw;
    for (int round = 0; round < 14; ++round) {
        int more = 0;
        for (int i = tid; i < ng; i += kSkNT) {
            const int c = S.gl[i];
            if (S.nin[c] != 1) continue;
            const unsigned long long w = vpw[c];
            if (!(w & kCwChain)) continue;
            const unsigned long long wj = vpw[cw_j(w)];
            const unsigned long long v = ((w & kPwVal) + (wj & kPwVal)) & kPwVal;
            vpw[c] = v | ((w | wj) & kCwPois) | (wj & (0xFFFull << 49)) | (wj & kCwChain);
            more |= (wj & kCwChain) != 0;
        }
        if (!__syncthreads_or(more)) break;
    }
    // 3. tails (S.qp[head] = its chain's tail; a head without a chain is its own)
    for (int i = tid; i < ng; i += kSkNT) {
        const int c = S.gl[i];
        S.qp[c] = (uint16_t)c;
    }
    __syncthreads();
    for (int i = tid; i < ng; i += kSkNT) {
        const int c = S.gl[i];
        const uint16_t p = S.sc[c];
        const bool tail = (p & kPtrFinal) || S.nin[p & 0xFFF] != 1;
        if (!tail) continue;
        if (S.nin[c] == 1) {
            const unsigned long long w = S.pw[c];
            if (!(w & kCwChain)) S.qp[cw_j(w)] = (uint16_t)c;  // else on a cycle
        }
    }
    __syncthreads();
    // 4. walkers over the heads; starts are the heads without donors, taken
    // from the global-cell list
    {
        int c = -1;
        unsigned long long w = 0;
        bool more = true;
        for (;;) {
            if (more) {
                const int was = c;
                hand_out_filtered(S, ng, c, more);
                if (was < 0 && c >= 0) w = S.pw[c];
            }
            // entries that are not starts leave lanes idle: stop only when
            // the list is exhausted too (more is warp-uniform)
            if (!__any_sync(0xffffffffu, c >= 0)) {
                if (!more) break;
                continue;
            }
            if (c < 0) continue;
            // the tail of c's chain and its value
            const int tl = S.qp[c];
            unsigned long long v = w & kPwVal, pois = (w >> 48) & 0xFFull;
            if (tl != c) {
                const unsigned long long wt = S.pw[tl];
                v = (v + (wt & kPwVal)) & kPwVal;
                pois |= wt & kCwPois;
            }
            const uint16_t p = S.sc[tl];
            int next = -1;
            if (!(p & kPtrFinal)) {
                const int t = p;
                const unsigned long long add = kPwOne | (pois ? kPwPois : 0ull) | v;
                const unsigned long long old = atomicAdd(&S.pw[t], add);
                if ((old >> 56) == kDone - 1) {
                    next = t;
                    w = old + add;
                }
            }
            c = next;
        }
    }
    __syncthreads();
    // 5. chain cells: the head's value plus their sums (only heads are read,
    // only chain cells written)
    for (int i = tid; i < ng; i += kSkNT) {
        const int c = S.gl[i];
        if (S.nin[c] != 1) continue;
        const unsigned long long w = S.pw[c];
        unsigned long long out = 0;  // unfinished (on or below a cycle)
        if (!(w & kCwChain)) {
            const unsigned long long wh = S.pw[cw_j(w)];
            if ((wh >> 56) == kDone) {
                const bool pois = (((wh >> 48) & 0xFFull) != 0) || (w & kCwPois);
                out = (unsigned long long)kDone << 56 | (pois ? kPwPois : 0ull) |
                      (((wh & kPwVal) + (w & kPwVal)) & kPwVal);
            }
        }
        S.pw[c] = out;
    }
}

// The same with two-float values (and areas beside them): a final cell pulls
// its in-tile global donors' values in code order, then arrives at its
// receiver (relaxed atomic between two fences: the donor's values are
// written before its arrival, the completing thread reads them after).
template <bool AREA, class S_>
__device__ void walk_pull(S_& S) {
    const int nst = S.qtail;
    int c = -1;
    bool more = true;
    for (;;) {
        if (more) hand_out(S, nst, c, more);
        if (!__any_sync(0xffffffffu, c >= 0)) break;
        if (c < 0) continue;
        uint32_t fl = S.pk[c] & (kPoison | kUp);
        df v = df{S.hi[c], S.lo[c]};
        unsigned long long a = 0;
        if constexpr (AREA) a = S.ar[c];
        for (uint32_t m = S.dm[c]; m; m &= m - 1) {
            const int k = __ffs(m) - 1;
            const int lj = c + offy(k) * SX + offx(k);
            fl |= S.pk[lj] & (kPoison | kUp);
            v = df_add(v, df{S.hi[lj], S.lo[lj]});
            if constexpr (AREA) a += S.ar[lj];
        }
        S.hi[c] = v.hi;
        S.lo[c] = v.lo;
        if constexpr (AREA) S.ar[c] = a;
        S.pk[c] = fl | kFin;
        const uint16_t p = S.sc[c];
        int next = -1;
        if (!(p & kPtrFinal)) {
            const int t = p;
            if (S.nin[t] == 1) {
                next = t;  // the receiver's only in-tile donor: continue without an arrival
            } else {
                __threadfence_block();
                const uint32_t old = atomicSub(&S.pk[t], 1u);
                if ((old & 15u) == 1u) {
                    __threadfence_block();
                    next = t;
                }
            }
        }
        c = next;
    }
}

// Tiles holding at least one global cell, listed once per call (one warp per
// tile reads the tile's rows of the global-cell bits).
__global__ void __launch_bounds__(256) k_skel_tiles(Prob P, EngineGlobals* G, int64_t ntiles) {
    if (__ldcg(&G->glist_count) < P.skel_min) return;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); t < ntiles; t += warps) {
        const TileGeo g = tile_geo(P, t);
        uint32_t any = 0;
        for (int ly = lane; ly < g.ey; ly += 32) {
            const int64_t b0 = (g.y0 + ly) * P.nx + g.x0, b1 = b0 + g.ex;  // bits [b0, b1)
            for (int64_t wd = b0 >> 5; wd <= (b1 - 1) >> 5; ++wd) {
                uint32_t m = __ldg(P.gbits + wd);
                const int64_t lo = wd << 5;
                if (b0 > lo) m &= ~0u << (b0 - lo);
                if (b1 < lo + 32) m &= (1u << (b1 - lo)) - 1u;
                any |= m;
            }
        }
        if (__any_sync(0xffffffffu, any != 0) && lane == 0) {
            const unsigned long long slot = atomicAdd(&G->skel_tiles, 1ull);
            P.sktiles[slot] = (uint32_t)t;
        }
    }
}

// Pass A: in-tile partial values, exits, entries and dependency lists.
template <bool W, bool AREA>
__global__ void __launch_bounds__(kSkNT, 3) k_skel_a(Prob P, EngineGlobals* G) {
    using Sm = SmemSk<W, AREA>;
    constexpr bool kPush = Sm::kPush;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm& S = *reinterpret_cast<Sm*>(smem_raw);
    if (__ldcg(&G->glist_count) < P.skel_min) return;
    const unsigned long long ntl = __ldcg(&G->skel_tiles);
    const int tid = threadIdx.x;
    for (unsigned long long it = blockIdx.x; it < ntl; it += gridDim.x) {
        const int64_t t = (int64_t)__ldcg(P.sktiles + it);
        const TileGeo g = tile_geo(P, t);
        __syncthreads();  // the previous tile's shared memory is no longer read
        if (tid == 0) {
            S.qtail = 0;
            S.head = 0;
        }
        load_tile(S, P, g);
        const int ng = S.ng;
        // ---- start values: rain (or 1) plus the final values of non-global
        // donors in code order; in-tile global donors counted
        for (int i0 = 0; i0 < ng; i0 += kSkNT) {  // warp-uniform trip count
            const int i = i0 + tid;
            int start = -1;
            if (i < ng) {
                const int c = S.gl[i];
                const int ly = c / SX, lx = c - ly * SX;
                const int r = (ly + 1) * SRX + lx + 1;
                const int64_t gi = (g.y0 + ly) * P.nx + g.x0 + lx;
                uint32_t loc = 0, din = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint8_t cj = S.cg[r + offy(k) * SRX + offx(k)];
                    if ((cj & 15u) != (uint8_t)opp(k)) continue;
                    if (!(cj & kGlob)) loc |= 1u << k;
                    else if (in_ext(lx + offx(k), ly + offy(k), g)) din |= 1u << k;
                }
                df v = df_make(0.0f);
                if constexpr (W) v = df_make(P.init ? rd_in(P.init, P, gi, 8) : 1.0f);
                unsigned long long a = 1;
                if (loc) {
                    float h[8], l[8];
                    unsigned long long av[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const bool on = (loc >> k) & 1u;
                        const int64_t gj = gi + offi(k, P.nx);
                        h[k] = l[k] = 0.0f;
                        av[k] = 0;
                        if constexpr (W) {
                            if (on) {
                                h[k] = rd_in(P.out_hi, P, gj, 30);
                                l[k] = rd_in(P.out_lo, P, gj, 31);
                            }
                        }
                        if constexpr (AREA) {
                            if (on) av[k] = (unsigned long long)__ldg(P.area + gj);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        if (!((loc >> k) & 1u)) continue;
                        if constexpr (W) v = df_add(v, df{h[k], l[k]});
                        a += av[k];
                    }
                }
                const uint32_t nin = __popc(din);
                S.nin[c] = (uint8_t)nin;
                S.sc[c] = succ_word(S.cg, c, r, g);
                if constexpr (kPush) {
                    S.pw[c] = (unsigned long long)(kDone - nin) << 56 | a;
                } else {
                    S.hi[c] = v.hi;
                    S.lo[c] = v.lo;
                    if constexpr (AREA) S.ar[c] = a;
                    S.pk[c] = nin;
                    S.dm[c] = (uint8_t)din;
                }
                if (nin == 0) start = c;
            }
            push_start(S, start);
        }
        __syncthreads();
        if constexpr (kPush) {
            // long straight chains (many cells per start): the walk does n
            // steps and its depth is hidden by the other blocks on the SM;
            // else the log-depth contraction
            if (ng >= kWalkCellsPerStart * S.qtail) walk_push(S);
            else contract_push(S, ng);
        } else {
            walk_pull<AREA>(S);
        }
        __syncthreads();
        // ---- where each boundary cell's in-tile path ends (one thread per
        // boundary cell follows the successor words; at most ng steps, so a
        // cycle ends the walk with "no end"), and its donors in other tiles
        const int nb = nboundary(g.ex, g.ey);
        for (int b = tid; b < SX * 4; b += kSkNT) S.bdep[b] = 0;
        __syncthreads();
        for (int b = tid; b < nb; b += kSkNT) {
            int lx, ly;
            bcell(b, g.ex, g.ey, lx, ly);
            const int r = (ly + 1) * SRX + lx + 1;
            uint16_t root = 0;
            int nd = 0;
            if (S.cg[r] & kGlob) {
                uint16_t p = S.sc[ly * SX + lx];
                for (int n = 0; n < ng && !(p & kPtrFinal); ++n) p = S.sc[p & 0xFFF];
                root = (p & kPtrFinal) ? p : 0;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint8_t cj = S.cg[r + offy(k) * SRX + offx(k)];
                    nd += (cj & kGlob) && (cj & 15u) == (uint8_t)opp(k) && !in_ext(lx + offx(k), ly + offy(k), g);
                }
                if constexpr (kPush) {
                    if (nd && (root & kPtrExit)) {
                        const int xc = root & 0xFFF;
                        atomicAdd(&S.bdep[bindex(xc - (xc / SX) * SX, xc / SX, g.ex, g.ey)], nd);
                    }
                }
            }
            S.broot[b] = root;
            S.bnd[b] = (uint8_t)nd;
        }
        __syncthreads();
        // ---- dependency lists (warp 0): entries in row-major boundary order;
        // an entry's donors in other tiles take consecutive slots of the list
        // of the exit its path reaches, in code order
        if (!kPush && tid < 32) {
            const unsigned lane = tid;
            for (int b = lane; b < SX * 4; b += 32) S.bslots[b] = 0;
            __syncwarp();
            for (int b0 = 0; b0 < nb; b0 += 32) {
                const int b = b0 + lane;
                int x = -1, nd = 0;
                if (b < nb) {
                    int lx, ly;
                    bcell(b, g.ex, g.ey, lx, ly);
                    const int r = (ly + 1) * SRX + lx + 1;
                    if (S.cg[r] & kGlob) {
                        nd = S.bnd[b];
                        const uint16_t p = S.broot[b];
                        if (nd && (p & kPtrExit)) {
                            const int xc = p & 0xFFF;
                            x = bindex(xc - (xc / SX) * SX, xc / SX, g.ex, g.ey);
                        }
                    }
                }
                S.wtmp[lane] = (uint8_t)nd;
                __syncwarp();
                const unsigned peers = __match_any_sync(0xffffffffu, x);
                if (x >= 0) {
                    int off = 0, tot = 0;
                    for (unsigned m = peers; m; m &= m - 1) {
                        const int l = __ffs(m) - 1;
                        if (l < (int)lane) off += S.wtmp[l];
                        tot += S.wtmp[l];
                    }
                    const int base = S.bslots[x];
                    S.brank[b] = (uint16_t)(base + off);
                    __syncwarp(peers);
                    if ((int)lane == __ffs(peers) - 1) S.bslots[x] = (uint16_t)(base + tot);
                }
                __syncwarp();
            }
            // list begins: exclusive scan over boundary cells in order
            int run = 0;
            for (int b0 = 0; b0 < nb; b0 += 32) {
                const int b = b0 + lane;
                const int v = b < nb ? S.bslots[b] : 0;
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((int)lane >= o) incl += u;
                }
                if (b < nb) S.bbeg[b] = (uint16_t)(run + incl - v);
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        __syncthreads();
        // ---- link words, dependency slots, walker starts (one thread per boundary cell)
        uint16_t* pool = P.skpool + t * kSkelPool;
        for (int b = tid; b < nb; b += kSkNT) {
            int lx, ly;
            bcell(b, g.ex, g.ey, lx, ly);
            const int c = ly * SX + lx, r = (ly + 1) * SRX + lx + 1;
            if (!(S.cg[r] & kGlob)) continue;
            const int64_t gi = (g.y0 + ly) * P.nx + g.x0 + lx;
            const uint16_t p = S.broot[b];
            const bool exit = (p & kPtrExit) && (p & 0xFFF) == c;
            const int nd = S.bnd[b];
            if (exit) {
                const unsigned long long len = kPush ? (unsigned long long)S.bdep[b] : S.bslots[b];
                bool fin;
                if constexpr (kPush) fin = (S.pw[c] >> 56) == kDone;
                else fin = (S.pk[c] & kFin) != 0;
                const unsigned long long pend = fin ? len : kLkNever;
                const unsigned long long beg = kPush ? 0ull : S.bbeg[b];
                P.link[gi] = (int64_t)(kLkExit | pend | (beg << 16) | (len << 32));
                if (fin && len == 0) {
                    const unsigned long long slot = atomicAdd(&G->fcount[0], 1ull);
                    P.skstarts[slot] = (unsigned long long)gi;
                }
            } else if (nd) {
                unsigned long long rec = 0;
                if (p & kPtrExit) {
                    const int xc = p & 0xFFF;
                    rec = kLkEntry | (unsigned long long)((g.y0 + xc / SX) * P.nx + g.x0 + (xc - (xc / SX) * SX));
                }
                P.link[gi] = (int64_t)rec;
            }
            if (!kPush && nd && (p & kPtrExit)) {
                const int xc = p & 0xFFF;
                const int xb = bindex(xc - (xc / SX) * SX, xc / SX, g.ex, g.ey);
                int s = S.bbeg[xb] + S.brank[b];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int j = r + offy(k) * SRX + offx(k);
                    const uint8_t cj = S.cg[j];
                    if ((cj & kGlob) && (cj & 15u) == (uint8_t)opp(k) && !in_ext(lx + offx(k), ly + offy(k), g))
                        if (FR_OK(s, kSkelPool, 32)) pool[s++] = (uint16_t)j;
                }
            }
        }
        // ---- in-tile partial values of the finished global cells
        for (int i = tid; i < ng; i += kSkNT) {
            const int c = S.gl[i];
            const int ly = c / SX, lx = c - ly * SX;
            const int64_t gi = (g.y0 + ly) * P.nx + g.x0 + lx;
            if constexpr (kPush) {
                const unsigned long long w = S.pw[c];
                if ((w >> 56) == kDone) wr_area(P, gi, w & kPwVal);
            } else {
                if (!(S.pk[c] & kFin)) continue;
                wr_f(P.out_hi, P, gi, S.hi[c], 33);
                wr_f(P.out_lo, P, gi, S.lo[c], 34);
                if constexpr (AREA) wr_area(P, gi, S.ar[c]);
            }
        }
    }
}

// Pass B: walkers over the exits.
template <bool W, bool AREA>
__global__ void __launch_bounds__(256) k_skel_walk(Prob P, EngineGlobals* G) {
    if (__ldcg(&G->glist_count) < P.skel_min) return;
    const unsigned long long count = __ldcg(&G->fcount[0]);
    const int tiles_x = (int)((P.nx + SX - 1) / SX);
    uint8_t* done = reinterpret_cast<uint8_t*>(P.cnt);
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        int64_t x = (int64_t)__ldcg(P.skstarts + i);
        if constexpr (AREA && !W) {
            // areas alone: every dependency adds its total into the exit's
            // area (exact integer atomics, any order), so the arrival that
            // completes the count finds the exit's total there
            for (;;) {
                const uint8_t k = rd_rb(P, x);
                const unsigned long long a = rd_area(P, x);
                if (FR_OK(x, ncell(P), 41)) done[x] = 1;
                if (k >= 8) break;
                const int64_t s = x + offi(k, P.nx);
                const unsigned long long rs = (unsigned long long)__ldcg(
                    reinterpret_cast<const unsigned long long*>(P.link) + s);
                int64_t q;
                if ((rs & kLkKind) == kLkExit) q = s;
                else if ((rs & kLkKind) == kLkEntry) q = (int64_t)(rs & kLkCell);
                else break;
                if (!FR_OK(q, ncell(P), 42)) break;
                atomicAdd(reinterpret_cast<unsigned long long*>(P.area) + q, a);
                cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> at(
                    reinterpret_cast<unsigned long long*>(P.link)[q]);
                const unsigned long long old = at.fetch_sub(1ull, cuda::memory_order_acq_rel);
                if ((old & 0xFFFFull) != 1ull) break;
                x = q;
            }
        } else {
            for (;;) {
                const uint8_t k = rd_rb(P, x);
                const unsigned long long rec = (unsigned long long)__ldcg(
                    reinterpret_cast<const unsigned long long*>(P.link) + x);
                const int begin = (int)((rec >> 16) & 0xFFFF), len = (int)((rec >> 32) & 0xFFFF);
                const int64_t yy = x / P.nx, xx = x - yy * P.nx;
                const int64_t tx = xx / SX, ty = yy / SY;
                const int64_t ox = tx * SX - 1, oy = ty * SY - 1;  // ring origin of x's tile
                const uint16_t* pool = P.skpool + (ty * tiles_x + tx) * kSkelPool;
                df v = df_make(0.0f);
                unsigned long long a = 0;
                if constexpr (W) v = df{rd_cg(P.out_hi, P, x, 35), rd_cg(P.out_lo, P, x, 36)};
                if constexpr (AREA) a = rd_area(P, x);
    #pragma unroll 1
                for (int s = 0; s < len; ++s) {
                    const int j = __ldcg(pool + begin + s);
                    const int ry = j / SRX, rx = j - ry * SRX;
                    const int64_t y = (oy + ry) * P.nx + (ox + rx);
                    if constexpr (W) v = df_add(v, df{rd_cg(P.out_hi, P, y, 37), rd_cg(P.out_lo, P, y, 38)});
                    if constexpr (AREA) a += rd_area(P, y);
                }
                if constexpr (W) {
                    wr_f(P.out_hi, P, x, v.hi, 39);
                    wr_f(P.out_lo, P, x, v.lo, 40);
                }
                if constexpr (AREA) wr_area(P, x, a);
                if (FR_OK(x, ncell(P), 41)) done[x] = 1;
                // the exit reached from this exit's receiver (an entry of the next tile)
                if (k >= 8) break;
                const int64_t s = x + offi(k, P.nx);
                const unsigned long long rs = (unsigned long long)__ldcg(
                    reinterpret_cast<const unsigned long long*>(P.link) + s);
                int64_t q;
                if ((rs & kLkKind) == kLkExit) q = s;
                else if ((rs & kLkKind) == kLkEntry) q = (int64_t)(rs & kLkCell);
                else break;
                if (!FR_OK(q, ncell(P), 42)) break;
                // release this exit's value; the completing arrival acquires all
                cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> at(
                    reinterpret_cast<unsigned long long*>(P.link)[q]);
                const unsigned long long old = at.fetch_sub(1ull, cuda::memory_order_acq_rel);
                if ((old & 0xFFFFull) != 1ull) break;
                x = q;
            }
        }
    }
}

// Pass C: inflows of the entries passed down the in-tile receivers; final
// values of the global cells; completion count.
template <bool W, bool AREA>
__global__ void __launch_bounds__(kSkNT, 3) k_skel_fix(Prob P, EngineGlobals* G,
                                                   unsigned long long total_cells) {
    using Sm = SmemSk<W, AREA>;
    constexpr bool kPush = Sm::kPush;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm& S = *reinterpret_cast<Sm*>(smem_raw);
    if (__ldcg(&G->glist_count) < P.skel_min) return;
    const unsigned long long ntl = __ldcg(&G->skel_tiles);
    const uint8_t* done_b = reinterpret_cast<const uint8_t*>(P.cnt);
    const int tid = threadIdx.x;
    unsigned long long done = 0;
    for (unsigned long long it = blockIdx.x; it < ntl; it += gridDim.x) {
        const int64_t t = (int64_t)__ldcg(P.sktiles + it);
        const TileGeo g = tile_geo(P, t);
        __syncthreads();
        if (tid == 0) {
            S.qtail = 0;
            S.head = 0;
        }
        load_tile(S, P, g);
        const int ng = S.ng;
        // ---- inflow of every entry: the totals of its donors in other tiles
        // (exits, final after pass B), one thread per boundary cell
        const int nb = nboundary(g.ex, g.ey);
        for (int b = tid; b < nb; b += kSkNT) {
            int lx, ly;
            bcell(b, g.ex, g.ey, lx, ly);
            const int r = (ly + 1) * SRX + lx + 1;
            if (!(S.cg[r] & kGlob)) continue;
            const int64_t gi = (g.y0 + ly) * P.nx + g.x0 + lx;
            uint32_t ext = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint8_t cj = S.cg[r + offy(k) * SRX + offx(k)];
                if ((cj & kGlob) && (cj & 15u) == (uint8_t)opp(k) && !in_ext(lx + offx(k), ly + offy(k), g))
                    ext |= 1u << k;
            }
            float h[8], l[8];
            unsigned long long av[8];
            uint8_t dn[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int64_t gj = gi + offi(k, P.nx);
                h[k] = l[k] = 0.0f;
                av[k] = 0;
                dn[k] = 1;
                if ((ext >> k) & 1u) {
                    dn[k] = done_b[gj];
                    if constexpr (W) {
                        h[k] = rd_cg(P.out_hi, P, gj, 43);
                        l[k] = rd_cg(P.out_lo, P, gj, 44);
                    }
                    if constexpr (AREA) av[k] = rd_area(P, gj);
                }
            }
            df v = df_make(0.0f);
            unsigned long long a = 0;
            uint32_t fl = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (!((ext >> k) & 1u)) continue;
                fl |= kUp;
                if (!dn[k]) fl |= kPoison;
                if constexpr (W) v = df_add(v, df{h[k], l[k]});
                a += av[k];
            }
            S.bval[b] = a;
            S.bfl[b] = fl;
            if constexpr (W) {
                S.bhi[b] = v.hi;
                S.blo[b] = v.lo;
            }
        }
        __syncthreads();
        for (int i0 = 0; i0 < ng; i0 += kSkNT) {  // warp-uniform trip count
            const int i = i0 + tid;
            int start = -1;
            if (i < ng) {
                const int c = S.gl[i];
                const int ly = c / SX, lx = c - ly * SX;
                const int r = (ly + 1) * SRX + lx + 1;
                uint32_t ext = 0, din = 0, fl = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint8_t cj = S.cg[r + offy(k) * SRX + offx(k)];
                    if (!(cj & kGlob) || (cj & 15u) != (uint8_t)opp(k)) continue;
                    if (in_ext(lx + offx(k), ly + offy(k), g)) din |= 1u << k;
                    else ext |= 1u << k;  // a donor in another tile: an exit, final after pass B
                }
                df v = df_make(0.0f);
                unsigned long long a = 0;
                if (ext) {  // an entry (on the boundary): its inflow from the pass above
                    const int b = bindex(lx, ly, g.ex, g.ey);
                    fl = S.bfl[b];
                    a = S.bval[b];
                    if constexpr (W) v = df{S.bhi[b], S.blo[b]};
                }
                const uint32_t nin = __popc(din);
                S.nin[c] = (uint8_t)nin;
                S.sc[c] = succ_word(S.cg, c, r, g);
                if constexpr (kPush) {
                    S.pw[c] = (unsigned long long)(kDone - nin) << 56 | ((fl & kPoison) ? kPwPois : 0ull) | a;
                } else {
                    S.hi[c] = v.hi;
                    S.lo[c] = v.lo;
                    if constexpr (AREA) S.ar[c] = a;
                    S.pk[c] = nin | fl;
                    S.dm[c] = (uint8_t)din;
                }
                if (nin == 0) start = c;
            }
            push_start(S, start);
        }
        __syncthreads();
        if constexpr (kPush) {
            // long straight chains (many cells per start): the walk does n
            // steps and its depth is hidden by the other blocks on the SM;
            // else the log-depth contraction
            if (ng >= kWalkCellsPerStart * S.qtail) walk_push(S);
            else contract_push(S, ng);
        } else {
            walk_pull<AREA>(S);
        }
        __syncthreads();
        // final values: L (pass A, in the outputs) plus the inflow sums, in
        // batches of eight cells per thread whose loads are issued together
        constexpr int B = 8;
        for (int i0 = 0; i0 < ng; i0 += B * kSkNT) {
            int64_t gix[B];
            bool upd[B];
#pragma unroll
            for (int q = 0; q < B; ++q) {
                const int i = i0 + q * kSkNT + tid;
                upd[q] = false;
                gix[q] = 0;
                if (i >= ng) continue;
                const int c = S.gl[i];
                const int ly = c / SX, lx = c - ly * SX;
                gix[q] = (g.y0 + ly) * P.nx + g.x0 + lx;
                if (S.sc[c] & kPtrExit) {  // an exit: final after pass B
                    done += done_b[gix[q]] ? 1 : 0;
                    continue;
                }
                if constexpr (kPush) {
                    const unsigned long long w = S.pw[c];
                    if ((w >> 56) != kDone || ((w >> 48) & 0xFFull)) continue;
                    ++done;
                    upd[q] = (w & kPwVal) != 0;  // inflow from other tiles
                } else {
                    const uint32_t pkc = S.pk[c];
                    if (!(pkc & kFin) || (pkc & kPoison)) continue;
                    ++done;
                    upd[q] = (pkc & kUp) != 0;  // else L is final
                }
            }
            float hh[B], ll[B];
            unsigned long long aa[B];
#pragma unroll
            for (int q = 0; q < B; ++q) {
                hh[q] = ll[q] = 0.0f;
                aa[q] = 0;
                if (!upd[q]) continue;
                if constexpr (W) {
                    hh[q] = rd_cg(P.out_hi, P, gix[q], 45);
                    ll[q] = rd_cg(P.out_lo, P, gix[q], 46);
                }
                if constexpr (AREA) aa[q] = rd_area(P, gix[q]);
            }
#pragma unroll
            for (int q = 0; q < B; ++q) {
                if (!upd[q]) continue;
                const int c = S.gl[i0 + q * kSkNT + tid];
                if constexpr (kPush) {
                    wr_area(P, gix[q], aa[q] + (S.pw[c] & kPwVal));
                } else {
                    const df v = df_add(df{hh[q], ll[q]}, df{S.hi[c], S.lo[c]});
                    wr_f(P.out_hi, P, gix[q], v.hi, 47);
                    wr_f(P.out_lo, P, gix[q], v.lo, 48);
                    if constexpr (AREA) wr_area(P, gix[q], aa[q] + S.ar[c]);
                }
            }
        }
    }
    // completion count; the last CTA checks that every cell was computed
    __shared__ unsigned long long s_done;
    for (int o = 16; o; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);
    __syncthreads();
    if (tid == 0) s_done = 0;
    __syncthreads();
    if ((tid & 31) == 0 && done) atomicAdd(&s_done, done);
    __syncthreads();
    if (tid == 0) {
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

template <class K>
int persistent_grid(K kernel, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kSkNT, smem) != cudaSuccess) return 0;
    return sms * (per > 0 ? per : 1);
}

template <bool W, bool AREA>
cudaError_t launch_skel_t(const Prob& P, EngineGlobals* G, cudaStream_t s) {
    constexpr size_t sm = sizeof(SmemSk<W, AREA>);
    static std::atomic<unsigned long long> set_a{0}, set_c{0};
    static int grid_a = 0, grid_c = 0;
    cudaError_t e = smem_limit_once(k_skel_a<W, AREA>, sm, set_a);
    if (e != cudaSuccess) return e;
    e = smem_limit_once(k_skel_fix<W, AREA>, sm, set_c);
    if (e != cudaSuccess) return e;
    if (!grid_a) grid_a = persistent_grid(k_skel_a<W, AREA>, sm);
    if (!grid_c) grid_c = persistent_grid(k_skel_fix<W, AREA>, sm);
    if (!grid_a || !grid_c) return cudaErrorInvalidConfiguration;
    const int64_t ntiles = skel_tiles(P.nx, P.ny);
    int tgrid = (int)((ntiles + 7) / 8);
    if (tgrid > 16 * 152) tgrid = 16 * 152;
    if (tgrid < 1) tgrid = 1;
    k_skel_tiles<<<tgrid, 256, 0, s>>>(P, G, ntiles);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_skel_a<W, AREA><<<grid_a, kSkNT, sm, s>>>(P, G);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_skel_walk<W, AREA><<<walker_grid(), 256, 0, s>>>(P, G);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_skel_fix<W, AREA><<<grid_c, kSkNT, sm, s>>>(P, G, (unsigned long long)(P.nx * P.ny));
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_d8_skeleton(bool want_w, bool want_area, const Prob& P, EngineGlobals* G,
                               cudaStream_t s) {
    if (want_w && want_area) return launch_skel_t<true, true>(P, G, s);
    if (want_w) return launch_skel_t<true, false>(P, G, s);
    return launch_skel_t<false, true>(P, G, s);
}

}  // namespace fr

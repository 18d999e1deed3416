// fr_halo.cu -- local phase over halo-extended tiles for MFD (slope-split)
// forward accumulation and for the adjoints of both routing rules.
//
// Same decomposition as the D8 forward kernel: each CTA solves an inner tile
// plus an H-cell halo exactly in shared memory (a per-subdomain high-to-low solve,
// Sec. 2.4, on overlapping subdomains), and only cells whose dependencies
// reach outside the extended region go to the global phase.  With several
// receivers per cell (App. A) dependency sets spread wider than D8 basins, so
// the halo is deeper: at 64x32 + 8 about 0.9 % of the cells of a rough
// fractal DEM stay global, against about 21 % for the same tiles without a
// halo.  The tiles are 64x64 (two blocks of about 103 KB and 384 threads per
// SM, 1.56 region cells per inner cell): smaller tiles that fit more blocks
// per SM (64x32, 48x48, 56x48, 40x40) were measured slower, their extra halo
// cells costing more than the occupancy gains; halos of 6 and 10 cells were
// slower than 8.
//
// The three modes differ only in the direction of the dependencies:
//   forward MFD   w_c = r_c    + sum over donors j    of f_{j->c} w_j
//   adjoint       g_c = gbar_c + sum over receivers k of f_{c->k} g_k
// (g = A^{-T} gbar, the transposed system of Eq. Aw=f: each cell's adjoint
// is its own gbar plus the fraction-weighted adjoints of its receivers; f = 1
// for D8).  A forward cell waits for its donors and then notifies its
// receivers; an adjoint cell waits for its receivers and notifies its donors.
// Fractions f_{j->k} = u_{j->k} / S_j (u = s^p, S_j the sum of cell j's
// weights) are computed once per cell by a fully parallel pass (mfd_fracs8)
// and read here, so the tile solve evaluates no powers.  The eight direction
// terms of a cell are accumulated in the fixed order of df_dot8, exactly as
// the global phase does, so a cell's value does not depend on which kernel
// computed it.
//
// Cells are finalised in a topological order (Sec. 3.2) discovered on the fly,
// without block barriers: every cell counts its pending in-region
// dependencies, and the lane whose decrement completes a count owns that
// cell.  A lane keeps one of the cells it completes and continues with it;
// the others go to a shared-memory queue from which idle lanes take work.
// A warp takes only queue slots that a producer has already reserved, so a
// wait for a slot is the few instructions between the producer's reservation
// and its store; a warp that finds the queue empty sleeps until new work is
// queued or no cell is held or queued anywhere in the CTA (the live count).
// One lane finalises one cell: its (up to eight) dependency terms are loaded
// side by side and summed in the fixed order, so the result does not depend
// on which lane computed it or when.
#include "fr_engine.cuh"

namespace fr {
namespace {

constexpr int kHaloTX = kMfdTileX, kHaloTY = kMfdTileY, kHaloH = 8;
constexpr int kHaloNT = 384;

struct HaloGeo {
    static constexpr int TX = kHaloTX, TY = kHaloTY, H = kHaloH;
    static constexpr int EX = TX + 2 * H, EY = TY + 2 * H, NE = EX * EY;  // extended region
    static constexpr int RX = EX + 2, RY = EY + 2, NR = RX * RY;         // plus a one-cell ring
    static_assert(NE < 65535, "local indices are 16-bit");
    static_assert(NE % 4 == 0, "state bytes are packed four to a word");
};

// Directions whose neighbour of region cell (ex, ey) lies inside the region.
__device__ __forceinline__ uint32_t region_mask(int ex, int ey) {
    uint32_t in = 0xFFu;
    if (ex == 0) in &= ~0x64u;                 // W NW SW
    if (ex == HaloGeo::EX - 1) in &= ~0x91u;   // E NE SE
    if (ey == 0) in &= ~0x32u;                 // N NE NW
    if (ey == HaloGeo::EY - 1) in &= ~0xC8u;   // S SW SE
    return in;
}

template <Mode M>
struct HaloMode {
    static constexpr bool kAdj = (M == Mode::AdjMfd || M == Mode::AdjD8);
    static constexpr bool kMfd = (M == Mode::FwdMfd || M == Mode::AdjMfd);
};

struct SmemHalo {
    static constexpr int NE = HaloGeo::NE, NR = HaloGeo::NR;
    float vhi[NE];        // value (water or adjoint), leading word
    float vlo[NE];        // value, trailing word
    uint32_t st[NE / 4];  // per cell byte: pending non-bare dependencies
    uint16_t queue[NE];   // ready cells (kSlotEmpty until written); each cell at most once
    uint8_t rb[NR];       // receiver masks of region + ring (0 outside the grid)
    uint8_t dm[NE];       // in-region dependencies (donors forward, receivers adjoint)
    uint8_t tm[NE];       // in-region targets (receivers forward, donors adjoint)
    uint8_t fin[NE];      // 1 final, 0 pending, 0x0F outside the grid
    uint8_t gf[NE];       // 1: a dependency chain leaves the region (solved globally)
    int head;             // queue slots taken
    int resv;             // queue slots reserved by producers
    int live;             // cells queued or held by a lane
    int gave_up;          // a bounded wait ran out
    unsigned long long done;
};
constexpr uint16_t kSlotEmpty = 0xFFFFu;

// Marks the global inner cells of a warp (all 32 lanes call; glob: this
// lane's cell gi is global): their bits, and list entries reserved with one
// atomic per warp.
__device__ __forceinline__ void mark_global_cells(const Prob& P, EngineGlobals* G, int64_t gi,
                                                  int pid, bool glob) {
    const unsigned m = __ballot_sync(0xffffffffu, glob);
    if (!m) return;
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long base = 0;
    if (lane == (unsigned)(__ffs(m) - 1)) base = atomicAdd(&G->glist_count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (glob) {
        atomicOr(P.gbits + (gi >> 5), 1u << (gi & 31));
        const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
        if (FR_OK((int64_t)slot, P.glist_cap, 17))
            P.glist[slot] = ((unsigned long long)pid << 40) | (unsigned long long)gi;
    }
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Warp-aggregated queue append: lane l appends the region cells c + off(k)
// for the set bits k < 8 of its mask `bits`, and c itself for bit 8.  Lane 0
// first adds (appended cells - finished) to the live count, then reserves the
// slots: the count never drops below the cells queued or held, so it reads
// zero only when the region has no work left.  The cells are stored after a
// block fence, so a consumer that reads a slot sees what the producer wrote
// before it.
__device__ __forceinline__ void queue_push(SmemHalo& S, int c, uint32_t bits, int finished) {
    const unsigned lane = threadIdx.x & 31u;
    if (!__any_sync(0xffffffffu, bits != 0)) {
        // the common step: nothing to queue, only finished cells to count
        if (lane == 0 && finished) atomicAdd(&S.live, -finished);
        return;
    }
    const unsigned lt = lanemask_lt();
    const uint32_t n = (uint32_t)__popc(bits);
    // exclusive prefix of n (at most 9) over the lanes, from the ballots of its bits
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const unsigned v = __ballot_sync(0xffffffffu, (n >> b) & 1u);
        pre += (uint32_t)__popc(v & lt) << b;
        tot += (uint32_t)__popc(v) << b;
    }
    int base = 0;
    if (lane == 0) {
        if ((int)tot != finished) atomicAdd(&S.live, (int)tot - finished);
        if (tot) base = atomicAdd(&S.resv, (int)tot);
    }
    if (tot == 0) return;
    base = __shfl_sync(0xffffffffu, base, 0);
    if (bits) {
        __threadfence_block();
        int slot = base + (int)pre;
        for (uint32_t m = bits; m; m &= m - 1) {
            const int k = __ffs(m) - 1;
            const int cell = k == 8 ? c : c + offy(k) * HaloGeo::EX + offx(k);
            if (slot < HaloGeo::NE)
                reinterpret_cast<volatile uint16_t*>(S.queue)[slot] = (uint16_t)cell;
            else
                S.gave_up = 1;  // unreachable: each cell is queued at most once
            ++slot;
        }
    }
}

// Problem and tile of this CTA in a batched launch: the problem whose tiles
// [prefix[p], prefix[p+1]) hold blockIdx.x.
__device__ __forceinline__ int batch_problem_halo(const int64_t* __restrict__ prefix, int nprob,
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

template <Mode M, bool BATCH>
__global__ void __launch_bounds__(kHaloNT, 2) k_local_halo(Prob Pone, EngineGlobals* G,
                                                           const Prob* __restrict__ probs,
                                                           const int64_t* __restrict__ prefix,
                                                           int nprob, unsigned long long limit_ns) {
    using HM = HaloMode<M>;
    constexpr int TX = HaloGeo::TX, TY = HaloGeo::TY, H = HaloGeo::H;
    constexpr int EX = HaloGeo::EX, NE = HaloGeo::NE;
    constexpr int RX = HaloGeo::RX;
    constexpr int NT = kHaloNT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemHalo& S = *reinterpret_cast<SmemHalo*>(smem_raw);
    uint8_t* stb = reinterpret_cast<uint8_t*>(S.st);
    const int tid = threadIdx.x;
    int64_t lt = (int64_t)blockIdx.x;
    const int pid = BATCH ? batch_problem_halo(prefix, nprob, lt) : 0;
    const Prob& P = BATCH ? probs[pid] : Pone;
    const int64_t tiles_x = (P.nx + TX - 1) / TX;
    const int64_t ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int64_t x0 = tx * TX, y0 = ty * TY;
    const int64_t ox = x0 - H - 1, oy = y0 - H - 1;  // ring origin (may be negative)
    if (tid == 0) {
        S.head = S.resv = S.live = S.gave_up = 0;
    }

    // The phases below walk the region row by row: warp w takes rows w,
    // w + NW, ...; lane l takes columns l, l + 32, ...  A tile whose ring lies
    // inside the grid skips the bounds checks.
    constexpr int NW = NT / 32;
    constexpr int EY = HaloGeo::EY, RY = HaloGeo::RY;
    const int warp = tid >> 5, lane_id = tid & 31;
    const bool interior = ox >= 0 && oy >= 0 && ox + RX <= P.nx && oy + RY <= P.ny;

    // ---- region + ring: receiver masks
    if (interior) {
        for (int ry = warp; ry < RY; ry += NW) {
            const uint8_t* src = P.rb + (oy + ry) * P.nx + ox;
            for (int rx = lane_id; rx < RX; rx += 32)
                S.rb[ry * RX + rx] = (uint8_t)recv_mask<HM::kMfd>(__ldg(src + rx));
        }
    } else {
        for (int ry = warp; ry < RY; ry += NW) {
            const int64_t gy = oy + ry;
            for (int rx = lane_id; rx < RX; rx += 32) {
                const int64_t gx = ox + rx;
                uint8_t m = 0;
                if (gx >= 0 && gy >= 0 && gx < P.nx && gy < P.ny)
                    m = (uint8_t)(recv_mask<HM::kMfd>(rd_rb(P, gy * P.nx + gx)) & grid_mask(gx, gy, P.nx, P.ny));
                S.rb[ry * RX + rx] = m;
            }
        }
    }
    if constexpr (HM::kMfd) {
        // warm L2 with the region's fractions, which the dependency pulls read
        // a few at a time: one prefetch per 128-byte line of every region row
        const int64_t gx0 = ox + 1 < 0 ? 0 : ox + 1;
        const int64_t gx1 = ox + 1 + EX > P.nx ? P.nx : ox + 1 + EX;
        if (gx1 > gx0) {
            const int lines = (int)(((gx1 - gx0) * 32 + 127) / 128) + 1;
            for (int ry = warp; ry < EY; ry += NW) {
                const int64_t gy = oy + 1 + ry;
                if (gy < 0 || gy >= P.ny) continue;
                const char* row = reinterpret_cast<const char*>(P.frac + (gy * P.nx + gx0) * 8);
                const char* end = reinterpret_cast<const char*>(P.frac + (gy * P.nx + gx1) * 8);
                for (int q = lane_id; q < lines; q += 32) {
                    const char* a = row + 128 * q;
                    if (a < end) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                }
            }
        }
    }
    __syncthreads();

    // ---- per region cell: dependencies and targets, bare / global flags,
    // initial value (rain forward; gbar adjoint)
    for (int ey = warp; ey < EY; ey += NW) {
        const int64_t gy = oy + ey + 1;
        const bool row_in = gy >= 0 && gy < P.ny;
        for (int ex = lane_id; ex < EX; ex += 32) {
            const int c = ey * EX + ex;
            const int r = (ey + 1) * RX + ex + 1;
            const int64_t gx = ox + ex + 1;
            uint8_t dmr = 0, tmr = 0, fin = 0x0F, b = 0;
            float vh = 0.0f, vl = 0.0f;
            if (interior || (row_in && gx >= 0 && gx < P.nx)) {
                const int64_t gi = gy * P.nx + gx;
                uint32_t don = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    don |= (uint32_t)((S.rb[r + offy(k) * RX + offx(k)] >> opp(k)) & 1u) << k;
                const uint32_t rcv = S.rb[r];
                const uint32_t dep = HM::kAdj ? rcv : don;
                const uint32_t tgt = HM::kAdj ? don : rcv;
                const uint32_t in = region_mask(ex, ey);
                dmr = (uint8_t)(dep & in);
                tmr = (uint8_t)(tgt & in);
                b = (dep & ~in) ? (uint8_t)1 : (uint8_t)0;
                fin = dep == 0;
                if constexpr (!HM::kAdj) {
                    vh = P.init ? rd_in(P.init, P, gi, 8) : 1.0f;
                } else if (P.init) {
                    vh = rd_in(P.init, P, gi, 8);
                } else if (!rcv) {
                    // L = sum over sinks of w^2: gbar = 2 w at a sink, 0 elsewhere
                    vh = __fmul_rn(2.0f, rd_in(P.wf, P, gi, 9));
                    vl = P.wf_lo ? __fmul_rn(2.0f, rd_in(P.wf_lo, P, gi, 10)) : 0.0f;
                }
            }
            S.dm[c] = dmr;
            S.tm[c] = tmr;
            S.fin[c] = fin;
            S.gf[c] = b;
            S.queue[c] = kSlotEmpty;
            S.vhi[c] = vh;
            S.vlo[c] = vl;
        }
    }
    __syncthreads();

    // ---- counts of non-bare in-region dependencies; cells with none are
    // ready at once and start the queue (every lane of a warp runs the same
    // number of column steps, as queue_push needs)
    for (int ey = warp; ey < EY; ey += NW) {
        for (int ex0 = 0; ex0 < EX; ex0 += 32) {
            const int ex = ex0 + lane_id;
            const int c = ey * EX + ex;
            uint32_t start = 0;
            if (ex < EX) {
                uint32_t n = 0;
                if (S.fin[c] == 0) {
                    const uint32_t dm = S.dm[c];
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        n += ((dm >> k) & 1u) && S.fin[c + offy(k) * EX + offx(k)] != 1;
                    start = n == 0;
                }
                stb[c] = (uint8_t)n;
            }
            queue_push(S, c, start ? 0x100u : 0u, 0);  // bit 8: the cell itself
        }
    }
    __syncthreads();

    // ---- dataflow over the region: finalise ready cells, pass readiness on
    {
        const unsigned lane = tid & 31u;
        int cur = -1;                 // the cell this lane holds
        unsigned long long idle_since = 0;
        for (;;) {
            // idle lanes take reserved queue slots, in lane order
            const unsigned idle = __ballot_sync(0xffffffffu, cur < 0);
            if (idle) {
                int h = 0, n = 0;
                if (lane == 0) {
                    int hh = ld_volatile(&S.head);
                    for (int tries = 0; tries < 4096; ++tries) {
                        const int avail = ld_volatile(&S.resv) - hh;
                        n = avail < __popc(idle) ? avail : __popc(idle);
                        if (n <= 0) {
                            n = 0;
                            break;
                        }
                        const int prev = atomicCAS(&S.head, hh, hh + n);
                        if (prev == hh) break;
                        hh = prev;
                        n = 0;
                    }
                    h = hh;
                }
                h = __shfl_sync(0xffffffffu, h, 0);
                n = __shfl_sync(0xffffffffu, n, 0);
                const int rank = __popc(idle & lanemask_lt());
                if (cur < 0 && rank < n && h + rank < NE) {
                    const volatile uint16_t* q = reinterpret_cast<const volatile uint16_t*>(S.queue);
                    uint16_t v = q[h + rank];
                    if (v == kSlotEmpty) {
                        // the producer reserved this slot and stores it next
                        const unsigned long long t0 = global_ns();
                        while ((v = q[h + rank]) == kSlotEmpty)
                            if (global_ns() - t0 > limit_ns) break;
                    }
                    if (v != kSlotEmpty) cur = v;
                    else S.gave_up = 1;
                }
            }
            if (!__any_sync(0xffffffffu, cur >= 0)) {
                // nothing held here and nothing queued: done when no cell is
                // held or queued anywhere, else wait for more work (lane 0
                // decides for the warp)
                int stop = 0;
                if (lane == 0) {
                    if (ld_volatile(&S.live) == 0) {
                        stop = 1;
                    } else {
                        const unsigned long long t = global_ns();
                        if (!idle_since) {
                            idle_since = t;
                        } else if (t - idle_since > limit_ns) {
                            S.gave_up = 1;
                            stop = 1;
                        }
                    }
                }
                if (__shfl_sync(0xffffffffu, stop, 0)) break;
                __nanosleep(128);
                continue;
            }
            idle_since = 0;
            uint32_t ready = 0;  // codes of targets this lane completed
            if (cur >= 0) {
                const int c = cur;
                __threadfence_block();  // acquire: the dependencies' values and flags
                const bool glob = S.gf[c] != 0;
                if (!glob) {
                    // dependency terms, loaded side by side, accumulated in
                    // the fixed order of df_dot8
                    const uint32_t dm = S.dm[c];
                    const float* fb = nullptr;
                    int64_t row = 0;
                    if constexpr (HM::kMfd) {
                        const int ey = c / EX, ex = c - ey * EX;
                        fb = P.frac + ((oy + ey + 1) * P.nx + (ox + ex + 1)) * 8;
                        row = P.nx * 8;
                    }
                    float f[8];
                    df vv[8];
                    float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f), f1 = f0;
                    if constexpr (HM::kMfd && HM::kAdj) {
                        // adjoint: c's own fractions towards its receivers, one 32-byte row
                        f0 = __ldg(reinterpret_cast<const float4*>(fb));
                        f1 = __ldg(reinterpret_cast<const float4*>(fb) + 1);
                    }
                    const float own[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        f[k] = 0.0f;
                        vv[k] = df_make(0.0f);
                        if (!((dm >> k) & 1u)) continue;
                        const int j = c + offy(k) * EX + offx(k);
                        vv[k] = {S.vhi[j], S.vlo[j]};
                        if constexpr (HM::kMfd) {
                            // forward: the donor's fraction towards c
                            f[k] = HM::kAdj ? own[k] : __ldg(fb + offy(k) * row + (offx(k) * 8 + opp(k)));
                        } else {
                            f[k] = 1.0f;
                        }
                    }
                    const df v = df_dot8(df{S.vhi[c], S.vlo[c]}, f, vv);
                    S.vhi[c] = v.hi;
                    S.vlo[c] = v.lo;
                }
                S.fin[c] = 1;
                // targets: pass on the global flag, then count down (release)
                const uint32_t tm = S.tm[c];
                if (glob) {
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if ((tm >> k) & 1u) S.gf[c + offy(k) * EX + offx(k)] = 1;
                }
                __threadfence_block();
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (!((tm >> k) & 1u)) continue;
                    const int t = c + offy(k) * EX + offx(k);
                    const uint32_t sh = 8u * (uint32_t)(t & 3);
                    const uint32_t old = atomicSub(&S.st[t >> 2], 1u << sh);
                    if (((old >> sh) & 0x0Fu) == 1u) ready |= 1u << k;
                }
            }
            // keep one completed target, queue the rest; then the live count
            // gains the queued cells and loses the finished ones
            int next = -1;
            if (ready) {
                const int k = __ffs(ready) - 1;
                ready &= ready - 1;
                next = cur + offy(k) * EX + offx(k);
            }
            const unsigned fin_w = __ballot_sync(0xffffffffu, cur >= 0 && next < 0);
            queue_push(S, cur, ready, __popc(fin_w));
            cur = next;
        }
    }
    __syncthreads();

    // ---- inner tile: publish final cells, list global ones (every lane of a
    // warp runs the same steps, as mark_global_cells needs)
    unsigned long long done = 0;
    for (int ly = warp; ly < TY; ly += NW) {
        const int64_t gy = y0 + ly;
        for (int lx0 = 0; lx0 < TX; lx0 += 32) {  // warp-uniform steps
            const int lx = lx0 + lane_id;
            const int64_t gx = x0 + lx;
            const bool in_grid = lx < TX && gx < P.nx && gy < P.ny;
            const int c = (ly + H) * EX + (lx < TX ? lx : 0) + H;
            const int64_t gi = gy * P.nx + gx;
            const bool glob = in_grid && S.gf[c];
            mark_global_cells(P, G, gi, pid, glob);
            // cells never reached (a cycle in a caller's routing) stay unpublished
            if (!in_grid || glob || S.fin[c] != 1) continue;
            ++done;
            wr_f(P.out_hi, P, gi, S.vhi[c], 27);
            // the global phase pulls this trailing word if a target leaves the
            // inner tile (another tile may list it as global) or is global here
            bool need_lo = P.lo_full;
            const uint32_t tm = S.tm[c];
            uint32_t out = 0;  // directions that leave the inner tile
            if (lx == 0) out |= 0x64u;       // W NW SW
            if (lx == TX - 1) out |= 0x91u;  // E NE SE
            if (ly == 0) out |= 0x32u;       // N NE NW
            if (ly == TY - 1) out |= 0xC8u;  // S SW SE
            need_lo |= (tm & out) != 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                need_lo |= ((tm >> k) & 1u) && S.gf[c + offy(k) * EX + offx(k)];
            if (need_lo) wr_f(P.out_lo, P, gi, S.vlo[c], 28);
        }
    }
    for (int o = 16; o; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);
    if (tid == 0) S.done = 0;
    __syncthreads();
    if ((tid & 31) == 0 && done) atomicAdd(&S.done, done);
    __syncthreads();
    if (tid == 0) {
        if (S.done) atomicAdd(&G->done_cells, S.done);
        if (S.gave_up) atomicMax(&G->status, kStatusNoProgress);
    }
}

template <Mode M, bool BATCH>
cudaError_t launch_local_halo(const Prob& P, EngineGlobals* G, const Prob* probs,
                              const int64_t* prefix, int nprob, int64_t tiles, cudaStream_t s) {
    constexpr size_t sm = sizeof(SmemHalo);
    static std::atomic<unsigned long long> set_on{0};
    cudaError_t e = smem_limit_once(k_local_halo<M, BATCH>, sm, set_on);
    if (e != cudaSuccess) return e;
    if (tiles > 0)
        k_local_halo<M, BATCH><<<(unsigned)tiles, kHaloNT, sm, s>>>(P, G, probs, prefix, nprob,
                                                                  wait_limit_ns());
    return cudaGetLastError();
}

template <Mode M>
cudaError_t launch_halo_single(const Prob& P, EngineGlobals* G, cudaStream_t s) {
    const int64_t tiles = ((P.nx + kHaloTX - 1) / kHaloTX) * ((P.ny + kHaloTY - 1) / kHaloTY);
    cudaError_t e = launch_local_halo<M, false>(P, G, nullptr, nullptr, 1, tiles, s);
    if (e != cudaSuccess) return e;
    return launch_global<M, true, false>(nullptr, P, G, (unsigned long long)(P.nx * P.ny), s);
}

}  // namespace

// MFD forward accumulation: halo-tile local phase + level-synchronous global phase.
cudaError_t launch_mfd_forward(const Prob& P, EngineGlobals* G, cudaStream_t s) {
    return launch_halo_single<Mode::FwdMfd>(P, G, s);
}

// Adjoint (D8 or MFD): halo-tile local phase + level-synchronous global phase.
cudaError_t launch_adjoint(bool mfd, const Prob& P, EngineGlobals* G, cudaStream_t s) {
    return mfd ? launch_halo_single<Mode::AdjMfd>(P, G, s) : launch_halo_single<Mode::AdjD8>(P, G, s);
}

// Batched MFD forward: the CTAs of all problems' tiles in one launch, then one
// global phase.
cudaError_t launch_mfd_forward_batch(const Prob* probs, const int64_t* prefix, int nprob,
                                     int64_t tiles, unsigned long long total_cells,
                                     EngineGlobals* G, cudaStream_t s) {
    Prob none{};
    cudaError_t e = launch_local_halo<Mode::FwdMfd, true>(none, G, probs, prefix, nprob, tiles, s);
    if (e != cudaSuccess) return e;
    return launch_global<Mode::FwdMfd, true, false>(probs, none, G, total_cells, s);
}

}  // namespace fr

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
// halo.  The tiles are 64x64 (two blocks of about 96 KB per SM): measured
// 14 % faster per 8192^2 route than 64x32 (three blocks per SM), which has
// 1.875 region cells per inner cell against 1.56; halos of 6 and 10 cells
// were slower than 8.
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
// terms of a cell are summed in the fixed pairwise order of df_tree8, exactly
// as the global phase does, so a cell's value does not depend on which kernel
// computed it.
//
// Cells are finalised level by level from compact lists (a topological order,
// Sec. 3.2).  One thread finalises one cell of a level: its (up to eight)
// dependency terms are loaded side by side and summed in the fixed order.
#include "fr_engine.cuh"

namespace fr {
namespace {

constexpr int kHaloTX = kMfdTileX, kHaloTY = kMfdTileY, kHaloH = 8;
constexpr int kHaloNT = 512;

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
    uint32_t st[NE / 4];  // per cell byte: pending non-bare dependencies (bits 0-3), kG
    uint16_t queue[NE];   // level lists, appended one after another
    uint8_t rb[NR];       // receiver masks of region + ring (0 outside the grid)
    uint8_t dm[NE];       // in-region dependencies (donors forward, receivers adjoint)
    uint8_t tm[NE];       // in-region targets (receivers forward, donors adjoint)
    uint8_t fin[NE];      // 1 final, 0 pending, 0x0F outside the grid
    int qtail;
    int lcnt[3];          // sizes of the levels being appended (rotating)
    unsigned long long done;
};

__device__ __forceinline__ uint32_t st_byte(const uint32_t* st, int c) {
    return (st[c >> 2] >> (8 * (c & 3))) & 0xFFu;
}

// Marks one global inner cell: its bit and a list entry.
__device__ __forceinline__ void mark_global_cell(const Prob& P, EngineGlobals* G, int64_t gi,
                                                 int pid) {
    atomicOr(P.gbits + (gi >> 5), 1u << (gi & 31));
    const unsigned long long slot = atomicAdd(&G->glist_count, 1ull);
    if (FR_OK((int64_t)slot, P.glist_cap, 17))
        P.glist[slot] = ((unsigned long long)pid << 40) | (unsigned long long)gi;
}

// Warp-aggregated append of one optional cell per lane (all lanes call).
// (with cnt: appends after position `end`, counting in *cnt; the start list
// uses the queue tail itself)
__device__ __forceinline__ void push_cell(SmemHalo& S, int cell, int end = 0, int* cnt = nullptr) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned pm = __ballot_sync(0xffffffffu, cell >= 0);
    if (!pm) return;
    int b0 = 0;
    if (lane == (unsigned)(__ffs(pm) - 1))
        b0 = cnt ? end + atomicAdd(cnt, __popc(pm)) : atomicAdd(&S.qtail, __popc(pm));
    b0 = __shfl_sync(0xffffffffu, b0, __ffs(pm) - 1);
    if (cell >= 0) S.queue[b0 + __popc(pm & ((1u << lane) - 1u))] = (uint16_t)cell;
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
                                                           int nprob) {
    using HM = HaloMode<M>;
    constexpr int TX = HaloGeo::TX, TY = HaloGeo::TY, H = HaloGeo::H;
    constexpr int EX = HaloGeo::EX, NE = HaloGeo::NE;
    constexpr int RX = HaloGeo::RX, NR = HaloGeo::NR;
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
        S.qtail = 0;
        S.lcnt[0] = S.lcnt[1] = S.lcnt[2] = 0;
    }

    // ---- region + ring: receiver masks
    for (int i = tid; i < NR; i += NT) {
        const int ry = i / RX, rx = i - ry * RX;
        const int64_t gx = ox + rx, gy = oy + ry;
        uint8_t m = 0;
        if (gx >= 0 && gy >= 0 && gx < P.nx && gy < P.ny)
            m = (uint8_t)(recv_mask<HM::kMfd>(rd_rb(P, gy * P.nx + gx)) & grid_mask(gx, gy, P.nx, P.ny));
        S.rb[i] = m;
    }
    if constexpr (HM::kMfd) {
        // warm L2 with the region's fractions, which the level pulls read a few
        // at a time: one prefetch per 128-byte line of every region row
        constexpr int EY = HaloGeo::EY;
        const int64_t gx0 = ox + 1 < 0 ? 0 : ox + 1;
        const int64_t gx1 = ox + 1 + EX > P.nx ? P.nx : ox + 1 + EX;
        if (gx1 > gx0) {
            const int lines = (int)(((gx1 - gx0) * 32 + 127) / 128) + 1;
            for (int i = tid; i < EY * lines; i += NT) {
                const int ry = i / lines, q = i - ry * lines;
                const int64_t gy = oy + 1 + ry;
                if (gy < 0 || gy >= P.ny) continue;
                const char* row = reinterpret_cast<const char*>(P.frac + (gy * P.nx + gx0) * 8);
                const char* a = row + 128 * q;
                if (a < reinterpret_cast<const char*>(P.frac + (gy * P.nx + gx1) * 8))
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
            }
        }
    }
    __syncthreads();

    // ---- per region cell: dependencies and targets, bare / global flags,
    // initial value (rain forward; gbar adjoint)
    for (int c = tid; c < NE; c += NT) {
        const int ey = c / EX, ex = c - ey * EX;
        const int r = (ey + 1) * RX + ex + 1;
        const int64_t gx = ox + ex + 1, gy = oy + ey + 1;
        uint8_t dmr = 0, tmr = 0, fin = 0x0F, b = 0;
        float vh = 0.0f, vl = 0.0f;
        if (gx >= 0 && gy >= 0 && gx < P.nx && gy < P.ny) {
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
            b = (dep & ~in) ? (uint8_t)kG : (uint8_t)0;
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
        stb[c] = b;
        S.vhi[c] = vh;
        S.vlo[c] = vl;
    }
    __syncthreads();

    // ---- counts of non-bare in-region dependencies; cells with none start the first level
    for (int c0 = 0; c0 < NE; c0 += NT) {
        const int c = c0 + tid;
        int start = -1;
        if (c < NE && S.fin[c] == 0) {
            uint32_t n = 0;
            for (uint32_t m = S.dm[c]; m; m &= m - 1) {
                const int k = __ffs(m) - 1;
                n += S.fin[c + offy(k) * EX + offx(k)] != 1;
            }
            stb[c] |= (uint8_t)n;
            if (n == 0) start = c;
        }
        push_cell(S, start);
    }
    __syncthreads();

    // ---- levels: finalise each level's list, collect the next one
    {
        // level L appends after its own end `hi`, counting in lcnt[(L + 1) % 3];
        // thread 0 clears lcnt[(L + 2) % 3] (last read before the previous
        // barrier, next used after this one): one barrier per level
        int lo = 0, hi = S.qtail, level = 0;
        while (lo < hi) {
            if (tid == 0) S.lcnt[(level + 2) % 3] = 0;
            int* const lcnt = &S.lcnt[(level + 1) % 3];
            for (int base = lo; base < hi; base += NT) {
                const int i = base + tid;
                int c = 0;
                uint32_t ready = 0;  // codes of targets whose count reached zero
                if (i < hi) {
                    c = S.queue[i];
                    const bool glob = st_byte(S.st, c) & kG;
                    if (!glob) {
                        // dependency terms, loaded side by side, summed in the
                        // fixed pairwise order of df_tree8
                        const uint32_t dm = S.dm[c];
                        int64_t gc = 0;
                        if constexpr (HM::kMfd) {
                            const int ey = c / EX, ex = c - ey * EX;
                            gc = (oy + ey + 1) * P.nx + (ox + ex + 1);
                        }
                        df term[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            term[k] = df_make(0.0f);
                            if (!((dm >> k) & 1u)) continue;
                            const int j = c + offy(k) * EX + offx(k);
                            const df vj = {S.vhi[j], S.vlo[j]};
                            if constexpr (HM::kMfd) {
                                // forward: the donor's fraction towards c; adjoint:
                                // c's own fraction towards the receiver
                                const int64_t fi = HM::kAdj ? gc * 8 + k : (gc + offi(k, P.nx)) * 8 + opp(k);
                                term[k] = mfd_frac(__ldg(P.frac + fi), vj);
                            } else {
                                term[k] = vj;
                            }
                        }
                        const df v = df_add(df{S.vhi[c], S.vlo[c]}, df_tree8(term));
                        S.vhi[c] = v.hi;
                        S.vlo[c] = v.lo;
                    }
                    S.fin[c] = 1;
                    // targets: pass on the global flag, count down
                    for (uint32_t m = S.tm[c]; m; m &= m - 1) {
                        const int k = __ffs(m) - 1;
                        const int t = c + offy(k) * EX + offx(k);
                        const uint32_t sh = 8u * (uint32_t)(t & 3);
                        if (glob) atomicOr(&S.st[t >> 2], kG << sh);
                        const uint32_t old = atomicSub(&S.st[t >> 2], 1u << sh);
                        if (((old >> sh) & 0x0Fu) == 1u) ready |= 1u << k;
                    }
                }
                // append the ready targets, one warp-aggregated append per round
                while (__any_sync(0xffffffffu, ready != 0)) {
                    int cell = -1;
                    if (ready) {
                        const int k = __ffs(ready) - 1;
                        ready &= ready - 1;
                        cell = c + offy(k) * EX + offx(k);
                    }
                    push_cell(S, cell, hi, lcnt);
                }
            }
            __syncthreads();  // the level's values and the next list are complete
            lo = hi;
            hi += *lcnt;
            ++level;
        }
    }

    // ---- inner tile: publish final cells, list global ones
    unsigned long long done = 0;
    for (int i = tid; i < TX * TY; i += NT) {
        const int ly = i / TX, lx = i - ly * TX;
        const int64_t gx = x0 + lx, gy = y0 + ly;
        if (gx >= P.nx || gy >= P.ny) continue;
        const int c = (ly + H) * EX + lx + H;
        const int64_t gi = gy * P.nx + gx;
        if (st_byte(S.st, c) & kG) {
            mark_global_cell(P, G, gi, pid);
            continue;
        }
        if (S.fin[c] != 1) continue;  // never reached (a cycle in a caller's routing)
        ++done;
        wr_f(P.out_hi, P, gi, S.vhi[c], 27);
        bool need_lo = P.lo_full;
        if (!need_lo) {
            // the global phase pulls this trailing word if a target leaves the
            // inner tile (another tile may list it as global) or is global here
            for (uint32_t mm = S.tm[c]; mm; mm &= mm - 1) {
                const int k = __ffs(mm) - 1;
                const int lxr = lx + offx(k), lyr = ly + offy(k);
                if (lxr < 0 || lyr < 0 || lxr >= TX || lyr >= TY ||
                    (st_byte(S.st, c + offy(k) * EX + offx(k)) & kG)) {
                    need_lo = true;
                    break;
                }
            }
        }
        if (need_lo) wr_f(P.out_lo, P, gi, S.vlo[c], 28);
    }
    for (int o = 16; o; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);
    if (tid == 0) S.done = 0;
    __syncthreads();
    if ((tid & 31) == 0 && done) atomicAdd(&S.done, done);
    __syncthreads();
    if (tid == 0 && S.done) atomicAdd(&G->done_cells, S.done);
}

template <Mode M, bool BATCH>
cudaError_t launch_local_halo(const Prob& P, EngineGlobals* G, const Prob* probs,
                              const int64_t* prefix, int nprob, int64_t tiles, cudaStream_t s) {
    constexpr size_t sm = sizeof(SmemHalo);
    static std::atomic<unsigned long long> set_on{0};
    cudaError_t e = smem_limit_once(k_local_halo<M, BATCH>, sm, set_on);
    if (e != cudaSuccess) return e;
    if (tiles > 0) k_local_halo<M, BATCH><<<(unsigned)tiles, kHaloNT, sm, s>>>(P, G, probs, prefix, nprob);
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

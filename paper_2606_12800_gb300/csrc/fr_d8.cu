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
// Solve: a cell without donors ("bare", about two thirds of a rough DEM) is
// final at once.  Every other cell waits for its non-bare in-region donors
// (a count).  The cells are then finalised level by level (a topological
// order, Sec. 3.2): the first level is every cell with nothing to wait for;
// each finished cell decrements its receiver's count, and a receiver whose
// count reaches zero is appended to the next level with one warp-aggregated
// append.  Every level is a compact list, so all lanes of a warp have work.
// Each cell is visited once, donor values are pulled in fixed code order
// (deterministic two-float sums; exact 16-bit local areas), and a routing
// cycle simply leaves its cells unvisited.
//
// Tiles away from the grid boundary take a vector path: code and rain rows are
// copied asynchronously (cp.async) in one batch, and the donor masks, bare
// flags and counts of four consecutive cells are computed together on packed
// bytes (a byte-permute builds each neighbour vector, an exact zero-byte test
// compares four codes at once).  Tiles touching the boundary take a scalar
// path with bounds tests.
#include <cuda/atomic>

#include "fr_engine.cuh"

namespace fr {
namespace {

constexpr int D8H = 4;
constexpr int NT8 = 512;

template <int TX_, int TY_>
struct D8Geo {
    static constexpr int TX = TX_, TY = TY_, H = D8H;
    static constexpr int EX = TX + 2 * H, EY = TY + 2 * H, NE = EX * EY;  // extended region
    static constexpr int RY = EY + 2;  // region plus a one-cell ring
    static constexpr int CP = EX + 8;  // padded row pitch (bytes) of ring-sized byte arrays
    // Ring coordinates (rx, ry), 0 <= rx < EX + 2, live at byte ry * CP + rx + 3;
    // region cell (ex, ey) is ring cell (ex + 1, ey + 1), byte (ey + 1) * CP + ex + 4,
    // so groups of four region cells starting at ex % 4 == 0 are word aligned.
    static_assert(NE < 65535, "local areas and indices are 16-bit");
    static_assert(EX % 4 == 0 && CP % 8 == 0 && TX % 4 == 0, "four-cell groups");
};

template <class Gm, bool W, bool AREA>
struct SmemD8 {
    static constexpr int NE = Gm::NE;
    float vhi[W ? NE : 4];
    float vlo[W ? NE : 4];
    uint16_t area[AREA ? NE : 4];
    uint16_t tgt[NE];              // in-region receiver index, 0xFFFF if none
    uint32_t st[NE / 4];           // per cell byte: missing non-bare donors (bits 0-3), kG
    uint8_t dm[NE];                // in-region donor mask
    uint8_t fin[NE];               // 1 final (bare or visited), 0 pending, 0x0F outside the grid
    alignas(16) uint8_t code[Gm::RY * Gm::CP];  // receiver codes of region + ring, padded rows
    alignas(16) uint8_t nbp[Gm::RY * Gm::CP];   // 1 where a region cell is not bare
    uint16_t queue[NE];            // level lists, appended one after another
    int qtail;                     // end of the start list (the first level)
    int lcnt[3];                   // sizes of the levels being appended (rotating)
    unsigned long long done;
};

__device__ __forceinline__ uint32_t stget(const uint32_t* st, int c) {
    return (st[c >> 2] >> (8 * (c & 3))) & 0xFFu;
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

// Marks one global inner cell (rare): its bit and a list entry.
__device__ __forceinline__ void mark_one(const Prob& P, EngineGlobals* G, int64_t gi, int pid) {
    atomicOr(P.gbits + (gi >> 5), 1u << (gi & 31));
    const unsigned long long slot = atomicAdd(&G->glist_count, 1ull);
    if (FR_OK((int64_t)slot, P.glist_cap, 17))
        P.glist[slot] = ((unsigned long long)pid << 40) | (unsigned long long)gi;
}

// Warp-aggregated append of up to four cells per lane (all lanes call).
template <class S_>
__device__ __forceinline__ void push_starts(S_& S, int n, const int (&cells)[4]) {
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
__global__ void __launch_bounds__(NT8) k_local_d8(Prob Pone, EngineGlobals* G,
                                                  const Prob* __restrict__ probs,
                                                  const int64_t* __restrict__ prefix, int nprob) {
    constexpr int TX = Gm::TX, TY = Gm::TY, H = Gm::H, EX = Gm::EX, EY = Gm::EY, NE = Gm::NE;
    constexpr int RY = Gm::RY, CP = Gm::CP;
    using Sm = SmemD8<Gm, W, AREA>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm& S = *reinterpret_cast<Sm*>(smem_raw);
    const int tid = threadIdx.x;
    int64_t lt = (int64_t)blockIdx.x;
    const int pid = BATCH ? batch_problem(prefix, nprob, lt) : 0;
    const Prob& P = BATCH ? probs[pid] : Pone;
    const int64_t tiles_x = (P.nx + TX - 1) / TX;
    const int64_t ty = lt / tiles_x, tx = lt - ty * tiles_x;
    const int64_t x0 = tx * TX, y0 = ty * TY;
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
    uint8_t* stb = reinterpret_cast<uint8_t*>(S.st);
    if (tid == 0) {
        S.qtail = 0;
        S.lcnt[0] = S.lcnt[1] = S.lcnt[2] = 0;
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
                    if (FR_OK(g + 3, ncell(P), 8)) cp_async16(S.vhi + ey * EX + 4 * q, P.init + g);
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
        // ---- donor masks, bare / global flags, receivers (4 cells per thread)
        for (int gq = tid; gq < NE / 4; gq += NT8) {
            const int ey = gq / (EX / 4), ex = (gq - ey * (EX / 4)) * 4;
            const int w1 = (ex + 4) >> 2;
            const Row3 up = row3(S.code + ey * CP, w1);
            const Row3 mid = row3(S.code + (ey + 1) * CP, w1);
            const Row3 dn = row3(S.code + (ey + 2) * CP, w1);
            uint32_t dmf = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                dmf |= zero_bytes(nbr(up, mid, dn, k) ^ (0x01010101u * (uint32_t)opp(k))) >> (7 - k);
            uint32_t in = 0xFFFFFFFFu;
            if (ex == 0) in &= ~0x64u;                   // W NW SW of the first cell
            if (ex == EX - 4) in &= ~(0x91u << 24);      // E NE SE of the last cell
            if (ey == 0) in &= ~0x32323232u;             // N NE NW
            if (ey == EY - 1) in &= ~0xC8C8C8C8u;        // S SW SE
            const uint32_t bare = zero_bytes(dmf) >> 7;  // 1 per bare cell
            const uint32_t glob = (~zero_bytes(dmf & ~in) & 0x80808080u) >> 3;  // kG
            const int c = ey * EX + ex;
            reinterpret_cast<uint32_t*>(S.dm)[c >> 2] = dmf & in;
            reinterpret_cast<uint32_t*>(S.fin)[c >> 2] = bare;
            S.st[c >> 2] = glob;
            reinterpret_cast<uint32_t*>(S.nbp + (ey + 1) * CP)[w1] = bare ^ 0x01010101u;
            uint32_t t01 = 0, t23 = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t k = (mid.c >> (8 * q)) & 0xFFu;
                uint32_t t = 0xFFFFu;
                if (k < 8) {
                    const int xr = ex + q + offx((int)k), yr = ey + offy((int)k);
                    if (xr >= 0 && yr >= 0 && xr < EX && yr < EY) t = (uint32_t)(yr * EX + xr);
                }
                if (q < 2) t01 |= t << (16 * q);
                else t23 |= t << (16 * (q - 2));
            }
            *reinterpret_cast<uint2*>(S.tgt + c) = make_uint2(t01, t23);
            if constexpr (W) {
                if (!P.init) *reinterpret_cast<float4*>(S.vhi + c) = make_float4(1.f, 1.f, 1.f, 1.f);
                *reinterpret_cast<float4*>(S.vlo + c) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if constexpr (AREA) *reinterpret_cast<uint2*>(S.area + c) = make_uint2(0x00010001u, 0x00010001u);
        }
        __syncthreads();
        // ---- counts of non-bare in-region donors; cells with none start level 1
        for (int gq0 = 0; gq0 < NE / 4; gq0 += NT8) {
            const int gq = gq0 + tid;
            int cells[4];
            int n = 0;
            if (gq < NE / 4) {
                const int ey = gq / (EX / 4), ex = (gq - ey * (EX / 4)) * 4;
                const int c = ey * EX + ex;
                const uint32_t dmr = reinterpret_cast<const uint32_t*>(S.dm)[c >> 2];
                uint32_t nb = 0;
                if (dmr) {
                    const int w1 = (ex + 4) >> 2;
                    const Row3 up = row3(S.nbp + ey * CP, w1);
                    const Row3 mid = row3(S.nbp + (ey + 1) * CP, w1);
                    const Row3 dn = row3(S.nbp + (ey + 2) * CP, w1);
#pragma unroll
                    for (int k = 0; k < 8; ++k) nb |= (nbr(up, mid, dn, k) & 0x01010101u) << k;
                }
                const uint32_t cnt = popc_bytes(nb & dmr);
                S.st[c >> 2] |= cnt;
                const uint32_t fin = reinterpret_cast<const uint32_t*>(S.fin)[c >> 2];
                const uint32_t st_mask = zero_bytes(fin) & zero_bytes(cnt);  // not bare, no wait
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if ((st_mask >> (8 * q + 7)) & 1u) cells[n++] = c + q;
            }
            push_starts(S, n, cells);
        }
        __syncthreads();
    } else {
        // ---- scalar path (tiles touching the grid boundary)
        for (int i = tid; i < RY * CP; i += NT8) {
            const int ry = i / CP, rx = i - ry * CP - 3;
            uint8_t code = kSink;
            if (rx >= gx_lo && rx < gx_hi && ry >= gy_lo && ry < gy_hi) {
                code = rd_rb(P, (oy + ry) * P.nx + (ox + rx));
                if (code < 8) {
                    const int xr = rx + offx(code), yr = ry + offy(code);
                    if (xr < gx_lo || xr >= gx_hi || yr < gy_lo || yr >= gy_hi) code = kSink;
                } else {
                    code = kSink;
                }
            }
            S.code[i] = code;
        }
        __syncthreads();
        for (int c = tid; c < NE; c += NT8) {
            const int ey = c / EX, ex = c - ey * EX;
            const int rx = ex + 1, ry = ey + 1;
            uint8_t b = 0, dmr = 0, bare = 0x0F;  // outside the grid: never solved
            uint16_t t = 0xFFFFu;
            if (rx >= gx_lo && rx < gx_hi && ry >= gy_lo && ry < gy_hi) {
                const int r = ry * CP + rx + 3;
                uint32_t dm = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    dm |= (uint32_t)(S.code[r + offy(k) * CP + offx(k)] == (uint8_t)opp(k)) << k;
                uint32_t in = 0xFFu;
                if (ex == 0) in &= ~0x64u;
                if (ex == EX - 1) in &= ~0x91u;
                if (ey == 0) in &= ~0x32u;
                if (ey == EY - 1) in &= ~0xC8u;
                dmr = (uint8_t)(dm & in);
                b = (uint8_t)((dm & ~in) ? kG : 0u);
                bare = dm == 0;
                const uint8_t k = S.code[r];
                if (k < 8) {
                    const int xr = ex + offx(k), yr = ey + offy(k);
                    if (xr >= 0 && yr >= 0 && xr < EX && yr < EY) t = (uint16_t)(yr * EX + xr);
                }
                if constexpr (W) {
                    const int64_t gi = (oy + ry) * P.nx + (ox + rx);
                    S.vhi[c] = P.init ? rd_in(P.init, P, gi, 8) : 1.0f;
                    S.vlo[c] = 0.0f;
                }
                if constexpr (AREA) S.area[c] = 1;
            }
            S.dm[c] = dmr;
            S.fin[c] = bare;
            S.tgt[c] = t;
            stb[c] = b;
        }
        __syncthreads();
        uint8_t cnt_own[(NE + NT8 - 1) / NT8];
        int nq = 0;
        for (int c = tid; c < NE; c += NT8, ++nq) {
            uint32_t n = 0;
            for (uint32_t m = S.dm[c]; m; m &= m - 1) {
                const int k = __ffs(m) - 1;
                n += S.fin[c + offy(k) * EX + offx(k)] != 1;
            }
            cnt_own[nq] = (uint8_t)n;
        }
        __syncthreads();
        nq = 0;
        for (int c0 = 0; c0 < NE; c0 += NT8, ++nq) {
            const int c = c0 + tid;
            int cells[4];
            int n = 0;
            if (c < NE) {
                stb[c] |= cnt_own[nq];
                if (S.fin[c] == 0 && cnt_own[nq] == 0) cells[n++] = c;
            }
            push_starts(S, n, cells);
        }
        __syncthreads();
    }

    // ---- levels: finalise each level's list, collect the next one
    {
        const unsigned lane = tid & 31u;
        // level L appends the next level after its own end `hi`, counting in
        // lcnt[(L + 1) % 3]; thread 0 clears lcnt[(L + 2) % 3], last read before
        // the previous barrier and next used after this level's barrier, so one
        // barrier per level orders everything
        int lo = 0, hi = S.qtail, level = 0;
        while (lo < hi) {
            if (tid == 0) S.lcnt[(level + 2) % 3] = 0;
            int* const lcnt = &S.lcnt[(level + 1) % 3];
            for (int base = lo; base < hi; base += NT8) {
                const int i = base + tid;
                int push = -1;
                if (i < hi) {
                    const int c = S.queue[i];
                    const bool glob = stget(S.st, c) & kG;
                    const uint32_t dm = S.dm[c];
                    const int t = S.tgt[c];
                    if (!glob && dm) {
                        // pull the donors' values in ascending code order (set bits of dm)
                        df v;
                        uint32_t a = 0;
                        if constexpr (W) v = {S.vhi[c], S.vlo[c]};
                        if constexpr (AREA) a = S.area[c];
                        for (uint32_t m = dm; m; m &= m - 1) {
                            const int k = __ffs(m) - 1;
                            const int j = c + offy(k) * EX + offx(k);
                            if constexpr (W) v = df_add(v, df{S.vhi[j], S.vlo[j]});
                            if constexpr (AREA) a += S.area[j];
                        }
                        if constexpr (W) {
                            S.vhi[c] = v.hi;
                            S.vlo[c] = v.lo;
                        }
                        if constexpr (AREA) S.area[c] = (uint16_t)a;
                    }
                    S.fin[c] = 1;
                    if (t != 0xFFFF) {
                        // counts are read only after the level barrier: relaxed atomics
                        const uint32_t sh = 8u * (uint32_t)(t & 3);
                        if (glob) atomicOr(&S.st[t >> 2], kG << sh);
                        const uint32_t old = atomicSub(&S.st[t >> 2], 1u << sh);
                        if (((old >> sh) & 0x0Fu) == 1u) push = t;
                    }
                }
                const unsigned pm = __ballot_sync(0xffffffffu, push >= 0);
                if (pm) {
                    int b0 = 0;
                    if (lane == (unsigned)(__ffs(pm) - 1)) b0 = hi + atomicAdd(lcnt, __popc(pm));
                    b0 = __shfl_sync(0xffffffffu, b0, __ffs(pm) - 1);
                    if (push >= 0) S.queue[b0 + __popc(pm & ((1u << lane) - 1u))] = (uint16_t)push;
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
    auto need_lo_of = [&](int c, int lx, int ly) -> bool {
        // a cell's trailing word is pulled later when its receiver leaves the
        // inner tile (another tile may list it as global) or is global here
        const uint8_t code = S.code[(ly + H + 1) * CP + lx + H + 4];
        if (code >= 8) return false;
        const int lxr = lx + offx(code), lyr = ly + offy(code);
        if (lxr < 0 || lyr < 0 || lxr >= TX || lyr >= TY) return true;
        return stget(S.st, c + offy(code) * EX + offx(code)) & kG;
    };
    auto publish_one = [&](int lx, int ly) {
        const int64_t gx = x0 + lx, gy = y0 + ly;
        if (gx >= P.nx || gy >= P.ny) return;
        const int c = (ly + H) * EX + lx + H;
        const int64_t gi = gy * P.nx + gx;
        if (stget(S.st, c) & kG) {
            mark_one(P, G, gi, pid);
            return;
        }
        if (S.fin[c] != 1) return;  // never reached (a cycle)
        ++done;
        if constexpr (W) {
            wr_f(P.out_hi, P, gi, S.vhi[c], 27);
            if (P.lo_full || need_lo_of(c, lx, ly)) wr_f(P.out_lo, P, gi, S.vlo[c], 28);
        }
        if constexpr (AREA) wr_area(P, gi, S.area[c]);
    };
    if (vec && x0 + TX <= P.nx && y0 + TY <= P.ny) {
        for (int gq = tid; gq < TX * TY / 4; gq += NT8) {
            const int ly = gq / (TX / 4), lx = (gq - ly * (TX / 4)) * 4;
            const int c = (ly + H) * EX + lx + H;
            const uint32_t st4 = S.st[c >> 2];
            const uint32_t fin4 = reinterpret_cast<const uint32_t*>(S.fin)[c >> 2];
            if ((st4 & 0x10101010u) || fin4 != 0x01010101u) {
                for (int q = 0; q < 4; ++q) publish_one(lx + q, ly);  // rare: global or unreached
                continue;
            }
            done += 4;
            const int64_t gi = (y0 + ly) * P.nx + x0 + lx;
            if constexpr (W) {
                *reinterpret_cast<float4*>(P.out_hi + gi) = *reinterpret_cast<const float4*>(S.vhi + c);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (P.lo_full || need_lo_of(c + q, lx + q, ly))
                        wr_f(P.out_lo, P, gi + q, S.vlo[c + q], 28);
            }
            if constexpr (AREA) {
                const uint2 a = *reinterpret_cast<const uint2*>(S.area + c);
                ulonglong2* out = reinterpret_cast<ulonglong2*>(P.area + gi);
                out[0] = make_ulonglong2(a.x & 0xFFFFu, a.x >> 16);
                out[1] = make_ulonglong2(a.y & 0xFFFFu, a.y >> 16);
            }
        }
    } else {
        for (int i = tid; i < TX * TY; i += NT8) {
            const int ly = i / TX, lx = i - ly * TX;
            publish_one(lx, ly);
        }
    }
    for (int o = 16; o; o >>= 1) done += __shfl_down_sync(0xffffffffu, done, o);
    if (tid == 0) S.done = 0;
    __syncthreads();
    if ((tid & 31) == 0 && done) atomicAdd(&S.done, done);
    __syncthreads();
    if (tid == 0 && S.done) atomicAdd(&G->done_cells, S.done);
}

template <class Gm, bool W, bool AREA, bool BATCH>
cudaError_t launch_local_d8(const Prob& P, EngineGlobals* G, const Prob* probs,
                            const int64_t* prefix, int nprob, int64_t tiles, cudaStream_t s) {
    constexpr size_t sm = sizeof(SmemD8<Gm, W, AREA>);
    cudaError_t e = cudaFuncSetAttribute(k_local_d8<Gm, W, AREA, BATCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (tiles > 0) k_local_d8<Gm, W, AREA, BATCH><<<(unsigned)tiles, NT8, sm, s>>>(P, G, probs, prefix, nprob);
    return cudaGetLastError();
}

template <class Gm, bool W, bool AREA>
cudaError_t launch_d8(const Prob& P, EngineGlobals* G, cudaStream_t s) {
    const int64_t tiles = ((P.nx + Gm::TX - 1) / Gm::TX) * ((P.ny + Gm::TY - 1) / Gm::TY);
    cudaError_t e = launch_local_d8<Gm, W, AREA, false>(P, G, nullptr, nullptr, 1, tiles, s);
    if (e != cudaSuccess) return e;
    return launch_global<Mode::FwdD8, W, AREA>(nullptr, P, G, (unsigned long long)(P.nx * P.ny), s);
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
using GeoD8s = D8Geo<kD8TileX / 2, kD8TileY>;   // geometry 1: 64x32, three CTAs per SM

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
    // 64x32 inner tiles: measured fastest at 4096^2 (three CTAs per SM)
    if (want_w && want_area) return launch_d8<GeoD8s, true, true>(P, G, s);
    if (want_w) return launch_d8<GeoD8s, true, false>(P, G, s);
    return launch_d8<GeoD8s, false, true>(P, G, s);
}

// Batched D8 forward: the CTAs of all problems' tiles in one launch (tile
// prefix of the chosen geometry), then one walker phase.
cudaError_t launch_d8_forward_batch(int geo, bool want_w, bool want_area, const Prob* probs,
                                    const int64_t* prefix, int nprob, int64_t tiles,
                                    unsigned long long total_cells, EngineGlobals* G, cudaStream_t s) {
    if (geo == 1) return d8_batch_w<GeoD8s>(want_w, want_area, probs, prefix, nprob, tiles, total_cells, G, s);
    return d8_batch_w<GeoD8>(want_w, want_area, probs, prefix, nprob, tiles, total_cells, G, s);
}

}  // namespace fr

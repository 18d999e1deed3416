// fr_d8.cu -- local phase of D8 forward accumulation over halo-extended tiles.
//
// Each CTA owns an inner tile of D8X x D8Y cells and solves the extended
// region (inner tile plus a D8H-cell halo on every side) exactly in shared
// memory: the paper's per-subdomain high-to-low solve (Sec. 2.4), with
// overlapping subdomains.  An inner cell is final unless its upstream basin
// reaches outside the extended region ("global"); on the synthetic fractal
// DEMs a 4-cell halo leaves about 0.03 % of the cells global, which the walker
// kernel of fr_engine.cuh then finishes.  Halo cells are solved only to feed
// the inner ones and are not written.
//
// Solve: a cell without donors ("bare", about two thirds of a rough DEM) is
// final at once.  The other cells are finalised in rounds: each thread keeps a
// bit mask of its own pending cells and finalises a cell once all of its
// non-bare in-region donors are final (a topological order, Sec. 3.2), pulling
// the donors' values in fixed code order (deterministic two-float sums; exact
// 16-bit local areas).  There are no atomics; the rounds stop when nothing is
// pending or a round makes no progress (a routing cycle).
//
// Tiles away from the grid boundary take a vector path: receiver codes arrive
// as 32-bit words, and the donor masks, bare flags and non-bare donor masks of four
// consecutive cells are computed together on packed bytes (a byte-permute
// builds each neighbour vector, an exact zero-byte test compares four codes
// at once).  Tiles touching the boundary take a scalar path with bounds tests.
#include <cuda/atomic>

#include "fr_engine.cuh"

namespace fr {
namespace {

constexpr int D8X = 128, D8Y = 32, D8H = 4;
constexpr int EX = D8X + 2 * D8H, EY = D8Y + 2 * D8H, NE = EX * EY;  // extended region
constexpr int RY8 = EY + 2;  // region plus a one-cell ring
constexpr int CP = EX + 8;   // padded row pitch (bytes) of ring-sized byte arrays
// Ring coordinates (rx, ry), 0 <= rx < EX + 2, live at byte ry * CP + rx + 3;
// region cell (ex, ey) is ring cell (ex + 1, ey + 1), byte (ey + 1) * CP + ex + 4,
// so groups of four region cells starting at ex % 4 == 0 are word aligned.
constexpr int NT8 = 512;
static_assert(NE < 65536, "local areas are 16-bit");
static_assert(EX % 4 == 0 && CP % 4 == 0 && D8X % 4 == 0, "four-cell groups");

template <bool W, bool AREA>
struct SmemD8 {
    float vhi[W ? NE : 4];
    float vlo[W ? NE : 4];
    uint16_t area[AREA ? NE : 4];
    uint32_t st[NE / 4];      // per cell byte: kG once the cell is known to be global
    uint8_t dm[NE];           // in-region donor mask
    uint8_t nbdm[NE];         // in-region donors that are not bare
    uint8_t fin[NE];          // 1 final, 0 pending (0x0F outside the grid)
    uint8_t code[RY8 * CP];   // receiver codes of region + ring, padded rows
    uint8_t nbp[RY8 * CP];    // 1 where a region cell has a donor (not bare), padded rows
    unsigned long long done;
};

__device__ __forceinline__ uint32_t stget(const uint32_t* st, int c) {
    return (st[c >> 2] >> (8 * (c & 3))) & 0xFFu;
}

// 0x80 in each byte of x that is zero, 0 elsewhere (exact, no carries between bytes).
__device__ __forceinline__ uint32_t zero_bytes(uint32_t x) {
    return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
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

// Marks one global inner cell (rare): its bit and a list entry.
__device__ __forceinline__ void mark_one(const Prob& P, EngineGlobals* G, int64_t gi) {
    atomicOr(P.gbits + (gi >> 5), 1u << (gi & 31));
    const unsigned long long slot = atomicAdd(&G->glist_count, 1ull);
    if (FR_OK((int64_t)slot, P.glist_cap, 17)) P.glist[slot] = (unsigned long long)gi;
}

template <bool W, bool AREA>
__global__ void __launch_bounds__(NT8) k_local_d8(Prob P, EngineGlobals* G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemD8<W, AREA>& S = *reinterpret_cast<SmemD8<W, AREA>*>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t tiles_x = (P.nx + D8X - 1) / D8X;
    const int64_t ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    const int64_t x0 = tx * D8X, y0 = ty * D8Y;
    // ring origin (may be negative) and the grid's extent in ring coordinates
    const int64_t ox = x0 - D8H - 1, oy = y0 - D8H - 1;
    const int gx_hi = (int)(P.nx - ox < EX + 2 ? P.nx - ox : EX + 2);
    const int gy_hi = (int)(P.ny - oy < RY8 ? P.ny - oy : RY8);
    const int gx_lo = (int)(ox < 0 ? -ox : 0), gy_lo = (int)(oy < 0 ? -oy : 0);
    // vector path: the padded ring rows [x0 - 8, x0 + EX) are inside the grid,
    // and the arrays allow aligned word / float4 access
    const bool vec = x0 >= 8 && x0 + EX <= P.nx && oy >= 0 && oy + RY8 <= P.ny &&
                     (P.nx & 3) == 0 && ((uintptr_t)P.rb & 3) == 0 &&
                     (!W || !P.init || ((uintptr_t)P.init & 15) == 0) &&
                     (!W || ((uintptr_t)P.out_hi & 15) == 0) &&
                     (!AREA || ((uintptr_t)P.area & 15) == 0);
    uint8_t* stb = reinterpret_cast<uint8_t*>(S.st);

    if (vec) {
        // ---- codes: whole padded rows as words (byte b <-> grid x = x0 - 8 + b)
        for (int i = tid; i < RY8 * (CP / 4); i += NT8) {
            const int ry = i / (CP / 4), w = i - ry * (CP / 4);
            const int64_t g = (oy + ry) * P.nx + (x0 - 8 + 4 * w);
            reinterpret_cast<uint32_t*>(S.code)[i] =
                FR_OK(g + 3, ncell(P), 1) ? __ldg(reinterpret_cast<const uint32_t*>(P.rb + g)) : 0xFFFFFFFFu;
        }
        __syncthreads();
        // ---- donor masks, bare flags, global flags, initial values (4 cells / thread)
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
            if constexpr (W) {
                const int64_t g = (oy + ey + 1) * P.nx + (x0 - D8H + ex);
                float4 r = make_float4(1.f, 1.f, 1.f, 1.f);
                if (P.init && FR_OK(g + 3, ncell(P), 8))
                    r = __ldg(reinterpret_cast<const float4*>(P.init + g));
                *reinterpret_cast<float4*>(S.vhi + c) = r;
                *reinterpret_cast<float4*>(S.vlo + c) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if constexpr (AREA) *reinterpret_cast<uint2*>(S.area + c) = make_uint2(0x00010001u, 0x00010001u);
        }
        __syncthreads();
        // ---- non-bare donor masks
        for (int gq = tid; gq < NE / 4; gq += NT8) {
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
            reinterpret_cast<uint32_t*>(S.nbdm)[c >> 2] = nb & dmr;
        }
        __syncthreads();
    } else {
        // ---- scalar path (tiles touching the grid boundary)
        for (int i = tid; i < RY8 * CP; i += NT8) {
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
            uint8_t b = 0;
            uint8_t dmr = 0, bare = 0x0F;  // outside the grid: never solved
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
                if constexpr (W) {
                    const int64_t gi = (oy + ry) * P.nx + (ox + rx);
                    S.vhi[c] = P.init ? rd_in(P.init, P, gi, 8) : 1.0f;
                    S.vlo[c] = 0.0f;
                }
                if constexpr (AREA) S.area[c] = 1;
            }
            S.dm[c] = dmr;
            S.fin[c] = bare;
            stb[c] = b;
        }
        __syncthreads();
        for (int c = tid; c < NE; c += NT8) {
            uint32_t nb = 0;
            for (uint32_t m = S.dm[c]; m; m &= m - 1) {
                const int k = __ffs(m) - 1;
                if (S.fin[c + offy(k) * EX + offx(k)] != 1) nb |= 1u << k;
            }
            S.nbdm[c] = (uint8_t)nb;
        }
        __syncthreads();
    }

    // ---- rounds: finalise pending cells whose non-bare donors are final
    {
        constexpr int KMAX = (NE + NT8 - 1) / NT8;
        static_assert(KMAX <= 32, "pending cells fit a 32-bit mask");
        uint32_t pend = 0;
        for (int k = 0; k < KMAX; ++k) {
            const int c = tid + k * NT8;
            if (c < NE && S.fin[c] == 0) pend |= 1u << k;
        }
        while (true) {
            uint32_t progress = 0;
            for (uint32_t m = pend; m; m &= m - 1) {
                const int k = __ffs(m) - 1;
                const int c = tid + k * NT8;
                const uint32_t nbd = S.nbdm[c];
                bool ready = true;
                uint32_t g = stb[c] & kG;
                for (uint32_t q = nbd; q; q &= q - 1) {
                    const int j = c + offy(__ffs(q) - 1) * EX + offx(__ffs(q) - 1);
                    if (reinterpret_cast<volatile uint8_t*>(S.fin)[j] != 1) {
                        ready = false;
                        break;
                    }
                    g |= stb[j] & kG;
                }
                if (!ready) continue;
                __threadfence_block();  // donors' values are visible once their flags are
                if (!g) {
                    const uint32_t dm = S.dm[c];
                    df v;
                    uint32_t a = 0;
                    if constexpr (W) v = {S.vhi[c], S.vlo[c]};
                    if constexpr (AREA) a = S.area[c];
                    for (uint32_t q = dm; q; q &= q - 1) {
                        const int kk = __ffs(q) - 1;
                        const int j = c + offy(kk) * EX + offx(kk);
                        if constexpr (W) v = df_add(v, df{S.vhi[j], S.vlo[j]});
                        if constexpr (AREA) a += S.area[j];
                    }
                    if constexpr (W) {
                        S.vhi[c] = v.hi;
                        S.vlo[c] = v.lo;
                    }
                    if constexpr (AREA) S.area[c] = (uint16_t)a;
                } else {
                    stb[c] = (uint8_t)kG;
                }
                __threadfence_block();  // publish the value before the flag
                reinterpret_cast<volatile uint8_t*>(S.fin)[c] = 1;
                pend &= ~(1u << k);
                progress = 1;
            }
            if (!__syncthreads_or(pend != 0)) break;
            if (!__syncthreads_or(progress)) break;  // a cycle: nothing can finish
        }
    }
    __syncthreads();

    // ---- inner tile: publish final cells, list global ones
    unsigned long long done = 0;
    auto need_lo_of = [&](int lx, int ly) -> bool {
        // a cell's trailing word is pulled later when its receiver leaves the
        // inner tile (another tile may list it as global) or is global here
        const uint8_t code = S.code[(ly + D8H + 1) * CP + lx + D8H + 4];
        if (code >= 8) return false;
        const int lxr = lx + offx(code), lyr = ly + offy(code);
        return lxr < 0 || lyr < 0 || lxr >= D8X || lyr >= D8Y ||
               (stget(S.st, (lyr + D8H) * EX + lxr + D8H) & kG);
    };
    auto publish_one = [&](int lx, int ly) {
        const int ex = lx + D8H, ey = ly + D8H;
        const int64_t gx = x0 + lx, gy = y0 + ly;
        if (gx >= P.nx || gy >= P.ny) return;
        const int c = ey * EX + ex;
        const int64_t gi = gy * P.nx + gx;
        if (stget(S.st, c) & kG) {
            mark_one(P, G, gi);
            return;
        }
        if (S.fin[c] != 1) return;  // never reached (a cycle)
        ++done;
        if constexpr (W) {
            wr_f(P.out_hi, P, gi, S.vhi[c], 27);
            if (P.lo_full || need_lo_of(lx, ly)) wr_f(P.out_lo, P, gi, S.vlo[c], 28);
        }
        if constexpr (AREA) wr_area(P, gi, S.area[c]);
    };
    if (vec && x0 + D8X <= P.nx && y0 + D8Y <= P.ny) {
        for (int gq = tid; gq < D8X * D8Y / 4; gq += NT8) {
            const int ly = gq / (D8X / 4), lx = (gq - ly * (D8X / 4)) * 4;
            const int c = (ly + D8H) * EX + lx + D8H;
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
                    if (P.lo_full || need_lo_of(lx + q, ly)) wr_f(P.out_lo, P, gi + q, S.vlo[c + q], 28);
            }
            if constexpr (AREA) {
                const uint2 a = *reinterpret_cast<const uint2*>(S.area + c);
                ulonglong2* out = reinterpret_cast<ulonglong2*>(P.area + gi);
                out[0] = make_ulonglong2(a.x & 0xFFFFu, a.x >> 16);
                out[1] = make_ulonglong2(a.y & 0xFFFFu, a.y >> 16);
            }
        }
    } else {
        for (int i = tid; i < D8X * D8Y; i += NT8) {
            const int ly = i / D8X, lx = i - ly * D8X;
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

template <bool W, bool AREA>
cudaError_t launch_d8(const Prob& P, EngineGlobals* G, cudaStream_t s) {
    constexpr size_t sm = sizeof(SmemD8<W, AREA>);
    cudaError_t e = cudaFuncSetAttribute(k_local_d8<W, AREA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t tiles = ((P.nx + D8X - 1) / D8X) * ((P.ny + D8Y - 1) / D8Y);
    k_local_d8<W, AREA><<<(unsigned)tiles, NT8, sm, s>>>(P, G);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_global<Mode::FwdD8, W, AREA><<<walker_grid(), 256, 0, s>>>(nullptr, P, G,
                                                                 (unsigned long long)(P.nx * P.ny));
    return cudaGetLastError();
}

}  // namespace

// D8 forward accumulation: halo-tile local phase + walker phase.
cudaError_t launch_d8_forward(bool want_w, bool want_area, const Prob& P, EngineGlobals* G,
                              cudaStream_t s) {
    if (want_w && want_area) return launch_d8<true, true>(P, G, s);
    if (want_w) return launch_d8<true, false>(P, G, s);
    return launch_d8<false, true>(P, G, s);
}

}  // namespace fr

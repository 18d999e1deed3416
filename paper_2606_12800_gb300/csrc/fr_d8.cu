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
// Within the region every cell has at most one receiver, so a finished cell is
// continued by the thread that completes its receiver's count ("last
// arriver", shared-memory atomics): each cell is visited once, with no rounds
// and no barriers inside the solve.  Values are pulled from donors in fixed
// code order (deterministic two-float sums; exact 16-bit local areas).
#include "fr_engine.cuh"

namespace fr {
namespace {

constexpr int D8X = 128, D8Y = 32, D8H = 4;
constexpr int EX = D8X + 2 * D8H, EY = D8Y + 2 * D8H, NE = EX * EY;  // extended region
constexpr int RX8 = EX + 2, RY8 = EY + 2;                            // plus a one-cell ring
constexpr int NT8 = 512;
static_assert(NE < 65536, "local areas are 16-bit");

template <bool W, bool AREA>
struct SmemD8 {
    float vhi[W ? NE : 1];
    float vlo[W ? NE : 1];
    uint16_t area[AREA ? NE : 1];
    uint32_t st[NE / 4 + 1];   // per cell: in-region donors missing (bits 0-3), kG, kDone
    uint8_t dm[NE];            // in-region donor mask
    uint8_t code[RX8 * RY8];   // receiver codes of the region and its ring (kSink = none)
    unsigned long long done;
};

__device__ __forceinline__ uint32_t stget(const uint32_t* st, int c) {
    return (st[c >> 2] >> (8 * (c & 3))) & 0xFFu;
}

template <bool W, bool AREA>
__global__ void __launch_bounds__(NT8) k_local_d8(Prob P, EngineGlobals* G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemD8<W, AREA>& S = *reinterpret_cast<SmemD8<W, AREA>*>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t tiles_x = (P.nx + D8X - 1) / D8X;
    const int64_t ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    // region origin (may be negative) and the grid's extent relative to it
    const int64_t ox = tx * D8X - D8H - 1, oy = ty * D8Y - D8H - 1;  // ring origin
    // ring coordinates inside the grid: gx_lo <= rx < gx_hi, gy_lo <= ry < gy_hi
    const int gx_hi = (int)(P.nx - ox < RX8 ? P.nx - ox : RX8);
    const int gy_hi = (int)(P.ny - oy < RY8 ? P.ny - oy : RY8);
    const int gx_lo = (int)(ox < 0 ? -ox : 0), gy_lo = (int)(oy < 0 ? -oy : 0);

    // receiver codes of region + ring; codes leaving the grid become "none"
    for (int i = tid; i < RX8 * RY8; i += NT8) {
        const int ry = i / RX8, rx = i - ry * RX8;
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

    // region cells: in-region donors, missing-donor counts, initial values
    uint8_t* stb = reinterpret_cast<uint8_t*>(S.st);
    for (int c = tid; c < NE; c += NT8) {
        const int ey = c / EX, ex = c - ey * EX;
        const int rx = ex + 1, ry = ey + 1;
        uint8_t b = 0x0F;  // outside the grid: never solved
        uint8_t dmr = 0;
        if (rx >= gx_lo && rx < gx_hi && ry >= gy_lo && ry < gy_hi) {
            const int r = ry * RX8 + rx;
            uint32_t dm = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                dm |= (uint32_t)(S.code[r + offy(k) * RX8 + offx(k)] == (uint8_t)opp(k)) << k;
            // donors that lie in the ring (outside the region) make the cell global
            uint32_t in = 0xFFu;
            if (ex == 0) in &= ~((1u << 2) | (1u << 5) | (1u << 6));
            if (ex == EX - 1) in &= ~((1u << 0) | (1u << 4) | (1u << 7));
            if (ey == 0) in &= ~((1u << 1) | (1u << 4) | (1u << 5));
            if (ey == EY - 1) in &= ~((1u << 3) | (1u << 6) | (1u << 7));
            dmr = (uint8_t)(dm & in);
            b = (uint8_t)(__popc(dmr) | ((dm & ~in) ? kG : 0u));
            if constexpr (W) {
                const int64_t gi = (oy + ry) * P.nx + (ox + rx);
                S.vhi[c] = P.init ? rd_in(P.init, P, gi, 8) : 1.0f;
                S.vlo[c] = 0.0f;
            }
            if constexpr (AREA) S.area[c] = 1;
        }
        S.dm[c] = dmr;
        stb[c] = b;
    }
    __syncthreads();

    // chain walks from every cell without in-region donors
    for (int c0 = tid; c0 < NE; c0 += NT8) {
        if (S.dm[c0] != 0 || (stb[c0] & 0x0Fu) != 0) continue;
        int c = c0;
        while (true) {
            const uint32_t b = stget(S.st, c);
            const bool glob = b & kG;
            const uint32_t dm = S.dm[c];
            if (!glob && dm) {
                if constexpr (W) {
                    df v = {S.vhi[c], S.vlo[c]};
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if ((dm >> k) & 1u) {
                            const int j = c + offy(k) * EX + offx(k);
                            v = df_add(v, df{S.vhi[j], S.vlo[j]});
                        }
                    S.vhi[c] = v.hi;
                    S.vlo[c] = v.lo;
                }
                if constexpr (AREA) {
                    uint32_t a = S.area[c];
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if ((dm >> k) & 1u) a += S.area[c + offy(k) * EX + offx(k)];
                    S.area[c] = (uint16_t)a;
                }
            }
            const int ey = c / EX, ex = c - ey * EX;
            const uint8_t code = S.code[(ey + 1) * RX8 + ex + 1];
            atomicOr(&S.st[c >> 2], kDone << (8 * (c & 3)));
            if (code >= 8) break;
            const int xr = ex + offx(code), yr = ey + offy(code);
            if (xr < 0 || yr < 0 || xr >= EX || yr >= EY) break;  // leaves the region
            const int t = yr * EX + xr;
            const uint32_t sh = 8u * (uint32_t)(t & 3);
            if (glob) atomicOr(&S.st[t >> 2], kG << sh);
            __threadfence_block();
            const uint32_t old = atomicSub(&S.st[t >> 2], 1u << sh);
            if (((old >> sh) & 0x0Fu) != 1u) break;
            __threadfence_block();
            c = t;
        }
    }
    __syncthreads();

    // inner tile: publish final cells, list global ones
    unsigned long long done = 0;
    for (int i = tid; i < D8X * D8Y; i += NT8) {
        const int ly = i / D8X, lx = i - ly * D8X;
        const int ex = lx + D8H, ey = ly + D8H;
        const int rx = ex + 1, ry = ey + 1;
        const bool valid = rx < gx_hi && ry < gy_hi;
        const int c = ey * EX + ex;
        const uint32_t b = valid ? stget(S.st, c) : 0u;
        const int64_t gi = (oy + ry) * P.nx + (ox + rx);
        const bool glob = valid && (b & kG);
        mark_global(P, G, glob, gi, 0);
        if (!valid || glob || !(b & kDone)) continue;
        ++done;
        if constexpr (W) {
            wr_f(P.out_hi, P, gi, S.vhi[c], 27);
            bool need_lo = P.lo_full;
            if (!need_lo) {
                // pulled later if the receiver leaves the inner tile or is global
                const uint8_t code = S.code[ry * RX8 + rx];
                if (code < 8) {
                    const int lxr = lx + offx(code), lyr = ly + offy(code);
                    need_lo = lxr < 0 || lyr < 0 || lxr >= D8X || lyr >= D8Y ||
                              (stget(S.st, (lyr + D8H) * EX + lxr + D8H) & kG);
                }
            }
            if (need_lo) wr_f(P.out_lo, P, gi, S.vlo[c], 28);
        }
        if constexpr (AREA) wr_area(P, gi, S.area[c]);
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

// fr_receivers.cu -- local flow routing kernels (paper Sec. 2.1 for D8,
// App. A for the multi-receiver split).
//
// Each CTA stages a (TY+4) x (TX+4) elevation tile (two-cell halo) in shared
// memory, computes the routing byte of the tile plus a one-cell ring, and from
// the ring the number of donors of each tile cell.  Outside the grid the tile
// holds +inf, which is never strictly lower than anything.
#include <cmath>

#include "fr_internal.h"
#include "fr_tma.cuh"

namespace fr {

namespace {

constexpr int RTX = kRecvTileX;  // receiver tile width (cells)
constexpr int RTY = kRecvTileY;  // receiver tile height
constexpr int RNT = 256;  // threads
constexpr int HX = RTX + 4, HY = RTY + 4;
constexpr int RX = RTX + 2, RY = RTY + 2;

__device__ __forceinline__ void load_z_tile(float* zs, const float* __restrict__ z, int64_t nx,
                                            int64_t ny, int64_t x0, int64_t y0) {
    const float inf = __int_as_float(0x7f800000);
    for (int i = threadIdx.x; i < HX * HY; i += RNT) {
        int ly = i / HX, lx = i - ly * HX;
        int64_t gx = x0 + lx - 2, gy = y0 + ly - 2;
        float v = inf;
        if (gx >= 0 && gy >= 0 && gx < nx && gy < ny && FR_OK(gy * nx + gx, nx * ny, 40))
            v = __ldg(z + gy * nx + gx);
        zs[i] = v;
    }
}

// Neighbour elevations of ring-tile cell (rx, ry) (ring coordinates: tile
// cell (0,0) is (1,1)).
__device__ __forceinline__ void gather8(const float* zs, int rx, int ry, float (&zn)[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) zn[k] = zs[(ry + 1 + offy(k)) * HX + (rx + 1 + offx(k))];
}

__device__ __forceinline__ void tile_origin(int64_t nx, int64_t& x0, int64_t& y0) {
    const int64_t tiles_x = (nx + RTX - 1) / RTX;
    const int64_t ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    x0 = tx * RTX;
    y0 = ty * RTY;
}

// D8 codes of RTX x RTY tile cells; each thread computes four consecutive
// cells of a row from a 3 x 6 register window.  Tiles away from the grid
// boundary skip all edge and bounds tests.
template <bool INDEG, bool LOWEST>
__device__ __forceinline__ void recv_d8_tile(const float* __restrict__ z, int64_t nx, int64_t ny,
                                             float c_orth, float c_diag, uint32_t flags,
                                             uint8_t* __restrict__ dir,
                                             uint8_t* __restrict__ indeg, int64_t x0,
                                             int64_t y0) {
    __shared__ float zs[HX * HY];
    __shared__ uint8_t ds[RX * RY];
    const bool lowest = LOWEST;
    const bool edge_route = flags & kEdgeRoute;
    const bool d4 = flags & kD4;
    const float inf = __int_as_float(0x7f800000);
    const bool interior = x0 >= 2 && y0 >= 2 && x0 + RTX + 2 <= nx && y0 + RTY + 2 <= ny;
    if (interior) {
        // row by row: a warp per row, lanes along it
        const float* base = z + (y0 - 2) * nx + (x0 - 2);
        const int lane = threadIdx.x & 31;
        for (int ly = threadIdx.x >> 5; ly < HY; ly += RNT / 32) {
            const float* row = base + (int64_t)ly * nx;
#pragma unroll
            for (int lx = lane; lx < HX; lx += 32) zs[ly * HX + lx] = __ldg(row + lx);
        }
    } else {
        load_z_tile(zs, z, nx, ny, x0, y0);
    }
    __syncthreads();
    // four cells per thread: tile row r = (t >> 5) + 8 j, columns 4 (t & 31) .. + 3
    const int qx = (threadIdx.x & 31) * 4;
    for (int r = threadIdx.x >> 5; r < RTY; r += RNT / 32) {
        float w[3][6];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 6; ++b) w[a][b] = zs[(r + 1 + a) * HX + qx + 1 + b];
        uint32_t packed = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint8_t code;
            if (!d4) {  // uniform over the launch: the common path carries no selects
                const float zn[8] = {w[1][q + 2], w[0][q + 1], w[1][q], w[2][q + 1],
                                     w[0][q + 2], w[0][q], w[2][q], w[2][q + 2]};
                code = (uint8_t)d8_code_sel<LOWEST>(w[1][q + 1], zn, c_orth, c_diag);
            } else {
                // D4: the diagonals read +inf, which is never strictly lower
                const float zn[8] = {w[1][q + 2], w[0][q + 1], w[1][q], w[2][q + 1], inf, inf, inf, inf};
                code = (uint8_t)d8_code_sel<LOWEST>(w[1][q + 1], zn, c_orth, c_diag);
            }
            if (!interior) {  // interior tiles hold no edge cell and no cell off the grid
                const int64_t gx = x0 + qx + q, gy = y0 + r;
                if (gx >= nx || gy >= ny || (!edge_route && is_edge(gx, gy, nx, ny))) code = kSink;
            }
            packed |= (uint32_t)code << (8 * q);
            if (INDEG) ds[(r + 1) * RX + qx + q + 1] = code;
        }
        const int64_t gy = y0 + r;
        if (gy < ny) {
            const int64_t gi = gy * nx + x0 + qx;
            if (interior && ((uintptr_t)(dir + gi) & 3) == 0) {
                *reinterpret_cast<uint32_t*>(dir + gi) = packed;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (x0 + qx + q < nx) dir[gi + q] = (uint8_t)(packed >> (8 * q));
            }
        }
    }
    if (INDEG) {
        // the ring around the tile, then the donor counts
        for (int i = threadIdx.x; i < 2 * RX + 2 * RTY; i += RNT) {
            int ry, rx;
            if (i < RX) { ry = 0; rx = i; }
            else if (i < 2 * RX) { ry = RY - 1; rx = i - RX; }
            else if (i < 2 * RX + RTY) { ry = i - 2 * RX + 1; rx = 0; }
            else { ry = i - 2 * RX - RTY + 1; rx = RX - 1; }
            const int64_t gx = x0 + rx - 1, gy = y0 + ry - 1;
            uint8_t code = kSink;
            if (gx >= 0 && gy >= 0 && gx < nx && gy < ny &&
                (edge_route || !is_edge(gx, gy, nx, ny))) {
                float zn[8];
                gather8(zs, rx, ry, zn);
                if (d4) zn[4] = zn[5] = zn[6] = zn[7] = inf;
                code = d8_code(zs[(ry + 1) * HX + (rx + 1)], zn, c_orth, c_diag, lowest);
            }
            ds[ry * RX + rx] = code;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < RTX * RTY; i += RNT) {
            const int ly = i / RTX, lx = i - ly * RTX;
            const int64_t gx = x0 + lx, gy = y0 + ly;
            if (gx >= nx || gy >= ny) continue;
            int n = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                n += ds[(ly + 1 + offy(k)) * RX + (lx + 1 + offx(k))] == (uint8_t)opp(k);
            indeg[gy * nx + gx] = (uint8_t)n;
        }
    }
}

template <bool INDEG, bool LOWEST>
__global__ void __launch_bounds__(RNT) k_receivers_d8(const float* __restrict__ z, int64_t nx,
                                                      int64_t ny, float c_orth, float c_diag,
                                                      uint32_t flags, uint8_t* __restrict__ dir,
                                                      uint8_t* __restrict__ indeg) {
    int64_t x0, y0;
    tile_origin(nx, x0, y0);
    recv_d8_tile<INDEG, LOWEST>(z, nx, ny, c_orth, c_diag, flags, dir, indeg, x0, y0);
}

// ---------------------------------------------------------------- TMA path
// D8 codes without donor counts, by a persistent kernel: each CTA walks its
// tiles of TTX x TTY cells, the elevations of a tile plus a one-cell halo
// arriving by TMA into one of TNS shared-memory stages while the previous tiles
// are computed.  The box starts 4 cells left of the tile (its x coordinate a
// multiple of 4, as TMA requires), so it is TTX + 8 wide.  The kernel is bound
// by the ALU pipe (the compare-and-select chain of eight directions per cell);
// 128x64 tiles in two stages (three CTAs per SM) measured 4.7 % faster than
// 128x32 in three (four CTAs per SM) at 32768^2: fewer halo rows and fewer
// per-tile waits and barriers.
constexpr int TTX = 128, TTY = 64, TNS = 2;
constexpr int TBX = TTX + 8, TBY = TTY + 2;
constexpr unsigned kTileBytes = TBX * TBY * 4;
static_assert((TBX * 4) % 16 == 0, "TMA box rows are whole 16-byte units");

// Set when a TMA wait ran out (read and cleared by fr_get_status).
__device__ unsigned g_tma_wait_error;

struct alignas(128) TmaStage {  // TMA writes whole boxes to 128-byte aligned addresses
    float v[TBY * TBX];
};
struct TmaSmem {
    TmaStage buf[TNS];
    alignas(8) uint64_t bar[TNS];
};

template <bool LOWEST, bool D4>
__global__ void __launch_bounds__(256) k_receivers_d8_tma(const __grid_constant__ CUtensorMap zmap,
                                                          int64_t nx, int64_t ny, float c_orth,
                                                          float c_diag, uint32_t flags,
                                                          uint8_t* __restrict__ dir, int64_t ntiles,
                                                          int tiles_x, unsigned long long limit_ns) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TmaSmem& S = *reinterpret_cast<TmaSmem*>(smem_raw);
    const bool edge_route = flags & kEdgeRoute;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < TNS; ++s) mbar_init(&S.bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int64_t t, int s) {
        const int64_t ty = t / tiles_x, tx = t - ty * tiles_x;
        mbar_expect_tx(&S.bar[s], kTileBytes);
        tma_load_2d(S.buf[s].v, &zmap, (int)(tx * TTX - 4), (int)(ty * TTY - 1), &S.bar[s]);
    };
    if (tid == 0)
        for (int s = 0; s < TNS; ++s) {
            const int64_t t = (int64_t)blockIdx.x + (int64_t)s * gridDim.x;
            if (t < ntiles) issue(t, s);
        }
    const int lane = tid & 31, warp = tid >> 5, qx = 4 * lane;
    int i = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const int s = i % TNS;
        const bool ok = mbar_wait(&S.bar[s], (unsigned)(i / TNS) & 1u, limit_ns);
        if (__syncthreads_or(!ok)) {
            // the copy did not arrive: report, let the other copies in flight
            // land (bounded), and leave (the whole block takes this branch)
            if (tid == 0) {
                atomicOr(&g_tma_wait_error, 1u);
                for (int k = 1; k < TNS; ++k) {
                    const int64_t tk = t + (int64_t)k * gridDim.x;
                    if (tk < ntiles) mbar_wait(&S.bar[(i + k) % TNS], (unsigned)((i + k) / TNS) & 1u, limit_ns);
                }
            }
            __syncthreads();
            return;
        }
        const int64_t ty = t / tiles_x, tx = t - ty * tiles_x;
        const int64_t x0 = tx * TTX, y0 = ty * TTY;
        const bool interior = x0 >= 1 && y0 >= 1 && x0 + TTX + 1 <= nx && y0 + TTY + 1 <= ny;
        const float* b = S.buf[s].v;
        for (int r = warp; r < TTY; r += 8) {
            // 3 x 12 window: buffer rows r .. r + 2, columns qx .. qx + 11
            // (tile column c sits at buffer column c + 4)
            float w[3][12];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const float4 f = *reinterpret_cast<const float4*>(b + (r + a) * TBX + qx + 4 * v);
                    w[a][4 * v] = f.x;
                    w[a][4 * v + 1] = f.y;
                    w[a][4 * v + 2] = f.z;
                    w[a][4 * v + 3] = f.w;
                }
            uint32_t packed = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = q + 4;  // window column of the cell
                float zn[8];
                zn[0] = w[1][c + 1];
                zn[1] = w[0][c];
                zn[2] = w[1][c - 1];
                zn[3] = w[2][c];
                if (D4) {
                    zn[4] = zn[5] = zn[6] = zn[7] = __int_as_float(0x7f800000);
                } else {
                    zn[4] = w[0][c + 1];
                    zn[5] = w[0][c - 1];
                    zn[6] = w[2][c - 1];
                    zn[7] = w[2][c + 1];
                }
                uint32_t code = d8_code_sel<LOWEST>(w[1][c], zn, c_orth, c_diag);
                if (!interior) {
                    const int64_t gx = x0 + qx + q, gy = y0 + r;
                    if (gx >= nx || gy >= ny || (!edge_route && is_edge(gx, gy, nx, ny))) code = kSink;
                }
                packed |= code << (8 * q);
            }
            const int64_t gy = y0 + r;
            const int64_t gx = x0 + qx;
            if (gy < ny && gx < nx) {
                const int64_t gi = gy * nx + gx;
                if (gx + 3 < nx && ((uintptr_t)(dir + gi) & 3) == 0) {
                    *reinterpret_cast<uint32_t*>(dir + gi) = packed;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (gx + q < nx) dir[gi + q] = (uint8_t)(packed >> (8 * q));
                }
            }
        }
        __syncthreads();  // every thread is done with stage s
        if (tid == 0) {
            const int64_t tn = t + (int64_t)TNS * gridDim.x;
            if (tn < ntiles) {
                fence_proxy_async_smem();
                issue(tn, s);
            }
        }
    }
}

template <bool FRAC, bool INDEG>
__device__ __forceinline__ void recv_mfd_tile(const float* __restrict__ z, int64_t nx, int64_t ny,
                                              const MfdConst& mc, uint32_t flags,
                                              uint8_t* __restrict__ mask, float* __restrict__ frac,
                                              uint8_t* __restrict__ indeg, int64_t x0, int64_t y0) {
    __shared__ float zs[HX * HY];
    __shared__ uint8_t ms[RX * RY];
    load_z_tile(zs, z, nx, ny, x0, y0);
    __syncthreads();
    const bool edge_route = flags & kEdgeRoute;
    const int rx0 = INDEG ? 0 : 1, ry0 = INDEG ? 0 : 1;
    const int rw = INDEG ? RX : RTX, rh = INDEG ? RY : RTY;
    for (int i = threadIdx.x; i < rw * rh; i += RNT) {
        int ry = ry0 + i / rw, rx = rx0 + i % rw;
        int64_t gx = x0 + rx - 1, gy = y0 + ry - 1;
        uint8_t m = 0;
        if (gx >= 0 && gy >= 0 && gx < nx && gy < ny &&
            (edge_route || !is_edge(gx, gy, nx, ny))) {
            float zc = zs[(ry + 1) * HX + (rx + 1)];
            if (flags & kDinf) {
                float zn[8], f[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) zn[k] = zs[(ry + 1 + offy(k)) * HX + (rx + 1 + offx(k))];
                m = (uint8_t)dinf_cell(zc, zn, grid_mask8(gx, gy, nx, ny), mc.co_hi, mc.cd_hi, f);
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (zs[(ry + 1 + offy(k)) * HX + (rx + 1 + offx(k))] < zc) m |= (uint8_t)(1u << k);
            }
        }
        ms[ry * RX + rx] = m;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RTX * RTY; i += RNT) {
        int ly = i / RTX, lx = i - ly * RTX;
        int64_t gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        int64_t gi = gy * nx + gx;
        if (!FR_OK(gi, nx * ny, 42)) continue;
        uint8_t m = ms[(ly + 1) * RX + lx + 1];
        mask[gi] = m;
        if (FRAC) {
            float zn[8], f[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) zn[k] = zs[(ly + 2 + offy(k)) * HX + (lx + 2 + offx(k))];
            if (flags & kDinf) {
                if (m) dinf_cell(zs[(ly + 2) * HX + (lx + 2)], zn, grid_mask8(gx, gy, nx, ny), mc.co_hi,
                                 mc.cd_hi, f);
                else
#pragma unroll
                    for (int k = 0; k < 8; ++k) f[k] = 0.0f;
            } else {
                mfd_fracs8(zs[(ly + 2) * HX + (lx + 2)], zn, m, mc, f);
            }
            float4* fo = reinterpret_cast<float4*>(frac + gi * 8);
            fo[0] = make_float4(f[0], f[1], f[2], f[3]);
            fo[1] = make_float4(f[4], f[5], f[6], f[7]);
        }
        if (INDEG) {
            int n = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                n += (ms[(ly + 1 + offy(k)) * RX + (lx + 1 + offx(k))] >> opp(k)) & 1;
            indeg[gi] = (uint8_t)n;
        }
    }
}

template <bool FRAC, bool INDEG>
__global__ void __launch_bounds__(RNT) k_receivers_mfd(const float* __restrict__ z, int64_t nx,
                                                       int64_t ny, MfdConst mc, uint32_t flags,
                                                       uint8_t* __restrict__ mask,
                                                       float* __restrict__ frac,
                                                       uint8_t* __restrict__ indeg) {
    int64_t x0, y0;
    tile_origin(nx, x0, y0);
    recv_mfd_tile<FRAC, INDEG>(z, nx, ny, mc, flags, mask, frac, indeg, x0, y0);
}

// Fractions of given receiver masks (bits pointing off the grid are
// ignored): one cell per thread, elevations staged like the receiver tiles.
__global__ void __launch_bounds__(RNT) k_mfd_fractions(const float* __restrict__ z,
                                                       const uint8_t* __restrict__ mask,
                                                       int64_t nx, int64_t ny, MfdConst mc,
                                                       uint32_t flags, float* __restrict__ frac) {
    __shared__ float zs[HX * HY];
    int64_t x0, y0;
    tile_origin(nx, x0, y0);
    load_z_tile(zs, z, nx, ny, x0, y0);
    __syncthreads();
    for (int i = threadIdx.x; i < RTX * RTY; i += RNT) {
        const int ly = i / RTX, lx = i - ly * RTX;
        const int64_t gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const int64_t gi = gy * nx + gx;
        if (!FR_OK(gi, nx * ny, 43)) continue;
        const uint32_t m = mask[gi] & grid_mask8(gx, gy, nx, ny);
        float zn[8], f[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) zn[k] = zs[(ly + 2 + offy(k)) * HX + (lx + 2 + offx(k))];
        if (flags & kDinf) {
            // the D-infinity split of this cell (its receivers are the mask's)
            if (m) dinf_cell(zs[(ly + 2) * HX + (lx + 2)], zn, grid_mask8(gx, gy, nx, ny), mc.co_hi,
                             mc.cd_hi, f);
            else
#pragma unroll
                for (int k = 0; k < 8; ++k) f[k] = 0.0f;
        } else {
            mfd_fracs8(zs[(ly + 2) * HX + (lx + 2)], zn, m, mc, f);
        }
        float4* fo = reinterpret_cast<float4*>(frac + gi * 8);
        fo[0] = make_float4(f[0], f[1], f[2], f[3]);
        fo[1] = make_float4(f[4], f[5], f[6], f[7]);
    }
}

// Batched receivers: persistent CTAs claim receiver tiles of any problem.
// prefix[p] is the first receiver tile of problem p (prefix[nprob] = total).
__global__ void __launch_bounds__(RNT) k_receivers_batch(int kind, const Prob* __restrict__ probs,
                                                         const int64_t* __restrict__ prefix,
                                                         int nprob, uint32_t flags,
                                                         EngineGlobals* G) {
    __shared__ int64_t s_work;
    const int64_t total = prefix[nprob];
    while (true) {
        if (threadIdx.x == 0) s_work = (int64_t)atomicAdd(&G->recv_next, 1ull);
        __syncthreads();
        const int64_t w = s_work;
        __syncthreads();
        if (w >= total) break;
        int lo = 0, hi = nprob - 1;  // last p with prefix[p] <= w
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const Prob& P = probs[lo];
        const int64_t lt = w - prefix[lo];
        const int64_t tiles_x = (P.nx + RTX - 1) / RTX;
        const int64_t ty = lt / tiles_x, tx = lt - ty * tiles_x;
        if (kind == 0 && (flags & kD8Lowest))
            recv_d8_tile<false, true>(P.z, P.nx, P.ny, P.mc.co_hi, P.mc.cd_hi, flags,
                                      const_cast<uint8_t*>(P.rb), nullptr, tx * RTX, ty * RTY);
        else if (kind == 0)
            recv_d8_tile<false, false>(P.z, P.nx, P.ny, P.mc.co_hi, P.mc.cd_hi, flags,
                                       const_cast<uint8_t*>(P.rb), nullptr, tx * RTX, ty * RTY);
        else
            recv_mfd_tile<true, false>(P.z, P.nx, P.ny, P.mc, flags, const_cast<uint8_t*>(P.rb),
                                       const_cast<float*>(P.frac), nullptr, tx * RTX, ty * RTY);
        __syncthreads();
    }
}

__global__ void k_count_nonfinite(const float* __restrict__ z, int64_t n,
                                  unsigned long long* count) {
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        local += !isfinite(z[i]);
    for (int o = 16; o; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// Linear index of each cell's receiver (-1 for sinks and for codes that
// point out of the grid), four cells per thread step.
template <class I>
__global__ void __launch_bounds__(256) k_receiver_index(const uint8_t* __restrict__ dir, int64_t nx,
                                                        int64_t n, I* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t k = __ldg(dir + i);
        I r = (I)-1;
        if (k < 8) {
            const int64_t y = i / nx, x = i - y * nx;
            const int64_t xr = x + offx((int)k), yr = y + offy((int)k);
            if (xr >= 0 && yr >= 0 && xr < nx && yr * nx + xr < n) r = (I)(yr * nx + xr);
        }
        out[i] = r;
    }
}

template <bool LOWEST, bool D4>
cudaError_t launch_d8_tma(const CUtensorMap& map, int64_t nx, int64_t ny, float co, float cd,
                          uint32_t flags, uint8_t* dir, cudaStream_t s) {
    constexpr size_t sm = sizeof(TmaSmem);
    static std::atomic<unsigned long long> set_on{0};
    static int grid_per_sm = 0, sms = 0;
    cudaError_t e = smem_limit_once(k_receivers_d8_tma<LOWEST, D4>, sm, set_on);
    if (e != cudaSuccess) return e;
    if (!grid_per_sm) {
        int dev = 0, per = 0, n = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_receivers_d8_tma<LOWEST, D4>, 256, sm)) !=
            cudaSuccess)
            return e;
        sms = n;
        grid_per_sm = per > 0 ? per : 1;
    }
    const int tiles_x = (int)((nx + TTX - 1) / TTX);
    const int64_t ntiles = (int64_t)tiles_x * ((ny + TTY - 1) / TTY);
    int64_t grid = (int64_t)sms * grid_per_sm;
    if (grid > ntiles) grid = ntiles;
    k_receivers_d8_tma<LOWEST, D4><<<(unsigned)grid, 256, sm, s>>>(map, nx, ny, co, cd, flags, dir, ntiles,
                                                                   tiles_x, wait_limit_ns());
    return cudaGetLastError();
}

}  // namespace

bool encode_tile_map_f32(CUtensorMap* map, const float* base, int64_t nx, int64_t ny, int box_x,
                         int box_y) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    // cuTensorMapEncodeTiled from the CUDA driver API, looked up once (thread-safe static
    // initialisation)
    static const Encode fn = []() -> Encode {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<Encode>(p);
        return nullptr;
    }();
    if (!fn || (nx & 3) || ((uintptr_t)base & 15) || nx > (int64_t)1 << 31 || ny > (int64_t)1 << 31) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)nx * 4};
    const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA) == CUDA_SUCCESS;
}

cudaError_t read_clear_tma_error(unsigned* out, cudaStream_t s) {
    unsigned zero = 0;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_tma_wait_error);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(out, p, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (*out == 0) return cudaSuccess;
    if ((e = cudaMemcpyAsync(p, &zero, sizeof(unsigned), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t launch_receiver_index(const uint8_t* dir, int64_t nx, int64_t ny, bool wide, void* out,
                                  cudaStream_t s) {
    const int64_t n = nx * ny;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (wide)
        k_receiver_index<int64_t><<<(unsigned)blocks, 256, 0, s>>>(dir, nx, n, (int64_t*)out);
    else
        k_receiver_index<int32_t><<<(unsigned)blocks, 256, 0, s>>>(dir, nx, n, (int32_t*)out);
    return cudaGetLastError();
}

cudaError_t launch_receivers_d8(const float* z, int64_t nx, int64_t ny, double dx,
                                uint32_t flags, uint8_t* dir, uint8_t* indeg, cudaStream_t s) {
    const unsigned grid = (unsigned)(((nx + RTX - 1) / RTX) * ((ny + RTY - 1) / RTY));
    float co = (float)(1.0 / dx);
    float cd = (float)(1.0 / (std::sqrt(2.0) * dx));
    const bool lowest = flags & kD8Lowest;
    // codes alone on a TMA-addressable grid: the pipelined persistent kernel
    CUtensorMap map;
    if (!indeg && nx * ny >= (int64_t)TTX * TTY && encode_tile_map_f32(&map, z, nx, ny, TBX, TBY)) {
        const bool d4 = flags & kD4;
        if (lowest) return d4 ? launch_d8_tma<true, true>(map, nx, ny, co, cd, flags, dir, s)
                              : launch_d8_tma<true, false>(map, nx, ny, co, cd, flags, dir, s);
        return d4 ? launch_d8_tma<false, true>(map, nx, ny, co, cd, flags, dir, s)
                  : launch_d8_tma<false, false>(map, nx, ny, co, cd, flags, dir, s);
    }
    if (indeg && lowest)
        k_receivers_d8<true, true><<<grid, RNT, 0, s>>>(z, nx, ny, co, cd, flags, dir, indeg);
    else if (indeg)
        k_receivers_d8<true, false><<<grid, RNT, 0, s>>>(z, nx, ny, co, cd, flags, dir, indeg);
    else if (lowest)
        k_receivers_d8<false, true><<<grid, RNT, 0, s>>>(z, nx, ny, co, cd, flags, dir, nullptr);
    else
        k_receivers_d8<false, false><<<grid, RNT, 0, s>>>(z, nx, ny, co, cd, flags, dir, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_receivers_mfd(const float* z, int64_t nx, int64_t ny, double dx, double p,
                                 uint32_t flags, uint8_t* mask, float* frac, uint8_t* indeg,
                                 cudaStream_t s) {
    const unsigned grid = (unsigned)(((nx + RTX - 1) / RTX) * ((ny + RTY - 1) / RTY));
    MfdConst mc = make_mfd_const(dx, p);
    if (frac && indeg)
        k_receivers_mfd<true, true><<<grid, RNT, 0, s>>>(z, nx, ny, mc, flags, mask, frac, indeg);
    else if (frac)
        k_receivers_mfd<true, false><<<grid, RNT, 0, s>>>(z, nx, ny, mc, flags, mask, frac, nullptr);
    else if (indeg)
        k_receivers_mfd<false, true><<<grid, RNT, 0, s>>>(z, nx, ny, mc, flags, mask, nullptr, indeg);
    else
        k_receivers_mfd<false, false><<<grid, RNT, 0, s>>>(z, nx, ny, mc, flags, mask, nullptr,
                                                           nullptr);
    return cudaGetLastError();
}

cudaError_t launch_mfd_fractions(const float* z, const uint8_t* mask, int64_t nx, int64_t ny,
                                 double dx, double p, uint32_t flags, float* frac, cudaStream_t s) {
    const unsigned grid = (unsigned)(((nx + RTX - 1) / RTX) * ((ny + RTY - 1) / RTY));
    k_mfd_fractions<<<grid, RNT, 0, s>>>(z, mask, nx, ny, make_mfd_const(dx, p), flags, frac);
    return cudaGetLastError();
}

cudaError_t launch_receivers_batch(int kind, const Prob* probs, const int64_t* prefix, int nprob,
                                   uint32_t flags, EngineGlobals* G, int grid, cudaStream_t s) {
    k_receivers_batch<<<grid, RNT, 0, s>>>(kind, probs, prefix, nprob, flags, G);
    return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(const float* z, int64_t n, unsigned long long* count,
                                   cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_count_nonfinite<<<(unsigned)blocks, 256, 0, s>>>(z, n, count);
    return cudaGetLastError();
}

}  // namespace fr

#ifdef FR_DEBUG_BOUNDS
// Debug builds only: first out-of-range access seen by the receiver kernels.
extern "C" unsigned long long fr_debug_bad_receivers(void) {
    unsigned long long v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, fr::fr_debug_bad, sizeof(v));
    cudaMemcpyToSymbol(fr::fr_debug_bad, &z, sizeof(z));
    return v;
}
#endif

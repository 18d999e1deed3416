// fr_fill.cu -- depression filling, the step before the path: the paper routes
// a depression-filled DEM (Sec. 4).  The filled surface F is the least F >= z
// that keeps every edge cell at its own elevation and gives every interior
// cell a neighbour (of 8) lower by at least one fp32 step, i.e. the solution of
//     F_c = z_c                                             (edge cells)
//     F_c = max(z_c, succ(min over neighbours n of F_n))    (elsewhere),
// succ(x) being the next fp32 value above x.  D8 routing on F has sinks only
// on the edge.
//
// GPU form (Planchon-Darboux relaxation): F starts at z on the edge and +inf
// inside; every update lowers a cell to the right-hand side above, which is
// never below the solution, so the updates can run in any order and the
// iteration ends exactly at the solution.  A sweep is one launch: each CTA
// loads a 64x32 tile of F with a one-cell ring into shared memory and relaxes
// it in place until nothing moves (block barrier per pass), then writes the
// tile back.  Rings read values of neighbouring tiles that may be older or
// newer within the sweep; both are upper bounds, so the result is the same.
// The host repeats sweeps until one changes nothing: then every cell meets
// its equation, and the surface is the unique solution, bit for bit.
//
// A tile whose 3x3 neighbourhood of tiles changed nothing in the previous
// sweep is skipped (its cells and its ring are as they were when it last
// settled); each CTA records whether its tile changed, for the next sweep.
#include "fr_internal.h"

namespace fr {
namespace {

constexpr int kFTX = 64, kFTY = 32, kFNT = 256;
constexpr int kFRX = kFTX + 2, kFRY = kFTY + 2;
constexpr int kFLocalCap = 4 * (kFTX + kFTY);  // relaxation passes per tile and sweep

// The next fp32 value above x, from the ordering of IEEE-754 bit patterns:
// one more in the magnitude for x > 0, one less for x < 0, the smallest
// positive subnormal for either zero; +inf stays +inf.
__device__ __forceinline__ float fsucc(float x) {
    const int b = __float_as_int(x);
    if (b == 0x7f800000) return x;
    if ((b & 0x7fffffff) == 0) return __int_as_float(1);
    return __int_as_float(b > 0 ? b + 1 : b - 1);
}

__global__ void __launch_bounds__(kFNT) k_fill_init(const float* __restrict__ z, int64_t nx,
                                                    int64_t ny, float* __restrict__ F) {
    const float inf = __int_as_float(0x7f800000);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nx * ny;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = i / nx, x = i - y * nx;
        const bool edge = x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
        F[i] = edge ? z[i] : inf;
    }
}

__global__ void __launch_bounds__(kFNT) k_fill_sweep(const float* __restrict__ z, int64_t nx,
                                                     int64_t ny, float* F,
                                                     const uint8_t* __restrict__ act_prev,
                                                     uint8_t* __restrict__ act_next, int first,
                                                     unsigned long long* changed) {
    __shared__ float fs[kFRY * kFRX];
    __shared__ float zs[kFTY * kFTX];
    const float inf = __int_as_float(0x7f800000);
    const int tiles_x = (int)((nx + kFTX - 1) / kFTX);
    const int tiles_y = (int)((ny + kFTY - 1) / kFTY);
    const int ty = (int)blockIdx.x / tiles_x, tx = (int)blockIdx.x - ty * tiles_x;
    const int64_t x0 = (int64_t)tx * kFTX, y0 = (int64_t)ty * kFTY;
    if (!first) {
        // run only if this tile or one of its 8 neighbour tiles changed last sweep
        bool active = false;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int ux = tx + dx, uy = ty + dy;
                if (ux >= 0 && uy >= 0 && ux < tiles_x && uy < tiles_y && act_prev[uy * tiles_x + ux])
                    active = true;
            }
        if (!active) {
            if (threadIdx.x == 0) act_next[blockIdx.x] = 0;
            return;
        }
    }
    for (int i = threadIdx.x; i < kFRY * kFRX; i += kFNT) {
        const int ry = i / kFRX, rx = i - ry * kFRX;
        const int64_t gx = x0 + rx - 1, gy = y0 + ry - 1;
        // other CTAs write their tiles meanwhile: read through L2, any value seen
        // is an upper bound of the solution
        fs[i] = (gx >= 0 && gy >= 0 && gx < nx && gy < ny) ? __ldcg(F + gy * nx + gx) : inf;
    }
    for (int i = threadIdx.x; i < kFTY * kFTX; i += kFNT) {
        const int ly = i / kFTX, lx = i - ly * kFTX;
        const int64_t gx = x0 + lx, gy = y0 + ly;
        zs[i] = (gx < nx && gy < ny) ? __ldg(z + gy * nx + gx) : inf;
    }
    __syncthreads();
    bool any = false;
    for (int pass = 0; pass < kFLocalCap; ++pass) {
        bool moved = false;
        for (int i = threadIdx.x; i < kFTY * kFTX; i += kFNT) {
            const int ly = i / kFTX, lx = i - ly * kFTX;
            const int64_t gx = x0 + lx, gy = y0 + ly;
            if (gx >= nx - 1 || gy >= ny - 1 || gx == 0 || gy == 0) continue;  // edge or off the grid
            const int r = (ly + 1) * kFRX + lx + 1;
            float m = fs[r + 1];
            m = fminf(m, fs[r - 1]);
            m = fminf(m, fs[r - kFRX]);
            m = fminf(m, fs[r + kFRX]);
            m = fminf(m, fs[r - kFRX - 1]);
            m = fminf(m, fs[r - kFRX + 1]);
            m = fminf(m, fs[r + kFRX - 1]);
            m = fminf(m, fs[r + kFRX + 1]);
            const float s = fsucc(m), zc = zs[i];
            const float v = zc > s ? zc : s;
            if (v < fs[r]) {
                fs[r] = v;
                moved = true;
            }
        }
        if (!__syncthreads_or(moved)) break;
        any = true;
    }
    if (threadIdx.x == 0) act_next[blockIdx.x] = any ? 1 : 0;
    if (!any) return;
    for (int i = threadIdx.x; i < kFTY * kFTX; i += kFNT) {
        const int ly = i / kFTX, lx = i - ly * kFTX;
        const int64_t gx = x0 + lx, gy = y0 + ly;
        if (gx < nx && gy < ny) F[gy * nx + gx] = fs[(ly + 1) * kFRX + lx + 1];
    }
    if (threadIdx.x == 0) atomicAdd(changed, 1ull);
}

}  // namespace

cudaError_t fill_init(const float* z, int64_t nx, int64_t ny, float* F, cudaStream_t s) {
    int64_t blocks = (nx * ny + kFNT - 1) / kFNT;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_fill_init<<<(unsigned)blocks, kFNT, 0, s>>>(z, nx, ny, F);
    return cudaGetLastError();
}

int64_t fill_tiles(int64_t nx, int64_t ny) {
    return ((nx + kFTX - 1) / kFTX) * ((ny + kFTY - 1) / kFTY);
}

cudaError_t fill_sweep(const float* z, int64_t nx, int64_t ny, float* F, const uint8_t* act_prev,
                       uint8_t* act_next, bool first, unsigned long long* changed, cudaStream_t s) {
    k_fill_sweep<<<(unsigned)fill_tiles(nx, ny), kFNT, 0, s>>>(z, nx, ny, F, act_prev, act_next,
                                                              first ? 1 : 0, changed);
    return cudaGetLastError();
}

}  // namespace fr

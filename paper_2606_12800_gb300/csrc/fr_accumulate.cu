// fr_accumulate.cu -- the D8 walker grid, the mass-balance reduction and the
// MFD elevation-gradient stencil.
#include "fr_engine.cuh"

namespace fr {
namespace {

// ---------------------------------------------------------------- mass balance
constexpr int MB_NT = 256;

// Bit i set where byte i of the 16 routing bytes in v marks a sink (D8 code
// 0xFF, MFD empty mask).
template <bool MFD>
__device__ __forceinline__ uint32_t sink_bits16(const uint4 v) {
    const uint32_t words[4] = {v.x, v.y, v.z, v.w};
    uint32_t bits = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t zb = zero_bytes(MFD ? words[q] : ~words[q]);  // 0x80 per sink byte
        zb >>= 7;                                               // bit 0 of each byte
        bits |= ((zb & 1u) | ((zb >> 7) & 2u) | ((zb >> 14) & 4u) | ((zb >> 21) & 8u)) << (4 * q);
    }
    return bits;
}

// Partial sums of one block: rain (two-float), water at sinks (two-float) and
// area at sinks (exact).  Each thread takes chunks of 16 cells (16-byte routing
// load, four 16-byte rain loads; the rain of a chunk is summed pairwise) and
// then gathers only the chunk's sinks.  Grid-stride over chunks in a fixed
// order, so the result does not depend on scheduling.
template <bool MFD>
__global__ void __launch_bounds__(MB_NT) k_mass_partial(int64_t n, const uint8_t* __restrict__ rb,
                                                        const float* __restrict__ rain,
                                                        const float* __restrict__ w,
                                                        const float* __restrict__ w_lo,
                                                        const uint64_t* __restrict__ area,
                                                        double* __restrict__ partials) {
    df sw = df_make(0.0f), sr = df_make(0.0f);
    unsigned long long sa = 0;
    const int64_t stride = (int64_t)gridDim.x * MB_NT;
    const int64_t first = (int64_t)blockIdx.x * MB_NT + threadIdx.x;
    const bool vec = ((uintptr_t)rb & 15) == 0 && (!rain || ((uintptr_t)rain & 15) == 0);
    const int64_t nchunk = vec ? n / 16 : 0;
    auto sink_add = [&](int64_t i) {
        if (w) sw = df_add(sw, df{__ldg(w + i), w_lo ? __ldg(w_lo + i) : 0.0f});
        if (area) sa += __ldg(area + i);
    };
    for (int64_t c = first; c < nchunk; c += stride) {
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(rb) + c);
        if (rain) {
            const float4* r4 = reinterpret_cast<const float4*>(rain) + 4 * c;
            const float4 a0 = __ldg(r4), a1 = __ldg(r4 + 1), a2 = __ldg(r4 + 2), a3 = __ldg(r4 + 3);
            const df p0 = df_add(df_add(df_make(a0.x), df_make(a0.y)), df_add(df_make(a0.z), df_make(a0.w)));
            const df p1 = df_add(df_add(df_make(a1.x), df_make(a1.y)), df_add(df_make(a1.z), df_make(a1.w)));
            const df p2 = df_add(df_add(df_make(a2.x), df_make(a2.y)), df_add(df_make(a2.z), df_make(a2.w)));
            const df p3 = df_add(df_add(df_make(a3.x), df_make(a3.y)), df_add(df_make(a3.z), df_make(a3.w)));
            sr = df_add(sr, df_add(df_add(p0, p1), df_add(p2, p3)));
        } else {
            sr = df_add(sr, df_make(16.0f));
        }
        for (uint32_t m = sink_bits16<MFD>(b); m; m &= m - 1) sink_add(16 * c + (__ffs(m) - 1));
    }
    // cells after the last whole chunk (or all cells without the vector path)
    for (int64_t i = 16 * nchunk + first; i < n; i += stride) {
        const uint8_t bb = rb[i];
        sr = df_add(sr, df_make(rain ? rain[i] : 1.0f));
        if (MFD ? (bb == 0) : (bb == kSink)) sink_add(i);
    }
    double v0 = (double)sw.hi + (double)sw.lo, v1 = (double)sr.hi + (double)sr.lo;
    for (int o = 16; o; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
        sa += __shfl_down_sync(0xffffffffu, sa, o);
    }
    __shared__ double s0[MB_NT / 32], s1[MB_NT / 32];
    __shared__ unsigned long long s2[MB_NT / 32];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s0[warp] = v0;
        s1[warp] = v1;
        s2[warp] = sa;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        unsigned long long c = 0;
        for (int i = 0; i < MB_NT / 32; ++i) {
            a += s0[i];
            b += s1[i];
            c += s2[i];
        }
        partials[3 * blockIdx.x + 0] = a;
        partials[3 * blockIdx.x + 1] = b;
        reinterpret_cast<unsigned long long*>(partials)[3 * blockIdx.x + 2] = c;
    }
}

// Area term of the D8 mass balance from the sums an accumulation left in the
// workspace: the local phase's sum over the FR_SINK cells it finished plus,
// gathered here, the areas of the FR_SINK cells among the global cells (set
// bits of the global-cell bitmap).  Each cell is finished by exactly one of
// the two phases, so the total equals the sum over all FR_SINK cells.  Block b
// writes the area term of partials[3 b + 2]; with `unit` (no rain field) it
// also writes the other two terms (0, and the cell count in block 0), which
// k_mass_partial has written otherwise.
__global__ void __launch_bounds__(MB_NT) k_mass_sinks_ws(int64_t n, const uint8_t* __restrict__ rb,
                                                         const uint64_t* __restrict__ area,
                                                         const uint32_t* __restrict__ gbits,
                                                         const EngineGlobals* __restrict__ G,
                                                         bool unit, double* __restrict__ partials) {
    unsigned long long sa = 0;
    auto take = [&](int64_t wd, uint32_t m) {  // the set bits of bitmap word wd
        for (; m; m &= m - 1) {
            const int64_t i = 32 * wd + (__ffs(m) - 1);
            if (i < n && __ldg(rb + i) == kSink) sa += __ldg(area + i);
        }
    };
    // the bitmap in 16-byte groups of four words, four groups in flight per
    // thread (the bitmap is 256-byte aligned in the workspace)
    const int64_t words = (n + 31) / 32, quads = words / 4;
    const int64_t stride = (int64_t)gridDim.x * MB_NT, first = (int64_t)blockIdx.x * MB_NT + threadIdx.x;
    const uint4* g4 = reinterpret_cast<const uint4*>(gbits);
    for (int64_t q0 = first; q0 < quads; q0 += 4 * stride) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v[u] = q0 + u * stride < quads ? __ldg(g4 + q0 + u * stride) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!(v[u].x | v[u].y | v[u].z | v[u].w)) continue;
            const int64_t wd = 4 * (q0 + u * stride);
            take(wd, v[u].x);
            take(wd + 1, v[u].y);
            take(wd + 2, v[u].z);
            take(wd + 3, v[u].w);
        }
    }
    for (int64_t wd = 4 * quads + first; wd < words; wd += stride) take(wd, __ldg(gbits + wd));
    for (int o = 16; o; o >>= 1) sa += __shfl_down_sync(0xffffffffu, sa, o);
    __shared__ unsigned long long s2[MB_NT / 32];
    if ((threadIdx.x & 31) == 0) s2[threadIdx.x >> 5] = sa;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long c = blockIdx.x == 0 ? G->sink_area : 0ull;
        for (int i = 0; i < MB_NT / 32; ++i) c += s2[i];
        reinterpret_cast<unsigned long long*>(partials)[3 * blockIdx.x + 2] = c;
        if (unit) {
            partials[3 * blockIdx.x + 0] = 0.0;
            partials[3 * blockIdx.x + 1] = blockIdx.x == 0 ? (double)n : 0.0;
        }
    }
}

__global__ void k_mass_final(const double* __restrict__ partials, int nblocks, double* out) {
    __shared__ double s0[256], s1[256];
    __shared__ unsigned long long s2[256];
    double a = 0.0, b = 0.0;
    unsigned long long c = 0;
    for (int i = threadIdx.x; i < nblocks; i += 256) {
        a += partials[3 * i];
        b += partials[3 * i + 1];
        c += reinterpret_cast<const unsigned long long*>(partials)[3 * i + 2];
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    s2[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) {
            s0[threadIdx.x] += s0[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s0[0];
        out[1] = s1[0];
        out[2] = (double)s2[0];
    }
}

// ------------------------------------------------------ MFD elevation gradient
// dL/dz = g^T (dW/dz) w with the lower sets held fixed.  For a source cell c
// with lower neighbours j: u_j = s_j^p with s_j = (z_c - z_j) / d_j, S = sum
// u_j, f_j = u_j / S and G = sum f_j g_j.  Then du_j/dz_c = p u_j / (s_j d_j)
// = p u_j / (z_c - z_j), so the term of edge c -> j is
//   a_j = w_c (g_j - G) / S * p u_j / (z_c - z_j) = p w_c (g_j - G) f_j / (z_c - z_j),
// which needs only the stored fractions; dL/dz_c += sum_j a_j and
// dL/dz_j -= a_j.  Each thread gathers the terms that land on its own cell
// from itself and its eight neighbours.
constexpr int GTX = 32, GTY = 16, GNT = 256;
constexpr int GHX = GTX + 4, GHY = GTY + 4;  // two-cell halo

__device__ __forceinline__ void src_terms(const float* zs, const float* ghs, const float* gls,
                                          const uint8_t* ms, const float* __restrict__ fr,
                                          float w_hi, int hx, int hy, float p, float (&a)[8]) {
    const uint32_t m = ms[hy * GHX + hx];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.0f;
    if (!m) return;
    const float zc = zs[hy * GHX + hx];
    const float4 f0 = __ldg(reinterpret_cast<const float4*>(fr));
    const float4 f1 = __ldg(reinterpret_cast<const float4*>(fr) + 1);
    float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
    df gv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        gv[k] = df_make(0.0f);
        if (!((m >> k) & 1u)) {
            f[k] = 0.0f;
            continue;
        }
        const int j = (hy + offy(k)) * GHX + hx + offx(k);
        gv[k] = {ghs[j], gls[j]};
    }
    const df G = df_dot8(df_make(0.0f), f, gv);
    const float pw = __fmul_rn(p, w_hi);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (!((m >> k) & 1u)) continue;
        const float zj = zs[(hy + offy(k)) * GHX + hx + offx(k)];
        const float dg = df_add(gv[k], df{-G.hi, -G.lo}).hi;
        a[k] = __fdividef(__fmul_rn(__fmul_rn(pw, dg), f[k]), __fsub_rn(zc, zj));
    }
}

__global__ void __launch_bounds__(GNT) k_mfd_grad_z(Prob P, const float* __restrict__ g_hi,
                                                    const float* __restrict__ g_lo,
                                                    float* __restrict__ dLdz) {
    __shared__ float zs[GHX * GHY], ghs[GHX * GHY], gls[GHX * GHY];
    __shared__ uint8_t ms[GHX * GHY];
    __shared__ float as[(GTY + 2) * (GTX + 2)][8];
    const int64_t tiles_x = (P.nx + GTX - 1) / GTX;
    const int64_t ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    const int64_t x0 = tx * GTX, y0 = ty * GTY;
    for (int i = threadIdx.x; i < GHX * GHY; i += GNT) {
        int hy = i / GHX, hx = i - hy * GHX;
        int64_t gx = x0 + hx - 2, gy = y0 + hy - 2;
        bool in = gx >= 0 && gy >= 0 && gx < P.nx && gy < P.ny;
        int64_t gi = gy * P.nx + gx;
        zs[i] = in ? P.z[gi] : __int_as_float(0x7f800000);
        ghs[i] = in ? g_hi[gi] : 0.0f;
        gls[i] = (in && g_lo) ? g_lo[gi] : 0.0f;
        ms[i] = in ? P.rb[gi] : 0;
    }
    __syncthreads();
    // source terms of the tile and its one-cell ring
    for (int i = threadIdx.x; i < (GTX + 2) * (GTY + 2); i += GNT) {
        int ry = i / (GTX + 2), rx = i - ry * (GTX + 2);
        int64_t gx = x0 + rx - 1, gy = y0 + ry - 1;
        float a[8];
        if (gx >= 0 && gy >= 0 && gx < P.nx && gy < P.ny) {
            int64_t gi = gy * P.nx + gx;
            src_terms(zs, ghs, gls, ms, P.frac + gi * 8, P.wf[gi], rx + 1, ry + 1, P.mc.p, a);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) as[i][k] = a[k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < GTX * GTY; i += GNT) {
        int ly = i / GTX, lx = i - ly * GTX;
        int64_t gx = x0 + lx, gy = y0 + ly;
        if (gx >= P.nx || gy >= P.ny) continue;
        const int r = (ly + 1) * (GTX + 2) + lx + 1;
        df acc = df_make(0.0f);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc = df_add(acc, df_make(as[r][k]));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            // neighbour in direction k gives to this cell along code opp(k)
            int rn = (ly + 1 + offy(k)) * (GTX + 2) + lx + 1 + offx(k);
            acc = df_add(acc, df_make(-as[rn][opp(k)]));
        }
        dLdz[gy * P.nx + gx] = acc.hi;
    }
}

}  // namespace

// Persistent walker grid: a few CTAs per SM, grid-striding over the list.
int walker_grid() {
    static int grid = 0;
    if (!grid) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = (sms > 0 ? sms : 152) * 8;
    }
    return grid;
}

cudaError_t launch_mfd_grad_z(const Prob& P, const float* g_hi, const float* g_lo, float* dLdz,
                              cudaStream_t s) {
    const int64_t tiles = ((P.nx + GTX - 1) / GTX) * ((P.ny + GTY - 1) / GTY);
    k_mfd_grad_z<<<(unsigned)tiles, GNT, 0, s>>>(P, g_hi, g_lo, dLdz);
    return cudaGetLastError();
}

cudaError_t launch_mass_balance_ws(int64_t nx, int64_t ny, const uint8_t* rb, const float* rain,
                                   const uint64_t* area, const uint32_t* gbits,
                                   const EngineGlobals* G, double* partials, int nblocks,
                                   double* out, cudaStream_t s) {
    const int64_t n = nx * ny;
    cudaError_t e;
    if (rain) {  // the rain sum as in the full pass; its area term is replaced below
        k_mass_partial<false><<<nblocks, MB_NT, 0, s>>>(n, rb, rain, nullptr, nullptr, nullptr, partials);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_mass_sinks_ws<<<nblocks, MB_NT, 0, s>>>(n, rb, area, gbits, G, rain == nullptr, partials);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_mass_final<<<1, 256, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_mass_balance(int kind, int64_t nx, int64_t ny, const uint8_t* rb,
                                const float* rain, const float* w, const float* w_lo,
                                const uint64_t* area, double* partials, int nblocks, double* out,
                                cudaStream_t s) {
    const int64_t n = nx * ny;
    if (kind == 1)
        k_mass_partial<true><<<nblocks, MB_NT, 0, s>>>(n, rb, rain, w, w_lo, area, partials);
    else
        k_mass_partial<false><<<nblocks, MB_NT, 0, s>>>(n, rb, rain, w, w_lo, area, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mass_final<<<1, 256, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace fr

#ifdef FR_DEBUG_BOUNDS
// Debug builds only: first out-of-range (site << 48 | index) seen by the
// engine kernels of this translation unit (0 = none); clears it.
extern "C" unsigned long long fr_debug_bad_engine(void) {
    unsigned long long v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, fr::fr_debug_bad, sizeof(v));
    cudaMemcpyToSymbol(fr::fr_debug_bad, &z, sizeof(z));
    return v;
}
#endif

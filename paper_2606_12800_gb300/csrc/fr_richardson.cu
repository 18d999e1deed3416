// fr_richardson.cu -- the paper's own solver on one GPU: Richardson iteration
// for the "I+X" form of the flow-routing system (Sec. 3.3, App. B.1,
// Eq. richardson-I+X):
//     w^(l+1) = D^{-1} (r + R w^(l)),
// where the grid is partitioned into subdomains (here 64x32 tiles, one CTA
// each, in the role of the paper's processes), D holds the diagonal blocks of
// A (each subdomain's own cells) and R the rest (water that crosses a
// subdomain boundary).  One sweep is one launch: every tile solves its block
// exactly (high-to-low, here level by level in shared memory, Sec. 3.2) with
// the water its off-tile donors had in the previous iterate as inflow.  A
// stream that crosses tile boundaries C times is exact after C + 1 sweeps;
// the host stops after the first sweep that changes no value.
//
// A cell's eight direction terms (in-tile donors from this sweep, off-tile
// donors from the previous iterate) are accumulated in the fixed order of
// df_dot8, so the converged values are bit-identical from sweep to sweep.
#include "fr_engine.cuh"

namespace fr {
namespace {

constexpr int kRTX = 64, kRTY = 32, kRNT = 256;
constexpr int kRRX = kRTX + 2, kRRY = kRTY + 2, kRNC = kRTX * kRTY;

struct SmemRich {
    float vhi[kRNC];
    float vlo[kRNC];
    uint32_t st[kRNC / 4];    // per cell byte: pending in-tile donors (bits 0-3)
    uint16_t queue[kRNC];
    uint8_t rb[kRRX * kRRY];  // receiver masks of tile + ring (0 outside the grid)
    uint8_t dm[kRNC];         // in-tile donors
    uint8_t tm[kRNC];         // in-tile receivers
    uint8_t fin[kRNC];        // 1 final, 0 pending, 0x0F outside the grid
    int qtail;
    int lcnt[3];              // sizes of the levels being appended (rotating)
    unsigned long long changed, done;
};

__device__ __forceinline__ void push_rich(SmemRich& S, int cell, int end = 0, int* cnt = nullptr) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned pm = __ballot_sync(0xffffffffu, cell >= 0);
    if (!pm) return;
    int b0 = 0;
    if (lane == (unsigned)(__ffs(pm) - 1))
        b0 = cnt ? end + atomicAdd(cnt, __popc(pm)) : atomicAdd(&S.qtail, __popc(pm));
    b0 = __shfl_sync(0xffffffffu, b0, __ffs(pm) - 1);
    if (cell >= 0) S.queue[b0 + __popc(pm & ((1u << lane) - 1u))] = (uint16_t)cell;
}

// One sweep: prev -> next (two-float values, interleaved hi/lo); adds the
// number of cells whose value changed to counts[0] and of cells finalised to
// counts[1].
template <bool MFD>
__global__ void __launch_bounds__(kRNT) k_richardson_sweep(Prob P, const float2* __restrict__ prev,
                                                           float2* __restrict__ next,
                                                           unsigned long long* counts) {
    constexpr int TX = kRTX, TY = kRTY, RX = kRRX, NC = kRNC, NT = kRNT;
    __shared__ SmemRich S;
    const int tid = threadIdx.x;
    const int64_t tiles_x = (P.nx + TX - 1) / TX;
    const int64_t ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    const int64_t x0 = tx * TX, y0 = ty * TY;
    if (tid == 0) {
        S.qtail = 0;
        S.lcnt[0] = S.lcnt[1] = S.lcnt[2] = 0;
        S.changed = 0;
        S.done = 0;
    }
    for (int i = tid; i < RX * kRRY; i += NT) {
        const int ry = i / RX, rx = i - ry * RX;
        const int64_t gx = x0 + rx - 1, gy = y0 + ry - 1;
        uint8_t m = 0;
        if (gx >= 0 && gy >= 0 && gx < P.nx && gy < P.ny)
            m = (uint8_t)(recv_mask<MFD>(rd_rb(P, gy * P.nx + gx)) & grid_mask(gx, gy, P.nx, P.ny));
        S.rb[i] = m;
    }
    __syncthreads();
    for (int c = tid; c < NC; c += NT) {
        const int ly = c / TX, lx = c - ly * TX;
        const int r = (ly + 1) * RX + lx + 1;
        const int64_t gx = x0 + lx, gy = y0 + ly;
        uint8_t dmr = 0, tmr = 0, fin = 0x0F;
        float vh = 0.0f;
        if (gx < P.nx && gy < P.ny) {
            uint32_t don = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                don |= (uint32_t)((S.rb[r + offy(k) * RX + offx(k)] >> opp(k)) & 1u) << k;
            uint32_t in = 0xFFu;  // neighbours inside the tile
            if (lx == 0) in &= ~0x64u;
            if (lx == TX - 1) in &= ~0x91u;
            if (ly == 0) in &= ~0x32u;
            if (ly == TY - 1) in &= ~0xC8u;
            dmr = (uint8_t)(don & in);
            tmr = (uint8_t)(S.rb[r] & in);
            fin = 0;
            vh = P.init ? rd_in(P.init, P, gy * P.nx + gx, 8) : 1.0f;
        }
        S.dm[c] = dmr;
        S.tm[c] = tmr;
        S.fin[c] = fin;
        S.vhi[c] = vh;
        S.vlo[c] = 0.0f;
        reinterpret_cast<uint8_t*>(S.st)[c] = (uint8_t)__popc(dmr);
    }
    __syncthreads();
    for (int c0 = 0; c0 < NC; c0 += NT) {
        const int c = c0 + tid;
        push_rich(S, (c < NC && S.fin[c] == 0 && S.dm[c] == 0) ? c : -1);
    }
    __syncthreads();
    int lo = 0, hi = S.qtail, level = 0;
    unsigned long long nchanged = 0, ndone = 0;
    while (lo < hi) {
        if (tid == 0) S.lcnt[(level + 2) % 3] = 0;  // one barrier per level (as fr_halo.cu)
        int* const lcnt = &S.lcnt[(level + 1) % 3];
        for (int base = lo; base < hi; base += NT) {
            const int i = base + tid;
            int c = 0;
            uint32_t ready = 0;
            if (i < hi) {
                c = S.queue[i];
                const int ly = c / TX, lx = c - ly * TX;
                const int r = (ly + 1) * RX + lx + 1;
                const int64_t gc = (y0 + ly) * P.nx + (x0 + lx);
                // the eight donor terms: in-tile donors from this sweep, the
                // others from the previous iterate (R w^(l))
                float f[8];
                df vv[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    f[k] = 0.0f;
                    vv[k] = df_make(0.0f);
                    if (!((S.rb[r + offy(k) * RX + offx(k)] >> opp(k)) & 1u)) continue;
                    if ((S.dm[c] >> k) & 1u) {
                        const int j = c + offy(k) * TX + offx(k);
                        vv[k] = {S.vhi[j], S.vlo[j]};
                    } else {
                        const float2 pj = prev[gc + offi(k, P.nx)];
                        vv[k] = {pj.x, pj.y};
                    }
                    f[k] = MFD ? __ldg(P.frac + (gc + offi(k, P.nx)) * 8 + opp(k)) : 1.0f;
                }
                const df v = df_dot8(df{S.vhi[c], S.vlo[c]}, f, vv);
                S.vhi[c] = v.hi;
                S.vlo[c] = v.lo;
                S.fin[c] = 1;
                const float2 old = prev[gc];
                nchanged += (__float_as_uint(old.x) != __float_as_uint(v.hi) ||
                             __float_as_uint(old.y) != __float_as_uint(v.lo));
                next[gc] = make_float2(v.hi, v.lo);
                ++ndone;
                for (uint32_t m = S.tm[c]; m; m &= m - 1) {
                    const int k = __ffs(m) - 1;
                    const int t = c + offy(k) * TX + offx(k);
                    const uint32_t sh = 8u * (uint32_t)(t & 3);
                    const uint32_t o = atomicSub(&S.st[t >> 2], 1u << sh);
                    if (((o >> sh) & 0x0Fu) == 1u) ready |= 1u << k;
                }
            }
            while (__any_sync(0xffffffffu, ready != 0)) {
                int cell = -1;
                if (ready) {
                    const int k = __ffs(ready) - 1;
                    ready &= ready - 1;
                    cell = c + offy(k) * TX + offx(k);
                }
                push_rich(S, cell, hi, lcnt);
            }
        }
        __syncthreads();
        lo = hi;
        hi += *lcnt;
        ++level;
    }
    for (int o = 16; o; o >>= 1) {
        nchanged += __shfl_down_sync(0xffffffffu, nchanged, o);
        ndone += __shfl_down_sync(0xffffffffu, ndone, o);
    }
    if ((tid & 31) == 0 && nchanged) atomicAdd(&S.changed, nchanged);
    if ((tid & 31) == 0 && ndone) atomicAdd(&S.done, ndone);
    __syncthreads();
    if (tid == 0) {
        if (S.changed) atomicAdd(counts, S.changed);
        if (S.done) atomicAdd(counts + 1, S.done);
    }
}

// The converged two-float values into the caller's outputs.
__global__ void k_richardson_out(const float2* __restrict__ v, int64_t n, float* __restrict__ hi,
                                 float* __restrict__ lo) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = v[i];
        hi[i] = a.x;
        if (lo) lo[i] = a.y;
    }
}

}  // namespace

cudaError_t richardson_sweep(bool mfd, const Prob& P, const float2* prev, float2* next,
                             unsigned long long* counts, cudaStream_t s) {
    const unsigned grid = (unsigned)(((P.nx + kRTX - 1) / kRTX) * ((P.ny + kRTY - 1) / kRTY));
    if (mfd) k_richardson_sweep<true><<<grid, kRNT, 0, s>>>(P, prev, next, counts);
    else k_richardson_sweep<false><<<grid, kRNT, 0, s>>>(P, prev, next, counts);
    return cudaGetLastError();
}

cudaError_t richardson_output(const float2* v, int64_t n, float* hi, float* lo, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_richardson_out<<<(unsigned)blocks, 256, 0, s>>>(v, n, hi, lo);
    return cudaGetLastError();
}

}  // namespace fr

// fr_device.cuh -- device helpers shared by the flow-routing kernels.
//
// Neighbour codes follow the scan order E N W S NE NW SW SE (codes 0..7); the
// opposite of code k is k ^ 2.  Receiver rules are those of the paper's local
// flow routing (Sec. 2.1 for D8, App. A for the multi-receiver split) with the
// arithmetic fixed here so that every kernel that recomputes them gets the
// same bits.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace fr {

constexpr uint8_t kSink = 0xFF;
constexpr uint32_t kEdgeRoute = 0x1u;
constexpr uint32_t kD8Lowest = 0x2u;
constexpr uint32_t kD4 = 0x8u;
constexpr uint32_t kDinf = 0x10u;

// Offsets as 2-bit fields (offset + 1) packed per code, decoded with plain
// signed integer arithmetic (a nested-ternary form of these functions was
// zero-extended instead of sign-extended in non-unrolled loops).
__host__ __device__ __forceinline__ constexpr int offx(int k) {
    return (int)((33350u >> (2 * k)) & 3u) - 1;  // +1 0 -1 0 +1 -1 -1 +1
}
__host__ __device__ __forceinline__ constexpr int offy(int k) {
    return (int)((41105u >> (2 * k)) & 3u) - 1;  // 0 -1 0 +1 -1 -1 +1 +1
}
static_assert(offx(0) == 1 && offx(1) == 0 && offx(2) == -1 && offx(3) == 0 && offx(4) == 1 &&
              offx(5) == -1 && offx(6) == -1 && offx(7) == 1, "offx table");
static_assert(offy(0) == 0 && offy(1) == -1 && offy(2) == 0 && offy(3) == 1 && offy(4) == -1 &&
              offy(5) == -1 && offy(6) == 1 && offy(7) == 1, "offy table");
// Linear index offset of code k on a grid with nx columns.
__host__ __device__ __forceinline__ int64_t offi(int k, int64_t nx) {
    return (int64_t)offy(k) * nx + (int64_t)offx(k);
}
__host__ __device__ __forceinline__ constexpr int opp(int k) { return k ^ 2; }

// ---------------------------------------------------------------- two-float
// Unevaluated sum hi + lo with |lo| <= ulp(hi)/2 (Dekker / Knuth).  The _rn
// intrinsics keep the compiler from contracting or reassociating.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return {a, 0.0f}; }

__device__ __forceinline__ df df_norm(float s, float e) {
    float hi = __fadd_rn(s, e);
    float lo = __fsub_rn(e, __fsub_rn(hi, s));
    return {hi, lo};
}

// Knuth's two-sum of the leading words plus the trailing words.
__device__ __forceinline__ df df_add(df a, df b) {
    float s = __fadd_rn(a.hi, b.hi);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_norm(s, e);
}

__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_norm(p, e);
}

// Sum of eight two-float terms in a fixed pairwise order:
// ((t0 + t1) + (t2 + t3)) + ((t4 + t5) + (t6 + t7)).  Absent terms are zero,
// which df_add passes through exactly (the MFD normaliser S uses this order).
__device__ __forceinline__ df df_tree8(const df (&t)[8]) {
    const df a = df_add(df_add(t[0], t[1]), df_add(t[2], t[3]));
    const df b = df_add(df_add(t[4], t[5]), df_add(t[6], t[7]));
    return df_add(a, b);
}

// own + sum over k = 0..7 of f[k] * v[k], accumulated in ascending k with
// compensation (the Dot2 scheme of Ogita, Rump and Oishi, 2005, with two-float
// v): each product is split exactly by an FMA, each partial sum by Knuth's
// two-sum, and the rounding errors are summed in a second float that joins the
// result at the end.  Terms with f = 0 and v = 0 leave both floats unchanged,
// so absent neighbours may stay in the sum.  Every kernel that pulls a cell's
// value from its dependencies (water forward, adjoints backward) uses this one
// order, so a cell's value does not depend on which kernel computed it.
__device__ __forceinline__ df df_dot8(df own, const float (&f)[8], const df (&v)[8]) {
    float s = own.hi, c = own.lo;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float p = __fmul_rn(f[k], v[k].hi);
        float pe = __fmaf_rn(f[k], v[k].hi, -p);
        pe = __fmaf_rn(f[k], v[k].lo, pe);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(e, pe));
    }
    return df_norm(s, c);
}

// ------------------------------------------------------------ D8 predicate
// zn[k] = elevation of neighbour k, +inf where the neighbour lies outside the
// grid (never strictly lower).  Strictly lower neighbours only; the largest
// fl32(fl32(zc - zk) * c_k) wins, first in scan order on ties.
__device__ __forceinline__ uint8_t d8_code(float zc, const float (&zn)[8], float c_orth,
                                           float c_diag, bool lowest) {
    float best = -1.0f;
    uint8_t code = kSink;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float z = zn[k];
        if (z < zc) {
            float drop = __fsub_rn(zc, z);
            float s = lowest ? drop : __fmul_rn(drop, k < 4 ? c_orth : c_diag);
            if (s > best) {
                best = s;
                code = (uint8_t)k;
            }
        }
    }
    return code;
}

// The same selection without branches, for the rule fixed at compile time:
// d = fl32(zc - zk) > 0 exactly when zk < zc (a difference of two floats is
// zero only if they are equal; infinities and NaN compare false as above).
template <bool LOWEST>
__device__ __forceinline__ uint32_t d8_code_sel(float zc, const float (&zn)[8], float c_orth,
                                                float c_diag) {
    float best = -1.0f;
    uint32_t code = kSink;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float d = __fsub_rn(zc, zn[k]);
        const float s = LOWEST ? d : __fmul_rn(d, k < 4 ? c_orth : c_diag);
        const bool take = (d > 0.0f) & (s > best);
        best = take ? s : best;
        code = take ? (uint32_t)k : code;
    }
    return code;
}

// ------------------------------------------------------------ MFD weights
// Reciprocal distances 1/d_k as two-float, set on the host from FP64, and the
// exponent p split into its integer part pn and fraction pf (FP64, then
// rounded), so that s^p = s^pn * 2^(pf log2 s).
struct MfdConst {
    float co_hi, co_lo;  // 1/dx
    float cd_hi, cd_lo;  // 1/(sqrt(2) dx)
    float p;             // p rounded to fp32 (used for the first-order corrections)
    float pf;            // p - floor(p), rounded to fp32
    int pn;              // floor(p)
};

// Constants of the weight rule for grid spacing dx and exponent p (FP64 on the
// host or the device, then rounded; both give the same bits).
__host__ __device__ inline MfdConst make_mfd_const(double dx, double p) {
    MfdConst m;
    const double co = 1.0 / dx;
    const double cd = 1.0 / (sqrt(2.0) * dx);
    m.co_hi = (float)co;
    m.co_lo = (float)(co - (double)m.co_hi);
    m.cd_hi = (float)cd;
    m.cd_lo = (float)(cd - (double)m.cd_hi);
    m.p = (float)p;
    const double pn = floor(p);
    m.pn = (int)pn;
    m.pf = (float)(p - pn);
    return m;
}

// s^p for a positive normal s: s^pn (repeated products) times 2^(pf log2 s).
// log2 s = e + log2(m) from the exponent e and a mantissa m in [1/sqrt2, sqrt2]
// (hardware log2, absolute error at most 2^-22 there); pf * e is kept exact as
// a two-float (FMA); the power of two is split into an integer k and a rest
// |x| <= ln2/2, and e^x is summed as its Taylor series to degree 7 (truncation
// below 6e-9).  Relative error about 1e-7 for p in [1, 2], independent of the
// magnitude of s.  Other s (zero, subnormal, infinite, NaN) fall back to powf.
__device__ __forceinline__ float mfd_pow(float s, const MfdConst& c) {
    if (!(s >= 1.17549435e-38f && s <= 3.0e38f)) return powf(s, c.p);
    const int bits = __float_as_int(s);
    int e = ((bits >> 23) & 0xFF) - 127;
    float m = __int_as_float((bits & 0x007FFFFF) | 0x3F800000);
    if (m > 1.41421356f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float fe = (float)e;
    const float a = __fmul_rn(c.pf, fe);
    const float ae = __fmaf_rn(c.pf, fe, -a);
    const float b = __fmul_rn(c.pf, __log2f(m));
    float k = rintf(a);
    float r = __fadd_rn(__fadd_rn(__fsub_rn(a, k), b), ae);
    const float k2 = rintf(r);
    r = __fsub_rn(r, k2);
    k = __fadd_rn(k, k2);
    const float x = __fmul_rn(r, 0.693147180559945309f);
    float q = __fmaf_rn(x, 1.0f / 5040.0f, 1.0f / 720.0f);
    q = __fmaf_rn(x, q, 1.0f / 120.0f);
    q = __fmaf_rn(x, q, 1.0f / 24.0f);
    q = __fmaf_rn(x, q, 1.0f / 6.0f);
    q = __fmaf_rn(x, q, 0.5f);
    q = __fmaf_rn(x, q, 1.0f);
    q = __fmaf_rn(x, q, 1.0f);
    float y = __fmul_rn(q, __int_as_float(((int)k + 127) << 23));
#pragma unroll 1
    for (int i = 0; i < c.pn; ++i) y = __fmul_rn(y, s);
    return y;
}

// u_k = s_k^p for a strictly lower neighbour, s_k = (zc - zn)/d_k.  The drop
// and the product with 1/d are carried as two-float and the trailing word is
// applied as a first-order correction of the power: (s+e)^p ~ s^p (1 + p e/s)
// (the quotient e/s only scales a correction of relative size 1e-7, so a
// fast division suffices).
__device__ __forceinline__ float mfd_u(float zc, float zn, int k, const MfdConst& m) {
    float dz = __fsub_rn(zc, zn);
    float bb = __fsub_rn(dz, zc);
    float dze = __fadd_rn(__fsub_rn(zc, __fsub_rn(dz, bb)), __fsub_rn(-zn, bb));
    float ch = k < 4 ? m.co_hi : m.cd_hi;
    float cl = k < 4 ? m.co_lo : m.cd_lo;
    float s = __fmul_rn(dz, ch);
    float se = __fmaf_rn(dz, ch, -s);
    se = __fmaf_rn(dz, cl, se);
    se = __fmaf_rn(dze, ch, se);
    float u = mfd_pow(s, m);
    float corr = __fmul_rn(m.p, __fdividef(se, s));
    return __fmaf_rn(u, corr, u);
}

// Out-of-line copy of mfd_u for loops that would otherwise replicate powf.
static __device__ __noinline__ float mfd_u_call(float zc, float zn, int k, MfdConst m) {
    return mfd_u(zc, zn, k, m);
}

// Two-float reciprocal of the normaliser S = sum of u_k.
__device__ __forceinline__ df df_recip(df s) {
    float r = __frcp_rn(s.hi);
    float e = __fmaf_rn(-s.hi, r, 1.0f);
    e = __fmaf_rn(-s.lo, r, e);
    return df_norm(r, __fmul_rn(r, e));
}

// Fraction u * (1/S) as two-float.
__device__ __forceinline__ df mfd_frac(float u, df inv_s) {
    float p = __fmul_rn(u, inv_s.hi);
    float e = __fmaf_rn(u, inv_s.hi, -p);
    e = __fmaf_rn(u, inv_s.lo, e);
    return df_norm(p, e);
}

// 0x80 in each byte of x that is zero, 0 elsewhere (exact, no carries between bytes).
__device__ __forceinline__ uint32_t zero_bytes(uint32_t x) {
    return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
}

// The fractions of a cell with receiver mask m (App. A): f_k = u_k / S with
// S = sum of u_k over the mask, summed in the pairwise order of df_tree8 and
// inverted as two-float, each f_k rounded once to fp32; 0 where bit k is clear.
// Every MFD kernel takes its fractions from this one definition.
__device__ __forceinline__ void mfd_fracs8(float zc, const float (&zn)[8], uint32_t m,
                                           const MfdConst& mc, float (&f)[8]) {
    float u[8];
    df t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        u[k] = ((m >> k) & 1u) ? mfd_u(zc, zn[k], k, mc) : 0.0f;
        t[k] = df_make(u[k]);
    }
    const df inv = m ? df_recip(df_tree8(t)) : df_make(0.0f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = ((m >> k) & 1u) ? mfd_frac(u[k], inv).hi : 0.0f;
}

// D-infinity (Tarboton) receivers and fractions of one cell: the steepest of
// the eight triangular facets (cell, cardinal neighbour kc, the diagonal kd
// next to it; facet i: kc = ((i + 1) / 2) mod 4, kd = 4 + i / 2), chosen in
// fp32 on squared slopes with the same rounded operations as the oracle, then
// the split between kc and kd by the angle inside the facet:
//   f(kd) = atan2(s2, s1) / (pi/4),  f(kc) = atan2(s1 - s2, s1 + s2) / (pi/4)
// (s1 - s2 is exact in fp32 where f(kc) is small, s2 >= s1 / 2).  gm: the
// in-grid neighbours.  Returns the receiver mask.
__device__ __forceinline__ uint32_t dinf_cell(float zc, const float (&zn)[8], uint32_t gm,
                                              float c1, float cd, float (&f)[8]) {
    float best = -1.0f, b1 = 0.0f, b2 = 0.0f;
    int bi = -1, bkind = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int kc = ((i + 1) >> 1) & 3, kd = 4 + (i >> 1);
        if (!((gm >> kc) & 1u) || !((gm >> kd) & 1u)) continue;
        const float s1 = __fmul_rn(__fsub_rn(zc, zn[kc]), c1);
        const float s2 = __fmul_rn(__fsub_rn(zn[kc], zn[kd]), c1);
        float key;
        int kind;
        if (s2 <= 0.0f) {
            kind = 0;
            key = s1 > 0.0f ? __fmul_rn(s1, s1) : -1.0f;
        } else if (s2 >= s1) {
            kind = 2;
            const float sd = __fmul_rn(__fsub_rn(zc, zn[kd]), cd);
            key = sd > 0.0f ? __fmul_rn(sd, sd) : -1.0f;
        } else {
            kind = 1;
            key = __fadd_rn(__fmul_rn(s1, s1), __fmul_rn(s2, s2));
        }
        if (key > best) {
            best = key;
            bi = i;
            bkind = kind;
            b1 = s1;
            b2 = s2;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = 0.0f;
    if (bi < 0) return 0u;
    const int kc = ((bi + 1) >> 1) & 3, kd = 4 + (bi >> 1);
    if (bkind == 0) {
        f[kc] = 1.0f;
        return 1u << kc;
    }
    if (bkind == 2) {
        f[kd] = 1.0f;
        return 1u << kd;
    }
    constexpr float q = 1.27323954473516268615f;  // 4 / pi
    f[kd] = __fmul_rn(atan2f(b2, b1), q);
    f[kc] = __fmul_rn(atan2f(__fsub_rn(b1, b2), __fadd_rn(b1, b2)), q);
    return (1u << kc) | (1u << kd);
}

// ------------------------------------------------------------ byte counters
// Four 8-bit counters per 32-bit word; atomics add n << 8*(i & 3).  Counts
// never exceed 8, so no carry crosses into a neighbouring byte.
__device__ __forceinline__ uint32_t counter_add(uint32_t* words, int64_t i, uint32_t n) {
    uint32_t sh = 8u * (uint32_t)(i & 3);
    uint32_t old = atomicAdd(words + (i >> 2), n << sh);
    return ((old >> sh) & 0xFFu) + n;
}

// Neighbour codes of cell (x, y) that lie inside the grid.
__device__ __forceinline__ uint32_t grid_mask8(int64_t x, int64_t y, int64_t nx, int64_t ny) {
    uint32_t m = 0xFFu;
    if (x == 0) m &= ~0x64u;       // W NW SW
    if (x == nx - 1) m &= ~0x91u;  // E NE SE
    if (y == 0) m &= ~0x32u;       // N NE NW
    if (y == ny - 1) m &= ~0xC8u;  // S SW SE
    return m;
}

__device__ __forceinline__ bool is_edge(int64_t x, int64_t y, int64_t nx, int64_t ny) {
    return x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
}

// ------------------------------------------------------------ debug bounds
// With -DFR_DEBUG_BOUNDS every engine and receiver memory access is checked;
// the first out-of-range (site, index) is recorded in fr_debug_bad and the
// access is skipped.  Release builds compile the checks away.
#ifdef FR_DEBUG_BOUNDS
__device__ unsigned long long fr_debug_bad;
__device__ __forceinline__ bool fr_ok(int64_t i, int64_t n, unsigned site) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&fr_debug_bad, 0ull,
              ((unsigned long long)site << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull));
    return false;
}
#define FR_OK(i, n, site) ::fr::fr_ok((int64_t)(i), (int64_t)(n), (site))
#else
#define FR_OK(i, n, site) true
#endif

// Loads that bypass L1: values published by other CTAs after a fence.
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ uint64_t ld_cg(const uint64_t* p) {
    return (uint64_t)__ldcg((const unsigned long long*)p);
}

}  // namespace fr

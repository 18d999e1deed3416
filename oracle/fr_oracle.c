/*
 * fr_oracle.c -- plain, slow, obviously-correct CPU oracle for flow routing.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * (GPU) path never links, imports or calls it, and shares no code with it.
 *
 * What it computes (Bangerth, "Massively parallel flow routing and drainage
 * area determination"):
 *   - local flow routing (Sec. 2.1 and its footnote; App. A): each cell gives
 *     its water to the steepest lower neighbour (D8), or splits it among all
 *     lower neighbours (MFD, App. A, with Freeman-style weights);
 *   - global flow routing by the sequential high-to-low algorithm (Sec. 2.1,
 *     Eq. high-to-low-procedure and the "global flow routing" listing): sort
 *     cells high to low, start with w = r, pass each cell's water to its
 *     receiver(s) in that order;
 *   - the same result by a second valid processing order (Kahn topological
 *     order), which Sec. 3.2 says must give identical water amounts;
 *   - the matrix-free product y = A x (Sec. 3.1, "matrix-vector product with
 *     A"; App. A for the multi-receiver form), used for residual checks;
 *   - the adjoint g = A^{-T} gbar by a low-to-high sweep (A is lower triangular
 *     in high-to-low numbering, Sec. 2.4, so A^T is upper triangular and is
 *     solved from the lowest cell up), with dL/dr = g and dL/dz through the
 *     MFD weights;
 *   - per-cell helpers for sampled checks on grids too large for the sort:
 *     upstream basin size by breadth-first search over reversed edges, and the
 *     sink reached from a cell.
 *
 * Readings of the paper that this file fixes (the paper is silent on them):
 *   - grid is row-major, idx = y*nx + x; neighbour k has offset (dx_k, dy_k)
 *     in the scan order E(+1,0) N(0,-1) W(-1,0) S(0,+1) NE(+1,-1) NW(-1,-1)
 *     SW(-1,+1) SE(+1,+1); SINK = 0xFF;
 *   - D8 "steepest" compares slope_k = fl32(fl32(z_c - z_k) * c_k) with
 *     c_orth = fl32(1/dx), c_diag = fl32(1/(sqrt(2) dx)), over neighbours that
 *     are strictly lower; strict '>' so the first in scan order wins ties;
 *     "lowest" (flag) compares fl32(z_c - z_k) instead;
 *   - edge cells are sinks by default (they still receive water); with
 *     FR_EDGE_ROUTE they route to in-grid lower neighbours like other cells;
 *   - MFD: f_k = s_k^p / sum_j s_j^p over strictly lower neighbours,
 *     s_k = (z_c - z_k)/d_k, all in FP64;
 *   - a cell with no strictly lower neighbour is a sink (flats are sinks).
 *
 * Precision: FP64 for water and gradients, uint64 for unit-rain D8 areas.
 * The only fp32 arithmetic is the D8 slope predicate, so that the receiver
 * choice is defined bit-for-bit.  Compile with -ffp-contract=off.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_SINK 0xFFu
#define OR_EDGE_ROUTE 1u
#define OR_D8_LOWEST 2u
#define OR_D4 8u
#define OR_DINF 16u

static const int OFFX[8] = {+1, 0, -1, 0, +1, -1, -1, +1};
static const int OFFY[8] = {0, -1, 0, +1, -1, -1, +1, +1};

static int is_edge(int64_t x, int64_t y, int64_t nx, int64_t ny) {
    return x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
}

/* Local flow routing, D8 (Sec. 2.1: the neighbour that is lower and to which
 * the downhill gradient is steepest; footnote: none at the boundary).  With
 * OR_D4 only the four orthogonal neighbours are candidates (the D4 scheme
 * Sec. 2.1 names beside D8). */
void or_receivers_d8(const float* z, int64_t nx, int64_t ny, double dx, uint32_t flags,
                     uint8_t* dir) {
    float c_orth = (float)(1.0 / dx);
    float c_diag = (float)(1.0 / (sqrt(2.0) * dx));
    for (int64_t y = 0; y < ny; ++y) {
        for (int64_t x = 0; x < nx; ++x) {
            int64_t i = y * nx + x;
            dir[i] = OR_SINK;
            if (!(flags & OR_EDGE_ROUTE) && is_edge(x, y, nx, ny)) continue;
            float zc = z[i];
            float best = -1.0f;
            const int ncand = (flags & OR_D4) ? 4 : 8;
            for (int k = 0; k < ncand; ++k) {
                int64_t xn = x + OFFX[k], yn = y + OFFY[k];
                if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
                float zn = z[yn * nx + xn];
                if (!(zn < zc)) continue;
                float drop = zc - zn;
                float s;
                if (flags & OR_D8_LOWEST) s = drop;
                else s = drop * (k < 4 ? c_orth : c_diag);
                if (s > best) { best = s; dir[i] = (uint8_t)k; }
            }
        }
    }
}

/* Local flow routing, MFD (App. A): fractions of a cell's water given to each
 * strictly lower neighbour, f_k = s_k^p / sum_j s_j^p, FP64.  frac is N x 8,
 * zero where neighbour k is not a receiver.  mask bit k set iff f_k is a
 * receiver. */
/* D-infinity (Tarboton 1997) for one cell: the water goes down the steepest of
 * the eight triangular facets spanned by the cell, a cardinal neighbour e1 and
 * the diagonal neighbour e2 next to it, split between e1 and e2 by the angle
 * of the steepest direction within the facet.  Facet i pairs cardinal code
 * ((i + 1) / 2) mod 4 with diagonal code 4 + i / 2 (E-NE, N-NE, N-NW, W-NW,
 * W-SW, S-SW, S-SE, E-SE); facets with a neighbour off the grid are skipped.
 * The choice is made in fp32 on squared slopes, s1 = fl(fl(e0 - e1) c1) and
 * s2 = fl(fl(e1 - e2) c1) with c1 = fl32(1/dx), so that it is defined
 * bit-for-bit:
 *   s2 <= 0:        along e1 only, key s1^2 (if s1 > 0)
 *   s2 >= s1:       along e2 only, sd = fl(fl(e0 - e2) cd), cd = fl32(1/(sqrt2 dx)),
 *                   key sd^2 (if sd > 0)
 *   otherwise:      inside the facet, key s1^2 + s2^2;
 * the largest key wins, the first facet on ties; no positive key: a sink.
 * Inside a facet the fractions are exact functions of those slopes (FP64):
 *   f(e2) = atan2(s2, s1) / (pi/4),  f(e1) = atan2(s1 - s2, s1 + s2) / (pi/4)
 * (they sum to 1; the second form keeps f(e1) accurate where it is small). */
static void dinf_cell(const double* z, int64_t nx, int64_t ny, double dx, int64_t x, int64_t y,
                      uint8_t* mask, double* f) {
    const float c1 = (float)(1.0 / dx), cd = (float)(1.0 / (sqrt(2.0) * dx));
    const float e0 = (float)z[y * nx + x];
    float best = -1.0f, b1 = 0.0f, b2 = 0.0f;
    int bi = -1, bkind = 0;
    for (int i = 0; i < 8; ++i) {
        const int kc = ((i + 1) / 2) % 4, kd = 4 + i / 2;
        const int64_t xc = x + OFFX[kc], yc = y + OFFY[kc], xd = x + OFFX[kd], yd = y + OFFY[kd];
        if (xc < 0 || yc < 0 || xc >= nx || yc >= ny || xd < 0 || yd < 0 || xd >= nx || yd >= ny)
            continue;
        const float e1 = (float)z[yc * nx + xc], e2 = (float)z[yd * nx + xd];
        const float s1 = (e0 - e1) * c1, s2 = (e1 - e2) * c1;
        float key;
        int kind;
        if (s2 <= 0.0f) {
            kind = 0;
            key = s1 > 0.0f ? s1 * s1 : -1.0f;
        } else if (s2 >= s1) {
            kind = 2;
            const float sd = (e0 - e2) * cd;
            key = sd > 0.0f ? sd * sd : -1.0f;
        } else {
            kind = 1;
            key = s1 * s1 + s2 * s2;
        }
        if (key > best) { best = key; bi = i; bkind = kind; b1 = s1; b2 = s2; }
    }
    *mask = 0;
    for (int k = 0; k < 8; ++k) f[k] = 0.0;
    if (bi < 0) return;
    const int kc = ((bi + 1) / 2) % 4, kd = 4 + bi / 2;
    const double q = 4.0 / 3.14159265358979323846;
    if (bkind == 0) { f[kc] = 1.0; *mask = (uint8_t)(1u << kc); return; }
    if (bkind == 2) { f[kd] = 1.0; *mask = (uint8_t)(1u << kd); return; }
    f[kd] = atan2((double)b2, (double)b1) * q;
    f[kc] = atan2((double)b1 - (double)b2, (double)b1 + (double)b2) * q;
    *mask = (uint8_t)((1u << kc) | (1u << kd));
}

void or_receivers_mfd(const double* z, int64_t nx, int64_t ny, double dx, double p, uint32_t flags,
                      uint8_t* mask, double* frac) {
    if (flags & OR_DINF) {
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t i = y * nx + x;
                if (!(flags & OR_EDGE_ROUTE) && is_edge(x, y, nx, ny)) {
                    mask[i] = 0;
                    for (int k = 0; k < 8; ++k) frac[i * 8 + k] = 0.0;
                    continue;
                }
                dinf_cell(z, nx, ny, dx, x, y, &mask[i], &frac[i * 8]);
            }
        return;
    }
    for (int64_t y = 0; y < ny; ++y) {
        for (int64_t x = 0; x < nx; ++x) {
            int64_t i = y * nx + x;
            double u[8];
            double tot = 0.0;
            mask[i] = 0;
            for (int k = 0; k < 8; ++k) { u[k] = 0.0; frac[i * 8 + k] = 0.0; }
            if (!(flags & OR_EDGE_ROUTE) && is_edge(x, y, nx, ny)) continue;
            double zc = z[i];
            for (int k = 0; k < 8; ++k) {
                int64_t xn = x + OFFX[k], yn = y + OFFY[k];
                if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
                double zn = z[yn * nx + xn];
                if (!(zn < zc)) continue;
                double d = (k < 4) ? dx : sqrt(2.0) * dx;
                double s = (zc - zn) / d;
                u[k] = pow(s, p);
                mask[i] |= (uint8_t)(1u << k);
            }
            for (int k = 0; k < 8; ++k) tot += u[k];
            if (tot > 0.0)
                for (int k = 0; k < 8; ++k) frac[i * 8 + k] = u[k] / tot;
        }
    }
}

/* Number of donors of each cell (cells whose routing sends water to it). */
void or_indegree(const uint8_t* dir_or_mask, int is_mask, int64_t nx, int64_t ny, uint8_t* indeg) {
    int64_t n = nx * ny;
    memset(indeg, 0, (size_t)n);
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            int64_t i = y * nx + x;
            for (int k = 0; k < 8; ++k) {
                int sends = is_mask ? ((dir_or_mask[i] >> k) & 1) : (dir_or_mask[i] == k);
                if (!sends) continue;
                indeg[(y + OFFY[k]) * nx + (x + OFFX[k])] += 1;
            }
        }
}

/* ---- high-to-low order (Sec. 2.1: sort all nodes from high to low) ---- */
static const float* g_sort_z;
static int cmp_high_to_low(const void* a, const void* b) {
    int64_t ia = *(const int64_t*)a, ib = *(const int64_t*)b;
    float za = g_sort_z[ia], zb = g_sort_z[ib];
    if (za > zb) return -1;
    if (za < zb) return 1;
    return (ia < ib) ? -1 : (ia > ib);
}

static const double* g_sort_z64;
static int cmp_high_to_low64(const void* a, const void* b) {
    int64_t ia = *(const int64_t*)a, ib = *(const int64_t*)b;
    double za = g_sort_z64[ia], zb = g_sort_z64[ib];
    if (za > zb) return -1;
    if (za < zb) return 1;
    return (ia < ib) ? -1 : (ia > ib);
}

/* Same order for FP64 elevations (used when elevations are perturbed in FP64
 * for finite-difference checks of the elevation gradient). */
void or_high_to_low_order64(const double* z, int64_t n, int64_t* order) {
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    g_sort_z64 = z;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_high_to_low64);
}

/* order[0..n) = cell indices sorted by (z descending, index ascending).
 * Any order in which every cell comes after all of its higher neighbours is
 * valid (Sec. 3.2); water only moves to strictly lower cells, so this is one. */
void or_high_to_low_order(const float* z, int64_t n, int64_t* order) {
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    g_sort_z = z;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_high_to_low);
}

/* Global flow routing, D8 (Eq. high-to-low-procedure; listing "global flow
 * routing"): w = r, then for src high-to-low: w(dst) += w(src).
 * rain == NULL means unit rain.  w (FP64) and/or area (uint64, unit rain)
 * may be NULL. */
void or_accumulate_d8(const uint8_t* dir, const int64_t* order, const float* rain,
                      int64_t nx, int64_t ny, double* w, uint64_t* area) {
    int64_t n = nx * ny;
    if (w) for (int64_t i = 0; i < n; ++i) w[i] = rain ? (double)rain[i] : 1.0;
    if (area) for (int64_t i = 0; i < n; ++i) area[i] = 1;
    for (int64_t t = 0; t < n; ++t) {
        int64_t src = order[t];
        uint8_t d = dir[src];
        if (d == OR_SINK) continue;
        int64_t dst = src + OFFY[d] * nx + OFFX[d];
        if (w) w[dst] += w[src];
        if (area) area[dst] += area[src];
    }
}

/* Global flow routing, MFD (App. A: each column of A holds the fractions):
 * w = r, then for src high-to-low: w(dst_k) += f_k w(src). */
void or_accumulate_mfd(const double* frac, const int64_t* order, const float* rain,
                       int64_t nx, int64_t ny, double* w) {
    int64_t n = nx * ny;
    for (int64_t i = 0; i < n; ++i) w[i] = rain ? (double)rain[i] : 1.0;
    for (int64_t t = 0; t < n; ++t) {
        int64_t src = order[t];
        for (int k = 0; k < 8; ++k) {
            double f = frac[src * 8 + k];
            if (f == 0.0) continue;
            w[src + OFFY[k] * nx + OFFX[k]] += f * w[src];
        }
    }
}

/* A second valid processing order: Kahn's algorithm (a cell is ready once all
 * of its donors are done).  Sec. 3.2: only the processing order matters, so
 * the water amounts must equal those of the high-to-low sort.
 * dir_or_mask as in or_indegree; order_out receives the Kahn order. */
int64_t or_kahn_order(const uint8_t* dir_or_mask, int is_mask, int64_t nx, int64_t ny,
                      int64_t* order_out) {
    int64_t n = nx * ny;
    uint8_t* cnt = (uint8_t*)malloc((size_t)n);
    or_indegree(dir_or_mask, is_mask, nx, ny, cnt);
    int64_t head = 0, tail = 0;
    for (int64_t i = 0; i < n; ++i) if (cnt[i] == 0) order_out[tail++] = i;
    while (head < tail) {
        int64_t c = order_out[head++];
        int64_t x = c % nx, y = c / nx;
        for (int k = 0; k < 8; ++k) {
            int sends = is_mask ? ((dir_or_mask[c] >> k) & 1) : (dir_or_mask[c] == k);
            if (!sends) continue;
            int64_t d = (y + OFFY[k]) * nx + (x + OFFX[k]);
            if (--cnt[d] == 0) order_out[tail++] = d;
        }
    }
    free(cnt);
    return tail; /* == n unless the routing has a cycle */
}

/* Matrix-free y = A x (Sec. 3.1 "matrix-vector product with A; optimized", and
 * the multi-receiver form of App. A): y = x, then y(dst) -= f * x(src). */
void or_apply_A(const uint8_t* dir, const double* frac, int64_t nx, int64_t ny,
                const double* x, double* y) {
    int64_t n = nx * ny;
    for (int64_t i = 0; i < n; ++i) y[i] = x[i];
    for (int64_t src = 0; src < n; ++src) {
        if (frac) {
            for (int k = 0; k < 8; ++k) {
                double f = frac[src * 8 + k];
                if (f != 0.0) y[src + OFFY[k] * nx + OFFX[k]] -= f * x[src];
            }
        } else {
            uint8_t d = dir[src];
            if (d != OR_SINK) y[src + OFFY[d] * nx + OFFX[d]] -= x[src];
        }
    }
}

/* Adjoint: g = A^{-T} gbar.  Column src of A holds +1 on the diagonal and -f_k
 * in rows dst_k, so row src of A^T reads g(src) - sum_k f_k g(dst_k) = gbar(src).
 * Receivers are strictly lower, so a low-to-high sweep (the high-to-low order
 * reversed) has every g(dst_k) ready when src is reached.
 * frac == NULL selects D8 (dir).  gbar == NULL selects the loss
 * L = sum over sinks of w_s^2, i.e. gbar_s = 2 w_s at sinks and 0 elsewhere.
 * Returns g in g_out (== dL/dr). */
void or_adjoint(const uint8_t* dir, const double* frac, const int64_t* order,
                int64_t nx, int64_t ny, const double* w, const double* gbar, double* g) {
    int64_t n = nx * ny;
    for (int64_t i = 0; i < n; ++i) {
        if (gbar) { g[i] = gbar[i]; continue; }
        int sink;
        if (frac) {
            sink = 1;
            for (int k = 0; k < 8; ++k) if (frac[i * 8 + k] != 0.0) sink = 0;
        } else {
            sink = (dir[i] == OR_SINK);
        }
        g[i] = sink ? 2.0 * w[i] : 0.0;
    }
    for (int64_t t = n - 1; t >= 0; --t) {
        int64_t src = order[t];
        int64_t x = src % nx, y = src / nx;
        if (frac) {
            double acc = 0.0;
            for (int k = 0; k < 8; ++k) {
                double f = frac[src * 8 + k];
                if (f != 0.0) acc += f * g[(y + OFFY[k]) * nx + (x + OFFX[k])];
            }
            g[src] += acc;
        } else {
            uint8_t d = dir[src];
            if (d != OR_SINK) g[src] += g[(y + OFFY[d]) * nx + (x + OFFX[d])];
        }
    }
}

/* dL/dz for the MFD rule, given w = A^{-1} r and g = A^{-T} gbar.
 * dL/dtheta = g^T (dW/dtheta) w with W(dst_k, src) = f_k(src).  The fractions
 * of src depend on z_src and on z of its lower neighbours:
 *   u_k = s_k^p, s_k = (z_src - z_k)/d_k, f_k = u_k / S, S = sum_j u_j,
 *   dL/du_j = w_src (g_{dst_j} - G) / S,  G = sum_k f_k g_{dst_k},
 *   du_j/dz_src = p s_j^{p-1} / d_j = -du_j/dz_{dst_j}.
 * The lower set is held fixed (the derivative where it is constant). */
void or_mfd_grad_z(const double* z, int64_t nx, int64_t ny, double dx, double p, uint32_t flags,
                   const double* frac, const double* w, const double* g, double* dLdz) {
    int64_t n = nx * ny;
    for (int64_t i = 0; i < n; ++i) dLdz[i] = 0.0;
    for (int64_t y = 0; y < ny; ++y) {
        for (int64_t x = 0; x < nx; ++x) {
            int64_t src = y * nx + x;
            double s[8], u[8], S = 0.0, G = 0.0;
            int any = 0;
            for (int k = 0; k < 8; ++k) {
                s[k] = 0.0; u[k] = 0.0;
                if (frac[src * 8 + k] == 0.0) continue;
                int64_t dst = (y + OFFY[k]) * nx + (x + OFFX[k]);
                double d = (k < 4) ? dx : sqrt(2.0) * dx;
                s[k] = (z[src] - z[dst]) / d;
                u[k] = pow(s[k], p);
                S += u[k];
                any = 1;
            }
            if (!any) continue;
            for (int k = 0; k < 8; ++k) {
                if (u[k] == 0.0) continue;
                int64_t dst = (y + OFFY[k]) * nx + (x + OFFX[k]);
                G += (u[k] / S) * g[dst];
            }
            for (int k = 0; k < 8; ++k) {
                if (u[k] == 0.0) continue;
                int64_t dst = (y + OFFY[k]) * nx + (x + OFFX[k]);
                double d = (k < 4) ? dx : sqrt(2.0) * dx;
                double dLdu = w[src] * (g[dst] - G) / S;
                double dudz = p * pow(s[k], p - 1.0) / d;
                dLdz[src] += dLdu * dudz;
                dLdz[dst] -= dLdu * dudz;
            }
        }
    }
    (void)flags;
}

/* Mass balance (Sec. 4: outflow equals total rain): out[0] = sum of w over
 * sinks, out[1] = sum of r.  frac == NULL selects D8. */
void or_mass_balance(const uint8_t* dir, const uint8_t* mask, int64_t n, const float* rain,
                     const double* w, double* out) {
    double s = 0.0, r = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        int sink = mask ? (mask[i] == 0) : (dir[i] == OR_SINK);
        if (sink) s += w[i];
        r += rain ? (double)rain[i] : 1.0;
    }
    out[0] = s;
    out[1] = r;
}

/* Upstream basin size of one cell by breadth-first search over reversed D8
 * edges (the cell itself included): equals the unit-rain area at that cell.
 * work must hold nx*ny int64 entries; seen must hold nx*ny bytes, all zero on
 * entry; both are restored/zeroed on exit so the call can be repeated. */
uint64_t or_upstream_count(const uint8_t* dir, int64_t nx, int64_t ny, int64_t cell,
                           int64_t* work, uint8_t* seen) {
    int64_t head = 0, tail = 0;
    work[tail++] = cell;
    seen[cell] = 1;
    while (head < tail) {
        int64_t c = work[head++];
        int64_t x = c % nx, y = c / nx;
        for (int k = 0; k < 8; ++k) {
            int64_t xn = x + OFFX[k], yn = y + OFFY[k];
            if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
            int64_t nb = yn * nx + xn;
            /* nb donates to c iff its direction points back at c */
            int back = (k < 4) ? ((k + 2) & 3) : (4 + ((k - 4 + 2) & 3));
            if (dir[nb] == back && !seen[nb]) { seen[nb] = 1; work[tail++] = nb; }
        }
    }
    for (int64_t t = 0; t < tail; ++t) seen[work[t]] = 0;
    return (uint64_t)tail;
}

/* Sink reached from a cell by following D8 receivers (-1 if the walk exceeds
 * nx*ny steps, i.e. a cycle). */
int64_t or_sink_of(const uint8_t* dir, int64_t nx, int64_t ny, int64_t cell) {
    int64_t c = cell;
    for (int64_t steps = 0; steps <= nx * ny; ++steps) {
        uint8_t d = dir[c];
        if (d == OR_SINK) return c;
        c += OFFY[d] * nx + OFFX[d];
    }
    return -1;
}

/* ------------------------------------------------------------------------
 * Exact change of the loss L = sum over sinks of w^2 when one input of cell m
 * changes by `delta`, without re-solving the whole grid (for finite-difference
 * checks of the adjoint on grids too large for repeated full solves).
 *   mode 0: z[m] += delta.  Only the fractions of m and its eight neighbours
 *           depend on z[m].  With W' the new weights and w the old water,
 *           A' w' = r and A w = r give A' (w' - w) = (W' - W) w, so the change
 *           d = w' - w starts at the receivers of those nine cells and is
 *           passed on with the new fractions.  Returns NaN if the change
 *           would alter a receiver mask (the weights are then not smooth).
 *   mode 1: the rain of m += delta; d starts at m and is passed on with the
 *           unchanged fractions.
 * d travels strictly downhill, so cells are finalised in decreasing
 * (perturbed) elevation from a max-heap; the change of L is accumulated at
 * the sinks as 2 w d + d^2 (no cancellation against L itself).
 * dwork [n] (doubles) and mark [n] (bytes) must be zero on entry and are zero
 * again on return.
 */
typedef struct {
    const double* z;
    int64_t m;
    double zm;
} zview;

static double zv(const zview* v, int64_t i) { return i == v->m ? v->zm : v->z[i]; }

/* max-heap of cell indices ordered by (elevation desc, index asc) */
static int heap_before(const zview* v, int64_t a, int64_t b) {
    double za = zv(v, a), zb = zv(v, b);
    return za > zb || (za == zb && a < b);
}
static void heap_push(int64_t* h, int64_t* n, int64_t c, const zview* v) {
    int64_t i = (*n)++;
    h[i] = c;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!heap_before(v, h[i], h[p])) break;
        int64_t t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}
static int64_t heap_pop(int64_t* h, int64_t* n, const zview* v) {
    int64_t top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < *n && heap_before(v, h[l], h[b])) b = l;
        if (r < *n && heap_before(v, h[r], h[b])) b = r;
        if (b == i) break;
        int64_t t = h[i]; h[i] = h[b]; h[b] = t;
        i = b;
    }
    return top;
}

/* Mask and fractions of one cell (the rule of or_receivers_mfd) under view v. */
static void mfd_cell(const zview* v, int64_t nx, int64_t ny, double dx, double p, uint32_t flags,
                     int64_t i, uint8_t* mask, double* f) {
    int64_t x = i % nx, y = i / nx;
    double u[8], tot = 0.0;
    *mask = 0;
    for (int k = 0; k < 8; ++k) { u[k] = 0.0; f[k] = 0.0; }
    if (!(flags & OR_EDGE_ROUTE) && is_edge(x, y, nx, ny)) return;
    double zc = zv(v, i);
    for (int k = 0; k < 8; ++k) {
        int64_t xn = x + OFFX[k], yn = y + OFFY[k];
        if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
        double zn = zv(v, yn * nx + xn);
        if (!(zn < zc)) continue;
        double d = (k < 4) ? dx : sqrt(2.0) * dx;
        u[k] = pow((zc - zn) / d, p);
        *mask |= (uint8_t)(1u << k);
    }
    for (int k = 0; k < 8; ++k) tot += u[k];
    if (tot > 0.0)
        for (int k = 0; k < 8; ++k) f[k] = u[k] / tot;
}

double or_mfd_delta_loss(const double* z, int64_t nx, int64_t ny, double dx, double p,
                         uint32_t flags, const uint8_t* mask, const double* frac, const double* w,
                         int64_t m, double delta, int mode, double* dwork, uint8_t* mark) {
    zview v = {z, m, mode == 0 ? z[m] + delta : z[m]};
    /* the nine cells whose fractions may change, and their new fractions */
    int64_t aff[9];
    double fnew[9][8];
    int naff = 0;
    int64_t mx = m % nx, my = m / nx;
    if (mode == 0) {
        for (int k = -1; k < 8; ++k) {
            int64_t xn = mx + (k < 0 ? 0 : OFFX[k]), yn = my + (k < 0 ? 0 : OFFY[k]);
            if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
            int64_t a = yn * nx + xn;
            uint8_t mk;
            mfd_cell(&v, nx, ny, dx, p, flags, a, &mk, fnew[naff]);
            if (mk != mask[a]) return NAN;
            aff[naff++] = a;
        }
    }
    int64_t cap = 1024, nheap = 0;
    int64_t* heap = (int64_t*)malloc((size_t)cap * sizeof(int64_t));
    if (!heap) return NAN;
#define OR_ADD(cell, amount)                                                       \
    do {                                                                           \
        int64_t c_ = (cell);                                                       \
        dwork[c_] += (amount);                                                     \
        if (!mark[c_]) {                                                           \
            mark[c_] = 1;                                                          \
            if (nheap == cap) {                                                    \
                cap *= 2;                                                          \
                int64_t* nh = (int64_t*)realloc(heap, (size_t)cap * sizeof(int64_t)); \
                if (!nh) { free(heap); return NAN; }                               \
                heap = nh;                                                         \
            }                                                                      \
            heap_push(heap, &nheap, c_, &v);                                       \
        }                                                                          \
    } while (0)
    if (mode == 0) {
        for (int q = 0; q < naff; ++q) {
            int64_t a = aff[q];
            for (int k = 0; k < 8; ++k) {
                if (!((mask[a] >> k) & 1u)) continue;
                double ds = (fnew[q][k] - frac[a * 8 + k]) * w[a];
                OR_ADD(a + OFFY[k] * nx + OFFX[k], ds);
            }
        }
    } else {
        OR_ADD(m, delta);
    }
    double dL = 0.0;
    while (nheap > 0) {
        int64_t c = heap_pop(heap, &nheap, &v);
        double d = dwork[c];
        dwork[c] = 0.0;
        mark[c] = 0;
        if (mask[c] == 0) {
            dL += 2.0 * w[c] * d + d * d;
            continue;
        }
        const double* fc = frac + c * 8;
        for (int q = 0; q < naff; ++q)
            if (aff[q] == c) fc = fnew[q];
        for (int k = 0; k < 8; ++k)
            if ((mask[c] >> k) & 1u) OR_ADD(c + OFFY[k] * nx + OFFX[k], d * fc[k]);
    }
#undef OR_ADD
    free(heap);
    return dL;
}

/* ------------------------------------------------------------------ depression filling
 * The paper routes a depression-filled DEM (Sec. 4); filling is the step before
 * the path.  Reading taken: the least surface F >= z that keeps every edge
 * cell at its own elevation and gives every interior cell a neighbour (of 8)
 * that is strictly lower, by at least one fp32 step -- so that D8 routing on F
 * has sinks only on the edge.  Equivalently, the unique solution of
 *     F_c = z_c at edge cells,
 *     F_c = max(z_c, min over neighbours n of succ(F_n)) elsewhere,
 * succ(x) being the next fp32 value above x.  Computed by priority-flood: the
 * edge cells seed a min-heap; each popped cell gives every not yet reached
 * neighbour n the value max(z_n, succ(F_c)).  Cells leave the heap in
 * non-decreasing F, so each cell is reached from its lowest neighbour. */
static float succf(float x) { return nextafterf(x, INFINITY); }

typedef struct { float f; int64_t i; } fill_item;

static int fill_before(fill_item a, fill_item b) { return a.f < b.f || (a.f == b.f && a.i < b.i); }

static void fill_push(fill_item* h, int64_t* n, fill_item it) {
    int64_t k = (*n)++;
    h[k] = it;
    while (k > 0) {
        int64_t p = (k - 1) / 2;
        if (!fill_before(h[k], h[p])) break;
        fill_item t = h[k]; h[k] = h[p]; h[p] = t;
        k = p;
    }
}

static fill_item fill_pop(fill_item* h, int64_t* n) {
    fill_item top = h[0];
    h[0] = h[--(*n)];
    int64_t k = 0;
    for (;;) {
        int64_t l = 2 * k + 1, r = l + 1, m = k;
        if (l < *n && fill_before(h[l], h[m])) m = l;
        if (r < *n && fill_before(h[r], h[m])) m = r;
        if (m == k) break;
        fill_item t = h[k]; h[k] = h[m]; h[m] = t;
        k = m;
    }
    return top;
}

int or_fill(const float* z, int64_t nx, int64_t ny, float* out) {
    const int64_t n = nx * ny;
    fill_item* heap = (fill_item*)malloc((size_t)n * sizeof(fill_item));
    uint8_t* seen = (uint8_t*)calloc((size_t)n, 1);
    if (!heap || !seen) { free(heap); free(seen); return -1; }
    int64_t hn = 0;
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            int64_t i = y * nx + x;
            if (!is_edge(x, y, nx, ny)) continue;
            out[i] = z[i];
            seen[i] = 1;
            fill_item it = {z[i], i};
            fill_push(heap, &hn, it);
        }
    while (hn > 0) {
        fill_item c = fill_pop(heap, &hn);
        int64_t cx = c.i % nx, cy = c.i / nx;
        for (int k = 0; k < 8; ++k) {
            int64_t xn = cx + OFFX[k], yn = cy + OFFY[k];
            if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
            int64_t j = yn * nx + xn;
            if (seen[j]) continue;
            seen[j] = 1;
            float s = succf(c.f);
            out[j] = z[j] > s ? z[j] : s;
            fill_item it = {out[j], j};
            fill_push(heap, &hn, it);
        }
    }
    free(heap);
    free(seen);
    return 0;
}

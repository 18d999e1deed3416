/*
 * fr.h -- C ABI of the GB300 flow-routing library (libfr.so).
 *
 * The library computes the data-parallel hot path of W. Bangerth, "Massively
 * parallel flow routing and drainage area determination":
 *   1. local flow routing: each DEM cell picks its receiver (D8 steepest
 *      descent, Sec. 2.1) or splits its water among all lower neighbours with
 *      slope-weighted fractions (MFD, App. A);
 *   2. global flow routing: the amount of water w at every cell, the solution
 *      of A w = r with A = I - W (Sec. 2.2, Eq. Aw=f), i.e. rain plus all water
 *      received from upstream, computed exactly (the result of the sequential
 *      high-to-low algorithm of Sec. 2.1);
 *   3. the adjoint of step 2 (gradients of a loss with respect to rain and,
 *      for MFD, elevation), a batched form over many independent DEMs, and a
 *      mass-balance check (Sec. 4: outflow equals total rain).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid      row-major, cell (x, y) at index y*nx + x, 0 <= x < nx (fastest).
 * Neighbour codes k = 0..7 in the scan order E(+1,0) N(0,-1) W(-1,0) S(0,+1)
 *           NE(+1,-1) NW(-1,-1) SW(-1,+1) SE(+1,+1); FR_SINK (0xFF) = no
 *           receiver.  Orthogonal distance dx, diagonal sqrt(2)*dx.
 * Memory    every array argument is a DEVICE pointer to caller-owned memory
 *           (cudaMalloc or equivalent), unless stated otherwise.  The library
 *           allocates nothing in these calls; scratch comes from the caller's
 *           workspace `ws` of at least the size returned by the matching
 *           *_workspace_size query, 256-byte aligned.  Workspace contents need
 *           not be initialised and are not preserved between calls.
 * Streams   `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *           stream).  All work is enqueued on it; calls return without
 *           synchronising.  Inputs must stay valid and outputs must not be
 *           read until the stream has reached the end of the call.
 * Errors    argument errors are detected synchronously and returned before
 *           anything is enqueued.  Launch errors return FR_ERR_CUDA.  Errors
 *           found on the device (a routing graph with a cycle, a device-side
 *           wait that reached its limit) are written to a status word inside
 *           the workspace; read it with fr_get_status() after the stream has
 *           synchronised.  On a device-side error the outputs are unspecified.
 * Flags     bit-or of the FR_* flag macros below; unknown bits are rejected.
 */
#ifndef FR_H
#define FR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FR_OK = 0,
    FR_ERR_INVALID_ARG = 1, /* null pointer, non-positive size, bad flag, nx*ny overflow */
    FR_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed */
    FR_ERR_WORKSPACE = 3,   /* workspace NULL, too small or not 256-byte aligned */
    FR_ERR_NONFINITE = 4,   /* FR_CHECK_FINITE: the DEM holds NaN or Inf */
    FR_ERR_NO_PROGRESS = 5, /* device: not every cell was reached (cycle in the routing) */
    FR_ERR_UNSUPPORTED = 6  /* valid request the library does not implement (dL/dz under FR_DINF) */
} fr_status;

/* ---- flags ---------------------------------------------------------------
 * Edge cells (x == 0, y == 0, x == nx-1, y == ny-1).  The paper's footnote to
 * Sec. 2.1 gives boundary cells no receiver; its Fig. 1 example routes them.
 *   FR_EDGE_SINK  (default) edge cells are sinks; they still receive water.
 *   FR_EDGE_ROUTE edge cells route to in-grid lower neighbours like any cell.
 * D8 rule.  Sec. 2.1 picks the lower neighbour with the steepest downhill
 * gradient; the introduction speaks of the lowest-lying neighbour.
 *   FR_D8_STEEPEST (default) maximise fl32(fl32(z_c - z_k) * c_k),
 *                  c_orth = fl32(1/dx), c_diag = fl32(1/(sqrt(2)*dx)).
 *   FR_D8_LOWEST   maximise fl32(z_c - z_k).
 * Both consider only strictly lower neighbours (flats are sinks) and break
 * ties with strict '>' in scan order (the first code wins).
 *   FR_D4          D8 routing only (rejected for MFD): consider the four
 *                  orthogonal neighbours E N W S alone, the D4 scheme that
 *                  Sec. 2.1 names beside D8.
 *   FR_DINF        MFD routing only (rejected for D8): Tarboton's D-infinity
 *                  split, the other multiple-flow-direction scheme App. A
 *                  names, instead of the slope-power split (p is then unused).
 *                  Water goes down the steepest of the eight triangular facets
 *                  (cell, cardinal neighbour, the diagonal next to it), chosen in
 *                  fp32 on squared slopes (s1 = fl(fl(z - z_card) / dx),
 *                  s2 = fl(fl(z_card - z_diag) / dx); along the cardinal if
 *                  s2 <= 0, along the diagonal if s2 >= s1, else inside the
 *                  facet), first facet on ties, and is split f_diag =
 *                  atan2(s2, s1) / (pi/4), f_card = atan2(s1 - s2, s1 + s2) / (pi/4).
 *                  dL/dz of the adjoint is not available for it.
 *   FR_CHECK_FINITE reject a DEM holding NaN or Inf (FR_ERR_NONFINITE; this
 *                  check synchronises the stream).
 * Global phase of D8 accumulation (fr_accumulate with a D8 routing, whose
 * fr_routing.flags carry these, and fr_route_d8).  Cells whose upstream basin
 * leaves their tile are finished either by walkers that follow the receivers
 * one cell per step, or by a solve on the skeleton of a 64x64 tiling whose
 * steps cross a whole tile (Sec. 2.4's skeleton of the domain decomposition);
 * the second wins on DEMs with long rivers (depression-filled, planar), the
 * first on rough ones.  By default the library picks the skeleton solve when
 * at least 1/512 of the cells need the global phase.  Both give the same
 * areas; real-valued water differs only in the order of two-float additions.
 *   FR_GLOBAL_WALKERS  always the cell walkers.
 *   FR_GLOBAL_SKELETON always the skeleton solve (grids too small for its
 *                  scratch, under about 64x64 cells, use the walkers).
 * Routing flag of MFD routings (fr_routing.flags), for fr_accumulate and
 * fr_route_adjoint: the checkpoint of the weights between a forward route and
 * its adjoint.  By default both calls recompute the fractions from the DEM
 * into the workspace (a stored copy would take 32 bytes per cell).
 *   FR_WEIGHTS_IN_WORKSPACE  the workspace already holds this routing's
 *                  fractions: fr_route_mfd, fr_accumulate or fr_route_adjoint
 *                  left them there, called with the same routing (mask, DEM,
 *                  dx, p and the receiver flags) and the same workspace, and
 *                  no call on a different routing used that workspace since.
 *                  The call reads them instead of recomputing them.  The
 *                  library cannot check this; wrong fractions give wrong
 *                  results, not an error.  D8 routings and the receiver,
 *                  fused route and batch calls reject this flag.
 * Routing flag of D8 routings, for fr_mass_balance: the area term formed where
 * the areas are produced.  An accumulation with areas sums the areas of the
 * FR_SINK cells its local phase finishes into the workspace and marks the
 * cells it leaves to its global phase there.
 *   FR_SINK_SUMS_IN_WORKSPACE  the workspace holds these records of the
 *                  accumulation that wrote `area` for this routing: that
 *                  fr_accumulate or fr_route_d8 call (with areas) was the
 *                  last call on the workspace other than fr_mass_balance and
 *                  fr_get_status.  fr_mass_balance then takes the area term
 *                  from them and reads `area` only at the FR_SINK cells among
 *                  the global cells, instead of at every FR_SINK cell; the
 *                  result is the same.  It needs `area` and no `w`; with
 *                  `rain` the rain term is still summed over the field.
 *                  fr_accumulate and fr_route_adjoint ignore the flag; MFD
 *                  routings and the receiver, fused route and batch calls
 *                  reject it.  As with FR_WEIGHTS_IN_WORKSPACE, the library
 *                  cannot check the claim.
 */
#define FR_EDGE_SINK 0x0u
#define FR_EDGE_ROUTE 0x1u
#define FR_D8_STEEPEST 0x0u
#define FR_D8_LOWEST 0x2u
#define FR_CHECK_FINITE 0x4u
#define FR_D4 0x8u
#define FR_DINF 0x10u
#define FR_GLOBAL_WALKERS 0x20u
#define FR_GLOBAL_SKELETON 0x40u
#define FR_WEIGHTS_IN_WORKSPACE 0x80u
#define FR_SINK_SUMS_IN_WORKSPACE 0x100u

#define FR_SINK 0xFFu

/* Largest MFD slope exponent p accepted (the weights take floor(p) products). */
#define FR_MFD_MAX_P 64.0

typedef enum { FR_ROUTING_D8 = 0, FR_ROUTING_MFD = 1 } fr_routing_kind;

/* Operation codes for fr_workspace_size. */
typedef enum {
    FR_OP_RECEIVERS = 0,
    FR_OP_ACCUMULATE = 1,
    FR_OP_ADJOINT = 2,
    FR_OP_MASS_BALANCE = 3,
    FR_OP_ROUTE = 4, /* receivers + accumulate in one call (fr_route_d8) */
    FR_OP_MFD = 5,   /* any operation on an MFD routing (fr_accumulate, fr_route_mfd,
                        fr_route_adjoint): the common workspace plus the fractions of
                        every cell, 32 bytes per cell */
    FR_OP_FILL = 6   /* fr_fill: 256 bytes plus two bytes per 64x32 tile */
} fr_op;

/*
 * Local flow routing, D8 (Sec. 2.1, footnote 2; App. A first paragraph).
 *   dem       [ny*nx] float32 elevations (metres).
 *   nx, ny    grid size, both >= 1, nx*ny < 2^40.
 *   dx        grid spacing (> 0, finite); only the slope rule depends on it.
 *   flags     FR_EDGE_*, FR_D8_*, FR_D4, FR_CHECK_FINITE.
 *   dir_out   [ny*nx] uint8: receiver code 0..7 or FR_SINK.
 *   indeg_out [ny*nx] uint8 or NULL: number of donors of each cell (0..8).
 * Results are bit-identical to the rule stated above.
 */
fr_status fr_receivers_d8(const float* dem, int64_t nx, int64_t ny, double dx, uint32_t flags,
                          uint8_t* dir_out, uint8_t* indeg_out, void* stream);

/*
 * Local flow routing, multiple flow directions (App. A: water split among
 * the lower neighbours with fractions f_k; Freeman-style slope weights).
 *   f_k = s_k^p / sum_j s_j^p over strictly lower neighbours j,
 *   s_k = (z_c - z_k) / d_k, d_k = dx or sqrt(2)*dx.
 *   mask_out  [ny*nx] uint8: bit k set iff neighbour k receives water
 *             (0 = sink).
 *   frac_out  [ny*nx*8] float32 or NULL: f_k per cell and code, 0 where bit k
 *             is clear: f_k = u_k * (1/S) with the weights u_k = s_k^p, their
 *             sum S in a fixed pairwise order and 1/S as two-float, each f_k
 *             rounded once to fp32.  These are the fractions every MFD
 *             operation of this library uses.
 *   indeg_out [ny*nx] uint8 or NULL: number of donors.
 *   p         exponent, 0 < p <= FR_MFD_MAX_P (1.1 in the benchmark configuration).
 */
fr_status fr_receivers_mfd(const float* dem, int64_t nx, int64_t ny, double dx, double p,
                           uint32_t flags, uint8_t* mask_out, float* frac_out,
                           uint8_t* indeg_out, void* stream);

/* Routing description consumed by fr_accumulate / fr_route_adjoint /
 * fr_mass_balance.  All pointers are device pointers. */
typedef struct {
    int32_t kind;         /* FR_ROUTING_D8 or FR_ROUTING_MFD */
    int32_t reserved;     /* must be 0 */
    int64_t nx, ny;
    const uint8_t* dir;   /* D8: [ny*nx] codes from fr_receivers_d8 */
    const uint8_t* mask;  /* MFD: [ny*nx] receiver masks from fr_receivers_mfd */
    const float* dem;     /* MFD: [ny*nx] elevations; the fractions are computed
                             from them into the workspace (the arithmetic of
                             fr_receivers_mfd's frac_out) */
    double dx;            /* MFD: grid spacing */
    double p;             /* MFD: slope exponent */
    uint32_t flags;       /* MFD: the flags given to fr_receivers_mfd; D8: 0 or one of
                             FR_GLOBAL_WALKERS / FR_GLOBAL_SKELETON */
    uint32_t reserved2;   /* must be 0 */
} fr_routing;

/*
 * Global flow routing: w = A^{-1} r (Sec. 2.2), the exact result of the
 * high-to-low algorithm (Sec. 2.1, Eq. high-to-low-procedure) computed in
 * parallel.  Every cell holds its own rain plus everything its donors pass
 * on; sinks keep their water.
 *   rain      [ny*nx] float32 >= 0, or NULL for unit rain (1 per cell).
 *   w_out     [ny*nx] float32 or NULL: water per cell, the leading word of a
 *             compensated two-float sum (relative error against an FP64 solve
 *             about 1e-7 for D8 and MFD: the rounding of the leading word, plus
 *             the fp32 fractions for MFD).
 *   w_lo_out  [ny*nx] float32 or NULL: trailing word of that sum
 *             (w ~= w_out + w_lo_out).
 *   area_out  [ny*nx] uint64 or NULL: D8 only -- unit-rain drainage area in
 *             cells (Sec. 1, "a note on terminology"), exact.  Ignores rain.
 * At least one output must be non-NULL.  Requires ws of
 * fr_workspace_size(FR_OP_ACCUMULATE, nx, ny, flags) bytes for D8,
 * fr_workspace_size(FR_OP_MFD, nx, ny, flags) for MFD.
 * A routing graph with a cycle leaves FR_ERR_NO_PROGRESS in the status word.
 */
fr_status fr_accumulate(const fr_routing* routing, const float* rain, float* w_out,
                        float* w_lo_out, uint64_t* area_out, void* ws, size_t ws_bytes,
                        void* stream);

/*
 * Depression filling, the step before the path: the paper routes a
 * depression-filled DEM (Sec. 4).  filled_out receives the least surface
 * F >= dem that keeps every edge cell at its own elevation and gives every
 * interior cell a neighbour (of 8) lower by at least one fp32 step:
 *     F = dem on the edge,  F_c = max(dem_c, succ(min over neighbours of F_n)),
 * succ(x) the next fp32 value above x.  D8 routing on F (fr_receivers_d8,
 * default flags) then has sinks only on the edge.  The result is unique and
 * bit-reproducible.
 *   dem          [ny*nx] float32, finite (FR_CHECK_FINITE checks it).
 *   flags        0 or FR_CHECK_FINITE.
 *   filled_out   [ny*nx] float32, not overlapping dem.
 *   max_sweeps   >= 1: relaxation sweeps over 64x32 tiles allowed; a sweep
 *                that changes nothing ends the call.  FR_ERR_NO_PROGRESS if
 *                the surface is still moving after max_sweeps (filled_out
 *                then holds an upper bound of F).
 *   sweeps_out   host int32 or NULL: sweeps run, the last one changing nothing.
 * Workspace: fr_workspace_size(FR_OP_FILL, nx, ny, flags).
 * Synchronises the stream after every batch of eight sweeps.
 */
fr_status fr_fill(const float* dem, int64_t nx, int64_t ny, uint32_t flags, float* filled_out,
                  int32_t max_sweeps, int32_t* sweeps_out, void* ws, size_t ws_bytes,
                  void* stream);

/*
 * The paper's own parallel solver, run on one GPU (Sec. 2.4, 3.3, 3.4,
 * App. B.1): Richardson iteration for the "I+X" form of A w = r,
 *     w^(l+1) = T(w^(l)),  T(w) = D^{-1} (r + R w),  w^(0) = 0
 * (Eq. richardson-I+X), with 64x32 tiles as the subdomains: D^{-1} is each
 * tile's exact high-to-low solve and R w passes water across tile
 * boundaries.  order = 1 is I+X.  order = 2 is the (I-X)(I+X) scheme of
 * Sec. 3.4: one Richardson step on the preconditioned system equals two
 * applications of T; order = k applies T k times per iteration (the longer
 * preconditioner series Sec. 3.4 mentions).  A stream crossing tile
 * boundaries C times is exact after C + 1 applications of T, that is after
 * ceil((C + 1) / order) iterations.  The loop stops at the first sweep that
 * changes no value; the result equals fr_accumulate's up to the order of
 * additions (also fixed here).  Offered as the paper's method for
 * comparison: fr_accumulate reaches the exact result in two launches.
 *   w_out, w_lo_out  as fr_accumulate (w_out required).
 *   order            1 .. 64.
 *   max_iterations   >= 1; FR_ERR_NO_PROGRESS if more would be needed.
 *   iterations_out   host int32 or NULL: iterations until exact.
 * Synchronises the stream after every sweep.  Workspace as fr_accumulate.
 */
fr_status fr_accumulate_richardson(const fr_routing* routing, const float* rain, float* w_out,
                                   float* w_lo_out, int32_t order, int32_t max_iterations,
                                   int32_t* iterations_out, void* ws, size_t ws_bytes,
                                   void* stream);

/*
 * Receivers + accumulation in one call (D8): the direction grid goes to
 * dir_out if non-NULL, else to the workspace.  Outputs as fr_accumulate.
 * Workspace: fr_workspace_size(FR_OP_ROUTE, nx, ny, flags).
 */
fr_status fr_route_d8(const float* dem, int64_t nx, int64_t ny, double dx, uint32_t flags,
                      const float* rain, float* w_out, float* w_lo_out, uint64_t* area_out,
                      uint8_t* dir_out, void* ws, size_t ws_bytes, void* stream);

/*
 * fr_route_d8 without a caller-supplied workspace, for callers that cannot
 * allocate device memory: a plugin host that passes only input and output
 * buffers, an application whose own pool allocator has reserved the device
 * memory, or a loop that cannot take cudaMalloc/cudaFree's implicit device
 * synchronisation.  The paper has no counterpart; this is an interface
 * convenience of this library.
 *   Arguments, outputs and results as fr_route_d8 (all data pointers are
 *   device pointers; dir_out may be NULL).
 *   Limit: nx*ny <= FR_NOALLOC_MAX_CELLS; larger grids return
 *   FR_ERR_INVALID_ARG before any device work.
 *   Scratch: one file-scope device array of about 22 bytes per cell of that
 *   limit (about 23 MB), which every GPU that loads the library holds until
 *   the process exits.  The first call on a device looks up the array's
 *   address there (cudaGetSymbolAddress, with that device current); make that
 *   first call before any stream capture.  No call allocates or frees device
 *   memory.
 *   Sharing: every call on a device uses the same array and finds the last
 *   call's contents in it; the parts that must start at zero are cleared on
 *   the caller's stream at the start of each call.  Calls whose GPU work
 *   overlaps (different streams, or different host threads on one device)
 *   race on the array and give wrong results; serialise them.
 *   Device-side errors (a cycle in the routing) are not reported: the status
 *   word lives in the array, which fr_get_status cannot address.  Argument
 *   errors are returned as usual.
 *   The array's address is looked up once per device and kept: do not call
 *   this after a device reset (cudaDeviceReset) in the same process.
 */
#define FR_NOALLOC_MAX_CELLS ((int64_t)1 << 20)
fr_status fr_route_d8_noalloc(const float* dem, int64_t nx, int64_t ny, double dx, uint32_t flags,
                              const float* rain, float* w_out, float* w_lo_out,
                              uint64_t* area_out, uint8_t* dir_out, void* stream);

/* Receivers + accumulation in one call (MFD): masks and fractions in one
 * pass, then the accumulation.  mask_out may be NULL.
 * Workspace: fr_workspace_size(FR_OP_MFD, nx, ny, flags). */
fr_status fr_route_mfd(const float* dem, int64_t nx, int64_t ny, double dx, double p,
                       uint32_t flags, const float* rain, float* w_out, float* w_lo_out,
                       uint8_t* mask_out, void* ws, size_t ws_bytes, void* stream);

/*
 * Adjoint of global flow routing.  With g = A^{-T} gbar (the transposed
 * system: each cell's adjoint equals its own gbar plus the fraction-weighted
 * adjoints of its receivers, so it is solved from the sinks upstream):
 *   dLdr = g                              (dL/d rain)
 *   dLdz = g^T (dW/dz) w                  (MFD only; through the fractions,
 *                                          lower sets held fixed)
 *   w, w_lo   forward result (w_lo may be NULL); used for gbar at sinks and
 *             for dLdz.
 *   dLdw      [ny*nx] float32 = gbar, or NULL for L = sum over sinks of w^2
 *             (gbar = 2 w at sinks, 0 elsewhere).
 *   dLdr_out  [ny*nx] float32 (required).
 *   dLdz_out  [ny*nx] float32 or NULL; must be NULL for D8 (the D8 routing is
 *             piecewise constant in z, so dL/dz = 0 almost everywhere).
 * Workspace: fr_workspace_size(FR_OP_ADJOINT, nx, ny, flags) for D8,
 * fr_workspace_size(FR_OP_MFD, nx, ny, flags) for MFD.
 */
fr_status fr_route_adjoint(const fr_routing* routing, const float* w, const float* w_lo,
                           const float* dLdw, float* dLdr_out, float* dLdz_out, void* ws,
                           size_t ws_bytes, void* stream);

/*
 * Mass balance (Sec. 4: the water leaving through the sinks equals the total
 * rain).  Writes three doubles to out_dev (device memory):
 *   out_dev[0] = sum over sinks of (w + w_lo)   (0 if w is NULL)
 *   out_dev[1] = sum of rain (nx*ny for unit rain)
 *   out_dev[2] = sum over sinks of area         (0 if area is NULL), exact
 * Sinks are the cells whose routing byte is FR_SINK (D8) or 0 (MFD).
 * The reduction order is fixed, so repeated calls give identical bits.
 * Workspace: fr_workspace_size(FR_OP_MASS_BALANCE, nx, ny, flags).  With
 * FR_SINK_SUMS_IN_WORKSPACE (D8 routings; w NULL, area given) the area term
 * comes from the records the accumulation left in the same workspace.
 */
fr_status fr_mass_balance(const fr_routing* routing, const float* rain, const float* w,
                          const float* w_lo, const uint64_t* area, double* out_dev, void* ws,
                          size_t ws_bytes, void* stream);

/* One independent DEM of a batch (all pointers device pointers). */
typedef struct {
    const float* dem;   /* [ny*nx] */
    const float* rain;  /* [ny*nx] or NULL (unit rain) */
    float* w_out;       /* [ny*nx] or NULL */
    float* w_lo_out;    /* [ny*nx] or NULL */
    uint64_t* area_out; /* [ny*nx] or NULL; D8 only */
    uint8_t* route_out; /* [ny*nx] direction codes (D8) / masks (MFD), required */
    int64_t nx, ny;
    double dx;
} fr_tile;

/*
 * Batched routing of many independent DEMs of uneven size (receivers +
 * accumulation for every tile) with one launch per stage over all tiles,
 * persistent CTAs taking work from device-side counters; the sequence reads
 * no host memory when it executes and can be captured in a CUDA graph.
 * At most 2^24 - 1 tiles per call.  All
 * tiles must request the same outputs (w_out / area_out set for all or none;
 * area_out only with FR_ROUTING_D8, w_out required with FR_ROUTING_MFD).
 * flags: FR_EDGE_ROUTE; with FR_ROUTING_D8 also FR_D8_LOWEST and FR_D4; with
 * FR_ROUTING_MFD also FR_DINF (no FR_CHECK_FINITE).
 *   tiles_host  [ntiles] host array (read during the call only).
 *   tiles_dev   [ntiles] device copy of the same array, provided by the
 *               caller (so that no host memory is read at execution time).
 *   kind        FR_ROUTING_D8 or FR_ROUTING_MFD; p the MFD exponent.
 * Workspace: fr_batch_workspace_size(tiles_host, ntiles, kind, flags).
 */
fr_status fr_route_batch(const fr_tile* tiles_host, const fr_tile* tiles_dev, int32_t ntiles,
                         int32_t kind, double p, uint32_t flags, void* ws, size_t ws_bytes,
                         void* stream);
size_t fr_batch_workspace_size(const fr_tile* tiles_host, int32_t ntiles, int32_t kind,
                               uint32_t flags);

/*
 * Autotuner of the batched route: runs fr_route_batch with several CTA counts
 * for its persistent receiver stage and, for D8, each inner-tile geometry of
 * the local stage (128x32, 64x32, 96x48), synchronising the stream after each
 * trial, and keeps the fastest for later fr_route_batch calls of the same
 * kind in this process.  Same arguments as fr_route_batch; not for use during
 * stream capture.  The outputs hold a valid result afterwards.
 */
fr_status fr_batch_autotune(const fr_tile* tiles_host, const fr_tile* tiles_dev, int32_t ntiles,
                            int32_t kind, double p, uint32_t flags, void* ws, size_t ws_bytes,
                            void* stream);

/*
 * Receiver indices from D8 codes: out[i] = linear index (y*nx + x) of cell
 * i's receiver, or -1 where cell i is a sink (or its code points out of the
 * grid).  The receiver array r(i) of Sec. 2.1 in index form, for callers that
 * work with indices rather than the direction bytes of fr_receivers_d8.
 *   dir          [ny*nx] uint8 codes (fr_receivers_d8).
 *   index_bytes  4 (int32; requires nx*ny <= INT32_MAX) or 8 (int64).
 *   idx_out      [ny*nx] int32 or int64.
 * Needs no workspace.
 */
fr_status fr_receiver_index(const uint8_t* dir, int64_t nx, int64_t ny, int32_t index_bytes,
                            void* idx_out, void* stream);

/*
 * Time limit of device-side waits (the grid barrier between the rounds of the
 * MFD and adjoint global phases), in nanoseconds of the GPU's global timer; a
 * wait that runs out leaves FR_ERR_NO_PROGRESS in the status word and the
 * kernel returns.  Applies to calls enqueued after it, in every thread of the
 * process.  Default 10 s.  Returns the previous limit.
 */
uint64_t fr_set_wait_limit(uint64_t ns);

/* Workspace bytes an operation needs for an nx-by-ny grid (0 if the sizes
 * are invalid).  FR_OP_RECEIVERS needs none. */
size_t fr_workspace_size(int32_t op, int64_t nx, int64_t ny, uint32_t flags);

/* Synchronises `stream`, then reads and clears the device status word kept
 * in the workspace of the last call that used `ws`. */
fr_status fr_get_status(const void* ws, size_t ws_bytes, void* stream);

/* Static English description of a status code. */
const char* fr_status_string(fr_status s);

/* Library version as major*10000 + minor*100 + patch. */
int32_t fr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FR_H */

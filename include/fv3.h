/*
 * fv3.h -- C-ABI of the GB300 FV3 acoustic-substep library (libfv3.so).
 *
 * What it computes: the nonhydrostatic acoustic substep of the FV3 dynamical
 * core on a doubly-periodic tile or on the six-tile gnomonic cubed sphere
 * (arxiv 2205.04148, Section II: the innermost loop, integrating on
 * Lagrangian surfaces, with halo exchanges at several execution points;
 * Section IX-B: riem_solver_c; Section IX-C: fv_tp_2d; Section V-C: halo
 * exchange with the orientation transform between cube faces).  The paper
 * gives no equation; the discretisation is the one documented with the
 * library (readings R1-R13: PPM transport with a monotone limiter, Lin-Rood
 * splitting, del-4 damping, a semi-implicit tridiagonal column solve, the
 * contour-integral C-grid pressure gradient).
 *
 * Conventions
 *  - Fields live on the device in the library layout: every member (ensemble
 *    state) has nt tiles (1 periodic, 6 cube) of n x n cells and nz levels
 *    with a halo of 3; each plane has `rows` rows of `pitch` elements and
 *    element (i, j) of the interior sits at (j + 3) * pitch + ox + i (i, j may
 *    be -3 .. n + 3).  A 3-D field is [tile][level][plane]; the fields of all
 *    members are concatenated at member offsets.  Query the layout with
 *    fv3_get_layout, the element count of a field with fv3_field_elems.
 *  - Staggering (D-grid): u, the x-wind, on y-faces (i in [0,n), j in [0,n]);
 *    v, the y-wind, on x-faces (i in [0,n], j in [0,n)); w, delp, pt, delz and
 *    tracers at cell centres.  pt is temperature (K), delp the layer pressure
 *    thickness (Pa), delz the (negative) layer height thickness (m), k = 0 the
 *    model top.  Faces on a tile edge are stored by both tiles; the tile with
 *    the lower index owns them (periodic: faces i = 0, j = 0).
 *  - Element type: double (FV3_FP64) or float (FV3_FP32 and FV3_FP32_M64,
 *    "FP32-bulk": all stencils in FP32, the column solve and global sums in
 *    FP64), fixed at fv3_init_grid.  FV3_FP32 reads FP32 copies of the metric
 *    terms (areas, lengths, grid-angle sin/cos, Coriolis); FV3_FP32_M64 keeps
 *    them in FP64 and forms every product with a metric term in FP64, rounding
 *    to FP32 where the result is stored.
 *  - Ownership: the caller allocates and owns the state buffers (device
 *    memory, base address aligned to 128 bytes) and the streams; the library
 *    owns the metric terms, halo plans, intermediates, solver scratch and
 *    CUDA graphs, released by fv3_destroy.
 *  - Streams: every call is stream-ordered on `stream` (a cudaStream_t; 0 is
 *    the legacy default stream) and does not synchronise unless stated.
 *  - Errors: no call aborts.  Every call validates its arguments and returns a
 *    status; fv3_last_error returns a message for the last failure of a
 *    context.  Conditions detected by kernels (Courant number >= 1, too many
 *    tracer subcycles) are latched in a device status word and reported by
 *    fv3_check_status.
 */
#ifndef FV3_H
#define FV3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fv3_ctx fv3_ctx;
typedef void* fv3_stream; /* cudaStream_t */

typedef enum {
  FV3_OK = 0,
  FV3_ERR_ARG = -1,         /* null pointer or value out of range */
  FV3_ERR_SHAPE = -2,       /* sizes inconsistent with the context */
  FV3_ERR_ALIGN = -3,       /* buffer base not 128-byte aligned */
  FV3_ERR_CUDA = -4,        /* a CUDA call failed (message in fv3_last_error) */
  FV3_ERR_NONFINITE = -5,   /* non-finite value found */
  FV3_ERR_CFL = -6,         /* a Courant number reached 1 */
  FV3_ERR_TIMEOUT = -7,     /* a bounded device wait gave up */
  FV3_ERR_UNSUPPORTED = -8  /* option not built */
} fv3_status;

enum { FV3_GRID_PERIODIC = 0, FV3_GRID_CUBED = 1 };
enum { FV3_FP64 = 0, FV3_FP32 = 1, FV3_FP32_M64 = 2 };
/* field kinds: cell levels, x-face levels, y-face levels, cell interfaces (nz+1) */
enum { FV3_KIND_CELL = 0, FV3_KIND_XFACE = 1, FV3_KIND_YFACE = 2, FV3_KIND_IFACE = 3 };
/* fv3_halo_fill field mask bits */
enum {
  FV3_HALO_WIND = 1,  /* u, v (D-grid vector pair, rotated across cube edges) */
  FV3_HALO_W = 2,
  FV3_HALO_DELP = 4,
  FV3_HALO_PT = 8,
  FV3_HALO_DELZ = 16,
  FV3_HALO_TRACERS = 32
};

typedef struct {
  int grid_type;         /* FV3_GRID_PERIODIC or FV3_GRID_CUBED */
  int npx;               /* cells per tile edge (all members, if member_npx is NULL); >= 8 */
  int npz;               /* vertical levels; >= 2 */
  int n_members;         /* independent states advanced together; >= 1 */
  const int* member_npx; /* host array [n_members] of per-member npx, or NULL */
  int precision;         /* FV3_FP64, FV3_FP32 or FV3_FP32_M64 */
  double dx;             /* periodic grid spacing (m) */
  double radius;         /* sphere radius (m), cube only */
  double omega;          /* rotation rate (1/s), cube only */
} fv3_grid_desc;

typedef struct {
  void *u, *v, *w, *delp, *pt, *delz; /* device, library layout, all members */
  void* const* q;                     /* host array of nq device tracer fields */
  int nq;                             /* 0 .. 16 */
} fv3_state;

typedef struct {
  double dt;     /* acoustic substep (s) */
  int n_split;   /* substeps per remapping step (fv3_run_dyn) */
  int nord;      /* damping order: 1 (del-4) */
  int hord;      /* face values: 0 monotone PPM; 1 learned network for delp, pt and tracers */
  double d4_bg;  /* damping coefficient (0.12) */
  double a_imp;  /* implicit weight of the column solve (1 = fully implicit) */
  double dz_min; /* minimum layer thickness (m) */
  double ptop;   /* model-top pressure (Pa) */
  double grav, rdgas, cp_air;
  const void* mlp; /* hord 1: device float[1313] network parameters (see fv3_mlp_forward) */
  int remap;       /* 1: fv3_run_dyn ends every remapping step with fv3_vertical_remap */
  int nh_full;     /* 1: each acoustic substep ends with update_dz_d, riem_solver3 and the
                      D-grid nonhydrostatic pressure gradient (reading R17; Fig. 2) */
  int d2c_ord;     /* C-grid winds in c_sw from the D-grid winds: 2 (mean of the four
                      surrounding values) or 4 (four-point Lagrange along, then across;
                      reading R18); 0 means 2 */
  double d2_bg;    /* divergence damping of the D-grid winds (reading R19): background
                      coefficient (0: off) */
  double dddmp;    /* and Smagorinsky coefficient on the deformation (0: off); the
                      damping coefficient is min area x max(d2_bg, min(0.2, dddmp dt |def|)) */
} fv3_params;

typedef struct {
  int n, nz, ntiles;    /* cells per tile edge, levels, tiles */
  int pitch, rows, ox;  /* plane geometry (elements) */
  long long plane;      /* elements per plane */
  long long offset3;    /* member offset in CELL / XFACE / YFACE fields */
  long long offseti;    /* member offset in IFACE fields */
} fv3_layout;

/* Build the grid (metric terms in FP64, Section II), the halo plans (Section
 * V-C) and all internal buffers.  *out receives the context.  Returns
 * FV3_ERR_ARG / FV3_ERR_SHAPE for bad descriptors, FV3_ERR_CUDA when device
 * memory cannot be had. */
fv3_status fv3_init_grid(fv3_ctx** out, const fv3_grid_desc* desc, fv3_stream stream);

/* Release every library-owned resource of ctx (NULL is allowed). */
void fv3_destroy(fv3_ctx* ctx);

/* Message of the last failure on ctx ("" if none; a static string if ctx is NULL). */
const char* fv3_last_error(const fv3_ctx* ctx);

/* Elements (of fv3_elem_size bytes) of one field of `kind`, all members. */
size_t fv3_field_elems(const fv3_ctx* ctx, int kind);
size_t fv3_elem_size(const fv3_ctx* ctx);

/* Plane geometry and offsets of member `member`. */
fv3_status fv3_get_layout(const fv3_ctx* ctx, int member, fv3_layout* out);

/* Copy a dense array of member `member` into (import) or out of (export) a
 * field in the library layout.  Dense layout [tile][level][nj][ni] with
 * (ni, nj) = (n, n) cells, (n+1, n) x-faces, (n, n+1) y-faces, levels nz (nz+1
 * for IFACE).  dense_is_host:
 *   FV3_DENSE_DEVICE (0): the dense array is device memory (a pack kernel);
 *   FV3_DENSE_HOST (1): host memory, copied through a staging buffer; host
 *     exports return after the copy completed;
 *   FV3_DENSE_HOST_ASYNC (2): page-locked host memory, asynchronous: the
 *     call returns once the copy is enqueued on `stream`, and the host array
 *     must stay untouched until the stream has passed it.  With dense
 *     elements of the library's precision (dense_is_double = 1 for FP64, 0
 *     for FP32) one 3-D copy-engine transfer between the dense array and the
 *     field's interior, no kernel (so it never waits for multiprocessors held
 *     by a substep on another stream).  Otherwise a contiguous copy into one
 *     of four device staging slots plus the converting pack kernel, both on
 *     `stream`; a slot is reused only after its previous copy completed (an
 *     event, whatever stream that ran on), and is allocated on first use with
 *     room for any field of the context.  Lets a caller overlap the I/O of
 *     one state with the substeps of another on a second stream.
 *   Any other value: FV3_ERR_ARG.
 * dense_is_double: dense elements are double (else float).
 * Errors: FV3_ERR_ARG (NULL buffer, bad kind or member), FV3_ERR_ALIGN (field
 * not 128-byte aligned), FV3_ERR_CUDA (a copy or launch failed). */
enum { FV3_DENSE_DEVICE = 0, FV3_DENSE_HOST = 1, FV3_DENSE_HOST_ASYNC = 2 };
fv3_status fv3_import(fv3_ctx* ctx, int kind, void* field, const void* dense, int dense_is_host, int dense_is_double,
                      int member, fv3_stream stream);
fv3_status fv3_export(fv3_ctx* ctx, int kind, const void* field, void* dense, int dense_is_host, int dense_is_double,
                      int member, fv3_stream stream);

/* One entry of a halo plan: the slot at element offset `dst` of a level
 * plane of tile `dst_tile` takes the value at offset `src` of tile `src_tile`
 * (same level) times `sign`; sign 0: no value exists (a cube-corner slot, set
 * to NaN).  Offsets index one padded plane (`pitch` elements per row, see
 * fv3_layout).  Vector plans: flags bit 0 set when the slot is in the y-face
 * array (u of the D-grid pair, vc of the C-grid pair), bit 1 when the source
 * is. */
typedef struct {
  int32_t dst, src, dst_tile, src_tile, sign, flags;
} fv3_halo_entry;
enum { FV3_PLAN_CELL = 0, FV3_PLAN_DGRID = 2, FV3_PLAN_CGRID = 3 };

/* The halo plan of kind FV3_PLAN_CELL (scalars, halo 3), FV3_PLAN_DGRID (the
 * D-grid winds: v on x-faces, u on y-faces) or FV3_PLAN_CGRID (the C-grid
 * winds: uc on x-faces, vc on y-faces) of member `member` of the grid `desc`:
 * the plan fv3_halo_fill applies (Section V-C), built on the host without a
 * device.  For a caller that places the tiles of a member on different
 * devices, every entry whose src_tile lives elsewhere is a value to receive
 * (the paper's halo exchange between ranks).  Writes min(total, cap) entries
 * to `out` (which may be NULL when cap is 0), *total = the number of entries,
 * and, if `layout` is not NULL, the member's plane geometry for the
 * descriptor's precision (its offsets are those of fv3_get_layout).  Errors:
 * as fv3_init_grid for the descriptor (FV3_ERR_ARG, FV3_ERR_SHAPE);
 * FV3_ERR_ARG for a bad member, kind or NULL total. */
fv3_status fv3_halo_plan(const fv3_grid_desc* desc, int member, int kind, fv3_halo_entry* out, size_t cap,
                         size_t* total, fv3_layout* layout);

/* Device side of a halo exchange between ranks that hold different tiles of
 * one member (Section V-C; tiles on several GPUs).  A rank's part of the plan
 * of fv3_halo_plan, split by tile owner, is lists of element offsets (int64,
 * device) into its field buffer (device, elements of elem_size 4 or 8 bytes):
 *   fv3_halo_gather:  out[e] = sign[e] * field[src[e]]  (the message to a
 *                     peer; sign int8 +-1, NULL for +1);
 *   fv3_halo_scatter: field[dst[e]] = in[e]  (a peer's message; in NULL
 *                     writes NaN, for halo slots that have no value);
 *   fv3_halo_copy:    field[dst[e]] = sign[e] * field[src[e]]  (slots filled
 *                     from the rank's own tiles; dst and src must be disjoint
 *                     sets, as halo slots are filled from interior values).
 * e < count; count = 0 is a no-op.  The messages travel between ranks through
 * the caller's transport.  Errors: FV3_ERR_ARG (count < 0, elem_size not 4 or
 * 8, a NULL array), FV3_ERR_CUDA (launch failure). */
fv3_status fv3_halo_gather(const void* field, int elem_size, const int64_t* src, const int8_t* sign, int64_t count,
                           void* out, fv3_stream stream);
fv3_status fv3_halo_scatter(void* field, int elem_size, const int64_t* dst, const void* in, int64_t count,
                            fv3_stream stream);
fv3_status fv3_halo_copy(void* field, int elem_size, const int64_t* src, const int64_t* dst, const int8_t* sign,
                         int64_t count, fv3_stream stream);

/* Fill the halos (strips of 3, owner copies of shared tile-edge faces, cube
 * corner slots) of the fields selected by `field_mask` (FV3_HALO_*), all
 * members: Section V-C, on the device. */
fv3_status fv3_halo_fill(fv3_ctx* ctx, const fv3_state* state, unsigned field_mask, fv3_stream stream);

/* One acoustic substep (Section II): halo fill, c_sw, update_dz_c,
 * riem_solver_c, p_grad_c, C-grid halo fill, d_sw with fv_tp_2d and del-4
 * damping.  u, v, w, delp, pt are advanced in place (delz and tracers are
 * inputs only). */
fv3_status fv3_acoustic_substep(fv3_ctx* ctx, const fv3_state* state, const fv3_params* params, fv3_stream stream);

/* n_steps remapping steps (Section II): each is params->n_split acoustic
 * substeps with accumulated mass fluxes and Courant numbers, then tracer
 * transport (tracer_2d) of the state's nq tracers.  The step is captured once
 * as a CUDA graph per state pointers and parameters and replayed; the graphs
 * of the last four such keys are kept (least recently used evicted). */
fv3_status fv3_run_dyn(fv3_ctx* ctx, const fv3_state* state, const fv3_params* params, int n_steps,
                       fv3_stream stream);

/* Vertical remapping (Section II: the model integrates on Lagrangian
 * surfaces and remaps them to reference levels; reading R16).  Every column of
 * every member: the reference layers are equally spaced in pressure between
 * params->ptop and the column's surface pressure (ptop + sum of delp, kept);
 * each field is reconstructed per layer as a monotone-limited parabola and
 * integrated exactly over the overlaps of the old and new layers.  delp
 * becomes the reference thickness; pt, w and the tracers are remapped as
 * mass-weighted means, delz through delz / delp (column height kept); u and v
 * on their face columns, whose interfaces are the means of the two adjacent
 * cell columns' interfaces.  Column mass, tracer and momentum integrals are
 * conserved to round-off.  The state is updated in place (the halo rings of
 * delp are filled, the other halos are left stale).  FP64 arithmetic for
 * both precisions.  Errors as fv3_acoustic_substep. */
fv3_status fv3_vertical_remap(fv3_ctx* ctx, const fv3_state* state, const fv3_params* params, fv3_stream stream);

/* fv_tp_2d alone (Section IX-C, "2-D mass-conserving flux-form transport";
 * readings R4-R6): the face fluxes of the scalar q for the given Courant
 * numbers and area fluxes -- Lin-Rood inner/outer PPM sweeps in both orders,
 * face value = mean of the two, flux = face value x area flux (x mass flux
 * when mfx/mfy are given) -- plus, when damp > 0, the del-4 damping flux
 * damp * (L_{i-1} - L_i) * dy/dxc with L the discrete Laplacian of q.  The same
 * transport runs inside fv3_acoustic_substep (d_sw) and fv3_run_dyn
 * (tracer_2d); this entry point exposes it for tests and module timings.
 *
 * All arrays are device arrays of the context's precision in the library
 * layout, every level of every tile of every member: q cell field
 * (FV3_KIND_CELL); crx, xfx, mfx, fx x-face fields (FV3_KIND_XFACE: between
 * cells i-1 and i); cry, yfx, mfy, fy y-face fields (FV3_KIND_YFACE).  mfx
 * and mfy: both NULL (area fluxes) or both set.  The halo rings of q, crx/cry,
 * xfx/yfx and mfx/mfy are filled by this call (C-grid vector rule for the
 * face pairs), so they are written as well as read; fx and fy receive the
 * interior faces.  |crx|, |cry| must not exceed 1 (not checked here; at 1 a
 * face passes its upwind cell's mean exactly).
 * Errors: FV3_ERR_ARG (NULL pointer, mfx without mfy, damp < 0 or not
 * finite), FV3_ERR_ALIGN (a pointer not 128-byte aligned). */
fv3_status fv3_fv_tp_2d(fv3_ctx* ctx, void* q, void* crx, void* cry, void* xfx, void* yfx, void* mfx, void* mfy,
                        double damp, void* fx, void* fy, fv3_stream stream);

/* Scan the interior of the state's fields (u, v, w, delp, pt, delz and the
 * tracers) of every member for NaN or Inf; synchronizes `stream` and returns
 * FV3_ERR_NONFINITE if one is found (else the pending status, as
 * fv3_check_status).  Failure detection without any device fault (no
 * counterpart in the paper). */
fv3_status fv3_check_finite(fv3_ctx* ctx, const fv3_state* state, fv3_stream stream);

/* Global mass sum(delp * area) per member in FP64 (Neumaier-compensated, fixed
 * order).  out_per_member: host array [n_members]; returns after the sum is
 * on the host. */
fv3_status fv3_mass_sum(fv3_ctx* ctx, const fv3_state* state, double* out_per_member, fv3_stream stream);

/* Synchronise `stream` and report (then clear) the kernel status word:
 * FV3_ERR_CFL, FV3_ERR_UNSUPPORTED (tracer subcycles beyond 4) or FV3_OK. */
fv3_status fv3_check_status(fv3_ctx* ctx, fv3_stream stream);

/* ---- test exports (same conventions) ---- */

/* Dense copy of one FP64 metric term of `member` into host memory: cells
 * (area, rarea, fA) [nt][n][n]; y-faces (dx, rdx, dyc, rdyc, cosy, siny)
 * [nt][n+1][n]; x-faces (dy, rdy, dxc, rdxc, cosx, sinx) [nt][n][n+1];
 * corners (fC, rareac) [nt][n+1][n+1]. */
fv3_status fv3_get_metric(fv3_ctx* ctx, const char* name, int member, double* dense_host);

/* Run the substep only up to stage `stop_after` (0 halo fill, 1 c_sw, 2
 * update_dz_c, 3 riem_solver_c, 4 p_grad_c, 5 everything) without advancing
 * the state, then copy an intermediate of member `member` to host (dense,
 * double): uc, fx1 (x-faces), vc, fy1 (y-faces), delpc, ptc, wc, delzc
 * (cells), pef, gz (interfaces). */
fv3_status fv3_stage(fv3_ctx* ctx, const fv3_state* state, const fv3_params* params, int stop_after,
                     fv3_stream stream);
fv3_status fv3_get_intermediate(fv3_ctx* ctx, const char* name, int member, double* dense_host, fv3_stream stream);

/* Enqueue only stage `stage` of the substep, `reps` times, on the current
 * intermediates (0 halo fill, 1 c_sw, 2 update_dz_c, 3 riem_solver_c, 4 pef/gz
 * halo + p_grad_c, 5 C-grid halo, 6 d_sw); run fv3_stage first so that its
 * inputs exist.  Used to time one kernel with events on `stream`; the state
 * is not advanced. */
fv3_status fv3_launch_stage(fv3_ctx* ctx, const fv3_state* state, const fv3_params* params, int stage, int reps,
                            fv3_stream stream);

/* Kernels the library has enqueued on ctx so far (graph replays included). */
long long fv3_kernel_launches(const fv3_ctx* ctx);

/* Machine calibration (paper Section IX-A: bandwidth test and copy stencil):
 * what = 0 FP64 multiply-add throughput, 1 FP32 multiply-add throughput, 2
 * copy stencil over one halo-padded FP64 3-D field of the context.  Enqueues
 * one launch on `stream` and returns its work (flops, or bytes read + written)
 * in *work_per_launch; time it with events on the same stream. */
fv3_status fv3_calibrate(fv3_ctx* ctx, int what, fv3_stream stream, double* work_per_launch);

/* Accuracy check of the kernels' FP64 helpers (no counterpart in the paper;
 * for tests).  Device arrays of n doubles.  what = 0: out = 1/x by the
 * Newton-refined hardware reciprocal the transport and the column solve use;
 * what = 1: out = ln((x + y) / x), the log pressure ratio (atanh series for
 * small y / (2x + y)); what = 2: out = y / ln((x + y) / x), the layer pressure
 * of the column solve's gas-law split (series of u / atanh(u) for small
 * u = y / (2x + y)); what = 3: out = 1/x from one reciprocal of x y (the
 * column solve's thickness and pressure-sum reciprocals together, x y in the
 * normal range); what = 4: out = x rounded to float and widened back to
 * double by the integer-pipe conversion of the column solve's FP32 inputs.
 * FV3_ERR_ARG for an unknown `what`, n < 0 or a NULL array;
 * FV3_ERR_CUDA if the launch fails. */
fv3_status fv3_math_check(int what, const double* x, const double* y, double* out, int n, fv3_stream stream);

/* Block shape (bx x by cells) and level chunk of the horizontal kernels
 * (c_sw, d_sw, tracer_2d).  Compiled shapes: 32x8, 32x16, 64x8, 16x16;
 * 1 <= kchunk <= npz.  Drops the cached remapping-step graphs.  Defaults at
 * fv3_init_grid: FP64 16x16, kchunk 1, persistent launches; FP32 32x8,
 * kchunk min(4, npz), one CTA per work item. */
fv3_status fv3_set_tiles(fv3_ctx* ctx, int bx, int by, int kchunk);
fv3_status fv3_get_tiles(const fv3_ctx* ctx, int* bx, int* by, int* kchunk);

/* on != 0: the horizontal kernels (c_sw, d_sw, tracer_2d) run as persistent
 * launches -- a grid of (SMs x resident blocks) CTAs that stride over the
 * work list of (member, tile, block, level chunk) items of all members --
 * instead of one CTA per item.  Drops the cached graph. */
fv3_status fv3_set_persistent(fv3_ctx* ctx, int on);
/* *on = the launch mode set by fv3_set_persistent or chosen by fv3_autotune. */
fv3_status fv3_get_persistent(const fv3_ctx* ctx, int* on);

/* Autotuner (the paper's transfer tuning, Section VII-B, as an empirical
 * search): times c_sw + d_sw on `state` for every compiled block shape,
 * level chunks 1, 4, 16 and both launch modes (one CTA per item, persistent),
 * keeps the fastest (fv3_set_tiles, fv3_set_persistent) and returns its
 * time per (c_sw + d_sw) in *best_ms (may be NULL).  Synchronises `stream`. */
fv3_status fv3_autotune(fv3_ctx* ctx, const fv3_state* state, const fv3_params* params, fv3_stream stream,
                        double* best_ms);

/* fv3_autotune for a shape that will be transferred to other grids (the
 * paper's transfer tuning, Section VII-B): only block shapes that cover every
 * tile size in sizes[n_sizes] (cells per tile edge) with whole blocks are
 * tried, when at least one does (the kernels have full-block instantiations
 * whose loops have compile-time extents); otherwise every shape.  Errors as
 * fv3_autotune, and FV3_ERR_ARG for n_sizes < 0, sizes NULL with n_sizes > 0,
 * or a size < 1. */
fv3_status fv3_autotune_for(fv3_ctx* ctx, const fv3_state* state, const fv3_params* params, fv3_stream stream,
                            double* best_ms, const int* sizes, int n_sizes);

/* ---- learned face values (reading R14; the paper has no learned part) ----
 * Network: 6 -> 32 -> 32 -> 1 with tanh, parameters float[1313] on the device
 * (W1[6][32] at 0, b1 at 192, W2[32][32] at 224, b2 at 1248, W3[32] at 1280,
 * b3 at 1312).  Inputs per face: the six cells of the PPM face stencil minus
 * their mean, over their standard deviation sig (+ 1e-12 |mean|).  The
 * learned face value is the plain PPM face value + sig * y, y the
 * mirror-symmetric network output; plain PPM where that value leaves the
 * range of the two cells next to the face or is negative.  Tensor-core
 * evaluation (bfloat16 operands, float accumulation, hardware tanh). */

/* y[n] = network(x[n][6]); symmetric != 0 averages x and the reversed x. */
fv3_status fv3_mlp_forward(const float* w, const float* x, int n, int symmetric, float* y, fv3_stream stream);

/* Floats of workspace fv3_mlp_grad needs for n samples. */
size_t fv3_mlp_work_floats(int n);

/* grad[1313] = d/dw sum_s 0.5 * weight * (ys(x_s) - t_s)^2 with the
 * mirror-symmetric network ys; *loss receives the sum (device pointers;
 * loss may be NULL).  Deterministic (fixed-order reduction). */
fv3_status fv3_mlp_grad(const float* w, const float* x, const float* t, int n, float weight, float* work,
                        float* grad, float* loss, fv3_stream stream);

/* The same gradient in float arithmetic without bfloat16 rounding (SIMT,
 * library tanhf): the reference the tensor-core gradient and the float
 * training path are checked against (no counterpart in the paper).  Work:
 * fv3_mlp_work_floats_fp32(n) floats.  Deterministic; slow (one thread per
 * parameter sums over the samples), meant for checks, not training. */
size_t fv3_mlp_work_floats_fp32(int n);
fv3_status fv3_mlp_grad_fp32(const float* w, const float* x, const float* t, int n, float weight, float* work,
                             float* grad, float* loss, fv3_stream stream);

/* Single-stencil exports of the FP64 transport's face arithmetic (readings R4
 * and R14; Section IX-C for the PPM face values), for forming training
 * targets and for tests.  q6: device double[n][6], six consecutive cell means
 * along a sweep, the face between q6[f][2] and q6[f][3]; cr: device double[n]
 * Courant numbers at that face (|cr| <= 1).  Outputs (device, each may be
 * NULL): plain[n] the plain PPM face value (edge values, limiter, swept mean
 * of the upwind cell's parabola, as inside fv3_fv_tp_2d); edge[n] the clamped
 * fourth-order edge value between q6[f][2] and q6[f][3]; x[n][6], sig[n] the
 * network inputs and standard deviation (float).  n = 0 is a no-op.  Errors:
 * FV3_ERR_ARG (q6 NULL, n < 0, cr NULL with plain requested), FV3_ERR_CUDA
 * (launch failure). */
fv3_status fv3_face_stencils(const double* q6, const double* cr, int n, double* plain, double* edge, float* x,
                             float* sig, fv3_stream stream);

/* Learned face values of n stencils as the FP64 transport forms them with
 * the network w (device float[1313]): value[n] (device) is the plain PPM face
 * value + sig * y where that lies in [min(q6[f][2], q6[f][3]), max(...)] and
 * is not negative, else the plain value.  Arguments as fv3_face_stencils. */
fv3_status fv3_learned_faces(const float* w, const double* q6, const double* cr, int n, double* value,
                             fv3_stream stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected, step >= 1) on
 * float master weights w with moments m, v. */
fv3_status fv3_mlp_adam(float* w, float* m, float* v, const float* grad, int step, float lr, fv3_stream stream);

/* Column solve of riem_solver_c for callers that cannot allocate device
 * memory (no counterpart in the paper).  Code that runs under a fixed,
 * pre-reserved memory budget, or inside a host framework that owns the whole
 * device pool, cannot create a context with fv3_init_grid (which allocates).
 * This entry point needs no context and calls no allocator: the caller passes
 * device arrays, level-major (element (k, col) at k * ncol + col), FP64:
 * inputs delpc, ptc, wc, delzc [nz][ncol]; outputs pef, gz [nz+1][ncol]; only
 * params->dt (the solve uses dt/2), ptop, grav, rdgas, cp_air and a_imp are
 * read.  Scratch is one fixed 32 MiB array inside the library's GPU image
 * (held on every GPU that loads the library until the process exits), so
 * 5 * nz * ncol must not exceed 4,194,304 (e.g. ncol <= 10485 at nz = 80);
 * larger sizes return FV3_ERR_SHAPE without launching.  The first call on a
 * device looks up the scratch address on that device; with lazy module
 * loading (the CUDA default) that lookup loads the library's module there and
 * so reserves the 32 MiB array and the kernel image.  Make that first call
 * (or any other fv3 call on the device) before entering a region where
 * nothing may be allocated, and before any stream capture; later calls
 * allocate nothing.  The looked-up address does not survive a device reset
 * (cudaDeviceReset): do not call this entry point across one.  All calls
 * share the one scratch array, so calls that may run at the same time on the
 * GPU (different streams, or host threads) race and must be ordered by the
 * caller; nothing in the scratch has to start at zero, every value read is
 * written first in the same call.  Errors: FV3_ERR_ARG (a NULL pointer;
 * dt, grav, a_imp, rdgas or ptop not positive; cp_air <= rdgas),
 * FV3_ERR_SHAPE (ncol < 1, nz < 2, or beyond the scratch), FV3_ERR_CUDA (the
 * address lookup or the launch failed). */
fv3_status fv3_riem_solver_c_noalloc(int ncol, int nz, const double* delpc, const double* ptc, const double* wc,
                                     const double* delzc, double* pef, double* gz, const fv3_params* params,
                                     fv3_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* FV3_H */

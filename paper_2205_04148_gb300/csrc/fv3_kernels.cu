// fv3_kernels.cu -- sm_103a kernels of one FV3 acoustic substep.
//
// arxiv 2205.04148, Section II (the acoustic substep: c_sw, riem_solver_c,
// p_grad_c, d_sw with halo exchanges between them), Section IX-B
// (riem_solver_c: semi-implicit tridiagonal column solve), Section IX-C
// (fv_tp_2d: 2-D mass-conserving flux-form transport), Section V-B (corner and
// edge specialisations), Section VII-A (I-contiguous layout, horizontal
// stencils with I on threadIdx.x, vertical solvers with K inside a thread;
// consecutive statements fused into one kernel with redundant computation of
// the halo they need).
//
// The paper prints no equation; the formulas are the design readings R1-R13
// (Colella-Woodward PPM with a monotone limiter, Lin-Rood inner/outer
// splitting, del-4 damping fluxes, Lin 1997 contour pressure gradient, a
// Chen-et-al.-style semi-implicit column).  Every kernel is templated on the
// arithmetic type R: double for the FP64 path, float for the FP32-bulk path
// (whose column solve still runs in double).
//
// Horizontal kernels: one CTA = one 2-D block (BX x BY cells) of one tile of
// one member, looping over a chunk of levels.  The block and its halo of 3
// live in shared memory; every phase is a 2-D loop over the range it must
// produce, separated by barriers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "fv3_kernels.cuh"
#include "fv3_math.cuh"
#include "fv3_mlp.cuh"

// The file is compiled as three translation units so that the two
// precisions' kernels build in parallel: FV3_TU=1 the shared host code and
// utility kernels, FV3_TU=64 the FP64 substep and tracer kernels, FV3_TU=32
// the FP32 ones.  Without FV3_TU it is all of them in one unit.
#ifndef FV3_TU
#define FV3_TU 0
#endif
#define FV3_TU_MAIN (FV3_TU == 0 || FV3_TU == 1)
#define FV3_TU_F64 (FV3_TU == 0 || FV3_TU == 64)
#define FV3_TU_F32 (FV3_TU == 0 || FV3_TU == 32)
#define FV3_TU_F32M64 (FV3_TU == 0 || FV3_TU == 33)

namespace fv3 {

template <typename R>
__device__ __forceinline__ R qnan();
template <>
__device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <>
__device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }

// *p += v for an element with one writer per launch: with v of the element's
// type an addition performed at the memory side (a reduction whose result
// is not read back: the same sum, without the load's round trip); with a
// wider v (FP64 metric products on an FP32 field) the sum is formed in the
// wider type and rounded once, as the expression p[0] + v is
template <typename R, typename T>
__device__ __forceinline__ void add_to(R* p, T v) {
  if constexpr (std::is_same_v<R, T>) atomicAdd(p, v);
  else *p = (R)((T)*p + v);
}

// sign and magnitude tests (FP64 on the integer pipe)
template <typename R>
__device__ __forceinline__ bool positive(R c) { return c > R(0); }
template <>
__device__ __forceinline__ bool positive<double>(double c) { return __double_as_longlong(c) > 0; }
// |c| < 1 (false for NaN; FP64 on the integer pipe)
template <typename R>
__device__ __forceinline__ bool below_one(R c) { return fabs(c) < R(1); }
template <>
__device__ __forceinline__ bool below_one<double>(double c) {
  return (__double_as_longlong(c) & 0x7fffffffffffffffLL) < 0x3ff0000000000000LL;
}
// the smaller of a and b, as fmin for numbers (FP64: compared on the
// integer pipe, on the order-preserving keys of the bit patterns)
template <typename R>
__device__ __forceinline__ R min_of(R a, R b) { return fmin(a, b); }
template <>
__device__ __forceinline__ double min_of<double>(double a, double b) { return okey(a) < okey(b) ? a : b; }
template <typename R>
__device__ __forceinline__ R magnitude(R c) { return fabs(c); }
template <>
__device__ __forceinline__ double magnitude<double>(double c) {
  return __longlong_as_double(__double_as_longlong(c) & 0x7fffffffffffffffLL);
}

// ------------------------------------------------------------------------
// PPM (reading R4)
// ------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R ppm_edge(R qm, R q0, R q1, R qp) {
  R al = R(7.0 / 12.0) * (q0 + q1) - R(1.0 / 12.0) * (qm + qp);
  return fmin(fmax(al, fmin(q0, q1)), fmax(q0, q1));
}

// A face's Courant number c as the sweeps keep it: w = 1 - |c|, the part of
// the upwind cell that does not cross the face in a step, carrying the sign
// of the upwind side (+w when c > 0: the cell before the face is upwind; -w
// when c <= 0; a zero weight keeps the side in its sign bit, see
// upwind_before).  Formed once per face, it spares every face value of every
// sweep and field a 1 - |c| of its own.  Requires |c| <= 1 (the Courant
// guard flags |c| >= 1).
template <typename R>
__device__ __forceinline__ R upwind_weight(R c) {
  const R w = R(1) - magnitude(c);
  return positive(c) ? w : -w;
}

// the side an upwind weight names: the sign bit (so that |c| = 1, w = 0,
// keeps its side: +0 before the face, -0 after it)
template <typename R>
__device__ __forceinline__ bool upwind_before(R cw) {
  if constexpr (sizeof(R) == 8) return __double_as_longlong(cw) >= 0;
  else return __float_as_int(cw) >= 0;
}

// a b + c with one rounding
template <typename R>
__device__ __forceinline__ R fmadd(R a, R b, R c) {
  if constexpr (sizeof(R) == 8) return fma(a, b, c);
  else return fmaf(a, b, c);
}

// the mean over the swept part of the upwind cell's limited parabola (mean
// qu, deviations bl and br at its two edges): qu + w (w (bl + br) - y), y the
// deviation at the cell's far edge from the face (bl when the cell before the
// face is upwind) -- the value of qu + (1 - |c|) (x - |c| (bl + br)), x the
// deviation at the near edge, since x - (bl + br) = -y
template <typename R>
__device__ __forceinline__ R swept_mean(R qu, R bl, R br, R cw) {
  const R w = magnitude(cw);
  const R y = upwind_before(cw) ? bl : br;
  return fmadd(w, fmadd(w, bl + br, -y), qu);
}

// face value at the face left of q[0] (between q[-s] and q[0]) for the
// upwind weight cw of the face; the upwind cell is picked first so the warp
// does one evaluation.
template <typename R>
__device__ __forceinline__ R ppm_face(const R* q, int s, R cw) {
  const R* p = upwind_before(cw) ? q - s : q;
  const R qu = p[0];
  R bl = ppm_edge(p[-2 * s], p[-s], p[0], p[s]) - qu;
  R br = ppm_edge(p[-s], p[0], p[s], p[2 * s]) - qu;
  ppm_limit(bl, br);
  return swept_mean(qu, bl, br, cw);
}

// FP64 specialisations (order-preserving integer keys, fv3_math.cuh)
template <>
__device__ __forceinline__ double ppm_edge<double>(double qm, double q0, double q1, double qp) {
  const double al = (7.0 / 12.0) * (q0 + q1) - (1.0 / 12.0) * (qm + qp);
  const long long k0 = okey(q0), k1 = okey(q1), ka = okey(al);
  const bool o = k0 < k1;
  const double lo = o ? q0 : q1, hi = o ? q1 : q0;
  const long long klo = o ? k0 : k1, khi = o ? k1 : k0;
  return ka < klo ? lo : (ka > khi ? hi : al);
}

template <>
__device__ __forceinline__ double upwind_weight<double>(double c) {
  const long long b = __double_as_longlong(c);
  const double w = 1.0 - __longlong_as_double(b & 0x7fffffffffffffffLL);
  return __longlong_as_double(__double_as_longlong(w) ^ (b > 0 ? 0LL : (long long)0x8000000000000000ULL));
}


// ------------------------------------------------------------------------
// per-tile metric view: element (i, j) at p[j * pitch + i]
// ------------------------------------------------------------------------
template <typename R>
struct TM {
  const R *area, *rarea, *fA, *dx, *rdx, *dyc, *rdyc, *cosy, *siny, *rsin2y, *dy, *rdy, *dxc, *rdxc, *cosx, *sinx,
      *rsin2x, *fC, *rareac, *wx, *wy, *kfx, *kcx, *kfy, *kcy;
  int pitch;
};
#define MT(name, j, i) __ldg(m.name + (long long)(j) * m.pitch + (i))

template <typename R>
__device__ __forceinline__ TM<R> tile_metric(const Metric<R>& M, const Geo& g, int t) {
  const long long o = g.off2 + (long long)t * g.plane + (long long)HALO * g.pitch + g.ox;
  TM<R> m;
  m.area = M.area + o; m.rarea = M.rarea + o; m.fA = M.fA + o;
  m.dx = M.dx + o; m.rdx = M.rdx + o; m.dyc = M.dyc + o; m.rdyc = M.rdyc + o;
  m.cosy = M.cosy + o; m.siny = M.siny + o; m.rsin2y = M.rsin2y + o;
  m.dy = M.dy + o; m.rdy = M.rdy + o; m.dxc = M.dxc + o; m.rdxc = M.rdxc + o;
  m.cosx = M.cosx + o; m.sinx = M.sinx + o; m.rsin2x = M.rsin2x + o;
  m.fC = M.fC + o; m.rareac = M.rareac + o;
  m.wx = M.wx + o; m.wy = M.wy + o;
  m.kfx = M.kfx + o; m.kcx = M.kcx + o; m.kfy = M.kfy + o; m.kcy = M.kcy + o;
  m.pitch = g.pitch;
  return m;
}

// the metric a kernel with metric type MR reads: the FP64 master copy, or
// the copy in the arithmetic precision
template <typename MR, typename A>
__device__ __forceinline__ Metric<MR> metric_sel(const A& a) {
  if constexpr (sizeof(MR) == 8) return a.Md;
  else return a.M;
}

// origin (i = j = 0) of level k of tile t in a [tile][nlev][plane] field
__device__ __forceinline__ long long fld0(const Geo& g, long long off, int nlev, int t, int k) {
  return off + ((long long)t * nlev + k) * g.plane + (long long)HALO * g.pitch + g.ox;
}

// CTA block and its shared-memory frame (halo 3 on every side)
struct Blk {
  int x0, x1, y0, y1, SX;
  __device__ __forceinline__ int L(int i, int j) const { return (j - y0 + 3) * SX + (i - x0 + 3); }
};

// 2-D loop over [ilo, ihi) x [jlo, jhi), flattened over all threads of the
// block so that every warp but the last is full (the ranges are a few cells
// wider than a warp; a row-per-warp loop would leave most lanes of a second
// pass idle, and on this GPU an FP64 warp instruction costs its full pipe
// time whatever its active lanes).  Runtime extents: row j = floor((e + 1/2)
// / w) from a float reciprocal (the fractional part of (e + 1/2) / w is at
// least 1/(2w) away from an integer, far more than the float error for these
// sizes).  CW: the caller's extents fold to constants (a full block of a
// compile-time shape), and the index arithmetic per point is a few integer
// adds.
// rot (in warps, running over the loops between two barriers): the loop's
// first pass starts at warp rot, so its last, partial pass falls on the
// warps after the ones that took the previous loop's last pass, and the
// loops of one barrier interval share out their passes as one flat loop
// would (without it the low warps take the extra pass of every loop and the
// barrier waits for them).  Blocks of NT threads (a multiple of 32; 256 but
// for the FP64 d_sw).
template <bool CW = false, int NT = 256, typename F>
__device__ __forceinline__ void for2(int& rot, int ilo, int ihi, int jlo, int jhi, F f) {
  const int w = ihi - ilo, h = jhi - jlo;
  if (w <= 0 || h <= 0) return;
  const int total = w * h;
  const int tid = (int)(threadIdx.y * blockDim.x + threadIdx.x);
  constexpr bool POW2 = (NT & (NT - 1)) == 0;
  int e0 = tid - 32 * rot;
  if constexpr (POW2) e0 &= NT - 1;
  else if (e0 < 0) e0 += NT;
  if constexpr (CW) {
    // extents known at compile time (full blocks): the first point by a
    // division by the constant width, then steps of 256 points as constant
    // increments of (i, j)
    int j = e0 / w, i = e0 - j * w;
    const int dj = NT / w, di = NT - dj * w;
#pragma unroll 1
    for (int e = e0; e < total; e += NT) {
      f(ilo + i, jlo + j);
      i += di;
      j += dj;
      if (i >= w) {
        i -= w;
        ++j;
      }
    }
  } else {
    const float rw = 1.0f / (float)w;
    for (int e = e0; e < total; e += NT) {
      const int j = (int)(((float)e + 0.5f) * rw);
      f(ilo + (e - j * w), jlo + j);
    }
  }
  if constexpr (POW2) rot = (rot + (total + 31) / 32) & (NT / 32 - 1);
  else rot = (rot + (total + 31) / 32) % (NT / 32);
}

// a loop on its own (the warps' first pass from warp 0)
template <bool CW = false, int NT = 256, typename F>
__device__ __forceinline__ void for2(int ilo, int ihi, int jlo, int jhi, F f) {
  int rot = 0;
  for2<CW, NT>(rot, ilo, ihi, jlo, jhi, f);
}

// The block's tile with its halo of 3 ([x0 - 3, x1 + 3) x [y0 - 3, y1 + 3)),
// fetched into NP registers per thread (the points of the flat loop of for2,
// 256 threads) and later put into shared memory: the loads are in flight
// while the block computes.  q: origin of the level.
template <int NP, typename R>
__device__ __forceinline__ void tile_fetch(const R* q, R (&reg)[NP], const Blk& B, int P) {
  const int w = B.x1 - B.x0 + 6, total = w * (B.y1 - B.y0 + 6);
  const float rw = 1.0f / (float)w;
  const int tid = (int)(threadIdx.y * blockDim.x + threadIdx.x);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int e = tid + p * 256;
    if (e < total) {
      const int j = (int)(((float)e + 0.5f) * rw);
      reg[p] = q[(long long)(B.y0 - 3 + j) * P + (B.x0 - 3 + e - j * w)];
    }
  }
}

template <int NP, typename R>
__device__ __forceinline__ void tile_put(R* Q, const R (&reg)[NP], const Blk& B) {
  const int w = B.x1 - B.x0 + 6, total = w * (B.y1 - B.y0 + 6);
  const float rw = 1.0f / (float)w;
  const int tid = (int)(threadIdx.y * blockDim.x + threadIdx.x);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int e = tid + p * 256;
    if (e < total) {
      const int j = (int)(((float)e + 0.5f) * rw);
      Q[j * B.SX + (e - j * w)] = reg[p];
    }
  }
}

// Cube corners (reading R3): rewrite the 3x3 missing-quadrant cells of a
// shared-memory scalar from the block's own strips, turned about the corner:
// role 0 for sweeps along x (from the W/E strip), 1 along y (S/N strip).
template <typename R>
__device__ __forceinline__ void corner_roles(R* Q, const Blk& B, int n, int role) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid >= 36) return;
  const int c = tid / 9, pa = tid % 3, pb = (tid / 3) % 3;
  const int ox = (c & 1) ? 1 : -1, oy = (c & 2) ? 1 : -1;
  const bool here = (ox < 0 ? B.x0 == 0 : B.x1 == n) && (oy < 0 ? B.y0 == 0 : B.y1 == n);
  if (!here) return;
  const int i = ox < 0 ? -1 - pa : n + pa;
  const int j = oy < 0 ? -1 - pb : n + pb;
  int si, sj;
  if (role == 0) {
    si = ox < 0 ? -1 - pb : n + pb;
    sj = oy < 0 ? pa : n - 1 - pa;
  } else {
    si = ox < 0 ? pb : n - 1 - pb;
    sj = oy < 0 ? -1 - pa : n + pa;
  }
  Q[B.L(i, j)] = Q[B.L(si, sj)];
}

// shared-memory arrays of the transport
// MR: the type of the metric terms (R, or double in the FP32-bulk mode that
// keeps the metric in FP64: every product with a metric term is then formed
// in FP64 and rounded to R where it is stored)
template <typename R, typename MR = R>
struct TS {
  R *CRX, *XFX, *CRY, *YFX, *FY2, *FX2, *QIJ, *LAP, *AL;
  MR *RDXd, *RDYd;
  // metric terms of the block's tile staged in shared memory once per work
  // item (area, 1/area; the damping weights wx, wy in the damped transports)
  MR *AREA, *RAREA, *WX, *WY;
};

// FP64 kernels keep the reciprocal denominators of the two inner updates in
// shared memory (a quotient costs several FP64 pipe slots); the FP32 kernels
// recompute them (cheap on the FP32 pipe) and spend those two arrays on the
// damping weights, so that four FP32 blocks still fit an SM
template <typename R>
constexpr bool kStoreRD = sizeof(R) == 8;

// the plain FP64 tracer kernel transports its tracers in pairs (six more
// shared-memory arrays: two FP64 blocks still fit an SM; four FP32 ones
// would not)
template <typename R, bool LEARN>
constexpr bool kTracerPair = sizeof(R) == 8 && !LEARN;

// 1 / (area + the two area fluxes) of the y- and x-inner updates at l
template <typename R, typename MR>
__device__ __forceinline__ MR inner_rdy(const TS<R, MR>& S, int l, int SX) {
  if constexpr (kStoreRD<R>) return S.RDYd[l];
  else return rcp<MR>(S.AREA[l] + S.YFX[l] - S.YFX[l + SX]);
}
template <typename R, typename MR>
__device__ __forceinline__ MR inner_rdx(const TS<R, MR>& S, int l) {
  if constexpr (kStoreRD<R>) return S.RDXd[l];
  else return rcp<MR>(S.AREA[l] + S.XFX[l] - S.XFX[l + 1]);
}

// the stored denominators (kStoreRD): y over [x0-3, x1+3) x [y0, y1), x over
// [x0, x1) x [y0-3, y1+3); read after the next barrier
template <int NT = 256, typename R, typename MR>
__device__ __forceinline__ void inner_denominators(const TS<R, MR>& S, const Blk& B) {
  if constexpr (kStoreRD<R>) {
    const int x0 = B.x0, x1 = B.x1, y0 = B.y0, y1 = B.y1, SX = B.SX;
    int rot = 0;
    for2<false, NT>(rot, x0 - 3, x1 + 3, y0, y1, [&](int i, int j) {
      const int l = B.L(i, j);
      S.RDYd[l] = rcp(S.AREA[l] + S.YFX[l] - S.YFX[l + SX]);
    });
    for2<false, NT>(rot, x0, x1, y0 - 3, y1 + 3, [&](int i, int j) {
      const int l = B.L(i, j);
      S.RDXd[l] = rcp(S.AREA[l] + S.XFX[l] - S.XFX[l + 1]);
    });
  }
}

// shared-memory arrays after the base ones of a kernel, counted in elements
// of R: area, 1/area, the stored denominators (kStoreRD) and the damping
// weights (if `weights`), each of type MR, plus one element of alignment
// slack when MR is wider than R
template <typename R, typename MR = R>
__host__ __device__ constexpr int extra_arrays(bool weights) {
  return 2 + (kStoreRD<R> ? 2 : 0) + (weights ? 2 : 0);
}
template <typename R, typename MR = R>
__host__ __device__ constexpr size_t extra_bytes(int SA, bool weights) {
  return (size_t)extra_arrays<R, MR>(weights) * SA * sizeof(MR) + (sizeof(MR) > sizeof(R) ? sizeof(MR) : 0);
}
template <typename R, typename MR>
__device__ __forceinline__ void assign_extra(TS<R, MR>& S, R* base, int SA, bool weights) {
  // MR arrays start on an MR boundary
  MR* p = reinterpret_cast<MR*>((reinterpret_cast<uintptr_t>(base) + sizeof(MR) - 1) & ~(uintptr_t)(sizeof(MR) - 1));
  S.AREA = p; p += SA;
  S.RAREA = p; p += SA;
  if (kStoreRD<R>) { S.RDXd = p; p += SA; S.RDYd = p; p += SA; } else { S.RDXd = nullptr; S.RDYd = nullptr; }
  if (weights) { S.WX = p; p += SA; S.WY = p; } else { S.WX = nullptr; S.WY = nullptr; }
}

// the metric terms of the block's tile into shared memory: area and 1/area
// over the tile, wx and wy over the faces the damping reads, times wscale
// (the square root of the damping coefficient: the gradients and the
// damping flux each take one factor, so the flux carries the coefficient
// without a multiply of its own)
template <int BX = 0, int BY = 0, bool FULL = false, int NT = 256, typename R, typename MR>
__device__ __forceinline__ void stage_metric(const TS<R, MR>& S, const Blk& B, const TM<MR>& m, bool weights,
                                             MR wscale = MR(1)) {
  const int x0 = B.x0, x1 = FULL ? x0 + BX : B.x1, y0 = B.y0, y1 = FULL ? y0 + BY : B.y1;
  int rot = 0;
  for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0 - 3, y1 + 3, [&](int i, int j) {
    const int l = B.L(i, j);
    S.AREA[l] = MT(area, j, i);
    S.RAREA[l] = MT(rarea, j, i);
  });
  if (weights) {
    for2<FULL, NT>(rot, x0 - 1, x1 + 2, y0 - 1, y1 + 1, [&](int i, int j) { S.WX[B.L(i, j)] = wscale * MT(wx, j, i); });
    for2<FULL, NT>(rot, x0 - 1, x1 + 1, y0 - 1, y1 + 2, [&](int i, int j) { S.WY[B.L(i, j)] = wscale * MT(wy, j, i); });
  }
}


// face value at face l from precomputed edge values AL (AL[l] is the edge
// between cells l - s and l) for the upwind weight cw of the face: limited
// parabola of the upwind cell, swept mean
template <typename R>
__device__ __forceinline__ R ppm_face_al(const R* Q, const R* AL, int l, int s, R cw) {
  const int p = upwind_before(cw) ? l - s : l;
  const R qu = Q[p];
  R bl = AL[p] - qu, br = AL[p + s] - qu;
  ppm_limit(bl, br);
  return swept_mean(qu, bl, br, cw);
}

// a lies in [min(qa, qb), max(qa, qb)] and is not negative (FP64: on the
// integer pipe, with the order-preserving keys of the bit patterns)
template <typename R>
__device__ __forceinline__ bool within_cells(R a, R qa, R qb) {
  const R lo = qa < qb ? qa : qb, hi = qa < qb ? qb : qa;
  return a >= lo && a <= hi && a >= R(0);
}
template <>
__device__ __forceinline__ bool within_cells<double>(double a, double qa, double qb) {
  const long long ka = okey(a), k0 = okey(qa), k1 = okey(qb);
  const long long lo = k0 < k1 ? k0 : k1, hi = k0 < k1 ? k1 : k0;
  return ka >= lo && ka <= hi && ka >= 0;
}

// damping of a transport: none, always, or where the coefficient is not zero
enum { DAMP_NO = 0, DAMP_YES = 1, DAMP_RT = 2 };
template <int DM, typename R>
__device__ __forceinline__ bool damped(R damp) {
  if constexpr (DM == DAMP_RT) return damp != R(0);
  else return DM == DAMP_YES;
}

// Learned face values (reading R14) over a 2-D range of faces with stride s
// along the sweep: the plain PPM face value plus the mirror-symmetric
// network's correction sig * y, or the plain value alone where the sum leaves
// the range of the two cells or is negative (every learned field is
// positive).  All lanes of a warp take part in the tensor-core evaluation;
// padding lanes repeat a valid face and do not store.
template <typename R>
__device__ void learned_faces(const R* Q, const R* AL, const R* CC, R* OUT, int ilo, int ihi, int jlo, int jhi,
                              int s, const Blk& B, const MlpFrag& F) {
  const int w = ihi - ilo, total = w * (jhi - jlo);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int warp = tid >> 5, nwarps = (blockDim.x * blockDim.y) >> 5, lane = tid & 31;
  for (int base = warp * 32; base < total; base += nwarps * 32) {
    const int e = base + lane;
    const bool valid = e < total;
    const int ee = valid ? e : base;
    const int i = ilo + ee % w, j = jlo + ee / w;
    const int l = B.L(i, j);
    const R plain = ppm_face_al(Q, AL, l, s, CC[l]);
    R q[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = Q[l + (k - 3) * s];
    float x[6], xr[6];
    const float sig = mlp_inputs(q, x, xr);
    const float y1 = mlp_warp(F, x);
    const float y2 = mlp_warp(F, xr);
    const float corr = __fmul_rn(__fmul_rn(0.5f, __fadd_rn(y1, y2)), sig);
    const R a = plain + widen<R>(corr);
    if (valid) OUT[l] = within_cells(a, q[2], q[3]) ? a : plain;
  }
}

// The flux through a face from its outer face value f and the inner
// sweep's face value fi: the mean of the two times the mass or area flux mf,
// plus, if damped, the del-4 flux (lap - lapm) w, w the staged weight that
// carries the square root of the coefficient (the Laplacians carry the
// other), weighted by the mean of wdp over the face's two cells (at l - s
// and l) if WDP.  As 0.5 (f + fi) mf + (lap - lapm) w [(wdp_l-s + wdp_l) / 2],
// with the halving moved to where it costs no multiply of its own.
template <bool WDP, typename R, typename MR>
__device__ __forceinline__ R face_flux(R f, R fi, R mf, bool dmp, R lap, R lapm, MR w, const R* wdp, int l, int s) {
  const R g = (f + fi) * mf;  // twice the advective flux
  if (!dmp) return R(0.5) * g;
  const R dl = (lap - lapm) * w;
  if constexpr (WDP) return R(0.5) * fmadd(dl, wdp[l - s] + wdp[l], g);
  else return fmadd(R(0.5), g, dl);
}

// fv_tp_2d (reading R5) + optional delnflux (R6) of the shared-memory scalar
// Q on the block: fluxes on x-faces [x0, x1] x [y0, y1) -> FXO and y-faces
// [x0, x1) x [y0, y1] -> FYO.  mfx/mfy: mass fluxes (null: area fluxes).
// damp > 0 adds the del-4 flux, weighted by 1/2 (wdp_{i-1} + wdp_i) if wdp;
// the staged weights WX, WY carry the square root of damp (stage_metric).
// Every PPM sweep first computes each edge value once (AL), then the face
// values; the Laplacian of the damping is the divergence of face gradients.
// The same transport for the FP32 path in four phases: on the FP32 pipe an
// edge value costs less than the shared-memory round trip, the loop
// overhead and the barrier of a separate edge phase, so each face value
// forms its two edge values itself (ppm_face: the same operations as
// ppm_edge + ppm_face_al, the same bits), the inner x-update goes to the
// edge array, which is free, and the phases that do not read each other's
// results share a barrier:
//   1  y-faces of Q (FY2) and the damping gradients GY
//   2  inner y-update (QIJ), x-faces of Q (FX2) and the gradients GX
//   3  Laplacian (LAP) and inner x-update (into AL)
//   4  outer x-faces of QIJ and outer y-faces of the x-updated field, fluxes
// The damping gradients live in the output arrays until the Laplacian is
// formed, as in transport().
template <int BX, int BY, bool FULL, int DM, bool WDP, int NT = 256, typename R, typename MR>
__device__ void transport_fused(R* Q, const TS<R, MR>& S, const Blk& B, int n, bool cc, const R* mfx, const R* mfy,
                                R damp, const R* wdp, R* FXO, R* FYO) {
  const int x0 = B.x0, x1 = FULL ? x0 + BX : B.x1, y0 = B.y0, y1 = FULL ? y0 + BY : B.y1, SX = B.SX;
  const bool dmp = damped<DM>(damp);
  R* const GX = FXO;
  R* const GY = FYO;
  R* const QJ = S.AL;  // the x-updated field
  int rot = 0;  // warp rotation of the loops of one barrier interval (for2)
  __syncthreads();  // Q (and the strips the corner turn reads) complete
  if (cc) {  // blocks at a cube corner: the missing quadrant for the y-sweep
    corner_roles(Q, B, n, 1);
    __syncthreads();
  }
  // 1: y-faces of the plain field (y-role corners)
  for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0, y1 + 1, [&](int i, int j) {
    const int l = B.L(i, j);
    S.FY2[l] = ppm_face(Q + l, SX, S.CRY[l]);
  });
  if (dmp)
    for2<FULL, NT>(rot, x0 - 1, x1 + 1, y0 - 1, y1 + 2, [&](int i, int j) {
      const int l = B.L(i, j);
      GY[l] = (Q[l] - Q[l - SX]) * S.WY[l];
    });
  __syncthreads();
  // 2: inner y-update in every column of the block and its halo
  for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0, y1, [&](int i, int j) {
    const int l = B.L(i, j);
    S.QIJ[l] = (Q[l] * S.AREA[l] + S.FY2[l] * S.YFX[l] - S.FY2[l + SX] * S.YFX[l + SX]) * inner_rdy(S, l, SX);
  });
  if (cc) {  // x-role corners: touches only missing-quadrant cells, which
             // the inner y-update does not read; the x-faces below do
    corner_roles(Q, B, n, 0);
    __syncthreads();
  }
  // x-faces of the plain field (x-role corners)
  for2<FULL, NT>(rot, x0, x1 + 1, y0 - 3, y1 + 3, [&](int i, int j) {
    const int l = B.L(i, j);
    S.FX2[l] = ppm_face(Q + l, 1, S.CRX[l]);
  });
  if (dmp)
    for2<FULL, NT>(rot, x0 - 1, x1 + 2, y0 - 1, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      GX[l] = (Q[l] - Q[l - 1]) * S.WX[l];
    });
  __syncthreads();
  // 3: Laplacian of the damping, inner x-update in every row of the block
  // and its halo
  if (dmp)
    for2<FULL, NT>(rot, x0 - 1, x1 + 1, y0 - 1, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      S.LAP[l] = (GX[l + 1] - GX[l] + GY[l + SX] - GY[l]) * S.RAREA[l];
    });
  for2<FULL, NT>(rot, x0, x1, y0 - 3, y1 + 3, [&](int i, int j) {
    const int l = B.L(i, j);
    QJ[l] = (Q[l] * S.AREA[l] + S.FX2[l] * S.XFX[l] - S.FX2[l + 1] * S.XFX[l + 1]) * inner_rdx(S, l);
  });
  __syncthreads();
  // 4: outer x-faces of the y-updated field and outer y-faces of the
  // x-updated field; fluxes = mean face value x (mass or area) flux, plus
  // the del-4 damping flux
  for2<FULL, NT>(rot, x0, x1 + 1, y0, y1, [&](int i, int j) {
    const int l = B.L(i, j);
    FXO[l] = face_flux<WDP>(ppm_face(S.QIJ + l, 1, S.CRX[l]), S.FX2[l], mfx ? mfx[l] : S.XFX[l], dmp, S.LAP[l],
                            S.LAP[l - 1], S.WX[l], wdp, l, 1);
  });
  for2<FULL, NT>(rot, x0, x1, y0, y1 + 1, [&](int i, int j) {
    const int l = B.L(i, j);
    FYO[l] = face_flux<WDP>(ppm_face(QJ + l, SX, S.CRY[l]), S.FY2[l], mfy ? mfy[l] : S.YFX[l], dmp, S.LAP[l],
                            S.LAP[l - SX], S.WY[l], wdp, l, SX);
  });
  __syncthreads();
}

// DM: DAMP_NO (no damping), DAMP_YES (the del-4 terms formed whatever the
// coefficient; a zero coefficient adds zeros) or DAMP_RT (damping where the
// coefficient is not zero, decided at run time); WDP: the damping flux is
// weighted by the mean of wdp over the face.  Compile-time choices keep the
// terms a transport does not form out of its loops altogether (a term
// switched off at run time inside a loop may still be issued, with no lane
// active, and FP64 instructions cost their pipe time either way).
template <typename R, bool LEARN = false, int BX = 0, int BY = 0, bool FULL = false, int DM = DAMP_RT,
          bool WDP = false, int NT = 256, typename MR = R>
__device__ void transport(R* Q, const TS<R, MR>& S, const Blk& B, const TM<MR>& m, int n, bool cc, const R* mfx,
                          const R* mfy, R damp, const R* wdp, R* FXO, R* FYO, const float* mlp = nullptr) {
  const int x0 = B.x0, x1 = FULL ? x0 + BX : B.x1, y0 = B.y0, y1 = FULL ? y0 + BY : B.y1, SX = B.SX;
  if constexpr (sizeof(R) == 4 && !LEARN) {
    transport_fused<BX, BY, FULL, DM, WDP, NT>(Q, S, B, n, cc, mfx, mfy, damp, wdp, FXO, FYO);
    return;
  }
  const bool dmp = damped<DM>(damp);
  int rot = 0;  // warp rotation of the loops of one barrier interval (for2)
  // the damping gradients live in the output arrays until the Laplacian is
  // formed; the fluxes are written only after it
  R* const GX = FXO;
  R* const GY = FYO;
  // the damped transports (d_sw, fv_tp_2d) have the weights wx, wy staged
  MlpFrag F;
  if (LEARN) mlp_load(mlp, F);
  // the fluxes of x-face / y-face l from its outer face value, with the
  // del-4 damping added where they are formed (the Laplacian is complete by
  // then)
  auto flux_x = [&](int l, R f) -> R {
    return face_flux<WDP>(f, S.FX2[l], mfx ? mfx[l] : S.XFX[l], dmp, S.LAP[l], S.LAP[l - 1], S.WX[l], wdp, l, 1);
  };
  auto flux_y = [&](int l, R f) -> R {
    return face_flux<WDP>(f, S.FY2[l], mfy ? mfy[l] : S.YFX[l], dmp, S.LAP[l], S.LAP[l - SX], S.WY[l], wdp, l,
                          SX);
  };
  __syncthreads();  // Q (and the strips the corner turn reads) complete
  if (cc) {  // blocks at a cube corner: the missing quadrant for the y-sweep
    corner_roles(Q, B, n, 1);
    __syncthreads();
  }
  // y-sweep of the plain field (y-role corners): edges, then faces
  for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0 - 1, y1 + 2, [&](int i, int j) {
    const int l = B.L(i, j);
    S.AL[l] = ppm_edge(Q[l - 2 * SX], Q[l - SX], Q[l], Q[l + SX]);
  });
  if (dmp)
    for2<FULL, NT>(rot, x0 - 1, x1 + 1, y0 - 1, y1 + 2, [&](int i, int j) {
      const int l = B.L(i, j);
      GY[l] = (Q[l] - Q[l - SX]) * S.WY[l];
    });
  __syncthreads();
  if (LEARN)
    learned_faces(Q, S.AL, S.CRY, S.FY2, x0 - 3, x1 + 3, y0, y1 + 1, SX, B, F);
  else
    for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      S.FY2[l] = ppm_face_al(Q, S.AL, l, SX, S.CRY[l]);
    });
  __syncthreads();
  // inner y-update in every column of the block and its halo
  for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0, y1, [&](int i, int j) {
    const int l = B.L(i, j);
    S.QIJ[l] = (Q[l] * S.AREA[l] + S.FY2[l] * S.YFX[l] - S.FY2[l + SX] * S.YFX[l + SX]) * inner_rdy(S, l, SX);
  });
  // the x-edges below read Q and write AL and GX, which the inner y-update
  // does not touch: a barrier only where the x-role corners rewrite Q
  if (cc) {
    corner_roles(Q, B, n, 0);  // touches only missing-quadrant cells
    __syncthreads();
  }
  // x-sweep of the plain field (x-role corners)
  for2<FULL, NT>(rot, x0 - 1, x1 + 2, y0 - 3, y1 + 3, [&](int i, int j) {
    const int l = B.L(i, j);
    S.AL[l] = ppm_edge(Q[l - 2], Q[l - 1], Q[l], Q[l + 1]);
  });
  if (dmp)
    for2<FULL, NT>(rot, x0 - 1, x1 + 2, y0 - 1, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      GX[l] = (Q[l] - Q[l - 1]) * S.WX[l];
    });
  __syncthreads();
  if (LEARN)
    learned_faces(Q, S.AL, S.CRX, S.FX2, x0, x1 + 1, y0 - 3, y1 + 3, 1, B, F);
  else
    for2<FULL, NT>(rot, x0, x1 + 1, y0 - 3, y1 + 3, [&](int i, int j) {
      const int l = B.L(i, j);
      S.FX2[l] = ppm_face_al(Q, S.AL, l, 1, S.CRX[l]);
    });
  if (dmp)
    for2<FULL, NT>(rot, x0 - 1, x1 + 1, y0 - 1, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      S.LAP[l] = (GX[l + 1] - GX[l] + GY[l + SX] - GY[l]) * S.RAREA[l];
    });
  __syncthreads();
  // outer x-sweep of the y-updated field
  for2<FULL, NT>(rot, x0 - 1, x1 + 2, y0, y1, [&](int i, int j) {
    const int l = B.L(i, j);
    S.AL[l] = ppm_edge(S.QIJ[l - 2], S.QIJ[l - 1], S.QIJ[l], S.QIJ[l + 1]);
  });
  __syncthreads();
  if (LEARN) {
    learned_faces(S.QIJ, S.AL, S.CRX, FXO, x0, x1 + 1, y0, y1, 1, B, F);
    __syncthreads();
    for2<FULL, NT>(rot, x0, x1 + 1, y0, y1, [&](int i, int j) {
      const int l = B.L(i, j);
      FXO[l] = flux_x(l, FXO[l]);
    });
  } else {
    for2<FULL, NT>(rot, x0, x1 + 1, y0, y1, [&](int i, int j) {
      const int l = B.L(i, j);
      FXO[l] = flux_x(l, ppm_face_al(S.QIJ, S.AL, l, 1, S.CRX[l]));
    });
  }
  __syncthreads();
  // inner x-update in every row of the block and its halo
  for2<FULL, NT>(rot, x0, x1, y0 - 3, y1 + 3, [&](int i, int j) {
    const int l = B.L(i, j);
    S.QIJ[l] = (Q[l] * S.AREA[l] + S.FX2[l] * S.XFX[l] - S.FX2[l + 1] * S.XFX[l + 1]) * inner_rdx(S, l);
  });
  __syncthreads();
  // outer y-sweep of the x-updated field
  for2<FULL, NT>(rot, x0, x1, y0 - 1, y1 + 2, [&](int i, int j) {
    const int l = B.L(i, j);
    S.AL[l] = ppm_edge(S.QIJ[l - 2 * SX], S.QIJ[l - SX], S.QIJ[l], S.QIJ[l + SX]);
  });
  __syncthreads();
  if (LEARN) {
    learned_faces(S.QIJ, S.AL, S.CRY, FYO, x0, x1, y0, y1 + 1, SX, B, F);
    __syncthreads();
    for2<FULL, NT>(rot, x0, x1, y0, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      FYO[l] = flux_y(l, FYO[l]);
    });
  } else {
    for2<FULL, NT>(rot, x0, x1, y0, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      FYO[l] = flux_y(l, ppm_face_al(S.QIJ, S.AL, l, SX, S.CRY[l]));
    });
  }
  __syncthreads();
}

// Two scalars transported together (tracer_2d, no damping, plain PPM): the
// steps of transport() above, each phase doing both fields, so that every
// barrier is shared by twice the FP64 work.  Per field: the tile Q, the edge,
// face and inner-update arrays and the output fluxes.
template <typename R>
struct TF {
  R *Q, *AL, *FY2, *FX2, *QIJ, *FXO, *FYO;
};

template <int BX, int BY, bool FULL, typename R, typename MR>
__device__ void transport_pair(const TF<R>* F, const TS<R, MR>& S, const Blk& B, int n, bool cc, const R* mfx,
                               const R* mfy) {
  const int x0 = B.x0, x1 = FULL ? x0 + BX : B.x1, y0 = B.y0, y1 = FULL ? y0 + BY : B.y1, SX = B.SX;
  int rot = 0;  // warp rotation of the loops of one barrier interval (for2)
  __syncthreads();  // both tiles complete
  if (cc) {
    corner_roles(F[0].Q, B, n, 1);
    corner_roles(F[1].Q, B, n, 1);
    __syncthreads();
  }
  for2<FULL>(rot, x0 - 3, x1 + 3, y0 - 1, y1 + 2, [&](int i, int j) {
    const int l = B.L(i, j);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const R* Q = F[f].Q;
      F[f].AL[l] = ppm_edge(Q[l - 2 * SX], Q[l - SX], Q[l], Q[l + SX]);
    }
  });
  __syncthreads();
  for2<FULL>(rot, x0 - 3, x1 + 3, y0, y1 + 1, [&](int i, int j) {
    const int l = B.L(i, j);
#pragma unroll
    for (int f = 0; f < 2; ++f) F[f].FY2[l] = ppm_face_al(F[f].Q, F[f].AL, l, SX, S.CRY[l]);
  });
  __syncthreads();
  for2<FULL>(rot, x0 - 3, x1 + 3, y0, y1, [&](int i, int j) {
    const int l = B.L(i, j);
    const MR rd = inner_rdy(S, l, SX);
#pragma unroll
    for (int f = 0; f < 2; ++f)
      F[f].QIJ[l] = (F[f].Q[l] * S.AREA[l] + F[f].FY2[l] * S.YFX[l] - F[f].FY2[l + SX] * S.YFX[l + SX]) * rd;
  });
  if (cc) {  // touches only missing-quadrant cells; else the x-edges need no barrier
    corner_roles(F[0].Q, B, n, 0);
    corner_roles(F[1].Q, B, n, 0);
    __syncthreads();
  }
  for2<FULL>(rot, x0 - 1, x1 + 2, y0 - 3, y1 + 3, [&](int i, int j) {
    const int l = B.L(i, j);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const R* Q = F[f].Q;
      F[f].AL[l] = ppm_edge(Q[l - 2], Q[l - 1], Q[l], Q[l + 1]);
    }
  });
  __syncthreads();
  for2<FULL>(rot, x0, x1 + 1, y0 - 3, y1 + 3, [&](int i, int j) {
    const int l = B.L(i, j);
#pragma unroll
    for (int f = 0; f < 2; ++f) F[f].FX2[l] = ppm_face_al(F[f].Q, F[f].AL, l, 1, S.CRX[l]);
  });
  __syncthreads();
  for2<FULL>(rot, x0 - 1, x1 + 2, y0, y1, [&](int i, int j) {
    const int l = B.L(i, j);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const R* Q = F[f].QIJ;
      F[f].AL[l] = ppm_edge(Q[l - 2], Q[l - 1], Q[l], Q[l + 1]);
    }
  });
  __syncthreads();
  for2<FULL>(rot, x0, x1 + 1, y0, y1, [&](int i, int j) {
    const int l = B.L(i, j);
    const R hw = R(0.5) * mfx[l];  // half the mass flux, shared by the two fields
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const R v = ppm_face_al(F[f].QIJ, F[f].AL, l, 1, S.CRX[l]);
      F[f].FXO[l] = (v + F[f].FX2[l]) * hw;
    }
  });
  __syncthreads();
  for2<FULL>(rot, x0, x1, y0 - 3, y1 + 3, [&](int i, int j) {
    const int l = B.L(i, j);
    const MR rd = inner_rdx(S, l);
#pragma unroll
    for (int f = 0; f < 2; ++f)
      F[f].QIJ[l] = (F[f].Q[l] * S.AREA[l] + F[f].FX2[l] * S.XFX[l] - F[f].FX2[l + 1] * S.XFX[l + 1]) * rd;
  });
  __syncthreads();
  for2<FULL>(rot, x0, x1, y0 - 1, y1 + 2, [&](int i, int j) {
    const int l = B.L(i, j);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const R* Q = F[f].QIJ;
      F[f].AL[l] = ppm_edge(Q[l - 2 * SX], Q[l - SX], Q[l], Q[l + SX]);
    }
  });
  __syncthreads();
  for2<FULL>(rot, x0, x1, y0, y1 + 1, [&](int i, int j) {
    const int l = B.L(i, j);
    const R hw = R(0.5) * mfy[l];  // half the mass flux, shared by the two fields
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const R v = ppm_face_al(F[f].QIJ, F[f].AL, l, SX, S.CRY[l]);
      F[f].FYO[l] = (v + F[f].FY2[l]) * hw;
    }
  });
  __syncthreads();
}

// Courant numbers and area fluxes (reading R11) into shared memory (the
// Courant numbers as upwind weights), plus the reciprocal denominators of the
// two inner updates.  uc/vc: global, origin of the level.  guard: returns
// whether a face of the block's own (|c| < 1 checked on the west and south
// faces of its cells) breaks the Courant condition.  acx, afx, acy, afy
// (level origins, or null): the remapping step's sums of the Courant numbers
// and area fluxes, added for the faces the block writes (its cells' west and
// south faces, and the tile's east and north edge faces).
template <int BX = 0, int BY = 0, bool FULL = false, int NT = 256, typename R, typename MR>
__device__ bool courant(const R* uc, const R* vc, const R* Vs, const R* Us, const TS<R, MR>& S, const Blk& B,
                        const TM<MR>& m, const Geo& g, R dt, bool guard, R* acx, R* afx, R* acy, R* afy) {
  const int x0 = B.x0, x1 = FULL ? x0 + BX : B.x1, y0 = B.y0, y1 = FULL ? y0 + BY : B.y1;
  const int P = g.pitch;
  const bool xe = x1 == g.n, ye = y1 == g.n;
  bool bad = false;
  int rot = 0;
  for2<FULL, NT>(rot, x0, x1 + 1, y0 - 3, y1 + 3, [&](int i, int j) {
    const int l = B.L(i, j);
    // dt ut dy sin and dt ut sin / dxc with ut = (uc - cos v) / sin^2
    const auto du = dt * (uc[(long long)j * P + i] - MT(cosx, j, i) * Vs[l]);
    const R fx = du * MT(kfx, j, i), c = du * MT(kcx, j, i);
    S.XFX[l] = fx;
    S.CRX[l] = upwind_weight(c);
    const bool row = j >= y0 && j < y1;
    if (guard && row && i < x1) bad |= !below_one(c);
    if (acx && row && (i < x1 || xe)) {
      atomicAdd(acx + (long long)j * P + i, c);
      atomicAdd(afx + (long long)j * P + i, fx);
    }
  });
  for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0, y1 + 1, [&](int i, int j) {
    const int l = B.L(i, j);
    const auto dv = dt * (vc[(long long)j * P + i] - MT(cosy, j, i) * Us[l]);
    const R fy = dv * MT(kfy, j, i), c = dv * MT(kcy, j, i);
    S.YFX[l] = fy;
    S.CRY[l] = upwind_weight(c);
    const bool col = i >= x0 && i < x1;
    if (guard && col && j < y1) bad |= !below_one(c);
    if (acy && col && (j < y1 || ye)) {
      atomicAdd(acy + (long long)j * P + i, c);
      atomicAdd(afy + (long long)j * P + i, fy);
    }
  });
  __syncthreads();
  inner_denominators<NT>(S, B);
  return bad;
}

// ------------------------------------------------------------------------
// d_sw (reading R11): one level of a block per loop iteration
// ------------------------------------------------------------------------
// FULL: every block of every member is a full BX x BY block (the tiles'
// sizes are multiples of the block shape), so the extents of every 2-D loop
// are compile-time constants
// threads of a d_sw block: the plain FP64 kernel takes nine warps (two
// blocks of 288 threads x 112 registers fill the register file, 18 warps per
// SM to feed the FP64 pipe instead of 16), the others eight
template <typename R, bool LEARN>
constexpr int kDswThreads = (sizeof(R) == 8 && !LEARN) ? 288 : 256;

template <typename R, int BX, int BY, bool LEARN, typename MR = R, bool FULL = false>
__global__ void __launch_bounds__(kDswThreads<R, LEARN>, (sizeof(R) == 8 || LEARN) ? 2 : (sizeof(MR) == 8 ? 3 : 4))
    k_d_sw(StepArgs<R> a, int kchunk, int nwork) {
  constexpr int NT = kDswThreads<R, LEARN>;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int SX = BX + 7, SY = BY + 7, SA = SX * SY;
  R* sb = reinterpret_cast<R*>(smraw);
  R *DP = sb, *PT = sb + SA, *W = sb + 2 * SA, *U = sb + 3 * SA, *V = sb + 4 * SA;
  R *MFX = sb + 5 * SA, *MFY = sb + 6 * SA, *FXO = sb + 7 * SA, *FYO = sb + 8 * SA, *DPN = sb + 9 * SA;
  R* KE = DPN;  // 1/delp_new is dead once pt and w are written
  TS<R, MR> S;
  S.CRX = sb + 10 * SA; S.XFX = sb + 11 * SA; S.CRY = sb + 12 * SA; S.YFX = sb + 13 * SA;
  S.FY2 = sb + 14 * SA; S.FX2 = sb + 15 * SA; S.QIJ = sb + 16 * SA; S.LAP = sb + 17 * SA; S.AL = sb + 18 * SA;
  assign_extra(S, sb + 19 * SA, SA, true);
  (void)SY;

  const int kz = (a.geo[0].nz + kchunk - 1) / kchunk;
  // work items (block, level chunk): one per CTA, or strided over a
  // persistent grid
  for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
  const Item it = a.items[wi / kz];
  const Geo g = a.geo[it.m];
  const int n = g.n, P = g.pitch;
  Blk B{it.x0, FULL ? it.x0 + BX : min(it.x0 + BX, n), it.y0, FULL ? it.y0 + BY : min(it.y0 + BY, n), SX};
  const bool cc = g.cubed && (B.x0 == 0 || B.x1 == n) && (B.y0 == 0 || B.y1 == n);
  const TM<MR> m = tile_metric(metric_sel<MR>(a), g, it.t);
  const R dt = (R)a.P.dt, hdt = R(0.5) * dt, qdt = R(0.25) * dt;
  const double dd = a.P.d4_bg * g.da_min;
  const R damp = (R)(dd * dd);
  const int k0 = (wi % kz) * kchunk, k1 = min(k0 + kchunk, g.nz);
  const int x0 = B.x0, x1 = FULL ? x0 + BX : B.x1, y0 = B.y0, y1 = FULL ? y0 + BY : B.y1;
  // read after the first barrier of the level loop; the damping weights
  // carry d4_bg da_min, the square root of the coefficient
  stage_metric<BX, BY, FULL, NT>(S, B, m, true, (MR)dd);
  for (int k = k0; k < k1; ++k) {
    const long long o = fld0(g, g.off3, g.nz, it.t, k);
    const R *u = a.u + o, *v = a.v + o, *w = a.w + o, *dp = a.delp + o, *pt = a.pt + o;
    const R *uc = a.uc + o, *vc = a.vc + o;
    int rot = 0;  // warp rotation of the loops of one barrier interval (for2)
    auto G = [&](int j, int i) { return (long long)j * P + i; };
    for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0 - 3, y1 + 3, [&](int i, int j) {
      const int l = B.L(i, j);
      const long long q = G(j, i);
      DP[l] = dp[q];
      PT[l] = pt[q];
      W[l] = w[q];
    });
    for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0 - 3, y1 + 4, [&](int i, int j) { U[B.L(i, j)] = u[G(j, i)]; });
    for2<FULL, NT>(rot, x0 - 3, x1 + 4, y0 - 3, y1 + 3, [&](int i, int j) { V[B.L(i, j)] = v[G(j, i)]; });
    __syncthreads();
    {
      R* const acx = a.amfx ? a.acrx + o : nullptr;
      const bool bad = courant<BX, BY, FULL, NT>(uc, vc, V, U, S, B, m, g, dt, a.status != nullptr, acx,
                                             a.amfx ? a.axfx + o : nullptr, a.amfx ? a.acry + o : nullptr,
                                             a.amfx ? a.ayfx + o : nullptr);
      if (bad) atomicOr(a.status, ST_CFL);  // Courant-number guard on the block's own faces
    }
    // mass
    transport<R, LEARN, BX, BY, FULL, DAMP_YES, false, NT>(DP, S, B, m, n, cc, (const R*)nullptr, (const R*)nullptr, damp,
                                      (const R*)nullptr, MFX, MFY, a.mlp);
    R* dpo = a.delp_o + o;
    for2<FULL, NT>(rot, x0, x1, y0, y1, [&](int i, int j) {
      const int l = B.L(i, j);
      const R d = DP[l] + (MFX[l] - MFX[l + 1] + MFY[l] - MFY[l + SX]) * S.RAREA[l];
      DPN[l] = rcp(d);  // reciprocal, used by pt and w
      dpo[G(j, i)] = d;
    });
    // pt and w with the mass fluxes and mass-weighted damping
    for (int fld = 0; fld < 2; ++fld) {
      R* Q = fld == 0 ? PT : W;
      R* out = (fld == 0 ? a.pt_o : a.w_o) + o;
      if (LEARN && fld == 0)
        transport<R, LEARN, BX, BY, FULL, DAMP_YES, true, NT>(Q, S, B, m, n, cc, MFX, MFY, damp, DP, FXO, FYO, a.mlp);
      else
        transport<R, false, BX, BY, FULL, DAMP_YES, true, NT>(Q, S, B, m, n, cc, MFX, MFY, damp, DP, FXO, FYO);
      for2<FULL, NT>(rot, x0, x1, y0, y1, [&](int i, int j) {
        const int l = B.L(i, j);
        out[G(j, i)] =
            (Q[l] * DP[l] + (FXO[l] - FXO[l + 1] + FYO[l] - FYO[l + SX]) * S.RAREA[l]) * DPN[l];
      });
    }
    __syncthreads();
    // cell absolute vorticity (into PT)
    for2<FULL, NT>(rot, x0 - 3, x1 + 3, y0 - 3, y1 + 3, [&](int i, int j) {
      const int l = B.L(i, j);
      PT[l] = (U[l] * MT(dx, j, i) - U[l + SX] * MT(dx, j + 1, i) + V[l + 1] * MT(dy, j, i + 1) -
               V[l] * MT(dy, j, i)) * S.RAREA[l] + MT(fA, j, i);
    });
    transport<R, false, BX, BY, FULL, DAMP_YES, false, NT>(PT, S, B, m, n, cc, (const R*)nullptr, (const R*)nullptr, damp,
                                      (const R*)nullptr, FXO, FYO);
    // kinetic energy at corners from upwind-PPM corner winds.  FP64: the
    // edge values of u along x and of v along y once each (into the free
    // transport arrays AL and QIJ), as the transports do, instead of two per
    // corner and wind; FP32 forms them in the corner loop (cheaper there than
    // the barrier)
    if constexpr (kStoreRD<R>) {
      for2<FULL, NT>(rot, x0 - 1, x1 + 2, y0, y1 + 1, [&](int i, int j) {
        const int l = B.L(i, j);
        S.AL[l] = ppm_edge(U[l - 2], U[l - 1], U[l], U[l + 1]);
      });
      for2<FULL, NT>(rot, x0, x1 + 1, y0 - 1, y1 + 2, [&](int i, int j) {
        const int l = B.L(i, j);
        S.QIJ[l] = ppm_edge(V[l - 2 * SX], V[l - SX], V[l], V[l + SX]);
      });
      __syncthreads();
    }
    for2<FULL, NT>(rot, x0, x1 + 1, y0, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      // twice the corner winds (their halvings moved into hdt and qdt)
      const R ua2 = uc[G(j - 1, i)] + uc[G(j, i)];
      const R va2 = vc[G(j, i - 1)] + vc[G(j, i)];
      // the upwind edge length's reciprocal: one load of the chosen face
      const R cu = hdt * ua2 * MT(rdx, j, positive(ua2) ? i - 1 : i);
      const R cv = hdt * va2 * MT(rdy, positive(va2) ? j - 1 : j, i);
      const R wu = upwind_weight(cu), wv = upwind_weight(cv);
      R ub, vb;
      if constexpr (kStoreRD<R>) {
        ub = ppm_face_al(U, S.AL, l, 1, wu);
        vb = ppm_face_al(V, S.QIJ, l, SX, wv);
      } else {
        ub = ppm_face(U + l, 1, wu);
        vb = ppm_face(V + l, SX, wv);
      }
      KE[l] = qdt * (ub * ua2 + vb * va2);
    });
    __syncthreads();
    R *uo = a.u_o + o, *vo = a.v_o + o;
    for2<FULL, NT>(rot, x0, x1, y0, y1 + (y1 == n ? 1 : 0), [&](int i, int j) {
      const int l = B.L(i, j);
      uo[G(j, i)] = U[l] + (FYO[l] + KE[l] - KE[l + 1]) * MT(rdx, j, i);
    });
    for2<FULL, NT>(rot, x0, x1 + (x1 == n ? 1 : 0), y0, y1, [&](int i, int j) {
      const int l = B.L(i, j);
      vo[G(j, i)] = V[l] + (-FXO[l] + KE[l] - KE[l + SX]) * MT(rdy, j, i);
    });
    if (a.xfxd) {  // the D-grid area fluxes for update_dz_d (reading R17)
      for2<FULL, NT>(rot, x0, x1 + (x1 == n ? 1 : 0), y0, y1, [&](int i, int j) { a.xfxd[o + G(j, i)] = S.XFX[B.L(i, j)]; });
      for2<FULL, NT>(rot, x0, x1, y0, y1 + (y1 == n ? 1 : 0), [&](int i, int j) { a.yfxd[o + G(j, i)] = S.YFX[B.L(i, j)]; });
    }
    if (a.amfx) {
      // the remapping step's sums (the Courant numbers and area fluxes were
      // added where they were formed): each face has one writer per launch,
      // so an addition performed at the memory side (a reduction whose
      // result is not read back) gives the sum a load-add-store gives,
      // without the load's round trip
      for2<FULL, NT>(rot, x0, x1 + (x1 == n ? 1 : 0), y0, y1, [&](int i, int j) {
        atomicAdd(a.amfx + o + G(j, i), MFX[B.L(i, j)]);
      });
      for2<FULL, NT>(rot, x0, x1, y0, y1 + (y1 == n ? 1 : 0), [&](int i, int j) {
        atomicAdd(a.amfy + o + G(j, i), MFY[B.L(i, j)]);
      });
    }
    __syncthreads();
  }
  }
}

// ------------------------------------------------------------------------
// c_sw (reading R7)
// ------------------------------------------------------------------------
template <typename R, int BX, int BY, typename MR = R, bool FULL = false>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 3 : 4) k_c_sw(StepArgs<R> a, int kchunk, int nwork) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int SX = BX + 7, SY = BY + 7, SA = SX * SY;
  R* sb = reinterpret_cast<R*>(smraw);
  R *U = sb, *V = sb + SA, *DP = sb + 2 * SA, *PT = sb + 3 * SA, *W = sb + 4 * SA;
  R *UC0 = sb + 5 * SA, *VC0 = sb + 6 * SA, *UT = sb + 7 * SA, *VT = sb + 8 * SA, *KE = sb + 9 * SA;
  R *VO = sb + 10 * SA, *FX1 = sb + 11 * SA, *FY1 = sb + 12 * SA;
  (void)SY;
  const int kz = (a.geo[0].nz + kchunk - 1) / kchunk;
  for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
  const Item it = a.items[wi / kz];
  const Geo g = a.geo[it.m];
  const int n = g.n, P = g.pitch;
  Blk B{it.x0, FULL ? it.x0 + BX : min(it.x0 + BX, n), it.y0, FULL ? it.y0 + BY : min(it.y0 + BY, n), SX};
  const int x0 = B.x0, x1 = FULL ? x0 + BX : B.x1, y0 = B.y0, y1 = FULL ? y0 + BY : B.y1;
  const TM<MR> m = tile_metric(metric_sel<MR>(a), g, it.t);
  const R dt2 = R(0.5 * a.P.dt), dt2e = R(0.125) * dt2;
  const int k0 = (wi % kz) * kchunk, k1 = min(k0 + kchunk, g.nz);
  auto G = [&](int j, int i) { return (long long)j * P + i; };
  for (int k = k0; k < k1; ++k) {
    const long long o = fld0(g, g.off3, g.nz, it.t, k);
    const R *u = a.u + o, *v = a.v + o, *w = a.w + o, *dp = a.delp + o, *pt = a.pt + o;
    const bool ord4 = a.P.d2c_ord == 4;
    if (ord4) {  // the fourth-order stencils reach one ring further
      for2<FULL>(x0 - 3, x1 + 3, y0 - 2, y1 + 3, [&](int i, int j) { U[B.L(i, j)] = u[G(j, i)]; });
      for2<FULL>(x0 - 2, x1 + 3, y0 - 3, y1 + 3, [&](int i, int j) { V[B.L(i, j)] = v[G(j, i)]; });
    } else {
      for2<FULL>(x0 - 2, x1 + 2, y0 - 1, y1 + 2, [&](int i, int j) { U[B.L(i, j)] = u[G(j, i)]; });
      for2<FULL>(x0 - 1, x1 + 2, y0 - 2, y1 + 2, [&](int i, int j) { V[B.L(i, j)] = v[G(j, i)]; });
    }
    for2<FULL>(x0 - 1, x1 + 1, y0 - 1, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      const long long q = G(j, i);
      DP[l] = dp[q];
      PT[l] = pt[q];
      W[l] = w[q];
    });
    __syncthreads();
    // C-grid winds from the D-grid: the mean of the four surrounding values
    // (reading R7) or four-point Lagrange interpolation (-1, 9, 9, -1) / 16
    // along the component's direction, then across (reading R18)
    auto lag4 = [](R a0, R a1, R a2, R a3) { return R(0.0625) * (R(9) * (a1 + a2) - (a0 + a3)); };
    for2<FULL>(x0 - 1, x1 + 2, y0 - 1, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      R c0;
      if (ord4) {
        auto ax = [&](int r) { return lag4(U[r - 2], U[r - 1], U[r], U[r + 1]); };
        c0 = lag4(ax(l - SX), ax(l), ax(l + SX), ax(l + 2 * SX));
      } else {
        c0 = R(0.25) * (U[l - 1] + U[l] + U[l - 1 + SX] + U[l + SX]);
      }
      UC0[l] = c0;
      UT[l] = (c0 - MT(cosx, j, i) * V[l]) * MT(rsin2x, j, i);
    });
    for2<FULL>(x0 - 1, x1 + 1, y0 - 1, y1 + 2, [&](int i, int j) {
      const int l = B.L(i, j);
      R c0;
      if (ord4) {
        auto by = [&](int r) { return lag4(V[r - 2 * SX], V[r - SX], V[r], V[r + SX]); };
        c0 = lag4(by(l - 1), by(l), by(l + 1), by(l + 2));
      } else {
        c0 = R(0.25) * (V[l - SX] + V[l - SX + 1] + V[l] + V[l + 1]);
      }
      VC0[l] = c0;
      VT[l] = (c0 - MT(cosy, j, i) * U[l]) * MT(rsin2y, j, i);
    });
    __syncthreads();
    R *fx1 = a.fx1 + o, *fy1 = a.fy1 + o;
    for2<FULL>(x0, x1 + 1, y0, y1, [&](int i, int j) {
      const int l = B.L(i, j);
      const R f = dt2 * UT[l] * MT(dy, j, i) * MT(sinx, j, i);
      FX1[l] = f;
      if (i < x1 || x1 == n) fx1[G(j, i)] = f;
    });
    for2<FULL>(x0, x1, y0, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      const R f = dt2 * VT[l] * MT(dx, j, i) * MT(siny, j, i);
      FY1[l] = f;
      if (j < y1 || y1 == n) fy1[G(j, i)] = f;
    });
    for2<FULL>(x0 - 1, x1 + 1, y0 - 1, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      // twice the cell-centre winds; their halvings squared fold into dt2 / 8
      const R ua2 = UT[l] + UT[l + 1];
      const R va2 = VT[l] + VT[l + SX];
      KE[l] = dt2e * (ua2 * ua2 + va2 * va2);
    });
    for2<FULL>(x0, x1 + 1, y0, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      const R ts = UC0[l - SX] * MT(dxc, j - 1, i);
      R te = VC0[l] * MT(dyc, j, i);
      const R tn = UC0[l] * MT(dxc, j, i);
      R tw = VC0[l - 1] * MT(dyc, j, i - 1);
      if (g.cubed && (i == 0 || i == n) && (j == 0 || j == n)) {  // cube corner: triangle
        if (i == 0) tw = R(0);
        else te = R(0);
      }
      VO[l] = (ts + te - tn - tw) * MT(rareac, j, i) + MT(fC, j, i);
    });
    __syncthreads();
    R *dpc = a.delpc + o, *ptc = a.ptc + o, *wcc = a.wc + o;
    for2<FULL>(x0, x1, y0, y1, [&](int i, int j) {
      const int l = B.L(i, j);
      const int up[4] = {positive(FX1[l]) ? l - 1 : l, positive(FX1[l + 1]) ? l : l + 1,
                         positive(FY1[l]) ? l - SX : l, positive(FY1[l + SX]) ? l : l + SX};
      const R F[4] = {FX1[l], FX1[l + 1], FY1[l], FY1[l + SX]};
      R fm[4], fp[4], fw[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        fm[f] = F[f] * DP[up[f]];
        fp[f] = fm[f] * PT[up[f]];
        fw[f] = fm[f] * W[up[f]];
      }
      const MR ra = MT(rarea, j, i);
      const R d = DP[l] + (fm[0] - fm[1] + fm[2] - fm[3]) * ra;
      dpc[G(j, i)] = d;
      const R rdn = rcp(d);
      ptc[G(j, i)] = (PT[l] * DP[l] + (fp[0] - fp[1] + fp[2] - fp[3]) * ra) * rdn;
      wcc[G(j, i)] = (W[l] * DP[l] + (fw[0] - fw[1] + fw[2] - fw[3]) * ra) * rdn;
    });
    R *uco = a.uc + o, *vco = a.vc + o;
    for2<FULL>(x0, x1 + (x1 == n ? 1 : 0), y0, y1, [&](int i, int j) {
      const int l = B.L(i, j);
      uco[G(j, i)] = UC0[l] + dt2 * R(0.5) * (VO[l] + VO[l + SX]) * V[l] + (KE[l - 1] - KE[l]) * MT(rdxc, j, i);
    });
    for2<FULL>(x0, x1, y0, y1 + (y1 == n ? 1 : 0), [&](int i, int j) {
      const int l = B.L(i, j);
      vco[G(j, i)] = VC0[l] - dt2 * R(0.5) * (VO[l] + VO[l + 1]) * U[l] + (KE[l - SX] - KE[l]) * MT(rdyc, j, i);
    });
    __syncthreads();
  }
  }
}

// ------------------------------------------------------------------------
// update_dz_c (reading R8): blocks of 16 x 8 columns marching up from the
// surface, the interface geopotential of the block and of its ring (the
// columns around it, corners excluded) exchanged in shared memory level by
// level.  128 threads: thread t owns the inner column (t % 16, t / 16) and
// its west and south faces; threads 0 .. 47 also own one ring column (8 on
// the west and east sides, 16 on the south and north sides), the east ring
// the block's last x-face and the north ring its last y-face.  Every warp
// holds inner columns, so the FP64 update of the inner cells runs on full
// warps (ring threads of their own would issue it with no lane active).
// The blocks are small so that a C96 sphere (55,296 columns, 432 blocks)
// spreads evenly over the SMs: a block's level march is sequential, and the
// busiest SM sets the time.
// ------------------------------------------------------------------------
template <typename R, typename MR = R>
__global__ void __launch_bounds__(kDzBX * kDzBY) k_update_dz_c(StepArgs<R> a) {
  constexpr int BX = kDzBX, BY = kDzBY, W = BX + 2, H = BY + 2;
  __shared__ R GZ[W * H];
  __shared__ R SXF[W * H], SYF[W * H];  // twice the level-mean flux of the west / south face of a frame cell
  const Item it = a.items[blockIdx.x];
  const Geo g = a.geo[it.m];
  const int n = g.n, P = g.pitch, nz = g.nz;
  const int x0 = it.x0, y0 = it.y0, x1 = min(x0 + BX, n), y1 = min(y0 + BY, n);
  const int t = (int)threadIdx.x;
  const int i = x0 + t % BX, j = y0 + t / BX;
  const bool inner = i < x1 && j < y1;
  const int l = (j - y0 + 1) * W + (i - x0 + 1);
  // the ring column of threads 0 .. 2 (BX + BY) - 1: west, east, south, north
  const int side = t < BY ? 0 : (t < 2 * BY ? 1 : (t < 2 * BY + BX ? 2 : 3));
  const int pos = side == 0 ? t : (side == 1 ? t - BY : (side == 2 ? t - 2 * BY : t - 2 * BY - BX));
  const int ri = side == 0 ? x0 - 1 : (side == 1 ? x1 : x0 + pos);
  const int rj = side <= 1 ? y0 + pos : (side == 2 ? y0 - 1 : y1);
  const bool ring = t < 2 * (BX + BY) && (side <= 1 ? rj < y1 : ri < x1);
  const bool rfx = ring && side == 1, rfy = ring && side == 3;
  const int rl = (rj - y0 + 1) * W + (ri - x0 + 1);
  const TM<MR> m = tile_metric(metric_sel<MR>(a), g, it.t);
  const R grav = (R)a.P.grav, dzmin = (R)a.P.dz_min, rgrav = (R)(1.0 / a.P.grav);
  const long long q = (long long)j * P + i, rq = (long long)rj * P + ri;
  const int lo[4] = {l - 1, l, l - W, l};
  const int hi[4] = {l, l + 1, l, l + W};
  auto lev = [&](int K) { return fld0(g, g.off3, nz, it.t, K); };
  // The level loop is sequential: the loads run ahead of it (delz one level,
  // the fluxes two levels), so their latency overlaps the level before.  The
  // update is written with twice the level-mean fluxes S = fx(K-1) + fx(K)
  // (2 fx(0) at the top) and twice the area: numerator and denominator both
  // scale by exactly 2, so the quotient is the one of the mean fluxes.
  const MR ar2 = inner ? MR(2) * MT(area, j, i) : MR(1);
  R gzr = R(0), gzn_below = R(0), rgz = R(0);
  R xb = R(0), xa = R(0), xn = R(0), yb = R(0), ya = R(0), yn = R(0);  // levels K, K - 1, K - 2
  R fb = R(0), fa = R(0), fn = R(0);                                    // the ring face's flux
  const R* rflux = rfx ? a.fx1 : a.fy1;
  R dzk = R(0), rdz = R(0);
  {
    const long long o = lev(nz - 1), o1 = lev(nz - 2);  // nz >= 2
    if (inner) {
      dzk = a.delz[o + q];
      xb = a.fx1[o + q]; xa = a.fx1[o1 + q];
      yb = a.fy1[o + q]; ya = a.fy1[o1 + q];
    }
    if (ring) rdz = a.delz[o + rq];
    if (rfx || rfy) { fb = rflux[o + rq]; fa = rflux[o1 + rq]; }
  }
  for (int K = nz - 1; K >= 0; --K) {
    const long long o = lev(K);
    R dzn = R(0), rdzn = R(0);
    if (K > 0) {
      if (inner) dzn = a.delz[o - g.plane + q];
      if (ring) rdzn = a.delz[o - g.plane + rq];
    }
    if (K >= 2) {
      const long long o2 = o - 2 * g.plane;
      if (inner) { xn = a.fx1[o2 + q]; yn = a.fy1[o2 + q]; }
      if (rfx || rfy) fn = rflux[o2 + rq];
    }
    if (inner) {
      gzr = gzr - grav * dzk;
      GZ[l] = gzr;
      SXF[l] = K == 0 ? R(2) * xb : xa + xb;
      SYF[l] = K == 0 ? R(2) * yb : ya + yb;
    }
    if (ring) {
      rgz = rgz - grav * rdz;
      GZ[rl] = rgz;
      if (rfx) SXF[rl] = K == 0 ? R(2) * fb : fa + fb;
      if (rfy) SYF[rl] = K == 0 ? R(2) * fb : fa + fb;
    }
    __syncthreads();
    if (inner) {
      const R S[4] = {SXF[l], SXF[l + 1], SYF[l], SYF[l + W]};
      R Gf[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) Gf[f] = S[f] * (positive(S[f]) ? GZ[lo[f]] : GZ[hi[f]]);
      const R gzn = (GZ[l] * ar2 + Gf[0] - Gf[1] + Gf[2] - Gf[3]) * rcp(ar2 + S[0] - S[1] + S[2] - S[3]);
      a.delzc[o + q] = min_of((gzn_below - gzn) * rgrav, -dzmin);
      gzn_below = gzn;
    }
    xb = xa; xa = xn; yb = ya; ya = yn;
    fb = fa; fa = fn;
    dzk = dzn;
    rdz = rdzn;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------
// riem_solver_c (Section IX-B, reading R9): one thread per column, FP64 in
// both precision modes.  Top-down: interface pressure, gas-law pressure and
// its perturbation, coefficients and the forward Thomas sweep into scratch;
// bottom-up: back-substitution, new thickness, perturbation pressure, pef and
// gz.  Scratch layout [5][nz][ncol], coalesced across the warp along i.
// ------------------------------------------------------------------------
// FULL (riem_solver3, reading R17): the whole substep dt instead of dt/2,
// and the new layer w (mean of its two interface values) and delz written
// back (w_o, delz_o)
// One warp per CTA: the columns of a tile are few for this GPU (one thread
// each, 7 to 12 warps per SM at C96 / C192), so the work is spread over the
// SMs in units of one warp; with CTAs of four warps (some partly empty) some
// SMs held twice the FP64 work of others.
constexpr int kRiemCols = 32;

template <typename R, bool FULL>
__global__ void __launch_bounds__(kRiemCols) k_riem_c(StepArgs<R> a, const RowItem* rows) {
  const RowItem r = rows[blockIdx.y];
  const Geo g = a.geo[r.m];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int nz = g.nz;
  const long long col = g.colbase + ((long long)r.t * g.n + r.j) * g.n + i;
  const long long NC = a.ncol;
  double* s_cp = a.scratch;
  double* s_dp = a.scratch + (long long)nz * NC;
  double* s_C = a.scratch + 2LL * nz * NC;
  double* s_pp = a.scratch + 3LL * nz * NC;
  double* s_pe = a.scratch + 4LL * nz * NC;
  const double dt = FULL ? a.P.dt : 0.5 * a.P.dt, grav = a.P.grav, rd = a.P.rdgas, aimp = a.P.a_imp;
  const double kappa = a.P.rdgas / a.P.cp_air, gama = 1.0 / (1.0 - kappa);
  // the loop-invariant quotients once; per level one reciprocal for the
  // thickness and the interface pressure sum together (rcp_pair) and one for
  // the pivot (FP64 here is 2 lanes per SM per clock, and a quotient costs
  // several of them).  kA2: a quarter of 1 / (g dt), so that (dp above + dp)
  // kA2 is half the interface mass term m / dt of the tridiagonal row.
  const double rgrav = 1.0 / grav, rdt = 1.0 / dt, cC = aimp * dt * gama, rd_g = rd / grav;
  const double kA2 = 0.25 * rgrav * rdt;
  const long long q = (long long)r.j * g.pitch + i;
  double pe = a.P.ptop, dpp = 0.0, wcp = 0.0, Cp = 0.0, ppp = 0.0, cpp = 0.0, dpv = 0.0;
  // Software pipeline over the levels: iteration k forms the coefficients of
  // level k + 1 (gas-law and hydrostatic pressures, C, the tridiagonal row)
  // and runs the elimination step of level k.  The two chains do not depend
  // on each other, so the scheduler interleaves them (a warp's sweep is
  // sequential and FP64 latency would otherwise stall it); the loads run two
  // levels ahead.  The arithmetic of every value is the one-level-at-a-time
  // sweep's.
  const long long o0 = fld0(g, g.off3, nz, r.t, 0) + q;
  const long long plane = g.plane;
  struct Row { double la, di, up, rhs; };
  auto coef = [&](int k, R dpr, R ptr, R wcr, R dzr) -> Row {
    const double dpk = to_f64(dpr), ptk = to_f64(ptr), wck = to_f64(wcr), dzk = to_f64(dzr);
    const double pen = pe + dpk, sum = pe + pen;
    double rdz, rsum;
    rcp_pair(dzk, sum, rdz, rsum);
    const double p = -dpk * rd_g * ptk * rdz;
    const double ph = layer_mean_pressure(sum, rsum, pen, pe, dpk);
    const double pp = p - ph;
    const double C = -cC * p * rdz;
    // the interface mass over dt is m / dt = 2 A2 (the top interface: half
    // its layer, dpp = 0 there), and its w the mean of the two layers'
    // (the top interface: its layer's; wcp = wck there), so that
    // m / dt * w = A2 (wcp + wck)
    const double A2 = (dpp + dpk) * kA2;
    Row w;
    w.la = -Cp;                        // lower (layer above the interface)
    w.di = fma(2.0, A2, Cp) + C;       // diagonal
    w.up = k < nz - 1 ? -C : 0.0;      // upper
    w.rhs = fma(A2, wcp + wck, pp) - ppp;
    const long long sidx = (long long)k * NC + col;
    s_C[sidx] = C;
    s_pp[sidx] = pp;
    s_pe[sidx] = pe;
    pe = pen;
    dpp = dpk;
    wcp = wck;
    Cp = C;
    ppp = pp;
    return w;
  };
  auto eliminate = [&](int k, const Row& w) {
    double cpk, dpt;
    if (k == 0) {
      const double rden = rcp(w.di);
      cpk = w.up * rden;
      dpt = w.rhs * rden;
    } else {
      const double rden = rcp(w.di - w.la * cpp);
      cpk = w.up * rden;
      dpt = (w.rhs - w.la * dpv) * rden;
    }
    const long long sidx = (long long)k * NC + col;
    s_cp[sidx] = cpk;
    s_dp[sidx] = dpt;
    cpp = cpk;
    dpv = dpt;
  };
  R ndp = a.delpc[o0], npt = a.ptc[o0], nwc = a.wc[o0], ndz = a.delzc[o0];
  wcp = to_f64(nwc);
  Row cur = coef(0, ndp, npt, nwc, ndz);
  {
    const long long on = o0 + plane;  // nz >= 2
    ndp = a.delpc[on]; npt = a.ptc[on]; nwc = a.wc[on]; ndz = a.delzc[on];
  }
  for (int k = 0; k < nz - 1; ++k) {
    const R dpr = ndp, ptr = npt, wcr = nwc, dzr = ndz;
    const long long on = o0 + (long long)min(k + 2, nz - 1) * plane;
    ndp = a.delpc[on]; npt = a.ptc[on]; nwc = a.wc[on]; ndz = a.delzc[on];
    const Row nxt = coef(k + 1, dpr, ptr, wcr, dzr);
    eliminate(k, cur);
    cur = nxt;
  }
  eliminate(nz - 1, cur);
  const double pe_bot = pe, raimp = 1.0 / aimp;
  double Wn = 0.0, gzv = 0.0, ppn_below = 0.0;
  {
    const long long ob = fld0(g, g.offi, nz + 1, r.t, nz) + q;
    a.gz[ob] = R(0);
  }
  // bottom-up, the loads of level k - 1 issued before level k is computed
  long long sidx = (long long)(nz - 1) * NC + col;
  double bdp = s_dp[sidx], bcp = s_cp[sidx], bpp = s_pp[sidx], bC = s_C[sidx], bpe = 0.0;
  R bdz = a.delzc[fld0(g, g.off3, nz, r.t, nz - 1) + q];
  for (int k = nz - 1; k >= 0; --k) {
    const double dpk = bdp, cpk = bcp, ppk = bpp, Ck = bC, pek = bpe, dzk = to_f64(bdz);
    const long long o = fld0(g, g.off3, nz, r.t, k) + q;
    if (k > 0) {
      bpe = s_pe[sidx];  // hydrostatic pressure of the interface below layer k - 1
      sidx -= NC;
      bdp = s_dp[sidx]; bcp = s_cp[sidx]; bpp = s_pp[sidx]; bC = s_C[sidx];
      bdz = a.delzc[o - g.plane];
    }
    const double Wk = dpk - cpk * Wn;
    const double dzn = dzk + dt * (Wn - Wk);
    const double ppn = ppk + Ck * (Wn - Wk) * raimp;
    if (FULL) {
      a.w_o[o] = (R)(0.5 * (Wk + Wn));
      a.delz_o[o] = (R)dzn;
    }
    gzv = gzv - grav * dzn;
    const long long oi = fld0(g, g.offi, nz + 1, r.t, k) + q;
    const long long oib = fld0(g, g.offi, nz + 1, r.t, k + 1) + q;
    a.gz[oi] = (R)gzv;
    // pef of the interface below layer k
    double pef;
    if (k == nz - 1) pef = pe_bot + ppn;
    else pef = pek + 0.5 * (ppn + ppn_below);
    a.pef[oib] = (R)pef;
    ppn_below = ppn;
    Wn = Wk;
  }
  a.pef[fld0(g, g.offi, nz + 1, r.t, 0) + q] = (R)a.P.ptop;
}

// ------------------------------------------------------------------------
// p_grad_c (reading R10): the first nbi x nbi blocks of a plane are 16 x 16
// cells, one thread per cell (i, j) updating its west x-face and its south
// y-face; the blocks after them take the east x-faces (i = n) and the north
// y-faces (j = n) of the tile as one flat list, 32 to a warp (a block of
// cells at the edge would hold one face per row).  Plane list entries
// (m, t, k).
// ------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R pgrad(R gA0, R gA1, R gB0, R gB1, R pA0, R pA1, R pB0, R pB1) {
  return ((gA1 - gB0) * (pB1 - pA0) + (gA0 - gB1) * (pA1 - pB0)) * rcp(pA1 - pA0 + pB1 - pB0);
}

template <typename R, typename MR = R>
__global__ void __launch_bounds__(256) k_p_grad_c(StepArgs<R> a, const int4* planes, int nbi) {
  const int4 pl = planes[blockIdx.z];
  const Geo g = a.geo[pl.x];
  const int n = g.n, b = (int)blockIdx.x;
  int i, j;
  bool xf = true, yf = true;
  if (b < nbi * nbi) {
    i = (b % nbi) * 16 + (int)threadIdx.x;
    j = (b / nbi) * 16 + (int)threadIdx.y;
    if (i >= n || j >= n) return;
  } else {
    const int e = (b - nbi * nbi) * 256 + (int)(threadIdx.y * 16 + threadIdx.x);
    if (e >= 2 * n) return;
    xf = e < n;
    yf = !xf;
    i = xf ? n : e - n;
    j = xf ? e : n;
  }
  const int t = pl.y, k = pl.z;
  const TM<MR> m = tile_metric(metric_sel<MR>(a), g, t);
  const R dt2 = R(0.5 * a.P.dt);
  const long long o = fld0(g, g.off3, g.nz, t, k);
  const R* p0 = a.pef + fld0(g, g.offi, g.nz + 1, t, k);
  const R* p1 = a.pef + fld0(g, g.offi, g.nz + 1, t, k + 1);
  const R* z0 = a.gz + fld0(g, g.offi, g.nz + 1, t, k);
  const R* z1 = a.gz + fld0(g, g.offi, g.nz + 1, t, k + 1);
  const long long B = (long long)j * g.pitch + i;
  if (xf) {
    const long long A = B - 1;
    add_to(a.uc + o + B, dt2 * MT(rdxc, j, i) * pgrad(z0[A], z1[A], z0[B], z1[B], p0[A], p1[A], p0[B], p1[B]));
  }
  if (yf) {
    const long long A = B - g.pitch;
    add_to(a.vc + o + B, dt2 * MT(rdyc, j, i) * pgrad(z0[A], z1[A], z0[B], z1[B], p0[A], p1[A], p0[B], p1[B]));
  }
}

// ------------------------------------------------------------------------
// Divergence damping (reading R19), after d_sw: at every corner the
// divergence and tension of the start-of-d_sw D-grid winds over the dual
// cell, the shear at the four surrounding cell centres, the coefficient
// c = da_min max(d2_bg, min(0.2, dddmp dt |deformation|)) and cd = c x div;
// d_sw's corner kinetic energy minus cd enters the wind update, so
// u += (cd(i+1, j) - cd(i, j)) rdx and v += (cd(i, j+1) - cd(i, j)) rdy.
// None at the cube corners.  One thread per (i, j) of a level plane.
// ------------------------------------------------------------------------
template <typename R, typename MR>
__device__ __forceinline__ R cell_shear(const R* u, const R* v, const TM<MR>& m, const Geo& g, int j, int i) {
  const long long P = g.pitch;
  return (u[(j + 1) * P + i] * MT(dx, j + 1, i) - u[j * P + i] * MT(dx, j, i) + v[j * P + i + 1] * MT(dy, j, i + 1) -
          v[j * P + i] * MT(dy, j, i)) * MT(rarea, j, i);
}

// a 16 x 16 block of corners (i0 + tx, j0 + ty): the shears of the 18 x 18
// cells around them and the damping of the 17 x 17 corners the block's faces
// need are formed once each, in shared memory
template <typename R, typename MR = R>
__global__ void __launch_bounds__(256) k_div_damp(StepArgs<R> a, const int4* planes) {
  __shared__ R s_sh[18][18];
  __shared__ R s_cd[17][17];
  const int4 pl = planes[blockIdx.z];
  const Geo g = a.geo[pl.x];
  const int n = g.n;
  const int i0 = blockIdx.x * 16, j0 = blockIdx.y * 16;
  if (i0 > n || j0 > n) return;  // the whole block (uniform)
  const int tid = threadIdx.y * 16 + threadIdx.x;
  const int t = pl.y, k = pl.z;
  const TM<MR> m = tile_metric(metric_sel<MR>(a), g, t);
  const long long o = fld0(g, g.off3, g.nz, t, k);
  const R *u = a.u + o, *v = a.v + o;
  const R d2 = (R)a.P.d2_bg, sm = (R)(a.P.dddmp * a.P.dt);
  for (int e = tid; e < 18 * 18; e += 256) {  // cells j0 - 1 .. j0 + 16, i0 - 1 .. i0 + 16
    const int jj = e / 18, ii = e - jj * 18;
    const int cj = j0 - 1 + jj, ci = i0 - 1 + ii;
    s_sh[jj][ii] = (cj <= n && ci <= n) ? cell_shear(u, v, m, g, cj, ci) : R(0);
  }
  __syncthreads();
  for (int e = tid; e < 17 * 17; e += 256) {  // corners j0 .. j0 + 16, i0 .. i0 + 16
    const int jj = e / 17, ii = e - jj * 17;
    const int j = j0 + jj, i = i0 + ii;
    R cd = R(0);
    if (j <= n && i <= n && !(g.cubed && (i == 0 || i == n) && (j == 0 || j == n))) {
      const long long P = g.pitch;
      const R fe = u[j * P + i] * MT(dyc, j, i) * MT(siny, j, i);
      const R fw = u[j * P + i - 1] * MT(dyc, j, i - 1) * MT(siny, j, i - 1);
      const R fn = v[j * P + i] * MT(dxc, j, i) * MT(sinx, j, i);
      const R fs = v[(j - 1) * P + i] * MT(dxc, j - 1, i) * MT(sinx, j - 1, i);
      const R div = (fe - fw + fn - fs) * MT(rareac, j, i);
      const R ten = (fe - fw - (fn - fs)) * MT(rareac, j, i);
      const R sh = R(0.25) * ((s_sh[jj][ii] + s_sh[jj][ii + 1]) + (s_sh[jj + 1][ii] + s_sh[jj + 1][ii + 1]));
      const R coef = fmax(d2, fmin(R(0.2), sm * sqrt(ten * ten + sh * sh)));
      cd = (R)g.da_min * coef * div;
    }
    s_cd[jj][ii] = cd;
  }
  __syncthreads();
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  if (i > n || j > n) return;
  const R c0 = s_cd[threadIdx.y][threadIdx.x];
  const long long q = o + (long long)j * g.pitch + i;
  if (i < n) add_to(a.u_o + q, (s_cd[threadIdx.y][threadIdx.x + 1] - c0) * MT(rdx, j, i));
  if (j < n) add_to(a.v_o + q, (s_cd[threadIdx.y + 1][threadIdx.x] - c0) * MT(rdy, j, i));
}

// ------------------------------------------------------------------------
// D-grid nonhydrostatic pressure gradient (reading R17): the contour form of
// R10 along each cell edge between its corners A and B, with pef and gz at
// the corners the means of the surrounding cells (three at a cube corner).
// One thread per (i, j): the y-face (u) and the x-face (v) at (i, j).
// ------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R corner_mean(const R* p, const Geo& g, int j, int i) {
  const int n = g.n, P = g.pitch;
  auto C = [&](int jj, int ii) { return p[(long long)jj * P + ii]; };
  if (g.cubed && (i == 0 || i == n) && (j == 0 || j == n)) {
    const int mi = i == 0 ? -1 : n, mj = j == 0 ? -1 : n;
    R sum = R(0);
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        const int ci = i + di, cj = j + dj;
        if (ci == mi && cj == mj) continue;
        sum += C(cj, ci);
      }
    return sum / R(3);
  }
  return R(0.25) * ((C(j - 1, i - 1) + C(j - 1, i)) + (C(j, i - 1) + C(j, i)));
}

// a 16 x 16 block of faces: the corner means of pef and gz at the two
// interfaces for its 17 x 17 corners are formed once each in shared memory
template <typename R, typename MR = R>
__global__ void __launch_bounds__(256) k_p_grad_d(StepArgs<R> a, const int4* planes) {
  __shared__ R s_c[4][17][17];  // pef top, pef bottom, gz top, gz bottom
  const int4 pl = planes[blockIdx.z];
  const Geo g = a.geo[pl.x];
  const int n = g.n;
  const int i0 = blockIdx.x * 16, j0 = blockIdx.y * 16;
  if (i0 > n || j0 > n) return;  // the whole block (uniform)
  const int tid = threadIdx.y * 16 + threadIdx.x;
  const int t = pl.y, k = pl.z;
  const long long oi0 = fld0(g, g.offi, g.nz + 1, t, k), oi1 = fld0(g, g.offi, g.nz + 1, t, k + 1);
  const R* src[4] = {a.pef + oi0, a.pef + oi1, a.gz + oi0, a.gz + oi1};
  for (int e = tid; e < 17 * 17; e += 256) {
    const int jj = e / 17, ii = e - jj * 17;
    const int j = j0 + jj, i = i0 + ii;
    if (j > n || i > n) continue;
#pragma unroll
    for (int f = 0; f < 4; ++f) s_c[f][jj][ii] = corner_mean(src[f], g, j, i);
  }
  __syncthreads();
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  if (i > n || j > n) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const TM<MR> m = tile_metric(metric_sel<MR>(a), g, t);
  const long long o = fld0(g, g.off3, g.nz, t, k) + (long long)j * g.pitch + i;
  const R dt = (R)a.P.dt;
  const R pA0 = s_c[0][ty][tx], pA1 = s_c[1][ty][tx], gA0 = s_c[2][ty][tx], gA1 = s_c[3][ty][tx];
  if (i < n)  // u on the y-face (i, j): corners (i, j) and (i + 1, j)
    add_to(a.u_o + o, dt * MT(rdx, j, i) *
                          pgrad(gA0, gA1, s_c[2][ty][tx + 1], s_c[3][ty][tx + 1], pA0, pA1, s_c[0][ty][tx + 1],
                                s_c[1][ty][tx + 1]));
  if (j < n)  // v on the x-face (i, j): corners (i, j) and (i, j + 1)
    add_to(a.v_o + o, dt * MT(rdy, j, i) *
                          pgrad(gA0, gA1, s_c[2][ty + 1][tx], s_c[3][ty + 1][tx], pA0, pA1, s_c[0][ty + 1][tx],
                                s_c[1][ty + 1][tx]));
}

// ------------------------------------------------------------------------
// halo fill (Section V-C): gather over the resolved plan
// ------------------------------------------------------------------------
template <typename R>
__global__ void k_halo(const HaloBatch b, const Geo* geo) {
  const HaloField& f = b.f[blockIdx.z];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (e >= f.count || k >= f.nlev) return;
  const HaloEntry E = f.ent[e];
  const Geo& g = geo[E.m];
  const long long mo = f.iface ? g.offi : g.off3;
  R* dst = (E.flags & 1) ? (R*)f.ya : (R*)f.xa;
  const R* src = (E.flags & 2) ? (const R*)f.ya : (const R*)f.xa;
  const long long d = mo + ((long long)E.dt * f.nlev + k) * g.plane + E.dst;
  R v;
  if (E.sign == 0) {
    v = qnan<R>();
  } else {
    const R s = src[mo + ((long long)E.st * f.nlev + k) * g.plane + E.src];
    v = E.sign > 0 ? s : -s;
  }
  dst[d] = v;
}

// ------------------------------------------------------------------------
// tracer_2d subcycle (reading R12)
// ------------------------------------------------------------------------
template <typename R, int BX, int BY, bool LEARN, typename MR = R, bool FULL = false>
__global__ void __launch_bounds__(256, (sizeof(R) == 8 || LEARN) ? 2 : 4)
    k_tracer(TracerArgs<R> a, int kchunk, int nwork) {
  if (a.it >= *a.nsplt) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int SX = BX + 7, SA = SX * (BY + 7);
  R* sb = reinterpret_cast<R*>(smraw);
  R *Q = sb, *MFX = sb + SA, *MFY = sb + 2 * SA, *FXO = sb + 3 * SA, *FYO = sb + 4 * SA, *D0 = sb + 5 * SA,
    *D1 = sb + 6 * SA;
  TS<R, MR> S;
  S.CRX = sb + 7 * SA; S.XFX = sb + 8 * SA; S.CRY = sb + 9 * SA; S.YFX = sb + 10 * SA;
  S.FY2 = sb + 11 * SA; S.FX2 = sb + 12 * SA; S.QIJ = sb + 13 * SA; S.LAP = sb + 14 * SA; S.AL = sb + 15 * SA;
  assign_extra(S, sb + 16 * SA, SA, false);  // no damping of tracers
  // the plain FP64 kernel transports tracers in pairs (kTracerPair): the
  // second field's arrays follow, its tile in the unused Laplacian array
  constexpr bool PAIR = kTracerPair<R, LEARN>;
  R* const sb2 = sb + (16 + extra_arrays<R>(false)) * SA;
  const TF<R> TFP[2] = {{Q, S.AL, S.FY2, S.FX2, S.QIJ, FXO, FYO},
                        {S.LAP, sb2, sb2 + SA, sb2 + 2 * SA, sb2 + 3 * SA, sb2 + 4 * SA, sb2 + 5 * SA}};
  const int kz = (a.geo[0].nz + kchunk - 1) / kchunk;
  for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
  const Item it = a.items[wi / kz];
  const Geo g = a.geo[it.m];
  const int n = g.n, P = g.pitch;
  Blk B{it.x0, FULL ? it.x0 + BX : min(it.x0 + BX, n), it.y0, FULL ? it.y0 + BY : min(it.y0 + BY, n), SX};
  const int x0 = B.x0, x1 = FULL ? x0 + BX : B.x1, y0 = B.y0, y1 = FULL ? y0 + BY : B.y1;
  const bool cc = g.cubed && (x0 == 0 || x1 == n) && (y0 == 0 || y1 == n);
  const TM<MR> m = tile_metric(metric_sel<MR>(a), g, it.t);
  const int nsplt = *a.nsplt;
  const R fr = R(1) / R(nsplt);
  const int k0 = (wi % kz) * kchunk, k1 = min(k0 + kchunk, g.nz);
  auto G = [&](int j, int i) { return (long long)j * P + i; };
  stage_metric<BX, BY, FULL>(S, B, m, false);  // read after the first barrier of the level loop
  for (int k = k0; k < k1; ++k) {
    const long long o = fld0(g, g.off3, g.nz, it.t, k);
    int rot = 0;  // warp rotation of the loops of one barrier interval (for2)
    // the remapping step's sums, divided among the subcycles (a multiply by
    // 1 left out altogether when there is one: a branch for the whole block)
    auto split = [&](bool one) {
      for2<FULL>(rot, x0, x1 + 1, y0 - 3, y1 + 3, [&](int i, int j) {
        const int l = B.L(i, j);
        const long long q = o + G(j, i);
        S.CRX[l] = upwind_weight(one ? a.acrx[q] : a.acrx[q] * fr);
        S.XFX[l] = one ? a.axfx[q] : a.axfx[q] * fr;
        MFX[l] = one ? a.amfx[q] : a.amfx[q] * fr;
      });
      for2<FULL>(rot, x0 - 3, x1 + 3, y0, y1 + 1, [&](int i, int j) {
        const int l = B.L(i, j);
        const long long q = o + G(j, i);
        S.CRY[l] = upwind_weight(one ? a.acry[q] : a.acry[q] * fr);
        S.YFX[l] = one ? a.ayfx[q] : a.ayfx[q] * fr;
        MFY[l] = one ? a.amfy[q] : a.amfy[q] * fr;
      });
    };
    if (nsplt == 1) split(true);
    else split(false);
    __syncthreads();
    inner_denominators(S, B);
    for2<FULL>(rot, x0, x1, y0, y1, [&](int i, int j) {
      const int l = B.L(i, j);
      const R d0 = a.dp0[o + G(j, i)];
      const R d1 = d0 + (MFX[l] - MFX[l + 1] + MFY[l] - MFY[l + SX]) * S.RAREA[l];
      // the factors every tracer's update takes: q_new = q dp0 / dp1 + (flux
      // divergence) / (area dp1)
      const R r = rcp(d1);
      D0[l] = d0 * r;
      D1[l] = S.RAREA[l] * r;
      a.dp1[o + G(j, i)] = d1;
    });
    // each tracer's tile (block + halo 3) is fetched into registers while the
    // previous tracer is transported (the plain kernel; the learned one has
    // no registers to spare)
    constexpr int NPRE = LEARN ? 1 : ((BX + 6) * (BY + 6) + 255) / 256;
    R pre[NPRE];
    if constexpr (PAIR) {
      R pre2[NPRE];
      tile_fetch<NPRE>(a.q[0] + o, pre, B, P);
      if (a.nq > 1) tile_fetch<NPRE>(a.q[1] + o, pre2, B, P);
      for (int tq = 0; tq < a.nq; tq += 2) {
        const bool two = tq + 1 < a.nq;
        __syncthreads();
        tile_put<NPRE>(TFP[0].Q, pre, B);
        if (two) tile_put<NPRE>(TFP[1].Q, pre2, B);
        if (tq + 2 < a.nq) tile_fetch<NPRE>(a.q[tq + 2] + o, pre, B, P);
        if (tq + 3 < a.nq) tile_fetch<NPRE>(a.q[tq + 3] + o, pre2, B, P);
        if (two)
          transport_pair<BX, BY, FULL>(TFP, S, B, n, cc, MFX, MFY);
        else
          transport<R, false, BX, BY, FULL, DAMP_NO>(Q, S, B, m, n, cc, MFX, MFY, R(0), (const R*)nullptr, FXO, FYO);
        for (int f = 0; f < (two ? 2 : 1); ++f) {
          R* qo = a.q_o[tq + f] + o;
          const TF<R>& T = TFP[f];
          for2<FULL>(rot, x0, x1, y0, y1, [&](int i, int j) {
            const int l = B.L(i, j);
            qo[G(j, i)] = T.Q[l] * D0[l] + (T.FXO[l] - T.FXO[l + 1] + T.FYO[l] - T.FYO[l + SX]) * D1[l];
          });
        }
      }
    } else {
    if (!LEARN) tile_fetch<NPRE>(a.q[0] + o, pre, B, P);
    for (int tq = 0; tq < a.nq; ++tq) {
      __syncthreads();
      if (LEARN) {
        const R* q = a.q[tq] + o;
        for2<FULL>(rot, x0 - 3, x1 + 3, y0 - 3, y1 + 3, [&](int i, int j) { Q[B.L(i, j)] = q[G(j, i)]; });
      } else {
        tile_put<NPRE>(Q, pre, B);
        if (tq + 1 < a.nq) tile_fetch<NPRE>(a.q[tq + 1] + o, pre, B, P);
      }
      transport<R, LEARN, BX, BY, FULL, DAMP_NO>(Q, S, B, m, n, cc, MFX, MFY, R(0), (const R*)nullptr, FXO, FYO,
                                                  a.mlp);
      R* qo = a.q_o[tq] + o;
      for2<FULL>(rot, x0, x1, y0, y1, [&](int i, int j) {
        const int l = B.L(i, j);
        qo[G(j, i)] = Q[l] * D0[l] + (FXO[l] - FXO[l + 1] + FYO[l] - FYO[l + SX]) * D1[l];
      });
    }
    }
    __syncthreads();
  }
  }
}

// ------------------------------------------------------------------------
// standalone fv_tp_2d (Section IX-C; readings R5, R6): fluxes of one scalar
// field for given Courant numbers and area fluxes (and optionally mass
// fluxes), every level of every tile of every member.  The same transport as
// inside d_sw and tracer_2d, with the fluxes written out.
// ------------------------------------------------------------------------
template <typename R, int BX, int BY, typename MR = R>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 2 : 4) k_fv_tp_2d(TpArgs<R> a, int kchunk, int nwork) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int SX = BX + 7, SA = SX * (BY + 7);
  R* sb = reinterpret_cast<R*>(smraw);
  R *Q = sb, *MFX = sb + SA, *MFY = sb + 2 * SA, *FXO = sb + 3 * SA, *FYO = sb + 4 * SA;
  TS<R, MR> S;
  S.CRX = sb + 5 * SA; S.XFX = sb + 6 * SA; S.CRY = sb + 7 * SA; S.YFX = sb + 8 * SA;
  S.FY2 = sb + 9 * SA; S.FX2 = sb + 10 * SA; S.QIJ = sb + 11 * SA; S.LAP = sb + 12 * SA; S.AL = sb + 13 * SA;
  assign_extra(S, sb + 14 * SA, SA, true);
  const bool mass = a.mfx != nullptr;
  const R damp = (R)a.damp;
  const int kz = (a.geo[0].nz + kchunk - 1) / kchunk;
  for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
  const Item it = a.items[wi / kz];
  const Geo g = a.geo[it.m];
  const int n = g.n, P = g.pitch;
  Blk B{it.x0, min(it.x0 + BX, n), it.y0, min(it.y0 + BY, n), SX};
  const int x0 = B.x0, x1 = B.x1, y0 = B.y0, y1 = B.y1;
  const bool cc = g.cubed && (x0 == 0 || x1 == n) && (y0 == 0 || y1 == n);
  const TM<MR> m = tile_metric(metric_sel<MR>(a), g, it.t);
  const int k0 = (wi % kz) * kchunk, k1 = min(k0 + kchunk, g.nz);
  auto G = [&](int j, int i) { return (long long)j * P + i; };
  // read after the first barrier of the level loop; the damping weights
  // carry the square root of the coefficient
  stage_metric(S, B, m, damp != R(0), (MR)sqrt(a.damp));
  for (int k = k0; k < k1; ++k) {
    const long long o = fld0(g, g.off3, g.nz, it.t, k);
    for2(x0, x1 + 1, y0 - 3, y1 + 3, [&](int i, int j) {
      const int l = B.L(i, j);
      const long long q = o + G(j, i);
      S.CRX[l] = upwind_weight(a.crx[q]);
      S.XFX[l] = a.xfx[q];
      if (mass) MFX[l] = a.mfx[q];
    });
    for2(x0 - 3, x1 + 3, y0, y1 + 1, [&](int i, int j) {
      const int l = B.L(i, j);
      const long long q = o + G(j, i);
      S.CRY[l] = upwind_weight(a.cry[q]);
      S.YFX[l] = a.yfx[q];
      if (mass) MFY[l] = a.mfy[q];
    });
    for2(x0 - 3, x1 + 3, y0 - 3, y1 + 3, [&](int i, int j) { Q[B.L(i, j)] = a.q[o + G(j, i)]; });
    __syncthreads();
    inner_denominators(S, B);
    transport<R, false>(Q, S, B, m, n, cc, mass ? MFX : (const R*)nullptr, mass ? MFY : (const R*)nullptr, damp,
                        (const R*)nullptr, FXO, FYO);
    for2(x0, x1 + (x1 == n ? 1 : 0), y0, y1, [&](int i, int j) { a.fx[o + G(j, i)] = FXO[B.L(i, j)]; });
    for2(x0, x1, y0, y1 + (y1 == n ? 1 : 0), [&](int i, int j) { a.fy[o + G(j, i)] = FYO[B.L(i, j)]; });
    __syncthreads();
  }
  }
}

// largest |accumulated Courant number| over interior faces -> subcycles
template <typename R>
__global__ void k_cmax(const Geo* geo, const int4* planes, const R* acrx, const R* acry, unsigned* cmax_bits) {
  const int4 pl = planes[blockIdx.z];
  const Geo g = geo[pl.x];
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  float c = 0.f;
  if (i < g.n && j < g.n) {
    const long long o = fld0(g, g.off3, g.nz, pl.y, pl.z) + (long long)j * g.pitch + i;
    c = (float)fmax(fabs((double)acrx[o]), fabs((double)acry[o]));
  }
  for (int s = 16; s > 0; s >>= 1) c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, s));
  if ((threadIdx.x & 31) == 0) atomicMax(cmax_bits, __float_as_uint(c));
}

template <typename R>
__global__ void k_nsplt(const unsigned* cmax_bits, int* nsplt, int nmax, unsigned* status, const R* dummy) {
  (void)dummy;
  const float c = __uint_as_float(*cmax_bits);
  int s = (int)ceilf(c);
  if (s < 1) s = 1;
  if (s > nmax) {
    atomicOr(status, ST_NSPLT);
    s = nmax;
  }
  *nsplt = s;
}

// copy [0, n] x [0, n] of every level plane (cells and both face kinds) from
// src to dst; gated on the subcycle count when gate != null
template <typename R>
__global__ void k_copy_planes(const Geo* geo, const int4* planes, const CopyArgs<R> a, const int* gate, int it) {
  if (gate && it >= *gate) return;
  const int4 pl = planes[blockIdx.z];
  const Geo g = geo[pl.x];
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.n || j > g.n) return;
  const long long o = fld0(g, g.off3, g.nz, pl.y, pl.z) + (long long)j * g.pitch + i;
  for (int f = 0; f < a.nf; ++f) a.dst[f][o] = a.src[f][o];
}

// flag any non-finite interior value of the listed fields (kind 0 cells,
// 1 x-faces, 2 y-faces) in the status word
template <typename R>
struct CheckArgs {
  const R* src[MAX_TRACERS + 1];
  int kind[MAX_TRACERS + 1];
  int nf;
};

template <typename R>
__global__ void k_check_finite(const Geo* geo, const int4* planes, const CheckArgs<R> a, unsigned* status) {
  const int4 pl = planes[blockIdx.z];
  const Geo g = geo[pl.x];
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = g.n;
  if (i > n || j > n) return;
  const long long o = fld0(g, g.off3, g.nz, pl.y, pl.z) + (long long)j * g.pitch + i;
  bool bad = false;
  for (int f = 0; f < a.nf; ++f) {
    const int kind = a.kind[f];
    const bool in = (i < n || kind == 1) && (j < n || kind == 2) && !(i == n && j == n);
    if (in) bad |= !isfinite((double)a.src[f][o]);
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

// ------------------------------------------------------------------------
// global mass (reading R13): sum of delp * area per member, FP64,
// Neumaier-compensated, fixed order (block partials, then one thread).
// ------------------------------------------------------------------------
__device__ __forceinline__ void neu_add(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

template <typename R>
__global__ void k_mass_partial(const Geo* geo, const int4* planes, const R* delp, const double* area,
                               double* partial) {
  const int4 pl = planes[blockIdx.x];
  const Geo g = geo[pl.x];
  __shared__ double ss[256], sc[256];
  double s = 0.0, c = 0.0;
  const long long o = fld0(g, g.off3, g.nz, pl.y, pl.z);
  const long long oa = g.off2 + (long long)pl.y * g.plane + (long long)HALO * g.pitch + g.ox;
  for (int e = threadIdx.x; e < g.n * g.n; e += blockDim.x) {
    const int j = e / g.n, i = e % g.n;
    const long long q = (long long)j * g.pitch + i;
    neu_add(s, c, (double)delp[o + q] * area[oa + q]);
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, Cc = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      neu_add(S, Cc, ss[t]);
      Cc += sc[t];
    }
    partial[2 * blockIdx.x] = S;
    partial[2 * blockIdx.x + 1] = Cc;
  }
}

#if FV3_TU_MAIN
__global__ void k_mass_final(const double* partial, const int* first, int nmem, double* out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmem) return;
  double S = 0.0, Cc = 0.0;
  for (int b = first[m]; b < first[m + 1]; ++b) {
    neu_add(S, Cc, partial[2 * b]);
    Cc += partial[2 * b + 1];
  }
  out[m] = S + Cc;
}
#endif


// ------------------------------------------------------------------------
// dense <-> padded layout (argument marshalling for import / export)
// kind: 0 cells (n x n), 1 x-faces (n x n+1), 2 y-faces (n+1 x n), 3 corners
// (n+1 x n+1); iface: 0 level fields, 1 interface fields, 2 metric planes
// ------------------------------------------------------------------------
template <typename R, typename D>
__global__ void k_pack(const Geo* geo, int mem, int kind, int nlev, int iface, R* padded, D* dense, int dir) {
  const Geo g = geo[mem];
  const int n = g.n, ni = n + (kind == 1 || kind == 3), nj = n + (kind == 2 || kind == 3);
  const long long total = (long long)g.nt * nlev * nj * ni;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % ni);
    const int j = (int)((e / ni) % nj);
    const long long tk = e / ((long long)ni * nj);
    const int k = (int)(tk % nlev), t = (int)(tk / nlev);
    const long long base = iface == 1 ? g.offi : iface == 2 ? g.off2 : g.off3;
    const long long o = fld0(g, base, nlev, t, k) + (long long)j * g.pitch + i;
    if (dir == 0) padded[o] = (R)dense[e];
    else dense[e] = (D)padded[o];
  }
}


// ------------------------------------------------------------------------
// orchestration: the launches of one substep / tracer step / utilities
// ------------------------------------------------------------------------
template <typename R>
Metric<R> metric_of(const Ctx& c);
template <>
inline Metric<double> metric_of<double>(const Ctx& c) { return c.Md; }
template <>
inline Metric<float> metric_of<float>(const Ctx& c) { return c.Mf; }

template <typename K>
static void set_smem(K kern, size_t bytes) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// block shapes compiled for the horizontal kernels (picked at run time by
// fv3_set_tiles / fv3_autotune)
#define FV3_DISPATCH_SHAPE(BXv, BYv, CALL) \
  do {                                     \
    if (BXv == 32 && BYv == 8) {           \
      CALL(32, 8);                         \
    } else if (BXv == 32 && BYv == 16) {   \
      CALL(32, 16);                        \
    } else if (BXv == 64 && BYv == 8) {    \
      CALL(64, 8);                         \
    } else {                               \
      CALL(16, 16);                        \
    }                                      \
  } while (0)

#if FV3_TU_MAIN
bool shape_supported(int bx, int by) {
  return (bx == 32 && by == 8) || (bx == 32 && by == 16) || (bx == 64 && by == 8) || (bx == 16 && by == 16);
}
#endif


// grid of a horizontal kernel: one CTA per work item, or (persistent mode)
// as many CTAs as fit on the GPU at once, each striding over the work list
template <typename K>
static dim3 work_grid(const Ctx& c, K kern, size_t smem, int nwork, int threads = 256) {
  if (c.persistent <= 0) return dim3(nwork);
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const int g = sms * per_sm;
  return dim3(g < nwork ? g : nwork);
}

// the d_sw and tracer kernels exist with and without learned face values
// (separate instantiations: the network's fragments need registers the
// plain kernel does not)
template <typename R, int X, int Y, bool L, typename MR, bool F = false>
static void launch_d_sw(const Ctx& c, const StepArgs<R>& a, size_t sm, int nwork, cudaStream_t st) {
  set_smem(k_d_sw<R, X, Y, L, MR, F>, sm);
  constexpr int nt = kDswThreads<R, L>;
  k_d_sw<R, X, Y, L, MR, F><<<work_grid(c, k_d_sw<R, X, Y, L, MR, F>, sm, nwork, nt), dim3(32, nt / 32), sm, st>>>(
      a, c.kchunk, nwork);
}

template <typename R, int X, int Y, typename MR, bool F = false>
static void launch_c_sw(const Ctx& c, const StepArgs<R>& a, size_t sm, int nwork, cudaStream_t st) {
  set_smem(k_c_sw<R, X, Y, MR, F>, sm);
  k_c_sw<R, X, Y, MR, F><<<work_grid(c, k_c_sw<R, X, Y, MR, F>, sm, nwork), dim3(32, 8), sm, st>>>(a, c.kchunk,
                                                                                                  nwork);
}

// every member's tiles are made of full blocks of the current shape
[[maybe_unused]] static bool full_blocks(const Ctx& c) {
  for (const Geo& g : c.geo)
    if (g.n % c.BX != 0 || g.n % c.BY != 0) return false;
  return true;
}

template <typename R, int X, int Y, bool L, typename MR, bool F = false>
static void launch_tracer(const Ctx& c, const TracerArgs<R>& a, size_t sm, int nwork, cudaStream_t st) {
  set_smem(k_tracer<R, X, Y, L, MR, F>, sm);
  k_tracer<R, X, Y, L, MR, F><<<work_grid(c, k_tracer<R, X, Y, L, MR, F>, sm, nwork), dim3(32, 8), sm, st>>>(
      a, c.kchunk, nwork);
}

[[maybe_unused]] static size_t blk_smem(const Ctx& c, int arrays) {
  return (size_t)arrays * (c.BX + 7) * (c.BY + 7) * c.esize;
}

// base arrays of R plus the metric arrays of MR (extra_bytes)
template <typename R, typename MR>
[[maybe_unused]] static size_t blk_smem_mr(const Ctx& c, int arrays, bool weights) {
  return blk_smem(c, arrays) + extra_bytes<R, MR>((c.BX + 7) * (c.BY + 7), weights);
}

#if FV3_TU_MAIN
void enqueue_halo_fields(Ctx& c, const std::vector<HaloField>& fields, cudaStream_t st) {
  for (size_t base = 0; base < fields.size(); base += MAX_HALO_FIELDS) {
    HaloBatch b{};
    int nf = 0, maxc = 0, maxl = 0;
    for (size_t i = base; i < fields.size() && nf < MAX_HALO_FIELDS; ++i, ++nf) {
      b.f[nf] = fields[i];
      maxc = std::max(maxc, fields[i].count);
      maxl = std::max(maxl, fields[i].nlev);
    }
    if (maxc == 0) continue;
    dim3 grid((maxc + 255) / 256, maxl, nf);
    if (c.prec == 0) k_halo<double><<<grid, 256, 0, st>>>(b, c.geo_d);
    else k_halo<float><<<grid, 256, 0, st>>>(b, c.geo_d);
    ++c.launches;
  }
}
#endif


static HaloField hf(const Ctx& c, int kind, void* xa, void* ya, int nlev, int iface) {
  HaloField f{};
  f.xa = xa;
  f.ya = ya;
  f.ent = c.plan_d[kind];
  f.count = c.plan_n[kind];
  f.nlev = nlev;
  f.iface = iface;
  return f;
}

#if FV3_TU_MAIN
void enqueue_halo_prognostics(Ctx& c, const StateView& s, cudaStream_t st) {
  std::vector<HaloField> F;
  F.push_back(hf(c, K_DGRID, s.v, s.u, c.nz, 0));
  F.push_back(hf(c, K_CELL3, s.w, nullptr, c.nz, 0));
  F.push_back(hf(c, K_CELL3, s.delp, nullptr, c.nz, 0));
  F.push_back(hf(c, K_CELL3, s.pt, nullptr, c.nz, 0));
  F.push_back(hf(c, K_CELL3, s.delz, nullptr, c.nz, 0));
  enqueue_halo_fields(c, F, st);
}
#endif


template <typename R, typename MR = R>
static void substep_t(Ctx& c, const StateView& in, const StateView& out, const Params& P, bool acc,
                      cudaStream_t st, int stop_after, int only) {
  StepArgs<R> a{};
  a.geo = c.geo_d;
  a.items = c.items_hz;
  a.M = metric_of<R>(c);
  a.Md = c.Md;
  a.P = P;
  a.u = (const R*)in.u; a.v = (const R*)in.v; a.w = (const R*)in.w;
  a.delp = (const R*)in.delp; a.pt = (const R*)in.pt; a.delz = (const R*)in.delz;
  a.u_o = (R*)out.u; a.v_o = (R*)out.v; a.w_o = (R*)out.w; a.delp_o = (R*)out.delp; a.pt_o = (R*)out.pt;
  a.uc = (R*)c.uc; a.vc = (R*)c.vc; a.delpc = (R*)c.delpc; a.ptc = (R*)c.ptc; a.wc = (R*)c.wc;
  a.delzc = (R*)c.delzc; a.fx1 = (R*)c.fx1; a.fy1 = (R*)c.fy1; a.pef = (R*)c.pef; a.gz = (R*)c.gz;
  a.scratch = c.scratch;
  a.ncol = c.ncol;
  a.mlp = P.mlp;
  if (acc) {
    a.amfx = (R*)c.amfx; a.amfy = (R*)c.amfy; a.acrx = (R*)c.acrx; a.acry = (R*)c.acry;
    a.axfx = (R*)c.axfx; a.ayfx = (R*)c.ayfx;
  }
  a.status = c.status;
  const int kz = (c.nz + c.kchunk - 1) / c.kchunk;
  const int nwork = c.n_items_hz * kz;
  // stage ids: 0 halo fill, 1 c_sw, 2 update_dz_c, 3 riem_solver_c,
  // 4 pef/gz halo + p_grad_c, 5 C-grid halo, 6 d_sw
  // 7 update_dz_d, 8 riem_solver3, 9 pef/gz halo + D-grid p_grad (nh_full)
  auto run = [&](int stage) {
    if (stage >= 7 && !P.nh_full) return false;
    if (only >= 0) return stage == only;
    const int last = (stop_after == 5 || stop_after == 6) ? 6 : stop_after;
    return stage <= last;
  };
  if (P.nh_full) {
    a.xfxd = (R*)c.fx1;  // c_sw's fluxes are dead once update_dz_c has run
    a.yfxd = (R*)c.fy1;
    a.delz_o = (R*)out.delz;
  }
  if (run(0)) enqueue_halo_prognostics(c, in, st);
  if (run(1)) {  // c_sw
    const size_t sm = blk_smem(c, 13);
    const bool full = full_blocks(c);
#define FV3_CSW(X, Y)                                                                  \
  (full ? launch_c_sw<R, X, Y, MR, true>(c, a, sm, nwork, st) : launch_c_sw<R, X, Y, MR>(c, a, sm, nwork, st))
    FV3_DISPATCH_SHAPE(c.BX, c.BY, FV3_CSW);
#undef FV3_CSW
    ++c.launches;
  }
  if (run(2)) {  // update_dz_c
    StepArgs<R> b = a;
    b.items = c.items_dz;
    k_update_dz_c<R, MR><<<dim3(c.n_items_dz), dim3(kDzBX * kDzBY), 0, st>>>(b);
    ++c.launches;
  }
  if (run(3)) {  // riem_solver_c
    k_riem_c<R, false><<<dim3((c.max_n + kRiemCols - 1) / kRiemCols, c.n_rows), kRiemCols, 0, st>>>(a, c.rows);
    ++c.launches;
  }
  if (run(4)) {  // pef, gz one ring into the halo, then p_grad_c
    std::vector<HaloField> F;
    F.push_back(hf(c, K_CELL1, c.pef, nullptr, c.nz + 1, 1));
    F.push_back(hf(c, K_CELL1, c.gz, nullptr, c.nz + 1, 1));
    enqueue_halo_fields(c, F, st);
    const int nbi = (c.max_n + 15) / 16, ne = (2 * c.max_n + 255) / 256;
    k_p_grad_c<R, MR><<<dim3(nbi * nbi + ne, 1, c.n_planes), dim3(16, 16), 0, st>>>(a, c.planes, nbi);
    ++c.launches;
  }
  if (run(5)) {  // C-grid winds into the halo
    std::vector<HaloField> F;
    F.push_back(hf(c, K_CGRID, c.uc, c.vc, c.nz, 0));
    enqueue_halo_fields(c, F, st);
  }
  if (run(6)) {  // d_sw
    const size_t sm = blk_smem_mr<R, MR>(c, 19, true);
    const bool learn = P.hord == 1 && P.mlp;
    const bool full = full_blocks(c);
#define FV3_DSW(X, Y)                                                                  \
  (learn  ? launch_d_sw<R, X, Y, true, MR>(c, a, sm, nwork, st)                        \
   : full ? launch_d_sw<R, X, Y, false, MR, true>(c, a, sm, nwork, st)                 \
          : launch_d_sw<R, X, Y, false, MR>(c, a, sm, nwork, st))
    FV3_DISPATCH_SHAPE(c.BX, c.BY, FV3_DSW);
#undef FV3_DSW
    ++c.launches;
  }
  if (run(6) && (P.d2_bg > 0.0 || P.dddmp > 0.0)) {  // divergence damping of d_sw's winds
    const int nb = (c.max_n + 1 + 15) / 16;
    k_div_damp<R, MR><<<dim3(nb, nb, c.n_planes), dim3(16, 16), 0, st>>>(a, c.planes);
    ++c.launches;
  }
  if (run(7)) {  // update_dz_d: the D-grid area fluxes of d_sw over the state delz
    StepArgs<R> b = a;
    b.items = c.items_dz;
    k_update_dz_c<R, MR><<<dim3(c.n_items_dz), dim3(kDzBX * kDzBY), 0, st>>>(b);
    ++c.launches;
  }
  if (run(8)) {  // riem_solver3 on the state after d_sw
    StepArgs<R> b = a;
    b.delpc = (R*)out.delp;
    b.ptc = (R*)out.pt;
    b.wc = (R*)out.w;
    k_riem_c<R, true><<<dim3((c.max_n + kRiemCols - 1) / kRiemCols, c.n_rows), kRiemCols, 0, st>>>(b, c.rows);
    ++c.launches;
  }
  if (run(9)) {  // pef, gz into the halo, then the D-grid pressure gradient
    // (the corner means need the diagonal halo cells too, which the depth-1
    // plan of p_grad_c leaves out: the full plan fills them)
    std::vector<HaloField> F;
    F.push_back(hf(c, K_CELL3, c.pef, nullptr, c.nz + 1, 1));
    F.push_back(hf(c, K_CELL3, c.gz, nullptr, c.nz + 1, 1));
    enqueue_halo_fields(c, F, st);
    const int nb = (c.max_n + 1 + 15) / 16;
    k_p_grad_d<R, MR><<<dim3(nb, nb, c.n_planes), dim3(16, 16), 0, st>>>(a, c.planes);
    ++c.launches;
  }
}

#if FV3_TU_F64
void enqueue_substep_f64(Ctx& c, const StateView& in, const StateView& out, const Params& P, bool accumulate,
                         cudaStream_t st, int stop_after, int only) {
  substep_t<double>(c, in, out, P, accumulate, st, stop_after, only);
}
#endif
#if FV3_TU_F32
void enqueue_substep_f32(Ctx& c, const StateView& in, const StateView& out, const Params& P, bool accumulate,
                         cudaStream_t st, int stop_after, int only) {
  substep_t<float>(c, in, out, P, accumulate, st, stop_after, only);
}
#endif
#if FV3_TU_F32M64
void enqueue_substep_f32m64(Ctx& c, const StateView& in, const StateView& out, const Params& P, bool accumulate,
                            cudaStream_t st, int stop_after, int only) {
  substep_t<float, double>(c, in, out, P, accumulate, st, stop_after, only);
}
#endif
#if FV3_TU_MAIN
void enqueue_substep(Ctx& c, const StateView& in, const StateView& out, const Params& P, bool accumulate,
                     cudaStream_t st, int stop_after, int only) {
  if (c.prec == 0) enqueue_substep_f64(c, in, out, P, accumulate, st, stop_after, only);
  else if (c.prec == 2) enqueue_substep_f32m64(c, in, out, P, accumulate, st, stop_after, only);
  else enqueue_substep_f32(c, in, out, P, accumulate, st, stop_after, only);
}
#endif

template <typename R>
static void copy_planes_t(Ctx& c, const std::vector<std::pair<void*, const void*>>& pairs, const int* gate, int it,
                          cudaStream_t st) {
  CopyArgs<R> a{};
  a.nf = (int)pairs.size();
  for (int f = 0; f < a.nf; ++f) {
    a.dst[f] = (R*)pairs[f].first;
    a.src[f] = (const R*)pairs[f].second;
  }
  const int nb = c.max_n + 1;
  k_copy_planes<R><<<dim3((nb + 31) / 32, (nb + 7) / 8, c.n_planes), dim3(32, 8), 0, st>>>(c.geo_d, c.planes, a,
                                                                                             gate, it);
  ++c.launches;
}

static void copy_planes(Ctx& c, const std::vector<std::pair<void*, const void*>>& pairs, const int* gate, int it,
                        cudaStream_t st) {
  if (c.prec == 0) copy_planes_t<double>(c, pairs, gate, it, st);
  else copy_planes_t<float>(c, pairs, gate, it, st);
}

#if FV3_TU_MAIN
void enqueue_copy_state(Ctx& c, const StateView& dst, const StateView& src, cudaStream_t st) {
  copy_planes(c, {{dst.u, src.u}, {dst.v, src.v}, {dst.w, src.w}, {dst.delp, src.delp}, {dst.pt, src.pt}}, nullptr,
              0, st);
}

// vertical remapping (reading R16): delp halo for the face columns, the
// column kernel into the context's buffers, then back into the state
void enqueue_remap(Ctx& c, const StateView& s, const Params& P, cudaStream_t st) {
  std::vector<HaloField> F;
  F.push_back(hf(c, K_CELL3, s.delp, nullptr, c.nz, 0));
  enqueue_halo_fields(c, F, st);
  enqueue_remap_kernel(c, s, P.ptop, st);
  std::vector<std::pair<void*, const void*>> pairs = {{s.u, c.nu},   {s.v, c.nv},   {s.w, c.nw},
                                                      {s.delp, c.ndelp}, {s.pt, c.npt}, {s.delz, c.delzc}};
  for (int q = 0; q < s.nq; ++q) pairs.push_back({s.q[q], c.qtmp[q]});
  for (size_t b = 0; b < pairs.size(); b += MAX_TRACERS + 1) {
    std::vector<std::pair<void*, const void*>> part(pairs.begin() + b,
                                                    pairs.begin() + std::min(pairs.size(), b + MAX_TRACERS + 1));
    copy_planes(c, part, nullptr, 0, st);
  }
}

void enqueue_zero_acc(Ctx& c, cudaStream_t st) {
  const size_t b = c.elems3 * c.esize;
  void* acc[6] = {c.amfx, c.amfy, c.acrx, c.acry, c.axfx, c.ayfx};
  for (void* p : acc) cudaMemsetAsync(p, 0, b, st);
}

void enqueue_save_dpstart(Ctx& c, const void* delp, cudaStream_t st) {
  copy_planes(c, {{c.dpstart, delp}}, nullptr, 0, st);
}
#endif


template <typename R, typename MR = R>
static void tracers_t(Ctx& c, const StateView& s, const Params& P, cudaStream_t st) {
  std::vector<HaloField> F;
  F.push_back(hf(c, K_CGRID, c.amfx, c.amfy, c.nz, 0));
  F.push_back(hf(c, K_CGRID, c.acrx, c.acry, c.nz, 0));
  F.push_back(hf(c, K_CGRID, c.axfx, c.ayfx, c.nz, 0));
  enqueue_halo_fields(c, F, st);
  cudaMemsetAsync(c.cmax, 0, sizeof(unsigned), st);
  {
    const int nb = (c.max_n + 15) / 16;
    k_cmax<R><<<dim3(nb, nb, c.n_planes), dim3(16, 16), 0, st>>>(c.geo_d, c.planes, (const R*)c.acrx,
                                                                 (const R*)c.acry, c.cmax);
    k_nsplt<R><<<1, 1, 0, st>>>(c.cmax, c.nsplt, NSPLT_MAX, c.status, (const R*)nullptr);
    c.launches += 2;
  }
  copy_planes(c, {{c.dp0, c.dpstart}}, nullptr, 0, st);
  TracerArgs<R> a{};
  a.geo = c.geo_d;
  a.items = c.items_hz;
  a.M = metric_of<R>(c);
  a.Md = c.Md;
  a.nq = s.nq;
  a.nsplt = c.nsplt;
  for (int q = 0; q < s.nq; ++q) {
    a.q[q] = (const R*)s.q[q];
    a.q_o[q] = (R*)c.qtmp[q];
  }
  a.acrx = (const R*)c.acrx; a.acry = (const R*)c.acry; a.axfx = (const R*)c.axfx; a.ayfx = (const R*)c.ayfx;
  a.amfx = (const R*)c.amfx; a.amfy = (const R*)c.amfy;
  a.dp0 = (const R*)c.dp0;
  a.dp1 = (R*)c.dp1;
  a.mlp = P.mlp;
  a.learn = P.hord == 1 && P.mlp != nullptr;
  const int kz = (c.nz + c.kchunk - 1) / c.kchunk;
  const int nwork = c.n_items_hz * kz;
  const bool pair = a.learn ? kTracerPair<R, true> : kTracerPair<R, false>;
  const size_t sm = blk_smem_mr<R, MR>(c, 16 + (pair ? 6 : 0), false);
  const bool full = full_blocks(c);
  for (int it = 0; it < NSPLT_MAX; ++it) {
    std::vector<HaloField> Q;
    for (int q = 0; q < s.nq; ++q) Q.push_back(hf(c, K_CELL3, s.q[q], nullptr, c.nz, 0));
    enqueue_halo_fields(c, Q, st);
    a.it = it;
#define FV3_TRC(X, Y)                                                                  \
  (a.learn ? launch_tracer<R, X, Y, true, MR>(c, a, sm, nwork, st)                     \
   : full  ? launch_tracer<R, X, Y, false, MR, true>(c, a, sm, nwork, st)                \
           : launch_tracer<R, X, Y, false, MR>(c, a, sm, nwork, st))
    FV3_DISPATCH_SHAPE(c.BX, c.BY, FV3_TRC);
#undef FV3_TRC
    ++c.launches;
    std::vector<std::pair<void*, const void*>> pairs;
    for (int q = 0; q < s.nq; ++q) pairs.push_back({s.q[q], c.qtmp[q]});
    pairs.push_back({c.dp0, c.dp1});
    copy_planes(c, pairs, c.nsplt, it, st);
  }
}

#if FV3_TU_F64
void enqueue_tracers_f64(Ctx& c, const StateView& s, const Params& P, cudaStream_t st) {
  tracers_t<double>(c, s, P, st);
}
#endif
#if FV3_TU_F32
void enqueue_tracers_f32(Ctx& c, const StateView& s, const Params& P, cudaStream_t st) {
  tracers_t<float>(c, s, P, st);
}
#endif
#if FV3_TU_F32M64
void enqueue_tracers_f32m64(Ctx& c, const StateView& s, const Params& P, cudaStream_t st) {
  tracers_t<float, double>(c, s, P, st);
}
#endif
template <typename R, typename MR = R>
static void fv_tp_2d_t(Ctx& c, const TpPtrs& p, cudaStream_t st) {
  TpArgs<R> a{};
  a.geo = c.geo_d;
  a.items = c.items_hz;
  a.M = metric_of<R>(c);
  a.Md = c.Md;
  a.q = (const R*)p.q; a.crx = (const R*)p.crx; a.cry = (const R*)p.cry;
  a.xfx = (const R*)p.xfx; a.yfx = (const R*)p.yfx;
  a.mfx = (const R*)p.mfx; a.mfy = (const R*)p.mfy;
  a.fx = (R*)p.fx; a.fy = (R*)p.fy;
  a.damp = p.damp;
  const int kz = (c.nz + c.kchunk - 1) / c.kchunk;
  const int nwork = c.n_items_hz * kz;
  const size_t sm = blk_smem_mr<R, MR>(c, 14, true);
#define FV3_TP(X, Y)                                                                   \
  set_smem(k_fv_tp_2d<R, X, Y, MR>, sm);                                               \
  k_fv_tp_2d<R, X, Y, MR><<<work_grid(c, k_fv_tp_2d<R, X, Y, MR>, sm, nwork), dim3(32, 8), sm, st>>>(a, c.kchunk, \
                                                                                                     nwork)
  FV3_DISPATCH_SHAPE(c.BX, c.BY, FV3_TP);
#undef FV3_TP
  ++c.launches;
}
#if FV3_TU_F64
void enqueue_fv_tp_2d_f64(Ctx& c, const TpPtrs& p, cudaStream_t st) { fv_tp_2d_t<double>(c, p, st); }
#endif
#if FV3_TU_F32
void enqueue_fv_tp_2d_f32(Ctx& c, const TpPtrs& p, cudaStream_t st) { fv_tp_2d_t<float>(c, p, st); }
#endif
#if FV3_TU_F32M64
void enqueue_fv_tp_2d_f32m64(Ctx& c, const TpPtrs& p, cudaStream_t st) { fv_tp_2d_t<float, double>(c, p, st); }
#endif

#if FV3_TU_MAIN
void enqueue_fv_tp_2d(Ctx& c, const TpPtrs& p, cudaStream_t st) {
  std::vector<HaloField> F;
  F.push_back(hf(c, K_CELL3, p.q, nullptr, c.nz, 0));
  F.push_back(hf(c, K_CGRID, p.crx, p.cry, c.nz, 0));
  F.push_back(hf(c, K_CGRID, p.xfx, p.yfx, c.nz, 0));
  if (p.mfx) F.push_back(hf(c, K_CGRID, p.mfx, p.mfy, c.nz, 0));
  enqueue_halo_fields(c, F, st);
  if (c.prec == 0) enqueue_fv_tp_2d_f64(c, p, st);
  else if (c.prec == 2) enqueue_fv_tp_2d_f32m64(c, p, st);
  else enqueue_fv_tp_2d_f32(c, p, st);
}

void enqueue_tracers(Ctx& c, const StateView& s, const Params& P, cudaStream_t st) {
  if (s.nq <= 0) return;
  if (c.prec == 0) enqueue_tracers_f64(c, s, P, st);
  else if (c.prec == 2) enqueue_tracers_f32m64(c, s, P, st);
  else enqueue_tracers_f32(c, s, P, st);
}
#endif

#if FV3_TU_MAIN
template <typename R>
static void check_finite_t(Ctx& c, const StateView& s, cudaStream_t st) {
  CheckArgs<R> a{};
  const void* f[6] = {s.u, s.v, s.w, s.delp, s.pt, s.delz};
  const int k6[6] = {2, 1, 0, 0, 0, 0};
  std::vector<std::pair<const void*, int>> all;
  for (int q = 0; q < 6; ++q) all.push_back({f[q], k6[q]});
  for (int q = 0; q < s.nq; ++q) all.push_back({s.q[q], 0});
  for (size_t b = 0; b < all.size(); b += MAX_TRACERS + 1) {
    a.nf = 0;
    for (size_t q = b; q < all.size() && a.nf < MAX_TRACERS + 1; ++q, ++a.nf) {
      a.src[a.nf] = (const R*)all[q].first;
      a.kind[a.nf] = all[q].second;
    }
    const int nb = c.max_n + 1;
    k_check_finite<R><<<dim3((nb + 31) / 32, (nb + 7) / 8, c.n_planes), dim3(32, 8), 0, st>>>(c.geo_d, c.planes, a,
                                                                                               c.status);
    ++c.launches;
  }
}

void enqueue_check_finite(Ctx& c, const StateView& s, cudaStream_t st) {
  if (c.prec == 0) check_finite_t<double>(c, s, st);
  else check_finite_t<float>(c, s, st);
}

void enqueue_mass(Ctx& c, const void* delp, cudaStream_t st) {
  if (c.prec == 0)
    k_mass_partial<double><<<c.n_planes, 256, 0, st>>>(c.geo_d, c.planes, (const double*)delp, c.Md.area,
                                                       c.mass_part);
  else
    k_mass_partial<float><<<c.n_planes, 256, 0, st>>>(c.geo_d, c.planes, (const float*)delp, c.Md.area,
                                                      c.mass_part);
  k_mass_final<<<(c.nmem + 63) / 64, 64, 0, st>>>(c.mass_part, c.mass_first, c.nmem, c.mass_out);
  c.launches += 2;
}

void enqueue_pack(Ctx& c, int member, int kind, int nlev, int iface, void* padded, void* dense, int dense_is_double,
                  int dir, cudaStream_t st) {
  const int blocks = 1024;
  ++c.launches;
  if (c.prec == 0 || iface == 2) {
    if (dense_is_double)
      k_pack<double, double><<<blocks, 256, 0, st>>>(c.geo_d, member, kind, nlev, iface, (double*)padded,
                                                     (double*)dense, dir);
    else
      k_pack<double, float><<<blocks, 256, 0, st>>>(c.geo_d, member, kind, nlev, iface, (double*)padded,
                                                    (float*)dense, dir);
  } else {
    if (dense_is_double)
      k_pack<float, double><<<blocks, 256, 0, st>>>(c.geo_d, member, kind, nlev, iface, (float*)padded,
                                                    (double*)dense, dir);
    else
      k_pack<float, float><<<blocks, 256, 0, st>>>(c.geo_d, member, kind, nlev, iface, (float*)padded,
                                                   (float*)dense, dir);
  }
}

#endif

#if FV3_TU_F64
// ------------------------------------------------------------------------
// stencil exports (FP64; readings R4, R14): the PPM face value, the clamped
// edge value and the network inputs of single six-cell stencils q6[f][0..5]
// (the face between q6[f][2] and q6[f][3]), formed by the same device
// functions as the transports (edge values first, then the limited parabola
// of the upwind cell), and the learned face value of the FP64 transport
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_face_stencils(const double* q6, const double* cr, int n, double* plain,
                                                       double* edge, float* x, float* sig) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n; f += gridDim.x * blockDim.x) {
    double q[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = q6[6 * (long long)f + k];
    if (plain) {
      // AL[l]: edge between q[l - 1] and q[l], l = 2, 3, 4
      double al[5];
#pragma unroll
      for (int l = 2; l <= 4; ++l) al[l] = ppm_edge<double>(q[l - 2], q[l - 1], q[l], q[l + 1]);
      plain[f] = ppm_face_al<double>(q, al, 3, 1, upwind_weight(cr[f]));
    }
    if (edge) edge[f] = ppm_edge<double>(q[1], q[2], q[3], q[4]);
    if (x || sig) {
      float xi[6], xr[6];
      const float sg = mlp_inputs<double>(q, xi, xr);
      if (x)
        for (int k = 0; k < 6; ++k) x[6 * (long long)f + k] = xi[k];
      if (sig) sig[f] = sg;
    }
  }
}

// learned face values: 256 stencils per CTA laid out as rows of a
// shared-memory tile (cells i = -3 .. 2 of row j, the face at i = 0), so that
// the transport's warp-level evaluation learned_faces runs unchanged
constexpr int kStencilRows = 256, kStencilSX = 8;

__global__ void __launch_bounds__(256) k_learned_stencils(const float* w, const double* q6, const double* cr, int n,
                                                          double* value) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int SA = (kStencilRows + 6) * kStencilSX;
  double* Q = reinterpret_cast<double*>(smraw);
  double *AL = Q + SA, *CC = Q + 2 * SA, *OUT = Q + 3 * SA;
  MlpFrag F;
  mlp_load(w, F);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int f0 = blockIdx.x * kStencilRows; f0 < n; f0 += gridDim.x * kStencilRows) {
    const int rows = min(kStencilRows, n - f0);
    const Blk B{0, 1, 0, rows, kStencilSX};
    for (int e = tid; e < rows * 6; e += 256) {
      const int j = e / 6, k = e % 6;
      Q[B.L(k - 3, j)] = q6[6 * (long long)(f0 + j) + k];
    }
    for (int j = tid; j < rows; j += 256) CC[B.L(0, j)] = upwind_weight(cr[f0 + j]);
    __syncthreads();
    for (int e = tid; e < rows * 3; e += 256) {
      const int j = e / 3, i = e % 3 - 1;  // edges i = -1, 0, 1
      const int l = B.L(i, j);
      AL[l] = ppm_edge<double>(Q[l - 2], Q[l - 1], Q[l], Q[l + 1]);
    }
    __syncthreads();
    learned_faces<double>(Q, AL, CC, OUT, 0, 1, 0, rows, 1, B, F);
    __syncthreads();
    for (int j = tid; j < rows; j += 256) value[f0 + j] = OUT[B.L(0, j)];
    __syncthreads();
  }
}

cudaError_t launch_face_stencils(const double* q6, const double* cr, int n, double* plain, double* edge, float* x,
                                 float* sig, cudaStream_t st) {
  const int blocks = std::min((n + 255) / 256, 152 * 8);
  k_face_stencils<<<blocks, 256, 0, st>>>(q6, cr, n, plain, edge, x, sig);
  return cudaGetLastError();
}

cudaError_t launch_learned_stencils(const float* w, const double* q6, const double* cr, int n, double* value,
                                    cudaStream_t st) {
  const size_t sm = 4 * sizeof(double) * (kStencilRows + 6) * kStencilSX;
  cudaError_t e = cudaFuncSetAttribute(k_learned_stencils, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int blocks = std::min((n + kStencilRows - 1) / kStencilRows, 152 * 2);
  k_learned_stencils<<<blocks, dim3(32, 8), sm, st>>>(w, q6, cr, n, value);
  return cudaGetLastError();
}
#endif

}  // namespace fv3

// fv3_dev.cuh -- device-side layout and helpers of the FV3 substep library.
//
// Layout (paper Section VII-A3/A4: I-contiguous FORTRAN order, pre-padded so
// that the first interior element of every row is 128-byte aligned; horizontal
// stencils map I to threadIdx.x, vertical solvers keep K inside a thread).
// One member ("domain") = nt tiles of n x n cells, nz levels, halo 3.
// Every field plane of a member uses the same geometry: `rows` = n + 1 + 2*3
// rows of `pitch` elements; element (i, j) of a plane sits at
// (j + 3) * pitch + ox + i, with ox the aligned column of i = 0.  Cell, x-face,
// y-face and corner arrays all use that geometry (faces have one more column
// or row).  A 3-D field of a member is [tile][level][plane]; the fields of all
// members are concatenated in one buffer at per-member offsets.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fv3 {

constexpr int HALO = 3;

// status bits raised by kernels (read by fv3_check_status)
enum : unsigned { ST_CFL = 1u, ST_NONFINITE = 2u, ST_NSPLT = 4u };

struct Geo {            // per member, device side
  int n, nz, nt, cubed; // cells per tile edge, levels, tiles, cube flag
  int pitch, rows, ox;  // row pitch (elements), rows per plane, column of i = 0
  int pad0;
  long long plane;      // elements per plane
  long long off3;       // offset of the member in [tile][nz][plane] buffers
  long long offi;       // offset in interface buffers [tile][nz+1][plane]
  long long off2;       // offset in metric buffers [tile][plane]
  long long colbase;    // first column id of the member (riem scratch)
  double da_min;        // smallest cell area of the member (damping scale)
};

__host__ __device__ inline long long pidx(const Geo& g, int j, int i) {
  return (long long)(j + HALO) * g.pitch + g.ox + i;
}

// metric of all members (FP64 master copy and the arithmetic-precision copy)
template <typename R>
struct Metric {
  const R *area, *rarea, *fA;                          // cells
  const R *dx, *rdx, *dyc, *rdyc, *cosy, *siny, *rsin2y; // y-faces
  const R *dy, *rdy, *dxc, *rdxc, *cosx, *sinx, *rsin2x; // x-faces
  const R *fC, *rareac;                                // corners
  const R *wx, *wy;  // dy/dxc on x-faces, dx/dyc on y-faces (damping weights)
  // area-flux and Courant-number factors of the contravariant wind:
  // dy / sin and 1 / (dxc sin) on x-faces, dx / sin and 1 / (dyc sin) on
  // y-faces (xfx = dt (uc - cos v) kfx, crx = dt (uc - cos v) kcx)
  const R *kfx, *kcx, *kfy, *kcy;
};

struct Params {
  double dt, d4_bg, a_imp, dz_min, ptop, grav, rdgas, cp_air, d2_bg, dddmp;
  int n_split, nord, hord, remap, nh_full, d2c_ord;
  const float* mlp;  // face-value network parameters (hord 1)
};

// halo-plan entry: destination slot <- sign * source value (sign 0: NaN)
struct HaloEntry {
  int dst, src;          // plane offsets (pidx) of destination and source
  short m;               // member
  unsigned char dt, st;  // destination / source tile
  signed char sign;      // +1, -1, or 0 for "no value" (NaN)
  unsigned char flags;   // bit 0: destination is the y-face array; bit 1: source is
  short pad;
};

// work item of the horizontal kernels: one CTA block of one tile of a member
struct Item {
  int m, t, x0, y0;
};

}  // namespace fv3

// fv3_remap.cu -- vertical remapping of every column (reading R16).
//
// arxiv 2205.04148, Section II: the dynamical core integrates on Lagrangian
// surfaces and remaps them to reference levels after the acoustic substeps.
// The paper gives no formula; the reading: reference layers equally spaced in
// pressure between the model top and the column's surface pressure; each
// field reconstructed per layer as a parabola (edge values and monotone
// limiter of the horizontal PPM, reading R4; the outermost edges take the
// layer values and the edges next to them the mean of their two layers) and
// integrated exactly over the overlaps of old and new layers.  delp becomes
// the reference thickness; pt, w and the tracers are mass-weighted means;
// delz is remapped as delz / delp; u and v on their face columns, whose
// interfaces are the means of the two neighbouring cell columns' interfaces.
//
// One thread per column and group of up to four cell fields (u on y-face
// columns and v on x-face columns alone), levels in sequence: the old and new
// interfaces advance together, so the walk over the overlaps needs only a
// four-layer window of each field, and the overlap geometry is formed once
// for the group.  Arithmetic in FP64 for both storage precisions.
#include <cuda_runtime.h>

#include "fv3_kernels.cuh"
#include "fv3_math.cuh"

namespace fv3 {

// edge e (between layers e-1 and e) from the layer means qm2..qp1 =
// q[e-2], q[e-1], q[e], q[e+1] (entries outside the column are not read)
__device__ __forceinline__ double remap_edge(int e, int nz, double qm2, double qm1, double q0, double qp1) {
  if (e == 0) return q0;
  if (e == nz) return qm1;
  const double a = (e == 1 || e == nz - 1) ? 0.5 * (qm1 + q0)
                                           : 7.0 / 12.0 * (qm1 + q0) - 1.0 / 12.0 * (qm2 + qp1);
  // clamp into the range of the two layers, compares on the integer pipe
  const long long k0 = okey(qm1), k1 = okey(q0), ka = okey(a);
  const bool o = k0 < k1;
  const double lo = o ? qm1 : q0, hi = o ? q0 : qm1;
  return ka < (o ? k0 : k1) ? lo : (ka > (o ? k1 : k0) ? hi : a);
}

template <typename R>
struct ColumnSrc {  // one field of one column: value(k), level stride
  const R* p;
  const R* dp;  // non-null: the value is p / dp (delz as delz / delp)
  long long stride;
  __device__ __forceinline__ double at(int k) const {
    const double v = (double)p[k * stride];
    return dp ? v * rcp((double)dp[k * stride]) : v;
  }
};

// interfaces of a column (cell column a, or the mean of cell columns a and b)
template <typename R>
struct ColumnP {
  const R* dpa;
  const R* dpb;  // null for a cell column
  long long stride;
  double ptop, psa, psb, rnz;
  int nz;
  // old interfaces below layer k of columns a and b from those above it
  __device__ __forceinline__ void next_old(int k, double pe_a, double pe_b, double* na, double* nb) const {
    *na = pe_a + (double)dpa[k * stride];
    *nb = dpb ? pe_b + (double)dpb[k * stride] : 0.0;
  }
  // new interface k of column a (or b)
  __device__ __forceinline__ double pn1(double ps, int k) const {
    return k == nz ? ps : ptop + (ps - ptop) * ((double)k * rnz);
  }
  __device__ __forceinline__ double pn(int k) const {
    return dpb ? 0.5 * (pn1(psa, k) + pn1(psb, k)) : pn1(psa, k);
  }
};

// Remap NF fields of one column together: the overlaps of old and new layers
// (their pressure widths and the weights of the parabola terms) are formed
// once and applied to every field.  The limited parabola of an old layer
// (mean qb, edge values qb + bl and qb + br) integrates over the fraction
// [x1, x2] of the layer, of pressure width w, to
//   w (qb + bl (1 - 2 s1 + s2) + br (s2 - s1)),  s1 = x1 + x2,
//   s2 = x1^2 + x1 x2 + x2^2
// (a whole layer gives w qb).  out(f, k, value, dpn) receives the new layer
// means.
template <int NF, typename R, typename F>
__device__ void remap_walk(const ColumnP<R>& C, const ColumnSrc<R> (&src)[NF], F out) {
  const int nz = C.nz;
  // per field the window q[m-1 .. m+2] (the right edge of layer m needs no more)
  double w1[NF], w2[NF], w3[NF], w4[NF], al[NF], bl[NF], br[NF], mass[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    w1[f] = 0.0;
    w2[f] = src[f].at(0);
    w3[f] = nz > 1 ? src[f].at(1) : 0.0;
    w4[f] = nz > 2 ? src[f].at(2) : 0.0;
    al[f] = remap_edge(0, nz, 0.0, 0.0, w2[f], 0.0);  // left edge of layer 0
    mass[f] = 0.0;
  }
  double pa = C.ptop, pb = C.ptop;  // old interfaces of columns a, b
  int k = 0;
  double pn_lo = C.pn(0), pn_hi = C.pn(1);
  for (int m = 0; m < nz && k < nz; ++m) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const double ar = remap_edge(m + 1, nz, w1[f], w2[f], w3[f], w4[f]);  // right edge of layer m
      bl[f] = al[f] - w2[f];
      br[f] = ar - w2[f];
      ppm_limit(bl[f], br[f]);
      al[f] = ar;
    }
    double na, nb;
    C.next_old(m, pa, pb, &na, &nb);
    const double pe_lo = C.dpb ? 0.5 * (pa + pb) : pa;
    const double pe_hi = C.dpb ? 0.5 * (na + nb) : na;
    const double rdp = rcp(pe_hi - pe_lo);
    double x = pe_lo;
    while (true) {
      // pressures are positive: their bit patterns order like the values
      const long long khi = __double_as_longlong(pe_hi), knh = __double_as_longlong(pn_hi);
      const double top = knh < khi ? pn_hi : pe_hi;
      if (__double_as_longlong(top) > __double_as_longlong(x)) {
        const double x1 = (x - pe_lo) * rdp, x2 = (top - pe_lo) * rdp;
        const double s1 = x1 + x2, s2 = fma(x1, s1, x2 * x2);
        const double w = top - x, wl = w * (1.0 - 2.0 * s1 + s2), wr = w * (s2 - s1);
#pragma unroll
        for (int f = 0; f < NF; ++f) mass[f] = fma(w, w2[f], fma(wl, bl[f], fma(wr, br[f], mass[f])));
      }
      if (knh <= khi) {  // new layer k ends inside old layer m
        const double dpn = pn_hi - pn_lo, rdpn = rcp(dpn);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          out(f, k, mass[f] * rdpn, dpn);
          mass[f] = 0.0;
        }
        ++k;
        x = __double_as_longlong(top) > __double_as_longlong(x) ? top : x;
        if (k == nz) break;
        pn_lo = pn_hi;
        pn_hi = C.pn(k + 1);
        continue;
      }
      break;
    }
    pa = na;
    pb = nb;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      w1[f] = w2[f];
      w2[f] = w3[f];
      w3[f] = w4[f];
      w4[f] = m + 3 < nz ? src[f].at(m + 3) : 0.0;
    }
  }
}

// cell fields in groups of up to RG per thread
constexpr int RG = 4;

template <int NF, typename R>
__device__ __forceinline__ void remap_cells(const RemapArgs<R>& a, const ColumnP<R>& C, long long bq, int f0) {
  ColumnSrc<R> src[NF];
  R* o[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    src[f] = ColumnSrc<R>{a.in[f0 + f] + bq, f0 + f == 2 ? a.delp + bq : nullptr, C.stride};
    o[f] = a.out[f0 + f] + bq;
  }
  R* dpo = a.delp_o + bq;
  const long long stride = C.stride;
  remap_walk<NF>(C, src, [&](int f, int k, double v, double dpn) {
    o[f][k * stride] = (R)(f0 + f == 2 ? v * dpn : v);  // delz from delz / delp
    if (f0 + f == 0) dpo[k * stride] = (R)dpn;
  });
}

template <typename R>
__global__ void __launch_bounds__(128) k_remap(RemapArgs<R> a, const RowItem* rows) {
  const RowItem r = rows[blockIdx.y];
  const Geo g = a.geo[r.m];
  // z < ng: cell fields RG z .. RG z + RG - 1 (field 0 also writes delp);
  // ng: u (y-faces); ng + 1: v (x-faces)
  const int ng = (a.nf + RG - 1) / RG;
  const int z = blockIdx.z;
  const int kind = z < ng ? 0 : z == ng ? 1 : 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = r.j, n = g.n, nz = g.nz;
  if (kind == 0 && (i >= n || j >= n)) return;
  if (kind == 1 && (i >= n || j > n)) return;
  if (kind == 2 && (i > n || j >= n)) return;
  // origin (i = j = 0) of level 0 of tile t; levels are one plane apart
  const long long base = g.off3 + (long long)r.t * nz * g.plane + (long long)HALO * g.pitch + g.ox;
  const long long stride = g.plane;
  const long long q = (long long)j * g.pitch + i;
  // cell columns a (and b for the faces)
  const long long qa = kind == 1 ? q - g.pitch : kind == 2 ? q - 1 : q;
  ColumnP<R> C;
  C.dpa = a.delp + base + qa;
  C.dpb = kind == 0 ? nullptr : a.delp + base + q;
  C.stride = stride;
  C.ptop = a.ptop;
  C.nz = nz;
  C.rnz = 1.0 / nz;
  double psa = a.ptop, psb = a.ptop;
  for (int k = 0; k < nz; ++k) {
    psa += (double)C.dpa[k * stride];
    if (C.dpb) psb += (double)C.dpb[k * stride];
  }
  C.psa = psa;
  C.psb = psb;
  if (kind == 0) {
    const int f0 = z * RG, nfz = min(RG, a.nf - f0);
    if (nfz == 4) remap_cells<4>(a, C, base + q, f0);
    else if (nfz == 3) remap_cells<3>(a, C, base + q, f0);
    else if (nfz == 2) remap_cells<2>(a, C, base + q, f0);
    else remap_cells<1>(a, C, base + q, f0);
  } else {
    ColumnSrc<R> src[1] = {ColumnSrc<R>{(kind == 1 ? a.u : a.v) + base + q, nullptr, stride}};
    R* o = (kind == 1 ? a.u_o : a.v_o) + base + q;
    remap_walk<1>(C, src, [&](int, int k, double v, double) { o[k * stride] = (R)v; });
  }
}

template <typename R>
static void remap_t(Ctx& c, const RemapArgs<R>& a, cudaStream_t st) {
  const int nb = (c.max_n + 1 + 127) / 128;
  k_remap<R><<<dim3(nb, c.n_rows_f, (a.nf + RG - 1) / RG + 2), 128, 0, st>>>(a, c.rows_f);
  ++c.launches;
}

void enqueue_remap_kernel(Ctx& c, const StateView& s, double ptop, cudaStream_t st) {
  if (c.prec == 0) {
    RemapArgs<double> a{};
    a.geo = c.geo_d;
    a.ptop = ptop;
    a.delp = (const double*)s.delp;
    a.delp_o = (double*)c.ndelp;
    const void* in[3] = {s.pt, s.w, s.delz};
    void* out[3] = {c.npt, c.nw, c.delzc};
    for (int f = 0; f < 3; ++f) {
      a.in[f] = (const double*)in[f];
      a.out[f] = (double*)out[f];
    }
    for (int q = 0; q < s.nq; ++q) {
      a.in[3 + q] = (const double*)s.q[q];
      a.out[3 + q] = (double*)c.qtmp[q];
    }
    a.nf = 3 + s.nq;
    a.u = (const double*)s.u;
    a.v = (const double*)s.v;
    a.u_o = (double*)c.nu;
    a.v_o = (double*)c.nv;
    remap_t(c, a, st);
  } else {
    RemapArgs<float> a{};
    a.geo = c.geo_d;
    a.ptop = ptop;
    a.delp = (const float*)s.delp;
    a.delp_o = (float*)c.ndelp;
    const void* in[3] = {s.pt, s.w, s.delz};
    void* out[3] = {c.npt, c.nw, c.delzc};
    for (int f = 0; f < 3; ++f) {
      a.in[f] = (const float*)in[f];
      a.out[f] = (float*)out[f];
    }
    for (int q = 0; q < s.nq; ++q) {
      a.in[3 + q] = (const float*)s.q[q];
      a.out[3 + q] = (float*)c.qtmp[q];
    }
    a.nf = 3 + s.nq;
    a.u = (const float*)s.u;
    a.v = (const float*)s.v;
    a.u_o = (float*)c.nu;
    a.v_o = (float*)c.nv;
    remap_t(c, a, st);
  }
}

}  // namespace fv3

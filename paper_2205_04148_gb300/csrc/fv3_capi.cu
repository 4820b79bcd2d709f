// fv3_capi.cu -- the C-ABI of include/fv3.h: context, layout, validation,
// streams and the CUDA graph of a remapping step.
//
// The paper compiles the whole time-stepping loop into one library invoked as
// a single call (arxiv 2205.04148, Section II, Fig. 2 caption; Section VI-B
// orchestration).  Here every entry point only enqueues kernels on the
// caller's stream; fv3_run_dyn captures one remapping step (n_split acoustic
// substeps and the tracer step) into a CUDA graph once and replays it.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fv3.h"
#include "fv3_kernels.cuh"

using namespace fv3;

// staging slots of the asynchronous host copies: a slot is reused only after
// the event recorded behind its last copy, on whatever stream that ran
struct Slot {
  void* buf = nullptr;
  size_t bytes = 0;
  cudaEvent_t done = nullptr;
};
constexpr int kSlots = 4;

struct fv3_ctx {
  Ctx c;
  cudaStream_t cap = nullptr;   // private stream used only to capture graphs
  void* stage = nullptr;        // staging buffer for host <-> device copies
  size_t stage_bytes = 0;
  Slot ring[kSlots];            // staging of the asynchronous host copies
  int ring_next = 0;
};

namespace {

fv3_status fail(fv3_ctx* x, fv3_status s, const std::string& msg) {
  if (x) x->c.err = msg;
  return s;
}

#define CK(x, call)                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail(x, FV3_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
cudaError_t dalloc(Ctx& c, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e == cudaSuccess) {
    c.owned.push_back(q);
    *p = (T*)q;
  }
  return e;
}

cudaError_t dalloc_bytes(Ctx& c, void** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 1));
  if (e == cudaSuccess) {
    c.owned.push_back(q);
    *p = q;
    e = cudaMemset(q, 0, std::max<size_t>(bytes, 1));
  }
  return e;
}

bool aligned(const void* p) { return ((uintptr_t)p & 127u) == 0; }

fv3_status check_state(fv3_ctx* x, const fv3_state* s, bool need_tracers) {
  if (!s) return fail(x, FV3_ERR_ARG, "state is NULL");
  const void* f[6] = {s->u, s->v, s->w, s->delp, s->pt, s->delz};
  for (const void* p : f) {
    if (!p) return fail(x, FV3_ERR_ARG, "a state field is NULL");
    if (!aligned(p)) return fail(x, FV3_ERR_ALIGN, "a state field is not 128-byte aligned");
  }
  if (s->nq < 0 || s->nq > MAX_TRACERS) return fail(x, FV3_ERR_ARG, "nq out of range (0..16)");
  if (s->nq > 0) {
    if (!s->q) return fail(x, FV3_ERR_ARG, "q is NULL with nq > 0");
    for (int i = 0; i < s->nq; ++i) {
      if (!s->q[i]) return fail(x, FV3_ERR_ARG, "a tracer field is NULL");
      if (!aligned(s->q[i])) return fail(x, FV3_ERR_ALIGN, "a tracer field is not 128-byte aligned");
    }
  }
  (void)need_tracers;
  return FV3_OK;
}

fv3_status check_params(fv3_ctx* x, const fv3_params* p) {
  if (!p) return fail(x, FV3_ERR_ARG, "params is NULL");
  if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(x, FV3_ERR_ARG, "dt must be positive");
  if (p->n_split < 1) return fail(x, FV3_ERR_ARG, "n_split must be >= 1");
  if (p->nord != 1) return fail(x, FV3_ERR_UNSUPPORTED, "only nord = 1 (del-4 damping) is built");
  if (p->hord != 0 && p->hord != 1) return fail(x, FV3_ERR_UNSUPPORTED, "hord must be 0 (PPM) or 1 (learned)");
  if (p->hord == 1 && !p->mlp) return fail(x, FV3_ERR_ARG, "hord = 1 needs the network parameters (mlp)");
  if (p->remap != 0 && p->remap != 1) return fail(x, FV3_ERR_ARG, "remap must be 0 or 1");
  if (p->nh_full != 0 && p->nh_full != 1) return fail(x, FV3_ERR_ARG, "nh_full must be 0 or 1");
  if (p->d2c_ord != 0 && p->d2c_ord != 2 && p->d2c_ord != 4) return fail(x, FV3_ERR_ARG, "d2c_ord must be 2 or 4");
  if (!(p->d2_bg >= 0.0) || !(p->dddmp >= 0.0) || !std::isfinite(p->d2_bg) || !std::isfinite(p->dddmp))
    return fail(x, FV3_ERR_ARG, "d2_bg and dddmp must be finite and >= 0");
  if (!(p->a_imp > 0) || !(p->grav > 0) || !(p->rdgas > 0) || !(p->cp_air > p->rdgas) || !(p->ptop > 0) ||
      !(p->dz_min >= 0) || !(p->d4_bg >= 0))
    return fail(x, FV3_ERR_ARG, "physical constant out of range");
  return FV3_OK;
}

StateView view(const fv3_state* s) {
  StateView v{};
  v.u = s->u; v.v = s->v; v.w = s->w; v.delp = s->delp; v.pt = s->pt; v.delz = s->delz;
  v.nq = s->nq;
  for (int i = 0; i < s->nq; ++i) v.q[i] = s->q[i];
  return v;
}

Params to_params(const fv3_params* p) {
  Params P{};
  P.dt = p->dt; P.d4_bg = p->d4_bg; P.a_imp = p->a_imp; P.dz_min = p->dz_min; P.ptop = p->ptop;
  P.grav = p->grav; P.rdgas = p->rdgas; P.cp_air = p->cp_air;
  P.n_split = p->n_split; P.nord = p->nord; P.hord = p->hord; P.remap = p->remap; P.nh_full = p->nh_full;
  P.d2c_ord = p->d2c_ord == 0 ? 2 : p->d2c_ord;
  P.d2_bg = p->d2_bg;
  P.dddmp = p->dddmp;
  P.mlp = (const float*)p->mlp;
  return P;
}

// captured remapping steps kept at once (a few states or parameter sets)
constexpr int kMaxGraphs = 4;

void drop_graphs(Ctx& c) {
  for (Ctx::Graph& e : c.graphs) cudaGraphExecDestroy(e.exec);
  c.graphs.clear();
}

fv3_status ensure_stage(fv3_ctx* x, size_t bytes) {
  if (x->stage_bytes >= bytes) return FV3_OK;
  if (x->stage) cudaFree(x->stage);
  x->stage = nullptr;
  x->stage_bytes = 0;
  CK(x, cudaMalloc(&x->stage, bytes));
  x->stage_bytes = bytes;
  return FV3_OK;
}

std::vector<Item> block_items(const Ctx& c, int bx, int by) {
  std::vector<Item> hz;
  for (int m = 0; m < c.nmem; ++m) {
    const Geo& g = c.geo[m];
    for (int t = 0; t < g.nt; ++t)
      for (int y0 = 0; y0 < g.n; y0 += by)
        for (int x0 = 0; x0 < g.n; x0 += bx) hz.push_back({m, t, x0, y0});
  }
  return hz;
}

size_t dense_count(const Geo& g, int kind, int nlev) {
  const int n = g.n;
  const int ni = n + (kind == 1 || kind == 3), nj = n + (kind == 2 || kind == 3);
  return (size_t)g.nt * nlev * nj * ni;
}

}  // namespace

// ---------------------------------------------------------------------------
namespace {

// descriptor checks shared by fv3_init_grid and fv3_halo_plan; npx per member
fv3_status check_desc(const fv3_grid_desc* d, std::vector<int>& npx) {
  if (d->grid_type != FV3_GRID_PERIODIC && d->grid_type != FV3_GRID_CUBED) return FV3_ERR_ARG;
  if (d->precision != FV3_FP64 && d->precision != FV3_FP32 && d->precision != FV3_FP32_M64) return FV3_ERR_ARG;
  if (d->n_members < 1 || d->n_members > 4096 || d->npz < 2 || d->npz > 1024) return FV3_ERR_SHAPE;
  if (d->grid_type == FV3_GRID_PERIODIC && !(d->dx > 0)) return FV3_ERR_ARG;
  if (d->grid_type == FV3_GRID_CUBED && (!(d->radius > 0) || !std::isfinite(d->omega))) return FV3_ERR_ARG;
  npx.assign(d->n_members, 0);
  for (int m = 0; m < d->n_members; ++m) {
    npx[m] = d->member_npx ? d->member_npx[m] : d->npx;
    if (npx[m] < 8 || npx[m] > 4096) return FV3_ERR_SHAPE;
  }
  return FV3_OK;
}

// plane geometry of one member (offsets left to the caller)
void plane_geo(int n, int nz, int nt, bool cubed, int esize, Geo& g) {
  const int align = 128 / esize;  // elements per 128 bytes
  g.n = n;
  g.nz = nz;
  g.nt = nt;
  g.cubed = cubed ? 1 : 0;
  g.ox = align;  // first interior element of a row on a 128-byte boundary
  g.pitch = ((g.ox + g.n + 1 + HALO) + align - 1) / align * align;
  g.rows = g.n + 1 + 2 * HALO;
  g.plane = (long long)g.rows * g.pitch;
}

}  // namespace

extern "C" fv3_status fv3_init_grid(fv3_ctx** out, const fv3_grid_desc* d, fv3_stream stream) {
  (void)stream;
  if (!out || !d) return FV3_ERR_ARG;
  *out = nullptr;
  std::vector<int> npx;
  const fv3_status dr = check_desc(d, npx);
  if (dr != FV3_OK) return dr;
  fv3_ctx* x = new fv3_ctx();
  Ctx& c = x->c;
  c.spec.cubed = d->grid_type == FV3_GRID_CUBED;
  c.spec.dx = d->dx;
  c.spec.radius = d->radius;
  c.spec.omega = d->omega;
  c.nz = d->npz;
  c.nmem = d->n_members;
  c.prec = d->precision;
  c.esize = c.prec == FV3_FP64 ? 8 : 4;
  // default launch shapes, the autotuner's picks on one C96 x 80 state: FP64
  // 16 x 16 blocks, one level per work item, persistent grid; FP32 32 x 8
  // blocks, four levels per work item
  if (c.prec == FV3_FP64) {
    c.BX = 16; c.BY = 16; c.kchunk = 1; c.persistent = 1;
  } else {
    c.BX = 32; c.BY = 8; c.kchunk = std::min(4, d->npz); c.persistent = 0;
  }
  const int nt = c.spec.cubed ? 6 : 1;
  long long o3 = 0, oi = 0, o2 = 0, oc = 0;
  c.geo.resize(c.nmem);
  std::vector<HostMetric> HM(c.nmem);
  std::vector<Plans> PL(c.nmem);
  for (int m = 0; m < c.nmem; ++m) {
    Geo& g = c.geo[m];
    plane_geo(npx[m], c.nz, nt, c.spec.cubed, c.esize, g);
    g.off3 = o3;
    g.offi = oi;
    g.off2 = o2;
    g.colbase = oc;
    o3 += (long long)nt * c.nz * g.plane;
    oi += (long long)nt * (c.nz + 1) * g.plane;
    o2 += (long long)nt * g.plane;
    oc += (long long)nt * g.n * g.n;
    build_metric(c.spec, m, g, HM[m], PL[m]);
    g.da_min = HM[m].da_min;
    c.max_n = std::max(c.max_n, g.n);
  }
  c.elems3 = (size_t)o3;
  c.elemsi = (size_t)oi;
  c.elems2 = (size_t)o2;
  c.ncol = oc;

#define FAIL_INIT(call)                                                          \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      c.err = std::string(#call) + ": " + cudaGetErrorString(e_);               \
      fv3_destroy(x);                                                            \
      return FV3_ERR_CUDA;                                                       \
    }                                                                            \
  } while (0)

  FAIL_INIT(cudaStreamCreateWithFlags(&x->cap, cudaStreamNonBlocking));
  FAIL_INIT(dalloc(c, &c.geo_d, c.nmem));
  FAIL_INIT(cudaMemcpy(c.geo_d, c.geo.data(), sizeof(Geo) * c.nmem, cudaMemcpyHostToDevice));

  // metric: concatenate members, FP64 and FP32 copies
  {
    const int NM = 25;
    std::vector<double> all[NM];
    for (int q = 0; q < NM; ++q) all[q].assign(c.elems2, NAN);
    for (int m = 0; m < c.nmem; ++m) {
      const HostMetric& M = HM[m];
      const std::vector<double>* src[NM] = {&M.area, &M.rarea, &M.fA, &M.dx, &M.rdx, &M.dyc, &M.rdyc,
                                            &M.cosy, &M.siny, nullptr, &M.dy, &M.rdy, &M.dxc, &M.rdxc,
                                            &M.cosx, &M.sinx, nullptr, &M.fC, &M.rareac, nullptr, nullptr,
                                            nullptr, nullptr, nullptr, nullptr};
      const long long o = c.geo[m].off2;
      for (int q = 0; q < NM; ++q)
        if (src[q]) std::copy(src[q]->begin(), src[q]->end(), all[q].begin() + o);
      for (size_t e = 0; e < M.siny.size(); ++e) {
        all[9][o + e] = 1.0 / (M.siny[e] * M.siny[e]);
        all[16][o + e] = 1.0 / (M.sinx[e] * M.sinx[e]);
        all[19][o + e] = M.dy[e] * M.rdxc[e];
        all[20][o + e] = M.dx[e] * M.rdyc[e];
        all[21][o + e] = M.dy[e] / M.sinx[e];
        all[22][o + e] = M.rdxc[e] / M.sinx[e];
        all[23][o + e] = M.dx[e] / M.siny[e];
        all[24][o + e] = M.rdyc[e] / M.siny[e];
      }
    }
    double* dptr[NM];
    float* fptr[NM];
    for (int q = 0; q < NM; ++q) {
      FAIL_INIT(dalloc(c, &dptr[q], c.elems2));
      FAIL_INIT(cudaMemcpy(dptr[q], all[q].data(), sizeof(double) * c.elems2, cudaMemcpyHostToDevice));
      std::vector<float> f(all[q].begin(), all[q].end());
      FAIL_INIT(dalloc(c, &fptr[q], c.elems2));
      FAIL_INIT(cudaMemcpy(fptr[q], f.data(), sizeof(float) * c.elems2, cudaMemcpyHostToDevice));
    }
    auto fill = [&](auto& M, auto** p) {
      M.area = p[0]; M.rarea = p[1]; M.fA = p[2]; M.dx = p[3]; M.rdx = p[4]; M.dyc = p[5]; M.rdyc = p[6];
      M.cosy = p[7]; M.siny = p[8]; M.rsin2y = p[9]; M.dy = p[10]; M.rdy = p[11]; M.dxc = p[12]; M.rdxc = p[13];
      M.cosx = p[14]; M.sinx = p[15]; M.rsin2x = p[16]; M.fC = p[17]; M.rareac = p[18];
      M.wx = p[19]; M.wy = p[20];
      M.kfx = p[21]; M.kcx = p[22]; M.kfy = p[23]; M.kcy = p[24];
    };
    fill(c.Md, dptr);
    fill(c.Mf, fptr);
  }
  // plans
  for (int k = 0; k < K_NUM; ++k) {
    std::vector<HaloEntry> all;
    for (int m = 0; m < c.nmem; ++m) all.insert(all.end(), PL[m].p[k].begin(), PL[m].p[k].end());
    c.plan_n[k] = (int)all.size();
    FAIL_INIT(dalloc(c, &c.plan_d[k], all.size()));
    if (!all.empty())
      FAIL_INIT(cudaMemcpy(c.plan_d[k], all.data(), sizeof(HaloEntry) * all.size(), cudaMemcpyHostToDevice));
  }
  // work lists
  {
    std::vector<Item> hz, dz;
    std::vector<RowItem> rows, rows_f;
    std::vector<int4> planes;
    std::vector<int> mfirst;
    for (int m = 0; m < c.nmem; ++m) {
      const Geo& g = c.geo[m];
      mfirst.push_back((int)planes.size());
      for (int t = 0; t < nt; ++t) {
        for (int y0 = 0; y0 < g.n; y0 += kDzBY)
          for (int x0 = 0; x0 < g.n; x0 += kDzBX) dz.push_back({m, t, x0, y0});
        for (int j = 0; j < g.n; ++j) rows.push_back({m, t, j, 0});
        for (int j = 0; j <= g.n; ++j) rows_f.push_back({m, t, j, 0});
        for (int k = 0; k < c.nz; ++k) planes.push_back(make_int4(m, t, k, 0));
      }
    }
    mfirst.push_back((int)planes.size());
    hz = block_items(c, c.BX, c.BY);
    c.n_items_hz = (int)hz.size();
    c.n_items_dz = (int)dz.size();
    c.n_rows = (int)rows.size();
    c.n_rows_f = (int)rows_f.size();
    c.n_planes = (int)planes.size();
    if (c.n_rows_f > 65535 || c.n_planes > 65535) {
      c.err = "too many tiles x levels for one launch";
      fv3_destroy(x);
      return FV3_ERR_SHAPE;
    }
    FAIL_INIT(dalloc(c, &c.items_hz, hz.size()));
    FAIL_INIT(cudaMemcpy(c.items_hz, hz.data(), sizeof(Item) * hz.size(), cudaMemcpyHostToDevice));
    FAIL_INIT(dalloc(c, &c.items_dz, dz.size()));
    FAIL_INIT(cudaMemcpy(c.items_dz, dz.data(), sizeof(Item) * dz.size(), cudaMemcpyHostToDevice));
    FAIL_INIT(dalloc(c, &c.rows, rows.size()));
    FAIL_INIT(cudaMemcpy(c.rows, rows.data(), sizeof(RowItem) * rows.size(), cudaMemcpyHostToDevice));
    FAIL_INIT(dalloc(c, &c.rows_f, rows_f.size()));
    FAIL_INIT(cudaMemcpy(c.rows_f, rows_f.data(), sizeof(RowItem) * rows_f.size(), cudaMemcpyHostToDevice));
    FAIL_INIT(dalloc(c, &c.planes, planes.size()));
    FAIL_INIT(cudaMemcpy(c.planes, planes.data(), sizeof(int4) * planes.size(), cudaMemcpyHostToDevice));
    FAIL_INIT(dalloc(c, &c.mass_first, mfirst.size()));
    FAIL_INIT(cudaMemcpy(c.mass_first, mfirst.data(), sizeof(int) * mfirst.size(), cudaMemcpyHostToDevice));
  }
  // internal buffers
  const size_t b3 = c.elems3 * c.esize, bi = c.elemsi * c.esize;
  void** f3[] = {&c.nu, &c.nv, &c.nw, &c.ndelp, &c.npt, &c.uc, &c.vc, &c.delpc, &c.ptc, &c.wc, &c.delzc,
                 &c.fx1, &c.fy1, &c.amfx, &c.amfy, &c.acrx, &c.acry, &c.axfx, &c.ayfx, &c.dp0, &c.dp1,
                 &c.dpstart};
  for (void** p : f3) FAIL_INIT(dalloc_bytes(c, p, b3));
  FAIL_INIT(dalloc_bytes(c, &c.pef, bi));
  FAIL_INIT(dalloc_bytes(c, &c.gz, bi));
  FAIL_INIT(dalloc(c, &c.scratch, (size_t)5 * c.nz * c.ncol));
  FAIL_INIT(dalloc(c, &c.status, 1));
  FAIL_INIT(cudaMemset(c.status, 0, sizeof(unsigned)));
  FAIL_INIT(dalloc(c, &c.cmax, 1));
  FAIL_INIT(dalloc(c, &c.nsplt, 1));
  FAIL_INIT(cudaMemset(c.nsplt, 0, sizeof(int)));
  FAIL_INIT(dalloc(c, &c.mass_part, 2 * (size_t)c.n_planes));
  FAIL_INIT(dalloc(c, &c.mass_out, c.nmem));
  FAIL_INIT(cudaDeviceSynchronize());
#undef FAIL_INIT
  *out = x;
  return FV3_OK;
}

extern "C" void fv3_destroy(fv3_ctx* x) {
  if (!x) return;
  drop_graphs(x->c);
  for (Slot& sl : x->ring) {
    if (sl.done) cudaEventSynchronize(sl.done);
    if (sl.buf) cudaFree(sl.buf);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  for (void* p : x->c.owned) cudaFree(p);
  if (x->stage) cudaFree(x->stage);
  if (x->cap) cudaStreamDestroy(x->cap);
  delete x;
}

extern "C" const char* fv3_last_error(const fv3_ctx* x) {
  if (!x) return "no context";
  return x->c.err.c_str();
}

extern "C" size_t fv3_field_elems(const fv3_ctx* x, int kind) {
  if (!x) return 0;
  if (kind == FV3_KIND_IFACE) return x->c.elemsi;
  if (kind == FV3_KIND_CELL || kind == FV3_KIND_XFACE || kind == FV3_KIND_YFACE) return x->c.elems3;
  return 0;
}

extern "C" size_t fv3_elem_size(const fv3_ctx* x) { return x ? (size_t)x->c.esize : 0; }

extern "C" fv3_status fv3_get_layout(const fv3_ctx* x, int member, fv3_layout* out) {
  if (!x || !out) return FV3_ERR_ARG;
  if (member < 0 || member >= x->c.nmem) return FV3_ERR_ARG;
  const Geo& g = x->c.geo[member];
  out->n = g.n; out->nz = g.nz; out->ntiles = g.nt;
  out->pitch = g.pitch; out->rows = g.rows; out->ox = g.ox;
  out->plane = g.plane; out->offset3 = g.off3; out->offseti = g.offi;
  return FV3_OK;
}

static fv3_status do_pack(fv3_ctx* x, int kind, void* field, void* dense, int host, int dbl, int member, int dir,
                          cudaStream_t st) {
  if (!x) return FV3_ERR_ARG;
  if (!field || !dense) return fail(x, FV3_ERR_ARG, "null buffer");
  if (kind < 0 || kind > 3) return fail(x, FV3_ERR_ARG, "bad field kind");
  if (member < 0 || member >= x->c.nmem) return fail(x, FV3_ERR_ARG, "bad member");
  if (!aligned(field)) return fail(x, FV3_ERR_ALIGN, "field not 128-byte aligned");
  const Geo& g = x->c.geo[member];
  const int iface = kind == FV3_KIND_IFACE ? 1 : 0;
  const int nlev = iface ? g.nz + 1 : g.nz;
  const int pk = kind == FV3_KIND_IFACE ? 0 : kind;  // interface fields are cell-shaped
  const size_t bytes = dense_count(g, pk, nlev) * (dbl ? 8 : 4);
  if (host == FV3_DENSE_HOST_ASYNC && dbl == (x->c.prec == FV3_FP64 ? 1 : 0)) {
    // same element type: one 3-D copy by the copy engine between the dense
    // host array and the field's interior (plane z = t * nlev + k, nj rows of
    // ni elements), no kernel, so it never waits for SMs held by the substep
    const size_t es = x->c.esize;
    const int n = g.n, ni = n + (pk == 1 || pk == 3), nj = n + (pk == 2 || pk == 3);
    const long long base = iface ? g.offi : g.off3;
    char* fo = (char*)field + (size_t)(base + (long long)HALO * g.pitch + g.ox) * es;
    cudaMemcpy3DParms cp{};
    cudaPitchedPtr fp = make_cudaPitchedPtr(fo, (size_t)g.pitch * es, (size_t)ni, (size_t)g.rows);
    cudaPitchedPtr hp = make_cudaPitchedPtr(dense, (size_t)ni * es, (size_t)ni, (size_t)nj);
    cp.extent = make_cudaExtent((size_t)ni * es, (size_t)nj, (size_t)g.nt * nlev);
    cp.srcPtr = dir == 0 ? hp : fp;
    cp.dstPtr = dir == 0 ? fp : hp;
    cp.kind = dir == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    CK(x, cudaMemcpy3DAsync(&cp, st));
    return FV3_OK;
  }
  if (host == FV3_DENSE_HOST_ASYNC) {
    // element type converted: one contiguous copy between the host array and
    // a staging slot, and the pack kernel between the slot and the field,
    // both on `st`
    Slot& sl = x->ring[x->ring_next];
    x->ring_next = (x->ring_next + 1) % kSlots;
    if (!sl.done) CK(x, cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    if (!sl.buf) {  // first use: large enough for any field of the context
      size_t most = bytes;
      for (const Geo& gm : x->c.geo)
        most = std::max(most, (size_t)gm.nt * (gm.nz + 1) * (gm.n + 1) * (gm.n + 1) * sizeof(double));
      CK(x, cudaMalloc(&sl.buf, most));
      sl.bytes = most;
    }
    if (sl.bytes < bytes) {  // grow: wait for the slot's last copy first
      CK(x, cudaEventSynchronize(sl.done));
      if (sl.buf) cudaFree(sl.buf);
      sl.buf = nullptr;
      sl.bytes = 0;
      CK(x, cudaMalloc(&sl.buf, bytes));
      sl.bytes = bytes;
    }
    CK(x, cudaStreamWaitEvent(st, sl.done, 0));
    if (dir == 0) CK(x, cudaMemcpyAsync(sl.buf, dense, bytes, cudaMemcpyHostToDevice, st));
    enqueue_pack(x->c, member, pk, nlev, iface, field, sl.buf, dbl, dir, st);
    CK(x, cudaGetLastError());
    if (dir == 1) CK(x, cudaMemcpyAsync(dense, sl.buf, bytes, cudaMemcpyDeviceToHost, st));
    CK(x, cudaEventRecord(sl.done, st));
    return FV3_OK;
  }
  if (host != 0 && host != FV3_DENSE_HOST) return fail(x, FV3_ERR_ARG, "bad dense_is_host");
  void* dd = dense;
  if (host) {
    fv3_status s = ensure_stage(x, bytes);
    if (s != FV3_OK) return s;
    dd = x->stage;
    if (dir == 0) CK(x, cudaMemcpyAsync(dd, dense, bytes, cudaMemcpyHostToDevice, st));
  }
  enqueue_pack(x->c, member, pk, nlev, iface, field, dd, dbl, dir, st);
  CK(x, cudaGetLastError());
  if (host && dir == 1) {
    CK(x, cudaMemcpyAsync(dense, dd, bytes, cudaMemcpyDeviceToHost, st));
    CK(x, cudaStreamSynchronize(st));
  }
  return FV3_OK;
}

extern "C" fv3_status fv3_halo_plan(const fv3_grid_desc* d, int member, int kind, fv3_halo_entry* out, size_t cap,
                                    size_t* total, fv3_layout* layout) {
  if (!d || !total) return FV3_ERR_ARG;
  std::vector<int> npx;
  const fv3_status dr = check_desc(d, npx);
  if (dr != FV3_OK) return dr;
  if (member < 0 || member >= d->n_members) return FV3_ERR_ARG;
  if (kind != FV3_PLAN_CELL && kind != FV3_PLAN_DGRID && kind != FV3_PLAN_CGRID) return FV3_ERR_ARG;
  if (cap > 0 && !out) return FV3_ERR_ARG;
  GridSpec spec{};
  spec.cubed = d->grid_type == FV3_GRID_CUBED;
  spec.dx = d->dx;
  spec.radius = d->radius;
  spec.omega = d->omega;
  const int nt = spec.cubed ? 6 : 1, esize = d->precision == FV3_FP64 ? 8 : 4;
  long long o3 = 0, oi = 0;  // member offsets, as fv3_init_grid lays them out
  Geo g{};
  for (int m = 0; m <= member; ++m) {
    plane_geo(npx[m], d->npz, nt, spec.cubed, esize, g);
    if (m < member) {
      o3 += (long long)nt * d->npz * g.plane;
      oi += (long long)nt * (d->npz + 1) * g.plane;
    }
  }
  g.off3 = o3;
  g.offi = oi;
  HostMetric M;
  Plans P;
  build_metric(spec, member, g, M, P);
  const PlanKind pk = kind == FV3_PLAN_CELL ? K_CELL3 : kind == FV3_PLAN_DGRID ? K_DGRID : K_CGRID;
  const std::vector<HaloEntry>& E = P.p[pk];
  *total = E.size();
  for (size_t e = 0; e < E.size() && e < cap; ++e) {
    out[e].dst = E[e].dst;
    out[e].src = E[e].src;
    out[e].dst_tile = E[e].dt;
    out[e].src_tile = E[e].st;
    out[e].sign = E[e].sign;
    out[e].flags = E[e].flags;
  }
  if (layout) {
    layout->n = g.n; layout->nz = g.nz; layout->ntiles = g.nt;
    layout->pitch = g.pitch; layout->rows = g.rows; layout->ox = g.ox;
    layout->plane = g.plane; layout->offset3 = g.off3; layout->offseti = g.offi;
  }
  return FV3_OK;
}

extern "C" fv3_status fv3_import(fv3_ctx* x, int kind, void* field, const void* dense, int dense_is_host,
                                 int dense_is_double, int member, fv3_stream stream) {
  return do_pack(x, kind, field, const_cast<void*>(dense), dense_is_host, dense_is_double, member, 0,
                 (cudaStream_t)stream);
}

extern "C" fv3_status fv3_export(fv3_ctx* x, int kind, const void* field, void* dense, int dense_is_host,
                                 int dense_is_double, int member, fv3_stream stream) {
  return do_pack(x, kind, const_cast<void*>(field), dense, dense_is_host, dense_is_double, member, 1,
                 (cudaStream_t)stream);
}

extern "C" fv3_status fv3_halo_fill(fv3_ctx* x, const fv3_state* s, unsigned mask, fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  fv3_status r = check_state(x, s, false);
  if (r != FV3_OK) return r;
  Ctx& c = x->c;
  std::vector<HaloField> F;
  auto cell = [&](void* p) {
    HaloField f{};
    f.xa = p; f.ent = c.plan_d[K_CELL3]; f.count = c.plan_n[K_CELL3]; f.nlev = c.nz;
    return f;
  };
  if (mask & FV3_HALO_WIND) {
    HaloField f{};
    f.xa = s->v; f.ya = s->u; f.ent = c.plan_d[K_DGRID]; f.count = c.plan_n[K_DGRID]; f.nlev = c.nz;
    F.push_back(f);
  }
  if (mask & FV3_HALO_W) F.push_back(cell(s->w));
  if (mask & FV3_HALO_DELP) F.push_back(cell(s->delp));
  if (mask & FV3_HALO_PT) F.push_back(cell(s->pt));
  if (mask & FV3_HALO_DELZ) F.push_back(cell(s->delz));
  if (mask & FV3_HALO_TRACERS)
    for (int q = 0; q < s->nq; ++q) F.push_back(cell(s->q[q]));
  enqueue_halo_fields(c, F, (cudaStream_t)stream);
  CK(x, cudaGetLastError());
  return FV3_OK;
}

static StateView internal_view(Ctx& c, const StateView& caller) {
  StateView v = caller;
  v.u = c.nu; v.v = c.nv; v.w = c.nw; v.delp = c.ndelp; v.pt = c.npt;
  return v;
}

extern "C" fv3_status fv3_acoustic_substep(fv3_ctx* x, const fv3_state* s, const fv3_params* p, fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  fv3_status r = check_state(x, s, false);
  if (r != FV3_OK) return r;
  r = check_params(x, p);
  if (r != FV3_OK) return r;
  Ctx& c = x->c;
  cudaStream_t st = (cudaStream_t)stream;
  const StateView in = view(s), nx = internal_view(c, in);
  enqueue_substep(c, in, nx, to_params(p), false, st);
  enqueue_copy_state(c, in, nx, st);
  CK(x, cudaGetLastError());
  return FV3_OK;
}

extern "C" fv3_status fv3_stage(fv3_ctx* x, const fv3_state* s, const fv3_params* p, int stop_after,
                                fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  fv3_status r = check_state(x, s, false);
  if (r != FV3_OK) return r;
  r = check_params(x, p);
  if (r != FV3_OK) return r;
  Ctx& c = x->c;
  const StateView in = view(s), nx = internal_view(c, in);
  enqueue_substep(c, in, nx, to_params(p), false, (cudaStream_t)stream, stop_after);
  CK(x, cudaGetLastError());
  return FV3_OK;
}

// one remapping step: n_split substeps (ping-pong between the caller's state
// and the internal next state), flux accumulation, tracer transport
static void enqueue_remap_step(Ctx& c, const StateView& in, const Params& P, cudaStream_t st) {
  const StateView nx = internal_view(c, in);
  enqueue_save_dpstart(c, in.delp, st);
  enqueue_zero_acc(c, st);
  for (int s = 0; s < P.n_split; ++s) {
    const bool even = (s % 2) == 0;
    enqueue_substep(c, even ? in : nx, even ? nx : in, P, true, st);
  }
  if (P.n_split % 2 == 1) enqueue_copy_state(c, in, nx, st);
  enqueue_tracers(c, in, P, st);
  if (P.remap) enqueue_remap(c, in, P, st);
}

extern "C" fv3_status fv3_vertical_remap(fv3_ctx* x, const fv3_state* s, const fv3_params* p, fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  fv3_status r = check_state(x, s, true);
  if (r != FV3_OK) return r;
  r = check_params(x, p);
  if (r != FV3_OK) return r;
  Ctx& c = x->c;
  for (int q = 0; q < s->nq; ++q)
    if (!c.qtmp[q]) CK(x, dalloc_bytes(c, &c.qtmp[q], c.elems3 * c.esize));
  enqueue_remap(c, view(s), to_params(p), (cudaStream_t)stream);
  CK(x, cudaGetLastError());
  return FV3_OK;
}

extern "C" fv3_status fv3_run_dyn(fv3_ctx* x, const fv3_state* s, const fv3_params* p, int n_steps,
                                  fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  fv3_status r = check_state(x, s, true);
  if (r != FV3_OK) return r;
  r = check_params(x, p);
  if (r != FV3_OK) return r;
  if (n_steps < 0) return fail(x, FV3_ERR_ARG, "n_steps < 0");
  Ctx& c = x->c;
  cudaStream_t st = (cudaStream_t)stream;
  const StateView in = view(s);
  const Params P = to_params(p);
  // tracer work buffers
  for (int q = 0; q < s->nq; ++q)
    if (!c.qtmp[q]) CK(x, dalloc_bytes(c, &c.qtmp[q], c.elems3 * c.esize));
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(x, cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) {  // caller is capturing: enqueue directly
    for (int k = 0; k < n_steps; ++k) enqueue_remap_step(c, in, P, st);
    CK(x, cudaGetLastError());
    return FV3_OK;
  }
  std::vector<unsigned char> key(sizeof(StateView) + sizeof(Params));
  std::memcpy(key.data(), &in, sizeof(StateView));
  std::memcpy(key.data() + sizeof(StateView), &P, sizeof(Params));
  Ctx::Graph* G = nullptr;
  for (Ctx::Graph& e : c.graphs)
    if (e.key == key) G = &e;
  if (!G) {
    if ((int)c.graphs.size() >= kMaxGraphs) {  // evict the least recently used
      size_t old = 0;
      for (size_t e = 1; e < c.graphs.size(); ++e)
        if (c.graphs[e].used < c.graphs[old].used) old = e;
      cudaGraphExecDestroy(c.graphs[old].exec);
      c.graphs.erase(c.graphs.begin() + (long)old);
    }
    CK(x, cudaStreamBeginCapture(x->cap, cudaStreamCaptureModeThreadLocal));
    const long long before = c.launches;
    enqueue_remap_step(c, in, P, x->cap);
    Ctx::Graph e;
    e.launches = c.launches - before;
    c.launches = before;
    cudaGraph_t g = nullptr;
    cudaError_t e1 = cudaStreamEndCapture(x->cap, &g);
    if (e1 != cudaSuccess) return fail(x, FV3_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1));
    cudaError_t e2 = cudaGraphInstantiate(&e.exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return fail(x, FV3_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
    e.key = key;
    c.graphs.push_back(e);
    G = &c.graphs.back();
  }
  G->used = ++c.graph_clock;
  for (int k = 0; k < n_steps; ++k) CK(x, cudaGraphLaunch(G->exec, st));
  c.launches += (long long)n_steps * G->launches;
  return FV3_OK;
}

extern "C" fv3_status fv3_fv_tp_2d(fv3_ctx* x, void* q, void* crx, void* cry, void* xfx, void* yfx, void* mfx,
                                   void* mfy, double damp, void* fx, void* fy, fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  void* need[7] = {q, crx, cry, xfx, yfx, fx, fy};
  for (void* p : need) {
    if (!p) return fail(x, FV3_ERR_ARG, "fv_tp_2d: a field is NULL");
    if (!aligned(p)) return fail(x, FV3_ERR_ALIGN, "fv_tp_2d: a field is not 128-byte aligned");
  }
  if ((mfx == nullptr) != (mfy == nullptr)) return fail(x, FV3_ERR_ARG, "fv_tp_2d: mfx and mfy go together");
  if (mfx && (!aligned(mfx) || !aligned(mfy)))
    return fail(x, FV3_ERR_ALIGN, "fv_tp_2d: a mass flux is not 128-byte aligned");
  if (!(damp >= 0.0) || !std::isfinite(damp)) return fail(x, FV3_ERR_ARG, "fv_tp_2d: damp must be >= 0");
  TpPtrs p{q, crx, cry, xfx, yfx, mfx, mfy, fx, fy, damp};
  enqueue_fv_tp_2d(x->c, p, (cudaStream_t)stream);
  CK(x, cudaGetLastError());
  return FV3_OK;
}

extern "C" fv3_status fv3_mass_sum(fv3_ctx* x, const fv3_state* s, double* out, fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  if (!s || !s->delp || !out) return fail(x, FV3_ERR_ARG, "null argument");
  Ctx& c = x->c;
  cudaStream_t st = (cudaStream_t)stream;
  enqueue_mass(c, s->delp, st);
  CK(x, cudaMemcpyAsync(out, c.mass_out, sizeof(double) * c.nmem, cudaMemcpyDeviceToHost, st));
  CK(x, cudaStreamSynchronize(st));
  return FV3_OK;
}

extern "C" fv3_status fv3_check_status(fv3_ctx* x, fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned h = 0;
  CK(x, cudaStreamSynchronize(st));
  CK(x, cudaMemcpy(&h, x->c.status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  CK(x, cudaMemset(x->c.status, 0, sizeof(unsigned)));
  if (h & ST_NONFINITE) return fail(x, FV3_ERR_NONFINITE, "a state field holds a non-finite value");
  if (h & ST_CFL) return fail(x, FV3_ERR_CFL, "a Courant number reached 1");
  if (h & ST_NSPLT) return fail(x, FV3_ERR_UNSUPPORTED, "tracer transport needed more than 4 subcycles");
  return FV3_OK;
}

extern "C" fv3_status fv3_check_finite(fv3_ctx* x, const fv3_state* s, fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  fv3_status r = check_state(x, s, false);
  if (r != FV3_OK) return r;
  enqueue_check_finite(x->c, view(s), (cudaStream_t)stream);
  CK(x, cudaGetLastError());
  return fv3_check_status(x, stream);
}

extern "C" fv3_status fv3_get_metric(fv3_ctx* x, const char* name, int member, double* dense) {
  if (!x || !name || !dense) return FV3_ERR_ARG;
  if (member < 0 || member >= x->c.nmem) return fail(x, FV3_ERR_ARG, "bad member");
  const Metric<double>& M = x->c.Md;
  struct E { const char* nm; const double* p; int kind; } tab[] = {
      {"area", M.area, 0}, {"rarea", M.rarea, 0}, {"fA", M.fA, 0}, {"dx", M.dx, 2}, {"rdx", M.rdx, 2},
      {"dyc", M.dyc, 2}, {"rdyc", M.rdyc, 2}, {"cosy", M.cosy, 2}, {"siny", M.siny, 2}, {"dy", M.dy, 1},
      {"rdy", M.rdy, 1}, {"dxc", M.dxc, 1}, {"rdxc", M.rdxc, 1}, {"cosx", M.cosx, 1}, {"sinx", M.sinx, 1},
      {"fC", M.fC, 3}, {"rareac", M.rareac, 3}};
  for (const E& e : tab)
    if (!std::strcmp(e.nm, name)) {
      const Geo& g = x->c.geo[member];
      const size_t bytes = dense_count(g, e.kind, 1) * 8;
      fv3_status s = ensure_stage(x, bytes);
      if (s != FV3_OK) return s;
      enqueue_pack(x->c, member, e.kind, 1, 2, const_cast<double*>(e.p), x->stage, 1, 1, 0);
      CK(x, cudaMemcpy(dense, x->stage, bytes, cudaMemcpyDeviceToHost));
      return FV3_OK;
    }
  return fail(x, FV3_ERR_ARG, std::string("unknown metric ") + name);
}

extern "C" fv3_status fv3_get_intermediate(fv3_ctx* x, const char* name, int member, double* dense,
                                           fv3_stream stream) {
  if (!x || !name || !dense) return FV3_ERR_ARG;
  Ctx& c = x->c;
  struct E { const char* nm; void* p; int kind; } tab[] = {
      {"uc", c.uc, 1}, {"fx1", c.fx1, 1}, {"vc", c.vc, 2}, {"fy1", c.fy1, 2}, {"delpc", c.delpc, 0},
      {"ptc", c.ptc, 0}, {"wc", c.wc, 0}, {"delzc", c.delzc, 0}, {"pef", c.pef, 3}, {"gz", c.gz, 3},
      {"mfx", c.amfx, 1}, {"mfy", c.amfy, 2}, {"crx", c.acrx, 1}, {"cry", c.acry, 2}, {"xfx", c.axfx, 1},
      {"yfx", c.ayfx, 2}};
  for (const E& e : tab)
    if (!std::strcmp(e.nm, name)) return fv3_export(x, e.kind, e.p, dense, 1, 1, member, stream);
  return fail(x, FV3_ERR_ARG, std::string("unknown intermediate ") + name);
}

extern "C" fv3_status fv3_launch_stage(fv3_ctx* x, const fv3_state* s, const fv3_params* p, int stage, int reps,
                                       fv3_stream stream) {
  if (!x) return FV3_ERR_ARG;
  fv3_status r = check_state(x, s, false);
  if (r != FV3_OK) return r;
  r = check_params(x, p);
  if (r != FV3_OK) return r;
  if (stage < 0 || stage > 6 || reps < 1) return fail(x, FV3_ERR_ARG, "stage 0..6, reps >= 1");
  Ctx& c = x->c;
  const StateView in = view(s), nx = internal_view(c, in);
  for (int k = 0; k < reps; ++k) enqueue_substep(c, in, nx, to_params(p), false, (cudaStream_t)stream, 99, stage);
  CK(x, cudaGetLastError());
  return FV3_OK;
}

extern "C" long long fv3_kernel_launches(const fv3_ctx* x) { return x ? x->c.launches : -1; }

extern "C" fv3_status fv3_calibrate(fv3_ctx* x, int what, fv3_stream stream, double* work_per_launch) {
  if (!x || !work_per_launch) return FV3_ERR_ARG;
  if (what < 0 || what > 2) return fail(x, FV3_ERR_ARG, "what: 0 fp64 fma, 1 fp32 fma, 2 fp64 copy stencil");
  *work_per_launch = enqueue_calibration(x->c, what, (cudaStream_t)stream);
  CK(x, cudaGetLastError());
  return FV3_OK;
}

extern "C" fv3_status fv3_set_tiles(fv3_ctx* x, int bx, int by, int kchunk) {
  if (!x) return FV3_ERR_ARG;
  Ctx& c = x->c;
  if (!shape_supported(bx, by)) return fail(x, FV3_ERR_UNSUPPORTED, "block shape not compiled");
  if (kchunk < 1 || kchunk > c.nz) return fail(x, FV3_ERR_ARG, "kchunk must be in [1, npz]");
  std::vector<Item> hz = block_items(c, bx, by);
  Item* d = nullptr;
  CK(x, dalloc(c, &d, hz.size()));
  CK(x, cudaMemcpy(d, hz.data(), sizeof(Item) * hz.size(), cudaMemcpyHostToDevice));
  c.items_hz = d;  // the previous list stays owned until destroy (graphs may refer to it)
  c.n_items_hz = (int)hz.size();
  c.BX = bx;
  c.BY = by;
  c.kchunk = kchunk;
  drop_graphs(c);
  return FV3_OK;
}

extern "C" fv3_status fv3_set_persistent(fv3_ctx* x, int on) {
  if (!x) return FV3_ERR_ARG;
  x->c.persistent = on ? 1 : 0;
  drop_graphs(x->c);
  return FV3_OK;
}

extern "C" fv3_status fv3_get_persistent(const fv3_ctx* x, int* on) {
  if (!x || !on) return FV3_ERR_ARG;
  *on = x->c.persistent;
  return FV3_OK;
}

extern "C" fv3_status fv3_get_tiles(const fv3_ctx* x, int* bx, int* by, int* kchunk) {
  if (!x || !bx || !by || !kchunk) return FV3_ERR_ARG;
  *bx = x->c.BX;
  *by = x->c.BY;
  *kchunk = x->c.kchunk;
  return FV3_OK;
}

// Empirical tuning of the block shape and level chunk of the horizontal
// kernels on the caller's state (the paper's transfer tuning, Section VII-B,
// searches transformation configurations on representative cutouts and
// transfers the best ones; here the search space is the compiled block
// shapes x level chunks, timed with events on the full d_sw + c_sw stages).
namespace {
// the search of fv3_autotune; sizes: tile sizes (cells per edge) whose tiles
// the chosen block shape must cover with whole blocks, if any shape does
fv3_status autotune_impl(fv3_ctx* x, const fv3_state* s, const fv3_params* p, fv3_stream stream, double* best_ms,
                         const std::vector<int>& sizes) {
  if (!x) return FV3_ERR_ARG;
  fv3_status r = check_state(x, s, false);
  if (r != FV3_OK) return r;
  r = check_params(x, p);
  if (r != FV3_OK) return r;
  Ctx& c = x->c;
  cudaStream_t st = (cudaStream_t)stream;
  const int all_shapes[4][2] = {{32, 8}, {32, 16}, {64, 8}, {16, 16}};
  // shapes that make every tile of the given sizes whole blocks (the kernels
  // then run their full-block instantiation); all shapes if none does
  std::vector<std::array<int, 2>> shapes;
  for (const auto& sh : all_shapes) {
    bool whole = true;
    for (int n : sizes) whole = whole && n % sh[0] == 0 && n % sh[1] == 0;
    if (whole) shapes.push_back({sh[0], sh[1]});
  }
  if (shapes.empty())
    for (const auto& sh : all_shapes) shapes.push_back({sh[0], sh[1]});
  const int chunks[3] = {1, 4, 16};
  const int pmodes[2] = {0, 1};
  const StateView in = view(s);
  const StateView nx = internal_view(c, in);
  const Params P = to_params(p);
  enqueue_substep(c, in, nx, P, false, st, 5);  // intermediates for the stage runs
  cudaEvent_t e0, e1;
  CK(x, cudaEventCreate(&e0));
  CK(x, cudaEventCreate(&e1));
  double best = 1e300;
  int bb[4] = {c.BX, c.BY, c.kchunk, c.persistent};
  for (int pm : pmodes)
  for (const auto& sh : shapes)
    for (int kc : chunks) {
      if (kc > c.nz) continue;
      if (fv3_set_tiles(x, sh[0], sh[1], kc) != FV3_OK) continue;
      c.persistent = pm;
      for (int w = 0; w < 2; ++w) {
        enqueue_substep(c, in, nx, P, false, st, 99, 1);
        enqueue_substep(c, in, nx, P, false, st, 99, 6);
      }
      CK(x, cudaEventRecord(e0, st));
      for (int rep = 0; rep < 3; ++rep) {
        enqueue_substep(c, in, nx, P, false, st, 99, 1);
        enqueue_substep(c, in, nx, P, false, st, 99, 6);
      }
      CK(x, cudaEventRecord(e1, st));
      CK(x, cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(x, cudaEventElapsedTime(&ms, e0, e1));
      if (ms / 3 < best) {
        best = ms / 3;
        bb[0] = sh[0];
        bb[1] = sh[1];
        bb[2] = kc;
        bb[3] = pm;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  r = fv3_set_tiles(x, bb[0], bb[1], bb[2]);
  c.persistent = bb[3];
  if (best_ms) *best_ms = best;
  return r;
}
}  // namespace

extern "C" fv3_status fv3_autotune(fv3_ctx* x, const fv3_state* s, const fv3_params* p, fv3_stream stream,
                                   double* best_ms) {
  return autotune_impl(x, s, p, stream, best_ms, {});
}

extern "C" fv3_status fv3_autotune_for(fv3_ctx* x, const fv3_state* s, const fv3_params* p, fv3_stream stream,
                                       double* best_ms, const int* sizes, int n_sizes) {
  if (n_sizes < 0 || (n_sizes > 0 && !sizes)) return FV3_ERR_ARG;
  std::vector<int> v(sizes, sizes + n_sizes);
  for (int n : v)
    if (n < 1) return FV3_ERR_ARG;
  return autotune_impl(x, s, p, stream, best_ms, v);
}

// ------------------------------------------------------------------------
// single-stencil exports (readings R4, R14)
// ------------------------------------------------------------------------
extern "C" fv3_status fv3_face_stencils(const double* q6, const double* cr, int n, double* plain, double* edge,
                                        float* x, float* sig, fv3_stream stream) {
  if (!q6 || n < 0 || (plain && !cr)) return FV3_ERR_ARG;
  if (n == 0) return FV3_OK;
  return fv3::launch_face_stencils(q6, cr, n, plain, edge, x, sig, (cudaStream_t)stream) == cudaSuccess
             ? FV3_OK
             : FV3_ERR_CUDA;
}

extern "C" fv3_status fv3_learned_faces(const float* w, const double* q6, const double* cr, int n, double* value,
                                        fv3_stream stream) {
  if (!w || !q6 || !cr || !value || n < 0) return FV3_ERR_ARG;
  if (n == 0) return FV3_OK;
  return fv3::launch_learned_stencils(w, q6, cr, n, value, (cudaStream_t)stream) == cudaSuccess ? FV3_OK
                                                                                               : FV3_ERR_CUDA;
}

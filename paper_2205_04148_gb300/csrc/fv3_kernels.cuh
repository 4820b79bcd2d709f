// fv3_kernels.cuh -- kernel argument blocks, the library context and the
// orchestration entry points shared by the two translation units (internal).
#pragma once
#include <string>
#include <vector>

#include "fv3_host.h"

namespace fv3 {

constexpr int MAX_TRACERS = 16;
constexpr int kDzBX = 16, kDzBY = 8;  // update_dz_c: blocks of 16 x 8 columns
constexpr int MAX_HALO_FIELDS = 24;
constexpr int NSPLT_MAX = 4;

template <typename R>
struct StepArgs {
  const Geo* geo;        // per member
  const Item* items;     // CTA work list
  Metric<R> M;           // metric in the arithmetic precision
  Metric<double> Md;     // the FP64 metric (kernels with FP64 metric terms)
  Params P;
  // prognostic state (in) and next state (out)
  const R *u, *v, *w, *delp, *pt, *delz;
  R *u_o, *v_o, *w_o, *delp_o, *pt_o;
  // C-grid intermediates
  R *uc, *vc, *delpc, *ptc, *wc, *delzc, *fx1, *fy1;
  R *pef, *gz;           // interface fields [tile][nz+1][plane]
  double* scratch;       // column-solver scratch, 5 * nz * ncol
  long long ncol;        // columns of all members
  // flux accumulators of the remapping step (null: not accumulating)
  R *amfx, *amfy, *acrx, *acry, *axfx, *ayfx;
  // closed substep (reading R17): d_sw's area fluxes out (null: not kept),
  // the column solve's new delz
  R *xfxd, *yfxd, *delz_o;
  unsigned* status;
  const float* mlp;      // face-value network (hord 1), float[1313] on the device
};

struct HaloField {
  void* xa;              // cell array, or x-face array of a pair
  void* ya;              // y-face array of a pair (null for cells)
  const HaloEntry* ent;  // entries
  int count;             // number of entries
  int nlev;              // levels of the field
  int iface;             // 1: interface field (member offsets offi)
  int pad;
};

struct HaloBatch {
  HaloField f[MAX_HALO_FIELDS];
};

template <typename R>
struct TracerArgs {
  const Geo* geo;
  const Item* items;
  Metric<R> M;
  Metric<double> Md;     // the FP64 metric (kernels with FP64 metric terms)
  int nq, it;            // tracers, subcycle index
  const int* nsplt;      // device: number of subcycles of this remapping step
  const R* q[MAX_TRACERS];
  R* q_o[MAX_TRACERS];
  const R *acrx, *acry, *axfx, *ayfx, *amfx, *amfy;
  const R* dp0;          // delp at the start of the subcycle
  R* dp1;                // delp after the subcycle
  const float* mlp;      // face-value network
  bool learn;            // tracers use learned face values
};

template <typename R>
struct CopyArgs {
  R* dst[MAX_TRACERS + 1];
  const R* src[MAX_TRACERS + 1];
  int nf;
};

struct RowItem {
  int m, t, j, pad;
};

// the library context behind the opaque fv3_ctx handle
struct Ctx {
  GridSpec spec{};
  // prec: 0 FP64; 1 FP32 bulk with FP32 copies of the metric; 2 FP32 bulk
  // with the metric terms in FP64
  int nz = 0, nmem = 0, prec = 0, esize = 8;
  std::vector<Geo> geo;
  Geo* geo_d = nullptr;
  size_t elems3 = 0, elemsi = 0, elems2 = 0;  // elements of a 3-D, interface, 2-D field
  long long ncol = 0;
  std::vector<double> da_min;
  // metric: FP64 master copy, and the FP32 copy for the FP32-bulk path
  Metric<double> Md{};
  Metric<float> Mf{};
  std::vector<void*> metric_bufs;
  // plans
  HaloEntry* plan_d[K_NUM] = {};
  int plan_n[K_NUM] = {};
  // work lists
  int BX = 32, BY = 8, kchunk = 8;
  int persistent = 0;  // 1: horizontal kernels run on a GPU-filling persistent grid
  Item* items_hz = nullptr;
  int n_items_hz = 0;
  Item* items_dz = nullptr;
  int n_items_dz = 0;
  RowItem* rows = nullptr;
  int n_rows = 0;
  RowItem* rows_f = nullptr;  // rows j = 0 .. n (face columns of the remap)
  int n_rows_f = 0;
  int max_n = 0;
  int4* planes = nullptr;  // (m, t, k) of every level plane
  int n_planes = 0;
  int* mass_first = nullptr;  // per-member first partial, nmem + 1
  // internal buffers (element type by prec)
  void *nu = nullptr, *nv = nullptr, *nw = nullptr, *ndelp = nullptr, *npt = nullptr;
  void *uc = nullptr, *vc = nullptr, *delpc = nullptr, *ptc = nullptr, *wc = nullptr, *delzc = nullptr;
  void *fx1 = nullptr, *fy1 = nullptr, *pef = nullptr, *gz = nullptr;
  double* scratch = nullptr;
  void *amfx = nullptr, *amfy = nullptr, *acrx = nullptr, *acry = nullptr, *axfx = nullptr, *ayfx = nullptr;
  void *dp0 = nullptr, *dp1 = nullptr, *dpstart = nullptr;
  void* qtmp[MAX_TRACERS] = {};
  unsigned* status = nullptr;
  unsigned* cmax = nullptr;
  int* nsplt = nullptr;
  double* mass_part = nullptr;
  double* mass_out = nullptr;
  std::vector<void*> owned;  // every device allocation, freed by destroy
  // kernels enqueued by the library (host count; graph replays add the
  // number captured in the graph)
  long long launches = 0;
  // graphs of one remapping step, one per (state, parameters) key, so that a
  // caller alternating between a few states replays instead of re-capturing
  struct Graph {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;  // kernels captured in it
    long long used = 0;      // last use, for eviction
  };
  std::vector<Graph> graphs;
  long long graph_clock = 0;
  std::string err;
};

struct StateView {  // caller state, device pointers in the library layout
  void *u, *v, *w, *delp, *pt, *delz;
  void* q[MAX_TRACERS];
  int nq;
};

struct ParamView {
  Params P;
};

// orchestration (fv3_kernels.cu); enqueue_pack: iface 2 = FP64 metric planes
void enqueue_halo_prognostics(Ctx& c, const StateView& s, cudaStream_t st);
void enqueue_substep(Ctx& c, const StateView& in, const StateView& out, const Params& P, bool accumulate,
                     cudaStream_t st, int stop_after = 99, int only = -1);
void enqueue_substep_f64(Ctx& c, const StateView& in, const StateView& out, const Params& P, bool accumulate,
                     cudaStream_t st, int stop_after, int only);
void enqueue_substep_f32(Ctx& c, const StateView& in, const StateView& out, const Params& P, bool accumulate,
                     cudaStream_t st, int stop_after, int only);
void enqueue_substep_f32m64(Ctx& c, const StateView& in, const StateView& out, const Params& P, bool accumulate,
                            cudaStream_t st, int stop_after, int only);
void enqueue_tracers_f64(Ctx& c, const StateView& s, const Params& P, cudaStream_t st);
void enqueue_tracers_f32(Ctx& c, const StateView& s, const Params& P, cudaStream_t st);
void enqueue_tracers_f32m64(Ctx& c, const StateView& s, const Params& P, cudaStream_t st);
void enqueue_tracers(Ctx& c, const StateView& s, const Params& P, cudaStream_t st);

// vertical remapping (fv3_remap.cu): caller's state in, context buffers out
template <typename R>
struct RemapArgs {
  const Geo* geo;
  double ptop;
  const R* delp;
  R* delp_o;
  const R* in[3 + MAX_TRACERS];  // pt, w, delz, tracers
  R* out[3 + MAX_TRACERS];
  int nf;
  const R *u, *v;
  R *u_o, *v_o;
};
void enqueue_remap_kernel(Ctx& c, const StateView& s, double ptop, cudaStream_t st);
void enqueue_remap(Ctx& c, const StateView& s, const Params& P, cudaStream_t st);

// standalone fv_tp_2d: caller's fields in the library layout
struct TpPtrs {
  void *q, *crx, *cry, *xfx, *yfx, *mfx, *mfy, *fx, *fy;
  double damp;
};
template <typename R>
struct TpArgs {
  const Geo* geo;
  const Item* items;
  Metric<R> M;
  Metric<double> Md;     // the FP64 metric (kernels with FP64 metric terms)
  const R *q, *crx, *cry, *xfx, *yfx, *mfx, *mfy;
  R *fx, *fy;
  double damp;
};
void enqueue_fv_tp_2d(Ctx& c, const TpPtrs& p, cudaStream_t st);
void enqueue_fv_tp_2d_f64(Ctx& c, const TpPtrs& p, cudaStream_t st);
void enqueue_fv_tp_2d_f32(Ctx& c, const TpPtrs& p, cudaStream_t st);
void enqueue_fv_tp_2d_f32m64(Ctx& c, const TpPtrs& p, cudaStream_t st);
void enqueue_mass(Ctx& c, const void* delp, cudaStream_t st);
void enqueue_check_finite(Ctx& c, const StateView& s, cudaStream_t st);
void enqueue_pack(Ctx& c, int member, int kind, int nlev, int iface, void* padded, void* dense, int dense_is_double,
                  int dir, cudaStream_t st);
void enqueue_halo_fields(Ctx& c, const std::vector<HaloField>& fields, cudaStream_t st);
void enqueue_copy_state(Ctx& c, const StateView& dst, const StateView& src, cudaStream_t st);
void enqueue_zero_acc(Ctx& c, cudaStream_t st);
void enqueue_save_dpstart(Ctx& c, const void* delp, cudaStream_t st);
bool shape_supported(int bx, int by);
// stencil exports (FP64, no context): plain PPM face values, clamped edge
// values and network inputs of six-cell stencils; learned face values
cudaError_t launch_face_stencils(const double* q6, const double* cr, int n, double* plain, double* edge, float* x,
                                 float* sig, cudaStream_t st);
cudaError_t launch_learned_stencils(const float* w, const double* q6, const double* cr, int n, double* value,
                                    cudaStream_t st);
// calibration kernels (fv3_calib.cu): returns work per launch (flops or bytes)
double enqueue_calibration(Ctx& c, int what, cudaStream_t st);

}  // namespace fv3

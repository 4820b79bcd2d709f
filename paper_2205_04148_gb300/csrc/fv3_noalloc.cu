// fv3_noalloc.cu -- a column-solver entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need the
// solve: code that runs inside a region where every buffer must be reserved
// up front (a real-time or inference loop with a fixed memory budget, a host
// framework that owns the whole device pool and forbids allocations from
// libraries, or a phase where an allocation could block on the device).  The
// regular path keeps its solver scratch in a context created by
// fv3_init_grid, which allocates.  This entry point needs no context: the
// caller passes its input and output arrays, and the scratch lives in a
// fixed-size array that is part of the library's GPU image.
//
// The scratch array is reserved on every GPU that loads this library and
// stays reserved until the process exits (32 MiB).  The host cannot use its
// name as a device address (in host code the name only stands for the
// symbol), so the address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device.  With lazy module loading (the CUDA default) that lookup is
// also what loads this file's module on the device, so the first call
// reserves the array and the kernel image: it must come before the region in
// which nothing may be allocated.  Later calls allocate nothing.  The cached
// address belongs to the context that was current at the first call; after
// a device reset (cudaDeviceReset) the module is loaded again and the array
// may move, so the entry point is not for use across a device reset.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "fv3.h"

namespace {

constexpr long long kScratchDoubles = 4LL << 20;  // 32 MiB of FP64 scratch
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// One thread per column; columns are independent.  Same solve as the
// library's riem_solver_c stage, on level-major arrays (element (k, col) at
// k * ncol + col) so that consecutive threads read consecutive addresses.
// Scratch per column: the forward-sweep coefficients, the layer coefficient
// C, the perturbation pressure and the hydrostatic interface pressure, each
// nz values.  Every scratch value a thread reads was written earlier by the
// same thread in the same call, so nothing needs clearing between calls.
__global__ void __launch_bounds__(128) k_riem_columns(int ncol, int nz, const double* __restrict__ delpc,
                                                      const double* __restrict__ ptc,
                                                      const double* __restrict__ wc,
                                                      const double* __restrict__ delzc, double* __restrict__ pef,
                                                      double* __restrict__ gz, double* scratch, double dt,
                                                      double ptop, double grav, double rdgas, double cp_air,
                                                      double a_imp) {
  const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  const long long N = ncol;
  double* s_cp = scratch;
  double* s_dp = scratch + (long long)nz * N;
  double* s_C = scratch + 2LL * nz * N;
  double* s_pp = scratch + 3LL * nz * N;
  double* s_pe = scratch + 4LL * nz * N;
  const double kappa = rdgas / cp_air, gama = 1.0 / (1.0 - kappa);
  double pe = ptop, dp_up = 0.0, w_up = 0.0, C_up = 0.0, pp_up = 0.0, cp_up = 0.0, d_up = 0.0;
  for (int k = 0; k < nz; ++k) {
    const long long e = (long long)k * N + col;
    const double dpk = delpc[e], tk = ptc[e], wk = wc[e], dzk = delzc[e];
    const double pe_dn = pe + dpk;
    const double p = -dpk * rdgas * tk / (grav * dzk);
    const double pp = p - dpk / log(pe_dn / pe);
    const double C = a_imp * dt * gama * p / (-dzk);
    const double mass = k == 0 ? 0.5 * dpk / grav : 0.5 * (dp_up + dpk) / grav;
    const double w_old = k == 0 ? wk : 0.5 * (w_up + wk);
    const double lower = -C_up;
    const double diag = mass / dt + C_up + C;
    const double upper = k < nz - 1 ? -C : 0.0;
    const double rhs = mass / dt * w_old + pp - pp_up;
    double cpk, dk;
    if (k == 0) {
      cpk = upper / diag;
      dk = rhs / diag;
    } else {
      const double den = diag - lower * cp_up;
      cpk = upper / den;
      dk = (rhs - lower * d_up) / den;
    }
    s_cp[e] = cpk;
    s_dp[e] = dk;
    s_C[e] = C;
    s_pp[e] = pp;
    s_pe[e] = pe;
    pe = pe_dn;
    dp_up = dpk;
    w_up = wk;
    C_up = C;
    pp_up = pp;
    cp_up = cpk;
    d_up = dk;
  }
  const double pe_bottom = pe;
  double w_below = 0.0, g = 0.0, ppn_below = 0.0;
  gz[(long long)nz * N + col] = 0.0;
  for (int k = nz - 1; k >= 0; --k) {
    const long long e = (long long)k * N + col;
    const double wk = s_dp[e] - s_cp[e] * w_below;
    const double dzn = delzc[e] + dt * (w_below - wk);
    const double ppn = s_pp[e] + s_C[e] * (w_below - wk) / a_imp;
    g = g - grav * dzn;
    gz[e] = g;
    const double pf = (k == nz - 1) ? pe_bottom + ppn : s_pe[e + N] + 0.5 * (ppn + ppn_below);
    pef[e + N] = pf;
    ppn_below = ppn;
    w_below = wk;
  }
  pef[col] = ptop;
}

}  // namespace

extern "C" fv3_status fv3_riem_solver_c_noalloc(int ncol, int nz, const double* delpc, const double* ptc,
                                                const double* wc, const double* delzc, double* pef, double* gz,
                                                const fv3_params* params, fv3_stream stream) {
  if (!delpc || !ptc || !wc || !delzc || !pef || !gz || !params) return FV3_ERR_ARG;
  if (ncol < 1 || nz < 2) return FV3_ERR_SHAPE;
  if (5LL * nz * (long long)ncol > kScratchDoubles) return FV3_ERR_SHAPE;  // beyond the fixed scratch
  if (!(params->dt > 0) || !(params->grav > 0) || !(params->a_imp > 0) || !(params->rdgas > 0) ||
      !(params->cp_air > params->rdgas) || !(params->ptop > 0))
    return FV3_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FV3_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return FV3_ERR_UNSUPPORTED;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {  // first call on this device: look the address up
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FV3_ERR_CUDA;
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  const int threads = 128;
  const unsigned blocks = (unsigned)((ncol + threads - 1) / threads);
  k_riem_columns<<<blocks, threads, 0, (cudaStream_t)stream>>>(ncol, nz, delpc, ptc, wc, delzc, pef, gz, scratch,
                                                               0.5 * params->dt, params->ptop, params->grav,
                                                               params->rdgas, params->cp_air, params->a_imp);
  if (cudaGetLastError() != cudaSuccess) return FV3_ERR_CUDA;
  return FV3_OK;
}

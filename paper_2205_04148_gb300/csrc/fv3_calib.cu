// fv3_calib.cu -- machine calibration kernels (not part of the substep).
//
// The paper bounds its kernels by measured machine peaks: a STREAM/CUDA
// bandwidth test and a one-input/one-output "copy stencil" on the target
// domain (arxiv 2205.04148, Section IX-A).  The same calibration is done here
// on the device: the copy stencil on a halo-padded FP64 3-D field of the
// context, and FP64 / FP32 fused multiply-add throughput (the FP64 rate
// bounds the FP64 substep, which is arithmetic-bound on this GPU).
#include <cuda_runtime.h>

#include "fv3.h"

#include "fv3_kernels.cuh"
#include "fv3_math.cuh"

namespace fv3 {

template <typename R, int CH>
__global__ void __launch_bounds__(256) k_fma_peak(R* sink, int iters, R a, R b) {
  R x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = R(threadIdx.x) * R(1e-3) + R(c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == R(-12345.0)) sink[blockIdx.x] = s;  // keeps the chains live
}

// copy the interior of every level plane of a padded FP64 field
__global__ void k_copy_stencil(const Geo* geo, const int4* planes, const double* src, double* dst) {
  const int4 pl = planes[blockIdx.z];
  const Geo g = geo[pl.x];
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.n || j >= g.n) return;
  const long long o = g.off3 + ((long long)pl.y * g.nz + pl.z) * g.plane + (long long)(j + HALO) * g.pitch + g.ox + i;
  dst[o] = src[o];
}

double enqueue_calibration(Ctx& c, int what, cudaStream_t st) {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256, iters = 2048;
  if (what == 0) {
    k_fma_peak<double, 8><<<blocks, threads, 0, st>>>((double*)c.nu, iters, 0.999999, 1e-7);
    ++c.launches;
    return 2.0 * 8 * iters * (double)blocks * threads;
  }
  if (what == 1) {
    k_fma_peak<float, 16><<<blocks, threads, 0, st>>>((float*)c.nu, iters * 4, 0.9999f, 1e-5f);
    ++c.launches;
    return 2.0 * 16 * iters * 4 * (double)blocks * threads;
  }
  // FP64 copy stencil: the interior cells of one 3-D field (requires FP64 buffers)
  if (c.prec != 0) return 0.0;
  const int nb = c.max_n;
  k_copy_stencil<<<dim3((nb + 31) / 32, (nb + 7) / 8, c.n_planes), dim3(32, 8), 0, st>>>(
      c.geo_d, c.planes, (const double*)c.nw, (double*)c.nu);
  ++c.launches;
  double cells = 0;
  for (const Geo& g : c.geo) cells += (double)g.nt * g.nz * g.n * g.n;
  return 16.0 * cells;
}

// element-wise FP64 helpers of the kernels, for their accuracy tests:
// what 0: out = rcp(x); 1: out = log_ratio(x + y, x, y);
// 2: out = layer_mean_pressure(x + y, x, y); 3: out = 1 / x from
// rcp_pair(x, y); 4: out = to_f64((float)x), the integer-pipe widening of a
// float
__global__ void k_math_check(int what, const double* x, const double* y, double* out, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double v;
  if (what == 0) v = rcp(x[e]);
  else if (what == 1) v = log_ratio(x[e] + y[e], x[e], y[e]);
  else if (what == 2) v = layer_mean_pressure(x[e] + y[e], x[e], y[e]);
  else if (what == 3) {
    double rb;
    rcp_pair(x[e], y[e], v, rb);
  } else {
    v = to_f64(__double2float_rn(x[e]));
  }
  out[e] = v;
}

}  // namespace fv3

extern "C" fv3_status fv3_math_check(int what, const double* x, const double* y, double* out, int n,
                                     fv3_stream stream) {
  if (n < 0 || what < 0 || what > 4 || (n > 0 && (!x || !out || (what >= 1 && !y)))) return FV3_ERR_ARG;
  if (n == 0) return FV3_OK;
  fv3::k_math_check<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(what, x, y, out, n);
  return cudaGetLastError() == cudaSuccess ? FV3_OK : FV3_ERR_CUDA;
}

// fv3_exchange.cu -- device side of the halo exchange between ranks that hold
// different tiles of one member (Section V-C: the halo exchange with the
// orientation transform between cube faces).
//
// A rank's part of the halo plan (fv3_halo_plan, split by tile owner on the
// host) is three lists of element offsets into its field buffer: values it
// sends to each peer (gathered with the vector sign into one contiguous
// message), halo slots it fills from its own tiles (copied with the sign),
// and halo slots each peer's message fills (scattered in plan order).  These
// kernels do the gathering, copying and scattering; the messages themselves
// travel between ranks through the caller's point-to-point transport.  Every
// launch is a grid-stride loop of independent elements: no element waits on
// another.
#include <cuda_runtime.h>

#include <cstdint>

#include "fv3.h"

namespace {

template <typename T>
__device__ __forceinline__ T nan_of();
template <>
__device__ __forceinline__ double nan_of<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <>
__device__ __forceinline__ float nan_of<float>() { return __int_as_float(0x7fc00000); }

template <typename T>
__global__ void k_gather(const T* __restrict__ field, const int64_t* __restrict__ src, const int8_t* __restrict__ sign,
                         int64_t count, T* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const T v = field[src[e]];
    out[e] = (sign && sign[e] < 0) ? -v : v;
  }
}

template <typename T>
__global__ void k_scatter(T* __restrict__ field, const int64_t* __restrict__ dst, const T* __restrict__ in,
                          int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    field[dst[e]] = in ? in[e] : nan_of<T>();
}

// destinations and sources are disjoint sets of the same buffer (halo slots
// are filled from interior values only), so the copies do not depend on
// their order
template <typename T>
__global__ void k_copy(T* field, const int64_t* __restrict__ src, const int64_t* __restrict__ dst,
                       const int8_t* __restrict__ sign, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const T v = field[src[e]];
    field[dst[e]] = (sign && sign[e] < 0) ? -v : v;
  }
}

unsigned blocks_for(int64_t count) {
  const int64_t b = (count + 255) / 256;
  return (unsigned)(b < 152 * 16 ? b : 152 * 16);
}

fv3_status done() { return cudaGetLastError() == cudaSuccess ? FV3_OK : FV3_ERR_CUDA; }

}  // namespace

extern "C" fv3_status fv3_halo_gather(const void* field, int elem_size, const int64_t* src, const int8_t* sign,
                                      int64_t count, void* out, fv3_stream stream) {
  if (count < 0 || (elem_size != 4 && elem_size != 8)) return FV3_ERR_ARG;
  if (count == 0) return FV3_OK;
  if (!field || !src || !out) return FV3_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (elem_size == 8)
    k_gather<double><<<blocks_for(count), 256, 0, st>>>((const double*)field, src, sign, count, (double*)out);
  else
    k_gather<float><<<blocks_for(count), 256, 0, st>>>((const float*)field, src, sign, count, (float*)out);
  return done();
}

extern "C" fv3_status fv3_halo_scatter(void* field, int elem_size, const int64_t* dst, const void* in, int64_t count,
                                       fv3_stream stream) {
  if (count < 0 || (elem_size != 4 && elem_size != 8)) return FV3_ERR_ARG;
  if (count == 0) return FV3_OK;
  if (!field || !dst) return FV3_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (elem_size == 8)
    k_scatter<double><<<blocks_for(count), 256, 0, st>>>((double*)field, dst, (const double*)in, count);
  else
    k_scatter<float><<<blocks_for(count), 256, 0, st>>>((float*)field, dst, (const float*)in, count);
  return done();
}

extern "C" fv3_status fv3_halo_copy(void* field, int elem_size, const int64_t* src, const int64_t* dst,
                                    const int8_t* sign, int64_t count, fv3_stream stream) {
  if (count < 0 || (elem_size != 4 && elem_size != 8)) return FV3_ERR_ARG;
  if (count == 0) return FV3_OK;
  if (!field || !src || !dst) return FV3_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (elem_size == 8)
    k_copy<double><<<blocks_for(count), 256, 0, st>>>((double*)field, src, dst, sign, count);
  else
    k_copy<float><<<blocks_for(count), 256, 0, st>>>((float*)field, src, dst, sign, count);
  return done();
}

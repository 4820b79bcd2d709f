// fv3_mlp.cu -- training and batch inference of the face-value network.
//
// Reading R14 (no counterpart in the paper): the network of fv3_mlp.cuh is
// trained on coarse-grained fine-grid face values with the mirror-symmetric
// objective 0.5 * (ys(x) - t)^2, ys(x) = (y(x) + y(reversed x)) / 2.  One
// fused kernel runs the forward pass and the backward pass of both stencil
// orders for chunks of 32 samples per warp on the tensor cores (mma.sync,
// bfloat16 operands, float accumulation): the activation gradients dh =
// dz W^T and the weight gradients dW = a^T dz, whose reduction dimension is the
// sample index (the activations are transposed through shared memory).
// Per-block partial gradients are summed in a fixed order by a second kernel
// (deterministic).  Adam updates float master weights.
#include <cuda_runtime.h>

#include "fv3.h"
#include "fv3_mlp.cuh"

namespace fv3 {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kPart = MLP_NP + 1;  // gradient + loss per block

__global__ void __launch_bounds__(kThreads) k_mlp_forward(const float* w, const float* x, int n, int sym,
                                                          float* y) {
  MlpFrag F;
  mlp_load(w, F);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int base = (blockIdx.x * kWarps + warp) * 32; base < n; base += gridDim.x * kWarps * 32) {
    const int s = base + lane;
    float xi[6], xr[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) xi[c] = s < n ? x[6 * s + c] : 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) xr[c] = xi[5 - c];
    float v = mlp_warp(F, xi);
    if (sym) v = 0.5f * (v + mlp_warp(F, xr));
    if (s < n) y[s] = v;
  }
}

struct WarpSmem {
  __nv_bfloat16 X[32][16];    // inputs of the 32 samples (columns 6..15 zero)
  __nv_bfloat16 H1[32][32];   // layer-1 activations, sample-major
  __nv_bfloat16 D2[32][32];   // layer-2 pre-activation gradients
  __nv_bfloat16 D1[32][32];   // layer-1 pre-activation gradients
};

__device__ __forceinline__ unsigned pk(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  __nv_bfloat162 v;
  v.x = lo;
  v.y = hi;
  return *reinterpret_cast<unsigned*>(&v);
}

__global__ void __launch_bounds__(kThreads) k_mlp_grad(const float* w, const float* x, const float* t, int n,
                                                       float wt, float* part) {
  __shared__ float G[kPart];
  __shared__ WarpSmem WS[kWarps];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tg = lane & 3;
  for (int i = tid; i < kPart; i += kThreads) G[i] = 0.f;
  MlpFrag F;
  mlp_load(w, F);
  // W2^T fragments for dh1 = dz2 W2^T: B[k = j][n = i] = W2[i][j]
  unsigned b2t[2][4][2];
  for (int kc = 0; kc < 2; ++kc)
    for (int ni = 0; ni < 4; ++ni) {
      const int i = ni * 8 + g, j = kc * 16 + 2 * tg;
      b2t[kc][ni][0] = pack_bf16(__ldg(w + MLP_W2 + i * 32 + j), __ldg(w + MLP_W2 + i * 32 + j + 1));
      b2t[kc][ni][1] = pack_bf16(__ldg(w + MLP_W2 + i * 32 + j + 8), __ldg(w + MLP_W2 + i * 32 + j + 9));
    }
  float w3c[4][2];
  for (int nt = 0; nt < 4; ++nt)
    for (int e = 0; e < 2; ++e) w3c[nt][e] = __ldg(w + MLP_W3 + nt * 8 + 2 * tg + e);
  float gw2[2][4][4] = {}, gw1[4][4] = {};
  float gw3[4][2] = {}, gb2[4][2] = {}, gb1[4][2] = {};
  float gb3 = 0.f, loss = 0.f;
  WarpSmem& S = WS[warp];
  __syncthreads();
  for (int base = (blockIdx.x * kWarps + warp) * 32; base < n; base += gridDim.x * kWarps * 32) {
    const int s = base + lane;
    const bool valid = s < n;
    float xi[6], xr[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) xi[c] = valid ? x[6 * s + c] : 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) xr[c] = xi[5 - c];
    MlpAct A1, A2;
    const float y1 = mlp_warp(F, xi, &A1);
    const float y2 = mlp_warp(F, xr, &A2);
    const float ys = 0.5f * (y1 + y2);
    const float r = valid ? ys - t[s] : 0.f;
    loss += 0.5f * r * r * wt;
    const float gy = 0.5f * r * wt;  // upstream gradient of each orientation
    gb3 += 2.f * gy;
    for (int o = 0; o < 2; ++o) {
      const MlpAct& A = o == 0 ? A1 : A2;
      const float* xo = o == 0 ? xi : xr;
      float gyr[2][2];
      for (int mt = 0; mt < 2; ++mt)
        for (int hf = 0; hf < 2; ++hf) gyr[mt][hf] = __shfl_sync(0xffffffffu, gy, 16 * mt + g + 8 * hf);
      // layer 3 and the layer-2 pre-activation gradient
      float dz2[2][4][4];
      for (int mt = 0; mt < 2; ++mt)
        for (int nt = 0; nt < 4; ++nt)
          for (int e = 0; e < 4; ++e) {
            const float h = A.h2[mt][nt][e], gr = gyr[mt][e >> 1];
            gw3[nt][e & 1] += h * gr;
            const float d = gr * w3c[nt][e & 1] * (1.f - h * h);
            dz2[mt][nt][e] = d;
            gb2[nt][e & 1] += d;
          }
      // dh1 = dz2 W2^T, then the layer-1 pre-activation gradient
      float dz1[2][4][4];
      for (int mt = 0; mt < 2; ++mt)
        for (int ni = 0; ni < 4; ++ni) {
          float d[4] = {0.f, 0.f, 0.f, 0.f};
          for (int kc = 0; kc < 2; ++kc) {
            const float* p = dz2[mt][2 * kc];
            const float* q = dz2[mt][2 * kc + 1];
            mma_bf16(d, pack_bf16(p[0], p[1]), pack_bf16(p[2], p[3]), pack_bf16(q[0], q[1]), pack_bf16(q[2], q[3]),
                     b2t[kc][ni][0], b2t[kc][ni][1]);
          }
          for (int e = 0; e < 4; ++e) {
            const float h = A.h1[mt][ni][e];
            dz1[mt][ni][e] = d[e] * (1.f - h * h);
            gb1[ni][e & 1] += dz1[mt][ni][e];
          }
        }
      // stage sample-major copies for the weight gradients (reduction over samples)
      for (int mt = 0; mt < 2; ++mt)
        for (int nt = 0; nt < 4; ++nt)
          for (int e = 0; e < 4; ++e) {
            const int f = 16 * mt + g + 8 * (e >> 1), col = nt * 8 + 2 * tg + (e & 1);
            S.H1[f][col] = __float2bfloat16_rn(A.h1[mt][nt][e]);
            S.D2[f][col] = __float2bfloat16_rn(dz2[mt][nt][e]);
            S.D1[f][col] = __float2bfloat16_rn(dz1[mt][nt][e]);
          }
#pragma unroll
      for (int c = 0; c < 16; ++c) S.X[lane][c] = __float2bfloat16_rn(c < 6 ? xo[c] : 0.f);
      __syncwarp();
      // dW2[i][j] += sum_f H1[f][i] D2[f][j]   (M = i, N = j, K = f)
      for (int kf = 0; kf < 2; ++kf) {
        const int f0 = 16 * kf + 2 * tg;
        unsigned bb[4][2];
        for (int nj = 0; nj < 4; ++nj) {
          const int j = 8 * nj + g;
          bb[nj][0] = pk(S.D2[f0][j], S.D2[f0 + 1][j]);
          bb[nj][1] = pk(S.D2[f0 + 8][j], S.D2[f0 + 9][j]);
        }
        for (int mi = 0; mi < 2; ++mi) {
          const int i = 16 * mi + g;
          const unsigned a0 = pk(S.H1[f0][i], S.H1[f0 + 1][i]);
          const unsigned a1 = pk(S.H1[f0][i + 8], S.H1[f0 + 1][i + 8]);
          const unsigned a2 = pk(S.H1[f0 + 8][i], S.H1[f0 + 9][i]);
          const unsigned a3 = pk(S.H1[f0 + 8][i + 8], S.H1[f0 + 9][i + 8]);
          for (int nj = 0; nj < 4; ++nj) mma_bf16(gw2[mi][nj], a0, a1, a2, a3, bb[nj][0], bb[nj][1]);
        }
        // dW1[m][j] += sum_f X[f][m] D1[f][j]   (M = m (inputs, 16), N = j, K = f)
        const unsigned a0 = pk(S.X[f0][g], S.X[f0 + 1][g]);
        const unsigned a2 = pk(S.X[f0 + 8][g], S.X[f0 + 9][g]);
        for (int nj = 0; nj < 4; ++nj) {
          const int j = 8 * nj + g;
          mma_bf16(gw1[nj], a0, 0u, a2, 0u, pk(S.D1[f0][j], S.D1[f0 + 1][j]), pk(S.D1[f0 + 8][j], S.D1[f0 + 9][j]));
        }
      }
      __syncwarp();
    }
  }
  // reduce the warp's register partials into the block's shared gradient
  for (int mi = 0; mi < 2; ++mi)
    for (int nj = 0; nj < 4; ++nj)
      for (int e = 0; e < 4; ++e) {
        const int i = 16 * mi + g + 8 * (e >> 1), j = 8 * nj + 2 * tg + (e & 1);
        atomicAdd(&G[MLP_W2 + i * 32 + j], gw2[mi][nj][e]);
      }
  for (int nj = 0; nj < 4; ++nj)
    for (int e = 0; e < 2; ++e)
      if (g < 6) atomicAdd(&G[MLP_W1 + g * 32 + 8 * nj + 2 * tg + e], gw1[nj][e]);
  for (int nt = 0; nt < 4; ++nt)
    for (int e = 0; e < 2; ++e) {
      float a = gw3[nt][e], b = gb2[nt][e], c = gb1[nt][e];
      for (int m = 4; m < 32; m <<= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, m);
        b += __shfl_xor_sync(0xffffffffu, b, m);
        c += __shfl_xor_sync(0xffffffffu, c, m);
      }
      if (g == 0) {
        atomicAdd(&G[MLP_W3 + nt * 8 + 2 * tg + e], a);
        atomicAdd(&G[MLP_B2 + nt * 8 + 2 * tg + e], b);
        atomicAdd(&G[MLP_B1 + nt * 8 + 2 * tg + e], c);
      }
    }
  for (int m = 1; m < 32; m <<= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, m);
    loss += __shfl_xor_sync(0xffffffffu, loss, m);
  }
  if (lane == 0) {
    atomicAdd(&G[MLP_B3], gb3);
    atomicAdd(&G[MLP_NP], loss);
  }
  __syncthreads();
  for (int i = tid; i < kPart; i += kThreads) part[(long long)blockIdx.x * kPart + i] = G[i];
}

__global__ void k_mlp_reduce(const float* part, int nblocks, float* grad, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > MLP_NP) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += part[(long long)b * kPart + p];
  if (p < MLP_NP) grad[p] = s;
  else if (loss) *loss = s;
}

__global__ void k_mlp_adam(float* w, float* m, float* v, const float* g, float lr, float b1, float b2, float c1,
                           float c2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NP) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.f - b1) * gp;
  const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  w[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
}

// FP32 reference gradient (SIMT, float arithmetic, library tanhf): the same
// objective as k_mlp_grad without bfloat16 rounding, for checking the
// tensor-core gradient and the float training path against the FP64 oracle.
// Pass 1 stores per sample and stencil order the inputs, activations and
// pre-activation gradients; pass 2 sums every parameter's gradient over the
// samples in a fixed order (one thread per parameter, deterministic).
constexpr int kAct = 6 + 32 + 32 + 32 + 32 + 1;  // x, h1, h2, d2, d1, dy per order

__global__ void k_mlp_fp32_act(const float* w, const float* x, const float* t, int n, float wt, float* act) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float* A = act + (long long)s * (2 * kAct + 1);
  float y[2];
  for (int o = 0; o < 2; ++o) {
    float* xo = A + o * kAct;
    float *h1 = xo + 6, *h2 = h1 + 32;
    for (int i = 0; i < 6; ++i) xo[i] = x[6 * s + (o ? 5 - i : i)];
    for (int j = 0; j < 32; ++j) {
      float z = w[MLP_B1 + j];
      for (int i = 0; i < 6; ++i) z = fmaf(xo[i], w[MLP_W1 + i * 32 + j], z);
      h1[j] = tanhf(z);
    }
    for (int j = 0; j < 32; ++j) {
      float z = w[MLP_B2 + j];
      for (int i = 0; i < 32; ++i) z = fmaf(h1[i], w[MLP_W2 + i * 32 + j], z);
      h2[j] = tanhf(z);
    }
    float v = w[MLP_B3];
    for (int i = 0; i < 32; ++i) v = fmaf(h2[i], w[MLP_W3 + i], v);
    y[o] = v;
  }
  const float ys = 0.5f * (y[0] + y[1]);
  const float r = ys - t[s];
  A[2 * kAct] = 0.5f * r * r * wt;
  const float dy = 0.5f * r * wt;  // d loss / d y of each order
  for (int o = 0; o < 2; ++o) {
    float* xo = A + o * kAct;
    float *h1 = xo + 6, *h2 = h1 + 32, *d2 = h2 + 32, *d1 = d2 + 32;
    for (int j = 0; j < 32; ++j) d2[j] = dy * w[MLP_W3 + j] * (1.f - h2[j] * h2[j]);
    for (int i = 0; i < 32; ++i) {
      float a = 0.f;
      for (int j = 0; j < 32; ++j) a = fmaf(w[MLP_W2 + i * 32 + j], d2[j], a);
      d1[i] = a * (1.f - h1[i] * h1[i]);
    }
    d1[32] = dy;  // the output's gradient, after d1
  }
}

__global__ void k_mlp_fp32_sum(const float* act, int n, float* grad, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > MLP_NP) return;
  float sum = 0.f;
  for (int s = 0; s < n; ++s) {
    const float* A = act + (long long)s * (2 * kAct + 1);
    if (p == MLP_NP) {
      sum += A[2 * kAct];
      continue;
    }
    for (int o = 0; o < 2; ++o) {
      const float* xo = A + o * kAct;
      const float *h1 = xo + 6, *h2 = h1 + 32, *d2 = h2 + 32, *d1 = d2 + 32;
      const float dy = d1[32];
      float g;
      if (p < MLP_B1) g = xo[p / 32] * d1[p % 32];
      else if (p < MLP_W2) g = d1[p - MLP_B1];
      else if (p < MLP_B2) g = h1[(p - MLP_W2) / 32] * d2[(p - MLP_W2) % 32];
      else if (p < MLP_W3) g = d2[p - MLP_B2];
      else if (p < MLP_B3) g = h2[p - MLP_W3] * dy;
      else g = dy;
      sum += g;
    }
  }
  if (p < MLP_NP) grad[p] = sum;
  else if (loss) *loss = sum;
}

int grad_blocks(int n) {
  const int per = kThreads;  // samples per block per pass
  int b = (n + per - 1) / per;
  return b < 1 ? 1 : (b > 512 ? 512 : b);
}

}  // namespace
}  // namespace fv3

using namespace fv3;

extern "C" fv3_status fv3_mlp_forward(const float* w, const float* x, int n, int symmetric, float* y,
                                      fv3_stream stream) {
  if (!w || !x || !y || n < 0) return FV3_ERR_ARG;
  if (n == 0) return FV3_OK;
  const int blocks = grad_blocks(n);
  k_mlp_forward<<<blocks, kThreads, 0, (cudaStream_t)stream>>>(w, x, n, symmetric, y);
  return cudaGetLastError() == cudaSuccess ? FV3_OK : FV3_ERR_CUDA;
}

extern "C" size_t fv3_mlp_work_floats(int n) { return (size_t)grad_blocks(n) * kPart; }

extern "C" fv3_status fv3_mlp_grad(const float* w, const float* x, const float* t, int n, float weight, float* work,
                                   float* grad, float* loss, fv3_stream stream) {
  if (!w || !x || !t || !work || !grad || n < 1) return FV3_ERR_ARG;
  const int blocks = grad_blocks(n);
  cudaStream_t st = (cudaStream_t)stream;
  k_mlp_grad<<<blocks, kThreads, 0, st>>>(w, x, t, n, weight, work);
  k_mlp_reduce<<<(MLP_NP + 1 + 255) / 256, 256, 0, st>>>(work, blocks, grad, loss);
  return cudaGetLastError() == cudaSuccess ? FV3_OK : FV3_ERR_CUDA;
}

extern "C" size_t fv3_mlp_work_floats_fp32(int n) { return (size_t)(n > 0 ? n : 0) * (2 * kAct + 1); }

extern "C" fv3_status fv3_mlp_grad_fp32(const float* w, const float* x, const float* t, int n, float weight,
                                        float* work, float* grad, float* loss, fv3_stream stream) {
  if (!w || !x || !t || !work || !grad || n < 1) return FV3_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  k_mlp_fp32_act<<<(n + 127) / 128, 128, 0, st>>>(w, x, t, n, weight, work);
  k_mlp_fp32_sum<<<(MLP_NP + 1 + 127) / 128, 128, 0, st>>>(work, n, grad, loss);
  return cudaGetLastError() == cudaSuccess ? FV3_OK : FV3_ERR_CUDA;
}

extern "C" fv3_status fv3_mlp_adam(float* w, float* m, float* v, const float* grad, int step, float lr,
                                   fv3_stream stream) {
  if (!w || !m || !v || !grad || step < 1) return FV3_ERR_ARG;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, m, v, grad, lr, b1, b2, c1, c2, 1e-8f);
  return cudaGetLastError() == cudaSuccess ? FV3_OK : FV3_ERR_CUDA;
}

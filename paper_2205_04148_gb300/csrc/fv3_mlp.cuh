// fv3_mlp.cuh -- warp-level tensor-core evaluation of the face-value network.
//
// The learned face value (reading R14; the paper has no learned component, it
// motivates coupling machine-learned models to the dynamical core in Section
// III-B) is a 6 -> 32 -> 32 -> 1 tanh network.  A warp evaluates it for 32
// faces at once with mma.sync m16n8k16 (bfloat16 inputs and weights, float
// accumulation): rows of the A operand are the warp's faces (two M tiles of
// 16), layer widths are the N dimension.  The float accumulator fragment of
// one layer has the same lane/element assignment as the A fragment of the
// next layer, so activations never leave registers.
//
// Parameters, flat float[1313]: W1[6][32] (input i -> hidden j at i*32+j),
// b1[32], W2[32][32], b2[32], W3[32], b3.
#pragma once
#include <cuda_bf16.h>

namespace fv3 {

constexpr int MLP_NP = 1313, MLP_W1 = 0, MLP_B1 = 192, MLP_W2 = 224, MLP_B2 = 1248, MLP_W3 = 1280, MLP_B3 = 1312;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<unsigned*>(&v);
}

// D += A(16x16, row) * B(16x8, col), bfloat16 in, float accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ int lane_id() { return (int)((threadIdx.y * blockDim.x + threadIdx.x) & 31); }

// weight fragments held by one lane (B operands) and the biases of the
// accumulator columns the lane owns
struct MlpFrag {
  unsigned b1[4][2];     // layer 1: n-tiles 0..3, K = inputs padded to 16
  unsigned b2[2][4][2];  // layer 2: k-chunks 0..1 x n-tiles 0..3
  unsigned b3[2][2];     // layer 3: k-chunks 0..1, one n-tile (column 0 = W3)
  float c1[4][2], c2[4][2], c3;
};

__device__ __forceinline__ float wget(const float* w, int i) { return __ldg(w + i); }

__device__ __forceinline__ void mlp_load(const float* w, MlpFrag& F) {
  const int lane = lane_id(), g = lane >> 2, t = lane & 3;
  for (int nt = 0; nt < 4; ++nt) {
    const int n = nt * 8 + g;
    auto w1 = [&](int k) { return k < 6 ? wget(w, MLP_W1 + k * 32 + n) : 0.f; };
    F.b1[nt][0] = pack_bf16(w1(2 * t), w1(2 * t + 1));
    F.b1[nt][1] = pack_bf16(w1(2 * t + 8), w1(2 * t + 9));
    for (int kc = 0; kc < 2; ++kc) {
      const int k = kc * 16 + 2 * t;
      F.b2[kc][nt][0] = pack_bf16(wget(w, MLP_W2 + k * 32 + n), wget(w, MLP_W2 + (k + 1) * 32 + n));
      F.b2[kc][nt][1] = pack_bf16(wget(w, MLP_W2 + (k + 8) * 32 + n), wget(w, MLP_W2 + (k + 9) * 32 + n));
    }
    for (int e = 0; e < 2; ++e) {
      F.c1[nt][e] = wget(w, MLP_B1 + nt * 8 + 2 * t + e);
      F.c2[nt][e] = wget(w, MLP_B2 + nt * 8 + 2 * t + e);
    }
  }
  for (int kc = 0; kc < 2; ++kc) {
    const int k = kc * 16 + 2 * t;
    F.b3[kc][0] = g == 0 ? pack_bf16(wget(w, MLP_W3 + k), wget(w, MLP_W3 + k + 1)) : 0u;
    F.b3[kc][1] = g == 0 ? pack_bf16(wget(w, MLP_W3 + k + 8), wget(w, MLP_W3 + k + 9)) : 0u;
  }
  F.c3 = wget(w, MLP_B3);
}

// activations of one warp: layer outputs in accumulator layout
// acc[mt][nt][e]: row (face) 16*mt + g + 8*(e >> 1), column nt*8 + 2t + (e & 1)
struct MlpAct {
  float h1[2][4][4], h2[2][4][4];
};

// x: this lane's six inputs.  Returns this lane's network output; fills A
// with the hidden activations (tanh outputs) when A is non-null.
__device__ __forceinline__ float mlp_warp(const MlpFrag& F, const float (&x)[6], MlpAct* A = nullptr) {
  const int lane = lane_id(), g = lane >> 2, t = lane & 3;
  float h1[2][4][4], h2[2][4][4];
  for (int mt = 0; mt < 2; ++mt) {
    unsigned a[2];
    for (int half = 0; half < 2; ++half) {  // rows g and g + 8 of this M tile
      const int src = 16 * mt + g + 8 * half;
      float xs[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) xs[c] = __shfl_sync(0xffffffffu, x[c], src);
      const float v0 = t == 0 ? xs[0] : t == 1 ? xs[2] : t == 2 ? xs[4] : 0.f;
      const float v1 = t == 0 ? xs[1] : t == 1 ? xs[3] : t == 2 ? xs[5] : 0.f;
      a[half] = pack_bf16(v0, v1);
    }
    for (int nt = 0; nt < 4; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(d, a[0], a[1], 0u, 0u, F.b1[nt][0], F.b1[nt][1]);
#pragma unroll
      for (int e = 0; e < 4; ++e) h1[mt][nt][e] = tanh_fast(d[e] + F.c1[nt][e & 1]);
    }
  }
  for (int mt = 0; mt < 2; ++mt)
    for (int nt = 0; nt < 4; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      for (int kc = 0; kc < 2; ++kc) {
        const float* p = h1[mt][2 * kc];
        const float* q = h1[mt][2 * kc + 1];
        mma_bf16(d, pack_bf16(p[0], p[1]), pack_bf16(p[2], p[3]), pack_bf16(q[0], q[1]), pack_bf16(q[2], q[3]),
                 F.b2[kc][nt][0], F.b2[kc][nt][1]);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) h2[mt][nt][e] = tanh_fast(d[e] + F.c2[nt][e & 1]);
    }
  float out[2][4];
  for (int mt = 0; mt < 2; ++mt) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kc = 0; kc < 2; ++kc) {
      const float* p = h2[mt][2 * kc];
      const float* q = h2[mt][2 * kc + 1];
      mma_bf16(d, pack_bf16(p[0], p[1]), pack_bf16(p[2], p[3]), pack_bf16(q[0], q[1]), pack_bf16(q[2], q[3]),
               F.b3[kc][0], F.b3[kc][1]);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) out[mt][e] = d[e];
  }
  if (A) {
    for (int mt = 0; mt < 2; ++mt)
      for (int nt = 0; nt < 4; ++nt)
        for (int e = 0; e < 4; ++e) {
          A->h1[mt][nt][e] = h1[mt][nt][e];
          A->h2[mt][nt][e] = h2[mt][nt][e];
        }
  }
  // column 0 of the output tile: lane 4r holds rows r (e = 0) and r + 8 (e = 2)
  const int mt = lane >> 4, r = lane & 15, src = 4 * (r & 7);
  const float s0 = __shfl_sync(0xffffffffu, out[0][0], src);
  const float s1 = __shfl_sync(0xffffffffu, out[0][2], src);
  const float s2 = __shfl_sync(0xffffffffu, out[1][0], src);
  const float s3 = __shfl_sync(0xffffffffu, out[1][2], src);
  const float y = mt == 0 ? (r < 8 ? s0 : s1) : (r < 8 ? s2 : s3);
  return y + F.c3;
}

// network inputs of a six-cell stencil (reading R14: x = (q - mean) / (sig +
// 1e-12 |mean|), sig the standard deviation): offsets d from the mean r of
// the two centre cells in the stencil's precision, rounded to float; then in
// float the mean m of the offsets, deviations e = d - m, sig and x = e / (sig
// + 1e-12 |r| + 1e-30) (|r| stands for the stencil mean's magnitude: the two
// differ by less than 5 sig), all sums in mirror pairs and without
// contraction so the reversed stencil gives the reversed inputs bit for bit.
// ar = |r| as a float.  Returns sig; xr = reversed x.
__device__ __forceinline__ float mlp_offsets_to_inputs(const float (&d)[6], float ar, float (&x)[6],
                                                      float (&xr)[6]) {
  const float sixth = 1.0f / 6.0f;
  const float m =
      __fmul_rn(__fadd_rn(__fadd_rn(__fadd_rn(d[0], d[5]), __fadd_rn(d[1], d[4])), __fadd_rn(d[2], d[3])), sixth);
  float e[6], sq[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    e[i] = __fsub_rn(d[i], m);
    sq[i] = __fmul_rn(e[i], e[i]);
  }
  const float v =
      __fmul_rn(__fadd_rn(__fadd_rn(__fadd_rn(sq[0], sq[5]), __fadd_rn(sq[1], sq[4])), __fadd_rn(sq[2], sq[3])), sixth);
  const float sig = __fsqrt_rn(v);
  const float inv = __fdiv_rn(1.0f, __fadd_rn(__fadd_rn(sig, __fmul_rn(1e-12f, ar)), 1e-30f));
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    x[i] = __fmul_rn(e[i], inv);
    xr[5 - i] = x[i];
  }
  return sig;
}

template <typename R>
__device__ __forceinline__ float mlp_inputs(const R (&q)[6], float (&x)[6], float (&xr)[6]);

// double -> float, round to nearest even (IEEE 754), on the integer pipe:
// the FP64 pipe (2 lanes per SM per clock) is the bottleneck of the learned
// transport.  Results below the float normal range flush to zero (the
// offsets they would encode are far below any stencil's variation).
__device__ __forceinline__ float to_float_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned long long m = b & 0xfffffffffffffULL;
  unsigned f = ((unsigned)e << 23) | (unsigned)(m >> 29);
  const unsigned long long rem = m & 0x1fffffffULL, half = 0x10000000ULL;
  f += (rem > half || (rem == half && (f & 1u))) ? 1u : 0u;  // a carry raises the exponent
  return __uint_as_float(sign | f);
}

// float -> double (exact for normal floats), on the integer pipe; float
// subnormals flush to zero
__device__ __forceinline__ double to_double(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const int e = (int)((b >> 23) & 0xff);
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ee = e == 255 ? 0x7ffULL : (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(sign | (ee << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

template <typename R>
__device__ __forceinline__ R widen(float x);
template <>
__device__ __forceinline__ double widen<double>(float x) { return to_double(x); }
template <>
__device__ __forceinline__ float widen<float>(float x) { return x; }

template <>
__device__ __forceinline__ float mlp_inputs<double>(const double (&q)[6], float (&x)[6], float (&xr)[6]) {
  const double r = __dmul_rn(0.5, __dadd_rn(q[2], q[3]));
  float d[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) d[i] = to_float_rn(__dsub_rn(q[i], r));
  return mlp_offsets_to_inputs(d, fabsf(to_float_rn(r)), x, xr);
}

template <>
__device__ __forceinline__ float mlp_inputs<float>(const float (&q)[6], float (&x)[6], float (&xr)[6]) {
  const float r = __fmul_rn(0.5f, __fadd_rn(q[2], q[3]));
  float d[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) d[i] = __fsub_rn(q[i], r);
  return mlp_offsets_to_inputs(d, fabsf(r), x, xr);
}

}  // namespace fv3

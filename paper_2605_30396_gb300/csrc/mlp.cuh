// Definitions shared by the proposal network's kernels (mlp.cu: training and
// the layer-by-layer forward; propose.cu: the fused inference kernel).  The
// element-wise arithmetic lives here once, written with explicit rounding
// intrinsics, so that both paths produce bit-identical activations and logits.
#pragma once

#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "host.hpp"

namespace dlsh {
namespace mlp {

constexpr int HID = 256;  // hidden width
constexpr int XIN = 64;   // input width (45 padded to a whole k-tile)

// Parameter vector layout (FP32 masters; a BF16 mirror has the same offsets).
struct Layout {
  long long W1, b1, W2, b2, W3, b3, n;
};
__host__ __device__ inline Layout layout(int K) {
  Layout L;
  L.W1 = 0;
  L.b1 = L.W1 + static_cast<long long>(HID) * XIN;
  L.W2 = L.b1 + HID;
  L.b2 = L.W2 + static_cast<long long>(HID) * HID;
  L.W3 = L.b2 + HID;
  L.b3 = L.W3 + static_cast<long long>(K) * HID;
  L.n = L.b3 + K;
  return L;
}

// Blob: P (FP32) | M1 (FP32) | M2 (FP32) | Pb (BF16) | step counter.
struct Blob {
  float* P;
  float* m1;
  float* m2;
  __nv_bfloat16* Pb;
  long long* step;
};
inline size_t carve_blob(void* base, int K, Blob& b) {
  const Layout L = layout(K);
  Carver c(base);
  b.P = c.take<float>(L.n);
  b.m1 = c.take<float>(L.n);
  b.m2 = c.take<float>(L.n);
  b.Pb = c.take<__nv_bfloat16>(L.n);
  b.step = c.take<long long>(2);
  return c.size();
}

// GELU, exact erf form: 0.5 z (1 + erf(z / sqrt 2)).
__device__ __forceinline__ float gelu_f(float z) {
  return __fmul_rn(__fmul_rn(0.5f, z), __fadd_rn(1.f, erff(__fmul_rn(z, 0.70710678118654752f))));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Pre-activation of an output unit: accumulator plus bias, one rounding.
__device__ __forceinline__ float add_bias(float acc, float bias) { return __fadd_rn(acc, bias); }

// Network input: x / ||x|| (0 when x = 0) for one 45-dim signal held by a
// warp: lane l holds x[l] in x0 and x[32 + l] in x1 (0 for l >= 13).  The
// squared norm is reduced over the warp in a fixed butterfly order.
__device__ __forceinline__ void normalise_pair(float x0, float x1, __nv_bfloat16& y0,
                                               __nv_bfloat16& y1) {
  float n2 = __fmaf_rn(x1, x1, __fmul_rn(x0, x0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n2 = __fadd_rn(n2, __shfl_xor_sync(0xffffffffu, n2, o));
  const float inv = n2 > 0.f ? rsqrtf(n2) : 0.f;
  y0 = __float2bfloat16(__fmul_rn(x0, inv));
  y1 = __float2bfloat16(__fmul_rn(x1, inv));
}

}  // namespace mlp
}  // namespace dlsh

// Learned precision predictor: inference rule (the PPM of Section 4.1; the
// regressor of Section 3.4 is replaced by a 5-32-32-5 MLP classifier over the
// bit widths 4/6/8/12/16).
//
// FP16 operands (weights, biases, normalised inputs, hidden activations) and
// FP32 accumulation: acc = b; for i ascending: acc = fma(W[o][i], x[i], acc).
// The product of two FP16 values is exact in FP32, so the FMA rounds exactly
// once, like fl32(acc + W*x). Hidden layers apply ReLU and round to FP16;
// logits stay FP32. The width is the fewest bits c whose best logit beats the
// best logit of every wider width by at least the margin tau,
// fl32(max_{i<=c} z_i - max_{i>c} z_i) >= tau, else 16 bits: tau = 0 is the
// argmax with ties to the narrower width, tau > 0 rounds uncertain pairs up
// and tau < 0 rounds them down.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "common.cuh"

namespace anns {

struct MlpParams16 {
  __half W1[32 * 5], b1[32], W2[32 * 32], b2[32], W3[5 * 32], b3[5];
  float mean[5], inv_std[5];
};

__device__ __forceinline__ uint8_t mlp_decide(const MlpParams16& P, const float f[5], float tau) {
  constexpr uint8_t kBits[5] = {4, 6, 8, 12, 16};
  float x[5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
    x[i] = __half2float(__float2half_rn(mul_rn(sub_rn(f[i], P.mean[i]), P.inv_std[i])));
  float h1[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    float acc = __half2float(P.b1[o]);
#pragma unroll
    for (int i = 0; i < 5; ++i) acc = fmaf(__half2float(P.W1[o * 5 + i]), x[i], acc);
    h1[o] = __half2float(__float2half_rn(fmaxf(acc, 0.f)));
  }
  float h2[32];
#pragma unroll 4
  for (int o = 0; o < 32; ++o) {
    float acc = __half2float(P.b2[o]);
#pragma unroll
    for (int i = 0; i < 32; ++i) acc = fmaf(__half2float(P.W2[o * 32 + i]), h1[i], acc);
    h2[o] = __half2float(__float2half_rn(fmaxf(acc, 0.f)));
  }
  float z[5];
#pragma unroll
  for (int o = 0; o < 5; ++o) {
    float acc = __half2float(P.b3[o]);
#pragma unroll
    for (int i = 0; i < 32; ++i) acc = fmaf(__half2float(P.W3[o * 32 + i]), h2[i], acc);
    z[o] = acc;
  }
  // the fewest bits c whose best logit (widths <= c) beats every wider width by tau
  int c = 4;
  float lo = -INFINITY;
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    lo = fmaxf(lo, z[cc]);
    float hi = -INFINITY;
#pragma unroll
    for (int o = cc + 1; o < 5; ++o) hi = fmaxf(hi, z[o]);
    if (c == 4 && sub_rn(lo, hi) >= tau) c = cc;
  }
  return kBits[c];
}

}  // namespace anns

// The learned car-dynamics surrogate: parameter layout and input features (device side).
//
//   features  z (16): X/20, Y/20, wrap(psi)/pi, (vx-5)/5, vy/2, r/3, delta/0.5, u_s/1.6,
//             u_t/1.8, zero padding (psi wrapped to (-pi, pi])
//   network   h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3
//   step      x' = x + y[0:7] * out_scale
// Parameters are one flat FP32 array: W1 [256][16], b1 [256], W2 [256][256], b2 [256],
// W3 [16][256], b3 [16] (row = output unit).
#pragma once
#include <cstddef>

namespace mppi {
namespace mlp {

constexpr int kIn = 16, kHid = 256, kOut = 16, kState = 7, kCtl = 2;
constexpr size_t kOffW1 = 0;
constexpr size_t kOffB1 = kOffW1 + static_cast<size_t>(kHid) * kIn;
constexpr size_t kOffW2 = kOffB1 + kHid;
constexpr size_t kOffB2 = kOffW2 + static_cast<size_t>(kHid) * kHid;
constexpr size_t kOffW3 = kOffB2 + kHid;
constexpr size_t kOffB3 = kOffW3 + static_cast<size_t>(kOut) * kHid;
constexpr size_t kNumParams = kOffB3 + kOut;

__host__ __device__ __forceinline__ float wrap_pi(float a) {
  return a - 6.283185307179586f * ceilf((a - 3.14159265358979f) * 0.15915494309189535f);
}

__host__ __device__ __forceinline__ void features(const float *x, const float *u, float *z) {
  z[0] = x[0] * (1.0f / 20.0f);
  z[1] = x[1] * (1.0f / 20.0f);
  z[2] = wrap_pi(x[2]) * 0.3183098861837907f;
  z[3] = (x[3] - 5.0f) * (1.0f / 5.0f);
  z[4] = x[4] * (1.0f / 2.0f);
  z[5] = x[5] * (1.0f / 3.0f);
  z[6] = x[6] * (1.0f / 0.5f);
  z[7] = u[0] * (1.0f / 1.6f);
  z[8] = u[1] * (1.0f / 1.8f);
#pragma unroll
  for (int i = 9; i < kIn; ++i) z[i] = 0.0f;
}

}  // namespace mlp
}  // namespace mppi

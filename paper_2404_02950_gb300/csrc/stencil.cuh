// Finite-difference weights of App. A (the "Laplacian" and "Gradient"
// stencils of accuracy 2G, G = 1, 2, 3 cells per side), as device constants.
#pragma once

namespace slh {

// Central second-difference weights w_m, m = 0..G (w_0 the centre weight).
template <int G>
__device__ __forceinline__ double lap_w(int m);
template <>
__device__ __forceinline__ double lap_w<1>(int m) { return m == 0 ? -2.0 : 1.0; }
template <>
__device__ __forceinline__ double lap_w<2>(int m) { return m == 0 ? -2.5 : (m == 1 ? 4.0 / 3.0 : -1.0 / 12.0); }
template <>
__device__ __forceinline__ double lap_w<3>(int m) {
  return m == 0 ? -49.0 / 18.0 : (m == 1 ? 1.5 : (m == 2 ? -0.15 : 1.0 / 90.0));
}

// Central first-difference weights: f'(0) ~ sum_{m=1..G} g_m (f(m) - f(-m)).
template <int G>
__device__ __forceinline__ double grad_w(int m);
template <>
__device__ __forceinline__ double grad_w<1>(int m) { return m == 1 ? 0.5 : 0.0; }
template <>
__device__ __forceinline__ double grad_w<2>(int m) { return m == 1 ? 2.0 / 3.0 : -1.0 / 12.0; }
template <>
__device__ __forceinline__ double grad_w<3>(int m) { return m == 1 ? 0.75 : (m == 2 ? -0.15 : 1.0 / 60.0); }

}  // namespace slh

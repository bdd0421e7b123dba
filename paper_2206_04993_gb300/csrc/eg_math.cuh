// Device-side pieces of the update rule shared by the kernel paths.
#pragma once

#include <cuda_runtime.h>

namespace sgep {

// Coefficients of the matrix form of Eq. (update), from the k x k terms
// [a (k*k) | G (k*k) | b (k)] with a_ij = v_i^T A_t v_j, G_ij = <v_i, [Bv]_j>,
// b_i = v_i^T B_t v_i:
//   s_j = max(G_jj, rho)                                  (clipping, Alg. 2)
//   c_i = sum_{j<i} a_ij G_ij / s_j                        (<v_i, [By]_j> terms)
//   T_ji = b_i a_ij / s_j for j < i, else 0                (<v_i, B v_i> [By]_j terms)
//   grad_i = b_i A_t v_i - (a_i - c_i) B_t v_i - sum_{j<i} T_ji [Bv]_j
// which is reward minus penalty with y_j = v_j / sqrt(s_j), [By]_j = [Bv]_j / sqrt(s_j).
// Block-cooperative; the caller synchronises afterwards.
__device__ inline void eg_coefficients(const float* __restrict__ terms, int k, float rho,
                                       float* coef_b, float* coef_ac, float* T) {
  const int kk = k * k;
  const float* a = terms;
  const float* G = terms + kk;
  const float* bd = terms + 2 * kk;
  for (int p = threadIdx.x; p < kk; p += blockDim.x) {
    const int j = p / k, i = p % k;
    float t = 0.f;
    if (j < i) t = bd[i] * a[i * k + j] / fmaxf(G[j * k + j], rho);
    T[p] = t;
  }
  // c_i: one thread per (i, j) term, then a short sum per i in a fixed order
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    float c0 = 0.f, c1 = 0.f;
    int j = 0;
    for (; j + 1 < i; j += 2) {
      c0 += a[i * k + j] * G[i * k + j] / fmaxf(G[j * k + j], rho);
      c1 += a[i * k + j + 1] * G[i * k + j + 1] / fmaxf(G[(j + 1) * k + j + 1], rho);
    }
    if (j < i) c0 += a[i * k + j] * G[i * k + j] / fmaxf(G[j * k + j], rho);
    coef_b[i] = bd[i];
    coef_ac[i] = a[i * k + i] - (c0 + c1);
  }
}

}  // namespace sgep

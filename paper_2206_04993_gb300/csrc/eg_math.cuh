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
// sden (k values, or null): the denominators s_j of Alg. 3 in place of the clipping.
// Block-cooperative; the caller synchronises afterwards.
__device__ inline void eg_coefficients(const float* __restrict__ terms, int k, float rho,
                                       float* coef_b, float* coef_ac, float* T,
                                       const float* sden = nullptr) {
  const int kk = k * k;
  const float* a = terms;
  const float* G = terms + kk;
  const float* bd = terms + 2 * kk;
  auto den = [&](int j) { return sden ? sden[j] : fmaxf(G[j * k + j], rho); };
  for (int p = threadIdx.x; p < kk; p += blockDim.x) {
    const int j = p / k, i = p % k;
    float t = 0.f;
    if (j < i) t = bd[i] * a[i * k + j] / den(j);
    T[p] = t;
  }
  // c_i: one thread per (i, j) term, then a short sum per i in a fixed order
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    float c0 = 0.f, c1 = 0.f;
    int j = 0;
    for (; j + 1 < i; j += 2) {
      c0 += a[i * k + j] * G[i * k + j] / den(j);
      c1 += a[i * k + j + 1] * G[i * k + j + 1] / den(j + 1);
    }
    if (j < i) c0 += a[i * k + j] * G[i * k + j] / den(j);
    coef_b[i] = bd[i];
    coef_ac[i] = a[i * k + i] - (c0 + c1);
  }
}

// Alg. 3's denominator exp(log rho + (log nu - log rho) sigmoid(z)), in (rho, nu).
__device__ __forceinline__ float smooth_den(float z, float log_rho, float log_nu) {
  const float sg = 1.f / (1.f + expf(-z));
  return expf(log_rho + (log_nu - log_rho) * sg);
}
// Alg. 3's z step: z + gamma (c - s) s (log nu - log rho) sigmoid(z) (1 - sigmoid(z)), where
// c = <v, [Bv]> and s = smooth_den(z) are taken at step t.
__device__ __forceinline__ float smooth_z_step(float z, float c, float gamma, float log_rho, float log_nu) {
  const float sg = 1.f / (1.f + expf(-z));
  const float s = expf(log_rho + (log_nu - log_rho) * sg);
  return fmaf(gamma, (c - s) * s * (log_nu - log_rho) * sg * (1.f - sg), z);
}
// Adam's player step (App. H.2.2) for one element with update direction g: updates the
// moments in place and returns the increment m_hat / (sqrt(s_hat) + eps).
__device__ __forceinline__ float adam_increment(float g, float& m, float& s, float b1, float b2, float eps, float bc1,
                                                float bc2) {
  m = fmaf(b1, m, (1.f - b1) * g);
  s = fmaf(b2, s, (1.f - b2) * g * g);
  return (m / bc1) / (sqrtf(s / bc2) + eps);
}

}  // namespace sgep

// LDA kind of the gamma-EigenGame products (generic SIMT path).
//
// The paper names LDA among the generalized eigenproblems of Sec. 1 but gives no
// estimators. Reading: A is the between-class scatter
//   A = sum_c pi_c (mu_c - mu)(mu_c - mu)^T,   mu = sum_c pi_c mu_c,
// with mu_c and pi_c = n_c / n the exact running class means and priors over every
// row seen so far (a step first adds all of its rows), and B_t is the within-class
// covariance of the minibatch's B rows, each centred by the mean of its class:
//   B_t V = X~^T (X~ V) / n_B,   x~_r = x_r - mu_{label r}.
// A V therefore costs O(C d k) from the class means (no pass over the rows):
//   W = (mu_c - mu)^T V  (C x k),   A V = sum_c (mu_c - mu) pi_c W_c.
// The k x k terms and the update are the generic ones.
#include <cuda_fp8.h>

#include <algorithm>

#include "generic_tiles.cuh"
#include "internal.h"

namespace sgep {
namespace {

using gt::kThreads;

// One tile per block; the tile functions live in generic_tiles.cuh.
__global__ void k_lda_counts(const int32_t* __restrict__ labels, int64_t b, int C, double* __restrict__ cnt,
                             float* __restrict__ pi, int* dflag) {
  __shared__ float smem[gt::kLdaCountsSmem];
  gt::lda_counts_tile(labels, b, C, cnt, pi, dflag, smem);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_lda_stats(const T* __restrict__ X, const float* __restrict__ rs,
                                                        const int32_t* __restrict__ labels, int64_t b, int64_t d,
                                                        int C, double* __restrict__ sum,
                                                        const double* __restrict__ cnt, float* __restrict__ mean,
                                                        float* __restrict__ M) {
  extern __shared__ float smem[];
  gt::lda_stats_tile(X, rs, labels, b, d, C, sum, cnt, mean, M, blockIdx.x, smem);
}

__global__ void __launch_bounds__(kThreads) k_lda_w(const float* __restrict__ M, const float* __restrict__ V,
                                                    int64_t d, int C, int k, float* __restrict__ W) {
  __shared__ float smem[gt::kLdaWSmem];
  gt::lda_w_tile(M, V, d, C, k, W, blockIdx.x, gridDim.x, smem);
}

__global__ void __launch_bounds__(kThreads) k_lda_av(const float* __restrict__ M, const float* __restrict__ pi,
                                                     const float* __restrict__ W, int64_t d, int C, int k,
                                                     float* __restrict__ AV) {
  __shared__ float smem[gt::kLdaAvSmem];
  gt::lda_av_tile(M, pi, W, d, C, k, AV, blockIdx.x, gridDim.x, smem);
}

}  // namespace

int lda_alloc(Ctx& c) {
  const int C = c.cfg.n_classes;
  const size_t cd = (size_t)C * c.d;
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.lda_sum, cd * sizeof(double)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.lda_cnt, (size_t)C * sizeof(double)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.lda_mean, cd * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.lda_M, cd * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.lda_pi, (size_t)C * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.lda_W, (size_t)C * c.k * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(c.lda_sum, 0, cd * sizeof(double)));
  SGEP_CUDA_TRY(cudaMemset(c.lda_cnt, 0, (size_t)C * sizeof(double)));
  SGEP_CUDA_TRY(cudaMemset(c.lda_mean, 0, cd * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(c.lda_M, 0, cd * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(c.lda_pi, 0, (size_t)C * sizeof(float)));
  return SGEP_OK;
}

void lda_free(Ctx& c) {
  cudaFree(c.lda_sum);
  cudaFree(c.lda_cnt);
  cudaFree(c.lda_mean);
  cudaFree(c.lda_M);
  cudaFree(c.lda_pi);
  cudaFree(c.lda_W);
  c.lda_sum = c.lda_cnt = nullptr;
  c.lda_mean = c.lda_M = c.lda_pi = c.lda_W = nullptr;
}

static int stats(Ctx& c, const void* X, const int32_t* labels, int64_t b, cudaStream_t s, const float* sx) {
  const int C = c.cfg.n_classes;
  k_lda_counts<<<1, kThreads, 0, s>>>(labels, b, C, c.lda_cnt, c.lda_pi, c.dflag);
  SGEP_CUDA_TRY(cudaGetLastError());
  const unsigned grid = (unsigned)((c.d + kThreads - 1) / kThreads);
  const size_t smem = (size_t)gt::lda_stats_smem(C) * sizeof(float);  // above 48 KB for C >= 16
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_lda_stats<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  SGEP_CUDA_TRY(
      cudaFuncSetAttribute(k_lda_stats<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  SGEP_CUDA_TRY(
      cudaFuncSetAttribute(k_lda_stats<__nv_fp8_e4m3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (c.cfg.dtype == SGEP_BF16)
    k_lda_stats<__nv_bfloat16><<<grid, kThreads, smem, s>>>((const __nv_bfloat16*)X, sx, labels, b, c.d, C,
                                                            c.lda_sum, c.lda_cnt, c.lda_mean, c.lda_M);
  else if (c.cfg.dtype == SGEP_FP8E4M3)
    k_lda_stats<__nv_fp8_e4m3><<<grid, kThreads, smem, s>>>((const __nv_fp8_e4m3*)X, sx, labels, b, c.d, C,
                                                            c.lda_sum, c.lda_cnt, c.lda_mean, c.lda_M);
  else
    k_lda_stats<float><<<grid, kThreads, smem, s>>>((const float*)X, sx, labels, b, c.d, C, c.lda_sum, c.lda_cnt,
                                                    c.lda_mean, c.lda_M);
  SGEP_CUDA_TRY(cudaGetLastError());
  c.launches += 2;
  return SGEP_OK;
}

int lda_refresh(Ctx& c, cudaStream_t s) { return stats(c, nullptr, nullptr, 0, s, nullptr); }

int lda_project_means(Ctx& c, cudaStream_t s) {
  SGEP_CUDA_TRY(cudaMemsetAsync(c.lda_W, 0, (size_t)c.cfg.n_classes * c.k * sizeof(float), s));
  const int grid = (int)std::min<int64_t>((c.d + 31) / 32, 2LL * c.num_sms);
  k_lda_w<<<grid, kThreads, 0, s>>>(c.lda_M, c.V, c.d, c.cfg.n_classes, c.k, c.lda_W);
  SGEP_CUDA_TRY(cudaGetLastError());
  ++c.launches;
  return SGEP_OK;
}

int lda_products(Ctx& c, const void* X, const int32_t* labels, int64_t b, cudaStream_t s, const float* sx) {
  int rc = stats(c, X, labels, b, s, sx);
  if (rc) return rc;
  SGEP_CUDA_TRY(cudaMemsetAsync(c.acc, 0, sizeof(float) * 2 * c.d * c.k, s));
  // B_t V from the B rows (second half when the batch is split), centred by class means
  const int64_t nA = c.cfg.split_AB ? b / 2 : 0;
  rc = generic_lda_within(c, (const char*)X + (size_t)nA * c.d * elem_size(c), labels + nA, b - nA, s,
                          sx ? sx + nA : nullptr);
  if (rc) return rc;
  // A V from the class means
  rc = lda_project_means(c, s);
  if (rc) return rc;
  const int grid = (int)std::min<int64_t>((c.d * c.k + kThreads - 1) / kThreads, 4LL * c.num_sms);
  k_lda_av<<<grid, kThreads, 0, s>>>(c.lda_M, c.lda_pi, c.lda_W, c.d, c.cfg.n_classes, c.k, c.acc);
  SGEP_CUDA_TRY(cudaGetLastError());
  ++c.launches;
  return SGEP_OK;
}

}  // namespace sgep

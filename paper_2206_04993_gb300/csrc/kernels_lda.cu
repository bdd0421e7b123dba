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

#include "internal.h"

namespace sgep {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float load_x(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_x(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float load_x(const __nv_fp8_e4m3* p, int64_t i) { return static_cast<float>(p[i]); }

// Counts of this minibatch's labels added to the running counts; priors. One block.
__global__ void k_lda_counts(const int32_t* __restrict__ labels, int64_t b, int C, double* __restrict__ cnt,
                             float* __restrict__ pi, int* dflag) {
  __shared__ unsigned h[kMaxClasses];
  __shared__ double total;
  const int tid = threadIdx.x;
  if (tid < kMaxClasses) h[tid] = 0;
  __syncthreads();
  bool bad = false;
  for (int64_t r = tid; r < b; r += blockDim.x) {
    const int lab = labels[r];
    if ((unsigned)lab < (unsigned)C) atomicAdd(&h[lab], 1u);
    else bad = true;
  }
  if (bad) atomicOr(dflag, kFlagBadLabel);
  __syncthreads();
  if (tid < C) cnt[tid] += (double)h[tid];
  __syncthreads();
  if (tid == 0) {
    double n = 0.0;
    for (int c = 0; c < C; ++c) n += cnt[c];
    total = n;
  }
  __syncthreads();
  if (tid < C) pi[tid] = total > 0.0 ? (float)(cnt[tid] / total) : 0.f;
}

// Per column: class sums += this minibatch's rows (skipped when b = 0), then the means,
// mu_c - mu and the class means used for centring. grid: ceil(d / 256) blocks, one
// column per thread; dynamic shared memory C x 256 floats.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_lda_stats(const T* __restrict__ X, const float* __restrict__ rs,
                                                        const int32_t* __restrict__ labels,
                                                        int64_t b, int64_t d, int C, double* __restrict__ sum,
                                                        const double* __restrict__ cnt, float* __restrict__ mean,
                                                        float* __restrict__ M) {
  extern __shared__ float acc[];  // [C][kThreads]
  __shared__ int labs[kThreads];
  const int tid = threadIdx.x;
  const int64_t col = (int64_t)blockIdx.x * kThreads + tid;
  for (int c = 0; c < C; ++c) acc[c * kThreads + tid] = 0.f;
  for (int64_t r0 = 0; r0 < b; r0 += kThreads) {
    __syncthreads();
    const int64_t rr = r0 + tid;
    const int lab = rr < b ? labels[rr] : -1;
    labs[tid] = (unsigned)lab < (unsigned)C ? lab : -1;  // bad labels are flagged by k_lda_counts
    __syncthreads();
    const int nr = (int)min((int64_t)kThreads, b - r0);
    if (col < d) {
      for (int q0 = 0; q0 < nr; q0 += 8) {
        float x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int64_t row = r0 + q0 + q;
          x[q] = (q0 + q < nr) ? load_x(X, row * d + col) * (rs ? rs[row] : 1.f) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int lab2 = (q0 + q < nr) ? labs[q0 + q] : -1;
          if (lab2 >= 0) acc[lab2 * kThreads + tid] += x[q];
        }
      }
    }
  }
  if (col >= d) return;
  double n = 0.0, tot = 0.0;
  for (int c = 0; c < C; ++c) {
    const double sc = sum[c * d + col] + (double)acc[c * kThreads + tid];
    sum[c * d + col] = sc;
    tot += sc;
    n += cnt[c];
  }
  const double mu = n > 0.0 ? tot / n : 0.0;
  for (int c = 0; c < C; ++c) {
    const double nc = cnt[c];
    const double mc = nc > 0.0 ? sum[c * d + col] / nc : 0.0;
    mean[c * d + col] = (float)mc;
    M[c * d + col] = nc > 0.0 ? (float)(mc - mu) : 0.f;
  }
}

// W[c][i] += sum over this block's columns of M[c][col] V[col][i] (W zeroed before).
__global__ void __launch_bounds__(kThreads) k_lda_w(const float* __restrict__ M, const float* __restrict__ V,
                                                    int64_t d, int C, int k, float* __restrict__ W) {
  constexpr int TC = 32;
  __shared__ float Ms[kMaxClasses][TC + 1];
  __shared__ float Vs[TC][64 + 1];
  const int tid = threadIdx.x;
  const int nout = C * k;
  float acc[(kMaxClasses * 64) / kThreads];
#pragma unroll
  for (int q = 0; q < (kMaxClasses * 64) / kThreads; ++q) acc[q] = 0.f;
  for (int64_t c0 = (int64_t)blockIdx.x * TC; c0 < d; c0 += (int64_t)gridDim.x * TC) {
    for (int e = tid; e < C * TC; e += kThreads) {
      const int c = e / TC, cc = e % TC;
      Ms[c][cc] = c0 + cc < d ? M[c * d + c0 + cc] : 0.f;
    }
    for (int e = tid; e < TC * k; e += kThreads) {
      const int cc = e / k, i = e % k;
      Vs[cc][i] = c0 + cc < d ? V[(c0 + cc) * k + i] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (kMaxClasses * 64) / kThreads; ++q) {
      const int p = tid + q * kThreads;
      if (p < nout) {
        const int c = p / k, i = p % k;
        float s = 0.f;
        for (int cc = 0; cc < TC; ++cc) s = fmaf(Ms[c][cc], Vs[cc][i], s);
        acc[q] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < (kMaxClasses * 64) / kThreads; ++q) {
    const int p = tid + q * kThreads;
    if (p < nout) atomicAdd(&W[p], acc[q]);
  }
}

// AV[col][i] = sum_c M[c][col] pi_c W[c][i].
__global__ void __launch_bounds__(kThreads) k_lda_av(const float* __restrict__ M, const float* __restrict__ pi,
                                                     const float* __restrict__ W, int64_t d, int C, int k,
                                                     float* __restrict__ AV) {
  __shared__ float PW[kMaxClasses * 64];
  for (int e = threadIdx.x; e < C * k; e += kThreads) PW[e] = pi[e / k] * W[e];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < d * k; e += (int64_t)gridDim.x * kThreads) {
    const int64_t col = e / k;
    const int i = (int)(e % k);
    float s = 0.f;
    for (int c = 0; c < C; ++c) s = fmaf(M[c * d + col], PW[c * k + i], s);
    AV[e] = s;
  }
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
  const size_t smem = (size_t)C * kThreads * sizeof(float);
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

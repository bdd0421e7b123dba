// Learned warm start: the sketch of the first minibatch and a per-row MLP that maps
// sketch rows to rows of the initial players V0, with hand-written forward, backward
// and Adam kernels. Not in the paper (which starts from random players, Alg. 2).
//
// Sketch: S = Z^T (Z Omega) / n, Z = [X Y] (n x d), Omega (d x m) fixed Gaussian, then
// every column of S divided by its root mean square over the d rows.
// Network on every row s of S: h1 = relu(W1 s + b1), h2 = relu(W2 h1 + b2),
// o = W3 h2 + b3, hidden width 64, m <= 32 inputs, k <= 32 outputs. Weights are used
// in BF16 (FP32 master copies are updated by Adam), all accumulation is FP32.
// Loss per instance with target V (the plain solver's solution):
// sum_i (1 - (o_i . v_i)^2 / (|o_i|^2 |v_i|^2)), averaged over the instances.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <type_traits>
#include <vector>

#include "generic_tiles.cuh"
#include "internal.h"

namespace sgep {
namespace {

constexpr int kH = 64;       // hidden width
constexpr int kMaxIn = 32;   // sketch width m
constexpr int kMaxOut = 32;  // players k
constexpr int kThreads = 256;

// ---- sketch ---------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_sk_project(const T* __restrict__ X, const T* __restrict__ Y, int64_t n,
                                                         int64_t dx, int64_t dy, const float* __restrict__ om, int m,
                                                         int64_t chunk, int nchunk_x, float* __restrict__ PQ,
                                                         int* dflag) {
  extern __shared__ __align__(16) float smem[];
  const gt::Centring none{nullptr, nullptr, 0, dflag};
  gt::project_tile(X, Y, n, dx, dy, om, m, chunk, nchunk_x, PQ, none, nullptr, nullptr, blockIdx.x, blockIdx.y,
                   smem);
}

// T = P + Q into the first half of every PQ row.
__global__ void k_sk_combine(float* __restrict__ PQ, int64_t n, int m) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / m;
    const int j = (int)(e % m);
    PQ[r * 2 * m + j] += PQ[r * 2 * m + m + j];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_sk_back(const T* __restrict__ X, const T* __restrict__ Y, int64_t n,
                                                      int64_t dx, int64_t dy, const float* __restrict__ PQ, int m,
                                                      int nblk_x, int64_t rows_per_split, float inv_n,
                                                      float* __restrict__ out, int* dflag) {
  extern __shared__ __align__(16) float smem[];
  const gt::Centring none{nullptr, nullptr, 0, dflag};
  // kind PCA: every column block reads the first half of the PQ rows (T)
  gt::backproject_tile(X, Y, n, dx, dy, n, SGEP_PCA, 0, PQ, m, nblk_x, rows_per_split, inv_n, 0.f, out, nullptr, none,
                       nullptr, nullptr, blockIdx.x, blockIdx.y, smem);
}

// Column root mean squares (one block per column), then S /= rms.
__global__ void k_sk_rms(const float* __restrict__ S, int64_t d, int m, float* __restrict__ rms) {
  __shared__ double red[kThreads];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < d; r += blockDim.x) {
    const double v = S[r * m + j];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) rms[j] = (float)sqrt(red[0] / (double)d);
}

__global__ void k_sk_scale(float* __restrict__ S, int64_t d, int m, const float* __restrict__ rms) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d * m; e += (int64_t)gridDim.x * blockDim.x) {
    const float r = rms[e % m];
    S[e] = r > 0.f ? S[e] / r : 0.f;
  }
}

// ---- network ----------------------------------------------------------------------
// Parameter vector layout (FP32): W1 (H x m) | b1 (H) | W2 (H x H) | b2 (H) | W3 (k x H) | b3 (k).
struct Shape {
  int m, k;
  __host__ __device__ int o_b1() const { return kH * m; }
  __host__ __device__ int o_w2() const { return o_b1() + kH; }
  __host__ __device__ int o_b2() const { return o_w2() + kH * kH; }
  __host__ __device__ int o_w3() const { return o_b2() + kH; }
  __host__ __device__ int o_b3() const { return o_w3() + k * kH; }
  __host__ __device__ int count() const { return o_b3() + k; }
};

// Shared copies of the (BF16-valued) weights, laid out for conflict-free reads:
// W1T[q][u], W2T[q][u] (forward, lane = unit u), W2[u][q] (backward, lane = input q),
// W3T[q][i] (forward, lane = output i), W3[i][u] (backward, lane = unit u).
struct SmemW {
  float* w1t;  // m x H
  float* w2t;  // H x H
  float* w2;   // H x H
  float* w3t;  // H x k
  float* w3;   // k x H
  float* b;    // b1 (H) | b2 (H) | b3 (k)
};

__device__ SmemW load_weights(const float* __restrict__ P, Shape sh, float* smem) {
  SmemW w;
  w.w1t = smem;
  w.w2t = w.w1t + kMaxIn * kH;
  w.w2 = w.w2t + kH * kH;
  w.w3t = w.w2 + kH * kH;
  w.w3 = w.w3t + kH * kMaxOut;
  w.b = w.w3 + kMaxOut * kH;
  for (int e = threadIdx.x; e < kH * sh.m; e += blockDim.x) {
    const int u = e / sh.m, q = e % sh.m;
    w.w1t[q * kH + u] = P[e];
  }
  for (int e = threadIdx.x; e < kH * kH; e += blockDim.x) {
    const int u = e / kH, q = e % kH;
    const float v = P[sh.o_w2() + e];
    w.w2t[q * kH + u] = v;
    w.w2[u * kH + q] = v;
  }
  for (int e = threadIdx.x; e < sh.k * kH; e += blockDim.x) {
    const int i = e / kH, u = e % kH;
    const float v = P[sh.o_w3() + e];
    w.w3t[u * kMaxOut + i] = v;
    w.w3[i * kH + u] = v;
  }
  for (int e = threadIdx.x; e < kH; e += blockDim.x) {
    w.b[e] = P[sh.o_b1() + e];
    w.b[kH + e] = P[sh.o_b2() + e];
  }
  for (int e = threadIdx.x; e < sh.k; e += blockDim.x) w.b[2 * kH + e] = P[sh.o_b3() + e];
  __syncthreads();
  return w;
}
constexpr int kSmemW = kMaxIn * kH + 2 * kH * kH + 2 * kH * kMaxOut + 2 * kH + kMaxOut;

// Forward, one warp per row: lane holds hidden units lane and lane + 32, output lane.
// Saves the pre-activations z1, z2 (rows x H) for the backward pass when non-null.
__global__ void __launch_bounds__(kThreads) k_mlp_forward(const float* __restrict__ Pw, Shape sh,
                                                          const float* __restrict__ S, int64_t rows,
                                                          float* __restrict__ O, float* __restrict__ Z1,
                                                          float* __restrict__ Z2) {
  extern __shared__ __align__(16) float smem[];
  const SmemW w = load_weights(Pw, sh, smem);
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows; r += nwarps) {
    const float s = lane < sh.m ? S[r * sh.m + lane] : 0.f;
    float z1a = w.b[lane], z1b = w.b[lane + 32];
    for (int q = 0; q < sh.m; ++q) {
      const float sq = __shfl_sync(0xffffffffu, s, q);
      z1a = fmaf(w.w1t[q * kH + lane], sq, z1a);
      z1b = fmaf(w.w1t[q * kH + lane + 32], sq, z1b);
    }
    const float h1a = fmaxf(z1a, 0.f), h1b = fmaxf(z1b, 0.f);
    float z2a = w.b[kH + lane], z2b = w.b[kH + lane + 32];
    for (int q = 0; q < 32; ++q) {
      const float x0 = __shfl_sync(0xffffffffu, h1a, q), x1 = __shfl_sync(0xffffffffu, h1b, q);
      z2a = fmaf(w.w2t[q * kH + lane], x0, z2a);
      z2a = fmaf(w.w2t[(q + 32) * kH + lane], x1, z2a);
      z2b = fmaf(w.w2t[q * kH + lane + 32], x0, z2b);
      z2b = fmaf(w.w2t[(q + 32) * kH + lane + 32], x1, z2b);
    }
    const float h2a = fmaxf(z2a, 0.f), h2b = fmaxf(z2b, 0.f);
    float o = lane < sh.k ? w.b[2 * kH + lane] : 0.f;
    for (int q = 0; q < 32; ++q) {
      const float x0 = __shfl_sync(0xffffffffu, h2a, q), x1 = __shfl_sync(0xffffffffu, h2b, q);
      if (lane < sh.k) {
        o = fmaf(w.w3t[q * kMaxOut + lane], x0, o);
        o = fmaf(w.w3t[(q + 32) * kMaxOut + lane], x1, o);
      }
    }
    if (lane < sh.k) O[r * sh.k + lane] = o;
    if (Z1) {
      Z1[r * kH + lane] = z1a;
      Z1[r * kH + lane + 32] = z1b;
      Z2[r * kH + lane] = z2a;
      Z2[r * kH + lane + 32] = z2b;
    }
  }
}

// Per-instance column sums c = o . v, a = |o|^2, t = |v|^2 (one block per instance) and
// the instance's loss into loss[inst].
__global__ void __launch_bounds__(kThreads) k_mlp_colstats(const float* __restrict__ O, const float* __restrict__ V,
                                                           const int64_t* __restrict__ seg, int k,
                                                           float* __restrict__ stats, double* __restrict__ loss) {
  __shared__ float red[3][kThreads];
  const int inst = blockIdx.x;
  const int64_t r0 = seg[inst], r1 = seg[inst + 1];
  const int tid = threadIdx.x;
  const int per = kThreads / k;  // rows handled together
  const int i = tid % k, rl = tid / k;
  float c = 0.f, a = 0.f, t = 0.f;
  if (rl < per)
    for (int64_t r = r0 + rl; r < r1; r += per) {
      const float o = O[r * k + i], v = V[r * k + i];
      c = fmaf(o, v, c);
      a = fmaf(o, o, a);
      t = fmaf(v, v, t);
    }
  red[0][tid] = rl < per ? c : 0.f;
  red[1][tid] = rl < per ? a : 0.f;
  red[2][tid] = rl < per ? t : 0.f;
  __syncthreads();
  if (tid < k) {
    float sc = 0.f, sa = 0.f, st = 0.f;
    for (int q = 0; q < per; ++q) {
      sc += red[0][q * k + tid];
      sa += red[1][q * k + tid];
      st += red[2][q * k + tid];
    }
    stats[(size_t)inst * 3 * k + tid] = sc;
    stats[(size_t)inst * 3 * k + k + tid] = sa;
    stats[(size_t)inst * 3 * k + 2 * k + tid] = st;
    red[0][tid] = 1.f - sc * sc / (sa * st);
  }
  __syncthreads();
  if (tid == 0) {
    double l = 0.0;
    for (int q = 0; q < k; ++q) l += red[0][q];
    loss[inst] = l;
  }
}

// Backward through the network, one warp per row: dO from the loss, then dH2 and dH1
// (rows x H, masked by the ReLUs), stored for the weight gradients.
__global__ void __launch_bounds__(kThreads) k_mlp_backward(const float* __restrict__ Pw, Shape sh,
                                                           const float* __restrict__ O, const float* __restrict__ V,
                                                           const float* __restrict__ Z1, const float* __restrict__ Z2,
                                                           const int64_t* __restrict__ seg, int n_inst,
                                                           const float* __restrict__ stats, float inv_n,
                                                           float* __restrict__ dO, float* __restrict__ dH2,
                                                           float* __restrict__ dH1) {
  extern __shared__ __align__(16) float smem[];
  const SmemW w = load_weights(Pw, sh, smem);
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t rows = seg[n_inst];
  for (int64_t r = warp; r < rows; r += nwarps) {
    int lo = 0, hi = n_inst - 1;  // instance of row r
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg[mid] <= r) lo = mid;
      else hi = mid - 1;
    }
    float g = 0.f;
    if (lane < sh.k) {
      const float* st = stats + (size_t)lo * 3 * sh.k;
      const float c = st[lane], a = st[sh.k + lane], t = st[2 * sh.k + lane];
      const float o = O[r * sh.k + lane], v = V[r * sh.k + lane];
      g = (2.f * c / (a * t)) * (c * o / a - v) * inv_n;
      dO[r * sh.k + lane] = g;
    }
    float d2a = 0.f, d2b = 0.f;
    for (int i = 0; i < sh.k; ++i) {
      const float gi = __shfl_sync(0xffffffffu, g, i);
      d2a = fmaf(w.w3[i * kH + lane], gi, d2a);
      d2b = fmaf(w.w3[i * kH + lane + 32], gi, d2b);
    }
    d2a = Z2[r * kH + lane] > 0.f ? d2a : 0.f;
    d2b = Z2[r * kH + lane + 32] > 0.f ? d2b : 0.f;
    dH2[r * kH + lane] = d2a;
    dH2[r * kH + lane + 32] = d2b;
    float d1a = 0.f, d1b = 0.f;
    for (int q = 0; q < 32; ++q) {
      const float x0 = __shfl_sync(0xffffffffu, d2a, q), x1 = __shfl_sync(0xffffffffu, d2b, q);
      d1a = fmaf(w.w2[q * kH + lane], x0, d1a);
      d1a = fmaf(w.w2[(q + 32) * kH + lane], x1, d1a);
      d1b = fmaf(w.w2[q * kH + lane + 32], x0, d1b);
      d1b = fmaf(w.w2[(q + 32) * kH + lane + 32], x1, d1b);
    }
    d1a = Z1[r * kH + lane] > 0.f ? d1a : 0.f;
    d1b = Z1[r * kH + lane + 32] > 0.f ? d1b : 0.f;
    dH1[r * kH + lane] = d1a;
    dH1[r * kH + lane + 32] = d1b;
  }
}

// Weight gradients as reductions over rows, per block partials (no atomics):
//   dW1 = dH1^T S, db1 = sum dH1, dW2 = dH2^T relu(Z1), db2 = sum dH2, dW3 = dO^T relu(Z2), db3 = sum dO.
// Rows are staged 32 at a time; thread j accumulates parameter entries j, j + 256, ...
__global__ void __launch_bounds__(kThreads) k_mlp_wgrad(Shape sh, const float* __restrict__ S,
                                                        const float* __restrict__ Z1, const float* __restrict__ Z2,
                                                        const float* __restrict__ dO, const float* __restrict__ dH2,
                                                        const float* __restrict__ dH1, int64_t rows,
                                                        float* __restrict__ part) {
  constexpr int R = 32;
  constexpr int kPer = (kH * kMaxIn + kH + kH * kH + kH + kMaxOut * kH + kMaxOut + kThreads - 1) / kThreads;
  __shared__ float s_s[R][kMaxIn + 1], s_h1[R][kH + 1], s_h2[R][kH + 1], s_d1[R][kH + 1], s_d2[R][kH + 1],
      s_o[R][kMaxOut + 1];
  const int tid = threadIdx.x;
  const int P = sh.count();
  float acc[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) acc[q] = 0.f;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < rows; r0 += (int64_t)gridDim.x * R) {
    const int nr = (int)min((int64_t)R, rows - r0);
    for (int e = tid; e < R * kH; e += kThreads) {
      const int rr = e / kH, u = e % kH;
      const bool ok = rr < nr;
      const int64_t g = (r0 + rr) * kH + u;
      s_h1[rr][u] = ok ? fmaxf(Z1[g], 0.f) : 0.f;
      s_h2[rr][u] = ok ? fmaxf(Z2[g], 0.f) : 0.f;
      s_d1[rr][u] = ok ? dH1[g] : 0.f;
      s_d2[rr][u] = ok ? dH2[g] : 0.f;
    }
    for (int e = tid; e < R * sh.m; e += kThreads) {
      const int rr = e / sh.m, q = e % sh.m;
      s_s[rr][q] = rr < nr ? S[(r0 + rr) * sh.m + q] : 0.f;
    }
    for (int e = tid; e < R * sh.k; e += kThreads) {
      const int rr = e / sh.k, i = e % sh.k;
      s_o[rr][i] = rr < nr ? dO[(r0 + rr) * sh.k + i] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int p = tid + q * kThreads;
      if (p >= P) continue;
      float s = 0.f;
      if (p < sh.o_b1()) {
        const int u = p / sh.m, j = p % sh.m;
        for (int rr = 0; rr < nr; ++rr) s = fmaf(s_d1[rr][u], s_s[rr][j], s);
      } else if (p < sh.o_w2()) {
        const int u = p - sh.o_b1();
        for (int rr = 0; rr < nr; ++rr) s += s_d1[rr][u];
      } else if (p < sh.o_b2()) {
        const int u = (p - sh.o_w2()) / kH, j = (p - sh.o_w2()) % kH;
        for (int rr = 0; rr < nr; ++rr) s = fmaf(s_d2[rr][u], s_h1[rr][j], s);
      } else if (p < sh.o_w3()) {
        const int u = p - sh.o_b2();
        for (int rr = 0; rr < nr; ++rr) s += s_d2[rr][u];
      } else if (p < sh.o_b3()) {
        const int i = (p - sh.o_w3()) / kH, j = (p - sh.o_w3()) % kH;
        for (int rr = 0; rr < nr; ++rr) s = fmaf(s_o[rr][i], s_h2[rr][j], s);
      } else {
        const int i = p - sh.o_b3();
        for (int rr = 0; rr < nr; ++rr) s += s_o[rr][i];
      }
      acc[q] += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int p = tid + q * kThreads;
    if (p < P) part[(size_t)blockIdx.x * P + p] = acc[q];
  }
}

__global__ void k_mlp_sum_parts(const float* __restrict__ part, int nparts, int P, float* __restrict__ grad) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int j = 0; j < nparts; ++j) s += part[(size_t)j * P + p];
    grad[p] = s;
  }
}

// Adam on the FP32 master parameters; the working copy rounds the weights (not the
// biases) to BF16.
__global__ void k_mlp_adam(float* __restrict__ master, float* __restrict__ work, float* __restrict__ mom,
                           float* __restrict__ var, const float* __restrict__ grad, Shape sh, float lr, float b1c,
                           float b2c) {
  const int P = sh.count();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const float g = grad[p];
    const float m = 0.9f * mom[p] + 0.1f * g;
    const float v = 0.999f * var[p] + 0.001f * g * g;
    mom[p] = m;
    var[p] = v;
    const float x = master[p] - lr * (m / b1c) / (sqrtf(v / b2c) + 1e-8f);
    master[p] = x;
    const bool bias = (p >= sh.o_b1() && p < sh.o_w2()) || (p >= sh.o_b2() && p < sh.o_w3()) || p >= sh.o_b3();
    work[p] = bias ? x : __bfloat162float(__float2bfloat16(x));
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side

struct MlpCtx {
  Shape sh{16, 16};
  float *master = nullptr, *work = nullptr, *mom = nullptr, *var = nullptr, *grad = nullptr;
  int64_t adam_t = 0;
  // activations and gradients for up to `cap` rows
  int64_t cap = 0;
  float *O = nullptr, *Z1 = nullptr, *Z2 = nullptr, *dO = nullptr, *dH1 = nullptr, *dH2 = nullptr;
  float* part = nullptr;
  int nparts = 0;
  float* stats = nullptr;
  double* loss = nullptr;
  int64_t* seg = nullptr;
  int inst_cap = 0;
  int num_sms = 0;
};

static void mlp_free_rows(MlpCtx& M) {
  cudaFree(M.O);
  cudaFree(M.Z1);
  cudaFree(M.Z2);
  cudaFree(M.dO);
  cudaFree(M.dH1);
  cudaFree(M.dH2);
  M.O = M.Z1 = M.Z2 = M.dO = M.dH1 = M.dH2 = nullptr;
  M.cap = 0;
}

void mlp_free(MlpCtx* M) {
  if (!M) return;
  cudaDeviceSynchronize();
  mlp_free_rows(*M);
  cudaFree(M->master);
  cudaFree(M->work);
  cudaFree(M->mom);
  cudaFree(M->var);
  cudaFree(M->grad);
  cudaFree(M->part);
  cudaFree(M->stats);
  cudaFree(M->loss);
  cudaFree(M->seg);
  delete M;
}

static int mlp_rows(MlpCtx& M, int64_t rows) {
  if (rows <= M.cap) return SGEP_OK;
  mlp_free_rows(M);
  const size_t r = (size_t)rows;
  SGEP_CUDA_TRY(cudaMalloc((void**)&M.O, r * kMaxOut * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&M.Z1, r * kH * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&M.Z2, r * kH * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&M.dO, r * kMaxOut * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&M.dH1, r * kH * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&M.dH2, r * kH * sizeof(float)));
  M.cap = rows;
  return SGEP_OK;
}

static int mlp_insts(MlpCtx& M, int n) {
  if (n <= M.inst_cap) return SGEP_OK;
  cudaFree(M.stats);
  cudaFree(M.loss);
  cudaFree(M.seg);
  SGEP_CUDA_TRY(cudaMalloc((void**)&M.stats, (size_t)n * 3 * kMaxOut * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&M.loss, (size_t)n * sizeof(double)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&M.seg, (size_t)(n + 1) * sizeof(int64_t)));
  M.inst_cap = n;
  return SGEP_OK;
}

int mlp_create(int m, int k, uint64_t seed, MlpCtx** out) {
  auto* M = new (std::nothrow) MlpCtx();
  if (!M) return SGEP_ENOMEM;
  M->sh = Shape{m, k};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&M->num_sms, cudaDevAttrMultiProcessorCount, dev);
  const int P = M->sh.count();
  M->nparts = std::max(1, 2 * M->num_sms);
  int rc = SGEP_OK;
  auto al = [&](float** p, size_t n) {
    if (!rc && cudaMalloc((void**)p, n * sizeof(float)) != cudaSuccess) rc = SGEP_ENOMEM;
  };
  al(&M->master, P);
  al(&M->work, P);
  al(&M->mom, P);
  al(&M->var, P);
  al(&M->grad, P);
  al(&M->part, (size_t)M->nparts * P);
  if (rc) {
    mlp_free(M);
    return rc;
  }
  // He-style initialisation from a seeded host generator
  std::mt19937_64 gen(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::vector<float> h(P, 0.f);
  const Shape& sh = M->sh;
  for (int e = 0; e < kH * m; ++e) h[e] = (float)(nd(gen) * std::sqrt(2.0 / m));
  for (int e = 0; e < kH * kH; ++e) h[sh.o_w2() + e] = (float)(nd(gen) * std::sqrt(2.0 / kH));
  for (int e = 0; e < k * kH; ++e) h[sh.o_w3() + e] = (float)(nd(gen) * std::sqrt(1.0 / kH));
  rc = mlp_set(*M, h.data());
  if (rc) {
    mlp_free(M);
    return rc;
  }
  *out = M;
  return SGEP_OK;
}

int mlp_set(MlpCtx& M, const float* host) {
  const int P = M.sh.count();
  std::vector<float> w(host, host + P);
  for (int p = 0; p < P; ++p) {
    const Shape& sh = M.sh;
    const bool bias = (p >= sh.o_b1() && p < sh.o_w2()) || (p >= sh.o_b2() && p < sh.o_w3()) || p >= sh.o_b3();
    if (!bias) w[p] = __bfloat162float(__float2bfloat16(w[p]));
  }
  SGEP_CUDA_TRY(cudaMemcpy(M.master, host, P * sizeof(float), cudaMemcpyHostToDevice));
  SGEP_CUDA_TRY(cudaMemcpy(M.work, w.data(), P * sizeof(float), cudaMemcpyHostToDevice));
  SGEP_CUDA_TRY(cudaMemset(M.mom, 0, P * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(M.var, 0, P * sizeof(float)));
  M.adam_t = 0;
  return SGEP_OK;
}

int mlp_get(const MlpCtx& M, float* host) {
  SGEP_CUDA_TRY(cudaMemcpy(host, M.work, M.sh.count() * sizeof(float), cudaMemcpyDeviceToHost));
  return SGEP_OK;
}

int mlp_param_count(const MlpCtx& M) { return M.sh.count(); }

static unsigned grid_for(const MlpCtx& M, int64_t rows) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, 4LL * M.num_sms));
}

int mlp_forward(MlpCtx& M, const float* S, int64_t rows, float* O, cudaStream_t s) {
  const size_t smem = (size_t)kSmemW * sizeof(float);
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_mlp_forward<<<grid_for(M, rows), kThreads, smem, s>>>(M.work, M.sh, S, rows, O, nullptr, nullptr);
  SGEP_CUDA_TRY(cudaGetLastError());
  return SGEP_OK;
}

int mlp_loss_grad(MlpCtx& M, const float* S, const float* V, const int64_t* seg_host, int n_inst, double* loss_out,
                  float* grad_host, cudaStream_t s) {
  const int64_t rows = seg_host[n_inst];
  int rc = mlp_rows(M, rows);
  if (!rc) rc = mlp_insts(M, n_inst);
  if (rc) return rc;
  SGEP_CUDA_TRY(cudaMemcpyAsync(M.seg, seg_host, (size_t)(n_inst + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  const size_t smem = (size_t)kSmemW * sizeof(float);
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_mlp_forward<<<grid_for(M, rows), kThreads, smem, s>>>(M.work, M.sh, S, rows, M.O, M.Z1, M.Z2);
  SGEP_CUDA_TRY(cudaGetLastError());
  k_mlp_colstats<<<n_inst, kThreads, 0, s>>>(M.O, V, M.seg, M.sh.k, M.stats, M.loss);
  SGEP_CUDA_TRY(cudaGetLastError());
  k_mlp_backward<<<grid_for(M, rows), kThreads, smem, s>>>(M.work, M.sh, M.O, V, M.Z1, M.Z2, M.seg, n_inst, M.stats,
                                                           1.f / (float)n_inst, M.dO, M.dH2, M.dH1);
  SGEP_CUDA_TRY(cudaGetLastError());
  const int nb = (int)std::min<int64_t>((rows + 31) / 32, M.nparts);
  k_mlp_wgrad<<<nb, kThreads, 0, s>>>(M.sh, S, M.Z1, M.Z2, M.dO, M.dH2, M.dH1, rows, M.part);
  SGEP_CUDA_TRY(cudaGetLastError());
  k_mlp_sum_parts<<<(M.sh.count() + 255) / 256, 256, 0, s>>>(M.part, nb, M.sh.count(), M.grad);
  SGEP_CUDA_TRY(cudaGetLastError());
  std::vector<double> l(n_inst);
  SGEP_CUDA_TRY(cudaMemcpyAsync(l.data(), M.loss, n_inst * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (grad_host)
    SGEP_CUDA_TRY(cudaMemcpyAsync(grad_host, M.grad, M.sh.count() * sizeof(float), cudaMemcpyDeviceToHost, s));
  SGEP_CUDA_TRY(cudaStreamSynchronize(s));
  if (loss_out) {
    double t = 0.0;
    for (double x : l) t += x;
    *loss_out = t / n_inst;
  }
  return SGEP_OK;
}

int mlp_adam(MlpCtx& M, float lr, cudaStream_t s) {
  M.adam_t += 1;
  const float b1c = 1.f - (float)std::pow(0.9, (double)M.adam_t);
  const float b2c = 1.f - (float)std::pow(0.999, (double)M.adam_t);
  k_mlp_adam<<<(M.sh.count() + 255) / 256, 256, 0, s>>>(M.master, M.work, M.mom, M.var, M.grad, M.sh, lr, b1c, b2c);
  SGEP_CUDA_TRY(cudaGetLastError());
  return SGEP_OK;
}

int sketch_rows(const void* X, const void* Y, int dtype, int64_t n, int64_t dx, int64_t dy, const float* om, int m,
                float* out, int num_sms, int* dflag, cudaStream_t s) {
  const int64_t d = dx + dy;
  float* PQ = nullptr;
  float* rms = nullptr;
  // stream-ordered allocations: no device-wide synchronisation
  SGEP_CUDA_TRY(cudaMallocAsync((void**)&PQ, (size_t)n * 2 * m * sizeof(float), s));
  if (cudaMallocAsync((void**)&rms, m * sizeof(float), s) != cudaSuccess) {
    cudaFreeAsync(PQ, s);
    return SGEP_ENOMEM;
  }
  int rc = SGEP_OK;
  cudaMemsetAsync(PQ, 0, (size_t)n * 2 * m * sizeof(float), s);
  cudaMemsetAsync(out, 0, (size_t)d * m * sizeof(float), s);
  const int64_t row_tiles = (n + gt::kProjRows - 1) / gt::kProjRows;
  int64_t chunk = 1024;
  while (chunk > 64 && row_tiles * ((d + chunk - 1) / chunk) < 2LL * num_sms) chunk /= 2;
  const int nchunk_x = (int)((dx + chunk - 1) / chunk), nchunk_y = dy ? (int)((dy + chunk - 1) / chunk) : 0;
  const int nblk_x = (int)((dx + 63) / 64), nblk_y = dy ? (int)((dy + 63) / 64) : 0;
  int splits = (int)std::max<int64_t>(1, std::min<int64_t>((2LL * num_sms + nblk_x + nblk_y - 1) / (nblk_x + nblk_y),
                                                           (n + 31) / 32));
  int64_t rps = ((n + splits - 1) / splits + 31) / 32 * 32;
  splits = (int)((n + rps - 1) / rps);
  const size_t sp = gt::kProjectSmem * sizeof(float), sb = gt::kBackprojectSmem * sizeof(float);
  auto launch = [&](auto tag) {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    cudaFuncSetAttribute(k_sk_project<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp);
    cudaFuncSetAttribute(k_sk_back<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    k_sk_project<T><<<dim3((unsigned)row_tiles, (unsigned)(nchunk_x + nchunk_y)), kThreads, sp, s>>>(
        (const T*)X, (const T*)Y, n, dx, dy, om, m, chunk, nchunk_x, PQ, dflag);
    k_sk_combine<<<(unsigned)std::min<int64_t>((n * m + 255) / 256, 4LL * num_sms), 256, 0, s>>>(PQ, n, m);
    k_sk_back<T><<<dim3((unsigned)(nblk_x + nblk_y), (unsigned)splits), kThreads, sb, s>>>(
        (const T*)X, (const T*)Y, n, dx, dy, PQ, m, nblk_x, rps, 1.f / (float)n, out, dflag);
  };
  if (dtype == SGEP_BF16) launch(static_cast<const __nv_bfloat16*>(nullptr));
  else launch(static_cast<const float*>(nullptr));
  k_sk_rms<<<m, kThreads, 0, s>>>(out, d, m, rms);
  k_sk_scale<<<(unsigned)std::min<int64_t>((d * m + 255) / 256, 4LL * num_sms), 256, 0, s>>>(out, d, m, rms);
  if (cudaGetLastError() != cudaSuccess) rc = SGEP_ECUDA;
  cudaFreeAsync(PQ, s);
  cudaFreeAsync(rms, s);
  if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = SGEP_ECUDA;
  return rc;
}

}  // namespace sgep

// ---------------------------------------------------------------------------
// C ABI (declared in include/sgep.h)

struct sgep_mlp_ctx {
  sgep::MlpCtx* impl;
};

namespace {
int warm_fail(int status, const char* msg) {
  sgep::set_error(msg);
  return status;
}
}  // namespace

extern "C" {

int sgep_sketch(const void* X, const void* Y, int dtype, int64_t n, int64_t d_x, int64_t d_y, const float* omega,
                int m, float* out, void* stream) {
  if (!X || !omega || !out || (d_y > 0 && !Y)) return warm_fail(SGEP_EINVAL, "NULL argument");
  if (n < 1 || d_x < 1 || d_y < 0 || m < 1 || m > sgep::kMaxIn) return warm_fail(SGEP_EINVAL, "bad shape");
  if (dtype != SGEP_F32 && dtype != SGEP_BF16) return warm_fail(SGEP_EINVAL, "sketch rows are FP32 or BF16");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return warm_fail(SGEP_ECUDA, "no CUDA device");
  int* flag = nullptr;  // the sketch passes no labels, so nothing is ever flagged here
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMallocAsync((void**)&flag, sizeof(int), s) != cudaSuccess) return warm_fail(SGEP_ENOMEM, "cudaMallocAsync");
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  int rc = sgep::sketch_rows(X, d_y > 0 ? Y : nullptr, dtype, n, d_x, d_y, omega, m, out, sms, flag, s);
  cudaFreeAsync(flag, s);
  cudaStreamSynchronize(s);
  return rc ? warm_fail(rc, "sketch failed") : SGEP_OK;
}

int sgep_mlp_create(int in_dim, int out_dim, uint64_t seed, sgep_mlp_t* out) {
  if (!out) return warm_fail(SGEP_EINVAL, "out is NULL");
  *out = nullptr;
  if (in_dim < 1 || in_dim > sgep::kMaxIn || out_dim < 1 || out_dim > sgep::kMaxOut)
    return warm_fail(SGEP_EINVAL, "in_dim and out_dim must be in 1..32");
  auto* w = new (std::nothrow) sgep_mlp_ctx();
  if (!w) return warm_fail(SGEP_ENOMEM, "host allocation failed");
  int rc = sgep::mlp_create(in_dim, out_dim, seed, &w->impl);
  if (rc) {
    delete w;
    return warm_fail(rc, "network allocation failed");
  }
  *out = w;
  return SGEP_OK;
}

int sgep_mlp_destroy(sgep_mlp_t m) {
  if (!m) return SGEP_OK;
  sgep::mlp_free(m->impl);
  delete m;
  return SGEP_OK;
}

int sgep_mlp_param_count(sgep_mlp_t m) { return m ? sgep::mlp_param_count(*m->impl) : -1; }

int sgep_mlp_get_params(sgep_mlp_t m, float* host) {
  if (!m || !host) return warm_fail(SGEP_EINVAL, "NULL argument");
  return sgep::mlp_get(*m->impl, host);
}

int sgep_mlp_set_params(sgep_mlp_t m, const float* host) {
  if (!m || !host) return warm_fail(SGEP_EINVAL, "NULL argument");
  return sgep::mlp_set(*m->impl, host);
}

int sgep_mlp_forward(sgep_mlp_t m, const float* S, int64_t rows, float* out, void* stream) {
  if (!m || !S || !out || rows < 1) return warm_fail(SGEP_EINVAL, "bad argument");
  return sgep::mlp_forward(*m->impl, S, rows, out, (cudaStream_t)stream);
}

int sgep_mlp_loss_grad(sgep_mlp_t m, const float* S, const float* V, const int64_t* seg, int n_inst, double* loss,
                       float* grad_host, void* stream) {
  if (!m || !S || !V || !seg || n_inst < 1) return warm_fail(SGEP_EINVAL, "bad argument");
  for (int i = 0; i < n_inst; ++i)
    if (seg[i + 1] <= seg[i]) return warm_fail(SGEP_EINVAL, "instance row ranges must be non-empty and increasing");
  if (seg[0] != 0) return warm_fail(SGEP_EINVAL, "seg[0] must be 0");
  return sgep::mlp_loss_grad(*m->impl, S, V, seg, n_inst, loss, grad_host, (cudaStream_t)stream);
}

int sgep_mlp_adam_step(sgep_mlp_t m, float lr, void* stream) {
  if (!m || !(lr > 0.f)) return warm_fail(SGEP_EINVAL, "bad argument");
  return sgep::mlp_adam(*m->impl, lr, (cudaStream_t)stream);
}

}  // extern "C"

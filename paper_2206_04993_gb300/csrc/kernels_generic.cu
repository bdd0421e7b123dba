// Generic multi-kernel SIMT path of the gamma-EigenGame step (Alg. 2, M = 1).
//
// One step is five kernels:
//   k_project      P = X V_x, Q = Y V_y for every row            (Alg. 2: A_t v, B_t v, first factor)
//   k_backproject  A_t V, B_t V = X^T [Q|P] / n                   (Alg. 2: mat-vecs, second factor)
//   k_gram         a_ij = v_i^T A_t v_j, b_i = v_i^T B_t v_i, G_ij = <v_i, [Bv]_j>
//   k_update       grad (Eq. update with clipped [By]_j), v_i + eta grad_i, [Bv] step
//   k_normalize    retraction v_i / ||v_i||
// It handles every shape (any d_x, d_y, b, 1 <= k <= 64) and both element
// types; the fused cluster and tensor-core paths are checked against it.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <type_traits>

#include "eg_math.cuh"
#include "internal.h"

namespace sgep {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxK = 64;

__device__ __forceinline__ float load_elem(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_elem(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}
__device__ __forceinline__ float load_elem(const __nv_fp8_e4m3* p, int64_t i) { return static_cast<float>(p[i]); }

// Element (row, i) of a row-major matrix, times the row's scale when there is one (FP8 rows).
template <typename T>
__device__ __forceinline__ float load_row_elem(const T* p, const float* scale, int64_t row, int64_t i) {
  const float x = load_elem(p, i);
  return scale ? x * scale[row] : x;
}

// Class-mean centring of LDA rows: x - mu_{label}. A label outside [0, C) is
// flagged and the row is left uncentred (the step then reports the bad label).
struct Centring {
  const float* mean;      // C x ld class means, or null (no centring)
  const int32_t* labels;  // labels of the rows passed to the kernel
  int C;
  int* dflag;
};

__device__ __forceinline__ float centred(const Centring& cz, float x, int64_t row, int64_t ld, int64_t col) {
  if (!cz.mean) return x;
  const int lab = cz.labels[row];
  if ((unsigned)lab >= (unsigned)cz.C) {
    atomicOr(cz.dflag, kFlagBadLabel);
    return x;
  }
  return x - cz.mean[(int64_t)lab * ld + col];
}

// ---------------------------------------------------------------------------
// k_project: PQ[r, 0:k] += X[r, cols] V[cols, :], PQ[r, k:2k] += Y[r, cols] V[d_x + cols, :]
// grid.x: row tiles of 32, grid.y: column chunks (X chunks first, then Y chunks),
// each chunk `chunk` columns wide. PQ must be zeroed.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_project(const T* __restrict__ X, const T* __restrict__ Y,
                                                      int64_t n, int64_t dx, int64_t dy,
                                                      const float* __restrict__ V, int k,
                                                      int64_t chunk, int nchunk_x,
                                                      float* __restrict__ PQ, const Centring cz,
                                                      const float* __restrict__ rsx,
                                                      const float* __restrict__ rsy) {
  constexpr int BR = 32, TC = 32;
  __shared__ float Xs[BR][TC + 1];
  __shared__ float Vs[TC][kMaxK];
  const int tid = threadIdx.x;
  const int r = tid >> 3;   // 0..31
  const int g = tid & 7;    // players g, g+8, ...
  const int64_t row0 = (int64_t)blockIdx.x * BR;
  const bool isY = (int)blockIdx.y >= nchunk_x;
  const int cidx = isY ? (int)blockIdx.y - nchunk_x : (int)blockIdx.y;
  const T* Z = isY ? Y : X;
  const float* rs = isY ? rsy : rsx;
  const int64_t ld = isY ? dy : dx;
  const int64_t voff = isY ? dx : 0;
  const int64_t c_begin = (int64_t)cidx * chunk;
  const int64_t c_end = min(c_begin + chunk, ld);
  float acc[kMaxK / 8];
#pragma unroll
  for (int m = 0; m < kMaxK / 8; ++m) acc[m] = 0.f;

  for (int64_t c0 = c_begin; c0 < c_end; c0 += TC) {
    for (int e = tid; e < BR * TC; e += kThreads) {
      const int rr = e / TC, cc = e % TC;
      const int64_t row = row0 + rr, col = c0 + cc;
      Xs[rr][cc] =
          (row < n && col < c_end) ? centred(cz, load_row_elem(Z, rs, row, row * ld + col), row, ld, col) : 0.f;
    }
    for (int e = tid; e < TC * k; e += kThreads) {
      const int cc = e / k, i = e % k;
      const int64_t col = c0 + cc;
      Vs[cc][i] = (col < c_end) ? V[(voff + col) * k + i] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < TC; ++cc) {
      const float x = Xs[r][cc];
#pragma unroll
      for (int m = 0; m < kMaxK / 8; ++m) {
        const int i = g + 8 * m;
        if (i < k) acc[m] = fmaf(x, Vs[cc][i], acc[m]);
      }
    }
    __syncthreads();
  }
  const int64_t row = row0 + r;
  if (row < n) {
#pragma unroll
    for (int m = 0; m < kMaxK / 8; ++m) {
      const int i = g + 8 * m;
      if (i < k) atomicAdd(&PQ[row * 2 * k + (isY ? k : 0) + i], acc[m]);
    }
  }
}

// ---------------------------------------------------------------------------
// k_backproject: for column c of X (or Y) and player i,
//   AV[c,i] += inv_nA * sum_{r in A rows} Z[r,c] W_A[r,i]
//   BV[c,i] += inv_nB * sum_{r in B rows} Z[r,c] W_B[r,i]
// where (CCA) W_A = Q for X columns / P for Y columns and W_B = P for X / Q for Y;
// (PCA) W_A = P over every row, no BV; (PLS) W_A as CCA over every row, no BV;
// (LDA) every row passed is a B row, centred by its class mean: W_B = P, no AV.
// grid.x: column blocks of 64 (X blocks then Y blocks), grid.y: row splits.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_backproject(
    const T* __restrict__ X, const T* __restrict__ Y, int64_t b, int64_t dx, int64_t dy,
    int64_t nA, int kind, int split, const float* __restrict__ PQ, int k, int nblk_x,
    int64_t rows_per_split, float inv_nA, float inv_nB, float* __restrict__ AV,
    float* __restrict__ BV, const Centring cz, const float* __restrict__ rsx, const float* __restrict__ rsy) {
  constexpr int TR = 32, CB = 64;
  __shared__ float Zs[TR][CB];
  __shared__ float Ws[TR][2 * kMaxK];
  const int tid = threadIdx.x;
  const int cl = tid & (CB - 1);
  const int g = tid >> 6;  // players g, g+4, ...
  const bool isY = (int)blockIdx.x >= nblk_x;
  const int bidx = isY ? (int)blockIdx.x - nblk_x : (int)blockIdx.x;
  const T* Z = isY ? Y : X;
  const float* rs = isY ? rsy : rsx;
  const int64_t ld = isY ? dy : dx;
  const int64_t col = (int64_t)bidx * CB + cl;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r_end = min(r_begin + rows_per_split, b);
  // column offsets into a PQ row: own projection (P for X, Q for Y) and cross projection
  const int own = isY ? k : 0;
  const int cross = isY ? 0 : k;
  const bool cca = kind == SGEP_CCA;
  const bool lda = kind == SGEP_LDA;
  float accA[kMaxK / 4], accB[kMaxK / 4];
#pragma unroll
  for (int m = 0; m < kMaxK / 4; ++m) accA[m] = accB[m] = 0.f;

  for (int64_t r0 = r_begin; r0 < r_end; r0 += TR) {
    for (int e = tid; e < TR * CB; e += kThreads) {
      const int rr = e / CB, cc = e % CB;
      const int64_t row = r0 + rr, cg = (int64_t)bidx * CB + cc;
      Zs[rr][cc] =
          (row < r_end && cg < ld) ? centred(cz, load_row_elem(Z, rs, row, row * ld + cg), row, ld, cg) : 0.f;
    }
    for (int e = tid; e < TR * 2 * k; e += kThreads) {
      const int rr = e / (2 * k), j = e % (2 * k);
      const int64_t row = r0 + rr;
      Ws[rr][j] = (row < r_end) ? PQ[row * 2 * k + j] : 0.f;
    }
    __syncthreads();
    const int nr = (int)min((int64_t)TR, r_end - r0);
    for (int rr = 0; rr < nr; ++rr) {
      const int64_t row = r0 + rr;
      const float z = Zs[rr][cl];
      // which estimate(s) this row feeds
      bool toA, toB;
      if (lda) {
        toA = false;
        toB = true;
      } else if (!cca) {
        toA = true;
        toB = false;
      } else if (split) {
        toA = row < nA;
        toB = !toA;
      } else {
        toA = toB = true;
      }
      const int offA = (kind == SGEP_PCA) ? 0 : cross;
      if (toA) {
#pragma unroll
        for (int m = 0; m < kMaxK / 4; ++m) {
          const int i = g + 4 * m;
          if (i < k) accA[m] = fmaf(z, Ws[rr][offA + i], accA[m]);
        }
      }
      if (toB) {
#pragma unroll
        for (int m = 0; m < kMaxK / 4; ++m) {
          const int i = g + 4 * m;
          if (i < k) accB[m] = fmaf(z, Ws[rr][own + i], accB[m]);
        }
      }
    }
    __syncthreads();
  }
  if (col < ld) {
    const int64_t gc = (isY ? dx : 0) + col;
#pragma unroll
    for (int m = 0; m < kMaxK / 4; ++m) {
      const int i = g + 4 * m;
      if (i < k) {
        if (!lda) atomicAdd(&AV[gc * k + i], accA[m] * inv_nA);
        if (cca || lda) atomicAdd(&BV[gc * k + i], accB[m] * inv_nB);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// k_gram: a_ij = sum_c V[c,i] AV[c,j];  G_ij = sum_c V[c,i] S[c,j];
//         b_i = sum_c V[c,i] (B_t V)[c,i] with B_t V = BV + eps V (or (1+eps) V when B = I).
// gram layout: [a (k*k) | G (k*k) | b (k) | norms (k)]; must be zeroed.
__global__ void __launch_bounds__(kThreads) k_gram(const float* __restrict__ V,
                                                   const float* __restrict__ S,
                                                   const float* __restrict__ AV,
                                                   const float* __restrict__ BV, int64_t d, int k,
                                                   float eps_B, int b_is_identity,
                                                   float* __restrict__ gram) {
  constexpr int CR = 32;
  extern __shared__ float sm[];
  float* Vs = sm;               // CR x k
  float* As = Vs + CR * k;      // CR x k
  float* Ss = As + CR * k;      // CR x k
  const int tid = threadIdx.x;
  const int kk = k * k;
  float ga[kMaxK * kMaxK / kThreads], gg[kMaxK * kMaxK / kThreads];
#pragma unroll
  for (int q = 0; q < kMaxK * kMaxK / kThreads; ++q) ga[q] = gg[q] = 0.f;
  float gb = 0.f;
  for (int64_t c0 = (int64_t)blockIdx.x * CR; c0 < d; c0 += (int64_t)gridDim.x * CR) {
    const int nr = (int)min((int64_t)CR, d - c0);
    for (int e = tid; e < CR * k; e += kThreads) {
      const int rr = e / k;
      const bool ok = rr < nr;
      const int64_t idx = c0 * k + e;
      Vs[e] = ok ? V[idx] : 0.f;
      As[e] = ok ? AV[idx] : 0.f;
      Ss[e] = ok ? S[idx] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxK * kMaxK / kThreads; ++q) {
      const int p = tid + q * kThreads;
      if (p < kk) {
        const int i = p / k, j = p % k;
        float sa = 0.f, sg = 0.f;
        for (int rr = 0; rr < nr; ++rr) {
          const float v = Vs[rr * k + i];
          sa = fmaf(v, As[rr * k + j], sa);
          sg = fmaf(v, Ss[rr * k + j], sg);
        }
        ga[q] += sa;
        gg[q] += sg;
      }
    }
    if (tid < k) {
      float sb = 0.f;
      for (int rr = 0; rr < nr; ++rr) {
        const float v = Vs[rr * k + tid];
        const float bv = b_is_identity ? (1.f + eps_B) * v : BV[(c0 + rr) * k + tid] + eps_B * v;
        sb = fmaf(v, bv, sb);
      }
      gb += sb;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kMaxK * kMaxK / kThreads; ++q) {
    const int p = tid + q * kThreads;
    if (p < kk) {
      atomicAdd(&gram[p], ga[q]);
      atomicAdd(&gram[kk + p], gg[q]);
    }
  }
  if (tid < k) atomicAdd(&gram[2 * kk + tid], gb);
}

// k_update: grad, V' = V + eta grad (into Vtmp), S <- S + gamma (B_t V - S), norms^2 of V'.
__global__ void __launch_bounds__(kThreads) k_update(const float* __restrict__ V, float* __restrict__ S,
                                                     const float* __restrict__ AV,
                                                     const float* __restrict__ BV, float* gram,
                                                     int64_t d, int k, float eta, float gamma,
                                                     float rho, float eps_B, int b_is_identity,
                                                     float* __restrict__ Vtmp,
                                                     float* __restrict__ grad_out) {
  extern __shared__ float sm[];
  float* T = sm;                 // k*k
  float* cb = T + k * k;         // k
  float* cac = cb + k;           // k
  float* nrm = cac + k;          // k
  const int rows = max(1, kThreads / k);
  float* Ss = nrm + k;           // rows x k
  eg_coefficients(gram, k, rho, cb, cac, T);
  for (int i = threadIdx.x; i < k; i += blockDim.x) nrm[i] = 0.f;
  __syncthreads();
  const int tid = threadIdx.x;
  const int rl = tid / k, i = tid % k;
  const bool active = rl < rows;
  float my_norm = 0.f;
  for (int64_t c0 = (int64_t)blockIdx.x * rows; c0 < d; c0 += (int64_t)gridDim.x * rows) {
    const int64_t c = c0 + rl;
    const bool ok = active && c < d;
    const int64_t idx = c * k + i;
    const float s_old = ok ? S[idx] : 0.f;
    if (active) Ss[rl * k + i] = s_old;
    __syncthreads();
    if (ok) {
      const float v = V[idx];
      const float bv = b_is_identity ? (1.f + eps_B) * v : BV[idx] + eps_B * v;
      float pen = 0.f;
      for (int j = 0; j < i; ++j) pen = fmaf(Ss[rl * k + j], T[j * k + i], pen);
      const float gr = cb[i] * AV[idx] - cac[i] * bv - pen;
      const float vn = fmaf(eta, gr, v);
      Vtmp[idx] = vn;
      S[idx] = fmaf(gamma, bv - s_old, s_old);
      if (grad_out) grad_out[idx] = gr;
      my_norm = fmaf(vn, vn, my_norm);
    }
    __syncthreads();
  }
  if (active) atomicAdd(&nrm[i], my_norm);
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) atomicAdd(&gram[2 * k * k + k + j], nrm[j]);
}

// k_normalize: v_i <- v'_i / ||v'_i||; flags non-finite norms.
__global__ void k_normalize(const float* __restrict__ Vtmp, const float* __restrict__ gram,
                            float* __restrict__ V, int64_t d, int k, int* dflag) {
  const int64_t n = d * k;
  const float* norms = gram + 2 * k * k + k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % k);
    const float nn = norms[i];
    const float v = Vtmp[e] / sqrtf(nn);
    if (!isfinite(v)) atomicOr(dflag, kFlagNonFinite);
    V[e] = v;
  }
}

// k_rayleigh: num_i += sum_r 2 P_ri Q_ri (CCA, PLS) or P_ri^2 (PCA, and LDA's B rows);
// den_i += P_ri^2 + Q_ri^2 (CCA).
__global__ void k_rayleigh(const float* __restrict__ PQ, int64_t n, int k, int kind,
                           double* __restrict__ rq) {
  const int i = threadIdx.x % k;
  const int lanes = blockDim.x / k;
  const int lr = threadIdx.x / k;
  if (lr >= lanes) return;
  double num = 0.0, den = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * lanes + lr; r < n; r += (int64_t)gridDim.x * lanes) {
    const double p = PQ[r * 2 * k + i];
    const double q = PQ[r * 2 * k + k + i];
    if (kind == SGEP_PCA || kind == SGEP_LDA) {
      num += p * p;
    } else {
      num += 2.0 * p * q;
      den += p * p + q * q;
    }
  }
  atomicAdd(&rq[i], num);
  atomicAdd(&rq[k + i], den);
}

inline int grid_cap(const Ctx& c, int per_sm) { return c.num_sms * per_sm; }

template <typename T>
int launch_project(Ctx& c, const T* X, const T* Y, int64_t n, cudaStream_t s, const Centring& cz,
                   const float* sx, const float* sy) {
  const int64_t row_tiles = (n + 31) / 32;
  // Column chunk: enough blocks to fill the GPU, at least 32 columns each.
  int64_t chunk = 1024;
  while (chunk > 64 && row_tiles * ((c.d + chunk - 1) / chunk) < 2LL * c.num_sms) chunk /= 2;
  const int nchunk_x = (int)((c.d_x + chunk - 1) / chunk);
  const int nchunk_y = c.has_y ? (int)((c.d_y + chunk - 1) / chunk) : 0;
  dim3 grid((unsigned)row_tiles, (unsigned)(nchunk_x + nchunk_y));
  k_project<T><<<grid, kThreads, 0, s>>>(X, Y, n, c.d_x, c.d_y, c.V, c.k, chunk, nchunk_x, c.PQ, cz, sx, sy);
  SGEP_CUDA_TRY(cudaGetLastError());
  ++c.launches;
  return SGEP_OK;
}

template <typename T>
int launch_backproject(Ctx& c, const T* X, const T* Y, int64_t b, cudaStream_t s, const Centring& cz,
                       const float* sx, const float* sy) {
  const int kind = c.cfg.kind;
  const bool cca = kind == SGEP_CCA;
  const int split = (cca && c.cfg.split_AB) ? 1 : 0;
  const int64_t nA = split ? b / 2 : b;
  const int64_t nB = split ? b - nA : b;  // LDA: every row passed is a B row (nB = b)
  const int nblk_x = (int)((c.d_x + 63) / 64);
  const int nblk_y = c.has_y ? (int)((c.d_y + 63) / 64) : 0;
  const int nblk = nblk_x + nblk_y;
  int splits = (int)((2LL * c.num_sms + nblk - 1) / nblk);
  splits = (int)std::max<int64_t>(1, std::min<int64_t>(splits, (b + 31) / 32));
  int64_t rows_per_split = (b + splits - 1) / splits;
  rows_per_split = ((rows_per_split + 31) / 32) * 32;
  splits = (int)((b + rows_per_split - 1) / rows_per_split);
  dim3 grid((unsigned)nblk, (unsigned)splits);
  float* AV = c.acc;
  float* BV = c.acc + c.d * c.k;
  k_backproject<T><<<grid, kThreads, 0, s>>>(X, Y, b, c.d_x, c.d_y, nA, kind, split, c.PQ, c.k,
                                             nblk_x, rows_per_split, 1.f / (float)nA,
                                             1.f / (float)nB, AV, BV, cz, sx, sy);
  SGEP_CUDA_TRY(cudaGetLastError());
  ++c.launches;
  return SGEP_OK;
}

}  // namespace

// Dispatch on the handle's element type.
template <typename F>
int by_dtype(const Ctx& c, F&& f) {
  if (c.cfg.dtype == SGEP_BF16) return f(static_cast<const __nv_bfloat16*>(nullptr));
  if (c.cfg.dtype == SGEP_FP8E4M3) return f(static_cast<const __nv_fp8_e4m3*>(nullptr));
  return f(static_cast<const float*>(nullptr));
}

int generic_project(Ctx& c, const void* X, const void* Y, int64_t n, cudaStream_t s, const float* center,
                    const int32_t* labels, const float* sx, const float* sy) {
  SGEP_CUDA_TRY(cudaMemsetAsync(c.PQ, 0, sizeof(float) * n * 2 * c.k, s));
  const Centring cz{center, labels, c.cfg.n_classes, c.dflag};
  return by_dtype(c, [&](auto tag) {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    return launch_project<T>(c, (const T*)X, (const T*)Y, n, s, cz, sx, sy);
  });
}

// LDA: BV = X~^T (X~ V) / n over the n rows passed (already the B rows), centred by class means.
int generic_lda_within(Ctx& c, const void* X, const int32_t* labels, int64_t n, cudaStream_t s, const float* sx) {
  int rc = generic_project(c, X, nullptr, n, s, c.lda_mean, labels, sx, nullptr);
  if (rc) return rc;
  const Centring cz{c.lda_mean, labels, c.cfg.n_classes, c.dflag};
  return by_dtype(c, [&](auto tag) {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    return launch_backproject<T>(c, (const T*)X, nullptr, n, s, cz, sx, nullptr);
  });
}

int generic_products(Ctx& c, const void* X, const void* Y, int64_t b, cudaStream_t s, const float* sx,
                     const float* sy) {
  int rc = generic_project(c, X, Y, b, s, nullptr, nullptr, sx, sy);
  if (rc) return rc;
  SGEP_CUDA_TRY(cudaMemsetAsync(c.acc, 0, sizeof(float) * 2 * c.d * c.k, s));
  const Centring none{nullptr, nullptr, 0, c.dflag};
  return by_dtype(c, [&](auto tag) {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    return launch_backproject<T>(c, (const T*)X, (const T*)Y, b, s, none, sx, sy);
  });
}

int generic_update(Ctx& c, float eta, float gamma, cudaStream_t s) {
  const int k = c.k;
  const int kk = k * k;
  SGEP_CUDA_TRY(cudaMemsetAsync(c.gram, 0, sizeof(float) * (2 * kk + 2 * k), s));
  const float* AV = c.acc;
  const float* BV = c.acc + c.d * k;
  const int gblocks = (int)std::min<int64_t>((c.d + 31) / 32, grid_cap(c, 2));
  const size_t gsm = sizeof(float) * 3 * 32 * k;
  k_gram<<<gblocks, kThreads, gsm, s>>>(c.V, c.S, AV, BV, c.d, k, c.cfg.eps_B,
                                        c.b_is_identity ? 1 : 0, c.gram);
  SGEP_CUDA_TRY(cudaGetLastError());
  const int rows = std::max(1, kThreads / k);
  const int ublocks = (int)std::min<int64_t>((c.d + rows - 1) / rows, grid_cap(c, 4));
  const size_t usm = sizeof(float) * (kk + 3 * k + rows * k);
  k_update<<<ublocks, kThreads, usm, s>>>(c.V, c.S, AV, BV, c.gram, c.d, k, eta, gamma, c.cfg.rho,
                                          c.cfg.eps_B, c.b_is_identity ? 1 : 0, c.Vtmp,
                                          c.cfg.debug ? c.grad : nullptr);
  SGEP_CUDA_TRY(cudaGetLastError());
  const int nblocks = (int)std::min<int64_t>((c.d * k + 255) / 256, grid_cap(c, 4));
  k_normalize<<<nblocks, 256, 0, s>>>(c.Vtmp, c.gram, c.V, c.d, k, c.dflag);
  SGEP_CUDA_TRY(cudaGetLastError());
  c.launches += 3;
  return SGEP_OK;
}

int generic_normalize(Ctx& c, cudaStream_t s) {
  const int nblocks = (int)std::min<int64_t>((c.d * c.k + 255) / 256, grid_cap(c, 4));
  k_normalize<<<nblocks, 256, 0, s>>>(c.Vtmp, c.gram, c.V, c.d, c.k, c.dflag);
  SGEP_CUDA_TRY(cudaGetLastError());
  c.launches += 2;
  return SGEP_OK;
}

int generic_rayleigh_sums(Ctx& c, int64_t n, cudaStream_t s) {
  const int k = c.k;
  const int lanes = std::max(1, 256 / k);
  const int blocks = (int)std::min<int64_t>((n + lanes - 1) / lanes, grid_cap(c, 2));
  k_rayleigh<<<blocks, lanes * k, 0, s>>>(c.PQ, n, k, c.cfg.kind, c.rq);
  SGEP_CUDA_TRY(cudaGetLastError());
  ++c.launches;
  return SGEP_OK;
}

}  // namespace sgep

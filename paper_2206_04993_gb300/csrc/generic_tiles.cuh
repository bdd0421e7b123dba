// Tiles of the generic SIMT step (Alg. 2, M = 1) as device functions.
//
// Each function is the work of one thread block of 256 threads on one tile,
// identified by explicit tile coordinates (bx, by) or a (tile, tile count) pair
// for grid-stride loops, with an explicit shared-memory workspace. The generic
// kernels launch them one tile per block (blockIdx); the batched kernel runs them
// for many problem instances from one persistent launch. All threads of the block
// must call a tile function together.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "eg_math.cuh"
#include "internal.h"

namespace sgep {
namespace gt {

constexpr int kThreads = 256;
constexpr int kMaxK = 64;

// Shared-memory floats each tile needs (k <= 64, C <= 32).
constexpr int kProjectSmem = 32 * 33 + 32 * kMaxK;
constexpr int kBackprojectSmem = 32 * 64 + 32 * 2 * kMaxK;
__host__ __device__ constexpr int gram_smem(int k) { return 3 * 32 * k; }
__host__ __device__ constexpr int update_smem(int k) {
  return k * k + 4 * k + (kThreads / k > 1 ? kThreads / k : 1) * k;
}
__host__ __device__ constexpr int lda_stats_smem(int C) { return C * kThreads + kThreads; }
constexpr int kLdaWSmem = kMaxClasses * 33 + 32 * (kMaxK + 1);
constexpr int kLdaAvSmem = kMaxClasses * kMaxK;
constexpr int kLdaCountsSmem = kMaxClasses + 2;  // histogram + a double

__device__ __forceinline__ float load_elem(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_elem(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float load_elem(const __nv_fp8_e4m3* p, int64_t i) { return static_cast<float>(p[i]); }

// Element i of a row-major matrix, times the row's scale when there is one (FP8 rows).
template <typename T>
__device__ __forceinline__ float load_row_elem(const T* p, const float* scale, int64_t row, int64_t i) {
  const float x = load_elem(p, i);
  return scale ? x * scale[row] : x;
}

// Class-mean centring of LDA rows: x - mu_{label}. A label outside [0, C) is
// flagged and the row is left uncentred (the step then reports the bad label).
// Running-mean centring (labels null): x - mean[col] for X rows, x - mean_y[col] for Y rows.
struct Centring {
  const float* mean;      // C x ld class means, or null (no centring)
  const int32_t* labels;  // labels of the rows passed to the kernel, or null (running means)
  int C;
  int* dflag;
  const float* mean_y = nullptr;  // running mean of the Y view
};

__device__ __forceinline__ float centred(const Centring& cz, float x, int64_t row, int64_t ld, int64_t col,
                                         bool isY = false) {
  if (!cz.mean) return x;
  if (!cz.labels) return x - (isY ? cz.mean_y : cz.mean)[col];
  const int lab = cz.labels[row];
  if ((unsigned)lab >= (unsigned)cz.C) {
    atomicOr(cz.dflag, kFlagBadLabel);
    return x;
  }
  return x - cz.mean[(int64_t)lab * ld + col];
}

// ---------------------------------------------------------------------------
// Projection: PQ[r, 0:k] += X[r, cols] V[cols, :], PQ[r, k:2k] += Y[r, cols] V[d_x + cols, :]
// Tile (bx, by): rows [32 bx, 32 bx + 32), column chunk by (X chunks first, then Y
// chunks), each `chunk` columns wide. PQ must be zeroed.
template <typename T>
__device__ void project_tile(const T* __restrict__ X, const T* __restrict__ Y, int64_t n, int64_t dx, int64_t dy,
                             const float* __restrict__ V, int k, int64_t chunk, int nchunk_x, float* __restrict__ PQ,
                             const Centring& cz, const float* __restrict__ rsx, const float* __restrict__ rsy,
                             int bx, int by, float* smem) {
  constexpr int BR = 32, TC = 32;
  float(*Xs)[TC + 1] = reinterpret_cast<float(*)[TC + 1]>(smem);
  float(*Vs)[kMaxK] = reinterpret_cast<float(*)[kMaxK]>(smem + BR * (TC + 1));
  const int tid = threadIdx.x;
  const int r = tid >> 3;   // 0..31
  const int g = tid & 7;    // players g, g+8, ...
  const int64_t row0 = (int64_t)bx * BR;
  const bool isY = by >= nchunk_x;
  const int cidx = isY ? by - nchunk_x : by;
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
          (row < n && col < c_end) ? centred(cz, load_row_elem(Z, rs, row, row * ld + col), row, ld, col, isY)
                                   : 0.f;
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
// Back-projection: for column c of X (or Y) and player i,
//   AV[c,i] += inv_nA * sum_{r in A rows} Z[r,c] W_A[r,i]
//   BV[c,i] += inv_nB * sum_{r in B rows} Z[r,c] W_B[r,i]
// where (CCA) W_A = Q for X columns / P for Y columns and W_B = P for X / Q for Y;
// (PCA) W_A = P over every row, no BV; (PLS) W_A as CCA over every row, no BV;
// (LDA) every row passed is a B row, centred by its class mean: W_B = P, no AV.
// Tile (bx, by): column block bx of 64 (X blocks then Y blocks), row split by.
template <typename T>
__device__ void backproject_tile(const T* __restrict__ X, const T* __restrict__ Y, int64_t b, int64_t dx,
                                 int64_t dy, int64_t nA, int kind, int split, const float* __restrict__ PQ, int k,
                                 int nblk_x, int64_t rows_per_split, float inv_nA, float inv_nB,
                                 float* __restrict__ AV, float* __restrict__ BV, const Centring& cz,
                                 const float* __restrict__ rsx, const float* __restrict__ rsy, int bx, int by,
                                 float* smem) {
  constexpr int TR = 32, CB = 64;
  float(*Zs)[CB] = reinterpret_cast<float(*)[CB]>(smem);
  float(*Ws)[2 * kMaxK] = reinterpret_cast<float(*)[2 * kMaxK]>(smem + TR * CB);
  const int tid = threadIdx.x;
  const int cl = tid & (CB - 1);
  const int g = tid >> 6;  // players g, g+4, ...
  const bool isY = bx >= nblk_x;
  const int bidx = isY ? bx - nblk_x : bx;
  const T* Z = isY ? Y : X;
  const float* rs = isY ? rsy : rsx;
  const int64_t ld = isY ? dy : dx;
  const int64_t col = (int64_t)bidx * CB + cl;
  const int64_t r_begin = (int64_t)by * rows_per_split;
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
          (row < r_end && cg < ld) ? centred(cz, load_row_elem(Z, rs, row, row * ld + cg), row, ld, cg, isY)
                                   : 0.f;
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
// k x k terms: a_ij = sum_c V[c,i] AV[c,j];  G_ij = sum_c V[c,i] S[c,j];
//              b_i = sum_c V[c,i] (B_t V)[c,i] with B_t V = BV + eps V (or (1+eps) V when B = I).
// gram layout: [a (k*k) | G (k*k) | b (k) | norms (k)]; must be zeroed. Grid-stride
// over 32-row chunks of V: tile `bx` of `nb`.
__device__ inline void gram_tile(const float* __restrict__ V, const float* __restrict__ S,
                                 const float* __restrict__ AV, const float* __restrict__ BV, int64_t d, int k,
                                 float eps_B, int b_is_identity, float* __restrict__ gram, int bx, int nb,
                                 float* smem) {
  constexpr int CR = 32;
  float* Vs = smem;             // CR x k
  float* As = Vs + CR * k;      // CR x k
  float* Ss = As + CR * k;      // CR x k
  const int tid = threadIdx.x;
  const int kk = k * k;
  float ga[kMaxK * kMaxK / kThreads], gg[kMaxK * kMaxK / kThreads];
#pragma unroll
  for (int q = 0; q < kMaxK * kMaxK / kThreads; ++q) ga[q] = gg[q] = 0.f;
  float gb = 0.f;
  for (int64_t c0 = (int64_t)bx * CR; c0 < d; c0 += (int64_t)nb * CR) {
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

// ---------------------------------------------------------------------------
// Update: grad, V' = V + eta grad (into Vtmp), S <- S + gamma (B_t V - S), norms^2 of V'
// into gram's norms slot. Grid-stride over groups of 256 / k rows: tile `bx` of `nb`.
__device__ inline void update_tile(const float* __restrict__ V, float* __restrict__ S, const float* __restrict__ AV,
                                   const float* __restrict__ BV, float* gram, int64_t d, int k, float eta,
                                   float gamma, float rho, float eps_B, int b_is_identity, float* __restrict__ Vtmp,
                                   float* __restrict__ grad_out, int bx, int nb, float* smem,
                                   const UpdVariant& var = UpdVariant()) {
  float* T = smem;               // k*k
  float* cb = T + k * k;         // k
  float* cac = cb + k;           // k
  float* nrm = cac + k;          // k
  float* sden = nrm + k;         // k: Alg. 3 denominators
  const int rows = max(1, kThreads / k);
  float* Ss = sden + k;          // rows x k
  if (var.z) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) sden[j] = smooth_den(var.z[j], var.log_rho, var.log_nu);
    __syncthreads();
  }
  eg_coefficients(gram, k, rho, cb, cac, T, var.z ? sden : nullptr);
  for (int i = threadIdx.x; i < k; i += blockDim.x) nrm[i] = 0.f;
  __syncthreads();
  const int tid = threadIdx.x;
  const int rl = tid / k, i = tid % k;
  const bool active = rl < rows;
  float my_norm = 0.f;
  for (int64_t c0 = (int64_t)bx * rows; c0 < d; c0 += (int64_t)nb * rows) {
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
      float step = gr;
      if (var.m) {  // Adam on the players
        float m = var.m[idx], s2 = var.s[idx];
        step = adam_increment(gr, m, s2, var.b1, var.b2, var.eps, var.bc1, var.bc2);
        var.m[idx] = m;
        var.s[idx] = s2;
      }
      const float vn = fmaf(eta, step, v);
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

// Retraction: v_i <- v'_i / ||v'_i||; flags non-finite norms. Grid-stride: tile `bx` of `nb`.
// With Alg. 3 (var.z) tile 0 also takes the z step from the k x k terms G_ii = <v_i, [Bv]_i>
// of step t (the update tiles have read z before this launch).
__device__ inline void normalize_tile(const float* __restrict__ Vtmp, const float* __restrict__ gram,
                                      float* __restrict__ V, int64_t d, int k, int* dflag, int bx, int nb,
                                      const UpdVariant& var = UpdVariant(), float gamma = 0.f) {
  const int64_t n = d * k;
  const float* norms = gram + 2 * k * k + k;
  if (var.z && bx == 0)
    for (int i = threadIdx.x; i < k; i += blockDim.x)
      var.z[i] = smooth_z_step(var.z[i], gram[k * k + i * k + i], gamma, var.log_rho, var.log_nu);
  for (int64_t e = (int64_t)bx * blockDim.x + threadIdx.x; e < n; e += (int64_t)nb * blockDim.x) {
    const int i = (int)(e % k);
    const float v = Vtmp[e] / sqrtf(norms[i]);
    if (!isfinite(v)) atomicOr(dflag, kFlagNonFinite);
    V[e] = v;
  }
}

// ---------------------------------------------------------------------------
// LDA (reading of Sec. 1; see kernels_lda.cu): running class statistics and the
// between-class products.

// Counts of the minibatch's labels added to the running counts; priors. One tile.
__device__ inline void lda_counts_tile(const int32_t* __restrict__ labels, int64_t b, int C, double* __restrict__ cnt,
                                       float* __restrict__ pi, int* dflag, float* smem) {
  unsigned* h = reinterpret_cast<unsigned*>(smem);
  double* total = reinterpret_cast<double*>(smem + kMaxClasses + (kMaxClasses & 1));
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
    *total = n;
  }
  __syncthreads();
  if (tid < C) pi[tid] = *total > 0.0 ? (float)(cnt[tid] / *total) : 0.f;
  __syncthreads();
}

// Columns [256 bx, 256 bx + 256): class sums += the minibatch rows (none when b = 0),
// then the class means, mu_c - mu, and the means used for centring.
template <typename T>
__device__ void lda_stats_tile(const T* __restrict__ X, const float* __restrict__ rs,
                               const int32_t* __restrict__ labels, int64_t b, int64_t d, int C,
                               double* __restrict__ sum, const double* __restrict__ cnt, float* __restrict__ mean,
                               float* __restrict__ M, int bx, float* smem) {
  float* acc = smem;                                             // [C][kThreads]
  int* labs = reinterpret_cast<int*>(smem + C * kThreads);       // [kThreads]
  const int tid = threadIdx.x;
  const int64_t col = (int64_t)bx * kThreads + tid;
  for (int c = 0; c < C; ++c) acc[c * kThreads + tid] = 0.f;
  for (int64_t r0 = 0; r0 < b; r0 += kThreads) {
    __syncthreads();
    const int64_t rr = r0 + tid;
    const int lab = rr < b ? labels[rr] : -1;
    labs[tid] = (unsigned)lab < (unsigned)C ? lab : -1;  // bad labels are flagged by the counts tile
    __syncthreads();
    const int nr = (int)min((int64_t)kThreads, b - r0);
    if (col < d) {
      for (int q0 = 0; q0 < nr; q0 += 8) {
        float x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int64_t row = r0 + q0 + q;
          x[q] = (q0 + q < nr) ? load_row_elem(X, rs, row, row * d + col) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int lab2 = (q0 + q < nr) ? labs[q0 + q] : -1;
          if (lab2 >= 0) acc[lab2 * kThreads + tid] += x[q];
        }
      }
    }
  }
  __syncthreads();
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

// W[c][i] += sum over this tile's columns of M[c][col] V[col][i] (W zeroed before).
// Grid-stride over 32-column chunks: tile `bx` of `nb`.
__device__ inline void lda_w_tile(const float* __restrict__ M, const float* __restrict__ V, int64_t d, int C, int k,
                                  float* __restrict__ W, int bx, int nb, float* smem) {
  constexpr int TC = 32;
  float(*Ms)[TC + 1] = reinterpret_cast<float(*)[TC + 1]>(smem);
  float(*Vs)[kMaxK + 1] = reinterpret_cast<float(*)[kMaxK + 1]>(smem + kMaxClasses * (TC + 1));
  const int tid = threadIdx.x;
  const int nout = C * k;
  float acc[(kMaxClasses * kMaxK) / kThreads];
#pragma unroll
  for (int q = 0; q < (kMaxClasses * kMaxK) / kThreads; ++q) acc[q] = 0.f;
  for (int64_t c0 = (int64_t)bx * TC; c0 < d; c0 += (int64_t)nb * TC) {
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
    for (int q = 0; q < (kMaxClasses * kMaxK) / kThreads; ++q) {
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
  for (int q = 0; q < (kMaxClasses * kMaxK) / kThreads; ++q) {
    const int p = tid + q * kThreads;
    if (p < nout) atomicAdd(&W[p], acc[q]);
  }
}

// AV[col][i] = sum_c M[c][col] pi_c W[c][i]. Grid-stride: tile `bx` of `nb`.
__device__ inline void lda_av_tile(const float* __restrict__ M, const float* __restrict__ pi,
                                   const float* __restrict__ W, int64_t d, int C, int k, float* __restrict__ AV,
                                   int bx, int nb, float* smem) {
  float* PW = smem;  // C x k
  for (int e = threadIdx.x; e < C * k; e += kThreads) PW[e] = pi[e / k] * W[e];
  __syncthreads();
  for (int64_t e = (int64_t)bx * kThreads + threadIdx.x; e < d * k; e += (int64_t)nb * kThreads) {
    const int64_t col = e / k;
    const int i = (int)(e % k);
    float s = 0.f;
    for (int c = 0; c < C; ++c) s = fmaf(M[c * d + col], PW[c * k + i], s);
    AV[e] = s;
  }
  __syncthreads();
}

}  // namespace gt
}  // namespace sgep

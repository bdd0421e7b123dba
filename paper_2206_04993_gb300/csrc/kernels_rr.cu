// Rayleigh-Ritz correction of the players (precision form).
//
// In the span of the current players, the k x k pencil (V^T A V) c = lambda (V^T B V) c
// is formed from an evaluation batch (FP64 sums of the FP32 row projections) and
// solved in FP64 on the device by the reduction of App. A (Prop. "Similar
// matrices"): Cholesky V^T B V = L L^T, M = L^-1 (V^T A V) L^-T, a cyclic Jacobi
// eigensolver for M, C = L^-T U. The players and the auxiliary variables are then
// rotated, V <- V C and [Bv] <- [Bv] C, and every column of both is divided by
// ||v'_i|| (the retraction to the unit sphere). Eigenvalues are returned in
// descending order; the columns of C are unit vectors of R^k whose largest-magnitude
// entry is positive.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace sgep {
namespace {

constexpr int kThreads = 256;
constexpr int kJacobiSweeps = 40;

// Asum += P^T Q + Q^T P (CCA, PLS) or P^T P (PCA); Bsum += P^T P + Q^T Q (CCA) or
// P^T P (LDA, whose rows are centred); PQ rows are [P | Q] (2k floats).
__global__ void __launch_bounds__(kThreads) k_rr_gram_pq(const float* __restrict__ PQ, int64_t m, int k, int kind,
                                                         double* __restrict__ Asum, double* __restrict__ Bsum) {
  constexpr int R = 32;
  extern __shared__ float rows[];  // R x 2k
  const int tid = threadIdx.x, kk = k * k;
  double a[(64 * 64) / kThreads], b[(64 * 64) / kThreads];
#pragma unroll
  for (int q = 0; q < (64 * 64) / kThreads; ++q) a[q] = b[q] = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < m; r0 += (int64_t)gridDim.x * R) {
    const int nr = (int)min((int64_t)R, m - r0);
    for (int e = tid; e < R * 2 * k; e += kThreads) rows[e] = e < nr * 2 * k ? PQ[r0 * 2 * k + e] : 0.f;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (64 * 64) / kThreads; ++q) {
      const int p = tid + q * kThreads;
      if (p < kk) {
        const int i = p / k, j = p % k;
        double sa = 0.0, sb = 0.0;
        for (int r = 0; r < nr; ++r) {
          const float* w = rows + r * 2 * k;
          const double pi = w[i], pj = w[j], qi = w[k + i], qj = w[k + j];
          if (kind == SGEP_CCA || kind == SGEP_PLS) sa += pi * qj + qi * pj;
          else if (kind == SGEP_PCA) sa += pi * pj;
          if (kind == SGEP_CCA) sb += pi * pj + qi * qj;
          else if (kind == SGEP_LDA) sb += pi * pj;
        }
        a[q] += sa;
        b[q] += sb;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < (64 * 64) / kThreads; ++q) {
    const int p = tid + q * kThreads;
    if (p < kk) {
      if (kind != SGEP_LDA) atomicAdd(&Asum[p], a[q]);
      if (kind == SGEP_CCA || kind == SGEP_LDA) atomicAdd(&Bsum[p], b[q]);
    }
  }
}

// VtV += V^T V over the rows of V (d x k).
__global__ void __launch_bounds__(kThreads) k_rr_gram_v(const float* __restrict__ V, int64_t d, int k,
                                                        double* __restrict__ VtV) {
  constexpr int R = 32;
  extern __shared__ float rows[];  // R x k
  const int tid = threadIdx.x, kk = k * k;
  double g[(64 * 64) / kThreads];
#pragma unroll
  for (int q = 0; q < (64 * 64) / kThreads; ++q) g[q] = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < d; r0 += (int64_t)gridDim.x * R) {
    const int nr = (int)min((int64_t)R, d - r0);
    for (int e = tid; e < R * k; e += kThreads) rows[e] = e < nr * k ? V[r0 * k + e] : 0.f;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (64 * 64) / kThreads; ++q) {
      const int p = tid + q * kThreads;
      if (p < kk) {
        const int i = p / k, j = p % k;
        double s = 0.0;
        for (int r = 0; r < nr; ++r) s += (double)rows[r * k + i] * rows[r * k + j];
        g[q] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < (64 * 64) / kThreads; ++q) {
    const int p = tid + q * kThreads;
    if (p < kk) atomicAdd(&VtV[p], g[q]);
  }
}

// The k x k generalized eigenproblem, one block, FP64, every loop bounded.
// Ak: LDA -> sum_c pi_c W_c^T W_c; else Asum / n. Bk: PCA, PLS -> V^T V; else Bsum / n;
// plus eps_B V^T V. Outputs C (k x k, columns ordered by descending eigenvalue) and lam.
__global__ void __launch_bounds__(kThreads) k_rr_solve(const double* __restrict__ Asum,
                                                       const double* __restrict__ Bsum,
                                                       const double* __restrict__ VtV, const float* __restrict__ W,
                                                       const float* __restrict__ pi, int C, double inv_n, int kind,
                                                       double eps_B, int k, double* __restrict__ Cout,
                                                       double* __restrict__ lam_out, int* dflag) {
  extern __shared__ double sm[];
  const int ld = k + 1;
  double* M = sm;           // k x ld: A, then L^-1 A L^-T, then its eigenvalues on the diagonal
  double* L = M + k * ld;   // k x ld: B, then its Cholesky factor
  double* U = L + k * ld;   // k x ld: eigenvectors of M
  double* Z = U + k * ld;   // k x ld: scratch
  __shared__ double cs[32], sn[32], red[kThreads], red2[kThreads];
  __shared__ int pp[32], qq[32], perm[64];
  __shared__ int bad, done;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < k * k; e += kThreads) {
    const int i = e / k, j = e % k;
    double a;
    if (kind == SGEP_LDA) {
      a = 0.0;
      for (int c = 0; c < C; ++c) a += (double)pi[c] * W[c * k + i] * W[c * k + j];
    } else {
      a = Asum[e] * inv_n;
    }
    double b = (kind == SGEP_PCA || kind == SGEP_PLS) ? VtV[e] : Bsum[e] * inv_n;
    b += eps_B * VtV[e];
    M[i * ld + j] = a;
    L[i * ld + j] = b;
    U[i * ld + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += kThreads) {  // symmetrise (each unordered pair once)
    const int i = e / k, j = e % k;
    if (i < j) {
      const double a = 0.5 * (M[i * ld + j] + M[j * ld + i]);
      const double b = 0.5 * (L[i * ld + j] + L[j * ld + i]);
      M[i * ld + j] = M[j * ld + i] = a;
      L[i * ld + j] = L[j * ld + i] = b;
    }
  }
  __syncthreads();
  // Cholesky, lower triangle in place
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      double s = L[j * ld + j];
      for (int p = 0; p < j; ++p) s -= L[j * ld + p] * L[j * ld + p];
      if (!(s > 0.0)) bad = 1;
      L[j * ld + j] = sqrt(s > 0.0 ? s : 1.0);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < k; i += kThreads) {
      double s = L[i * ld + j];
      for (int p = 0; p < j; ++p) s -= L[i * ld + p] * L[j * ld + p];
      L[i * ld + j] = s / L[j * ld + j];
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicOr(dflag, kFlagNotPD);
    return;
  }
  // Z = L^-1 A (columns independent)
  for (int c = tid; c < k; c += kThreads)
    for (int i = 0; i < k; ++i) {
      double s = M[i * ld + c];
      for (int p = 0; p < i; ++p) s -= L[i * ld + p] * Z[p * ld + c];
      Z[i * ld + c] = s / L[i * ld + i];
    }
  __syncthreads();
  // M = L^-1 Z^T = L^-1 A L^-T
  for (int c = tid; c < k; c += kThreads)
    for (int i = 0; i < k; ++i) {
      double s = Z[c * ld + i];
      for (int p = 0; p < i; ++p) s -= L[i * ld + p] * M[p * ld + c];
      M[i * ld + c] = s / L[i * ld + i];
    }
  __syncthreads();
  for (int e = tid; e < k * k; e += kThreads) {
    const int i = e / k, j = e % k;
    if (i < j) M[i * ld + j] = M[j * ld + i] = 0.5 * (M[i * ld + j] + M[j * ld + i]);
  }
  __syncthreads();
  // cyclic Jacobi, round-robin pairs (circle method over km players; index k is a
  // dummy when k is odd)
  const int km = k + (k & 1), half = km / 2;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < k * k; e += kThreads) {
      const int i = e / k, j = e % k;
      const double v = M[i * ld + j] * M[i * ld + j];
      tot += v;
      if (i != j) off += v;
    }
    red[tid] = off;
    red2[tid] = tot;
    __syncthreads();
    if (tid == 0) {
      double o = 0.0, t2 = 0.0;
      for (int i = 0; i < kThreads; ++i) {
        o += red[i];
        t2 += red2[i];
      }
      done = (o <= 1e-28 * t2) ? 1 : 0;
    }
    __syncthreads();
    if (done) break;
    for (int r = 0; r < km - 1; ++r) {
      if (tid < half) {
        int p, q;
        if (tid == 0) {
          p = 0;
          q = 1 + r;
        } else {
          p = 1 + (r + tid) % (km - 1);
          q = 1 + (r - tid + km - 1) % (km - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        if (q < k) {
          const double apq = M[p * ld + q];
          if (fabs(apq) > 1e-300) {
            const double th = (M[q * ld + q] - M[p * ld + p]) / (2.0 * apq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        pp[tid] = p;
        qq[tid] = q;
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      for (int e = tid; e < half * k; e += kThreads) {  // rows p, q of M
        const int t = e / k, j = e % k;
        const int p = pp[t], q = qq[t];
        if (q < k) {
          const double c = cs[t], s = sn[t];
          const double mp = M[p * ld + j], mq = M[q * ld + j];
          M[p * ld + j] = c * mp - s * mq;
          M[q * ld + j] = s * mp + c * mq;
        }
      }
      __syncthreads();
      for (int e = tid; e < half * k; e += kThreads) {  // columns p, q of M and of U
        const int t = e / k, i = e % k;
        const int p = pp[t], q = qq[t];
        if (q < k) {
          const double c = cs[t], s = sn[t];
          const double mp = M[i * ld + p], mq = M[i * ld + q];
          M[i * ld + p] = c * mp - s * mq;
          M[i * ld + q] = s * mp + c * mq;
          const double up = U[i * ld + p], uq = U[i * ld + q];
          U[i * ld + p] = c * up - s * uq;
          U[i * ld + q] = s * up + c * uq;
        }
      }
      __syncthreads();
    }
  }
  // descending order of the eigenvalues
  if (tid == 0) {
    for (int i = 0; i < k; ++i) perm[i] = i;
    for (int i = 0; i < k; ++i) {
      int best = i;
      for (int j = i + 1; j < k; ++j)
        if (M[perm[j] * ld + perm[j]] > M[perm[best] * ld + perm[best]]) best = j;
      const int t = perm[i];
      perm[i] = perm[best];
      perm[best] = t;
    }
  }
  __syncthreads();
  // C = L^-T U[:, perm], unit columns, largest-magnitude entry positive
  for (int c = tid; c < k; c += kThreads) {
    const int src = perm[c];
    for (int i = k - 1; i >= 0; --i) {
      double s = U[i * ld + src];
      for (int p = i + 1; p < k; ++p) s -= L[p * ld + i] * Z[p * ld + c];
      Z[i * ld + c] = s / L[i * ld + i];
    }
    double nrm = 0.0, big = 0.0;
    for (int i = 0; i < k; ++i) {
      const double v = Z[i * ld + c];
      nrm += v * v;
      if (fabs(v) > fabs(big)) big = v;
    }
    const double sc = (big < 0.0 ? -1.0 : 1.0) / sqrt(nrm);
    for (int i = 0; i < k; ++i) Cout[i * k + c] = Z[i * ld + c] * sc;
    lam_out[c] = M[src * ld + src];
  }
}

// Vtmp = V C, S <- S C (rows staged in shared memory), column sums of (V C)^2 into nrm.
__global__ void __launch_bounds__(kThreads) k_rr_apply(const float* __restrict__ V, float* __restrict__ S,
                                                       const double* __restrict__ Cm, int64_t d, int k,
                                                       float* __restrict__ Vtmp, double* __restrict__ nrm) {
  extern __shared__ double Cs[];  // k x k, then rows of V and S (float)
  float* vs = reinterpret_cast<float*>(Cs + k * k);
  const int R = max(1, kThreads / k);
  float* ss = vs + R * k;
  __shared__ double red[kThreads];
  const int tid = threadIdx.x;
  for (int e = tid; e < k * k; e += kThreads) Cs[e] = Cm[e];
  const int rl = tid / k, i = tid % k;
  const bool active = rl < R;
  double acc = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < d; r0 += (int64_t)gridDim.x * R) {
    __syncthreads();
    for (int e = tid; e < R * k; e += kThreads) {
      const int64_t row = r0 + e / k;
      vs[e] = row < d ? V[r0 * k + e] : 0.f;
      ss[e] = row < d ? S[r0 * k + e] : 0.f;
    }
    __syncthreads();
    const int64_t row = r0 + rl;
    if (active && row < d) {
      double v = 0.0, s = 0.0;
      for (int j = 0; j < k; ++j) {
        v += (double)vs[rl * k + j] * Cs[j * k + i];
        s += (double)ss[rl * k + j] * Cs[j * k + i];
      }
      Vtmp[row * k + i] = (float)v;
      S[row * k + i] = (float)s;
      acc += v * v;
    }
  }
  red[tid] = active ? acc : 0.0;
  __syncthreads();
  if (tid < k) {
    double s = 0.0;
    for (int r = 0; r < R; ++r) s += red[r * k + tid];
    atomicAdd(&nrm[tid], s);
  }
}

// V = Vtmp / ||.||, S = S / ||.|| column-wise; flags non-finite results.
__global__ void k_rr_scale(const float* __restrict__ Vtmp, float* __restrict__ V, float* __restrict__ S,
                           const double* __restrict__ nrm, int64_t n, int k, int* dflag) {
  bool badv = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double inv = 1.0 / sqrt(nrm[e % k]);
    const float v = (float)(Vtmp[e] * inv);
    V[e] = v;
    S[e] = (float)(S[e] * inv);
    badv |= !isfinite(v);
  }
  if (badv) atomicOr(dflag, kFlagNonFinite);
}

}  // namespace

int rr_correct(Ctx& c, const void* X, const void* Y, const float* sx, const float* sy, const int32_t* labels,
               int64_t n, double* lam_host, cudaStream_t s) {
  const int k = c.k, kk = k * k;
  if (!c.rr_buf) SGEP_CUDA_TRY(cudaMalloc((void**)&c.rr_buf, (size_t)(4 * kk + 2 * k) * sizeof(double)));
  double* Asum = c.rr_buf;
  double* Bsum = Asum + kk;
  double* VtV = Bsum + kk;
  double* Cm = VtV + kk;
  double* lam = Cm + kk;
  double* nrm = lam + k;
  SGEP_CUDA_TRY(cudaMemsetAsync(c.rr_buf, 0, (size_t)(4 * kk + 2 * k) * sizeof(double), s));
  const int kind = c.cfg.kind;
  const bool lda = kind == SGEP_LDA;
  const size_t esz = elem_size(c);
  for (int64_t r0 = 0; r0 < n; r0 += c.cfg.max_b) {
    const int64_t m = std::min<int64_t>(c.cfg.max_b, n - r0);
    const char* xs = (const char*)X + (size_t)r0 * c.d_x * esz;
    const char* ys = c.has_y ? (const char*)Y + (size_t)r0 * c.d_y * esz : nullptr;
    const float* sxs = sx ? sx + r0 : nullptr;
    const float* sys = sy ? sy + r0 : nullptr;
    int rc = generic_project(c, xs, ys, m, s, lda ? c.lda_mean : nullptr, lda ? labels + r0 : nullptr, sxs, sys);
    if (rc) return rc;
    const int grid = (int)std::min<int64_t>((m + 31) / 32, 2LL * c.num_sms);
    k_rr_gram_pq<<<grid, kThreads, (size_t)32 * 2 * k * sizeof(float), s>>>(c.PQ, m, k, kind, Asum, Bsum);
    SGEP_CUDA_TRY(cudaGetLastError());
  }
  {
    const int grid = (int)std::min<int64_t>((c.d + 31) / 32, 2LL * c.num_sms);
    k_rr_gram_v<<<grid, kThreads, (size_t)32 * k * sizeof(float), s>>>(c.V, c.d, k, VtV);
    SGEP_CUDA_TRY(cudaGetLastError());
  }
  if (lda) {
    int rc = lda_project_means(c, s);
    if (rc) return rc;
  }
  const size_t smem_solve = (size_t)4 * k * (k + 1) * sizeof(double);
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_rr_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_solve));
  k_rr_solve<<<1, kThreads, smem_solve, s>>>(Asum, Bsum, VtV, c.lda_W, c.lda_pi, lda ? c.cfg.n_classes : 0,
                                             1.0 / (double)n, kind, (double)c.cfg.eps_B, k, Cm, lam, c.dflag);
  SGEP_CUDA_TRY(cudaGetLastError());
  // a failed solve (B not positive definite) leaves V and S untouched: check first
  SGEP_CUDA_TRY(cudaStreamSynchronize(s));
  int flag = 0;
  SGEP_CUDA_TRY(cudaMemcpy(&flag, c.dflag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag & kFlagNotPD) return SGEP_OK;  // reported by the caller's flag check
  {
    const int R = std::max(1, kThreads / k);
    const size_t smem = (size_t)kk * sizeof(double) + (size_t)2 * R * k * sizeof(float);
    const int grid = (int)std::min<int64_t>((c.d + R - 1) / R, 4LL * c.num_sms);
    k_rr_apply<<<grid, kThreads, smem, s>>>(c.V, c.S, Cm, c.d, k, c.Vtmp, nrm);
    SGEP_CUDA_TRY(cudaGetLastError());
    const int64_t nn = c.d * k;
    k_rr_scale<<<(unsigned)std::min<int64_t>((nn + 255) / 256, 4LL * c.num_sms), 256, 0, s>>>(c.Vtmp, c.V, c.S, nrm,
                                                                                           nn, k, c.dflag);
    SGEP_CUDA_TRY(cudaGetLastError());
  }
  c.launches += 4 + (n + c.cfg.max_b - 1) / c.cfg.max_b * 2;
  if (lam_host) {
    SGEP_CUDA_TRY(cudaMemcpyAsync(lam_host, lam, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  SGEP_CUDA_TRY(cudaStreamSynchronize(s));
  return SGEP_OK;
}

}  // namespace sgep

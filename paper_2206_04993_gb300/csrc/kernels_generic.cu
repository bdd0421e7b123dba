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

#include "generic_tiles.cuh"
#include "internal.h"

namespace sgep {
namespace {

using gt::Centring;
using gt::kThreads;

// One tile per block; the tile functions live in generic_tiles.cuh.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_project(const T* __restrict__ X, const T* __restrict__ Y, int64_t n,
                                                      int64_t dx, int64_t dy, const float* __restrict__ V, int k,
                                                      int64_t chunk, int nchunk_x, float* __restrict__ PQ,
                                                      const Centring cz, const float* __restrict__ rsx,
                                                      const float* __restrict__ rsy) {
  extern __shared__ __align__(16) float smem[];
  gt::project_tile(X, Y, n, dx, dy, V, k, chunk, nchunk_x, PQ, cz, rsx, rsy, blockIdx.x, blockIdx.y, smem);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_backproject(
    const T* __restrict__ X, const T* __restrict__ Y, int64_t b, int64_t dx, int64_t dy, int64_t nA, int kind,
    int split, const float* __restrict__ PQ, int k, int nblk_x, int64_t rows_per_split, float inv_nA, float inv_nB,
    float* __restrict__ AV, float* __restrict__ BV, const Centring cz, const float* __restrict__ rsx,
    const float* __restrict__ rsy) {
  extern __shared__ __align__(16) float smem[];
  gt::backproject_tile(X, Y, b, dx, dy, nA, kind, split, PQ, k, nblk_x, rows_per_split, inv_nA, inv_nB, AV, BV, cz,
                       rsx, rsy, blockIdx.x, blockIdx.y, smem);
}

__global__ void __launch_bounds__(kThreads) k_gram(const float* __restrict__ V, const float* __restrict__ S,
                                                   const float* __restrict__ AV, const float* __restrict__ BV,
                                                   int64_t d, int k, float eps_B, int b_is_identity,
                                                   float* __restrict__ gram) {
  extern __shared__ __align__(16) float smem[];
  gt::gram_tile(V, S, AV, BV, d, k, eps_B, b_is_identity, gram, blockIdx.x, gridDim.x, smem);
}

__global__ void __launch_bounds__(kThreads) k_update(const float* __restrict__ V, float* __restrict__ S,
                                                     const float* __restrict__ AV, const float* __restrict__ BV,
                                                     float* gram, int64_t d, int k, float eta, float gamma,
                                                     float rho, float eps_B, int b_is_identity,
                                                     float* __restrict__ Vtmp, float* __restrict__ grad_out,
                                                     const UpdVariant var) {
  extern __shared__ __align__(16) float smem[];
  gt::update_tile(V, S, AV, BV, gram, d, k, eta, gamma, rho, eps_B, b_is_identity, Vtmp, grad_out, blockIdx.x,
                  gridDim.x, smem, var);
}

__global__ void k_normalize(const float* __restrict__ Vtmp, const float* __restrict__ gram, float* __restrict__ V,
                            int64_t d, int k, int* dflag, const UpdVariant var, float gamma) {
  gt::normalize_tile(Vtmp, gram, V, d, k, dflag, blockIdx.x, gridDim.x, var, gamma);
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

// The contraction tiles use more than the default 48 KB of dynamic shared memory.
template <typename K>
cudaError_t smem_optin(K kernel, int floats) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, floats * (int)sizeof(float));
}

template <typename T>
int launch_project(Ctx& c, const T* X, const T* Y, int64_t n, cudaStream_t s, const Centring& cz,
                   const float* sx, const float* sy) {
  const int64_t row_tiles = (n + gt::kProjRows - 1) / gt::kProjRows;
  // Column chunk: enough blocks to fill the GPU, at least 32 columns each.
  int64_t chunk = 1024;
  while (chunk > 64 && row_tiles * ((c.d + chunk - 1) / chunk) < 2LL * c.num_sms) chunk /= 2;
  const int nchunk_x = (int)((c.d_x + chunk - 1) / chunk);
  const int nchunk_y = c.has_y ? (int)((c.d_y + chunk - 1) / chunk) : 0;
  dim3 grid((unsigned)row_tiles, (unsigned)(nchunk_x + nchunk_y));
  SGEP_CUDA_TRY(smem_optin(k_project<T>, gt::kProjectSmem));
  k_project<T><<<grid, kThreads, gt::kProjectSmem * sizeof(float), s>>>(X, Y, n, c.d_x, c.d_y, c.V, c.k, chunk, nchunk_x, c.PQ, cz, sx, sy);
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
  SGEP_CUDA_TRY(smem_optin(k_backproject<T>, gt::kBackprojectSmem));
  k_backproject<T><<<grid, kThreads, gt::kBackprojectSmem * sizeof(float), s>>>(X, Y, b, c.d_x, c.d_y, nA, kind, split, c.PQ, c.k,
                                             nblk_x, rows_per_split, 1.f / (float)nA,
                                             1.f / (float)nB, AV, BV, cz, sx, sy);
  SGEP_CUDA_TRY(cudaGetLastError());
  ++c.launches;
  return SGEP_OK;
}

// ---- running-mean centring ----
// sums[c] += sum_{r < n} x_rc (FP64) for the ld columns of one view; 256 columns per block,
// rows split over gridDim.y.
template <typename T>
__global__ void k_colsum(const T* __restrict__ Z, int64_t n, int64_t ld, const float* __restrict__ rs,
                         double* __restrict__ sums) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ld) return;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * per, r1 = min(n, r0 + per);
  double acc = 0.0;
  for (int64_t r = r0; r < r1; ++r) acc += (double)gt::load_row_elem(Z, rs, r, r * ld + col);
  atomicAdd(&sums[col], acc);
}

__global__ void k_mean_from_sums(const double* __restrict__ sums, int64_t d, double count, float* __restrict__ mean) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d; e += (int64_t)gridDim.x * blockDim.x)
    mean[e] = count > 0.0 ? (float)(sums[e] / count) : 0.f;
}

// ---- ICA helpers ----
// w[r] = ||x_r||^2 for r < n (one warp per row; FP8 rows times their scale).
template <typename T>
__global__ void k_row_sqnorm(const T* __restrict__ X, int64_t n, int64_t d, const float* __restrict__ rs,
                             float* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += nw) {
    float s = 0.f;
    for (int64_t c = lane; c < d; c += 32) {
      const float x = gt::load_row_elem(X, rs, r, r * d + c);
      s = fmaf(x, x, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[r] = s;
  }
}

// PW[r, i] = w[r] PQ[r, i] for r < n, i < k (both with row stride 2k).
__global__ void k_weight_rows(const float* __restrict__ PQ, const float* __restrict__ w, int64_t n, int k,
                              float* __restrict__ PW) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k;
    const int i = (int)(e % k);
    PW[r * 2 * k + i] = w[r] * PQ[r * 2 * k + i];
  }
}

// out[0] = sum_{r < n} w[r] / n (one block, double accumulation).
__global__ void k_mean(const float* __restrict__ w, int64_t n, float* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s += w[r];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = (float)(red[0] / (double)n);
}

// A_t V = K - tr U - 2 W (kurtosis term, tr(B_2) B_3 V, B_2 B_3 V).
__global__ void k_ica_combine(float* __restrict__ AV, const float* __restrict__ U, const float* __restrict__ W,
                              const float* __restrict__ tr, int64_t n) {
  const float t = tr[0];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    AV[e] = AV[e] - t * U[e] - 2.f * W[e];
}

// out (n x 2k, first k columns used) = X M over n rows of one view, M d_x x k.
template <typename T>
int launch_project_with(Ctx& c, const T* X, int64_t n, const float* M, float* out, cudaStream_t s, const float* sx) {
  SGEP_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(float) * n * 2 * c.k, s));
  const int64_t row_tiles = (n + gt::kProjRows - 1) / gt::kProjRows;
  int64_t chunk = 1024;
  while (chunk > 64 && row_tiles * ((c.d_x + chunk - 1) / chunk) < 2LL * c.num_sms) chunk /= 2;
  const int nchunk_x = (int)((c.d_x + chunk - 1) / chunk);
  const Centring none{nullptr, nullptr, 0, c.dflag};
  dim3 grid((unsigned)row_tiles, (unsigned)nchunk_x);
  SGEP_CUDA_TRY(smem_optin(k_project<T>, gt::kProjectSmem));
  k_project<T><<<grid, kThreads, gt::kProjectSmem * sizeof(float), s>>>(X, nullptr, n, c.d_x, 0, M, c.k, chunk,
                                                                          nchunk_x, out, none, sx, nullptr);
  SGEP_CUDA_TRY(cudaGetLastError());
  ++c.launches;
  return SGEP_OK;
}

// out (d_x x k) += scale X^T P over n rows of one view (P with row stride 2k).
template <typename T>
int launch_bp_rows(Ctx& c, const T* X, int64_t n, const float* P, float* out, float scale, cudaStream_t s,
                   const float* sx) {
  const int nblk = (int)((c.d_x + 63) / 64);
  int splits = (int)((2LL * c.num_sms + nblk - 1) / nblk);
  splits = (int)std::max<int64_t>(1, std::min<int64_t>(splits, (n + 31) / 32));
  int64_t rows_per_split = (n + splits - 1) / splits;
  rows_per_split = ((rows_per_split + 31) / 32) * 32;
  splits = (int)((n + rows_per_split - 1) / rows_per_split);
  const Centring none{nullptr, nullptr, 0, c.dflag};
  dim3 grid((unsigned)nblk, (unsigned)splits);
  SGEP_CUDA_TRY(smem_optin(k_backproject<T>, gt::kBackprojectSmem));
  k_backproject<T><<<grid, kThreads, gt::kBackprojectSmem * sizeof(float), s>>>(
      X, nullptr, n, c.d_x, 0, n, SGEP_PCA, 0, P, c.k, nblk, rows_per_split, scale, scale, out, nullptr, none, sx,
      nullptr);
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

// Rows centred by class means (center, labels), else by the running means of a centring
// handle, else not centred.
static Centring centring_of(const Ctx& c, const float* center, const int32_t* labels) {
  if (center) return Centring{center, labels, c.cfg.n_classes, c.dflag};
  if (c.cen_mean) return Centring{c.cen_mean, nullptr, 1, c.dflag, c.cen_mean + c.d_x};
  return Centring{nullptr, nullptr, 0, c.dflag};
}

int generic_project(Ctx& c, const void* X, const void* Y, int64_t n, cudaStream_t s, const float* center,
                    const int32_t* labels, const float* sx, const float* sy) {
  SGEP_CUDA_TRY(cudaMemsetAsync(c.PQ, 0, sizeof(float) * n * 2 * c.k, s));
  const Centring cz = centring_of(c, center, labels);
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
  const Centring cz = centring_of(c, nullptr, nullptr);
  return by_dtype(c, [&](auto tag) {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    return launch_backproject<T>(c, (const T*)X, (const T*)Y, b, s, cz, sx, sy);
  });
}

int generic_update(Ctx& c, float eta, float gamma, cudaStream_t s) {
  const int k = c.k;
  const int kk = k * k;
  SGEP_CUDA_TRY(cudaMemsetAsync(c.gram, 0, sizeof(float) * (2 * kk + 2 * k), s));
  const float* AV = c.acc;
  const float* BV = c.acc + c.d * k;
  const int gblocks = (int)std::min<int64_t>((c.d + 31) / 32, grid_cap(c, 2));
  const size_t gsm = sizeof(float) * gt::gram_smem(k);
  k_gram<<<gblocks, kThreads, gsm, s>>>(c.V, c.S, AV, BV, c.d, k, c.cfg.eps_B,
                                        c.b_is_identity ? 1 : 0, c.gram);
  SGEP_CUDA_TRY(cudaGetLastError());
  const int rows = std::max(1, kThreads / k);
  const int64_t span = (int64_t)rows * gt::kUpdRows;
  const int ublocks = (int)std::min<int64_t>((c.d + span - 1) / span, grid_cap(c, 4));
  const size_t usm = sizeof(float) * gt::update_smem(k);
  SGEP_CUDA_TRY(smem_optin(k_update, gt::update_smem(k)));
  const UpdVariant var = next_variant(c);
  k_update<<<ublocks, kThreads, usm, s>>>(c.V, c.S, AV, BV, c.gram, c.d, k, eta, gamma, c.cfg.rho,
                                          c.cfg.eps_B, c.b_is_identity ? 1 : 0, c.Vtmp,
                                          c.cfg.debug ? c.grad : nullptr, var);
  SGEP_CUDA_TRY(cudaGetLastError());
  const int nblocks = (int)std::min<int64_t>((c.d * k + 255) / 256, grid_cap(c, 4));
  k_normalize<<<nblocks, 256, 0, s>>>(c.Vtmp, c.gram, c.V, c.d, k, c.dflag, var, gamma);
  SGEP_CUDA_TRY(cudaGetLastError());
  c.launches += 3;
  return SGEP_OK;
}

// Alg. 2 with M machines: acc_v += inv_m (v_i + eta grad_im) and acc_s += inv_m ([Bv]_i +
// gamma (B_tm v_i - [Bv]_i)) over the machines m, elementwise (both steps are affine in the
// machine's quantities, so this is the step with the averaged direction and increment).
__global__ void k_machine_accumulate(const float* __restrict__ vstep, const float* __restrict__ sstep,
                                     float* __restrict__ acc_v, float* __restrict__ acc_s, int64_t n, float inv_m) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    acc_v[e] = fmaf(inv_m, vstep[e], acc_v[e]);
    acc_s[e] = fmaf(inv_m, sstep[e], acc_s[e]);
  }
}

// Squared column norms of a d x k matrix, added into out[k] (zero on entry).
__global__ void k_col_norms(const float* __restrict__ A, int64_t d, int k, float* out) {
  const int i = threadIdx.x % k, lanes = blockDim.x / k, lr = threadIdx.x / k;
  if (lr >= lanes) return;
  float s2 = 0.f;
  for (int64_t r = (int64_t)blockIdx.x * lanes + lr; r < d; r += (int64_t)gridDim.x * lanes) {
    const float v = A[r * k + i];
    s2 = fmaf(v, v, s2);
  }
  atomicAdd(out + i, s2);
}

int generic_machines_step(Ctx& c, const void* X, const void* Y, int64_t b, cudaStream_t s, const float* sx,
                          const float* sy, float eta, float gamma) {
  const int M = c.cfg.machines, k = c.k, kk = k * k;
  const int64_t dk = c.d * k;
  float* accv = c.mach_buf;
  float* accs = accv + dk;
  float* Sm = accs + dk;  // the machine's [Bv] step (k_update steps its S argument in place)
  const size_t esz = elem_size(c);
  SGEP_CUDA_TRY(cudaMemsetAsync(accv, 0, 2 * (size_t)dk * sizeof(float), s));
  const int rows = std::max(1, kThreads / k);
  const int64_t span = (int64_t)rows * gt::kUpdRows;
  const int ublocks = (int)std::min<int64_t>((c.d + span - 1) / span, grid_cap(c, 4));
  const int gblocks = (int)std::min<int64_t>((c.d + 31) / 32, grid_cap(c, 2));
  const int eblocks = (int)std::min<int64_t>((dk + 255) / 256, grid_cap(c, 4));
  SGEP_CUDA_TRY(smem_optin(k_update, gt::update_smem(k)));
  for (int m = 0; m < M; ++m) {
    const int64_t r0 = b * m / M, r1 = b * (m + 1) / M;
    const char* xs = (const char*)X + (size_t)r0 * c.d_x * esz;
    const char* ys = c.has_y ? (const char*)Y + (size_t)r0 * c.d_y * esz : nullptr;
    int rc = generic_products(c, xs, ys, r1 - r0, s, sx ? sx + r0 : nullptr, sy ? sy + r0 : nullptr);
    if (rc) return rc;
    SGEP_CUDA_TRY(cudaMemsetAsync(c.gram, 0, sizeof(float) * (2 * kk + 2 * k), s));
    k_gram<<<gblocks, kThreads, sizeof(float) * gt::gram_smem(k), s>>>(c.V, c.S, c.acc, c.acc + dk, c.d, k,
                                                                       c.cfg.eps_B, c.b_is_identity ? 1 : 0, c.gram);
    SGEP_CUDA_TRY(cudaGetLastError());
    SGEP_CUDA_TRY(cudaMemcpyAsync(Sm, c.S, (size_t)dk * sizeof(float), cudaMemcpyDeviceToDevice, s));
    k_update<<<ublocks, kThreads, sizeof(float) * gt::update_smem(k), s>>>(
        c.V, Sm, c.acc, c.acc + dk, c.gram, c.d, k, eta, gamma, c.cfg.rho, c.cfg.eps_B, c.b_is_identity ? 1 : 0,
        c.Vtmp, nullptr, UpdVariant());
    SGEP_CUDA_TRY(cudaGetLastError());
    k_machine_accumulate<<<eblocks, 256, 0, s>>>(c.Vtmp, Sm, accv, accs, dk, 1.f / (float)M);
    SGEP_CUDA_TRY(cudaGetLastError());
    c.launches += 4;
  }
  // [Bv] <- the averaged step; V <- retraction of the averaged player step
  SGEP_CUDA_TRY(cudaMemcpyAsync(c.S, accs, (size_t)dk * sizeof(float), cudaMemcpyDeviceToDevice, s));
  float* norms = c.gram + 2 * kk + k;
  SGEP_CUDA_TRY(cudaMemsetAsync(norms, 0, (size_t)k * sizeof(float), s));
  const int lanes = std::max(1, 256 / k);
  k_col_norms<<<(unsigned)std::min<int64_t>((c.d + lanes - 1) / lanes, grid_cap(c, 2)), lanes * k, 0, s>>>(
      accv, c.d, k, norms);
  SGEP_CUDA_TRY(cudaGetLastError());
  k_normalize<<<eblocks, 256, 0, s>>>(accv, c.gram, c.V, c.d, k, c.dflag, UpdVariant(), 0.f);
  SGEP_CUDA_TRY(cudaGetLastError());
  c.launches += 2;
  c.debug_valid = 0;  // the update directions of the shards are not kept
  return SGEP_OK;
}

int generic_normalize(Ctx& c, cudaStream_t s) {
  const int nblocks = (int)std::min<int64_t>((c.d * c.k + 255) / 256, grid_cap(c, 4));
  k_normalize<<<nblocks, 256, 0, s>>>(c.Vtmp, c.gram, c.V, c.d, c.k, c.dflag, UpdVariant(), 0.f);
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

namespace sgep {

int ica_alloc(Ctx& c) {
  const size_t mb = (size_t)c.cfg.max_b, dk = (size_t)c.d * c.k;
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.ica_buf, (mb + 2 * mb * c.k + 2 * dk + 4) * sizeof(float)));
  return SGEP_OK;
}

// A_t V and B_t V of the ICA pencil (Sec. 1) from b rows: P = X V over every row, row norms
// w, the kurtosis term X_1^T (w . P_1) / n_1, U = B_3 V, tr = mean_2 w, W = B_2 U,
// A_t V = K - tr U - 2 W, B_t V = B_4 V. Quarters 1..4 of the rows when `split`, else all rows.
int ica_products(Ctx& c, const void* X, int64_t b, cudaStream_t s, const float* sx, bool split) {
  const int k = c.k;
  const size_t dk = (size_t)c.d * k, mb = (size_t)c.cfg.max_b;
  float* w = c.ica_buf;
  float* PW = w + mb;
  float* U = PW + 2 * mb * k;
  float* W = U + dk;
  float* tr = W + dk;
  float* AV = c.acc;
  float* BV = c.acc + dk;
  const int64_t q = split ? b / 4 : b;
  const int64_t lo[4] = {0, split ? q : 0, split ? 2 * q : 0, split ? 3 * q : 0};
  const int64_t nr[4] = {q, q, q, split ? b - 3 * q : b};
  SGEP_CUDA_TRY(cudaMemsetAsync(c.acc, 0, 2 * dk * sizeof(float), s));
  SGEP_CUDA_TRY(cudaMemsetAsync(U, 0, 2 * dk * sizeof(float), s));
  return by_dtype(c, [&](auto tag) {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    const T* Xt = static_cast<const T*>(X);
    auto rows = [&](int j) { return Xt + lo[j] * c.d_x; };
    auto rsc = [&](int j) { return sx ? sx + lo[j] : (const float*)nullptr; };
    int rc = launch_project_with<T>(c, Xt, b, c.V, c.PQ, s, sx);
    if (rc) return rc;
    const int64_t nw = split ? 2 * q : b;  // rows of the first two quarters
    k_row_sqnorm<T><<<(unsigned)std::min<int64_t>((nw + 7) / 8, 4 * c.num_sms), 256, 0, s>>>(Xt, nw, c.d_x, sx, w);
    SGEP_CUDA_TRY(cudaGetLastError());
    k_mean<<<1, 256, 0, s>>>(w + lo[1], nr[1], tr);
    SGEP_CUDA_TRY(cudaGetLastError());
    k_weight_rows<<<(unsigned)std::min<int64_t>((nr[0] * k + 255) / 256, 4 * c.num_sms), 256, 0, s>>>(
        c.PQ + lo[0] * 2 * k, w + lo[0], nr[0], k, PW);
    SGEP_CUDA_TRY(cudaGetLastError());
    c.launches += 3;
    rc = launch_bp_rows<T>(c, rows(0), nr[0], PW, AV, 1.f / (float)nr[0], s, rsc(0));
    if (!rc) rc = launch_bp_rows<T>(c, rows(2), nr[2], c.PQ + lo[2] * 2 * k, U, 1.f / (float)nr[2], s, rsc(2));
    if (!rc) rc = launch_bp_rows<T>(c, rows(3), nr[3], c.PQ + lo[3] * 2 * k, BV, 1.f / (float)nr[3], s, rsc(3));
    if (!rc) rc = launch_project_with<T>(c, rows(1), nr[1], U, PW, s, rsc(1));
    if (!rc) rc = launch_bp_rows<T>(c, rows(1), nr[1], PW, W, 1.f / (float)nr[1], s, rsc(1));
    if (rc) return rc;
    k_ica_combine<<<(unsigned)std::min<int64_t>(((int64_t)dk + 255) / 256, 4 * c.num_sms), 256, 0, s>>>(AV, U, W,
                                                                                                       tr, dk);
    SGEP_CUDA_TRY(cudaGetLastError());
    ++c.launches;
    return SGEP_OK;
  });
}

}  // namespace sgep

namespace sgep {

int centring_update(Ctx& c, const void* X, const void* Y, int64_t b, cudaStream_t s, const float* sx,
                    const float* sy) {
  const unsigned ysplit = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (b + 255) / 256));
  int rc = by_dtype(c, [&](auto tag) {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
    k_colsum<T><<<dim3((unsigned)((c.d_x + 255) / 256), ysplit), 256, 0, s>>>((const T*)X, b, c.d_x, sx, c.cen_sum);
    SGEP_CUDA_TRY(cudaGetLastError());
    if (c.has_y) {
      k_colsum<T><<<dim3((unsigned)((c.d_y + 255) / 256), ysplit), 256, 0, s>>>((const T*)Y, b, c.d_y, sy,
                                                                               c.cen_sum + c.d_x);
      SGEP_CUDA_TRY(cudaGetLastError());
    }
    return SGEP_OK;
  });
  if (rc) return rc;
  c.cen_count += (double)b;
  k_mean_from_sums<<<(unsigned)std::min<int64_t>((c.d + 255) / 256, 4 * c.num_sms), 256, 0, s>>>(
      c.cen_sum, c.d, c.cen_count, c.cen_mean);
  SGEP_CUDA_TRY(cudaGetLastError());
  c.launches += c.has_y ? 3 : 2;
  return SGEP_OK;
}

}  // namespace sgep

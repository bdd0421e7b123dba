// Tensor-core (tcgen05) path of the gamma-EigenGame products for BF16 minibatches
// with large d, plus a self-test of the MMA operand layouts it relies on.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "eg_math.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace sgep {

// ---------------------------------------------------------------------------
// Tensor maps (cuTensorMapEncodeTiled through the runtime's driver entry point)

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 2-D BF16 row-major matrix [rows][cols] (row stride `ld` elements); boxes of
// box_rows x box_cols with 128-byte swizzle (box_cols * 2 must be 128).
int make_map_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                  int box_cols) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available");
    return SGEP_ECUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SGEP_ECUDA;
  }
  return SGEP_OK;
}

// FP32 row-major matrix [rows][cols], boxes of box_rows x box_cols (box_cols * 4 <= 128 bytes)
// with 128-byte swizzle.
int make_map_f32(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                 int box_cols) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available");
    return SGEP_ECUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SGEP_ECUDA;
  }
  return SGEP_OK;
}

// 3-D view of a BF16 row-major matrix [rows][cols] (row stride `ld` elements) as (64 columns,
// rows, cols / 64 column groups): one box of box_rows rows x `groups` groups lands as `groups`
// consecutive [box_rows][64] sub-boxes with 128-byte swizzle, the layout of that many 2-D boxes
// of 64 columns, in one copy. Returns SGEP_ECUDA when the CUDA driver does not take the view.
int make_map_bf16_groups(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                         int groups) {
  auto fn = encode_fn();
  if (!fn || cols % 64) return SGEP_ECUDA;
  cuuint64_t dims[3] = {64, (cuuint64_t)rows, (cuuint64_t)(cols / 64)};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, 128};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, (cuuint32_t)groups};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SGEP_OK : SGEP_ECUDA;
}

namespace {

using namespace tc;

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// ---------------------------------------------------------------------------
// Self-test: one 128 x 64 x 64 product through TMA + tcgen05 + TMEM.
//  mode 0: D[r][n] = sum_k A[r][k] Bt[n][k], A K-major ([128][64] row-major)
//  mode 1: D[c][n] = sum_r T[r][c] Bt[n][r], A = T^T MN-major (T [64][128] row-major),
//          descriptor LBO = stride between 64-column groups, SBO = 8-row groups
//  mode 2: as mode 1 with the two strides exchanged
// Every address the descriptors can reach stays inside the 32 KB A region.
__global__ void __launch_bounds__(128) k_tc_selftest(const __grid_constant__ CUtensorMap mapA,
                                                     const __grid_constant__ CUtensorMap mapB, int mode,
                                                     float* __restrict__ out, int* flag) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint8_t* As = base;               // 32 KB
  uint8_t* Bs = base + 32768;       // 8 KB
  uint64_t* full = (uint64_t*)(base + 40960);
  uint64_t* done = full + 1;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* issued = (int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid / 32;
  if (warp == 0) {
    tmem_alloc(tmem_slot, 64);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(full, 1);
    mbar_init(done, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  if (tid == 0) {
    mbar_arrive_expect_tx(full, 16384 + 8192);
    if (mode == 0) {
      tma_load_2d(As, &mapA, 0, 0, full);
    } else {
      tma_load_2d(As, &mapA, 0, 0, full);
      tma_load_2d(As + 8192, &mapA, 64, 0, full);
    }
    tma_load_2d(Bs, &mapB, 0, 0, full);
    ok = mbar_wait(full, 0);
    if (ok) {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16(128, 64, mode == 0 ? 0 : 1, 0);
      for (int kk = 0; kk < 4; ++kk) {
        uint64_t a;
        if (mode == 0) a = desc_sw128(As + kk * 32, 16, 1024);
        else if (mode == 1) a = desc_sw128(As + kk * 2048, 8192, 1024);
        else a = desc_sw128(As + kk * 2048, 1024, 8192);
        const uint64_t b = desc_sw128(Bs + kk * 32, 16, 1024);
        mma_bf16(tmem, a, b, idesc, kk > 0 ? 1u : 0u);
      }
      mma_commit(done);
    } else {
      atomicOr(flag, kFlagTimeout);
    }
    *issued = ok ? 1 : 0;
  }
  __syncthreads();
  if (*issued) {
    const bool ready = mbar_wait(done, 0, 500000000ull);
    if (!ready) {
      if ((tid & 31) == 0) atomicOr(flag, kFlagTimeout);
    } else {
      tc_fence_after();
      const int q = warp & 3;
      float v[32];
      const int row = 32 * q + (tid & 31);
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16), v);
#pragma unroll
      for (int j = 0; j < 32; ++j) out[row * 64 + j] = v[j];
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) out[row * 64 + 32 + j] = v[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 64);
}

__global__ void k_fill_bf16(__nv_bfloat16* p, int n, uint32_t seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    p[i] = __float2bfloat16(((float)(h & 0xFFFF) / 32768.f) - 1.f);
  }
}

__global__ void k_selftest_ref(const __nv_bfloat16* A, const __nv_bfloat16* Bt, int mode, float* ref) {
  const int m = blockIdx.x, n = threadIdx.x;  // 128 x 64
  float s = 0.f;
  for (int kx = 0; kx < 64; ++kx) {
    const float a = mode == 0 ? __bfloat162float(A[m * 64 + kx]) : __bfloat162float(A[kx * 128 + m]);
    s = fmaf(a, __bfloat162float(Bt[n * 64 + kx]), s);
  }
  ref[m * 64 + n] = s;
}


// ---------------------------------------------------------------------------
// Products of one BF16 minibatch on the tensor cores.
//
// V (FP32) is split per element into a BF16 pair v = hi + lo (hi = bf16(v),
// lo = bf16(v - hi)), so X V is computed from 2k BF16 columns and summed in FP32;
// the pair keeps about 16 significant bits of V. The same split is used for the
// row projections P and Q that feed the back-projection.
//
//   k_tc_prep_v   Vt = [hi(V)^T ; lo(V)^T]  (64 x d BF16, players padded to 32)
//   k_tc_project  P = X V_x, Q = Y V_y      (tcgen05, rows in tiles of 128,
//                 columns split in S parts; partial tiles added with float4 atomics)
//   k_tc_prep_w   Pt = [hi(P)^T ; lo(P)^T], Qt likewise (64 x b BF16)
//   k_tc_backproject  A_t V = [X_A^T Q_A ; Y_A^T P_A] / n_A, B_t V = [X_B^T P_B ; Y_B^T Q_B] / n_B
//                 (tcgen05 with the row-major minibatch tile read transposed,
//                 CTAs own 256-column slices, accumulators stay in tensor memory,
//                 rows streamed last-first so the rows the projection read last are
//                 still in L2)

constexpr int kTcThreads = 192;     // warp 0: TMA, warp 1: MMA, warps 2-5: epilogue
constexpr int kP_Stages = 8;        // projection: 24 KB per stage
constexpr int kB_Stages = 5;        // back-projection: 40 KB per stage
constexpr int kTcKP = 32;           // players padded to 32 (N = 64 with hi/lo)

struct TcProjArgs {
  int64_t b, d_x, d_y;
  int splits;        // column splits per view
  int64_t cols_per_split;
  float* P;          // b x 32
  float* Q;          // b x 32
  int* dflag;
};

// V split into BF16 pairs (transposed, players padded to 32) and the d-side terms
// G_ij = <v_i, [Bv]_j>, vv_i = |v_i|^2 of the update, accumulated per block of 64 rows of V.
// grid: d/64 blocks of 256 threads. Gout (k*k) and vvout (k) must be zero on entry.
__global__ void __launch_bounds__(256) k_tc_prep_v(const float* __restrict__ V, const float* __restrict__ S,
                                                   int64_t d, int k, __nv_bfloat16* __restrict__ Vt,
                                                   float* __restrict__ Gout, float* __restrict__ vvout) {
  __shared__ float vs[64][kTcKP + 1];
  __shared__ float ss[64][kTcKP + 1];
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * 64;
  {
    // all loads of the block in flight before the first store (8 rows per thread)
    float rv[8], rs[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + 256 * u;
      const int r = e / kTcKP, i = e % kTcKP;
      const bool ok = c0 + r < d && i < k;
      rv[u] = ok ? __ldg(V + (c0 + r) * k + i) : 0.f;
      rs[u] = ok ? __ldg(S + (c0 + r) * k + i) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + 256 * u;
      vs[e / kTcKP][e % kTcKP] = rv[u];
      ss[e / kTcKP][e % kTcKP] = rs[u];
    }
  }
  __syncthreads();
  // transposed BF16 pairs: consecutive threads write consecutive columns
  for (int e = tid; e < 2 * kTcKP * 64; e += 256) {
    const int n = e / 64, r = e % 64;
    if (c0 + r >= d) continue;
    const float v = vs[r][n % kTcKP];
    const __nv_bfloat16 hi = __float2bfloat16(v);
    Vt[(int64_t)n * d + c0 + r] = n < kTcKP ? hi : __float2bfloat16(v - __bfloat162float(hi));
  }
  const int kk = k * k;
  for (int p = tid; p < kk + k; p += 256) {
    float s0 = 0.f, s1 = 0.f;
    if (p < kk) {
      const int i = p / k, j = p % k;
      for (int r = 0; r < 64; r += 2) {
        s0 = fmaf(vs[r][i], ss[r][j], s0);
        s1 = fmaf(vs[r + 1][i], ss[r + 1][j], s1);
      }
      atomicAdd(&Gout[p], s0 + s1);
    } else {
      const int i = p - kk;
      for (int r = 0; r < 64; r += 2) {
        s0 = fmaf(vs[r][i], vs[r][i], s0);
        s1 = fmaf(vs[r + 1][i], vs[r + 1][i], s1);
      }
      atomicAdd(&vvout[i], s0 + s1);
    }
  }
}

// P, Q split into BF16 pairs (transposed, row stride ldt; skipped when Pt is null) and the
// row-side terms a_ij = sum_A (P_i Q_j + Q_i P_j) / n_A, b_i = sum_B (P_i^2 + Q_i^2) / n_B.
// grid: b/16 blocks of 256 threads (16 rows each; the split point is a multiple of 64).
// aout (k*k) and bout (k) must be zero on entry.
__global__ void __launch_bounds__(256) k_tc_prep_w(const float* __restrict__ P, const float* __restrict__ Q,
                                                   int64_t b, int64_t ldt, int64_t nA, int k, float inv_nA,
                                                   float inv_nB, __nv_bfloat16* __restrict__ Pt,
                                                   __nv_bfloat16* __restrict__ Qt, float* __restrict__ aout,
                                                   float* __restrict__ bout) {
  constexpr int R = 16;
  __shared__ float ps[R][kTcKP + 1];
  __shared__ float qs[R][kTcKP + 1];
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  {
    float rp[2], rq[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + 256 * u;
      const int r = e / kTcKP, i = e % kTcKP;
      const bool ok = r0 + r < b;
      rp[u] = ok ? __ldcg(P + (r0 + r) * kTcKP + i) : 0.f;
      rq[u] = ok ? __ldcg(Q + (r0 + r) * kTcKP + i) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + 256 * u;
      ps[e / kTcKP][e % kTcKP] = rp[u];
      qs[e / kTcKP][e % kTcKP] = rq[u];
    }
  }
  __syncthreads();
  for (int e = tid; Pt != nullptr && e < 2 * kTcKP * R; e += 256) {
    const int n = e / R, r = e % R;
    if (r0 + r >= b) continue;
    const float p = ps[r][n % kTcKP], q = qs[r][n % kTcKP];
    const __nv_bfloat16 ph = __float2bfloat16(p), qh = __float2bfloat16(q);
    Pt[(int64_t)n * ldt + r0 + r] = n < kTcKP ? ph : __float2bfloat16(p - __bfloat162float(ph));
    Qt[(int64_t)n * ldt + r0 + r] = n < kTcKP ? qh : __float2bfloat16(q - __bfloat162float(qh));
  }
  const bool rowsA = r0 < nA;
  const int kk = k * k;
  for (int p = tid; p < kk + k; p += 256) {
    float s0 = 0.f, s1 = 0.f;
    if (p < kk && rowsA) {
      const int i = p / k, j = p % k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        s0 = fmaf(ps[r][i], qs[r][j], s0);
        s1 = fmaf(qs[r][i], ps[r][j], s1);
      }
      atomicAdd(&aout[p], (s0 + s1) * inv_nA);
    } else if (p >= kk && !rowsA) {
      const int i = p - kk;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        s0 = fmaf(ps[r][i], ps[r][i], s0);
        s1 = fmaf(qs[r][i], qs[r][i], s1);
      }
      atomicAdd(&bout[i], (s0 + s1) * inv_nB);
    }
  }
}

// Update of large-d problems (k <= 32): one warp per row c of V, lane i = player i, so every
// load and store is one 128-byte row; [Bv]_j of the row reach lane i by shuffles. Each block
// forms the coefficients of Eq. (update) from the k x k terms (with 1/max(G_jj, rho) once per j).
// Writes v + eta grad to Vtmp, the [Bv] step to S, and adds per-block column sums of
// (v + eta grad)^2 into the norms. gram: a | G | b | norms | vv.
__global__ void __launch_bounds__(256) k_tc_update(const float* __restrict__ V, float* __restrict__ S,
                                                   const float* __restrict__ AV, const float* __restrict__ BV,
                                                   const float* __restrict__ a, const float* __restrict__ bterm,
                                                   const float* __restrict__ G, const float* __restrict__ vv,
                                                   float* __restrict__ norms, int64_t d, int k, float rho,
                                                   float eta, float gamma, float eps_B,
                                                   float* __restrict__ Vtmp, float* __restrict__ grad_out) {
  __shared__ float T[kTcKP * kTcKP];
  __shared__ float cb[kTcKP], cac[kTcKP], inv_s[kTcKP];
  __shared__ float red[8][kTcKP];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int kk = k * k;
  if (tid < k) {
    inv_s[tid] = 1.f / fmaxf(G[tid * k + tid], rho);
    cb[tid] = fmaf(eps_B, vv[tid], bterm[tid]);
  }
  __syncthreads();
  for (int p = tid; p < kk; p += 256) {
    const int j = p / k, i = p % k;
    T[j * kTcKP + i] = j < i ? cb[i] * a[i * k + j] * inv_s[j] : 0.f;
  }
  if (tid < k) {
    float c = 0.f;
    for (int j = 0; j < tid; ++j) c = fmaf(a[tid * k + j] * G[tid * k + j], inv_s[j], c);
    cac[tid] = a[tid * k + tid] - c;
  }
  __syncthreads();
  const bool on = lane < k;
  float nr = 0.f;
  constexpr int U = 4;
  float v[U], sv[U], av[U], bv[U];
  int64_t g[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t c = (int64_t)blockIdx.x * (8 * U) + wid + 8 * u;
    g[u] = c * k + lane;
    const bool ok = on && c < d;
    v[u] = ok ? V[g[u]] : 0.f;
    sv[u] = ok ? S[g[u]] : 0.f;
    av[u] = ok ? AV[g[u]] : 0.f;
    bv[u] = ok ? BV[g[u]] : 0.f;
  }
  float pen[U];
#pragma unroll
  for (int u = 0; u < U; ++u) pen[u] = 0.f;
  for (int j = 0; j < k; ++j) {
    const float t = T[j * kTcKP + lane];
#pragma unroll
    for (int u = 0; u < U; ++u) pen[u] = fmaf(__shfl_sync(0xffffffffu, sv[u], j), t, pen[u]);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t c = (int64_t)blockIdx.x * (8 * U) + wid + 8 * u;
    if (!on || c >= d) continue;
    const float bve = fmaf(eps_B, v[u], bv[u]);
    const float gr = cb[lane] * av[u] - cac[lane] * bve - pen[u];
    const float vn = fmaf(eta, gr, v[u]);
    Vtmp[g[u]] = vn;
    S[g[u]] = fmaf(gamma, bve - sv[u], sv[u]);
    if (grad_out) grad_out[g[u]] = gr;
    nr = fmaf(vn, vn, nr);
  }
  red[wid][lane] = nr;
  __syncthreads();
  if (tid < k) {
    float s2 = 0.f;
    for (int w = 0; w < 8; ++w) s2 += red[w][tid];
    atomicAdd(&norms[tid], s2);
  }
}

// v_i <- v'_i / |v'_i|, four elements per thread (k is a multiple of 4 here).
__global__ void k_tc_normalize(const float* __restrict__ Vtmp, const float* __restrict__ norms,
                               float* __restrict__ V, int64_t n4, int k, int* dflag) {
  __shared__ float inv[kTcKP];
  if (threadIdx.x < k) inv[threadIdx.x] = 1.f / sqrtf(norms[threadIdx.x]);
  __syncthreads();
  const float4* src = reinterpret_cast<const float4*>(Vtmp);
  float4* dst = reinterpret_cast<float4*>(V);
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
    float4 v = src[e];
    const int i = (int)((e * 4) % k);
    v.x *= inv[i];
    v.y *= inv[i + 1];
    v.z *= inv[i + 2];
    v.w *= inv[i + 3];
    bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
    dst[e] = v;
  }
  if (bad) atomicOr(dflag, kFlagNonFinite);
}

// Update, retraction and the next step's V-side preparation in one launch, for
// large-d problems (k <= 32). Blocks of 256 threads own 128 rows of V; all blocks
// are resident (cooperative launch) and meet at one grid barrier.
//   phase 1: coefficients of Eq. (update) from a, G, b (and |v_i|^2 when eps_B > 0);
//            v' = v + eta grad and the [Bv] step S' = S + gamma (BV - S) per row, kept in
//            shared memory; the block's column sums of v'^2 are added into norms[slot]
//            (one atomic per column) and its partial of U = V'^T S' is stored.
//   barrier;
//   phase 2: v = v' / |v'| written out with its BF16 hi/lo pairs (the next step's
//            transposed V operand); block j adds a slice of the U partials over all blocks:
//            the next step's G = V^T S' = diag(1/|v'|) U, and |v_i|^2 = |v'_i|^2 / |v'_i|^2.
// The k x k terms are double-buffered by step parity: this launch reads slot `slot` and
// writes slot 1 - slot. After the barrier block 0 clears a and b (accumulated by the next
// step's products) and norms[1 - slot] (accumulated by the next update).
struct TcUpdArgs {
  const float* V;
  float* Vout;
  float* S;
  const float* AV;
  const float* BV;
  float* terms;   // a (kk) | b (k) | norms [2][k] | G [2][kk] | vv [2][k]
  float* part;    // per-block partials of U: [grid][32 * 32]
  float* dbg;     // a | G | b as used by this update (debug), or null
  float* grad_out;
  __nv_bfloat16* Vt;
  int64_t d;
  int k, slot;
  float rho, eta, gamma, eps_B;
  unsigned long long* bar;  // grid-barrier arrivals (monotone)
  unsigned long long bar_target;  // arrivals that complete this launch's barrier
  unsigned long long bar_ns;      // how long a block waits at the barrier before giving up
  int* dflag;
  unsigned long long* trace;  // [grid][8] globaltimer stamps of the phases, or null
  UpdVariant var;             // Adam on the players / Alg. 3 denominators, or plain Alg. 2
};

// acc[a][c] += x[a] y[c]: one 4 x 4 outer product.
__device__ __forceinline__ void tc_fma4x4(float (&acc)[4][4], const float4 x, const float4 y) {
  const float xa[4] = {x.x, x.y, x.z, x.w};
  const float ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(xa[a], ya[c], acc[a][c]);
}

// Bounded grid barrier: returns false (and flags a timeout) when the wait gives up.
__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, unsigned long long target, int* flag,
                                             int* ok_s, unsigned long long ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1ull);
    *ok_s = tc::spin_until_geq64(bar, target, ns) ? 1 : 0;
    if (!*ok_s) atomicOr(flag, kFlagTimeout);
  }
  __syncthreads();
  return *ok_s != 0;
}

// kVar: the Adam / Alg. 3 code is compiled in (the plain Alg. 2 update keeps its registers).
template <bool kVar>
__global__ void __launch_bounds__(256, 2) k_tc_update_fused(const TcUpdArgs u) {
  constexpr int R = 128;
  constexpr int KP = kTcKP;
  constexpr int SP = KP + 4;  // row stride of vs / ss: float4-aligned rows, 9 float4 (odd) per row
  static_assert(KP == 32 && R == 128, "micro-tile mappings below assume 32 players and 128 rows");
  __shared__ __align__(16) float T[KP * KP];
  __shared__ float cb[KP], cac[KP], inv_s[KP], inv_n[KP], nsq[KP], gdiag[KP];
  __shared__ float red[8][KP];
  __shared__ __align__(16) float vs[R][SP];
  __shared__ __align__(16) float ss[R][SP];
  __shared__ int ok_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int k = u.k, kk = k * k, slot = u.slot;
  const int nblk = (int)gridDim.x;
  auto stamp = [&](int ph) {
    if (u.trace && tid == 0) u.trace[blockIdx.x * 8 + ph] = tc::globaltimer();
  };
  stamp(0);
  float* a = u.terms;
  float* bt = a + kk;
  float* nrm = bt + k;             // [2][k]
  float* Gs = nrm + 2 * k;         // [2][kk]
  float* vvs = Gs + 2 * kk;        // [2][k]
  const float* G = Gs + slot * kk;
  const float* vv = vvs + slot * k;
  float* nsum = nrm + slot * k;    // column sums of v'^2 of this update (zero on entry)
  float* part_t = u.part;          // [nblk][KP * KP]
  const bool on = lane < k;
  const int64_t c0 = (int64_t)blockIdx.x * R;
  constexpr int U = 16;
  float v[U], sv[U], av[U], bv[U];
  {
    // a and G staged in shared memory (vs and ss are free until phase 1). Their loads go
    // first, then phase 1's rows (16 per warp), whose latency overlaps the coefficients'
    // setup (V, S and the Adam moments are not written by the products; AV and BV are
    // complete at launch).
    // Every block reads the same a and G, so their loads are as few and as wide as possible
    // (one float4 of each per thread when aligned: these hot lines are request-bound in L2).
    // Both are staged transposed (At[j k + i] = a_ij), so the reads below that walk a row of
    // a or G across the lanes (lane = i) hit consecutive banks.
    float* At = &vs[0][0];
    float* Gt = &ss[0][0];
    const bool vec = (kk % 4 == 0) && ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(G)) & 15) == 0;
    float xa[4], xg[4];
    if (vec) {
      const bool in = 4 * tid < kk;
      const float4 a4 = in ? __ldcg(reinterpret_cast<const float4*>(a) + tid) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 g4 = in ? __ldcg(reinterpret_cast<const float4*>(G) + tid) : make_float4(0.f, 0.f, 0.f, 0.f);
      xa[0] = a4.x, xa[1] = a4.y, xa[2] = a4.z, xa[3] = a4.w;
      xg[0] = g4.x, xg[1] = g4.y, xg[2] = g4.z, xg[3] = g4.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int p = tid + 256 * q;
        xa[q] = p < kk ? __ldcg(a + p) : 0.f;
        xg[q] = p < kk ? __ldcg(G + p) : 0.f;
      }
    }
    const float xb = tid < k ? __ldcg(bt + tid) : 0.f;
    const float xv = tid < k ? __ldcg(vv + tid) : 0.f;
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int r = wid + 8 * q;
      const int64_t g = (c0 + r) * k + lane;
      const bool ok = on && c0 + r < u.d;
      v[q] = ok ? u.V[g] : 0.f;  // plain load: this launch rewrites V
      sv[q] = ok ? u.S[g] : 0.f;
      av[q] = ok ? __ldcg(u.AV + g) : 0.f;
      bv[q] = ok ? __ldcg(u.BV + g) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = vec ? 4 * tid + q : tid + 256 * q;  // element p = i k + j of a and G
      if (p < kk) {
        const int t = (p % k) * k + p / k;
        At[t] = xa[q];
        Gt[t] = xg[q];
      }
    }
    if (tid < k) cb[tid] = fmaf(u.eps_B, xv, xb);
    __syncthreads();
    if (tid < k) {
      gdiag[tid] = Gt[tid * k + tid];  // <v_i, [Bv]_i> of step t (Alg. 3's z step)
      inv_s[tid] = 1.f / ((kVar && u.var.z) ? smooth_den(u.var.z[tid], u.var.log_rho, u.var.log_nu)
                                            : fmaxf(Gt[tid * k + tid], u.rho));
    }
    __syncthreads();
    for (int p = tid; p < KP * KP; p += 256) {  // zero outside k x k: read by the micro-tiles
      const int j = p / KP, i = p % KP;
      T[p] = (i < k && j < i) ? cb[i] * At[j * k + i] * inv_s[j] : 0.f;
    }
    if (tid < k) {
      float c = 0.f;
      for (int j = 0; j < tid; ++j) c = fmaf(At[j * k + tid] * Gt[j * k + tid], inv_s[j], c);
      cac[tid] = At[tid * k + tid] - c;
    }
    if (blockIdx.x == 0 && u.dbg) {  // the terms as used (debug), untransposed
      for (int p = tid; p < kk; p += 256) {
        const int t = (p % k) * k + p / k;
        u.dbg[p] = At[t];
        u.dbg[kk + p] = Gt[t];
      }
      if (tid < k) u.dbg[2 * kk + tid] = xb;
    }
    __syncthreads();
  }
  stamp(3);
  // ---- phase 1 (rows loaded above) ---------------------------------------------
  float nr = 0.f;
  {
    float am[kVar ? U : 1], as2[kVar ? U : 1];  // Adam moments of the rows
    if constexpr (kVar) {
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int r = wid + 8 * q;
        const int64_t g = (c0 + r) * k + lane;
        const bool ok = u.var.m && on && c0 + r < u.d;
        am[q] = ok ? u.var.m[g] : 0.f;
        as2[q] = ok ? u.var.s[g] : 0.f;
      }
    }
    // penalty PEN = S T over the block's rows (T_ji = 0 unless j < i): the old S rows in ss,
    // thread -> rows pr + 32a (a < 4) x players 4pc..4pc+3, result into vs
#pragma unroll
    for (int q = 0; q < U; ++q) ss[wid + 8 * q][lane] = sv[q];
    __syncthreads();
    {
      const int pr = tid & 31, pc = tid >> 5;
      float pacc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) pacc[a][c] = 0.f;
      for (int j0 = 0; j0 < k; j0 += 4) {
        float4 s4[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) s4[a] = *reinterpret_cast<const float4*>(&ss[pr + 32 * a][j0]);
        const float4 t0 = *reinterpret_cast<const float4*>(&T[(j0 + 0) * KP + 4 * pc]);
        const float4 t1 = *reinterpret_cast<const float4*>(&T[(j0 + 1) * KP + 4 * pc]);
        const float4 t2 = *reinterpret_cast<const float4*>(&T[(j0 + 2) * KP + 4 * pc]);
        const float4 t3 = *reinterpret_cast<const float4*>(&T[(j0 + 3) * KP + 4 * pc]);
        tc_fma4x4(pacc, make_float4(s4[0].x, s4[1].x, s4[2].x, s4[3].x), t0);
        tc_fma4x4(pacc, make_float4(s4[0].y, s4[1].y, s4[2].y, s4[3].y), t1);
        tc_fma4x4(pacc, make_float4(s4[0].z, s4[1].z, s4[2].z, s4[3].z), t2);
        tc_fma4x4(pacc, make_float4(s4[0].w, s4[1].w, s4[2].w, s4[3].w), t3);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
        *reinterpret_cast<float4*>(&vs[pr + 32 * a][4 * pc]) =
            make_float4(pacc[a][0], pacc[a][1], pacc[a][2], pacc[a][3]);
    }
    __syncthreads();
    stamp(4);
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int r = wid + 8 * q;
      const int64_t g = (c0 + r) * k + lane;
      const bool ok = on && c0 + r < u.d;
      const float bve = fmaf(u.eps_B, v[q], bv[q]);
      const float gr = cb[lane] * av[q] - cac[lane] * bve - vs[r][lane];
      float step = gr;
      if constexpr (kVar) {
        if (u.var.m) step = adam_increment(gr, am[q], as2[q], u.var.b1, u.var.b2, u.var.eps, u.var.bc1, u.var.bc2);
      }
      const float vn = ok ? fmaf(u.eta, step, v[q]) : 0.f;
      const float sn = ok ? fmaf(u.gamma, bve - sv[q], sv[q]) : 0.f;
      if (ok) {
        u.S[g] = sn;
        if (u.grad_out) u.grad_out[g] = gr;
        if constexpr (kVar) {
          if (u.var.m) {
            u.var.m[g] = am[q];
            u.var.s[g] = as2[q];
          }
        }
      }
      vs[r][lane] = vn;
      ss[r][lane] = sn;
      nr = fmaf(vn, vn, nr);
    }
  }
  stamp(6);
  red[wid][lane] = nr;
  __syncthreads();
  if (tid < k) {
    float s2 = 0.f;
    for (int w = 0; w < 8; ++w) s2 += red[w][tid];
    atomicAdd(nsum + tid, s2);
  }
  stamp(7);
  {
    // the block's partial of U = V'^T S': thread -> rows 4iq..4iq+3 x columns 4jq..4jq+3 of
    // U over the block rows rs, rs + 4, ...; the four row splits (lanes xor 8, 16) are added
    const int jq = tid & 7, rs = (tid >> 3) & 3, iq = tid >> 5;
    float uacc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) uacc[a][c] = 0.f;
#pragma unroll 4
    for (int r = rs; r < R; r += 4)
      tc_fma4x4(uacc, *reinterpret_cast<const float4*>(&vs[r][4 * iq]),
                *reinterpret_cast<const float4*>(&ss[r][4 * jq]));
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uacc[a][c] += __shfl_xor_sync(0xffffffffu, uacc[a][c], 8);
        uacc[a][c] += __shfl_xor_sync(0xffffffffu, uacc[a][c], 16);
      }
    if (rs == 0) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
        *reinterpret_cast<float4*>(part_t + (size_t)blockIdx.x * KP * KP + (4 * iq + a) * KP + 4 * jq) =
            make_float4(uacc[a][0], uacc[a][1], uacc[a][2], uacc[a][3]);
    }
  }
  stamp(1);
  if (!grid_barrier(u.bar, u.bar_target, u.dflag, &ok_s, u.bar_ns)) return;
  stamp(2);
  // this block's entries [e0, e0 + ne) of U: the first entry of each warp has its partials
  // (lanes over the first 256 blocks) in flight together with the norms
  const int per = (KP * KP + nblk - 1) / nblk;
  const int e0 = (int)blockIdx.x * per;
  const int ne = max(0, min(per, KP * KP - e0));
  float x0[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int blk = lane + 32 * q;
    x0[q] = (wid < ne && blk < nblk) ? __ldcg(part_t + (size_t)blk * KP * KP + e0 + wid) : 0.f;
  }
  if (blockIdx.x == 0) {  // every block has read a, b and z: clear a, b and next update's sums
    for (int p = tid; p < kk; p += 256) a[p] = 0.f;
    if (tid < k) {
      bt[tid] = 0.f;
      nrm[(1 - slot) * k + tid] = 0.f;
      if (kVar && u.var.z)
        u.var.z[tid] = smooth_z_step(u.var.z[tid], gdiag[tid], u.gamma, u.var.log_rho, u.var.log_nu);
    }
  }
  if (tid < KP) {
    const float s2 = tid < k ? __ldcg(nsum + tid) : 0.f;
    nsq[tid] = s2;
    inv_n[tid] = tid < k ? 1.f / sqrtf(s2) : 0.f;
  }
  __syncthreads();
  // ---- phase 2 -----------------------------------------------------------------
  bool bad = false;
  for (int e = tid; e < R * KP; e += 256) {
    const int r = e / KP, i = e % KP;
    const float v = vs[r][i] * inv_n[i];
    vs[r][i] = v;
    if (i < k && c0 + r < u.d) {
      u.Vout[(c0 + r) * k + i] = v;
      bad |= !isfinite(v);
    }
  }
  if (bad) atomicOr(u.dflag, kFlagNonFinite);
  __syncthreads();
  // transposed BF16 pairs: thread -> (four operand rows 4nq..4nq+3, two consecutive rows
  // of V), one float4 of each V row (operand rows n < KP: hi parts of column n; n >= KP:
  // lo parts of column n - KP)
  for (int e = tid; e < (2 * KP / 4) * (R / 2); e += 256) {
    const int nq = e / (R / 2), rp = 2 * (e % (R / 2));
    if (c0 + rp >= u.d) continue;  // d is even: rp + 1 < d as well
    const float4 x4 = *reinterpret_cast<const float4*>(&vs[rp][4 * (nq % (KP / 4))]);
    const float4 y4 = *reinterpret_cast<const float4*>(&vs[rp + 1][4 * (nq % (KP / 4))]);
    const float xs4[4] = {x4.x, x4.y, x4.z, x4.w}, ys4[4] = {y4.x, y4.y, y4.z, y4.w};
    const bool lo = nq >= KP / 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float v0 = xs4[c], v1 = ys4[c];
      __nv_bfloat162 w;
      if (!lo) {
        w = __floats2bfloat162_rn(v0, v1);
      } else {
        const float h0 = __bfloat162float(__float2bfloat16(v0)), h1 = __bfloat162float(__float2bfloat16(v1));
        w = __floats2bfloat162_rn(v0 - h0, v1 - h1);
      }
      *reinterpret_cast<__nv_bfloat162*>(u.Vt + (int64_t)(4 * nq + c) * u.d + c0 + rp) = w;
    }
  }
  // entries [j per, (j + 1) per) of U over all blocks -> the next step's G and |v|^2
  {
    float* Gn = Gs + (1 - slot) * kk;
    for (int el = wid; el < ne; el += 8) {  // warp per entry, lanes over the blocks
      float s2 = 0.f;
      int blk_start = lane;
      if (el == wid) {  // partials of the first 256 blocks already loaded
#pragma unroll
        for (int q = 0; q < 8; ++q) s2 += x0[q];
        blk_start = lane + 256;
      }
      for (int blk0 = blk_start; blk0 < nblk; blk0 += 256) {
        float x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int blk = blk0 + 32 * q;
          x[q] = blk < nblk ? __ldcg(part_t + (size_t)blk * KP * KP + e0 + el) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) s2 += x[q];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      const int te = e0 + el, i = te / KP, j = te % KP;
      if (lane == 0 && i < k && j < k) Gn[i * k + j] = inv_n[i] * s2;
    }
    if (blockIdx.x == 0 && tid < k) vvs[(1 - slot) * k + tid] = nsq[tid] * inv_n[tid] * inv_n[tid];
  }
  stamp(5);
}

// grid: (b/128 row tiles, 2 views, splits)
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_project(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
                 const __grid_constant__ CUtensorMap mapVt, const TcProjArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  constexpr int kA = 16384, kB = 8192, kStage = kA + kB;
  uint64_t* full = (uint64_t*)(base + kP_Stages * kStage);
  uint64_t* empty = full + kP_Stages;
  uint64_t* done = empty + kP_Stages;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* abort_flag = (int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  const int view = blockIdx.y;
  const int64_t row0 = (int64_t)blockIdx.x * 128;
  const int64_t c0 = (int64_t)blockIdx.z * a.cols_per_split;
  const int nk = (int)(a.cols_per_split / 64);
  const CUtensorMap* mZ = view ? &mapY : &mapX;
  const int64_t voff = view ? a.d_x : 0;

  if (warp == 1) {
    tmem_alloc(tmem_slot, 64);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kP_Stages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tensormap(mZ);
    prefetch_tensormap(&mapVt);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    const uint64_t keep = policy_evict_last();
    for (int ks = 0; ks < nk; ++ks) {
      const int st = ks % kP_Stages;
      if (ks >= kP_Stages && !mbar_wait(empty + st, ((ks / kP_Stages) - 1) & 1)) {
        atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        break;
      }
      if (*(volatile int*)abort_flag) break;
      uint8_t* sa = base + st * kStage;
      mbar_arrive_expect_tx(full + st, kStage);
      tma_load_2d(sa, mZ, (int)(c0 + (int64_t)ks * 64), (int)row0, full + st);
      tma_load_2d_hint(sa + kA, &mapVt, (int)(voff + c0 + (int64_t)ks * 64), 0, full + st, keep);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16(128, 64, 0, 0);
    bool ok = true;
    for (int ks = 0; ks < nk; ++ks) {
      const int st = ks % kP_Stages;
      if (!mbar_wait(full + st, (ks / kP_Stages) & 1)) {
        atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      uint8_t* sa = base + st * kStage;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma_bf16(tmem, desc_sw128(sa + kk * 32, 16, 1024), desc_sw128(sa + kA + kk * 32, 16, 1024), idesc,
                 (ks | kk) ? 1u : 0u);
      mma_commit(empty + st);
    }
    if (ok) mma_commit(done);
    else mbar_arrive(done);
  } else if (warp >= 2) {
    const bool ready = mbar_wait(done, 0);
    tc_fence_after();
    if (!ready) {
      if (lane == 0) atomicOr(a.dflag, kFlagTimeout);
    } else if (!*(volatile int*)abort_flag) {
      const int q = warp & 3;
      const int r = 32 * q + lane;
      float hi[32], lo[32];
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16), hi);
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32, lo);
      float* out = (view ? a.Q : a.P) + (row0 + r) * kTcKP;
      if (row0 + r < a.b) {
#pragma unroll
        for (int i = 0; i < kTcKP; i += 4)
          atomicAdd(reinterpret_cast<float4*>(out + i),
                    make_float4(hi[i] + lo[i], hi[i + 1] + lo[i + 1], hi[i + 2] + lo[i + 2], hi[i + 3] + lo[i + 3]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 64);
}

struct TcBackArgs {
  int64_t b, nA, d_x, d_y;
  int k, split, nslice_x;
  float inv_nA, inv_nB;
  float* AV;
  float* BV;
  int* dflag;
};

// grid: d/256 column slices (X slices first, then Y slices)
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_backproject(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
                     const __grid_constant__ CUtensorMap mapPt, const __grid_constant__ CUtensorMap mapQt,
                     const TcBackArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  constexpr int kA = 32768, kB = 8192, kStage = kA + kB;
  uint64_t* full = (uint64_t*)(base + kB_Stages * kStage);
  uint64_t* empty = full + kB_Stages;
  uint64_t* done = empty + kB_Stages;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* abort_flag = (int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  const bool isY = (int)blockIdx.x >= a.nslice_x;
  const int64_t c0 = (int64_t)(isY ? blockIdx.x - a.nslice_x : blockIdx.x) * 256;
  const int64_t goff = (isY ? a.d_x : 0) + c0;
  const CUtensorMap* mZ = isY ? &mapY : &mapX;
  // A rows use the other view's projection, B rows this view's
  const CUtensorMap* mWA = isY ? &mapPt : &mapQt;
  const CUtensorMap* mWB = isY ? &mapQt : &mapPt;
  const int nrb = (int)(a.b / 64);

  if (warp == 1) {
    tmem_alloc(tmem_slot, 256);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kB_Stages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tensormap(mZ);
    prefetch_tensormap(mWA);
    prefetch_tensormap(mWB);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    const uint64_t once = policy_evict_first();
    for (int s = 0; s < nrb; ++s) {
      const int st = s % kB_Stages;
      const int64_t r0 = (int64_t)(nrb - 1 - s) * 64;
      if (s >= kB_Stages && !mbar_wait(empty + st, ((s / kB_Stages) - 1) & 1)) {
        atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        break;
      }
      if (*(volatile int*)abort_flag) break;
      uint8_t* sa = base + st * kStage;
      const bool rowA = !a.split || r0 < a.nA;
      mbar_arrive_expect_tx(full + st, kStage);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        tma_load_2d_hint(sa + j * 8192, mZ, (int)(c0 + 64 * j), (int)r0, full + st, once);
      tma_load_2d(sa + kA, rowA ? mWA : mWB, (int)r0, 0, full + st);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16(128, 64, 1, 0);
    bool ok = true, usedA = false, usedB = false;
    for (int s = 0; s < nrb; ++s) {
      const int st = s % kB_Stages;
      const int64_t r0 = (int64_t)(nrb - 1 - s) * 64;
      if (!mbar_wait(full + st, (s / kB_Stages) & 1)) {
        atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      uint8_t* sa = base + st * kStage;
      const bool rowA = !a.split || r0 < a.nA;
      const uint32_t dbase = tmem + (rowA ? 0u : 128u);
      const bool used = rowA ? usedA : usedB;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(dbase + 64 * h, desc_sw128(sa + 2 * h * 8192 + kk * 2048, 8192, 1024),
                   desc_sw128(sa + kA + kk * 32, 16, 1024), idesc, (used || kk) ? 1u : 0u);
      if (rowA) usedA = true;
      else usedB = true;
      mma_commit(empty + st);
    }
    if (ok) mma_commit(done);
    else mbar_arrive(done);
  } else if (warp >= 2) {
    const bool ready = mbar_wait(done, 0);
    tc_fence_after();
    if (!ready) {
      if (lane == 0) atomicOr(a.dflag, kFlagTimeout);
    } else if (!*(volatile int*)abort_flag) {
      const int q = warp & 3;
      const int k = a.k;
#pragma unroll 1
      for (int which = 0; which < 2; ++which) {
        float* out = which == 0 ? a.AV : a.BV;
        const float sc = which == 0 ? a.inv_nA : a.inv_nB;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          float hi[32], lo[32];
          const uint32_t t = tmem + (uint32_t)(which * 128 + 64 * h) + ((uint32_t)(32 * q) << 16);
          tmem_ld32(t, hi);
          tmem_ld32(t + 32, lo);
          const int64_t col = goff + 128 * h + 32 * q + lane;
          for (int i = 0; i < k; ++i) out[col * k + i] = (hi[i] + lo[i]) * sc;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// FP32 minibatches on the tensor cores. Each FP32 tile that TMA lands (boxes of 32 columns,
// 128-byte swizzle) is split by converter warps into BF16 hi = bf16(x) and lo = bf16(x - hi),
// written in the layout TMA gives BF16 boxes of 64 columns; x - hi is exact in FP32, so hi + lo
// keeps about 16 significant bits of x. The MMAs add X_hi [V_hi | V_lo] + X_lo V_hi (the
// X_lo V_lo term is below the pairs' resolution), the same accumulator columns as the BF16 path.

// Four landing slots [FP32 tile 32 KB | operand box 8 KB] keep three tiles in flight from HBM;
// two conversion slots [BF16 hi 16 KB | BF16 lo 16 KB] take the converted tiles to the MMAs.
constexpr int kF32Land = 4, kF32ConvSlots = 2;
constexpr int kF32LandB = 40960, kF32ConvB = 32768;
constexpr size_t kF32Smem = (size_t)kF32Land * kF32LandB + (size_t)kF32ConvSlots * kF32ConvB + 1024 + 256;
constexpr int kF32Threads = 448;  // warps 0: TMA, 1: MMA, 2-5: epilogue, 6-13: converters
constexpr int kF32Conv = 256;     // converter threads

// FP32 tile of R rows x C columns (C / 32 boxes of [R][32]) into hi and lo (C / 64 boxes of
// [R][64] BF16 each); converter thread t of kF32Conv. Consecutive threads take consecutive rows
// of one 8-column group, so a quarter warp's 16-byte accesses fall in distinct banks. Each
// thread's items are unrolled with all their loads issued first.
template <int R, int C>
__device__ __forceinline__ void split_f32_tile(const uint8_t* src, uint8_t* hi, uint8_t* lo, int t) {
  constexpr int kItems = R * (C / 8) / kF32Conv;
  static_assert(R * (C / 8) % kF32Conv == 0, "items split evenly over the converter threads");
  float4 x0[kItems], x1[kItems];
#pragma unroll
  for (int u = 0; u < kItems; ++u) {
    const int it = t + u * kF32Conv;
    const int r = it % R, c = 8 * (it / R), rr = r & 7;
    const uint8_t* sb = src + (c / 32) * (R * 128) + (r >> 3) * 1024 + rr * 128;
    const int q = (c & 31) >> 2;
    x0[u] = *reinterpret_cast<const float4*>(sb + ((q ^ rr) << 4));
    x1[u] = *reinterpret_cast<const float4*>(sb + (((q + 1) ^ rr) << 4));
  }
#pragma unroll
  for (int u = 0; u < kItems; ++u) {
    const int it = t + u * kF32Conv;
    const int r = it % R, c = 8 * (it / R), rr = r & 7;
    const float xs[8] = {x0[u].x, x0[u].y, x0[u].z, x0[u].w, x1[u].x, x1[u].y, x1[u].z, x1[u].w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const __nv_bfloat162 hv = __floats2bfloat162_rn(xs[2 * v], xs[2 * v + 1]);
      const __nv_bfloat162 lv =
          __floats2bfloat162_rn(xs[2 * v] - __low2float(hv), xs[2 * v + 1] - __high2float(hv));
      h[v] = *reinterpret_cast<const uint32_t*>(&hv);
      l[v] = *reinterpret_cast<const uint32_t*>(&lv);
    }
    const int toff = (c / 64) * (R * 128) + (r >> 3) * 1024 + rr * 128 + ((((c & 63) >> 3) ^ rr) << 4);
    *reinterpret_cast<uint4*>(hi + toff) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo + toff) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// P = X V_x, Q = Y V_y from FP32 rows. grid: (b/128 row tiles, 2 views, splits). A landing
// slot is [X: two 128 x 32 FP32 boxes][V^T box 64 x 64], a conversion slot [hi 128 x 64][lo 128 x 64].
__global__ void __launch_bounds__(kF32Threads, 1)
    k_tc_project_f32(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
                     const __grid_constant__ CUtensorMap mapVt, const TcProjArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  constexpr int kX = 32768, kH = 16384;
  uint8_t* cbase = base + kF32Land * kF32LandB;
  uint64_t* full = (uint64_t*)(cbase + kF32ConvSlots * kF32ConvB);  // [kF32Land] tile and operand landed
  uint64_t* lempty = full + kF32Land;                                // [kF32Land] MMAs done with the operand
  uint64_t* cfull = lempty + kF32Land;                               // [kF32ConvSlots] tile converted
  uint64_t* cempty = cfull + kF32ConvSlots;                          // [kF32ConvSlots] MMAs done with it
  uint64_t* done = cempty + kF32ConvSlots;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* abort_flag = (int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  const int view = blockIdx.y;
  const int64_t row0 = (int64_t)blockIdx.x * 128;
  const int64_t c0 = (int64_t)blockIdx.z * a.cols_per_split;
  const int nk = (int)(a.cols_per_split / 64);
  const CUtensorMap* mZ = view ? &mapY : &mapX;
  const int64_t voff = view ? a.d_x : 0;

  if (warp == 1) {
    tmem_alloc(tmem_slot, 64);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kF32Land; ++s) {
      mbar_init(full + s, 1);
      mbar_init(lempty + s, 1);
    }
    for (int s = 0; s < kF32ConvSlots; ++s) {
      mbar_init(cfull + s, kF32Conv / 32);
      mbar_init(cempty + s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tensormap(mZ);
    prefetch_tensormap(&mapVt);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    const uint64_t keep = policy_evict_last();
    for (int ks = 0; ks < nk; ++ks) {
      const int st = ks % kF32Land;
      if (ks >= kF32Land && !mbar_wait(lempty + st, ((ks / kF32Land) - 1) & 1)) {
        atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        break;
      }
      if (*(volatile int*)abort_flag) break;
      uint8_t* sa = base + st * kF32LandB;
      mbar_arrive_expect_tx(full + st, kF32LandB);
      tma_load_2d(sa, mZ, (int)(c0 + (int64_t)ks * 64), (int)row0, full + st);
      tma_load_2d(sa + kX / 2, mZ, (int)(c0 + (int64_t)ks * 64 + 32), (int)row0, full + st);
      tma_load_2d_hint(sa + kX, &mapVt, (int)(voff + c0 + (int64_t)ks * 64), 0, full + st, keep);
    }
  } else if (warp >= 6) {
    // converters: each landed FP32 tile into its hi / lo BF16 tiles
    const int t = tid - 192;
    for (int ks = 0; ks < nk; ++ks) {
      const int st = ks % kF32Land, cs = ks % kF32ConvSlots;
      if (!mbar_wait(full + st, (ks / kF32Land) & 1) ||
          (ks >= kF32ConvSlots && !mbar_wait(cempty + cs, ((ks / kF32ConvSlots) - 1) & 1))) {
        if (lane == 0) atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        break;
      }
      if (*(volatile int*)abort_flag) break;
      uint8_t* cb = cbase + cs * kF32ConvB;
      split_f32_tile<128, 64>(base + st * kF32LandB, cb, cb + kH, t);
      fence_proxy_async_smem();  // the tiles are read by the tensor cores (async proxy)
      __syncwarp();
      if (lane == 0) mbar_arrive(cfull + cs);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t id64 = idesc_bf16(128, 64, 0, 0), id32 = idesc_bf16(128, 32, 0, 0);
    bool ok = true;
    for (int ks = 0; ks < nk; ++ks) {
      const int st = ks % kF32Land, cs = ks % kF32ConvSlots;
      if (!mbar_wait(cfull + cs, (ks / kF32ConvSlots) & 1) || *(volatile int*)abort_flag) {
        atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint8_t* vt = base + st * kF32LandB + kX;
      const uint8_t* xh = cbase + cs * kF32ConvB;
      const uint8_t* xl = xh + kH;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        mma_bf16(tmem, desc_sw128(xh + kk * 32, 16, 1024), desc_sw128(vt + kk * 32, 16, 1024), id64,
                 (ks | kk) ? 1u : 0u);
        mma_bf16(tmem, desc_sw128(xl + kk * 32, 16, 1024), desc_sw128(vt + kk * 32, 16, 1024), id32, 1u);
      }
      mma_commit(cempty + cs);
      mma_commit(lempty + st);
    }
    if (ok) mma_commit(done);
    else mbar_arrive(done);
  } else if (warp >= 2 && warp < 6) {
    const bool ready = mbar_wait(done, 0);
    tc_fence_after();
    if (!ready) {
      if (lane == 0) atomicOr(a.dflag, kFlagTimeout);
    } else if (!*(volatile int*)abort_flag) {
      const int q = warp & 3;
      const int r = 32 * q + lane;
      float hi[32], lo[32];
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16), hi);
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32, lo);
      float* out = (view ? a.Q : a.P) + (row0 + r) * kTcKP;
      if (row0 + r < a.b) {
#pragma unroll
        for (int i = 0; i < kTcKP; i += 4)
          atomicAdd(reinterpret_cast<float4*>(out + i),
                    make_float4(hi[i] + lo[i], hi[i + 1] + lo[i + 1], hi[i + 2] + lo[i + 2], hi[i + 3] + lo[i + 3]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 64);
}

// A_t V and B_t V from FP32 rows. grid: d/256 column slices (X slices first). Rows in 64-row
// blocks streamed last-first (the rows the projection read last are still in L2), each block
// in two steps of 128 columns: landing slot [X: four 64 x 32 FP32 boxes][operand 64 x 64],
// conversion slot [hi 2 x 64 x 64][lo 2 x 64 x 64].
__global__ void __launch_bounds__(kF32Threads, 1)
    k_tc_backproject_f32(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
                         const __grid_constant__ CUtensorMap mapPt, const __grid_constant__ CUtensorMap mapQt,
                         const TcBackArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  constexpr int kX = 32768, kH = 16384;
  uint8_t* cbase = base + kF32Land * kF32LandB;
  uint64_t* full = (uint64_t*)(cbase + kF32ConvSlots * kF32ConvB);  // [kF32Land] tile and operand landed
  uint64_t* lempty = full + kF32Land;                                // [kF32Land] MMAs done with the operand
  uint64_t* cfull = lempty + kF32Land;                               // [kF32ConvSlots] tile converted
  uint64_t* cempty = cfull + kF32ConvSlots;                          // [kF32ConvSlots] MMAs done with it
  uint64_t* done = cempty + kF32ConvSlots;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* abort_flag = (int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  const bool isY = (int)blockIdx.x >= a.nslice_x;
  const int64_t c0 = (int64_t)(isY ? blockIdx.x - a.nslice_x : blockIdx.x) * 256;
  const int64_t goff = (isY ? a.d_x : 0) + c0;
  const CUtensorMap* mZ = isY ? &mapY : &mapX;
  const CUtensorMap* mWA = isY ? &mapPt : &mapQt;
  const CUtensorMap* mWB = isY ? &mapQt : &mapPt;
  const int nrb = (int)(a.b / 64);
  const int nst = 2 * nrb;  // (row block, column half) steps

  if (warp == 1) {
    tmem_alloc(tmem_slot, 256);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kF32Land; ++s) {
      mbar_init(full + s, 1);
      mbar_init(lempty + s, 1);
    }
    for (int s = 0; s < kF32ConvSlots; ++s) {
      mbar_init(cfull + s, kF32Conv / 32);
      mbar_init(cempty + s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tensormap(mZ);
    prefetch_tensormap(mWA);
    prefetch_tensormap(mWB);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    const uint64_t once = policy_evict_first();
    for (int s = 0; s < nst; ++s) {
      const int st = s % kF32Land;
      const int64_t r0 = (int64_t)(nrb - 1 - s / 2) * 64;
      const int h = s & 1;
      if (s >= kF32Land && !mbar_wait(lempty + st, ((s / kF32Land) - 1) & 1)) {
        atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        break;
      }
      if (*(volatile int*)abort_flag) break;
      uint8_t* sa = base + st * kF32LandB;
      const bool rowA = !a.split || r0 < a.nA;
      mbar_arrive_expect_tx(full + st, kF32LandB);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        tma_load_2d_hint(sa + j * 8192, mZ, (int)(c0 + 128 * h + 32 * j), (int)r0, full + st, once);
      tma_load_2d(sa + kX, rowA ? mWA : mWB, (int)r0, 0, full + st);
    }
  } else if (warp >= 6) {
    const int t = tid - 192;
    for (int s = 0; s < nst; ++s) {
      const int st = s % kF32Land, cs = s % kF32ConvSlots;
      if (!mbar_wait(full + st, (s / kF32Land) & 1) ||
          (s >= kF32ConvSlots && !mbar_wait(cempty + cs, ((s / kF32ConvSlots) - 1) & 1))) {
        if (lane == 0) atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        break;
      }
      if (*(volatile int*)abort_flag) break;
      uint8_t* cb = cbase + cs * kF32ConvB;
      split_f32_tile<64, 128>(base + st * kF32LandB, cb, cb + kH, t);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(cfull + cs);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t id64 = idesc_bf16(128, 64, 1, 0), id32 = idesc_bf16(128, 32, 1, 0);
    bool ok = true;
    bool usedA[2] = {false, false}, usedB[2] = {false, false};
    for (int s = 0; s < nst; ++s) {
      const int st = s % kF32Land, cs = s % kF32ConvSlots;
      const int64_t r0 = (int64_t)(nrb - 1 - s / 2) * 64;
      const int h = s & 1;
      if (!mbar_wait(cfull + cs, (s / kF32ConvSlots) & 1) || *(volatile int*)abort_flag) {
        atomicOr(a.dflag, kFlagTimeout);
        *(volatile int*)abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint8_t* w = base + st * kF32LandB + kX;
      const uint8_t* xh = cbase + cs * kF32ConvB;
      const uint8_t* xl = xh + kH;
      const bool rowA = !a.split || r0 < a.nA;
      const uint32_t dcol = tmem + (rowA ? 0u : 128u) + 64 * h;
      const bool used = rowA ? usedA[h] : usedB[h];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        mma_bf16(dcol, desc_sw128(xh + kk * 2048, 8192, 1024), desc_sw128(w + kk * 32, 16, 1024), id64,
                 (used || kk) ? 1u : 0u);
        mma_bf16(dcol, desc_sw128(xl + kk * 2048, 8192, 1024), desc_sw128(w + kk * 32, 16, 1024), id32, 1u);
      }
      if (rowA) usedA[h] = true;
      else usedB[h] = true;
      mma_commit(cempty + cs);
      mma_commit(lempty + st);
    }
    if (ok) mma_commit(done);
    else mbar_arrive(done);
  } else if (warp >= 2 && warp < 6) {
    const bool ready = mbar_wait(done, 0);
    tc_fence_after();
    if (!ready) {
      if (lane == 0) atomicOr(a.dflag, kFlagTimeout);
    } else if (!*(volatile int*)abort_flag) {
      const int q = warp & 3;
      const int k = a.k;
#pragma unroll 1
      for (int which = 0; which < 2; ++which) {
        float* out = which == 0 ? a.AV : a.BV;
        const float sc = which == 0 ? a.inv_nA : a.inv_nB;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          float hi[32], lo[32];
          const uint32_t t = tmem + (uint32_t)(which * 128 + 64 * h) + ((uint32_t)(32 * q) << 16);
          tmem_ld32(t, hi);
          tmem_ld32(t + 32, lo);
          const int64_t col = goff + 128 * h + 32 * q + lane;
          for (int i = 0; i < k; ++i) out[col * k + i] = (hi[i] + lo[i]) * sc;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 256);
}

}  // namespace
}  // namespace sgep


namespace sgep {

size_t tc_terms_floats(int k) { return (size_t)3 * k * k + 5 * k; }

// Pointers into the k x k terms for step parity `slot`: a | b | norms[2] | G[2] | vv[2].
TcTerms tc_terms(const Ctx& c, int slot) {
  const int k = c.k, kk = k * k;
  TcTerms t;
  t.a = c.gram;
  t.b = c.gram + kk;
  t.norms = c.gram + kk + k + slot * k;
  t.G = c.gram + kk + 3 * k + slot * kk;
  t.vv = c.gram + 3 * kk + 3 * k + slot * k;
  return t;
}

bool tc_supported(const Ctx& c, const char** why) {
  const char* w = nullptr;
  if (c.cfg.dtype != SGEP_BF16 && c.cfg.dtype != SGEP_F32) w = "needs BF16 or FP32 minibatches";
  else if (c.cfg.kind != SGEP_CCA) w = "tensor-core path supports CCA";
  else if (!c.cfg.split_AB) w = "tensor-core path needs split A/B batches";
  else if (c.d_x != c.d_y) w = "tensor-core path needs d_x == d_y";
  else if (c.k > kTcKP) w = "k > 32";
  else if (c.d_x % 256 || c.d_y % 256) w = "d_x and d_y must be multiples of 256";
  else if (c.cfg.max_b % 128) w = "max_b must be a multiple of 128";
  if (why) *why = w;
  return w == nullptr;
}

int tc_alloc(Ctx& c) {
  const size_t mb = (size_t)c.cfg.max_b;
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_Vt, (size_t)2 * kTcKP * c.d * 2));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_PQ, 2 * mb * kTcKP * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_Pt, 2 * kTcKP * mb * 2));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_Qt, 2 * kTcKP * mb * 2));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_coef, (size_t)(c.k * c.k + 2 * c.k) * sizeof(float)));
  // k x k terms: a | b | norms [2] | G [2] | |v_i|^2 [2] (double-buffered by step parity)
  cudaFree(c.gram);
  c.gram = nullptr;
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.gram, tc_terms_floats(c.k) * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(c.gram, 0, tc_terms_floats(c.k) * sizeof(float)));
  if (c.cfg.debug) SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_dbg, (size_t)(2 * c.k * c.k + c.k) * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_bar, sizeof(unsigned long long)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_part,
                           (size_t)((c.d + 127) / 128) * (32 + kTcKP * kTcKP + kTcKP) * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(c.tc_bar, 0, sizeof(unsigned long long)));
  c.tc_bar_base = 0;
  c.tc_chain = 0;
  {
    const char* tr = getenv("SGEP_TRACE");
    if (tr && tr[0] == '1') {
      const size_t n = (size_t)((c.d + 127) / 128) * 8;
      SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_upd_trace, n * sizeof(unsigned long long)));
      SGEP_CUDA_TRY(cudaMemset(c.tc_upd_trace, 0, n * sizeof(unsigned long long)));
    }
  }
  {
    // the fused update needs every block resident at once
    int per_sm = 0;
    const int grid = (int)((c.d + 127) / 128);
    const bool var = c.adam_m || c.z;
    c.tc_upd_fused = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                         &per_sm, var ? k_tc_update_fused<true> : k_tc_update_fused<false>, 256, 0) ==
                             cudaSuccess &&
                         grid <= per_sm * c.num_sms
                     ? 1
                     : 0;
    cudaGetLastError();
  }
  if (c.cfg.dtype == SGEP_F32) {
    // FP32 rows: three stages of [FP32 tile | operand box | BF16 hi | BF16 lo]
    const size_t sf = kF32Smem;
    SGEP_CUDA_TRY(cudaFuncSetAttribute(k_tc_project_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf));
    SGEP_CUDA_TRY(cudaFuncSetAttribute(k_tc_backproject_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf));
    c.tc_smem_p = c.tc_smem_b = sf;
  } else {
    const size_t sp = kP_Stages * 24576 + 1024 + 256, sb = kB_Stages * 40960 + 1024 + 256;
    SGEP_CUDA_TRY(cudaFuncSetAttribute(k_tc_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp));
    SGEP_CUDA_TRY(cudaFuncSetAttribute(k_tc_backproject, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    c.tc_smem_p = sp;
    c.tc_smem_b = sb;
  }
  // The streamed one-read kernel is the default where the shape allows it
  // (SGEP_TC_STREAM=0 keeps the two-pass products).
  return tc_stream_setup(c);
}

void tc_free(Ctx& c) {
  tc_stream_free(c);
  cudaFree(c.tc_Vt);
  cudaFree(c.tc_PQ);
  cudaFree(c.tc_Pt);
  cudaFree(c.tc_Qt);
  cudaFree(c.tc_coef);
  c.tc_coef = nullptr;
  cudaFree(c.tc_dbg);
  c.tc_dbg = nullptr;
  cudaFree(c.tc_bar);
  c.tc_bar = nullptr;
  cudaFree(c.tc_part);
  c.tc_part = nullptr;
  cudaFree(c.tc_upd_trace);
  c.tc_upd_trace = nullptr;
  c.tc_Vt = nullptr;
  c.tc_PQ = nullptr;
  c.tc_Pt = c.tc_Qt = nullptr;
}

int tc_prepare_chain(Ctx& c, cudaStream_t s) {
  if (c.tc_chain) return SGEP_OK;
  const TcTerms tt = tc_terms(c, (int)(c.t & 1));
  SGEP_CUDA_TRY(cudaMemsetAsync(c.gram, 0, tc_terms_floats(c.k) * sizeof(float), s));
  k_tc_prep_v<<<(unsigned)((c.d + 63) / 64), 256, 0, s>>>(c.V, c.S, c.d, c.k, c.tc_Vt, tt.G, tt.vv);
  SGEP_CUDA_TRY(cudaGetLastError());
  ++c.launches;
  c.tc_chain = 1;
  return SGEP_OK;
}

int tc_products(Ctx& c, const void* X, const void* Y, int64_t b, cudaStream_t s, float eta, float gamma) {
  (void)eta;
  (void)gamma;
  const int split = c.cfg.split_AB ? 1 : 0;
  const int64_t nA = split ? b / 2 : b;
  c.tc_st_updated = 0;
  c.tc_acc_stale = 0;
  if (b % 128 || ((uintptr_t)X & 15) || ((uintptr_t)Y & 15) || (split && nA % 64)) {
    c.tc_generic_step = 1;
    return generic_products(c, X, Y, b, s);
  }
  c.tc_generic_step = 0;
  float* P = c.tc_PQ;
  float* Q = c.tc_PQ + (size_t)c.cfg.max_b * kTcKP;
  const int k = c.k;
  const int slot = (int)(c.t & 1);
  const TcTerms tt = tc_terms(c, slot);
  // 1. V split into BF16 pairs and the d-side terms -- unless the previous step's update
  //    produced them (and cleared the terms this step accumulates)
  int rc = tc_prepare_chain(c, s);
  if (rc) return rc;
  if (tc_stream_supported(c, b)) {
    // one read of the minibatch from HBM: products, row-side terms and update in one launch
    rc = tc_stream_steps(c, X, Y, b, 1, s);
    if (!rc) c.tc_st_updated = 1;
    return rc;
  }
  CUtensorMap mX1, mY1, mVt, mX2, mY2, mPt, mQt;
  const bool f32 = c.cfg.dtype == SGEP_F32;
  if (f32) {
    rc = make_map_f32(&mX1, X, b, c.d_x, c.d_x, 128, 32);
    if (!rc) rc = make_map_f32(&mY1, Y, b, c.d_y, c.d_y, 128, 32);
    if (!rc) rc = make_map_f32(&mX2, X, b, c.d_x, c.d_x, 64, 32);
    if (!rc) rc = make_map_f32(&mY2, Y, b, c.d_y, c.d_y, 64, 32);
  } else {
    rc = make_map_bf16(&mX1, X, b, c.d_x, c.d_x, 128, 64);
    if (!rc) rc = make_map_bf16(&mY1, Y, b, c.d_y, c.d_y, 128, 64);
    if (!rc) rc = make_map_bf16(&mX2, X, b, c.d_x, c.d_x, 64, 64);
    if (!rc) rc = make_map_bf16(&mY2, Y, b, c.d_y, c.d_y, 64, 64);
  }
  if (!rc) rc = make_map_bf16(&mVt, c.tc_Vt, 2 * kTcKP, c.d, c.d, 64, 64);
  if (rc) return rc;
  c.tc_pq_dirty = 1;  // the kernels below leave P and Q non-zero
  rc = make_map_bf16(&mPt, c.tc_Pt, 2 * kTcKP, b, c.cfg.max_b, 64, 64);
  if (!rc) rc = make_map_bf16(&mQt, c.tc_Qt, 2 * kTcKP, b, c.cfg.max_b, 64, 64);
  if (rc) return rc;
  // 2. projections (accumulated into P and Q)
  SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_PQ, 0, sizeof(float) * 2 * c.cfg.max_b * kTcKP, s));
  {
    TcProjArgs pa;
    pa.b = b;
    pa.d_x = c.d_x;
    pa.d_y = c.d_y;
    // column splits so that the grid covers the SMs; each split a multiple of 64 columns
    int splits = std::max(1, (int)(c.num_sms / (2 * (b / 128))));
    const int64_t dmin = std::min(c.d_x, c.d_y);
    while (splits > 1 && (dmin % (64LL * splits) != 0)) --splits;
    pa.splits = splits;
    pa.cols_per_split = c.d_x / splits;
    pa.P = P;
    pa.Q = Q;
    pa.dflag = c.dflag;
    dim3 grid((unsigned)(b / 128), 2, (unsigned)splits);
    if (f32) k_tc_project_f32<<<grid, kF32Threads, c.tc_smem_p, s>>>(mX1, mY1, mVt, pa);
    else k_tc_project<<<grid, kTcThreads, c.tc_smem_p, s>>>(mX1, mY1, mVt, pa);
    SGEP_CUDA_TRY(cudaGetLastError());
  }
  // 3. P, Q split into BF16 pairs (transposed), row-side terms a and b
  k_tc_prep_w<<<(unsigned)((b + 15) / 16), 256, 0, s>>>(P, Q, b, c.cfg.max_b, nA, k, 1.f / (float)nA,
                                                         1.f / (float)(split ? b - nA : b), c.tc_Pt, c.tc_Qt,
                                                         tt.a, tt.b);
  SGEP_CUDA_TRY(cudaGetLastError());
  // 4. back-projection into acc = [A_t V ; B_t V]
  {
    TcBackArgs ba;
    ba.b = b;
    ba.nA = nA;
    ba.d_x = c.d_x;
    ba.d_y = c.d_y;
    ba.k = c.k;
    ba.split = split;
    ba.nslice_x = (int)(c.d_x / 256);
    ba.inv_nA = 1.f / (float)nA;
    ba.inv_nB = 1.f / (float)(split ? b - nA : b);
    ba.AV = c.acc;
    ba.BV = c.acc + c.d * c.k;
    ba.dflag = c.dflag;
    if (f32) k_tc_backproject_f32<<<(unsigned)(c.d / 256), kF32Threads, c.tc_smem_b, s>>>(mX2, mY2, mPt, mQt, ba);
    else k_tc_backproject<<<(unsigned)(c.d / 256), kTcThreads, c.tc_smem_b, s>>>(mX2, mY2, mPt, mQt, ba);
    SGEP_CUDA_TRY(cudaGetLastError());
  }
  c.launches += 3;
  return SGEP_OK;
}

int tc_update(Ctx& c, float eta, float gamma, cudaStream_t s) {
  if (c.tc_st_updated) {  // the streamed launch applied the update and prepared the next step
    c.tc_st_updated = 0;
    c.tc_chain = 1;
    return SGEP_OK;
  }
  const int k = c.k;
  const int slot = (int)(c.t & 1);
  const TcTerms tt = tc_terms(c, slot);
  if (c.tc_upd_fused) {
    if (c.tc_bar_reset) {  // an aborted launch may have left the barrier count short
      SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_bar, 0, sizeof(unsigned long long), s));
      c.tc_bar_base = 0;
      c.tc_bar_reset = 0;
    }
    const unsigned grid = (unsigned)((c.d + 127) / 128);
    TcUpdArgs u;
    u.V = c.V;
    u.Vout = c.V;  // each block reads its rows in phase 1 and writes them in phase 2
    u.S = c.S;
    u.AV = c.acc;
    u.BV = c.acc + c.d * k;
    u.terms = c.gram;
    u.part = c.tc_part;
    u.dbg = c.cfg.debug ? c.tc_dbg : nullptr;
    u.grad_out = c.cfg.debug ? c.grad : nullptr;
    u.Vt = c.tc_Vt;
    u.d = c.d;
    u.k = k;
    u.slot = slot;
    u.rho = c.cfg.rho;
    u.eta = eta;
    u.gamma = gamma;
    u.eps_B = c.cfg.eps_B;
    u.bar = c.tc_bar;
    u.bar_target = c.tc_bar_base + grid;
    u.bar_ns = 2000000000ull;
    if (c.test_stall) {  // test hook: a barrier count nothing reaches, a short limit
      u.bar_target += 1;
      u.bar_ns = 20000000ull;
    }
    u.trace = c.tc_upd_trace;
    u.dflag = c.dflag;
    u.var = next_variant(c);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (u.var.m || u.var.z) SGEP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tc_update_fused<true>, u));
    else SGEP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tc_update_fused<false>, u));
    c.tc_bar_base += (unsigned long long)grid;  // one barrier
    c.tc_chain = 1;
    ++c.launches;
    return SGEP_OK;
  }
  c.tc_chain = 0;
  if (c.cfg.debug) {
    SGEP_CUDA_TRY(cudaMemcpyAsync(c.tc_dbg, tt.a, (size_t)k * k * sizeof(float), cudaMemcpyDeviceToDevice, s));
    SGEP_CUDA_TRY(
        cudaMemcpyAsync(c.tc_dbg + k * k, tt.G, (size_t)k * k * sizeof(float), cudaMemcpyDeviceToDevice, s));
    SGEP_CUDA_TRY(
        cudaMemcpyAsync(c.tc_dbg + 2 * k * k, tt.b, (size_t)k * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  k_tc_update<<<(unsigned)((c.d + 31) / 32), 256, 0, s>>>(c.V, c.S, c.acc, c.acc + c.d * k, tt.a, tt.b, tt.G,
                                                          tt.vv, tt.norms, c.d, k, c.cfg.rho, eta, gamma,
                                                          c.cfg.eps_B, c.Vtmp, c.cfg.debug ? c.grad : nullptr);
  SGEP_CUDA_TRY(cudaGetLastError());
  if (k % 4 == 0) {
    const int64_t n4 = c.d * k / 4;
    k_tc_normalize<<<(unsigned)std::min<int64_t>((n4 + 255) / 256, 4 * c.num_sms), 256, 0, s>>>(
        c.Vtmp, tt.norms, c.V, n4, k, c.dflag);
    SGEP_CUDA_TRY(cudaGetLastError());
    c.launches += 2;
    return SGEP_OK;
  }
  // k not a multiple of 4: the generic retraction
  return generic_normalize(c, s);
}

}  // namespace sgep

using namespace sgep;

extern "C" int sgep_tc_selftest(int mode, double* max_rel_err) {
  if (!max_rel_err || mode < 0 || mode > 2) {
    set_error("sgep_tc_selftest: bad arguments");
    return SGEP_EINVAL;
  }
  __nv_bfloat16 *A = nullptr, *Bt = nullptr;
  float *out = nullptr, *ref = nullptr;
  int* flag = nullptr;
  int rc = SGEP_OK;
  CUtensorMap mA, mB;
  const size_t smem = 40960 + 64 + 1024;
  std::vector<float> h_out(128 * 64), h_ref(128 * 64);
  int h_flag = 0;
  cudaError_t e = cudaMalloc((void**)&A, 128 * 64 * 2);
  if (e == cudaSuccess) e = cudaMalloc((void**)&Bt, 64 * 64 * 2);
  if (e == cudaSuccess) e = cudaMalloc((void**)&out, 128 * 64 * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ref, 128 * 64 * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&flag, sizeof(int));
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "sgep_tc_selftest alloc");
    goto done;
  }
  cudaMemset(flag, 0, sizeof(int));
  cudaMemset(out, 0, 128 * 64 * 4);
  k_fill_bf16<<<16, 256>>>(A, 128 * 64, 12345u);
  k_fill_bf16<<<16, 256>>>(Bt, 64 * 64, 777u);
  if (mode == 0) rc = make_map_bf16(&mA, A, 128, 64, 64, 128, 64);
  else rc = make_map_bf16(&mA, A, 64, 128, 128, 64, 64);
  if (!rc) rc = make_map_bf16(&mB, Bt, 64, 64, 64, 64, 64);
  if (rc) goto done;
  e = cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "cudaFuncSetAttribute");
    goto done;
  }
  k_tc_selftest<<<1, 128, smem>>>(mA, mB, mode, out, flag);
  k_selftest_ref<<<128, 64>>>(A, Bt, mode, ref);
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h_out.data(), out, h_out.size() * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h_ref.data(), ref, h_ref.size() * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "sgep_tc_selftest run");
    goto done;
  }
  if (h_flag) {
    set_error("sgep_tc_selftest: a bounded wait gave up");
    rc = SGEP_ETIMEOUT;
    goto done;
  }
  {
    double mx = 0.0, md = 0.0;
    for (size_t i = 0; i < h_ref.size(); ++i) {
      mx = std::max(mx, (double)std::fabs(h_ref[i]));
      md = std::max(md, (double)std::fabs(h_out[i] - h_ref[i]));
    }
    *max_rel_err = md / (mx > 0 ? mx : 1.0);
  }
done:
  cudaFree(A);
  cudaFree(Bt);
  cudaFree(out);
  cudaFree(ref);
  cudaFree(flag);
  return rc;
}

namespace sgep {
// SGEP_TRACE=1: phase times of the most recent fused update (stderr).
void tc_update_trace_report(Ctx& c) {
  if (!c.tc_upd_trace) return;
  const int n = (int)((c.d + 127) / 128);
  std::vector<unsigned long long> t((size_t)n * 8);
  if (cudaMemcpy(t.data(), c.tc_upd_trace, t.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return;
  unsigned long long g0 = ~0ull;
  for (int b = 0; b < n; ++b) g0 = std::min(g0, t[(size_t)b * 8]);
  std::fprintf(stderr, "[sgep trace] fused update, %d blocks (us from first start, median/max):", n);
  const char* names[8] = {"start", "coefficients", "penalty", "rows", "norms", "phase1", "barrier", "end"};
  const int ev[8] = {0, 3, 4, 6, 7, 1, 2, 5};
  for (int ph = 0; ph < 8; ++ph) {
    std::vector<double> v;
    for (int b = 0; b < n; ++b) v.push_back((t[(size_t)b * 8 + ev[ph]] - g0) / 1e3);
    std::sort(v.begin(), v.end());
    std::fprintf(stderr, " %s %.2f/%.2f", names[ph], v[v.size() / 2], v.back());
  }
  std::fprintf(stderr, "\n");
}
}  // namespace sgep

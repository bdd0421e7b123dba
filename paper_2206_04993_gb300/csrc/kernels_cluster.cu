// Cluster path: one fused kernel launch per gamma-EigenGame step (Alg. 2, M = 1)
// for d up to a few thousand.
//
// Layout. The grid is NC clusters of CL CTAs (CL = 8 or 16). Inside a cluster,
// CTA r owns a contiguous slice of the columns: the first cl_x CTAs slice X's
// d_x columns, the others slice Y's d_y columns, so one cluster covers all d
// columns and every CTA keeps its slice of V, [Bv] and the products on chip.
// Cluster c streams its own contiguous range of minibatch rows.
//
// Per launch (step t+1, with the update of step t still pending):
//   1. Update of step t (every cluster redundantly, each CTA on its slice):
//      k x k terms a_ij = v_i^T A_t v_j, G_ij = <v_i, [Bv]_j>, b_i = v_i^T B_t v_i
//      are summed over the slice, then over the cluster through distributed
//      shared memory (fixed order, so every cluster gets bit-identical values);
//      then grad (Eq. update with the clipped [By]_j), v + eta grad, the [Bv]
//      step, column norms (again reduced over the cluster) and the retraction.
//      Cluster 0 writes the new V and [Bv] to the other state buffer.
//   2. Products of step t+1: for each tile of 32 rows, every CTA forms its
//      partial projections X_tile V_slice, the cluster sums them through
//      distributed shared memory into P and Q for the tile, and each CTA
//      accumulates X_tile^T [Q|P] for its columns in registers; the tile is
//      read from HBM once. At the end each CTA adds its d-slice of A_t V and
//      B_t V into one of three accumulator slots (one written, one read, one
//      being cleared for the step after).
// There are no waits between clusters, so no launch can deadlock.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "eg_math.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace sgep {
namespace {

constexpr int kThreads = 256;
constexpr int kRows = 32;          // rows per tile
constexpr int kMaxElems = 8192;    // w * k per CTA
constexpr int kMaxW = 256;         // columns per CTA
constexpr int kPerThread = kMaxElems / kThreads;

struct ClArgs {
  const void* X;
  const void* Y;
  int64_t b, nA;
  int64_t d_x, d_y, d;
  int k, kind, split, b_is_identity;
  float inv_nA, inv_nB;
  const float* V_in;
  const float* S_in;
  float* V_out;
  float* S_out;
  const float* acc_prev;  // A_t V | B_t V of the pending step, or null
  float* acc_cur;         // slot the new products go to, or null (update only)
  float* acc_zero;        // slot cleared for the step after next, or null
  float eta, gamma, rho, eps_B;
  int cl_x, w_x, w_y, wmax;
  int64_t rows_per_cluster;
  int* dflag;
  float* grad_dbg;  // d x k update directions (cluster 0), or null
  float* gram_dbg;  // a | G | b | norms (cluster 0, rank 0), or null
};

__device__ __forceinline__ float ld_elem(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_elem(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

// out[i] = sum_{c < w} A[c*k + i] * B[c*k + i], summed in a fixed order.
__device__ void colsum_prod(const float* A, const float* B, int w, int k, float* scratch, float* out) {
  const int G = max(1, kThreads / k);
  const int t = threadIdx.x;
  const int i = t % k, g = t / k;
  if (g < G) {
    float s = 0.f;
    for (int c = g; c < w; c += G) s = fmaf(A[c * k + i], B[c * k + i], s);
    scratch[g * k + i] = s;
  }
  __syncthreads();
  if (t < k) {
    float s = 0.f;
    for (int gg = 0; gg < G; ++gg) s += scratch[gg * k + t];
    out[t] = s;
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_cluster_step(const ClArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int cid = (int)(blockIdx.x / CL);
  const int tid = threadIdx.x;
  const int k = a.k;
  const int kk = k * k;

  const bool isY = rank >= a.cl_x;
  const int vr = isY ? rank - a.cl_x : rank;
  const int64_t ld = isY ? a.d_y : a.d_x;
  const int wn = isY ? a.w_y : a.w_x;
  const int64_t c_lo = min((int64_t)vr * wn, ld);
  const int64_t c_hi = min(c_lo + wn, ld);
  const int w = (int)(c_hi - c_lo);
  const int64_t goff = (isY ? a.d_x : 0) + c_lo;  // first row of V owned here
  const int n_el = w * k;
  const int wm = a.wmax;

  extern __shared__ float sm[];
  float* Vs = sm;                    // wm*k: V slice (then the new V slice)
  float* As = Vs + wm * k;           // wm*k: A_t V slice (then v + eta grad)
  float* Ss = As + wm * k;           // wm*k: [Bv] slice
  float* Bs = Ss + wm * k;           // wm*k: B_t V slice (with the ridge)
  float* Xt = Bs + wm * k;           // kRows*wm: minibatch tile
  float* part = Xt + kRows * wm;     // 2*kRows*k: partial projections (double buffer)
  float* Wown = part + 2 * kRows * k;   // kRows*k: projection of this CTA's view
  float* Wcross = Wown + kRows * k;     // kRows*k: projection of the other view
  float* red = Wcross + kRows * k;      // 2k^2+k: partial a | G | b of this CTA
  float* nrmp = red + 2 * kk + k;       // k: partial column norms^2
  float* tot = nrmp + k;                // 2k^2+k: cluster totals
  float* Tm = tot + 2 * kk + k;         // k^2
  float* cb = Tm + kk;                  // k
  float* cac = cb + k;                  // k
  float* nrm = cac + k;                 // k
  float* scr = nrm + k;                 // kThreads scratch

  // Clear the accumulator slot of the step after next (whole grid shares the work).
  if (a.acc_zero) {
    const int64_t n = 2 * a.d * k;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + tid; e < n; e += (int64_t)gridDim.x * kThreads)
      a.acc_zero[e] = 0.f;
  }

  // ---------------- 1. pending update ----------------
  if (a.acc_prev) {
    const float* AVp = a.acc_prev;
    const float* BVp = a.acc_prev + a.d * k;
    const float e1 = 1.f + a.eps_B;
    for (int e = tid; e < n_el; e += kThreads) {
      const int64_t g = goff * k + e;
      const float v = a.V_in[g];
      Vs[e] = v;
      As[e] = AVp[g];
      Ss[e] = a.S_in[g];
      Bs[e] = a.b_is_identity ? e1 * v : fmaf(a.eps_B, v, BVp[g]);
    }
    __syncthreads();
    for (int p = tid; p < kk; p += kThreads) {
      const int i = p / k, j = p % k;
      float sa = 0.f, sg = 0.f;
      for (int c = 0; c < w; ++c) {
        const float v = Vs[c * k + i];
        sa = fmaf(v, As[c * k + j], sa);
        sg = fmaf(v, Ss[c * k + j], sg);
      }
      red[p] = sa;
      red[kk + p] = sg;
    }
    colsum_prod(Vs, Bs, w, k, scr, red + 2 * kk);
    cluster.sync();
    for (int p = tid; p < 2 * kk + k; p += kThreads) {
      float s = 0.f;
      for (int r = 0; r < CL; ++r) s += cluster.map_shared_rank(red, r)[p];
      tot[p] = s;
    }
    __syncthreads();
    eg_coefficients(tot, k, a.rho, cb, cac, Tm);
    __syncthreads();
    const bool writer = cid == 0;
    for (int e = tid; e < n_el; e += kThreads) {
      const int c = e / k, i = e % k;
      const int64_t g = goff * k + e;
      const float v = Vs[e];
      const float bv = Bs[e];
      float pen = 0.f;
      for (int j = 0; j < i; ++j) pen = fmaf(Ss[c * k + j], Tm[j * k + i], pen);
      const float gr = cb[i] * As[e] - cac[i] * bv - pen;
      if (writer) {
        const float s_old = Ss[e];
        a.S_out[g] = fmaf(a.gamma, bv - s_old, s_old);
        if (a.grad_dbg) a.grad_dbg[g] = gr;
      }
      As[e] = fmaf(a.eta, gr, v);
    }
    __syncthreads();
    colsum_prod(As, As, w, k, scr, nrmp);
    cluster.sync();
    for (int i = tid; i < k; i += kThreads) {
      float s = 0.f;
      for (int r = 0; r < CL; ++r) s += cluster.map_shared_rank(nrmp, r)[i];
      nrm[i] = s;
    }
    __syncthreads();
    for (int e = tid; e < n_el; e += kThreads) {
      const int i = e % k;
      const float v = As[e] / sqrtf(nrm[i]);
      if (!isfinite(v)) atomicOr(a.dflag, kFlagNonFinite);
      Vs[e] = v;
      if (writer) a.V_out[goff * k + e] = v;
    }
    if (writer && rank == 0 && a.gram_dbg) {
      for (int p = tid; p < 2 * kk + k; p += kThreads) a.gram_dbg[p] = tot[p];
      for (int i = tid; i < k; i += kThreads) a.gram_dbg[2 * kk + k + i] = nrm[i];
    }
    __syncthreads();
  } else {
    for (int e = tid; e < n_el; e += kThreads) Vs[e] = a.V_in[goff * k + e];
    __syncthreads();
  }

  // ---------------- 2. products of the new minibatch ----------------
  if (a.acc_cur) {
    const T* Z = (const T*)(isY ? a.Y : a.X);
    const int64_t row_lo = min((int64_t)cid * a.rows_per_cluster, a.b);
    const int64_t row_hi = min(row_lo + a.rows_per_cluster, a.b);
    const bool cca = a.kind == SGEP_CCA;
    const bool pca = a.kind == SGEP_PCA;
    const int own_lo = isY ? a.cl_x : 0, own_hi = isY ? CL : a.cl_x;
    const int cr_lo = isY ? 0 : a.cl_x, cr_hi = isY ? a.cl_x : CL;
    const float* WA = pca ? Wown : Wcross;
    float accA[kPerThread], accB[kPerThread];
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) accA[q] = accB[q] = 0.f;
    int buf = 0;
    for (int64_t r0 = row_lo; r0 < row_hi; r0 += kRows) {
      const int nr = (int)min((int64_t)kRows, row_hi - r0);
      for (int e = tid; e < kRows * wm; e += kThreads) {
        const int rr = e / wm, c = e % wm;
        Xt[e] = (rr < nr && c < w) ? ld_elem(Z, (r0 + rr) * ld + c_lo + c) : 0.f;
      }
      __syncthreads();
      float* pb = part + buf * kRows * k;
      for (int p = tid; p < kRows * k; p += kThreads) {
        const int rr = p / k, i = p % k;
        float s = 0.f;
        for (int c = 0; c < w; ++c) s = fmaf(Xt[rr * wm + c], Vs[c * k + i], s);
        pb[p] = s;
      }
      cluster.sync();
      for (int p = tid; p < kRows * k; p += kThreads) {
        float so = 0.f, sc = 0.f;
        for (int r = own_lo; r < own_hi; ++r) so += cluster.map_shared_rank(pb, r)[p];
        for (int r = cr_lo; r < cr_hi; ++r) sc += cluster.map_shared_rank(pb, r)[p];
        Wown[p] = so;
        Wcross[p] = sc;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kPerThread; ++q) {
        const int e = tid + q * kThreads;
        if (e < n_el) {
          const int c = e / k, i = e % k;
          float sa = accA[q], sb = accB[q];
          for (int rr = 0; rr < nr; ++rr) {
            const int64_t row = r0 + rr;
            const float x = Xt[rr * wm + c];
            const bool toA = !cca || !a.split || row < a.nA;
            const bool toB = cca && (!a.split || row >= a.nA);
            if (toA) sa = fmaf(x, WA[rr * k + i], sa);
            if (toB) sb = fmaf(x, Wown[rr * k + i], sb);
          }
          accA[q] = sa;
          accB[q] = sb;
        }
      }
      __syncthreads();
      buf ^= 1;
    }
    const bool hasA = row_lo < row_hi && (!cca || !a.split || row_lo < a.nA);
    const bool hasB = row_lo < row_hi && cca && (!a.split || row_hi > a.nA);
    float* AVc = a.acc_cur;
    float* BVc = a.acc_cur + a.d * k;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      const int e = tid + q * kThreads;
      if (e < n_el) {
        const int64_t g = goff * k + e;
        if (hasA) atomicAdd(&AVc[g], accA[q] * a.inv_nA);
        if (hasB) atomicAdd(&BVc[g], accB[q] * a.inv_nB);
      }
    }
  }
  // No CTA may leave while others can still read its shared memory.
  cluster.sync();
}

size_t smem_floats(int wm, int k) {
  return (size_t)4 * wm * k + (size_t)kRows * wm + (size_t)4 * kRows * k + 2 * (2 * k * k + k) + k +
         (size_t)k * k + 3 * k + kThreads;
}

// Column split of a cluster of CL CTAs: X gets cl_x CTAs, Y the rest.
void plan(const Ctx& c, int CL, int* cl_x, int* wx, int* wy) {
  if (!c.has_y) {
    *cl_x = CL;
  } else {
    int x = (int)((double)CL * (double)c.d_x / (double)c.d + 0.5);
    *cl_x = std::min(CL - 1, std::max(1, x));
  }
  *wx = (int)((c.d_x + *cl_x - 1) / *cl_x);
  *wy = c.has_y ? (int)((c.d_y + (CL - *cl_x) - 1) / (CL - *cl_x)) : 0;
}

template <typename T>
int launch(Ctx& c, const ClArgs& a, int NC, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(NC * c.cl_size));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = c.cl_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c.cl_size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SGEP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cluster_step<T>, a));
  ++c.launches;
  return SGEP_OK;
}

template <typename T>
int configure(Ctx& c) {
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_cluster_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)c.cl_smem));
  if (c.cl_size > 8)
    SGEP_CUDA_TRY(cudaFuncSetAttribute(k_cluster_step<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c.cl_size);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = c.cl_smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c.cl_size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  SGEP_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, k_cluster_step<T>, &cfg));
  if (nclusters < 1) {
    set_error("cluster path: no cluster of this size fits on the device");
    return SGEP_ELAUNCH;
  }
  return SGEP_OK;
}

ClArgs base_args(Ctx& c) {
  ClArgs a = {};
  a.d_x = c.d_x;
  a.d_y = c.d_y;
  a.d = c.d;
  a.k = c.k;
  a.kind = c.cfg.kind;
  a.split = (c.cfg.kind == SGEP_CCA && c.cfg.split_AB) ? 1 : 0;
  a.b_is_identity = c.b_is_identity ? 1 : 0;
  a.rho = c.cfg.rho;
  a.eps_B = c.cfg.eps_B;
  a.cl_x = c.cl_x;
  a.w_x = c.cl_wx;
  a.w_y = c.cl_wy;
  a.wmax = c.cl_wmax;
  a.dflag = c.dflag;
  a.grad_dbg = c.cfg.debug ? c.grad : nullptr;
  a.gram_dbg = c.cfg.debug ? c.gram : nullptr;
  return a;
}

int run(Ctx& c, const void* X, const void* Y, int64_t b, float eta, float gamma, cudaStream_t s) {
  ClArgs a = base_args(c);
  const int pending = c.cl_pending;
  const size_t slot = (size_t)2 * c.d * c.k;
  a.V_in = c.cl_V[c.cl_cur];
  a.S_in = c.cl_S[c.cl_cur];
  a.V_out = c.cl_V[1 - c.cl_cur];
  a.S_out = c.cl_S[1 - c.cl_cur];
  a.acc_prev = pending ? c.cl_acc + c.cl_slot * slot : nullptr;
  a.eta = c.cl_eta;
  a.gamma = c.cl_gamma;
  int NC = 1;
  const int next = (c.cl_slot + 1) % 3;
  if (X) {
    a.X = X;
    a.Y = Y;
    a.b = b;
    a.nA = a.split ? b / 2 : b;
    a.inv_nA = 1.f / (float)a.nA;
    a.inv_nB = a.split ? 1.f / (float)(b - a.nA) : 1.f / (float)b;
    a.acc_cur = c.cl_acc + next * slot;
    a.acc_zero = c.cl_acc + ((c.cl_slot + 2) % 3) * slot;
    const int max_nc = std::max(1, c.num_sms / c.cl_size);
    NC = (int)std::min<int64_t>(max_nc, std::max<int64_t>(1, (b + 2 * kRows - 1) / (2 * kRows)));
    a.rows_per_cluster = (b + NC - 1) / NC;
  }
  int rc = c.cfg.dtype == SGEP_BF16 ? launch<__nv_bfloat16>(c, a, NC, s) : launch<float>(c, a, NC, s);
  if (rc) return rc;
  if (pending) {
    c.cl_cur = 1 - c.cl_cur;
    c.debug_valid = c.cfg.debug;
  }
  if (X) {
    c.cl_slot = next;
    c.cl_pending = 1;
    c.cl_eta = eta;
    c.cl_gamma = gamma;
  } else {
    c.cl_pending = 0;
  }
  c.V = c.cl_V[c.cl_cur];
  c.S = c.cl_S[c.cl_cur];
  return SGEP_OK;
}

}  // namespace

bool cluster_supported(const Ctx& c, const char** why) {
  if (c.k > 32) {
    if (why) *why = "k > 32";
    return false;
  }
  for (int CL : {8, 16}) {
    int cl_x, wx, wy;
    plan(c, CL, &cl_x, &wx, &wy);
    const int wm = std::max(wx, wy);
    if (wm <= kMaxW && wm * c.k <= kMaxElems && smem_floats(wm, c.k) * 4 <= 227 * 1024) return true;
  }
  if (why) *why = "column slices too wide for shared memory (d too large)";
  return false;
}

int cluster_alloc(Ctx& c) {
  int chosen = 0;
  for (int CL : {8, 16}) {
    int cl_x, wx, wy;
    plan(c, CL, &cl_x, &wx, &wy);
    const int wm = std::max(wx, wy);
    if (wm <= kMaxW && wm * c.k <= kMaxElems && smem_floats(wm, c.k) * 4 <= 227 * 1024) {
      c.cl_size = CL;
      c.cl_x = cl_x;
      c.cl_wx = wx;
      c.cl_wy = wy;
      c.cl_wmax = wm;
      c.cl_smem = smem_floats(wm, c.k) * sizeof(float);
      chosen = CL;
      break;
    }
  }
  if (!chosen) return SGEP_ENOTSUP;
  int rc = c.cfg.dtype == SGEP_BF16 ? configure<__nv_bfloat16>(c) : configure<float>(c);
  if (rc) return rc;
  const size_t dk = (size_t)c.d * c.k;
  c.cl_V[0] = c.V;
  c.cl_S[0] = c.S;
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.cl_V[1], dk * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.cl_S[1], dk * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.cl_acc, 3 * 2 * dk * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(c.cl_acc, 0, 3 * 2 * dk * sizeof(float)));
  c.cl_cur = 0;
  c.cl_slot = 0;
  c.cl_pending = 0;
  return SGEP_OK;
}

void cluster_free(Ctx& c) {
  if (c.cl_V[0]) {
    c.V = c.cl_V[0];
    c.S = c.cl_S[0];
  }
  cudaFree(c.cl_V[1]);
  cudaFree(c.cl_S[1]);
  cudaFree(c.cl_acc);
  c.cl_V[1] = c.cl_S[1] = nullptr;
  c.cl_acc = nullptr;
}

int cluster_step(Ctx& c, const void* X, const void* Y, int64_t b, float eta, float gamma, cudaStream_t s) {
  return run(c, X, Y, b, eta, gamma, s);
}

int cluster_flush(Ctx& c, cudaStream_t s) {
  if (!c.cl_pending) return SGEP_OK;
  return run(c, nullptr, nullptr, 0, 0.f, 0.f, s);
}

int cluster_products(Ctx& c, float* AV, float* BV, cudaStream_t s) {
  const size_t dk = (size_t)c.d * c.k;
  const float* src = c.cl_acc + (size_t)c.cl_slot * 2 * dk;
  SGEP_CUDA_TRY(cudaMemcpyAsync(AV, src, dk * sizeof(float), cudaMemcpyDeviceToHost, s));
  SGEP_CUDA_TRY(cudaMemcpyAsync(BV, src + dk, dk * sizeof(float), cudaMemcpyDeviceToHost, s));
  SGEP_CUDA_TRY(cudaStreamSynchronize(s));
  return SGEP_OK;
}

}  // namespace sgep

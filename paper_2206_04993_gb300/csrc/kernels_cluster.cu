// Cluster path: one fused kernel launch per gamma-EigenGame step (Alg. 2, M = 1)
// for d up to a few thousand.
//
// Layout. The grid is NC clusters of CL CTAs (CL = 8 or 16). Inside a cluster,
// CTA r owns a contiguous slice of the columns: the first cl_x CTAs slice X's
// d_x columns, the others slice Y's d_y columns, so one cluster covers all d
// columns and every CTA keeps its slice of V and [Bv] on chip. Cluster c
// streams its own contiguous range of minibatch rows in chunks of 32.
//
// Per launch (step t+1, with the update of step t pending):
//   0. The minibatch rows of this cluster are prefetched into shared memory
//      with cp.async before anything else (they do not depend on step t).
//   1. Update of step t, redundantly in every cluster, each CTA on its slice:
//      G_ij = <v_i, [Bv]_j> and ||v_i||^2 are summed over the slice and then
//      over the cluster through distributed shared memory (fixed order, so all
//      clusters obtain bit-identical values); a_ij = v_i^T A_t v_j and
//      b_i = v_i^T B_t v_i were accumulated row-side by step t's launch.
//      Then grad (Eq. update with clipped [By]_j), v + eta grad, the [Bv] step,
//      column norms (cluster-reduced) and the retraction. Cluster 0 writes the
//      new V and [Bv] to the other state buffer.
//   2. Products of step t+1, per chunk of 32 rows: partial projections
//      X_chunk V_slice (4x4 register micro-tiles), summed over the cluster into
//      P and Q through distributed shared memory; the row-side k x k terms
//      a_ij = (P^T Q + Q^T P)/n_A, b_i = (|P_i|^2 + |Q_i|^2)/n_B; and the
//      back-projection X_chunk^T [Q|P] accumulated in registers. The chunk is
//      read from HBM once. Each CTA finally adds its d-slice of A_t V and B_t V
//      (and each cluster its k x k terms) into one of three slots: one being
//      written, one read by the next launch, one cleared for the launch after.
// There are no waits between clusters, so no launch can deadlock. Launches
// use programmatic dependent launch: step 0 runs before the wait for the
// previous launch.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "eg_math.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace sgep {
namespace {

constexpr int kThreads = 512;
constexpr int kMaxW = 256;      // padded columns per CTA
constexpr int kMaxKP = 32;      // padded players
constexpr int kRed = 8192;      // floats of the split-reduction buffer
constexpr int kEB = 4;          // slice elements per thread in flight in the update

struct ClArgs {
  const void* X;
  const void* Y;
  int64_t b, nA;
  int64_t d_x, d_y, d;
  int k, kp, kind, split, b_is_identity;
  float inv_nA, inv_nB;
  const float* V_in;
  const float* S_in;
  float* V_out;
  float* S_out;
  const float* acc_prev;   // A_t V | B_t V of the pending step, or null
  const float* gram_prev;  // a (k*k) | b (k) of the pending step
  float* acc_cur;          // slot the new products go to, or null (update only)
  float* gram_cur;
  float* acc_zero;         // slot cleared for the step after next, or null
  float* gram_zero;
  float eta, gamma, rho, eps_B;
  int cl_x, w_x, w_y, wp, xs, rs, lkp;
  int64_t rows_per_cluster;
  int async_ok;
  int* dflag;
  float* grad_dbg;  // d x k update directions (cluster 0), or null
  float* gram_dbg;  // a | G | b | norms (cluster 0, rank 0), or null
  unsigned long long* trace;  // per-CTA phase clocks, or null
};

constexpr int kTracePhases = 16;
__device__ __forceinline__ void mark(const ClArgs& a, int ph, long long t0) {
  if (a.trace && threadIdx.x == 0) a.trace[blockIdx.x * kTracePhases + ph] = (unsigned long long)(clock64() - t0);
}

__device__ __forceinline__ float ld_elem(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_elem(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&u.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&u.y);
  const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float comp(const float4& v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// out[i] = sum_{c < w} A[c*lda + i] * B[c*lda + i] for i < k, summed in a fixed order.
__device__ void colsum_prod(const float* A, const float* B, int lda, int w, int k, float* scratch,
                            float* out) {
  const int G = max(1, kThreads / k);
  const int t = threadIdx.x;
  const int i = t % k, g = t / k;
  if (g < G) {
    float s = 0.f;
    for (int c = g; c < w; c += G) s = fmaf(A[c * lda + i], B[c * lda + i], s);
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

// Sum over the ranks of the cluster (ranks in [lo, hi)) of a value in each CTA's shared
// memory, all remote loads in flight before the first add; fixed order.
template <int CL>
__device__ __forceinline__ float cluster_sum(cg::cluster_group& cluster, float* base, int idx, int lo, int hi) {
  float v[CL];
#pragma unroll
  for (int r = 0; r < CL; ++r) v[r] = (r >= lo && r < hi) ? cluster.map_shared_rank(base, r)[idx] : 0.f;
  float s = 0.f;
#pragma unroll
  for (int r = 0; r < CL; ++r) s += v[r];
  return s;
}

// Rows, column slice and output slots of one CTA's share of a step's products.
struct ProdGeom {
  int kind, split, async_ok;
  int k, kp, wp, xs, rs, cl_x, w;
  int64_t nA, ld, c_lo, goff, d;
  float inv_nA, inv_nB;
  int64_t row_lo, row_hi;  // rows of this cluster within the step
  float* acc_cur;          // A_t V | B_t V slot the products are added into
  float* gram_cur;         // a | b slot
};

// Copy of chunk j of the cluster's rows (rows row_lo + j rs .., this CTA's columns) into Xb:
// cp.async when rows and slices start on 16-byte boundaries, plain loads otherwise.
template <typename T>
__device__ __forceinline__ void issue_chunk(const ProdGeom& g, const T* Z, T* Xb, int j) {
  const int tid = threadIdx.x;
  const int64_t r0 = g.row_lo + (int64_t)j * g.rs;
  const int nr = (int)min((int64_t)g.rs, g.row_hi - r0);
  if (g.async_ok) {
    constexpr int V4 = 16 / sizeof(T);
    const int nvec = g.wp / V4;
    for (int e = tid; e < g.rs * nvec; e += kThreads) {
      const int rr = e / nvec, c = (e % nvec) * V4;
      T* d = Xb + rr * g.xs + c;
      if (rr < nr && c + V4 <= g.w) {
        cp_async16(d, Z + (r0 + rr) * g.ld + g.c_lo + c);
      } else {
#pragma unroll
        for (int u = 0; u < V4; ++u)
          d[u] = (rr < nr && c + u < g.w) ? Z[(r0 + rr) * g.ld + g.c_lo + c + u] : T(0.f);
      }
    }
    cp_async_commit();
  } else {
    for (int e = tid; e < g.rs * g.wp; e += kThreads) {
      const int rr = e / g.wp, c = e % g.wp;
      Xb[rr * g.xs + c] = (rr < nr && c < g.w) ? Z[(r0 + rr) * g.ld + g.c_lo + c] : T(0.f);
    }
  }
}

// One step's products in one CTA (chunk 0 already issued): per chunk of rows, partial
// projections X_chunk V_slice (4x4 register micro-tiles), summed over the cluster into P and Q
// through distributed shared memory; the row-side k x k terms a_ij = (P^T Q + Q^T P)/n_A,
// b_i = (|P_i|^2 + |Q_i|^2)/n_B; the back-projection X_chunk^T [Q|P] in registers. Finally the
// CTA's d-slice of A_t V and B_t V and its share of the k x k terms are added into the slot.
template <typename T, int CL, typename Mark, typename Hook>
__device__ __forceinline__ void products_phase(cg::cluster_group& cluster, int rank, const ProdGeom& g, const T* Z,
                                               T* Xb, const float* VP, float* part, float* Wo, float* Wc,
                                               float* red, Mark mark, Hook after_first_sync,
                                               const float* pscale = nullptr) {
  const int tid = threadIdx.x;
  const int k = g.k, kp = g.kp, wp = g.wp, xs = g.xs, w = g.w;
  const int kk = k * k;
  const bool isY = rank >= g.cl_x;
  const int64_t goff = g.goff, row_lo = g.row_lo, row_hi = g.row_hi;
  const int nch = (int)((row_hi - row_lo + g.rs - 1) / g.rs);
  const bool cca = g.kind == SGEP_CCA;
  const bool pca = g.kind == SGEP_PCA;
  const int own_lo = isY ? g.cl_x : 0, own_hi = isY ? CL : g.cl_x;
  const int cr_lo = isY ? 0 : g.cl_x, cr_hi = isY ? g.cl_x : CL;
  const float* WA = pca ? Wo : Wc;  // A rows: the other view's projection (CCA, PLS)
  const float* Pm = isY ? Wc : Wo;  // P = X V_x
  const float* Qm = isY ? Wo : Wc;  // Q = Y V_y
  const int RS = g.rs;               // rows per super-chunk (multiple of 8)
  const int R4 = RS / 4;
  const int kq = kp >> 2;
  // projection micro-tiles: rows prg + R4*m (m < 4) x players 4*ppq .. 4*ppq+3
  const int ntp = R4 * kq;
  const int nsp = max(1, kThreads / ntp);
  const int tp = tid % ntp, sp = tid / ntp;
  const int prg = tp / kq, ppq = tp % kq;
  const int pcw = ((wp + nsp * 4 - 1) / (nsp * 4)) * 4;
  // back-projection micro-tiles: columns 4*cgp .. +3 x players 4*pq .. +3
  const int ntb = (wp >> 2) * kq;
  const int nsb = ntb >= kThreads ? 1 : min(min(kThreads / ntb, RS), 1 + kRed / (ntb * 32));
  const int sb = ntb >= kThreads ? 0 : tid / ntb;
  const int my_tile = ntb >= kThreads ? tid : tid % ntb;
  const bool bp_on = my_tile < ntb && sb < nsb;
  const int cgp = my_tile / kq, bpq = my_tile % kq;
  // row-side k x k items owned by this CTA: a_ij (p < kk) and b_i (kk <= p < kk + k)
  const int gi = rank + CL * tid;
  const bool g_on = gi < kk + k;
  float gacc = 0.f;
  float accA[16], accB[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) accA[q] = accB[q] = 0.f;

  for (int j = 0; j < nch; ++j) {
    if (j > 0) issue_chunk<T>(g, Z, Xb, j);
    cp_async_wait_all();
    __syncthreads();
    if (j == 0) mark(8);
    const int64_t r0 = row_lo + (int64_t)j * RS;
    const int nr = (int)min((int64_t)RS, row_hi - r0);
    // rows of the super-chunk that estimate A and B
    int a_lo = 0, a_hi = nr, b_lo = 0, b_hi = 0;
    if (cca) {
      if (g.split) {
        const int cut = (int)max((int64_t)0, min((int64_t)nr, g.nA - r0));
        a_hi = cut;
        b_lo = cut;
        b_hi = nr;
      } else {
        b_hi = nr;
      }
    }
    // (a) partial projections of the rows on this slice
    if (sp < nsp) {
      float acc[4][4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][q] = 0.f;
      const int c_end = min(wp, (sp + 1) * pcw);
      for (int c4 = sp * pcw; c4 < c_end; c4 += 4) {
        float4 x[4], v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) x[m] = ld4(Xb + (prg + R4 * m) * xs + c4);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) v[cc] = ld4(VP + (c4 + cc) * kp + ppq * 4);
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const float xv = comp(x[m], cc);
            acc[m][0] = fmaf(xv, v[cc].x, acc[m][0]);
            acc[m][1] = fmaf(xv, v[cc].y, acc[m][1]);
            acc[m][2] = fmaf(xv, v[cc].z, acc[m][2]);
            acc[m][3] = fmaf(xv, v[cc].w, acc[m][3]);
          }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[((m * 4 + q) * nsp + sp) * ntp + tp] = acc[m][q];
    }
    __syncthreads();
    float* pb = part + (j & 1) * RS * kp;
    // reduce over the column splits, reading consecutive words: o = slot * ntp + tile
    for (int o = tid; o < 16 * ntp; o += kThreads) {
      const int slot = o / ntp, tile = o - slot * ntp;
      const int r = (slot >> 2) * R4 + tile / kq;
      const int i = (tile % kq) * 4 + (slot & 3);
      float s = 0.f;
      for (int u = 0; u < nsp; ++u) s += red[(slot * nsp + u) * ntp + tile];
      pb[r * kp + i] = s;
    }
    if (j == 0) mark(9);
    cluster.sync();
    if (j == 0) {
      mark(10);
      after_first_sync();
      if (pscale) __syncthreads();
    }
    // the projections made with unnormalised players are scaled by 1/|v'_i| here
    for (int o = tid; o < nr * kp; o += kThreads) {
      const float f = pscale ? pscale[o & (kp - 1)] : 1.f;
      Wo[o] = cluster_sum<CL>(cluster, pb, o, own_lo, own_hi) * f;
      Wc[o] = cluster_sum<CL>(cluster, pb, o, cr_lo, cr_hi) * f;
    }
    __syncthreads();
    if (j == 0) mark(11);
    // (b) row-side k x k terms
    if (g_on) {
      if (gi < kk) {
        const int i = gi / k, jj = gi % k;
        float g0 = 0.f, g1 = 0.f;
        for (int r = a_lo; r < a_hi; ++r) {
          if (pca) {
            g0 = fmaf(Pm[r * kp + i], Pm[r * kp + jj], g0);
          } else {
            g0 = fmaf(Pm[r * kp + i], Qm[r * kp + jj], g0);
            g1 = fmaf(Qm[r * kp + i], Pm[r * kp + jj], g1);
          }
        }
        gacc += g0 + g1;
      } else if (cca) {
        const int i = gi - kk;
        float g0 = 0.f, g1 = 0.f;
        for (int r = b_lo; r < b_hi; ++r) {
          const float p = Pm[r * kp + i], q = Qm[r * kp + i];
          g0 = fmaf(p, p, g0);
          g1 = fmaf(q, q, g1);
        }
        gacc += g0 + g1;
      }
    }
    // (c) back-projection X^T W into the registers
    if (bp_on) {
      for (int r = a_lo + sb; r < a_hi; r += nsb) {
        const float4 x = ld4(Xb + r * xs + cgp * 4);
        const float4 y = ld4(WA + r * kp + bpq * 4);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const float xv = comp(x, cc);
          accA[cc * 4 + 0] = fmaf(xv, y.x, accA[cc * 4 + 0]);
          accA[cc * 4 + 1] = fmaf(xv, y.y, accA[cc * 4 + 1]);
          accA[cc * 4 + 2] = fmaf(xv, y.z, accA[cc * 4 + 2]);
          accA[cc * 4 + 3] = fmaf(xv, y.w, accA[cc * 4 + 3]);
        }
      }
      for (int r = b_lo + sb; r < b_hi; r += nsb) {
        const float4 x = ld4(Xb + r * xs + cgp * 4);
        const float4 y = ld4(Wo + r * kp + bpq * 4);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const float xv = comp(x, cc);
          accB[cc * 4 + 0] = fmaf(xv, y.x, accB[cc * 4 + 0]);
          accB[cc * 4 + 1] = fmaf(xv, y.y, accB[cc * 4 + 1]);
          accB[cc * 4 + 2] = fmaf(xv, y.z, accB[cc * 4 + 2]);
          accB[cc * 4 + 3] = fmaf(xv, y.w, accB[cc * 4 + 3]);
        }
      }
    }
    __syncthreads();
  }
  mark(12);

  // combine the row splits of the back-projection, then add into the slot
  const bool hasA = row_lo < row_hi && (!cca || !g.split || row_lo < g.nA);
  const bool hasB = row_lo < row_hi && cca && (!g.split || row_hi > g.nA);
  if (nsb > 1) {
    // layout [value q][split][tile]: consecutive threads touch consecutive words
    const int nsm = nsb - 1;
    if (bp_on && sb > 0) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        red[(q * nsm + sb - 1) * ntb + my_tile] = accA[q];
        red[((16 + q) * nsm + sb - 1) * ntb + my_tile] = accB[q];
      }
    }
    __syncthreads();
    if (bp_on && sb == 0) {
      for (int u = 0; u < nsm; ++u) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          accA[q] += red[(q * nsm + u) * ntb + my_tile];
          accB[q] += red[((16 + q) * nsm + u) * ntb + my_tile];
        }
      }
    }
  }
  mark(13);
  float* AVc = g.acc_cur;
  float* BVc = g.acc_cur + g.d * k;
  if (bp_on && sb == 0) {
    const bool vec = (k & 3) == 0;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int c = cgp * 4 + cc;
      if (c >= w) continue;
      const int64_t g0 = (goff + c) * k + bpq * 4;
      if (vec && bpq * 4 < k) {
        if (hasA)
          atomicAdd(reinterpret_cast<float4*>(AVc + g0),
                    make_float4(accA[cc * 4] * g.inv_nA, accA[cc * 4 + 1] * g.inv_nA,
                                accA[cc * 4 + 2] * g.inv_nA, accA[cc * 4 + 3] * g.inv_nA));
        if (hasB)
          atomicAdd(reinterpret_cast<float4*>(BVc + g0),
                    make_float4(accB[cc * 4] * g.inv_nB, accB[cc * 4 + 1] * g.inv_nB,
                                accB[cc * 4 + 2] * g.inv_nB, accB[cc * 4 + 3] * g.inv_nB));
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (bpq * 4 + q >= k) continue;
          if (hasA) atomicAdd(AVc + g0 + q, accA[cc * 4 + q] * g.inv_nA);
          if (hasB) atomicAdd(BVc + g0 + q, accB[cc * 4 + q] * g.inv_nB);
        }
      }
    }
  }
  if (g_on && row_lo < row_hi) {
    if (gi < kk) {
      if (hasA) atomicAdd(&g.gram_cur[gi], gacc * g.inv_nA);
    } else if (cca && hasB) {
      atomicAdd(&g.gram_cur[gi], gacc * g.inv_nB);
    }
  }
}

template <typename T, int CLT>
__global__ void __launch_bounds__(kThreads, 1) k_cluster_step(const ClArgs a) {
  const long long t0 = clock64();
  if (a.trace && threadIdx.x == 0) {
    unsigned long long g;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g));
    a.trace[blockIdx.x * kTracePhases] = g;
  }
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int CL = CLT;
  const int rank = (int)cluster.block_rank();
  const int cid = (int)(blockIdx.x / CL);
  const int tid = threadIdx.x;
  const int k = a.k, kp = a.kp, wp = a.wp, xs = a.xs;
  const int kk = k * k;

  const bool isY = rank >= a.cl_x;
  const int vr = isY ? rank - a.cl_x : rank;
  const int64_t ld = isY ? a.d_y : a.d_x;
  const int wn = isY ? a.w_y : a.w_x;
  const int64_t c_lo = min((int64_t)vr * wn, ld);
  const int64_t c_hi = min(c_lo + wn, ld);
  const int w = (int)(c_hi - c_lo);
  const int64_t goff = (isY ? a.d_x : 0) + c_lo;  // first row of V owned here

  extern __shared__ __align__(16) float sm[];
  float* VP = sm;                      // wp*kp: V slice, then the new V slice (zero padded)
  float* SP = VP + wp * kp;            // wp*kp: [Bv] slice
  float* UP = SP + wp * kp;            // wp*kp: v + eta grad
  T* Xb = reinterpret_cast<T*>(UP + wp * kp);                 // rs*xs: minibatch rows
  float* part = reinterpret_cast<float*>(Xb + a.rs * xs);     // 2*rs*kp (double buffer)
  float* Wo = part + 2 * a.rs * kp;    // rs*kp: projection of this CTA's view
  float* Wc = Wo + a.rs * kp;          // rs*kp: projection of the other view
  float* red = Wc + a.rs * kp;         // kRed
  float* Gp = red + kRed;              // k*k + k: partial G | v.v   (read by the cluster)
  float* np_ = Gp + kk + k;            // k: partial norms^2          (read by the cluster)
  float* terms = np_ + k;              // 2k*k + k: a | G | b
  float* vv = terms + 2 * kk + k;      // k
  float* Tm = vv + k;                  // k*k
  float* cb = Tm + kk;                 // k
  float* cac = cb + k;                 // k
  float* nrm = cac + k;                // k
  float* scr = nrm + k;                // kThreads

  // ---- rows of this cluster; prefetch of its first super-chunk ----
  const bool products = a.acc_cur != nullptr;
  const int64_t row_lo = products ? min((int64_t)cid * a.rows_per_cluster, a.b) : 0;
  const int64_t row_hi = products ? min(row_lo + a.rows_per_cluster, a.b) : 0;
  const int nch = (int)((row_hi - row_lo + a.rs - 1) / a.rs);
  const T* Z = reinterpret_cast<const T*>(isY ? a.Y : a.X);
  ProdGeom g;
  g.kind = a.kind;
  g.split = a.split;
  g.async_ok = a.async_ok;
  g.k = k;
  g.kp = kp;
  g.wp = wp;
  g.xs = xs;
  g.rs = a.rs;
  g.cl_x = a.cl_x;
  g.w = w;
  g.nA = a.nA;
  g.ld = ld;
  g.c_lo = c_lo;
  g.goff = goff;
  g.d = a.d;
  g.inv_nA = a.inv_nA;
  g.inv_nB = a.inv_nB;
  g.row_lo = row_lo;
  g.row_hi = row_hi;
  g.acc_cur = a.acc_cur;
  g.gram_cur = a.gram_cur;
  if (products && nch > 0) issue_chunk<T>(g, Z, Xb, 0);

  // Everything below reads what the previous launch wrote.
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" :::);
  mark(a, 1, t0);

  // Clear the slots of the step after next (the whole grid shares the work).
  if (a.acc_zero) {
    const int64_t n = 2 * a.d * k;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + tid; e < n; e += (int64_t)gridDim.x * kThreads)
      a.acc_zero[e] = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + tid; e < kk + k; e += (int64_t)gridDim.x * kThreads)
      a.gram_zero[e] = 0.f;
  }

  // ---------------- 1. pending update ----------------
  const int ne = wp * kp;  // padded slice elements; thread owns e = tid + kThreads * u
  const bool pend = a.acc_prev != nullptr;
  for (int e0 = 0; e0 < ne; e0 += kEB * kThreads) {
    float rv[kEB], rs[kEB];
#pragma unroll
    for (int u = 0; u < kEB; ++u) {
      const int e = e0 + u * kThreads + tid;
      const int c = e / kp, i = e % kp;
      const bool ok = e < ne && c < w && i < k;
      const int64_t g = (goff + c) * k + i;
      rv[u] = ok ? __ldg(a.V_in + g) : 0.f;
      rs[u] = (ok && pend) ? __ldg(a.S_in + g) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kEB; ++u) {
      const int e = e0 + u * kThreads + tid;
      if (e < ne) {
        VP[e] = rv[u];
        if (pend) SP[e] = rs[u];
      }
    }
  }
  if (pend) {
    const float* AVp = a.acc_prev;
    const float* BVp = a.acc_prev + a.d * k;
    for (int p = tid; p < kk; p += kThreads) terms[p] = __ldg(a.gram_prev + p);
    __syncthreads();
    mark(a, 2, t0);
    for (int p = tid; p < kk; p += kThreads) {
      const int i = p / k, j = p % k;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int c = 0;
      for (; c + 3 < w; c += 4) {
        s0 = fmaf(VP[c * kp + i], SP[c * kp + j], s0);
        s1 = fmaf(VP[(c + 1) * kp + i], SP[(c + 1) * kp + j], s1);
        s2 = fmaf(VP[(c + 2) * kp + i], SP[(c + 2) * kp + j], s2);
        s3 = fmaf(VP[(c + 3) * kp + i], SP[(c + 3) * kp + j], s3);
      }
      for (; c < w; ++c) s0 = fmaf(VP[c * kp + i], SP[c * kp + j], s0);
      Gp[p] = (s0 + s1) + (s2 + s3);
    }
    colsum_prod(VP, VP, kp, w, k, scr, Gp + kk);
    mark(a, 3, t0);
    cluster.sync();
    mark(a, 4, t0);
    for (int p = tid; p < kk + k; p += kThreads) {
      const float s = cluster_sum<CL>(cluster, Gp, p, 0, CL);
      if (p < kk) terms[kk + p] = s;
      else vv[p - kk] = s;
    }
    __syncthreads();
    for (int i = tid; i < k; i += kThreads)
      terms[2 * kk + i] = a.b_is_identity ? (1.f + a.eps_B) * vv[i] : fmaf(a.eps_B, vv[i], a.gram_prev[kk + i]);
    __syncthreads();
    eg_coefficients(terms, k, a.rho, cb, cac, Tm);
    __syncthreads();
    mark(a, 5, t0);
    const bool writer = cid == 0;
    const float e1 = 1.f + a.eps_B;
    for (int e0 = 0; e0 < ne; e0 += kEB * kThreads) {
      float av[kEB], bvr[kEB], pen[kEB];
      int cu[kEB], iu[kEB];
      bool oku[kEB];
#pragma unroll
      for (int u = 0; u < kEB; ++u) {
        const int e = e0 + u * kThreads + tid;
        cu[u] = e / kp;
        iu[u] = e % kp;
        oku[u] = e < ne && cu[u] < w && iu[u] < k;
        const int64_t g = (goff + cu[u]) * k + iu[u];
        av[u] = oku[u] ? __ldg(AVp + g) : 0.f;
        bvr[u] = (oku[u] && !a.b_is_identity) ? __ldg(BVp + g) : 0.f;
        pen[u] = 0.f;
      }
      // penalty sum_{j<i} [Bv]_j T_ji; T_ji is zero for j >= i
      for (int j = 0; j < k; ++j) {
#pragma unroll
        for (int u = 0; u < kEB; ++u)
          if (oku[u]) pen[u] = fmaf(SP[cu[u] * kp + j], Tm[j * k + iu[u]], pen[u]);
      }
#pragma unroll
      for (int u = 0; u < kEB; ++u) {
        if (!oku[u]) continue;
        const int e = cu[u] * kp + iu[u];
        const int64_t g = (goff + cu[u]) * k + iu[u];
        const float v = VP[e];
        const float s_old = SP[e];
        const float bv = a.b_is_identity ? e1 * v : fmaf(a.eps_B, v, bvr[u]);
        const float gr = cb[iu[u]] * av[u] - cac[iu[u]] * bv - pen[u];
        if (writer) {
          a.S_out[g] = fmaf(a.gamma, bv - s_old, s_old);
          if (a.grad_dbg) a.grad_dbg[g] = gr;
        }
        UP[e] = fmaf(a.eta, gr, v);
      }
    }
    __syncthreads();
    mark(a, 6, t0);
    colsum_prod(UP, UP, kp, w, k, scr, np_);
    cluster.sync();
    for (int i = tid; i < k; i += kThreads) nrm[i] = cluster_sum<CL>(cluster, np_, i, 0, CL);
    __syncthreads();
    for (int e = tid; e < w * k; e += kThreads) {
      const int c = e / k, i = e % k;
      const float v = UP[c * kp + i] / sqrtf(nrm[i]);
      if (!isfinite(v)) atomicOr(a.dflag, kFlagNonFinite);
      VP[c * kp + i] = v;
      if (writer) a.V_out[goff * k + e] = v;
    }
    if (writer && rank == 0 && a.gram_dbg) {
      for (int p = tid; p < 2 * kk + k; p += kThreads) a.gram_dbg[p] = terms[p];
      for (int i = tid; i < k; i += kThreads) a.gram_dbg[2 * kk + k + i] = nrm[i];
    }
  }
  __syncthreads();
  mark(a, 7, t0);

  // ---------------- 2. products of the new minibatch ----------------
  if (products) {
    products_phase<T, CL>(cluster, rank, g, Z, Xb, VP, part, Wo, Wc, red, [&](int ph) { mark(a, ph, t0); },
                          [] {});
  }
  mark(a, 14, t0);
  // No CTA may leave while others can still read its shared memory.
  cluster.sync();
  mark(a, 15, t0);
}

// ---------------------------------------------------------------------------
// Several steps in one launch. Each step does the work of k_cluster_step (the pending
// update, then the products of the step's minibatch); between steps a bounded grid barrier
// takes the place of the launch boundary. The players' and auxiliary slices stay in shared
// memory, and the cluster sums G_ij = <v_i, [Bv]_j>, |v_i|^2 that the next update needs are
// formed after the CTA has arrived at the barrier, while the other CTAs are still adding
// their products. A CTA whose wait runs out records the timeout and stops waiting, but keeps
// executing every cluster barrier, so no cluster is left waiting on a barrier it will not reach.
constexpr int kMsMax = 64;  // steps of one launch

struct MsArgs {
  const void* X;            // nsteps * b rows (step s: rows s b .. s b + b - 1)
  const void* Y;
  int64_t b, nA;
  int64_t d_x, d_y, d;
  int k, kp, kind, split, b_is_identity;
  float inv_nA, inv_nB;
  float rho, eps_B;
  int cl_x, w_x, w_y, wp, xs, rs;
  int64_t rows_per_cluster;
  int async_ok;
  int nsteps;
  int pend0;                // step 0 first applies the update of products made before the launch
  int slot0;                // slot of those products; step s adds its own into (slot0 + s + 1) % 3
  float eta[kMsMax];        // step sizes of the update applied at the start of step s
  float gamma[kMsMax];
  const float* V_in;
  const float* S_in;
  float* V_out;             // state after the last applied update (cluster 0)
  float* S_out;
  float* acc;               // three slots of A_t V | B_t V (2 d k)
  float* gram;              // three slots of a | b (k k + k)
  unsigned* bar;            // grid-barrier arrivals (monotone across launches)
  unsigned bar_base;        // its value at the launch
  int* dflag;
  unsigned long long* trace;  // [grid][kTracePhases] globaltimer stamps of the step before the last, or null
};

// the second [Bv] buffer, its 16-byte alignment and the status word
size_t ms_extra_smem(int wp, int kp) { return (size_t)wp * kp * sizeof(float) + 32; }

template <typename T, int CLT>
__global__ void __launch_bounds__(kThreads, 1) k_cluster_steps(const __grid_constant__ MsArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int CL = CLT;
  const int rank = (int)cluster.block_rank();
  const int cid = (int)(blockIdx.x / CL);
  const int tid = threadIdx.x;
  const int k = a.k, kp = a.kp, wp = a.wp, xs = a.xs;
  const int kk = k * k;
  const bool isY = rank >= a.cl_x;
  const int vr = isY ? rank - a.cl_x : rank;
  const int64_t ld = isY ? a.d_y : a.d_x;
  const int wn = isY ? a.w_y : a.w_x;
  const int64_t c_lo = min((int64_t)vr * wn, ld);
  const int64_t c_hi = min(c_lo + wn, ld);
  const int w = (int)(c_hi - c_lo);
  const int64_t goff = (isY ? a.d_x : 0) + c_lo;
  const size_t dk = (size_t)a.d * k, gk = (size_t)kk + k;

  extern __shared__ __align__(16) float sm[];
  float* VP = sm;                      // wp*kp: the players' slice (unit columns)
  float* UP = VP + wp * kp;            // wp*kp: v + eta grad
  T* Xb = reinterpret_cast<T*>(UP + wp * kp);                 // rs*xs: minibatch rows
  float* part = reinterpret_cast<float*>(Xb + a.rs * xs);     // 2*rs*kp
  float* Wo = part + 2 * a.rs * kp;    // rs*kp
  float* Wc = Wo + a.rs * kp;          // rs*kp
  float* red = Wc + a.rs * kp;         // kRed
  float* Gp = red + kRed;              // k*k + k: partial G | v.v   (read by the cluster)
  float* rinv = Gp + kk + k;           // k: 1 / |v'_i| of the step's players
  float* terms = rinv + k;             // 2k*k + k: a | G | b
  float* vv = terms + 2 * kk + k;      // k
  float* Tm = vv + k;                  // k*k
  float* cb = Tm + kk;                 // k
  float* cac = cb + k;                 // k
  float* nrm = cac + k;                // k: |v'_i|^2
  float* scr = nrm + k;                // kThreads
  // wp*kp: [Bv] slice (two buffers, swapped by the update), 16-byte aligned for float4 reads
  float* SA = reinterpret_cast<float*>(((uintptr_t)(scr + kThreads) + 15) & ~(uintptr_t)15);
  int* dead_s = reinterpret_cast<int*>(SA + wp * kp + wp * kp);
  float* Scur = SA;
  float* Snew = SA + wp * kp;

  ProdGeom g;
  g.kind = a.kind;
  g.split = a.split;
  g.async_ok = a.async_ok;
  g.k = k;
  g.kp = kp;
  g.wp = wp;
  g.xs = xs;
  g.rs = a.rs;
  g.cl_x = a.cl_x;
  g.w = w;
  g.nA = a.nA;
  g.ld = ld;
  g.c_lo = c_lo;
  g.goff = goff;
  g.d = a.d;
  g.inv_nA = a.inv_nA;
  g.inv_nB = a.inv_nB;
  g.row_lo = min((int64_t)cid * a.rows_per_cluster, a.b);
  g.row_hi = min(g.row_lo + a.rows_per_cluster, a.b);
  const int nch = (int)((g.row_hi - g.row_lo + a.rs - 1) / a.rs);
  const T* Z0 = reinterpret_cast<const T*>(isY ? a.Y : a.X);
  if (nch > 0) issue_chunk<T>(g, Z0, Xb, 0);

  // resident slices of V and [Bv] (written before the launch)
  for (int e = tid; e < wp * kp; e += kThreads) {
    const int c = e / kp, i = e % kp;
    const bool ok = c < w && i < k;
    const int64_t gi = (goff + c) * k + i;
    VP[e] = ok ? __ldg(a.V_in + gi) : 0.f;
    Scur[e] = ok ? __ldg(a.S_in + gi) : 0.f;
    Snew[e] = 0.f;
  }
  if (tid == 0) *dead_s = 0;
  __syncthreads();

  // G_ij = <v_i, [Bv]_j> and |v_i|^2 of the current slices, summed over the cluster (fixed order)
  auto gram = [&](const float* Sc) {
    for (int p = tid; p < kk; p += kThreads) {
      const int i = p / k, j = p % k;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int c = 0;
      for (; c + 3 < w; c += 4) {
        s0 = fmaf(VP[c * kp + i], Sc[c * kp + j], s0);
        s1 = fmaf(VP[(c + 1) * kp + i], Sc[(c + 1) * kp + j], s1);
        s2 = fmaf(VP[(c + 2) * kp + i], Sc[(c + 2) * kp + j], s2);
        s3 = fmaf(VP[(c + 3) * kp + i], Sc[(c + 3) * kp + j], s3);
      }
      for (; c < w; ++c) s0 = fmaf(VP[c * kp + i], Sc[c * kp + j], s0);
      Gp[p] = (s0 + s1) + (s2 + s3);
    }
    colsum_prod(VP, VP, kp, w, k, scr, Gp + kk);
    cluster.sync();
    for (int p = tid; p < kk + k; p += kThreads) {
      const float s = cluster_sum<CL>(cluster, Gp, p, 0, CL);
      if (p < kk) terms[kk + p] = s;
      else vv[p - kk] = s;
    }
    __syncthreads();
  };
  if (a.pend0) gram(Scur);
  // partial G_ij = sum_c v_ci s_cj and |v_i|^2 over the slice: 4 x 4 register tiles of the
  // padded kp x kp output, column groups c = cg, cg + ncg, ..., the groups summed in a fixed
  // order into Gp (the cluster sums are taken at the products' first cluster barrier)
  // partial tiles stored as float4 rows with row stride kp + 4 (a quarter warp's stores then fall
  // in distinct banks); the column groups are as many as red and scr hold
  const int gt_n = (kp / 4) * (kp / 4);             // tiles
  const int gt_ld = kp + 4, gt_rs = kp * gt_ld;     // row stride, group stride
  const int gt_cg = min(min(kThreads / gt_n, kThreads / kp), kRed / gt_rs);
  auto gram_partial = [&](const float* PV, const float* Sc) {
    const int tile = tid % gt_n, cg = tid / gt_n;
    const int ti = tile / (kp / 4), tj = tile % (kp / 4);
    if (cg < gt_cg) {
      float acc[4][4] = {};
      float n2[4] = {};
      for (int c = cg; c < w; c += gt_cg) {
        const float4 v = *reinterpret_cast<const float4*>(PV + c * kp + 4 * ti);
        const float4 t = *reinterpret_cast<const float4*>(Sc + c * kp + 4 * tj);
        const float va[4] = {v.x, v.y, v.z, v.w};
        const float ta[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int x = 0; x < 4; ++x) {
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(va[x], ta[y], acc[x][y]);
          n2[x] = fmaf(va[x], va[x], n2[x]);
        }
      }
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        *reinterpret_cast<float4*>(red + cg * gt_rs + (4 * ti + x) * gt_ld + 4 * tj) =
            make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
        if (tj == 0) scr[cg * kp + 4 * ti + x] = n2[x];
      }
    }
    __syncthreads();
    for (int p = tid; p < kk + k; p += kThreads) {
      float sum = 0.f;
      if (p < kk) {
        const int o = (p / k) * gt_ld + p % k;
        for (int u = 0; u < gt_cg; ++u) sum += red[u * gt_rs + o];
      } else {
        for (int u = 0; u < gt_cg; ++u) sum += scr[u * kp + p - kk];
      }
      Gp[p] = sum;
    }
    __syncthreads();
  };
  // cluster sums of the partials: |v'_i|^2, 1/|v'_i| and |v_i|^2 of the retracted players
  // v_i = v'_i / |v'_i|, and <v'_i, [Bv]_j> (its row i is scaled by 1/|v'_i| at the next
  // update); `scaled` says whether the partials were of unnormalised players
  bool scaled = false;
  for (int i = tid; i < k; i += kThreads) rinv[i] = 1.f;
  __syncthreads();
  auto gram_sum = [&]() {
    for (int p = tid; p < kk + k; p += kThreads) {
      const float sv = cluster_sum<CL>(cluster, Gp, p, 0, CL);
      if (p < kk) {
        terms[kk + p] = sv;
      } else {
        const int i = p - kk;
        const float r = scaled ? 1.f / sqrtf(sv) : 1.f;
        nrm[i] = sv;
        rinv[i] = r;
        vv[i] = scaled ? sv * r * r : sv;
      }
    }
  };

  bool applied = false;  // an update has changed the resident slices
  for (int s = 0; s < a.nsteps; ++s) {
    // phase stamps of the step before the last: 0 top, 1 barrier passed, 2 coefficients,
    // 3 update directions, 4 norms summed, 5 players retracted, 8-14 products, 15 Gram done
    auto stamp = [&](int ev) {
      if (a.trace && tid == 0 && s == a.nsteps - 2) a.trace[(size_t)blockIdx.x * kTracePhases + ev] = tc::globaltimer();
    };
    stamp(0);
    const bool pend = s > 0 || a.pend0;
    const int pslot = (a.slot0 + s) % 3;  // products waiting for their update
    const int wslot = (pslot + 1) % 3;    // this step's products
    const int zslot = (pslot + 2) % 3;    // read by the previous step, written by the next one
    const T* Z = Z0 + (size_t)s * (size_t)a.b * (size_t)ld;
    if (s > 0) {
      // every CTA has added the previous step's products
      if (tid == 0 && !*dead_s && !tc::spin_until_geq(a.bar, a.bar_base + (unsigned)s * gridDim.x)) {
        atomicOr(a.dflag, kFlagTimeout);
        *dead_s = 1;
      }
      __syncthreads();
    }
    stamp(1);
    {
      float* az = a.acc + zslot * 2 * dk;
      float* gz = a.gram + zslot * gk;
      for (int64_t e = (int64_t)blockIdx.x * kThreads + tid; e < (int64_t)(2 * dk); e += (int64_t)gridDim.x * kThreads)
        az[e] = 0.f;
      for (int64_t e = (int64_t)blockIdx.x * kThreads + tid; e < (int64_t)gk; e += (int64_t)gridDim.x * kThreads)
        gz[e] = 0.f;
    }
    if (pend) {
      // ---- the pending update (Alg. 2), on the resident slices ----
      const float* AVp = a.acc + pslot * 2 * dk;
      const float* BVp = AVp + dk;
      const float* gp = a.gram + pslot * gk;
      const int ne = wp * kp;
      float av[kEB], bvr[kEB], pen[kEB];
      int cu[kEB], iu[kEB];
      bool oku[kEB];
      auto load_block = [&](int e0) {  // A_t V and B_t V of this thread's elements of block e0
#pragma unroll
        for (int u = 0; u < kEB; ++u) {
          const int e = e0 + u * kThreads + tid;
          cu[u] = e / kp;
          iu[u] = e % kp;
          oku[u] = e < ne && cu[u] < w && iu[u] < k;
          const int64_t gi = (goff + cu[u]) * k + iu[u];
          av[u] = oku[u] ? __ldcg(AVp + gi) : 0.f;
          bvr[u] = (oku[u] && !a.b_is_identity) ? __ldcg(BVp + gi) : 0.f;
          pen[u] = 0.f;
        }
      };
      load_block(0);  // in flight while the coefficients are built
      for (int p = tid; p < kk; p += kThreads) {
        terms[p] = __ldcg(gp + p);
        terms[kk + p] *= rinv[p / k];  // G of the retracted players
      }
      for (int i = tid; i < k; i += kThreads)
        terms[2 * kk + i] = a.b_is_identity ? (1.f + a.eps_B) * vv[i] : fmaf(a.eps_B, vv[i], __ldcg(gp + kk + i));
      __syncthreads();
      // coefficients of Eq. (update): T_ji = b_i a_ij / s_j (j < i), c_i = sum_{j<i} a_ij G_ij / s_j,
      // with s_j = max(G_jj, rho) inverted once and c_i summed by one warp per player
      {
        const float* ta = terms;
        const float* tG = terms + kk;
        const float* tb = terms + 2 * kk;
        for (int j = tid; j < k; j += kThreads) scr[j] = 1.f / fmaxf(tG[j * k + j], a.rho);
        __syncthreads();
        for (int p = tid; p < kk; p += kThreads) {
          const int j = p / k, i = p % k;
          Tm[p] = j < i ? tb[i] * ta[i * k + j] * scr[j] : 0.f;
        }
        const int wid = tid >> 5, ln = tid & 31;
        for (int i = wid; i < k; i += kThreads / 32) {
          float c = ln < i ? ta[i * k + ln] * tG[i * k + ln] * scr[ln] : 0.f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
          if (ln == 0) {
            cb[i] = tb[i];
            cac[i] = ta[i * k + i] - c;
          }
        }
      }
      __syncthreads();
      stamp(2);
      const float eta = a.eta[s], gamma = a.gamma[s];
      const float e1 = 1.f + a.eps_B;
      for (int e0 = 0; e0 < ne; e0 += kEB * kThreads) {
        if (e0 > 0) load_block(e0);
        // penalty sum_{j<i} [Bv]_j T_ji; T_ji is zero for j >= i
        for (int j = 0; j < k; ++j) {
#pragma unroll
          for (int u = 0; u < kEB; ++u)
            if (oku[u]) pen[u] = fmaf(Scur[cu[u] * kp + j], Tm[j * k + iu[u]], pen[u]);
        }
#pragma unroll
        for (int u = 0; u < kEB; ++u) {
          const int e = e0 + u * kThreads + tid;
          if (e >= ne) continue;
          if (!oku[u]) {
            UP[e] = 0.f;
            Snew[e] = 0.f;
            continue;
          }
          const float v = VP[e];
          const float s_old = Scur[e];
          const float bv = a.b_is_identity ? e1 * v : fmaf(a.eps_B, v, bvr[u]);
          const float gr = cb[iu[u]] * av[u] - cac[iu[u]] * bv - pen[u];
          Snew[e] = fmaf(gamma, bv - s_old, s_old);
          UP[e] = fmaf(eta, gr, v);
        }
      }
      __syncthreads();
      stamp(3);
    }
    // Retraction deferred: the products use v' = v + eta grad, and the partial |v'_i|^2 and
    // <v'_i, [Bv]'_j> are summed over the cluster at the products' first cluster barrier, where
    // the gathered projections are scaled by 1/|v'_i| (the projections of the retracted players)
    const float* PV = pend ? UP : VP;
    const float* PS = pend ? Snew : Scur;
    scaled = pend;
    gram_partial(PV, PS);
    stamp(5);
    // ---- products of this step's minibatch ----
    g.acc_cur = a.acc + wslot * 2 * dk;
    g.gram_cur = a.gram + wslot * gk;
    products_phase<T, CL>(cluster, rank, g, Z, Xb, PV, part, Wo, Wc, red, [&](int ph) { stamp(ph); }, gram_sum,
                          pend ? rinv : nullptr);
    if (nch == 0) {  // no chunk, so no barrier inside the products (the same in the whole cluster)
      cluster.sync();
      gram_sum();
    }
    // work that does not depend on the products' atomics, while they complete: the next step's
    // first rows and the retraction itself
    if (s + 1 < a.nsteps && nch > 0) issue_chunk<T>(g, Z + (size_t)a.b * (size_t)ld, Xb, 0);
    if (pend) {
      __syncthreads();
      for (int e = tid; e < wp * kp; e += kThreads) {
        const int c = e / kp, i = e % kp;
        float v = 0.f;
        if (c < w && i < k) {
          v = UP[e] / sqrtf(nrm[i]);
          if (!isfinite(v)) atomicOr(a.dflag, kFlagNonFinite);
        }
        VP[e] = v;
      }
      float* t = Scur;
      Scur = Snew;
      Snew = t;
      applied = true;
    }
    if (s + 1 < a.nsteps) {
      // arrive: this CTA's products and clears are in
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        atomicAdd(a.bar, 1u);
      }
      stamp(15);
    }
    __syncthreads();
  }
  // the state after the last applied update
  if (applied && cid == 0) {
    for (int e = tid; e < w * k; e += kThreads) {
      const int c = e / k, i = e % k;
      a.V_out[goff * k + e] = VP[c * kp + i];
      a.S_out[goff * k + e] = Scur[c * kp + i];
    }
  }
  // No CTA may leave while others can still read its shared memory.
  cluster.sync();
}

struct Plan {
  int CL, cl_x, wx, wy, wp, kp, lkp, xs, rs;
  size_t smem;
};

size_t smem_bytes(int wp, int kp, int k, int xs, int esz, int rs) {
  const size_t f = (size_t)3 * wp * kp + (size_t)4 * rs * kp + kRed + (size_t)(k * k + k) + k +
                   (size_t)(2 * k * k + k) + k + (size_t)k * k + 3 * k + kThreads;
  return f * sizeof(float) + (size_t)rs * xs * esz + 64;
}

// Column split (X gets cl_x CTAs of the cluster, Y the rest), padding and the number of
// minibatch rows a CTA keeps resident (rs, a multiple of 8 chosen to cover the rows one
// cluster streams when shared memory allows).
bool make_plan(const Ctx& c, int CL, int max_clusters, Plan* p) {
  p->CL = CL;
  if (!c.has_y) {
    p->cl_x = CL;
  } else {
    int x = (int)((double)CL * (double)c.d_x / (double)c.d + 0.5);
    p->cl_x = std::min(CL - 1, std::max(1, x));
  }
  p->wx = (int)((c.d_x + p->cl_x - 1) / p->cl_x);
  p->wy = c.has_y ? (int)((c.d_y + (CL - p->cl_x) - 1) / (CL - p->cl_x)) : 0;
  const int wm = std::max(p->wx, p->wy);
  p->wp = ((wm + 7) / 8) * 8;
  p->kp = 4;
  p->lkp = 2;
  while (p->kp < c.k) {
    p->kp *= 2;
    ++p->lkp;
  }
  const int esz = c.cfg.dtype == SGEP_BF16 ? 2 : 4;
  p->xs = p->wp + (esz == 4 ? 4 : 8);
  const int nc = std::max(1, std::min(c.num_sms / CL, max_clusters > 0 ? max_clusters : c.num_sms / CL));
  const int64_t rows = (c.cfg.max_b + nc - 1) / nc;
  // resident rows: a multiple of 8 (the micro-tiles need 4), at most 128
  int rs = (int)std::min<int64_t>(128, ((rows + 7) / 8) * 8);
  while (rs > 8 && smem_bytes(p->wp, p->kp, c.k, p->xs, esz, rs) > 227 * 1024) rs -= 8;
  p->rs = rs;
  p->smem = smem_bytes(p->wp, p->kp, c.k, p->xs, esz, rs);
  return p->wp <= kMaxW && p->kp <= kMaxKP && p->smem <= 227 * 1024;
}

template <typename T, int CLT>
int launch(Ctx& c, const ClArgs& a, int NC, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(NC * c.cl_size));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = c.cl_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c.cl_size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = c.cl_pdl ? 2 : 1;
  SGEP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cluster_step<T, CLT>, a));
  ++c.launches;
  return SGEP_OK;
}

template <typename T, int CLT>
int configure(Ctx& c) {
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_cluster_step<T, CLT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)c.cl_smem));
  if (CLT > 8)
    SGEP_CUDA_TRY(cudaFuncSetAttribute(k_cluster_step<T, CLT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
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
  SGEP_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, k_cluster_step<T, CLT>, &cfg));
  if (nclusters < 1) {
    set_error("cluster path: no cluster of this size fits on the device");
    return SGEP_ELAUNCH;
  }
  c.cl_max_clusters = nclusters;
  return SGEP_OK;
}

int run(Ctx& c, const void* X, const void* Y, int64_t b, float eta, float gamma, cudaStream_t s) {
  ClArgs a = {};
  a.d_x = c.d_x;
  a.d_y = c.d_y;
  a.d = c.d;
  a.k = c.k;
  a.kp = c.cl_kp;
  a.kind = c.cfg.kind;
  a.split = (c.cfg.kind == SGEP_CCA && c.cfg.split_AB) ? 1 : 0;
  a.b_is_identity = c.b_is_identity ? 1 : 0;
  a.rho = c.cfg.rho;
  a.eps_B = c.cfg.eps_B;
  a.cl_x = c.cl_x;
  a.w_x = c.cl_wx;
  a.w_y = c.cl_wy;
  a.wp = c.cl_wmax;
  a.xs = c.cl_xs;
  a.rs = c.cl_rs;
  a.lkp = c.cl_lkp;
  a.dflag = c.dflag;
  a.grad_dbg = c.cfg.debug ? c.grad : nullptr;
  a.gram_dbg = c.cfg.debug ? c.gram : nullptr;
  a.trace = X ? c.trace : nullptr;
  const int pending = c.cl_pending;
  const size_t slot = (size_t)2 * c.d * c.k;
  const size_t gslot = (size_t)c.k * c.k + c.k;
  a.V_in = c.cl_V[c.cl_cur];
  a.S_in = c.cl_S[c.cl_cur];
  a.V_out = c.cl_V[1 - c.cl_cur];
  a.S_out = c.cl_S[1 - c.cl_cur];
  a.acc_prev = pending ? c.cl_acc + c.cl_slot * slot : nullptr;
  a.gram_prev = pending ? c.cl_gram + c.cl_slot * gslot : nullptr;
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
    a.gram_cur = c.cl_gram + next * gslot;
    a.acc_zero = c.cl_acc + ((c.cl_slot + 2) % 3) * slot;
    a.gram_zero = c.cl_gram + ((c.cl_slot + 2) % 3) * gslot;
    const int max_nc = std::max(1, std::min(c.num_sms / c.cl_size, c.cl_max_clusters));
    NC = (int)std::min<int64_t>(max_nc, std::max<int64_t>(1, (b + 63) / 64));
    a.rows_per_cluster = (b + NC - 1) / NC;
    const bool aligned = ((uintptr_t)X % 16 == 0) && (!c.has_y || (uintptr_t)Y % 16 == 0);
    a.async_ok = (aligned && c.cl_async_shape) ? 1 : 0;
  }
  int rc;
  if (c.cfg.dtype == SGEP_BF16)
    rc = c.cl_size == 16 ? launch<__nv_bfloat16, 16>(c, a, NC, s) : launch<__nv_bfloat16, 8>(c, a, NC, s);
  else
    rc = c.cl_size == 16 ? launch<float, 16>(c, a, NC, s) : launch<float, 8>(c, a, NC, s);
  if (rc) return rc;
  if (X) {
    c.cl_last_grid = NC * c.cl_size;
    c.cl_ms_traced = 0;
  }
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

template <typename T, int CLT>
int ms_configure(Ctx& c) {
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_cluster_steps<T, CLT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)c.cl_ms_smem));
  if (CLT > 8)
    SGEP_CUDA_TRY(cudaFuncSetAttribute(k_cluster_steps<T, CLT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c.cl_size);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = c.cl_ms_smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c.cl_size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  SGEP_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, k_cluster_steps<T, CLT>, &cfg));
  c.cl_ms_max_clusters = n;
  return SGEP_OK;
}

// Cooperative launch: every CTA is resident, so the grid barrier between steps cannot wait
// on a CTA that has not started.
template <typename T, int CLT>
int ms_launch(Ctx& c, const MsArgs& a, int NC, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(NC * c.cl_size));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = c.cl_ms_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c.cl_size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = c.cl_ms_coop ? 2 : 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_cluster_steps<T, CLT>, a);
  if (e != cudaSuccess && c.cl_ms_coop) {
    // the CUDA driver refused the cooperative attribute with clusters: the grid never exceeds the
    // co-resident clusters and every wait is bounded, so launch without it
    cudaGetLastError();
    c.cl_ms_coop = 0;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_cluster_steps<T, CLT>, a);
  }
  SGEP_CUDA_TRY(e);
  ++c.launches;
  return SGEP_OK;
}

int ms_conf(Ctx& c) {
  if (c.cfg.dtype == SGEP_BF16)
    return c.cl_size == 16 ? ms_configure<__nv_bfloat16, 16>(c) : ms_configure<__nv_bfloat16, 8>(c);
  return c.cl_size == 16 ? ms_configure<float, 16>(c) : ms_configure<float, 8>(c);
}

}  // namespace

bool cluster_supported(const Ctx& c, const char** why) {
  if (c.k > kMaxKP) {
    if (why) *why = "k > 32";
    return false;
  }
  Plan p;
  if (make_plan(c, 8, 0, &p) || make_plan(c, 16, 0, &p)) return true;
  if (why) *why = "column slices too wide for shared memory (d too large)";
  return false;
}

int cluster_alloc(Ctx& c) {
  Plan p;
  if (!make_plan(c, 8, 0, &p) && !make_plan(c, 16, 0, &p)) return SGEP_ENOTSUP;
  auto adopt = [&](const Plan& q) {
    c.cl_size = q.CL;
    c.cl_x = q.cl_x;
    c.cl_wx = q.wx;
    c.cl_wy = q.wy;
    c.cl_wmax = q.wp;
    c.cl_kp = q.kp;
    c.cl_lkp = q.lkp;
    c.cl_xs = q.xs;
    c.cl_rs = q.rs;
    c.cl_smem = q.smem;
  };
  adopt(p);
  auto conf = [&]() {
    if (c.cfg.dtype == SGEP_BF16)
      return c.cl_size == 16 ? configure<__nv_bfloat16, 16>(c) : configure<__nv_bfloat16, 8>(c);
    return c.cl_size == 16 ? configure<float, 16>(c) : configure<float, 8>(c);
  };
  int rc = conf();
  if (rc) return rc;
  // re-plan the resident rows with the number of clusters that fit at once
  if (make_plan(c, c.cl_size, c.cl_max_clusters, &p) && p.smem != c.cl_smem) {
    adopt(p);
    rc = conf();
    if (rc) return rc;
  }
  const int esz = c.cfg.dtype == SGEP_BF16 ? 2 : 4;
  c.cl_async_shape = (c.d_x * esz % 16 == 0) && (!c.has_y || c.d_y * esz % 16 == 0) &&
                     (p.wx * esz % 16 == 0) && (!c.has_y || p.wy * esz % 16 == 0);
  const size_t dk = (size_t)c.d * c.k;
  const size_t gk = (size_t)c.k * c.k + c.k;
  c.cl_V[0] = c.V;
  c.cl_S[0] = c.S;
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.cl_V[1], dk * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.cl_S[1], dk * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.cl_acc, 3 * 2 * dk * sizeof(float)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.cl_gram, 3 * gk * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(c.cl_acc, 0, 3 * 2 * dk * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(c.cl_gram, 0, 3 * gk * sizeof(float)));
  c.cl_cur = 0;
  c.cl_slot = 0;
  c.cl_pending = 0;
  const char* pdl = getenv("SGEP_PDL");
  c.cl_pdl = (pdl && pdl[0] == '0') ? 0 : 1;
  const char* tr = getenv("SGEP_TRACE");
  if (tr && tr[0] == '1') {
    SGEP_CUDA_TRY(cudaMalloc((void**)&c.trace, (size_t)4096 * kTracePhases * sizeof(unsigned long long)));
    SGEP_CUDA_TRY(cudaMemset(c.trace, 0, (size_t)4096 * kTracePhases * sizeof(unsigned long long)));
  }
  // several steps per launch (sgep_step_many) where the resident second [Bv] buffer fits;
  // SGEP_CLUSTER_MS=0 keeps one launch per step
  c.cl_ms_ok = 0;
  const char* ms = getenv("SGEP_CLUSTER_MS");
  c.cl_ms_smem = c.cl_smem + ms_extra_smem(c.cl_wmax, c.cl_kp);
  if (!(ms && ms[0] == '0') && c.cl_ms_smem <= 227 * 1024 && ms_conf(c) == SGEP_OK && c.cl_ms_max_clusters > 0) {
    SGEP_CUDA_TRY(cudaMalloc((void**)&c.cl_bar, sizeof(unsigned)));
    SGEP_CUDA_TRY(cudaMemset(c.cl_bar, 0, sizeof(unsigned)));
    c.cl_bar_count = 0;
    c.cl_ms_ok = 1;
    c.cl_ms_coop = 1;
  }
  cudaGetLastError();
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
  cudaFree(c.cl_gram);
  cudaFree(c.cl_bar);
  c.cl_bar = nullptr;
  c.cl_ms_ok = 0;
  cudaFree(c.trace);
  c.trace = nullptr;
  c.cl_V[1] = c.cl_S[1] = nullptr;
  c.cl_acc = nullptr;
  c.cl_gram = nullptr;
}

int cluster_step(Ctx& c, const void* X, const void* Y, int64_t b, float eta, float gamma, cudaStream_t s) {
  return run(c, X, Y, b, eta, gamma, s);
}

int cluster_flush(Ctx& c, cudaStream_t s) {
  if (!c.cl_pending) return SGEP_OK;
  return run(c, nullptr, nullptr, 0, 0.f, 0.f, s);
}

int cluster_max_steps() { return kMsMax; }

bool cluster_steps_usable(const Ctx& c) { return c.cl_ms_ok && !c.cfg.debug; }

// `nsteps` consecutive minibatches X[s b .. s b + b) (and Y) in one launch: the pending
// update (if any), then per step its products and the next step's update; the last step's
// products stay pending, as after the same number of cluster_step calls.
int cluster_steps(Ctx& c, const void* X, const void* Y, int64_t b, int nsteps, cudaStream_t s) {
  if (nsteps < 1 || nsteps > kMsMax || !c.cl_ms_ok) {
    set_error("cluster_steps: nsteps out of range or multi-step kernel not available");
    return SGEP_EINVAL;
  }
  MsArgs a = {};
  a.X = X;
  a.Y = Y;
  a.b = b;
  a.split = (c.cfg.kind == SGEP_CCA && c.cfg.split_AB) ? 1 : 0;
  a.nA = a.split ? b / 2 : b;
  a.inv_nA = 1.f / (float)a.nA;
  a.inv_nB = a.split ? 1.f / (float)(b - a.nA) : 1.f / (float)b;
  a.d_x = c.d_x;
  a.d_y = c.d_y;
  a.d = c.d;
  a.k = c.k;
  a.kp = c.cl_kp;
  a.kind = c.cfg.kind;
  a.b_is_identity = c.b_is_identity ? 1 : 0;
  a.rho = c.cfg.rho;
  a.eps_B = c.cfg.eps_B;
  a.cl_x = c.cl_x;
  a.w_x = c.cl_wx;
  a.w_y = c.cl_wy;
  a.wp = c.cl_wmax;
  a.xs = c.cl_xs;
  a.rs = c.cl_rs;
  const int max_nc = std::max(1, std::min(c.num_sms / c.cl_size, c.cl_ms_max_clusters));
  const int NC = (int)std::min<int64_t>(max_nc, std::max<int64_t>(1, (b + 63) / 64));
  a.rows_per_cluster = (b + NC - 1) / NC;
  const bool aligned = ((uintptr_t)X % 16 == 0) && (!c.has_y || (uintptr_t)Y % 16 == 0);
  a.async_ok = (aligned && c.cl_async_shape) ? 1 : 0;
  a.nsteps = nsteps;
  a.pend0 = c.cl_pending;
  a.slot0 = c.cl_slot;
  for (int st = 0; st < nsteps; ++st) {
    // step st applies the update of minibatch st - 1 (step c.t + st of the schedule)
    a.eta[st] = st == 0 ? c.cl_eta : (float)schedule_eta(c.cfg, c.t + st);
    a.gamma[st] = st == 0 ? c.cl_gamma : c.cfg.gamma0;
  }
  a.V_in = c.cl_V[c.cl_cur];
  a.S_in = c.cl_S[c.cl_cur];
  a.V_out = c.cl_V[1 - c.cl_cur];
  a.S_out = c.cl_S[1 - c.cl_cur];
  a.acc = c.cl_acc;
  a.gram = c.cl_gram;
  const unsigned grid = (unsigned)(NC * c.cl_size);
  if (c.cl_bar_count > (1u << 30)) {  // restart the arrival counter long before it could wrap
    SGEP_CUDA_TRY(cudaMemsetAsync(c.cl_bar, 0, sizeof(unsigned), s));
    c.cl_bar_count = 0;
  }
  a.bar = c.cl_bar;
  a.bar_base = c.cl_bar_count;
  a.dflag = c.dflag;
  a.trace = nsteps >= 2 ? c.trace : nullptr;
  if (a.trace) SGEP_CUDA_TRY(cudaMemsetAsync(c.trace, 0, (size_t)4096 * kTracePhases * sizeof(unsigned long long), s));
  int rc;
  if (c.cfg.dtype == SGEP_BF16)
    rc = c.cl_size == 16 ? ms_launch<__nv_bfloat16, 16>(c, a, NC, s) : ms_launch<__nv_bfloat16, 8>(c, a, NC, s);
  else
    rc = c.cl_size == 16 ? ms_launch<float, 16>(c, a, NC, s) : ms_launch<float, 8>(c, a, NC, s);
  if (rc) return rc;
  c.cl_bar_count += (unsigned)(nsteps - 1) * grid;
  c.cl_last_grid = (int)grid;
  c.cl_ms_traced = a.trace ? 1 : 0;
  if (c.cl_pending || nsteps > 1) c.cl_cur = 1 - c.cl_cur;  // an update was applied
  c.cl_slot = (c.cl_slot + nsteps) % 3;
  c.cl_pending = 1;
  c.cl_eta = (float)schedule_eta(c.cfg, c.t + nsteps);
  c.cl_gamma = c.cfg.gamma0;
  c.debug_valid = 0;
  c.V = c.cl_V[c.cl_cur];
  c.S = c.cl_S[c.cl_cur];
  return SGEP_OK;
}

void cluster_trace_report(Ctx& c) {
  if (!c.trace || c.cl_last_grid <= 0) return;
  const int n = c.cl_last_grid;
  std::vector<unsigned long long> t((size_t)n * kTracePhases);
  if (cudaMemcpy(t.data(), c.trace, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
    return;
  unsigned long long g0 = ~0ull, g1 = 0;
  for (int b = 0; b < n; ++b) {
    g0 = std::min(g0, t[(size_t)b * kTracePhases]);
    g1 = std::max(g1, t[(size_t)b * kTracePhases]);
  }
  std::fprintf(stderr, "[sgep trace] grid %d CTAs (cluster %d, max co-resident clusters %d); CTA start spread %.2f us\n",
               n, c.cl_size, c.cl_max_clusters, (double)(g1 - g0) / 1e3);
  if (c.cl_ms_traced) {
    // globaltimer stamps of one step of a multi-step launch, relative to the earliest step start
    std::fprintf(stderr, "[sgep trace] multi-step launch, the step before the last (us from its earliest start, median / max over CTAs):");
    for (int ph = 1; ph < kTracePhases; ++ph) {
      std::vector<double> v;
      for (int b = 0; b < n; ++b)
        if (t[(size_t)b * kTracePhases + ph]) v.push_back((double)(t[(size_t)b * kTracePhases + ph] - g0) / 1e3);
      if (v.empty()) continue;
      std::sort(v.begin(), v.end());
      std::fprintf(stderr, " %d:%.2f/%.2f", ph, v[v.size() / 2], v.back());
    }
    std::fprintf(stderr, "\n");
    return;
  }
  std::fprintf(stderr, "[sgep trace] phase clocks (median / max over CTAs, SM cycles from CTA start):");
  for (int ph = 1; ph < kTracePhases; ++ph) {
    std::vector<unsigned long long> v;
    for (int b = 0; b < n; ++b) v.push_back(t[(size_t)b * kTracePhases + ph]);
    std::sort(v.begin(), v.end());
    std::fprintf(stderr, " %d:%llu/%llu", ph, v[v.size() / 2], v.back());
  }
  std::fprintf(stderr, "\n");
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

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

#include <type_traits>

#include "eg_math.cuh"
#include "internal.h"

namespace sgep {
namespace gt {

constexpr int kThreads = 256;
constexpr int kMaxK = 64;

// Register-tiled SIMT contractions (projection and back-projection). Both tiles stage a
// block of rows and the players' weights in shared memory, rows padded by kPad floats so
// every float4 read is aligned and the 8 lanes of one 128-bit access phase hit distinct
// banks; every thread keeps a 4 x 4 micro-tile of accumulators, one float4 of data and one
// float4 of weights per 16 FMAs. The k players form ceil(k/4) player quads; the threads
// left after one thread per (data quad, player quad) split the contraction dimension, and
// their partial sums are added in shared memory before one atomic per output. The next
// stage's loads are written before the current stage is computed: the data rows (any element
// type, centred or scaled) into registers, the FP32 weights by cp.async into the other half
// of a double buffer (zero-filled where masked). The compiler may still issue a register load
// next to its use, so plain FP32 rows take the cp.async ring below instead.
constexpr int kPad = 4;
constexpr int kWS = kMaxK + kPad;  // staged row stride of V, P and Q (floats)
constexpr int kProjRows = 64;      // rows of one projection tile
constexpr int kProjCols = 32;      // columns staged per projection stage
constexpr int kProjXS = kProjRows + kPad;
constexpr int kBpRows = 32;        // rows staged per back-projection stage
constexpr int kBpCols = 64;        // columns of one back-projection tile
constexpr int kBpZS = kBpCols + kPad;
constexpr int kRedFloats = kThreads * 16;  // split partials: splits x 64 x 4 ceil(k/4) <= 4096
constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Plain FP32 rows (no centring, no row scale) skip the registers: rows and weights go to
// shared memory by cp.async through a ring of stages, so several stages are in flight
// while one is computed. The projection's ring keeps its rows row-major (stride kPRXS:
// an odd number of float4, so 8 consecutive rows at one column quad hit distinct banks).
constexpr int kProjRing = 4;
constexpr int kBpRing = 3;
constexpr int kPRXS = kProjCols + kPad;
// BF16 rows land in their own buffer of each stage (row stride an odd number of 16-byte
// chunks) and are widened to FP32 into the stage, centred if they are, before it is read.
constexpr int kPLB = kProjCols + 8;  // BF16 landing row stride of the projection ring
constexpr int kBLB = kBpCols + 16;   // ... and of the back-projection ring (also 256 x 5 value pairs)
constexpr int kProjRingSmem = kProjRing * (kProjRows * kPRXS + kProjCols * kWS + kProjRows * kPLB / 2);
constexpr int kBpRingSmem = kBpRing * (kBpRows * kBpZS + 2 * kBpRows * kWS + kBpRows * kBLB / 2);

// Shared-memory floats each tile needs (k <= 64, C <= 32). The register path's weights are
// double-buffered.
constexpr int kProjectSmem = cmax(cmax(kProjCols * kProjXS + 2 * kProjCols * kWS, kRedFloats), kProjRingSmem);
constexpr int kBackprojectSmem = cmax(cmax(kBpRows * kBpZS + 4 * kBpRows * kWS, kRedFloats), kBpRingSmem);
// k x k terms: four staged 32-row chunks (V, AV, S, BV) of row stride ceil(k/4)*4 + 4, or the
// split partials of one k x k matrix, whichever is larger.
__host__ __device__ constexpr int gram_smem(int k) {
  return 4 * 32 * (((k + 3) / 4) * 4 + 4) > kThreads * 16 ? 4 * 32 * (((k + 3) / 4) * 4 + 4) : kThreads * 16;
}
constexpr int kUpdRows = 4;  // rows per thread per iteration of the update tile
__host__ __device__ constexpr int update_smem(int k) {
  return k * k + 4 * k + kUpdRows * (kThreads / k > 1 ? kThreads / k : 1) * k + 2 * k * k + k;
}
constexpr int kStatsRows = 16;  // rows per cp.async block of the LDA statistics (FP32 rows)
__host__ __device__ constexpr int lda_stats_smem(int C) { return C * kThreads + kThreads + 2 * kStatsRows * kThreads; }
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

// acc[a][c] += x[a] w[c]: one 4 x 4 outer product.
__device__ __forceinline__ void fma4x4(float (&acc)[4][4], const float4 x, const float4 w) {
  const float xa[4] = {x.x, x.y, x.z, x.w};
  const float wa[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(xa[a], wa[c], acc[a][c]);
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// 4-byte asynchronous global -> shared copy; zero-fills the destination when !valid (no read).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit_all() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// 16-byte variant (both addresses 16-byte aligned); zero-fills when !valid.
__device__ __forceinline__ void cp_async16z(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
template <int N>
__device__ __forceinline__ void cp_async_wait_pending() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Zero the player columns [k, 4 ceil(k/4)) of `rows` staged rows of stride kWS, so the
// last player quad multiplies zeros.
__device__ __forceinline__ void zero_player_pad(float* W, int rows, int k) {
  const int pad = ((k + 3) & ~3) - k;
  if (pad == 0) return;
  for (int e = threadIdx.x; e < rows * pad; e += kThreads) W[(e / pad) * kWS + k + e % pad] = 0.f;
}

// Adds the split partials of the 4 x 4 micro-tiles (thread (o, sp): data group dq = o % 16,
// player quad pq = o / 16; accumulator row a is data index r = rmul dq + astride a) and issues
// one atomicAdd(out[orow(r) + i], scale * sum) per output r < 64 with valid(r), i < k.
// `red` must not overlap data still being read.
template <typename Valid, typename OutRow>
__device__ __forceinline__ void reduce_quads(const float (&acc)[4][4], bool active, int splits, int sp, int dq,
                                             int pq, int k, float scale, float* red, float* out, Valid valid,
                                             OutRow orow, int rmul = 4, int astride = 1) {
  const int kp = (k + 3) & ~3;
  if (splits == 1) {
    if (active) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int r = rmul * dq + astride * a;
        if (!valid(r)) continue;
        const int64_t base = orow(r);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (4 * pq + c < k) atomicAdd(&out[base + 4 * pq + c], scale * acc[a][c]);
      }
    }
  } else {
    if (active) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
        *reinterpret_cast<float4*>(red + ((sp * 64) + rmul * dq + astride * a) * kp + 4 * pq) =
            make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * k; e += kThreads) {
      const int r = e / k, i = e % k;
      if (!valid(r)) continue;
      float sum = 0.f;
      for (int s2 = 0; s2 < splits; ++s2) sum += red[(s2 * 64 + r) * kp + i];
      atomicAdd(&out[orow(r) + i], scale * sum);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Projection of FP32 rows through the cp.async ring (same tile and result as project_tile).
// Stage st holds rows [row0, row0 + 64) x columns [c0, c0 + 32) row-major and V's rows
// [c0, c0 + 32); a thread owns rows rq + 16a (a < 4) and one player quad, and per column quad
// reads 4 float4 of rows and 4 float4 of V for 64 FMAs. With `cz`, each landed stage is centred
// in shared memory (a thread: one row, 8 columns) before it is read.
// The 8 BF16 values at element a, a + 1, .. of a matrix of `total` values, widened, from the
// five aligned value pairs staged from element a & ~1 on. Values whose column is past `ncols`
// (columns left in the row from a), or of a row that is not valid, are zero; a pair that
// reached past the matrix's last value was not staged and is read directly.
__device__ __forceinline__ void widen_pairs(const uint32_t* slot, const __nv_bfloat16* Z, int64_t a, int64_t total,
                                            bool row_ok, int64_t ncols, float (&out)[8]) {
  const int64_t p0 = a & ~(int64_t)1;
  const int sh = (int)(a - p0);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int e = u + sh;  // position in the staged pairs
    float v = 0.f;
    if (row_ok && u < ncols) {
      if (p0 + 2 * (e >> 1) + 1 < total) {
        const uint32_t w = slot[e >> 1];
        v = __uint_as_float((e & 1) ? (w & 0xffff0000u) : (w << 16));
      } else {
        v = __bfloat162float(Z[a + u]);
      }
    }
    out[u] = v;
  }
}
__device__ __forceinline__ void widen_pairs(const uint32_t*, const float*, int64_t, int64_t, bool, int64_t,
                                            float (&out)[8]) {
  for (int u = 0; u < 8; ++u) out[u] = 0.f;
}

template <typename T>
__device__ inline void project_tile_ring(const T* __restrict__ X, const T* __restrict__ Y, int64_t n, int64_t dx,
                                         int64_t dy, const float* __restrict__ V, int k, int64_t chunk,
                                         int nchunk_x, float* __restrict__ PQ, int bx, int by, float* smem,
                                         const Centring* cz = nullptr) {
  constexpr bool kB = !std::is_same<T, float>::value;  // BF16 rows: landed, then widened in shared memory
  constexpr int NS = kProjRing;
  constexpr int kXStage = kProjRows * kPRXS, kVStage = kProjCols * kWS;
  float* Xs = smem;                // [NS][kProjRows][kPRXS]
  float* Vs = smem + NS * kXStage;  // [NS][kProjCols][kWS]
  __nv_bfloat16* Lb = reinterpret_cast<__nv_bfloat16*>(Vs + NS * kVStage);  // [NS][kProjRows][kPLB]
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)bx * kProjRows;
  const bool isY = by >= nchunk_x;
  const int cidx = isY ? by - nchunk_x : by;
  const T* Z = isY ? Y : X;
  const int64_t ld = isY ? dy : dx;
  const int64_t voff = isY ? dx : 0;
  const int64_t c_begin = (int64_t)cidx * chunk;
  const int64_t c_end = min(c_begin + chunk, ld);
  const int nst = (int)((c_end - c_begin + kProjCols - 1) / kProjCols);
  const int kp = (k + 3) & ~3;
  const int nq = kp >> 2;
  const int ot = 16 * nq;           // threads with one (row group, player quad)
  const int splits = kThreads / ot;  // column-quad splits
  const bool active = tid < ot * splits;
  const int o = tid % ot, sp = tid / ot;
  const int rq = o % 16, pq = o / 16;
  // 16-byte copies when the row pitch and base allow (then a stage's columns are all valid
  // or all past the end together), else 4-byte copies.
  const bool x16 = (ld % 4 == 0) && aligned16(Z);
  // BF16 rows (the caller checked 4-byte alignment): 16-byte copies when the rows allow
  const bool b16 = kB && ld % 8 == 0 && aligned16(Z);
  const bool v16 = (k % 4 == 0) && aligned16(V);
  // staging roles: 16-byte rows xq + 32j, column quad xm (4-byte: rows xr + 8j, column xc);
  // V rows vq + 16j, player quad vm (4-byte: rows vr + 4j, player vi)
  const int xm = tid % 8, xq = tid / 8, xc = tid % kProjCols, xr = tid / kProjCols;
  const int vm = tid % 16, vq = tid / 16, vi = tid % 64, vr = tid / 64;
  const T* zrow = x16 ? Z + (row0 + xq) * ld + 4 * xm : Z + (row0 + xr) * ld + xc;

  auto issue = [&](int st) {
    if (st < nst) {
      float* xs = Xs + (st % NS) * kXStage;
      float* vs = Vs + (st % NS) * kVStage;
      const int64_t c0 = c_begin + (int64_t)st * kProjCols;
      if constexpr (kB) {
        __nv_bfloat16* lb = Lb + (st % NS) * kProjRows * kPLB;
        if (b16) {  // one 16-byte copy (8 values) per thread: row tid / 4, columns 8 (tid % 4) ..
          const int r = tid / 4, c = 8 * (tid % 4);
          const bool v = row0 + r < n && c0 + c < c_end;
          cp_async16z(reinterpret_cast<float*>(lb + r * kPLB + c),
                      reinterpret_cast<const float*>(v ? Z + (row0 + r) * ld + c0 + c : Z), v);
        } else {  // the five aligned value pairs holding this thread's 8 values (row tid / 4)
          const int r = tid / 4, c = 8 * (tid % 4);
          const int64_t a = (row0 + r) * ld + c0 + c, p0 = a & ~(int64_t)1;
          const bool v = row0 + r < n && c0 + c < c_end;
          uint32_t* slot = reinterpret_cast<uint32_t*>(lb) + 5 * tid;
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            const bool ok = v && p0 + 2 * j + 1 < n * ld;
            cp_async4(reinterpret_cast<float*>(slot + j), reinterpret_cast<const float*>(ok ? Z + p0 + 2 * j : Z), ok);
          }
        }
      } else if (x16) {
        const bool cv = c0 + 4 * xm < c_end;
#pragma unroll
        for (int j = 0; j < kProjRows / 32; ++j) {
          const bool v = cv && row0 + xq + 32 * j < n;
          cp_async16z(xs + (xq + 32 * j) * kPRXS + 4 * xm, v ? zrow + 32 * j * ld + c0 : Z, v);
        }
      } else {
        const bool cv = c0 + xc < c_end;
#pragma unroll
        for (int j = 0; j < kProjRows / 8; ++j) {
          const bool v = cv && row0 + xr + 8 * j < n;
          cp_async4(xs + (xr + 8 * j) * kPRXS + xc, v ? zrow + 8 * j * ld + c0 : Z, v);
        }
      }
      if (v16) {
        if (vm < nq) {
#pragma unroll
          for (int j = 0; j < kProjCols / 16; ++j) {
            const int64_t c = c0 + vq + 16 * j;
            const bool v = c < c_end;
            cp_async16z(vs + (vq + 16 * j) * kWS + 4 * vm, v ? V + (voff + c) * k + 4 * vm : V, v);
          }
        }
      } else if (vi < kp) {
#pragma unroll
        for (int j = 0; j < kProjCols / 4; ++j) {
          const int64_t c = c0 + vr + 4 * j;
          const bool v = vi < k && c < c_end;
          cp_async4(vs + (vr + 4 * j) * kWS + vi, v ? V + (voff + c) * k + vi : V, v);
        }
      }
    }
    cp_async_commit_all();  // empty groups keep one group per stage
  };

  // centring roles: row cr, columns cc8 .. cc8 + 7 of every stage (the row's label is fixed)
  static_assert(kProjRows * kProjCols / 8 == kThreads, "one centring item per thread");
  const int cr = tid / 4, cc8 = 8 * (tid % 4);
  bool crow = cz && row0 + cr < n;
  const float* mrow = nullptr;
  if (crow) {
    if (cz->labels) {
      const int lab = cz->labels[row0 + cr];
      if ((unsigned)lab >= (unsigned)cz->C) {  // flagged; the row stays uncentred
        atomicOr(cz->dflag, kFlagBadLabel);
        crow = false;
      } else {
        mrow = cz->mean + (int64_t)lab * ld;
      }
    } else {
      mrow = isY ? cz->mean_y : cz->mean;
    }
  }

  __syncthreads();  // the workspace may still be read by this block's previous tile
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
#pragma unroll
  for (int st = 0; st < NS - 1; ++st) issue(st);
  for (int st = 0; st < nst; ++st) {
    cp_async_wait_pending<NS - 2>();
    __syncthreads();       // stage st landed for every thread; stage st - 1 is no longer read
    issue(st + NS - 1);    // into the slot of stage st - 1
    if (kB) {  // widen the landed BF16 row values (and centre them)
      float xv[8];
      if (b16) {
        const uint4 raw = *reinterpret_cast<const uint4*>(Lb + (st % NS) * kProjRows * kPLB + cr * kPLB + cc8);
        const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 f = __bfloat1622float2(h2[u]);
          xv[2 * u] = f.x;
          xv[2 * u + 1] = f.y;
        }
      } else {
        widen_pairs(reinterpret_cast<const uint32_t*>(Lb + (st % NS) * kProjRows * kPLB) + 5 * tid, Z,
                    (row0 + cr) * ld + c_begin + (int64_t)st * kProjCols + cc8, n * ld, row0 + cr < n,
                    c_end - (c_begin + (int64_t)st * kProjCols + cc8), xv);
      }
      if (crow) {
        const int64_t c0 = c_begin + (int64_t)st * kProjCols + cc8;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c0 + u < c_end) xv[u] -= mrow[c0 + u];
      }
      float* xs = Xs + (st % NS) * kXStage + cr * kPRXS + cc8;
      *reinterpret_cast<float4*>(xs) = make_float4(xv[0], xv[1], xv[2], xv[3]);
      *reinterpret_cast<float4*>(xs + 4) = make_float4(xv[4], xv[5], xv[6], xv[7]);
      __syncthreads();
    } else if (cz) {
      if (crow) {
        float* xs = Xs + (st % NS) * kXStage + cr * kPRXS + cc8;
        const int64_t c0 = c_begin + (int64_t)st * kProjCols + cc8;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c0 + u < c_end) xs[u] -= mrow[c0 + u];
      }
      __syncthreads();
    }
    if (active) {
      const float* xs = Xs + (st % NS) * kXStage + rq * kPRXS;
      const float* vs = Vs + (st % NS) * kVStage + 4 * pq;
#pragma unroll 2
      for (int q = sp; q < kProjCols / 4; q += splits) {
        float4 xa[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) xa[a] = lds4(xs + 16 * a * kPRXS + 4 * q);
        fma4x4(acc, make_float4(xa[0].x, xa[1].x, xa[2].x, xa[3].x), lds4(vs + (4 * q + 0) * kWS));
        fma4x4(acc, make_float4(xa[0].y, xa[1].y, xa[2].y, xa[3].y), lds4(vs + (4 * q + 1) * kWS));
        fma4x4(acc, make_float4(xa[0].z, xa[1].z, xa[2].z, xa[3].z), lds4(vs + (4 * q + 2) * kWS));
        fma4x4(acc, make_float4(xa[0].w, xa[1].w, xa[2].w, xa[3].w), lds4(vs + (4 * q + 3) * kWS));
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int64_t pqoff = isY ? k : 0;
  reduce_quads(
      acc, active, splits, sp, rq, pq, k, 1.f, smem, PQ, [&](int r) { return row0 + r < n; },
      [&](int r) { return (row0 + r) * 2 * k + pqoff; }, 1, 16);
}

// Back-projection of FP32 rows through the cp.async ring (same tile and result as
// backproject_tile): stage st holds rows [r0, r0 + 32) of the 64-column block and their
// P / Q weights, masked per estimate by zero-filled copies. With `cz`, each landed stage is
// centred in shared memory (a thread: one row, 8 columns) before it is read.
template <typename T>
__device__ inline void backproject_tile_ring(const T* __restrict__ X, const T* __restrict__ Y, int64_t b, int64_t dx,
                                             int64_t dy, int64_t nA, int kind, int split,
                                             const float* __restrict__ PQ, int k, int nblk_x,
                                             int64_t rows_per_split, float inv_nA, float inv_nB,
                                             float* __restrict__ AV, float* __restrict__ BV, int bx, int by,
                                             float* smem, const Centring* cz = nullptr) {
  constexpr bool kB = !std::is_same<T, float>::value;  // BF16 rows: landed, then widened in shared memory
  constexpr int NS = kBpRing;
  constexpr int kZStage = kBpRows * kBpZS, kWStage = kBpRows * kWS;
  float* Zs = smem;                      // [NS][kBpRows][kBpZS]
  float* WA = smem + NS * kZStage;       // [NS][kBpRows][kWS]
  float* WB = WA + NS * kWStage;         // [NS][kBpRows][kWS]
  __nv_bfloat16* Lb = reinterpret_cast<__nv_bfloat16*>(WB + NS * kWStage);  // [NS][kBpRows][kBLB]
  const int tid = threadIdx.x;
  const bool isY = bx >= nblk_x;
  const int bidx = isY ? bx - nblk_x : bx;
  const T* Z = isY ? Y : X;
  const int64_t ld = isY ? dy : dx;
  const int64_t col0 = (int64_t)bidx * kBpCols;
  const int64_t r_begin = (int64_t)by * rows_per_split;
  const int64_t r_end = min(r_begin + rows_per_split, b);
  const int nst = (int)((max(r_end - r_begin, (int64_t)0) + kBpRows - 1) / kBpRows);
  const int own = isY ? k : 0;
  const int cross = isY ? 0 : k;
  const bool cca = kind == SGEP_CCA;
  const bool lda = kind == SGEP_LDA;
  const int offA = (kind == SGEP_PCA) ? 0 : cross;
  const bool splitAB = cca && split;
  // the estimates this tile's rows feed (with split A/B rows, a row split inside one half
  // feeds one of them: its other weights are not staged and its other sums not reduced)
  const bool wantA = !lda && (!splitAB || r_begin < nA), wantB = (cca || lda) && (!splitAB || r_end > nA);
  const int kp = (k + 3) & ~3;
  const int nq = kp >> 2;
  const int ot = 16 * nq;           // threads with one (column quad, player quad)
  const int splits = kThreads / ot;  // row splits
  const bool active = tid < ot * splits;
  const int o = tid % ot, sp = tid / ot;
  const int cq = o % 16, pq = o / 16;
  // 16-byte copies when the row pitch and bases allow, else 4-byte copies
  const bool z16 = (ld % 4 == 0) && aligned16(Z);
  // BF16 rows (the caller checked 4-byte alignment): 16-byte copies when the rows allow
  const bool b16 = kB && ld % 8 == 0 && aligned16(Z);
  const bool w16 = (k % 4 == 0) && aligned16(PQ);
  // staging roles: 16-byte rows sq + 16j at column (or player) quad sm; 4-byte rows sr + 4j
  // at column (or player) sc
  const int sm = tid % 16, sq = tid / 16, sc = tid % 64, sr = tid / 64;
  const bool ccol = z16 ? col0 + 4 * sm < ld : col0 + sc < ld;
  const T* zcol = z16 ? Z + col0 + 4 * sm : Z + col0 + sc;

  auto issue = [&](int st) {
    if (st < nst) {
      const int64_t r0 = r_begin + (int64_t)st * kBpRows;
      float* zs = Zs + (st % NS) * kZStage;
      float* wa = WA + (st % NS) * kWStage;
      float* wb = WB + (st % NS) * kWStage;
      if constexpr (kB) {
        __nv_bfloat16* lb = Lb + (st % NS) * kBpRows * kBLB;
        if (b16) {  // one 16-byte copy (8 values) per thread: row tid / 8, columns 8 (tid % 8) ..
          const int r = tid / 8, c = 8 * (tid % 8);
          const bool v = r0 + r < r_end && col0 + c < ld;
          cp_async16z(reinterpret_cast<float*>(lb + r * kBLB + c),
                      reinterpret_cast<const float*>(v ? Z + (r0 + r) * ld + col0 + c : Z), v);
        } else {  // the five aligned value pairs holding this thread's 8 values (row tid / 8)
          const int r = tid / 8, c = 8 * (tid % 8);
          const int64_t a = (r0 + r) * ld + col0 + c, p0 = a & ~(int64_t)1;
          const bool v = r0 + r < r_end && col0 + c < ld;
          uint32_t* slot = reinterpret_cast<uint32_t*>(lb) + 5 * tid;
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            const bool ok = v && p0 + 2 * j + 1 < b * ld;
            cp_async4(reinterpret_cast<float*>(slot + j), reinterpret_cast<const float*>(ok ? Z + p0 + 2 * j : Z), ok);
          }
        }
      } else if (z16) {
#pragma unroll
        for (int j = 0; j < kBpRows / 16; ++j) {
          const int64_t row = r0 + sq + 16 * j;
          const bool v = ccol && row < r_end;
          cp_async16z(zs + (sq + 16 * j) * kBpZS + 4 * sm, v ? zcol + row * ld : Z, v);
        }
      } else {
#pragma unroll
        for (int j = 0; j < kBpRows / 4; ++j) {
          const int64_t row = r0 + sr + 4 * j;
          const bool v = ccol && row < r_end;
          cp_async4(zs + (sr + 4 * j) * kBpZS + sc, v ? zcol + row * ld : Z, v);
        }
      }
      if (w16) {
        if (sm < nq) {
#pragma unroll
          for (int j = 0; j < kBpRows / 16; ++j) {
            const int64_t row = r0 + sq + 16 * j;
            const bool in = row < r_end;
            if (wantA) {
              const bool v = in && (!splitAB || row < nA);
              cp_async16z(wa + (sq + 16 * j) * kWS + 4 * sm, v ? PQ + row * 2 * k + offA + 4 * sm : PQ, v);
            }
            if (wantB) {
              const bool v = in && (!splitAB || row >= nA);
              cp_async16z(wb + (sq + 16 * j) * kWS + 4 * sm, v ? PQ + row * 2 * k + own + 4 * sm : PQ, v);
            }
          }
        }
      } else if (sc < kp) {
#pragma unroll
        for (int j = 0; j < kBpRows / 4; ++j) {
          const int64_t row = r0 + sr + 4 * j;
          const bool in = sc < k && row < r_end;
          if (wantA) {
            const bool v = in && (!splitAB || row < nA);
            cp_async4(wa + (sr + 4 * j) * kWS + sc, v ? PQ + row * 2 * k + offA + sc : PQ, v);
          }
          if (wantB) {
            const bool v = in && (!splitAB || row >= nA);
            cp_async4(wb + (sr + 4 * j) * kWS + sc, v ? PQ + row * 2 * k + own + sc : PQ, v);
          }
        }
      }
    }
    cp_async_commit_all();
  };

  __syncthreads();  // the workspace may still be read by this block's previous tile
  float accA[4][4], accB[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) accA[a][c] = accB[a][c] = 0.f;
#pragma unroll
  for (int st = 0; st < NS - 1; ++st) issue(st);
  static_assert(kBpRows * kBpCols / 8 == kThreads, "one centring item per thread");
  const int cr = tid / 8, cc8 = 8 * (tid % 8);  // centring roles: row cr, columns cc8 .. cc8 + 7
  for (int st = 0; st < nst; ++st) {
    cp_async_wait_pending<NS - 2>();
    __syncthreads();
    issue(st + NS - 1);
    const int64_t r0 = r_begin + (int64_t)st * kBpRows;
    const int nr = (int)min((int64_t)kBpRows, r_end - r0);
    if (kB || cz) {
      const int64_t row = r0 + cr;
      const float* mrow = nullptr;
      if (cz && row < r_end) {
        mrow = isY ? cz->mean_y : cz->mean;
        if (cz->labels) {
          const int lab = cz->labels[row];
          if ((unsigned)lab >= (unsigned)cz->C) {  // flagged; the row stays uncentred
            atomicOr(cz->dflag, kFlagBadLabel);
            mrow = nullptr;
          } else {
            mrow = cz->mean + (int64_t)lab * ld;
          }
        }
      }
      float* zs = Zs + (st % NS) * kZStage + cr * kBpZS + cc8;
      if (kB) {  // widen the landed BF16 row values (and centre them)
        float zv[8];
        if (b16) {
          const uint4 raw = *reinterpret_cast<const uint4*>(Lb + (st % NS) * kBpRows * kBLB + cr * kBLB + cc8);
          const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 f = __bfloat1622float2(h2[u]);
            zv[2 * u] = f.x;
            zv[2 * u + 1] = f.y;
          }
        } else {
          widen_pairs(reinterpret_cast<const uint32_t*>(Lb + (st % NS) * kBpRows * kBLB) + 5 * tid, Z,
                      row * ld + col0 + cc8, b * ld, row < r_end, ld - (col0 + cc8), zv);
        }
        if (mrow) {
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (col0 + cc8 + u < ld) zv[u] -= mrow[col0 + cc8 + u];
        }
        *reinterpret_cast<float4*>(zs) = make_float4(zv[0], zv[1], zv[2], zv[3]);
        *reinterpret_cast<float4*>(zs + 4) = make_float4(zv[4], zv[5], zv[6], zv[7]);
      } else if (mrow) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (col0 + cc8 + u < ld) zs[u] -= mrow[col0 + cc8 + u];
      }
      __syncthreads();
    }
    const bool useA = wantA && (!splitAB || r0 < nA);
    const bool useB = wantB && (!splitAB || r0 + nr > nA);
    if (active) {
      const float* zs = Zs + (st % NS) * kZStage + 4 * cq;
      const float* wa = WA + (st % NS) * kWStage + 4 * pq;
      const float* wb = WB + (st % NS) * kWStage + 4 * pq;
      if (useA && useB) {
#pragma unroll 2
        for (int rr = sp; rr < nr; rr += splits) {
          const float4 z = lds4(zs + rr * kBpZS);
          fma4x4(accA, z, lds4(wa + rr * kWS));
          fma4x4(accB, z, lds4(wb + rr * kWS));
        }
      } else if (useA) {
#pragma unroll 4
        for (int rr = sp; rr < nr; rr += splits) fma4x4(accA, lds4(zs + rr * kBpZS), lds4(wa + rr * kWS));
      } else if (useB) {
#pragma unroll 4
        for (int rr = sp; rr < nr; rr += splits) fma4x4(accB, lds4(zs + rr * kBpZS), lds4(wb + rr * kWS));
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int64_t coff = isY ? dx : 0;
  auto valid = [&](int c) { return col0 + c < ld; };
  auto orow = [&](int c) { return (coff + col0 + c) * k; };
  if (wantA) reduce_quads(accA, active, splits, sp, cq, pq, k, inv_nA, smem, AV, valid, orow);
  if (wantB) reduce_quads(accB, active, splits, sp, cq, pq, k, inv_nB, smem, BV, valid, orow);
}

// ---------------------------------------------------------------------------
// Projection: PQ[r, 0:k] += X[r, cols] V[cols, :], PQ[r, k:2k] += Y[r, cols] V[d_x + cols, :]
// Tile (bx, by): rows [kProjRows bx, kProjRows (bx + 1)), column chunk by (X chunks first,
// then Y chunks), each `chunk` columns wide. PQ must be zeroed. A thread owns 4 rows x 4
// players; the rows are staged transposed (column-major) so its 4 rows are one float4.
template <typename T>
__device__ void project_tile(const T* __restrict__ X, const T* __restrict__ Y, int64_t n, int64_t dx, int64_t dy,
                             const float* __restrict__ V, int k, int64_t chunk, int nchunk_x, float* __restrict__ PQ,
                             const Centring& cz, const float* __restrict__ rsx, const float* __restrict__ rsy,
                             int bx, int by, float* smem) {
  static_assert(kProjRows == 64 && kProjRows * kProjCols % (4 * kThreads) == 0, "projection staging");
  if constexpr (std::is_same<T, float>::value) {
    if (!rsx && !rsy) {  // FP32 rows without a row scale: the cp.async ring (centred in shared memory)
      project_tile_ring<float>(X, Y, n, dx, dy, V, k, chunk, nchunk_x, PQ, bx, by, smem, cz.mean ? &cz : nullptr);
      return;
    }
  } else if constexpr (std::is_same<T, __nv_bfloat16>::value) {
    // BF16 rows through the ring (16-byte copies, or the aligned value pairs holding a thread's values)
    const T* Z = by >= nchunk_x ? Y : X;
    if (!rsx && !rsy && chunk % 8 == 0 && ((uintptr_t)Z & 3) == 0) {
      project_tile_ring<T>(X, Y, n, dx, dy, V, k, chunk, nchunk_x, PQ, bx, by, smem, cz.mean ? &cz : nullptr);
      return;
    }
  }
  float* Xt = smem;                        // [kProjCols][kProjXS]: Xt[c][r] = Z[row0 + r, c0 + c]
  float* Vs = smem + kProjCols * kProjXS;  // [2][kProjCols][kWS]
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)bx * kProjRows;
  const bool isY = by >= nchunk_x;
  const int cidx = isY ? by - nchunk_x : by;
  const T* Z = isY ? Y : X;
  const float* rs = isY ? rsy : rsx;
  const int64_t ld = isY ? dy : dx;
  const int64_t voff = isY ? dx : 0;
  const int64_t c_begin = (int64_t)cidx * chunk;
  const int64_t c_end = min(c_begin + chunk, ld);
  const int nq = (k + 3) >> 2;
  const int ot = (kProjRows / 4) * nq;  // threads with one (row quad, player quad)
  const int splits = kThreads / ot;     // column splits
  const bool active = tid < ot * splits;
  const int o = tid % ot, sp = tid / ot;
  const int rq = o % (kProjRows / 4), pq = o / (kProjRows / 4);

  constexpr int kXR = kProjRows * kProjCols / (4 * kThreads);  // row quads staged per thread
  float xr[kXR][4];
  auto load_x = [&](int64_t c0) {
#pragma unroll
    for (int j = 0; j < kXR; ++j) {
      const int slot = tid + kThreads * j;
      const int cc = slot % kProjCols, q = slot / kProjCols;
      const int64_t col = c0 + cc;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t row = row0 + 4 * q + a;
        xr[j][a] = (row < n && col < c_end) ? centred(cz, load_row_elem(Z, rs, row, row * ld + col), row, ld, col, isY)
                                            : 0.f;
      }
    }
  };
  auto load_v = [&](int64_t c0, float* dst) {
    for (int e = tid; e < kProjCols * k; e += kThreads) {
      const int cc = e / k, i = e % k;
      const int64_t col = c0 + cc;
      cp_async4(dst + cc * kWS + i, col < c_end ? V + (voff + col) * k + i : V, col < c_end);
    }
    cp_async_commit_all();
  };
  auto store_x = [&]() {
#pragma unroll
    for (int j = 0; j < kXR; ++j) {
      const int slot = tid + kThreads * j;
      const int cc = slot % kProjCols, q = slot / kProjCols;
      *reinterpret_cast<float4*>(Xt + cc * kProjXS + 4 * q) = make_float4(xr[j][0], xr[j][1], xr[j][2], xr[j][3]);
    }
  };

  __syncthreads();  // the workspace may still be read by this block's previous tile
  zero_player_pad(Vs, 2 * kProjCols, k);
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
  if (c_begin < c_end) {
    load_v(c_begin, Vs);
    load_x(c_begin);
  }
  int buf = 0;
  for (int64_t c0 = c_begin; c0 < c_end; c0 += kProjCols, buf ^= 1) {
    store_x();
    cp_async_wait_all();
    __syncthreads();
    if (c0 + kProjCols < c_end) {
      load_v(c0 + kProjCols, Vs + (buf ^ 1) * kProjCols * kWS);
      load_x(c0 + kProjCols);
    }
    if (active) {
      // column quads split across threads, columns in order within a quad: the same
      // summation order as project_tile_ring, so both row paths give identical sums
      const float* Vb = Vs + buf * kProjCols * kWS;
#pragma unroll 2
      for (int q = sp; q < kProjCols / 4; q += splits)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          fma4x4(acc, lds4(Xt + (4 * q + c) * kProjXS + 4 * rq), lds4(Vb + (4 * q + c) * kWS + 4 * pq));
    }
    __syncthreads();
  }
  const int64_t pqoff = isY ? k : 0;
  reduce_quads(
      acc, active, splits, sp, rq, pq, k, 1.f, smem, PQ, [&](int r) { return row0 + r < n; },
      [&](int r) { return (row0 + r) * 2 * k + pqoff; });
}

// ---------------------------------------------------------------------------
// Back-projection: for column c of X (or Y) and player i,
//   AV[c,i] += inv_nA * sum_{r in A rows} Z[r,c] W_A[r,i]
//   BV[c,i] += inv_nB * sum_{r in B rows} Z[r,c] W_B[r,i]
// where (CCA) W_A = Q for X columns / P for Y columns and W_B = P for X / Q for Y;
// (PCA) W_A = P over every row, no BV; (PLS) W_A as CCA over every row, no BV;
// (LDA) every row passed is a B row, centred by its class mean: W_B = P, no AV.
// Tile (bx, by): column block bx of kBpCols (X blocks then Y blocks), row split by.
// A thread owns 4 columns x 4 players of each estimate; rows of the other estimate are
// staged with zero weights, and a stage with no row of an estimate skips it.
template <typename T>
__device__ void backproject_tile(const T* __restrict__ X, const T* __restrict__ Y, int64_t b, int64_t dx,
                                 int64_t dy, int64_t nA, int kind, int split, const float* __restrict__ PQ, int k,
                                 int nblk_x, int64_t rows_per_split, float inv_nA, float inv_nB,
                                 float* __restrict__ AV, float* __restrict__ BV, const Centring& cz,
                                 const float* __restrict__ rsx, const float* __restrict__ rsy, int bx, int by,
                                 float* smem) {
  static_assert(kBpCols == 64 && kBpRows * kBpCols % kThreads == 0, "back-projection staging");
  if constexpr (std::is_same<T, float>::value) {
    if (!rsx && !rsy) {  // FP32 rows without a row scale: the cp.async ring (centred in shared memory)
      backproject_tile_ring<float>(X, Y, b, dx, dy, nA, kind, split, PQ, k, nblk_x, rows_per_split, inv_nA, inv_nB,
                                   AV, BV, bx, by, smem, cz.mean ? &cz : nullptr);
      return;
    }
  } else if constexpr (std::is_same<T, __nv_bfloat16>::value) {
    // BF16 rows through the ring (16-byte copies, or the aligned value pairs holding a thread's values)
    const T* Z = bx >= nblk_x ? Y : X;
    if (!rsx && !rsy && ((uintptr_t)Z & 3) == 0) {
      backproject_tile_ring<T>(X, Y, b, dx, dy, nA, kind, split, PQ, k, nblk_x, rows_per_split, inv_nA, inv_nB, AV,
                               BV, bx, by, smem, cz.mean ? &cz : nullptr);
      return;
    }
  }
  float* Zs = smem;                       // [kBpRows][kBpZS]
  float* WA = smem + kBpRows * kBpZS;     // [2][kBpRows][kWS]
  float* WB = WA + 2 * kBpRows * kWS;     // [2][kBpRows][kWS]
  const int tid = threadIdx.x;
  const bool isY = bx >= nblk_x;
  const int bidx = isY ? bx - nblk_x : bx;
  const T* Z = isY ? Y : X;
  const float* rs = isY ? rsy : rsx;
  const int64_t ld = isY ? dy : dx;
  const int64_t col0 = (int64_t)bidx * kBpCols;
  const int64_t r_begin = (int64_t)by * rows_per_split;
  const int64_t r_end = min(r_begin + rows_per_split, b);
  // column offsets into a PQ row: own projection (P for X, Q for Y) and cross projection
  const int own = isY ? k : 0;
  const int cross = isY ? 0 : k;
  const bool cca = kind == SGEP_CCA;
  const bool lda = kind == SGEP_LDA;
  const int offA = (kind == SGEP_PCA) ? 0 : cross;
  const bool splitAB = cca && split;
  // the estimates this tile's rows feed (a row split inside one A/B half feeds one of them)
  const bool wantA = !lda && (!splitAB || r_begin < nA), wantB = (cca || lda) && (!splitAB || r_end > nA);
  const int nq = (k + 3) >> 2;
  const int ot = (kBpCols / 4) * nq;  // threads with one (column quad, player quad)
  const int splits = kThreads / ot;   // row splits
  const bool active = tid < ot * splits;
  const int o = tid % ot, sp = tid / ot;
  const int cq = o % (kBpCols / 4), pq = o / (kBpCols / 4);

  constexpr int kZR = kBpRows * kBpCols / kThreads;
  float zr[kZR];
  auto load_z = [&](int64_t r0) {
#pragma unroll
    for (int j = 0; j < kZR; ++j) {
      const int slot = tid + kThreads * j;
      const int cc = slot % kBpCols, rr = slot / kBpCols;
      const int64_t row = r0 + rr, cg = col0 + cc;
      zr[j] = (row < r_end && cg < ld) ? centred(cz, load_row_elem(Z, rs, row, row * ld + cg), row, ld, cg, isY)
                                       : 0.f;
    }
  };
  // P / Q rows of the stage, each into the estimate(s) it feeds (zeros elsewhere)
  auto load_w = [&](int64_t r0, int bsel) {
    float* wa = WA + bsel * kBpRows * kWS;
    float* wb = WB + bsel * kBpRows * kWS;
    for (int e = tid; e < kBpRows * k; e += kThreads) {
      const int rr = e / k, i = e % k;
      const int64_t row = r0 + rr;
      const bool in = row < r_end;
      if (wantA) {
        const bool v = in && (!splitAB || row < nA);
        cp_async4(wa + rr * kWS + i, v ? PQ + row * 2 * k + offA + i : PQ, v);
      }
      if (wantB) {
        const bool v = in && (!splitAB || row >= nA);
        cp_async4(wb + rr * kWS + i, v ? PQ + row * 2 * k + own + i : PQ, v);
      }
    }
    cp_async_commit_all();
  };
  auto store_z = [&]() {
#pragma unroll
    for (int j = 0; j < kZR; ++j) {
      const int slot = tid + kThreads * j;
      Zs[(slot / kBpCols) * kBpZS + slot % kBpCols] = zr[j];
    }
  };

  __syncthreads();  // the workspace may still be read by this block's previous tile
  zero_player_pad(WA, 4 * kBpRows, k);  // both buffers of WA and WB
  float accA[4][4], accB[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) accA[a][c] = accB[a][c] = 0.f;
  if (r_begin < r_end) {
    load_w(r_begin, 0);
    load_z(r_begin);
  }
  int buf = 0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kBpRows, buf ^= 1) {
    store_z();
    cp_async_wait_all();
    __syncthreads();
    const int nr = (int)min((int64_t)kBpRows, r_end - r0);
    const bool useA = wantA && (!splitAB || r0 < nA);
    const bool useB = wantB && (!splitAB || r0 + nr > nA);
    if (r0 + kBpRows < r_end) {
      load_w(r0 + kBpRows, buf ^ 1);
      load_z(r0 + kBpRows);
    }
    if (active) {
      const float* wa = WA + buf * kBpRows * kWS + 4 * pq;
      const float* wb = WB + buf * kBpRows * kWS + 4 * pq;
      const float* zs = Zs + 4 * cq;
      if (useA && useB) {
#pragma unroll 2
        for (int rr = sp; rr < nr; rr += splits) {
          const float4 z = lds4(zs + rr * kBpZS);
          fma4x4(accA, z, lds4(wa + rr * kWS));
          fma4x4(accB, z, lds4(wb + rr * kWS));
        }
      } else if (useA) {
#pragma unroll 4
        for (int rr = sp; rr < nr; rr += splits) fma4x4(accA, lds4(zs + rr * kBpZS), lds4(wa + rr * kWS));
      } else if (useB) {
#pragma unroll 4
        for (int rr = sp; rr < nr; rr += splits) fma4x4(accB, lds4(zs + rr * kBpZS), lds4(wb + rr * kWS));
      }
    }
    __syncthreads();
  }
  const int64_t coff = isY ? dx : 0;
  auto valid = [&](int c) { return col0 + c < ld; };
  auto orow = [&](int c) { return (coff + col0 + c) * k; };
  if (wantA) reduce_quads(accA, active, splits, sp, cq, pq, k, inv_nA, smem, AV, valid, orow);
  if (wantB) reduce_quads(accB, active, splits, sp, cq, pq, k, inv_nB, smem, BV, valid, orow);
}

// ---------------------------------------------------------------------------
// k x k terms: a_ij = sum_c V[c,i] AV[c,j];  G_ij = sum_c V[c,i] S[c,j];
//              b_i = sum_c V[c,i] (B_t V)[c,i] with B_t V = BV + eps V (or (1+eps) V when B = I).
// gram layout: [a (k*k) | G (k*k) | b (k) | norms (k)]; must be zeroed. Grid-stride
// over 32-row chunks of V: tile `bx` of `nb`. Each chunk's rows of V, AV, S and BV are
// staged (players padded to a multiple of 4 with zeros); a thread owns a 4 x 4 block
// (players 4iq.., 4jq..) of both a and G over the rows of its split, so one float4 of V,
// of AV and of S feed 32 FMAs. The splits' partials are added in shared memory, then one
// atomic per entry.
__device__ inline void gram_tile(const float* __restrict__ V, const float* __restrict__ S,
                                 const float* __restrict__ AV, const float* __restrict__ BV, int64_t d, int k,
                                 float eps_B, int b_is_identity, float* __restrict__ gram, int bx, int nb,
                                 float* smem) {
  constexpr int CR = 32;
  const int kp = (k + 3) & ~3, nq = kp >> 2;
  const int gs = kp + 4;         // staged row stride
  float* Vs = smem;              // CR x gs
  float* As = Vs + CR * gs;
  float* Ss = As + CR * gs;
  float* Bs = Ss + CR * gs;
  const int tid = threadIdx.x;
  const int kk = k * k;
  const int tiles = nq * nq;
  const int splits = min(kThreads / tiles, CR);
  const int t = tid % tiles, sp = tid / tiles;
  const bool active = sp < splits;
  const int iq = t / nq, jq = t % nq;
  const int si = tid % 64, sr = tid / 64;  // staging: player si of rows sr + 4u
  float acc_a[4][4], acc_g[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc_a[x][y] = acc_g[x][y] = 0.f;
  float gb = 0.f;
  __syncthreads();  // the workspace may still be read by this block's previous tile
  for (int64_t c0 = (int64_t)bx * CR; c0 < d; c0 += (int64_t)nb * CR) {
    const int nr = (int)min((int64_t)CR, d - c0);
    if (si < kp) {
      float xv[CR / 4], xa[CR / 4], xs[CR / 4], xb[CR / 4];
#pragma unroll
      for (int u = 0; u < CR / 4; ++u) {
        const int rr = sr + 4 * u;
        const bool ok = si < k && rr < nr;
        const int64_t idx = (c0 + rr) * k + si;
        xv[u] = ok ? V[idx] : 0.f;
        xa[u] = ok ? AV[idx] : 0.f;
        xs[u] = ok ? S[idx] : 0.f;
        xb[u] = (ok && !b_is_identity) ? BV[idx] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < CR / 4; ++u) {
        const int o = (sr + 4 * u) * gs + si;
        Vs[o] = xv[u];
        As[o] = xa[u];
        Ss[o] = xs[u];
        Bs[o] = xb[u];
        // <v_i, B_t v_i>: this thread's rows of player si, summed in registers
        gb = fmaf(xv[u], b_is_identity ? (1.f + eps_B) * xv[u] : xb[u] + eps_B * xv[u], gb);
      }
    }
    __syncthreads();
    if (active) {
      for (int rr = sp; rr < nr; rr += splits) {
        const float4 v4 = lds4(Vs + rr * gs + 4 * iq);
        fma4x4(acc_a, v4, lds4(As + rr * gs + 4 * jq));
        fma4x4(acc_g, v4, lds4(Ss + rr * gs + 4 * jq));
      }
    }
    __syncthreads();
  }
  // add the splits' partials of a, then of G (red aliases the staging buffers)
  float* red = smem;  // [splits][kp][kp]
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    if (active) {
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const float* src = m == 0 ? acc_a[x] : acc_g[x];
        *reinterpret_cast<float4*>(red + (sp * kp + 4 * iq + x) * kp + 4 * jq) =
            make_float4(src[0], src[1], src[2], src[3]);
      }
    }
    __syncthreads();
    for (int p = tid; p < kk; p += kThreads) {
      const int i = p / k, j = p % k;
      float sum = 0.f;
      for (int s2 = 0; s2 < splits; ++s2) sum += red[(s2 * kp + i) * kp + j];
      atomicAdd(&gram[m * kk + p], sum);
    }
    __syncthreads();
  }
  if (si < k) atomicAdd(&gram[2 * kk + si], gb);  // one partial per staging row group
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
  float* Ss = sden + k;          // kUpdRows * rows x k
  float* terms = Ss + kUpdRows * rows * k;  // a | G | b of the step, staged
  for (int p = threadIdx.x; p < 2 * k * k + k; p += blockDim.x) terms[p] = gram[p];
  if (var.z)
    for (int j = threadIdx.x; j < k; j += blockDim.x) sden[j] = smooth_den(var.z[j], var.log_rho, var.log_nu);
  __syncthreads();
  eg_coefficients(terms, k, rho, cb, cac, T, var.z ? sden : nullptr);
  for (int i = threadIdx.x; i < k; i += blockDim.x) nrm[i] = 0.f;
  __syncthreads();
  const int tid = threadIdx.x;
  const int rl = tid / k, i = tid % k;
  const bool active = rl < rows;
  float my_norm = 0.f;
  // kUpdRows rows per thread per iteration (rows rl + rows u), every load in flight at once
  const int64_t span = (int64_t)rows * kUpdRows;
  for (int64_t c0 = (int64_t)bx * span; c0 < d; c0 += (int64_t)nb * span) {
    float xs[kUpdRows], xv[kUpdRows], xa[kUpdRows], xb[kUpdRows];
#pragma unroll
    for (int u = 0; u < kUpdRows; ++u) {
      const int64_t c = c0 + rl + (int64_t)rows * u;
      const bool ok = active && c < d;
      const int64_t idx = c * k + i;
      xs[u] = ok ? S[idx] : 0.f;
      xv[u] = ok ? V[idx] : 0.f;
      xa[u] = ok ? AV[idx] : 0.f;
      xb[u] = (ok && !b_is_identity) ? BV[idx] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kUpdRows; ++u)
      if (active) Ss[(rl + rows * u) * k + i] = xs[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kUpdRows; ++u) {
      const int64_t c = c0 + rl + (int64_t)rows * u;
      const bool ok = active && c < d;
      const int64_t idx = c * k + i;
      const float s_old = xs[u];
      const int srow = (rl + rows * u) * k;
      if (ok) {
        const float v = xv[u];
        const float bv = b_is_identity ? (1.f + eps_B) * v : xb[u] + eps_B * v;
        float pen = 0.f;
        for (int j = 0; j < i; ++j) pen = fmaf(Ss[srow + j], T[j * k + i], pen);
        const float gr = cb[i] * xa[u] - cac[i] * bv - pen;
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
  float* xs = smem + C * kThreads + kThreads;                    // [2][kStatsRows][kThreads]
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
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
      if (!rs && ((uintptr_t)X & 3) == 0) {
        // BF16 rows: each thread stages, by 4-byte cp.async (double-buffered, blocks of kStatsRows
        // rows), the aligned value pair that holds its column's value and keeps its half (no
        // barrier: a thread reads only what it copied). A pair that would reach past the
        // matrix's last value is read directly instead.
        const int64_t total = b * d;
        auto issue = [&](int s0, int buf) {
#pragma unroll
          for (int q = 0; q < kStatsRows; ++q) {
            const int64_t a = (r0 + s0 + q) * d + col;
            const bool ok = col < d && s0 + q < nr && (a | 1) < total;
            cp_async4(xs + (buf * kStatsRows + q) * kThreads + tid,
                      reinterpret_cast<const float*>(ok ? X + (a & ~(int64_t)1) : X), ok);
          }
          cp_async_commit_all();
        };
        if (col >= d) continue;
        issue(0, 0);
        int buf = 0;
        for (int s0 = 0; s0 < nr; s0 += kStatsRows, buf ^= 1) {
          if (s0 + kStatsRows < nr) {
            issue(s0 + kStatsRows, buf ^ 1);
            cp_async_wait_pending<1>();
          } else {
            cp_async_wait_all();
          }
#pragma unroll
          for (int q = 0; q < kStatsRows; ++q) {
            const int lab2 = (s0 + q < nr) ? labs[s0 + q] : -1;
            if (lab2 >= 0) {
              const int64_t a = (r0 + s0 + q) * d + col;
              float v;
              if ((a | 1) < total) {
                const __nv_bfloat162 pr =
                    *reinterpret_cast<const __nv_bfloat162*>(xs + (buf * kStatsRows + q) * kThreads + tid);
                v = (a & 1) ? __high2float(pr) : __low2float(pr);
              } else {
                v = __bfloat162float(X[a]);
              }
              acc[lab2 * kThreads + tid] += v;
            }
          }
        }
        continue;
      }
    }
    if (col >= d) continue;
    if constexpr (std::is_same<T, float>::value) {
      if (!rs) {
        // Plain FP32 rows: each thread stages its own column in blocks of kStatsRows rows by
        // cp.async (double-buffered), so the loads of a block are in flight together and
        // ahead of the additions (no barrier: a thread reads only what it copied).
        const float* xcol = X + col;
        auto issue = [&](int s0, int buf) {
#pragma unroll
          for (int q = 0; q < kStatsRows; ++q) {
            const bool ok = s0 + q < nr;
            cp_async4(xs + (buf * kStatsRows + q) * kThreads + tid, ok ? xcol + (r0 + s0 + q) * d : xcol, ok);
          }
          cp_async_commit_all();
        };
        issue(0, 0);
        int buf = 0;
        for (int s0 = 0; s0 < nr; s0 += kStatsRows, buf ^= 1) {
          if (s0 + kStatsRows < nr) {
            issue(s0 + kStatsRows, buf ^ 1);
            cp_async_wait_pending<1>();
          } else {
            cp_async_wait_all();
          }
#pragma unroll
          for (int q = 0; q < kStatsRows; ++q) {
            const int lab2 = (s0 + q < nr) ? labs[s0 + q] : -1;
            if (lab2 >= 0) acc[lab2 * kThreads + tid] += xs[(buf * kStatsRows + q) * kThreads + tid];
          }
        }
        continue;
      }
    }
    {
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

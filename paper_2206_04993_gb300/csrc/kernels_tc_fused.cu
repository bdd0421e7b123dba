// One-read tensor-core products of a BF16 minibatch (large d): X V and X^T (X V)
// with the minibatch streamed from HBM once.
//
// Grid: one persistent CTA per 256-column slice of X and of Y (2 * d_x / 256
// CTAs, launched cooperatively so that all of them are resident). Rows are
// processed in blocks of 128. For every row block:
//   A. TMA brings the block's tile of the slice from HBM (four 128 x 64 boxes);
//      tcgen05 multiplies it by the slice of V^T (BF16 hi/lo pairs, resident in
//      shared memory) into a double-buffered TMEM tile: the slice's partial row
//      projections.
//   B. Four epilogue warps move the partial projections to shared memory
//      (double-buffered) and a bulk reduce-add (TMA, performed at L2) sums them
//      into one of kRep replicas of the row block's P (X CTAs) or Q (Y CTAs),
//      chosen by the slice index; a release counter records the contribution
//      once the reduction is complete. With replicas, each element receives
//      d_x / 256 / kRep reductions instead of d_x / 256: reductions into one
//      L2 location serialise, and that serialisation bounded the step.
//   C. Combiner CTAs (kComb extra CTAs on otherwise idle SMs) wait until all
//      CTAs of a view have contributed to a row block, add its replicas, write
//      the final P or Q rows, clear the replicas and release a second counter.
//   D. A builder group (four warps) waits for the final rows of the view a row
//      block needs (the other view for rows that estimate A, its own view for
//      rows that estimate B), bulk-copies them to shared memory and writes
//      their BF16 hi/lo pairs as a 128-byte-swizzled K-major operand.
//   E. The tile is fetched again -- from L2, some microseconds after A -- in four
//      64-row x 128-column items, and tcgen05 multiplies each item's transpose
//      (the row-major tile read MN-major) by the operand into the slice's
//      A_t V or B_t V accumulators, which stay in TMEM for the whole step and
//      are written out once.
// A and B run ahead of C, D and E; only C and D wait on other CTAs, and nothing
// they wait for depends on D or E, so the pipeline cannot deadlock. Every wait is
// time-bounded: on expiry the kernel records SGEP's timeout bit and winds down.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "internal.h"
#include "tc_common.cuh"

namespace sgep {
namespace {

using namespace tc;

// w0 TMA(A), w1 MMA(A), w2-5 publish + write-out, w6 TMA+MMA(E), w7-10 W builders
constexpr int kThreads = 352;
constexpr int kRep = 8;   // replicas of P and Q
constexpr int kComb = 8;  // combiner CTAs (half per view)
constexpr int kBuilder0 = 7;
constexpr int kAStages = 4;
constexpr int kDStages = 3;
constexpr int kVT = 32768;     // V^T slice: four 64 x 64 boxes
constexpr int kABox = 16384;   // one 128 x 64 box of the minibatch
constexpr int kDItem = 16384;  // 64 rows x 128 columns: two 64 x 64 boxes
constexpr int kWT = 16384;     // W operand: two 64 x 64 boxes
constexpr int kStg = 16384;    // 128 rows x 32 FP32 partial projections
constexpr int kPst = 16384;    // 128 rows x 32 FP32 summed projections (two 64-row halves)
constexpr int kBars = 26;
constexpr size_t kSmem = kVT + kAStages * kABox + kDStages * kDItem + 2 * kWT + 2 * kStg + kPst + 1024 + 512;
static_assert(kSmem <= 232448, "shared memory budget");

struct FusedArgs {
  int64_t b, nA, d_x;
  int nrb;      // row blocks (b / 128)
  int nslice;   // 256-column slices per view (CTAs per view)
  int k;
  float inv_nA, inv_nB;
  float* Pg;        // [2][b][32] final row projections (P then Q), written by the combiners
  float* Prep;      // [kRep][2][b][32] replicas, zero at launch (the combiners clear them again)
  unsigned* cnt;    // [2][nrb] contributions reduced, then [2][nrb] final rows written; zeroed before launch
  float* AV;        // d x k
  float* BV;        // d x k
  int* dflag;
  unsigned long long* trace;  // [CTA][nrb + 1][kEv] globaltimer stamps, or null
};

// Trace events per row block; row nrb of a CTA holds its start and end.
constexpr int kEv = 9;
enum { kEvMma1 = 0, kEvReduce, kEvReadDone, kEvRelease, kEvCombined, kEvCounter, kEvPFull, kEvW, kEvMma2 };

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// Two FP32 values as packed BF16 (first value in the low half).
__device__ __forceinline__ uint32_t pack2_bf16(float first, float second) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(first, second);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Combiner CTA: adds the replicas of the row blocks rb = first, first + kComb / 2, ...
// of one view into the final rows, clears the replicas and releases the blocks.
__device__ void combine_blocks(const FusedArgs& a, uint8_t* base) {
  float* RB = reinterpret_cast<float*>(base);  // [kRep][128][32]
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + kRep * 16384);
  volatile int* ok_s = reinterpret_cast<volatile int*>(bar + 1);
  const int ci = (int)blockIdx.x - 2 * a.nslice;
  const int per_view = kComb / 2;
  const int view = ci / per_view, first = ci % per_view;
  const int nrb = a.nrb, tid = threadIdx.x;
  unsigned* cnt_part = a.cnt;
  unsigned* cnt_final = a.cnt + 2 * nrb;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  int it = 0;
  bool inflight = false;
  for (int rb = first; rb < nrb; rb += per_view, ++it) {
    if (tid == 0) {
      const bool ok = spin_until_geq(cnt_part + view * nrb + rb, (unsigned)a.nslice);
      if (ok) {
        fence_proxy_async_global();
        mbar_arrive_expect_tx(bar, kRep * 16384);
        for (int r = 0; r < kRep; ++r)
          bulk_load_g2s(RB + r * 4096, a.Prep + (((size_t)r * 2 + view) * a.b + (size_t)rb * 128) * 32, 16384, bar);
        inflight = true;
      } else {
        atomicOr(a.dflag, kFlagTimeout);
      }
      *ok_s = ok ? 1 : 0;
    }
    __syncthreads();
    if (!*ok_s) break;
    if (!mbar_wait(bar, it & 1)) {  // every thread waits; a failure is recorded and the block skipped
      atomicOr(a.dflag, kFlagTimeout);
    } else {
      if (tid == 0) inflight = false;
      const float4* r4 = reinterpret_cast<const float4*>(RB);
      float4* out = reinterpret_cast<float4*>(a.Pg + ((size_t)view * a.b + (size_t)rb * 128) * 32);
      for (int i = tid; i < 1024; i += kThreads) {
        float4 v = r4[i];
#pragma unroll
        for (int r = 1; r < kRep; ++r) {
          const float4 w = r4[r * 1024 + i];
          v.x += w.x;
          v.y += w.y;
          v.z += w.z;
          v.w += w.w;
        }
        out[i] = v;
#pragma unroll
        for (int r = 0; r < kRep; ++r)
          reinterpret_cast<float4*>(a.Prep + (((size_t)r * 2 + view) * a.b + (size_t)rb * 128) * 32)[i] =
              make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      red_release_add(cnt_final + view * nrb + rb, 1u);
      if (a.trace) a.trace[((size_t)blockIdx.x * (nrb + 1) + rb) * kEv + kEvCombined] = globaltimer();
    }
  }
  if (tid == 0 && inflight) mbar_wait(bar, it & 1, 100000000ull);  // copies land before the CTA exits
}

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_fused(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
               const __grid_constant__ CUtensorMap mapX64, const __grid_constant__ CUtensorMap mapY64,
               const __grid_constant__ CUtensorMap mapVt, const FusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  if ((int)blockIdx.x >= 2 * a.nslice) {
    combine_blocks(a, base);
    return;
  }
  uint8_t* VT = base;
  uint8_t* AST = VT + kVT;
  uint8_t* DST = AST + kAStages * kABox;
  uint8_t* WT = DST + kDStages * kDItem;
  float* STG = reinterpret_cast<float*>(WT + 2 * kWT);  // [2][128][32]
  float* PST = STG + 2 * (kStg / 4);                     // [128][32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(PST) + kPst);
  uint64_t* a_full = bars;          // [4]
  uint64_t* a_empty = bars + 4;     // [4]
  uint64_t* d1_full = bars + 8;     // [2]
  uint64_t* d1_empty = bars + 10;   // [2]
  uint64_t* d_full = bars + 12;     // [3]
  uint64_t* d_empty = bars + 15;    // [3]
  uint64_t* w_full = bars + 18;     // [2]
  uint64_t* w_empty = bars + 20;    // [2]
  uint64_t* vt_full = bars + 22;
  uint64_t* acc_done = bars + 23;
  uint64_t* p_full = bars + 24;     // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* used = reinterpret_cast<volatile int*>(tmem_slot + 2);  // [AV h0, AV h1, BV h0, BV h1]
  volatile int* pub_ok = used + 4;    // decisions broadcast to a group of warps
  volatile int* wo_ok = used + 5;
  volatile int* b_ok = used + 6;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int view = (int)blockIdx.x >= a.nslice ? 1 : 0;
  const int slice = (int)blockIdx.x - view * a.nslice;
  const int64_t col0 = (int64_t)slice * 256;
  const int64_t goff = (view ? a.d_x : 0) + col0;
  const CUtensorMap* mZ = view ? &mapY : &mapX;
  const CUtensorMap* mZ64 = view ? &mapY64 : &mapX64;
  const int nrb = a.nrb;
  unsigned* cnt_part = a.cnt;
  unsigned* cnt_final = a.cnt + 2 * nrb;

  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < kBars; ++i) mbar_init(bars + i, 1);
    *abort_flag = 0;
    for (int i = 0; i < 4; ++i) used[i] = 0;
    fence_mbar_init();
    prefetch_tensormap(mZ);
    prefetch_tensormap(mZ64);
    prefetch_tensormap(&mapVt);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto stamp = [&](int rb, int ev) {
    if (a.trace) a.trace[((size_t)blockIdx.x * (nrb + 1) + rb) * kEv + ev] = globaltimer();
  };
  if (tid == 0) stamp(nrb, 0);
  auto fail = [&]() {
    atomicOr(a.dflag, kFlagTimeout);
    *abort_flag = 1;
  };

  if (warp == 0) {
    // ---- A: HBM tiles of the slice -------------------------------------------
    if (lane == 0) {
      mbar_arrive_expect_tx(vt_full, kVT);
      for (int j = 0; j < 4; ++j) tma_load_2d(VT + j * 8192, &mapVt, (int)(goff + 64 * j), 0, vt_full);
      int issued = 0;
      for (int i = 0; i < nrb * 4 && !*abort_flag; ++i) {
        const int st = i & (kAStages - 1);
        if (i >= kAStages && !mbar_wait(a_empty + st, ((i / kAStages) - 1) & 1)) {
          fail();
          break;
        }
        mbar_arrive_expect_tx(a_full + st, kABox);
        tma_load_2d(AST + st * kABox, mZ, (int)(col0 + 64 * (i & 3)), (i >> 2) * 128, a_full + st);
        issued = i + 1;
      }
      // the copies of the last stages land before the CTA may exit
      for (int i = issued > kAStages ? issued - kAStages : 0; i < issued; ++i)
        mbar_wait(a_full + (i & (kAStages - 1)), (i / kAStages) & 1, 100000000ull);
      mbar_wait(vt_full, 0, 100000000ull);
    }
  } else if (warp == 1) {
    // ---- A: partial projections X_tile V_slice -------------------------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, 64, 0, 0);
      bool ok = mbar_wait(vt_full, 0);
      for (int rb = 0; ok && rb < nrb; ++rb) {
        const int buf = rb & 1;
        if (rb >= 2 && !mbar_wait(d1_empty + buf, ((rb >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int bx = 0; bx < 4; ++bx) {
          const int i = rb * 4 + bx, st = i & (kAStages - 1);
          if (!mbar_wait(a_full + st, (i / kAStages) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16(tmem + 64 * buf, desc_sw128(AST + st * kABox + kk * 32, 16, 1024),
                     desc_sw128(VT + bx * 8192 + kk * 32, 16, 1024), idesc, (bx | kk) ? 1u : 0u);
          mma_commit(a_empty + st);
        }
        if (!ok) break;
        mma_commit(d1_full + buf);
        stamp(rb, kEvMma1);
      }
      if (!ok) fail();
    }
  } else if (warp <= 5) {
    // ---- B: publish the partial projections ----------------------------------
    // Staging is double-buffered and a block's counter is released two blocks
    // later, so up to three reductions are in flight.
    const int ptid = tid - 64;
    const int q = warp & 3;
    const int r = 32 * q + lane;
    float* rep = a.Prep + ((size_t)(slice % kRep) * 2 + view) * a.b * 32;
    for (int rb = 0; rb < nrb; ++rb) {
      const int buf = rb & 1;
      float* stg = STG + buf * (kStg / 4);
      if (ptid == 0) {
        *pub_ok = mbar_wait(d1_full + buf, (rb >> 1) & 1) ? 1 : 0;
        bulk_wait_read<1>();  // the reduction two blocks back has read this staging buffer
        if (rb >= 1) stamp(rb - 1, kEvReadDone);
      }
      named_barrier(1, 128);
      if (!*pub_ok) {
        if (ptid == 0) fail();
        break;
      }
      tc_fence_after();
      float hi[32], lo[32];
      tmem_ld32(tmem + 64 * buf + ((uint32_t)(32 * q) << 16), hi);
      tmem_ld32(tmem + 64 * buf + 32 + ((uint32_t)(32 * q) << 16), lo);
      tc_fence_before();
      float4* dst = reinterpret_cast<float4*>(stg + r * 32);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        dst[j] = make_float4(hi[4 * j] + lo[4 * j], hi[4 * j + 1] + lo[4 * j + 1], hi[4 * j + 2] + lo[4 * j + 2],
                             hi[4 * j + 3] + lo[4 * j + 3]);
      fence_proxy_async_smem();
      named_barrier(1, 128);  // TMEM tile read and staging written by all four warps
      if (ptid == 0) {
        mbar_arrive(d1_empty + buf);
        bulk_reduce_add_f32(rep + (size_t)rb * 128 * 32, stg, kStg);
        bulk_commit();
        stamp(rb, kEvReduce);
        bulk_wait<2>();  // reductions up to block rb - 2 are complete: publish them
        if (rb >= 2) {
          fence_proxy_async_global();
          __threadfence();
          red_release_add(cnt_part + view * nrb + rb - 2, 1u);
          stamp(rb - 2, kEvRelease);
        }
      }
    }
    if (ptid == 0) {
      bulk_wait<0>();  // no reduction may still read the staging buffers when the CTA exits
      if (!*abort_flag) {
        fence_proxy_async_global();
        __threadfence();
        for (int rb = nrb >= 2 ? nrb - 2 : 0; rb < nrb; ++rb) {
          red_release_add(cnt_part + view * nrb + rb, 1u);
          stamp(rb, kEvRelease);
        }
      }
    }
  } else if (warp == 6) {
    // ---- D: tiles again (L2) and X_tile^T W into the accumulators -------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, 64, 1, 0);
      const uint64_t once = policy_evict_first();
      bool ok = true;
      bool u[4] = {false, false, false, false};
      const int nitems = 4 * nrb;  // item j: row block j / 4, column half (j / 2) % 2, row half j % 2
      int issued = 0;
      auto issue = [&](int j) -> bool {
        const int st = j % kDStages;
        if (j >= kDStages && !mbar_wait(d_empty + st, ((j / kDStages) - 1) & 1)) return false;
        mbar_arrive_expect_tx(d_full + st, kDItem);
        const int rb = j >> 2, h = (j >> 1) & 1, g = j & 1;
        for (int jj = 0; jj < 2; ++jj)
          tma_load_2d_hint(DST + st * kDItem + jj * 8192, mZ64, (int)(col0 + 128 * h + 64 * jj), rb * 128 + 64 * g,
                           d_full + st, once);
        return true;
      };
      while (ok && issued < nitems && issued < kDStages) ok = issue(issued++);
      for (int j = 0; ok && j < nitems; ++j) {
        const int rb = j >> 2, h = (j >> 1) & 1, g = j & 1, st = j % kDStages;
        const int wb = rb & 1;
        if ((j & 3) == 0 && !mbar_wait(w_full + wb, (rb >> 1) & 1)) {
          ok = false;
          break;
        }
        if (!mbar_wait(d_full + st, (j / kDStages) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int rowA = (int64_t)rb * 128 < a.nA;
        const int slot = (rowA ? 0 : 2) + h;
        const uint32_t acc = tmem + 128 + 64 * slot;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(acc, desc_sw128(DST + st * kDItem + kk * 2048, 8192, 1024),
                   desc_sw128(WT + wb * kWT + g * 8192 + kk * 32, 16, 1024), idesc, (u[slot] || kk) ? 1u : 0u);
        u[slot] = true;
        mma_commit(d_empty + st);
        if ((j & 3) == 3) {
          mma_commit(w_empty + wb);
          stamp(rb, kEvMma2);
        }
        // refill the stage of item j - 1 (its MMA is queued ahead of item j's)
        while (ok && issued < nitems && issued <= j + kDStages - 1) ok = issue(issued++);
      }
      for (int i = 0; i < 4; ++i) used[i] = u[i] ? 1 : 0;
      if (ok) {
        mma_commit(acc_done);
      } else {
        fail();
        mbar_arrive(acc_done);
        for (int st = 0; st < kDStages; ++st) {  // the copies of the last items land before the CTA may exit
          int last = -1;
          for (int j = st; j < issued; j += kDStages) last = j;
          if (last >= 0) mbar_wait(d_full + st, (last / kDStages) & 1, 100000000ull);
        }
      }
    }
  } else {
    // ---- C: W operand of each row block (BF16 hi/lo pairs, swizzled K-major) -
    // Builder warp bw converts the 64-row half bw / 2 (W box bw / 2), projection
    // columns 16 (bw % 2) .. 16 (bw % 2) + 15. Lane 0 of the first builder warp
    // waits for the counters, issues the copies and makes every decision the
    // four warps act on.
    const int bw = warp - kBuilder0;
    const int g = bw >> 1;
    const int cb = 4 * (bw & 1);  // first float4 of this warp's columns
    const bool leader = bw == 0 && lane == 0;
    auto need_of = [&](int rb) { return ((int64_t)rb * 128 < a.nA) ? 1 - view : view; };
    auto fetch = [&](int rb) {
      for (int hh = 0; hh < 2; ++hh) {
        mbar_arrive_expect_tx(p_full + hh, 8192);
        bulk_load_g2s(PST + hh * 2048, a.Pg + ((size_t)need_of(rb) * a.b + (size_t)rb * 128 + 64 * hh) * 32, 8192,
                      p_full + hh);
      }
    };
    int issued = 0;  // leader: row blocks whose copies were issued
    if (leader) {
      const bool ok = spin_until_geq(cnt_final + need_of(0) * nrb, 1u);
      if (ok) {
        stamp(0, kEvCounter);
        fence_proxy_async_global();
        fetch(0);
        issued = 1;
      } else {
        fail();
      }
    }
    const int rr = 2 * lane;  // row pair within the 64-row half
    const float4* s0 = reinterpret_cast<const float4*>(PST + (64 * g + rr) * 32);
    const float4* s1 = s0 + 8;
    const uint32_t inrow = (uint32_t)(rr & 7) * 2;
    const uint32_t chunk = (uint32_t)rr >> 3;
    for (int rb = 0; rb < nrb; ++rb) {
      const int wb = rb & 1;
      if (leader) {
        bool ok = !*abort_flag;
        if (ok && rb >= 2) ok = mbar_wait(w_empty + wb, ((rb >> 1) - 1) & 1);
        if (!ok) fail();
        *b_ok = ok ? 1 : 0;
      }
      named_barrier(2, 128);
      if (!*b_ok) break;
      int okw = 1;
      if (lane == 0) {
        okw = mbar_wait(p_full + g, rb & 1) ? 1 : 0;
        if (leader) stamp(rb, kEvPFull);
      }
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (okw) {
        uint8_t* box = WT + wb * kWT + g * 8192;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int jj = cb + ((j + lane) & 3);  // rotated: few bank conflicts on the loads
          const float4 v0 = s0[jj], v1 = s1[jj];
          const float x0[4] = {v0.x, v0.y, v0.z, v0.w};
          const float x1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const uint32_t nh = 4 * jj + e, nl = 32 + nh;
            const uint32_t hp = pack2_bf16(x0[e], x1[e]);
            const float h0 = __uint_as_float(hp << 16), h1 = __uint_as_float(hp & 0xffff0000u);
            *reinterpret_cast<uint32_t*>(box + nh * 128 + ((chunk ^ (nh & 7)) << 4) + inrow) = hp;
            *reinterpret_cast<uint32_t*>(box + nl * 128 + ((chunk ^ (nl & 7)) << 4) + inrow) =
                pack2_bf16(x0[e] - h0, x1[e] - h1);
          }
        }
        fence_proxy_async_smem();  // W visible to the tensor core; PST reads ordered before the next copy
      } else if (lane == 0) {
        fail();
      }
      named_barrier(2, 128);  // the block's operand is complete (or a warp failed)
      if (leader) {
        if (!*abort_flag) {
          mbar_arrive(w_full + wb);
          stamp(rb, kEvW);
          if (rb + 1 < nrb) {
            if (spin_until_geq(cnt_final + need_of(rb + 1) * nrb + rb + 1, 1u)) {
              stamp(rb + 1, kEvCounter);
              fence_proxy_async_global();
              fetch(rb + 1);
              issued = rb + 2;
            } else {
              fail();
            }
          }
        }
      }
    }
    if (leader && issued > 0)  // copies in flight land before the CTA may exit
      for (int hh = 0; hh < 2; ++hh) mbar_wait(p_full + hh, (issued - 1) & 1, 100000000ull);
  }

  // ---- write-out of the accumulators (warps 2-5) ------------------------------
  __syncthreads();  // every role has left its loop; used[] is visible
  if (warp >= 2 && warp <= 5) {
    if (tid == 64) *wo_ok = (mbar_wait(acc_done, 0, 4000000000ull) && !*abort_flag) ? 1 : 0;
    named_barrier(1, 128);
    tc_fence_after();
    if (*wo_ok) {
      const int q = warp & 3;
      const int k = a.k;
#pragma unroll 1
      for (int slot = 0; slot < 4; ++slot) {
        float* out = slot < 2 ? a.AV : a.BV;
        const float sc = slot < 2 ? a.inv_nA : a.inv_nB;
        const int h = slot & 1;
        const int64_t col = goff + 128 * h + 32 * q + lane;
        if (!used[slot]) {
          for (int i = 0; i < k; ++i) out[col * k + i] = 0.f;
          continue;
        }
        float hi[32], lo[32];
        const uint32_t t = tmem + 128 + 64 * slot + ((uint32_t)(32 * q) << 16);
        tmem_ld32(t, hi);
        tmem_ld32(t + 32, lo);
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < k) out[col * k + i] = (hi[i] + lo[i]) * sc;
      }
    } else if (tid == 64) {
      atomicOr(a.dflag, kFlagTimeout);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0) stamp(nrb, 1);
  if (warp == 1) tmem_dealloc(tmem, 512);
}

}  // namespace

bool tc_fused_supported(const Ctx& c, int64_t b) {
  return c.d_x == c.d_y && c.d_x % 256 == 0 && 2 * (c.d_x / 256) + kComb <= c.num_sms && b % 256 == 0 &&
         c.cfg.split_AB;
}

int tc_fused_setup(Ctx& c) {
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_tc_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
  const size_t nrb = (size_t)c.cfg.max_b / 128;
  SGEP_CUDA_TRY(cudaMalloc(&c.tc_fused_buf, 4 * nrb * sizeof(unsigned)));
  c.tc_fused_bytes = 4 * nrb * sizeof(unsigned);
  const size_t rep = (size_t)kRep * 2 * c.cfg.max_b * 32 * sizeof(float);
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_fused_rep, rep));
  SGEP_CUDA_TRY(cudaMemset(c.tc_fused_rep, 0, rep));
  c.tc_fused_dirty = 0;
  const char* tr = getenv("SGEP_TRACE");
  if (tr && tr[0] == '1') {
    const size_t n = (size_t)c.num_sms * (nrb + 1) * kEv;
    SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_trace, n * sizeof(unsigned long long)));
    SGEP_CUDA_TRY(cudaMemset(c.tc_trace, 0, n * sizeof(unsigned long long)));
  }
  return SGEP_OK;
}

// acc = [A_t V ; B_t V] of one BF16 minibatch with one read of the minibatch from HBM.
// Vt (BF16 pairs of V) must be current; the row projections land in tc_PQ (P, then Q).
// mX / mY: 128 x 64 boxes; mX64 / mY64: 64 x 64 boxes of the same matrices.
int tc_fused_products(Ctx& c, const CUtensorMap& mX, const CUtensorMap& mY, const CUtensorMap& mX64,
                      const CUtensorMap& mY64, const CUtensorMap& mVt, int64_t b, cudaStream_t s) {
  const int nrb = (int)(b / 128);
  unsigned* cnt = reinterpret_cast<unsigned*>(c.tc_fused_buf);
  SGEP_CUDA_TRY(cudaMemsetAsync(cnt, 0, 4 * (size_t)nrb * sizeof(unsigned), s));
  if (c.tc_fused_dirty) {  // an aborted launch may have left partial sums in the replicas
    SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_fused_rep, 0, (size_t)kRep * 2 * c.cfg.max_b * 32 * sizeof(float), s));
    c.tc_fused_dirty = 0;
  }
  FusedArgs fa;
  fa.b = c.cfg.max_b;  // row stride of the halves of Pg and of the replicas
  fa.nA = b / 2;
  fa.d_x = c.d_x;
  fa.nrb = nrb;
  fa.nslice = (int)(c.d_x / 256);
  fa.k = c.k;
  fa.inv_nA = 1.f / (float)(b / 2);
  fa.inv_nB = 1.f / (float)(b - b / 2);
  fa.Pg = c.tc_PQ;  // [2][max_b][32]; rows [0, b) of each half are written
  fa.Prep = c.tc_fused_rep;
  fa.cnt = cnt;
  fa.AV = c.acc;
  fa.BV = c.acc + c.d * c.k;
  fa.dflag = c.dflag;
  fa.trace = c.tc_trace;
  c.tc_trace_grid = 2 * fa.nslice + kComb;
  c.tc_trace_nrb = nrb;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * fa.nslice + kComb));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: they wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SGEP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tc_fused, mX, mY, mX64, mY64, mVt, fa));
  ++c.launches;
  return SGEP_OK;
}

void tc_fused_trace_report(Ctx& c) {
  const int n = c.tc_trace_grid, nrb = c.tc_trace_nrb;
  if (!c.tc_trace || n <= 0) return;
  std::vector<unsigned long long> t((size_t)n * (nrb + 1) * kEv);
  if (cudaMemcpy(t.data(), c.tc_trace, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
    return;
  auto at = [&](int cta, int rb, int ev) { return t[((size_t)cta * (nrb + 1) + rb) * kEv + ev]; };
  unsigned long long g0 = ~0ull, s1 = 0, e0 = ~0ull, e1 = 0;
  for (int b = 0; b < n; ++b) {
    g0 = std::min(g0, at(b, nrb, 0));
    s1 = std::max(s1, at(b, nrb, 0));
    e0 = std::min(e0, at(b, nrb, 1));
    e1 = std::max(e1, at(b, nrb, 1));
  }
  std::fprintf(stderr,
               "[sgep trace] one-read kernel: %d CTAs (%d combiners), %d row blocks; start spread %.2f us, end "
               "%.2f-%.2f us\n",
               n, kComb, nrb, (s1 - g0) / 1e3, (e0 - g0) / 1e3, (e1 - g0) / 1e3);
  const char* names[kEv] = {"mma1", "reduce", "rdone", "release", "comb", "count", "pfull", "W", "mma2"};
  std::vector<int> rbs = {0, 1, 2, 3, nrb / 4, nrb / 2, 3 * nrb / 4, nrb - 2, nrb - 1};
  for (int rb : rbs) {
    if (rb < 0 || rb >= nrb) continue;
    std::fprintf(stderr, "[sgep trace] rb %3d (us, median/max over CTAs):", rb);
    for (int ev = 0; ev < kEv; ++ev) {
      std::vector<double> v;
      for (int b = 0; b < n; ++b)
        if (at(b, rb, ev)) v.push_back((at(b, rb, ev) - g0) / 1e3);
      std::sort(v.begin(), v.end());
      if (v.empty()) v.push_back(-1.0);
      std::fprintf(stderr, " %s %.2f/%.2f", names[ev], v[v.size() / 2], v.back());
    }
    std::fprintf(stderr, "\n");
  }
}

}  // namespace sgep

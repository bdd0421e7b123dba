// Streamed tensor-core steps of a BF16 minibatch sequence (large d): products, row-side
// terms and the update of Alg. 2 for one or more consecutive steps in one launch.
//
// Alg. 2 needs, per minibatch, the row projections P = X V_x, Q = Y V_y and the
// back-projections A_t V = [X_A^T Q_A ; Y_A^T P_A] / n_A, B_t V = [X_B^T P_B ; Y_B^T Q_B] / n_B.
// A row can be back-projected only once its projection is summed over all d
// columns, so a minibatch larger than shared memory is read twice. Here the
// second read comes from L2: rows are processed in chunks of kR rows (16 MB at
// d = 32768), and the back-projection of chunk c runs while chunk c + 1 streams
// in from HBM.
//
// Grid: G = d / 256 persistent CTAs, all resident (cooperative launch), one per SM.
//  * Projection role. Chunk c holds kR / 128 row tiles; its tiles are
//    (row tile, view, column split) with splits = d_x / (2 kR) column splits of
//    2 kR columns, exactly G tiles, so CTA j takes the same (view, split) in every
//    chunk and keeps its slice of V^T (BF16 hi/lo pairs, 64 x 2 kR) resident in
//    shared memory. tcgen05 multiplies 128 x 64 boxes of the minibatch by it into one of
//    four TMEM tiles; four epilogue warps stage each finished tile in shared memory and
//    one of four reducer warps adds it into P or Q with one bulk reduction (performed
//    at L2), waits for it and releases a per-row-tile counter.
//  * Builders. Helper CTAs on the SMs the streaming CTAs leave idle (their loads do not
//    queue behind the minibatch stream) take the row tiles' 64-row halves in turn: wait
//    for the tile's counter, turn the summed P and Q rows into the transposed BF16
//    hi/lo operand of the back-projection, release a per-half flag, then add the
//    row-side terms a_ij = sum_A (P_i Q_j + Q_i P_j) / n_A or b_i = sum_B (P_i^2 + Q_i^2)
//    / n_B and clear the rows for the next step.
//  * Back-projection role. CTA j owns a 256-column slice of X or Y (the rows j*256 ..
//    j*256 + 255 of V) and streams every row of it (from L2) in 64-row steps once the
//    step's row tile is built; tcgen05 multiplies each step's transpose by the operand into
//    four TMEM accumulators (A_t V, B_t V x two 128-column halves).
//  * Update role. When its accumulators and every row-side term of the step are in,
//    warps 4-11 of CTA j apply Eq. (update), the player step and the auxiliary step to
//    the slice's 256 rows (one row per thread, A_t V and B_t V read from tensor memory),
//    and write the rows of V, [Bv] and the next step's V^T operand.
// Several steps run in one launch. Within it the retraction of Alg. 2 is deferred: a
// step leaves v'_i = v_i + eta grad_i in memory, with its squared norm n_i^2 and the
// Gram U = V'^T [Bv]' summed over all CTAs by atomics; the next step projects with V'
// and divides what it gets by n_i (P, Q, A_t V, B_t V and the row-side terms are linear or
// bilinear in the players), which is the retraction v_i = v'_i / n_i applied exactly.
// The projection of the next step in CTA j therefore waits only for the two CTAs that
// own its V^T columns (per-CTA flags), never for the whole grid. The last step of the
// launch normalises behind one grid barrier, so between launches V is on the unit sphere.
// The projection runs at most kLag chunks ahead of the CTA's own back-projection so the
// rows it re-reads are still in L2. Waits only ever point at earlier chunks or steps,
// so the pipeline cannot deadlock; every wait is time-bounded and records the timeout bit
// of the device error word.
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

// Streaming CTAs: w0 projection TMA, w1 projection MMA (and the V^T slice loads), w2
// back-projection TMA, w3 back-projection MMA, w4-7 projection epilogue, w8-11 reducers
// (chunk g: warp 8 + g % 4 sums the staged tile into P or Q and releases it); w4-11 also
// run the update at the end of every step. Helper CTAs: w8-11 builders.
constexpr int kThreads = 384;
constexpr int kR = 256;         // rows per chunk (16 MB at d = 32768)
constexpr int kPS = 4;          // projection stages (one 128 x 64 box each)
constexpr int kBS = 2;          // back-projection stages (four 64 x 64 boxes + the operand box)
constexpr int kLagDefault = 5;  // chunks the projection may run ahead of the back-projection
constexpr int kPfNextDefault = 3;  // next-step chunks prefetched into L2 at the end of a step
constexpr int kMaxHelpers = 24; // builder CTAs on SMs the streaming CTAs leave idle
constexpr int kAcc = 4;         // projection accumulators in tensor memory (64 columns each)
constexpr int kVtBoxes = 2 * kR / 64;
constexpr int kVtB = kVtBoxes * 8192;  // resident V^T slice: 2 kR columns in 64 x 64 boxes
constexpr int kPBox = 16384;
constexpr int kBStage = 40960;
constexpr int kStgRows = 64;    // builder staging (helper CTAs, in the V^T region): 64 rows of P and Q
constexpr int kEStg = 128 * 32 * 4;  // epilogue staging: one 128 x 32 FP32 projection tile
constexpr int kNumBars = 2 * kPS + 2 * kAcc + 2 * kBS + 5 + 2 + 4 + 1;
constexpr size_t kSmem = (size_t)kVtB + kPS * kPBox + kBS * kBStage + kEStg + kNumBars * 8 + 64 + 1024;
static_assert(2 * kStgRows * 32 * 4 <= kVtB, "builder staging fits in the V^T region");
static_assert(2 * kStgRows * 32 * 4 + (3 * 32 * 32 + 4 * 32) * 4 <= kVtB,
              "builder staging and the coefficient scratch fit in the V^T region");
static_assert(kSmem <= 232448, "shared memory budget");
constexpr int kKP = 32;         // players padded to 32
constexpr int kTerms = kKP * kKP + kKP;  // one slot of row-side terms a (k x k) | b (k), or |v'|^2 | U
constexpr int kMaxSteps = 64;   // steps of one launch
constexpr int kCoef = kKP * kKP + 3 * kKP;  // one slot of update coefficients: T | b | a_ii - c_i | 1/n
// update scratch: V' and [Bv] rows [256][kRS] (16-byte aligned rows) in the back-projection stages
constexpr int kRS = 36;
static_assert(2 * 256 * kRS * 4 <= kBS * kBStage, "update rows fit in the back-projection stages");
static_assert(3 * kKP * kKP * 4 + 4 * kKP * 4 + 8 * kKP * 4 <= kEStg, "update coefficients fit in the staging tile");

struct StreamArgs {
  int64_t b, nA, d_x, ldt;  // ldt: row stride (elements) of Pt and Qt
  int64_t d;
  int k, nchunk, splits;
  int G;                    // streaming CTAs; CTAs G .. gridDim.x - 1 are builder helpers
  int H;                    // helper CTAs
  int lag;                  // chunks the projection may run ahead of the CTA's back-projection
  int nsteps;               // consecutive minibatches of this launch (rows s*b .. s*b + b - 1)
  int serial;               // the next step's projection also waits for the CTA's own update
  int bp_groups;            // mapX64 / mapY64 are 3-D views: one copy per 64-row back-projection step
  int pf_next;              // chunks of the next step's projection tile prefetched into L2, one as each of
                            // this step's last chunks is back-projected (0: two chunks at the step start)
  unsigned e0;              // steps streamed since the counters were cleared (epoch of step 0)
  float inv_nA, inv_nB;
  float rho, gamma, eps_B;
  float eta[kMaxSteps];     // step size of every step
  float* P;                 // [rows][32], zero on entry; the builders clear the rows again
  float* Q;
  __nv_bfloat16* Pt;        // [64][ldt] BF16 hi (0..31) / lo (32..63) pairs, transposed
  __nv_bfloat16* Qt;
  unsigned* cnt;            // [b / 128] projection contributions (monotone over steps)
  unsigned* wready;         // [b / 64] operand of the 64-row half built (monotone)
  unsigned* terms_done;     // row-side items added by the builders (monotone)
  unsigned* bar;            // grid-barrier arrivals (one barrier per launch, monotone)
  unsigned bar_target;
  unsigned* grams_done;     // helper CTAs (those owning a slice) that added a step's |v'|^2 and U (monotone)
  unsigned grams_base;      // its value at the launch
  unsigned* upd_done;       // [G] updates finished by CTA j: the V^T operand is written (monotone)
  unsigned* rows_done;      // [G] ... and the rows of V and [Bv] (monotone)
  unsigned* coef_ready;     // steps whose update coefficients are written (monotone)
  float* cbuf;              // [2][kCoef] update coefficients of step e in slot e & 1
  float* abbuf;             // [3][kTerms] row-side terms a | b of step e in slot e % 3
  float* ubuf;              // [3][kTerms] |v'_i|^2 | U of the V' left by step e - 1, slot e % 3
  float* V;                 // d x k, read and rewritten
  float* S;                 // d x k [Bv]
  const float* G0;          // k x k G_ij = <v_i, [Bv]_j> of the launch's first step
  const float* vv0;         // k |v_i|^2 of the launch's first step
  float* Gn;                // where the last step leaves G and |v_i|^2 for the next launch
  float* vvn;
  __nv_bfloat16* Vt;        // V^T operand (BF16 hi/lo pairs, 64 x d), rewritten every step
  float* AV;                // d x k products of the last step (debug), or null
  float* BV;
  float* dbg;               // a | G | b as used by the last step (debug), or null
  float* grad_out;          // update directions of the last step (debug), or null
  int* dflag;
  unsigned long long* trace;  // [G + H][nchunk + 2][kEv] globaltimer stamps of the last step, or null
  unsigned long long* trace2;  // [G][16] row-work stamps of the step before the last, or null
};

// Trace events per chunk (last step of the launch); row nchunk of a CTA holds start,
// projection end, back-projection end, end, then the last step's update phases (4 ..);
// row nchunk + 1 the update phases of the step before it.
constexpr int kEv = 12;
enum { kEvIssue = 0, kEvMma, kEvRelease, kEvBuildStart, kEvBuilt, kEvWSeen, kEvBpDone, kEvTerms };

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ uint32_t pack2_bf16(float first, float second) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(first, second);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// (hi, lo) BF16 split of two consecutive values: hi = bf16(v), lo = bf16(v - hi).
__device__ __forceinline__ uint32_t pack2_lo_bf16(float v0, float v1) {
  const float h0 = __bfloat162float(__float2bfloat16(v0)), h1 = __bfloat162float(__float2bfloat16(v1));
  return pack2_bf16(v0 - h0, v1 - h1);
}

// Waits (bounded) until a volatile shared counter reaches `target`.
__device__ __forceinline__ bool wait_shared_geq(volatile int* p, int target, uint64_t ns = 2000000000ull) {
  if (*p >= target) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (*p >= target) return true;
    if ((it & 63u) == 0 && globaltimer() - t0 > ns) return false;
    __nanosleep(64);
  }
}

// The k x k coefficients of step e's update, computed once per step by the 128 builder threads
// (bt) of the helper CTA that added the step's last row-side item: with the deferred norms
// n_i (step s > 0: n_i^2 and U from ubuf[e % 3]; step 0: n_i = 1, G and |v_i|^2 from G0, vv0),
// a_ij = a'_ij / (n_i n_j), b_i = b'_i / n_i^2 (+ eps_B |v_i|^2), G = diag(1/n) U, s_j =
// max(G_jj, rho), T_ji = b_i a_ij / s_j (j < i, else 0), c_i = sum_{j<i} a_ij G_ij / s_j.
// Writes T | b | a_ii - c_i | 1/n into cbuf[e & 1] (and a | G | b to dbg at the launch's last
// step), then releases coef_ready. sm: 3 * 32 * 32 + 4 * 32 floats. False on a timeout.
__device__ __forceinline__ bool build_coefficients(const StreamArgs& a, int s, unsigned e, int bt, float* sm,
                                                volatile int* ok) {
  const int k = a.k, kk = k * k;
  float* Am = sm;                // [32][32]
  float* Gm = Am + kKP * kKP;    // [32][32]
  float* T = Gm + kKP * kKP;     // [32][32]
  float* cb = T + kKP * kKP;
  float* cac = cb + kKP;
  float* inv_s = cac + kKP;
  float* inv_n = inv_s + kKP;
  const float* ab = a.abbuf + (size_t)(e % 3) * kTerms;
  const float* ub = a.ubuf + (size_t)(e % 3) * kTerms;
  if (bt == 0)
    *ok = (s == 0 || spin_until_geq(a.grams_done, a.grams_base + (unsigned)(s * min(a.H, a.G)))) ? 1 : 0;
  named_barrier(2, 128);
  if (!*ok) return false;
  // every load in flight at once (kk <= 8 * 128)
  float la[8], lg[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int p = bt + 128 * u;
    const int i = p / k, jj = p - i * k;
    la[u] = p < kk ? __ldcg(ab + p) : 0.f;
    lg[u] = p < kk ? (s == 0 ? __ldcg(a.G0 + p) : __ldcg(ub + kKP + i * kKP + jj)) : 0.f;
  }
  const float nsq = (s > 0 && bt < k) ? __ldcg(ub + bt) : 1.f;
  const float bq = bt < k ? __ldcg(ab + kk + bt) : 0.f;
  const float vv = (s == 0 && bt < k) ? __ldcg(a.vv0 + bt) : 1.f;
  if (bt < kKP) inv_n[bt] = bt < k ? (s == 0 ? 1.f : 1.f / sqrtf(nsq)) : 0.f;
  named_barrier(2, 128);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int p = bt + 128 * u;
    const int i = p / k, jj = p - i * k;
    if (p < kk) {
      Am[i * kKP + jj] = la[u] * inv_n[i] * inv_n[jj];
      Gm[i * kKP + jj] = s == 0 ? lg[u] : lg[u] * inv_n[i];
    }
  }
  if (bt < kKP) cb[bt] = bt < k ? fmaf(a.eps_B, vv, bq * inv_n[bt] * inv_n[bt]) : 0.f;
  named_barrier(2, 128);
  if (bt < kKP) inv_s[bt] = bt < k ? 1.f / fmaxf(Gm[bt * kKP + bt], a.rho) : 0.f;
  named_barrier(2, 128);
  for (int p = bt; p < kKP * kKP; p += 128) {
    const int jj = p / kKP, i = p % kKP;
    T[p] = (jj < i && i < k) ? cb[i] * Am[i * kKP + jj] * inv_s[jj] : 0.f;
  }
  {
    // c_i: warp w takes players 8w .. 8w + 7, the lanes run over j
    const int w = bt >> 5, lane = bt & 31;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = 8 * w + u;
      float c = (lane < i && i < k) ? Am[i * kKP + lane] * Gm[i * kKP + lane] * inv_s[lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if (lane == 0) cac[i] = i < k ? Am[i * kKP + i] - c : 0.f;
    }
  }
  named_barrier(2, 128);
  float* cf = a.cbuf + (size_t)(e & 1) * kCoef;
  for (int p = bt; p < kKP * kKP; p += 128) cf[p] = T[p];
  if (bt < kKP) {
    cf[kKP * kKP + bt] = cb[bt];
    cf[kKP * kKP + kKP + bt] = cac[bt];
    cf[kKP * kKP + 2 * kKP + bt] = inv_n[bt];
  }
  if (s == a.nsteps - 1 && a.dbg) {  // a | G | b as used (b without eps_B)
    for (int p = bt; p < kk; p += 128) {
      const int i = p / k, jj = p - i * k;
      a.dbg[p] = Am[i * kKP + jj];
      a.dbg[kk + p] = Gm[i * kKP + jj];
    }
    if (bt < k) a.dbg[2 * kk + bt] = __ldcg(ab + kk + bt) * inv_n[bt] * inv_n[bt];
  }
  __threadfence();
  named_barrier(2, 128);
  if (bt == 0) red_release_add(a.coef_ready, 1u);
  return true;
}

// 8 consecutive FP32 columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
// Waits for this thread's tensor-memory loads; the registers they fill are operands, so
// no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&a)[8], uint32_t (&b)[8], uint32_t (&c)[8],
                                               uint32_t (&d)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                 "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                 "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3]), "+r"(c[4]), "+r"(c[5]), "+r"(c[6]), "+r"(c[7]),
                 "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5]), "+r"(d[6]), "+r"(d[7])
               :
               : "memory");
}

// The update of Alg. 2 for the CTA's 256 rows of V (rows goff .. goff + 255), by warps 4-11
// (ut = tid - 128: row ut of the slice; TMEM lane ut & 127 of accumulator half ut >> 7).
// V in memory holds v'_i = n_i v_i (step s > 0: the previous step's retraction deferred; step 0:
// n_i = 1). A_t V' and B_t V' (TMEM) scaled by 1/n are the step's A_t V and B_t V; the k x k
// coefficients of Eq. (update) in matrix form, grad = A_t V diag(b) - B_t V diag(a - c) - [Bv] T
// (T_ji = b_i a_ij / s_j for j < i, c_i = sum_{j<i} a_ij G_ij / s_j, s_j = max(G_jj, rho)), come
// from cbuf (build_coefficients); then v'' = v + eta grad, [Bv]'' = [Bv] + gamma (B_t v - [Bv]).
// A non-final step writes the BF16 pairs of v'' (the next step's operand; the retraction
// deferred) and releases them, then the rows of v'' and [Bv]'' (the helpers form their Grams);
// the final step adds |v''_i|^2 and V''^T [Bv]'' into ubuf[(e + 1) % 3], normalises behind a
// grid barrier and leaves G, |v_i|^2 for the next launch. br_free is arrived on when the
// back-projection stages (the update's scratch) may be reused. False on a timeout (recorded).
__device__ __forceinline__ bool run_update(const StreamArgs& a, int s, unsigned e, int j, int64_t goff,
                                           uint32_t tmem_bp, uint8_t* BR, float* ESTG, uint64_t* bp_done,
                                           uint64_t* bp_free, uint64_t* br_free, volatile int* ok,
                                           volatile int* abort_flag, int tid, int warp, int lane) {
  const int ut = tid - 128;
  const int q = warp & 3, h = ut >> 7;
  const int k = a.k, kk = k * k;
  const bool last = s == a.nsteps - 1;
  float* vs = reinterpret_cast<float*>(BR);  // [256][36] V' rows, then v''
  float* ss = vs + 256 * kRS;                // [256][36] [Bv] rows, then [Bv]''
  float* T = ESTG;                           // [32][32] T_ji at j * 32 + i
  float* cb = T + kKP * kKP;                 // b_i (+ eps_B |v_i|^2)
  float* cac = cb + kKP;                     // a_ii - c_i
  float* inv_n = cac + kKP;                  // 1 / n_i
  float* red8 = inv_n + kKP;                 // [8][32]
  float* ubn = a.ubuf + (size_t)((e + 1) % 3) * kTerms;
  const bool tr = a.trace && ut == 0 && s >= a.nsteps - 2;
  // quarter stamps of thread 0's row work (step before the last), in row nchunk + 1 events 0..3
  // and the spare trace area after the per-CTA rows
  const bool qtr = a.trace && ut == 0 && s == a.nsteps - 2;
  auto qstamp = [&](int ev) {  // ev 0..15
    if (qtr) a.trace2[(size_t)j * 16 + ev] = globaltimer();
  };
  auto ustamp = [&](int ev) {  // ev 0..7
    if (tr) a.trace[((size_t)j * (a.nchunk + 2) + a.nchunk + (last ? 0 : 1)) * kEv + 4 + ev] = globaltimer();
  };
  // 1. the slice's accumulators are complete; its rows of V' and [Bv] into shared memory
  if (ut == 0) *ok = mbar_wait(bp_done, (uint32_t)(s & 1)) && !*abort_flag ? 1 : 0;
  named_barrier(3, 256);
  if (!*ok) return false;
  ustamp(0);
  tc_fence_after();
  if ((k & 3) == 0) {
    const float4* gv = reinterpret_cast<const float4*>(a.V + goff * k);
    const float4* gs = reinterpret_cast<const float4*>(a.S + goff * k);
    const int n4 = 64 * k;
    for (int base = 0; base < n4; base += 256 * 4) {
      float4 xv[4], xs[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int el = base + ut + 256 * u;
        if (el < n4) {
          xv[u] = __ldcg(gv + el);
          xs[u] = __ldcg(gs + el);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int el = base + ut + 256 * u;
        if (el < n4) {
          const int row = (4 * el) / k, i = 4 * el - row * k;
          *reinterpret_cast<float4*>(vs + row * kRS + i) = xv[u];
          *reinterpret_cast<float4*>(ss + row * kRS + i) = xs[u];
        }
      }
    }
  } else {
    for (int el = ut; el < 256 * k; el += 256) {
      const int row = el / k, i = el - row * k;
      vs[row * kRS + i] = __ldcg(a.V + goff * k + el);
      ss[row * kRS + i] = __ldcg(a.S + goff * k + el);
    }
  }
  for (int el = ut; el < 256 * (kKP - k); el += 256) {  // players k .. 31 of every row are zero
    const int row = el / (kKP - k), i = k + el % (kKP - k);
    vs[row * kRS + i] = 0.f;
    ss[row * kRS + i] = 0.f;
  }
  // 2. the step's coefficients (computed once, by the builder that added its last row-side item)
  if (ut == 0) *ok = spin_until_geq(a.coef_ready, e + 1) && !*abort_flag ? 1 : 0;
  named_barrier(3, 256);
  if (!*ok) return false;
  ustamp(1);
  {
    const float* cf = a.cbuf + (size_t)(e & 1) * kCoef;
    float t[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) t[u] = __ldcg(cf + ut + 256 * u);
    const float c0 = ut < kKP ? __ldcg(cf + kKP * kKP + ut) : 0.f;
    const float c1 = ut < kKP ? __ldcg(cf + kKP * kKP + kKP + ut) : 0.f;
    const float c2 = ut < kKP ? __ldcg(cf + kKP * kKP + 2 * kKP + ut) : 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) T[ut + 256 * u] = t[u];
    if (ut < kKP) {
      cb[ut] = c0;
      cac[ut] = c1;
      inv_n[ut] = c2;
    }
  }
  named_barrier(3, 256);
  ustamp(2);
  ustamp(3);
  // 3. one row per thread, players in quarters of 8 (A_t V' and B_t V' from tensor memory)
  const float eta = a.eta[s];
  {
    const int row = ut;
    const int64_t c = goff + row;
    float4* v4 = reinterpret_cast<float4*>(vs + row * kRS);
    float4* s4 = reinterpret_cast<float4*>(ss + row * kRS);
    const uint32_t ta0 = tmem_bp + (uint32_t)(64 * h) + ((uint32_t)(32 * q) << 16);
    uint32_t x[8], lo[8], y[8], ylo[8];
    tmem_ld8_nowait(ta0, x);  // quarter 0 of A_t V' (hi, lo) and B_t V' in flight during the penalty
    tmem_ld8_nowait(ta0 + 32, lo);
    tmem_ld8_nowait(ta0 + 128, y);
    tmem_ld8_nowait(ta0 + 128 + 32, ylo);
    qstamp(0);
    // penalty_i = sum_{j<i} [Bv]_j T_ji for every player (T_ji = 0 unless j < i < k): [Bv]_j from
    // shared memory, the zero triangle skipped at compile time
    float gr[kKP];
#pragma unroll
    for (int i = 0; i < kKP; ++i) gr[i] = 0.f;
#pragma unroll
    for (int jj = 0; jj < kKP - 1; ++jj) {
      const float sj = ss[row * kRS + jj];
#pragma unroll
      for (int i4 = (jj + 1) / 4; i4 < kKP / 4; ++i4) {
        const float4 t = *reinterpret_cast<const float4*>(T + jj * kKP + 4 * i4);
        gr[4 * i4] = fmaf(sj, t.x, gr[4 * i4]);
        gr[4 * i4 + 1] = fmaf(sj, t.y, gr[4 * i4 + 1]);
        gr[4 * i4 + 2] = fmaf(sj, t.z, gr[4 * i4 + 2]);
        gr[4 * i4 + 3] = fmaf(sj, t.w, gr[4 * i4 + 3]);
      }
    }
    qstamp(1);
    float chk = 0.f;
#pragma unroll
    for (int qq = 0; qq < kKP / 8; ++qq) {
      const int i0 = 8 * qq;
      if (qq > 0) {
        tmem_ld8_nowait(ta0 + i0, x);
        tmem_ld8_nowait(ta0 + 32 + i0, lo);
        tmem_ld8_nowait(ta0 + 128 + i0, y);
        tmem_ld8_nowait(ta0 + 128 + 32 + i0, ylo);
      }
      const float4 va = v4[2 * qq], vb = v4[2 * qq + 1];
      const float4 sa = s4[2 * qq], sb = s4[2 * qq + 1];
      const float vq[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
      const float sq[8] = {sa.x, sa.y, sa.z, sa.w, sb.x, sb.y, sb.z, sb.w};
      tmem_wait_ld32(x, lo, y, ylo);
      float vn[8], sn[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + u;
        const float v = vq[u] * inv_n[i];
        const float av = (__uint_as_float(x[u]) + __uint_as_float(lo[u])) * a.inv_nA * inv_n[i];
        const float bvr = (__uint_as_float(y[u]) + __uint_as_float(ylo[u])) * a.inv_nB * inv_n[i];
        const float bv = fmaf(a.eps_B, v, bvr);
        const float g = cb[i] * av - gr[i] - cac[i] * bv;
        vn[u] = i < k ? fmaf(eta, g, v) : 0.f;
        sn[u] = i < k ? fmaf(a.gamma, bv - sq[u], sq[u]) : 0.f;
        chk += vn[u] + sn[u];
        if (last && i < k && a.AV) {  // debug readback: update direction, A_t V, B_t V
          a.grad_out[c * k + i] = g;
          a.AV[c * k + i] = av;
          a.BV[c * k + i] = bvr;
        }
      }
      v4[2 * qq] = make_float4(vn[0], vn[1], vn[2], vn[3]);
      v4[2 * qq + 1] = make_float4(vn[4], vn[5], vn[6], vn[7]);
      s4[2 * qq] = make_float4(sn[0], sn[1], sn[2], sn[3]);
      s4[2 * qq + 1] = make_float4(sn[4], sn[5], sn[6], sn[7]);
      qstamp(2 + qq);
    }
    if (!isfinite(chk)) atomicOr(a.dflag, kFlagNonFinite);
  }
  tc_fence_before();
  named_barrier(3, 256);
  if (ut == 0) mbar_arrive(bp_free);  // the accumulators may be overwritten by the next step
  ustamp(4);
  // BF16 (hi, lo) pairs of rows of vs, transposed into the V^T operand: item (operand row n,
  // 8 consecutive rows); the lanes of a warp take 32 consecutive n (conflict-free reads)
  auto write_operand = [&]() {
    for (int el = ut; el < 2 * kKP * 32; el += 256) {
      const int n = el & 63, r0 = (el >> 6) * 8, pl = n & 31;
      float v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = vs[(r0 + m) * kRS + pl];
      uint4 w;
      if (n < kKP) {
        w = make_uint4(pack2_bf16(v[0], v[1]), pack2_bf16(v[2], v[3]), pack2_bf16(v[4], v[5]), pack2_bf16(v[6], v[7]));
      } else {
        w = make_uint4(pack2_lo_bf16(v[0], v[1]), pack2_lo_bf16(v[2], v[3]), pack2_lo_bf16(v[4], v[5]),
                       pack2_lo_bf16(v[6], v[7]));
      }
      *reinterpret_cast<uint4*>(a.Vt + (int64_t)n * a.d + goff + r0) = w;
    }
  };
  // |v''_i|^2 and V''^T [Bv]'' of the slice into the next slot (atomics)
  auto add_grams = [&]() {
    {
      const int i = ut & 31, g = ut >> 5;
      float s2 = 0.f;
#pragma unroll 8
      for (int row = 32 * g; row < 32 * g + 32; ++row) s2 = fmaf(vs[row * kRS + i], vs[row * kRS + i], s2);
      red8[g * kKP + i] = s2;
    }
    {
      // 4 x 4 block (players i0.., l0..) of U over a quarter of the rows (rows = rq mod 4);
      // warp = i block, lane = (row quarter, l block); the quarters are added by shuffles
      const int i0 = 4 * (warp - 4), l0 = 4 * (lane & 7), rq = lane >> 3;
      float u[4][4] = {};
#pragma unroll 4
      for (int it = 0; it < 64; ++it) {
        const int row = 4 * it + rq;  // interleaved: the four quarters' rows fall in different banks
        const float4 v = *reinterpret_cast<const float4*>(vs + row * kRS + i0);
        const float4 t = *reinterpret_cast<const float4*>(ss + row * kRS + l0);
        const float vv4[4] = {v.x, v.y, v.z, v.w}, tt[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int r2 = 0; r2 < 4; ++r2) u[p][r2] = fmaf(vv4[p], tt[r2], u[p][r2]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) {
          u[p][r2] += __shfl_xor_sync(0xffffffffu, u[p][r2], 8);
          u[p][r2] += __shfl_xor_sync(0xffffffffu, u[p][r2], 16);
        }
      if (rq == 0) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int r2 = 0; r2 < 4; ++r2)
            if (i0 + p < k && l0 + r2 < k) atomicAdd(ubn + kKP + (i0 + p) * kKP + l0 + r2, u[p][r2]);
      }
    }
    named_barrier(3, 256);
    if (ut < k) {
      float s2 = 0.f;
#pragma unroll
      for (int g = 0; g < 8; ++g) s2 += red8[g * kKP + ut];
      atomicAdd(ubn + ut, s2);
    }
  };
  auto write_rows = [&]() {  // rows of V (v'' or v''/n) and [Bv]''
    if ((k & 3) == 0) {
      const int k4 = k / 4;
      float4* gv = reinterpret_cast<float4*>(a.V + goff * k);
      float4* gs = reinterpret_cast<float4*>(a.S + goff * k);
      for (int el = ut; el < 256 * k4; el += 256) {
        const int row = el / k4, i = 4 * (el - row * k4);
        gv[el] = *reinterpret_cast<const float4*>(vs + row * kRS + i);
        gs[el] = *reinterpret_cast<const float4*>(ss + row * kRS + i);
      }
    } else {
      for (int el = ut; el < 256 * k; el += 256) {
        const int row = el / k, i = el - row * k;
        a.V[goff * k + el] = vs[row * kRS + i];
        a.S[goff * k + el] = ss[row * kRS + i];
      }
    }
  };
  auto clear_slots = [&]() {  // CTA 0: slots read by the previous step in every CTA, for step e + 2
    if (j == 0) {
      float* ab2 = a.abbuf + (size_t)((e + 2) % 3) * kTerms;
      float* ub2 = a.ubuf + (size_t)((e + 2) % 3) * kTerms;
      for (int p = ut; p < kTerms; p += 256) {
        ab2[p] = 0.f;
        ub2[p] = 0.f;
      }
    }
  };
  if (!last) {
    // 4. the next step's operand first (what its projections wait for), released; then the
    //    rows of V'' and [Bv]'' (the helpers read them for the Grams of the next update)
    write_operand();
    fence_proxy_async_global();  // the operand is read by TMA (async proxy) in other CTAs
    __threadfence();
    named_barrier(3, 256);
    if (ut == 0) red_release_add(a.upd_done + j, 1u);
    ustamp(5);
    write_rows();
    clear_slots();
    __threadfence();
    named_barrier(3, 256);
    if (ut == 0) {
      red_release_add(a.rows_done + j, 1u);
      mbar_arrive(br_free);
    }
    ustamp(7);
    return true;
  }
  // final step: every CTA's |v''|^2 and U, a grid barrier, then the normalised players
  add_grams();
  __threadfence();
  named_barrier(3, 256);
  ustamp(5);
  if (ut == 0) {
    atomicAdd(a.bar, 1u);
    *ok = spin_until_geq(a.bar, a.bar_target) ? 1 : 0;
  }
  named_barrier(3, 256);
  if (!*ok) return false;
  ustamp(6);
  if (ut < kKP) inv_n[ut] = ut < k ? 1.f / sqrtf(__ldcg(ubn + ut)) : 0.f;
  named_barrier(3, 256);
  for (int el = ut; el < 256 * kKP; el += 256) {
    const int row = el / kKP, i = el % kKP;
    vs[row * kRS + i] *= inv_n[i];
  }
  if (j == 0) {  // G_il = U_il / n_i and |v_i|^2 of the normalised players for the next launch
    for (int p = ut; p < kk; p += 256) {
      const int i = p / k, l = p - i * k;
      a.Gn[p] = __ldcg(ubn + kKP + i * kKP + l) * inv_n[i];
    }
    if (ut < k) a.vvn[ut] = __ldcg(ubn + ut) * inv_n[ut] * inv_n[ut];
  }
  named_barrier(3, 256);
  write_operand();
  write_rows();
  clear_slots();
  fence_proxy_async_global();
  __threadfence();
  named_barrier(3, 256);
  if (ut == 0) {
    red_release_add(a.upd_done + j, 1u);
    red_release_add(a.rows_done + j, 1u);
    mbar_arrive(br_free);
  }
  ustamp(7);
  return true;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_stream(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
                const __grid_constant__ CUtensorMap mapX64, const __grid_constant__ CUtensorMap mapY64,
                const __grid_constant__ CUtensorMap mapVt, const __grid_constant__ CUtensorMap mapPt,
                const __grid_constant__ CUtensorMap mapQt, const __grid_constant__ StreamArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  uint8_t* VT = base;
  uint8_t* PR = VT + kVtB;
  uint8_t* BR = PR + kPS * kPBox;
  float* ESTG = reinterpret_cast<float*>(BR + kBS * kBStage);  // [128][32] (streaming CTAs)
  float* Ps = reinterpret_cast<float*>(VT);                    // [kStgRows][32] (helper CTAs)
  float* Qs = Ps + kStgRows * 32;                              // [kStgRows][32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(ESTG + 128 * 32);
  uint64_t* p_full = bars;                 // [kPS]
  uint64_t* p_empty = p_full + kPS;        // [kPS]
  uint64_t* acc_full = p_empty + kPS;      // [kAcc]
  uint64_t* acc_empty = acc_full + kAcc;   // [kAcc]
  uint64_t* b_full = acc_empty + kAcc;     // [kBS]
  uint64_t* b_empty = b_full + kBS;        // [kBS]
  uint64_t* vt_full = b_empty + kBS;       // the step's V^T slice has landed
  uint64_t* vt_free = vt_full + 1;         // the step's projection MMAs are complete
  uint64_t* bp_done = vt_free + 1;         // the step's back-projection MMAs are complete
  uint64_t* bp_free = bp_done + 1;         // the update has read the accumulators
  uint64_t* br_free = bp_free + 1;         // the update is done with its scratch (the back-projection stages)
  uint64_t* mma_fin = br_free + 1;         // [2]
  uint64_t* stg_full = mma_fin + 2;        // [4] staged tile of chunk g ready for reducer g % 4
  uint64_t* stg_empty = stg_full + 4;      // the reduction of the staged tile has read it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* bp_loaded = abort_flag + 1;  // chunks whose back-projection rows have landed (all steps)
  volatile int* epi_ok = abort_flag + 2;
  volatile int* bld_ok = abort_flag + 3;
  volatile int* upd_ok = abort_flag + 4;
  volatile int* bld_last = abort_flag + 6;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = a.G, j = (int)blockIdx.x;
  const bool helper = j >= G;
  const int H = (int)gridDim.x - G;
  const int splits = a.splits;
  const int nsteps = a.nsteps;
  // projection tile of this CTA (the same in every chunk)
  const int p_split = j % splits;
  const int p_view = (j / splits) & 1;
  const int p_rtl = j / (2 * splits);
  constexpr int kRT = kR / 128;  // row tiles per chunk
  const int64_t p_col0 = (int64_t)p_split * (2 * kR);
  // back-projection slice of this CTA: rows goff .. goff + 255 of V
  const int nslice = G / 2;
  const int b_view = j >= nslice ? 1 : 0;
  const int64_t b_c0 = (int64_t)(j - b_view * nslice) * 256;
  const int64_t b_goff = (b_view ? a.d_x : 0) + b_c0;
  const int nchunk = a.nchunk;
  const int nrt = nchunk * kRT;
  const int lastS = nsteps - 1;

  if (warp == 1 && !helper) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < kNumBars; ++i) mbar_init(bars + i, 1);
    *abort_flag = 0;
    *bp_loaded = 0;
    fence_mbar_init();
    prefetch_tensormap(p_view ? &mapY : &mapX);
    prefetch_tensormap(b_view ? &mapY64 : &mapX64);
    prefetch_tensormap(&mapVt);
    prefetch_tensormap(&mapPt);
    prefetch_tensormap(&mapQt);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tmem_bp = tmem;          // 256 columns: A_t V (h0, h1), B_t V (h0, h1)
  const uint32_t tmem_p = tmem + 256;     // kAcc x 64 columns: projection tiles
  auto stamp = [&](int ev) {
    if (a.trace) a.trace[((size_t)j * (nchunk + 2) + nchunk) * kEv + ev] = globaltimer();
  };
  auto cstamp = [&](int s, int c, int ev) {
    if (a.trace && s == lastS) a.trace[((size_t)j * (nchunk + 2) + c) * kEv + ev] = globaltimer();
  };
  auto fail = [&]() {
    atomicOr(a.dflag, kFlagTimeout);
    *abort_flag = 1;
  };
  if (tid == 0) stamp(0);

  if (helper) {
    if (warp < 8 && j - G < G) {  // helpers that own at least one slice (the others never release)
      // ---- Grams of the next update: |v_i|^2 and U = V^T [Bv] over the rows the streaming
      //      CTAs' updates just wrote (step s reads the players of step s, still unnormalised),
      //      slices hid, hid + H, ... accumulated in registers, then added into ubuf[e % 3] ----
      const int gt = tid;  // 0..255
      const int k = a.k;
      const int hid = j - G;
      float* vs = reinterpret_cast<float*>(BR);  // [256][kRS]
      float* ss = vs + 256 * kRS;
      float* red8 = ESTG;                        // [8][32]
      volatile int* g_ok = abort_flag + 5;
      const int i0 = 4 * warp, l0 = 4 * (lane & 7), rq = lane >> 3;
      auto hstamp = [&](int s, int ev) {  // the last step's Gram phase of this helper
        if (a.trace2 && gt == 0 && s == nsteps - 1) a.trace2[(size_t)j * 16 + ev] = globaltimer();
      };
      for (int s = 1; s < nsteps; ++s) {
        const unsigned e = a.e0 + (unsigned)s;
        float u[4][4] = {};
        float s2 = 0.f;
        bool alive = true;
        hstamp(s, 0);
        for (int sl = hid; sl < G; sl += H) {
          if (gt == 0) *g_ok = !*abort_flag && spin_until_geq(a.rows_done + sl, e) ? 1 : 0;
          named_barrier(4, 256);
          if (!*g_ok) {
            if (gt == 0) fail();
            alive = false;
            break;
          }
          if (sl == hid) hstamp(s, 1);
          const int64_t goff = (int64_t)sl * 256;
          if ((k & 3) == 0) {  // all of the slice's float4 loads in flight (8 of V and 8 of S per thread at k = 32)
            const float4* gv = reinterpret_cast<const float4*>(a.V + goff * k);
            const float4* gs = reinterpret_cast<const float4*>(a.S + goff * k);
            const int n4 = 64 * k, k4 = k / 4;
            for (int base = 0; base < n4; base += 256 * 8) {
              float4 xv[8], xs[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int el = base + gt + 256 * u;
                if (el < n4) {
                  xv[u] = __ldcg(gv + el);
                  xs[u] = __ldcg(gs + el);
                }
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int el = base + gt + 256 * u;
                if (el < n4) {
                  const int row = el / k4, i = 4 * (el - row * k4);
                  *reinterpret_cast<float4*>(vs + row * kRS + i) = xv[u];
                  *reinterpret_cast<float4*>(ss + row * kRS + i) = xs[u];
                }
              }
            }
          } else {
            for (int el = gt; el < 256 * k; el += 256) {
              const int row = el / k, i = el - row * k;
              vs[row * kRS + i] = __ldcg(a.V + goff * k + el);
              ss[row * kRS + i] = __ldcg(a.S + goff * k + el);
            }
          }
          for (int el = gt; el < 256 * (kKP - k); el += 256) {
            const int row = el / (kKP - k), i = k + el % (kKP - k);
            vs[row * kRS + i] = 0.f;
            ss[row * kRS + i] = 0.f;
          }
          named_barrier(4, 256);
          {
            const int i = gt & 31, g = gt >> 5;
#pragma unroll 8
            for (int row = 32 * g; row < 32 * g + 32; ++row) s2 = fmaf(vs[row * kRS + i], vs[row * kRS + i], s2);
          }
#pragma unroll 4
          for (int it = 0; it < 64; ++it) {
            const int row = 4 * it + rq;
            const float4 v = *reinterpret_cast<const float4*>(vs + row * kRS + i0);
            const float4 t = *reinterpret_cast<const float4*>(ss + row * kRS + l0);
            const float vv4[4] = {v.x, v.y, v.z, v.w}, tt[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int r2 = 0; r2 < 4; ++r2) u[p][r2] = fmaf(vv4[p], tt[r2], u[p][r2]);
          }
          named_barrier(4, 256);  // the next slice overwrites the rows
        }
        if (!alive) break;
        float* ub = a.ubuf + (size_t)(e % 3) * kTerms;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int r2 = 0; r2 < 4; ++r2) {
            u[p][r2] += __shfl_xor_sync(0xffffffffu, u[p][r2], 8);
            u[p][r2] += __shfl_xor_sync(0xffffffffu, u[p][r2], 16);
          }
        if (rq == 0) {
#pragma unroll
          for (int p = 0; p < 4; ++p)
            if (i0 + p < k)
              atomicAdd(reinterpret_cast<float4*>(ub + kKP + (i0 + p) * kKP + l0),
                        make_float4(u[p][0], u[p][1], u[p][2], u[p][3]));
        }
        red8[(gt >> 5) * kKP + (gt & 31)] = s2;
        named_barrier(4, 256);
        if (gt < k) {
          float t2 = 0.f;
#pragma unroll
          for (int g = 0; g < 8; ++g) t2 += red8[g * kKP + gt];
          atomicAdd(ub + gt, t2);
        }
        __threadfence();
        named_barrier(4, 256);
        if (gt == 0) red_release_add(a.grams_done, 1u);
        hstamp(s, 2);
      }
    } else if (warp >= 8) {
      // ---- builders: summed rows -> BF16 hi/lo operand, then the row-side terms ----
      const int bt = tid - 256;
      const int k = a.k;
      constexpr int kU = kStgRows * 8 / 128;    // float4 of P (and of Q) per thread per pass
      // rows [r0, r0 + kStgRows) of P and Q into shared memory
      auto stage = [&](int64_t r0) {
        const float4* gp = reinterpret_cast<const float4*>(a.P + r0 * 32);
        const float4* gq = reinterpret_cast<const float4*>(a.Q + r0 * 32);
        float4 vp[kU], vq[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          vp[u] = __ldcg(gp + bt + 128 * u);
          vq[u] = __ldcg(gq + bt + 128 * u);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          reinterpret_cast<float4*>(Ps)[bt + 128 * u] = vp[u];
          reinterpret_cast<float4*>(Qs)[bt + 128 * u] = vq[u];
        }
      };
      bool alive = true;
      for (int s = 0; s < nsteps && alive; ++s) {
        const unsigned e = a.e0 + (unsigned)s;
        float* ta = a.abbuf + (size_t)(e % 3) * kTerms;  // a (k x k) | b (k) of this step
        float* tb = ta + k * k;
        for (int item = 0; item < 2 * nrt; ++item) {  // item = (row tile, 64-row half)
          if (item % H != j - G) continue;
          const int rt = item >> 1;
          const int64_t r0 = (int64_t)item * kStgRows;
          if (bt == 0) {
            bool ok = !*abort_flag && spin_until_geq(a.cnt + rt, (e + 1) * (unsigned)(2 * splits));
            *bld_ok = ok ? 1 : 0;
          }
          named_barrier(2, 128);
          if (bt == 0 && (item & 1) == 0) cstamp(s, rt / kRT, kEvBuildStart);
          if (!*bld_ok) {
            if (bt == 0) fail();
            alive = false;
            break;
          }
          // the operand Pt[n][r] (n < 32: hi, n >= 32: lo of P[r][n mod 32]) of the half, released
          stage(r0);
          named_barrier(2, 128);
          {
            const int n = bt >> 1, rr = (bt & 1) * (kStgRows / 2), pl = n & 31;
            const bool lo = n >= 32;
#pragma unroll
            for (int which = 0; which < 2; ++which) {
              const float* src = which ? Qs : Ps;
              __nv_bfloat16* dst = (which ? a.Qt : a.Pt) + (int64_t)n * a.ldt + r0 + rr;
#pragma unroll
              for (int u = 0; u < kStgRows / 16; ++u) {
                uint32_t w[4];
#pragma unroll
                for (int el = 0; el < 4; ++el) {
                  const float v0 = src[(rr + 8 * u + 2 * el) * 32 + pl];
                  const float v1 = src[(rr + 8 * u + 2 * el + 1) * 32 + pl];
                  w[el] = lo ? pack2_lo_bf16(v0, v1) : pack2_bf16(v0, v1);
                }
                *reinterpret_cast<uint4*>(dst + 8 * u) = make_uint4(w[0], w[1], w[2], w[3]);
              }
            }
          }
          fence_proxy_async_global();  // the operand is read by TMA (async proxy) in other CTAs
          __threadfence();
          named_barrier(2, 128);
          if (bt == 0) {
            red_release_add(a.wready + item, 1u);
            if ((item & 1) == 0) cstamp(s, rt / kRT, kEvBuilt);
          }
          // off the back-projection's path: a_ij = sum_A (P_i Q_j + Q_i P_j) / n_A or
          // b_i = sum_B (P_i^2 + Q_i^2) / n_B over the half's rows (still staged); rows cleared
          // for the next step
          {
            float4* gp = reinterpret_cast<float4*>(a.P + r0 * 32);
            float4* gq = reinterpret_cast<float4*>(a.Q + r0 * 32);
#pragma unroll
            for (int u = 0; u < kU; ++u) {
              gp[bt + 128 * u] = make_float4(0.f, 0.f, 0.f, 0.f);
              gq[bt + 128 * u] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
          }
          if (r0 < a.nA) {
            const int i0 = (bt >> 4) * 4, j0 = (bt & 15) * 2;
            float acc[4][2] = {};
#pragma unroll 4
            for (int rr = 0; rr < kStgRows; ++rr) {
              const float4 pi = *reinterpret_cast<const float4*>(Ps + rr * 32 + i0);
              const float4 qi = *reinterpret_cast<const float4*>(Qs + rr * 32 + i0);
              const float2 pj = *reinterpret_cast<const float2*>(Ps + rr * 32 + j0);
              const float2 qj = *reinterpret_cast<const float2*>(Qs + rr * 32 + j0);
              const float pv[4] = {pi.x, pi.y, pi.z, pi.w}, qv[4] = {qi.x, qi.y, qi.z, qi.w};
#pragma unroll
              for (int p = 0; p < 4; ++p) {
                acc[p][0] = fmaf(pv[p], qj.x, fmaf(qv[p], pj.x, acc[p][0]));
                acc[p][1] = fmaf(pv[p], qj.y, fmaf(qv[p], pj.y, acc[p][1]));
              }
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int el = 0; el < 2; ++el)
                if (i0 + p < k && j0 + el < k) atomicAdd(ta + (i0 + p) * k + j0 + el, acc[p][el] * a.inv_nA);
          } else {
            const int i = bt & 31, g = bt >> 5;
            float s2 = 0.f;
            for (int rr = g * (kStgRows / 4); rr < (g + 1) * (kStgRows / 4); ++rr) {
              const float p = Ps[rr * 32 + i], qv = Qs[rr * 32 + i];
              s2 = fmaf(p, p, fmaf(qv, qv, s2));
            }
            if (i < k) atomicAdd(tb + i, s2 * a.inv_nB);
          }
          __threadfence();
          named_barrier(2, 128);  // staging is reused by the next item
          if (bt == 0) {
            // the builder whose item completes the step's count computes the coefficients
            const unsigned before = atom_add_acq_rel(a.terms_done, 1u);
            *bld_last = before + 1 == (e + 1) * (unsigned)(2 * nrt) ? 1 : 0;
            if ((item & 1) == 0) cstamp(s, rt / kRT, kEvTerms);
          }
          named_barrier(2, 128);
          if (*bld_last && !build_coefficients(a, s, e, bt, reinterpret_cast<float*>(VT) + 2 * kStgRows * 32,
                                               bld_ok)) {
            if (bt == 0) fail();
            alive = false;
            break;
          }
        }
      }
    }
  } else if (warp == 0) {
    // ---- projection loads: the row tiles of every step from HBM ------------------
    if (lane == 0) {
      const CUtensorMap* mZ = p_view ? &mapY : &mapX;
      const int nks = 2 * kR / 64;
      int i = 0;
      bool ok = true;
      for (int s = 0; ok && s < nsteps; ++s) {
        for (int c = 0; c < nchunk; ++c) {
          const int gc = s * nchunk + c;
          if (*abort_flag) {
            ok = false;
            break;
          }
          if (gc >= a.lag && !wait_shared_geq(bp_loaded, gc - a.lag + 1)) {
            fail();
            ok = false;
            break;
          }
          const int row0 = (int)((int64_t)s * a.b) + (c * kRT + p_rtl) * 128;
          cstamp(s, c, kEvIssue);
          if (s > 0 && c == 0 && a.pf_next == 0) {
            // the step's first two tiles into L2 while the previous step's update runs (the
            // stages hold only half a tile, and HBM is idle during the update)
            for (int cc = 0; cc < 2 && cc < nchunk; ++cc)
              for (int ks = 0; ks < nks; ++ks)
                tma_prefetch_2d(mZ, (int)(p_col0 + 64 * ks), (int)((int64_t)s * a.b) + (cc * kRT + p_rtl) * 128);
          }
          for (int ks = 0; ks < nks; ++ks, ++i) {
            const int st = i % kPS;
            if (i >= kPS && !mbar_wait(p_empty + st, ((i / kPS) - 1) & 1)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(p_full + st, kPBox);
            tma_load_2d(PR + st * kPBox, mZ, (int)(p_col0 + 64 * ks), row0, p_full + st);
          }
          if (!ok) {
            fail();
            break;
          }
        }
      }
      // every issued copy lands before the CTA may exit
      for (int q = i > kPS ? i - kPS : 0; q < i; ++q) mbar_wait(p_full + (q % kPS), (q / kPS) & 1, 100000000ull);
    }
  } else if (warp == 1) {
    // ---- V^T slice of every step, projection MMAs: D[128 rows x 64] += X box . V^T box^T ----
    if (lane == 0) {
      const int voff = (int)((p_view ? a.d_x : 0) + p_col0);
      // the two CTAs whose update writes these V^T columns
      const int src0 = voff / 256, src1 = src0 + 1;
      const uint32_t idesc = idesc_bf16(128, 64, 0, 0);
      const int nks = 2 * kR / 64;
      bool ok = true;
      bool vt_pending = false;  // a V^T load was issued and has not been waited for
      int i = 0;
      for (int s = 0; ok && s < nsteps; ++s) {
        const unsigned e = a.e0 + (unsigned)s;
        if (s > 0) {
          // the previous step's MMAs have read the slice; its sources have written the new one
          mma_commit(vt_free);
          ok = mbar_wait(vt_free, (uint32_t)((s - 1) & 1)) && !*abort_flag &&
               spin_until_geq(a.upd_done + src0, e) && spin_until_geq(a.upd_done + src1, e) &&
               (!a.serial || spin_until_geq(a.upd_done + j, e));
          if (!ok) break;
          fence_proxy_async_global();
        }
        mbar_arrive_expect_tx(vt_full, kVtB);
        for (int jb = 0; jb < kVtBoxes; ++jb) tma_load_2d(VT + jb * 8192, &mapVt, voff + 64 * jb, 0, vt_full);
        vt_pending = true;
        if (!mbar_wait(vt_full, (uint32_t)(s & 1))) {
          ok = false;
          break;
        }
        vt_pending = false;
        for (int c = 0; ok && c < nchunk; ++c) {
          const int gc = s * nchunk + c;
          const int buf = gc % kAcc;
          if (gc >= kAcc && !mbar_wait(acc_empty + buf, ((gc / kAcc) - 1) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (int ks = 0; ks < nks; ++ks, ++i) {
            const int st = i % kPS;
            if (!mbar_wait(p_full + st, (i / kPS) & 1)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint8_t* sa = PR + st * kPBox;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(tmem_p + 64 * buf, desc_sw128(sa + kk * 32, 16, 1024),
                       desc_sw128(VT + ks * 8192 + kk * 32, 16, 1024), idesc, (ks | kk) ? 1u : 0u);
            mma_commit(p_empty + st);
          }
          if (!ok) break;
          mma_commit(acc_full + buf);
          cstamp(s, c, kEvMma);
        }
      }
      if (!ok) fail();
      if (vt_pending) mbar_wait(vt_full, (uint32_t)((nsteps - 1) & 1), 100000000ull);
      mma_commit(mma_fin);  // every MMA of this thread completes before the teardown
      mbar_wait(mma_fin, 0, 100000000ull);
    }
  } else if (warp == 2) {
    // ---- back-projection loads: 64-row steps of the slice, from L2 -----------
    if (lane == 0) {
      const CUtensorMap* mZ = b_view ? &mapY64 : &mapX64;
      // A rows use the other view's projection, B rows this view's
      const CUtensorMap* mWA = b_view ? &mapPt : &mapQt;
      const CUtensorMap* mWB = b_view ? &mapQt : &mapPt;
      const uint64_t once = policy_evict_first();
      // the next step's projection tile of chunk cc, into L2 once this step's back-projection
      // has moved past chunk nchunk - pf_next + cc (the L2 footprint stays at the re-read window)
      const CUtensorMap* mP = p_view ? &mapY : &mapX;
      const int pf0 = nchunk - a.pf_next + 1;
      auto prefetch_next = [&](int s, int c) {
        const int cc = c - pf0;
        if (a.pf_next <= 0 || s + 1 >= nsteps || cc < 0 || cc >= nchunk || cc >= a.pf_next) return;
        const int row = (int)((int64_t)(s + 1) * a.b) + (cc * kRT + p_rtl) * 128;
        for (int ks = 0; ks < 2 * kR / 64; ++ks) tma_prefetch_2d(mP, (int)(p_col0 + 64 * ks), row);
      };
      int i = 0;
      bool ok = true;
      for (int s = 0; ok && s < nsteps; ++s) {
        const unsigned e = a.e0 + (unsigned)s;
        // the previous step's update is done with the stages (its scratch)
        if (s > 0 && !mbar_wait(br_free, (uint32_t)((s - 1) & 1))) {
          ok = false;
          break;
        }
        for (int c = 0; ok && c < nchunk && !*abort_flag; ++c) {
          prefetch_next(s, c);
          for (int h = 0; h < kR / 64; ++h, ++i) {
            const int r0 = c * kR + 64 * h;  // row of the step
            if (!spin_until_geq(a.wready + (r0 >> 6), e + 1)) {
              ok = false;
              break;
            }
            fence_proxy_async_global();
            if (h == 0) cstamp(s, c, kEvWSeen);
            const int st = i % kBS;
            if (i >= kBS && !mbar_wait(b_empty + st, ((i / kBS) - 1) & 1)) {
              ok = false;
              break;
            }
            uint8_t* sa = BR + st * kBStage;
            mbar_arrive_expect_tx(b_full + st, kBStage);
            const int rg = (int)((int64_t)s * a.b) + r0;
            if (a.bp_groups)  // the four 64-column boxes in one copy (3-D view of the rows)
              tma_load_3d_hint(sa, mZ, 0, rg, (int)(b_c0 / 64), b_full + st, once);
            else
#pragma unroll
              for (int jb = 0; jb < 4; ++jb)
                tma_load_2d_hint(sa + jb * 8192, mZ, (int)(b_c0 + 64 * jb), rg, b_full + st, once);
            tma_load_2d(sa + 32768, r0 < a.nA ? mWA : mWB, r0, 0, b_full + st);
          }
        }
        if (ok) prefetch_next(s, nchunk);
      }
      if (!ok) fail();
      for (int q = i > kBS ? i - kBS : 0; q < i; ++q) mbar_wait(b_full + (q % kBS), (q / kBS) & 1, 100000000ull);
    }
  } else if (warp == 3) {
    // ---- back-projection MMAs: acc[128 cols x 64] += X step^T . W ------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, 64, 1, 0);
      bool ok = true;
      int i = 0;
      for (int s = 0; ok && s < nsteps; ++s) {
        // the previous step's update has read the accumulators
        if (s > 0 && !mbar_wait(bp_free, (uint32_t)((s - 1) & 1))) {
          ok = false;
          break;
        }
        tc_fence_after();
        bool usedA = false, usedB = false;
        for (int c = 0; ok && c < nchunk; ++c) {
          for (int hh = 0; hh < kR / 64; ++hh, ++i) {
            const int r0 = c * kR + 64 * hh;
            const int st = i % kBS;
            if (!mbar_wait(b_full + st, (i / kBS) & 1)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint8_t* sa = BR + st * kBStage;
            const bool rowA = r0 < a.nA;
            const uint32_t dbase = tmem_bp + (rowA ? 0u : 128u);
            const bool used = rowA ? usedA : usedB;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_bf16(dbase + 64 * h, desc_sw128(sa + 2 * h * 8192 + kk * 2048, 8192, 1024),
                         desc_sw128(sa + 32768 + kk * 32, 16, 1024), idesc, (used || kk) ? 1u : 0u);
            if (rowA) usedA = true;
            else usedB = true;
            mma_commit(b_empty + st);
          }
          if (ok) {
            *bp_loaded = s * nchunk + c + 1;
            cstamp(s, c, kEvBpDone);
          }
        }
        if (ok) mma_commit(bp_done);
      }
      if (!ok) {
        fail();
        mbar_arrive(bp_done);
      }
      mma_commit(mma_fin + 1);
      mbar_wait(mma_fin + 1, 0, 100000000ull);
    }
  } else {
    // ---- warps 4-7: projection epilogue; warps 8-11: reducers; then the update ----
    const bool epi = warp < 8;
    const int etid = tid - 128;  // 0..127 (epilogue)
    const int q = warp & 3;
    const int r = 32 * q + lane;
    float* dstv = p_view ? a.Q : a.P;
    bool alive = true;
    for (int s = 0; alive && s < nsteps; ++s) {
      const unsigned e = a.e0 + (unsigned)s;
      if (epi) {
        // partial rows of each chunk into the staging tile for its reducer
        for (int c = 0; c < nchunk; ++c) {
          const int gc = s * nchunk + c;
          const int buf = gc % kAcc;
          if (etid == 0) {
            *epi_ok = mbar_wait(acc_full + buf, (gc / kAcc) & 1) && !*abort_flag ? 1 : 0;
            if (c == nchunk - 1) {  // the update reads these rows when the step's products are in
              bulk_prefetch_l2(a.V + b_goff * a.k, (uint32_t)(256 * a.k * 4));
              bulk_prefetch_l2(a.S + b_goff * a.k, (uint32_t)(256 * a.k * 4));
            }
          }
          named_barrier(1, 128);
          if (!*epi_ok) {
            if (etid == 0) fail();
            alive = false;
            break;
          }
          tc_fence_after();
          float hi[32], lo[32];
          tmem_ld32(tmem_p + 64 * buf + ((uint32_t)(32 * q) << 16), hi);
          tmem_ld32(tmem_p + 64 * buf + 32 + ((uint32_t)(32 * q) << 16), lo);
          tc_fence_before();
          // the reduction of the previous chunk has read the staging tile
          if (etid == 0) *epi_ok = (gc == 0 || mbar_wait(stg_empty, (gc - 1) & 1)) && !*abort_flag ? 1 : 0;
          named_barrier(1, 128);
          if (!*epi_ok) {
            if (etid == 0) fail();
            alive = false;
            break;
          }
          float4* srow = reinterpret_cast<float4*>(ESTG + r * 32);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            srow[i] = make_float4(hi[4 * i] + lo[4 * i], hi[4 * i + 1] + lo[4 * i + 1], hi[4 * i + 2] + lo[4 * i + 2],
                                  hi[4 * i + 3] + lo[4 * i + 3]);
          fence_proxy_async_smem();  // the tile is read by the bulk reduction (async proxy)
          named_barrier(1, 128);
          if (etid == 0) {
            mbar_arrive(acc_empty + buf);
            mbar_arrive(stg_full + (gc & 3));
          }
        }
      } else if (lane == 0) {
        // staged projection tile -> P or Q (bulk add at L2), then release the row tile
        const int w = warp - 8;
        for (int c = 0; c < nchunk; ++c) {
          const int gc = s * nchunk + c;
          if ((gc & 3) != w) continue;
          if (!mbar_wait(stg_full + w, (uint32_t)((gc >> 2) & 1)) || *abort_flag) {
            fail();
            alive = false;
            break;
          }
          const int rt = c * kRT + p_rtl;
          bulk_reduce_add_f32(dstv + (int64_t)rt * 128 * 32, ESTG, kEStg);
          bulk_commit();
          bulk_wait_read<0>();
          mbar_arrive(stg_empty);
          bulk_wait<0>();
          fence_proxy_async_global();
          __threadfence();
          red_release_add(a.cnt + rt, 1u);
          cstamp(s, c, kEvRelease);
        }
      }
      // every warp of the group learns whether another one gave up
      named_barrier(3, 256);
      if (*abort_flag) alive = false;
      named_barrier(3, 256);
      if (!alive) break;
      if (s == lastS && tid == 128) stamp(1);
      if (!run_update(a, s, e, j, b_goff, tmem_bp, BR, ESTG, bp_done, bp_free, br_free, upd_ok, abort_flag, tid,
                      warp, lane)) {
        if (tid == 128) fail();
        alive = false;
      }
    }
    if (tid == 128) stamp(2);
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0) stamp(3);
  if (warp == 1 && !helper) tmem_dealloc(tmem, 512);
}

}  // namespace

// The streamed kernel takes CCA with d_x == d_y, d_x a multiple of 2 kR (one column split
// per (view, CTA) pair), one resident CTA per 256 columns, minibatches of whole chunks and
// Alg. 2's plain step (Adam and Alg. 3 take the two-pass products).
bool tc_stream_supported(const Ctx& c, int64_t b) {
  return c.tc_st_ok && c.cfg.dtype == SGEP_BF16 && c.d_x == c.d_y && c.d_x % (2 * kR) == 0 && c.d_x / 128 < c.num_sms && b % 256 == 0 &&
         b > 0 && b <= c.cfg.max_b && c.cfg.split_AB && c.k <= 32 && !c.adam_m && !c.z;
}

int tc_stream_max_steps() { return kMaxSteps; }

static size_t counters_len(const Ctx& c) {
  const size_t nrt = (size_t)c.cfg.max_b / 128;
  // [nrt] contributions | [2 nrt] operand flags | terms | barrier | Grams | coefficients |
  // [num_sms] per-CTA operands | [num_sms] per-CTA rows
  return 3 * nrt + 4 + 2 * (size_t)c.num_sms;
}
constexpr size_t kTermFloats = 6 * (size_t)kTerms + 2 * (size_t)kCoef;  // abbuf | ubuf | cbuf

int tc_stream_setup(Ctx& c) {
  c.tc_st_ok = 0;
  const char* env = getenv("SGEP_TC_STREAM");
  if (env && env[0] == '0') return SGEP_OK;
  if (c.cfg.dtype != SGEP_BF16) return SGEP_OK;  // the streamed kernel reads BF16 rows
  if (c.d_x != c.d_y || c.d_x % (2 * kR) != 0 || c.d_x / 128 >= c.num_sms) return SGEP_OK;
  int per_sm = 0;
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_tc_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_stream, kThreads, kSmem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return SGEP_OK;
  }
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_st_cnt, counters_len(c) * sizeof(unsigned)));
  SGEP_CUDA_TRY(cudaMemset(c.tc_st_cnt, 0, counters_len(c) * sizeof(unsigned)));
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_st_terms, kTermFloats * sizeof(float)));
  SGEP_CUDA_TRY(cudaMemset(c.tc_st_terms, 0, kTermFloats * sizeof(float)));
  c.tc_st_last_b = 0;
  // tuning knobs: SGEP_TC_LAG (chunks the projection may run ahead, 2..8; each chunk is
  // 256 rows of the minibatch kept in L2) and SGEP_TC_HELPERS (builder CTAs, 1..24)
  const char* lag = getenv("SGEP_TC_LAG");
  c.tc_st_lag = lag ? std::max(2, std::min(8, atoi(lag))) : kLagDefault;
  // SGEP_TC_PFN: chunks of the next step prefetched into L2 during a step's last chunks (0..8)
  const char* pfn = getenv("SGEP_TC_PFN");
  c.tc_st_pfn = pfn ? std::max(0, std::min(8, atoi(pfn))) : kPfNextDefault;
  const char* hl = getenv("SGEP_TC_HELPERS");
  c.tc_st_helpers = hl ? std::max(1, std::min(kMaxHelpers, atoi(hl))) : kMaxHelpers;
  c.tc_st_epoch = 0;
  c.tc_st_launch = 0;
  c.tc_st_reset = 0;
  c.tc_pq_dirty = 1;
  const char* tr = getenv("SGEP_TRACE");
  if (tr && tr[0] == '1') {
    const size_t n = (size_t)c.num_sms * ((size_t)c.cfg.max_b / kR + 2) * kEv + (size_t)c.num_sms * 16;
    SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_st_trace, n * sizeof(unsigned long long)));
    SGEP_CUDA_TRY(cudaMemset(c.tc_st_trace, 0, n * sizeof(unsigned long long)));
  }
  c.tc_st_ok = 1;
  return SGEP_OK;
}

void tc_stream_free(Ctx& c) {
  cudaFree(c.tc_st_cnt);
  c.tc_st_cnt = nullptr;
  cudaFree(c.tc_st_terms);
  c.tc_st_terms = nullptr;
  cudaFree(c.tc_st_trace);
  c.tc_st_trace = nullptr;
  c.tc_st_ok = 0;
}

// `nsteps` consecutive steps of Alg. 2 on BF16 minibatches X[s b .. s b + b) (and Y), each
// read from HBM once: products, row-side terms and the update in one cooperative launch.
// V, [Bv], the V^T operand and the d-side terms of slot (c.t & 1) must be current (the
// chain of tensor-core steps); the launch leaves them current for step c.t + nsteps.
int tc_stream_steps(Ctx& c, const void* X, const void* Y, int64_t b, int nsteps, cudaStream_t s) {
  if (nsteps < 1 || nsteps > kMaxSteps) {
    set_error("tc_stream_steps: nsteps out of range");
    return SGEP_EINVAL;
  }
  const size_t nrt_max = (size_t)c.cfg.max_b / 128;
  float* P = c.tc_PQ;
  float* Q = c.tc_PQ + (size_t)c.cfg.max_b * 32;
  // counters are monotone over steps of one minibatch size; restart them (and the row sums
  // and term slots) after an aborted launch, when the size changes and before they could wrap
  if (c.tc_st_reset || c.tc_st_epoch + (unsigned)nsteps >= (1u << 20) || b != c.tc_st_last_b) {
    SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_st_cnt, 0, counters_len(c) * sizeof(unsigned), s));
    SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_st_terms, 0, kTermFloats * sizeof(float), s));
    c.tc_st_last_b = b;
    c.tc_st_epoch = 0;
    c.tc_st_launch = 0;
    c.tc_st_grams = 0;
    c.tc_st_reset = 0;
    c.tc_pq_dirty = 1;
  }
  if (c.tc_pq_dirty) {
    SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_PQ, 0, 2 * (size_t)c.cfg.max_b * 32 * sizeof(float), s));
    c.tc_pq_dirty = 0;
  }
  const int64_t rows = b * nsteps;
  CUtensorMap mX, mY, mX64, mY64, mVt, mPt, mQt;
  int rc = make_map_bf16(&mX, X, rows, c.d_x, c.d_x, 128, 64);
  if (!rc) rc = make_map_bf16(&mY, Y, rows, c.d_y, c.d_y, 128, 64);
  // the back-projection's 64-row steps: one copy of 64 rows x 256 columns through a 3-D view
  // where the CUDA driver takes it (SGEP_TC_BP_GROUPS=0 keeps four 2-D boxes per step)
  const char* bg = getenv("SGEP_TC_BP_GROUPS");
  int bp_groups = !(bg && bg[0] == '0') && make_map_bf16_groups(&mX64, X, rows, c.d_x, c.d_x, 64, 4) == SGEP_OK &&
                  make_map_bf16_groups(&mY64, Y, rows, c.d_y, c.d_y, 64, 4) == SGEP_OK;
  if (!bp_groups) {
    if (!rc) rc = make_map_bf16(&mX64, X, rows, c.d_x, c.d_x, 64, 64);
    if (!rc) rc = make_map_bf16(&mY64, Y, rows, c.d_y, c.d_y, 64, 64);
  }
  if (!rc) rc = make_map_bf16(&mVt, c.tc_Vt, 2 * 32, c.d, c.d, 64, 64);
  if (!rc) rc = make_map_bf16(&mPt, c.tc_Pt, 2 * 32, b, c.cfg.max_b, 64, 64);
  if (!rc) rc = make_map_bf16(&mQt, c.tc_Qt, 2 * 32, b, c.cfg.max_b, 64, 64);
  if (rc) return rc;
  const int G = (int)(c.d_x / 128);
  const int H = std::min(c.tc_st_helpers, c.num_sms - G);  // builder helpers on otherwise idle SMs
  const int k = c.k;
  const int slot0 = (int)(c.t & 1), slot_last = (int)((c.t + nsteps - 1) & 1);
  const TcTerms t0 = tc_terms(c, slot0), tn = tc_terms(c, 1 - slot_last);
  StreamArgs sa = {};
  sa.G = G;
  sa.lag = c.tc_st_lag;
  sa.nsteps = nsteps;
  sa.bp_groups = bp_groups;
  sa.pf_next = c.tc_st_pfn;
  c.tc_st_bp_groups = bp_groups;
  {
    const char* se = getenv("SGEP_TC_SERIAL");
    sa.serial = (se && se[0] == '1') ? 1 : 0;
  }
  sa.e0 = c.tc_st_epoch;
  sa.b = b;
  sa.nA = b / 2;
  sa.d_x = c.d_x;
  sa.d = c.d;
  sa.ldt = c.cfg.max_b;
  sa.k = k;
  sa.nchunk = (int)(b / kR);
  sa.splits = (int)(c.d_x / (2 * kR));
  sa.inv_nA = 1.f / (float)(b / 2);
  sa.inv_nB = 1.f / (float)(b - b / 2);
  sa.rho = c.cfg.rho;
  sa.gamma = c.cfg.gamma0;
  sa.eps_B = c.cfg.eps_B;
  for (int st = 0; st < nsteps; ++st) sa.eta[st] = (float)schedule_eta(c.cfg, c.t + st + 1);
  sa.P = P;
  sa.Q = Q;
  sa.Pt = c.tc_Pt;
  sa.Qt = c.tc_Qt;
  sa.cnt = c.tc_st_cnt;
  sa.wready = c.tc_st_cnt + nrt_max;
  sa.terms_done = c.tc_st_cnt + 3 * nrt_max;
  sa.bar = sa.terms_done + 1;
  sa.grams_done = sa.terms_done + 2;
  sa.coef_ready = sa.terms_done + 3;
  sa.grams_base = c.tc_st_grams;
  sa.H = H;
  sa.upd_done = sa.terms_done + 4;
  sa.rows_done = sa.upd_done + c.num_sms;
  sa.bar_target = (c.tc_st_launch + 1) * (unsigned)G;
  sa.abbuf = c.tc_st_terms;
  sa.ubuf = c.tc_st_terms + 3 * kTerms;
  sa.cbuf = c.tc_st_terms + 6 * kTerms;
  sa.V = c.V;
  sa.S = c.S;
  sa.G0 = t0.G;
  sa.vv0 = t0.vv;
  sa.Gn = tn.G;
  sa.vvn = tn.vv;
  sa.Vt = c.tc_Vt;
  const bool dbg = c.cfg.debug != 0;
  sa.AV = dbg ? c.acc : nullptr;
  sa.BV = dbg ? c.acc + c.d * k : nullptr;
  sa.dbg = dbg ? c.tc_dbg : nullptr;
  sa.grad_out = dbg ? c.grad : nullptr;
  sa.dflag = c.dflag;
  sa.trace = c.tc_st_trace;
  sa.trace2 = c.tc_st_trace ? c.tc_st_trace + (size_t)c.num_sms * ((size_t)c.cfg.max_b / kR + 2) * kEv : nullptr;
  c.tc_st_nchunk = sa.nchunk;
  if (c.tc_st_trace)
    SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_st_trace, 0,
                                  ((size_t)c.num_sms * ((size_t)c.cfg.max_b / kR + 2) * kEv + (size_t)c.num_sms * 16) *
                                      sizeof(unsigned long long),
                                  s));
  c.tc_st_grid = G + H;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(G + H));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: they wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SGEP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tc_stream, mX, mY, mX64, mY64, mVt, mPt, mQt, sa));
  c.tc_st_epoch += (unsigned)nsteps;
  c.tc_st_grams += (unsigned)((nsteps - 1) * std::min(H, G));  // one release per step by each slice owner
  ++c.tc_st_launch;
  c.tc_acc_stale = dbg ? 0 : 1;
  c.tc_chain = 1;
  ++c.launches;
  return SGEP_OK;
}

// SGEP_TRACE=1: per-chunk event times of the last step of the most recent streamed launch (stderr).
void tc_stream_trace_report(Ctx& c) {
  if (!c.tc_st_trace || !c.tc_st_nchunk) return;
  const int n = c.tc_st_grid, nc = c.tc_st_nchunk;
  std::vector<unsigned long long> t((size_t)n * (nc + 2) * kEv);
  if (cudaMemcpy(t.data(), c.tc_st_trace, t.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return;
  auto at = [&](int cta, int ch, int ev) { return t[((size_t)cta * (nc + 2) + ch) * kEv + ev]; };
  unsigned long long g0 = ~0ull;
  for (int b = 0; b < n; ++b)
    if (at(b, nc, 0)) g0 = std::min(g0, at(b, nc, 0));
  auto row = [&](int ch, const char* const* names, int ev0, int nev) {
    for (int ev = ev0; ev < ev0 + nev; ++ev) {
      std::vector<double> v;
      for (int b = 0; b < n; ++b)
        if (at(b, ch, ev) >= g0) v.push_back(((double)at(b, ch, ev) - (double)g0) / 1e3);
      std::sort(v.begin(), v.end());
      if (v.empty()) continue;
      std::fprintf(stderr, " %s %.2f/%.2f", names[ev - ev0], v[v.size() / 2], v.back());
    }
    std::fprintf(stderr, "\n");
  };
  const char* tot[4] = {"start", "proj", "end", "exit"};
  std::fprintf(stderr, "[sgep trace] streamed steps, %d CTAs (%d helpers), %d chunks, back-projection copies %s (us, median/max):",
               n, n - (int)(c.d_x / 128), nc, c.tc_st_bp_groups ? "3-D" : "2-D");
  row(nc, tot, 0, 4);
  const char* upd[8] = {"entry", "terms", "coef", "T", "rows", "operand/grams", "bar", "done"};
  std::fprintf(stderr, "[sgep trace]   update, last step:");
  row(nc, upd, 4, 8);
  std::fprintf(stderr, "[sgep trace]   update, step before:");
  row(nc + 1, upd, 4, 8);
  {
    std::vector<unsigned long long> t2((size_t)n * 16);
    const size_t off = (size_t)c.num_sms * ((size_t)c.cfg.max_b / kR + 2) * kEv;
    if (cudaMemcpy(t2.data(), c.tc_st_trace + off, t2.size() * 8, cudaMemcpyDeviceToHost) == cudaSuccess) {
      std::fprintf(stderr, "[sgep trace]   row work quarters (start, issued, waited, stored), CTA 0:");
      for (int ev = 0; ev < 16; ++ev)
        std::fprintf(stderr, " %.2f", t2[ev] >= g0 ? ((double)t2[ev] - (double)g0) / 1e3 : -1.0);
      std::fprintf(stderr, "\n");
    }
  }
  {
    std::vector<unsigned long long> t2((size_t)n * 16);
    const size_t off = (size_t)c.num_sms * ((size_t)c.cfg.max_b / kR + 2) * kEv;
    const int G = (int)(c.d_x / 128);
    if (cudaMemcpy(t2.data(), c.tc_st_trace + off, t2.size() * 8, cudaMemcpyDeviceToHost) == cudaSuccess) {
      const char* hn[3] = {"step", "first slice", "released"};
      std::fprintf(stderr, "[sgep trace]   helper Grams, last step:");
      for (int ev = 0; ev < 3; ++ev) {
        std::vector<double> v;
        for (int b = G; b < n; ++b)
          if (t2[(size_t)b * 16 + ev] >= g0) v.push_back(((double)t2[(size_t)b * 16 + ev] - (double)g0) / 1e3);
        std::sort(v.begin(), v.end());
        if (!v.empty()) std::fprintf(stderr, " %s %.2f/%.2f", hn[ev], v[v.size() / 2], v.back());
      }
      std::fprintf(stderr, "\n");
    }
  }
  const char* names[8] = {"issue", "mma", "release", "build0", "built", "Wseen", "bpdone", "terms"};
  for (int ch : {0, 1, 2, nc / 2, nc - 2, nc - 1}) {
    if (ch < 0 || ch >= nc) continue;
    std::fprintf(stderr, "[sgep trace]   chunk %2d:", ch);
    row(ch, names, 0, 8);
  }
}

}  // namespace sgep

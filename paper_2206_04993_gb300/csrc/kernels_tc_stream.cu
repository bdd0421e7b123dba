// One-read tensor-core products of a BF16 minibatch (large d), chunked through L2.
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
//  * Back-projection role. CTA j owns a 256-column slice of X or Y and streams
//    every row of it (from L2) in 64-row steps once the step's row tile is built;
//    tcgen05 multiplies each step's transpose by the operand into four TMEM
//    accumulators (A_t V, B_t V x two 128-column halves) written once at the end.
// The projection runs at most kLag chunks ahead of the CTA's own back-projection
// so the rows it re-reads are still in L2. Nothing the projection or the builders
// wait for depends on the back-projection, and waits only ever point at earlier
// chunks, so the pipeline cannot deadlock; every wait is time-bounded and records
// the timeout bit of the device error word.
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

// Streaming CTAs: w0 projection TMA, w1 projection MMA, w2 back-projection TMA,
// w3 back-projection MMA, w4-7 projection epilogue then A_t V / B_t V write-out, w8-11
// reducers (chunk c: warp 8 + c % 4 sums the staged tile into P or Q and releases it).
// Helper CTAs: w8-11 builders.
constexpr int kThreads = 384;
constexpr int kR = 256;         // rows per chunk (16 MB at d = 32768)
constexpr int kPS = 4;          // projection stages (one 128 x 64 box each)
constexpr int kBS = 2;          // back-projection stages (four 64 x 64 boxes + the operand box)
constexpr int kLagDefault = 5;  // chunks the projection may run ahead of the back-projection
constexpr int kMaxHelpers = 24; // builder CTAs on SMs the streaming CTAs leave idle
constexpr int kAcc = 4;         // projection accumulators in tensor memory (64 columns each)
constexpr int kVtBoxes = 2 * kR / 64;
constexpr int kVtB = kVtBoxes * 8192;  // resident V^T slice: 2 kR columns in 64 x 64 boxes
constexpr int kPBox = 16384;
constexpr int kBStage = 40960;
constexpr int kStgRows = 64;    // builder staging (helper CTAs, in the V^T region): 64 rows of P and Q
constexpr int kEStg = 128 * 32 * 4;  // epilogue staging: one 128 x 32 FP32 projection tile
constexpr int kNumBars = 2 * kPS + 2 * kAcc + 2 * kBS + 1 + 1 + 2 + 4 + 1;
constexpr size_t kSmem = (size_t)kVtB + kPS * kPBox + kBS * kBStage + kEStg + kNumBars * 8 + 64 + 1024;
static_assert(2 * kStgRows * 32 * 4 <= kVtB, "builder staging fits in the V^T region");
static_assert(kSmem <= 232448, "shared memory budget");
constexpr int kRTc = kR / 128;  // row tiles per chunk

struct StreamArgs {
  int64_t b, nA, d_x, ldt;  // ldt: row stride (elements) of Pt and Qt
  int k, nchunk, splits;
  int G;                    // streaming CTAs; CTAs G .. gridDim.x - 1 are builder helpers
  int lag;                  // chunks the projection may run ahead of the CTA's back-projection
  float inv_nA, inv_nB;
  float* P;                 // [rows][32], zero on entry; the builders clear the rows again
  float* Q;
  __nv_bfloat16* Pt;        // [64][ldt] BF16 hi (0..31) / lo (32..63) pairs, transposed
  __nv_bfloat16* Qt;
  unsigned* cnt;            // [b / 128] projection contributions (monotone over launches)
  unsigned* wready;         // [b / 64] operand of the 64-row half built (monotone)
  unsigned cnt_target, w_target;
  float* a;                 // k x k row-side terms (accumulated)
  float* bterm;             // k
  float* AV;                // d x k
  float* BV;
  int* dflag;
  unsigned long long* trace;  // [G][nchunk + 1][kEv] globaltimer stamps, or null
  // fused update (Eq. update, the player and auxiliary steps, the retraction) when fuse != 0
  int fuse;
  float* V;                 // d x k, read and rewritten
  float* S;                 // d x k [Bv]
  float* terms;             // a (kk) | b (k) | norms [2][k] | G [2][kk] | vv [2][k]
  float* part;              // per-CTA partials: [G][32] column sums, then [G][32 * 32 + 32]
  float* dbg;               // a | G | b as used (debug), or null
  float* grad_out;          // update directions (debug), or null
  __nv_bfloat16* Vt;        // next step's V operand (BF16 hi/lo pairs, 64 x d)
  int64_t d;
  int slot;                 // step parity of the k x k terms read by this update
  float rho, eta, gamma, eps_B;
  unsigned* bar;            // grid-barrier arrivals of the streaming CTAs (monotone)
  unsigned bar_base;        // arrivals before this launch
  unsigned* terms_done;     // row-side terms added by the builders (monotone)
  unsigned terms_target;
};

// Trace events per chunk; row nchunk of a CTA holds start, projection end, back-projection end, end.
constexpr int kEv = 8;
enum { kEvIssue = 0, kEvMma, kEvRelease, kEvBuildStart, kEvBuilt, kEvWSeen, kEvBpDone, kEvTerms };

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ uint32_t pack2_bf16(float first, float second) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(first, second);
  return *reinterpret_cast<const uint32_t*>(&h);
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

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Bounded barrier of the streaming CTAs (epilogue group of each): false on timeout.
__device__ __forceinline__ bool stream_barrier(const StreamArgs& a, unsigned target, int etid, volatile int* ok) {
  named_barrier(1, 128);
  if (etid == 0) {
    __threadfence();
    atomicAdd(a.bar, 1u);
    *ok = spin_until_geq(a.bar, target) ? 1 : 0;
    if (!*ok) atomicOr(a.dflag, kFlagTimeout);
  }
  named_barrier(1, 128);
  return *ok != 0;
}

// The update of Alg. 2 for the CTA's 256 rows of V, run by the epilogue group (128 threads,
// thread r of the group owns rows r and 128 + r of the slice) once every row-side term is in:
//   phase 1: coefficients of Eq. (update) from a, G, b (and |v_i|^2 when eps_B > 0); with
//            A_t V and B_t V from tensor memory, v' = v + eta grad and [Bv]' = [Bv] + gamma
//            (B_t v - [Bv]); per-CTA column sums of v'^2;
//   barrier; phase 2: v = v' / |v'| (the retraction) written out with its BF16 hi/lo pairs
//            (the next step's operand); per-CTA partials of the next step's G = V^T [Bv]' and
//            |v_i|^2;
//   barrier; phase 3: CTA j adds a slice of those partials.
// The k x k terms are double-buffered by step parity (read slot, write 1 - slot); CTA 0
// clears a and b after the first barrier, when every CTA has read them.
__device__ __forceinline__ void fused_update(const StreamArgs& a, int etid, int q, int lane, int r, int j,
                                          int64_t b_goff, uint32_t tmem_bp, uint8_t* PR, uint8_t* BR,
                                          volatile int* ok, volatile int* abort_flag) {
  constexpr int KP = 32, KT = KP * KP + KP;
  const int k = a.k, kk = k * k, slot = a.slot, G = a.G;
  float* vs = reinterpret_cast<float*>(BR);  // [256][33] v', then v
  float* ss = vs + 256 * 33;                 // [256][33] [Bv]'
  float* T = reinterpret_cast<float*>(PR);   // [32][32]
  float* Am = T + KP * KP;
  float* Gm = Am + KP * KP;
  float* cb = Gm + KP * KP;
  float* cac = cb + KP;
  float* inv_s = cac + KP;
  float* inv_n = inv_s + KP;
  float* red = inv_n + KP;                   // [4][KT]
  float* ta = a.terms;
  float* tb = ta + kk;
  float* nrm = tb + k;
  float* Gs = nrm + 2 * k;
  float* vvs = Gs + 2 * kk;
  const float* Gc = Gs + slot * kk;
  const float* vvc = vvs + slot * k;
  float* part_n = a.part;
  float* part_t = a.part + (size_t)G * KP;
  auto ustamp = [&](int ev) {  // events 4..7 of the CTA's summary row
    if (a.trace && etid == 0) a.trace[((size_t)j * (a.nchunk + 1) + a.nchunk) * kEv + ev] = globaltimer();
  };
  if (etid == 0) *ok = spin_until_geq(a.terms_done, a.terms_target) ? 1 : 0;
  named_barrier(1, 128);
  if (!*ok) {
    if (etid == 0) atomicOr(a.dflag, kFlagTimeout);
    return;
  }
  ustamp(4);
  for (int p = etid; p < kk; p += 128) {
    Am[p] = __ldcg(ta + p);
    Gm[p] = __ldcg(Gc + p);
  }
  if (etid < KP) cb[etid] = etid < k ? fmaf(a.eps_B, __ldcg(vvc + etid), __ldcg(tb + etid)) : 0.f;
  named_barrier(1, 128);
  if (etid < k) inv_s[etid] = 1.f / fmaxf(Gm[etid * k + etid], a.rho);
  named_barrier(1, 128);
  for (int p = etid; p < KP * KP; p += 128) {
    const int jj = p / KP, i = p % KP;
    T[p] = (jj < i && i < k) ? cb[i] * Am[i * k + jj] * inv_s[jj] : 0.f;
  }
  if (etid < KP) {
    float c = 0.f;
    if (etid < k)
      for (int jj = 0; jj < etid; ++jj) c = fmaf(Am[etid * k + jj] * Gm[etid * k + jj], inv_s[jj], c);
    cac[etid] = etid < k ? Am[etid * k + etid] - c : 0.f;
  }
  named_barrier(1, 128);
  // ---- phase 1 ----------------------------------------------------------------
  // the slice's rows of V and [Bv] (256 k contiguous floats each) into shared memory
  if ((k & 3) == 0) {  // eight float4 loads of each in flight per thread
    const float4* gv = reinterpret_cast<const float4*>(a.V + b_goff * k);
    const float4* gs = reinterpret_cast<const float4*>(a.S + b_goff * k);
    const int n4 = 64 * k;
    for (int base = 0; base < n4; base += 128 * 8) {
      float4 xv[8], xs[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = base + etid + 128 * u;
        if (e < n4) {
          xv[u] = gv[e];
          xs[u] = gs[e];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = base + etid + 128 * u;
        if (e < n4) {
          const int row = (4 * e) / k, i = 4 * e - row * k;
          float* dv = vs + row * 33 + i;
          float* ds = ss + row * 33 + i;
          dv[0] = xv[u].x, dv[1] = xv[u].y, dv[2] = xv[u].z, dv[3] = xv[u].w;
          ds[0] = xs[u].x, ds[1] = xs[u].y, ds[2] = xs[u].z, ds[3] = xs[u].w;
        }
      }
    }
  } else {
    const float* gv = a.V + b_goff * k;
    const float* gs = a.S + b_goff * k;
    for (int base = 0; base < 256 * k; base += 128 * 8) {
      float xv[8], xs[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = base + etid + 128 * u;
        if (e < 256 * k) {
          xv[u] = gv[e];
          xs[u] = gs[e];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = base + etid + 128 * u;
        if (e < 256 * k) {
          const int row = e / k, i = e - row * k;
          vs[row * 33 + i] = xv[u];
          ss[row * 33 + i] = xs[u];
        }
      }
    }
  }
  named_barrier(1, 128);
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int row = 128 * h + r;
    const int64_t c = b_goff + row;
    const float* sv = ss + row * 33;  // this thread's row of [Bv] (zero beyond k: see T)
    // penalty sum_j [Bv]_j T_ji for every player first: the row of [Bv] is overwritten below
    float gr[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) gr[i] = 0.f;
#pragma unroll 4
    for (int jj = 0; jj < k; ++jj) {
      const float sj = sv[jj];
#pragma unroll
      for (int i = 0; i < 32; ++i) gr[i] = fmaf(sj, T[jj * KP + i], gr[i]);
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int i0 = 16 * half;
      float x[16], lo[16];
      const uint32_t ta0 = tmem_bp + (uint32_t)(64 * h) + ((uint32_t)(32 * q) << 16);
      tmem_ld16(ta0 + i0, x);  // A_t v (hi, lo)
      tmem_ld16(ta0 + 32 + i0, lo);
#pragma unroll
      for (int i = 0; i < 16; ++i) gr[i0 + i] = cb[i0 + i] * ((x[i] + lo[i]) * a.inv_nA) - gr[i0 + i];
      tmem_ld16(ta0 + 128 + i0, x);  // B_t v (hi, lo)
      tmem_ld16(ta0 + 128 + 32 + i0, lo);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int ii = i0 + i;
        const float v = ii < k ? vs[row * 33 + ii] : 0.f;
        const float bve = fmaf(a.eps_B, v, (x[i] + lo[i]) * a.inv_nB);
        const float g = gr[ii] - cac[ii] * bve;
        const float vn = ii < k ? fmaf(a.eta, g, v) : 0.f;
        const float s0 = ii < k ? sv[ii] : 0.f;
        const float sn = ii < k ? fmaf(a.gamma, bve - s0, s0) : 0.f;
        if (ii < k && a.grad_out) a.grad_out[c * k + ii] = g;
        vs[row * 33 + ii] = vn;
        ss[row * 33 + ii] = sn;
      }
    }
  }
  named_barrier(1, 128);
  {
    float* gs = a.S + b_goff * k;  // [Bv]' rows out, coalesced
    for (int e = etid; e < 256 * k; e += 128) {
      const int row = e / k, i = e - row * k;
      gs[e] = ss[row * 33 + i];
    }
  }
  {
    const int i = etid & 31, g = etid >> 5;
    float s2 = 0.f;
    for (int row = 64 * g; row < 64 * g + 64; ++row) s2 = fmaf(vs[row * 33 + i], vs[row * 33 + i], s2);
    red[g * KP + i] = s2;
  }
  named_barrier(1, 128);
  if (etid < KP) part_n[(size_t)j * KP + etid] = red[etid] + red[KP + etid] + red[2 * KP + etid] + red[3 * KP + etid];
  ustamp(5);
  if (!stream_barrier(a, a.bar_base + (unsigned)G, etid, ok)) return;
  ustamp(6);
  if (j == 0) {  // every CTA has read a, G and b: keep them (debug) and clear a and b
    if (a.dbg) {
      for (int p = etid; p < kk; p += 128) {
        a.dbg[p] = Am[p];
        a.dbg[kk + p] = Gm[p];
      }
      if (etid < k) a.dbg[2 * kk + etid] = __ldcg(tb + etid);
    }
    for (int p = etid; p < kk; p += 128) ta[p] = 0.f;
    if (etid < k) tb[etid] = 0.f;
  }
  {
    const int i = etid & 31, g = etid >> 5;
    float s2 = 0.f;
    for (int blk0 = g; blk0 < G; blk0 += 4 * 8) {  // eight loads in flight
      float x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int blk = blk0 + 4 * u;
        x[u] = blk < G ? __ldcg(part_n + (size_t)blk * KP + i) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) s2 += x[u];
    }
    red[g * KP + i] = s2;
  }
  named_barrier(1, 128);
  if (etid < KP) {
    const float s2 = red[etid] + red[KP + etid] + red[2 * KP + etid] + red[3 * KP + etid];
    inv_n[etid] = etid < k ? 1.f / sqrtf(s2) : 0.f;
    if (j == 0 && etid < k) nrm[slot * k + etid] = s2;
  }
  named_barrier(1, 128);
  // ---- phase 2 ----------------------------------------------------------------
  bool bad = false;
  for (int e = etid; e < 256 * KP; e += 128) {
    const int row = e / KP, i = e % KP;
    vs[row * 33 + i] *= inv_n[i];
  }
  named_barrier(1, 128);
  {
    float* gv = a.V + b_goff * k;  // coalesced
    for (int e = etid; e < 256 * k; e += 128) {
      const int row = e / k, i = e - row * k;
      const float v = vs[row * 33 + i];
      gv[e] = v;
      bad |= !isfinite(v);
    }
  }
  if (bad) atomicOr(a.dflag, kFlagNonFinite);
  named_barrier(1, 128);
  // transposed BF16 pairs: (operand row n, two consecutive rows of V)
  for (int e = etid; e < 2 * KP * 128; e += 128) {
    const int n = e / 128, rp = 2 * (e % 128);
    const float v0 = vs[rp * 33 + (n % KP)], v1 = vs[(rp + 1) * 33 + (n % KP)];
    uint32_t w;
    if (n < KP) {
      w = pack2_bf16(v0, v1);
    } else {
      const float h0 = __bfloat162float(__float2bfloat16(v0)), h1 = __bfloat162float(__float2bfloat16(v1));
      w = pack2_bf16(v0 - h0, v1 - h1);
    }
    *reinterpret_cast<uint32_t*>(a.Vt + (int64_t)n * a.d + b_goff + rp) = w;
  }
  // partials of G = V^T [Bv]' (4 x 4 tiles, two 128-row groups) and |v_i|^2
  {
    const int tl = etid & 63, rg = etid >> 6;
    const int i0 = 4 * (tl & 7), j0 = 4 * (tl >> 3);
    float acc[4][4] = {};
    for (int row = 128 * rg; row < 128 * rg + 128; ++row) {
      float x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = vs[row * 33 + i0 + u];
        y[u] = ss[row * 33 + j0 + u];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[p][u] = fmaf(x[p], y[u], acc[p][u]);
    }
    float nv = 0.f;
    {
      const int i = etid & 31, g = etid >> 5;
      for (int row = 64 * g; row < 64 * g + 64; ++row) nv = fmaf(vs[row * 33 + i], vs[row * 33 + i], nv);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int u = 0; u < 4; ++u) red[rg * KT + (i0 + p) * KP + j0 + u] = acc[p][u];
    named_barrier(1, 128);
    // |v_i|^2 of the four 64-row groups into the spare rows 2 and 3 of red
    red[2 * KT + (etid >> 5) * KP + (etid & 31)] = nv;
    named_barrier(1, 128);
    for (int e = etid; e < KT; e += 128) {
      float val;
      if (e < KP * KP) {
        val = red[e] + red[KT + e];
      } else {
        const int i = e - KP * KP;
        val = red[2 * KT + i] + red[2 * KT + KP + i] + red[2 * KT + 2 * KP + i] + red[2 * KT + 3 * KP + i];
      }
      part_t[(size_t)j * KT + e] = val;
    }
  }
  if (!stream_barrier(a, a.bar_base + 2u * (unsigned)G, etid, ok)) return;
  ustamp(7);
  // ---- phase 3: entries [j per, (j + 1) per) of the next step's terms ----------
  {
    const int per = (KT + G - 1) / G;
    const int e0 = j * per;
    const int ne = max(0, min(per, KT - e0));
    float* Gn = Gs + (1 - slot) * kk;
    float* vvn = vvs + (1 - slot) * k;
    for (int el = q; el < ne; el += 4) {
      float s2 = 0.f;
      for (int b0 = lane; b0 < G; b0 += 32 * 5) {  // five loads in flight per lane
        float x[5];
#pragma unroll
        for (int u = 0; u < 5; ++u) {
          const int blk = b0 + 32 * u;
          x[u] = blk < G ? __ldcg(part_t + (size_t)blk * KT + e0 + el) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 5; ++u) s2 += x[u];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) {
        const int te = e0 + el;
        if (te < KP * KP) {
          const int i = te / KP, jj = te % KP;
          if (i < k && jj < k) Gn[i * k + jj] = s2;
        } else if (te - KP * KP < k) {
          vvn[te - KP * KP] = s2;
        }
      }
    }
  }
  (void)abort_flag;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_stream(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
                const __grid_constant__ CUtensorMap mapX64, const __grid_constant__ CUtensorMap mapY64,
                const __grid_constant__ CUtensorMap mapVt, const __grid_constant__ CUtensorMap mapPt,
                const __grid_constant__ CUtensorMap mapQt, const StreamArgs a) {
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
  uint64_t* vt_full = b_empty + kBS;
  uint64_t* bp_done = vt_full + 1;
  uint64_t* mma_fin = bp_done + 1;         // [2]
  uint64_t* stg_full = mma_fin + 2;        // [4] staged tile of chunk c ready for reducer c % 4
  uint64_t* stg_empty = stg_full + 4;      // the reduction of the staged tile has read it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* bp_loaded = abort_flag + 1;  // chunks whose back-projection rows have landed
  volatile int* epi_ok = abort_flag + 2;
  volatile int* bld_ok = abort_flag + 3;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = a.G, j = (int)blockIdx.x;
  const bool helper = j >= G;
  const int H = (int)gridDim.x - G;
  const int splits = a.splits;
  // projection tile of this CTA (the same in every chunk)
  const int p_split = j % splits;
  const int p_view = (j / splits) & 1;
  const int p_rtl = j / (2 * splits);
  constexpr int kRT = kR / 128;  // row tiles per chunk
  const int64_t p_col0 = (int64_t)p_split * (2 * kR);
  // back-projection slice of this CTA
  const int nslice = G / 2;
  const int b_view = j >= nslice ? 1 : 0;
  const int64_t b_c0 = (int64_t)(j - b_view * nslice) * 256;
  const int64_t b_goff = (b_view ? a.d_x : 0) + b_c0;
  const int nchunk = a.nchunk;
  const int nrt = nchunk * kRT;

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
    if (a.trace) a.trace[((size_t)j * (nchunk + 1) + nchunk) * kEv + ev] = globaltimer();
  };
  auto cstamp = [&](int c, int ev) {
    if (a.trace) a.trace[((size_t)j * (nchunk + 1) + c) * kEv + ev] = globaltimer();
  };
  auto fail = [&]() {
    atomicOr(a.dflag, kFlagTimeout);
    *abort_flag = 1;
  };
  if (tid == 0) stamp(0);

  if (helper) {
    if (warp >= 8) {
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
    for (int item = 0; item < 2 * nrt; ++item) {  // item = (row tile, 64-row half)
      if (item % H != j - G) continue;
      const int rt = item >> 1;
      const int64_t r0 = (int64_t)item * kStgRows;
      if (bt == 0) {
        bool ok = !*abort_flag && spin_until_geq(a.cnt + rt, a.cnt_target);
        *bld_ok = ok ? 1 : 0;
      }
      named_barrier(2, 128);
      if (bt == 0 && (item & 1) == 0) cstamp(rt / kRT, kEvBuildStart);
      if (!*bld_ok) {
        if (bt == 0) fail();
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
            for (int e = 0; e < 4; ++e) {
              const float v0 = src[(rr + 8 * u + 2 * e) * 32 + pl];
              const float v1 = src[(rr + 8 * u + 2 * e + 1) * 32 + pl];
              if (!lo) {
                w[e] = pack2_bf16(v0, v1);
              } else {
                const float h0 = __bfloat162float(__float2bfloat16(v0));
                const float h1 = __bfloat162float(__float2bfloat16(v1));
                w[e] = pack2_bf16(v0 - h0, v1 - h1);
              }
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
        if ((item & 1) == 0) cstamp(rt / kRT, kEvBuilt);
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
          for (int e = 0; e < 2; ++e)
            if (i0 + p < k && j0 + e < k) atomicAdd(a.a + (i0 + p) * k + j0 + e, acc[p][e] * a.inv_nA);
      } else {
        const int i = bt & 31, g = bt >> 5;
        float s2 = 0.f;
        for (int rr = g * (kStgRows / 4); rr < (g + 1) * (kStgRows / 4); ++rr) {
          const float p = Ps[rr * 32 + i], qv = Qs[rr * 32 + i];
          s2 = fmaf(p, p, fmaf(qv, qv, s2));
        }
        if (i < k) atomicAdd(a.bterm + i, s2 * a.inv_nB);
      }
      __threadfence();
      named_barrier(2, 128);  // staging is reused by the next item
      if (bt == 0) {
        red_release_add(a.terms_done, 1u);
        if ((item & 1) == 0) cstamp(rt / kRT, kEvTerms);
      }
    }
    }
  } else if (warp == 0) {
    // ---- projection: resident V^T slice, then the row tiles from HBM ----------
    if (lane == 0) {
      const CUtensorMap* mZ = p_view ? &mapY : &mapX;
      const int voff = (int)((p_view ? a.d_x : 0) + p_col0);
      mbar_arrive_expect_tx(vt_full, kVtB);
      for (int jb = 0; jb < kVtBoxes; ++jb) tma_load_2d(VT + jb * 8192, &mapVt, voff + 64 * jb, 0, vt_full);
      const int nks = 2 * kR / 64;
      int i = 0;
      for (int c = 0; c < nchunk && !*abort_flag; ++c) {
        if (c >= a.lag && !wait_shared_geq(bp_loaded, c - a.lag + 1)) {
          fail();
          break;
        }
        const int row0 = (c * kRT + p_rtl) * 128;
        cstamp(c, kEvIssue);
        bool ok = true;
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
      // every issued copy lands before the CTA may exit
      for (int q = i > kPS ? i - kPS : 0; q < i; ++q) mbar_wait(p_full + (q % kPS), (q / kPS) & 1, 100000000ull);
      mbar_wait(vt_full, 0, 100000000ull);
    }
  } else if (warp == 1) {
    // ---- projection MMAs: D[128 rows x 64] += X box (128 x 64) . V^T box^T ----
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, 64, 0, 0);
      const int nks = 2 * kR / 64;
      bool ok = mbar_wait(vt_full, 0);
      int i = 0;
      for (int c = 0; ok && c < nchunk; ++c) {
        const int buf = c % kAcc;
        if (c >= kAcc && !mbar_wait(acc_empty + buf, ((c / kAcc) - 1) & 1)) {
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
        cstamp(c, kEvMma);
      }
      if (!ok) fail();
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
      int i = 0;
      bool ok = true;
      for (int c = 0; ok && c < nchunk && !*abort_flag; ++c) {
        for (int s = 0; s < kR / 64; ++s, ++i) {
          const int r0 = c * kR + 64 * s;
          if (!spin_until_geq(a.wready + (r0 >> 6), a.w_target)) {
            ok = false;
            break;
          }
          fence_proxy_async_global();
          if (s == 0) cstamp(c, kEvWSeen);
          const int st = i % kBS;
          if (i >= kBS && !mbar_wait(b_empty + st, ((i / kBS) - 1) & 1)) {
            ok = false;
            break;
          }
          uint8_t* sa = BR + st * kBStage;
          mbar_arrive_expect_tx(b_full + st, kBStage);
#pragma unroll
          for (int jb = 0; jb < 4; ++jb)
            tma_load_2d_hint(sa + jb * 8192, mZ, (int)(b_c0 + 64 * jb), r0, b_full + st, once);
          tma_load_2d(sa + 32768, r0 < a.nA ? mWA : mWB, r0, 0, b_full + st);
        }
      }
      if (!ok) fail();
      for (int q = i > kBS ? i - kBS : 0; q < i; ++q) mbar_wait(b_full + (q % kBS), (q / kBS) & 1, 100000000ull);
    }
  } else if (warp == 3) {
    // ---- back-projection MMAs: acc[128 cols x 64] += X step^T . W ------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, 64, 1, 0);
      bool ok = true, usedA = false, usedB = false;
      int i = 0;
      for (int c = 0; ok && c < nchunk; ++c) {
        for (int s = 0; s < kR / 64; ++s, ++i) {
          const int r0 = c * kR + 64 * s;
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
          *bp_loaded = c + 1;
          cstamp(c, kEvBpDone);
        }
      }
      if (ok) mma_commit(bp_done);
      else {
        fail();
        mbar_arrive(bp_done);
      }
      mma_commit(mma_fin + 1);
      mbar_wait(mma_fin + 1, 0, 100000000ull);
    }
  } else if (warp < 8) {
    // ---- projection epilogue: partial rows into P / Q, release the row tile ----
    const int etid = tid - 128;
    const int q = warp & 3;
    const int r = 32 * q + lane;
    for (int c = 0; c < nchunk; ++c) {
      const int buf = c % kAcc;
      if (etid == 0) *epi_ok = mbar_wait(acc_full + buf, (c / kAcc) & 1) && !*abort_flag ? 1 : 0;
      named_barrier(1, 128);
      if (!*epi_ok) {
        if (etid == 0) fail();
        break;
      }
      tc_fence_after();
      float hi[32], lo[32];
      tmem_ld32(tmem_p + 64 * buf + ((uint32_t)(32 * q) << 16), hi);
      tmem_ld32(tmem_p + 64 * buf + 32 + ((uint32_t)(32 * q) << 16), lo);
      tc_fence_before();
      // the reduction of the previous chunk has read the staging tile
      if (etid == 0) *epi_ok = (c == 0 || mbar_wait(stg_empty, (c - 1) & 1)) && !*abort_flag ? 1 : 0;
      named_barrier(1, 128);
      if (!*epi_ok) {
        if (etid == 0) fail();
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
        mbar_arrive(stg_full + (c & 3));
      }
    }
    if (etid == 0) stamp(1);
    // ---- A_t V and B_t V of the slice ------------------------------------------
    if (etid == 0) *epi_ok = mbar_wait(bp_done, 0) && !*abort_flag ? 1 : 0;
    named_barrier(1, 128);
    if (*epi_ok) {
      tc_fence_after();
      const int k = a.k;
      if (a.AV != nullptr) {  // kept for readback (always when the update is not fused)
#pragma unroll 1
        for (int which = 0; which < 2; ++which) {
          float* outm = which == 0 ? a.AV : a.BV;
          const float sc = which == 0 ? a.inv_nA : a.inv_nB;
#pragma unroll 1
          for (int h = 0; h < 2; ++h) {
            float hi[32], lo[32];
            const uint32_t t = tmem_bp + (uint32_t)(which * 128 + 64 * h) + ((uint32_t)(32 * q) << 16);
            tmem_ld32(t, hi);
            tmem_ld32(t + 32, lo);
            float* o = outm + (b_goff + 128 * h + r) * k;
            if ((k & 3) == 0) {
#pragma unroll
              for (int i = 0; i < 32; i += 4)
                if (i < k)
                  *reinterpret_cast<float4*>(o + i) = make_float4(
                      (hi[i] + lo[i]) * sc, (hi[i + 1] + lo[i + 1]) * sc, (hi[i + 2] + lo[i + 2]) * sc,
                      (hi[i + 3] + lo[i + 3]) * sc);
            } else {
#pragma unroll
              for (int i = 0; i < 32; ++i)
                if (i < k) o[i] = (hi[i] + lo[i]) * sc;
            }
          }
        }
      }
      if (a.fuse) fused_update(a, etid, q, lane, r, j, b_goff, tmem_bp, PR, BR, epi_ok, abort_flag);
      tc_fence_before();
    } else if (etid == 0) {
      fail();
    }
    if (etid == 0) stamp(2);
  } else if (lane == 0) {
    // ---- reducers: staged projection tile -> P or Q (bulk add at L2), then release ----
    const int w = warp - 8;
    float* dstv = p_view ? a.Q : a.P;
    bool pending = false;
    for (int c = w, use = 0; c < nchunk; c += 4, ++use) {
      if (!mbar_wait(stg_full + w, use & 1) || *abort_flag) {
        fail();
        break;
      }
      const int rt = c * kRT + p_rtl;
      bulk_reduce_add_f32(dstv + (int64_t)rt * 128 * 32, ESTG, kEStg);
      bulk_commit();
      pending = true;
      bulk_wait_read<0>();
      mbar_arrive(stg_empty);
      bulk_wait<0>();
      pending = false;
      fence_proxy_async_global();
      __threadfence();
      red_release_add(a.cnt + rt, 1u);
      cstamp(c, kEvRelease);
    }
    if (pending) bulk_wait<0>();
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0) stamp(3);
  if (warp == 1 && !helper) tmem_dealloc(tmem, 512);
}

}  // namespace

// The streamed kernel takes CCA with d_x == d_y, d_x a multiple of 2 kR (one column split
// per (view, CTA) pair), one resident CTA per 256 columns, and minibatches of whole chunks.
bool tc_stream_supported(const Ctx& c, int64_t b) {
  return c.tc_st_ok && c.d_x == c.d_y && c.d_x % (2 * kR) == 0 && c.d_x / 128 < c.num_sms && b % 256 == 0 &&
         b > 0 && b <= c.cfg.max_b && c.cfg.split_AB && c.k <= 32;
}

int tc_stream_setup(Ctx& c) {
  c.tc_st_ok = 0;
  const char* env = getenv("SGEP_TC_STREAM");
  if (env && env[0] == '0') return SGEP_OK;
  if (c.d_x != c.d_y || c.d_x % (2 * kR) != 0 || c.d_x / 128 >= c.num_sms) return SGEP_OK;
  int per_sm = 0;
  SGEP_CUDA_TRY(cudaFuncSetAttribute(k_tc_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_stream, kThreads, kSmem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return SGEP_OK;
  }
  const size_t nrt = (size_t)c.cfg.max_b / 128;
  // [nrt] contributions | [2 nrt] operand flags | terms added | grid-barrier arrivals
  SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_st_cnt, (3 * nrt + 2) * sizeof(unsigned)));
  SGEP_CUDA_TRY(cudaMemset(c.tc_st_cnt, 0, (3 * nrt + 2) * sizeof(unsigned)));
  c.tc_st_last_b = 0;
  // SGEP_TC_STREAM_UPDATE=1 applies the update in the same launch (four warps per SM run it,
  // which is slower on GB300 than the separate fused-update kernel's 2048 warps)
  const char* fu = getenv("SGEP_TC_STREAM_UPDATE");
  c.tc_st_fuse = (fu && fu[0] == '1' && !c.adam_m && !c.z) ? 1 : 0;  // the in-launch update is Alg. 2's
  // tuning knobs: SGEP_TC_LAG (chunks the projection may run ahead, 2..8; each chunk is
  // 256 rows of the minibatch kept in L2) and SGEP_TC_HELPERS (builder CTAs, 1..24)
  const char* lag = getenv("SGEP_TC_LAG");
  c.tc_st_lag = lag ? std::max(2, std::min(8, atoi(lag))) : kLagDefault;
  const char* hl = getenv("SGEP_TC_HELPERS");
  c.tc_st_helpers = hl ? std::max(1, std::min(kMaxHelpers, atoi(hl))) : kMaxHelpers;
  c.tc_st_epoch = 0;
  c.tc_st_reset = 0;
  c.tc_pq_dirty = 1;
  const char* tr = getenv("SGEP_TRACE");
  if (tr && tr[0] == '1') {
    const size_t n = (size_t)c.num_sms * (nrt / kRTc + 1) * kEv;
    SGEP_CUDA_TRY(cudaMalloc((void**)&c.tc_st_trace, n * sizeof(unsigned long long)));
    SGEP_CUDA_TRY(cudaMemset(c.tc_st_trace, 0, n * sizeof(unsigned long long)));
  }
  c.tc_st_ok = 1;
  return SGEP_OK;
}

void tc_stream_free(Ctx& c) {
  cudaFree(c.tc_st_cnt);
  c.tc_st_cnt = nullptr;
  cudaFree(c.tc_st_trace);
  c.tc_st_trace = nullptr;
  c.tc_st_ok = 0;
}

// acc = [A_t V ; B_t V] and the row-side terms a, b of one BF16 minibatch, reading the
// minibatch from HBM once. Vt must be current. mX / mY: 128 x 64 boxes; mX64 / mY64:
// 64 x 64 boxes of the same matrices; mPt / mQt: 64 x 64 boxes of the operands.
int tc_stream_products(Ctx& c, const CUtensorMap& mX, const CUtensorMap& mY, const CUtensorMap& mX64,
                       const CUtensorMap& mY64, const CUtensorMap& mVt, const CUtensorMap& mPt,
                       const CUtensorMap& mQt, float* a_terms, float* b_terms, int64_t b, float eta, float gamma,
                       cudaStream_t s) {
  const size_t nrt_max = (size_t)c.cfg.max_b / 128;
  float* P = c.tc_PQ;
  float* Q = c.tc_PQ + (size_t)c.cfg.max_b * 32;
  // counters are monotone over launches of one minibatch size; restart them (and the row
  // sums) after an aborted launch, when the size changes and well before they could wrap
  if (c.tc_st_reset || c.tc_st_epoch >= (1u << 20) || b != c.tc_st_last_b) {
    SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_st_cnt, 0, (3 * nrt_max + 2) * sizeof(unsigned), s));
    c.tc_st_last_b = b;
    c.tc_st_epoch = 0;
    c.tc_st_reset = 0;
    c.tc_pq_dirty = 1;
  }
  if (c.tc_pq_dirty) {
    SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_PQ, 0, 2 * (size_t)c.cfg.max_b * 32 * sizeof(float), s));
    c.tc_pq_dirty = 0;
  }
  const int G = (int)(c.d_x / 128);
  const int H = std::min(c.tc_st_helpers, c.num_sms - G);  // builder helpers on otherwise idle SMs
  StreamArgs sa;
  sa.G = G;
  sa.lag = c.tc_st_lag;
  sa.b = b;
  sa.nA = b / 2;
  sa.d_x = c.d_x;
  sa.ldt = c.cfg.max_b;
  sa.k = c.k;
  sa.nchunk = (int)(b / kR);
  sa.splits = (int)(c.d_x / (2 * kR));
  sa.inv_nA = 1.f / (float)(b / 2);
  sa.inv_nB = 1.f / (float)(b - b / 2);
  sa.P = P;
  sa.Q = Q;
  sa.Pt = c.tc_Pt;
  sa.Qt = c.tc_Qt;
  sa.cnt = c.tc_st_cnt;
  sa.wready = c.tc_st_cnt + nrt_max;
  sa.cnt_target = (c.tc_st_epoch + 1) * (unsigned)(2 * sa.splits);
  sa.w_target = c.tc_st_epoch + 1;
  sa.a = a_terms;
  sa.bterm = b_terms;
  // the products are kept for readback unless the update is fused and the handle is not debugging
  const bool keep = !c.tc_st_fuse || c.cfg.debug;
  sa.AV = keep ? c.acc : nullptr;
  sa.BV = keep ? c.acc + c.d * c.k : nullptr;
  sa.dflag = c.dflag;
  const int nrt = (int)(b / 128);
  sa.fuse = c.tc_st_fuse;
  sa.V = c.V;
  sa.S = c.S;
  sa.terms = c.gram;
  sa.part = c.tc_part;
  sa.dbg = c.cfg.debug ? c.tc_dbg : nullptr;
  sa.grad_out = c.cfg.debug ? c.grad : nullptr;
  sa.Vt = c.tc_Vt;
  sa.d = c.d;
  sa.slot = (int)(c.t & 1);
  sa.rho = c.cfg.rho;
  sa.eta = eta;
  sa.gamma = gamma;
  sa.eps_B = c.cfg.eps_B;
  sa.terms_done = c.tc_st_cnt + 3 * nrt_max;
  sa.bar = c.tc_st_cnt + 3 * nrt_max + 1;
  sa.terms_target = (c.tc_st_epoch + 1) * (unsigned)(2 * nrt);
  sa.bar_base = c.tc_st_epoch * 2u * (unsigned)G;
  sa.trace = c.tc_st_trace;
  c.tc_st_nchunk = sa.nchunk;
  if (c.tc_st_trace)
    SGEP_CUDA_TRY(cudaMemsetAsync(c.tc_st_trace, 0,
                                  (size_t)c.num_sms * ((size_t)c.cfg.max_b / kR + 1) * kEv * sizeof(unsigned long long), s));
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
  ++c.tc_st_epoch;
  c.tc_st_updated = sa.fuse;  // the step's update is done; tc_update launches nothing
  c.tc_acc_stale = keep ? 0 : 1;
  ++c.launches;
  return SGEP_OK;
}

// SGEP_TRACE=1: per-chunk event times of the most recent streamed launch (stderr).
void tc_stream_trace_report(Ctx& c) {
  if (!c.tc_st_trace || !c.tc_st_nchunk) return;
  const int n = c.tc_st_grid, nc = c.tc_st_nchunk;
  std::vector<unsigned long long> t((size_t)n * (nc + 1) * kEv);
  if (cudaMemcpy(t.data(), c.tc_st_trace, t.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return;
  auto at = [&](int cta, int ch, int ev) { return t[((size_t)cta * (nc + 1) + ch) * kEv + ev]; };
  unsigned long long g0 = ~0ull;
  for (int b = 0; b < n; ++b) g0 = std::min(g0, at(b, nc, 0));
  auto row = [&](int ch, const char* const* names, int nev) {
    for (int ev = 0; ev < nev; ++ev) {
      std::vector<double> v;
      for (int b = 0; b < n; ++b)
        if (at(b, ch, ev) >= g0) v.push_back((at(b, ch, ev) - g0) / 1e3);
      std::sort(v.begin(), v.end());
      if (v.empty()) continue;
      std::fprintf(stderr, " %s %.2f/%.2f", names[ev], v[v.size() / 2], v.back());
    }
    std::fprintf(stderr, "\n");
  };
  const char* tot[8] = {"start", "proj", "backproj", "end", "terms", "upd1", "bar1", "bar2"};
  std::fprintf(stderr, "[sgep trace] streamed products, %d CTAs (%d helpers), %d chunks (us, median/max):", n,
               n - (int)(c.d_x / 128), nc);
  row(nc, tot, 8);
  const char* names[8] = {"issue", "mma", "release", "build0", "built", "Wseen", "bpdone", "terms"};
  for (int ch : {0, 1, 2, nc / 2, nc - 2, nc - 1}) {
    if (ch < 0 || ch >= nc) continue;
    std::fprintf(stderr, "[sgep trace]   chunk %2d:", ch);
    row(ch, names, 8);
  }
}

}  // namespace sgep

// Batching form: many independent SGEP instances (uneven d, k, kind, element type)
// advanced together, one step of every instance per call.
//
// Every instance is a generic-path handle. One step of the batch is eight phases,
// each a work list of tiles over all instances (the tile functions of the generic
// path, generic_tiles.cuh):
//   0 zero the instance's P/Q, products, k x k terms (and LDA W); LDA label counts
//   1 LDA class statistics
//   2 projection tiles             3 back-projection tiles (+ LDA W = M^T V tiles)
//   4 LDA A V from the class means 5 k x k terms
//   6 update and aux step          7 retraction
// Mode 0 runs all eight phases in one persistent cooperative launch with bounded grid
// barriers between phases; mode 1 launches one kernel per phase. The per-step
// descriptor table (row pointers, b, eta per instance) is copied from pinned host
// memory; the copy and the launch(es) can be captured in a CUDA graph and replayed.
// The work partition (projection chunk width, back-projection row-split height, mode
// and blocks per SM) is picked by sgep_batch_autotune, which times candidates on the
// device and caches the winner per batch signature.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "generic_tiles.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace sgep {

constexpr int kPhases = 8;

struct InstDesc {
  int kind, dtype, k, C, split, b_is_identity;
  int64_t d_x, d_y, d, b, nA, nrows_proj;  // nrows_proj: rows of the projection (LDA: B rows)
  float eta, gamma, rho, eps_B;
  const void* X;
  const void* Y;
  const float* sx;
  const float* sy;
  const int32_t* labels;
  float *V, *S, *Vtmp, *PQ, *acc, *gram, *grad;
  int* dflag;
  double *lda_sum, *lda_cnt;
  float *lda_mean, *lda_M, *lda_pi, *lda_W;
  // work partition
  int64_t chunk, rows_per_split;
  int nchunk_x, nchunk_y, row_tiles, nblk_x, nblk_y, bp_splits;
  int zero_items, stats_items, ldaw_items, ldaav_items, gram_items, upd_items, norm_items;
  int items[kPhases];
  int off[kPhases];  // first item of this instance in each phase
};

struct BatchHeader {
  int n;
  int total[kPhases];
  unsigned long long bar_base;  // barrier arrivals before this launch
  unsigned long long work_base[kPhases];  // persistent mode: items claimed per phase before this launch
};

namespace {

using gt::kThreads;
// the largest tile workspace: the back-projection's, or the LDA statistics' (C = 32)
constexpr int kSmemFloats = gt::cmax(gt::lda_stats_smem(kMaxClasses), gt::kBackprojectSmem);
static_assert(kSmemFloats >= gt::kBackprojectSmem && kSmemFloats >= gt::kProjectSmem &&
                  kSmemFloats >= gt::gram_smem(64) &&
                  kSmemFloats >= gt::update_smem(1) && kSmemFloats >= gt::update_smem(gt::kMaxK) &&
                  kSmemFloats >= gt::kLdaWSmem,
              "batch workspace");

constexpr int max_update_smem(int k = 1, int m = 0) {
  return k > gt::kMaxK ? m : max_update_smem(k + 1, gt::cmax(m, gt::update_smem(k)));
}
// Shared-memory floats of each phase's tiles: a launch of one phase asks for its own, so the
// phases with small workspaces keep more blocks resident.
constexpr int kPhaseSmemFloats[kPhases] = {gt::kLdaCountsSmem,
                                           gt::lda_stats_smem(kMaxClasses),
                                           gt::kProjectSmem,
                                           gt::cmax(gt::kBackprojectSmem, gt::kLdaWSmem),
                                           gt::kLdaAvSmem,
                                           gt::gram_smem(gt::kMaxK),
                                           max_update_smem(),
                                           0};
static_assert(gt::gram_smem(gt::kMaxK) >= gt::gram_smem(1), "the k x k terms' workspace grows with k");
static_assert(kSmemFloats >= max_update_smem(), "the persistent launch holds every phase's workspace");

__device__ int find_instance(const InstDesc* inst, int n, int phase, int item) {
  int lo = 0, hi = n - 1;  // last instance whose offset <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].off[phase] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__device__ __forceinline__ void run_typed(const InstDesc& I, int phase, int li, float* smem) {
  const T* X = static_cast<const T*>(I.X);
  const T* Y = static_cast<const T*>(I.Y);
  const bool lda = I.kind == SGEP_LDA;
  // LDA: the projection and the within-class back-projection run over the B rows
  const size_t xoff = lda ? (size_t)I.nA * I.d : 0;
  const int32_t* lab = lda ? I.labels + I.nA : nullptr;
  const float* sx = I.sx ? I.sx + (lda ? I.nA : 0) : nullptr;
  const gt::Centring cz{lda ? I.lda_mean : nullptr, lab, I.C, I.dflag};
  if (phase == 1) {
    gt::lda_stats_tile(X, I.sx, I.labels, I.b, I.d, I.C, I.lda_sum, I.lda_cnt, I.lda_mean, I.lda_M, li, smem);
  } else if (phase == 2) {
    const int bx = li % I.row_tiles, by = li / I.row_tiles;
    gt::project_tile(X + xoff, Y, I.nrows_proj, I.d_x, I.d_y, I.V, I.k, I.chunk, I.nchunk_x, I.PQ, cz, sx, I.sy, bx,
                     by, smem);
  } else if (phase == 3) {
    const int nbp = (I.nblk_x + I.nblk_y) * I.bp_splits;
    if (li < nbp) {
      const int bx = li % (I.nblk_x + I.nblk_y), by = li / (I.nblk_x + I.nblk_y);
      const float inv_nA = 1.f / (float)I.nA;
      const float inv_nB = 1.f / (float)(lda ? I.nrows_proj : (I.split ? I.b - I.nA : I.b));
      gt::backproject_tile(X + xoff, Y, I.nrows_proj, I.d_x, I.d_y, lda ? 0 : I.nA, I.kind, I.split, I.PQ, I.k,
                           I.nblk_x, I.rows_per_split, inv_nA, inv_nB, I.acc, I.acc + I.d * I.k, cz, sx, I.sy, bx,
                           by, smem);
    } else {
      gt::lda_w_tile(I.lda_M, I.V, I.d, I.C, I.k, I.lda_W, li - nbp, I.ldaw_items, smem);
    }
  }
}

// Element type of every instance's rows, fixed at compile time when a batch is uniform (FP32 or
// BF16 rows: only that type's tiles are compiled into the kernels, which keeps them within their
// register budget), or kAnyRows: chosen per instance.
constexpr int kAnyRows = -1;

template <int DT>
__device__ __forceinline__ void run_rows(const InstDesc& I, int phase, int li, float* smem) {
  if constexpr (DT == SGEP_F32) {
    run_typed<float>(I, phase, li, smem);
  } else if constexpr (DT == SGEP_BF16) {
    run_typed<__nv_bfloat16>(I, phase, li, smem);
  } else {
    if (I.dtype == SGEP_BF16) run_typed<__nv_bfloat16>(I, phase, li, smem);
    else if (I.dtype == SGEP_FP8E4M3) run_typed<__nv_fp8_e4m3>(I, phase, li, smem);
    else run_typed<float>(I, phase, li, smem);
  }
}

template <int DT>
__device__ __forceinline__ void run_item(const InstDesc& I, int phase, int li, float* smem) {
  switch (phase) {
    case 0: {
      if (I.kind == SGEP_LDA && li == I.zero_items) {  // the label counts tile
        gt::lda_counts_tile(I.labels, I.b, I.C, I.lda_cnt, I.lda_pi, I.dflag, smem);
        return;
      }
      // zero P/Q rows, products, k x k terms and W: one contiguous span of each
      const int64_t npq = I.nrows_proj * 2 * I.k, nacc = 2 * I.d * I.k, ngr = 2 * (int64_t)I.k * I.k + 2 * I.k;
      const int64_t nw = I.kind == SGEP_LDA ? (int64_t)I.C * I.k : 0;
      const int64_t total = npq + nacc + ngr + nw;
      for (int64_t e = (int64_t)li * kThreads + threadIdx.x; e < total; e += (int64_t)I.zero_items * kThreads) {
        if (e < npq) I.PQ[e] = 0.f;
        else if (e < npq + nacc) I.acc[e - npq] = 0.f;
        else if (e < npq + nacc + ngr) I.gram[e - npq - nacc] = 0.f;
        else I.lda_W[e - npq - nacc - ngr] = 0.f;
      }
      return;
    }
    case 1:
    case 2:
    case 3:
      run_rows<DT>(I, phase, li, smem);
      return;
    case 4:
      gt::lda_av_tile(I.lda_M, I.lda_pi, I.lda_W, I.d, I.C, I.k, I.acc, li, I.ldaav_items, smem);
      return;
    case 5:
      gt::gram_tile(I.V, I.S, I.acc, I.acc + I.d * I.k, I.d, I.k, I.eps_B, I.b_is_identity, I.gram, li, I.gram_items,
                    smem);
      return;
    case 6:
      gt::update_tile(I.V, I.S, I.acc, I.acc + I.d * I.k, I.gram, I.d, I.k, I.eta, I.gamma, I.rho, I.eps_B,
                      I.b_is_identity, I.Vtmp, I.grad, li, I.upd_items, smem);
      return;
    default:
      gt::normalize_tile(I.Vtmp, I.gram, I.V, I.d, I.k, I.dflag, li, I.norm_items);
      return;
  }
}

template <int DT>
__device__ __forceinline__ void run_phase(const BatchHeader* h, const InstDesc* inst, int phase, float* smem) {
  const int total = h->total[phase];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int i = find_instance(inst, h->n, phase, it);
    run_item<DT>(inst[i], phase, it - inst[i].off[phase], smem);
    __syncthreads();  // the workspace is reused by the next item
  }
}

// One launch per phase: one kernel per phase (and, for the phases that read rows, per element
// type of a uniform batch), so each is compiled (registers, spills) for its own tiles only.
template <int P, int DT>
__global__ void __launch_bounds__(kThreads, 2) k_batch_phase(const BatchHeader* __restrict__ h,
                                                          const InstDesc* __restrict__ inst) {
  extern __shared__ __align__(16) float smem[];
  run_phase<DT>(h, inst, P, smem);
}

// only phases 1-3 read rows; the others have one kernel whatever the element type
constexpr int phase_rows(int P, int DT) { return (P >= 1 && P <= 3) ? DT : kAnyRows; }

template <int DT, int P = 0>
void set_phase_smem(int smem) {
  if constexpr (P < kPhases) {
    cudaFuncSetAttribute(k_batch_phase<P, phase_rows(P, DT)>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    set_phase_smem<DT, P + 1>(smem);
  }
}

template <int DT, int P = 0>
void launch_phase(int phase, unsigned grid, size_t smem, cudaStream_t s, const BatchHeader* dh,
                  const InstDesc* di) {
  if constexpr (P < kPhases) {
    if (phase == P) k_batch_phase<P, phase_rows(P, DT)><<<grid, kThreads, smem, s>>>(dh, di);
    else launch_phase<DT, P + 1>(phase, grid, smem, s, dh, di);
  }
}

// Persistent mode: the blocks claim a phase's items one at a time from a counter (monotone
// across launches; each block ends a phase with one claim past the last item), so items of
// uneven cost spread over the blocks as they finish.
template <int DT>
__device__ void run_phase_claimed(const BatchHeader* h, const InstDesc* inst, int phase, float* smem,
                                  unsigned long long* work, int* it_s) {
  const int total = h->total[phase];
  const unsigned long long base = h->work_base[phase];
  for (;;) {
    if (threadIdx.x == 0) *it_s = (int)min(atomicAdd(work + phase, 1ull) - base, (unsigned long long)total);
    __syncthreads();
    const int it = *it_s;
    if (it >= total) break;
    const int i = find_instance(inst, h->n, phase, it);
    run_item<DT>(inst[i], phase, it - inst[i].off[phase], smem);
    __syncthreads();  // the workspace and the claimed index are reused by the next item
  }
}

template <int DT>
__global__ void __launch_bounds__(kThreads, 2) k_batch_persistent(const BatchHeader* __restrict__ h,
                                                               const InstDesc* __restrict__ inst,
                                                               unsigned long long* bar, int* dflag) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int ok_s;
  __shared__ int it_s;
  const unsigned long long base = h->bar_base;
  for (int phase = 0; phase < kPhases; ++phase) {
    run_phase_claimed<DT>(h, inst, phase, smem, bar + 1, &it_s);
    if (phase + 1 == kPhases) break;
    // bounded grid barrier: arrivals are counted monotonically across launches
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(bar, 1ull);
      ok_s = tc::spin_until_geq64(bar, base + (unsigned long long)(phase + 1) * gridDim.x) ? 1 : 0;
      if (!ok_s) atomicOr(dflag, kFlagTimeout);
    }
    __syncthreads();
    if (!ok_s) return;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side

struct BatchTuning {
  int mode = 0;           // 0 persistent, 1 one launch per phase
  int blocks_per_sm = 2;  // persistent grid
  int chunk_cap = 1024;   // projection chunk width (columns)
  int rows_cap = 128;     // back-projection row-split height
};

struct BatchCtx {
  std::vector<Ctx*> h;
  int n = 0, num_sms = 0, device = 0, max_pers_blocks = 0;
  int rows_dt = kAnyRows;  // SGEP_F32 or SGEP_BF16 when every instance's rows have that type
  BatchTuning tune;
  int use_graph = 0;
  // pinned descriptor tables (two, alternating) and their device copies
  char* host_tab[2] = {nullptr, nullptr};
  char* dev_tab[2] = {nullptr, nullptr};
  size_t tab_bytes = 0;
  cudaEvent_t done[2] = {nullptr, nullptr};
  int cur = 0;
  unsigned long long* bar = nullptr;  // [1 + kPhases]: grid-barrier arrivals, then the phases' claims
  unsigned long long bar_base = 0;
  unsigned long long work_base[kPhases] = {};
  int* dflag = nullptr;  // batch-level flag (barrier timeouts)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_key[2] = {-1, -1};  // launch-shape key the graph was captured for
  int64_t launches = 0;
};

static void destroy_graphs(BatchCtx& B) {
  for (int j = 0; j < 2; ++j) {
    if (B.graph[j]) cudaGraphExecDestroy(B.graph[j]);
    B.graph[j] = nullptr;
    B.graph_key[j] = -1;
  }
}

void batch_free(BatchCtx* B) {
  if (!B) return;
  cudaDeviceSynchronize();
  destroy_graphs(*B);
  for (int j = 0; j < 2; ++j) {
    cudaFreeHost(B->host_tab[j]);
    cudaFree(B->dev_tab[j]);
    if (B->done[j]) cudaEventDestroy(B->done[j]);
  }
  cudaFree(B->bar);
  cudaFree(B->dflag);
  delete B;
}

int batch_create(Ctx** hs, int n, BatchCtx** out) {
  auto* B = new (std::nothrow) BatchCtx();
  if (!B) return SGEP_ENOMEM;
  B->h.assign(hs, hs + n);
  B->n = n;
  B->device = hs[0]->device;
  B->num_sms = hs[0]->num_sms;
  B->tab_bytes = sizeof(BatchHeader) + 64 + (size_t)n * sizeof(InstDesc);
  for (int j = 0; j < 2; ++j) {
    if (cudaHostAlloc((void**)&B->host_tab[j], B->tab_bytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaMalloc((void**)&B->dev_tab[j], B->tab_bytes) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->done[j], cudaEventDisableTiming) != cudaSuccess) {
      batch_free(B);
      return SGEP_ENOMEM;
    }
  }
  if (cudaMalloc((void**)&B->bar, (1 + kPhases) * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc((void**)&B->dflag, sizeof(int)) != cudaSuccess) {
    batch_free(B);
    return SGEP_ENOMEM;
  }
  cudaMemset(B->bar, 0, (1 + kPhases) * sizeof(unsigned long long));
  cudaMemset(B->dflag, 0, sizeof(int));
  B->rows_dt = hs[0]->cfg.dtype;
  for (int i = 1; i < n; ++i)
    if (hs[i]->cfg.dtype != B->rows_dt) B->rows_dt = kAnyRows;
  if (B->rows_dt != SGEP_F32 && B->rows_dt != SGEP_BF16) B->rows_dt = kAnyRows;
  const size_t smem = (size_t)kSmemFloats * sizeof(float);
  int per_sm = 0;
  cudaError_t occ;
  if (B->rows_dt == SGEP_F32) {
    set_phase_smem<SGEP_F32>((int)smem);
    cudaFuncSetAttribute(k_batch_persistent<SGEP_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    occ = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent<SGEP_F32>, kThreads, smem);
  } else if (B->rows_dt == SGEP_BF16) {
    set_phase_smem<SGEP_BF16>((int)smem);
    cudaFuncSetAttribute(k_batch_persistent<SGEP_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    occ = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent<SGEP_BF16>, kThreads, smem);
  } else {
    set_phase_smem<kAnyRows>((int)smem);
    cudaFuncSetAttribute(k_batch_persistent<kAnyRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    occ = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent<kAnyRows>, kThreads, smem);
  }
  if (occ != cudaSuccess) per_sm = 1;
  cudaGetLastError();
  B->max_pers_blocks = std::max(1, per_sm);
  B->tune.blocks_per_sm = std::min(2, B->max_pers_blocks);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    batch_free(B);
    return SGEP_ECUDA;
  }
  *out = B;
  return SGEP_OK;
}

// Work partition of one instance for `b` rows, and its item counts per phase.
static void partition(const BatchCtx& B, const Ctx& c, int64_t b, InstDesc& D) {
  const int kind = c.cfg.kind;
  const bool lda = kind == SGEP_LDA;
  D.kind = kind;
  D.dtype = c.cfg.dtype;
  D.k = c.k;
  D.C = lda ? c.cfg.n_classes : 0;
  D.split = ((kind == SGEP_CCA || lda) && c.cfg.split_AB) ? 1 : 0;
  D.b_is_identity = c.b_is_identity ? 1 : 0;
  D.d_x = c.d_x;
  D.d_y = c.has_y ? c.d_y : 0;
  D.d = c.d;
  D.b = b;
  D.nA = D.split ? b / 2 : (lda ? 0 : b);
  D.nrows_proj = lda ? b - D.nA : b;
  D.row_tiles = (int)((D.nrows_proj + gt::kProjRows - 1) / gt::kProjRows);
  int64_t chunk = B.tune.chunk_cap;
  // keep a few column chunks per row tile so that small-b instances still spread out
  while (chunk > 64 && (int64_t)D.row_tiles * ((c.d + chunk - 1) / chunk) < 8) chunk /= 2;
  D.chunk = chunk;
  D.nchunk_x = (int)((D.d_x + chunk - 1) / chunk);
  D.nchunk_y = c.has_y ? (int)((D.d_y + chunk - 1) / chunk) : 0;
  D.nblk_x = (int)((D.d_x + 63) / 64);
  D.nblk_y = c.has_y ? (int)((D.d_y + 63) / 64) : 0;
  D.rows_per_split = std::max<int64_t>(32, ((int64_t)B.tune.rows_cap + 31) / 32 * 32);
  D.bp_splits = (int)std::max<int64_t>(1, (D.nrows_proj + D.rows_per_split - 1) / D.rows_per_split);
  const int64_t zero_floats =
      D.nrows_proj * 2 * c.k + 2 * c.d * c.k + 2 * (int64_t)c.k * c.k + 2 * c.k + (lda ? (int64_t)D.C * c.k : 0);
  D.zero_items = (int)std::max<int64_t>(1, (zero_floats + 8 * kThreads - 1) / (8 * kThreads));
  D.stats_items = lda ? (int)((c.d + kThreads - 1) / kThreads) : 0;
  D.ldaw_items = lda ? (int)std::max<int64_t>(1, std::min<int64_t>((c.d + 31) / 32, 16)) : 0;
  D.ldaav_items = lda ? (int)std::max<int64_t>(1, std::min<int64_t>((c.d * c.k + kThreads - 1) / kThreads, 32)) : 0;
  D.gram_items = (int)std::max<int64_t>(1, std::min<int64_t>((c.d + 31) / 32, 32));
  const int64_t span = (int64_t)std::max(1, kThreads / c.k) * gt::kUpdRows;
  D.upd_items = (int)std::max<int64_t>(1, std::min<int64_t>((c.d + span - 1) / span, 32));
  D.norm_items = (int)std::max<int64_t>(1, std::min<int64_t>((c.d * c.k + kThreads - 1) / kThreads, 32));
  D.items[0] = D.zero_items + (lda ? 1 : 0);
  D.items[1] = D.stats_items;
  D.items[2] = D.row_tiles * (D.nchunk_x + D.nchunk_y);
  D.items[3] = (D.nblk_x + D.nblk_y) * D.bp_splits + D.ldaw_items;
  D.items[4] = D.ldaav_items;
  D.items[5] = D.gram_items;
  D.items[6] = D.upd_items;
  D.items[7] = D.norm_items;
}

// Fill the pinned table for this step; returns the launch-shape key (item totals).
static int fill_table(BatchCtx& B, char* tab, const void* const* X, const void* const* Y, const float* const* sx,
                      const float* const* sy, const int32_t* const* labels, const int64_t* b) {
  auto* hd = reinterpret_cast<BatchHeader*>(tab);
  auto* inst = reinterpret_cast<InstDesc*>(tab + ((sizeof(BatchHeader) + 63) / 64) * 64);
  std::memset(hd, 0, sizeof(BatchHeader));
  hd->n = B.n;
  for (int i = 0; i < B.n; ++i) {
    Ctx& c = *B.h[i];
    InstDesc& D = inst[i];
    std::memset(&D, 0, sizeof(D));
    partition(B, c, b[i], D);
    D.eta = (float)schedule_eta(c.cfg, c.t + 1);
    D.gamma = c.cfg.gamma0;
    D.rho = c.cfg.rho;
    D.eps_B = c.cfg.eps_B;
    D.X = X[i];
    D.Y = Y ? Y[i] : nullptr;
    D.sx = sx ? sx[i] : nullptr;
    D.sy = sy ? sy[i] : nullptr;
    D.labels = labels ? labels[i] : nullptr;
    D.V = c.V;
    D.S = c.S;
    D.Vtmp = c.Vtmp;
    D.PQ = c.PQ;
    D.acc = c.acc;
    D.gram = c.gram;
    D.grad = c.cfg.debug ? c.grad : nullptr;
    D.dflag = c.dflag;
    D.lda_sum = c.lda_sum;
    D.lda_cnt = c.lda_cnt;
    D.lda_mean = c.lda_mean;
    D.lda_M = c.lda_M;
    D.lda_pi = c.lda_pi;
    D.lda_W = c.lda_W;
    for (int p = 0; p < kPhases; ++p) {
      D.off[p] = hd->total[p];
      hd->total[p] += D.items[p];
    }
  }
  hd->bar_base = B.bar_base;
  for (int p = 0; p < kPhases; ++p) hd->work_base[p] = B.work_base[p];
  int key = B.tune.mode * 7919 + B.tune.blocks_per_sm;
  for (int p = 0; p < kPhases; ++p) key = key * 31 + hd->total[p];
  return key;
}

// Enqueue the table copy and the launch(es) of one step on `s`.
static int enqueue_step(BatchCtx& B, int j, cudaStream_t s) {
  const auto* hd = reinterpret_cast<const BatchHeader*>(B.host_tab[j]);
  const BatchHeader* dh = reinterpret_cast<const BatchHeader*>(B.dev_tab[j]);
  const InstDesc* di = reinterpret_cast<const InstDesc*>(B.dev_tab[j] + ((sizeof(BatchHeader) + 63) / 64) * 64);
  SGEP_CUDA_TRY(cudaMemcpyAsync(B.dev_tab[j], B.host_tab[j], B.tab_bytes, cudaMemcpyHostToDevice, s));
  const size_t smem = (size_t)kSmemFloats * sizeof(float);
  if (B.tune.mode == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(B.tune.blocks_per_sm * B.num_sms));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (B.rows_dt == SGEP_F32)
      SGEP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_batch_persistent<SGEP_F32>, dh, di, B.bar, B.dflag));
    else if (B.rows_dt == SGEP_BF16)
      SGEP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_batch_persistent<SGEP_BF16>, dh, di, B.bar, B.dflag));
    else
      SGEP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_batch_persistent<kAnyRows>, dh, di, B.bar, B.dflag));
    ++B.launches;
  } else {
    for (int p = 0; p < kPhases; ++p) {
      if (hd->total[p] == 0) continue;
      const unsigned grid = (unsigned)std::min(hd->total[p], 8 * B.num_sms);
      const size_t psm = (size_t)kPhaseSmemFloats[p] * sizeof(float);
      if (B.rows_dt == SGEP_F32) launch_phase<SGEP_F32>(p, grid, psm, s, dh, di);
      else if (B.rows_dt == SGEP_BF16) launch_phase<SGEP_BF16>(p, grid, psm, s, dh, di);
      else launch_phase<kAnyRows>(p, grid, psm, s, dh, di);
      SGEP_CUDA_TRY(cudaGetLastError());
      ++B.launches;
    }
  }
  return SGEP_OK;
}

int batch_step(BatchCtx& B, const void* const* X, const void* const* Y, const float* const* sx,
               const float* const* sy, const int32_t* const* labels, const int64_t* b, cudaStream_t s) {
  const int j = B.cur;
  B.cur ^= 1;
  // the table j was last read by the launch two steps back
  SGEP_CUDA_TRY(cudaEventSynchronize(B.done[j]));
  const int key = fill_table(B, B.host_tab[j], X, Y, sx, sy, labels, b);
  if (B.use_graph) {
    if (!B.graph[j] || B.graph_key[j] != key) {
      if (B.graph[j]) cudaGraphExecDestroy(B.graph[j]);
      B.graph[j] = nullptr;
      cudaStream_t cs;
      SGEP_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      const int64_t counted = B.launches;  // capturing launches nothing
      int rc = e == cudaSuccess ? enqueue_step(B, j, cs) : SGEP_ECUDA;
      B.launches = counted;
      cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      if (rc == SGEP_OK && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&B.graph[j], g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (rc) return rc;
      SGEP_CUDA_TRY(e2);
      B.graph_key[j] = key;
    }
    SGEP_CUDA_TRY(cudaGraphLaunch(B.graph[j], s));
    const auto* hd = reinterpret_cast<const BatchHeader*>(B.host_tab[j]);
    if (B.tune.mode == 0) {
      B.launches += 1;
    } else {
      for (int p = 0; p < kPhases; ++p) B.launches += hd->total[p] > 0 ? 1 : 0;
    }
  } else {
    int rc = enqueue_step(B, j, s);
    if (rc) return rc;
  }
  SGEP_CUDA_TRY(cudaEventRecord(B.done[j], s));
  if (B.tune.mode == 0) {
    const unsigned long long grid = (unsigned long long)B.tune.blocks_per_sm * B.num_sms;
    B.bar_base += (unsigned long long)(kPhases - 1) * grid;
    const auto* hd = reinterpret_cast<const BatchHeader*>(B.host_tab[j]);
    for (int p = 0; p < kPhases; ++p) B.work_base[p] += (unsigned long long)hd->total[p] + grid;
  }
  for (auto* c : B.h) {
    c->t += 1;
    c->debug_valid = c->cfg.debug;
  }
  return SGEP_OK;
}

int batch_sync(BatchCtx& B, cudaStream_t s) {
  SGEP_CUDA_TRY(cudaStreamSynchronize(s));
  int flag = 0;
  SGEP_CUDA_TRY(cudaMemcpy(&flag, B.dflag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    SGEP_CUDA_TRY(cudaMemset(B.dflag, 0, sizeof(int)));
    // the counts may be short
    SGEP_CUDA_TRY(cudaMemset(B.bar, 0, (1 + kPhases) * sizeof(unsigned long long)));
    B.bar_base = 0;
    for (auto& w : B.work_base) w = 0;
    return SGEP_ETIMEOUT;
  }
  return SGEP_OK;
}

void batch_set(BatchCtx& B, int mode, int blocks_per_sm, int chunk_cap, int rows_cap, int use_graph) {
  if (mode >= 0) B.tune.mode = mode ? 1 : 0;
  if (blocks_per_sm > 0) B.tune.blocks_per_sm = std::min(blocks_per_sm, B.max_pers_blocks);
  if (chunk_cap > 0) B.tune.chunk_cap = std::max(64, std::min(chunk_cap, 4096));
  if (rows_cap > 0) B.tune.rows_cap = std::max(32, std::min(rows_cap, 1 << 20));
  if (use_graph >= 0) B.use_graph = use_graph ? 1 : 0;
  destroy_graphs(B);
}

void batch_get(const BatchCtx& B, int* out5) {
  out5[0] = B.tune.mode;
  out5[1] = B.tune.blocks_per_sm;
  out5[2] = B.tune.chunk_cap;
  out5[3] = B.tune.rows_cap;
  out5[4] = B.use_graph;
}

int64_t batch_launches(const BatchCtx& B) { return B.launches; }

// Times candidates on the device (state saved first and restored after) and keeps the
// fastest; winners are cached per batch signature (kind, dtype, d_x, d_y, k, b of every
// instance) for the life of the process.
int batch_autotune(BatchCtx& B, const void* const* X, const void* const* Y, const float* const* sx,
                   const float* const* sy, const int32_t* const* labels, const int64_t* b, int reps, int* best5) {
  static std::mutex mu;
  static std::map<std::string, BatchTuning> cache;
  std::string sig;
  for (int i = 0; i < B.n; ++i) {
    const Ctx& c = *B.h[i];
    sig += std::to_string(c.cfg.kind) + "," + std::to_string(c.cfg.dtype) + "," + std::to_string(c.d_x) + "," +
           std::to_string(c.d_y) + "," + std::to_string(c.k) + "," + std::to_string(b[i]) + ";";
  }
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(sig);
    if (it != cache.end()) {
      B.tune = it->second;
      destroy_graphs(B);
      batch_get(B, best5);
      return SGEP_OK;
    }
  }
  reps = std::max(1, reps);
  // save the state every step changes (V, [Bv], step count, LDA statistics)
  std::vector<float*> save_vs(B.n, nullptr);
  std::vector<double*> save_lda(B.n, nullptr);
  std::vector<int64_t> save_t(B.n);
  int rc = SGEP_OK;
  for (int i = 0; i < B.n && !rc; ++i) {
    Ctx& c = *B.h[i];
    const size_t dk = (size_t)c.d * c.k;
    if (cudaMalloc((void**)&save_vs[i], 2 * dk * sizeof(float)) != cudaSuccess) rc = SGEP_ENOMEM;
    if (!rc) {
      cudaMemcpy(save_vs[i], c.V, dk * sizeof(float), cudaMemcpyDeviceToDevice);
      cudaMemcpy(save_vs[i] + dk, c.S, dk * sizeof(float), cudaMemcpyDeviceToDevice);
    }
    if (!rc && c.cfg.kind == SGEP_LDA) {
      const size_t cd = (size_t)c.cfg.n_classes * c.d;
      if (cudaMalloc((void**)&save_lda[i], (cd + c.cfg.n_classes) * sizeof(double)) != cudaSuccess) rc = SGEP_ENOMEM;
      if (!rc) {
        cudaMemcpy(save_lda[i], c.lda_sum, cd * sizeof(double), cudaMemcpyDeviceToDevice);
        cudaMemcpy(save_lda[i] + cd, c.lda_cnt, c.cfg.n_classes * sizeof(double), cudaMemcpyDeviceToDevice);
      }
    }
    save_t[i] = c.t;
  }
  const BatchTuning start = B.tune;
  const int graph_was = B.use_graph;
  BatchTuning best = start;
  float best_ms = 1e30f;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
              cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = SGEP_ECUDA;
  std::vector<BatchTuning> cands;
  for (int mode = 0; mode < 2; ++mode)
    for (int chunk : {256, 512, 1024})
      for (int rows : {64, 128, 256})
        for (int bps : {1, 2, 4}) {
          if (mode == 1 && bps != 1) continue;
          if (mode == 0 && bps > B.max_pers_blocks) continue;
          BatchTuning t;
          t.mode = mode;
          t.blocks_per_sm = mode == 0 ? bps : start.blocks_per_sm;
          t.chunk_cap = chunk;
          t.rows_cap = rows;
          cands.push_back(t);
        }
  for (const BatchTuning& t : cands) {
    if (rc) break;
    B.tune = t;
    destroy_graphs(B);
    rc = batch_step(B, X, Y, sx, sy, labels, b, s);  // warm-up (and graph capture)
    for (int r = 0; r < reps && !rc; ++r) {
      if (r == 0) cudaEventRecord(e0, s);
      rc = batch_step(B, X, Y, sx, sy, labels, b, s);
    }
    if (rc) break;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = SGEP_ECUDA;
      break;
    }
    rc = batch_sync(B, s);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (!rc && ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  // restore the state
  for (int i = 0; i < B.n; ++i) {
    Ctx& c = *B.h[i];
    const size_t dk = (size_t)c.d * c.k;
    if (save_vs[i]) {
      cudaMemcpy(c.V, save_vs[i], dk * sizeof(float), cudaMemcpyDeviceToDevice);
      cudaMemcpy(c.S, save_vs[i] + dk, dk * sizeof(float), cudaMemcpyDeviceToDevice);
      cudaFree(save_vs[i]);
    }
    if (save_lda[i]) {
      const size_t cd = (size_t)c.cfg.n_classes * c.d;
      cudaMemcpy(c.lda_sum, save_lda[i], cd * sizeof(double), cudaMemcpyDeviceToDevice);
      cudaMemcpy(c.lda_cnt, save_lda[i] + cd, c.cfg.n_classes * sizeof(double), cudaMemcpyDeviceToDevice);
      cudaFree(save_lda[i]);
      lda_refresh(c, nullptr);
    }
    c.t = save_t[i];
    c.debug_valid = 0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaDeviceSynchronize();
  B.tune = rc ? start : best;
  B.use_graph = graph_was;
  destroy_graphs(B);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(mu);
    cache[sig] = best;
  }
  batch_get(B, best5);
  return SGEP_OK;
}

}  // namespace sgep

// ---------------------------------------------------------------------------
// C ABI (declared in include/sgep.h)

struct sgep_batch_ctx {
  sgep::BatchCtx* impl;
};

namespace {

int batch_fail(int status, const char* msg) {
  sgep::set_error(msg);
  return status;
}

// Per-instance argument checks of one batch step (the same rules as sgep_step).
int check_rows(const sgep::BatchCtx& B, const void* const* X, const void* const* Y, const float* const* sx,
               const float* const* sy, const int32_t* const* labels, const int64_t* rows) {
  if (!X || !rows) return batch_fail(SGEP_EINVAL, "X and rows arrays are required");
  for (int i = 0; i < B.n; ++i) {
    const sgep::Ctx& c = *B.h[i];
    if (!X[i]) return batch_fail(SGEP_EINVAL, "X[i] is NULL");
    if (c.has_y && (!Y || !Y[i])) return batch_fail(SGEP_EINVAL, "Y[i] is NULL for a two-view instance");
    if (c.cfg.kind == SGEP_LDA && (!labels || !labels[i])) return batch_fail(SGEP_EINVAL, "LDA needs labels");
    const bool fp8 = c.cfg.dtype == SGEP_FP8E4M3;
    const float* a = sx ? sx[i] : nullptr;
    const float* b2 = sy ? sy[i] : nullptr;
    if (fp8 && (!a || (c.has_y && !b2))) return batch_fail(SGEP_EINVAL, "FP8 rows need their row scales");
    if (!fp8 && (a || b2)) return batch_fail(SGEP_EINVAL, "row scales are for FP8 rows only");
    const bool split = (c.cfg.kind == SGEP_CCA || c.cfg.kind == SGEP_LDA) && c.cfg.split_AB;
    if (rows[i] < (split ? 2 : 1) || rows[i] > c.cfg.max_b) return batch_fail(SGEP_EINVAL, "rows[i] out of range");
  }
  return SGEP_OK;
}

}  // namespace

extern "C" {

int sgep_batch_create(const sgep_t* handles, int n, sgep_batch_t* out) {
  if (!out) return batch_fail(SGEP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!handles || n < 1) return batch_fail(SGEP_EINVAL, "need n >= 1 handles");
  std::vector<sgep::Ctx*> hs(n);
  for (int i = 0; i < n; ++i) {
    if (!handles[i]) return batch_fail(SGEP_EINVAL, "handle is NULL");
    hs[i] = handles[i];
    if (hs[i]->path != SGEP_PATH_GENERIC)
      return batch_fail(SGEP_EINVAL, "batched instances must be created with path = SGEP_PATH_GENERIC");
    if (hs[i]->cfg.kind == SGEP_ICA) return batch_fail(SGEP_ENOTSUP, "batched instances cannot be ICA");
    if (hs[i]->adam_m || hs[i]->z || hs[i]->cen_sum)
      return batch_fail(SGEP_ENOTSUP, "batched instances take Alg. 2's plain step (no Adam, Alg. 3 or centring)");
    if (hs[i]->device != hs[0]->device) return batch_fail(SGEP_EINVAL, "instances on different devices");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return batch_fail(SGEP_EINVAL, "a handle appears twice");
    int rc = sgep_sync(handles[i], nullptr);  // no pending work or unreported error
    if (rc) return rc;
  }
  auto* w = new (std::nothrow) sgep_batch_ctx();
  if (!w) return batch_fail(SGEP_ENOMEM, "host allocation failed");
  int rc = sgep::batch_create(hs.data(), n, &w->impl);
  if (rc) {
    delete w;
    return batch_fail(rc, "batch allocation failed");
  }
  *out = w;
  return SGEP_OK;
}

int sgep_batch_destroy(sgep_batch_t b) {
  if (!b) return SGEP_OK;
  sgep::batch_free(b->impl);
  delete b;
  return SGEP_OK;
}

int sgep_batch_step(sgep_batch_t b, const void* const* X, const void* const* Y, const float* const* row_scale_x,
                    const float* const* row_scale_y, const int32_t* const* labels, const int64_t* rows,
                    void* stream) {
  if (!b) return batch_fail(SGEP_EINVAL, "batch is NULL");
  int rc = check_rows(*b->impl, X, Y, row_scale_x, row_scale_y, labels, rows);
  if (rc) return rc;
  return sgep::batch_step(*b->impl, X, Y, row_scale_x, row_scale_y, labels, rows, (cudaStream_t)stream);
}

int sgep_batch_sync(sgep_batch_t b, void* stream) {
  if (!b) return batch_fail(SGEP_EINVAL, "batch is NULL");
  int rc = sgep::batch_sync(*b->impl, (cudaStream_t)stream);
  if (rc) return batch_fail(rc, "a bounded grid barrier of the batched launch gave up");
  for (auto* c : b->impl->h) {
    rc = sgep_sync(static_cast<sgep_t>(c), stream);
    if (rc) return rc;
  }
  return SGEP_OK;
}

int sgep_batch_configure(sgep_batch_t b, int mode, int blocks_per_sm, int chunk_cap, int rows_cap, int use_graph) {
  if (!b) return batch_fail(SGEP_EINVAL, "batch is NULL");
  if (mode > 1 || blocks_per_sm > 64 || chunk_cap > 4096 || use_graph > 1)
    return batch_fail(SGEP_EINVAL, "configuration value out of range");
  int rc = sgep_batch_sync(b, nullptr);
  if (rc) return rc;
  sgep::batch_set(*b->impl, mode, blocks_per_sm, chunk_cap, rows_cap, use_graph);
  return SGEP_OK;
}

int sgep_batch_get_config(sgep_batch_t b, int* out5) {
  if (!b || !out5) return batch_fail(SGEP_EINVAL, "NULL argument");
  sgep::batch_get(*b->impl, out5);
  return SGEP_OK;
}

int sgep_batch_autotune(sgep_batch_t b, const void* const* X, const void* const* Y, const float* const* row_scale_x,
                        const float* const* row_scale_y, const int32_t* const* labels, const int64_t* rows, int reps,
                        int* out5) {
  if (!b || !out5) return batch_fail(SGEP_EINVAL, "NULL argument");
  int rc = check_rows(*b->impl, X, Y, row_scale_x, row_scale_y, labels, rows);
  if (rc) return rc;
  rc = sgep_batch_sync(b, nullptr);
  if (rc) return rc;
  rc = sgep::batch_autotune(*b->impl, X, Y, row_scale_x, row_scale_y, labels, rows, reps, out5);
  if (rc) return batch_fail(rc, "autotuning failed");
  return sgep_batch_sync(b, nullptr);
}

int64_t sgep_batch_launch_count(sgep_batch_t b) { return b ? sgep::batch_launches(*b->impl) : -1; }

}  // extern "C"

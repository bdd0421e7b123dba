// Internal declarations shared by the host-side ABI and the kernel files.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sgep.h"

namespace sgep {

// Per-handle device state. All device buffers are allocated once by sgep_init.
// Variant parameters of one update (Adam on the players, App. H.2.2; smooth
// denominators, Alg. 3). Null pointers select Alg. 2's plain step / clipping.
struct UpdVariant {
  float* m = nullptr;  // d x k Adam moments (read and written)
  float* s = nullptr;
  float b1 = 0.f, b2 = 0.f, eps = 0.f;
  float bc1 = 1.f, bc2 = 1.f;  // 1 - b1^t, 1 - b2^t for this step
  float* z = nullptr;  // k scalars of Alg. 3 (updated after the step)
  float log_rho = 0.f, log_nu = 0.f;
};

struct Ctx {
  sgep_config cfg;
  int64_t d_x = 0, d_y = 0, d = 0;
  int k = 0;
  int path = SGEP_PATH_GENERIC;
  int device = 0;
  int num_sms = 0;
  bool b_is_identity = false;  // PCA, PLS
  bool has_y = false;          // CCA, PLS

  float* V = nullptr;      // d x k, player vectors v_i (columns)
  float* S = nullptr;      // d x k, auxiliary variables [Bv]_i
  float* Vtmp = nullptr;   // d x k, v_i + eta grad_i before the retraction
  float* PQ = nullptr;     // max_b x 2k, row projections [X V_x | Y V_y]
  float* acc = nullptr;    // 2 x d x k: A_t V then B_t V
  float* gram = nullptr;   // k*k (a_ij), k*k (G_ij), k (b_i), k (norms^2)
  float* grad = nullptr;   // d x k update directions (debug only)
  double* rq = nullptr;    // 2k doubles: Rayleigh numerator / denominator sums
  int* dflag = nullptr;    // device error word: bit 0 non-finite, bit 1 timeout
  float* adam_m = nullptr; // Adam: d x k first moments, then (adam_s) d x k second moments
  float* adam_s = nullptr;
  int64_t adam_t = 0;      // Adam steps since the moments were last reset
  float* z = nullptr;      // Alg. 3: k scalars z_i
  float* ica_buf = nullptr;  // ICA: row norms (max_b) | weighted projections (max_b x 2k) | U, W (d x k each) | tr
  double* cen_sum = nullptr; // running-mean centring: column sums of every row seen (X then Y, d)
  float* cen_mean = nullptr; // their means (d)
  double cen_count = 0.0;    // rows seen

  // cluster path: ping-pong state buffers and three accumulator slots
  float* cl_V[2] = {nullptr, nullptr};
  float* cl_S[2] = {nullptr, nullptr};
  float* cl_acc = nullptr;     // 3 slots of 2 x d x k
  int cl_cur = 0;              // state buffer holding V_t, [Bv]_t
  int cl_slot = 0;             // accumulator slot written by the most recent step
  int cl_pending = 0;          // products of one step are waiting for their update
  float cl_eta = 0.f, cl_gamma = 0.f;  // step sizes of the pending update
  int cl_size = 8;             // CTAs per cluster
  int cl_x = 4;                // CTAs of a cluster on X columns (rest on Y)
  int cl_wx = 0, cl_wy = 0, cl_wmax = 0;  // column-slice widths (cl_wmax padded to 8)
  int cl_kp = 4;               // players padded to a power of two (>= 4)
  int cl_lkp = 2;              // log2(cl_kp)
  int cl_rs = 32;              // minibatch rows resident per CTA
  int cl_xs = 0;               // shared-memory row stride of a minibatch chunk (elements)
  int cl_async_shape = 0;      // rows and slices start on 16-byte boundaries
  int cl_pdl = 1;              // programmatic dependent launch
  float* cl_gram = nullptr;    // 3 slots of k*k + k row-side terms
  int cl_max_clusters = 0;     // co-resident clusters reported by the occupancy API
  int cl_last_grid = 0;        // CTAs of the most recent launch
  int cl_ms_ok = 0;            // the multi-step kernel is configured
  int cl_ms_coop = 1;          // it is launched cooperatively
  int cl_ms_traced = 0;        // the trace buffer holds a multi-step launch's stamps
  size_t cl_ms_smem = 0;       // its shared memory
  int cl_ms_max_clusters = 0;  // its co-resident clusters
  unsigned* cl_bar = nullptr;  // its grid-barrier arrival counter
  unsigned cl_bar_count = 0;   // arrivals so far
  unsigned long long* trace = nullptr;  // SGEP_TRACE=1: per-CTA phase timestamps
  size_t cl_smem = 0;

  // tensor-core path
  __nv_bfloat16* tc_Vt = nullptr;  // 64 x d: BF16 hi/lo pairs of V (transposed)
  float* tc_PQ = nullptr;          // 2 x max_b x 32: row projections P, Q
  __nv_bfloat16* tc_Pt = nullptr;  // 64 x max_b: BF16 hi/lo pairs of P (transposed)
  __nv_bfloat16* tc_Qt = nullptr;
  float* tc_coef = nullptr;        // k*k + 2k update coefficients
  int tc_generic_step = 0;         // the last step's shape needed the generic products
  float* tc_dbg = nullptr;         // a | G | b used by the last tensor-core update (debug)
  unsigned long long* tc_bar = nullptr;  // grid-barrier arrivals of the fused update
  float* tc_part = nullptr;              // its per-block partial sums
  unsigned long long* tc_upd_trace = nullptr;  // SGEP_TRACE=1: its phase times
  unsigned long long tc_bar_base = 0;    // arrivals expected before the next launch
  int tc_upd_fused = 0;            // the fused update fits on the device (all blocks resident)
  int tc_chain = 0;                // the last update prepared this step's V operand and d-side terms
  int tc_bar_reset = 0;            // the barrier count must be cleared before the next launch
  size_t tc_smem_p = 0, tc_smem_b = 0;
  // one-read streamed products (kernels_tc_stream.cu)
  int tc_st_ok = 0;                // the streamed kernel is set up for this handle
  unsigned* tc_st_cnt = nullptr;   // [max_b / 128] contributions, then [max_b / 128] operand-ready flags
  unsigned tc_st_epoch = 0;        // streamed steps since the counters were last cleared
  int tc_st_reset = 0;             // clear the counters (and the row sums) before the next launch
  int tc_pq_dirty = 0;             // P and Q hold values another kernel left behind
  unsigned long long* tc_st_trace = nullptr;  // SGEP_TRACE=1: per-CTA, per-chunk event times
  int tc_st_nchunk = 0;            // chunks of the most recent streamed launch
  int tc_st_grid = 0;              // its CTAs (streaming + builder helpers)
  int tc_st_lag = 5, tc_st_helpers = 24;  // tuning knobs (SGEP_TC_LAG, SGEP_TC_HELPERS)
  int tc_st_pfn = 3;                       // next-step chunks prefetched into L2 (SGEP_TC_PFN)
  float* tc_st_terms = nullptr;    // [3] row-side term slots a | b, then [3] slots |v'|^2 | U
  unsigned tc_st_launch = 0;       // streamed launches since the counters were last cleared
  unsigned tc_st_grams = 0;        // helper Gram contributions since then
  int tc_st_bp_groups = 0;         // the last streamed launch loaded its back-projection rows in one copy per step
  int tc_st_updated = 0;           // the most recent streamed launch applied the step's update
  int64_t tc_st_last_b = 0;        // minibatch size the counters were last used with
  int tc_acc_stale = 0;            // acc does not hold the last step's products (not kept)

  // LDA: running class statistics (exact cumulative sums over every row seen)
  double* lda_sum = nullptr;  // C x d class sums
  double* lda_cnt = nullptr;  // C class counts
  float* lda_mean = nullptr;  // C x d class means
  float* lda_M = nullptr;     // C x d mu_c - mu
  float* lda_pi = nullptr;    // C priors n_c / n
  float* lda_W = nullptr;     // C x k: (mu_c - mu)^T V
  double* rr_buf = nullptr;   // Rayleigh-Ritz: k x k sums, C, eigenvalues, norms (FP64)
  int64_t rr_every = 0;       // periodic Rayleigh-Ritz: every this many steps (0: none)
  const void* rr_X = nullptr; // its evaluation rows (caller-owned device memory)
  const void* rr_Y = nullptr;
  const float* rr_sx = nullptr;
  const float* rr_sy = nullptr;
  const int32_t* rr_labels = nullptr;
  int64_t rr_n = 0;

  int64_t t = 0;       // iterations applied (Alg. 2's t)
  float* mach_buf = nullptr;  // machines > 1: 3 x d x k (V' sum, [Bv]' sum, [Bv] copy)
  int test_stall = 0;   // SGEP_TEST_STALL=1 at init: the fused update's grid barrier never completes
  int64_t launches = 0; // kernels launched
  int debug_valid = 0; // sgep_debug_update has data
};

// Flag bits of Ctx::dflag.
constexpr int kFlagNonFinite = 1;
constexpr int kFlagTimeout = 2;
constexpr int kFlagBadLabel = 4;
constexpr int kFlagNotPD = 8;    // Rayleigh-Ritz: V^T B V not positive definite
constexpr int kMaxClasses = 32;  // LDA classes

// Error reporting (thread-local message).
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define SGEP_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return ::sgep::cuda_fail(_e, #expr); \
  } while (0)

// Step-size schedule (App. H.2.2), evaluated on the host.
double schedule_eta(const sgep_config& c, int64_t t);
// The variant parameters of the next update (advances the Adam step count).
UpdVariant next_variant(Ctx& c);

// ---- generic SIMT path (kernels_generic.cu) ----
// Products of one minibatch: acc <- [A_t V ; B_t V], PQ scratch.
// Bytes per element of X and Y for the handle's dtype.
inline size_t elem_size(const Ctx& c) { return c.cfg.dtype == SGEP_F32 ? 4 : (c.cfg.dtype == SGEP_BF16 ? 2 : 1); }

int generic_products(Ctx& c, const void* X, const void* Y, int64_t b, cudaStream_t s,
                     const float* sx = nullptr, const float* sy = nullptr);
// Update from acc: grams, update, retraction. eta/gamma of this step.
int generic_update(Ctx& c, float eta, float gamma, cudaStream_t s);
// One step of Alg. 2 with cfg.machines shards of the b rows: per-shard products, update
// directions and auxiliary increments, averaged over the shards before the steps.
int generic_machines_step(Ctx& c, const void* X, const void* Y, int64_t b, cudaStream_t s, const float* sx,
                          const float* sy, float eta, float gamma);
// Row projections of n rows into PQ (n <= max_b), zeroing PQ first.
// sx, sy: per-row scales of FP8 rows (null otherwise); center/labels: LDA centring.
int generic_project(Ctx& c, const void* X, const void* Y, int64_t n, cudaStream_t s,
                    const float* center = nullptr, const int32_t* labels = nullptr, const float* sx = nullptr,
                    const float* sy = nullptr);
// Running-mean centring (kernels_generic.cu): adds b rows to the running sums, refreshes the means.
int centring_update(Ctx& c, const void* X, const void* Y, int64_t b, cudaStream_t s, const float* sx,
                    const float* sy);
// ICA (kernels_generic.cu): acc <- [A_t V ; B_t V] of b rows, quarters when `split`.
int ica_alloc(Ctx& c);
int ica_products(Ctx& c, const void* X, int64_t b, cudaStream_t s, const float* sx, bool split);
// LDA: BV = X~^T (X~ V) / n over n rows centred by the class means (kernels_generic.cu).
int generic_lda_within(Ctx& c, const void* X, const int32_t* labels, int64_t n, cudaStream_t s,
                       const float* sx = nullptr);

// Learned warm start (kernels_warm.cu).
struct MlpCtx;
int mlp_create(int m, int k, uint64_t seed, MlpCtx** out);
void mlp_free(MlpCtx* M);
int mlp_set(MlpCtx& M, const float* host);
int mlp_get(const MlpCtx& M, float* host);
int mlp_param_count(const MlpCtx& M);
int mlp_forward(MlpCtx& M, const float* S, int64_t rows, float* O, cudaStream_t s);
int mlp_loss_grad(MlpCtx& M, const float* S, const float* V, const int64_t* seg_host, int n_inst, double* loss_out,
                  float* grad_host, cudaStream_t s);
int mlp_adam(MlpCtx& M, float lr, cudaStream_t s);
int sketch_rows(const void* X, const void* Y, int dtype, int64_t n, int64_t dx, int64_t dy, const float* om, int m,
                float* out, int num_sms, int* dflag, cudaStream_t s);

// Batching form (kernels_batch.cu).
struct BatchCtx;
int batch_create(Ctx** hs, int n, BatchCtx** out);
void batch_free(BatchCtx* B);
int batch_step(BatchCtx& B, const void* const* X, const void* const* Y, const float* const* sx,
               const float* const* sy, const int32_t* const* labels, const int64_t* b, cudaStream_t s);
int batch_sync(BatchCtx& B, cudaStream_t s);
void batch_set(BatchCtx& B, int mode, int blocks_per_sm, int chunk_cap, int rows_cap, int use_graph);
void batch_get(const BatchCtx& B, int* out5);
int64_t batch_launches(const BatchCtx& B);
int batch_autotune(BatchCtx& B, const void* const* X, const void* const* Y, const float* const* sx,
                   const float* const* sy, const int32_t* const* labels, const int64_t* b, int reps, int* best5);
double schedule_eta(const sgep_config& cfg, int64_t t);

// Rayleigh-Ritz correction of V and [Bv] on n evaluation rows (kernels_rr.cu).
int rr_correct(Ctx& c, const void* X, const void* Y, const float* sx, const float* sy, const int32_t* labels,
               int64_t n, double* lam_host, cudaStream_t s);

// LDA (kernels_lda.cu): class statistics and the between-class products.
int lda_alloc(Ctx& c);
void lda_free(Ctx& c);
// Adds the minibatch rows to the class statistics, then acc = [A_t V ; B_t V].
int lda_products(Ctx& c, const void* X, const int32_t* labels, int64_t b, cudaStream_t s, const float* sx);
// Recomputes means, mu_c - mu and priors from the sums and counts (after a state load).
int lda_refresh(Ctx& c, cudaStream_t s);
// W = (mu_c - mu)^T V into lda_W (C x k) for the current V.
int lda_project_means(Ctx& c, cudaStream_t s);
// Retraction V <- Vtmp / ||Vtmp|| with the norms in gram (counts the update launch too).
int generic_normalize(Ctx& c, cudaStream_t s);
// Rayleigh sums of the n rows in PQ accumulated into rq (double).
int generic_rayleigh_sums(Ctx& c, int64_t n, cudaStream_t s);

// ---- tensor-core path (kernels_tc.cu) ----
// 2-D BF16 row-major tensor map, 128-byte swizzle, box_rows x box_cols (box_cols * 2 == 128).
int make_map_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                  int box_cols);
// The same matrix viewed as (64 columns, rows, column groups): a box of box_rows x `groups`
// groups lands as `groups` consecutive 2-D boxes of 64 columns (one copy).
int make_map_f32(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                 int box_cols);
int make_map_bf16_groups(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                         int groups);
bool tc_supported(const Ctx& c, const char** why);
int tc_alloc(Ctx& c);
void tc_free(Ctx& c);
// acc <- [A_t V ; B_t V] of a BF16 minibatch on the tensor cores. eta, gamma: the step's
// sizes, used when the streamed launch also applies the update.
int tc_products(Ctx& c, const void* X, const void* Y, int64_t b, cudaStream_t s, float eta, float gamma);
// k x k terms of the tensor-core path, double-buffered by step parity.
struct TcTerms {
  float *a, *b, *norms, *G, *vv;
};
size_t tc_terms_floats(int k);
TcTerms tc_terms(const Ctx& c, int slot);

// Streamed tensor-core steps (kernels_tc_stream.cu): products, row-side terms and update.
bool tc_stream_supported(const Ctx& c, int64_t b);
int tc_stream_setup(Ctx& c);
void tc_stream_free(Ctx& c);
// nsteps (<= tc_stream_max_steps()) consecutive steps of Alg. 2 in one launch: products,
// row-side terms and the update of each; X and Y hold nsteps minibatches of b rows.
int tc_stream_steps(Ctx& c, const void* X, const void* Y, int64_t b, int nsteps, cudaStream_t s);
int tc_stream_max_steps();
// V split into BF16 pairs and the d-side terms of slot (c.t & 1), unless the chain of
// tensor-core steps left them current.
int tc_prepare_chain(Ctx& c, cudaStream_t s);
void tc_stream_trace_report(Ctx& c);
// Update from acc with the k x k terms the tensor-core products accumulated.
int tc_update(Ctx& c, float eta, float gamma, cudaStream_t s);

// ---- cluster path (kernels_cluster.cu) ----
bool cluster_supported(const Ctx& c, const char** why);
int cluster_alloc(Ctx& c);
void cluster_free(Ctx& c);
// One fused launch: pending update (if any) then the products of (X, Y).
int cluster_step(Ctx& c, const void* X, const void* Y, int64_t b, float eta, float gamma,
                 cudaStream_t s);
// Apply a pending update (no new minibatch).
int cluster_flush(Ctx& c, cudaStream_t s);
// Several consecutive minibatches in one persistent launch (grid barrier between steps).
int cluster_steps(Ctx& c, const void* X, const void* Y, int64_t b, int nsteps, cudaStream_t s);
int cluster_max_steps();
bool cluster_steps_usable(const Ctx& c);
// Copy the pending products into acc layout (d x k AV, d x k BV) for debugging.
int cluster_products(Ctx& c, float* AV, float* BV, cudaStream_t s);
void tc_update_trace_report(Ctx& c);
// SGEP_TRACE=1: print per-phase times of the most recent cluster launch to stderr.
void cluster_trace_report(Ctx& c);

}  // namespace sgep

// The opaque handle type of the ABI is the context itself.
struct sgep_ctx : public sgep::Ctx {};

/*
 * sgep.h -- C ABI of libsgep: the minibatch gamma-EigenGame iteration for the
 * top-k symmetric generalized eigenproblem  A v = lambda B v  on one GB300
 * (sm_103a).
 *
 * Method: Gemp, Chen, McWilliams, "The Symmetric Generalized Eigenvalue
 * Problem as a Nash Equilibrium" (arXiv 2206.04993), Alg. 2 ("Stochastic
 * gamma-EigenGame") with M = 1 machine; the update direction is Eq. (update)
 * of Sec. 3, A and B are expectations of outer products (Sec. 1) and are never
 * formed: each step streams one minibatch through  X V  and  X^T (X V).
 *
 * Conventions shared by every entry point
 *  - Every function returns SGEP_OK (0) or a negative status code below.
 *    Nothing throws across the ABI. sgep_last_error() describes the most
 *    recent failure of the calling thread.
 *  - A handle owns all of its device state (V, [Bv], accumulators, scratch).
 *    It is not thread-safe: calls on one handle must not overlap, and work
 *    enqueued on different streams for one handle must not overlap on the GPU.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Device work is enqueued asynchronously on it; device-side
 *    errors (non-finite values, exhausted spin limits) are recorded in a
 *    device flag and reported by the next synchronising call (sgep_sync,
 *    sgep_get_V, sgep_get_eigenvalues, sgep_get_state, sgep_debug_*).
 *  - Data matrices are row-major, one sample per row: X is b x d_x, Y is
 *    b x d_y, element (r, c) at X[r * d_x + c]. Their element type is the
 *    handle's dtype (float for SGEP_F32, bfloat16 bit patterns for
 *    SGEP_BF16, FP8 e4m3 bytes for SGEP_FP8E4M3 together with one float
 *    scale per row: the row's values are scale_r * e4m3(code)). They are
 *    caller-owned DEVICE pointers and must stay valid
 *    until the work on `stream` has completed.
 *  - The player matrix V (and [Bv], called S here) is d x k row-major float:
 *    element (c, i) at V[c * k + i], so column i is the player vector v_i
 *    and d = d_x + d_y (d = d_x for PCA and LDA).
 */
#ifndef SGEP_H_
#define SGEP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SGEP_OK          0
#define SGEP_EINVAL     (-1)  /* invalid argument or configuration            */
#define SGEP_ENOMEM     (-2)  /* device or host allocation failed             */
#define SGEP_ECUDA      (-3)  /* a CUDA runtime call failed                   */
#define SGEP_ETIMEOUT   (-4)  /* a bounded device-side wait gave up           */
#define SGEP_ENONFINITE (-5)  /* NaN or Inf appeared in the player vectors    */
#define SGEP_ELAUNCH    (-6)  /* a kernel could not be launched as configured */
#define SGEP_ESTATE     (-7)  /* state blob malformed / wrong shape / version */
#define SGEP_ENOTSUP    (-8)  /* combination not supported by this build      */

/* ---- problem kinds (Sec. 1) --------------------------------------------- */
#define SGEP_PCA 0  /* A = E[x x^T], B = I                                       */
#define SGEP_CCA 1  /* A = [[0, E xy^T], [E yx^T, 0]], B = blockdiag(E xx^T, E yy^T) */
#define SGEP_PLS 2  /* A as CCA, B = I (reading of Sec. 1, which gives no formula) */
#define SGEP_LDA 3  /* between-class A from running class means, within-class B  */
#define SGEP_ICA 4  /* A = E[<x,x> x x^T] - tr(B) B - 2 B^2, B = E[x x^T] (excess kurtosis) */
/* ICA (Sec. 1): d_y = 0, generic path. Reading of "independent data batches": with
 * split_AB = 1 the rows form four quarters (the last takes the remainder, b >= 4): the
 * kurtosis term of A_t from the first, tr(B) and the outer B of B^2 from the second, the
 * inner B from the third, B_t from the fourth, so every product pairs independent rows.
 * With split_AB = 0 every term uses every row. sgep_get_eigenvalues takes at most max_b
 * rows for ICA (A is not a sum over rows); sgep_rayleigh_ritz does not take ICA. */
/* LDA (Sec. 1 names it without estimators; reading): the handle keeps the exact
 * running class sums and counts of every row seen (FP64); a step first adds all
 * of its rows, then uses A = sum_c pi_c (mu_c - mu)(mu_c - mu)^T (pi_c = n_c / n,
 * mu = sum_c pi_c mu_c) and B_t = the covariance of the B rows, each centred by
 * the mean of its class. d_y = 0; labels are int32 in [0, n_classes), 2 <= n_classes
 * <= 32. LDA runs on the generic path. rank(A) <= n_classes - 1, so only the top
 * n_classes - 1 generalized eigenvalues are nonzero. */

/* ---- element type of X and Y ------------------------------------------- */
#define SGEP_F32      0
#define SGEP_BF16     1
#define SGEP_FP8E4M3  2  /* e4m3 codes with per-row float scales (generic path) */

/* ---- step-size schedules (App. H.2.2) ----------------------------------- */
#define SGEP_SCHED_CONST          0  /* eta_t = eta0                                   */
#define SGEP_SCHED_HOLD_HARMONIC  1  /* eta0 up to t_c, then ~1/(t+Delta), eta_T at T  */
#define SGEP_SCHED_WARMUP_HARMONIC 2 /* linear warm-up to eta0 at t_c, then as above   */

/* ---- kernel path selection --------------------------------------------- */
#define SGEP_OPT_SGD  0  /* player step of Alg. 2                                       */
#define SGEP_OPT_ADAM 1  /* Adam on the players (App. H.2.2)                           */
#define SGEP_ALG2     0  /* clipped denominators (Alg. 2)                              */
#define SGEP_ALG3     1  /* smooth denominators with scalars z_j (Alg. 3, App. E.2)    */

#define SGEP_PATH_AUTO    0  /* pick by shape and dtype                         */
#define SGEP_PATH_GENERIC 1  /* multi-kernel SIMT path, any shape               */
#define SGEP_PATH_CLUSTER 2  /* one fused cluster kernel per step, d <= 4096    */
#define SGEP_PATH_TC      3  /* tcgen05 tensor-core fused path, BF16, large d   */

typedef struct sgep_ctx* sgep_t;

/* Configuration of one problem instance. Fill with sgep_config_default()
 * and override fields; unknown future fields keep their defaults. */
typedef struct {
  int32_t  kind;       /* SGEP_PCA / SGEP_CCA / SGEP_PLS                          */
  int32_t  dtype;      /* SGEP_F32, SGEP_BF16 or SGEP_FP8E4M3 (element type of X, Y) */
  int64_t  d_x;        /* columns of X (>= 1)                                      */
  int64_t  d_y;        /* columns of Y (>= 1 for CCA/PLS, must be 0 for PCA)       */
  int32_t  k;          /* number of players, 1 <= k <= 64 and k <= d              */
  int32_t  n_classes;  /* LDA only: number of classes, 2..32                         */
  float    eta0;       /* player step size eta (Alg. 2 "step size sequence")      */
  float    gamma0;     /* auxiliary step size gamma_t (constant; beta_t in App. H) */
  float    rho;        /* clipping floor of <v_j, [Bv]_j> (Alg. 2), > 0           */
  float    eps_B;      /* optional ridge: B_t + eps_B I (App. G); default 0        */
  int32_t  schedule;   /* SGEP_SCHED_*                                              */
  int32_t  split_AB;   /* 1: rows [0, b/2) estimate A, rows [b/2, b) estimate B   */
                       /* (independent batches of Alg. 2); 0: all rows for both    */
  int64_t  t_c;        /* schedule knee (App. H.2.2)                               */
  int64_t  T;          /* schedule horizon: eta_t reaches eta_T at t = T           */
  float    eta_T;      /* final step size                                          */
  int32_t  path;       /* SGEP_PATH_*                                              */
  uint64_t seed;       /* seed of the initial V (Philox-4x32-10 + Box-Muller)      */
  int64_t  max_b;      /* largest minibatch (rows) a step or readout chunk may use */
  int32_t  debug;      /* 1: keep update directions and k x k terms for sgep_debug_update */
  int32_t  optimizer;  /* SGEP_OPT_SGD: Alg. 2's step v + eta grad; SGEP_OPT_ADAM: Adam on the */
                       /* players (App. H.2.2): v + eta m_hat / (sqrt(s_hat) + adam_eps)        */
  float    adam_b1;    /* Adam moment decays and floor (defaults 0.9, 0.999, 1e-8; App. H.2.2) */
  float    adam_b2;
  float    adam_eps;
  int32_t  variant;    /* SGEP_ALG2: clipped denominators max(<v_j,[Bv]_j>, rho) (Alg. 2);     */
                       /* SGEP_ALG3: smooth denominators exp(log rho + (log nu - log rho)       */
                       /* sigmoid(z_j)) with one scalar z_j per player (Alg. 3, App. E.2)       */
  float    nu;         /* Alg. 3: upper bound on lambda_max(B), > rho                           */
  int32_t  center;     /* 1: centre every row by the exact running mean of all rows seen      */
                       /* (App. H.2.2 "mean estimates are learned"; the pencils of Sec. 1     */
                       /* assume zero-mean data). PCA, CCA, PLS on the generic path. A step   */
                       /* adds its rows to the running sums first, then centres them.         */
  int32_t  machines;   /* M of Alg. 2 (default 1): the b rows of a step form M consecutive      */
                       /* shards of b / M rows (the last takes the remainder); each shard is a  */
                       /* machine's minibatch with its own A/B split, its update direction and  */
                       /* auxiliary increment B_tm v_i - [Bv]_i are averaged over the machines   */
                       /* before the player and auxiliary steps. M > 1: CCA, PCA, PLS on the     */
                       /* generic path, Alg. 2's plain step (no Adam, Alg. 3 or centring).       */
  int32_t  reserved0;  /* must be 0 */
} sgep_config;

/* Fill `cfg` with defaults: CCA, F32, k = 1, eta0 = 0.1, gamma0 = 1, rho = 1e-6,
 * eps_B = 0, constant schedule, split_AB = 1, path AUTO, seed 0, max_b 4096,
 * optimizer SGD (Adam decays 0.9, 0.999, floor 1e-8), variant Alg. 2.
 * Adam and Alg. 3 run on the generic and tensor-core paths (AUTO avoids the cluster
 * path for them); their state (Adam moments, z) is reset by sgep_set_V / sgep_set_VS
 * and travels in the state blob.
 * Returns SGEP_EINVAL if cfg is NULL. */
int sgep_config_default(sgep_config* cfg);

/* Create a handle (Alg. 2 initialisation): allocate device state on the
 * current CUDA device, draw v_i ~ N(0, I_d) and scale each to unit norm
 * (Alg. 2, line "v_i ~ S^{d-1}"), and set [Bv]_i = v_i (Alg. 2, auxiliary
 * initialisation). Synchronous. On error *out is left NULL and nothing leaks.
 * Errors: SGEP_EINVAL (bad shape/kind/dtype/rho/k), SGEP_ENOMEM, SGEP_ECUDA,
 * SGEP_ENOTSUP (a forced path that cannot run the shape or kind). */
int sgep_init(const sgep_config* cfg, sgep_t* out);

/* Free every resource of the handle (synchronises the device first).
 * NULL is accepted. */
int sgep_destroy(sgep_t h);

/* One iteration of Alg. 2 (M = 1) on the minibatch (X, Y) of b rows:
 * A_t and B_t are the minibatch estimates (split per cfg.split_AB),
 * the update direction is Eq. (update) with the clipped auxiliary terms,
 * v_i <- (v_i + eta_t grad_i) / ||.||, [Bv]_i <- [Bv]_i + gamma_t (B_t v_i - [Bv]_i),
 * all players reading the state of step t. Asynchronous on `stream`.
 * X: device, b x d_x; Y: device, b x d_y (NULL for PCA and LDA);
 * row_scale_x, row_scale_y: FP8E4M3 only, device, b floats each (NULL for the
 * other dtypes and for a missing view); labels: LDA
 * only, device, b int32 class labels in [0, n_classes) (NULL otherwise). A label
 * outside the range is reported as SGEP_EINVAL by the next synchronising call
 * (its row is then left uncentred; no out-of-bounds access happens).
 * Requires 2 <= b <= max_b when split_AB = 1 (1 <= b otherwise).
 * The work of a step may be completed lazily by the next step or by the
 * next synchronising call. Errors: SGEP_EINVAL, SGEP_ECUDA, SGEP_ELAUNCH. */
int sgep_step(sgep_t h, const void* X, const void* Y, const float* row_scale_x,
              const float* row_scale_y, const int32_t* labels, int64_t b, void* stream);

/* `nsteps` consecutive iterations on minibatches stored back to back:
 * step s reads rows [s*b, (s+1)*b) of X and Y (and of the row scales and labels).
 * Same contract as sgep_step. */
int sgep_step_many(sgep_t h, const void* X, const void* Y, const float* row_scale_x,
                   const float* row_scale_y, const int32_t* labels, int64_t b, int64_t nsteps,
                   void* stream);

/* Wait for the handle's work on `stream` and report device-side errors
 * (SGEP_ENONFINITE, SGEP_ETIMEOUT). Clears the recorded error. */
int sgep_sync(sgep_t h, void* stream);

/* Copy V (d x k row-major float) to `out` (device pointer if on_device,
 * else host). Completes pending work and synchronises `stream`. */
int sgep_get_V(sgep_t h, float* out, int on_device, void* stream);

/* Copy the auxiliary variables [Bv] (d x k row-major float) to `out`. */
int sgep_get_S(sgep_t h, float* out, int on_device, void* stream);

/* Replace V by `V` (d x k row-major float, host or device) and reset
 * [Bv] <- V (warm start, Alg. 2 auxiliary initialisation). Columns are used
 * as given (callers pass unit-norm columns). Synchronous. */
int sgep_set_V(sgep_t h, const float* V, int on_device, void* stream);

/* Replace both V and [Bv] (S may not equal V). Synchronous. */
int sgep_set_VS(sgep_t h, const float* V, const float* S, int on_device, void* stream);

/* Generalized Rayleigh quotients lambda_i = <v_i, A v_i> / <v_i, B v_i>
 * (Sec. 2, below Eq. util_new) with A and B estimated on the n evaluation
 * rows (X, Y) (all rows for both; App. H.2.2 evaluates on a larger batch than
 * it trains on). Sums are accumulated in double. out_k: host, k doubles.
 * LDA: <v_i, A v_i> comes from the handle's class statistics (the readout does
 * not update them) and <v_i, B v_i> from the n rows centred by their class
 * means; labels (device, n int32) are required.
 * Synchronous. Any n >= 1 (processed in chunks of max_b rows). */
int sgep_get_eigenvalues(sgep_t h, const void* X, const void* Y, const float* row_scale_x,
                         const float* row_scale_y, const int32_t* labels, int64_t n,
                         double* out_k, void* stream);

/* Rayleigh-Ritz correction (precision form): on the n evaluation rows (X, Y,
 * labels as for sgep_get_eigenvalues; A and B estimated on all rows, in FP64
 * sums of the FP32 row projections), solve the k x k pencil
 * (V^T A V) c = lambda (V^T B V) c in FP64 on the device (Cholesky reduction and
 * Jacobi, App. A), set V <- V C and [Bv] <- [Bv] C, and divide every column of
 * both by ||v'_i|| (unit sphere). The players become the Ritz vectors of their
 * span, ordered by descending Ritz value; lambda_out (host, k doubles, may be
 * NULL) receives those values. The paper has no such step: it is a correction
 * applied between iterations to win back accuracy lost to low-precision data.
 * Synchronous. Errors: SGEP_EINVAL, SGEP_ENONFINITE (V^T B V not positive
 * definite: V and [Bv] are then left unchanged), SGEP_ECUDA. */
int sgep_rayleigh_ritz(sgep_t h, const void* X, const void* Y, const float* row_scale_x,
                       const float* row_scale_y, const int32_t* labels, int64_t n,
                       double* lambda_out, void* stream);

/* Periodic Rayleigh-Ritz correction (precision form): after every step whose count
 * t (sgep_step_count) is a multiple of `every`, sgep_step and sgep_step_many apply
 * sgep_rayleigh_ritz on the evaluation rows given here (same meaning and layout as
 * its arguments; device pointers owned by the caller, which must keep them valid and
 * unchanged while the schedule is set). The correction is the Ritz step of App. A
 * (Prop. "Similar matrices") on the span of the players, taken every `every` steps of
 * Alg. 2; sgep_step_many splits its launches at those steps. every = 0 removes the
 * schedule (the pointers may then be NULL). The corrections run on the step's stream
 * and synchronise it. Errors: SGEP_EINVAL (every < 0, NULL rows or labels when
 * needed, n < 1, bad scales), SGEP_ENOTSUP (ICA). A correction that finds V^T B V not
 * positive definite makes the step report SGEP_ENONFINITE (V and [Bv] unchanged). */
int sgep_set_rr_every(sgep_t h, int64_t every, const void* X, const void* Y, const float* row_scale_x,
                      const float* row_scale_y, const int32_t* labels, int64_t n);

/* ---- batching form ------------------------------------------------------
 * Many independent problems (uneven kind, d_x, d_y, k, element type) advanced
 * together: one call runs one step of every instance. The paper has no batched
 * form; this groups independent Alg. 2 iterations. Every handle must have been
 * created with path = SGEP_PATH_GENERIC (the batch runs the generic tiles); it
 * stays owned by the caller, must outlive the batch, and must not be stepped on
 * its own while the batch may have work in flight (sgep_batch_sync first).
 * Per-instance results and errors are read through the handles as usual. */
typedef struct sgep_batch_ctx* sgep_batch_t;

/* Group n handles (host array) into a batch. Synchronises every handle first.
 * Errors: SGEP_EINVAL (NULL, duplicate, non-generic handle), SGEP_ENOTSUP (a handle
 * with Adam or Alg. 3), SGEP_ENOMEM. */
int sgep_batch_create(const sgep_t* handles, int n, sgep_batch_t* out);

/* Free the batch (not the handles). NULL is accepted. */
int sgep_batch_destroy(sgep_batch_t b);

/* One step of every instance. X, Y, row_scale_x, row_scale_y, labels: host
 * arrays of n device pointers with the meaning of sgep_step's arguments for
 * instance i (Y, the scale arrays and labels may be NULL when no instance needs
 * them); rows: host array of n row counts. Asynchronous on `stream`: a table of
 * per-instance descriptors is copied from pinned host memory, then either one
 * persistent cooperative launch runs the eight phases of the step (zeroing, LDA
 * class statistics, projection, back-projection, LDA between-class products, k x k
 * terms, update, retraction) separated by bounded grid barriers (mode 0), or one
 * launch per phase (mode 1); with use_graph the copy and the launch(es) are
 * captured in a CUDA graph once per launch shape and replayed. */
int sgep_batch_step(sgep_batch_t b, const void* const* X, const void* const* Y,
                    const float* const* row_scale_x, const float* const* row_scale_y,
                    const int32_t* const* labels, const int64_t* rows, void* stream);

/* Wait for the batch's work on `stream`; report a barrier timeout of the batched
 * launch (SGEP_ETIMEOUT) or the first instance error (as sgep_sync). */
int sgep_batch_sync(sgep_batch_t b, void* stream);

/* Set the launch configuration; a negative or zero value keeps the current one.
 * mode: 0 persistent, 1 one launch per phase; blocks_per_sm: persistent grid
 * (capped by occupancy); chunk_cap: projection tile width in columns (64..4096);
 * rows_cap: back-projection tile height in rows (>= 32); use_graph: 0 or 1. */
int sgep_batch_configure(sgep_batch_t b, int mode, int blocks_per_sm, int chunk_cap,
                         int rows_cap, int use_graph);

/* The current configuration: out5 = {mode, blocks_per_sm, chunk_cap, rows_cap, use_graph}. */
int sgep_batch_get_config(sgep_batch_t b, int* out5);

/* Autotuner: time every candidate configuration (mode x chunk_cap in {256, 512,
 * 1024} x rows_cap in {64, 128, 256} x blocks_per_sm in {1, 2, 4} for mode 0) for
 * `reps` steps on these rows, keep the fastest, and cache it for this batch
 * signature (kind, dtype, d_x, d_y, k, rows of every instance) for the life of the
 * process. The instances' state (V, [Bv], step count, LDA statistics) is saved
 * before and restored after. out5 receives the chosen configuration. Synchronous. */
int sgep_batch_autotune(sgep_batch_t b, const void* const* X, const void* const* Y,
                        const float* const* row_scale_x, const float* const* row_scale_y,
                        const int32_t* const* labels, const int64_t* rows, int reps, int* out5);

/* Kernel launches issued by the batch so far (a graph replay counts its kernels). */
int64_t sgep_batch_launch_count(sgep_batch_t b);

/* ---- learned warm start --------------------------------------------------
 * Not in the paper, which starts from random players (Alg. 2): a random sketch of
 * the first minibatch is mapped row by row to an initial V by a small network
 * trained on the plain solver's solutions; the plain iteration then runs from it
 * (sgep_set_V), and stays the fallback. */
typedef struct sgep_mlp_ctx* sgep_mlp_t;

/* Sketch S = Z^T (Z Omega) / n of n rows Z = [X Y] (device, dtype SGEP_F32 or
 * SGEP_BF16; Y NULL when d_y = 0), Omega device d x m row-major float (d = d_x + d_y,
 * m <= 32); every column of S is then divided by its root mean square over the d
 * rows. out: device d x m row-major float. Synchronous. */
int sgep_sketch(const void* X, const void* Y, int dtype, int64_t n, int64_t d_x, int64_t d_y,
                const float* omega, int m, float* out, void* stream);

/* Per-row network in_dim (m <= 32) -> 64 -> 64 -> out_dim (k <= 32) with ReLUs;
 * weights used in BF16 (FP32 master copies), FP32 accumulation; seeded He
 * initialisation. Errors: SGEP_EINVAL, SGEP_ENOMEM. */
int sgep_mlp_create(int in_dim, int out_dim, uint64_t seed, sgep_mlp_t* out);
int sgep_mlp_destroy(sgep_mlp_t m);

/* Number of parameters P; their layout (row-major): W1 (64 x m) | b1 (64) |
 * W2 (64 x 64) | b2 (64) | W3 (k x 64) | b3 (k). */
int sgep_mlp_param_count(sgep_mlp_t m);

/* Copy the parameters as used (weights rounded to BF16) to host `host` (P floats). */
int sgep_mlp_get_params(sgep_mlp_t m, float* host);

/* Set the master parameters from host (P floats; weights are used rounded to BF16)
 * and reset the optimiser state. Synchronous. */
int sgep_mlp_set_params(sgep_mlp_t m, const float* host);

/* out (device rows x k) = network applied to every row of S (device rows x m). */
int sgep_mlp_forward(sgep_mlp_t m, const float* S, int64_t rows, float* out, void* stream);

/* Loss and gradients on a batch of instances: rows seg[i] .. seg[i+1] - 1 of S
 * (device, rows x m) and of the targets V (device, rows x k) belong to instance i
 * (seg: host, n_inst + 1 increasing offsets, seg[0] = 0). Loss = mean over the
 * instances of sum_i (1 - (o_i . v_i)^2 / (|o_i|^2 |v_i|^2)) (sign- and scale-
 * invariant per column). The gradients stay on the device for sgep_mlp_adam_step;
 * grad_host (P floats, may be NULL) receives a copy. Synchronous. */
int sgep_mlp_loss_grad(sgep_mlp_t m, const float* S, const float* V, const int64_t* seg, int n_inst,
                       double* loss, float* grad_host, void* stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with the last gradients. */
int sgep_mlp_adam_step(sgep_mlp_t m, float lr, void* stream);

/* Serialise the state (versioned header, V, [Bv], step counter; LDA also its
 * class sums, C x d doubles, and counts, C doubles) into `buf`.
 * If buf is NULL, only writes the required size to *nbytes. Synchronous. */
int sgep_get_state(sgep_t h, void* buf, size_t* nbytes);

/* Restore a state written by sgep_get_state for the same kind, d_x, d_y, k.
 * Errors: SGEP_ESTATE on a malformed or mismatched blob. Synchronous. */
int sgep_set_state(sgep_t h, const void* buf, size_t nbytes);

/* Number of iterations applied so far (t of Alg. 2). */
int64_t sgep_step_count(sgep_t h);

/* The step size eta_t the handle uses at iteration t (1-based). */
double sgep_eta_at(sgep_t h, int64_t t);

/* Kernel path the handle runs (SGEP_PATH_GENERIC / _CLUSTER / _TC). */
int sgep_path(sgep_t h);

/* Number of CUDA kernels the handle has launched since sgep_init (memsets and
 * copies are not counted). Returns -1 for a NULL handle. */
int64_t sgep_launch_count(sgep_t h);

/* Diagnostics for parity tests. sgep_debug_products copies the minibatch
 * products of the most recent step, A_t V and B_t V (each d x k row-major,
 * host), before the update was applied (for PCA and PLS, where B = I, B_t V is
 * not formed and BV is zero-filled). sgep_debug_update (needs cfg.debug=1)
 * copies the update direction grad (d x k), and the k x k terms
 * [a_ij = v_i^T A_t v_j (k*k), b_i = v_i^T B_t v_i (k), G_ij = <v_i, [Bv]_j> (k*k)]
 * into `terms` (2 k^2 + k doubles) of the most recent completed step. Synchronous. */
int sgep_debug_products(sgep_t h, float* AV, float* BV);
int sgep_debug_update(sgep_t h, float* grad, double* terms);

/* Diagnostic of the tensor-core building blocks (TMA loads with 128-byte
 * swizzle, tcgen05.mma BF16 -> FP32 in tensor memory, tcgen05.ld): runs one
 * 128 x 64 x 64 product on the current device and writes the largest error
 * relative to a SIMT FP32 reference into *max_rel_err. mode 0: A K-major;
 * modes 1 and 2: A MN-major (transposed) with the two descriptor strides in
 * either order. Allocates its own buffers; synchronous. */
int sgep_tc_selftest(int mode, double* max_rel_err);

/* ---- allocation-free step ----------------------------------------------- */
/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory themselves: plugins inside a host application
 * that owns the GPU's memory through its own pool and only hands out fixed
 * buffers, services that must keep their device footprint constant after
 * start-up, and tight loops where cudaMalloc/cudaFree (which can synchronise
 * the whole device) are not allowed.
 *
 * sgep_step_noalloc performs the same iteration as sgep_step on the generic
 * path, for a problem described by `cfg` (kind, dtype, d_x, d_y, k, rho,
 * eps_B, split_AB, step-size schedule; path, seed, max_b and debug are
 * ignored), starting from the caller's state V and S = [Bv] (device, d x k
 * row-major float) and writing the new state to V_out and S_out (device,
 * d x k; they may be the same buffers as V and S). `t` (>= 1) is the
 * iteration number that selects eta_t from the schedule. X and Y are as for
 * sgep_step. It never calls cudaMalloc or cudaFree: the temporaries of the
 * step live in one fixed array of SGEP_NOALLOC_SCRATCH_BYTES in device memory,
 * which every GPU that loads this library keeps until the process exits.
 * A shape needs 4*(2k^2 + 2k + 2bk + 3dk) bytes plus a few hundred bytes of
 * alignment; larger shapes are rejected with SGEP_EINVAL and a message.
 *  - The first call on each device looks up the device address of the array
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before starting any stream capture.
 *  - Every call on a device shares the one array, which keeps the contents
 *    of the previous call (the call clears what must start at zero). Calls
 *    whose work overlaps on the GPU (other streams, other host threads) race
 *    on it and corrupt each other's results: serialise them.
 *  - Asynchronous on `stream`; non-finite values are not reported (inspect
 *    V_out). Errors: SGEP_EINVAL (also for cfg->optimizer = Adam or
 *    cfg->variant = Alg. 3, whose state does not fit this call), SGEP_ECUDA. */
#define SGEP_NOALLOC_SCRATCH_BYTES 4194304
int sgep_step_noalloc(const sgep_config* cfg, const void* X, const void* Y, int64_t b,
                      const float* V, const float* S, float* V_out, float* S_out,
                      int64_t t, void* stream);

/* Human-readable name of a status code (static string). */
const char* sgep_strerror(int status);

/* Description of the most recent failure on the calling thread ("" if none). */
const char* sgep_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SGEP_H_ */

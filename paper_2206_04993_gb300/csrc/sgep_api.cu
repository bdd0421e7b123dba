// Host side of the C ABI declared in include/sgep.h: handle lifetime,
// argument checks, the step-size schedule, path dispatch, state blobs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace sgep {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SGEP_ENOMEM : SGEP_ECUDA;
}

static int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

// App. H.2.2: warm-up (or hold) until t_c, then eta proportional to 1/(t + Delta) with
// Delta chosen so that eta_T is reached at t = T.
double schedule_eta(const sgep_config& c, int64_t t) {
  const double eta0 = c.eta0;
  if (c.schedule == SGEP_SCHED_CONST) return eta0;
  const double tc = (double)c.t_c, T = (double)c.T, etaT = c.eta_T;
  const double delta = (etaT * T - eta0 * tc) / (eta0 - etaT);
  if ((double)t <= tc) return c.schedule == SGEP_SCHED_HOLD_HARMONIC ? eta0 : eta0 * (double)t / tc;
  return eta0 * (tc + delta) / ((double)t + delta);
}

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for the initial V.
static void philox4x32(uint32_t ctr[4], uint32_t key[2]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)M0 * ctr[0];
    const uint64_t p1 = (uint64_t)M1 * ctr[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t c0 = hi1 ^ ctr[1] ^ k0, c2 = hi0 ^ ctr[3] ^ k1;
    ctr[0] = c0;
    ctr[1] = lo1;
    ctr[2] = c2;
    ctr[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

static void gaussian_init(std::vector<float>& V, int64_t d, int k, uint64_t seed) {
  // column i gets Philox counters (i, c/2, 0, 0); Box-Muller pairs.
  std::vector<double> col(d);
  const double two_pi = 6.283185307179586476925286766559;
  for (int i = 0; i < k; ++i) {
    double nrm = 0.0;
    for (int64_t c = 0; c < d; c += 2) {
      uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(c >> 1), (uint32_t)((uint64_t)c >> 33), 0u};
      uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
      philox4x32(ctr, key);
      const double u1 = ((double)ctr[0] + 1.0) / 4294967296.0;  // (0, 1]
      const double u2 = (double)ctr[1] / 4294967296.0;
      const double r = std::sqrt(-2.0 * std::log(u1));
      col[c] = r * std::cos(two_pi * u2);
      if (c + 1 < d) col[c + 1] = r * std::sin(two_pi * u2);
    }
    for (int64_t c = 0; c < d; ++c) nrm += col[c] * col[c];
    nrm = std::sqrt(nrm);
    for (int64_t c = 0; c < d; ++c) V[c * k + i] = (float)(col[c] / nrm);
  }
}

static void free_ctx(sgep_ctx* c) {
  if (!c) return;
  cluster_free(*c);
  tc_free(*c);
  lda_free(*c);
  cudaFree(c->rr_buf);
  cudaFree(c->V);
  cudaFree(c->S);
  cudaFree(c->Vtmp);
  cudaFree(c->PQ);
  cudaFree(c->acc);
  cudaFree(c->gram);
  cudaFree(c->grad);
  cudaFree(c->rq);
  cudaFree(c->dflag);
  cudaFree(c->adam_m);
  cudaFree(c->z);
  cudaFree(c->ica_buf);
  cudaFree(c->mach_buf);
  cudaFree(c->cen_sum);
  cudaFree(c->cen_mean);
  delete c;
}

static int check_flag(Ctx& c) {
  int flag = 0;
  SGEP_CUDA_TRY(cudaMemcpy(&flag, c.dflag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    SGEP_CUDA_TRY(cudaMemset(c.dflag, 0, sizeof(int)));
    if (flag & kFlagTimeout) {
      c.tc_bar_reset = 1;    // an aborted update may leave a short barrier count
      c.tc_st_reset = 1;     // ... and an aborted streamed launch short counters and row sums
      c.tc_chain = 0;
      return fail(SGEP_ETIMEOUT, "a bounded device-side wait gave up");
    }
    if (flag & kFlagBadLabel) return fail(SGEP_EINVAL, "a label is outside [0, n_classes)");
    if (flag & kFlagNotPD)
      return fail(SGEP_ENONFINITE, "V^T B V is not positive definite (players not independent)");
    if (flag & kFlagNonFinite) return fail(SGEP_ENONFINITE, "non-finite values in V");
  }
  return SGEP_OK;
}

// Completes a step whose update is still pending (cluster path) and synchronises.
static int complete(Ctx& c, cudaStream_t s) {
  if (c.path == SGEP_PATH_CLUSTER && c.cl_pending) {
    int rc = cluster_flush(c, s);
    if (rc) return rc;
  }
  SGEP_CUDA_TRY(cudaStreamSynchronize(s));
  return check_flag(c);
}

UpdVariant next_variant(Ctx& c) {
  UpdVariant v;
  if (c.adam_m) {
    ++c.adam_t;
    v.m = c.adam_m;
    v.s = c.adam_s;
    v.b1 = c.cfg.adam_b1;
    v.b2 = c.cfg.adam_b2;
    v.eps = c.cfg.adam_eps;
    v.bc1 = (float)(1.0 - std::pow((double)c.cfg.adam_b1, (double)c.adam_t));
    v.bc2 = (float)(1.0 - std::pow((double)c.cfg.adam_b2, (double)c.adam_t));
  }
  if (c.z) {
    v.z = c.z;
    v.log_rho = std::log(c.cfg.rho);
    v.log_nu = std::log(c.cfg.nu);
  }
  return v;
}

}  // namespace sgep

using namespace sgep;

static_assert(sizeof(sgep_config) == 136, "sgep_config layout changed: update the bindings");

extern "C" {

int sgep_config_default(sgep_config* cfg) {
  if (!cfg) return fail(SGEP_EINVAL, "cfg is NULL");
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->kind = SGEP_CCA;
  cfg->dtype = SGEP_F32;
  cfg->d_x = 1;
  cfg->d_y = 1;
  cfg->k = 1;
  cfg->eta0 = 0.1f;
  cfg->gamma0 = 1.0f;
  cfg->rho = 1e-6f;
  cfg->eps_B = 0.0f;
  cfg->schedule = SGEP_SCHED_CONST;
  cfg->split_AB = 1;
  cfg->t_c = 1;
  cfg->T = 2;
  cfg->eta_T = 0.1f;
  cfg->path = SGEP_PATH_AUTO;
  cfg->seed = 0;
  cfg->max_b = 4096;
  cfg->debug = 0;
  cfg->optimizer = SGEP_OPT_SGD;
  cfg->adam_b1 = 0.9f;
  cfg->adam_b2 = 0.999f;
  cfg->adam_eps = 1e-8f;
  cfg->variant = SGEP_ALG2;
  cfg->nu = 0.f;
  cfg->machines = 1;
  return SGEP_OK;
}

int sgep_init(const sgep_config* cfg, sgep_t* out) {
  if (!out) return fail(SGEP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(SGEP_EINVAL, "cfg is NULL");
  const sgep_config& g = *cfg;
  if (g.kind != SGEP_PCA && g.kind != SGEP_CCA && g.kind != SGEP_PLS && g.kind != SGEP_LDA && g.kind != SGEP_ICA)
    return fail(SGEP_EINVAL, "unknown kind");
  if (g.kind == SGEP_LDA && (g.n_classes < 2 || g.n_classes > kMaxClasses))
    return fail(SGEP_EINVAL, "LDA needs 2 <= n_classes <= 32");
  if (g.dtype != SGEP_F32 && g.dtype != SGEP_BF16 && g.dtype != SGEP_FP8E4M3)
    return fail(SGEP_EINVAL, "unknown dtype");
  if (g.d_x < 1) return fail(SGEP_EINVAL, "d_x must be >= 1");
  const bool one_view = g.kind == SGEP_PCA || g.kind == SGEP_LDA || g.kind == SGEP_ICA;
  if (one_view && g.d_y != 0) return fail(SGEP_EINVAL, "PCA, LDA and ICA require d_y = 0");
  if (!one_view && g.d_y < 1) return fail(SGEP_EINVAL, "CCA/PLS require d_y >= 1");
  const int64_t d = g.d_x + g.d_y;
  if (g.k < 1 || g.k > 64 || g.k > d) return fail(SGEP_EINVAL, "k must satisfy 1 <= k <= min(64, d)");
  if (!(g.rho > 0.f) || !std::isfinite(g.rho)) return fail(SGEP_EINVAL, "rho must be > 0");
  if (!std::isfinite(g.eta0) || !std::isfinite(g.gamma0) || !std::isfinite(g.eps_B) || g.eps_B < 0.f)
    return fail(SGEP_EINVAL, "eta0, gamma0 must be finite and eps_B >= 0");
  if (g.schedule < 0 || g.schedule > 2) return fail(SGEP_EINVAL, "unknown schedule");
  if (g.schedule != SGEP_SCHED_CONST &&
      (g.t_c < 1 || g.T <= g.t_c || !(g.eta_T > 0.f) || !(g.eta_T < g.eta0)))
    return fail(SGEP_EINVAL, "schedule needs 1 <= t_c < T and 0 < eta_T < eta0");
  if (g.max_b < 2 || g.max_b > (1LL << 24)) return fail(SGEP_EINVAL, "max_b out of range");
  if (g.path < 0 || g.path > 3) return fail(SGEP_EINVAL, "unknown path");
  if (g.optimizer != SGEP_OPT_SGD && g.optimizer != SGEP_OPT_ADAM) return fail(SGEP_EINVAL, "unknown optimizer");
  if (g.optimizer == SGEP_OPT_ADAM &&
      (!(g.adam_b1 >= 0.f && g.adam_b1 < 1.f) || !(g.adam_b2 >= 0.f && g.adam_b2 < 1.f) || !(g.adam_eps >= 0.f) ||
       !std::isfinite(g.adam_eps)))
    return fail(SGEP_EINVAL, "Adam needs 0 <= b1, b2 < 1 and a finite eps >= 0");
  if (g.variant != SGEP_ALG2 && g.variant != SGEP_ALG3) return fail(SGEP_EINVAL, "unknown variant");
  if (g.variant == SGEP_ALG3 && !(g.nu > g.rho && std::isfinite(g.nu)))
    return fail(SGEP_EINVAL, "Alg. 3 needs a finite nu > rho");
  const bool variants = g.optimizer == SGEP_OPT_ADAM || g.variant == SGEP_ALG3;
  if (g.center != 0 && g.center != 1) return fail(SGEP_EINVAL, "center must be 0 or 1");
  if (g.center && g.kind != SGEP_PCA && g.kind != SGEP_CCA && g.kind != SGEP_PLS)
    return fail(SGEP_EINVAL, "running-mean centring is for PCA, CCA and PLS (LDA centres by class means)");
  if (g.machines < 1 || g.reserved0 != 0) return fail(SGEP_EINVAL, "machines must be >= 1 (reserved0 = 0)");
  if (g.machines > 1 &&
      ((g.kind != SGEP_CCA && g.kind != SGEP_PCA && g.kind != SGEP_PLS) || variants || g.center ||
       (g.path != SGEP_PATH_AUTO && g.path != SGEP_PATH_GENERIC)))
    return fail(SGEP_ENOTSUP, "machines > 1: CCA, PCA or PLS with Alg. 2's plain step on the generic path");

  sgep_ctx* c = new (std::nothrow) sgep_ctx();
  if (!c) return fail(SGEP_ENOMEM, "host allocation failed");
  c->cfg = g;
  c->d_x = g.d_x;
  c->d_y = g.d_y;
  c->d = d;
  c->k = g.k;
  c->b_is_identity = (g.kind == SGEP_PCA || g.kind == SGEP_PLS);
  c->has_y = !one_view;
  {
    // test hook for the bounded waits: the fused tensor-core update's grid barrier waits for
    // one arrival too many (nothing sends it) and gives up after 20 ms
    const char* st = std::getenv("SGEP_TEST_STALL");
    c->test_stall = (st && st[0] == '1') ? 1 : 0;
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(e, "cudaGetDevice");
  }
  const size_t dk = (size_t)d * g.k;
  const size_t kk = (size_t)g.k * g.k;
  struct {
    void** p;
    size_t n;
  } allocs[] = {
      {(void**)&c->V, dk * sizeof(float)},
      {(void**)&c->S, dk * sizeof(float)},
      {(void**)&c->Vtmp, dk * sizeof(float)},
      {(void**)&c->PQ, (size_t)g.max_b * 2 * g.k * sizeof(float)},
      {(void**)&c->acc, 2 * dk * sizeof(float)},
      {(void**)&c->gram, (2 * kk + 2 * g.k) * sizeof(float)},
      {(void**)&c->rq, 2 * g.k * sizeof(double)},
      {(void**)&c->dflag, sizeof(int)},
  };
  for (auto& a : allocs) {
    e = cudaMalloc(a.p, a.n);
    if (e != cudaSuccess) {
      free_ctx(c);
      return cuda_fail(e, "cudaMalloc (state)");
    }
  }
  if (g.debug) {
    e = cudaMalloc((void**)&c->grad, dk * sizeof(float));
    if (e != cudaSuccess) {
      free_ctx(c);
      return cuda_fail(e, "cudaMalloc (debug)");
    }
  }
  if (g.optimizer == SGEP_OPT_ADAM) {  // Adam moments, zero at the start
    e = cudaMalloc((void**)&c->adam_m, 2 * dk * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->adam_m, 0, 2 * dk * sizeof(float));
    if (e != cudaSuccess) {
      free_ctx(c);
      return cuda_fail(e, "cudaMalloc (Adam moments)");
    }
    c->adam_s = c->adam_m + dk;
  }
  if (g.variant == SGEP_ALG3) {  // z_i = 0 at the start (Alg. 3)
    e = cudaMalloc((void**)&c->z, (size_t)g.k * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->z, 0, (size_t)g.k * sizeof(float));
    if (e != cudaSuccess) {
      free_ctx(c);
      return cuda_fail(e, "cudaMalloc (Alg. 3 scalars)");
    }
  }
  cudaMemset(c->dflag, 0, sizeof(int));
  cudaMemset(c->acc, 0, 2 * dk * sizeof(float));

  // Path selection.
  const char* why = nullptr;
  const bool cl_ok = cluster_supported(*c, &why);
  const bool generic_only =
      g.kind == SGEP_LDA || g.kind == SGEP_ICA || g.dtype == SGEP_FP8E4M3 || g.center || g.machines > 1;
  if (generic_only && g.path != SGEP_PATH_AUTO && g.path != SGEP_PATH_GENERIC) {
    free_ctx(c);
    return fail(SGEP_ENOTSUP, "LDA, ICA, FP8 rows and running-mean centring run on the generic path only");
  }
  if (g.center) {  // running sums and means start at zero
    e = cudaMalloc((void**)&c->cen_sum, (size_t)d * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(c->cen_sum, 0, (size_t)d * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->cen_mean, (size_t)d * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->cen_mean, 0, (size_t)d * sizeof(float));
    if (e != cudaSuccess) {
      free_ctx(c);
      return cuda_fail(e, "cudaMalloc (running means)");
    }
  }
  if (generic_only) c->path = SGEP_PATH_GENERIC;
  if (g.machines > 1) {  // per-machine averaging: V' and [Bv]' accumulators and a copy of [Bv]
    e = cudaMalloc((void**)&c->mach_buf, 3 * dk * sizeof(float));
    if (e != cudaSuccess) {
      free_ctx(c);
      return cuda_fail(e, "cudaMalloc (machines)");
    }
  }
  if (g.kind == SGEP_ICA) {
    int rc = ica_alloc(*c);
    if (rc) {
      free_ctx(c);
      return rc;
    }
  } else if (g.kind == SGEP_LDA) {
    int rc = lda_alloc(*c);
    if (rc) {
      free_ctx(c);
      return rc;
    }
  } else if (generic_only) {
    // FP8 rows: the generic kernels dequantise with the per-row scales
  } else if (g.path == SGEP_PATH_AUTO) {
    c->path = (cl_ok && !variants) ? SGEP_PATH_CLUSTER
                                   : (tc_supported(*c, nullptr) ? SGEP_PATH_TC : SGEP_PATH_GENERIC);
  } else if (g.path == SGEP_PATH_CLUSTER) {
    if (variants) {
      free_ctx(c);
      return fail(SGEP_ENOTSUP, "cluster path: Adam and Alg. 3 run on the generic and tensor-core paths");
    }
    if (!cl_ok) {
      free_ctx(c);
      return fail(SGEP_ENOTSUP, std::string("cluster path: ") + (why ? why : "unsupported"));
    }
    c->path = SGEP_PATH_CLUSTER;
  } else if (g.path == SGEP_PATH_TC) {
    const char* tw = nullptr;
    if (!tc_supported(*c, &tw)) {
      free_ctx(c);
      return fail(SGEP_ENOTSUP, std::string("tensor-core path: ") + tw);
    }
    c->path = SGEP_PATH_TC;
  } else {
    c->path = SGEP_PATH_GENERIC;
  }
  if (c->path == SGEP_PATH_CLUSTER || c->path == SGEP_PATH_TC) {
    int rc = c->path == SGEP_PATH_CLUSTER ? cluster_alloc(*c) : tc_alloc(*c);
    if (rc) {
      free_ctx(c);
      return rc;
    }
    if (c->path == SGEP_PATH_TC && variants && !c->tc_upd_fused) {
      // Adam and Alg. 3 are in the fused tensor-core update, which needs every block resident
      if (g.path == SGEP_PATH_TC) {
        free_ctx(c);
        return fail(SGEP_ENOTSUP, "tensor-core path: Adam / Alg. 3 need the fused update (d too large)");
      }
      tc_free(*c);
      c->path = SGEP_PATH_GENERIC;
    }
  }

  std::vector<float> V0(dk);
  gaussian_init(V0, d, g.k, g.seed);
  e = cudaMemcpy(c->V, V0.data(), dk * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->S, V0.data(), dk * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(e, "initialising V");
  }
  *out = c;
  return SGEP_OK;
}

int sgep_destroy(sgep_t h) {
  if (!h) return SGEP_OK;
  cudaDeviceSynchronize();
  free_ctx(h);
  return SGEP_OK;
}

// Row scales: required for FP8 rows (one per row and view), absent otherwise.
static int scale_checks(const Ctx& c, const float* sx, const float* sy) {
  if (c.cfg.dtype == SGEP_FP8E4M3) {
    if (!sx || (c.has_y && !sy)) return fail(SGEP_EINVAL, "FP8 rows need their row scales");
    if (!c.has_y && sy) return fail(SGEP_EINVAL, "row_scale_y given for a one-view problem");
  } else if (sx || sy) {
    return fail(SGEP_EINVAL, "row scales are for FP8 rows only");
  }
  return SGEP_OK;
}

static int step_checks(Ctx& c, const void* X, const void* Y, const float* sx, const float* sy,
                       const int32_t* labels, int64_t b) {
  if (!X) return fail(SGEP_EINVAL, "X is NULL");
  if (c.has_y && !Y) return fail(SGEP_EINVAL, "Y is NULL");
  if (int rc = scale_checks(c, sx, sy)) return rc;
  if (c.cfg.kind == SGEP_LDA && !labels) return fail(SGEP_EINVAL, "LDA needs labels");
  const bool split = (c.cfg.kind == SGEP_CCA || c.cfg.kind == SGEP_LDA || c.cfg.kind == SGEP_ICA) && c.cfg.split_AB;
  const int64_t bmin = split ? (c.cfg.kind == SGEP_ICA ? 4 : 2) : 1;
  if (b < bmin * c.cfg.machines)
    return fail(SGEP_EINVAL, "b too small (split batches need b >= 2, ICA quarters b >= 4, per machine)");
  if (b > c.cfg.max_b) return fail(SGEP_EINVAL, "b exceeds max_b");
  return SGEP_OK;
}

// The periodic Rayleigh-Ritz correction, when step count c.t is due for one.
static int rr_if_due(Ctx& c, cudaStream_t s) {
  if (c.rr_every <= 0 || c.t % c.rr_every != 0) return SGEP_OK;
  int rc = rr_correct(c, c.rr_X, c.rr_Y, c.rr_sx, c.rr_sy, c.rr_labels, c.rr_n, nullptr, s);
  c.tc_chain = 0;  // V and [Bv] changed outside the step
  if (rc) return rc;
  return check_flag(c);
}

static int do_step(Ctx& c, const void* X, const void* Y, const float* sx, const float* sy, const int32_t* labels,
                   int64_t b, cudaStream_t s) {
  const int64_t t = c.t + 1;
  const float eta = (float)schedule_eta(c.cfg, t);
  const float gamma = c.cfg.gamma0;
  int rc;
  if (c.path == SGEP_PATH_CLUSTER) {
    rc = cluster_step(c, X, Y, b, eta, gamma, s);
  } else {
    if (c.path == SGEP_PATH_TC) {
      rc = tc_products(c, X, Y, b, s, eta, gamma);
      if (!rc && c.tc_generic_step) c.tc_chain = 0;
      if (!rc) rc = c.tc_generic_step ? generic_update(c, eta, gamma, s) : tc_update(c, eta, gamma, s);
    } else {
      rc = c.cen_sum ? centring_update(c, X, Y, b, s, sx, sy) : SGEP_OK;  // the step's rows first
      if (!rc && c.cfg.machines > 1) {
        rc = generic_machines_step(c, X, Y, b, s, sx, sy, eta, gamma);
      } else {
        if (!rc) {
          if (c.cfg.kind == SGEP_LDA) rc = lda_products(c, X, labels, b, s, sx);
          else if (c.cfg.kind == SGEP_ICA) rc = ica_products(c, X, b, s, sx, c.cfg.split_AB != 0);
          else rc = generic_products(c, X, Y, b, s, sx, sy);
        }
        if (!rc) rc = generic_update(c, eta, gamma, s);
      }
    }
    if (!rc) c.debug_valid = c.cfg.machines > 1 ? 0 : c.cfg.debug;  // shards keep no directions
  }
  if (!rc) c.t = t;
  if (!rc && c.path != SGEP_PATH_CLUSTER) rc = rr_if_due(c, s);
  return rc;
}

int sgep_step(sgep_t h, const void* X, const void* Y, const float* row_scale_x, const float* row_scale_y,
              const int32_t* labels, int64_t b, void* stream) {
  if (!h) return fail(SGEP_EINVAL, "handle is NULL");
  int rc = step_checks(*h, X, Y, row_scale_x, row_scale_y, labels, b);
  if (rc) return rc;
  return do_step(*h, X, Y, row_scale_x, row_scale_y, labels, b, (cudaStream_t)stream);
}

int sgep_step_many(sgep_t h, const void* X, const void* Y, const float* row_scale_x, const float* row_scale_y,
                   const int32_t* labels, int64_t b, int64_t nsteps, void* stream) {
  if (!h) return fail(SGEP_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(SGEP_EINVAL, "nsteps < 0");
  int rc = step_checks(*h, X, Y, row_scale_x, row_scale_y, labels, b);
  if (rc) return rc;
  const size_t esz = elem_size(*h);
  Ctx& c = *h;
  if (c.path == SGEP_PATH_TC && tc_stream_supported(c, b) && !((uintptr_t)X & 15) && !((uintptr_t)Y & 15)) {
    // consecutive minibatches of the streamed tensor-core path: several steps per launch
    for (int64_t s0 = 0; s0 < nsteps;) {
      int64_t lim = std::min<int64_t>(nsteps - s0, tc_stream_max_steps());
      if (c.rr_every > 0) lim = std::min<int64_t>(lim, c.rr_every - c.t % c.rr_every);  // stop at a correction
      const int n = (int)lim;
      const char* xs = (const char*)X + (size_t)s0 * b * c.d_x * esz;
      const char* ys = (const char*)Y + (size_t)s0 * b * c.d_y * esz;
      rc = tc_prepare_chain(c, (cudaStream_t)stream);
      if (!rc) rc = tc_stream_steps(c, xs, ys, b, n, (cudaStream_t)stream);
      if (rc) return rc;
      c.t += n;
      c.tc_generic_step = 0;
      c.debug_valid = c.cfg.debug;
      s0 += n;
      rc = rr_if_due(c, (cudaStream_t)stream);
      if (rc) return rc;
    }
    return SGEP_OK;
  }
  if (c.path == SGEP_PATH_CLUSTER && nsteps > 1 && cluster_steps_usable(c)) {
    // consecutive minibatches of the cluster path: several steps per persistent launch
    for (int64_t s0 = 0; s0 < nsteps;) {
      const int n = (int)std::min<int64_t>(nsteps - s0, cluster_max_steps());
      const char* xs = (const char*)X + (size_t)s0 * b * c.d_x * esz;
      const char* ys = Y ? (const char*)Y + (size_t)s0 * b * c.d_y * esz : nullptr;
      rc = cluster_steps(c, xs, ys, b, n, (cudaStream_t)stream);
      if (rc) return rc;
      c.t += n;
      s0 += n;
    }
    return SGEP_OK;
  }
  for (int64_t s = 0; s < nsteps; ++s) {
    const char* xs = (const char*)X + (size_t)s * b * h->d_x * esz;
    const char* ys = Y ? (const char*)Y + (size_t)s * b * h->d_y * esz : nullptr;
    const int32_t* ls = labels ? labels + s * b : nullptr;
    const float* sxs = row_scale_x ? row_scale_x + s * b : nullptr;
    const float* sys = row_scale_y ? row_scale_y + s * b : nullptr;
    rc = do_step(*h, xs, ys, sxs, sys, ls, b, (cudaStream_t)stream);
    if (rc) return rc;
  }
  return SGEP_OK;
}

int sgep_sync(sgep_t h, void* stream) {
  if (!h) return fail(SGEP_EINVAL, "handle is NULL");
  int rc = complete(*h, (cudaStream_t)stream);
  if (h->trace) cluster_trace_report(*h);
  if (h->tc_upd_trace) tc_update_trace_report(*h);
  if (h->tc_st_trace) tc_stream_trace_report(*h);
  return rc;
}

// Completes pending work first: the cluster path swaps its state buffers when it does,
// so the source pointer is read only afterwards.
static int copy_out(Ctx& c, bool want_S, float* out, int on_device, void* stream) {
  if (!out) return fail(SGEP_EINVAL, "out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = complete(c, s);
  if (rc) return rc;
  const float* src = want_S ? c.S : c.V;
  SGEP_CUDA_TRY(cudaMemcpyAsync(out, src, sizeof(float) * c.d * c.k,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  SGEP_CUDA_TRY(cudaStreamSynchronize(s));
  return SGEP_OK;
}

int sgep_get_V(sgep_t h, float* out, int on_device, void* stream) {
  if (!h) return fail(SGEP_EINVAL, "handle is NULL");
  return copy_out(*h, false, out, on_device, stream);
}

int sgep_get_S(sgep_t h, float* out, int on_device, void* stream) {
  if (!h) return fail(SGEP_EINVAL, "handle is NULL");
  return copy_out(*h, true, out, on_device, stream);
}

int sgep_set_VS(sgep_t h, const float* V, const float* S, int on_device, void* stream) {
  if (!h) return fail(SGEP_EINVAL, "handle is NULL");
  if (!V || !S) return fail(SGEP_EINVAL, "V or S is NULL");
  Ctx& c = *h;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = complete(c, s);
  if (rc) return rc;
  const cudaMemcpyKind kd = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  SGEP_CUDA_TRY(cudaMemcpyAsync(c.V, V, sizeof(float) * c.d * c.k, kd, s));
  SGEP_CUDA_TRY(cudaMemcpyAsync(c.S, S, sizeof(float) * c.d * c.k, kd, s));
  // a new start: Adam's moments and Alg. 3's scalars restart from zero as at sgep_init
  if (c.adam_m) SGEP_CUDA_TRY(cudaMemsetAsync(c.adam_m, 0, 2 * sizeof(float) * c.d * c.k, s));
  if (c.z) SGEP_CUDA_TRY(cudaMemsetAsync(c.z, 0, sizeof(float) * c.k, s));
  c.adam_t = 0;
  SGEP_CUDA_TRY(cudaStreamSynchronize(s));
  c.debug_valid = 0;
  c.tc_chain = 0;
  return SGEP_OK;
}

int sgep_set_V(sgep_t h, const float* V, int on_device, void* stream) {
  return sgep_set_VS(h, V, V, on_device, stream);
}

int sgep_get_eigenvalues(sgep_t h, const void* X, const void* Y, const float* row_scale_x,
                         const float* row_scale_y, const int32_t* labels, int64_t n, double* out_k,
                         void* stream) {
  if (!h) return fail(SGEP_EINVAL, "handle is NULL");
  Ctx& c = *h;
  if (!X || (c.has_y && !Y) || !out_k) return fail(SGEP_EINVAL, "NULL argument");
  const bool lda = c.cfg.kind == SGEP_LDA;
  if (lda && !labels) return fail(SGEP_EINVAL, "LDA needs labels");
  if (n < 1) return fail(SGEP_EINVAL, "n must be >= 1");
  if (int e = scale_checks(c, row_scale_x, row_scale_y)) return e;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = complete(c, s);
  if (rc) return rc;
  const int k = c.k;
  if (c.cfg.kind == SGEP_ICA) {
    // A is not a sum over rows: the n rows form one unsplit estimate; v_i^T A v_i / v_i^T B v_i
    if (n > c.cfg.max_b) return fail(SGEP_EINVAL, "ICA eigenvalues take at most max_b rows");
    rc = ica_products(c, X, n, s, row_scale_x, false);
    if (rc) return rc;
    const size_t dk = (size_t)c.d * k;
    std::vector<float> V(dk), AV(dk), BV(dk);
    SGEP_CUDA_TRY(cudaMemcpyAsync(V.data(), c.V, dk * sizeof(float), cudaMemcpyDeviceToHost, s));
    SGEP_CUDA_TRY(cudaMemcpyAsync(AV.data(), c.acc, dk * sizeof(float), cudaMemcpyDeviceToHost, s));
    SGEP_CUDA_TRY(cudaMemcpyAsync(BV.data(), c.acc + dk, dk * sizeof(float), cudaMemcpyDeviceToHost, s));
    SGEP_CUDA_TRY(cudaStreamSynchronize(s));
    rc = check_flag(c);
    if (rc) return rc;
    for (int i = 0; i < k; ++i) {
      double num = 0.0, den = 0.0;
      for (int64_t r = 0; r < c.d; ++r) {
        num += (double)V[r * k + i] * AV[r * k + i];
        den += (double)V[r * k + i] * BV[r * k + i];
      }
      out_k[i] = num / den;
    }
    c.debug_valid = 0;
    return SGEP_OK;
  }
  SGEP_CUDA_TRY(cudaMemsetAsync(c.rq, 0, sizeof(double) * 2 * k, s));
  const size_t esz = elem_size(c);
  for (int64_t r0 = 0; r0 < n; r0 += c.cfg.max_b) {
    const int64_t m = std::min<int64_t>(c.cfg.max_b, n - r0);
    const char* xs = (const char*)X + (size_t)r0 * c.d_x * esz;
    const char* ys = c.has_y ? (const char*)Y + (size_t)r0 * c.d_y * esz : nullptr;
    // LDA: rows centred by the running class means (the readout does not update them)
    rc = generic_project(c, xs, ys, m, s, lda ? c.lda_mean : nullptr, lda ? labels + r0 : nullptr,
                         row_scale_x ? row_scale_x + r0 : nullptr, row_scale_y ? row_scale_y + r0 : nullptr);
    if (!rc) rc = generic_rayleigh_sums(c, m, s);
    if (rc) return rc;
  }
  std::vector<double> sums(2 * k);
  std::vector<float> V((size_t)c.d * k);
  SGEP_CUDA_TRY(cudaMemcpyAsync(sums.data(), c.rq, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, s));
  SGEP_CUDA_TRY(cudaMemcpyAsync(V.data(), c.V, sizeof(float) * V.size(), cudaMemcpyDeviceToHost, s));
  // LDA: v_i^T A v_i = sum_c pi_c ((mu_c - mu)^T v_i)^2 from the class statistics
  const int C = lda ? c.cfg.n_classes : 0;
  std::vector<float> W((size_t)C * k), pi(C);
  if (lda) {
    rc = lda_project_means(c, s);
    if (rc) return rc;
    SGEP_CUDA_TRY(cudaMemcpyAsync(W.data(), c.lda_W, sizeof(float) * W.size(), cudaMemcpyDeviceToHost, s));
    SGEP_CUDA_TRY(cudaMemcpyAsync(pi.data(), c.lda_pi, sizeof(float) * C, cudaMemcpyDeviceToHost, s));
  }
  SGEP_CUDA_TRY(cudaStreamSynchronize(s));
  rc = check_flag(c);
  if (rc) return rc;
  for (int i = 0; i < k; ++i) {
    double vv = 0.0;
    for (int64_t r = 0; r < c.d; ++r) vv += (double)V[r * k + i] * V[r * k + i];
    double num = sums[i] / (double)n;
    double den = c.b_is_identity ? vv : sums[k + i] / (double)n;
    if (lda) {
      num = 0.0;
      for (int cl = 0; cl < C; ++cl) num += (double)pi[cl] * W[cl * k + i] * W[cl * k + i];
      den = sums[i] / (double)n;  // sum of squared projections of the centred rows
    }
    den += (double)c.cfg.eps_B * vv;
    out_k[i] = num / den;
  }
  return SGEP_OK;
}

// State blob: header then V and S (float, d x k each).
// LDA appends its class sums (C x d doubles) and counts (C doubles) to the state.
static size_t lda_state_bytes(const Ctx& c) {
  return c.cfg.kind == SGEP_LDA ? ((size_t)c.cfg.n_classes * c.d + c.cfg.n_classes) * sizeof(double) : 0;
}
// Adam moments (2 d k floats) and their step count; Alg. 3's k scalars z; the running
// column sums (d doubles) and row count of a centring handle.
static size_t variant_state_bytes(const Ctx& c) {
  const size_t dk = (size_t)c.d * c.k;
  return (c.adam_m ? 2 * dk * sizeof(float) + sizeof(int64_t) : 0) + (c.z ? (size_t)c.k * sizeof(float) : 0) +
         (c.cen_sum ? ((size_t)c.d + 1) * sizeof(double) : 0);
}
static int32_t variant_flags(const Ctx& c) { return (c.adam_m ? 1 : 0) | (c.z ? 2 : 0) | (c.cen_sum ? 4 : 0); }

struct StateHeader {
  char magic[8];
  int32_t version;
  int32_t kind;
  int64_t d_x, d_y;
  int32_t k;
  int32_t variants;  // bit 0: Adam moments follow, bit 1: Alg. 3 scalars follow
  int64_t t;
};

int sgep_rayleigh_ritz(sgep_t h, const void* X, const void* Y, const float* row_scale_x,
                       const float* row_scale_y, const int32_t* labels, int64_t n, double* lambda_out,
                       void* stream) {
  if (!h) return fail(SGEP_EINVAL, "handle is NULL");
  Ctx& c = *h;
  if (!X || (c.has_y && !Y)) return fail(SGEP_EINVAL, "NULL argument");
  if (c.cfg.kind == SGEP_LDA && !labels) return fail(SGEP_EINVAL, "LDA needs labels");
  if (c.cfg.kind == SGEP_ICA) return fail(SGEP_ENOTSUP, "the Rayleigh-Ritz correction does not take ICA");
  if (n < 1) return fail(SGEP_EINVAL, "n must be >= 1");
  if (int e = scale_checks(c, row_scale_x, row_scale_y)) return e;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = complete(c, s);
  if (rc) return rc;
  rc = rr_correct(c, X, Y, row_scale_x, row_scale_y, labels, n, lambda_out, s);
  c.tc_chain = 0;  // V and [Bv] changed outside the step
  c.debug_valid = 0;
  if (rc) return rc;
  return check_flag(c);
}

int sgep_set_rr_every(sgep_t h, int64_t every, const void* X, const void* Y, const float* row_scale_x,
                      const float* row_scale_y, const int32_t* labels, int64_t n) {
  if (!h) return fail(SGEP_EINVAL, "handle is NULL");
  Ctx& c = *h;
  if (every < 0) return fail(SGEP_EINVAL, "every must be >= 0");
  if (every == 0) {
    c.rr_every = 0;
    c.rr_X = c.rr_Y = nullptr;
    c.rr_sx = c.rr_sy = nullptr;
    c.rr_labels = nullptr;
    c.rr_n = 0;
    return SGEP_OK;
  }
  if (c.cfg.kind == SGEP_ICA) return fail(SGEP_ENOTSUP, "the Rayleigh-Ritz correction does not take ICA");
  if (c.path == SGEP_PATH_CLUSTER)
    return fail(SGEP_ENOTSUP, "the cluster path keeps its update pending: call sgep_rayleigh_ritz between steps");
  if (!X || (c.has_y && !Y)) return fail(SGEP_EINVAL, "NULL argument");
  if (c.cfg.kind == SGEP_LDA && !labels) return fail(SGEP_EINVAL, "LDA needs labels");
  if (n < 1) return fail(SGEP_EINVAL, "n must be >= 1");
  if (int e = scale_checks(c, row_scale_x, row_scale_y)) return e;
  c.rr_every = every;
  c.rr_X = X;
  c.rr_Y = Y;
  c.rr_sx = row_scale_x;
  c.rr_sy = row_scale_y;
  c.rr_labels = labels;
  c.rr_n = n;
  return SGEP_OK;
}

int sgep_get_state(sgep_t h, void* buf, size_t* nbytes) {
  if (!h || !nbytes) return fail(SGEP_EINVAL, "NULL argument");
  Ctx& c = *h;
  const size_t dk = (size_t)c.d * c.k;
  const size_t need = sizeof(StateHeader) + 2 * dk * sizeof(float) + lda_state_bytes(c) + variant_state_bytes(c);
  if (!buf) {
    *nbytes = need;
    return SGEP_OK;
  }
  if (*nbytes < need) return fail(SGEP_EINVAL, "buffer too small");
  int rc = complete(c, (cudaStream_t)0);
  if (rc) return rc;
  StateHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "SGEPSTAT", 8);
  hd.version = 1;
  hd.kind = c.cfg.kind;
  hd.d_x = c.d_x;
  hd.d_y = c.d_y;
  hd.k = c.k;
  hd.variants = variant_flags(c);
  hd.t = c.t;
  char* p = (char*)buf;
  std::memcpy(p, &hd, sizeof(hd));
  SGEP_CUDA_TRY(cudaMemcpy(p + sizeof(hd), c.V, dk * sizeof(float), cudaMemcpyDeviceToHost));
  SGEP_CUDA_TRY(cudaMemcpy(p + sizeof(hd) + dk * sizeof(float), c.S, dk * sizeof(float),
                           cudaMemcpyDeviceToHost));
  if (c.cfg.kind == SGEP_LDA) {  // class sums, then counts
    char* q = p + sizeof(hd) + 2 * dk * sizeof(float);
    const size_t cd = (size_t)c.cfg.n_classes * c.d;
    SGEP_CUDA_TRY(cudaMemcpy(q, c.lda_sum, cd * sizeof(double), cudaMemcpyDeviceToHost));
    SGEP_CUDA_TRY(cudaMemcpy(q + cd * sizeof(double), c.lda_cnt, c.cfg.n_classes * sizeof(double),
                             cudaMemcpyDeviceToHost));
  }
  {
    char* q = p + sizeof(hd) + 2 * dk * sizeof(float) + lda_state_bytes(c);
    if (c.adam_m) {  // m, s, step count
      SGEP_CUDA_TRY(cudaMemcpy(q, c.adam_m, 2 * dk * sizeof(float), cudaMemcpyDeviceToHost));
      std::memcpy(q + 2 * dk * sizeof(float), &c.adam_t, sizeof(int64_t));
      q += 2 * dk * sizeof(float) + sizeof(int64_t);
    }
    if (c.z) {
      SGEP_CUDA_TRY(cudaMemcpy(q, c.z, (size_t)c.k * sizeof(float), cudaMemcpyDeviceToHost));
      q += (size_t)c.k * sizeof(float);
    }
    if (c.cen_sum) {
      SGEP_CUDA_TRY(cudaMemcpy(q, c.cen_sum, (size_t)c.d * sizeof(double), cudaMemcpyDeviceToHost));
      std::memcpy(q + (size_t)c.d * sizeof(double), &c.cen_count, sizeof(double));
    }
  }
  *nbytes = need;
  return SGEP_OK;
}

int sgep_set_state(sgep_t h, const void* buf, size_t nbytes) {
  if (!h || !buf) return fail(SGEP_EINVAL, "NULL argument");
  Ctx& c = *h;
  const size_t dk = (size_t)c.d * c.k;
  if (nbytes < sizeof(StateHeader)) return fail(SGEP_ESTATE, "state blob too short");
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, "SGEPSTAT", 8) != 0 || hd.version != 1)
    return fail(SGEP_ESTATE, "not a state blob of this version");
  if (hd.kind != c.cfg.kind || hd.d_x != c.d_x || hd.d_y != c.d_y || hd.k != c.k)
    return fail(SGEP_ESTATE, "state blob has a different kind or shape");
  if (hd.variants != variant_flags(c))
    return fail(SGEP_ESTATE, "state blob has a different optimizer or variant");
  if (nbytes != sizeof(StateHeader) + 2 * dk * sizeof(float) + lda_state_bytes(c) + variant_state_bytes(c))
    return fail(SGEP_ESTATE, "state blob has the wrong size");
  int rc = complete(c, (cudaStream_t)0);
  if (rc) return rc;
  const char* p = (const char*)buf + sizeof(hd);
  SGEP_CUDA_TRY(cudaMemcpy(c.V, p, dk * sizeof(float), cudaMemcpyHostToDevice));
  SGEP_CUDA_TRY(cudaMemcpy(c.S, p + dk * sizeof(float), dk * sizeof(float), cudaMemcpyHostToDevice));
  if (c.cfg.kind == SGEP_LDA) {
    const char* q = p + 2 * dk * sizeof(float);
    const size_t cd = (size_t)c.cfg.n_classes * c.d;
    SGEP_CUDA_TRY(cudaMemcpy(c.lda_sum, q, cd * sizeof(double), cudaMemcpyHostToDevice));
    SGEP_CUDA_TRY(cudaMemcpy(c.lda_cnt, q + cd * sizeof(double), c.cfg.n_classes * sizeof(double),
                             cudaMemcpyHostToDevice));
    rc = lda_refresh(c, (cudaStream_t)0);
    if (rc) return rc;
    SGEP_CUDA_TRY(cudaDeviceSynchronize());
  }
  {
    const char* q = p + 2 * dk * sizeof(float) + lda_state_bytes(c);
    if (c.adam_m) {
      SGEP_CUDA_TRY(cudaMemcpy(c.adam_m, q, 2 * dk * sizeof(float), cudaMemcpyHostToDevice));
      std::memcpy(&c.adam_t, q + 2 * dk * sizeof(float), sizeof(int64_t));
      q += 2 * dk * sizeof(float) + sizeof(int64_t);
    }
    if (c.z) {
      SGEP_CUDA_TRY(cudaMemcpy(c.z, q, (size_t)c.k * sizeof(float), cudaMemcpyHostToDevice));
      q += (size_t)c.k * sizeof(float);
    }
    if (c.cen_sum) {  // sums and count, then the means they give
      SGEP_CUDA_TRY(cudaMemcpy(c.cen_sum, q, (size_t)c.d * sizeof(double), cudaMemcpyHostToDevice));
      std::memcpy(&c.cen_count, q + (size_t)c.d * sizeof(double), sizeof(double));
      rc = centring_update(c, nullptr, nullptr, 0, (cudaStream_t)0, nullptr, nullptr);
      if (rc) return rc;
      SGEP_CUDA_TRY(cudaDeviceSynchronize());
    }
  }
  c.t = hd.t;
  c.debug_valid = 0;
  c.tc_chain = 0;
  return SGEP_OK;
}

int64_t sgep_step_count(sgep_t h) { return h ? h->t : -1; }

double sgep_eta_at(sgep_t h, int64_t t) { return h ? schedule_eta(h->cfg, t) : 0.0; }

int sgep_path(sgep_t h) { return h ? h->path : SGEP_EINVAL; }

int64_t sgep_launch_count(sgep_t h) { return h ? h->launches : -1; }

int sgep_debug_products(sgep_t h, float* AV, float* BV) {
  if (!h || !AV || !BV) return fail(SGEP_EINVAL, "NULL argument");
  Ctx& c = *h;
  const size_t dk = (size_t)c.d * c.k;
  if (c.path == SGEP_PATH_CLUSTER) {
    if (!c.cl_pending) return fail(SGEP_ESTATE, "no pending products (call right after sgep_step)");
    SGEP_CUDA_TRY(cudaDeviceSynchronize());
    return cluster_products(c, AV, BV, (cudaStream_t)0);
  }
  if (c.tc_acc_stale)
    return fail(SGEP_ESTATE, "the tensor-core step kept no products (create the handle with debug = 1)");
  SGEP_CUDA_TRY(cudaDeviceSynchronize());
  SGEP_CUDA_TRY(cudaMemcpy(AV, c.acc, dk * sizeof(float), cudaMemcpyDeviceToHost));
  if (c.b_is_identity) {
    std::memset(BV, 0, dk * sizeof(float));  // B = I: B_t V is not formed
  } else {
    SGEP_CUDA_TRY(cudaMemcpy(BV, c.acc + dk, dk * sizeof(float), cudaMemcpyDeviceToHost));
  }
  return SGEP_OK;
}

int sgep_debug_update(sgep_t h, float* grad, double* terms) {
  if (!h || !grad || !terms) return fail(SGEP_EINVAL, "NULL argument");
  Ctx& c = *h;
  if (!c.cfg.debug) return fail(SGEP_ESTATE, "handle was created with debug = 0");
  int rc = complete(c, (cudaStream_t)0);
  if (rc) return rc;
  if (!c.debug_valid) return fail(SGEP_ESTATE, "no completed step since the state was set");
  const size_t dk = (size_t)c.d * c.k;
  const int k = c.k;
  SGEP_CUDA_TRY(cudaMemcpy(grad, c.grad, dk * sizeof(float), cudaMemcpyDeviceToHost));
  std::vector<float> g(2 * k * k + 2 * k);
  const bool from_tc = c.path == SGEP_PATH_TC && !c.tc_generic_step;  // a | G | b kept by the update
  SGEP_CUDA_TRY(cudaMemcpy(g.data(), from_tc ? c.tc_dbg : c.gram,
                           (from_tc ? 2 * k * k + k : g.size()) * sizeof(float), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 2 * k * k + k; ++i) terms[i] = g[i];
  return SGEP_OK;
}

const char* sgep_strerror(int status) {
  switch (status) {
    case SGEP_OK: return "ok";
    case SGEP_EINVAL: return "invalid argument";
    case SGEP_ENOMEM: return "out of memory";
    case SGEP_ECUDA: return "CUDA error";
    case SGEP_ETIMEOUT: return "device wait timed out";
    case SGEP_ENONFINITE: return "non-finite values";
    case SGEP_ELAUNCH: return "launch configuration not possible";
    case SGEP_ESTATE: return "bad state";
    case SGEP_ENOTSUP: return "not supported";
    default: return "unknown status";
  }
}

const char* sgep_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

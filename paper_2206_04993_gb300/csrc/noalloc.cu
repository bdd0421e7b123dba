// sgep_step_noalloc: one gamma-EigenGame step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host application that owns all device
// memory through its own pool and hands plugins fixed buffers, code that must
// not grow the process's device footprint after start-up, or a latency-bound
// loop where an allocation (which can synchronise the device) is not allowed.
// Such a caller passes its own inputs (X, Y, V, [Bv]) and outputs (V', [Bv]');
// the temporaries of the step live in the fixed-size device array below,
// which every GPU that loads this library holds until the process exits.
//
// The step runs the same kernels as the handle-based generic path; only the
// location of their scratch differs.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "internal.h"

namespace sgep {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SGEP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch per device
int g_num_sms[kMaxDevices] = {};

inline size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// Bytes of scratch one step needs: error word, k x k terms, row projections,
// the two d x k products and the pre-retraction V.
size_t scratch_bytes(int64_t d, int k, int64_t b) {
  const size_t kk = (size_t)k * k;
  return align256(sizeof(int)) + align256((2 * kk + 2 * k) * sizeof(float)) +
         align256((size_t)b * 2 * k * sizeof(float)) + align256(2 * (size_t)d * k * sizeof(float)) +
         align256((size_t)d * k * sizeof(float));
}

// Per-device set-up: the host-side symbol is only a stand-in, so the device
// address of the array is looked up once per device with that device current.
int device_scratch(int dev, void** addr, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sgep_step_noalloc: device ordinal out of range");
    return SGEP_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    g_num_sms[dev] = n;
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  *sms = g_num_sms[dev];
  return SGEP_OK;
}

int bad(const char* msg) {
  set_error(std::string("sgep_step_noalloc: ") + msg);
  return SGEP_EINVAL;
}

}  // namespace
}  // namespace sgep

using namespace sgep;

extern "C" int sgep_step_noalloc(const sgep_config* cfg, const void* X, const void* Y, int64_t b,
                                 const float* V, const float* S, float* V_out, float* S_out,
                                 int64_t t, void* stream) {
  if (!cfg) return bad("cfg is NULL");
  const sgep_config& g = *cfg;
  if (g.kind != SGEP_PCA && g.kind != SGEP_CCA && g.kind != SGEP_PLS)
    return bad("kind must be PCA, CCA or PLS");
  if (g.dtype != SGEP_F32 && g.dtype != SGEP_BF16) return bad("unknown dtype");
  if (g.d_x < 1 || (g.kind == SGEP_PCA ? g.d_y != 0 : g.d_y < 1)) return bad("bad d_x / d_y");
  const int64_t d = g.d_x + g.d_y;
  if (g.k < 1 || g.k > 64 || g.k > d) return bad("k must satisfy 1 <= k <= min(64, d)");
  if (!(g.rho > 0.f) || !std::isfinite(g.rho) || !(g.eps_B >= 0.f)) return bad("rho > 0 and eps_B >= 0 required");
  if (g.schedule < 0 || g.schedule > 2 ||
      (g.schedule != SGEP_SCHED_CONST && (g.t_c < 1 || g.T <= g.t_c || !(g.eta_T > 0.f) || !(g.eta_T < g.eta0))))
    return bad("invalid schedule");
  if (!X || (g.kind != SGEP_PCA && !Y) || !V || !S || !V_out || !S_out) return bad("NULL pointer");
  const bool split = g.kind == SGEP_CCA && g.split_AB;
  if (b < (split ? 2 : 1)) return bad("b too small (split batches need b >= 2)");
  if (t < 1) return bad("t must be >= 1");
  const size_t need = scratch_bytes(d, g.k, b);
  if (need > (size_t)SGEP_NOALLOC_SCRATCH_BYTES)
    return bad(("shape needs " + std::to_string(need) + " bytes of scratch, more than the fixed " +
                std::to_string((size_t)SGEP_NOALLOC_SCRATCH_BYTES) + " (reduce b, d or k)").c_str());

  if (g.optimizer != SGEP_OPT_SGD || g.variant != SGEP_ALG2 || g.center)
    return bad("Adam, Alg. 3 and running-mean centring keep state beyond V and [Bv]; use a handle (sgep_step)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  void* base = nullptr;
  int sms = 0;
  int rc = device_scratch(dev, &base, &sms);
  if (rc) return rc;

  // A context on the stack whose buffers all point into the caller's memory or the array.
  Ctx c;
  c.cfg = g;
  c.cfg.debug = 0;
  c.cfg.max_b = b;
  c.d_x = g.d_x;
  c.d_y = g.d_y;
  c.d = d;
  c.k = g.k;
  c.device = dev;
  c.num_sms = sms;
  c.b_is_identity = (g.kind == SGEP_PCA || g.kind == SGEP_PLS);
  c.has_y = (g.kind != SGEP_PCA);
  unsigned char* p = (unsigned char*)base;
  const size_t kk = (size_t)g.k * g.k;
  c.dflag = (int*)p;
  p += align256(sizeof(int));
  c.gram = (float*)p;
  p += align256((2 * kk + 2 * g.k) * sizeof(float));
  c.PQ = (float*)p;
  p += align256((size_t)b * 2 * g.k * sizeof(float));
  c.acc = (float*)p;
  p += align256(2 * (size_t)d * g.k * sizeof(float));
  c.Vtmp = (float*)p;
  // The kernels read V and [Bv] from, and write them back to, the output buffers.
  c.V = V_out;
  c.S = S_out;

  cudaStream_t s = (cudaStream_t)stream;
  const size_t dk_bytes = (size_t)d * g.k * sizeof(float);
  if (V_out != V) {
    e = cudaMemcpyAsync(V_out, V, dk_bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(V_out)");
  }
  if (S_out != S) {
    e = cudaMemcpyAsync(S_out, S, dk_bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(S_out)");
  }
  // The array keeps the previous call's contents: the error word is cleared here, the
  // accumulators and k x k terms are cleared by the step itself before use.
  e = cudaMemsetAsync(c.dflag, 0, sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(flag)");
  rc = generic_products(c, X, Y, b, s);
  if (rc) return rc;
  return generic_update(c, (float)schedule_eta(g, t), g.gamma0, s);
}

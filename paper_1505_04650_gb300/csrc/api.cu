// Status strings, ABI version and device queries.
#include <cstdlib>
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace cnmf {

// Largest grid (CTAs) of the persistent and per-SM-sized kernels launched
// from this host thread (0: the device's SM count); see
// cnmf_set_thread_cta_limit.
static thread_local int t_cta_limit = 0;

// SM count of the current device, or the calling thread's CTA limit when
// that is smaller.  Every grid that is sized per SM comes from here, so the
// limit bounds the SMs one call occupies.
int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return 1;
  }
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
        cudaSuccess)
      (void)cudaGetLastError();
    cached[dev] = v > 0 ? v : 1;
  }
  const int full = cached[dev];
  return (t_cta_limit > 0 && t_cta_limit < full) ? t_cta_limit : full;
}

bool pdl_enabled() {
  static const bool on = getenv("CNMF_NO_PDL") == nullptr;
  return on;
}

int max_smem_optin() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return 48 * 1024;
  }
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                               dev) != cudaSuccess)
      (void)cudaGetLastError();
    cached[dev] = v > 0 ? v : 48 * 1024;
  }
  return cached[dev];
}

size_t static_smem(const void* func) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return fa.sharedSizeBytes;
}

bool set_max_smem(const void* func, size_t bytes) {
  if (bytes + static_smem(func) > (size_t)max_smem_optin()) return false;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return true;
}

bool ensure_max_smem(const void* func, size_t bytes) {
  struct Done { const void* f; int dev; size_t bytes; };
  static std::mutex mu;
  static Done done[256];
  static int ndone = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lk(mu);
  for (int i = 0; i < ndone; ++i)
    if (done[i].f == func && done[i].dev == dev && done[i].bytes >= bytes)
      return true;
  if (!set_max_smem(func, bytes)) return false;
  if (ndone < 256) done[ndone++] = Done{func, dev, bytes};
  return true;
}

static thread_local char g_err[320];

void record_cuda_error(cudaError_t e, const char* file, int line) {
  const char* base = file;
  for (const char* p = file; *p; ++p)
    if (*p == '/') base = p + 1;
  snprintf(g_err, sizeof(g_err), "%s (%s) at %s:%d", cudaGetErrorName(e),
           cudaGetErrorString(e), base, line);
}

}  // namespace cnmf

extern "C" const char* cnmf_last_error(void) { return cnmf::g_err; }

extern "C" const char* cnmf_status_string(int32_t status) {
  switch (status) {
    case CNMF_OK: return "CNMF_OK";
    case CNMF_E_INVALID_ARG: return "CNMF_E_INVALID_ARG: invalid argument";
    case CNMF_E_WORKSPACE: return "CNMF_E_WORKSPACE: workspace too small";
    case CNMF_E_CUDA: return "CNMF_E_CUDA: CUDA launch or runtime error";
    case CNMF_E_CHOLESKY:
      return "CNMF_E_CHOLESKY: Gram matrix not numerically positive definite";
    case CNMF_E_NONFINITE: return "CNMF_E_NONFINITE: NaN or Inf encountered";
    case CNMF_E_TIMEOUT: return "CNMF_E_TIMEOUT: grid barrier wait expired";
    default: return "CNMF_E_UNKNOWN";
  }
}

extern "C" int32_t cnmf_abi_version(void) { return 1; }

// Self-test of the bounded grid barrier (see cnmf.h).
namespace cnmf {
__global__ void k_barrier_selftest(unsigned* bar, int rounds, int skip,
                                   uint64_t timeout_ns, int32_t* status,
                                   int32_t* out_rounds) {
  int passed = 0;
  for (int i = 0; i < rounds; ++i) {
    if ((int)blockIdx.x == skip) return;   // this CTA never arrives
    if (!grid_barrier(bar, status, timeout_ns)) break;
    ++passed;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && out_rounds) *out_rounds = passed;
}
// Ring exchange through tagged words (the ADMM sweep loop's synchronisation):
// in round t every CTA publishes (c + t, tag t) in buffer t & 1 and waits
// for the round-t words of both neighbours, so no CTA gets two rounds ahead
// of a reader of its buffer.
__global__ void k_tagwait_selftest(unsigned* bar, uint64_t* words, int rounds,
                                   int skip, uint64_t timeout_ns,
                                   int32_t* status, int32_t* out_rounds) {
  if (threadIdx.x != 0) return;
  const int G = gridDim.x, c = blockIdx.x;
  int passed = 0;
  for (int t = 1; t <= rounds; ++t) {
    if (c == skip) return;                 // this CTA never publishes
    uint64_t* buf = words + (size_t)(t & 1) * G;
    tag_put<float>(buf + c, (float)(c + t), (uint32_t)t);
    bool ok = true;
    const int nb[2] = {(c + 1) % G, (c + G - 1) % G};
    for (int j = 0; j < 2 && ok; ++j) {
      uint64_t w = ld_relaxed_u64(buf + nb[j]);
      ok = tag_spin(buf + nb[j], (uint32_t)t, w, bar, status, timeout_ns);
      if (ok && tag_value<float>(&w) != (float)(nb[j] + t)) {
        set_status(status, CNMF_E_NONFINITE);
        ok = false;
      }
    }
    if (!ok) break;
    ++passed;
  }
  if (c == 0 && out_rounds) *out_rounds = passed;
}
}  // namespace cnmf

extern "C" cnmf_status cnmf_tagwait_selftest(int32_t ctas, int32_t rounds,
                                             int32_t skip, int32_t timeout_ms,
                                             void* ws, size_t ws_bytes,
                                             int32_t* dev_status,
                                             int32_t* out_rounds,
                                             cnmf_stream_t stream) {
  if (ctas < 1 || ctas > cnmf::num_sms() || rounds < 0 || timeout_ms < 1 ||
      timeout_ms > 10000 || !ws || !dev_status ||
      ws_bytes < 256 + 16 * (size_t)ctas)
    return CNMF_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* bar = (unsigned*)ws;
  uint64_t* words = (uint64_t*)((char*)ws + 256);
  CNMF_CUDA(cudaMemsetAsync(ws, 0, 256 + 16 * (size_t)ctas, s));
  uint64_t tns = (uint64_t)timeout_ms * 1000000ull;
  void* args[] = {&bar, &words, &rounds, &skip, &tns, &dev_status, &out_rounds};
  // co-resident CTAs: a cooperative launch (they wait on one another)
  CNMF_CUDA(cudaLaunchCooperativeKernel((const void*)cnmf::k_tagwait_selftest,
                                        dim3(ctas), dim3(32), args, 0, s));
  return CNMF_OK;
}

extern "C" cnmf_status cnmf_barrier_selftest(int32_t ctas, int32_t rounds,
                                             int32_t skip, int32_t timeout_ms,
                                             void* ws, size_t ws_bytes,
                                             int32_t* dev_status,
                                             int32_t* out_rounds,
                                             cnmf_stream_t stream) {
  if (ctas < 1 || ctas > cnmf::num_sms() || rounds < 0 || timeout_ms < 1 ||
      timeout_ms > 10000 || !ws || ws_bytes < 256 || !dev_status)
    return CNMF_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* bar = (unsigned*)ws;
  CNMF_CUDA(cudaMemsetAsync(bar, 0, 256, s));
  uint64_t tns = (uint64_t)timeout_ms * 1000000ull;
  void* args[] = {&bar, &rounds, &skip, &tns, &dev_status, &out_rounds};
  CNMF_CUDA(cudaLaunchCooperativeKernel((const void*)cnmf::k_barrier_selftest,
                                        dim3(ctas), dim3(128), args, 0, s));
  return CNMF_OK;
}

extern "C" cnmf_status cnmf_set_thread_cta_limit(int32_t ctas) {
  if (ctas < 0) return CNMF_E_INVALID_ARG;
  cnmf::t_cta_limit = ctas;
  return CNMF_OK;
}

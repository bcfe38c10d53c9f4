// Shared device/host helpers for the compressed-NMF library (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "cnmf.h"

namespace cnmf {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// Element loads: A may be stored as double, float or bfloat16; arithmetic is
// done in the working type W (double for FP64 inputs, float otherwise).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(bf16 x) { return __bfloat162float(x); }
__device__ __forceinline__ double to_f(double x) { return x; }

template <typename W, typename T>
__device__ __forceinline__ W widen(T x) {
  return static_cast<W>(to_f(x));
}

// 4 consecutive elements from shared memory (16-, 8- or 32-byte aligned).
template <typename W, typename T>
__device__ __forceinline__ void lds4(const T* p, W out[4]);

template <>
__device__ __forceinline__ void lds4<float, float>(const float* p, float o[4]) {
  float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void lds4<float, bf16>(const bf16* p, float o[4]) {
  uint2 v = *reinterpret_cast<const uint2*>(p);
  o[0] = __uint_as_float(v.x << 16);
  o[1] = __uint_as_float(v.x & 0xFFFF0000u);
  o[2] = __uint_as_float(v.y << 16);
  o[3] = __uint_as_float(v.y & 0xFFFF0000u);
}
template <>
__device__ __forceinline__ void lds4<double, double>(const double* p,
                                                     double o[4]) {
  double2 a = *reinterpret_cast<const double2*>(p);
  double2 b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// Four consecutive W values to shared memory (16-byte aligned address).
template <typename W>
__device__ __forceinline__ void sts4(W* p, const W v[4]) {
  if constexpr (sizeof(W) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
}

// N consecutive W values from shared memory, vectorised when possible.
template <int N, typename W>
__device__ __forceinline__ void ldsN(const W* p, W* o) {
  if constexpr (sizeof(W) == 4 && N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 4) {
      float4 v = *reinterpret_cast<const float4*>(p + i);
      o[i] = v.x; o[i + 1] = v.y; o[i + 2] = v.z; o[i + 3] = v.w;
    }
  } else if constexpr (N % 2 == 0) {
    typedef typename std::conditional<sizeof(W) == 4, float2, double2>::type V2;
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      V2 v = *reinterpret_cast<const V2*>(p + i);
      o[i] = v.x; o[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] = p[i];
  }
}

// ---------------------------------------------------------------------------
// cp.async (16-byte global -> shared copies, L2-only caching)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s),
               "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::);
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// ---------------------------------------------------------------------------
// Status word: the first device-detected error wins; flag bits
// (CNMF_STATUS_NEGATIVE_A) are kept beside it and do not count as an error.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int32_t* st, int32_t code) {
  if (!st) return;
  int32_t old = atomicCAS(st, 0, code);   // the common case: no flag set
  while (old != 0 && (old & CNMF_STATUS_CODE_MASK) == 0) {
    const int32_t prev = atomicCAS(st, old, old | code);
    if (prev == old) return;
    old = prev;
  }
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Grid barrier for a cooperative (co-resident) grid, with a bounded wait.
// bar[0] counts arrivals since the launch (the caller zeroes it before the
// launch); bit 31 is the abort flag.  Arrival k of a CTA is ticket
// t = atomicAdd(bar, 1); the barrier it belongs to opens when the count
// reaches (t / G + 1) G, G the number of CTAs, so nothing is ever reset and
// the only round trips on the critical path are the last arrival's add and
// the waiters' next poll.  Returns false when the grid must stop (timeout
// here or elsewhere); the timeout sets CNMF_E_TIMEOUT in *status and raises
// the abort bit, so every other CTA leaves its own wait promptly.
// ---------------------------------------------------------------------------
constexpr unsigned GRID_ABORT = 0x80000000u;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, int32_t* status,
                                             uint64_t timeout_ns) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned G = gridDim.x * gridDim.y;
    __threadfence();   // this CTA's writes (ordered by the barrier above)
    const unsigned t = atomicAdd(&bar[0], 1u);
    if (t & GRID_ABORT) {
      ok = 0;
    } else {
      const unsigned target = (t / G + 1u) * G;
      uint64_t t0 = 0;
      unsigned spins = 0;
      for (;;) {
        const unsigned v = ld_acquire_gpu(&bar[0]);
        if (v & GRID_ABORT) { ok = 0; break; }
        if (v >= target) break;
        if ((++spins & 63u) == 0) {
          const uint64_t now = globaltimer_ns();
          if (t0 == 0) t0 = now;
          else if (now - t0 > timeout_ns) {
            set_status(status, CNMF_E_TIMEOUT);
            atomicOr(&bar[0], GRID_ABORT);
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// ---------------------------------------------------------------------------
// Tagged words: a 32-bit payload and a 32-bit tag in one 64-bit word, stored
// and loaded as single aligned 64-bit accesses (single-copy atomic), so a
// reader that sees the tag it expects also sees the payload stored with it.
// Producers and consumers of per-sweep data synchronise through the data
// itself instead of a grid barrier.  A value of type W takes sizeof(W) / 4
// words, each carrying the tag.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

template <typename W>
__device__ __forceinline__ void tag_put(uint64_t* p, W v, uint32_t tag) {
  const uint64_t t = (uint64_t)tag << 32;
  if constexpr (sizeof(W) == 4) {
    st_relaxed_u64(p, t | __float_as_uint(v));
  } else {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    st_relaxed_u64(p, t | (b & 0xffffffffull));
    st_relaxed_u64(p + 1, t | (b >> 32));
  }
}

template <typename W>
__device__ __forceinline__ W tag_value(const uint64_t* w) {
  if constexpr (sizeof(W) == 4) {
    return __uint_as_float((uint32_t)w[0]);
  } else {
    return __longlong_as_double(
        (long long)(((w[1] & 0xffffffffull) << 32) | (w[0] & 0xffffffffull)));
  }
}

// Re-read *p until it carries `tag` (w: the value already read).  The wait
// is bounded like grid_barrier's: false after timeout_ns (CNMF_E_TIMEOUT,
// abort bit raised in bar[0]) or when another CTA raised the abort bit.
__device__ __forceinline__ bool tag_spin(const uint64_t* p, uint32_t tag,
                                         uint64_t& w, unsigned* bar,
                                         int32_t* status,
                                         uint64_t timeout_ns) {
  uint64_t t0 = 0;
  unsigned spins = 0;
  while ((uint32_t)(w >> 32) != tag) {
    if ((++spins & 63u) == 0) {
      if (ld_acquire_gpu(bar) & GRID_ABORT) return false;
      const uint64_t now = globaltimer_ns();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > timeout_ns) {
        set_status(status, CNMF_E_TIMEOUT);
        atomicOr(bar, GRID_ABORT);
        return false;
      }
    }
    w = ld_relaxed_u64(p);
  }
  return true;
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
struct Carve {
  // Bump allocator over the caller's workspace (256-byte aligned pieces).
  char* base;
  size_t cap;
  size_t off;
  __host__ Carve(void* b, size_t c) : base((char*)b), cap(c), off(0) {}
  template <typename T>
  __host__ T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += bytes;
    return p;
  }
  __host__ bool fits() const { return off <= cap; }
};

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of a pass chain (sketch pass,
// CholeskyQR) are launched with programmatic stream serialisation, so a
// kernel's CTAs can be scheduled, and run their set-up, while the kernel
// before it in the stream finishes.  Every kernel so launched calls
// pdl_wait() before it touches memory that an earlier kernel writes or
// reads (griddepcontrol.wait returns once the preceding grid has completed
// and its writes are visible; it returns at once in a normally launched
// kernel).  Because each kernel of the chain waits before it completes,
// the wait covers every earlier kernel of the stream, not only the one
// before.  A kernel calls pdl_release() to let the next kernel launch
// before it ends (without it, the next one launches as its CTAs exit).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
bool pdl_enabled();   // false with CNMF_NO_PDL set in the environment

// kernel<<<grid, block, smem, s>>>(args...) with programmatic stream
// serialisation (where enabled); the launch error is left for
// CNMF_CHECK_LAUNCH.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block,
                       size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  (void)cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

int num_sms();                       // SM count of the current device
int max_smem_optin();                // opt-in shared memory per block (bytes)
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) that never leaves a
// pending error behind; returns false if `bytes` is not allowed.
bool set_max_smem(const void* func, size_t bytes);
size_t static_smem(const void* func);  // static shared memory of a kernel
// set_max_smem once per (kernel, device): the attribute belongs to the
// current device's context, so a process that uses several GPUs raises it
// on each of them.  Thread-safe; false if `bytes` is not allowed.
bool ensure_max_smem(const void* func, size_t bytes);
// Remembers (per host thread) the CUDA error behind the last CNMF_E_CUDA.
void record_cuda_error(cudaError_t e, const char* file, int line);
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int pad_k(int k) { return k <= 16 ? 16 : (k <= 32 ? 32 : (k <= 48 ? 48 : (k <= 64 ? 64 : (k <= 80 ? 80 : (k <= 96 ? 96 : 128))))); }
inline size_t wbytes(cnmf_dtype t) { return t == CNMF_F64 ? 8 : 4; }

}  // namespace cnmf

#define CNMF_CHECK_LAUNCH()                                   \
  do {                                                        \
    cudaError_t _e = cudaPeekAtLastError();                   \
    if (_e != cudaSuccess) {                                  \
      (void)cudaGetLastError();                               \
      cnmf::record_cuda_error(_e, __FILE__, __LINE__);        \
      return CNMF_E_CUDA;                                     \
    }                                                         \
  } while (0)

// Check a CUDA runtime call that returns cudaError_t.
#define CNMF_CUDA(call)                                       \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) {                                  \
      (void)cudaGetLastError();                               \
      cnmf::record_cuda_error(_e, __FILE__, __LINE__);        \
      return CNMF_E_CUDA;                                     \
    }                                                         \
  } while (0)

#define CNMF_TRY(expr)                  \
  do {                                  \
    cnmf_status _s = (expr);            \
    if (_s != CNMF_OK) return _s;       \
  } while (0)

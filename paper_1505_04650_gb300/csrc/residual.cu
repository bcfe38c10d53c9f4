// Relative reconstruction error of Sec. V: ||A - U V||_F^2 and ||A||_F^2 in
// one read of A.  64 x 64 tiles of A; the matching 64 rows of U and of
// Vt = V^T are staged in shared memory and each thread forms a 4 x 4 block
// of U V^T (FMA over r), subtracts it from A and accumulates squares (FP32
// within a tile, FP64 across tiles).  A persistent grid writes one FP64
// partial pair per CTA; a second launch sums them in CTA order.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

constexpr int RS_NT = 256;
constexpr int RS_T = 64;

// The tiles cta, cta + ncta, ... of one problem; the CTA's FP64 pair goes
// to part[0], part[1].
template <typename TA, typename W>
__device__ __forceinline__ void res_tiles(const TA* __restrict__ A, int64_t m,
                                          int64_t n, int64_t lda,
                                          const W* __restrict__ U,
                                          const W* __restrict__ Vt, int r,
                                          int64_t cta, int64_t ncta,
                                          double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int RPAD = r + 1;
  W* Us = reinterpret_cast<W*>(smem);   // 64 x (r+1)
  W* Vs = Us + RS_T * RPAD;             // 64 x (r+1)
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int64_t tm = ceil_div(m, RS_T), tn = ceil_div(n, RS_T);
  const int64_t ntiles = tm * tn;
  double e2 = 0.0, a2 = 0.0;
  for (int64_t t = cta; t < ntiles; t += ncta) {
    const int64_t i0 = (t / tn) * RS_T, j0 = (t % tn) * RS_T;
    __syncthreads();
    for (int e = threadIdx.x; e < RS_T * r; e += RS_NT) {
      int i = e / r, b = e % r;
      Us[i * RPAD + b] = (i0 + i < m) ? U[(i0 + i) * r + b] : W(0);
      Vs[i * RPAD + b] = (j0 + i < n) ? Vt[(j0 + i) * r + b] : W(0);
    }
    __syncthreads();
    W acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = W(0);
    for (int l = 0; l < r; ++l) {
      W uu[4], vv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) uu[a] = Us[(ty + 16 * a) * RPAD + l];
#pragma unroll
      for (int b = 0; b < 4; ++b) vv[b] = Vs[(tx + 16 * b) * RPAD + l];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(uu[a], vv[b], acc[a][b]);
    }
    W se = W(0), sa = W(0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t i = i0 + ty + 16 * a;
      if (i >= m) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int64_t j = j0 + tx + 16 * b;
        if (j >= n) continue;
        W av = widen<W>(A[i * lda + j]);
        W df = av - acc[a][b];
        se = fma(df, df, se);
        sa = fma(av, av, sa);
      }
    }
    e2 += (double)se;
    a2 += (double)sa;
  }
  // block reduction in FP64 (fixed order)
  __shared__ double re[RS_NT], ra[RS_NT];
  re[threadIdx.x] = e2;
  ra[threadIdx.x] = a2;
  __syncthreads();
  for (int s = RS_NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      re[threadIdx.x] += re[threadIdx.x + s];
      ra[threadIdx.x] += ra[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[0] = re[0];
    part[1] = ra[0];
  }
}

template <typename TA, typename W>
__global__ void __launch_bounds__(RS_NT)
    k_residual(const TA* __restrict__ A, int64_t m, int64_t n, int64_t lda,
               const W* __restrict__ U, const W* __restrict__ Vt, int r,
               double* __restrict__ part) {
  res_tiles<TA, W>(A, m, n, lda, U, Vt, r, blockIdx.x, gridDim.x,
                   part + 2 * blockIdx.x);
}

// Many problems in one launch: blockIdx.y is the item, blockIdx.x one of
// its gridDim.x CTAs.  An item that does not fit the launch (r above max_r,
// bad sizes) reports CNMF_E_INVALID_ARG and gets NaN pairs.
template <typename TA, typename W>
__global__ void __launch_bounds__(RS_NT)
    k_residual_batched(const cnmf_residual_item* __restrict__ items,
                       int max_r, double* __restrict__ part,
                       int32_t* __restrict__ status) {
  const cnmf_residual_item it = items[blockIdx.y];
  double* p = part + 2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
  const bool ok = it.A && it.U && it.Vt && it.m >= 1 && it.n >= 1 &&
                  it.lda >= it.n && it.r >= 1 && it.r <= max_r;
  if (!ok) {   // uniform per block
    if (threadIdx.x == 0) {
      p[0] = p[1] = __longlong_as_double(0x7ff8000000000000ll);
      if (blockIdx.x == 0) set_status(status, CNMF_E_INVALID_ARG);
    }
    return;
  }
  res_tiles<TA, W>((const TA*)it.A, it.m, it.n, it.lda, (const W*)it.U,
                   (const W*)it.Vt, it.r, blockIdx.x, gridDim.x, p);
}

// out2[2 i], out2[2 i + 1] = the sums of item i's G pairs, in CTA order
__global__ void k_residual_sum_batched(const double* __restrict__ part, int G,
                                       int nitems, double* __restrict__ out2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nitems) return;
  double e = 0.0, a = 0.0;
  for (int g = 0; g < G; ++g) {
    e += part[2 * ((size_t)i * G + g)];
    a += part[2 * ((size_t)i * G + g) + 1];
  }
  out2[2 * i] = e;
  out2[2 * i + 1] = a;
}

template <typename TA, typename W>
static cnmf_status run_res_batched(const cnmf_residual_item* items, int nitems,
                                   int max_r, int G, double* out2, void* ws,
                                   int32_t* status, cudaStream_t s) {
  const size_t smem = sizeof(W) * 2 * RS_T * (max_r + 1);
  if (!ensure_max_smem((const void*)k_residual_batched<TA, W>,
                       sizeof(W) * 2 * RS_T * 129))
    return CNMF_E_INVALID_ARG;
  double* part = (double*)ws;
  k_residual_batched<TA, W><<<dim3(G, nitems), RS_NT, smem, s>>>(
      items, max_r, part, status);
  CNMF_CHECK_LAUNCH();
  k_residual_sum_batched<<<(unsigned)ceil_div(nitems, 128), 128, 0, s>>>(
      part, G, nitems, out2);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

__global__ void k_residual_sum(const double* __restrict__ part, int G,
                               double* __restrict__ out2) {
  if (threadIdx.x == 0) {
    double e = 0.0, a = 0.0;
    for (int g = 0; g < G; ++g) { e += part[2 * g]; a += part[2 * g + 1]; }
    out2[0] = e;
    out2[1] = a;
  }
}

static int res_grid(int64_t m, int64_t n) {
  int64_t tiles = ceil_div(m, RS_T) * ceil_div(n, RS_T);
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 4 * num_sms()));
}

template <typename TA, typename W>
static cnmf_status run_res(const void* A, int64_t m, int64_t n, int64_t lda,
                           const void* U, const void* Vt, int r, double* out2,
                           void* ws, cudaStream_t s) {
  const int G = res_grid(m, n);
  const size_t smem = sizeof(W) * 2 * RS_T * (r + 1);
  // raised once per (kernel, device): a second GPU needs its own raise
  if (!ensure_max_smem((const void*)k_residual<TA, W>,
                       sizeof(W) * 2 * RS_T * 129))
    return CNMF_E_INVALID_ARG;
  double* part = (double*)ws;
  k_residual<TA, W><<<G, RS_NT, smem, s>>>((const TA*)A, m, n, lda,
                                           (const W*)U, (const W*)Vt, r, part);
  CNMF_CHECK_LAUNCH();
  k_residual_sum<<<1, 32, 0, s>>>(part, G, out2);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

// ---------------------------------------------------------------------------
// Scratch for cnmf_residual_noalloc: the per-CTA partial pairs of k_residual
// live in this file-scope device array instead of a caller workspace.  Every
// GPU that loads the library holds it (16 KiB) until the process exits.
// Host code must not pass the symbol itself to a kernel -- on the host it is
// only a stand-in -- so its device address is looked up once per device.
// ---------------------------------------------------------------------------
constexpr int RS_NOALLOC_MAX_CTAS = 1024;
static __device__ __align__(256) double g_res_scratch[2 * RS_NOALLOC_MAX_CTAS];

static std::mutex g_res_scratch_mu;
static double* g_res_scratch_dev[64];

// Device address of g_res_scratch on the current device (looked up on the
// first call made with that device current).
static cnmf_status res_scratch_address(double** out) {
  int dev = 0;
  CNMF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return CNMF_E_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_res_scratch_mu);
  if (!g_res_scratch_dev[dev]) {
    void* p = nullptr;
    CNMF_CUDA(cudaGetSymbolAddress(&p, g_res_scratch));
    g_res_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_res_scratch_dev[dev];
  return CNMF_OK;
}

}  // namespace cnmf

using namespace cnmf;

extern "C" cnmf_status cnmf_residual_noalloc(const void* A, cnmf_dtype a_type,
                                             int64_t m, int64_t n, int64_t lda,
                                             const void* U, const void* Vt,
                                             cnmf_dtype w_type, int32_t r,
                                             double* out2,
                                             cnmf_stream_t stream) {
  if (!A || !U || !Vt || !out2 || m < 1 || n < 1 || lda < n || r < 1 ||
      r > 128 || (a_type != CNMF_F64 && a_type != CNMF_F32 &&
                  a_type != CNMF_BF16) ||
      (w_type != CNMF_F64 && w_type != CNMF_F32) ||
      (a_type == CNMF_F64) != (w_type == CNMF_F64))
    return CNMF_E_INVALID_ARG;
  // The grid (one partial pair per CTA) must fit the static scratch.
  if (res_grid(m, n) > RS_NOALLOC_MAX_CTAS) return CNMF_E_WORKSPACE;
  double* scratch = nullptr;
  CNMF_TRY(res_scratch_address(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  if (a_type == CNMF_F64)
    return run_res<double, double>(A, m, n, lda, U, Vt, r, out2, scratch, s);
  if (a_type == CNMF_F32)
    return run_res<float, float>(A, m, n, lda, U, Vt, r, out2, scratch, s);
  return run_res<bf16, float>(A, m, n, lda, U, Vt, r, out2, scratch, s);
}

extern "C" size_t cnmf_residual_batched_workspace(int32_t nitems,
                                                  int32_t ctas_per_item) {
  if (nitems < 1 || ctas_per_item < 1 || ctas_per_item > 1024) return 0;
  return (size_t)2 * sizeof(double) * nitems * ctas_per_item + 256;
}

extern "C" cnmf_status cnmf_residual_batched(
    const cnmf_residual_item* items, int32_t nitems, cnmf_dtype a_type,
    cnmf_dtype w_type, int32_t max_r, int32_t ctas_per_item, double* out2,
    void* ws, size_t ws_bytes, int32_t* dev_status, cnmf_stream_t stream) {
  if (!items || !out2 || !ws || nitems < 1 || nitems > 65535 || max_r < 1 ||
      max_r > 128 || ctas_per_item < 1 || ctas_per_item > 1024 ||
      (a_type != CNMF_F64 && a_type != CNMF_F32 && a_type != CNMF_BF16) ||
      (w_type != CNMF_F64 && w_type != CNMF_F32) ||
      (a_type == CNMF_F64) != (w_type == CNMF_F64))
    return CNMF_E_INVALID_ARG;
  if (ws_bytes < cnmf_residual_batched_workspace(nitems, ctas_per_item))
    return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (a_type == CNMF_F64)
    return run_res_batched<double, double>(items, nitems, max_r,
                                           ctas_per_item, out2, ws,
                                           dev_status, s);
  if (a_type == CNMF_F32)
    return run_res_batched<float, float>(items, nitems, max_r, ctas_per_item,
                                         out2, ws, dev_status, s);
  return run_res_batched<bf16, float>(items, nitems, max_r, ctas_per_item,
                                      out2, ws, dev_status, s);
}

extern "C" size_t cnmf_residual_workspace(int64_t m, int64_t n, int32_t r,
                                          cnmf_dtype a_type) {
  (void)r; (void)a_type;
  if (m < 1 || n < 1) return 0;
  return (size_t)2 * sizeof(double) * res_grid(m, n) + 256;
}

extern "C" cnmf_status cnmf_residual(const void* A, cnmf_dtype a_type,
                                     int64_t m, int64_t n, int64_t lda,
                                     const void* U, const void* Vt,
                                     cnmf_dtype w_type, int32_t r,
                                     double* out2, void* ws, size_t ws_bytes,
                                     cnmf_stream_t stream) {
  if (!A || !U || !Vt || !out2 || !ws || m < 1 || n < 1 || lda < n || r < 1 ||
      r > 128 || (a_type != CNMF_F64 && a_type != CNMF_F32 &&
                  a_type != CNMF_BF16) ||
      (w_type != CNMF_F64 && w_type != CNMF_F32) ||
      (a_type == CNMF_F64) != (w_type == CNMF_F64))
    return CNMF_E_INVALID_ARG;
  if (ws_bytes < cnmf_residual_workspace(m, n, r, a_type))
    return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (a_type == CNMF_F64)
    return run_res<double, double>(A, m, n, lda, U, Vt, r, out2, ws, s);
  if (a_type == CNMF_F32)
    return run_res<float, float>(A, m, n, lda, U, Vt, r, out2, ws, s);
  return run_res<bf16, float>(A, m, n, lda, U, Vt, r, out2, ws, s);
}

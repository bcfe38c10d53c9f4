// Nonnegativity check of A.  NMF and SNMF are stated for a nonnegative
// data matrix (Sec. II, problem statement of NMF; Sec. IV, separable NMF).
// A negative entry is not an error for the compression (a random
// projection of any matrix is defined), so it is reported, not rejected:
// the flag bit CNMF_STATUS_NEGATIVE_A is ORed into *dev_status, beside
// whatever error code the status word holds.
//
// One read of A (HBM-bound): one warp per row at a time; where the base
// and the row pitch are multiples of 16 bytes, 16-byte loads (four in
// flight per lane) over the row's whole chunks and scalar loads for its
// tail, otherwise scalar loads.  Only the n entries of each row are read,
// never the padding up to lda.  A value is negative when it compares below
// zero: -0.0 and NaN are not.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

constexpr int CK_NT = 256;

static bool ck_type(cnmf_dtype t) {
  return t == CNMF_F64 || t == CNMF_F32 || t == CNMF_BF16;
}

__device__ __forceinline__ bool ck_neg(double v) { return v < 0.0; }
__device__ __forceinline__ bool ck_neg(float v) { return v < 0.0f; }
__device__ __forceinline__ bool ck_neg(bf16 v) {
  return __bfloat162float(v) < 0.0f;
}

// any negative value among the 16 bytes of one chunk of T values
template <typename T>
__device__ __forceinline__ bool ck_chunk(const uint4& c) {
  constexpr int K = 16 / sizeof(T);
  const T* v = reinterpret_cast<const T*>(&c);
  bool neg = false;
#pragma unroll
  for (int k = 0; k < K; ++k) neg |= ck_neg(v[k]);
  return neg;
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(CK_NT)
    k_check_nonneg(const T* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                   int32_t* __restrict__ status) {
  constexpr int K = 16 / sizeof(T);   // values per 16-byte chunk
  const int lane = threadIdx.x % 32;
  const int64_t warp = ((int64_t)blockIdx.x * CK_NT + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * CK_NT / 32;
  bool neg = false;
  for (int64_t i = warp; i < m; i += nwarps) {
    const T* row = A + i * lda;
    int64_t j0 = 0;
    if (VEC) {
      const int64_t nc = n / K;   // whole chunks of the row
      const uint4* rc = reinterpret_cast<const uint4*>(row);
      int64_t c = lane;
      for (; c + 96 < nc; c += 128) {
        const uint4 a = __ldcs(rc + c), b = __ldcs(rc + c + 32),
                    d = __ldcs(rc + c + 64), e = __ldcs(rc + c + 96);
        neg |= ck_chunk<T>(a) | ck_chunk<T>(b) | ck_chunk<T>(d) |
               ck_chunk<T>(e);
      }
      for (; c < nc; c += 32) neg |= ck_chunk<T>(__ldcs(rc + c));
      j0 = nc * K;
    }
    for (int64_t j = j0 + lane; j < n; j += 32) neg |= ck_neg(row[j]);
  }
  if (__any_sync(~0u, neg) && lane == 0)
    atomicOr(status, (int32_t)CNMF_STATUS_NEGATIVE_A);
}

template <typename T>
static cnmf_status run_check(const void* A, int64_t m, int64_t n, int64_t lda,
                             int32_t* status, cudaStream_t s) {
  const bool vec = (uintptr_t)A % 16 == 0 &&
                   (lda * (int64_t)sizeof(T)) % 16 == 0;
  // eight CTAs (64 warps) per SM, or one warp per row if fewer
  const int64_t want = std::min<int64_t>((int64_t)num_sms() * 8,
                                         ceil_div(m, CK_NT / 32));
  const unsigned grid = (unsigned)std::max<int64_t>(want, 1);
  if (vec)
    k_check_nonneg<T, true><<<grid, CK_NT, 0, s>>>((const T*)A, m, n, lda,
                                                    status);
  else
    k_check_nonneg<T, false><<<grid, CK_NT, 0, s>>>((const T*)A, m, n, lda,
                                                     status);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

}  // namespace cnmf

using namespace cnmf;

extern "C" cnmf_status cnmf_check_nonnegative(const void* A,
                                              cnmf_dtype a_type, int64_t m,
                                              int64_t n, int64_t lda,
                                              int32_t* dev_status,
                                              cnmf_stream_t stream) {
  if (!A || !dev_status || !ck_type(a_type) || m < 1 || n < 1 || lda < n)
    return CNMF_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  switch (a_type) {
    case CNMF_F64: return run_check<double>(A, m, n, lda, dev_status, s);
    case CNMF_F32: return run_check<float>(A, m, n, lda, dev_status, s);
    default: return run_check<bf16>(A, m, n, lda, dev_status, s);
  }
}

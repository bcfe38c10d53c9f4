// Counter-based Gaussian test matrices (Alg. 1, first step: Omega with
// i.i.d. N(0, 1) entries).  Philox4x32-10 (Salmon et al., SC'11) written
// from its published round function, then Box-Muller (1958) in FP64.
#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0,
                                             uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
  uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
  uint32_t n0 = hi1 ^ c[1] ^ k0;
  uint32_t n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0,
                                              uint32_t k1) {
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    philox_round(c, k0, k1);
  }
}

__device__ __forceinline__ void philox_block(uint64_t seed, uint32_t stream,
                                             uint64_t b, uint32_t out[4]) {
  out[0] = (uint32_t)b;
  out[1] = (uint32_t)(b >> 32);
  out[2] = stream;
  out[3] = 0;
  philox4x32_10(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

template <typename W>
__global__ void k_gaussian(uint64_t seed, uint32_t stream, int64_t count,
                           W* __restrict__ out) {
  int64_t nblocks = (count + 3) / 4;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblocks;
       b += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x[4];
    philox_block(seed, stream, (uint64_t)b, x);
    double z[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double u1 = ((double)x[2 * h] + 0.5) * 0x1p-32;
      double u2 = ((double)x[2 * h + 1] + 0.5) * 0x1p-32;
      double rad = sqrt(-2.0 * log(u1));
      double s, c;
      sincospi(2.0 * u2, &s, &c);
      z[2 * h] = rad * c;
      z[2 * h + 1] = rad * s;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int64_t e = 4 * b + i;
      if (e < count) out[e] = (W)z[i];
    }
  }
}

__global__ void k_philox_words(uint64_t seed, uint32_t stream, int64_t first,
                               int64_t nblocks, uint32_t* __restrict__ out) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblocks;
       b += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x[4];
    philox_block(seed, stream, (uint64_t)(first + b), x);
#pragma unroll
    for (int i = 0; i < 4; ++i) out[4 * b + i] = x[i];
  }
}

cnmf_status launch_gaussian(uint64_t seed, uint32_t stream_id, int64_t count,
                            cnmf_dtype t, void* out, cudaStream_t s) {
  if (count <= 0) return CNMF_OK;
  int64_t nb = (count + 3) / 4;
  int grid = (int)std::min<int64_t>(ceil_div(nb, 256), 4 * num_sms());
  if (t == CNMF_F64)
    k_gaussian<double><<<grid, 256, 0, s>>>(seed, stream_id, count,
                                            (double*)out);
  else
    k_gaussian<float><<<grid, 256, 0, s>>>(seed, stream_id, count,
                                           (float*)out);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

}  // namespace cnmf

using namespace cnmf;

extern "C" cnmf_status cnmf_gaussian(uint64_t seed, uint32_t stream_id,
                                     int64_t rows, int64_t cols,
                                     cnmf_dtype out_type, void* out,
                                     cnmf_stream_t stream) {
  if (rows < 0 || cols < 0 || (out_type != CNMF_F64 && out_type != CNMF_F32))
    return CNMF_E_INVALID_ARG;
  if (rows * cols > 0 && !out) return CNMF_E_INVALID_ARG;
  return launch_gaussian(seed, stream_id, rows * cols, out_type, out,
                         (cudaStream_t)stream);
}

extern "C" cnmf_status cnmf_philox_words(uint64_t seed, uint32_t stream_id,
                                         int64_t first_block, int64_t nblocks,
                                         uint32_t* out, cnmf_stream_t stream) {
  if (first_block < 0 || nblocks < 0 || (nblocks > 0 && !out))
    return CNMF_E_INVALID_ARG;
  if (nblocks == 0) return CNMF_OK;
  int grid = (int)std::min<int64_t>(ceil_div(nblocks, 256), 4 * num_sms());
  k_philox_words<<<grid, 256, 0, (cudaStream_t)stream>>>(
      seed, stream_id, first_block, nblocks, out);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

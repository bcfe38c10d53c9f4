// Launch side of the batched compressed ADMM kernel (admm_batch.cuh).
#include <mutex>

#include "admm_impl.cuh"

namespace cnmf {

// Largest dynamic shared memory any item with r <= max_r, d <= max_d needs.
static size_t batch_smem(int max_r, int max_d, int dmax) {
  size_t best = 0;
  for (int r = 1; r <= max_r; ++r) {
    const int d = max_d;
    BatchSmem b(r, d, dmax);
    best = std::max(best, (size_t)b.total * sizeof(float));
  }
  return best;
}

template <int DMAX, int RMAX, int CS>
static cnmf_status launch_batch(const cnmf_batch_item* items, int n,
                                int sweeps, int max_r, int max_d,
                                int32_t* st, cudaStream_t s) {
  const void* fn = (const void*)k_admm_batch<float, DMAX, RMAX, CS>;
  const size_t smem = batch_smem(max_r, max_d, DMAX);
  if (smem > admm_limit(fn)) return CNMF_E_INVALID_ARG;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * CS));
  cfg.blockDim = dim3(AD_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CNMF_CUDA(cudaLaunchKernelEx(&cfg, k_admm_batch<float, DMAX, RMAX, CS>,
                               items, n, sweeps, st));
  return CNMF_OK;
}

template <int DMAX, int RMAX>
static cnmf_status launch_cs(const cnmf_batch_item* items, int n, int sweeps,
                             int cs, int max_r, int max_d, int32_t* st,
                             cudaStream_t s) {
  switch (cs) {
    case 1: return launch_batch<DMAX, RMAX, 1>(items, n, sweeps, max_r, max_d, st, s);
    case 2: return launch_batch<DMAX, RMAX, 2>(items, n, sweeps, max_r, max_d, st, s);
    case 4: return launch_batch<DMAX, RMAX, 4>(items, n, sweeps, max_r, max_d, st, s);
    case 8: return launch_batch<DMAX, RMAX, 8>(items, n, sweeps, max_r, max_d, st, s);
  }
  return CNMF_E_INVALID_ARG;
}

}  // namespace cnmf

using namespace cnmf;

extern "C" size_t cnmf_batch_scratch_bytes(int32_t r, int32_t d) {
  if (r < 1 || d < r) return 0;
  return (((size_t)2 * d * r * sizeof(float)) + 255) & ~size_t(255);
}

extern "C" cnmf_status cnmf_factor_batched(const cnmf_batch_item* items,
                                           int32_t nitems, int32_t sweeps,
                                           int32_t cluster_size, int32_t max_r,
                                           int32_t max_d, int32_t* dev_status,
                                           cnmf_stream_t stream) {
  if (!items || nitems < 0 || sweeps < 0 || max_r < 1 || max_r > 32 ||
      max_d < max_r || max_d > 64 ||
      (cluster_size != 1 && cluster_size != 2 && cluster_size != 4 &&
       cluster_size != 8))
    return CNMF_E_INVALID_ARG;
  if (nitems == 0) return CNMF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (max_d <= 32 && max_r <= 16)
    return launch_cs<32, 16>(items, nitems, sweeps, cluster_size, max_r, max_d,
                             dev_status, s);
  if (max_d <= 32)
    return launch_cs<32, 32>(items, nitems, sweeps, cluster_size, max_r, max_d,
                             dev_status, s);
  return launch_cs<64, 32>(items, nitems, sweeps, cluster_size, max_r, max_d,
                           dev_status, s);
}

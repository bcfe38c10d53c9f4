// double instantiation of the compressed ADMM kernels (Alg. 4); see
// admm_impl.cuh.
#include "admm_impl.cuh"

namespace cnmf {
cnmf_status run_factor_f64(const void* L, const void* Rt, const void* At,
                           int64_t m, int64_t n, int r, int d,
                           const cnmf_admm_params* p, void* U, void* Vt,
                           void* state, int resume, void* ws, size_t ws_bytes,
                           int32_t* status, cudaStream_t s) {
  return run_factor<double>(L, Rt, At, m, n, r, d, p, U, Vt, state, resume, ws,
                         ws_bytes, status, s);
}
}  // namespace cnmf

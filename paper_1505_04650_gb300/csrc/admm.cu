// C-ABI entry points of the compressed ADMM NMF iteration (Alg. 4).  The
// kernels and the launch planning live in admm_impl.cuh; admm_f32.cu and
// admm_f64.cu instantiate them per working precision.
#include "admm_impl.cuh"

namespace cnmf {
cnmf_status run_factor_f32(const void* L, const void* Rt, const void* At,
                           int64_t m, int64_t n, int r, int d,
                           const cnmf_admm_params* p, void* U, void* Vt,
                           void* state, int resume, void* ws, size_t ws_bytes,
                           int32_t* status, cudaStream_t s);
cnmf_status run_factor_f64(const void* L, const void* Rt, const void* At,
                           int64_t m, int64_t n, int r, int d,
                           const cnmf_admm_params* p, void* U, void* Vt,
                           void* state, int resume, void* ws, size_t ws_bytes,
                           int32_t* status, cudaStream_t s);
}  // namespace cnmf

using namespace cnmf;

extern "C" size_t cnmf_factor_workspace(int64_t m, int64_t n, int32_t r,
                                        int32_t d, cnmf_dtype w_type) {
  if (m < 1 || n < 1 || r < 1 || d < r || d > 128 || r > 64 ||
      (w_type != CNMF_F64 && w_type != CNMF_F32))
    return 0;
  return factor_ws(r, d, wbytes(w_type), num_sms());
}

extern "C" size_t cnmf_factor_state_bytes(int64_t m, int64_t n, int32_t r,
                                          int32_t d, cnmf_dtype w_type) {
  if (m < 1 || n < 1 || r < 1 || d < r ||
      (w_type != CNMF_F64 && w_type != CNMF_F32))
    return 0;
  return state_bytes(m, n, r, d, wbytes(w_type));
}

extern "C" cnmf_status cnmf_factor(const void* L, const void* Rt,
                                   const void* Atilde, cnmf_dtype w_type,
                                   int64_t m, int64_t n, int32_t r, int32_t d,
                                   const cnmf_admm_params* p, void* U,
                                   void* Vt, void* state, int32_t resume,
                                   void* ws, size_t ws_bytes,
                                   int32_t* dev_status, cnmf_stream_t stream) {
  if (!L || !Rt || !Atilde || !p || !U || !Vt || !state || !ws || m < 1 ||
      n < 1 || r < 1 || d < r || d > 128 || r > 64 || d > m || d > n ||
      p->iters < 0 || !(p->lambda > 0) || !(p->phi > 0) ||
      (w_type != CNMF_F64 && w_type != CNMF_F32))
    return CNMF_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (w_type == CNMF_F64)
    return run_factor_f64(L, Rt, Atilde, m, n, r, d, p, U, Vt, state, resume,
                          ws, ws_bytes, dev_status, s);
  return run_factor_f32(L, Rt, Atilde, m, n, r, d, p, U, Vt, state, resume,
                        ws, ws_bytes, dev_status, s);
}

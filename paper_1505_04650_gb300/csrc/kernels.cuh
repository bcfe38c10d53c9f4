// Internal launchers shared between the library's translation units.
#pragma once

#include "common.cuh"

namespace cnmf {

cnmf_status launch_gaussian(uint64_t seed, uint32_t stream_id, int64_t count,
                            cnmf_dtype t, void* out, cudaStream_t s);

// ---- products with A (Alg. 1 power scheme) -------------------------------
// Z (P x kz, pitch ldz) = op(A) B, op(A) = A (P = m, S = n) or A^T (P = n,
// S = m); B is S x kb (pitch ldb), columns kb..KP-1 read as zero.
struct ProdArgs {
  const void* A;
  cnmf_dtype a_type;
  int64_t m, n, lda;
  bool trans;
  const void* B;
  int64_t ldb;
  int kb;
  void* Z;
  int64_t ldz;
  int kz;
  int32_t* status = nullptr;   // device status word (tensor-core path waits)
};
size_t prod_workspace(int64_t m, int64_t n, int k, cnmf_dtype a_type);
cnmf_status launch_prod(const ProdArgs& a, void* ws, size_t ws_bytes,
                        cudaStream_t s);
// tensor-core path for BF16-stored A (tc.cu)
bool tc_applicable(const ProdArgs& a);
size_t tc_workspace(int64_t m, int64_t n, int k);
cnmf_status launch_prod_tc(const ProdArgs& a, void* ws, int32_t* status,
                           cudaStream_t s);
// fix-up of split 128-row output tiles (sketch.cu), FP32 partials
cnmf_status launch_prod_fixup_f32(void* Z, int64_t ldz, int kz, int64_t P,
                                  const float* part, int64_t U,
                                  int64_t chunks, int64_t G, int KP,
                                  cudaStream_t s);

// ---- fused two-sided pass (fused.cu): Zm = A X (m x k, pitch ldzm) and
//      Zn = A^T Y (n x k, pitch ldzn) from one read of A; FP32 or BF16 A,
//      k <= 32, A 16-byte aligned with 16-byte row pitch; X = NULL (Y = NULL)
//      leaves that product out ----------------------------------------------
struct FusedArgs {
  const void* A;
  cnmf_dtype a_type;
  int64_t m, n, lda;
  const void* X;       // n x k, pitch ldx (FP32)
  int64_t ldx;
  const void* Y;       // m x k, pitch ldy (FP32)
  int64_t ldy;
  int k;
  void* Zm;
  int64_t ldzm;
  void* Zn;
  int64_t ldzn;
  int32_t* status;
};
size_t fused_workspace(int64_t m, int64_t n, int k, cnmf_dtype a_type);
bool fused_applicable(const void* A, cnmf_dtype a_type, int64_t m, int64_t n,
                      int64_t lda, int k, bool has_x = true, bool has_y = true);
cnmf_status launch_fused(const FusedArgs& a, void* ws, size_t ws_bytes,
                         cudaStream_t s);

// ---- CholeskyQR2 on up to two tall panels at once --------------------------
struct OrthPanel {
  void* Y;       // in: rows x k panel (pitch ld); out: Q (pitch ldo) in Q
  int64_t rows;
  int64_t ld;
  void* Q;       // may equal Y when ldo == ld
  int64_t ldo;
};
size_t orth_workspace(int64_t max_rows, int k, cnmf_dtype w);
// sweeps = 2: CholeskyQR2, the unique thin Q.  sweeps = 1: one shifted
// CholeskyQR sweep, Q1 = Y R1^-1 -- a well-conditioned basis of the same
// span that differs from the thin Q by an upper-triangular factor, which
// the power passes in between final orthonormalisations do not need.
cnmf_status launch_orth(const OrthPanel* p, int npanels, int k, cnmf_dtype w,
                        void* ws, size_t ws_bytes, int32_t* dev_status,
                        cudaStream_t s, int sweeps = 2);

// ---- R^-1 (KP x KP, W-typed, KP = pad_k(k)) of the Cholesky factor of
//      Y^T Y + shift_abs I (FP64-accurate Gram, FP64 Cholesky) -------------
cnmf_status launch_gram_chol(const void* Y, int64_t ld, int64_t rows, int k,
                             cnmf_dtype w, double shift_abs, void* rinv_out,
                             void* ws, size_t ws_bytes, int32_t* status,
                             cudaStream_t s);

// ---- C (kx x ky, W-typed, pitch ldc) = X^T Y over `rows` rows --------------
size_t cross_workspace(int64_t rows, int k, cnmf_dtype w);
cnmf_status launch_cross(const void* X, int64_t ldx, const void* Y,
                         int64_t ldy, int64_t rows, int k, cnmf_dtype w,
                         void* C, int64_t ldc, void* ws, size_t ws_bytes,
                         cudaStream_t s);

// ---- copy a rows x k block between pitches (W-typed) -----------------------
cnmf_status launch_copy2d(const void* src, int64_t lds, void* dst, int64_t ldd,
                          int64_t rows, int k, cnmf_dtype w, cudaStream_t s);

}  // namespace cnmf

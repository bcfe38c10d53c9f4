// Uncompressed ADMM NMF baseline: Alg. 4 with L = I_m and R = I_n (then
// Atilde = A, Xt = X (m x r), Yt = Y (r x n); Sec. III problem "nmfEquiv",
// the ADMM of Xu et al.).  One sweep:
//   X <- (A Y^T + lam U - Lam)(Y Y^T + lam I)^-1
//   Y <- (X^T X + phi I)^-1 (X^T A + phi V - Phi)
//   U <- P+(X + Lam/lam);  Lam <- Lam + xi lam (X - U)
//   V <- P+(Y + Phi/phi);  Phi <- Phi + xi phi (Y - V)
// Tall operands are stored transposed where needed (Yt = Y^T, Vt, Phit are
// n x r).  Per sweep: A Y^T and A^T X are products with A (the dominant
// cost: two reads of A), the r x r inverses come from an FP64-accurate Gram
// and FP64 Cholesky, and one row kernel per side applies the inverse and the
// projection / multiplier updates.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

constexpr int PL_NT = 256;
constexpr int PL_ROWS = 32;

// rows i: M = Z + c P1 - P2;  X = M Rinv Rinv^T;  P1' = P+(X + P2/c);
// P2' = P2 + xi c (X - P1').  Writes X (pitch r), P1, P2.
template <typename W, int RP>
__global__ void __launch_bounds__(PL_NT)
    k_plain_rows(int64_t rows, int r, const W* __restrict__ Z, W* P1, W* P2,
                 W* __restrict__ X, const W* __restrict__ rinv, W c, W xi) {
  constexpr int PITCH = RP + 4;
  constexpr int TN = RP / 8;
  extern __shared__ __align__(16) unsigned char smem[];
  W* Rs = reinterpret_cast<W*>(smem);       // RP x RP (upper)
  W* Ms = Rs + RP * RP;                     // PL_ROWS x PITCH
  W* Ts = Ms + PL_ROWS * PITCH;             // PL_ROWS x PITCH
  for (int i = threadIdx.x; i < RP * RP; i += PL_NT) Rs[i] = rinv[i];
  const int rr = threadIdx.x / 8, c0 = (threadIdx.x % 8) * TN;
  const int64_t G = gridDim.x, cb = blockIdx.x;
  const int64_t r0 = (cb * rows) / G, r1 = ((cb + 1) * rows) / G;
  for (int64_t rb = r0; rb < r1; rb += PL_ROWS) {
    const int nr = (int)std::min<int64_t>(PL_ROWS, r1 - rb);
    for (int e = threadIdx.x; e < PL_ROWS * RP; e += PL_NT) {
      int i = e / RP, b = e % RP;
      W v = W(0);
      if (i < nr && b < r) {
        int64_t g = (rb + i) * r + b;
        v = Z[g] + c * P1[g] - P2[g];
      }
      Ms[i * PITCH + b] = v;
    }
    __syncthreads();
    W t[TN];
#pragma unroll
    for (int q = 0; q < TN; ++q) t[q] = W(0);
    for (int l = 0; l < RP; ++l) {
      W mv = Ms[rr * PITCH + l];
#pragma unroll
      for (int q = 0; q < TN; ++q) t[q] = fma(mv, Rs[l * RP + c0 + q], t[q]);
    }
#pragma unroll
    for (int q = 0; q < TN; ++q) Ts[rr * PITCH + c0 + q] = t[q];
    __syncthreads();
    W x[TN];
#pragma unroll
    for (int q = 0; q < TN; ++q) x[q] = W(0);
    for (int l = 0; l < RP; ++l) {
      W tv = Ts[rr * PITCH + l];
#pragma unroll
      for (int q = 0; q < TN; ++q) x[q] = fma(tv, Rs[(c0 + q) * RP + l], x[q]);
    }
    if (rr < nr) {
#pragma unroll
      for (int q = 0; q < TN; ++q) {
        const int b = c0 + q;
        if (b >= r) continue;
        const int64_t g = (rb + rr) * r + b;
        const W p2 = P2[g];
        W p1 = x[q] + p2 / c;
        p1 = p1 > W(0) ? p1 : W(0);
        X[g] = x[q];
        P1[g] = p1;
        P2[g] = p2 + xi * c * (x[q] - p1);
      }
    }
    __syncthreads();
  }
}

static int plain_rp(int r) { return pad_k(r); }

__global__ void k_add_count(int64_t* kc, int64_t v) { *kc += v; }

struct PlainLayout {
  void *Z, *Wn, *rinv, *prod_ws, *gram_ws;
  size_t prod_bytes, gram_bytes, bytes;
};

static PlainLayout plain_layout(void* ws, int64_t m, int64_t n, int r,
                                cnmf_dtype a_type) {
  PlainLayout L;
  cnmf_dtype w = a_type == CNMF_F64 ? CNMF_F64 : CNMF_F32;
  size_t e = wbytes(w);
  Carve cv(ws, SIZE_MAX);
  L.Z = cv.take<char>((size_t)m * r * e);
  L.Wn = cv.take<char>((size_t)n * r * e);
  L.rinv = cv.take<char>((size_t)2 * 128 * 128 * e);
  L.prod_bytes = prod_workspace(m, n, r, a_type);
  L.prod_ws = cv.take<char>(L.prod_bytes);
  L.gram_bytes = orth_workspace(std::max(m, n), r, w);
  L.gram_ws = cv.take<char>(L.gram_bytes);
  L.bytes = cv.off;
  return L;
}

static size_t plain_state(int64_t m, int64_t n, int r, size_t e) {
  size_t b = ((size_t)2 * m * r + (size_t)2 * n * r) * e;
  return ((b + 7) & ~size_t(7)) + 8;
}

template <typename W, int RP>
static cnmf_status rows_launch(int64_t rows, int r, const void* Z, void* P1,
                               void* P2, void* X, const void* rinv, double c,
                               double xi, cudaStream_t s) {
  const size_t smem = sizeof(W) * (RP * RP + 2 * PL_ROWS * (RP + 4));
  ensure_max_smem((const void*)k_plain_rows<W, RP>, smem);
  int G = (int)std::max<int64_t>(
      1, std::min<int64_t>(2 * num_sms(), ceil_div(rows, PL_ROWS)));
  k_plain_rows<W, RP><<<G, PL_NT, smem, s>>>(rows, r, (const W*)Z, (W*)P1,
                                             (W*)P2, (W*)X, (const W*)rinv,
                                             (W)c, (W)xi);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

template <typename W>
static cnmf_status rows_dispatch(int64_t rows, int r, const void* Z, void* P1,
                                 void* P2, void* X, const void* rinv, double c,
                                 double xi, cudaStream_t s) {
  switch (plain_rp(r)) {
    case 16: return rows_launch<W, 16>(rows, r, Z, P1, P2, X, rinv, c, xi, s);
    case 32: return rows_launch<W, 32>(rows, r, Z, P1, P2, X, rinv, c, xi, s);
    case 48: return rows_launch<W, 48>(rows, r, Z, P1, P2, X, rinv, c, xi, s);
    default: return rows_launch<W, 64>(rows, r, Z, P1, P2, X, rinv, c, xi, s);
  }
}

}  // namespace cnmf

using namespace cnmf;

extern "C" size_t cnmf_plain_workspace(int64_t m, int64_t n, int32_t r,
                                       cnmf_dtype a_type) {
  if (m < 1 || n < 1 || r < 1 || r > 64) return 0;
  return plain_layout(nullptr, m, n, r, a_type).bytes;
}

extern "C" size_t cnmf_plain_state_bytes(int64_t m, int64_t n, int32_t r,
                                         cnmf_dtype a_type) {
  if (m < 1 || n < 1 || r < 1) return 0;
  return plain_state(m, n, r, a_type == CNMF_F64 ? 8 : 4);
}

extern "C" cnmf_status cnmf_factor_plain(const void* A, cnmf_dtype a_type,
                                         int64_t m, int64_t n, int64_t lda,
                                         int32_t r, const cnmf_admm_params* p,
                                         void* U, void* Vt, void* state,
                                         int32_t resume, void* ws,
                                         size_t ws_bytes, int32_t* dev_status,
                                         cnmf_stream_t stream) {
  if ((a_type != CNMF_F64 && a_type != CNMF_F32 && a_type != CNMF_BF16) ||
      !A || !p || !U || !Vt || !state || !ws || m < 1 || n < 1 || lda < n ||
      r < 1 || r > 64 || r > m || r > n || p->iters < 0 || !(p->lambda > 0) ||
      !(p->phi > 0))
    return CNMF_E_INVALID_ARG;
  PlainLayout lay = plain_layout(ws, m, n, r, a_type);
  if (ws_bytes < lay.bytes) return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const cnmf_dtype w = a_type == CNMF_F64 ? CNMF_F64 : CNMF_F32;
  const size_t e = wbytes(w);
  char* st = (char*)state;
  void* Lam = st;
  void* Phit = st + (size_t)m * r * e;
  void* Yt = st + (size_t)(m + n) * r * e;
  void* X = st + (size_t)(m + 2 * n) * r * e;
  int64_t* kc = (int64_t*)(st + plain_state(m, n, r, e) - 8);
  if (!resume) {
    CNMF_CUDA(cudaMemsetAsync(Lam, 0, (size_t)m * r * e, s));
    CNMF_CUDA(cudaMemsetAsync(Phit, 0, (size_t)n * r * e, s));
    CNMF_CUDA(cudaMemsetAsync(kc, 0, 8, s));
    CNMF_CUDA(cudaMemcpyAsync(Yt, Vt, (size_t)n * r * e,
                              cudaMemcpyDeviceToDevice, s));
  }
  const int KP = pad_k(r);
  char* rinvY = (char*)lay.rinv;
  char* rinvX = rinvY + (size_t)128 * 128 * e;
  for (int it = 0; it < p->iters; ++it) {
    // X-step: Z = A Y^T; (Y Y^T + lam I)^-1 via Cholesky
    ProdArgs pa{A, a_type, m, n, lda, false, Yt, r, r, lay.Z, r, r, dev_status};
    CNMF_TRY(launch_prod(pa, lay.prod_ws, lay.prod_bytes, s));
    CNMF_TRY(launch_gram_chol(Yt, r, n, r, w, p->lambda, rinvY, lay.gram_ws,
                              lay.gram_bytes, dev_status, s));
    CNMF_TRY(w == CNMF_F64
                 ? rows_dispatch<double>(m, r, lay.Z, U, Lam, X, rinvY,
                                         p->lambda, p->xi, s)
                 : rows_dispatch<float>(m, r, lay.Z, U, Lam, X, rinvY,
                                        p->lambda, p->xi, s));
    // Y-step with the new X: W = A^T X; (X^T X + phi I)^-1
    CNMF_TRY(launch_gram_chol(X, r, m, r, w, p->phi, rinvX, lay.gram_ws,
                              lay.gram_bytes, dev_status, s));
    ProdArgs pt{A, a_type, m, n, lda, true, X, r, r, lay.Wn, r, r, dev_status};
    CNMF_TRY(launch_prod(pt, lay.prod_ws, lay.prod_bytes, s));
    CNMF_TRY(w == CNMF_F64
                 ? rows_dispatch<double>(n, r, lay.Wn, Vt, Phit, Yt, rinvX,
                                         p->phi, p->xi, s)
                 : rows_dispatch<float>(n, r, lay.Wn, Vt, Phit, Yt, rinvX,
                                        p->phi, p->xi, s));
  }
  (void)KP;
  if (p->iters > 0) {
    k_add_count<<<1, 1, 0, s>>>(kc, p->iters);
    CNMF_CHECK_LAUNCH();
  }
  return CNMF_OK;
}

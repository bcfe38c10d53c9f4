// Compressed separable NMF column selection (Alg. 3, steps 1-2; Sec. IV).
//
// Step 1: Q = Alg.1(A): A Omega, then q times (A^T Q -> orth, A Z -> orth),
//         re-orthonormalised (CholeskyQR2) after every product.
// Step 2: Rhat = Q^T A, formed as its transpose Rhat_t = A^T Q (n x d): one
//         more product with A.  The r extreme columns of Rhat are found with
//         the successive projection algorithm (Araujo et al. 2001; Gillis &
//         Vavasis 2014): repeat r times -- take the column of largest squared
//         norm (ties -> lowest index), normalise it to u, and project every
//         column onto the orthogonal complement of u.
// One SPA step is one launch over the rows of Rhat_t (L2-resident at the
// sizes this targets): each warp projects its rows with the previous u,
// computes the new squared norms, and keeps its best (norm, index); the last
// CTA to finish (atomic ticket) reduces the per-CTA candidates in CTA order,
// records the anchor and writes the next u.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

constexpr int SPA_NT = 256;

struct SpaCand {
  double val;
  long long idx;
};

__device__ __forceinline__ bool better(double v, long long i, double bv,
                                       long long bi) {
  return v > bv || (v == bv && i < bi);
}

template <typename W, int KPW>  // KPW = elements per lane (KP / 32)
__global__ void __launch_bounds__(SPA_NT)
    k_spa_step(W* __restrict__ Rh, int64_t n, int d, int64_t ld, int step,
               W* __restrict__ u, SpaCand* __restrict__ cand,
               int64_t* __restrict__ anchors, unsigned* __restrict__ ticket,
               int32_t* status) {
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int nwarps = SPA_NT / 32;
  const int64_t G = gridDim.x, c = blockIdx.x;
  const int64_t j0 = (c * n) / G, j1 = ((c + 1) * n) / G;
  W uu[KPW];
#pragma unroll
  for (int q = 0; q < KPW; ++q) {
    int k = lane + 32 * q;
    uu[q] = (step > 0 && k < d) ? __ldcg(u + k) : W(0);
  }
  double best = -1.0;
  long long besti = 0x7fffffffffffffffLL;
  for (int64_t j = j0 + warp; j < j1; j += nwarps) {
    W x[KPW];
    W* row = Rh + j * ld;
#pragma unroll
    for (int q = 0; q < KPW; ++q) {
      int k = lane + 32 * q;
      x[q] = k < d ? row[k] : W(0);
    }
    if (step > 0) {
      W dot = W(0);
#pragma unroll
      for (int q = 0; q < KPW; ++q) dot = fma(x[q], uu[q], dot);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
#pragma unroll
      for (int q = 0; q < KPW; ++q) {
        x[q] = fma(-dot, uu[q], x[q]);
        int k = lane + 32 * q;
        if (k < d) row[k] = x[q];
      }
    }
    W nn = W(0);
#pragma unroll
    for (int q = 0; q < KPW; ++q) nn = fma(x[q], x[q], nn);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    double v = (double)nn;
    if (!isfinite(v)) {
      if (lane == 0) set_status(status, CNMF_E_NONFINITE);
      v = -1.0;
    }
    if (better(v, (long long)j, best, besti)) { best = v; besti = j; }
  }
  __shared__ double sv[SPA_NT / 32];
  __shared__ long long si[SPA_NT / 32];
  if (lane == 0) { sv[warp] = best; si[warp] = besti; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = sv[0];
    long long bi = si[0];
    for (int w = 1; w < nwarps; ++w)
      if (better(sv[w], si[w], bv, bi)) { bv = sv[w]; bi = si[w]; }
    cand[c].val = bv;
    cand[c].idx = bi;
  }
  __shared__ int last_s;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(ticket, 1u);
    last_s = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  __shared__ long long win_s;
  if (threadIdx.x == 0) {
    double bv = -2.0;
    long long bi = 0x7fffffffffffffffLL;
    for (int64_t g = 0; g < G; ++g) {
      double v = __ldcg(&cand[g].val);
      long long i = __ldcg(&cand[g].idx);
      if (better(v, i, bv, bi)) { bv = v; bi = i; }
    }
    anchors[step] = bi;
    win_s = bi;
    *ticket = 0;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const W* row = Rh + win_s * ld;
    W x[KPW];
    W nn = W(0);
#pragma unroll
    for (int q = 0; q < KPW; ++q) {
      int k = lane + 32 * q;
      x[q] = k < d ? __ldcg(row + k) : W(0);
      nn = fma(x[q], x[q], nn);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    const W inv = nn > W(0) ? W(1) / sqrt(nn) : W(0);
#pragma unroll
    for (int q = 0; q < KPW; ++q) {
      int k = lane + 32 * q;
      if (k < d) u[k] = x[q] * inv;
    }
  }
}

template <typename W, int KPW>
static cnmf_status spa_launch(W* Rh, int64_t n, int d, int64_t ld, int r,
                              W* u, SpaCand* cand, int64_t* anchors,
                              unsigned* ticket, int G, int32_t* status,
                              cudaStream_t s) {
  for (int step = 0; step < r; ++step) {
    k_spa_step<W, KPW><<<G, SPA_NT, 0, s>>>(Rh, n, d, ld, step, u, cand,
                                            anchors, ticket, status);
    CNMF_CHECK_LAUNCH();
  }
  return CNMF_OK;
}

struct SnmfLayout {
  void *om, *m0, *n0, *rh, *u, *cand, *ticket, *prod_ws, *orth_ws;
  size_t prod_bytes, orth_bytes, bytes;
  int KP;
};

static int spa_grid(int64_t n) {
  return (int)std::max<int64_t>(
      1, std::min<int64_t>(2 * num_sms(), ceil_div(n, 64)));
}

static SnmfLayout snmf_layout(void* ws, int64_t m, int64_t n, int d,
                              cnmf_dtype a_type) {
  SnmfLayout L;
  cnmf_dtype w = a_type == CNMF_F64 ? CNMF_F64 : CNMF_F32;
  size_t e = wbytes(w);
  L.KP = pad_k(d);
  Carve cv(ws, SIZE_MAX);
  L.om = cv.take<char>((size_t)n * d * e);
  L.m0 = cv.take<char>((size_t)m * L.KP * e);
  L.n0 = cv.take<char>((size_t)n * L.KP * e);
  L.rh = cv.take<char>((size_t)n * L.KP * e);
  L.u = cv.take<char>((size_t)128 * e);
  L.cand = cv.take<SpaCand>((size_t)spa_grid(n));
  L.ticket = cv.take<unsigned>(64);
  L.prod_bytes = prod_workspace(m, n, d, a_type);
  L.prod_ws = cv.take<char>(L.prod_bytes);
  L.orth_bytes = orth_workspace(std::max(m, n), d, w);
  L.orth_ws = cv.take<char>(L.orth_bytes);
  L.bytes = cv.off;
  return L;
}

}  // namespace cnmf

using namespace cnmf;

extern "C" size_t snmf_select_workspace(int64_t m, int64_t n, int32_t d,
                                        cnmf_dtype a_type) {
  if (m < 1 || n < 1 || d < 1 || d > 128) return 0;
  return snmf_layout(nullptr, m, n, d, a_type).bytes;
}

extern "C" cnmf_status snmf_select(const void* A, cnmf_dtype a_type,
                                   int64_t m, int64_t n, int64_t lda,
                                   int32_t r, int32_t d, int32_t q,
                                   uint64_t seed, const void* Omega,
                                   int64_t* anchors, void* Rhat_t, void* ws,
                                   size_t ws_bytes, int32_t* dev_status,
                                   cnmf_stream_t stream) {
  if ((a_type != CNMF_F64 && a_type != CNMF_F32 && a_type != CNMF_BF16) ||
      !A || !anchors || !ws || m < 1 || n < 1 || lda < n || r < 1 || d < r ||
      d > 128 || d > m || d > n || q < 0 || q > 64)
    return CNMF_E_INVALID_ARG;
  SnmfLayout lay = snmf_layout(ws, m, n, d, a_type);
  if (ws_bytes < lay.bytes) return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const cnmf_dtype w = a_type == CNMF_F64 ? CNMF_F64 : CNMF_F32;
  const int KP = lay.KP;
  const void* X = Omega;
  int64_t ldx = d;
  if (!X) {
    CNMF_TRY(launch_gaussian(seed, 0, n * (int64_t)d, w, lay.om, s));
    X = lay.om;
  }
  // Q0 = orth(A Omega)
  ProdArgs p0{A, a_type, m, n, lda, false, X, ldx, d, lay.m0, KP, d, dev_status};
  CNMF_TRY(launch_prod(p0, lay.prod_ws, lay.prod_bytes, s));
  // one CholeskyQR sweep between products, CholeskyQR2 for the final Q
  // (see cnmf_compress)
  OrthPanel om{lay.m0, m, KP, lay.m0, KP};
  CNMF_TRY(launch_orth(&om, 1, d, w, lay.orth_ws, lay.orth_bytes, dev_status,
                       s, q == 0 ? 2 : 1));
  OrthPanel on{lay.n0, n, KP, lay.n0, KP};
  for (int j = 0; j < q; ++j) {
    ProdArgs pt{A, a_type, m, n, lda, true, lay.m0, KP, d, lay.n0, KP, d, dev_status};
    CNMF_TRY(launch_prod(pt, lay.prod_ws, lay.prod_bytes, s));
    CNMF_TRY(launch_orth(&on, 1, d, w, lay.orth_ws, lay.orth_bytes,
                         dev_status, s, 1));
    ProdArgs pa{A, a_type, m, n, lda, false, lay.n0, KP, d, lay.m0, KP, d, dev_status};
    CNMF_TRY(launch_prod(pa, lay.prod_ws, lay.prod_bytes, s));
    CNMF_TRY(launch_orth(&om, 1, d, w, lay.orth_ws, lay.orth_bytes,
                         dev_status, s, j == q - 1 ? 2 : 1));
  }
  // Rhat^T = A^T Q  (n x d)
  ProdArgs pr{A, a_type, m, n, lda, true, lay.m0, KP, d, lay.rh, KP, d, dev_status};
  CNMF_TRY(launch_prod(pr, lay.prod_ws, lay.prod_bytes, s));
  if (Rhat_t)
    CNMF_TRY(launch_copy2d(lay.rh, KP, Rhat_t, d, n, d, w, s));
  CNMF_CUDA(cudaMemsetAsync(lay.ticket, 0, sizeof(unsigned), s));
  const int G = spa_grid(n);
  const int kpw = (d + 31) / 32;
  if (w == CNMF_F64) {
    double* rh = (double*)lay.rh;
    double* u = (double*)lay.u;
    switch (kpw) {
      case 1: return spa_launch<double, 1>(rh, n, d, KP, r, u, (SpaCand*)lay.cand, anchors, (unsigned*)lay.ticket, G, dev_status, s);
      case 2: return spa_launch<double, 2>(rh, n, d, KP, r, u, (SpaCand*)lay.cand, anchors, (unsigned*)lay.ticket, G, dev_status, s);
      case 3: return spa_launch<double, 3>(rh, n, d, KP, r, u, (SpaCand*)lay.cand, anchors, (unsigned*)lay.ticket, G, dev_status, s);
      default: return spa_launch<double, 4>(rh, n, d, KP, r, u, (SpaCand*)lay.cand, anchors, (unsigned*)lay.ticket, G, dev_status, s);
    }
  }
  float* rh = (float*)lay.rh;
  float* u = (float*)lay.u;
  switch (kpw) {
    case 1: return spa_launch<float, 1>(rh, n, d, KP, r, u, (SpaCand*)lay.cand, anchors, (unsigned*)lay.ticket, G, dev_status, s);
    case 2: return spa_launch<float, 2>(rh, n, d, KP, r, u, (SpaCand*)lay.cand, anchors, (unsigned*)lay.ticket, G, dev_status, s);
    case 3: return spa_launch<float, 3>(rh, n, d, KP, r, u, (SpaCand*)lay.cand, anchors, (unsigned*)lay.ticket, G, dev_status, s);
    default: return spa_launch<float, 4>(rh, n, d, KP, r, u, (SpaCand*)lay.cand, anchors, (unsigned*)lay.ticket, G, dev_status, s);
  }
}

// Right factor of compressed separable NMF (Alg. 3 step 3; Sec. IV): for
// every column i of Rhat (d x n),
//   Y[:, i] = argmin_{h >= 0} || Rhat[:, i] - Rhat[:, K] h ||_2 .
// All n problems share the matrix B = Rhat[:, K] (d x r), so they share its
// Gram matrix G = B^T B (r x r); only b_i = B^T Rhat[:, i] differs.  The
// paper leaves the NNLS solver open; this one is projected cyclic
// coordinate descent on 1/2 h^T G h - b^T h, one column per thread:
//   h_j <- max(0, h_j - g_j / G_jj),  g <- g + (h_j,new - h_j,old) G[:, j]
// with g = G h - b (recomputed exactly every 16 sweeps, so rounding does not
// drift), until the projected gradient max_j (h_j > 0 ? |g_j| : max(-g_j, 0))
// is at most tol * max_j |b_j|, or max_sweeps.  Each step is the exact
// minimiser along one coordinate of a strictly convex quadratic (G SPD when
// B has full column rank), so the iterates converge to the unique minimiser.
//
// The sweeps start from the unconstrained minimiser G^-1 b with its negative
// entries set to zero: when it has none (most columns of a near-separable
// matrix) it is the answer, and otherwise a close start.
//
// The same batched solver runs both steps of compressed alternating NMF
// with exact nonnegative least-squares steps (Alg. 2, Sec. III; the paper
// allows any NNLS method): the X step solves, for every row of A-check,
// against Y-check^T, and the Y step, for every column of A-hat, against
// X-hat.
//
// The other inner solver of Alg. 2 is the semi-NMF multiplicative update of
// Ding, Li & Jordan (2010, Eq. 8; the compressed matrices have both signs):
// for min_{X >= 0} ||M - X F|| (F: r x d) with P = M F^T, Q = F F^T and the
// positive / negative parts B+ = (|B| + B) / 2, B- = (|B| - B) / 2,
//   X <- X * sqrt((P+ + X Q-) / (P- + X Q+))   entrywise,
// a zero denominator floored at 1e-300 (a reading: the paper and Ding et
// al. leave it open).  k_mu_step does one such update for every row, one
// row per thread, with F and Q in shared memory.
//
// Launches: (1) one CTA gathers B from the rows K of Rhat^T and forms G and
// G^-1 (Gauss-Jordan in FP64);
// (2) the library's product kernel forms Bt = Rhat^T B (n x r, = b_i^T by
// rows); (3) k_nnls: 128 columns per CTA, b staged through shared memory
// for coalesced loads, Y written by rows (coalesced over columns).
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

constexpr int NN_NT = 128;

// B (d x r, pitch rp) = rows K of Rt (n x d) transposed; G (r x r, pitch
// rp) = B^T B in W arithmetic; gd[j] = 1 / G_jj (0 for a zero column);
// Gi (r x r, pitch rp) = G^-1 by Gauss-Jordan in FP64 (no pivoting: G is
// SPD when B has full column rank; a zero pivot leaves its row at zero, and
// the solver then starts from whatever finite point that gives).
template <typename W>
constexpr size_t nnls_setup_smem(int d, int rp, int r) {
  return (((size_t)d * rp * sizeof(W) + 15) & ~size_t(15)) +
         (size_t)r * 2 * r * sizeof(double) + (size_t)r * sizeof(double);
}

// B comes either from the rows K of Rt (K non-null) or from Bsrc with
// B[k][j] = Bsrc[k sk + j sj].
template <typename W>
__global__ void __launch_bounds__(256)
    k_nnls_setup(const W* __restrict__ Rt, int64_t n, int d, int64_t ld,
                 const int64_t* __restrict__ K, const W* __restrict__ Bsrc,
                 int64_t sk, int64_t sj, int r, int rp, W* __restrict__ B,
                 W* __restrict__ G, W* __restrict__ gd, W* __restrict__ Gi,
                 int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* Bs = reinterpret_cast<W*>(smem_raw);   // d x rp
  double* J = reinterpret_cast<double*>(
      smem_raw + (((size_t)d * rp * sizeof(W) + 15) & ~size_t(15)));  // r x 2r
  double* fac = J + (size_t)r * 2 * r;                                 // r
  __shared__ double pk_s;
  __shared__ int bad_s;
  if (threadIdx.x == 0) bad_s = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < d * r; e += blockDim.x) {
    const int k = e / r, j = e % r;
    W v = W(0);
    if (K) {
      const int64_t kj = K[j];
      if (kj < 0 || kj >= n) bad_s = 1;
      else v = Rt[kj * ld + k];
    } else {
      v = Bsrc[k * sk + j * sj];
    }
    Bs[k * rp + j] = v;
    B[k * rp + j] = v;
  }
  __syncthreads();
  if (bad_s) {
    if (threadIdx.x == 0) set_status(status, CNMF_E_INVALID_ARG);
    return;
  }
  const int r2 = 2 * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e / r, c = e % r;
    W s = W(0);
    for (int k = 0; k < d; ++k) s = fma(Bs[k * rp + a], Bs[k * rp + c], s);
    G[a * rp + c] = s;
    J[a * r2 + c] = (double)s;
    J[a * r2 + r + c] = a == c ? 1.0 : 0.0;
    if (a == c) gd[a] = s > W(0) ? W(1) / s : W(0);
  }
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      const double p = J[k * r2 + k];
      pk_s = p > 0.0 ? 1.0 / p : 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < r2; c += blockDim.x) J[k * r2 + c] *= pk_s;
    for (int a = threadIdx.x; a < r; a += blockDim.x)
      if (a != k) fac[a] = J[a * r2 + k];
    __syncthreads();
    for (int e = threadIdx.x; e < r * r2; e += blockDim.x) {
      const int a = e / r2, c = e % r2;
      if (a != k) J[e] = fma(-fac[a], J[k * r2 + c], J[e]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e / r, c = e % r;
    Gi[a * rp + c] = (W)J[a * r2 + r + c];
  }
}

// One column per thread.  Bt (n x r, pitch r) holds b_i by rows; solution
// i, entry j goes to Y[j ysj + i ysc].  G, 1/diag(G) and the tile's b rows are staged in shared
// memory (dynamic: nnls_smem bytes); the column-j slice of G that a step
// needs is the same for every lane (broadcast).
template <typename W, int RMAX>
constexpr size_t nnls_smem() {
  return ((size_t)2 * RMAX * RMAX + RMAX + (size_t)NN_NT * (RMAX + 1)) *
         sizeof(W);
}

template <typename W, int RMAX>
__global__ void __launch_bounds__(NN_NT)
    k_nnls(const W* __restrict__ Bt, int64_t n, int r, int rp,
           const W* __restrict__ G, const W* __restrict__ gd,
           const W* __restrict__ Gi, int max_sweeps, W tol,
           W* __restrict__ Y, int64_t ysj, int64_t ysc,
           int32_t* __restrict__ unconverged,
           const int32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the set-up kernel found an anchor index out of range (or an earlier
  // step failed): G and its inverse were not formed, so there is nothing to
  // solve; Y is left unwritten and the status word already says why
  if (status && *reinterpret_cast<const volatile int32_t*>(status) != 0) return;
  W* Gs = reinterpret_cast<W*>(smem_raw);       // RMAX x RMAX
  W* Gis = Gs + RMAX * RMAX;                     // RMAX x RMAX
  W* gds = Gis + RMAX * RMAX;                    // RMAX
  W* bts = gds + RMAX;                           // NN_NT x (RMAX + 1)
  for (int e = threadIdx.x; e < RMAX * RMAX; e += NN_NT) {
    const int a = e / RMAX, c = e % RMAX;
    Gs[e] = (a < r && c < r) ? G[a * rp + c] : W(0);
    Gis[e] = (a < r && c < r) ? Gi[a * rp + c] : W(0);
  }
  for (int e = threadIdx.x; e < RMAX; e += NN_NT) gds[e] = e < r ? gd[e] : W(0);
  for (int64_t t0 = (int64_t)blockIdx.x * NN_NT; t0 < n;
       t0 += (int64_t)gridDim.x * NN_NT) {
    const int64_t cnt = min((int64_t)NN_NT, n - t0);
    __syncthreads();
    // this tile's b rows: cnt x r contiguous values, coalesced; padding 0
    for (int64_t e = threadIdx.x; e < (int64_t)NN_NT * RMAX; e += NN_NT) {
      const int64_t i = e / RMAX;
      const int j = (int)(e % RMAX);
      bts[i * (RMAX + 1) + j] =
          (i < cnt && j < r) ? Bt[(t0 + i) * r + j] : W(0);
    }
    __syncthreads();
    const W* b = bts + threadIdx.x * (RMAX + 1);   // this column's b
    const int64_t col = t0 + threadIdx.x;
    const bool have = threadIdx.x < cnt;
    W h[RMAX], g[RMAX];
    W bmax = W(0);
    // start: the unconstrained minimiser G^-1 b with its negative entries
    // set to zero -- already the answer when it has none (most columns of a
    // near-separable matrix), else a close starting point
#pragma unroll
    for (int a = 0; a < RMAX; ++a) {
      W sacc = W(0);
#pragma unroll
      for (int c = 0; c < RMAX; ++c) sacc = fma(Gis[a * RMAX + c], b[c], sacc);
      h[a] = sacc > W(0) ? sacc : W(0);   // NaN -> 0
      const W ab = fabs(b[a]);
      bmax = ab > bmax ? ab : bmax;
    }
    const W lim = tol * bmax;
    bool conv = false;
    // sweep sw: exact gradient g = G h - b every 16 sweeps (no drift), the
    // stopping test, then one cyclic pass over the coordinates
    for (int sw = 0; sw <= max_sweeps; ++sw) {
      if ((sw & 15) == 0) {
#pragma unroll
        for (int a = 0; a < RMAX; ++a) {
          W sacc = -b[a];
#pragma unroll
          for (int c = 0; c < RMAX; ++c) sacc = fma(Gs[a * RMAX + c], h[c], sacc);
          g[a] = sacc;
        }
      }
      W pg = W(0);
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
        const W v = h[j] > W(0) ? fabs(g[j]) : (g[j] < W(0) ? -g[j] : W(0));
        pg = (v > pg || v != v) ? v : pg;   // a NaN stays in pg
      }
      // NaN (from NaN or Inf in b or G) is never converged: the column
      // stops at once and is counted as unconverged
      conv = pg <= lim;
      const bool bad = pg != pg;
      // the warp runs until every lane is done (lanes past n count as done)
      if (__all_sync(0xffffffffu, conv || bad || !have) || sw == max_sweeps)
        break;
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
        if (j < r) {
          W hn = h[j] - g[j] * gds[j];
          hn = hn > W(0) ? hn : W(0);
          const W dl = hn - h[j];
          h[j] = hn;
          const W* gc = Gs + j * RMAX;   // G symmetric: row j = column j
#pragma unroll
          for (int a = 0; a < RMAX; ++a) g[a] = fma(dl, gc[a], g[a]);
        }
      }
    }
    if (have) {
#pragma unroll
      for (int j = 0; j < RMAX; ++j)
        if (j < r) Y[(int64_t)j * ysj + col * ysc] = h[j];
      if (!conv && unconverged) atomicAdd(unconverged, 1);
    }
  }
}

template <typename W, int RMAX>
static cnmf_status nnls_launch(int grid, const W* Bt, int64_t n, int r,
                               int rp, const W* G, const W* gd, const W* Gi,
                               int max_sweeps, W tol, W* Y, int64_t ysj,
                               int64_t ysc, int32_t* unconverged,
                               const int32_t* status, cudaStream_t s) {
  constexpr size_t smem = nnls_smem<W, RMAX>();
  if (cudaFuncSetAttribute((const void*)k_nnls<W, RMAX>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return CNMF_E_CUDA;
  k_nnls<W, RMAX><<<grid, NN_NT, smem, s>>>(Bt, n, r, rp, G, gd, Gi,
                                            max_sweeps, tol, Y, ysj, ysc,
                                            unconverged, status);
  CNMF_CUDA(cudaGetLastError());
  return CNMF_OK;
}

struct NnlsLayout {
  void* B;
  void* G;
  void* gd;
  void* Gi;
  void* bt;
  void* prod_ws;
  size_t prod_bytes;
  size_t bytes;
};

static NnlsLayout nnls_layout(void* ws, int64_t n, int d, int r,
                              cnmf_dtype w) {
  Carve cv(ws, SIZE_MAX);
  NnlsLayout L;
  const size_t e = wbytes(w);
  const int rp = r;
  L.B = cv.take<char>((size_t)d * rp * e);
  L.G = cv.take<char>((size_t)r * rp * e);
  L.gd = cv.take<char>((size_t)r * e);
  L.Gi = cv.take<char>((size_t)r * rp * e);
  L.bt = cv.take<char>((size_t)n * r * e);
  L.prod_bytes = prod_workspace(n, d, r, w);
  L.prod_ws = cv.take<char>(L.prod_bytes);
  L.bytes = cv.off;
  return L;
}

// Solves, for every row i of M (rows x d, pitch ldm), min_{h >= 0}
// ||M[i] - h^T B^T||, B (d x r) gathered from the rows K of Rt (pitch ld)
// or read from Bsrc with strides (sk, sj); solution i, entry j to
// Y[j ysj + i ysc].
template <typename W>
static cnmf_status nnls_run(const W* M, int64_t ldm, int64_t rows, int d,
                            const W* Rt, int64_t nrt, int64_t ld,
                            const int64_t* K, const W* Bsrc, int64_t sk,
                            int64_t sj, int r, int max_sweeps, double tol,
                            W* Y, int64_t ysj, int64_t ysc,
                            int32_t* unconverged, const NnlsLayout& L,
                            int32_t* status, cudaStream_t s) {
  const int rp = r;
  // dynamic shared memory plus the kernel's static words may pass the
  // default 48 KiB: always raise the limit to what this launch needs
  const size_t smem = nnls_setup_smem<W>(d, rp, r);
  if (cudaFuncSetAttribute((const void*)k_nnls_setup<W>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return CNMF_E_CUDA;
  k_nnls_setup<W><<<1, 256, smem, s>>>(Rt, nrt, d, ld, K, Bsrc, sk, sj, r, rp,
                                       (W*)L.B, (W*)L.G, (W*)L.gd, (W*)L.Gi,
                                       status);
  CNMF_CUDA(cudaGetLastError());
  // right-hand sides for every row: Bt = M B (rows x r)
  const cnmf_dtype w = sizeof(W) == 8 ? CNMF_F64 : CNMF_F32;
  ProdArgs p{M, w, rows, d, ldm, false, L.B, rp, r, L.bt, r, r, status};
  CNMF_TRY(launch_prod(p, L.prod_ws, L.prod_bytes, s));
  const int64_t tiles = (rows + NN_NT - 1) / NN_NT;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 8 * num_sms()));
  const W t = (W)tol;
  if (r <= 16)
    return nnls_launch<W, 16>(grid, (const W*)L.bt, rows, r, rp, (const W*)L.G,
                              (const W*)L.gd, (const W*)L.Gi, max_sweeps, t, Y,
                              ysj, ysc, unconverged, status, s);
  if (r <= 32)
    return nnls_launch<W, 32>(grid, (const W*)L.bt, rows, r, rp, (const W*)L.G,
                              (const W*)L.gd, (const W*)L.Gi, max_sweeps, t, Y,
                              ysj, ysc, unconverged, status, s);
  return nnls_launch<W, 64>(grid, (const W*)L.bt, rows, r, rp, (const W*)L.G,
                            (const W*)L.gd, (const W*)L.Gi, max_sweeps, t, Y,
                            ysj, ysc, unconverged, status, s);
}

struct AlsLayout {
  void* ach;    // A-check = A R^T, m x d
  void* aht;    // A-hat^T = A^T L, n x d
  void* yc;     // Y-check = Y R^T, r x d
  void* xh;     // X-hat = L^T X, d x r
  void* prod_ws;
  size_t prod_bytes;
  NnlsLayout nn;
  size_t bytes;
};

static AlsLayout als_layout(void* ws, int64_t m, int64_t n, int r, int d,
                            cnmf_dtype a_type) {
  Carve cv(ws, SIZE_MAX);
  AlsLayout L;
  const cnmf_dtype w = a_type == CNMF_F64 ? CNMF_F64 : CNMF_F32;
  const size_t e = wbytes(w);
  L.ach = cv.take<char>((size_t)m * d * e);
  L.aht = cv.take<char>((size_t)n * d * e);
  L.yc = cv.take<char>((size_t)r * d * e);
  L.xh = cv.take<char>((size_t)d * r * e);
  size_t pb = prod_workspace(m, n, d, a_type);
  pb = std::max(pb, prod_workspace(r, n, d, w));
  pb = std::max(pb, prod_workspace(m, d, r, w));
  L.prod_bytes = pb;
  L.prod_ws = cv.take<char>(pb);
  char* nb = (char*)(ws ? (char*)ws + cv.off : nullptr);
  L.nn = nnls_layout(nb, std::max(m, n), d, r, w);
  cv.take<char>(L.nn.bytes);
  L.bytes = cv.off;
  return L;
}

template <typename W>
static cnmf_status als_inputs(const void* A, cnmf_dtype a_type, int64_t m,
                              int64_t n, int64_t lda, const W* Lm,
                              const W* Rt, int d, const AlsLayout& L,
                              int32_t* status, cudaStream_t s);

template <typename W>
static cnmf_status als_run(const void* A, cnmf_dtype a_type, int64_t m,
                           int64_t n, int64_t lda, const W* Lm, const W* Rt,
                           int r, int d, int iters, int max_sweeps,
                           double tol, W* X, W* Y, int32_t* unconverged,
                           const AlsLayout& L, int32_t* status,
                           cudaStream_t s) {
  const cnmf_dtype w = sizeof(W) == 8 ? CNMF_F64 : CNMF_F32;
  W* ach = (W*)L.ach;
  W* aht = (W*)L.aht;
  W* yc = (W*)L.yc;
  W* xh = (W*)L.xh;
  // A-check = A R^T (m x d), A-hat^T = A^T L (n x d)
  CNMF_TRY(als_inputs<W>(A, a_type, m, n, lda, Lm, Rt, d, L, status, s));
  for (int it = 0; it < iters; ++it) {
    // Y-check = Y R^T (r x d)
    ProdArgs py{Y, w, r, n, n, false, Rt, d, d, yc, d, d, status};
    CNMF_TRY(launch_prod(py, L.prod_ws, L.prod_bytes, s));
    // X: row i = argmin_{x >= 0} ||A-check[i] - x Y-check||; B = Y-check^T
    CNMF_TRY(nnls_run<W>(ach, d, m, d, nullptr, 0, 0, nullptr, yc, 1, d, r,
                         max_sweeps, tol, X, 1, r, unconverged, L.nn, status,
                         s));
    // X-hat = L^T X (d x r)
    ProdArgs px{Lm, w, m, d, d, true, X, r, r, xh, r, r, status};
    CNMF_TRY(launch_prod(px, L.prod_ws, L.prod_bytes, s));
    // Y: column j = argmin_{y >= 0} ||A-hat[:, j] - X-hat y||; B = X-hat
    CNMF_TRY(nnls_run<W>(aht, d, n, d, nullptr, 0, 0, nullptr, xh, r, 1, r,
                         max_sweeps, tol, Y, n, 1, unconverged, L.nn, status,
                         s));
  }
  return CNMF_OK;
}

// ---------------------------------------------------------------------------
// Multiplicative update (Alg. 2 inner solver, Ding et al. Eq. 8): for every
// row i of M (rows x d, pitch ldm), x = X[i, :] (x_k at X[i si + k sk]),
//   p = M[i] F^T,  x_k <- x_k sqrt((p+_k + (x Q-)_k) / max(p-_k + (x Q+)_k,
//   1e-300)),  Q = F F^T,
// F (r x d) read as F[k][c] = Fs[k fk + c fc].  Every block forms F and Q
// in shared memory (r^2 d multiply-adds, in a fixed order, so every row
// sees the same Q).  A non-finite result sets CNMF_E_NONFINITE.
// ---------------------------------------------------------------------------
constexpr int MU_NT = 128;

template <typename W, int RMAX>
__global__ void __launch_bounds__(MU_NT)
    k_mu_step(const W* __restrict__ M, int64_t ldm, int64_t rows, int d,
              const W* __restrict__ Fs, int64_t fk, int64_t fc, int r,
              W* __restrict__ X, int64_t si, int64_t sk,
              int32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* F = reinterpret_cast<W*>(smem_raw);    // RMAX x d
  W* Q = F + (size_t)RMAX * d;              // RMAX x RMAX
  for (int e = threadIdx.x; e < r * d; e += MU_NT) {
    const int k = e / d, c = e - k * d;
    F[k * d + c] = Fs[k * fk + c * fc];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += MU_NT) {
    const int k = e / r, l = e - k * r;
    W q = W(0);
    for (int c = 0; c < d; ++c) q = fma(F[k * d + c], F[l * d + c], q);
    Q[k * RMAX + l] = q;
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * MU_NT + threadIdx.x;
  if (i >= rows) return;
  W p[RMAX], x[RMAX];
#pragma unroll
  for (int k = 0; k < RMAX; ++k) {
    p[k] = W(0);
    x[k] = k < r ? X[i * si + k * sk] : W(0);
  }
  const W* mi = M + i * ldm;
  for (int c = 0; c < d; ++c) {
    const W v = mi[c];
#pragma unroll
    for (int k = 0; k < RMAX; ++k)
      if (k < r) p[k] = fma(v, F[k * d + c], p[k]);
  }
  bool bad = false;
#pragma unroll
  for (int k = 0; k < RMAX; ++k) {
    if (k >= r) break;
    W num = p[k] > W(0) ? p[k] : W(0);
    W den = p[k] < W(0) ? -p[k] : W(0);
    for (int l = 0; l < r; ++l) {
      const W q = Q[l * RMAX + k];
      if (q < W(0)) num = fma(x[l], -q, num);
      else den = fma(x[l], q, den);
    }
    const W floor_den = sizeof(W) == 8 ? W(1e-300) : W(1e-38);
    const W xn = x[k] * sqrt(num / (den > floor_den ? den : floor_den));
    bad |= !isfinite((double)xn);
    X[i * si + k * sk] = xn;
  }
  if (bad) set_status(status, CNMF_E_NONFINITE);
}

template <typename W>
static cnmf_status mu_launch(const W* M, int64_t ldm, int64_t rows, int d,
                             const W* Fs, int64_t fk, int64_t fc, int r, W* X,
                             int64_t si, int64_t sk, int32_t* status,
                             cudaStream_t s) {
  const unsigned grid = (unsigned)ceil_div(rows, MU_NT);
#define MU_CASE(RM)                                                          \
  {                                                                          \
    const size_t smem = sizeof(W) * ((size_t)RM * d + (size_t)RM * RM);      \
    if (!ensure_max_smem((const void*)k_mu_step<W, RM>, smem))               \
      return CNMF_E_INVALID_ARG;                                             \
    k_mu_step<W, RM><<<grid, MU_NT, smem, s>>>(M, ldm, rows, d, Fs, fk, fc,  \
                                               r, X, si, sk, status);        \
    CNMF_CHECK_LAUNCH();                                                     \
    return CNMF_OK;                                                          \
  }
  if (r <= 16) MU_CASE(16)
  if (r <= 32) MU_CASE(32)
  MU_CASE(64)
#undef MU_CASE
}

// A-check = A R^T (m x d) and A-hat^T = A^T L (n x d): one fused read of A
// where the fused pass applies, else one read per product.
template <typename W>
static cnmf_status als_inputs(const void* A, cnmf_dtype a_type, int64_t m,
                              int64_t n, int64_t lda, const W* Lm,
                              const W* Rt, int d, const AlsLayout& L,
                              int32_t* status, cudaStream_t s) {
  if (fused_applicable(A, a_type, m, n, lda, d)) {
    FusedArgs fa{A, a_type, m, n, lda, Rt, d, Lm, d, d, L.ach, d, L.aht, d,
                 status};
    return launch_fused(fa, L.prod_ws, L.prod_bytes, s);
  }
  ProdArgs pc{A, a_type, m, n, lda, false, Rt, d, d, L.ach, d, d, status};
  CNMF_TRY(launch_prod(pc, L.prod_ws, L.prod_bytes, s));
  ProdArgs ph{A, a_type, m, n, lda, true, Lm, d, d, L.aht, d, d, status};
  return launch_prod(ph, L.prod_ws, L.prod_bytes, s);
}

template <typename W>
static cnmf_status mu_run(const void* A, cnmf_dtype a_type, int64_t m,
                          int64_t n, int64_t lda, const W* Lm, const W* Rt,
                          int r, int d, int iters, W* X, W* Y,
                          const AlsLayout& L, int32_t* status,
                          cudaStream_t s) {
  const cnmf_dtype w = sizeof(W) == 8 ? CNMF_F64 : CNMF_F32;
  W* ach = (W*)L.ach;
  W* aht = (W*)L.aht;
  W* yc = (W*)L.yc;
  W* xh = (W*)L.xh;
  CNMF_TRY(als_inputs<W>(A, a_type, m, n, lda, Lm, Rt, d, L, status, s));
  for (int it = 0; it < iters; ++it) {
    // Y-check = Y R^T (r x d)
    ProdArgs py{Y, w, r, n, n, false, Rt, d, d, yc, d, d, status};
    CNMF_TRY(launch_prod(py, L.prod_ws, L.prod_bytes, s));
    // X step: M = A-check, F = Y-check; X row i at X[i r + k]
    CNMF_TRY(mu_launch<W>(ach, d, m, d, yc, d, 1, r, X, r, 1, status, s));
    // X-hat = L^T X (d x r)
    ProdArgs px{Lm, w, m, d, d, true, X, r, r, xh, r, r, status};
    CNMF_TRY(launch_prod(px, L.prod_ws, L.prod_bytes, s));
    // Y step (transposed): M = A-hat^T, F = X-hat^T (F[k][c] = xh[c r + k]),
    // row j of Y^T = column j of Y (Y[k n + j])
    CNMF_TRY(mu_launch<W>(aht, d, n, d, xh, 1, r, r, Y, 1, n, status, s));
  }
  return CNMF_OK;
}

}  // namespace cnmf

using namespace cnmf;

extern "C" size_t snmf_right_factor_workspace(int64_t n, int32_t d, int32_t r,
                                              cnmf_dtype w_type) {
  if (n < 1 || d < 1 || d > 128 || r < 1 || r > 64 || r > d ||
      (w_type != CNMF_F64 && w_type != CNMF_F32))
    return 0;
  return nnls_layout(nullptr, n, d, r, w_type).bytes;
}

extern "C" cnmf_status snmf_right_factor(const void* Rhat_t, cnmf_dtype w_type,
                                         int64_t n, int32_t d, int64_t ld,
                                         const int64_t* anchors, int32_t r,
                                         int32_t max_sweeps, double tol,
                                         void* Y, int64_t ldy,
                                         int32_t* unconverged, void* ws,
                                         size_t ws_bytes, int32_t* dev_status,
                                         cnmf_stream_t stream) {
  if ((w_type != CNMF_F64 && w_type != CNMF_F32) || !Rhat_t || !anchors ||
      !Y || !ws || n < 1 || d < 1 || d > 128 || ld < d || r < 1 || r > 64 ||
      r > d || ldy < n || max_sweeps < 1 || !(tol >= 0.0))
    return CNMF_E_INVALID_ARG;
  NnlsLayout L = nnls_layout(ws, n, d, r, w_type);
  if (ws_bytes < L.bytes) return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (w_type == CNMF_F64)
    return nnls_run<double>((const double*)Rhat_t, ld, n, d,
                            (const double*)Rhat_t, n, ld, anchors, nullptr, 0,
                            0, r, max_sweeps, tol, (double*)Y, ldy, 1,
                            unconverged, L, dev_status, s);
  return nnls_run<float>((const float*)Rhat_t, ld, n, d, (const float*)Rhat_t,
                         n, ld, anchors, nullptr, 0, 0, r, max_sweeps, tol,
                         (float*)Y, ldy, 1, unconverged, L, dev_status, s);
}

extern "C" size_t cnmf_factor_als_workspace(int64_t m, int64_t n, int32_t r,
                                            int32_t d, cnmf_dtype a_type) {
  if (m < 1 || n < 1 || d < 1 || d > 128 || r < 1 || r > 64 || r > d ||
      (a_type != CNMF_F64 && a_type != CNMF_F32 && a_type != CNMF_BF16))
    return 0;
  return als_layout(nullptr, m, n, r, d, a_type).bytes;
}

extern "C" cnmf_status cnmf_factor_als(const void* A, cnmf_dtype a_type,
                                       int64_t m, int64_t n, int64_t lda,
                                       const void* L, const void* Rt,
                                       int32_t r, int32_t d, int32_t iters,
                                       int32_t max_sweeps, double tol, void* X,
                                       void* Y, int32_t* unconverged, void* ws,
                                       size_t ws_bytes, int32_t* dev_status,
                                       cnmf_stream_t stream) {
  if ((a_type != CNMF_F64 && a_type != CNMF_F32 && a_type != CNMF_BF16) ||
      !A || !L || !Rt || !X || !Y || !ws || m < 1 || n < 1 || lda < n ||
      d < 1 || d > 128 || d > m || d > n || r < 1 || r > 64 || r > d ||
      iters < 0 || max_sweeps < 1 || !(tol >= 0.0))
    return CNMF_E_INVALID_ARG;
  AlsLayout lay = als_layout(ws, m, n, r, d, a_type);
  if (ws_bytes < lay.bytes) return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (a_type == CNMF_F64)
    return als_run<double>(A, a_type, m, n, lda, (const double*)L,
                           (const double*)Rt, r, d, iters, max_sweeps, tol,
                           (double*)X, (double*)Y, unconverged, lay,
                           dev_status, s);
  return als_run<float>(A, a_type, m, n, lda, (const float*)L,
                        (const float*)Rt, r, d, iters, max_sweeps, tol,
                        (float*)X, (float*)Y, unconverged, lay, dev_status, s);
}

extern "C" size_t cnmf_factor_mu_workspace(int64_t m, int64_t n, int32_t r,
                                           int32_t d, cnmf_dtype a_type) {
  return cnmf_factor_als_workspace(m, n, r, d, a_type);
}

extern "C" cnmf_status cnmf_factor_mu(const void* A, cnmf_dtype a_type,
                                      int64_t m, int64_t n, int64_t lda,
                                      const void* L, const void* Rt, int32_t r,
                                      int32_t d, int32_t iters, void* X,
                                      void* Y, void* ws, size_t ws_bytes,
                                      int32_t* dev_status,
                                      cnmf_stream_t stream) {
  if ((a_type != CNMF_F64 && a_type != CNMF_F32 && a_type != CNMF_BF16) ||
      !A || !L || !Rt || !X || !Y || !ws || m < 1 || n < 1 || lda < n ||
      d < 1 || d > 128 || d > m || d > n || r < 1 || r > 64 || r > d ||
      iters < 0)
    return CNMF_E_INVALID_ARG;
  AlsLayout lay = als_layout(ws, m, n, r, d, a_type);
  if (ws_bytes < lay.bytes) return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (a_type == CNMF_F64)
    return mu_run<double>(A, a_type, m, n, lda, (const double*)L,
                          (const double*)Rt, r, d, iters, (double*)X,
                          (double*)Y, lay, dev_status, s);
  return mu_run<float>(A, a_type, m, n, lda, (const float*)L,
                       (const float*)Rt, r, d, iters, (float*)X, (float*)Y,
                       lay, dev_status, s);
}

// Orthonormal basis of a tall panel ("QR decomposition", last step of
// Alg. 1) by CholeskyQR2, plus small cross products C = X^T Y (used for
// A-tilde = L^T (A R^T), Alg. 4 setup).
//
// CholeskyQR2: G = Y^T Y; G + s I = R^T R (Cholesky); Q1 = Y R^-1; then the
// same once more on Q1 without shift.  Q = Y (R2 R1)^-1 is the unique thin
// Q factor of Y with positive diagonal, whatever invertible R1 is used, so
// the small shift s (which keeps the first Cholesky defined when Y is close
// to rank deficient) does not change the result.
//
// Precision: the Gram matrices are accumulated FP64-accurately.  For FP32
// panels each product a*b is split exactly into hi + lo with one FMA and
// summed with Knuth's TwoSum (double-float accumulation on the FP32 pipe;
// GB300's FP64 pipe is far slower).  Per-CTA partials are summed in FP64 in
// CTA order; the Cholesky factorisation runs in FP64 in one CTA; the
// triangular inverse and the row updates run in the working precision.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

constexpr int OR_NT = 256;
constexpr int OR_ROWS = 32;  // rows staged per block
constexpr int FIN_E = 32;    // Gram entries reduced per k_finish CTA

template <typename W>
struct GAcc;
template <>
struct GAcc<float> {
  float s, c;
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float a, float b) {
    float p = a * b;
    float pe = fmaf(a, b, -p);          // exact: a*b = p + pe
    float t = s + p;                     // TwoSum(s, p) = t + e exactly
    float bb = t - s;
    float e = (s - (t - bb)) + (p - bb);
    s = t;
    c += e + pe;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <>
struct GAcc<double> {
  double s;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

template <int KP, bool SYM>
struct GramMap {
  static constexpr int NB = KP / 4;
  static constexpr int NSUB = SYM ? NB * (NB + 1) / 2 : NB * NB;
  static constexpr int SPT = (NSUB + OR_NT - 1) / OR_NT;
  static constexpr int PITCH = KP + 4;  // staged rows: 16B aligned, skewed
  __device__ static void block_of(int sb, int& ba, int& bb) {
    if (SYM) {
      int r = 0, rem = sb;
      while (rem >= NB - r) { rem -= NB - r; ++r; }
      ba = r; bb = r + rem;
    } else {
      ba = sb / NB; bb = sb % NB;
    }
  }
};

template <typename W, int KP, bool SYM>
struct GramState {
  typedef GramMap<KP, SYM> M;
  GAcc<W> acc[M::SPT][16];
  int ba[M::SPT], bb[M::SPT];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int j = 0; j < M::SPT; ++j) {
      int sb = threadIdx.x + j * OR_NT;
      if (sb < M::NSUB) M::block_of(sb, ba[j], bb[j]); else { ba[j] = -1; bb[j] = -1; }
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[j][e].zero();
    }
  }
  // rows of Xs / Ys staged with pitch M::PITCH
  __device__ __forceinline__ void accumulate(const W* Xs, const W* Ys, int nrows) {
#pragma unroll
    for (int j = 0; j < M::SPT; ++j) {
      if (ba[j] < 0) continue;
      for (int r = 0; r < nrows; ++r) {
        W x[4], y[4];
        ldsN<4, W>(Xs + r * M::PITCH + 4 * ba[j], x);
        ldsN<4, W>(Ys + r * M::PITCH + 4 * bb[j], y);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[j][a * 4 + b].add(x[a], y[b]);
      }
    }
  }
  __device__ __forceinline__ void store(double* out) const {
#pragma unroll
    for (int j = 0; j < M::SPT; ++j) {
      if (ba[j] < 0) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          out[(4 * ba[j] + a) * KP + 4 * bb[j] + b] = acc[j][a * 4 + b].value();
    }
  }
};

struct PanelDesc {
  const void* X;   // gram: X == Y (sym) or the left factor (cross)
  const void* Y;
  int64_t ldx, ldy, rows;
};

template <typename W, int KP>
__device__ __forceinline__ void stage_rows(W* dst, const W* __restrict__ src,
                                           int64_t ld, int64_t r0, int nrows,
                                           int k) {
  constexpr int PITCH = KP + 4;
  for (int e = threadIdx.x; e < OR_ROWS * KP; e += OR_NT) {
    int r = e / KP, c = e % KP;
    dst[r * PITCH + c] = (r < nrows && c < k) ? src[(r0 + r) * ld + c] : W(0);
  }
}

// Gram (SYM) or cross products over row ranges; per-CTA partials, FP64.
template <typename W, int KP, bool SYM>
__global__ void __launch_bounds__(OR_NT)
    k_gram(PanelDesc p0, PanelDesc p1, int k, double* __restrict__ part) {
  typedef GramMap<KP, SYM> M;
  extern __shared__ __align__(16) unsigned char smem[];
  W* Xs = reinterpret_cast<W*>(smem);
  W* Ys = SYM ? Xs : Xs + OR_ROWS * M::PITCH;
  const PanelDesc& P = blockIdx.y ? p1 : p0;
  const int64_t G = gridDim.x, c = blockIdx.x;
  const int64_t r0 = (c * P.rows) / G, r1 = ((c + 1) * P.rows) / G;
  GramState<W, KP, SYM> gs;
  gs.init();
  for (int64_t rb = r0; rb < r1; rb += OR_ROWS) {
    int nr = (int)std::min<int64_t>(OR_ROWS, r1 - rb);
    stage_rows<W, KP>(Xs, (const W*)P.X, P.ldx, rb, nr, k);
    if (!SYM) stage_rows<W, KP>(Ys, (const W*)P.Y, P.ldy, rb, nr, k);
    __syncthreads();
    gs.accumulate(Xs, SYM ? Xs : Ys, nr);
    __syncthreads();
  }
  gs.store(part + ((size_t)blockIdx.y * G + c) * KP * KP);
}

// Sum partials (CTA order).  mode 0: write C (W, pitch ldc, k x k).
// mode 1: the last CTA of each panel factors G + shift I = R^T R (FP64) and
// writes R^-1 (W, KP x KP, zero outside the upper k x k triangle).
template <typename W, int KP>
__global__ void __launch_bounds__(OR_NT)
    k_finish(const double* __restrict__ part, int64_t G, int k, int mode,
             double shift_rel, double shift_abs, double* __restrict__ gfull,
             W* __restrict__ out0, W* __restrict__ out1, int64_t ldc,
             unsigned* __restrict__ tickets, int32_t* status) {
  // Each CTA sums FIN_E entries; FIN_S threads per entry split the CTAs
  // (thread j takes partials j, j + FIN_S, ...), then one thread adds the
  // FIN_S sub-sums in order -- a fixed order, so the result is deterministic.
  constexpr int FIN_S = OR_NT / FIN_E;
  __shared__ double red[FIN_E][FIN_S + 1];
  const int p = blockIdx.y;
  const int le = threadIdx.x / FIN_S, sub = threadIdx.x % FIN_S;
  const int e = blockIdx.x * FIN_E + le;
  const int a = e / KP, b = e % KP;
  W* out = p ? out1 : out0;
  const bool want = e < KP * KP && (mode == 0 || a <= b) && a < k && b < k;
  double s = 0.0;
  if (want) {
    const double* src = part + (size_t)p * G * KP * KP + e;
#pragma unroll 4
    for (int64_t c = sub; c < G; c += FIN_S) s += src[(size_t)c * KP * KP];
  }
  red[le][sub] = s;
  __syncthreads();
  if (sub == 0 && e < KP * KP && (mode == 0 || a <= b)) {
    double t = 0.0;
    for (int j = 0; j < FIN_S; ++j) t += red[le][j];
    if (mode == 0) {
      if (a < k && b < k) out[a * ldc + b] = (W)t;
    } else {
      gfull[(size_t)p * KP * KP + e] = want ? t : 0.0;
    }
  }
  if (mode == 0) return;

  __shared__ int last_s;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(&tickets[p], 1u);
    last_s = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last_s) return;
  __threadfence();

  extern __shared__ __align__(16) unsigned char smem[];
  double* R = reinterpret_cast<double*>(smem);                // KP x KP
  __shared__ double trace_s;
  __shared__ int bad_s;
  const volatile double* gv = gfull + (size_t)p * KP * KP;
  for (int i = threadIdx.x; i < KP * KP; i += OR_NT) {
    int ia = i / KP, ib = i % KP;
    R[i] = (ia <= ib && ia < k && ib < k) ? gv[i] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    int bad = 0;
    for (int j = 0; j < k; ++j) tr += R[j * KP + j];
    if (!isfinite(tr)) bad = CNMF_E_NONFINITE;
    trace_s = tr;
    bad_s = bad;
  }
  __syncthreads();
  if (bad_s) {
    if (threadIdx.x == 0) set_status(status, bad_s);
  }
  const double shift = shift_rel * trace_s + shift_abs;
  for (int j = threadIdx.x; j < k; j += OR_NT) R[j * KP + j] += shift;
  __syncthreads();
  // right-looking Cholesky, upper factor in place
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      double d = R[j * KP + j];
      if (!(d > 0.0) || !isfinite(d)) {
        set_status(status, isfinite(d) ? CNMF_E_CHOLESKY : CNMF_E_NONFINITE);
        d = 1.0;
      }
      R[j * KP + j] = sqrt(d);
    }
    __syncthreads();
    const double dj = R[j * KP + j];
    for (int l = j + 1 + threadIdx.x; l < k; l += OR_NT) R[j * KP + l] /= dj;
    __syncthreads();
    const int nt = k - j - 1;
    for (int t = threadIdx.x; t < nt * nt; t += OR_NT) {
      int ia = j + 1 + t / nt, ib = j + 1 + t % nt;
      if (ia <= ib) R[ia * KP + ib] -= R[j * KP + ia] * R[j * KP + ib];
    }
    __syncthreads();
  }
  // R^-1 (upper) straight into `out`: thread jc owns column jc, rows
  // bottom-up in lockstep (so R[i][l] reads are broadcasts).
  for (int jc = threadIdx.x; jc < KP; jc += OR_NT) {
    for (int i = KP - 1; i >= 0; --i) {
      W v = W(0);
      if (i <= jc && jc < k) {
        W s = (i == jc) ? W(1) : W(0);
        for (int l = i + 1; l <= jc; ++l) s -= (W)R[i * KP + l] * out[l * KP + jc];
        v = s / (W)R[i * KP + i];
      }
      out[i * KP + jc] = v;
    }
  }
  if (threadIdx.x == 0) tickets[p] = 0;
}

// Q = Y Rinv (in place allowed); optional Gram partials of Q.
template <typename W, int KP, bool GRAM>
__global__ void __launch_bounds__(OR_NT)
    k_apply(PanelDesc p0, PanelDesc p1, W* q0, W* q1, int64_t ldq0,
            int64_t ldq1, int k, const W* __restrict__ rinv,
            double* __restrict__ part) {
  typedef GramMap<KP, true> M;
  constexpr int PITCH = KP + 4;
  constexpr int TN = KP / 8;
  extern __shared__ __align__(16) unsigned char smem[];
  W* Rs = reinterpret_cast<W*>(smem);        // KP x KP
  W* Ys = Rs + KP * KP;                      // OR_ROWS x PITCH
  W* Qs = Ys + OR_ROWS * PITCH;              // OR_ROWS x PITCH
  const int p = blockIdx.y;
  const PanelDesc& P = p ? p1 : p0;
  W* Q = p ? q1 : q0;
  const int64_t ldq = p ? ldq1 : ldq0;
  const W* Ri = rinv + (size_t)p * KP * KP;
  for (int i = threadIdx.x; i < KP * KP; i += OR_NT) Rs[i] = Ri[i];
  const int64_t G = gridDim.x, c = blockIdx.x;
  const int64_t r0 = (c * P.rows) / G, r1 = ((c + 1) * P.rows) / G;
  GramState<W, KP, true> gs;
  if (GRAM) gs.init();
  const int r = threadIdx.x / 8, c0 = (threadIdx.x % 8) * TN;
  for (int64_t rb = r0; rb < r1; rb += OR_ROWS) {
    int nr = (int)std::min<int64_t>(OR_ROWS, r1 - rb);
    stage_rows<W, KP>(Ys, (const W*)P.Y, P.ldy, rb, nr, k);
    __syncthreads();
    W q[TN];
#pragma unroll
    for (int t = 0; t < TN; ++t) q[t] = W(0);
    for (int l = 0; l < KP; ++l) {
      W y = Ys[r * PITCH + l];
      W rr[TN];
      ldsN<TN, W>(Rs + l * KP + c0, rr);
#pragma unroll
      for (int t = 0; t < TN; ++t) q[t] = fma(y, rr[t], q[t]);
    }
#pragma unroll
    for (int t = 0; t < TN; ++t) Qs[r * PITCH + c0 + t] = q[t];
    __syncthreads();
    for (int e = threadIdx.x; e < OR_ROWS * KP; e += OR_NT) {
      int rr = e / KP, cc = e % KP;
      if (rr < nr && cc < k) Q[(rb + rr) * ldq + cc] = Qs[rr * PITCH + cc];
    }
    if (GRAM) gs.accumulate(Qs, Qs, nr);
    __syncthreads();
  }
  if (GRAM) gs.store(part + ((size_t)p * G + c) * KP * KP);
}

static int orth_kp(int k) { return pad_k(k); }

template <typename W>
static int gram_grid(int64_t rows) {
  int64_t g = std::max<int64_t>(1, std::min<int64_t>(num_sms(), ceil_div(rows, 128)));
  return (int)g;
}

size_t orth_workspace(int64_t max_rows, int k, cnmf_dtype w) {
  int KP = orth_kp(k);
  size_t G = gram_grid<float>(max_rows);
  size_t b = 0;
  b += ((2 * G * KP * KP * 8) + 255) & ~size_t(255);   // partials
  b += ((2 * KP * KP * 8) + 255) & ~size_t(255);       // gfull
  b += ((2 * KP * KP * wbytes(w)) + 255) & ~size_t(255);  // rinv
  b += 256;                                             // tickets
  return b;
}

size_t cross_workspace(int64_t rows, int k, cnmf_dtype w) {
  return orth_workspace(rows, k, w);
}

template <typename W, int KP>
static void set_smem_attrs() {
  static std::once_flag once;
  std::call_once(once, [] {
    size_t fin = sizeof(double) * KP * KP;
    set_max_smem((const void*)k_finish<W, KP>, fin);
    size_t ap = sizeof(W) * (KP * KP + 2 * OR_ROWS * (KP + 4));
    size_t gx = sizeof(W) * 2 * OR_ROWS * (KP + 4);
    set_max_smem((const void*)k_gram<W, KP, false>, gx);
    set_max_smem((const void*)k_gram<W, KP, true>, gx);
    set_max_smem((const void*)k_apply<W, KP, true>, ap);
    set_max_smem((const void*)k_apply<W, KP, false>, ap);
  });
}

template <typename W, int KP>
static cnmf_status run_orth(const OrthPanel* pp, int np, int k, void* ws,
                            int32_t* status, cudaStream_t s) {
  set_smem_attrs<W, KP>();
  int64_t maxr = 0;
  for (int i = 0; i < np; ++i) maxr = std::max(maxr, pp[i].rows);
  const int G = gram_grid<W>(maxr);
  Carve cv(ws, SIZE_MAX);
  double* part = cv.take<double>((size_t)2 * G * KP * KP);
  double* gfull = cv.take<double>((size_t)2 * KP * KP);
  W* rinv = cv.take<W>((size_t)2 * KP * KP);
  unsigned* tickets = cv.take<unsigned>(64);
  CNMF_CUDA(cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned), s));
  PanelDesc d[2];
  for (int i = 0; i < 2; ++i) {
    const OrthPanel& o = pp[std::min(i, np - 1)];
    d[i] = PanelDesc{o.Y, o.Y, o.ld, o.ld, o.rows};
  }
  dim3 grid(G, np);
  const int nfin = (int)ceil_div((int64_t)KP * KP, FIN_E);
  const size_t fin_smem = sizeof(double) * KP * KP;
  const size_t ap_smem = sizeof(W) * (KP * KP + 2 * OR_ROWS * (KP + 4));
  const double shift = sizeof(W) == 8 ? 1e-13 : 1e-11;

  k_gram<W, KP, true><<<grid, OR_NT, sizeof(W) * OR_ROWS * (KP + 4), s>>>(
      d[0], d[1], k, part);
  CNMF_CHECK_LAUNCH();
  k_finish<W, KP><<<dim3(nfin, np), OR_NT, fin_smem, s>>>(
      part, G, k, 1, shift, 0.0, gfull, rinv, rinv + KP * KP, 0, tickets, status);
  CNMF_CHECK_LAUNCH();
  k_apply<W, KP, true><<<grid, OR_NT, ap_smem, s>>>(
      d[0], d[1], (W*)d[0].Y, (W*)d[1].Y, d[0].ldy, d[1].ldy, k, rinv, part);
  CNMF_CHECK_LAUNCH();
  k_finish<W, KP><<<dim3(nfin, np), OR_NT, fin_smem, s>>>(
      part, G, k, 1, 0.0, 0.0, gfull, rinv, rinv + KP * KP, 0, tickets, status);
  CNMF_CHECK_LAUNCH();
  W* q0 = (W*)pp[0].Q;
  W* q1 = (W*)pp[std::min(1, np - 1)].Q;
  k_apply<W, KP, false><<<grid, OR_NT, ap_smem, s>>>(
      d[0], d[1], q0, q1, pp[0].ldo, pp[std::min(1, np - 1)].ldo, k, rinv,
      part);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

template <typename W, int KP>
static cnmf_status run_cross(const void* X, int64_t ldx, const void* Y,
                             int64_t ldy, int64_t rows, int k, void* C,
                             int64_t ldc, void* ws, cudaStream_t s) {
  set_smem_attrs<W, KP>();
  const int G = gram_grid<W>(rows);
  Carve cv(ws, SIZE_MAX);
  double* part = cv.take<double>((size_t)2 * G * KP * KP);
  PanelDesc d{X, Y, ldx, ldy, rows};
  k_gram<W, KP, false><<<dim3(G, 1), OR_NT,
                         sizeof(W) * 2 * OR_ROWS * (KP + 4), s>>>(d, d, k,
                                                                  part);
  CNMF_CHECK_LAUNCH();
  const int nfin = (int)ceil_div((int64_t)KP * KP, FIN_E);
  k_finish<W, KP><<<dim3(nfin, 1), OR_NT, 0, s>>>(
      part, G, k, 0, 0.0, 0.0, nullptr, (W*)C, (W*)C, ldc, nullptr, nullptr);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

template <typename W, int KP>
static cnmf_status run_gram_chol(const void* Y, int64_t ld, int64_t rows,
                                 int k, double shift_abs, void* rinv_out,
                                 void* ws, int32_t* status, cudaStream_t s) {
  set_smem_attrs<W, KP>();
  const int G = gram_grid<W>(rows);
  Carve cv(ws, SIZE_MAX);
  double* part = cv.take<double>((size_t)2 * G * KP * KP);
  double* gfull = cv.take<double>((size_t)2 * KP * KP);
  cv.take<W>((size_t)2 * KP * KP);
  unsigned* tickets = cv.take<unsigned>(64);
  CNMF_CUDA(cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned), s));
  PanelDesc d{Y, Y, ld, ld, rows};
  k_gram<W, KP, true><<<dim3(G, 1), OR_NT, sizeof(W) * OR_ROWS * (KP + 4), s>>>(
      d, d, k, part);
  CNMF_CHECK_LAUNCH();
  const int nfin = (int)ceil_div((int64_t)KP * KP, FIN_E);
  const size_t fin_smem = sizeof(double) * KP * KP;
  k_finish<W, KP><<<dim3(nfin, 1), OR_NT, fin_smem, s>>>(
      part, G, k, 1, 0.0, shift_abs, gfull, (W*)rinv_out, (W*)rinv_out, 0,
      tickets, status);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

template <typename W>
static cnmf_status orth_dispatch(const OrthPanel* p, int np, int k, void* ws,
                                 int32_t* st, cudaStream_t s) {
  switch (orth_kp(k)) {
    case 16: return run_orth<W, 16>(p, np, k, ws, st, s);
    case 32: return run_orth<W, 32>(p, np, k, ws, st, s);
    case 48: return run_orth<W, 48>(p, np, k, ws, st, s);
    case 64: return run_orth<W, 64>(p, np, k, ws, st, s);
    case 80: return run_orth<W, 80>(p, np, k, ws, st, s);
    case 96: return run_orth<W, 96>(p, np, k, ws, st, s);
    default: return run_orth<W, 128>(p, np, k, ws, st, s);
  }
}

template <typename W>
static cnmf_status cross_dispatch(const void* X, int64_t ldx, const void* Y,
                                  int64_t ldy, int64_t rows, int k, void* C,
                                  int64_t ldc, void* ws, cudaStream_t s) {
  switch (orth_kp(k)) {
    case 16: return run_cross<W, 16>(X, ldx, Y, ldy, rows, k, C, ldc, ws, s);
    case 32: return run_cross<W, 32>(X, ldx, Y, ldy, rows, k, C, ldc, ws, s);
    case 48: return run_cross<W, 48>(X, ldx, Y, ldy, rows, k, C, ldc, ws, s);
    case 64: return run_cross<W, 64>(X, ldx, Y, ldy, rows, k, C, ldc, ws, s);
    case 80: return run_cross<W, 80>(X, ldx, Y, ldy, rows, k, C, ldc, ws, s);
    case 96: return run_cross<W, 96>(X, ldx, Y, ldy, rows, k, C, ldc, ws, s);
    default: return run_cross<W, 128>(X, ldx, Y, ldy, rows, k, C, ldc, ws, s);
  }
}

cnmf_status launch_gram_chol(const void* Y, int64_t ld, int64_t rows, int k,
                             cnmf_dtype w, double shift_abs, void* rinv_out,
                             void* ws, size_t ws_bytes, int32_t* status,
                             cudaStream_t s) {
  if (ws_bytes < orth_workspace(rows, k, w)) return CNMF_E_WORKSPACE;
#define GC_CASE(KPV)                                                        \
  case KPV:                                                                 \
    return w == CNMF_F64                                                    \
               ? run_gram_chol<double, KPV>(Y, ld, rows, k, shift_abs,      \
                                            rinv_out, ws, status, s)        \
               : run_gram_chol<float, KPV>(Y, ld, rows, k, shift_abs,       \
                                           rinv_out, ws, status, s);
  switch (orth_kp(k)) {
    GC_CASE(16)
    GC_CASE(32)
    GC_CASE(48)
    GC_CASE(64)
    GC_CASE(80)
    GC_CASE(96)
    GC_CASE(128)
  }
#undef GC_CASE
  return CNMF_E_INVALID_ARG;
}

cnmf_status launch_orth(const OrthPanel* p, int np, int k, cnmf_dtype w,
                        void* ws, size_t ws_bytes, int32_t* st,
                        cudaStream_t s) {
  int64_t maxr = 0;
  for (int i = 0; i < np; ++i) maxr = std::max(maxr, p[i].rows);
  if (ws_bytes < orth_workspace(maxr, k, w)) return CNMF_E_WORKSPACE;
  return w == CNMF_F64 ? orth_dispatch<double>(p, np, k, ws, st, s)
                       : orth_dispatch<float>(p, np, k, ws, st, s);
}

cnmf_status launch_cross(const void* X, int64_t ldx, const void* Y,
                         int64_t ldy, int64_t rows, int k, cnmf_dtype w,
                         void* C, int64_t ldc, void* ws, size_t ws_bytes,
                         cudaStream_t s) {
  if (ws_bytes < cross_workspace(rows, k, w)) return CNMF_E_WORKSPACE;
  return w == CNMF_F64
             ? cross_dispatch<double>(X, ldx, Y, ldy, rows, k, C, ldc, ws, s)
             : cross_dispatch<float>(X, ldx, Y, ldy, rows, k, C, ldc, ws, s);
}

cnmf_status launch_copy2d(const void* src, int64_t lds, void* dst, int64_t ldd,
                          int64_t rows, int k, cnmf_dtype w, cudaStream_t s) {
  if (rows == 0) return CNMF_OK;
  size_t e = wbytes(w);
  CNMF_CUDA(cudaMemcpy2DAsync(dst, ldd * e, src, lds * e, k * e, rows,
                              cudaMemcpyDeviceToDevice, s));
  return CNMF_OK;
}

}  // namespace cnmf

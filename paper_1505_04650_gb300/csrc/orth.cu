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
  // With fewer 4x4 sub-blocks than threads, RPH threads share a sub-block
  // and take every RPH-th staged row; their sums are added in phase order.
  static constexpr int RPH = NSUB >= OR_NT ? 1 : OR_NT / NSUB;
  static constexpr int SPT = (NSUB + OR_NT - 1) / OR_NT;
  static constexpr int PITCH = KP + 4;  // staged rows: 16B aligned, skewed
  // shared scratch (doubles) that store() needs for the phase sums
  static constexpr int RED = RPH > 1 ? RPH * NSUB * 16 : 0;
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
  int ph;
  __device__ __forceinline__ void init() {
    ph = M::RPH > 1 ? (int)threadIdx.x / M::NSUB : 0;
#pragma unroll
    for (int j = 0; j < M::SPT; ++j) {
      const int sb = M::RPH > 1 ? (int)threadIdx.x % M::NSUB
                                : (int)threadIdx.x + j * OR_NT;
      if (sb < M::NSUB && ph < M::RPH) M::block_of(sb, ba[j], bb[j]);
      else { ba[j] = -1; bb[j] = -1; }
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[j][e].zero();
    }
  }
  // rows of Xs / Ys staged with pitch M::PITCH
  __device__ __forceinline__ void accumulate(const W* Xs, const W* Ys, int nrows) {
#pragma unroll
    for (int j = 0; j < M::SPT; ++j) {
      if (ba[j] < 0) continue;
      for (int r = ph; r < nrows; r += M::RPH) {
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
  // Called by every thread of the block.  `red`: M::RED doubles of shared
  // memory (unused when M::RPH == 1).
  __device__ __forceinline__ void store(double* out, double* red) const {
    if (M::RPH == 1) {
#pragma unroll
      for (int j = 0; j < M::SPT; ++j) {
        if (ba[j] < 0) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
            out[(4 * ba[j] + a) * KP + 4 * bb[j] + b] = acc[j][a * 4 + b].value();
      }
      return;
    }
    const int sb = (int)threadIdx.x % M::NSUB;
    __syncthreads();   // the caller's staging buffers may alias `red`
    if (ba[0] >= 0)
#pragma unroll
      for (int e = 0; e < 16; ++e)
        red[(ph * M::NSUB + sb) * 16 + e] = acc[0][e].value();
    __syncthreads();
    if (ba[0] >= 0 && ph == 0) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        double t = 0.0;
        for (int q = 0; q < M::RPH; ++q) t += red[(q * M::NSUB + sb) * 16 + e];
        out[(4 * ba[0] + e / 4) * KP + 4 * bb[0] + e % 4] = t;
      }
    }
  }
};

struct PanelDesc {
  const void* X;   // gram: X == Y (sym) or the left factor (cross)
  const void* Y;
  int64_t ldx, ldy, rows;
};

// One tile of OR_ROWS panel rows held in registers on its way to shared
// memory: all loads are issued before the first use, and the next tile is
// loaded while the current one is being consumed.
template <typename W, int KP>
struct RowTile {
  static constexpr int NIT = OR_ROWS * KP / OR_NT;
  W v[NIT];
  __device__ __forceinline__ void load(const W* __restrict__ src, int64_t ld,
                                       int64_t r0, int nrows, int k) {
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const int e = threadIdx.x + it * OR_NT;
      const int r = e / KP, c = e % KP;
      v[it] = (r < nrows && c < k) ? src[(r0 + r) * ld + c] : W(0);
    }
  }
  __device__ __forceinline__ void store(W* dst) const {
    constexpr int PITCH = KP + 4;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const int e = threadIdx.x + it * OR_NT;
      dst[(e / KP) * PITCH + e % KP] = v[it];
    }
  }
};

// Gram (SYM) or cross products over row ranges; per-CTA partials, FP64.
template <typename W, int KP, bool SYM>
__global__ void __launch_bounds__(OR_NT)
    k_gram(PanelDesc p0, PanelDesc p1, int k, double* __restrict__ part,
           unsigned* __restrict__ tickets) {
  typedef GramMap<KP, SYM> M;
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_wait();   // the panels come from the kernels before
  // the tickets of the k_finish launches that follow start at zero (each
  // k_finish's last CTA puts its ticket back to zero)
  if (tickets && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < 2)
    tickets[threadIdx.x] = 0u;
  W* Xs = reinterpret_cast<W*>(smem);
  W* Ys = SYM ? Xs : Xs + OR_ROWS * M::PITCH;
  const PanelDesc& P = blockIdx.y ? p1 : p0;
  const int64_t G = gridDim.x, c = blockIdx.x;
  const int64_t r0 = (c * P.rows) / G, r1 = ((c + 1) * P.rows) / G;
  GramState<W, KP, SYM> gs;
  gs.init();
  RowTile<W, KP> tx, ty;
  if (r0 < r1) {
    const int nr = (int)std::min<int64_t>(OR_ROWS, r1 - r0);
    tx.load((const W*)P.X, P.ldx, r0, nr, k);
    if (!SYM) ty.load((const W*)P.Y, P.ldy, r0, nr, k);
  }
  for (int64_t rb = r0; rb < r1; rb += OR_ROWS) {
    const int nr = (int)std::min<int64_t>(OR_ROWS, r1 - rb);
    tx.store(Xs);
    if (!SYM) ty.store(Ys);
    __syncthreads();
    const int64_t rn = rb + OR_ROWS;
    if (rn < r1) {   // next tile in flight during the accumulation
      const int nn = (int)std::min<int64_t>(OR_ROWS, r1 - rn);
      tx.load((const W*)P.X, P.ldx, rn, nn, k);
      if (!SYM) ty.load((const W*)P.Y, P.ldy, rn, nn, k);
    }
    gs.accumulate(Xs, SYM ? Xs : Ys, nr);
    __syncthreads();
  }
  gs.store(part + ((size_t)blockIdx.y * G + c) * KP * KP,
           reinterpret_cast<double*>(smem));
}

// Double-float numbers for the small factorisations of FP32 panels: value
// = hi + lo with |lo| <= ulp(hi) / 2, on the FP32 pipe (GB300's FP64 pipe
// is a small fraction of it).  Built from error-free transformations --
// Knuth's TwoSum, Dekker's FastTwoSum, the FMA product split -- and one
// Newton correction for the square root and the reciprocal (Karp and
// Markstein's scheme); about 2^-44 relative per operation.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_fast(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  DF s = df_two_sum(x.hi, y.hi);
  const DF t = df_two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = df_fast(s.hi, s.lo);
  s.lo += t.lo;
  return df_fast(s.hi, s.lo);
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_fast(p, e);
}
// sqrt and reciprocal: an FP32 seed (the hardware approximations, a few
// ulps) and one Newton correction from the exactly formed residual, which
// squares the seed's relative error (Karp and Markstein's scheme).
__device__ __forceinline__ DF df_sqrt(DF x) {   // x > 0
  const float y = rsqrtf(x.hi);                 // ~ x^-1/2
  const float r = x.hi * y;
  const float p = r * r, pe = fmaf(r, r, -p);
  const float res = ((x.hi - p) - pe) + x.lo;   // x - r^2
  return df_fast(r, res * (0.5f * y));
}
__device__ __forceinline__ DF df_rcp(DF y) {
  const float q = __fdividef(1.0f, y.hi);       // ~ 1 / y
  const DF qy = df_mul(DF{q, 0.0f}, y);
  const DF res = df_add(DF{1.0f, 0.0f}, DF{-qy.hi, -qy.lo});   // 1 - q y
  return df_fast(q, res.hi * q);
}

// Arithmetic of the Cholesky factorisation: FP64 for FP64 panels,
// double-float for FP32 ones.  Both elements are 8 bytes.
struct ArF64 {
  typedef double T;
  static __device__ __forceinline__ T from(double d) { return d; }
  static __device__ __forceinline__ double lead(T x) { return x; }
  static __device__ __forceinline__ T one() { return 1.0; }
  static __device__ __forceinline__ T root(T x) { return sqrt(x); }
  static __device__ __forceinline__ T rcp(T x) { return 1.0 / x; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  // c - a b s
  static __device__ __forceinline__ T update(T c, T a, T b, T s) {
    return fma(-s, a * b, c);
  }
};
struct ArDF {
  typedef DF T;
  static __device__ __forceinline__ T from(double d) {
    const float h = (float)d;
    return DF{h, (float)(d - (double)h)};
  }
  static __device__ __forceinline__ double lead(T x) { return (double)x.hi; }
  static __device__ __forceinline__ T one() { return DF{1.0f, 0.0f}; }
  static __device__ __forceinline__ T root(T x) { return df_sqrt(x); }
  static __device__ __forceinline__ T rcp(T x) { return df_rcp(x); }
  static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
  static __device__ __forceinline__ T update(T c, T a, T b, T s) {
    const DF t = df_mul(df_mul(a, b), s);
    return df_add(c, DF{-t.hi, -t.lo});
  }
};
template <typename W>
struct ArOf;
template <>
struct ArOf<double> { typedef ArF64 type; };
template <>
struct ArOf<float> { typedef ArDF type; };

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
  pdl_wait();   // the Gram partials
  __shared__ double red[FIN_E][FIN_S + 1];
  const int p = blockIdx.y;
  const int le = threadIdx.x / FIN_S, sub = threadIdx.x % FIN_S;
  const int e = blockIdx.x * FIN_E + le;
  const int a = e / KP, b = e % KP;
  W* out = p ? out1 : out0;
  const bool want = e < KP * KP && (mode == 0 || a <= b) && a < k && b < k;
  double s = 0.0;
  if (want) {
    // this thread's partials (CTAs sub, sub + FIN_S, ...) all in flight at
    // once, then added in CTA order
    const double* src = part + (size_t)p * G * KP * KP + e;
    for (int64_t c0 = sub; c0 < G; c0 += 24 * FIN_S) {
      double v[24];
#pragma unroll
      for (int j = 0; j < 24; ++j) {
        const int64_t c = c0 + (int64_t)j * FIN_S;
        v[j] = c < G ? __ldcg(src + (size_t)c * KP * KP) : 0.0;
      }
#pragma unroll
      for (int j = 0; j < 24; ++j) s += v[j];
    }
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

  typedef typename ArOf<W>::type Ar;
  typedef typename Ar::T T;
  static_assert(sizeof(T) == 8, "8-byte factor entries");
  extern __shared__ __align__(16) unsigned char smem[];
  T* R = reinterpret_cast<T*>(smem);                       // KP x KP
  __shared__ double trace_s;
  __shared__ int bad_s;
  // the other CTAs' sums: L2 reads (after the ticket's fence), all issued
  // at once; the Gram's upper triangle is staged in the factor's slots
  const double* gp = gfull + (size_t)p * KP * KP;
  double* Gs = reinterpret_cast<double*>(R);   // same 8-byte slots
  for (int i = threadIdx.x; i < KP * KP; i += OR_NT) {
    const int ia = i / KP, ib = i % KP;
    Gs[i] = (ia <= ib && ia < k && ib < k) ? __ldcg(gp + i) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int j = 0; j < k; ++j) tr += Gs[j * KP + j];
    trace_s = tr;
    bad_s = isfinite(tr) ? 0 : CNMF_E_NONFINITE;
    if (bad_s) set_status(status, bad_s);
  }
  __syncthreads();
  const double shift = shift_rel * trace_s + shift_abs;
  for (int i = threadIdx.x; i < KP * KP; i += OR_NT) {
    const int ia = i / KP, ib = i % KP;
    const double g = Gs[i] + ((ia == ib && ia < k) ? shift : 0.0);
    R[i] = Ar::from(g);
  }
  __syncthreads();
  // Right-looking Cholesky, upper factor in place, one barrier per pivot,
  // with the pivot's reciprocal off the other threads' path: in the phase
  // of pivot j, warps 0 and 1 both form the update of the diagonal entry
  // j + 1 (the same arithmetic, so the same value); warp 0 then forms
  // 1/R_{j+1,j+1}^2, which the next phase's trailing update needs, and
  // warp 1 the root and its reciprocal, which only the scaling of row j + 1
  // (one phase later still) needs.  The other warps update the rest of the
  // trailing triangle with the unscaled row j times 1/R_jj^2; everyone
  // scales row j - 1, which nobody reads in this phase.
  __shared__ T piv_s[3][3];   // {root, 1/root, 1/root^2}, pivot j in j % 3
  auto bad_pivot = [&](T d) {
    const double dl = Ar::lead(d);
    if (!(dl > 0.0) || !isfinite(dl)) {
      if (threadIdx.x == 0)
        set_status(status, isfinite(dl) ? CNMF_E_CHOLESKY : CNMF_E_NONFINITE);
      return true;
    }
    return false;
  };
  // warp 0 forms 1/d (lane 0 stores it), warp 1 the root and its
  // reciprocal; whole warps, so no lane of them waits on a diverged path
  const int warp = threadIdx.x >> 5;
  auto pivot_parts = [&](int j, T d) {
    if (bad_pivot(d)) d = Ar::one();
    if (warp == 0) {
      const T iv2 = Ar::rcp(d);
      if (threadIdx.x == 0) piv_s[j % 3][2] = iv2;
    } else {
      const T rt = Ar::root(d);
      const T iv = Ar::rcp(rt);
      if (threadIdx.x == 32) {
        piv_s[j % 3][0] = rt;
        piv_s[j % 3][1] = iv;
      }
    }
  };
  if (warp < 2 && k > 0) pivot_parts(0, R[0]);
  __syncthreads();
  // phase j reads slots (j - 1) % 3 and j % 3 and writes (j + 1) % 3
  for (int j = 0; j <= k; ++j) {
    if (j > 0) {   // scale row j - 1
      const int jp = j - 1;
      const T iv = piv_s[jp % 3][1];
      for (int l = jp + 1 + threadIdx.x; l < k; l += OR_NT)
        R[jp * KP + l] = Ar::mul(R[jp * KP + l], iv);
      if (threadIdx.x == 0) R[jp * KP + jp] = piv_s[jp % 3][0];
    }
    if (j == k) break;
    const T iv2 = piv_s[j % 3][2];
    const int nt = k - j - 1;
    if (warp < 2) {
      if (nt > 0) {
        // (not stored: the updated entry is only ever the next pivot, and
        // its slot receives the root when row j + 1 is scaled)
        const T dn = Ar::update(R[(j + 1) * KP + j + 1], R[j * KP + j + 1],
                                R[j * KP + j + 1], iv2);
        pivot_parts(j + 1, dn);
      }
    } else {
      // entries t = 1 .. nt^2 - 1 of the trailing square (t = 0 is the
      // diagonal entry above) over warps 2 and up
      for (int t = 1 + threadIdx.x - 64; t < nt * nt; t += OR_NT - 64) {
        const int ia = j + 1 + t / nt, ib = j + 1 + t % nt;
        if (ia <= ib)
          R[ia * KP + ib] =
              Ar::update(R[ia * KP + ib], R[j * KP + ia], R[j * KP + ib], iv2);
      }
    }
    __syncthreads();
  }
  __syncthreads();
  // R^-1 in the working precision, in place in `Ri` (upper, k x k), column
  // by column: column j needs the inverted leading block and a copy of the
  // old column j.  GI threads per row share each dot product and add their
  // parts by shuffles in a fixed order; the copy of column j + 1 is taken in
  // the same phase (double buffer); diagonal reciprocals are formed first,
  // all at once.
  constexpr int GI = OR_NT / KP >= 16 ? 16 : OR_NT / KP >= 8 ? 8
                     : OR_NT / KP >= 4 ? 4 : 2;
  static_assert(GI * KP <= OR_NT, "one row group per KP row");
  // FP64 panels invert in place in R; FP32 ones in a copy after it
  W* tail = reinterpret_cast<W*>(R + KP * KP);
  W* Ri = sizeof(W) == 8 ? reinterpret_cast<W*>(R) : tail;   // KP x KP
  W* colv = sizeof(W) == 8 ? tail : tail + KP * KP;          // 2 x KP
  W* dinv = colv + 2 * KP;                                   // KP
  for (int i = threadIdx.x; i < KP * KP; i += OR_NT) {
    const int ia = i / KP, ib = i % KP;
    Ri[i] = (ia <= ib && ib < k) ? (W)Ar::lead(R[i]) : W(0);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += OR_NT) dinv[j] = W(1) / Ri[j * KP + j];
  if (threadIdx.x == 0) colv[0] = Ri[0];
  __syncthreads();
  const int irow = threadIdx.x / GI, ig = threadIdx.x % GI;
  for (int j = 0; j < k; ++j) {
    const W* cj = colv + (j & 1) * KP;
    W* cn = colv + ((j + 1) & 1) * KP;
    W x = W(0);
    if (irow < j)
      for (int l = irow + ig; l < j; l += GI) x = fma(Ri[irow * KP + l], cj[l], x);
#pragma unroll
    for (int o = GI / 2; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o, GI);
    if (j + 1 < k)
      for (int l = threadIdx.x; l <= j + 1; l += OR_NT) cn[l] = Ri[l * KP + j + 1];
    if (ig == 0 && irow < j) Ri[irow * KP + j] = -dinv[j] * x;
    if (threadIdx.x == 0) Ri[j * KP + j] = dinv[j];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < KP * KP; i += OR_NT) out[i] = Ri[i];
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
  pdl_wait();   // R^-1 from k_finish, the panel
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
  RowTile<W, KP> ty;
  if (r0 < r1) ty.load((const W*)P.Y, P.ldy, r0, (int)std::min<int64_t>(OR_ROWS, r1 - r0), k);
  for (int64_t rb = r0; rb < r1; rb += OR_ROWS) {
    int nr = (int)std::min<int64_t>(OR_ROWS, r1 - rb);
    ty.store(Ys);
    __syncthreads();
    const int64_t rn = rb + OR_ROWS;
    if (rn < r1)
      ty.load((const W*)P.Y, P.ldy, rn, (int)std::min<int64_t>(OR_ROWS, r1 - rn), k);
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
  if (GRAM) gs.store(part + ((size_t)p * G + c) * KP * KP,
                     reinterpret_cast<double*>(smem));
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
static size_t finish_smem() {
  return sizeof(double) * KP * KP +
         sizeof(W) * ((sizeof(W) == 8 ? 0 : KP * KP) + 3 * KP);
}
template <typename W, int KP, bool SYM>
static size_t gram_smem() {
  const size_t stage = sizeof(W) * (SYM ? 1 : 2) * OR_ROWS * (KP + 4);
  return std::max(stage, sizeof(double) * GramMap<KP, SYM>::RED);
}
template <typename W, int KP>
static size_t apply_smem() {
  const size_t stage = sizeof(W) * (KP * KP + 2 * OR_ROWS * (KP + 4));
  return std::max(stage, sizeof(double) * GramMap<KP, true>::RED);
}

// The attribute belongs to the current device's context: raised once per
// (kernel, device).
template <typename W, int KP>
static void set_smem_attrs() {
  ensure_max_smem((const void*)k_finish<W, KP>, finish_smem<W, KP>());
  const size_t ap = apply_smem<W, KP>();
  ensure_max_smem((const void*)k_gram<W, KP, false>, gram_smem<W, KP, false>());
  ensure_max_smem((const void*)k_gram<W, KP, true>, gram_smem<W, KP, true>());
  ensure_max_smem((const void*)k_apply<W, KP, true>, ap);
  ensure_max_smem((const void*)k_apply<W, KP, false>, ap);
}

template <typename W, int KP>
static cnmf_status run_orth(const OrthPanel* pp, int np, int k, void* ws,
                            int32_t* status, cudaStream_t s, int sweeps) {
  set_smem_attrs<W, KP>();
  int64_t maxr = 0;
  for (int i = 0; i < np; ++i) maxr = std::max(maxr, pp[i].rows);
  const int G = gram_grid<W>(maxr);
  Carve cv(ws, SIZE_MAX);
  double* part = cv.take<double>((size_t)2 * G * KP * KP);
  double* gfull = cv.take<double>((size_t)2 * KP * KP);
  W* rinv = cv.take<W>((size_t)2 * KP * KP);
  unsigned* tickets = cv.take<unsigned>(64);   // zeroed by k_gram
  PanelDesc d[2];
  for (int i = 0; i < 2; ++i) {
    const OrthPanel& o = pp[std::min(i, np - 1)];
    d[i] = PanelDesc{o.Y, o.Y, o.ld, o.ld, o.rows};
  }
  dim3 grid(G, np);
  const int nfin = (int)ceil_div((int64_t)KP * KP, FIN_E);
  const size_t fin_smem = finish_smem<W, KP>();
  const size_t ap_smem = apply_smem<W, KP>();
  const double shift = sizeof(W) == 8 ? 1e-13 : 1e-11;

  launch_pdl(k_gram<W, KP, true>, grid, dim3(OR_NT), gram_smem<W, KP, true>(),
             s, d[0], d[1], k, part, tickets);
  CNMF_CHECK_LAUNCH();
  launch_pdl(k_finish<W, KP>, dim3(nfin, np), dim3(OR_NT), fin_smem, s, part,
             (int64_t)G, k, 1, shift, 0.0, gfull, rinv, rinv + KP * KP,
             (int64_t)0, tickets, status);
  CNMF_CHECK_LAUNCH();
  W* q0 = (W*)pp[0].Q;
  W* q1 = (W*)pp[std::min(1, np - 1)].Q;
  if (sweeps == 1) {
    launch_pdl(k_apply<W, KP, false>, grid, dim3(OR_NT), ap_smem, s, d[0],
               d[1], q0, q1, pp[0].ldo, pp[std::min(1, np - 1)].ldo, k,
               (const W*)rinv, part);
    CNMF_CHECK_LAUNCH();
    return CNMF_OK;
  }
  launch_pdl(k_apply<W, KP, true>, grid, dim3(OR_NT), ap_smem, s, d[0], d[1],
             (W*)d[0].Y, (W*)d[1].Y, d[0].ldy, d[1].ldy, k, (const W*)rinv,
             part);
  CNMF_CHECK_LAUNCH();
  launch_pdl(k_finish<W, KP>, dim3(nfin, np), dim3(OR_NT), fin_smem, s, part,
             (int64_t)G, k, 1, 0.0, 0.0, gfull, rinv, rinv + KP * KP,
             (int64_t)0, tickets, status);
  CNMF_CHECK_LAUNCH();
  launch_pdl(k_apply<W, KP, false>, grid, dim3(OR_NT), ap_smem, s, d[0], d[1],
             q0, q1, pp[0].ldo, pp[std::min(1, np - 1)].ldo, k, (const W*)rinv,
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
  launch_pdl(k_gram<W, KP, false>, dim3(G, 1), dim3(OR_NT),
             gram_smem<W, KP, false>(), s, d, d, k, part,
             (unsigned*)nullptr);
  CNMF_CHECK_LAUNCH();
  const int nfin = (int)ceil_div((int64_t)KP * KP, FIN_E);
  launch_pdl(k_finish<W, KP>, dim3(nfin, 1), dim3(OR_NT), 0, s, part,
             (int64_t)G, k, 0, 0.0, 0.0, (double*)nullptr, (W*)C, (W*)C, ldc,
             (unsigned*)nullptr, (int32_t*)nullptr);
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
  unsigned* tickets = cv.take<unsigned>(64);   // zeroed by k_gram
  PanelDesc d{Y, Y, ld, ld, rows};
  launch_pdl(k_gram<W, KP, true>, dim3(G, 1), dim3(OR_NT),
             gram_smem<W, KP, true>(), s, d, d, k, part, tickets);
  CNMF_CHECK_LAUNCH();
  const int nfin = (int)ceil_div((int64_t)KP * KP, FIN_E);
  const size_t fin_smem = finish_smem<W, KP>();
  launch_pdl(k_finish<W, KP>, dim3(nfin, 1), dim3(OR_NT), fin_smem, s, part,
             (int64_t)G, k, 1, 0.0, shift_abs, gfull, (W*)rinv_out,
             (W*)rinv_out, (int64_t)0, tickets, status);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

template <typename W>
static cnmf_status orth_dispatch(const OrthPanel* p, int np, int k, void* ws,
                                 int32_t* st, cudaStream_t s, int sw) {
  switch (orth_kp(k)) {
    case 16: return run_orth<W, 16>(p, np, k, ws, st, s, sw);
    case 32: return run_orth<W, 32>(p, np, k, ws, st, s, sw);
    case 48: return run_orth<W, 48>(p, np, k, ws, st, s, sw);
    case 64: return run_orth<W, 64>(p, np, k, ws, st, s, sw);
    case 80: return run_orth<W, 80>(p, np, k, ws, st, s, sw);
    case 96: return run_orth<W, 96>(p, np, k, ws, st, s, sw);
    default: return run_orth<W, 128>(p, np, k, ws, st, s, sw);
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
                        cudaStream_t s, int sweeps) {
  int64_t maxr = 0;
  for (int i = 0; i < np; ++i) maxr = std::max(maxr, p[i].rows);
  if (ws_bytes < orth_workspace(maxr, k, w)) return CNMF_E_WORKSPACE;
  if (sweeps != 1 && sweeps != 2) return CNMF_E_INVALID_ARG;
  return w == CNMF_F64 ? orth_dispatch<double>(p, np, k, ws, st, s, sweeps)
                       : orth_dispatch<float>(p, np, k, ws, st, s, sweeps);
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


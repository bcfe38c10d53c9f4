// Compressed ADMM NMF (Alg. 4, App. B) as one persistent cooperative kernel.
//
// Per sweep, every CTA first redoes the small r x r / d x r algebra in
// shared memory (the same inputs, the same arithmetic, so every CTA holds
// bitwise the same Xt, Yt):
//   Xt <- (Atilde Yt^T + SX)(Yt Yt^T + lam I)^-1,  SX = L^T (lam U - Lam)
//   Yt <- (Xt^T Xt + phi I)^-1 (Xt^T Atilde + SY), SY = (phi V - Phi) R^T
// then sweeps its own rows of the tall state:
//   U-rows:  T = L Xt; U <- P+(T + Lam/lam); Lam <- Lam + xi lam (T - U)
//   V-rows:  S = (Yt R)^T = Rt Yt^T; V^T <- P+(S + Phi^T/phi);
//            Phi^T <- Phi^T + xi phi (S - V^T)
// (U and V use the old multipliers, as printed) and accumulates its share
// of the NEXT sweep's SX = L^T (lam U - Lam) and SY = (phi V - Phi) R^T from
// the rows it just wrote.  The shares are summed over CTAs in CTA order
// (CTA c sums slice c of the entries): the generic kernel here with two
// bounded grid barriers per sweep, the register-tiled kernel (admm_fast.cuh)
// through tagged words without grid barriers.  The small algebra runs in
// the working precision: the r x r systems are SPD and well scaled by
// lam, phi > 0.
#include <algorithm>
#include <mutex>

#pragma once
#include <cooperative_groups.h>
#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

constexpr int AD_NT = 256;
constexpr int AD_BR = 64;  // rows per staged block

template <typename W>
__device__ __forceinline__ W fma_rn(W a, W b, W c);
template <>
__device__ __forceinline__ float fma_rn<float>(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}
template <>
__device__ __forceinline__ double fma_rn<double>(double a, double b, double c) {
  return __fma_rn(a, b, c);
}

template <typename W>
struct AdmmArgs {
  const W* L;
  const W* Rt;
  const W* At;
  W* U;
  W* Vt;
  W* Lam;
  W* Phit;
  W* Yt;      // state r x d
  W* Xt;      // state d x r
  int64_t* kcount;
  W* Zs;      // state: kept inverses, 2 x r x r
  W* SX;      // d x r (reduced)
  W* SY;      // r x d (reduced)
  W* part;    // G x (2 d r + r d)
  unsigned* bar;
  int32_t* status;
  int64_t m, n;
  int r, d;
  W lam, phi, xi;
  int iters;
  int resume;
  uint64_t timeout_ns;
  double* phase_ns;   // optional: CTA 0's time per phase, summed over sweeps
  int phase_ns_len;
  int64_t mu, nv;     // max rows per CTA on the U side / V side
  // Side split of the fast kernel (0: every CTA sweeps rows of both
  // sides): CTAs [0, Gu) own U rows, [Gu, G) own V rows.  U-side CTAs
  // stop the small algebra after the X update and read Yt^T, which the
  // first V-side CTA publishes in Ypub (two buffers, by sweep parity).
  int Gu;
  W* Ypub;
  // Sweep loop of the fast kernel: tagged words (payload + sweep tag, see
  // tag_put) in place of grid barriers: per-CTA shares (2 x G x 2 d r
  // values, by sweep parity), the reduced SX, SY^T (3 x 2 d r, by sweep
  // mod 3) and the published Yt^T (2 x d RP, by parity).
  uint64_t* tpart;
  uint64_t* tsxy;
  uint64_t* typ;
};

struct AdmmSmem {
  // element offsets into the dynamic shared buffer
  int At, Yt, Xt, MY, G, V, SXp, SYp, Blk, Wb, total;
  __host__ __device__ AdmmSmem(int r, int d) {
    int o = 0;
    auto take = [&](int64_t n) { int p = o; o += (int)((n + 3) & ~3); return p; };
    At = take(d * d);
    Yt = take(r * d);
    Xt = take(d * r);
    MY = take(r * d > d * r ? r * d : d * r);
    G = take(r * r);
    V = take(r);
    SXp = take(d * r);
    SYp = take(r * d);
    Blk = take(AD_BR * d);
    Wb = take(AD_BR * r);
    total = o;
  }
};

// In-place inverse of an r x r SPD matrix in shared memory with the sweep
// operator (Beaton 1964): pivoting on j in turn, with v = column j,
//   G[i][k] -= v_i v_k / d  (i, k != j),  G[i][j] = G[j][i] = v_i / d,
//   G[j][j] = -1 / d,   d = v_j;
// after all r pivots G holds -G^-1.  In this order it is Gaussian
// elimination without pivoting, which is stable for SPD matrices.  Two
// block barriers per pivot; `v` is r scratch elements.
template <typename W>
__device__ void spd_sweep_inverse(W* G, W* v, int r, int32_t* status) {
  for (int j = 0; j < r; ++j) {
    for (int i = threadIdx.x; i < r; i += AD_NT) v[i] = G[i * r + j];
    __syncthreads();
    W d = v[j];
    if (!(d > W(0))) {
      if (threadIdx.x == 0)
        set_status(status, isfinite((double)d) ? CNMF_E_CHOLESKY
                                               : CNMF_E_NONFINITE);
      d = W(1);
    }
    const W id = W(1) / d;
    for (int e = threadIdx.x; e < r * r; e += AD_NT) {
      const int i = e / r, k = e % r;
      W g;
      if (i == j && k == j) g = -id;
      else if (i == j) g = v[k] * id;
      else if (k == j) g = v[i] * id;
      else g = G[e] - v[i] * v[k] * id;
      G[e] = g;
    }
    __syncthreads();
  }
}

// One sweep's small algebra (all threads of the CTA).
template <typename W>
__device__ void small_phase(const AdmmArgs<W>& a, W* sm, const AdmmSmem& o) {
  const int r = a.r, d = a.d;
  W* At = sm + o.At;
  W* Yt = sm + o.Yt;
  W* Xt = sm + o.Xt;
  W* MY = sm + o.MY;
  W* G = sm + o.G;
  W* v = sm + o.V;
  // MX (d x r) = Atilde Yt^T + SX -> MY buffer (as d x r);  G = Yt Yt^T + lam I
  for (int e = threadIdx.x; e < d * r; e += AD_NT) {
    int i = e / r, b = e % r;
    W s = __ldcg(a.SX + e);
    for (int c = 0; c < d; ++c) s = fma(At[i * d + c], Yt[b * d + c], s);
    MY[e] = s;
  }
  for (int e = threadIdx.x; e < r * r; e += AD_NT) {
    int b = e / r, b2 = e % r;
    W s = (b == b2) ? a.lam : W(0);
    for (int c = 0; c < d; ++c) s = fma(Yt[b * d + c], Yt[b2 * d + c], s);
    G[e] = s;
  }
  __syncthreads();
  spd_sweep_inverse(G, v, r, a.status);      // G = -(Yt Yt^T + lam I)^-1
  // Xt = MX (Yt Yt^T + lam I)^-1
  for (int e = threadIdx.x; e < d * r; e += AD_NT) {
    int i = e / r, b = e % r;
    W s = W(0);
    for (int c = 0; c < r; ++c) s = fma(MY[i * r + c], G[c * r + b], s);
    Xt[e] = -s;
  }
  __syncthreads();
  // MY (r x d) = Xt^T Atilde + SY;  G = Xt^T Xt + phi I
  for (int e = threadIdx.x; e < r * d; e += AD_NT) {
    int b = e / d, c = e % d;
    W s = __ldcg(a.SY + e);
    for (int i = 0; i < d; ++i) s = fma(Xt[i * r + b], At[i * d + c], s);
    MY[e] = s;
  }
  for (int e = threadIdx.x; e < r * r; e += AD_NT) {
    int b = e / r, b2 = e % r;
    W s = (b == b2) ? a.phi : W(0);
    for (int i = 0; i < d; ++i) s = fma(Xt[i * r + b], Xt[i * r + b2], s);
    G[e] = s;
  }
  __syncthreads();
  spd_sweep_inverse(G, v, r, a.status);      // G = -(Xt^T Xt + phi I)^-1
  // Yt = (Xt^T Xt + phi I)^-1 MY
  for (int e = threadIdx.x; e < r * d; e += AD_NT) {
    int b = e / d, c = e % d;
    W s = W(0);
    for (int k = 0; k < r; ++k) s = fma(G[b * r + k], MY[k * d + c], s);
    s = -s;
    if (!isfinite((double)s)) set_status(a.status, CNMF_E_NONFINITE);
    Yt[e] = s;
  }
  __syncthreads();
}

// mode 0: setup (fresh): Lam = Phi = 0, accumulate SX from lam U, SY from
//         phi V, and Yt0 = V R^T (third block of partials).
// mode 1: setup (resume): accumulate SX, SY from the stored state.
// mode 2: ADMM sweep rows with the Xt, Yt in smem.
template <typename W>
__device__ void sweep_rows(const AdmmArgs<W>& a, W* sm, const AdmmSmem& o,
                           int mode) {
  const int r = a.r, d = a.d;
  const int64_t G = gridDim.x, c = blockIdx.x;
  W* SXp = sm + o.SXp;
  W* SYp = sm + o.SYp;
  W* Blk = sm + o.Blk;
  W* Wb = sm + o.Wb;
  const W* Xt = sm + o.Xt;
  const W* Yt = sm + o.Yt;
  W* Y0p = sm + o.MY;  // r x d accumulator for Yt0 (mode 0 only)
  for (int e = threadIdx.x; e < d * r; e += AD_NT) {
    SXp[e] = W(0);
    SYp[e] = W(0);
    if (mode == 0) Y0p[e] = W(0);
  }
  __syncthreads();
  // ---- U side: rows of L, U, Lam
  {
    const int64_t i0 = (c * a.m) / G, i1 = ((c + 1) * a.m) / G;
    for (int64_t ib = i0; ib < i1; ib += AD_BR) {
      const int nr = (int)(i1 - ib < AD_BR ? i1 - ib : AD_BR);
      for (int e = threadIdx.x; e < nr * d; e += AD_NT)
        Blk[e] = a.L[ib * d + e];
      __syncthreads();
      for (int e = threadIdx.x; e < nr * r; e += AD_NT) {
        const int64_t g = ib * r + e;
        W w;
        if (mode == 2) {
          const int i = e / r, b = e % r;
          W t = W(0);
          for (int k = 0; k < d; ++k) t = fma(Blk[i * d + k], Xt[k * r + b], t);
          const W lamo = a.Lam[g];
          W u = t + lamo / a.lam;
          u = u > W(0) ? u : W(0);
          const W lamn = lamo + a.xi * a.lam * (t - u);
          a.U[g] = u;
          a.Lam[g] = lamn;
          w = fma_rn<W>(a.lam, u, -lamn);
        } else if (mode == 0) {
          a.Lam[g] = W(0);
          w = fma_rn<W>(a.lam, a.U[g], -W(0));
        } else {
          w = fma_rn<W>(a.lam, a.U[g], -a.Lam[g]);
        }
        Wb[e] = w;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < d * r; e += AD_NT) {
        const int k = e / r, b = e % r;
        W s = SXp[e];
        for (int i = 0; i < nr; ++i) s = fma(Blk[i * d + k], Wb[i * r + b], s);
        SXp[e] = s;
      }
      __syncthreads();
    }
  }
  // ---- V side: rows of Rt, Vt, Phit
  {
    const int64_t j0 = (c * a.n) / G, j1 = ((c + 1) * a.n) / G;
    for (int64_t jb = j0; jb < j1; jb += AD_BR) {
      const int nr = (int)(j1 - jb < AD_BR ? j1 - jb : AD_BR);
      for (int e = threadIdx.x; e < nr * d; e += AD_NT)
        Blk[e] = a.Rt[jb * d + e];
      __syncthreads();
      for (int e = threadIdx.x; e < nr * r; e += AD_NT) {
        const int64_t g = jb * r + e;
        W w;
        if (mode == 2) {
          const int j = e / r, b = e % r;
          W s = W(0);
          for (int k = 0; k < d; ++k) s = fma(Blk[j * d + k], Yt[b * d + k], s);
          const W phio = a.Phit[g];
          W v = s + phio / a.phi;
          v = v > W(0) ? v : W(0);
          const W phin = phio + a.xi * a.phi * (s - v);
          a.Vt[g] = v;
          a.Phit[g] = phin;
          w = fma_rn<W>(a.phi, v, -phin);
        } else if (mode == 0) {
          a.Phit[g] = W(0);
          w = fma_rn<W>(a.phi, a.Vt[g], -W(0));
        } else {
          w = fma_rn<W>(a.phi, a.Vt[g], -a.Phit[g]);
        }
        Wb[e] = w;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < r * d; e += AD_NT) {
        const int b = e / d, k = e % d;
        W s = SYp[e];
        for (int j = 0; j < nr; ++j) s = fma(Wb[j * r + b], Blk[j * d + k], s);
        SYp[e] = s;
        if (mode == 0) {
          W y = Y0p[e];
          for (int j = 0; j < nr; ++j)
            y = fma(a.Vt[(jb + j) * r + b], Blk[j * d + k], y);
          Y0p[e] = y;
        }
      }
      __syncthreads();
    }
  }
  // ---- publish this CTA's shares
  const int E = 2 * d * r + (mode == 0 ? r * d : 0);
  W* dst = a.part + (size_t)c * (3 * d * r);
  for (int e = threadIdx.x; e < E; e += AD_NT) {
    W v;
    if (e < d * r) v = SXp[e];
    else if (e < 2 * d * r) v = SYp[e - d * r];
    else v = Y0p[e - 2 * d * r];
    dst[e] = v;
  }
}


// Sum slice `blockIdx.x` of the shares over CTAs.  One warp per entry:
// lane l adds the partials of CTAs l, l+32, ... in order, then a fixed
// xor-shuffle tree combines the lanes, so the result is deterministic.
template <typename W>
__device__ void reduce_shares(const AdmmArgs<W>& a, int with_y0) {
  const int dr = a.d * a.r;
  const int E = 2 * dr + (with_y0 ? dr : 0);
  const int64_t G = gridDim.x, c = blockIdx.x;
  const int e0 = (int)((c * E) / G), e1 = (int)(((c + 1) * E) / G);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int e = e0 + warp; e < e1; e += AD_NT / 32) {
    W s = W(0);
    const W* p = a.part + e;
#pragma unroll 4
    for (int64_t g = lane; g < G; g += 32) s += __ldcg(p + (size_t)g * 3 * dr);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (e < dr) a.SX[e] = s;
      else if (e < 2 * dr) a.SY[e - dr] = s;
      else a.Yt[e - 2 * dr] = s;
    }
  }
}

// Generic path (any d <= 128, r <= 64): block-parallel small algebra and
// row sweeps streamed through shared memory in blocks of AD_BR rows.
template <typename W>
__global__ void __launch_bounds__(AD_NT) k_admm(AdmmArgs<W> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sm = reinterpret_cast<W*>(smem_raw);
  const AdmmSmem o(a.r, a.d);
  const int r = a.r, d = a.d;
  const bool prof = a.phase_ns && blockIdx.x == 0 && threadIdx.x == 0;
  uint64_t tph[5] = {0, 0, 0, 0, 0};
  for (int e = threadIdx.x; e < d * d; e += AD_NT) sm[o.At + e] = a.At[e];
  __syncthreads();
  sweep_rows<W>(a, sm, o, a.resume ? 1 : 0);
  if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;
  reduce_shares<W>(a, a.resume ? 0 : 1);
  if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;
  for (int e = threadIdx.x; e < r * d; e += AD_NT) sm[o.Yt + e] = __ldcg(a.Yt + e);
  __syncthreads();
  for (int it = 0; it < a.iters; ++it) {
    uint64_t t0 = prof ? globaltimer_ns() : 0;
    small_phase<W>(a, sm, o);
    uint64_t t1 = prof ? globaltimer_ns() : 0;
    sweep_rows<W>(a, sm, o, 2);
    uint64_t t2 = prof ? globaltimer_ns() : 0;
    if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;
    uint64_t t3 = prof ? globaltimer_ns() : 0;
    reduce_shares<W>(a, 0);
    uint64_t t4 = prof ? globaltimer_ns() : 0;
    if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;
    if (prof) {
      uint64_t t5 = globaltimer_ns();
      tph[0] += t1 - t0; tph[1] += t2 - t1; tph[2] += t3 - t2;
      tph[3] += t4 - t3; tph[4] += t5 - t4;
    }
  }
  if (blockIdx.x == 0) {
    for (int e = threadIdx.x; e < r * d; e += AD_NT) {
      a.Yt[e] = sm[o.Yt + e];
      if (a.iters > 0) a.Xt[e] = sm[o.Xt + e];
    }
    if (threadIdx.x == 0) *a.kcount += a.iters;
  }
  if (prof)
    for (int i = 0; i < 5; ++i) a.phase_ns[i] += (double)tph[i];
}

#include "admm_fast.cuh"
#include "admm_batch.cuh"

// State: Lam, Phit, Yt, Xt (W), then int64 k at the next 8-byte boundary
// (state_core), then the two kept r x r inverses (W).
inline size_t state_core(int64_t m, int64_t n, int r, int d, size_t e) {
  const size_t b = ((size_t)m * r + (size_t)n * r + 2 * (size_t)r * d) * e;
  return (b + 7) & ~size_t(7);
}
inline size_t state_bytes(int64_t m, int64_t n, int r, int d, size_t e) {
  return state_core(m, n, r, d, e) + 8 +
         ((2 * (size_t)r * r * e + 7) & ~size_t(7));
}

// Tagged-word counts of the fast kernel's sweep loop (sizeof(W) / 4 words
// per value).
inline size_t tag_part_words(int r, int d, size_t e, int G) {
  return (size_t)2 * G * 2 * d * r * (e / 4);
}
inline size_t tag_sxy_words(int r, int d, size_t e) {
  return (size_t)3 * 2 * d * r * (e / 4);
}
inline size_t tag_y_words(int r, int d, size_t e) {
  return (size_t)2 * d * ((r + 3) & ~3) * (e / 4);
}

inline size_t factor_ws(int r, int d, size_t e, int G) {
  Carve cv(nullptr, SIZE_MAX);
  cv.take<char>((size_t)d * r * e);
  cv.take<char>((size_t)r * d * e);
  cv.take<char>((size_t)G * 3 * d * r * e);
  cv.take<unsigned>(64);
  cv.take<char>((size_t)2 * d * ((r + 3) & ~3) * e);   // Ypub
  cv.take<uint64_t>(tag_part_words(r, d, e, G));
  cv.take<uint64_t>(tag_sxy_words(r, d, e));
  cv.take<uint64_t>(tag_y_words(r, d, e));
  return cv.off;
}

struct AdmmPlan {
  int G, Gu;
  const void* fn;
  size_t smem;
  int64_t mu, nv;
};

// U/V split of the fast kernel's CTAs.  A U-side CTA stops the small
// algebra after the X update, so it starts its rows earlier than a V-side
// CTA by the second half of the chain; past a fixed start-up cost that both
// sides pay, rows cost about 2e-5 d r us each.  Gu balances m / Gu row costs
// against dt + n / (G - Gu) row costs.  dt = 2.3 us is the measured best on
// GB300 at m = 20000, n = 10000, d = 30, r = 20 (the Y half itself takes
// about 3.3 us, but the U side also waits for the lead's Yt; the time per
// sweep is flat within 1% for Gu from 54 to 73 there).
inline int split_gu(int64_t m, int64_t n, int r, int d, int G) {
  if (G < 2) return 0;
  const double c = 2e-5 * d * r, dt = 2.3;
  int best = 0;
  double bt = 1e300;
  for (int gu = 1; gu < G; ++gu) {
    const double tu = (double)((m + gu - 1) / gu) * c;
    const double tv = dt + (double)((n + (G - gu) - 1) / (G - gu)) * c;
    const double t = tu > tv ? tu : tv;
    if (t < bt) { bt = t; best = gu; }
  }
  return best;
}

// Opt-in shared memory left for a kernel's dynamic buffer (set once).
inline size_t admm_limit(const void* fn) {
  static std::mutex mu;
  static const void* fns[16];
  static size_t lim[16];
  static int nf = 0;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < nf; ++i)
    if (fns[i] == fn) return lim[i];
  size_t l = (size_t)max_smem_optin() - static_smem(fn);
  if (!set_max_smem(fn, l)) l = 48 * 1024;
  if (nf < 16) { fns[nf] = fn; lim[nf] = l; ++nf; }
  return l;
}

inline bool coop_ok(const void* fn, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, AD_NT,
                                                    smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return per_sm >= 1;
}

template <typename W, int DMAX, int RMAX, bool RES>
static bool plan_fast(AdmmPlan& P, int r, int d) {
  const void* fn = (const void*)k_admm_fast<W, DMAX, RMAX, RES>;
  FastSmem o(r, d, RES, P.mu, P.nv, DMAX, P.Gu > 0);
  const size_t smem = (size_t)o.total * sizeof(W);
  if (smem > admm_limit(fn) || !coop_ok(fn, smem)) return false;
  P.fn = fn;
  P.smem = smem;
  return true;
}

template <typename W>
static bool admm_plan(AdmmPlan& P, int64_t m, int64_t n, int r, int d) {
  P.G = (int)std::min<int64_t>(std::max<int64_t>(1, ceil_div(m + n, AD_BR)),
                               (int64_t)num_sms());
  P.Gu = split_gu(m, n, r, d, P.G);
  P.mu = P.Gu ? ceil_div(m, P.Gu) : ceil_div(m, P.G);
  P.nv = P.Gu ? ceil_div(n, P.G - P.Gu) : ceil_div(n, P.G);
  if (r <= 16 && d <= 32) {
    if (plan_fast<W, 32, 16, true>(P, r, d)) return true;
    if (plan_fast<W, 32, 16, false>(P, r, d)) return true;
  }
  if (r <= 32 && d <= 32) {
    if (plan_fast<W, 32, 32, true>(P, r, d)) return true;
    if (plan_fast<W, 32, 32, false>(P, r, d)) return true;
  }
  if (r <= 32 && d <= 64) {
    if (plan_fast<W, 64, 32, true>(P, r, d)) return true;
    if (plan_fast<W, 64, 32, false>(P, r, d)) return true;
  }
  const void* fn = (const void*)k_admm<W>;
  AdmmSmem o(r, d);
  P.Gu = 0;
  P.mu = ceil_div(m, P.G);
  P.nv = ceil_div(n, P.G);
  P.smem = (size_t)o.total * sizeof(W);
  P.fn = fn;
  return P.smem <= admm_limit(fn) && coop_ok(fn, P.smem);
}

template <typename W>
static cnmf_status run_factor(const void* L, const void* Rt, const void* At,
                              int64_t m, int64_t n, int r, int d,
                              const cnmf_admm_params* p, void* U, void* Vt,
                              void* state, int resume, void* ws,
                              size_t ws_bytes, int32_t* status,
                              cudaStream_t s) {
  AdmmPlan P;
  if (!admm_plan<W>(P, m, n, r, d)) return CNMF_E_INVALID_ARG;
  const int G = P.G;
  const size_t e = sizeof(W);
  if (ws_bytes < factor_ws(r, d, e, num_sms())) return CNMF_E_WORKSPACE;
  Carve cv(ws, ws_bytes);
  AdmmArgs<W> a;
  a.SX = cv.take<W>((size_t)d * r);
  a.SY = cv.take<W>((size_t)r * d);
  a.part = cv.take<W>((size_t)G * 3 * d * r);
  a.bar = cv.take<unsigned>(64);
  a.Ypub = (W*)cv.take<char>((size_t)2 * d * ((r + 3) & ~3) * e);
  a.tpart = cv.take<uint64_t>(tag_part_words(r, d, e, G));
  a.tsxy = cv.take<uint64_t>(tag_sxy_words(r, d, e));
  a.typ = cv.take<uint64_t>(tag_y_words(r, d, e));
  a.Gu = P.Gu;
  char* st = (char*)state;
  a.Lam = (W*)st;
  a.Phit = a.Lam + (size_t)m * r;
  a.Yt = a.Phit + (size_t)n * r;
  a.Xt = a.Yt + (size_t)r * d;
  a.kcount = (int64_t*)(st + state_core(m, n, r, d, e));
  a.Zs = (W*)(st + state_core(m, n, r, d, e) + 8);
  a.L = (const W*)L; a.Rt = (const W*)Rt; a.At = (const W*)At;
  a.U = (W*)U; a.Vt = (W*)Vt;
  a.status = status;
  a.m = m; a.n = n; a.r = r; a.d = d;
  a.lam = (W)p->lambda; a.phi = (W)p->phi; a.xi = (W)p->xi;
  a.iters = p->iters;
  a.resume = resume;
  a.timeout_ns = (uint64_t)(p->barrier_timeout_ms > 0 ? p->barrier_timeout_ms
                                                      : 2000) * 1000000ull;
  a.phase_ns = p->phase_ns;
  a.phase_ns_len = p->phase_ns_len;
  a.mu = P.mu;
  a.nv = P.nv;
  CNMF_CUDA(cudaMemsetAsync(a.bar, 0, 64 * sizeof(unsigned), s));
  if (!resume) CNMF_CUDA(cudaMemsetAsync(a.kcount, 0, 8, s));
  void* args[] = {&a};
  CNMF_CUDA(cudaLaunchCooperativeKernel(P.fn, dim3(G), dim3(AD_NT), args,
                                        P.smem, s));
  return CNMF_OK;
}

}  // namespace cnmf

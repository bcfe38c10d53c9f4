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
// (CTA c sums slice c of the entries), with two bounded grid barriers per
// sweep.  The small algebra runs in the working precision: the r x r
// systems are SPD and well scaled by lam, phi > 0.
#include <algorithm>
#include <mutex>

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
};

struct AdmmSmem {
  // element offsets into the dynamic shared buffer
  int At, Yt, Xt, MY, G, SXp, SYp, Blk, Wb, total;
  __host__ __device__ AdmmSmem(int r, int d) {
    int o = 0;
    auto take = [&](int n) { int p = o; o += (n + 3) & ~3; return p; };
    At = take(d * d);
    Yt = take(r * d);
    Xt = take(d * r);
    MY = take(r * d);
    G = take(r * r);
    SXp = take(d * r);
    SYp = take(r * d);
    Blk = take(AD_BR * d);
    Wb = take(AD_BR * r);
    total = o;
  }
};

// In-place Cholesky G = C C^T (lower C) of an r x r SPD matrix in smem.
template <typename W>
__device__ void chol_lower(W* G, int r, int32_t* status) {
  for (int j = 0; j < r; ++j) {
    if (threadIdx.x == 0) {
      W dj = G[j * r + j];
      if (!(dj > W(0))) {
        set_status(status, isfinite((double)dj) ? CNMF_E_CHOLESKY
                                                : CNMF_E_NONFINITE);
        dj = W(1);
      }
      G[j * r + j] = sqrt(dj);
    }
    __syncthreads();
    const W inv = W(1) / G[j * r + j];
    for (int i = j + 1 + threadIdx.x; i < r; i += AD_NT) G[i * r + j] *= inv;
    __syncthreads();
    const int nt = r - j - 1;
    for (int t = threadIdx.x; t < nt * nt; t += AD_NT) {
      int i = j + 1 + t / nt, k = j + 1 + t % nt;
      if (k <= i) G[i * r + k] -= G[i * r + j] * G[k * r + j];
    }
    __syncthreads();
  }
}

// Solve G x = b for `nrhs` right-hand sides given G = C C^T (lower C).
// Right-hand side t is B[t * sr + i * sc], i < r; solved in place.
template <typename W>
__device__ void chol_solve(const W* C, int r, W* B, int nrhs, int sr, int sc) {
  for (int t = threadIdx.x; t < nrhs; t += AD_NT) {
    W* b = B + t * sr;
    for (int i = 0; i < r; ++i) {
      W s = b[i * sc];
      for (int k = 0; k < i; ++k) s -= C[i * r + k] * b[k * sc];
      b[i * sc] = s / C[i * r + i];
    }
    for (int i = r - 1; i >= 0; --i) {
      W s = b[i * sc];
      for (int k = i + 1; k < r; ++k) s -= C[k * r + i] * b[k * sc];
      b[i * sc] = s / C[i * r + i];
    }
  }
  __syncthreads();
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
  // MX (d x r) = Atilde Yt^T + SX  -> Xt buffer;  G = Yt Yt^T + lam I
  for (int e = threadIdx.x; e < d * r; e += AD_NT) {
    int i = e / r, b = e % r;
    W s = __ldcg(a.SX + e);
    for (int c = 0; c < d; ++c) s = fma(At[i * d + c], Yt[b * d + c], s);
    Xt[e] = s;
  }
  for (int e = threadIdx.x; e < r * r; e += AD_NT) {
    int b = e / r, b2 = e % r;
    W s = (b == b2) ? a.lam : W(0);
    for (int c = 0; c < d; ++c) s = fma(Yt[b * d + c], Yt[b2 * d + c], s);
    G[e] = s;
  }
  __syncthreads();
  chol_lower(G, r, a.status);
  chol_solve(G, r, Xt, d, r, 1);      // rows of Xt: (Yt Yt^T + lam I) x = MX_i
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
  chol_lower(G, r, a.status);
  chol_solve(G, r, MY, d, 1, d);      // columns of MY
  for (int e = threadIdx.x; e < r * d; e += AD_NT) {
    W v = MY[e];
    if (!isfinite((double)v)) set_status(a.status, CNMF_E_NONFINITE);
    Yt[e] = v;
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

// Sum slice `blockIdx.x` of the shares over CTAs (in CTA order).
template <typename W>
__device__ void reduce_shares(const AdmmArgs<W>& a, int with_y0) {
  const int dr = a.d * a.r;
  const int E = 2 * dr + (with_y0 ? dr : 0);
  const int64_t G = gridDim.x, c = blockIdx.x;
  const int e0 = (int)((c * E) / G), e1 = (int)(((c + 1) * E) / G);
  for (int e = e0 + threadIdx.x; e < e1; e += AD_NT) {
    W s = W(0);
    for (int64_t g = 0; g < G; ++g) s += __ldcg(a.part + (size_t)g * 3 * dr + e);
    if (e < dr) a.SX[e] = s;
    else if (e < 2 * dr) a.SY[e - dr] = s;
    else a.Yt[e - 2 * dr] = s;
  }
}

template <typename W>
__global__ void __launch_bounds__(AD_NT) k_admm(AdmmArgs<W> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sm = reinterpret_cast<W*>(smem_raw);
  const AdmmSmem o(a.r, a.d);
  const int r = a.r, d = a.d;
  for (int e = threadIdx.x; e < d * d; e += AD_NT) sm[o.At + e] = a.At[e];
  __syncthreads();

  // setup: SX, SY (and Yt0 on a fresh start) from the stored U, V, Lam, Phi
  sweep_rows<W>(a, sm, o, a.resume ? 1 : 0);
  if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;
  reduce_shares<W>(a, a.resume ? 0 : 1);
  if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;

  for (int e = threadIdx.x; e < r * d; e += AD_NT) sm[o.Yt + e] = __ldcg(a.Yt + e);
  __syncthreads();
  for (int it = 0; it < a.iters; ++it) {
    small_phase<W>(a, sm, o);
    sweep_rows<W>(a, sm, o, 2);
    if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;
    reduce_shares<W>(a, 0);
    if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;
  }
  if (blockIdx.x == 0) {
    for (int e = threadIdx.x; e < r * d; e += AD_NT) {
      a.Yt[e] = sm[o.Yt + e];
      if (a.iters > 0) a.Xt[e] = sm[o.Xt + e];
    }
    if (threadIdx.x == 0) *a.kcount += a.iters;
  }
}

static size_t state_bytes(int64_t m, int64_t n, int r, int d, size_t e) {
  size_t b = ((size_t)m * r + (size_t)n * r + 2 * (size_t)r * d) * e;
  return ((b + 7) & ~size_t(7)) + 8;
}

static size_t factor_ws(int r, int d, size_t e, int G) {
  Carve cv(nullptr, SIZE_MAX);
  cv.take<char>((size_t)d * r * e);
  cv.take<char>((size_t)r * d * e);
  cv.take<char>((size_t)G * 3 * d * r * e);
  cv.take<unsigned>(64);
  return cv.off;
}

template <typename W>
static int admm_grid(int64_t m, int64_t n, int r, int d, size_t* smem) {
  AdmmSmem o(r, d);
  *smem = (size_t)o.total * sizeof(W);
  static std::once_flag once;
  static size_t limit = 0;
  std::call_once(once, [] {
    limit = (size_t)max_smem_optin() - static_smem((const void*)k_admm<W>);
    if (!set_max_smem((const void*)k_admm<W>, limit)) limit = 48 * 1024;
  });
  if (*smem > limit) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_admm<W>, AD_NT,
                                                    *smem) != cudaSuccess)
    (void)cudaGetLastError();
  if (per_sm < 1) return 0;
  int64_t want = std::max<int64_t>(1, ceil_div(m + n, 2 * AD_BR));
  return (int)std::min<int64_t>(want, (int64_t)num_sms());
}

template <typename W>
static cnmf_status run_factor(const void* L, const void* Rt, const void* At,
                              int64_t m, int64_t n, int r, int d,
                              const cnmf_admm_params* p, void* U, void* Vt,
                              void* state, int resume, void* ws,
                              size_t ws_bytes, int32_t* status,
                              cudaStream_t s) {
  size_t smem = 0;
  const int G = admm_grid<W>(m, n, r, d, &smem);
  if (G < 1) return CNMF_E_INVALID_ARG;
  const size_t e = sizeof(W);
  if (ws_bytes < factor_ws(r, d, e, num_sms())) return CNMF_E_WORKSPACE;
  Carve cv(ws, ws_bytes);
  AdmmArgs<W> a;
  a.SX = cv.take<W>((size_t)d * r);
  a.SY = cv.take<W>((size_t)r * d);
  a.part = cv.take<W>((size_t)G * 3 * d * r);
  a.bar = cv.take<unsigned>(64);
  char* st = (char*)state;
  a.Lam = (W*)st;
  a.Phit = a.Lam + (size_t)m * r;
  a.Yt = a.Phit + (size_t)n * r;
  a.Xt = a.Yt + (size_t)r * d;
  a.kcount = (int64_t*)(st + state_bytes(m, n, r, d, e) - 8);
  a.L = (const W*)L; a.Rt = (const W*)Rt; a.At = (const W*)At;
  a.U = (W*)U; a.Vt = (W*)Vt;
  a.status = status;
  a.m = m; a.n = n; a.r = r; a.d = d;
  a.lam = (W)p->lambda; a.phi = (W)p->phi; a.xi = (W)p->xi;
  a.iters = p->iters;
  a.resume = resume;
  a.timeout_ns = (uint64_t)(p->barrier_timeout_ms > 0 ? p->barrier_timeout_ms
                                                      : 2000) * 1000000ull;
  CNMF_CUDA(cudaMemsetAsync(a.bar, 0, 64 * sizeof(unsigned), s));
  if (!resume) CNMF_CUDA(cudaMemsetAsync(a.kcount, 0, 8, s));
  void* args[] = {&a};
  CNMF_CUDA(cudaLaunchCooperativeKernel((const void*)k_admm<W>, dim3(G),
                                        dim3(AD_NT), args, smem, s));
  return CNMF_OK;
}

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
    return run_factor<double>(L, Rt, Atilde, m, n, r, d, p, U, Vt, state,
                              resume, ws, ws_bytes, dev_status, s);
  return run_factor<float>(L, Rt, Atilde, m, n, r, d, p, U, Vt, state, resume,
                           ws, ws_bytes, dev_status, s);
}

// Products with A for the structured random compression (Alg. 1 power
// scheme, Sec. II; applied to A and A^T in Sec. III; Q^T A in Alg. 3).
//
//   Z = A B    (P = m output rows, reduction over S = n)   trans = false
//   Z = A^T B  (P = n output rows, reduction over S = m)   trans = true
//
// B is thin (k <= 128 columns, padded to KP).  CUDA-core FMA kernel:
// 128 x 32 tiles of A staged through shared memory with a 3-stage cp.async
// pipeline in A's natural row-major orientation (so both products read the
// same coalesced 16-byte chunks), 4 x KP/8 register micro-tiles, FP32 (or
// FP64) accumulation.  Work is split evenly over a grid of exactly
// (SMs x resident CTAs): CTA c takes the contiguous range of
// (output tile, reduction chunk) units [c U / G, (c+1) U / G).  A tile
// finished inside one CTA is written directly; split tiles are written as
// per-CTA partials and summed in CTA order by a fix-up kernel, so results
// are deterministic and no floating-point atomics are used.
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

constexpr int SK_BP = 128;
constexpr int SK_BS = 32;
constexpr int SK_NT = 256;
constexpr int SK_TM = 4;

template <typename TA, typename W, int KP, bool TRANS>
struct SkCfg {
  static constexpr int STAGES = sizeof(TA) == 8 ? 2 : 3;
  static constexpr int TN = KP / 8;
  static constexpr int A_ROWS = TRANS ? SK_BS : SK_BP;
  static constexpr int A_COLS = TRANS ? SK_BP : SK_BS;
  static constexpr int A_PITCH = A_COLS + 16 / (int)sizeof(TA);
  static constexpr int A_ELEMS = A_ROWS * A_PITCH;
  static constexpr int B_ELEMS = SK_BS * KP;
  static constexpr size_t A_BYTES = (size_t)A_ELEMS * sizeof(TA);
  static constexpr size_t STAGE_BYTES = A_BYTES + (size_t)B_ELEMS * sizeof(W);
  static constexpr size_t SMEM = STAGES * STAGE_BYTES;
};

__host__ __device__ __forceinline__ int64_t split_start(int64_t c, int64_t U,
                                                        int64_t G) {
  return (c * U) / G;
}
__host__ __device__ __forceinline__ int64_t split_owner(int64_t u, int64_t U,
                                                        int64_t G) {
  int64_t c = ((u + 1) * G + U - 1) / U - 1;
  return c < G - 1 ? c : G - 1;
}

template <typename TA, typename W, int KP, bool TRANS>
__device__ __forceinline__ void sk_load_tile(
    TA* As, W* Bs, const TA* __restrict__ A, int64_t m, int64_t n, int64_t lda,
    bool a_vec, const W* __restrict__ B, int64_t S, int64_t ldb, int kb,
    bool b_vec, int64_t p0, int64_t s0) {
  typedef SkCfg<TA, W, KP, TRANS> C;
  constexpr int EA = 16 / sizeof(TA);
  constexpr int CPR = C::A_COLS / EA;
  const int64_t grow = TRANS ? s0 : p0;
  const int64_t gcol = TRANS ? p0 : s0;
  for (int c = threadIdx.x; c < C::A_ROWS * CPR; c += SK_NT) {
    int row = c / CPR, cc = c % CPR;
    int64_t gi = grow + row, gj = gcol + (int64_t)cc * EA;
    TA* dst = As + row * C::A_PITCH + cc * EA;
    if (a_vec && gi < m && gj + EA <= n) {
      cp_async16(dst, A + gi * lda + gj);
    } else {
#pragma unroll
      for (int e = 0; e < EA; ++e)
        dst[e] = (gi < m && gj + e < n) ? A[gi * lda + gj + e] : TA(0.0f);
    }
  }
  constexpr int EB = 16 / sizeof(W);
  constexpr int CPRB = KP / EB;
  for (int c = threadIdx.x; c < SK_BS * CPRB; c += SK_NT) {
    int row = c / CPRB, cc = c % CPRB;
    int64_t gs = s0 + row;
    int col = cc * EB;
    W* dst = Bs + row * KP + col;
    if (b_vec && gs < S && col + EB <= kb) {
      cp_async16(dst, B + gs * ldb + col);
    } else {
#pragma unroll
      for (int e = 0; e < EB; ++e)
        dst[e] = (gs < S && col + e < kb) ? B[gs * ldb + col + e] : W(0);
    }
  }
}

template <typename TA, typename W, int KP, bool TRANS>
__global__ void __launch_bounds__(SK_NT)
    k_prod(const TA* __restrict__ A, int64_t m, int64_t n, int64_t lda,
           int a_vec, const W* __restrict__ B, int64_t ldb, int kb, int b_vec,
           W* __restrict__ Z, int64_t ldz, int kz, W* __restrict__ part,
           int64_t U, int64_t chunks) {
  typedef SkCfg<TA, W, KP, TRANS> C;
  constexpr int TN = C::TN;
  constexpr int ST = C::STAGES;
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t P = TRANS ? n : m;
  const int64_t S = TRANS ? m : n;
  const int tid = threadIdx.x;
  const int tc = tid % 8, tr = tid / 8;
  const int64_t G = gridDim.x;
  const int64_t c = blockIdx.x;
  const int64_t u0 = split_start(c, U, G), u1 = split_start(c + 1, U, G);

  auto As_of = [&](int st) {
    return reinterpret_cast<TA*>(smem + (size_t)st * C::STAGE_BYTES);
  };
  auto Bs_of = [&](int st) {
    return reinterpret_cast<W*>(smem + (size_t)st * C::STAGE_BYTES +
                                C::A_BYTES);
  };

  int64_t u = u0;
  bool first_tile = true;
  while (u < u1) {
    const int64_t tp = u / chunks;
    const int64_t ts0 = u % chunks;
    const int64_t ts1 = min(chunks, ts0 + (u1 - u));
    const int nst = (int)(ts1 - ts0);
    const int64_t p0 = tp * SK_BP;

    W acc[SK_TM][TN];
#pragma unroll
    for (int i = 0; i < SK_TM; ++i)
#pragma unroll
      for (int t = 0; t < TN; ++t) acc[i][t] = W(0);

#pragma unroll
    for (int st = 0; st < ST - 1; ++st) {
      if (st < nst)
        sk_load_tile<TA, W, KP, TRANS>(As_of(st), Bs_of(st), A, m, n, lda,
                                       a_vec, B, S, ldb, kb, b_vec, p0,
                                       (ts0 + st) * SK_BS);
      cp_async_commit();
    }
    for (int it = 0; it < nst; ++it) {
      cp_async_wait<ST - 2>();
      __syncthreads();
      {
        int nx = it + ST - 1;
        if (nx < nst)
          sk_load_tile<TA, W, KP, TRANS>(As_of(nx % ST), Bs_of(nx % ST), A, m,
                                         n, lda, a_vec, B, S, ldb, kb, b_vec,
                                         p0, (ts0 + nx) * SK_BS);
        cp_async_commit();
      }
      const TA* As = As_of(it % ST);
      const W* Bs = Bs_of(it % ST);
      if constexpr (!TRANS) {
#pragma unroll 2
        for (int s = 0; s < SK_BS; s += 4) {
          W a[SK_TM][4];
#pragma unroll
          for (int i = 0; i < SK_TM; ++i)
            lds4<W, TA>(As + (tr + 32 * i) * C::A_PITCH + s, a[i]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            W b[TN];
            ldsN<TN, W>(Bs + (s + q) * KP + tc * TN, b);
#pragma unroll
            for (int i = 0; i < SK_TM; ++i)
#pragma unroll
              for (int t = 0; t < TN; ++t) acc[i][t] = fma(a[i][q], b[t], acc[i][t]);
          }
        }
      } else {
#pragma unroll 4
        for (int s = 0; s < SK_BS; ++s) {
          W a[4];
          lds4<W, TA>(As + s * C::A_PITCH + 4 * tr, a);
          W b[TN];
          ldsN<TN, W>(Bs + s * KP + tc * TN, b);
#pragma unroll
          for (int i = 0; i < SK_TM; ++i)
#pragma unroll
            for (int t = 0; t < TN; ++t) acc[i][t] = fma(a[i], b[t], acc[i][t]);
        }
      }
    }
    cp_async_wait<0>();
    __syncthreads();

    const bool whole = (ts0 == 0 && ts1 == chunks);
    W* dst;
    int64_t ld;
    if (whole) {
      dst = Z + p0 * ldz;
      ld = ldz;
    } else {
      dst = part + ((size_t)c * 2 + (first_tile ? 0 : 1)) * SK_BP * KP;
      ld = KP;
    }
#pragma unroll
    for (int i = 0; i < SK_TM; ++i) {
      int lp = TRANS ? (4 * tr + i) : (tr + 32 * i);
      if (p0 + lp >= P) continue;
      W* row = dst + (int64_t)lp * ld + tc * TN;
#pragma unroll
      for (int t = 0; t < TN; ++t)
        if (!whole || tc * TN + t < kz) row[t] = acc[i][t];
    }
    first_tile = false;
    u = ts1 + tp * chunks;
  }
}

// Sum the per-CTA partials of split output tiles, in CTA order.  The
// contributing CTAs of the tile and their partial slots are worked out once
// per CTA (64-bit integer divisions) and kept in shared memory.
constexpr int FIX_MAX = 1024;

template <typename W, int KP>
__global__ void k_prod_fixup(W* __restrict__ Z, int64_t ldz, int kz, int64_t P,
                             const W* __restrict__ part, int64_t U,
                             int64_t chunks, int64_t G) {
  __shared__ int64_t off[FIX_MAX];
  __shared__ int nc_s;
  const int64_t tp = blockIdx.x;
  const int64_t ua = tp * chunks, ub = ua + chunks - 1;
  const int64_t ca = split_owner(ua, U, G), cb = split_owner(ub, U, G);
  if (ca == cb) return;  // whole tile written directly by one CTA
  const int nc = (int)(cb - ca + 1);
  for (int j = threadIdx.x; j < nc && j < FIX_MAX; j += blockDim.x) {
    const int64_t c = ca + j;
    const int slot = (split_start(c, U, G) / chunks == tp) ? 0 : 1;
    off[j] = ((int64_t)c * 2 + slot) * SK_BP * KP;
  }
  if (threadIdx.x == 0) nc_s = nc;
  __syncthreads();
  const int64_t p0 = tp * SK_BP;
  // blockIdx.y splits the tile's entries: one or a few per thread, so the
  // partial loads of all entries are in flight together
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < SK_BP * KP;
       e += blockDim.x * gridDim.y) {
    int lp = e / KP, col = e % KP;
    if (p0 + lp >= P || col >= kz) continue;
    W s = W(0);
    int j = 0;
    for (; j < nc_s && j < FIX_MAX; ++j) s += part[off[j] + e];
    for (; j < nc_s; ++j) {  // more contributors than the cache holds
      const int64_t c = ca + j;
      const int slot = (split_start(c, U, G) / chunks == tp) ? 0 : 1;
      s += part[((int64_t)c * 2 + slot) * SK_BP * KP + e];
    }
    Z[(p0 + lp) * ldz + col] = s;
  }
}

template <typename TA, typename W, int KP, bool TRANS>
static int sk_grid_slots() {
  typedef SkCfg<TA, W, KP, TRANS> C;
  static int resident = 0;   // CTAs per SM (the same on every GB300)
  static std::once_flag once;
  auto kern = k_prod<TA, W, KP, TRANS>;
  ensure_max_smem((const void*)kern, C::SMEM);   // per device
  std::call_once(once, [kern] {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SK_NT,
                                                      C::SMEM) != cudaSuccess)
      (void)cudaGetLastError();
    resident = std::min(4, std::max(1, per_sm));
  });
  // num_sms() follows the calling thread's CTA limit, so it is read per call
  return resident * num_sms();
}

template <typename TA, typename W, int KP, bool TRANS>
static cnmf_status run_prod(const ProdArgs& a, void* ws, cudaStream_t s) {
  typedef SkCfg<TA, W, KP, TRANS> C;
  const int64_t P = TRANS ? a.n : a.m;
  const int64_t S = TRANS ? a.m : a.n;
  if (P == 0) return CNMF_OK;
  const int64_t tiles = ceil_div(P, SK_BP);
  const int64_t chunks = std::max<int64_t>(1, ceil_div(S, SK_BS));
  const int64_t U = tiles * chunks;
  const int64_t G = std::min<int64_t>(U, sk_grid_slots<TA, W, KP, TRANS>());
  const bool a_vec = ((uintptr_t)a.A % 16 == 0) &&
                     ((a.lda * (int64_t)sizeof(TA)) % 16 == 0);
  const bool b_vec = ((uintptr_t)a.B % 16 == 0) &&
                     ((a.ldb * (int64_t)sizeof(W)) % 16 == 0);
  W* part = reinterpret_cast<W*>(ws);
  k_prod<TA, W, KP, TRANS><<<(unsigned)G, SK_NT, C::SMEM, s>>>(
      (const TA*)a.A, a.m, a.n, a.lda, a_vec, (const W*)a.B, a.ldb, a.kb,
      b_vec, (W*)a.Z, a.ldz, a.kz, part, U, chunks);
  CNMF_CHECK_LAUNCH();
  if (chunks > 1) {
    k_prod_fixup<W, KP><<<dim3((unsigned)tiles, KP / 2), 256, 0, s>>>(
        (W*)a.Z, a.ldz, a.kz, P, part, U, chunks, G);
    CNMF_CHECK_LAUNCH();
  }
  return CNMF_OK;
}

template <typename TA, typename W, bool TRANS>
static cnmf_status dispatch_kp(const ProdArgs& a, void* ws, cudaStream_t s) {
  switch (pad_k(std::max(a.kb, a.kz))) {
    case 16: return run_prod<TA, W, 16, TRANS>(a, ws, s);
    case 32: return run_prod<TA, W, 32, TRANS>(a, ws, s);
    case 48:
    case 64: return run_prod<TA, W, 64, TRANS>(a, ws, s);
    case 80:
    case 96: return run_prod<TA, W, 96, TRANS>(a, ws, s);
    default: return run_prod<TA, W, 128, TRANS>(a, ws, s);
  }
}

static int prod_kp(int k) {
  int p = pad_k(k);
  if (p == 48) return 64;
  if (p == 80) return 96;
  return p;
}

size_t prod_workspace(int64_t m, int64_t n, int k, cnmf_dtype a_type) {
  // two partial tiles per CTA; at most 4 resident CTAs per SM.
  size_t w = a_type == CNMF_F64 ? 8 : 4;
  size_t b = (size_t)4 * num_sms() * 2 * SK_BP * prod_kp(k) * w + 256;
  if (a_type != CNMF_F64) {
    b = std::max(b, tc_workspace(m, n, k));
    b = std::max(b, fused_workspace(m, n, k, a_type));
  }
  return b;
}

cnmf_status launch_prod_fixup_f32(void* Z, int64_t ldz, int kz, int64_t P,
                                  const float* part, int64_t U,
                                  int64_t chunks, int64_t G, int KP,
                                  cudaStream_t s) {
  const unsigned tiles = (unsigned)ceil_div(P, SK_BP);
#define FIX_CASE(K)                                                      \
  case K:                                                                \
    k_prod_fixup<float, K><<<dim3(tiles, K / 2), 256, 0, s>>>(            \
        (float*)Z, ldz, kz, P,                                           \
                                                 part, U, chunks, G);    \
    break;
  switch (KP) {
    FIX_CASE(16)
    FIX_CASE(32)
    FIX_CASE(48)
    FIX_CASE(64)
    FIX_CASE(80)
    FIX_CASE(96)
    FIX_CASE(128)
    default: return CNMF_E_INVALID_ARG;
  }
#undef FIX_CASE
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

static bool tc_disabled() {
  static int v = -1;
  if (v < 0) v = getenv("CNMF_NO_TENSOR_CORES") != nullptr ? 1 : 0;
  return v == 1;
}

cnmf_status launch_prod(const ProdArgs& a, void* ws, size_t ws_bytes,
                        cudaStream_t s) {
  if (ws_bytes < prod_workspace(a.m, a.n, std::max(a.kb, a.kz), a.a_type))
    return CNMF_E_WORKSPACE;
  if (a.a_type != CNMF_F64 && !tc_disabled() && tc_applicable(a))
    return launch_prod_tc(a, ws, a.status, s);
  if (a.a_type == CNMF_F64)
    return a.trans ? dispatch_kp<double, double, true>(a, ws, s)
                   : dispatch_kp<double, double, false>(a, ws, s);
  if (a.a_type == CNMF_F32)
    return a.trans ? dispatch_kp<float, float, true>(a, ws, s)
                   : dispatch_kp<float, float, false>(a, ws, s);
  return a.trans ? dispatch_kp<bf16, float, true>(a, ws, s)
                 : dispatch_kp<bf16, float, false>(a, ws, s);
}

}  // namespace cnmf

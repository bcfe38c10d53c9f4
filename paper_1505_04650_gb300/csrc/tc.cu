// Tensor-core products with A (the sketch products of the compression,
// Alg. 1 power scheme on A and A^T), for BF16- and FP32-stored A:
//
//   Z = A B    (output rows i of A; A tile K-major)           trans = false
//   Z = A^T B  (output rows j = columns of A; A tile MN-major) trans = true
//
// B (FP32, S x k) is first packed into "hi | lo" planes, transposed so that
// the reduction index is contiguous: Bp[c][s] = hi(B[s][c]) and Bp[KP + c][s]
// = lo = B[s][c] - hi.  One MMA with N = 2 KP yields A B_hi and A B_lo side
// by side in TMEM; the epilogue adds the two halves in FP32.
//  * BF16 A (kind::f16): hi, lo are bf16 (|B - hi - lo| <= 2^-18 |B|); A is
//    used exactly as stored.
//  * FP32 A (kind::tf32, 3xTF32 split): hi = B rounded to TF32, lo = the FP32
//    remainder.  The tensor core reads A truncated to TF32 (A_hi); four
//    converter warps write A_lo = A - A_hi into tensor memory (for A^T B
//    A_hi as well, transposed, since an MN-major TF32 operand is not
//    usable) and a second MMA, A from TMEM, adds A_lo B_hi into the hi
//    half.  The dropped terms (A_lo B_lo and the TF32 truncation of the lo
//    parts) are about 2^-20 of |A||B|.
//
// Kernel (one CTA per SM, persistent, stream-K split of (output tile,
// 128-byte reduction chunk) units like the CUDA-core kernel, sharing its
// fix-up): warp 0 lane 0 issues TMA loads (128-byte swizzle) into an
// N-stage mbarrier ring; warp 1 allocates TMEM and lane 0 issues
// tcgen05.mma (M = 128, N = 2 KP, K = 16 bf16 / 8 tf32, FP32 accumulate)
// into one of two TMEM accumulators; for FP32 A, warps 8-11 produce the
// TMEM A operands per stage; warps 4-7 drain finished accumulators with
// tcgen05.ld and write FP32 rows (or split-tile partials).  Every wait is
// bounded: on expiry the kernel records CNMF_E_TIMEOUT, drains its own
// copies and MMAs (bounded), frees TMEM and returns.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace cnmf {

constexpr int TC_BM = 128;   // output rows per tile (MMA M)

// Warp roles: 0 TMA, 1 MMA, 4-7 epilogue, 8-11 (FP32 A) the converters that
// put A_lo (A K-major) or A_hi and A_lo (A MN-major) into tensor memory.
template <int KP, bool F32, bool TRANS>
struct TcCfg {
  static constexpr bool TMEM_A = F32;               // A operand(s) in TMEM
  static constexpr int NT = TMEM_A ? 384 : 256;
  static constexpr int ESZ = F32 ? 4 : 2;           // bytes per A / B element
  static constexpr int BK = 128 / ESZ;              // reduction per stage
  static constexpr int N = 2 * KP;
  static constexpr int A_BYTES = TC_BM * 128;       // 16 KiB
  static constexpr int B_BYTES = N * 128;           // N rows x 128 B
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int ST_FIT = (200 * 1024) / STAGE;
  // TMEM: NACC accumulators of N columns, then (TMEM_A) per stage ACOLS
  // columns: A_lo (K-major A, whose A_hi the MMA reads from shared
  // memory), or A_hi and A_lo (MN-major A).
  static constexpr int ACOLS = TRANS ? 2 * BK : BK;
  static constexpr int NACC = (!TMEM_A || 512 - 2 * N >= 3 * ACOLS) ? 2 : 1;
  static constexpr int ST_TMEM = TMEM_A ? (512 - NACC * N) / ACOLS : 8;
  static constexpr int ST_A = ST_FIT < ST_TMEM ? ST_FIT : ST_TMEM;
  static constexpr int STAGES = ST_A > 8 ? 8 : ST_A;
  static constexpr int TMEM_COLS = TMEM_A ? 512
                                   : NACC * N <= 64 ? 64
                                   : NACC * N <= 128 ? 128
                                   : NACC * N <= 256 ? 256 : 512;
  static constexpr int A_TMEM = NACC * N;           // first A column
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE;
  static_assert(STAGES >= 2, "pipeline needs two stages");
};

__host__ __device__ __forceinline__ int64_t tc_split_start(int64_t c, int64_t U,
                                                           int64_t G) {
  return (c * U) / G;
}

// ---------------------------------------------------------------------------
// B (S x kb, FP32, pitch ldb) -> Bp (2 KP x spad, bf16 or TF32-valued FP32),
// transposed hi | lo.
// ---------------------------------------------------------------------------
template <bool F32>
__global__ void k_pack_panel(const float* __restrict__ B, int64_t S,
                             int64_t ldb, int kb, int KP,
                             void* __restrict__ Bpv, int64_t spad) {
  __shared__ float tile[32][33];
  const int64_t s0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t s = s0 + r;
    const int c = c0 + tx;
    tile[r][tx] = (s < S && c < kb) ? B[s * ldb + c] : 0.0f;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += 8) {
    const int c = c0 + cc;
    const int64_t s = s0 + tx;
    if (c >= KP || s >= spad) continue;
    const float v = tile[tx][cc];
    if (F32) {
      float* Bp = reinterpret_cast<float*>(Bpv);
      const float hi = tf32_rna(v);
      Bp[(int64_t)c * spad + s] = hi;
      Bp[(int64_t)(KP + c) * spad + s] = tf32_rna(v - hi);
    } else {
      bf16* Bp = reinterpret_cast<bf16*>(Bpv);
      const bf16 hi = __float2bfloat16_rn(v);
      Bp[(int64_t)c * spad + s] = hi;
      Bp[(int64_t)(KP + c) * spad + s] =
          __float2bfloat16_rn(v - __bfloat162float(hi));
    }
  }
}

// ---------------------------------------------------------------------------
// The product kernel
// ---------------------------------------------------------------------------
template <int KP, bool TRANS, bool F32>
__global__ void __launch_bounds__((TcCfg<KP, F32, TRANS>::NT), 1)
    k_tc_prod(const __grid_constant__ CUtensorMap tmA,
              const __grid_constant__ CUtensorMap tmB, int64_t P,
              float* __restrict__ Z, int64_t ldz, int kz,
              float* __restrict__ part, int64_t U, int64_t chunks,
              int32_t* status) {
  typedef TcCfg<KP, F32, TRANS> C;
  constexpr int N = C::N;
  constexpr int ST = C::STAGES;
  constexpr int NACC = C::NACC;
  constexpr bool TMEM_A = C::TMEM_A;
  constexpr int BK = C::BK;
  constexpr int MMA_K = F32 ? 8 : 16;                // reduction per MMA
  // A from TMEM is K-major; from shared memory K-major unless TRANS
  constexpr bool A_MN = TRANS && !TMEM_A;
  constexpr uint32_t IDESC = idesc_mk(TC_BM, N, A_MN, F32);
  constexpr uint32_t IDESC_HI = idesc_mk(TC_BM, KP, A_MN, F32);
  // MN-major A: one TMA box per 128-byte chunk of the MN index
  constexpr int MN_CHUNK = 128 / C::ESZ;             // 64 bf16 / 32 fp32
  constexpr int BOX_BYTES = MN_CHUNK * BK * C::ESZ;  // bytes of one box
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[8], empty_bar[8], lo_bar[8];
  __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], drain_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t G = gridDim.x, c = blockIdx.x;
  const int64_t u0 = tc_split_start(c, U, G), u1 = tc_split_start(c + 1, U, G);

  if (threadIdx.x == 0) {
    for (int i = 0; i < ST; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
      mbar_init(&lo_bar[i], 4);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf_bar[i], 1);
      mbar_init(&acce_bar[i], 128);
    }
    mbar_init(&drain_bar, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::
            "r"(smem_u32(&tmem_base_s)),
        "r"(C::TMEM_COLS)
        : "memory");
    asm volatile(
        "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::
            : "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int stage = 0;
    uint32_t phase = 0;
    uint32_t issued_phase[8];
    bool issued[8];
    for (int i = 0; i < 8; ++i) { issued[i] = false; issued_phase[i] = 0; }
    int64_t u = u0;
    bool ok = true;
    while (ok && u < u1) {
      const int64_t tp = u / chunks, ts0 = u % chunks;
      const int64_t ts1 = min(chunks, ts0 + (u1 - u));
      for (int64_t ts = ts0; ts < ts1; ++ts) {
        if (!mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_s, status)) {
          ok = false;
          break;
        }
        unsigned char* sa = smem + (size_t)stage * C::STAGE;
        unsigned char* sb = sa + C::A_BYTES;
        mbar_expect_tx(&full_bar[stage], (uint32_t)(C::A_BYTES + C::B_BYTES));
        if (!TRANS) {
          tma_load_2d(sa, &tmA, (int)(ts * BK), (int)(tp * TC_BM),
                      &full_bar[stage]);
        } else {
#pragma unroll
          for (int b = 0; b < TC_BM / MN_CHUNK; ++b)
            tma_load_2d(sa + b * BOX_BYTES, &tmA,
                        (int)(tp * TC_BM + b * MN_CHUNK), (int)(ts * BK),
                        &full_bar[stage]);
        }
        tma_load_2d(sb, &tmB, (int)(ts * BK), 0, &full_bar[stage]);
        issued[stage] = true;
        issued_phase[stage] = phase;
        if (++stage == ST) { stage = 0; phase ^= 1u; }
      }
      u = tp * chunks + ts1;
    }
    // drain: every copy this thread issued has landed before teardown
    for (int i = 0; i < ST; ++i)
      if (issued[i]) {
        if (!mbar_try(&full_bar[i], issued_phase[i])) {
          const uint64_t t0 = globaltimer_ns();
          while (!mbar_try(&full_bar[i], issued_phase[i]) &&
                 globaltimer_ns() - t0 < 2000000000ull) {
          }
        }
      }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int stage = 0;
    uint32_t phase = 0;
    int ab = 0;
    uint32_t aphase = 0;
    bool any = false;
    int64_t u = u0;
    bool ok = true;
    while (ok && u < u1) {
      const int64_t tp = u / chunks, ts0 = u % chunks;
      const int64_t ts1 = min(chunks, ts0 + (u1 - u));
      if (!mbar_wait(&acce_bar[ab], aphase ^ 1u, &abort_s, status)) break;
      tc_fence_after();
      const uint32_t dtm = tmem + (uint32_t)(ab * N);
      for (int64_t ts = ts0; ts < ts1; ++ts) {
        if (!mbar_wait(&full_bar[stage], phase, &abort_s, status) ||
            (F32 && !mbar_wait(&lo_bar[stage], phase, &abort_s, status))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + (size_t)stage * C::STAGE);
        const uint32_t sb = sa + C::A_BYTES;
        const uint32_t at = tmem + (uint32_t)(C::A_TMEM + stage * C::ACOLS);
        if (TMEM_A && TRANS) {
          // A_hi . [B_hi | B_lo], then A_lo . B_hi, A from this stage's
          // TMEM columns
#pragma unroll
          for (int kk = 0; kk < BK / MMA_K; ++kk)
            tc_mma_tf32_ta(dtm, at + kk * MMA_K, sdesc(sb + kk * 32, 16, 1024),
                           IDESC, (ts > ts0 || kk > 0) ? 1u : 0u);
#pragma unroll
          for (int kk = 0; kk < BK / MMA_K; ++kk)
            tc_mma_tf32_ta(dtm, at + BK + kk * MMA_K,
                           sdesc(sb + kk * 32, 16, 1024), IDESC_HI, 1u);
          any = true;
        } else {
#pragma unroll
        for (int kk = 0; kk < BK / MMA_K; ++kk) {
          // K-major: the next MMA_K elements sit 32 bytes further along the
          // swizzled row; MN-major: MMA_K rows of 128 bytes further.
          const uint64_t ad =
              !TRANS ? sdesc(sa + kk * 32, 16, 1024)
                     : sdesc(sa + kk * MMA_K * 128, BOX_BYTES, 1024);
          const uint64_t bd = sdesc(sb + kk * 32, 16, 1024);
          const uint32_t acc = (ts > ts0 || kk > 0) ? 1u : 0u;
          if (F32) tc_mma_tf32(dtm, ad, bd, IDESC, acc);
          else tc_mma(dtm, ad, bd, IDESC, acc);
          any = true;
        }
        if (F32) {   // A_lo (TMEM) . B_hi into the hi half
#pragma unroll
          for (int kk = 0; kk < BK / MMA_K; ++kk)
            tc_mma_tf32_ta(dtm, at + kk * MMA_K, sdesc(sb + kk * 32, 16, 1024),
                           IDESC_HI, 1u);
        }
        }
        tc_commit(&empty_bar[stage]);
        if (++stage == ST) { stage = 0; phase ^= 1u; }
      }
      if (!ok) break;
      tc_commit(&accf_bar[ab]);
      if (++ab == NACC) { ab = 0; aphase ^= 1u; }
      u = tp * chunks + ts1;
    }
    if (any) {   // all MMAs complete before TMEM is released
      tc_commit(&drain_bar);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try(&drain_bar, 0) && globaltimer_ns() - t0 < 2000000000ull) {
      }
    }
  } else if (TMEM_A && warp >= 8) {
    // ---------------- A operands into TMEM (FP32 A) ----------------
    // Warp 8 + w owns TMEM lanes 32 w .. 32 w + 31.  The tensor core reads
    // an FP32 operand as TF32 (the low 13 mantissa bits ignored), so
    // A_hi = A as stored and A_lo = A - A_hi exactly.
    //  * K-major tile (A X): lane l takes row i = 32 w + l of the tile, its
    //    eight 16-byte chunks swizzled by i mod 8, and stores its A_lo row.
    //  * MN-major tile (A^T Y): lane l reads column j = 32 w + l (row i of
    //    TMA box w is 128 bytes, chunks swizzled by i mod 8), so TMEM lane j
    //    gets row j of A^T: A_hi and A_lo, K-major.
    const int w = warp - 8;
    int stage = 0;
    uint32_t phase = 0;
    int64_t u = u0;
    bool ok = true;
    while (ok && u < u1) {
      const int64_t tp = u / chunks, ts0 = u % chunks;
      const int64_t ts1 = min(chunks, ts0 + (u1 - u));
      for (int64_t ts = ts0; ts < ts1; ++ts) {
        if (!mbar_wait(&full_bar[stage], phase, &abort_s, status)) {
          ok = false;
          break;
        }
        const uint32_t ta = tmem + ((uint32_t)(32 * w) << 16) +
                            (uint32_t)(C::A_TMEM + stage * C::ACOLS);
        uint32_t lo[32];
        if (!TRANS) {
          const int i = 32 * w + lane;
          const unsigned char* rowp = smem + (size_t)stage * C::STAGE + i * 128;
#pragma unroll
          for (int cch = 0; cch < 8; ++cch) {
            const float4 v = *reinterpret_cast<const float4*>(
                rowp + ((cch ^ (i & 7)) << 4));
            const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
              lo[4 * cch + q] = __float_as_uint(
                  e[q] - __uint_as_float(__float_as_uint(e[q]) & 0xFFFFE000u));
          }
          tc_st32(ta, lo);
        } else {
          const unsigned char* box = smem + (size_t)stage * C::STAGE +
                                     w * BOX_BYTES + (lane & 3) * 4;
          uint32_t hi[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float v = *reinterpret_cast<const float*>(
                box + i * 128 + ((((lane >> 2) ^ i) & 7) << 4));
            hi[i] = __float_as_uint(v);
            lo[i] = __float_as_uint(v - __uint_as_float(hi[i] & 0xFFFFE000u));
          }
          tc_st32(ta, hi);
          tc_st32(ta + BK, lo);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&lo_bar[stage]);
        if (++stage == ST) { stage = 0; phase ^= 1u; }
      }
      u = tp * chunks + ts1;
    }
  } else if (warp >= 4 && warp < 8) {
    // ---------------- epilogue ----------------
    const int q = warp - 4;                 // TMEM lane quarter
    const int row = 32 * q + lane;
    int ab = 0;
    uint32_t aphase = 0;
    int64_t u = u0;
    bool first = true;
    while (u < u1) {
      const int64_t tp = u / chunks, ts0 = u % chunks;
      const int64_t ts1 = min(chunks, ts0 + (u1 - u));
      if (!mbar_wait(&accf_bar[ab], aphase, &abort_s, status)) break;
      tc_fence_after();
      const bool whole = (ts0 == 0 && ts1 == chunks);
      const int64_t p = tp * TC_BM + row;
      float* dst = whole ? (p < P ? Z + p * ldz : nullptr)
                         : part + (((size_t)c * 2 + (first ? 0 : 1)) * TC_BM +
                                   row) * KP;
      const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * N);
#pragma unroll 1
      for (int c0 = 0; c0 < KP; c0 += 16) {
        float hi[16], lo[16];
        tc_ld16(tbase + c0, hi);
        tc_ld16(tbase + KP + c0, lo);
        if (dst) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int col = c0 + t;
            if (!whole || col < kz) dst[col] = hi[t] + lo[t];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&acce_bar[ab]);
      if (++ab == NACC) { ab = 0; aphase ^= 1u; }
      first = false;
      u = tp * chunks + ts1;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                     tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int tc_kp(int k) { return pad_k(k); }

size_t tc_workspace(int64_t m, int64_t n, int k) {
  // split-tile partials, then the packed B panel (4 bytes per element covers
  // both the bf16 and the TF32 packing)
  const int KP = tc_kp(k);
  const int64_t spad = (std::max(m, n) + 7) / 8 * 8;
  size_t b = 0;
  b += (((size_t)num_sms() * 2 * TC_BM * KP * 4) + 255) & ~size_t(255);
  b += (((size_t)2 * KP * spad * 4) + 255) & ~size_t(255);
  return b + 256;
}

bool tc_applicable(const ProdArgs& a) {
  if (a.a_type != CNMF_BF16 && a.a_type != CNMF_F32) return false;
  const int64_t es = a.a_type == CNMF_F32 ? 4 : 2;
  if ((uintptr_t)a.A % 16 != 0 || (a.lda * es) % 16 != 0) return false;
  if (std::max(a.kb, a.kz) > 128 || a.m < 1 || a.n < 1) return false;
  if (a.m >= (1ll << 31) || a.n >= (1ll << 31)) return false;
  return tmap_encoder() != nullptr;
}

template <int KP, bool TRANS, bool F32>
static cnmf_status run_tc(const ProdArgs& a, void* ws, int32_t* status,
                          cudaStream_t s) {
  typedef TcCfg<KP, F32, TRANS> C;
  // raised once per (kernel, device)
  if (!ensure_max_smem((const void*)k_tc_prod<KP, TRANS, F32>, C::SMEM))
    return CNMF_E_INVALID_ARG;
  const int64_t P = TRANS ? a.n : a.m;
  const int64_t S = TRANS ? a.m : a.n;
  const int64_t spad = (S + 7) / 8 * 8;
  Carve cv(ws, SIZE_MAX);
  float* part = cv.take<float>((size_t)num_sms() * 2 * TC_BM * KP);
  void* Bp = cv.take<char>((size_t)2 * KP * spad * C::ESZ);
  // pack B
  dim3 pg((unsigned)ceil_div(spad, 32), (unsigned)ceil_div(KP, 32));
  k_pack_panel<F32><<<pg, 256, 0, s>>>((const float*)a.B, S, a.ldb, a.kb, KP,
                                       Bp, spad);
  CNMF_CHECK_LAUNCH();
  CUtensorMap ta, tb;
  bool ok;
  constexpr int MN_CHUNK = 128 / C::ESZ;
  if (!TRANS)
    ok = make_map(&ta, a.A, F32, (uint64_t)a.n, (uint64_t)a.m,
                  (uint64_t)a.lda * C::ESZ, C::BK, TC_BM);
  else
    ok = make_map(&ta, a.A, F32, (uint64_t)a.n, (uint64_t)a.m,
                  (uint64_t)a.lda * C::ESZ, MN_CHUNK, C::BK);
  ok = ok && make_map(&tb, Bp, F32, (uint64_t)spad, (uint64_t)(2 * KP),
                      (uint64_t)spad * C::ESZ, C::BK, 2 * KP);
  if (!ok) return CNMF_E_INVALID_ARG;
  const int64_t tiles = ceil_div(P, TC_BM);
  const int64_t chunks = std::max<int64_t>(1, ceil_div(S, C::BK));
  const int64_t U = tiles * chunks;
  const int64_t G = std::min<int64_t>(U, num_sms());
  k_tc_prod<KP, TRANS, F32><<<(unsigned)G, C::NT, C::SMEM, s>>>(
      ta, tb, P, (float*)a.Z, a.ldz, a.kz, part, U, chunks, status);
  CNMF_CHECK_LAUNCH();
  if (chunks > 1)
    CNMF_TRY(launch_prod_fixup_f32(a.Z, a.ldz, a.kz, P, part, U, chunks, G, KP,
                                   s));
  return CNMF_OK;
}

cnmf_status launch_prod_tc(const ProdArgs& a, void* ws, int32_t* status,
                           cudaStream_t s) {
  const int KP = tc_kp(std::max(a.kb, a.kz));
  const bool f32 = a.a_type == CNMF_F32;
#define TC_CASE(K)                                                        \
  case K:                                                                 \
    if (f32)                                                              \
      return a.trans ? run_tc<K, true, true>(a, ws, status, s)            \
                     : run_tc<K, false, true>(a, ws, status, s);          \
    return a.trans ? run_tc<K, true, false>(a, ws, status, s)             \
                   : run_tc<K, false, false>(a, ws, status, s);
  switch (KP) {
    TC_CASE(16)
    TC_CASE(32)
    TC_CASE(48)
    TC_CASE(64)
    TC_CASE(80)
    TC_CASE(96)
    TC_CASE(128)
  }
#undef TC_CASE
  return CNMF_E_INVALID_ARG;
}

}  // namespace cnmf

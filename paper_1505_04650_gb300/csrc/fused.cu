// Fused two-sided sketch pass: one power pass of the structured random
// compression applied to A and A^T (Alg. 1 power scheme, Sec. III),
//
//   Zm = A X   (m x k, from X n x k)   and   Zn = A^T Y   (n x k, from Y m x k),
//
// computed from ONE read of A.  At every pass the left chain needs one of
// the two products and the right chain the other, so a pass of the
// two-sided compression is exactly this pair.  Either side may be left out
// (a one-sided product, as in A-check = A R^T).
//
// A is cut into 128 x 128 tiles.  Each tile is loaded once by TMA (128-byte
// swizzle) and feeds both products on the tensor cores (tcgen05 kind::f16,
// bf16 operands, FP32 accumulation in tensor memory) from the same shared
// memory:
//  * A X:   M = the tile's 128 rows i, K = its columns j; A read K-major.
//  * A^T Y: M = the tile's 128 columns j, K = its rows i; the same bytes
//    read MN-major.
// BF16 A is used as stored.  FP32 A is split in place by converter warps
// into two bf16 tiles, A_hi = bf16(A) and A_lo = bf16(A - A_hi), both
// rounded to nearest, so |A - A_hi - A_lo| <= 2^-18 |A|; both products take
// both terms.  X and Y (FP32) are split the same way into bf16 hi | lo
// planes, packed transposed (the K-major B operand).  A X places them side
// by side along N (N = 2 KP), so one MMA forms A X_hi and A X_lo together
// and the epilogue adds the halves; A^T Y adds them in its accumulator
// through two MMAs.  Every product of two bf16 values is exact in FP32, so
// the result is (A_hi + A_lo)(X_hi + X_lo) up to FP32 accumulation, minus,
// for FP32 A, the term A_lo Y_lo of A^T Y (below 2^-18 of |A||Y|).
//
// Work order (stream-K over tiles, one persistent CTA per SM): the tile
// columns are cut into groups of Tj (as many A^T Y accumulators as tensor
// memory holds); tiles are ordered (group, row, column) and CTA c takes the
// contiguous range [c U / G, (c + 1) U / G) of the U tiles.  Along a row of
// a group the A X accumulator (double-buffered) collects the row's columns;
// over the rows of its range a CTA keeps one A^T Y accumulator per column
// of the group.  Finished accumulators go to partial slots in the
// workspace, and a second kernel sums each row's (column's) slots in a
// fixed order, so the output does not depend on timing and no
// floating-point atomics are used.
//
// Warp roles: 0 lane 0 TMA of A tiles (stage ring), 1 lane 0 the A X MMAs,
// 3 lane 0 the A^T Y MMAs, 2 lane 0 TMA of the group's X tiles and of the Y
// tiles, 4-7 epilogue (tcgen05.ld, partials), 8-15 (FP32 A) the converters.
// Every wait is bounded: on expiry the kernel records CNMF_E_TIMEOUT, lets
// its own copies and MMAs finish (bounded), frees tensor memory and returns.
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace cnmf {

constexpr int FU_T = 128;                      // tile edge
constexpr int FU_BOX = FU_T * 128;             // 128 rows x 128 bytes
constexpr int FU_SMEM = 232448 - 1024 - 512;   // dynamic budget (opt-in max
                                               // minus alignment and static)

template <int KP, bool F32>
struct FuCfg {
  static constexpr int ESZ = F32 ? 4 : 2;
  static constexpr int BOXW = 128 / ESZ;        // tile columns per TMA box
  static constexpr int NBOX = FU_T / BOXW;      // 4 (FP32) / 2 (BF16)
  static constexpr int A_BYTES = NBOX * FU_BOX;
  static constexpr int NTERM = F32 ? 2 : 1;     // bf16 terms of A
  static constexpr int LO_OFF = 2 * FU_BOX;     // A_lo after A_hi (FP32)
  static constexpr int P_BOX = 2 * KP * 128;    // KP hi rows, KP lo rows
  static constexpr int P_LO = KP * 128;         // lo rows inside a box
  static constexpr int P_BYTES = 2 * P_BOX;     // 128 values along K
  static constexpr int STAGE = A_BYTES + P_BYTES;   // A tile + X tile
  static constexpr int YBUF = 2;
  static constexpr int ST_FIT = (FU_SMEM - YBUF * P_BYTES) / STAGE;
  static constexpr int STAGES = ST_FIT > 4 ? 4 : ST_FIT;
  static constexpr size_t SMEM =
      1024 + (size_t)STAGES * STAGE + (size_t)YBUF * P_BYTES;
  // A X accumulators (two, double-buffered) hold the hi and lo parts side
  // by side (N = 2 KP: one MMA per K-chunk and term); the A^T Y
  // accumulators (one per column of a group) take the hi and lo parts
  // through two MMAs into KP columns, so tensor memory holds
  // (512 - 4 KP) / KP of them -- fewer A X partials
  static constexpr int ZX = 2 * KP;
  static constexpr int ZY = KP;
  static constexpr int NCONV = F32 ? 16 : 0;    // converter warps
  static constexpr int NT = 256 + 32 * NCONV;
  static_assert(STAGES >= 2, "fused pass needs two stages");
  static_assert(!F32 || NBOX == 4, "converter mapping assumes 4 FP32 boxes");
};

// Geometry of the tile walk (identical in every role and in the host code).
struct FuGeom {
  int TI, TJ;        // tile rows / columns of A
  int Tj, NG, wlast; // group width, groups, width of the last group
  int G;             // CTAs
  int64_t U;         // tiles
  int has_x, has_y;  // which products (A X, A^T Y) this launch forms
  int z2col;         // first tensor-memory column of the A^T Y accumulators
};

struct FuPos {
  int64_t u;
  int g, i, jl;      // group, tile row, column in group
  int w;             // columns of this group
};

__host__ __device__ __forceinline__ int fu_w(const FuGeom& q, int g) {
  return g == q.NG - 1 ? q.wlast : q.Tj;
}
// first tile of group g
__host__ __device__ __forceinline__ int64_t fu_gs(const FuGeom& q, int g) {
  return (int64_t)g * q.TI * q.Tj;
}
// the CTA whose range holds tile u
__host__ __device__ __forceinline__ int fu_owner(const FuGeom& q, int64_t u) {
  const int64_t c = ((u + 1) * q.G + q.U - 1) / q.U - 1;
  return (int)(c < q.G - 1 ? c : q.G - 1);
}
__host__ __device__ __forceinline__ int64_t fu_start(const FuGeom& q, int c) {
  return (int64_t)c * q.U / q.G;
}

__device__ __forceinline__ void fu_decode(const FuGeom& q, int64_t u,
                                          FuPos& p) {
  p.u = u;
  const int64_t gfull = (int64_t)q.TI * q.Tj;
  const int64_t gq = u / gfull;
  p.g = gq < q.NG - 1 ? (int)gq : q.NG - 1;
  const int64_t r = u - fu_gs(q, p.g);
  p.w = fu_w(q, p.g);
  p.i = (int)(r / p.w);
  p.jl = (int)(r - (int64_t)p.i * p.w);
}
__device__ __forceinline__ void fu_next(const FuGeom& q, FuPos& p) {
  ++p.u;
  if (++p.jl < p.w) return;
  p.jl = 0;
  if (++p.i < q.TI) return;
  p.i = 0;
  ++p.g;
  p.w = fu_w(q, p.g < q.NG ? p.g : q.NG - 1);
}

struct FuOut {
  float* Zm;
  int64_t ldzm;
  float* Zn;
  int64_t ldzn;
  int kz;
  int64_t m, n;
  float* P1;          // A X partials: (segments + G) slots of 128 x KP
  float* P2;          // A^T Y partials: (groups + G) x Tj slots of 128 x KP
  int32_t* status;
};

// ---------------------------------------------------------------------------
// X (n x kb) and Y (m x kb), FP32 with pitches, -> transposed bf16 hi | lo
// planes Xp (2 KP x spn) and Yp (2 KP x spm); z = 0 packs X, z = 1 packs Y
// (a NULL panel is skipped).
// ---------------------------------------------------------------------------
__global__ void k_fu_pack(const float* __restrict__ X, int64_t ldx, int64_t n,
                          const float* __restrict__ Y, int64_t ldy, int64_t m,
                          int kb, int KP, bf16* __restrict__ Xp, int64_t spn,
                          bf16* __restrict__ Yp, int64_t spm) {
  __shared__ float tile[32][33];
  // X, Y come from the kernel before; once they can be read, the fused
  // pass may launch and start its loads of A
  pdl_wait();
  pdl_release();
  const bool xs = blockIdx.z == 0;
  const float* B = xs ? X : Y;
  if (!B) return;
  const int64_t ldb = xs ? ldx : ldy;
  const int64_t S = xs ? n : m;
  const int64_t spad = xs ? spn : spm;
  bf16* Bp = xs ? Xp : Yp;
  const int64_t s0 = (int64_t)blockIdx.x * 32;
  if (s0 >= spad) return;
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
    const bf16 hi = __float2bfloat16_rn(v);
    Bp[(int64_t)c * spad + s] = hi;
    Bp[(int64_t)(KP + c) * spad + s] =
        __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// Eight FP32 values -> bf16 hi and lo parts, packed in tile-column order.
__device__ __forceinline__ void fu_split8(const float4& a, const float4& b,
                                          uint4& hi, uint4& lo) {
  const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint32_t h[4], l[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const __nv_bfloat162 hv = __floats2bfloat162_rn(x[2 * t], x[2 * t + 1]);
    const float2 hf = __bfloat1622float2(hv);
    const __nv_bfloat162 lv =
        __floats2bfloat162_rn(x[2 * t] - hf.x, x[2 * t + 1] - hf.y);
    h[t] = *reinterpret_cast<const uint32_t*>(&hv);
    l[t] = *reinterpret_cast<const uint32_t*>(&lv);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// ---------------------------------------------------------------------------
// The fused kernel
// ---------------------------------------------------------------------------
template <int KP, bool F32>
__global__ void __launch_bounds__((FuCfg<KP, F32>::NT), 1)
    k_fused_pass(const __grid_constant__ CUtensorMap tmA,
                 const __grid_constant__ CUtensorMap tmX,
                 const __grid_constant__ CUtensorMap tmY, const FuGeom geo,
                 const FuOut out) {
  typedef FuCfg<KP, F32> C;
  constexpr int ST = C::STAGES;
  constexpr int YB = C::YBUF;
  constexpr uint32_t ID_X = idesc_mk(FU_T, C::ZX, false, false);
  constexpr uint32_t ID_T = idesc_mk(FU_T, C::ZY, true, false);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[4], conv_bar[4], empty_bar[4];
  __shared__ __align__(8) uint64_t y_full[2], y_empty[2];
  __shared__ __align__(8) uint64_t z1_full[2], z1_empty[2], z2_full,
      z2_empty[16],
      drain_bar[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* ysm = smem + (size_t)ST * C::STAGE;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int c = blockIdx.x;
  const int64_t u0 = fu_start(geo, c), u1 = fu_start(geo, c + 1);
  const bool hx = geo.has_x != 0, hy = geo.has_y != 0;
  int32_t* status = out.status;

  if (threadIdx.x == 0) {
    for (int i = 0; i < ST; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&conv_bar[i], C::NCONV > 0 ? C::NCONV : 1);
      // one commit per issuing thread (A X, A^T Y)
      mbar_init(&empty_bar[i], (uint32_t)(geo.has_x + geo.has_y));
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&y_full[i], 1);
      mbar_init(&y_empty[i], 1);
      mbar_init(&z1_full[i], 1);
      mbar_init(&z1_empty[i], 128);
      mbar_init(&drain_bar[i], 1);
    }
    mbar_init(&z2_full, 1);
    for (int i = 0; i < 16; ++i) mbar_init(&z2_empty[i], 128);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::
            "r"(smem_u32(&tmem_base_s)),
        "r"(512)
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
    // ---------------- TMA: A tile (+ X tile) per stage ----------------
    const uint64_t pol = l2_evict_first();
    const uint32_t bytes = (uint32_t)(C::A_BYTES + (hx ? C::P_BYTES : 0));
    int s = 0;
    uint32_t ph = 0;
    int64_t nissued = 0;
    FuPos p, pd;
    fu_decode(geo, u0, p);
    pd = p;
    // The first min(ST, tiles) stages get their A tiles before the wait for
    // the kernel before (A is no output of it); their X tiles, which it
    // writes, follow the wait, before any stage is reused.
    const int64_t npre = u1 - u0 < ST ? u1 - u0 : ST;
    bool waited = false;
    auto load_x = [&](int st, const FuPos& q) {
      unsigned char* sx = smem + (size_t)st * C::STAGE + C::A_BYTES;
      const int jt = q.g * geo.Tj + q.jl;
#pragma unroll
      for (int b = 0; b < 2; ++b)
        tma_load_2d(sx + b * C::P_BOX, &tmX, jt * FU_T + b * 64, 0,
                    &full_bar[st]);
    };
    auto release_x = [&]() {
      pdl_wait();
      waited = true;
      if (!hx) return;
      for (int64_t t = 0; t < nissued && t < npre; ++t, fu_next(geo, pd))
        load_x((int)t, pd);
    };
    for (int64_t u = u0; u < u1; ++u, fu_next(geo, p)) {
      if (!waited && u - u0 == npre) release_x();
      if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_s, status)) break;
      unsigned char* sa = smem + (size_t)s * C::STAGE;
      const int jt = p.g * geo.Tj + p.jl;
      mbar_expect_tx(&full_bar[s], bytes);
#pragma unroll
      for (int b = 0; b < C::NBOX; ++b)
        tma_load_2d_hint(sa + b * FU_BOX, &tmA, jt * FU_T + b * C::BOXW,
                         p.i * FU_T, &full_bar[s], pol);
      if (hx && waited) load_x(s, p);
      ++nissued;
      if (++s == ST) { s = 0; ph ^= 1u; }
    }
    if (!waited) release_x();
    // every copy has landed before exit (bounded): the last ST loads
    for (int64_t t = nissued - 1; t >= 0 && t >= nissued - ST; --t) {
      uint64_t* fb = &full_bar[t % ST];
      const uint32_t fph = (uint32_t)((t / ST) & 1);
      const uint64_t t0 = globaltimer_ns();
      while (!mbar_try(fb, fph) && globaltimer_ns() - t0 < 2000000000ull) {
      }
    }
  } else if (warp == 2 && lane == 0) {
    // ---------------- TMA: Y tile per row segment ----------------
    pdl_wait();   // Y comes from the kernel before
    if (hy) {
      int yb = 0;
      uint32_t yph = 0;
      int64_t nissued = 0;
      FuPos p;
      fu_decode(geo, u0, p);
      for (int64_t u = u0; u < u1; ++u, fu_next(geo, p)) {
        if (!(u == u0 || p.jl == 0)) continue;
        if (!mbar_wait(&y_empty[yb], yph ^ 1u, &abort_s, status)) break;
        unsigned char* sy = ysm + (size_t)yb * C::P_BYTES;
        mbar_expect_tx(&y_full[yb], (uint32_t)C::P_BYTES);
#pragma unroll
        for (int b = 0; b < 2; ++b)
          tma_load_2d(sy + b * C::P_BOX, &tmY, p.i * FU_T + b * 64, 0,
                      &y_full[yb]);
        ++nissued;
        if (++yb == YB) { yb = 0; yph ^= 1u; }
      }
      for (int64_t t = nissued - 1; t >= 0 && t >= nissued - YB; --t) {
        uint64_t* fb = &y_full[t % YB];
        const uint32_t fph = (uint32_t)((t / YB) & 1);
        const uint64_t t0 = globaltimer_ns();
        while (!mbar_try(fb, fph) && globaltimer_ns() - t0 < 2000000000ull) {
        }
      }
    }
  } else if ((warp == 1 || warp == 3) && lane == 0) {
    // ---------------- MMA issue ----------------
    // Two issuing threads: warp 1 forms A X (accumulators Z1, one per row
    // segment, double-buffered), warp 3 forms A^T Y (accumulators Z2, one
    // per column of the group).  Each releases a stage with its own commit,
    // so the two MMA streams are issued side by side from two SM
    // sub-partitions.  Per K-chunk of 16 and per bf16 term of A: one A X
    // MMA on the panel's hi | lo rows; A^T Y MMAs on the hi rows and on the
    // lo rows (FP32 A: A_lo Y_lo, below 2^-18 of |A||Y|, is left out).
    const bool is_x = warp == 1;
    if ((is_x && hx) || (!is_x && hy)) {
      int s = 0, zb = 0, yb = 0;
      uint32_t ph = 0, zph = 0, yph = 0;
      // bit jl: parity of the number of drains of A^T Y accumulator jl so
      // far (the epilogue drains columns 0 .. w - 1 at every run's end)
      uint32_t drained = 0;
      uint32_t touched = 0;
      bool any = false;
      const uint32_t smem0 = smem_u32(smem);
      const uint32_t ys0 = smem_u32(ysm);
      FuPos p;
      fu_decode(geo, u0, p);
      for (int64_t u = u0; u < u1; ++u, fu_next(geo, p)) {
        const bool seg_first = (u == u0) || p.jl == 0;
        const bool seg_last = (u == u1 - 1) || p.jl == p.w - 1;
        const bool run_first = (u == u0) || (p.i == 0 && p.jl == 0);
        const bool run_last =
            (u == u1 - 1) || (p.i == geo.TI - 1 && p.jl == p.w - 1);
        if (is_x) {
          if (seg_first &&
              !mbar_wait(&z1_empty[zb], zph ^ 1u, &abort_s, status))
            break;
        } else {
          if (run_first) touched = 0;
          // the first MMA of a run into accumulator jl waits only for the
          // epilogue to have drained that accumulator, so a new run starts
          // while the previous run's other columns are still being drained
          if (((touched >> p.jl) & 1u) == 0 &&
              !mbar_wait(&z2_empty[p.jl], ((drained >> p.jl) & 1u) ^ 1u,
                         &abort_s, status))
            break;
          if (seg_first && !mbar_wait(&y_full[yb], yph, &abort_s, status))
            break;
        }
        if (!mbar_wait(F32 ? &conv_bar[s] : &full_bar[s], ph, &abort_s,
                       status))
          break;
        tc_fence_after();
        const uint32_t sa = smem0 + (uint32_t)(s * C::STAGE);
        // Descriptors of the stage's first K-chunk; a K-chunk further is the
        // descriptor plus the byte offset / 16 (the start-address field).
        if (is_x) {
          const uint32_t z1 = tmem + (uint32_t)(zb * C::ZX);
          const uint64_t dA = sdesc(sa, 16, 1024);   // K-major: rows i
          const uint64_t dX = sdesc(sa + C::A_BYTES, 16, 1024);
#pragma unroll
          for (int kc = 0; kc < FU_T / 16; ++kc) {
            // 16 columns j of the tile: box kc / 4, chunk kc % 4
            const uint64_t pk =
                (uint64_t)(((kc >> 2) * C::P_BOX + (kc & 3) * 32) >> 4);
            const uint64_t ak =
                (uint64_t)(((kc >> 2) * FU_BOX + (kc & 3) * 32) >> 4);
#pragma unroll
            for (int t = 0; t < C::NTERM; ++t)
              tc_mma(z1, dA + (uint64_t)((t * C::LO_OFF) >> 4) + ak, dX + pk,
                     ID_X, (seg_first && kc == 0 && t == 0) ? 0u : 1u);
          }
          tc_commit(&empty_bar[s]);
          if (seg_last) tc_commit(&z1_full[zb]);
          if (seg_last && ++zb == 2) { zb = 0; zph ^= 1u; }
        } else {
          const uint32_t z2 = tmem + (uint32_t)(geo.z2col + p.jl * C::ZY);
          const bool fresh2 = ((touched >> p.jl) & 1u) == 0;
          const uint64_t dAt = sdesc(sa, FU_BOX, 1024);   // MN-major: cols j
          const uint64_t dY =
              sdesc(ys0 + (uint32_t)(yb * C::P_BYTES), 16, 1024);
#pragma unroll
          for (int kc = 0; kc < FU_T / 16; ++kc) {
            // 16 rows i of the tile
            const uint64_t pk =
                (uint64_t)(((kc >> 2) * C::P_BOX + (kc & 3) * 32) >> 4);
            const uint64_t tk = (uint64_t)((kc * 16 * 128) >> 4);
#pragma unroll
            for (int t = 0; t < C::NTERM; ++t) {
              const uint64_t a = dAt + (uint64_t)((t * C::LO_OFF) >> 4) + tk;
              tc_mma(z2, a, dY + pk, ID_T,
                     (fresh2 && kc == 0 && t == 0) ? 0u : 1u);
              if (t == 0)
                tc_mma(z2, a, dY + pk + (uint64_t)(C::P_LO >> 4), ID_T, 1u);
            }
          }
          touched |= 1u << p.jl;
          tc_commit(&empty_bar[s]);
          if (seg_last) tc_commit(&y_empty[yb]);
          if (run_last) tc_commit(&z2_full);
          if (seg_last && ++yb == YB) { yb = 0; yph ^= 1u; }
          if (run_last) drained ^= p.w >= 32 ? ~0u : (1u << p.w) - 1u;
        }
        any = true;
        if (++s == ST) { s = 0; ph ^= 1u; }
      }
      if (any) {   // own MMAs complete before tensor memory is freed
        uint64_t* db = &drain_bar[is_x ? 0 : 1];
        tc_commit(db);
        const uint64_t t0 = globaltimer_ns();
        while (!mbar_try(db, 0) && globaltimer_ns() - t0 < 2000000000ull) {
        }
      }
    }
  } else if (F32 && warp >= 8) {
    // ---------------- FP32 tile -> bf16 A_hi | A_lo, in place ----------------
    // Thread t: tile row i = t % 128 and quarter qq = t / 128: bf16 box
    // cb = qq / 2, its columns 32 hh .. 32 hh + 31 (hh = qq % 2) = FP32 box
    // fb = 2 cb + hh.  A_hi box cb takes the bytes of FP32 box cb, A_lo box
    // cb those of FP32 box 2 + cb, so all 512 threads read their values
    // before any of them writes.
    const int t = threadIdx.x - 256;
    const int i = t & 127, qq = t >> 7, cb = qq >> 1, hh = qq & 1;
    const int sw = i & 7;
    int s = 0;
    uint32_t ph = 0;
    for (int64_t u = u0; u < u1; ++u) {
      const bool ok = mbar_wait(&full_bar[s], ph, &abort_s, status);
      if (!named_and(2, 32 * C::NCONV, ok)) break;
      unsigned char* sa = smem + (size_t)s * C::STAGE;
      const unsigned char* row = sa + (2 * cb + hh) * FU_BOX + i * 128;
      float4 v[8];
#pragma unroll
      for (int qa = 0; qa < 8; ++qa)
        v[qa] = *reinterpret_cast<const float4*>(row + ((qa ^ sw) << 4));
      named_sync(2, 32 * C::NCONV);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint4 hi, lo;
        fu_split8(v[2 * k], v[2 * k + 1], hi, lo);
        const int q8 = 4 * hh + k;    // 8-column chunk of the bf16 box
        const int off = cb * FU_BOX + i * 128 + ((q8 ^ sw) << 4);
        *reinterpret_cast<uint4*>(sa + off) = hi;
        *reinterpret_cast<uint4*>(sa + C::LO_OFF + off) = lo;
      }
      // generic-proxy writes become visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv_bar[s]);
      if (++s == ST) { s = 0; ph ^= 1u; }
    }
  } else if (warp >= 4 && warp < 8) {
    // ---------------- epilogue: accumulators -> partial slots ----------------
    // A row segment's A X accumulator goes to its piece slot (segment + c);
    // at the end of a run, the run's A^T Y accumulator of every column of
    // the group goes to slot (group + c) Tj + column -- zeros for a column
    // this CTA did not reach in the run, so every slot that k_fu_reduce
    // reads has been written.  A slot is stored column by column (element
    // (r, j) at j 128 + r), so a warp's store of one column is one 128-byte
    // line.
    pdl_wait();   // the partial slots were read by the kernels before
    const int q = warp - 4;                 // tensor-memory lane quarter
    const int row = 32 * q + lane;          // row of the accumulators
    const uint32_t tl = (uint32_t)(32 * q) << 16;
    int zb = 0;
    uint32_t zph = 0, z2ph = 0;
    uint32_t touched = 0;
    FuPos p;
    fu_decode(geo, u0, p);
    for (int64_t u = u0; u < u1; ++u, fu_next(geo, p)) {
      const bool seg_last = (u == u1 - 1) || p.jl == p.w - 1;
      const bool run_first = (u == u0) || (p.i == 0 && p.jl == 0);
      const bool run_last =
          (u == u1 - 1) || (p.i == geo.TI - 1 && p.jl == p.w - 1);
      if (run_first) touched = 0;
      touched |= 1u << p.jl;
      if (hx && seg_last) {
        if (!named_and(1, 128, mbar_wait(&z1_full[zb], zph, &abort_s, status)))
          break;
        tc_fence_after();
        const int64_t seg = (int64_t)p.g * geo.TI + p.i;
        float* dst = out.P1 + (size_t)(seg + c) * FU_T * KP + row;
        const uint32_t zt = tmem + tl + (uint32_t)(zb * C::ZX);
#pragma unroll 1
        for (int c0 = 0; c0 < KP; c0 += 16) {
          float v[16], lo[16];
          tc_ld16(zt + c0, v);
          tc_ld16(zt + KP + c0, lo);
#pragma unroll
          for (int t = 0; t < 16; ++t)
            dst[(size_t)(c0 + t) * FU_T] = v[t] + lo[t];
        }
        tc_fence_before();
        mbar_arrive(&z1_empty[zb]);
        if (++zb == 2) { zb = 0; zph ^= 1u; }
      }
      if (hy && run_last) {
        if (!named_and(1, 128, mbar_wait(&z2_full, z2ph, &abort_s, status)))
          break;
        z2ph ^= 1u;
        tc_fence_after();
#pragma unroll 1
        for (int jl = 0; jl < p.w; ++jl) {
          float* dst =
              out.P2 + ((size_t)(p.g + c) * geo.Tj + jl) * FU_T * KP + row;
          const bool t_on = (touched >> jl) & 1u;
          const uint32_t zt = tmem + tl + (uint32_t)(geo.z2col + jl * C::ZY);
#pragma unroll 1
          for (int c0 = 0; c0 < KP; c0 += 16) {
            float v[16];
            if (t_on) {
              tc_ld16(zt + c0, v);
            } else {
#pragma unroll
              for (int t = 0; t < 16; ++t) v[t] = 0.0f;
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) dst[(size_t)(c0 + t) * FU_T] = v[t];
          }
          tc_fence_before();
          mbar_arrive(&z2_empty[jl]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                     tmem),
                 "r"(512)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Sum of the partial slots, in a fixed order.  With A X formed, tiles
// 0 .. TI - 1 are the 128-row tiles of Zm = A X: for each group in order,
// the pieces of the row's segment in CTA order.  With A^T Y formed, the
// next TJ tiles are the 128-row tiles of Zn = A^T Y: the runs of the
// column's group in CTA order.  Each output tile is split over KP / 8
// blocks of 256 threads, one float4 of the tile per thread; warp 0 lists
// the slots in shared memory first (one group per lane, then a prefix
// sum); each thread then adds its float4 of every slot, eight loads in
// flight, in slot order.
// ---------------------------------------------------------------------------
constexpr int FU_RED_MAX = 2048;
constexpr int FU_RED_NT = 256;

template <int KP>
__global__ void __launch_bounds__(FU_RED_NT)
    k_fu_reduce(const FuGeom geo, const FuOut out) {
  constexpr int RQ = FU_T * KP / 4 / FU_RED_NT;   // blocks per tile: 4 / 2
  static_assert(RQ * FU_RED_NT * 4 == FU_T * KP, "one float4 per thread");
  __shared__ int64_t off[FU_RED_MAX];
  __shared__ int ns_s;
  pdl_wait();   // the fused pass's partial slots
  const int tile = (int)blockIdx.x / RQ, part = (int)blockIdx.x % RQ;
  const int nrow_blocks = geo.has_x ? geo.TI : 0;
  const bool rows = tile < nrow_blocks;
  const int t = rows ? tile : tile - nrow_blocks;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int ns = 0;
    if (rows) {
      // row tile t: one segment per group, split over its owners
      int base = 0;
      for (int g0 = 0; g0 < geo.NG; g0 += 32) {
        const int g = g0 + lane;
        int ca = 0, cnt = 0;
        int64_t first = 0;
        if (g < geo.NG) {
          const int w = fu_w(geo, g);
          const int64_t ua = fu_gs(geo, g) + (int64_t)t * w;
          ca = fu_owner(geo, ua);
          cnt = fu_owner(geo, ua + w - 1) - ca + 1;
          first = ((int64_t)g * geo.TI + t + ca) * FU_T * KP;
        }
        int incl = cnt;
#pragma unroll
        for (int dlt = 1; dlt < 32; dlt <<= 1) {
          const int v = __shfl_up_sync(~0u, incl, dlt);
          if (lane >= dlt) incl += v;
        }
        const int pos = base + incl - cnt;
        for (int k = 0; k < cnt; ++k)
          if (pos + k < FU_RED_MAX)
            off[pos + k] = first + (int64_t)k * FU_T * KP;
        base += __shfl_sync(~0u, incl, 31);
      }
      ns = base;
    } else {
      // column tile t of group g: the runs of the group's CTAs
      const int g = t / geo.Tj, jl = t % geo.Tj;
      const int64_t gs = fu_gs(geo, g);
      const int64_t ge = gs + (int64_t)geo.TI * fu_w(geo, g) - 1;
      const int ca = fu_owner(geo, gs);
      const int cnt = fu_owner(geo, ge) - ca + 1;
      for (int k = lane; k < cnt && k < FU_RED_MAX; k += 32)
        off[k] = (((int64_t)g + ca + k) * geo.Tj + jl) * FU_T * KP;
      ns = cnt;
    }
    if (lane == 0) ns_s = ns;
  }
  __syncthreads();
  const int ns = ns_s;
  if (ns > FU_RED_MAX) {   // more slots than the list holds: cannot happen
    if (threadIdx.x == 0) set_status(out.status, CNMF_E_WORKSPACE);
    return;
  }
  const float* P = rows ? out.P1 : out.P2;
  float* Z = rows ? out.Zm : out.Zn;
  const int64_t ldz = rows ? out.ldzm : out.ldzn;
  const int64_t P_rows = rows ? out.m : out.n;
  const int f = part * FU_RED_NT + (int)threadIdx.x;   // float4 of the tile
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  constexpr int B = 8;
  int k = 0;
  for (; k + B <= ns; k += B) {
    float4 v[B];
#pragma unroll
    for (int a = 0; a < B; ++a)
      v[a] = __ldcg(reinterpret_cast<const float4*>(P + off[k + a]) + f);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      acc.x += v[a].x; acc.y += v[a].y; acc.z += v[a].z; acc.w += v[a].w;
    }
  }
  for (; k < ns; ++k) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(P + off[k]) + f);
    acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
  }
  // slots are column-major: float4 f holds rows 4f % 128 .. + 3 of column
  // 4f / 128
  const int col = (4 * f) / FU_T, r0 = (4 * f) % FU_T;
  if (col >= out.kz) return;
  const float vv[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t prow = (int64_t)t * FU_T + r0 + q;
    if (prow < P_rows) Z[prow * ldz + col] = vv[q];
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct FuPlan {
  bool ok = false;
  bool f32 = false;
  int KP = 0;
  FuGeom geo{};
  int64_t spn = 0, spm = 0;
  size_t p1_slots = 0, p2_slots = 0;
  size_t bytes = 0;
};

// CNMF_UNFUSED_SKETCH selects one read of A per product (the product
// kernels); CNMF_NO_TENSOR_CORES the CUDA-core kernel, so it turns the
// fused (tensor-core) pass off as well.
static bool fu_disabled() {
  static int v = -1;
  if (v < 0)
    v = (getenv("CNMF_UNFUSED_SKETCH") != nullptr ||
         getenv("CNMF_NO_TENSOR_CORES") != nullptr)
            ? 1
            : 0;
  return v == 1;
}

static FuPlan fu_plan(int64_t m, int64_t n, int k, cnmf_dtype a_type,
                      bool has_x, bool has_y) {
  FuPlan pl;
  if (a_type != CNMF_F32 && a_type != CNMF_BF16) return pl;
  if (k < 1 || k > 32 || m < 1 || n < 1 || (!has_x && !has_y)) return pl;
  if (m >= (1ll << 31) || n >= (1ll << 31)) return pl;
  pl.f32 = a_type == CNMF_F32;
  pl.KP = k <= 16 ? 16 : 32;
  const int ZX = 2 * pl.KP, ZY = pl.KP;   // FuCfg::ZX, FuCfg::ZY
  FuGeom& q = pl.geo;
  q.has_x = has_x ? 1 : 0;
  q.has_y = has_y ? 1 : 0;
  q.TI = (int)ceil_div(m, FU_T);
  q.TJ = (int)ceil_div(n, FU_T);
  q.U = (int64_t)q.TI * q.TJ;
  q.z2col = has_x ? 2 * ZX : 0;
  // A^T Y accumulators: as many as tensor memory holds (at most 16, the
  // width of the epilogue's bit mask).  Without A^T Y the groups only bound
  // the length of an A X accumulation: FP32 accumulation on the tensor
  // cores truncates, so its bias grows with the number of accumulating
  // MMAs (about 2^-25 of the sum each); 8 tiles keep it near 1e-5 at most,
  // and the segments are then added in round-to-nearest FP32
  q.Tj = std::min({has_y ? (512 - q.z2col) / ZY : 8, 16, q.TJ});
  q.NG = (int)ceil_div(q.TJ, q.Tj);
  q.wlast = q.TJ - (q.NG - 1) * q.Tj;
  q.G = (int)std::min<int64_t>(q.U, num_sms());
  pl.spn = (n + 7) / 8 * 8;
  pl.spm = (m + 7) / 8 * 8;
  const int64_t nseg = (int64_t)q.TI * q.NG;
  pl.p1_slots = has_x ? (size_t)(nseg + q.G) : 0;
  pl.p2_slots = has_y ? (size_t)(q.NG + q.G) * q.Tj : 0;
  // the reduce kernel lists at most FU_RED_MAX slots per output tile
  if (q.NG + q.G > FU_RED_MAX) return pl;
  Carve cv(nullptr, SIZE_MAX);
  cv.take<bf16>((size_t)2 * pl.KP * pl.spn);
  cv.take<bf16>((size_t)2 * pl.KP * pl.spm);
  cv.take<float>(pl.p1_slots * FU_T * pl.KP);
  cv.take<float>(pl.p2_slots * FU_T * pl.KP);
  pl.bytes = cv.off + 256;
  pl.ok = true;
  return pl;
}

// Large enough for the two-sided pass and for either one-sided product (A^T Y
// alone keeps more accumulators in tensor memory, hence more slots).
size_t fused_workspace(int64_t m, int64_t n, int k, cnmf_dtype a_type) {
  size_t b = 0;
  for (int sides = 1; sides <= 3; ++sides) {
    const FuPlan pl = fu_plan(m, n, k, a_type, sides & 1, sides & 2);
    if (pl.ok) b = std::max(b, pl.bytes);
  }
  return b;
}

bool fused_applicable(const void* A, cnmf_dtype a_type, int64_t m, int64_t n,
                      int64_t lda, int k, bool has_x, bool has_y) {
  if (fu_disabled()) return false;
  if (!fu_plan(m, n, k, a_type, has_x, has_y).ok) return false;
  const int64_t es = a_type == CNMF_F32 ? 4 : 2;
  if ((uintptr_t)A % 16 != 0 || (lda * es) % 16 != 0) return false;
  return tmap_encoder() != nullptr;
}

template <int KP, bool F32>
static cnmf_status run_fused(const FusedArgs& a, const FuPlan& pl, void* ws,
                             cudaStream_t s) {
  typedef FuCfg<KP, F32> C;
  if (!ensure_max_smem((const void*)k_fused_pass<KP, F32>, C::SMEM))
    return CNMF_E_INVALID_ARG;
  const FuGeom& q = pl.geo;
  Carve cv(ws, SIZE_MAX);
  bf16* Xp = cv.take<bf16>((size_t)2 * KP * pl.spn);
  bf16* Yp = cv.take<bf16>((size_t)2 * KP * pl.spm);
  float* P1 = cv.take<float>(pl.p1_slots * FU_T * KP);
  float* P2 = cv.take<float>(pl.p2_slots * FU_T * KP);
  // pack the panels
  dim3 pg((unsigned)ceil_div(std::max(pl.spn, pl.spm), 32),
          (unsigned)ceil_div(KP, 32), 2);
  launch_pdl(k_fu_pack, pg, dim3(256), 0, s,
             q.has_x ? (const float*)a.X : nullptr, a.ldx, a.n,
             q.has_y ? (const float*)a.Y : nullptr, a.ldy, a.m, a.k, KP, Xp,
             pl.spn, Yp, pl.spm);
  CNMF_CHECK_LAUNCH();
  CUtensorMap ta, tx, ty;
  bool ok = make_map(&ta, a.A, F32, (uint64_t)a.n, (uint64_t)a.m,
                     (uint64_t)a.lda * C::ESZ, C::BOXW, FU_T);
  ok = ok && make_map(&tx, Xp, false, (uint64_t)pl.spn, (uint64_t)(2 * KP),
                      (uint64_t)pl.spn * 2, 64, 2 * KP);
  ok = ok && make_map(&ty, Yp, false, (uint64_t)pl.spm, (uint64_t)(2 * KP),
                      (uint64_t)pl.spm * 2, 64, 2 * KP);
  if (!ok) return CNMF_E_INVALID_ARG;
  FuOut o{(float*)a.Zm, a.ldzm, (float*)a.Zn, a.ldzn, a.k, a.m, a.n,
          P1, P2, a.status};
  launch_pdl(k_fused_pass<KP, F32>, dim3((unsigned)q.G), dim3(C::NT), C::SMEM,
             s, ta, tx, ty, q, o);
  CNMF_CHECK_LAUNCH();
  const int nred = ((q.has_x ? q.TI : 0) + (q.has_y ? q.TJ : 0)) * (KP / 8);
  launch_pdl(k_fu_reduce<KP>, dim3((unsigned)nred), dim3(FU_RED_NT), 0, s, q,
             o);
  CNMF_CHECK_LAUNCH();
  return CNMF_OK;
}

cnmf_status launch_fused(const FusedArgs& a, void* ws, size_t ws_bytes,
                         cudaStream_t s) {
  const FuPlan pl = fu_plan(a.m, a.n, a.k, a.a_type, a.X != nullptr,
                            a.Y != nullptr);
  if (!pl.ok) return CNMF_E_INVALID_ARG;
  if (ws_bytes < pl.bytes) return CNMF_E_WORKSPACE;
  if (pl.f32)
    return pl.KP == 16 ? run_fused<16, true>(a, pl, ws, s)
                       : run_fused<32, true>(a, pl, ws, s);
  return pl.KP == 16 ? run_fused<16, false>(a, pl, ws, s)
                     : run_fused<32, false>(a, pl, ws, s);
}

}  // namespace cnmf

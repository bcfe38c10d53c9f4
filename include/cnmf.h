/*
 * cnmf.h -- C ABI of the GB300 compressed-NMF / compressed-SNMF library.
 *
 * Method: Tepper & Sapiro, "Compressed Nonnegative Matrix Factorization is
 * Fast and Accurate".  The library implements the data-parallel hot path:
 *   - structured random compression (Alg. 1, Sec. II) applied to A and A^T
 *     (Sec. III), giving L (m x d) and R (d x n);
 *   - the compressed ADMM NMF iteration (Alg. 4, App. B) and, as a baseline,
 *     the same iteration with L = I, R = I (uncompressed ADMM, Sec. III);
 *   - compressed separable NMF column selection (Alg. 3, steps 1-2) with the
 *     successive projection algorithm on Q^T A (Sec. IV);
 *   - the relative reconstruction error used in Sec. V.
 *
 * Conventions (all entry points):
 *   - Matrices are row-major.  A is m x n with row pitch lda >= n elements.
 *     Tall panels are stored with the long dimension first: L is m x d,
 *     R is stored transposed as Rt = R^T (n x d), V as Vt = V^T (n x r),
 *     Phi as Phit = Phi^T (n x r), Rhat as Rhat_t = (Q^T A)^T (n x d).
 *   - Every pointer is a DEVICE pointer owned by the caller, unless stated.
 *     The library never allocates device memory; scratch space is the
 *     caller's workspace `ws`, whose size comes from the matching
 *     *_workspace() query (256-byte aligned pointer).  Its only state:
 *     per-device caches filled on first use (SM count, opt-in shared
 *     memory, kernel shared-memory limits raised once per device, the
 *     driver's tensor-map encoder, the device address of
 *     cnmf_residual_noalloc's static scratch), each guarded for
 *     concurrent first calls; the calling host thread's CTA limit
 *     (cnmf_set_thread_cta_limit); and the text of that thread's last
 *     CUDA error (cnmf_last_error).
 *   - All work is enqueued asynchronously on `stream` (a cudaStream_t).
 *   - Host-detected errors (bad sizes, NULL pointers, small workspace,
 *     launch failures) are returned immediately with NOTHING enqueued,
 *     except CNMF_E_CUDA from a failed launch after earlier launches.
 *   - Device-detected errors are written to *dev_status (device int32 that
 *     the caller zeroes; the first error wins): CNMF_E_CHOLESKY (a Gram
 *     matrix that is not numerically positive definite), CNMF_E_NONFINITE
 *     (NaN/Inf met in a panel or factor), CNMF_E_TIMEOUT (a bounded grid
 *     barrier wait expired; the kernel returns instead of hanging).
 *     The caller reads *dev_status after synchronising the stream.  The
 *     error code is (*dev_status & CNMF_STATUS_CODE_MASK); the high bits
 *     are flags that are not errors (CNMF_STATUS_NEGATIVE_A, set by
 *     cnmf_check_nonnegative), kept beside the error code.
 *   - Working precision W: FP64 when the input type is CNMF_F64, else FP32.
 *     Outputs and test matrices are in W.  A stored as CNMF_BF16 is widened
 *     to FP32 on load.
 *   - Same inputs and seed give bitwise-identical outputs (all reductions
 *     run in a fixed order; no floating-point atomics).
 */
#ifndef CNMF_H
#define CNMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cnmf_stream_t; /* == cudaStream_t */

typedef enum {
  CNMF_OK = 0,
  CNMF_E_INVALID_ARG = 1,
  CNMF_E_WORKSPACE = 2,
  CNMF_E_CUDA = 3,
  CNMF_E_CHOLESKY = 4,
  CNMF_E_NONFINITE = 5,
  CNMF_E_TIMEOUT = 6
} cnmf_status;

/* Bits of *dev_status: the error code (a cnmf_status) in the low bits, and
 * flags that are not errors in the high bits. */
#define CNMF_STATUS_CODE_MASK 0x0000FFFF
#define CNMF_STATUS_NEGATIVE_A 0x40000000 /* A holds an entry below zero */

/* Storage type of A (and, for CNMF_F64 / CNMF_F32, of W-typed buffers). */
typedef enum { CNMF_F64 = 0, CNMF_F32 = 1, CNMF_BF16 = 2 } cnmf_dtype;

/* Penalties lambda, phi and step xi of Alg. 4 (App. B); iters sweeps.
 * The paper sets xi = 1 and leaves lambda, phi unspecified. */
typedef struct {
  double lambda;
  double phi;
  double xi;
  int32_t iters;
  int32_t barrier_timeout_ms; /* 0 -> default (2000 ms) */
  /* Optional device array of phase_ns_len >= 5 doubles (NULL: off).
   * cnmf_factor adds the nanoseconds one CTA spends per phase, summed over
   * the sweeps (CTA 0, or with the register-tiled path's U/V split the
   * first V-side CTA): [0] small r x r algebra, [1] row sweep, [2] first
   * grid barrier, [3] cross-CTA reduction, [4] second grid barrier (the
   * register-tiled path has no grid barrier in its sweeps: [2] is its
   * cross-CTA reduction including the waits for the other CTAs' shares,
   * [3] and [4] stay zero); with
   * phase_ns_len >= 15 on the register-tiled path also the sub-steps:
   * [5] staging of the reduced shares, [6] Xt Grams, [7] Xt solve, [8] Yt
   * Grams, [9] Yt solve, [10] publishing Yt, [11] U-row updates, [12]
   * U-side lane sums, [13] V-row updates, [14] V-side lane sums; with
   * phase_ns_len >= 20 and the U/V split, [15..19] the phases [0..4] of
   * U-side CTA 0; with phase_ns_len >= 20 + 3 G (G CTAs) on that path,
   * [20 + 3c], [21 + 3c], [22 + 3c] the time CTA c spends in the small
   * algebra, the row sweep and the reduction with its waits.  Ignored by cnmf_factor_plain. */
  double* phase_ns;
  int32_t phase_ns_len;
  int32_t reserved;
} cnmf_admm_params;

/* Human-readable name of a status code (static string, never NULL). */
const char* cnmf_status_string(int32_t status);

/* Detail of the CUDA error behind the calling thread's last CNMF_E_CUDA
 * (error name, message, source location); "" if none.  Static per-thread
 * buffer owned by the library. */
const char* cnmf_last_error(void);

/* ABI version of this header (bumped on incompatible change). */
int32_t cnmf_abi_version(void);

/* ------------------------------------------------------------------------
 * Gaussian test matrices (Alg. 1, first step: Omega with i.i.d. N(0,1)).
 * Counter-based: Philox4x32-10 (Salmon et al., SC'11) + Box-Muller.
 * key = (seed mod 2^32, seed >> 32); counter = (b mod 2^32, b >> 32,
 * stream_id, 0) for block b = e / 4 of row-major element e; uniforms
 * u = (x + 0.5) 2^-32; (z0, z1) from words (0, 1), (z2, z3) from (2, 3);
 * element e takes z_{e mod 4}.  Box-Muller is evaluated in FP64.
 * ---------------------------------------------------------------------- */

/* out: rows x cols (row-major) in out_type (CNMF_F64 or CNMF_F32). */
cnmf_status cnmf_gaussian(uint64_t seed, uint32_t stream_id, int64_t rows,
                          int64_t cols, cnmf_dtype out_type, void* out,
                          cnmf_stream_t stream);

/* out: nblocks x 4 uint32 raw Philox words of blocks first_block.. . */
cnmf_status cnmf_philox_words(uint64_t seed, uint32_t stream_id,
                              int64_t first_block, int64_t nblocks,
                              uint32_t* out, cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * Building blocks of the compression (exposed for step-level checks).
 * ---------------------------------------------------------------------- */

/* One two-sided product pass over A (Alg. 1 power scheme, Sec. III):
 *   Zm = A X   (m x k, from X n x k)     and/or
 *   Zn = A^T Y (n x k, from Y m x k).
 * X, Y, Zm, Zn are W-typed with row pitch k.  Pass X = NULL / Zm = NULL
 * (or Y = NULL / Zn = NULL) to skip one side.  1 <= k <= 128.
 *   FP64 A (and A whose base or row pitch is not 16-byte aligned): CUDA-core
 *   FMA, one read of A per product, exact products rounded in W.
 *   FP32 / BF16 A: tensor cores (tcgen05, FP32 accumulation).  For k <= 32
 *   both products come from ONE read of A (fused pass): each 128 x 128
 *   tile feeds A X (tile K-major) and A^T Y (the same bytes MN-major); FP32
 *   A is split in shared memory into bf16 hi + lo parts (|A - hi - lo| <=
 *   2^-18 |A|).  For k > 32 each product reads A once (FP32 A as 3xTF32).
 *   X / Y are split into bf16 (3xTF32: TF32) hi + lo parts.  The products
 *   carry an extra relative error of at most 2^-17 (BF16 A) or 2^-16 (FP32
 *   A: the split of A and the dropped A_lo Y_lo term) of |A||X| besides
 *   FP32 accumulation.  Environment: CNMF_UNFUSED_SKETCH selects one read per
 *   product for k <= 32 too; CNMF_NO_TENSOR_CORES selects the CUDA-core
 *   kernel.
 * Results do not depend on timing (partial sums are added in a fixed
 * order).  dev_status (optional): CNMF_E_TIMEOUT if a bounded pipeline
 * wait expired. */
size_t cnmf_sketch_workspace(int64_t m, int64_t n, int32_t k,
                             cnmf_dtype a_type);
cnmf_status cnmf_sketch_pass(const void* A, cnmf_dtype a_type, int64_t m,
                             int64_t n, int64_t lda, int32_t k, const void* X,
                             const void* Y, void* Zm, void* Zn, void* ws,
                             size_t ws_bytes, int32_t* dev_status,
                             cnmf_stream_t stream);

/* Orthonormal basis (Alg. 1, last step: "QR decomposition") of a tall
 * panel Y (rows x k, W-typed, row pitch k, rows >= k), in place:
 * CholeskyQR2 with FP64-accurate Gram matrices (double-float accumulation
 * on FP32 data) and a small diagonal shift in the first sweep.  The result
 * equals the thin Q of Y with diag(R) > 0 (unique for full column rank). */
size_t cnmf_orth_workspace(int64_t rows, int32_t k, cnmf_dtype w_type);
cnmf_status cnmf_orth(void* Y, cnmf_dtype w_type, int64_t rows, int32_t k,
                      void* ws, size_t ws_bytes, int32_t* dev_status,
                      cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_compress: two-sided structured random compression (Alg. 1 on A and
 * A^T, Sec. III) with q power iterations and re-orthonormalisation after
 * every product, then A-tilde = L^T A R^T (Alg. 4 setup).
 *   A       m x n, a_type, pitch lda (>= n).  NMF expects A >= 0 (Sec. I);
 *           negative entries are not rejected (cnmf_check_nonnegative
 *           reports them).
 *   r, d    target rank and sketch size d = r + r_ov, 1 <= r <= d <=
 *           min(m, n), d <= 128.
 *   q       power iterations (Alg. 1 exponent w), 0 <= q <= 64.  The
 *           compression reads A 2q + 2 times when d <= 32 and A is FP32 or
 *           BF16 (2q + 1 fused passes and A-check), else 4q + 3 times.
 *   seed    Philox seed for Omega (stream 0, n x d, left chain) and Psi
 *           (stream 1, m x d, right chain), used when Omega/Psi are NULL.
 *   Omega, Psi  optional caller test matrices (W-typed, n x d and m x d).
 *   L       out, m x d, orthonormal columns.
 *   Rt      out, n x d, R^T (R has orthonormal rows).
 *   Atilde  out, d x d.
 * ---------------------------------------------------------------------- */
size_t cnmf_compress_workspace(int64_t m, int64_t n, int32_t d,
                               cnmf_dtype a_type);
cnmf_status cnmf_compress(const void* A, cnmf_dtype a_type, int64_t m,
                          int64_t n, int64_t lda, int32_t r, int32_t d,
                          int32_t q, uint64_t seed, const void* Omega,
                          const void* Psi, void* L, void* Rt, void* Atilde,
                          void* ws, size_t ws_bytes, int32_t* dev_status,
                          cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_compress_host: cnmf_compress for an A that does not stay in device
 * memory -- the paper's out-of-core setting (Sec. II, big-data solutions;
 * App. A): A in host memory is streamed through the GPU once per pass.
 *   A           m x n, pitch lda, in memory the copy engine reads (host
 *               memory: page-locked for the full copy rate, pageable works
 *               slower; a device pointer works too).  It must stay valid
 *               and unchanged until the stream has finished the call.
 *   block_rows  rows per block (>= 1): each block is copied into one of
 *               two device buffers of block_rows x n and goes through the
 *               same product kernels as cnmf_compress (the fused one-read
 *               pass for FP32 / BF16 and d <= 32); the blocks' shares of
 *               A^T Y are added in block order.  The copies run on a copy
 *               stream of the library's own (one non-blocking stream and
 *               five events per host thread and device, created on the
 *               thread's first call on that device and kept until exit),
 *               so the copy of block k + 1 overlaps block k's products;
 *               events order the two streams, and the call still returns
 *               with all its work ordered on `stream`.
 *   Everything else as cnmf_compress: the m x d and n x d panels, their
 *   CholeskyQR2 (whose Gram matrices are the sums over row blocks -- the
 *   one central reduction TSQR provides in the paper) and A-tilde stay in
 *   device memory, of which the call needs the workspace below plus L, Rt,
 *   Atilde (O((m + n) d) and block_rows x n, not m x n).  A is read from
 *   host memory 2q + 2 times (d <= 32, FP32/BF16) or 4q + 3 times.
 *   Results equal cnmf_compress's up to the order of FP32 additions.
 * ---------------------------------------------------------------------- */
size_t cnmf_compress_host_workspace(int64_t m, int64_t n, int32_t d,
                                    cnmf_dtype a_type, int64_t block_rows);
cnmf_status cnmf_compress_host(const void* A, cnmf_dtype a_type, int64_t m,
                               int64_t n, int64_t lda, int32_t r, int32_t d,
                               int32_t q, uint64_t seed, const void* Omega,
                               const void* Psi, void* L, void* Rt,
                               void* Atilde, int64_t block_rows, void* ws,
                               size_t ws_bytes, int32_t* dev_status,
                               cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_compress_gaussian: the Gaussian-compression baseline the paper
 * compares against (Sec. II, note on data-agnostic compression: Q =
 * s^-1/2 Omega), applied on both sides with s = d and no power iteration or
 * orthonormalisation:
 *   L = d^-1/2 Psi (m x d, Philox stream 1),  R^T = d^-1/2 Omega (n x d,
 *   stream 0) -- the test matrices cnmf_compress draws for the same seed --
 *   then A-tilde = L^T A R^T (d x d) as in cnmf_compress.
 * Arguments as cnmf_compress (same workspace query), without r, q, Omega
 * and Psi; L and Rt are dense (pitch d), in the working type.
 * ---------------------------------------------------------------------- */
cnmf_status cnmf_compress_gaussian(const void* A, cnmf_dtype a_type,
                                   int64_t m, int64_t n, int64_t lda,
                                   int32_t d, uint64_t seed, void* L,
                                   void* Rt, void* Atilde, void* ws,
                                   size_t ws_bytes, int32_t* dev_status,
                                   cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_factor: `p->iters` sweeps of compressed ADMM (Alg. 4, App. B):
 *   Xt <- (Atilde Yt^T + lam L^T U - L^T Lam)(Yt Yt^T + lam I)^-1
 *   Yt <- (Xt^T Xt + phi I)^-1 (Xt^T Atilde + phi V R^T - Phi R^T)
 *   U  <- P+(L Xt + Lam/lam),  V <- P+(Yt R + Phi/phi)
 *   Lam <- Lam + xi lam (L Xt - U),  Phi <- Phi + xi phi (Yt R - V)
 * One persistent cooperative launch; grid barriers are bounded.
 *   L (m x d), Rt (n x d), Atilde (d x d): from cnmf_compress (W-typed).
 *   U   in/out m x r.  On a fresh start (resume = 0): the initial U.
 *   Vt  in/out n x r (V^T).  On a fresh start: the initial V^T.
 *   state  in/out, cnmf_factor_state_bytes() bytes, W-typed sections in
 *          this order: Lam (m x r), Phit (n x r), Yt (r x d), Xt (d x r),
 *          then int64 k (sweeps done so far) at the next 8-byte boundary,
 *          then Zx, Zy (r x r each): -(Yt Yt^T + lam I)^-1 and
 *          -(Xt^T Xt + phi I)^-1 of the last sweep, from which the next
 *          sweep's inverses are refined (valid when k > 0).
 *          resume = 0: Yt <- V R^T, Lam = Phi = 0, k = 0 (Alg. 4 setup).
 *          resume = 1: continue from the state; the result is bitwise the
 *          same as an uninterrupted run.
 *   1 <= r <= d <= 128, r <= 64, lambda, phi > 0; the per-CTA working set
 *   of about d^2 + 5 d r + r^2 + 64 (d + r) values of W must fit in shared
 *   memory (FP32: d = 128 with r <= 32, d = 80 with r = 64; FP64: d = 64
 *   with r = 32); sizes beyond it return CNMF_E_INVALID_ARG.
 * ---------------------------------------------------------------------- */
size_t cnmf_factor_workspace(int64_t m, int64_t n, int32_t r, int32_t d,
                             cnmf_dtype w_type);
size_t cnmf_factor_state_bytes(int64_t m, int64_t n, int32_t r, int32_t d,
                               cnmf_dtype w_type);
cnmf_status cnmf_factor(const void* L, const void* Rt, const void* Atilde,
                        cnmf_dtype w_type, int64_t m, int64_t n, int32_t r,
                        int32_t d, const cnmf_admm_params* p, void* U,
                        void* Vt, void* state, int32_t resume, void* ws,
                        size_t ws_bytes, int32_t* dev_status,
                        cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_factor_batched: `sweeps` compressed ADMM sweeps (Alg. 4, FP32) for
 * each of `nitems` independent problems in ONE launch.  Each problem runs
 * on a cluster of `cluster_size` CTAs (1, 2, 4 or 8) that split its rows
 * and add their shares through distributed shared memory; there are no
 * grid-wide waits, and a problem's result does not depend on the other
 * problems in the launch.  A problem may run its sweeps over several
 * launches; the result is bitwise that of one launch with the total count.
 *   items   DEVICE array of nitems cnmf_batch_item (below); a slot with
 *           L == NULL or r == 0 is skipped.  Each item's buffers are its
 *           own: L (m x d), Rt (n x d), Atilde (d x d) from cnmf_compress;
 *           U (m x r) and Vt (n x r) in/out; state as in cnmf_factor
 *           (cnmf_factor_state_bytes, FP32); scratch of
 *           cnmf_batch_scratch_bytes(r, d) bytes kept between launches.
 *           flags & CNMF_BATCH_FRESH: start from U, V as given (Alg. 4
 *           setup: Yt = V R^T, Lam = Phi = 0); clear it for later launches.
 *           lambda <= 0 selects the balanced scale lambda = phi =
 *           c ||Atilde||_F / r, formed on the device from the item's
 *           Atilde, with c = 1 for lambda = 0 and c = -lambda for
 *           lambda < 0.
 *   max_r, max_d  bounds on the items' r and d (r <= 32, d <= 64, r <= d);
 *           they select the kernel variant and its shared-memory size.
 * The launch reads `items` when it runs, so a CUDA graph that captured it
 * can be replayed after the caller rewrites the device array.
 * ---------------------------------------------------------------------- */
#define CNMF_BATCH_FRESH 1
typedef struct {
  const void* L;
  const void* Rt;
  const void* Atilde;
  void* U;
  void* Vt;
  void* state;
  void* scratch;
  int64_t m, n;
  int32_t r, d;
  double lambda, phi, xi;
  int32_t flags;
  int32_t reserved;
} cnmf_batch_item;

size_t cnmf_batch_scratch_bytes(int32_t r, int32_t d);
cnmf_status cnmf_factor_batched(const cnmf_batch_item* items, int32_t nitems,
                                int32_t sweeps, int32_t cluster_size,
                                int32_t max_r, int32_t max_d,
                                int32_t* dev_status, cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_factor_plain: the uncompressed ADMM NMF baseline -- Alg. 4 with
 * L = I_m, R = I_n, Atilde = A (Sec. III, problem nmfEquiv; Xu et al.).
 * Each sweep reads A twice (A Y^T, then A^T X with the new X).
 *   A, a_type, m, n, lda as in cnmf_compress; W from a_type.
 *   U in/out m x r; Vt in/out n x r.
 *   state  cnmf_plain_state_bytes(): Lam (m x r), Phit (n x r), Yt (n x r,
 *          = Y^T), X (m x r), then int64 k.  resume as in cnmf_factor.
 * ---------------------------------------------------------------------- */
size_t cnmf_plain_workspace(int64_t m, int64_t n, int32_t r,
                            cnmf_dtype a_type);
size_t cnmf_plain_state_bytes(int64_t m, int64_t n, int32_t r,
                              cnmf_dtype a_type);
cnmf_status cnmf_factor_plain(const void* A, cnmf_dtype a_type, int64_t m,
                              int64_t n, int64_t lda, int32_t r,
                              const cnmf_admm_params* p, void* U, void* Vt,
                              void* state, int32_t resume, void* ws,
                              size_t ws_bytes, int32_t* dev_status,
                              cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * snmf_select: compressed separable NMF, Alg. 3 steps 1-2 (Sec. IV).
 *   Q = Alg.1(A) with q power iterations (one-sided, 2q + 1 products,
 *   re-orthonormalised after each), Rhat = Q^T A (d x n), then the
 *   successive projection algorithm on the columns of Rhat: r times pick
 *   j* = argmax_j ||Rhat[:, j]||^2 (ties -> lowest j), u = Rhat[:, j*] /
 *   ||.||, Rhat <- (I - u u^T) Rhat.
 *   Omega  optional n x d W-typed test matrix (else Philox stream 0).
 *   anchors  out, r int64 column indices in selection order.
 *   Rhat_t   optional out, n x d (= Rhat^T) BEFORE the SPA projections.
 *   1 <= r <= d <= min(m, n), d <= 128.
 * ---------------------------------------------------------------------- */
size_t snmf_select_workspace(int64_t m, int64_t n, int32_t d,
                             cnmf_dtype a_type);
cnmf_status snmf_select(const void* A, cnmf_dtype a_type, int64_t m,
                        int64_t n, int64_t lda, int32_t r, int32_t d,
                        int32_t q, uint64_t seed, const void* Omega,
                        int64_t* anchors, void* Rhat_t, void* ws,
                        size_t ws_bytes, int32_t* dev_status,
                        cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * snmf_right_factor: compressed separable NMF, Alg. 3 step 3 (Sec. IV):
 * for every column i of Rhat (d x n),
 *   Y[:, i] = argmin_{h >= 0} || Rhat[:, i] - Rhat[:, K] h ||_2 ,
 * the nonnegative least-squares fit by the r selected columns.  The paper
 * leaves the NNLS solver open; this one is projected cyclic coordinate
 * descent on the shared Gram matrix G = Rhat[:, K]^T Rhat[:, K] (one column
 * per thread), started from the unconstrained minimiser G^-1 b with its
 * negative entries set to zero, run until the projected gradient is at
 * most tol times
 * max_j |(Rhat[:, K]^T Rhat[:, i])_j| or for max_sweeps sweeps; when
 * Rhat[:, K] has full column rank the minimiser is unique and the sweeps
 * converge to it.
 *   Rhat_t   n x d (pitch ld >= d), = Rhat^T as snmf_select writes it;
 *            w_type CNMF_F64 or CNMF_F32 (arithmetic in w_type).
 *   anchors  device, r int64 column indices (snmf_select's); an index
 *            outside [0, n) sets CNMF_E_INVALID_ARG in *dev_status.
 *   Y        out, r x n (pitch ldy >= n), w_type.
 *   unconverged  optional device int32, incremented once per column that
 *            did not reach the tolerance within max_sweeps (the caller
 *            zeroes it).
 *   1 <= r <= min(d, 64), d <= 128, max_sweeps >= 1, tol >= 0.
 * ---------------------------------------------------------------------- */
size_t snmf_right_factor_workspace(int64_t n, int32_t d, int32_t r,
                                   cnmf_dtype w_type);
cnmf_status snmf_right_factor(const void* Rhat_t, cnmf_dtype w_type,
                              int64_t n, int32_t d, int64_t ld,
                              const int64_t* anchors, int32_t r,
                              int32_t max_sweeps, double tol, void* Y,
                              int64_t ldy, int32_t* unconverged, void* ws,
                              size_t ws_bytes, int32_t* dev_status,
                              cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_factor_als: compressed alternating NMF (Alg. 2, Sec. III) with exact
 * nonnegative least-squares steps (the paper admits any NNLS method; this
 * is the solver of snmf_right_factor).  With A-check = A R^T (m x d) and
 * A-hat = L^T A (d x n), `iters` times:
 *   Y-check = Y R^T;  X[i] = argmin_{x >= 0} ||A-check[i] - x Y-check||
 *   X-hat = L^T X;    Y[:, j] = argmin_{y >= 0} ||A-hat[:, j] - X-hat y||
 *   A  m x n (pitch lda) in a_type; L (m x d), Rt (n x d, = R^T) dense, in
 *      the working type (CNMF_F64 for F64 A, else CNMF_F32).
 *   X  out, m x r;  Y  in/out, r x n (the start Y0 on entry), working type.
 *   max_sweeps, tol  the NNLS stopping rule of snmf_right_factor, per step.
 *   unconverged  optional device int32, incremented per row or column that
 *      stopped on max_sweeps (over all steps; the caller zeroes it).
 *   1 <= r <= min(d, 64), d <= min(128, m, n), iters >= 0.
 * ---------------------------------------------------------------------- */
size_t cnmf_factor_als_workspace(int64_t m, int64_t n, int32_t r, int32_t d,
                                 cnmf_dtype a_type);
cnmf_status cnmf_factor_als(const void* A, cnmf_dtype a_type, int64_t m,
                            int64_t n, int64_t lda, const void* L,
                            const void* Rt, int32_t r, int32_t d,
                            int32_t iters, int32_t max_sweeps, double tol,
                            void* X, void* Y, int32_t* unconverged, void* ws,
                            size_t ws_bytes, int32_t* dev_status,
                            cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_factor_mu: compressed alternating NMF (Alg. 2, Sec. III) with the
 * multiplicative updates of Ding, Li & Jordan (2010, Eq. 8) -- the paper's
 * other inner solver -- in their semi-NMF form (A-check and A-hat have
 * entries of both signs).  With B+ = (|B| + B) / 2, B- = (|B| - B) / 2,
 * `iters` times:
 *   Y-check = Y R^T;  P = A-check Y-check^T, Q = Y-check Y-check^T,
 *     X <- X * sqrt((P+ + X Q-) / (P- + X Q+))             (entrywise)
 *   X-hat = L^T X;    P = A-hat^T X-hat, Q = X-hat^T X-hat,
 *     Y^T <- Y^T * sqrt((P+ + Y^T Q-) / (P- + Y^T Q+))
 * a zero denominator floored at 1e-300 (FP64) / 1e-38 (FP32); an entry
 * that is zero stays zero.
 *   A, L, Rt, r, d as in cnmf_factor_als (same workspace query).
 *   X  in/out, m x r (the start X0 on entry);  Y  in/out, r x n.
 *   dev_status: CNMF_E_NONFINITE if an update is not finite.
 * ---------------------------------------------------------------------- */
size_t cnmf_factor_mu_workspace(int64_t m, int64_t n, int32_t r, int32_t d,
                                cnmf_dtype a_type);
cnmf_status cnmf_factor_mu(const void* A, cnmf_dtype a_type, int64_t m,
                           int64_t n, int64_t lda, const void* L,
                           const void* Rt, int32_t r, int32_t d,
                           int32_t iters, void* X, void* Y, void* ws,
                           size_t ws_bytes, int32_t* dev_status,
                           cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_residual: out2[0] = ||A - U V||_F^2, out2[1] = ||A||_F^2 (FP64,
 * device), in one read of A (Sec. V reports sqrt(out2[0] / out2[1])).
 *   U m x r, Vt n x r in w_type (CNMF_F64 or CNMF_F32), 1 <= r <= 128.
 * ---------------------------------------------------------------------- */
size_t cnmf_residual_workspace(int64_t m, int64_t n, int32_t r,
                               cnmf_dtype a_type);
cnmf_status cnmf_residual(const void* A, cnmf_dtype a_type, int64_t m,
                          int64_t n, int64_t lda, const void* U,
                          const void* Vt, cnmf_dtype w_type, int32_t r,
                          double* out2, void* ws, size_t ws_bytes,
                          cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_check_nonnegative: reports whether A holds a negative entry.  NMF and
 * SNMF are posed for a nonnegative matrix (Sec. II, the NMF problem; Sec.
 * IV, separable NMF); the compression itself is defined for any A, so a
 * negative entry is reported, not rejected: the flag bit
 * CNMF_STATUS_NEGATIVE_A is ORed into *dev_status (required, device
 * int32), keeping the error code in its low bits.  An entry is negative
 * when it compares below zero (-0.0 and NaN are not).  Only the n entries
 * of each row are read, not the padding up to lda.  One read of A; the
 * compression entry points do not run it by themselves.
 * ---------------------------------------------------------------------- */
cnmf_status cnmf_check_nonnegative(const void* A, cnmf_dtype a_type,
                                   int64_t m, int64_t n, int64_t lda,
                                   int32_t* dev_status, cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_residual_batched: cnmf_residual for many problems in one launch (the
 * accuracy checks of a served batch).  Item i: out2[2 i] = ||A - U V||_F^2,
 * out2[2 i + 1] = ||A||_F^2 (FP64, device), one read of its A.
 *   items   DEVICE array of nitems cnmf_residual_item (below); all items
 *           share a_type and w_type (as in cnmf_residual); 1 <= r <= max_r
 *           <= 128 per item.  An item that breaks these rules gets NaN
 *           pairs and CNMF_E_INVALID_ARG in *dev_status (optional).
 *   ctas_per_item  CTAs that split each item's 64 x 64 tiles (1..1024);
 *           each item's sums run in CTA order, so results do not depend on
 *           timing (they may differ from cnmf_residual's in the last bits:
 *           another split of the same sums).
 *   ws      cnmf_residual_batched_workspace(nitems, ctas_per_item) bytes.
 * The launch reads `items` when it runs.
 * ---------------------------------------------------------------------- */
typedef struct {
  const void* A;   /* m x n, pitch lda */
  const void* U;   /* m x r */
  const void* Vt;  /* n x r */
  int64_t m, n, lda;
  int32_t r, reserved;
} cnmf_residual_item;
size_t cnmf_residual_batched_workspace(int32_t nitems, int32_t ctas_per_item);
cnmf_status cnmf_residual_batched(const cnmf_residual_item* items,
                                  int32_t nitems, cnmf_dtype a_type,
                                  cnmf_dtype w_type, int32_t max_r,
                                  int32_t ctas_per_item, double* out2,
                                  void* ws, size_t ws_bytes,
                                  int32_t* dev_status, cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_residual_noalloc: the same result as cnmf_residual, for callers that
 * cannot allocate device memory -- for example a plugin whose host
 * application owns every device allocation, code running while another
 * allocator has reserved all of device memory, or a latency-critical loop
 * that must not reach cudaMalloc and its implicit device synchronisation.
 * It takes no workspace and allocates nothing: its scratch (one FP64 pair
 * per CTA, at most 1024 CTAs) is a 16 KiB static device array inside the
 * library, which every GPU that loads the library keeps until exit.
 *   - Arguments as in cnmf_residual, minus ws / ws_bytes.
 *   - The first call on each device (with that device current) looks up the
 *     array's device address once; make that first call before any stream
 *     capture.
 *   - Returns CNMF_E_WORKSPACE if the launch would need more than 1024 CTAs
 *     (more than 256 SMs); nothing is enqueued then.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and must be serialised by
 *     the caller.  Nothing in the array needs to start at zero -- each call
 *     writes every partial it later reads.
 * (Library utility; the paper has no counterpart.)
 * ---------------------------------------------------------------------- */
cnmf_status cnmf_residual_noalloc(const void* A, cnmf_dtype a_type, int64_t m,
                                  int64_t n, int64_t lda, const void* U,
                                  const void* Vt, cnmf_dtype w_type, int32_t r,
                                  double* out2, cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_set_thread_cta_limit: caps the grid of every kernel that is sized
 * per SM (the tensor-core products, CholeskyQR, the cooperative ADMM
 * launch, ...) for the calls this host thread makes from now on: at most
 * `ctas` CTAs, so each such kernel occupies at most `ctas` SMs (one CTA per
 * SM).  0 restores the device's SM count.  Two independent calls on two
 * streams, each capped at half the SMs, then run side by side -- e.g. the
 * compression of one problem beside the latency-bound ADMM sweeps of
 * another.  Workspace queries made under a cap return the capped sizes;
 * a workspace sized without a cap fits every cap.  Results depend on the
 * cap only through the summation order of cross-CTA sums (within the
 * documented tolerances).  A cooperative ADMM launch below about 70 CTAs
 * may no longer keep its rows in shared memory at large m + n (slower, not
 * wrong).  Returns CNMF_E_INVALID_ARG for ctas < 0.
 * (Library utility; the paper has no counterpart.)
 * ---------------------------------------------------------------------- */
cnmf_status cnmf_set_thread_cta_limit(int32_t ctas);

/* ------------------------------------------------------------------------
 * cnmf_barrier_selftest: exercises the bounded grid barrier that the
 * persistent kernels (cnmf_factor) use.  A cooperative grid of `ctas` CTAs
 * (<= SM count) passes `rounds` barriers.  If 0 <= skip < ctas, CTA `skip`
 * leaves before the first barrier, so the others can never complete it:
 * they give up after timeout_ms (1..10000), write CNMF_E_TIMEOUT to
 * *dev_status and return -- nothing hangs.  With skip < 0 every barrier
 * completes and *dev_status stays 0.  *out_rounds (optional device int32)
 * receives the number of barriers CTA 0 passed.  ws: >= 256 bytes.
 * (Library self-test; the paper has no counterpart.)
 * ---------------------------------------------------------------------- */
cnmf_status cnmf_barrier_selftest(int32_t ctas, int32_t rounds, int32_t skip,
                                  int32_t timeout_ms, void* ws,
                                  size_t ws_bytes, int32_t* dev_status,
                                  int32_t* out_rounds, cnmf_stream_t stream);

/* ------------------------------------------------------------------------
 * cnmf_tagwait_selftest: exercises the bounded waits on tagged words (a
 * 32-bit payload and a 32-bit tag in one 64-bit word) through which
 * cnmf_factor's register-tiled sweep loop synchronises instead of grid
 * barriers.  A cooperative grid of `ctas` CTAs (<= SM count) runs `rounds`
 * rounds; in round t every CTA publishes a tagged word and waits for both
 * ring neighbours' round-t words.  If 0 <= skip < ctas, CTA `skip`
 * publishes nothing, so its neighbours give up after timeout_ms (1..10000),
 * write CNMF_E_TIMEOUT to *dev_status and raise the abort flag, and every
 * CTA returns -- nothing hangs.  With skip < 0 all rounds complete and
 * *dev_status stays 0.  *out_rounds (optional device int32) receives the
 * number of rounds CTA 0 completed.  ws: >= 256 + 16 ctas bytes.
 * (Library self-test; the paper has no counterpart.)
 * ---------------------------------------------------------------------- */
cnmf_status cnmf_tagwait_selftest(int32_t ctas, int32_t rounds, int32_t skip,
                                  int32_t timeout_ms, void* ws,
                                  size_t ws_bytes, int32_t* dev_status,
                                  int32_t* out_rounds, cnmf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CNMF_H */

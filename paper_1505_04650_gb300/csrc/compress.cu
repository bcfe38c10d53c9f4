// Two-sided structured random compression (Alg. 1 applied to A and A^T,
// Sec. III) and its building blocks, behind the C ABI.
//
// Pass t = 0 .. 2q forms one product A . X (n x d -> m x d) and one product
// A^T . Y (m x d -> n x d).  At even t the A-product belongs to the left
// chain (L: A Omega, A A^T A Omega, ...) and the A^T-product to the right
// chain (R^T: A^T Psi, ...); at odd t the roles swap.  Every product is
// re-orthonormalised before it feeds the next pass (one shifted CholeskyQR
// sweep; CholeskyQR2 on the last pass), so after pass 2q the m x d panel
// is L and the n x d panel is R^T.  One more product
// gives A-check = A R^T and then A-tilde = L^T A-check (Alg. 4 setup).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace cnmf {

static bool valid_type(cnmf_dtype t) {
  return t == CNMF_F64 || t == CNMF_F32 || t == CNMF_BF16;
}
static cnmf_dtype work_type(cnmf_dtype a) {
  return a == CNMF_F64 ? CNMF_F64 : CNMF_F32;
}

// x[0 .. count) *= c
template <typename W>
__global__ void k_scale(W* __restrict__ x, int64_t count, W c) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= c;
}

static cnmf_status launch_scale(void* x, int64_t count, cnmf_dtype w,
                                double c, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((count + 255) / 256, 4 * num_sms()));
  if (w == CNMF_F64)
    k_scale<double><<<grid, 256, 0, s>>>((double*)x, count, c);
  else
    k_scale<float><<<grid, 256, 0, s>>>((float*)x, count, (float)c);
  CNMF_CUDA(cudaGetLastError());
  return CNMF_OK;
}

struct CompressLayout {
  int KP;
  size_t bytes;
  // pieces (null base -> offsets only)
  void *om, *ps, *m0, *m1, *n0, *n1, *acheck, *prod_ws, *orth_ws;
  size_t prod_bytes, orth_bytes;
};

// prod_rows: the row count of the matrices the product kernels see (m, or
// the row-block size when A is streamed from host memory)
static CompressLayout compress_layout(void* ws, int64_t m, int64_t n, int d,
                                      cnmf_dtype a_type,
                                      int64_t prod_rows = -1) {
  CompressLayout L;
  cnmf_dtype w = work_type(a_type);
  size_t e = wbytes(w);
  L.KP = pad_k(d);
  Carve cv(ws, SIZE_MAX);
  L.om = cv.take<char>((size_t)n * d * e);
  L.ps = cv.take<char>((size_t)m * d * e);
  L.m0 = cv.take<char>((size_t)m * L.KP * e);
  L.m1 = cv.take<char>((size_t)m * L.KP * e);
  L.n0 = cv.take<char>((size_t)n * L.KP * e);
  L.n1 = cv.take<char>((size_t)n * L.KP * e);
  L.acheck = cv.take<char>((size_t)m * L.KP * e);
  L.prod_bytes = prod_workspace(prod_rows > 0 ? prod_rows : m, n, d, a_type);
  L.prod_ws = cv.take<char>(L.prod_bytes);
  L.orth_bytes = std::max(orth_workspace(std::max(m, n), d, w),
                          cross_workspace(m, d, w));
  L.orth_ws = cv.take<char>(L.orth_bytes);
  L.bytes = cv.off;
  return L;
}

// A-check = A R^T into the layout's m x KP panel: the one-sided form of the
// fused pass where it applies, else the product kernels.
static cnmf_status acheck_product(const void* A, cnmf_dtype a_type, int64_t m,
                                  int64_t n, int64_t lda, const void* Rt,
                                  int d, const CompressLayout& lay,
                                  int32_t* dev_status, cudaStream_t s) {
  if (fused_applicable(A, a_type, m, n, lda, d, true, false)) {
    FusedArgs fa{A, a_type, m, n, lda, Rt, d, nullptr, 0, d, lay.acheck,
                 lay.KP, nullptr, 0, dev_status};
    return launch_fused(fa, lay.prod_ws, lay.prod_bytes, s);
  }
  ProdArgs pc{A, a_type, m, n, lda, false, Rt, d, d, lay.acheck, lay.KP, d,
              dev_status};
  return launch_prod(pc, lay.prod_ws, lay.prod_bytes, s);
}

}  // namespace cnmf

using namespace cnmf;

extern "C" size_t cnmf_sketch_workspace(int64_t m, int64_t n, int32_t k,
                                        cnmf_dtype a_type) {
  if (m < 0 || n < 0 || k < 1 || k > 128 || !valid_type(a_type)) return 0;
  return prod_workspace(m, n, k, a_type);
}

extern "C" cnmf_status cnmf_sketch_pass(const void* A, cnmf_dtype a_type,
                                        int64_t m, int64_t n, int64_t lda,
                                        int32_t k, const void* X, const void* Y,
                                        void* Zm, void* Zn, void* ws,
                                        size_t ws_bytes, int32_t* dev_status,
                                        cnmf_stream_t stream) {
  if (!valid_type(a_type) || m < 1 || n < 1 || lda < n || k < 1 || k > 128 ||
      !A || (!X != !Zm) || (!Y != !Zn) || (!X && !Y) || !ws)
    return CNMF_E_INVALID_ARG;
  if (ws_bytes < prod_workspace(m, n, k, a_type)) return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (fused_applicable(A, a_type, m, n, lda, k, X != nullptr, Y != nullptr)) {
    FusedArgs fa{A, a_type, m, n, lda, X, k, Y, k, k, Zm, k, Zn, k, dev_status};
    return launch_fused(fa, ws, ws_bytes, s);
  }
  if (X) {
    ProdArgs pa{A, a_type, m, n, lda, false, X, k, k, Zm, k, k, dev_status};
    CNMF_TRY(launch_prod(pa, ws, ws_bytes, s));
  }
  if (Y) {
    ProdArgs pa{A, a_type, m, n, lda, true, Y, k, k, Zn, k, k, dev_status};
    CNMF_TRY(launch_prod(pa, ws, ws_bytes, s));
  }
  return CNMF_OK;
}

extern "C" size_t cnmf_orth_workspace(int64_t rows, int32_t k,
                                      cnmf_dtype w_type) {
  if (rows < 1 || k < 1 || k > 128 ||
      (w_type != CNMF_F64 && w_type != CNMF_F32))
    return 0;
  return orth_workspace(rows, k, w_type);
}

extern "C" cnmf_status cnmf_orth(void* Y, cnmf_dtype w_type, int64_t rows,
                                 int32_t k, void* ws, size_t ws_bytes,
                                 int32_t* dev_status, cnmf_stream_t stream) {
  if (!Y || !ws || rows < k || k < 1 || k > 128 ||
      (w_type != CNMF_F64 && w_type != CNMF_F32))
    return CNMF_E_INVALID_ARG;
  if (ws_bytes < orth_workspace(rows, k, w_type)) return CNMF_E_WORKSPACE;
  OrthPanel p{Y, rows, k, Y, k};
  return launch_orth(&p, 1, k, w_type, ws, ws_bytes, dev_status,
                     (cudaStream_t)stream);
}

extern "C" size_t cnmf_compress_workspace(int64_t m, int64_t n, int32_t d,
                                          cnmf_dtype a_type) {
  if (m < 1 || n < 1 || d < 1 || d > 128 || !valid_type(a_type)) return 0;
  return compress_layout(nullptr, m, n, d, a_type).bytes;
}

namespace cnmf {

// Where the passes over A come from: A resident in device memory, or A in
// host memory streamed through the GPU in row blocks.
struct PassSource {
  // Zm = A X (m x KP panel) and Zn = A^T Y (n x KP panel)
  virtual cnmf_status both(const void* X, int64_t ldx, const void* Y,
                           int64_t ldy, void* zm, void* zn) = 0;
  // Zm = A X only (A-check = A R^T)
  virtual cnmf_status left(const void* X, int64_t ldx, void* zm) = 0;
  virtual ~PassSource() = default;
};

// A in device memory: the fused pass (one read of A for both products)
// where it applies, else one read per product.
struct DeviceSource : PassSource {
  const void* A;
  cnmf_dtype a_type;
  int64_t m, n, lda;
  int d;
  const CompressLayout* lay;
  int32_t* status;
  cudaStream_t s;
  cnmf_status both(const void* X, int64_t ldx, const void* Y, int64_t ldy,
                   void* zm, void* zn) override {
    const int KP = lay->KP;
    if (fused_applicable(A, a_type, m, n, lda, d)) {
      FusedArgs fa{A, a_type, m, n, lda, X, ldx, Y, ldy, d, zm, KP, zn, KP,
                   status};
      return launch_fused(fa, lay->prod_ws, lay->prod_bytes, s);
    }
    ProdArgs pa{A, a_type, m, n, lda, false, X, ldx, d, zm, KP, d, status};
    CNMF_TRY(launch_prod(pa, lay->prod_ws, lay->prod_bytes, s));
    ProdArgs pt{A, a_type, m, n, lda, true, Y, ldy, d, zn, KP, d, status};
    return launch_prod(pt, lay->prod_ws, lay->prod_bytes, s);
  }
  cnmf_status left(const void* X, int64_t ldx, void* zm) override {
    const int KP = lay->KP;
    if (fused_applicable(A, a_type, m, n, lda, d, true, false)) {
      FusedArgs fa{A, a_type, m, n, lda, X, ldx, nullptr, 0, d, zm, KP,
                   nullptr, 0, status};
      return launch_fused(fa, lay->prod_ws, lay->prod_bytes, s);
    }
    ProdArgs pc{A, a_type, m, n, lda, false, X, ldx, d, zm, KP, d, status};
    return launch_prod(pc, lay->prod_ws, lay->prod_bytes, s);
  }
};

// x[i] = y[i] (first) or x[i] + y[i]
template <typename W>
__global__ void k_acc(W* __restrict__ x, const W* __restrict__ y,
                      int64_t count, int first) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = first ? y[i] : x[i] + y[i];
}

static cnmf_status launch_acc(void* x, const void* y, int64_t count,
                              bool first, cnmf_dtype w, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((count + 255) / 256, 4 * num_sms()));
  if (w == CNMF_F64)
    k_acc<double><<<grid, 256, 0, s>>>((double*)x, (const double*)y, count,
                                       first ? 1 : 0);
  else
    k_acc<float><<<grid, 256, 0, s>>>((float*)x, (const float*)y, count,
                                      first ? 1 : 0);
  CNMF_CUDA(cudaGetLastError());
  return CNMF_OK;
}

// A outside device memory (host memory; page-locked memory gives the full
// copy rate), streamed in row blocks: each block is copied into one device
// buffer with a 16-byte-aligned row pitch and goes through the device path;
// the blocks' shares of A^T Y are added in block order, so the result does
// not depend on timing.  The m x d and n x d panels, their
// orthonormalisation (CholeskyQR2: its Gram matrices are sums over row
// blocks of the resident panels, the one central reduction that TSQR plays
// in the paper's out-of-core setting) and A-tilde stay in device memory.
// The copy lane of the out-of-core passes: one non-blocking stream and
// five events per host thread and device, created on the thread's first
// out-of-core call on that device and kept until exit.  Block copies run on
// it, so the copy of block k + 1 overlaps the products of block k on the
// caller's stream; events order the two (no host synchronisation).
struct CopyLane {
  bool ok = false;
  cudaStream_t cs = nullptr;
  cudaEvent_t start = nullptr, copied[2] = {nullptr, nullptr},
              freed[2] = {nullptr, nullptr};
};
constexpr int LANE_DEVS = 16;

static CopyLane* copy_lane() {
  static thread_local CopyLane lanes[LANE_DEVS];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LANE_DEVS) {
    (void)cudaGetLastError();
    return nullptr;   // the caller's stream alone (no overlap)
  }
  CopyLane& l = lanes[dev];
  if (!l.ok) {
    const unsigned f = cudaEventDisableTiming;
    bool good =
        cudaStreamCreateWithFlags(&l.cs, cudaStreamNonBlocking) == cudaSuccess;
    good = good && cudaEventCreateWithFlags(&l.start, f) == cudaSuccess;
    for (int i = 0; i < 2 && good; ++i)
      good = cudaEventCreateWithFlags(&l.copied[i], f) == cudaSuccess &&
             cudaEventCreateWithFlags(&l.freed[i], f) == cudaSuccess;
    if (!good) {
      (void)cudaGetLastError();
      return nullptr;
    }
    l.ok = true;
  }
  return &l;
}

// A in host memory: each pass copies A in row blocks into one of two device
// buffers and runs the block through the same product kernels; the blocks'
// shares of A^T Y are added in block order.  With a copy lane, block k + 1
// is copied (lane stream) while block k's products run (caller's stream);
// block k + 2 reuses block k's buffer once its products are done.
struct HostSource : PassSource {
  const void* A;
  cnmf_dtype a_type;
  int64_t m, n, lda;
  int d;
  int64_t rows_blk;
  void* blk[2];      // rows_blk x ldb each, a_type
  int64_t ldb;
  void* znb;         // n x KP, the block's share of A^T Y
  const CompressLayout* lay;
  int32_t* status;
  cudaStream_t s;
  CopyLane* lane;    // null: copies on s, one after the other

  size_t es() const {
    return a_type == CNMF_F64 ? 8 : (a_type == CNMF_F32 ? 4 : 2);
  }
  // copy block k (rows i0 .. i0 + mb) into its buffer
  cnmf_status copy(int64_t k, int64_t i0, int64_t mb) {
    const size_t e = es();
    const int b = (int)(k & 1);
    cudaStream_t cs = lane ? lane->cs : s;
    if (lane && k >= 2) CNMF_CUDA(cudaStreamWaitEvent(cs, lane->freed[b], 0));
    CNMF_CUDA(cudaMemcpy2DAsync(blk[b], (size_t)ldb * e,
                                (const char*)A + (size_t)i0 * lda * e,
                                (size_t)lda * e, (size_t)n * e, (size_t)mb,
                                cudaMemcpyDefault, cs));
    if (lane) CNMF_CUDA(cudaEventRecord(lane->copied[b], cs));
    return CNMF_OK;
  }
  // block k's products wait for its copy (enqueued on s just before them,
  // after the copy of block k + 1 has been issued)
  cnmf_status arrived(int64_t k) {
    if (lane) CNMF_CUDA(cudaStreamWaitEvent(s, lane->copied[k & 1], 0));
    return CNMF_OK;
  }
  // the lane starts after everything already on s (the buffers' last
  // readers, the panels of the pass before)
  cnmf_status begin() {
    if (!lane) return CNMF_OK;
    CNMF_CUDA(cudaEventRecord(lane->start, s));
    CNMF_CUDA(cudaStreamWaitEvent(lane->cs, lane->start, 0));
    return CNMF_OK;
  }
  cnmf_status done(int64_t k) {
    if (lane) CNMF_CUDA(cudaEventRecord(lane->freed[k & 1], s));
    return CNMF_OK;
  }
  DeviceSource block(int64_t k, int64_t mb) const {
    DeviceSource b;
    b.A = blk[k & 1]; b.a_type = a_type; b.m = mb; b.n = n; b.lda = ldb;
    b.d = d; b.lay = lay; b.status = status; b.s = s;
    return b;
  }
  cnmf_status both(const void* X, int64_t ldx, const void* Y, int64_t ldy,
                   void* zm, void* zn) override {
    const size_t w = wbytes(work_type(a_type));
    const int KP = lay->KP;
    CNMF_TRY(begin());
    const int64_t nblk = ceil_div(m, rows_blk);
    // the first copy goes out ahead; then the copy of block k + 1 is issued
    // before block k's products
    CNMF_TRY(copy(0, 0, std::min(rows_blk, m)));
    for (int64_t k = 0; k < nblk; ++k) {
      const int64_t i0 = k * rows_blk;
      const int64_t mb = std::min(rows_blk, m - i0);
      if (k + 1 < nblk)
        CNMF_TRY(copy(k + 1, i0 + rows_blk,
                      std::min(rows_blk, m - i0 - rows_blk)));
      CNMF_TRY(arrived(k));
      DeviceSource b = block(k, mb);
      CNMF_TRY(b.both(X, ldx, (const char*)Y + (size_t)i0 * ldy * w, ldy,
                      (char*)zm + (size_t)i0 * KP * w, znb));
      CNMF_TRY(launch_acc(zn, znb, n * (int64_t)KP, i0 == 0,
                          work_type(a_type), s));
      CNMF_TRY(done(k));
    }
    return CNMF_OK;
  }
  cnmf_status left(const void* X, int64_t ldx, void* zm) override {
    const size_t w = wbytes(work_type(a_type));
    const int KP = lay->KP;
    CNMF_TRY(begin());
    const int64_t nblk = ceil_div(m, rows_blk);
    CNMF_TRY(copy(0, 0, std::min(rows_blk, m)));
    for (int64_t k = 0; k < nblk; ++k) {
      const int64_t i0 = k * rows_blk;
      const int64_t mb = std::min(rows_blk, m - i0);
      if (k + 1 < nblk)
        CNMF_TRY(copy(k + 1, i0 + rows_blk,
                      std::min(rows_blk, m - i0 - rows_blk)));
      CNMF_TRY(arrived(k));
      DeviceSource b = block(k, mb);
      CNMF_TRY(b.left(X, ldx, (char*)zm + (size_t)i0 * KP * w));
      CNMF_TRY(done(k));
    }
    return CNMF_OK;
  }
};

struct HostLayout {
  CompressLayout lay;
  int64_t rows_blk, ldb;
  void *blk[2], *znb;
  size_t bytes;
};

static HostLayout host_layout(void* ws, int64_t m, int64_t n, int d,
                              cnmf_dtype a_type, int64_t block_rows) {
  HostLayout H;
  H.rows_blk = std::min(block_rows, m);
  H.lay = compress_layout(ws, m, n, d, a_type, H.rows_blk);
  const size_t e = a_type == CNMF_F64 ? 8 : (a_type == CNMF_F32 ? 4 : 2);
  H.ldb = (n + 7) / 8 * 8;
  Carve cv(ws ? (char*)ws + H.lay.bytes : nullptr, SIZE_MAX);
  H.blk[0] = cv.take<char>((size_t)H.rows_blk * H.ldb * e);
  H.blk[1] = cv.take<char>((size_t)H.rows_blk * H.ldb * e);
  H.znb = cv.take<char>((size_t)n * H.lay.KP * wbytes(work_type(a_type)));
  H.bytes = H.lay.bytes + cv.off;
  return H;
}

// Alg. 1 on A and A^T (2q + 1 passes with re-orthonormalisation), then
// A-check and A-tilde, over any source of passes.
static cnmf_status compress_passes(PassSource& src, cnmf_dtype a_type,
                                   int64_t m, int64_t n, int r, int d, int q,
                                   uint64_t seed, const void* Omega,
                                   const void* Psi, void* L, void* Rt,
                                   void* Atilde, const CompressLayout& lay,
                                   int32_t* dev_status, cudaStream_t s) {
  (void)r;
  const cnmf_dtype w = work_type(a_type);
  const int KP = lay.KP;
  const void* X = Omega;   // n x d operand of the A-product
  int64_t ldx = d;
  const void* Y = Psi;     // m x d operand of the A^T-product
  int64_t ldy = d;
  if (!X) {
    CNMF_TRY(launch_gaussian(seed, 0, n * (int64_t)d, w, lay.om, s));
    X = lay.om;
  }
  if (!Y) {
    CNMF_TRY(launch_gaussian(seed, 1, m * (int64_t)d, w, lay.ps, s));
    Y = lay.ps;
  }
  void* mb[2] = {lay.m0, lay.m1};
  void* nb[2] = {lay.n0, lay.n1};
  const int T = 2 * q + 1;
  for (int t = 0; t < T; ++t) {
    const bool last = (t == T - 1);
    void* zm = mb[t & 1];
    void* zn = nb[t & 1];
    CNMF_TRY(src.both(X, ldx, Y, ldy, zm, zn));
    OrthPanel op[2] = {{zm, m, KP, last ? L : zm, last ? d : KP},
                       {zn, n, KP, last ? Rt : zn, last ? d : KP}};
    // the last pass gives L and R^T: the unique thin Q (CholeskyQR2); in
    // between, one sweep keeps the basis well conditioned with the same
    // span, and the final thin Q does not depend on the basis fed to the
    // product (it differs by an upper-triangular factor)
    CNMF_TRY(launch_orth(op, 2, d, w, lay.orth_ws, lay.orth_bytes, dev_status,
                         s, last ? 2 : 1));
    // next pass: A-product takes the n x d panel, A^T-product the m x d one
    X = zn; ldx = KP;
    Y = zm; ldy = KP;
  }
  // A-check = A R^T (m x d), then A-tilde = L^T A-check (d x d)
  CNMF_TRY(src.left(Rt, d, lay.acheck));
  CNMF_TRY(launch_cross(L, d, lay.acheck, KP, m, d, w, Atilde, d, lay.orth_ws,
                        lay.orth_bytes, s));
  return CNMF_OK;
}

}  // namespace cnmf

using namespace cnmf;

extern "C" cnmf_status cnmf_compress(const void* A, cnmf_dtype a_type,
                                     int64_t m, int64_t n, int64_t lda,
                                     int32_t r, int32_t d, int32_t q,
                                     uint64_t seed, const void* Omega,
                                     const void* Psi, void* L, void* Rt,
                                     void* Atilde, void* ws, size_t ws_bytes,
                                     int32_t* dev_status,
                                     cnmf_stream_t stream) {
  if (!valid_type(a_type) || !A || !L || !Rt || !Atilde || !ws || m < 1 ||
      n < 1 || lda < n || r < 1 || d < r || d > 128 || d > m || d > n ||
      q < 0 || q > 64)
    return CNMF_E_INVALID_ARG;
  CompressLayout lay = compress_layout(ws, m, n, d, a_type);
  if (ws_bytes < lay.bytes) return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceSource src;
  src.A = A; src.a_type = a_type; src.m = m; src.n = n; src.lda = lda;
  src.d = d; src.lay = &lay; src.status = dev_status; src.s = s;
  return compress_passes(src, a_type, m, n, r, d, q, seed, Omega, Psi, L, Rt,
                         Atilde, lay, dev_status, s);
}

extern "C" cnmf_status cnmf_compress_gaussian(const void* A, cnmf_dtype a_type,
                                              int64_t m, int64_t n,
                                              int64_t lda, int32_t d,
                                              uint64_t seed, void* L, void* Rt,
                                              void* Atilde, void* ws,
                                              size_t ws_bytes,
                                              int32_t* dev_status,
                                              cnmf_stream_t stream) {
  if (!valid_type(a_type) || !A || !L || !Rt || !Atilde || !ws || m < 1 ||
      n < 1 || lda < n || d < 1 || d > 128 || d > m || d > n)
    return CNMF_E_INVALID_ARG;
  CompressLayout lay = compress_layout(ws, m, n, d, a_type);
  if (ws_bytes < lay.bytes) return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const cnmf_dtype w = work_type(a_type);
  const int KP = lay.KP;
  // L = d^-1/2 Psi (stream 1, m x d), R^T = d^-1/2 Omega (stream 0, n x d):
  // the test matrices of cnmf_compress, without power iteration or
  // orthonormalisation
  const double c = 1.0 / std::sqrt((double)d);
  CNMF_TRY(launch_gaussian(seed, 1, m * (int64_t)d, w, L, s));
  CNMF_TRY(launch_scale(L, m * (int64_t)d, w, c, s));
  CNMF_TRY(launch_gaussian(seed, 0, n * (int64_t)d, w, Rt, s));
  CNMF_TRY(launch_scale(Rt, n * (int64_t)d, w, c, s));
  // A-check = A R^T (m x d), then A-tilde = L^T A-check (d x d)
  CNMF_TRY(acheck_product(A, a_type, m, n, lda, Rt, d, lay, dev_status, s));
  CNMF_TRY(launch_cross(L, d, lay.acheck, KP, m, d, w, Atilde, d, lay.orth_ws,
                        lay.orth_bytes, s));
  return CNMF_OK;
}

extern "C" size_t cnmf_compress_host_workspace(int64_t m, int64_t n, int32_t d,
                                               cnmf_dtype a_type,
                                               int64_t block_rows) {
  if (m < 1 || n < 1 || d < 1 || d > 128 || block_rows < 1 ||
      !valid_type(a_type))
    return 0;
  return host_layout(nullptr, m, n, d, a_type, block_rows).bytes;
}

extern "C" cnmf_status cnmf_compress_host(const void* A, cnmf_dtype a_type,
                                          int64_t m, int64_t n, int64_t lda,
                                          int32_t r, int32_t d, int32_t q,
                                          uint64_t seed, const void* Omega,
                                          const void* Psi, void* L, void* Rt,
                                          void* Atilde, int64_t block_rows,
                                          void* ws, size_t ws_bytes,
                                          int32_t* dev_status,
                                          cnmf_stream_t stream) {
  if (!valid_type(a_type) || !A || !L || !Rt || !Atilde || !ws || m < 1 ||
      n < 1 || lda < n || r < 1 || d < r || d > 128 || d > m || d > n ||
      q < 0 || q > 64 || block_rows < 1)
    return CNMF_E_INVALID_ARG;
  HostLayout H = host_layout(ws, m, n, d, a_type, block_rows);
  if (ws_bytes < H.bytes) return CNMF_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  HostSource src;
  src.A = A; src.a_type = a_type; src.m = m; src.n = n; src.lda = lda;
  src.d = d; src.rows_blk = H.rows_blk; src.blk[0] = H.blk[0];
  src.blk[1] = H.blk[1]; src.ldb = H.ldb; src.znb = H.znb; src.lay = &H.lay;
  src.status = dev_status; src.s = s; src.lane = copy_lane();
  return compress_passes(src, a_type, m, n, r, d, q, seed, Omega, Psi, L, Rt,
                         Atilde, H.lay, dev_status, s);
}

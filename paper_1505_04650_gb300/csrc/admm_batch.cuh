// Batched compressed ADMM (Alg. 4) for many independent small problems in
// one launch.  Included by admm_impl.cuh.
//
// Each problem is handled by one thread-block cluster of CS CTAs (CS = 1, 2,
// 4 or 8; the autotuner picks it per problem size).  The CTAs of a cluster
// split the problem's rows like the CTAs of the cooperative kernel, run the
// same register-tiled small algebra and row sweeps, and add their shares of
// the next SX, SY^T through distributed shared memory in rank order -- a
// hardware cluster barrier replaces the grid barriers, so nothing spins and
// a problem's arithmetic does not depend on which other problems share the
// launch (the same problem gives bitwise the same result alone or in a
// batch).  The reduced SX, SY^T are kept in the problem's scratch between
// launches, so a problem can run its sweeps over several launches (the
// serving loop's rounds) with exactly the arithmetic of one long run.
namespace cg = cooperative_groups;

struct BatchSmem {
  FastSmem f;
  int share0, share1, SX, SY, total;
  __host__ __device__ BatchSmem(int r, int d, int dmax)
      : f(r, d, false, 0, 0, dmax, false, false) {
    int o = f.total;
    auto take = [&](int n) { int p = o; o += (n + 3) & ~3; return p; };
    share0 = take(3 * d * r);
    share1 = take(3 * d * r);
    SX = take(d * r);
    SY = take(d * r);
    total = o;
  }
};

template <typename W, int DMAX, int RMAX, int CS>
__global__ void __launch_bounds__(AD_NT)
    k_admm_batch(const cnmf_batch_item* __restrict__ items, int nitems,
                 int sweeps, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sm = reinterpret_cast<W*>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int item = blockIdx.x / CS;
  const int rank = (int)cl.block_rank();
  if (item >= nitems) return;                      // uniform per cluster
  const cnmf_batch_item it = items[item];
  if (it.r < 1 || it.L == nullptr) return;         // empty slot
  AdmmArgs<W> a;
  a.L = (const W*)it.L; a.Rt = (const W*)it.Rt; a.At = (const W*)it.Atilde;
  a.U = (W*)it.U; a.Vt = (W*)it.Vt;
  a.m = it.m; a.n = it.n; a.r = it.r; a.d = it.d;
  a.Gu = 0;            // every CTA of the cluster sweeps both sides
  a.Ypub = nullptr;
  a.tpart = a.tsxy = a.typ = nullptr;
  const int r = a.r, d = a.d, dr = d * r;
  char* st = (char*)it.state;
  a.Lam = (W*)st;
  a.Phit = a.Lam + (size_t)a.m * r;
  a.Yt = a.Phit + (size_t)a.n * r;
  a.Xt = a.Yt + (size_t)r * d;
  // state layout of cnmf_factor: Lam, Phit, Yt, Xt, then int64 k
  const size_t sbytes =
      (((size_t)a.m * r + (size_t)a.n * r + 2 * (size_t)r * d) * sizeof(W) + 7) &
      ~size_t(7);
  a.kcount = (int64_t*)(st + sbytes);
  a.Zs = (W*)(st + sbytes + 8);
  W* keep = (W*)it.scratch;                        // reduced SX | SY^T
  a.SX = keep; a.SY = keep + dr;
  a.status = status;
  a.lam = (W)it.lambda; a.phi = (W)it.phi; a.xi = (W)it.xi;
  a.phase_ns = nullptr;
  const BatchSmem b(r, d, DMAX);
  const FastSmem& o = b.f;
  const int RP = o.RP;
  W* SXs = sm + b.SX;
  W* SYs = sm + b.SY;
  for (int e = threadIdx.x; e < d * d; e += AD_NT) {
    const W v = a.At[e];
    sm[o.At + e] = v;
    sm[o.AtT + (e % d) * d + e / d] = v;
  }
  for (int e = threadIdx.x; e < d * RP; e += AD_NT) {
    sm[o.YtT + e] = W(0);
    sm[o.Xt + e] = W(0);
  }
  __syncthreads();
  if (!(it.lambda > 0)) {
    // the balanced default lambda = phi = ||Atilde||_F / r, formed here
    // (FP64 squares, added in a fixed order) so the caller needs no host
    // round trip after the compression; a negative lambda scales it by
    // -lambda
    __shared__ double nrm_s[AD_NT / 32 + 1];
    double s = 0.0;
    for (int e = threadIdx.x; e < d * d; e += AD_NT) {
      const double v = (double)sm[o.At + e];
      s = fma(v, v, s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) nrm_s[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < AD_NT / 32; ++w) t += nrm_s[w];
      nrm_s[AD_NT / 32] = sqrt(t) / r;
    }
    __syncthreads();
    const double scale = it.lambda < 0 ? -it.lambda : 1.0;
    a.lam = a.phi = (W)(nrm_s[AD_NT / 32] * scale);
  }

  // cluster-wide sum of the shares in `buf` (entries [0, E)) in rank order
  auto reduce = [&](int buf, int E) {
    cl.sync();
    for (int e = threadIdx.x; e < E; e += AD_NT) {
      W s = W(0);
      for (int q = 0; q < CS; ++q) {
        const W* rem = cl.map_shared_rank(sm + buf, q);
        s += rem[e];
      }
      if (e < dr) SXs[e] = s;
      else if (e < 2 * dr) SYs[e - dr] = s;
      else {   // Yt0^T -> Yt (state) on a fresh start
        const int k = (e - 2 * dr) / r, bb = (e - 2 * dr) % r;
        if (rank == 0) a.Yt[bb * d + k] = s;
        sm[o.YtT + k * RP + bb] = s;
      }
    }
    __syncthreads();
  };

  int parity = 0;
  bool have = false;
  if (it.flags & CNMF_BATCH_FRESH) {
    sweep_fast<W, DMAX, false>(a, sm, o, 0, nullptr, CS, rank,
                               sm + b.share0);
    reduce(b.share0, 3 * dr);
    parity = 1;
    if (rank == 0 && threadIdx.x == 0) *a.kcount = 0;
  } else {
    for (int e = threadIdx.x; e < dr; e += AD_NT) {
      SXs[e] = keep[e];
      SYs[e] = keep[dr + e];
    }
    for (int e = threadIdx.x; e < dr; e += AD_NT) {
      const int k = e / r, bb = e % r;
      sm[o.YtT + k * RP + bb] = a.Yt[bb * d + k];
    }
    // the inverses the last launch kept (a problem's sweeps may be split
    // over launches with the arithmetic of one run)
    have = *a.kcount > 0;
    if (have) load_inverses<W>(a.Zs, r, RP, sm + o.Zx, sm + o.Zy);
    __syncthreads();
  }
  for (int s = 0; s < sweeps; ++s) {
    small_fast<W, DMAX, RMAX>(a, sm, o, have || s > 0, nullptr, SXs, SYs, true);
    const int buf = parity ? b.share1 : b.share0;
    sweep_fast<W, DMAX, false>(a, sm, o, 2, nullptr, CS, rank, sm + buf);
    reduce(buf, 2 * dr);
    parity ^= 1;
  }
  cl.sync();   // no CTA may leave while others read its shares
  if (rank == 0) {
    for (int e = threadIdx.x; e < dr; e += AD_NT) {
      const int k = e / r, bb = e % r;
      a.Yt[bb * d + k] = sm[o.YtT + k * RP + bb];
      if (sweeps > 0) a.Xt[e] = sm[o.Xt + k * RP + bb];
      keep[e] = SXs[e];
      keep[dr + e] = SYs[e];
    }
    if (sweeps > 0) store_inverses<W>(a.Zs, r, RP, sm + o.Zx, sm + o.Zy);
    if (threadIdx.x == 0) *a.kcount += sweeps;
  }
}


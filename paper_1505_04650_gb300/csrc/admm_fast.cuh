// Register-tiled path of the compressed ADMM kernel (Alg. 4) for d <= 64,
// r <= 32.  Included by admm.cu after the generic path.
//
// Layout: every matrix with an r-long dimension is stored with that
// dimension last and padded to RP = 4 ceil(r / 4) (zeros in the padding),
// so four consecutive columns are one 16-byte shared-memory load:
//   At, AtT d x d         Atilde and its transpose
//   YtT  d x RP           Yt^T
//   Xt   d x RP           Xt
//   M, T d x RP           MX (then MY^T), solve scratch
//   G    r x RP           Gram matrix (destroyed by the solve)
//   Zx, Zy r x RP         kept inverses -(Gram)^-1
//   E, F, H r x RP        solve scratch
// Shares of the next sweep's SX = L^T (lam U - Lam) and SY^T =
// R (phi V - Phi)^T (both d x r) are reduced in that layout.
//
// One small-algebra step is six block-wide phases when the kept inverses
// need one refinement term:
//   M  = SX + At Yt^T            G = Yt Yt^T + lam I
//   T  = -M Zx                   E = I + G Zx
//   Xt = T + T E                 Zx <- Zx + Zx E
//   M  = SY^T + At^T Xt          G = Xt^T Xt + phi I
//   T  = -M Zy                   E = I + G Zy
//   Yt^T = T + T E               Zy <- Zy + Zy E
// (Xt = M (Yt Yt^T + lam I)^-1, Yt^T = M (Xt^T Xt + phi I)^-1 = (G^-1
// MY)^T as G is symmetric.)  Each output quad C[p][4q..4q+3] is one
// thread's task: a length-S loop of one scalar load, one 16-byte load and
// four FMAs.

struct FastSmem {
  int RP, dp, nl;
  int At, AtT, YtT, Xt, M, T, G, Zx, Zy, E, F, H, v, mx, sSX, sSY, Red, sL, sU,
      sLam, sRt, sVt, sPhit, total;
  // dmax: the register tile width; resident rows are stored zero-padded to
  // dmax with pitch dmax + 4 (4 banks apart: the <= 8 rows one warp reads
  // with 16-byte loads hit distinct banks).
  // split: each CTA holds rows of one side only (U/V split), so the two
  // sides' resident rows share one region.
  // stage: room to stage the reduced shares SX, SY^T read from global memory.
  __host__ __device__ FastSmem(int r, int d, bool res, int64_t mu,
                               int64_t nv, int dmax, bool split = false,
                               bool stage = true) {
    RP = (r + 3) & ~3;
    dp = dmax + 4;
    nl = AD_NT / r;
    int o = 0;
    auto take = [&](int64_t n) { int p = o; o += (int)((n + 3) & ~3); return p; };
    At = take(d * d);
    AtT = take(d * d);
    YtT = take(d * RP);
    Xt = take(d * RP);
    M = take(d * RP);
    T = take(d * RP);
    G = take(r * RP);
    Zx = take(r * RP);
    Zy = take(r * RP);
    E = take(r * RP);
    F = take(r * RP);
    H = take(r * RP);
    v = take(2 * 32);
    mx = take(AD_NT / 32);
    sSX = stage ? take(d * r) : 0;
    sSY = stage ? take(d * r) : 0;
    Red = take((int64_t)nl * d * r);
    if (res && split) {
      const int64_t rows = mu > nv ? mu : nv;
      sL = sRt = take(rows * dp);
      sU = sVt = take(rows * r);
      sLam = sPhit = take(rows * r);
    } else {
      sL = res ? take(mu * dp) : 0;
      sU = res ? take(mu * r) : 0;
      sLam = res ? take(mu * r) : 0;
      sRt = res ? take(nv * dp) : 0;
      sVt = res ? take(nv * r) : 0;
      sPhit = res ? take(nv * r) : 0;
    }
    total = o;
  }
};

// C[p][4q..4q+3] = init + scale * sum_{s < S} A(p, s) B[s][4q..4q+3]
// for all tasks (p, q), p < P, q < RP/4; A(p, s) = A[p * sap + s * sas].
// With `amax`, each warp also writes the largest |C| entry (NaN wins) of
// its tasks to amax[warp] (every warp writes; the caller syncs).
template <typename W>
__device__ __forceinline__ void quad_mm(W* C, int RP, const W* A, int sap,
                                        int sas, const W* B, int P, int S,
                                        W scale, const W* init_g, int init_ld,
                                        int init_cols, W diag, int task0,
                                        bool init_smem, W* amax = nullptr,
                                        bool* nonfinite = nullptr) {
  const int Q = RP / 4;
  W mx = W(0);
  bool bad = false;
  for (int t = threadIdx.x - task0; t < P * Q; t += AD_NT) {
    if (t < 0) continue;
    const int p = t / Q, q = t % Q;
    W c0 = W(0), c1 = W(0), c2 = W(0), c3 = W(0);
    W ini[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = 4 * q + j;
      ini[j] = W(0);
      if (init_g && col < init_cols)
        ini[j] = init_smem ? init_g[p * init_ld + col]
                           : __ldcg(init_g + p * init_ld + col);
    }
    const W* ap = A + p * sap;
    const W* bp = B + 4 * q;
#pragma unroll 4
    for (int s = 0; s < S; ++s) {
      const W av = ap[s * sas];
      W b4[4];
      ldsN<4, W>(bp + s * RP, b4);
      c0 = fma(av, b4[0], c0);
      c1 = fma(av, b4[1], c1);
      c2 = fma(av, b4[2], c2);
      c3 = fma(av, b4[3], c3);
    }
    W o[4] = {c0 * scale, c1 * scale, c2 * scale, c3 * scale};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = 4 * q + j;
      o[j] += ini[j];
      if (col == p) o[j] += diag;
      if (col >= init_cols) o[j] = W(0);   // keep the padding at zero
      const W av = fabs(o[j]);
      mx = (av > mx || av != av) ? av : mx;
      bad |= !isfinite(o[j]);
    }
    sts4<W>(C + p * RP + 4 * q, o);
  }
  if (amax) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const W v = __shfl_xor_sync(0xffffffffu, mx, off);
      mx = (v > mx || v != v) ? v : mx;
    }
    if ((threadIdx.x & 31) == 0) amax[threadIdx.x >> 5] = mx;
  }
  if (nonfinite && bad) *nonfinite = true;
}

// One operand pair of dual_mm: C = init + scale * A B + diag I, with
// A(p, s) = A[p * sap + s * sas] (P rows), B (S x RP), init (P x init_ld,
// shared memory) or none.  qmaj: consecutive lanes take consecutive rows p
// of one column quad (pick it when A is read along p, sap = 1: the lanes of a
// quarter warp then share one 16-byte B load and read consecutive A words);
// otherwise consecutive lanes take the quads of one row.
template <typename W>
struct QProd {
  W* C;
  const W* A;
  int sap, sas;
  const W* B;
  int P;
  W scale;
  const W* init;
  int init_ld;
  W diag;
  bool qmaj;
};

// Two products with the same inner length S in one task loop (tasks of x
// first): every lane runs the same instructions whichever product its task
// belongs to, so a warp holding tasks of both does not run two loops.  Each
// output quad is one thread's task.  The padding columns (>= cols) are
// written as zeros.  amax (y's tasks only): each warp's largest |C| entry
// (NaN wins) to amax[warp] (every warp writes; the caller syncs).
// nonfinite: set when an entry of x's output is not finite.
template <typename W>
__device__ __forceinline__ void dual_mm(const QProd<W>& x, const QProd<W>& y,
                                        int RP, int S, int cols,
                                        W* amax = nullptr,
                                        bool* nonfinite = nullptr) {
  const int Q = RP / 4;
  const int n1 = x.P * Q, n2 = y.P * Q;
  W mx = W(0);
  bool bad = false;
  for (int t = threadIdx.x; t < n1 + n2; t += AD_NT) {
    const bool sec = t >= n1;
    const QProd<W>& g = sec ? y : x;
    const int u = sec ? t - n1 : t;
    const int p = g.qmaj ? u % g.P : u / Q;
    const int q = g.qmaj ? u / g.P : u % Q;
    const W* ap = g.A + p * g.sap;
    const W* bp = g.B + 4 * q;
    const int sas = g.sas;
    W c0 = W(0), c1 = W(0), c2 = W(0), c3 = W(0);
#pragma unroll 4
    for (int s = 0; s < S; ++s) {
      const W av = ap[s * sas];
      W b4[4];
      ldsN<4, W>(bp + s * RP, b4);
      c0 = fma(av, b4[0], c0);
      c1 = fma(av, b4[1], c1);
      c2 = fma(av, b4[2], c2);
      c3 = fma(av, b4[3], c3);
    }
    const W sc = g.scale, dg = g.diag;
    W o[4] = {c0 * sc, c1 * sc, c2 * sc, c3 * sc};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = 4 * q + j;
      if (g.init && col < cols) o[j] += g.init[p * g.init_ld + col];
      if (col == p) o[j] += dg;
      if (col >= cols) o[j] = W(0);   // keep the padding at zero
      const W av = fabs(o[j]);
      if (sec) mx = (av > mx || av != av) ? av : mx;
      else bad |= !isfinite(o[j]);
    }
    sts4<W>(g.C + p * RP + 4 * q, o);
  }
  if (amax) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const W v = __shfl_xor_sync(0xffffffffu, mx, off);
      mx = (v > mx || v != v) ? v : mx;
    }
    if ((threadIdx.x & 31) == 0) amax[threadIdx.x >> 5] = mx;
  }
  if (nonfinite && bad) *nonfinite = true;
}

__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

// -G^-1 in place for the leading r x r block of G (pitch RP <= RMAX): the
// sweep operator of spd_sweep_inverse with every entry quad held in a
// register of one thread for all pivots (thread (i, q) owns G[i][4q..4q+3]);
// the pivot column is published through a double-buffered shared vector, so
// each pivot costs one block barrier.  Rows/columns beyond r hold the
// identity and are never pivoted.
template <typename W, int RMAX>
__device__ void fast_sweep_inverse(W* G, W* vbuf, int r, int RP,
                                   int32_t* status) {
  constexpr int QM = RMAX / 4;
  const int t = threadIdx.x;
  const bool own = t < RMAX * QM;
  const int i = t / QM, q = t % QM;
  W g[4];
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int k = 4 * q + jj;
    g[jj] = (own && i < r && k < r) ? G[i * RP + k] : (i == k ? W(1) : W(0));
  }
  for (int j = 0; j < r; ++j) {
    W* v = vbuf + (j & 1) * 32;
    if (own && q == (j >> 2)) {
      const int jj = j & 3;
      v[i] = jj == 0 ? g[0] : (jj == 1 ? g[1] : (jj == 2 ? g[2] : g[3]));
    }
    __syncthreads();
    W dj = v[j];
    if (!(dj > W(0))) {
      if (t == 0)
        set_status(status, isfinite((double)dj) ? CNMF_E_CHOLESKY
                                                : CNMF_E_NONFINITE);
      dj = W(1);
    }
    const W id = fast_rcp(dj);
    if (own) {
      const W vi = v[i];
      const W vid = vi * id;
      W vk[4];
      ldsN<4, W>(v + 4 * q, vk);
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int k = 4 * q + jj;
        const W gen = fma(-vid, vk[jj], g[jj]);
        g[jj] = (i == j) ? ((k == j) ? -id : vk[jj] * id)
                         : ((k == j) ? vid : gen);
      }
    }
  }
  __syncthreads();
  if (own && i < r) {
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int k = 4 * q + jj;
      if (k < RP) G[i * RP + k] = (k < r) ? g[jj] : W(0);
    }
  }
  __syncthreads();
}

// The two kept inverses in the factor state: Zx then Zy, r x r each.
template <typename W>
__device__ void load_inverses(const W* Zs, int r, int RP, W* Zx, W* Zy) {
  for (int e = threadIdx.x; e < r * RP; e += AD_NT) {
    const int i = e / RP, k = e % RP;
    Zx[e] = k < r ? __ldcg(Zs + i * r + k) : W(0);
    Zy[e] = k < r ? __ldcg(Zs + r * r + i * r + k) : W(0);
  }
}
template <typename W>
__device__ void store_inverses(W* Zs, int r, int RP, const W* Zx,
                               const W* Zy) {
  for (int e = threadIdx.x; e < r * r; e += AD_NT) {
    const int i = e / r, k = e % r;
    Zs[e] = Zx[i * RP + k];
    Zs[r * r + e] = Zy[i * RP + k];
  }
}

// Xout = M Gm^-1 (P x RP) for the SPD Gm (r x RP, zero padding), with the
// inverse kept across sweeps.  The matrices of Alg. 4's two solves move
// little from one sweep to the next, so the previous sweep's Z = -Gm_prev^-1
// is refined: with E = I + Gm Z, -Gm^-1 = Z (I - E)^-1 = Z (I + E + E^2 +
// ...).  Both the solution and the new inverse are summed by Horner's rule
// from the same E:
//   T = -M Z,   X_j = T + X_{j-1} E,   Z_j = Z + Z_{j-1} E   (X_0 = T,
//   Z_0 = Z; residual E^{j+1}),
// so the solve costs one phase (T and E) plus one phase per term, and the
// product M Gm^-1 needs no phase of its own.  The number of terms follows
// max|E| so that the residual is below the working precision (FP32: |E| <=
// 3e-4: one, <= 5e-3: two, <= 2e-2: three, <= 4e-2: four terms); beyond
// that, and without a kept inverse, the sweep operator inverts Gm and one
// phase forms Xout = -M (-Gm^-1).  The choice depends only on the data, so
// every CTA makes the same one.
// Buffers: M is consumed (the odd Horner steps land there), T, E, F, H are
// scratch, Gm is destroyed.  The result lands in Xout.  Returns the buffer
// holding the new inverse: Z itself after the sweep operator (copied during
// the last phase), else F or H, which the caller copies into Z after the
// next block barrier and before F or H are written again.  `nonfinite`
// flags a non-finite entry of Xout.
template <typename W, int RMAX>
__device__ const W* solve_fast(W* Xout, W* M, W* T, int P, W* Gm, W* Z, W* E,
                               W* F, W* H, W* vbuf, W* wmax, int r, int RP,
                               bool have, int32_t* status, bool* nonfinite) {
  if (have) {
    // T = -M Z;  E = I + Gm Z (Gm symmetric: read along its columns), and
    // max |E| per warp into wmax (read by every thread until the next call:
    // nothing else writes it)
    dual_mm<W>({T, M, RP, 1, Z, P, W(-1), nullptr, 0, W(0), false},
               {E, Gm, 1, RP, Z, r, W(1), nullptr, 0, W(1), true}, RP, r, r,
               wmax);
    __syncthreads();
    W e = wmax[0];
    for (int w = 1; w < AD_NT / 32; ++w)
      e = (wmax[w] > e || wmax[w] != wmax[w]) ? wmax[w] : e;
    const bool f64 = sizeof(W) == 8;
    int terms = 0;
    if (f64) {
      terms = e <= W(1e-8) ? 1 : e <= W(2e-6) ? 2 : e <= W(1e-4) ? 3
              : e <= W(6e-4) ? 4 : 0;
    } else {
      terms = e <= W(3e-4) ? 1 : e <= W(5e-3) ? 2 : e <= W(2e-2) ? 3
              : e <= W(4e-2) ? 4 : 0;
    }
    if (terms > 0) {
      const W* xp = T;
      const W* zp = Z;
      for (int j = 1; j <= terms; ++j) {
        // the last step writes Xout; the ones before alternate with M
        W* xd = ((terms - j) & 1) ? M : Xout;
        W* zd = (j & 1) ? F : H;
        dual_mm<W>({xd, xp, RP, 1, E, P, W(1), T, RP, W(0), false},
                   {zd, zp, RP, 1, E, r, W(1), Z, RP, W(0), false}, RP, r, r,
                   nullptr, j == terms ? nonfinite : nullptr);
        __syncthreads();
        xp = xd;
        zp = zd;
      }
      return zp;
    }
  }
  fast_sweep_inverse<W, RMAX>(Gm, vbuf, r, RP, status);
  quad_mm<W>(Xout, RP, M, RP, 1, Gm, P, r, W(-1), nullptr, 0, r, W(0), 0,
             false, nullptr, nonfinite);
  for (int e = threadIdx.x; e < r * RP; e += AD_NT) Z[e] = Gm[e];
  __syncthreads();
  return Z;
}

// Tagged inputs and outputs of one sweep of the cooperative kernel.
struct SweepIO {
  const uint64_t* sxy;   // reduced SX then SY^T (2 d r values), or null:
  uint32_t stag;         //   a.SX, a.SY (plain, after a grid barrier)
  const uint64_t* yin;   // this sweep's Yt^T (d x RP) for a U-side CTA,
  uint32_t ytag;         //   or null (YtT holds it)
  uint64_t* yout;        // where the lead publishes Yt^T, or null
  uint32_t yotag;
};

// One small-algebra step of Alg. 4 (the Xt and Yt updates).
// SXp, SYp: the reduced shares -- global memory written by other CTAs
// (staged into shared memory first, one L2 round trip for all), or this
// CTA's shared memory when sxy_smem.  io: the cooperative kernel's tagged
// shares and Yt^T (null: plain a.SX, a.SY).  have: Zx, Zy hold the previous
// sweep's inverses.  half: stop after the X update (U-side CTAs of the
// split).  Returns false when a wait for tagged data gave up (timeout or
// abort; every thread of the CTA returns the same).
template <typename W, int DMAX, int RMAX>
__device__ bool small_fast(const AdmmArgs<W>& a, W* sm, const FastSmem& o,
                           bool have, uint64_t* sub = nullptr,
                           const W* SXp = nullptr, const W* SYp = nullptr,
                           bool sxy_smem = false, bool half = false,
                           const SweepIO* io = nullptr) {
  if (!SXp) { SXp = a.SX; SYp = a.SY; }
  const int r = a.r, d = a.d, RP = o.RP, dr = d * r;
  uint64_t tm = sub ? globaltimer_ns() : 0;
  auto mark = [&](int i) {
    if (sub) { uint64_t t = globaltimer_ns(); sub[i] += t - tm; tm = t; }
  };
  W* At = sm + o.At;
  W* AtT = sm + o.AtT;
  W* YtT = sm + o.YtT;
  W* Xt = sm + o.Xt;
  W* M = sm + o.M;
  W* T = sm + o.T;
  W* G = sm + o.G;
  W* Zx = sm + o.Zx;
  W* Zy = sm + o.Zy;
  W* E = sm + o.E;
  W* F = sm + o.F;
  W* H = sm + o.H;
  constexpr int KS = (DMAX * RMAX + AD_NT - 1) / AD_NT;
  constexpr int NW = sizeof(W) / 4;
  if (!sxy_smem && io && io->sxy) {
    // Sweep loop: the reduced shares (and on U-side CTAs this sweep's
    // Yt^T) are tagged words, all loads in flight at once.  Yt^T is needed
    // by the X Grams loop and is waited for first; the Grams products then
    // run while the shares may still be on their way, and SX is added to M
    // afterwards (the same sum as adding it in the loop's epilogue).
    const uint64_t* sx = io->sxy;
    const uint64_t* sy = io->sxy + (size_t)dr * NW;
    const uint64_t* yp = io->yin;
    const uint64_t dx = (uint64_t)io->stag << 32, dy = (uint64_t)io->ytag << 32;
    uint64_t wx[KS][NW], wy[KS][NW], wp[KS][NW];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int e = threadIdx.x + k * AD_NT;
#pragma unroll
      for (int h = 0; h < NW; ++h) {
        wx[k][h] = e < dr ? ld_relaxed_u64(sx + e * NW + h) : dx;
        wy[k][h] = (!half && e < dr) ? ld_relaxed_u64(sy + e * NW + h) : dx;
        wp[k][h] = (yp && e < d * RP) ? ld_relaxed_u64(yp + e * NW + h) : dy;
      }
    }
    bool ok = true;
    if (yp) {
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int e = threadIdx.x + k * AD_NT;
        if (e < d * RP) {
#pragma unroll
          for (int h = 0; h < NW; ++h)
            ok = ok && tag_spin(yp + e * NW + h, io->ytag, wp[k][h], a.bar,
                                a.status, a.timeout_ns);
          YtT[e] = tag_value<W>(wp[k]);
        }
      }
      if (__syncthreads_or(!ok)) return false;
    }
    mark(0);
    // At Yt^T (d x RP, At read along its columns from AtT);
    // G = Yt Yt^T + lam I  (r x RP)
    dual_mm<W>({M, AtT, 1, d, YtT, d, W(1), nullptr, 0, W(0), true},
               {G, YtT, 1, RP, YtT, r, W(1), nullptr, 0, a.lam, true}, RP,
               d, r);
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int e = threadIdx.x + k * AD_NT;
      if (e < dr) {
#pragma unroll
        for (int h = 0; h < NW; ++h) {
          ok = ok && tag_spin(sx + e * NW + h, io->stag, wx[k][h], a.bar,
                              a.status, a.timeout_ns);
          if (!half)
            ok = ok && tag_spin(sy + e * NW + h, io->stag, wy[k][h], a.bar,
                                a.status, a.timeout_ns);
        }
        sm[o.sSX + e] = tag_value<W>(wx[k]);
        if (!half) sm[o.sSY + e] = tag_value<W>(wy[k]);
      }
    }
    if (__syncthreads_or(!ok)) return false;
    // M = SX + At Yt^T
    for (int e = threadIdx.x; e < dr; e += AD_NT)
      M[(e / r) * RP + e % r] += sm[o.sSX + e];
    SYp = sm + o.sSY;
    __syncthreads();
  } else {
    W vy[KS];
    if (!sxy_smem) {
      // SX staged in shared memory before the X Grams; SY^T: loads issued
      // with it, stored after the X Grams loop
      W vx[KS];
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int e = threadIdx.x + k * AD_NT;
        vx[k] = e < dr ? __ldcg(SXp + e) : W(0);
        vy[k] = (!half && e < dr) ? __ldcg(SYp + e) : W(0);
      }
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int e = threadIdx.x + k * AD_NT;
        if (e < dr) sm[o.sSX + e] = vx[k];
      }
      SXp = sm + o.sSX;
      __syncthreads();
    }
    mark(0);
    // M = SX + At Yt^T  (d x RP, At read along its columns from AtT);
    // G = Yt Yt^T + lam I  (r x RP)
    dual_mm<W>({M, AtT, 1, d, YtT, d, W(1), SXp, r, W(0), true},
               {G, YtT, 1, RP, YtT, r, W(1), nullptr, 0, a.lam, true}, RP,
               d, r);
    if (!sxy_smem && !half) {
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int e = threadIdx.x + k * AD_NT;
        if (e < dr) sm[o.sSY + e] = vy[k];
      }
      SYp = sm + o.sSY;
    }
    __syncthreads();
  }
  mark(1);
  // Xt = M (Yt Yt^T + lam I)^-1
  const W* zx = solve_fast<W, RMAX>(Xt, M, T, d, G, Zx, E, F, H, sm + o.v,
                                    sm + o.mx, r, RP, have, a.status, nullptr);
  mark(2);
  if (half) {
    // F, H are next written in the next sweep's solve, after barriers
    if (zx != Zx)
      for (int e = threadIdx.x; e < r * RP; e += AD_NT) Zx[e] = zx[e];
    return true;
  }
  // M = SY^T + At^T Xt (d x RP);  G = Xt^T Xt + phi I;  the new Zx moves
  // home before the Y solve writes F, H
  dual_mm<W>({M, At, 1, d, Xt, d, W(1), SYp, r, W(0), true},
             {G, Xt, 1, RP, Xt, r, W(1), nullptr, 0, a.phi, true}, RP, d, r);
  if (zx != Zx)
    for (int e = threadIdx.x; e < r * RP; e += AD_NT) Zx[e] = zx[e];
  __syncthreads();
  mark(3);
  // Yt^T = M (Xt^T Xt + phi I)^-1 = (G^-1 MY)^T, G symmetric; a non-finite
  // entry of Yt (the chain's last link) flags CNMF_E_NONFINITE
  bool bad = false;
  const W* zy = solve_fast<W, RMAX>(YtT, M, T, d, G, Zy, E, F, H, sm + o.v,
                                    sm + o.mx, r, RP, have, a.status, &bad);
  if (bad) set_status(a.status, CNMF_E_NONFINITE);
  mark(4);
  // the last solve phase ended with a block barrier; Zy, F, H and YtT are
  // next written or read after further barriers
  if (zy != Zy)
    for (int e = threadIdx.x; e < r * RP; e += AD_NT) Zy[e] = zy[e];
  if (io && io->yout)
    for (int e = threadIdx.x; e < d * RP; e += AD_NT)
      tag_put<W>(io->yout + (size_t)e * (sizeof(W) / 4), YtT[e], io->yotag);
  mark(5);
  return true;
}

// Rows of `side` (0: U / L rows, 1 and 2: V / R^T rows) that CTA c of G
// owns: part c of G, or with the U/V split (a.Gu > 0) part c of Gu on the
// U side and part c - Gu of G - Gu on the V side (false: none).
template <typename W>
__device__ __forceinline__ bool side_rows(const AdmmArgs<W>& a, int side,
                                          int64_t G, int64_t c, int64_t& i0,
                                          int64_t& i1) {
  const bool vside = side > 0;
  const int64_t tot = vside ? a.n : a.m;
  int64_t gg = G, cc = c;
  if (a.Gu > 0) {
    if (vside != (c >= a.Gu)) return false;
    gg = vside ? G - a.Gu : a.Gu;
    cc = vside ? c - a.Gu : c;
  }
  i0 = (cc * tot) / gg;
  i1 = ((cc + 1) * tot) / gg;
  return true;
}

// Thread (l, b): column b of Xt (U side) or Yt^T (V side) in registers;
// rows l, l + nl, ... of this CTA; shares accumulated in registers and
// added over lanes in lane order.  mode 0: fresh setup (Lam = Phi = 0,
// shares of lam U and phi V, plus Yt0^T = R V^T); mode 1: resume setup;
// mode 2: ADMM row updates.
// This CTA is part c of G splitting the rows; its shares go to dst
// (3 d r entries: SX, SY^T, Yt0^T), or with tdst as tagged words (tag) to
// tdst (2 d r values: SX, SY^T).
template <typename W, int DMAX, bool RES>
__device__ void sweep_fast(const AdmmArgs<W>& a, W* sm, const FastSmem& o,
                           int mode, uint64_t* sub, int64_t G, int64_t c,
                           W* dst, uint64_t* tdst = nullptr,
                           uint32_t tag = 0) {
  uint64_t tm = sub ? globaltimer_ns() : 0;
  auto mark = [&](int i) {
    if (sub) { uint64_t t = globaltimer_ns(); sub[i] += t - tm; tm = t; }
  };
  const int r = a.r, d = a.d, dp = o.dp, RP = o.RP, nl = o.nl;
  const int b = threadIdx.x % r, lr = threadIdx.x / r;
  const bool active = lr < nl;
  const int dr = d * r;
  W* Red = sm + o.Red;
  for (int side = 0; side < 2 + (mode == 0 ? 1 : 0); ++side) {
    const bool vside = side > 0;
    int64_t i0, i1;
    if (!side_rows(a, side, G, c, i0, i1)) continue;   // uniform per CTA
    const W* rows = RES ? sm + (vside ? o.sRt : o.sL) : (vside ? a.Rt : a.L);
    const int64_t rstride = RES ? dp : d;
    W* P = RES ? sm + (vside ? o.sVt : o.sU) : (vside ? a.Vt : a.U);
    W* Qm = RES ? sm + (vside ? o.sPhit : o.sLam) : (vside ? a.Phit : a.Lam);
    const int64_t pbase = RES ? 0 : i0;
    const W pen = vside ? a.phi : a.lam;
    const W ipen = W(1) / pen;
    const W step = a.xi * pen;
    const W* coefsrc = sm + (vside ? o.YtT : o.Xt);
    W coef[DMAX], acc[DMAX];
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
      acc[k] = W(0);
      coef[k] = (mode == 2 && k < d) ? coefsrc[k * RP + b] : W(0);
    }
    if (active) {
      for (int64_t i = i0 + lr; i < i1; i += nl) {
        const W* row = rows + (i - i0 + (RES ? 0 : i0)) * rstride;
        const int64_t g = (i - i0 + pbase) * r + b;
        W x[DMAX];
        if constexpr (RES) {
#pragma unroll
          for (int k = 0; k < DMAX; k += 4) ldsN<4, W>(row + k, x + k);
        } else {
#pragma unroll
          for (int k = 0; k < DMAX; ++k) x[k] = k < d ? row[k] : W(0);
        }
        W w;
        if (side == 2) {
          w = P[g];                                  // Yt0^T = R V^T
        } else if (mode == 2) {
          W t4[4] = {W(0), W(0), W(0), W(0)};
#pragma unroll
          for (int k = 0; k < DMAX; ++k) t4[k & 3] = fma(x[k], coef[k], t4[k & 3]);
          const W t = (t4[0] + t4[1]) + (t4[2] + t4[3]);
          const W qo = Qm[g];
          W u = fma(qo, ipen, t);
          u = u > W(0) ? u : W(0);
          const W qn = fma(step, t - u, qo);
          P[g] = u;
          Qm[g] = qn;
          w = fma_rn<W>(pen, u, -qn);
        } else if (mode == 0) {
          Qm[g] = W(0);
          w = fma_rn<W>(pen, P[g], -W(0));
        } else {
          w = fma_rn<W>(pen, P[g], -Qm[g]);
        }
#pragma unroll
        for (int k = 0; k < DMAX; ++k) acc[k] = fma(x[k], w, acc[k]);
      }
#pragma unroll
      for (int k = 0; k < DMAX; ++k)
        if (k < d) Red[lr * dr + k * r + b] = acc[k];
    }
    __syncthreads();
    if (side < 2) mark(2 * side);
    // lane sums in lane order; the loads are issued before the adds
    for (int e = threadIdx.x; e < dr; e += AD_NT) {
      W v[AD_NT / 4];   // nl <= AD_NT / r; r >= 4 keeps this in bounds
      W t = W(0);
      int l = 0;
      for (; l + 8 <= nl; l += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = Red[(l + u) * dr + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) t += v[u];
      }
      for (; l < nl; ++l) t += Red[l * dr + e];
      if (tdst)
        tag_put<W>(tdst + (size_t)(side * dr + e) * (sizeof(W) / 4), t, tag);
      else
        dst[side * dr + e] = t;
    }
    __syncthreads();
    if (side < 2) mark(2 * side + 1);
  }
}

template <typename W>
__device__ void fast_resident_copy(const AdmmArgs<W>& a, W* sm,
                                   const FastSmem& o, int dir) {
  const int r = a.r, d = a.d, dp = o.dp;  // rows padded with zeros to dp
  const int64_t G = gridDim.x, c = blockIdx.x;
  for (int side = 0; side < 2; ++side) {
    int64_t i0, i1;
    if (!side_rows(a, side, G, c, i0, i1)) continue;
    const int64_t nr = i1 - i0;
    W* rs = sm + (side ? o.sRt : o.sL);
    const W* rg = side ? a.Rt : a.L;
    W* ps = sm + (side ? o.sVt : o.sU);
    W* pg = side ? a.Vt : a.U;
    W* qs = sm + (side ? o.sPhit : o.sLam);
    W* qg = side ? a.Phit : a.Lam;
    if (dir == 0) {
      for (int64_t e = threadIdx.x; e < nr * dp; e += AD_NT) {
        const int64_t ii = e / dp;
        const int k = (int)(e % dp);
        rs[e] = k < d ? rg[(i0 + ii) * d + k] : W(0);
      }
      for (int64_t e = threadIdx.x; e < nr * r; e += AD_NT) {
        ps[e] = pg[i0 * r + e];
        qs[e] = qg[i0 * r + e];
      }
    } else {
      for (int64_t e = threadIdx.x; e < nr * r; e += AD_NT) {
        pg[i0 * r + e] = ps[e];
        qg[i0 * r + e] = qs[e];
      }
    }
  }
  __syncthreads();
}

// Cross-CTA sums (one warp per entry, fixed order).  Entries: SX (d x r),
// SY^T (d x r) and, on a fresh start, Yt0^T (d x r), which is stored to the
// state as Yt (r x d).
template <typename W>
__device__ void reduce_fast(const AdmmArgs<W>& a, int with_y0) {
  const int dr = a.d * a.r;
  const int E = 2 * dr + (with_y0 ? dr : 0);
  const int64_t G = gridDim.x, c = blockIdx.x;
  const int e0 = (int)((c * E) / G), e1 = (int)(((c + 1) * E) / G);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int e = e0 + warp; e < e1; e += AD_NT / 32) {
    const W* p = a.part + e;
    // the CTAs holding rows of this entry's side
    int64_t gs = 0, ge = G;
    if (a.Gu > 0) {
      if (e < dr) ge = a.Gu;
      else gs = a.Gu;
    }
    // all of this lane's partials in flight at once (8 * 32 CTAs per
    // round), then added in CTA order
    W s = W(0);
    for (int64_t g0 = gs; g0 < ge; g0 += 8 * 32) {
      W v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t g = g0 + lane + 32 * j;
        v[j] = g < ge ? __ldcg(p + (size_t)g * 3 * dr) : W(0);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) s += v[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (e < dr) a.SX[e] = s;
      else if (e < 2 * dr) a.SY[e - dr] = s;
      else {
        const int k = (e - 2 * dr) / a.r, bb = (e - 2 * dr) % a.r;
        a.Yt[bb * a.d + k] = s;
      }
    }
  }
}

// The sweep loop's cross-CTA sums: this CTA's slice of the 2 d r entries
// (SX, then SY^T), one warp per entry, each summed in CTA order over the
// CTAs holding rows of its side, from sweep it's tagged shares P_it (tag
// it + 1, buffer it & 1) -- each load waits for its tag, so no grid barrier
// is needed -- and stored as the reduced shares S_it+1 (tag it + 2, buffer
// (it + 1) % 3).
// Buffer reuse.  Every CTA of sweep k + 1 waits (directly, or on the U side
// through the lead's Yt_k+1) for all of S_k+1, so for every reducer's
// reading of P_k: two share buffers suffice.  The U side can run one sweep
// ahead of a V-side CTA (it waits for the lead only), so S_it+1's SX part
// may be written while that CTA still reads S_it-1: three buffers of S.
// Returns false when a wait gave up.
template <typename W>
__device__ bool reduce_tagged(const AdmmArgs<W>& a, int it) {
  constexpr int NW = sizeof(W) / 4;
  const int dr = a.d * a.r, E = 2 * dr;
  const int64_t G = gridDim.x, c = blockIdx.x;
  const int e0 = (int)((c * E) / G), e1 = (int)(((c + 1) * E) / G);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const uint32_t tin = (uint32_t)it + 1, tout = (uint32_t)it + 2;
  const uint64_t* part = a.tpart + (size_t)(it & 1) * G * E * NW;
  uint64_t* out = a.tsxy + (size_t)((it + 1) % 3) * E * NW;
  const uint64_t dummy = (uint64_t)tin << 32;
  bool ok = true;
  for (int e = e0 + warp; e < e1; e += AD_NT / 32) {
    int64_t gs = 0, ge = G;
    if (a.Gu > 0) {
      if (e < dr) ge = a.Gu;
      else gs = a.Gu;
    }
    W s = W(0);
    for (int64_t g0 = gs; g0 < ge; g0 += 8 * 32) {
      uint64_t w[8][NW];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t g = g0 + lane + 32 * j;
#pragma unroll
        for (int h = 0; h < NW; ++h)
          w[j][h] = g < ge ? ld_relaxed_u64(part + ((size_t)g * E + e) * NW + h)
                           : dummy;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t g = g0 + lane + 32 * j;
        if (g < ge) {
#pragma unroll
          for (int h = 0; h < NW; ++h)
            ok = ok && tag_spin(part + ((size_t)g * E + e) * NW + h, tin,
                                w[j][h], a.bar, a.status, a.timeout_ns);
          s += tag_value<W>(w[j]);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (__all_sync(0xffffffffu, ok) && lane == 0)
      tag_put<W>(out + (size_t)e * NW, s, tout);
  }
  return !__syncthreads_or(!ok);
}

template <typename W, int DMAX, int RMAX, bool RES>
__global__ void __launch_bounds__(AD_NT) k_admm_fast(AdmmArgs<W> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sm = reinterpret_cast<W*>(smem_raw);
  const FastSmem o(a.r, a.d, RES, a.mu, a.nv, DMAX, a.Gu > 0);
  const int r = a.r, d = a.d, RP = o.RP;
  // with the U/V split: U-side CTAs stop after the X update; the first
  // V-side CTA (which has everything) publishes Yt^T, keeps the state and
  // is the one profiled
  const bool uside = a.Gu > 0 && (int)blockIdx.x < a.Gu;
  const int lead = a.Gu > 0 ? a.Gu : 0;
  const size_t ypsz = (size_t)d * RP;
  // profiled: the lead (sub-steps too) and, with the split, U-side CTA 0
  const bool prof = a.phase_ns && (int)blockIdx.x == lead && threadIdx.x == 0;
  const bool profu = a.phase_ns && a.Gu > 0 && blockIdx.x == 0 &&
                     threadIdx.x == 0 && a.phase_ns_len >= 20;
  // with room for it, every CTA's time in the small algebra, the row sweep
  // and the reduction
  const bool profc = a.phase_ns && threadIdx.x == 0 &&
                     a.phase_ns_len >= 20 + 3 * (int)gridDim.x;
  const bool pr = prof || profu || profc;
  uint64_t tw = 0, tr = 0, tb = 0;
  uint64_t tph[5] = {0, 0, 0, 0, 0};
  uint64_t tsub[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int e = threadIdx.x; e < d * d; e += AD_NT) {
    const W v = a.At[e];
    sm[o.At + e] = v;
    sm[o.AtT + (e % d) * d + e / d] = v;
  }
  for (int e = threadIdx.x; e < d * RP; e += AD_NT) {
    sm[o.YtT + e] = W(0);
    sm[o.Xt + e] = W(0);
  }
  if (RES) fast_resident_copy<W>(a, sm, o, 0);
  __syncthreads();

  // this CTA's tagged words start at tag 0 (no sweep uses it), so nothing
  // left by an earlier launch can pass for this launch's data; the setup's
  // grid barriers order the zeroing before every tagged read
  constexpr int NW = sizeof(W) / 4;
  const int E2 = 2 * d * r;
  const size_t cw = (size_t)E2 * NW;   // one CTA's shares, one parity
  for (int par = 0; par < 2; ++par)
    for (size_t e = threadIdx.x; e < cw; e += AD_NT)
      a.tpart[((size_t)par * gridDim.x + blockIdx.x) * cw + e] = 0;
  if (blockIdx.x == 0) {
    for (size_t e = threadIdx.x; e < 3 * cw; e += AD_NT) a.tsxy[e] = 0;
    for (size_t e = threadIdx.x; e < 2 * ypsz * NW; e += AD_NT) a.typ[e] = 0;
  }
  sweep_fast<W, DMAX, RES>(a, sm, o, a.resume ? 1 : 0, nullptr, gridDim.x,
                           blockIdx.x, a.part + (size_t)blockIdx.x * 3 * d * r);
  if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;
  reduce_fast<W>(a, a.resume ? 0 : 1);
  if (!grid_barrier(a.bar, a.status, a.timeout_ns)) return;
  for (int e = threadIdx.x; e < d * r; e += AD_NT) {
    const int k = e / r, bb = e % r;
    sm[o.YtT + k * RP + bb] = __ldcg(a.Yt + bb * d + k);
  }
  // a resumed run continues from the inverses the last launch kept
  const bool have0 = a.resume && __ldcg(a.kcount) > 0;
  if (have0) load_inverses<W>(a.Zs, r, RP, sm + o.Zx, sm + o.Zy);
  __syncthreads();
  // Sweep it reads the reduced shares S_it (sweep 0: a.SX, a.SY from the
  // setup; then tag it + 1, buffer it % 3) and, on the U side, Yt_it (tag
  // it, buffer it & 1, published by the lead in sweep it - 1); it writes
  // its shares P_it (tag it + 1, buffer it & 1), its slice of S_it+1 and,
  // on the lead, Yt_it+1.  A U-side CTA's reading of Yt_it ends before the
  // lead writes Yt_it+2: the lead waits for S_it+1, made from P_it.
  for (int it = 0; it < a.iters; ++it) {
    uint64_t t0 = pr ? globaltimer_ns() : 0;
    SweepIO io;
    io.sxy = it > 0 ? a.tsxy + (size_t)(it % 3) * cw : nullptr;
    io.stag = (uint32_t)it + 1;
    io.yin = (uside && it > 0) ? a.typ + (size_t)(it & 1) * ypsz * NW : nullptr;
    io.ytag = (uint32_t)it;
    io.yout = (a.Gu > 0 && (int)blockIdx.x == lead)
                  ? a.typ + (size_t)((it + 1) & 1) * ypsz * NW : nullptr;
    io.yotag = (uint32_t)it + 1;
    if (!small_fast<W, DMAX, RMAX>(a, sm, o, have0 || it > 0,
                                   prof ? tsub : nullptr, nullptr, nullptr,
                                   false, uside, &io))
      return;
    uint64_t t1 = pr ? globaltimer_ns() : 0;
    sweep_fast<W, DMAX, RES>(
        a, sm, o, 2, prof ? tsub + 6 : nullptr, gridDim.x, blockIdx.x, nullptr,
        a.tpart + ((size_t)(it & 1) * gridDim.x + blockIdx.x) * cw,
        (uint32_t)it + 1);
    uint64_t t2 = pr ? globaltimer_ns() : 0;
    if (!reduce_tagged<W>(a, it)) return;
    if (pr) {
      uint64_t t3 = globaltimer_ns();
      tw += t1 - t0; tr += t2 - t1; tb += t3 - t2;
      tph[0] += t1 - t0; tph[1] += t2 - t1; tph[2] += t3 - t2;
    }
  }
  if (RES) fast_resident_copy<W>(a, sm, o, 1);
  if ((int)blockIdx.x == lead) {
    for (int e = threadIdx.x; e < d * r; e += AD_NT) {
      const int k = e / r, bb = e % r;
      a.Yt[bb * d + k] = sm[o.YtT + k * RP + bb];
      if (a.iters > 0) a.Xt[e] = sm[o.Xt + k * RP + bb];
    }
    if (a.iters > 0) store_inverses<W>(a.Zs, r, RP, sm + o.Zx, sm + o.Zy);
    if (threadIdx.x == 0) *a.kcount += a.iters;
  }
  if (prof) {
    for (int i = 0; i < 5; ++i) a.phase_ns[i] += (double)tph[i];
    const int ns = a.phase_ns_len - 5 < 10 ? a.phase_ns_len - 5 : 10;
    for (int i = 0; i < ns; ++i) a.phase_ns[5 + i] += (double)tsub[i];
  }
  if (profu)
    for (int i = 0; i < 5; ++i) a.phase_ns[15 + i] += (double)tph[i];
  if (profc) {
    a.phase_ns[20 + 3 * blockIdx.x] += (double)tw;
    a.phase_ns[21 + 3 * blockIdx.x] += (double)tr;
    a.phase_ns[22 + 3 * blockIdx.x] += (double)tb;
  }
}

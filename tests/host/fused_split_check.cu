// Host-only check of the fused sketch pass's work split and partial-slot
// layout (the helpers of fused.cu compiled for the host, no device code
// runs): every tile has exactly one owner CTA whose range holds it, ranges
// tile the whole grid in order, every partial slot a CTA writes is unique
// and inside the workspace the plan reserves, and every slot the sum
// kernel lists for an output tile is one that was written.  Prints
// "ok <cases>" or the first violation.
#include "../../paper_1505_04650_gb300/csrc/fused.cu"

#include <cstdio>
#include <set>
#include <vector>

namespace cnmf {
int num_sms() { return 152; }
bool ensure_max_smem(const void*, size_t) { return false; }
void record_cuda_error(cudaError_t, const char*, int) {}
bool pdl_enabled() { return false; }
}  // namespace cnmf

using namespace cnmf;

static int fail(const char* what, long long a, long long b) {
  std::printf("FAIL %s %lld %lld\n", what, a, b);
  return 1;
}

static int check(int64_t m, int64_t n, int k, bool hx, bool hy, int G0) {
  FuGeom q{};
  q.has_x = hx;
  q.has_y = hy;
  q.TI = (int)ceil_div(m, FU_T);
  q.TJ = (int)ceil_div(n, FU_T);
  q.U = (int64_t)q.TI * q.TJ;
  const int KP = k <= 16 ? 16 : 32;
  q.z2col = hx ? 4 * KP : 0;
  q.Tj = std::min({hy ? (512 - q.z2col) / KP : 8, 16, q.TJ});
  q.NG = (int)ceil_div(q.TJ, q.Tj);
  q.wlast = q.TJ - (q.NG - 1) * q.Tj;
  q.G = (int)std::min<int64_t>(q.U, G0);
  if (fu_start(q, 0) != 0 || fu_start(q, q.G) != q.U)
    return fail("ends", fu_start(q, 0), fu_start(q, q.G));
  const int64_t gfull = (int64_t)q.TI * q.Tj;
  std::set<int64_t> s1, s2;
  for (int c = 0; c < q.G; ++c) {
    const int64_t a = fu_start(q, c), b = fu_start(q, c + 1);
    if (b <= a) return fail("empty range", c, a);
    for (int64_t u = a; u < b; ++u) {
      if (fu_owner(q, u) != c) return fail("owner", u, c);
      const int g = (int)std::min<int64_t>(u / gfull, q.NG - 1);
      const int64_t r = u - fu_gs(q, g);
      const int i = (int)(r / fu_w(q, g));
      // A X: one piece slot per (segment, CTA); A^T Y: (group + CTA) Tj + jl
      if (hx) s1.insert(((int64_t)g * q.TI + i) + c);
      if (hy) s2.insert((int64_t)g + c);
    }
  }
  // uniqueness of the slot indices written: a (segment, CTA) pair maps to
  // seg + c, which must not collide with another pair's
  std::set<std::pair<int64_t, int>> p1, p2;
  for (int c = 0; c < q.G; ++c)
    for (int64_t u = fu_start(q, c); u < fu_start(q, c + 1); ++u) {
      const int g = (int)std::min<int64_t>(u / gfull, q.NG - 1);
      const int i = (int)((u - fu_gs(q, g)) / fu_w(q, g));
      p1.insert({(int64_t)g * q.TI + i, c});
      p2.insert({(int64_t)g, c});
    }
  std::set<int64_t> idx1, idx2;
  for (auto& e : p1) {
    const int64_t sl = e.first + e.second;
    if (!idx1.insert(sl).second) return fail("P1 clash", e.first, e.second);
    if (sl >= (int64_t)q.TI * q.NG + q.G) return fail("P1 range", sl, 0);
  }
  for (auto& e : p2) {
    const int64_t sl = e.first + e.second;
    if (!idx2.insert(sl).second) return fail("P2 clash", e.first, e.second);
    if (sl >= q.NG + q.G) return fail("P2 range", sl, 0);
  }
  // the sum kernel's lists: row tile t takes, per group, the owners of its
  // segment; column tile (g, jl) the owners of the group's tiles
  if (hx)
    for (int t = 0; t < q.TI; ++t)
      for (int g = 0; g < q.NG; ++g) {
        const int w = fu_w(q, g);
        const int64_t ua = fu_gs(q, g) + (int64_t)t * w;
        const int ca = fu_owner(q, ua), cb = fu_owner(q, ua + w - 1);
        for (int c = ca; c <= cb; ++c)
          if (!p1.count({(int64_t)g * q.TI + t, c}))
            return fail("row list", t, c);
      }
  if (hy)
    for (int g = 0; g < q.NG; ++g) {
      const int64_t gs = fu_gs(q, g), ge = gs + (int64_t)q.TI * fu_w(q, g) - 1;
      for (int c = fu_owner(q, gs); c <= fu_owner(q, ge); ++c)
        if (!p2.count({(int64_t)g, c})) return fail("col list", g, c);
    }
  return 0;
}

int main() {
  const int64_t sizes[][2] = {{20000, 10000}, {10000, 100000}, {300, 200},
                              {128, 128},     {129, 4000},     {4000, 129},
                              {1, 1},         {200, 70000},    {20000, 3000},
                              {1000, 1000},   {128, 256000},   {50000, 300}};
  int cases = 0;
  for (auto& z : sizes)
    for (int k : {8, 30})
      for (int sd = 1; sd <= 3; ++sd)
        for (int G0 : {152, 76, 48, 7, 1}) {
          if (check(z[0], z[1], k, sd & 1, sd & 2, G0)) {
            std::printf("case m=%lld n=%lld k=%d sides=%d G=%d\n",
                        (long long)z[0], (long long)z[1], k, sd, G0);
            return 1;
          }
          ++cases;
        }
  std::printf("ok %d\n", cases);
  return 0;
}

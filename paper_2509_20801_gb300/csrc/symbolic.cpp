// Geometric nested dissection of a strip's local node box (host side).
// See symbolic.h for the construction; Sec. 2.4 / Eq. 22 of the paper.
#include "symbolic.h"

#include <stdexcept>
#include <string>

namespace stdd {
namespace {

struct Builder {
  Shape &S;
  int W, H, leaf;
  std::vector<int> pos;  // node -> index inside the front being linked, else -1

  Builder(Shape &s, int w, int h, int l) : S(s), W(w), H(h), leaf(l), pos((size_t)w * h, -1) {}

  int build(int x0, int x1, int y0, int y1, int level) {
    if (x1 <= x0 || y1 <= y0) return -1;
    const int w = x1 - x0, h = y1 - y0;
    std::vector<int> piv;
    int c0 = -1, c1 = -1;
    if ((long long)w * h <= leaf) {
      piv.reserve((size_t)w * h);
      for (int x = x0; x < x1; ++x)
        for (int y = y0; y < y1; ++y) piv.push_back(x * H + y);
    } else if (h >= w) {  // cut the longer (y) side by the middle node row
      const int ys = y0 + h / 2;
      c0 = build(x0, x1, y0, ys, level + 1);
      c1 = build(x0, x1, ys + 1, y1, level + 1);
      for (int x = x0; x < x1; ++x) piv.push_back(x * H + ys);
    } else {              // cut the longer (x) side by the middle node column
      const int xs = x0 + w / 2;
      c0 = build(x0, xs, y0, y1, level + 1);
      c1 = build(xs + 1, x1, y0, y1, level + 1);
      for (int y = y0; y < y1; ++y) piv.push_back(xs * H + y);
    }
    // ring: 5-point neighbours of the box that lie outside it
    std::vector<int> ring;
    if (y0 > 0)
      for (int x = x0; x < x1; ++x) ring.push_back(x * H + (y0 - 1));
    if (y1 < H)
      for (int x = x0; x < x1; ++x) ring.push_back(x * H + y1);
    if (x0 > 0)
      for (int y = y0; y < y1; ++y) ring.push_back((x0 - 1) * H + y);
    if (x1 < W)
      for (int y = y0; y < y1; ++y) ring.push_back(x1 * H + y);

    SymFront f;
    f.p = (int)piv.size();
    f.b = (int)ring.size();
    f.level = level;
    f.child[0] = c0;
    f.child[1] = c1;
    f.node_off = (int64_t)S.nodes.size();
    S.nodes.insert(S.nodes.end(), piv.begin(), piv.end());
    S.nodes.insert(S.nodes.end(), ring.begin(), ring.end());
    const int id = (int)S.fronts.size();
    const int n = f.p + f.b;
    for (int k = 0; k < n; ++k) pos[S.nodes[f.node_off + k]] = k;
    for (int ci = 0; ci < 2; ++ci) {
      const int c = f.child[ci];
      if (c < 0) continue;
      SymFront &ch = S.fronts[c];
      ch.parent = id;
      f.cmap_off[ci] = (int64_t)S.cmap.size();
      f.inv_off[ci] = (int64_t)S.inv.size();
      S.inv.insert(S.inv.end(), (size_t)n, -1);
      const int chn = ch.p + ch.b;
      for (int k = 0; k < ch.b; ++k) {
        const int node = S.nodes[ch.node_off + ch.p + k];
        const int at = pos[node];
        if (at < 0) throw std::logic_error("nested dissection: child ring node outside parent front");
        S.cmap.push_back(at);
        S.inv[f.inv_off[ci] + at] = k;
      }
      (void)chn;
    }
    for (int k = 0; k < n; ++k) pos[S.nodes[f.node_off + k]] = -1;
    S.fronts.push_back(f);
    return id;
  }
};

}  // namespace

void nd_analyze(int W, int H, int leaf_max, Shape &S) {
  if (W < 1 || H < 1 || leaf_max < 1) throw std::invalid_argument("nd_analyze: bad box");
  S = Shape();
  S.W = W;
  S.H = H;
  S.leaf_max = leaf_max;
  Builder B(S, W, H, leaf_max);
  B.build(0, W, 0, H, 0);
  int64_t off = 0;
  for (auto &f : S.fronts) {
    f.fac_off = off;
    const int64_t p = f.p, b = f.b, n = p + b;
    off += p * (p + 2 * b);
    // Gauss-Jordan sweep of p pivots over the whole n x n front
    S.factor_cflops += double(p) * double(n) * double(n);
    // LU count: pivot k updates the (n-k-1)^2 trailing block, sum of m^2 for m = b .. n-1
    auto sq = [](double x) { return x * (x + 1) * (2 * x + 1) / 6.0; };
    S.factor_cflops_lu += sq(double(n - 1)) - sq(double(b - 1));
    S.solve_cflops += double(p) * double(p) + 2.0 * double(p) * double(b);
    if (f.level + 1 > S.depth) S.depth = f.level + 1;
    if (f.p > S.max_p) S.max_p = f.p;
    if (f.b > S.max_b) S.max_b = f.b;
  }
  S.factor_entries = off;
}

}  // namespace stdd

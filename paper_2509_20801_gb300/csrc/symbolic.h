// Nested-dissection symbolic analysis of one strip's local box (host).
//
// Sec. 2.4 of the paper factors every local matrix as A = P^T L U Q^T with
// fill-reducing permutations (Eq. 22).  Here the permutation is geometric
// nested dissection of the W x H node box (Lipton-Rose-Tarjan): a box whose
// node count exceeds `leaf_max` is cut by its middle node line across the
// longer side; the line is a separator front whose pivots are the line's
// nodes and whose border is the ring of nodes just outside the box (5-point
// neighbours only).  Leaf boxes are fronts that eliminate all their nodes.
// Because of the 5-point stencil the ring of a child box lies in its
// parent's separator plus the parent's ring, which gives the extend-add maps.
#pragma once
#include <cstdint>
#include <vector>

namespace stdd {

struct SymFront {
  int p = 0;            // pivots (separator or leaf nodes)
  int b = 0;            // border (ring) nodes
  int level = 0;        // depth from the root
  int parent = -1;
  int child[2] = {-1, -1};
  int64_t node_off = 0; // nodes[node_off .. +p+b): pivots then ring; node = x*H + y
  int64_t cmap_off[2] = {-1, -1};  // child ring index -> this front's index (b_child ints)
  int64_t inv_off[2] = {-1, -1};   // this front's index -> child ring index or -1 (p+b ints)
  int64_t fac_off = 0;  // complex entries before this front in the strip's factor block
};

struct Shape {
  int W = 0, H = 0, leaf_max = 0;
  std::vector<SymFront> fronts;     // elimination order: children before parents
  std::vector<int> nodes;
  std::vector<int> cmap;
  std::vector<int> inv;
  int depth = 0;                    // number of levels
  int64_t factor_entries = 0;       // sum p*(p + 2b)
  double factor_cflops = 0;         // complex multiply-adds of the factorization (sum p n^2)
  double factor_cflops_lu = 0;      // the same elimination counted as LU: sum over pivots of
                                    // the trailing block, (n-k-1)^2 for pivot k
  double solve_cflops = 0;          // complex multiply-adds of one fwd+bwd solve
  int max_p = 0, max_b = 0;
};

// Builds the analysis for a W x H box.  Throws std::invalid_argument on bad sizes.
void nd_analyze(int W, int H, int leaf_max, Shape &out);

}  // namespace stdd

// Global-grid kernels of the hot path: the matrix-free stretched 5-point
// operator (Eq. 2 with the PML stretching of Eq. 9), the residual, the
// restriction of a global field to every strip's owned columns (R_i^I) and
// the synthesis of the strips' full local fields (sum_i E_i, Eq. 21).
//
// Fields are complex128 interleaved, node g = i*ny + j (y fastest), so a
// strip's local box is one contiguous slice of the global vector: restriction
// and synthesis are coalesced copies.  One thread per node, grid-stride; the
// x-neighbours at g +- ny are one grid row away and come from L2.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace stdd {

long long g_launches = 0;

namespace {

constexpr int TPB = 256;

inline int grid_for(int64_t n) {
  return (int)std::min<int64_t>((n + TPB - 1) / TPB, 152 * 16);
}

__device__ __forceinline__ double2 apply_row_ij(const GridDev &g, const double2 *__restrict__ x, int64_t idx, int i,
                                                int j) {
  return grid_row(g, x, idx, i, j);
}

__device__ __forceinline__ double2 apply_row(const GridDev &g, const double2 *__restrict__ x, int64_t idx) {
  const int i = (int)(idx / g.ny), j = (int)(idx - (int64_t)i * g.ny);
  return apply_row_ij(g, x, idx, i, j);
}

// grid-stride walk over all nodes with (i, j) advanced incrementally (no
// division per node): f(idx, i, j) for every node of this thread
template <typename F> __device__ __forceinline__ void for_nodes(const GridDev &g, F f) {
  const int64_t n = (int64_t)g.nx * g.ny, stride = (int64_t)gridDim.x * TPB;
  int64_t idx = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (idx >= n) return;
  int i = (int)(idx / g.ny), j = (int)(idx - (int64_t)i * g.ny);
  const int si = (int)(stride / g.ny), sj = (int)(stride - (int64_t)si * g.ny);
  for (; idx < n; idx += stride) {
    f(idx, i, j);
    i += si;
    j += sj;
    if (j >= g.ny) {
      j -= g.ny;
      ++i;
    }
  }
}

__global__ void __launch_bounds__(TPB) k_stencil(GridDev g, const double2 *__restrict__ x, double2 *__restrict__ y) {
  for_nodes(g, [&](int64_t idx, int i, int j) { y[idx] = apply_row_ij(g, x, idx, i, j); });
}

__global__ void __launch_bounds__(TPB) k_residual(GridDev g, const double2 *__restrict__ b,
                                                  const double2 *__restrict__ x, double2 *__restrict__ r) {
  for_nodes(g, [&](int64_t idx, int i, int j) { r[idx] = csub(b[idx], apply_row_ij(g, x, idx, i, j)); });
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_restrict(const StripDev *__restrict__ strips, int ny,
                                                  const double2 *__restrict__ v, void *tloc) {
  using C = typename CT<R>::T;
  const StripDev s = strips[blockIdx.y];
  const int64_t nl = (int64_t)(s.x1 - s.x0) * ny;
  const int64_t lo = (int64_t)(s.c0 - s.x0) * ny, hi = (int64_t)(s.c1 - s.x0) * ny;
  C *t = reinterpret_cast<C *>(tloc) + s.vec_off;
  const double2 *vs = v + (int64_t)s.x0 * ny;
  for (int64_t l = (int64_t)blockIdx.x * TPB + threadIdx.x; l < nl; l += (int64_t)gridDim.x * TPB)
    t[l] = (l >= lo && l < hi) ? to_c(vs[l], C()) : czero<C>();
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_synthesize(const StripDev *__restrict__ strips, int nsub, int nx,
                                                    int ny, const int *__restrict__ col_strip,
                                                    const void *tloc, double2 *__restrict__ z) {
  using C = typename CT<R>::T;
  const C *t = reinterpret_cast<const C *>(tloc);
  const int64_t n = (int64_t)nx * ny;
  for (int64_t g = (int64_t)blockIdx.x * TPB + threadIdx.x; g < n; g += (int64_t)gridDim.x * TPB) {
    const int i = (int)(g / ny);
    const int k = col_strip[i];
    double2 acc = make_double2(0.0, 0.0);
    for (int kk = max(0, k - 1); kk <= min(nsub - 1, k + 1); ++kk) {
      const StripDev s = strips[kk];
      if (i >= s.x0 && i < s.x1) acc = cadd(acc, to_d(t[s.vec_off + g - (int64_t)s.x0 * ny]));
    }
    z[g] = acc;
  }
}

// 2-D (checkerboard) boxes: local node (lx, ly) of box s is global node
// (x0 + lx, y0 + ly); R_s^I keeps the owned block [c0, c1) x [r0, r1)
template <typename R>
__global__ void __launch_bounds__(TPB) k_restrict_box(const StripDev *__restrict__ boxes, int ny,
                                                      const double2 *__restrict__ v, void *tloc) {
  using C = typename CT<R>::T;
  const StripDev s = boxes[blockIdx.y];
  const int Hl = s.y1 - s.y0;
  const int64_t nl = (int64_t)(s.x1 - s.x0) * Hl;
  C *t = reinterpret_cast<C *>(tloc) + s.vec_off;
  for (int64_t l = (int64_t)blockIdx.x * TPB + threadIdx.x; l < nl; l += (int64_t)gridDim.x * TPB) {
    const int lx = (int)(l / Hl), ly = (int)(l - (int64_t)lx * Hl);
    const int gx = s.x0 + lx, gy = s.y0 + ly;
    t[l] = (gx >= s.c0 && gx < s.c1 && gy >= s.r0 && gy < s.r1) ? to_c(v[(int64_t)gx * ny + gy], C()) : czero<C>();
  }
}

// z = sum_k E_k local[k] over boxes: node (i, j) is covered by at most the
// 3 x 3 boxes around its owner (col_box[i], row_box[j]); summed in box order
// (x-major), each box id kx * py + ky
template <typename R>
__global__ void __launch_bounds__(TPB) k_synthesize_box(const StripDev *__restrict__ boxes, int px, int py, int nx,
                                                        int ny, const int *__restrict__ col_box,
                                                        const int *__restrict__ row_box, const void *tloc,
                                                        double2 *__restrict__ z) {
  using C = typename CT<R>::T;
  const C *t = reinterpret_cast<const C *>(tloc);
  const int64_t n = (int64_t)nx * ny;
  for (int64_t g = (int64_t)blockIdx.x * TPB + threadIdx.x; g < n; g += (int64_t)gridDim.x * TPB) {
    const int i = (int)(g / ny), j = (int)(g - (int64_t)i * ny);
    const int kx = col_box[i], ky = row_box[j];
    double2 acc = make_double2(0.0, 0.0);
    for (int bx = max(0, kx - 1); bx <= min(px - 1, kx + 1); ++bx)
      for (int by = max(0, ky - 1); by <= min(py - 1, ky + 1); ++by) {
        const StripDev s = boxes[bx * py + by];
        if (i >= s.x0 && i < s.x1 && j >= s.y0 && j < s.y1)
          acc = cadd(acc, to_d(t[s.vec_off + (int64_t)(i - s.x0) * (s.y1 - s.y0) + (j - s.y0)]));
      }
    z[g] = acc;
  }
}

// one strip s: t = R_s^I (v - A z) on its local box (zero off the owned
// columns), the source of its local solve in the multiplicative order
template <typename R>
__global__ void __launch_bounds__(TPB) k_restrict_residual_strip(GridDev g, StripDev s, const double2 *__restrict__ v,
                                                                 const double2 *__restrict__ z, void *tloc) {
  using C = typename CT<R>::T;
  const int64_t nl = (int64_t)(s.x1 - s.x0) * g.ny;
  const int64_t lo = (int64_t)(s.c0 - s.x0) * g.ny, hi = (int64_t)(s.c1 - s.x0) * g.ny;
  const int64_t g0 = (int64_t)s.x0 * g.ny;
  C *t = reinterpret_cast<C *>(tloc) + s.vec_off;
  for (int64_t l = (int64_t)blockIdx.x * TPB + threadIdx.x; l < nl; l += (int64_t)gridDim.x * TPB)
    t[l] = (l >= lo && l < hi) ? to_c(csub(v[g0 + l], apply_row(g, z, g0 + l)), C()) : czero<C>();
}

// z += E_s e_s: the strip's full local field added on its local box
template <typename R>
__global__ void __launch_bounds__(TPB) k_add_strip(StripDev s, int ny, const void *tloc, double2 *__restrict__ z) {
  using C = typename CT<R>::T;
  const C *t = reinterpret_cast<const C *>(tloc) + s.vec_off;
  const int64_t nl = (int64_t)(s.x1 - s.x0) * ny;
  double2 *zs = z + (int64_t)s.x0 * ny;
  for (int64_t l = (int64_t)blockIdx.x * TPB + threadIdx.x; l < nl; l += (int64_t)gridDim.x * TPB)
    zs[l] = cadd(zs[l], to_d(t[l]));
}

// ---- band space: vectors on a union of column intervals (first column,
// width); element bi of the band vector <-> global node, the interval found
// by binary search over the element offsets
__device__ __forceinline__ int64_t band_node(int64_t bi, const int2 *__restrict__ iv, const int64_t *__restrict__ off,
                                           int niv, int ny) {
  int lo = 0, hi = niv - 1;  // largest k with off[k] <= bi
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= bi) lo = mid;
    else hi = mid - 1;
  }
  return (int64_t)iv[lo].x * ny + (bi - off[lo]);
}

// every strip's local source R_s^I G(s): the band vector s placed on its
// columns (colband = band offset of a column's first element, -1 off the
// band), kept on the strip's owned columns
template <typename R>
__global__ void __launch_bounds__(TPB) k_restrict_band(const StripDev *__restrict__ strips, int ny,
                                                       const int64_t *__restrict__ colband,
                                                       const double2 *__restrict__ s, void *tloc) {
  using C = typename CT<R>::T;
  const StripDev st = strips[blockIdx.y];
  const int64_t nl = (int64_t)(st.x1 - st.x0) * ny;
  const int64_t lo = (int64_t)(st.c0 - st.x0) * ny, hi = (int64_t)(st.c1 - st.x0) * ny;
  C *t = reinterpret_cast<C *>(tloc) + st.vec_off;
  for (int64_t l = (int64_t)blockIdx.x * TPB + threadIdx.x; l < nl; l += (int64_t)gridDim.x * TPB) {
    C v = czero<C>();
    if (l >= lo && l < hi) {
      const int col = st.x0 + (int)(l / ny);
      const int64_t cb = colband[col];
      if (cb >= 0) v = to_c(s[cb + l % ny], C());
    }
    t[l] = v;
  }
}

// z = sum_k E_k local[k] on the band's columns widened by one (the nodes the
// stencil on the band reads), gather form as k_synthesize
template <typename R>
__global__ void __launch_bounds__(TPB) k_synthesize_band(const StripDev *__restrict__ strips, int nsub, int ny,
                                                         const int *__restrict__ col_strip, const int2 *__restrict__ iv,
                                                         const int64_t *__restrict__ off, int niv, int64_t nb,
                                                         const void *tloc, double2 *__restrict__ z) {
  using C = typename CT<R>::T;
  const C *t = reinterpret_cast<const C *>(tloc);
  for (int64_t bi = (int64_t)blockIdx.x * TPB + threadIdx.x; bi < nb; bi += (int64_t)gridDim.x * TPB) {
    const int64_t g = band_node(bi, iv, off, niv, ny);
    const int i = (int)(g / ny);
    const int k = col_strip[i];
    double2 acc = make_double2(0.0, 0.0);
    for (int kk = max(0, k - 1); kk <= min(nsub - 1, k + 1); ++kk) {
      const StripDev s = strips[kk];
      if (i >= s.x0 && i < s.x1) acc = cadd(acc, to_d(t[s.vec_off + g - (int64_t)s.x0 * ny]));
    }
    z[g] = acc;
  }
}

// y[bi] = +-((A z)(g) - (sub ? sub[g or bi] : 0)) on the band: sub_global
// selects whether sub is a global (1) or a band (0) vector, neg the sign
__global__ void __launch_bounds__(TPB) k_stencil_band(GridDev g, const int2 *__restrict__ iv,
                                                      const int64_t *__restrict__ off, int niv, int64_t nb,
                                                      const double2 *__restrict__ z, const double2 *__restrict__ sub,
                                                      int sub_global, int neg, double2 *__restrict__ y) {
  for (int64_t bi = (int64_t)blockIdx.x * TPB + threadIdx.x; bi < nb; bi += (int64_t)gridDim.x * TPB) {
    const int64_t gi = band_node(bi, iv, off, niv, g.ny);
    double2 v = apply_row(g, z, gi);
    if (sub) v = csub(v, sub[sub_global ? gi : bi]);
    if (neg) v = make_double2(-v.x, -v.y);
    y[bi] = v;
  }
}

// r = a - b (band vectors)
__global__ void __launch_bounds__(TPB) k_vsub(const double2 *__restrict__ a, const double2 *__restrict__ b,
                                              double2 *__restrict__ r, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB)
    r[i] = csub(a[i], b[i]);
}

// band <-> global: y[bi] = x[g] (gather), or x[g] += y[bi] (scatter-add)
__global__ void __launch_bounds__(TPB) k_band_copy(const int2 *__restrict__ iv, const int64_t *__restrict__ off,
                                                   int niv, int64_t nb, int ny, double2 *__restrict__ x,
                                                   double2 *__restrict__ y, int to_band) {
  for (int64_t bi = (int64_t)blockIdx.x * TPB + threadIdx.x; bi < nb; bi += (int64_t)gridDim.x * TPB) {
    const int64_t gi = band_node(bi, iv, off, niv, ny);
    if (to_band) y[bi] = x[gi];
    else x[gi] = cadd(x[gi], y[bi]);
  }
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_to_local(const double2 *__restrict__ v, void *tloc, int64_t n) {
  using C = typename CT<R>::T;
  C *t = reinterpret_cast<C *>(tloc);
  for (int64_t l = (int64_t)blockIdx.x * TPB + threadIdx.x; l < n; l += (int64_t)gridDim.x * TPB)
    t[l] = to_c(v[l], C());
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_from_local(const void *tloc, double2 *__restrict__ z, int64_t n) {
  using C = typename CT<R>::T;
  const C *t = reinterpret_cast<const C *>(tloc);
  for (int64_t l = (int64_t)blockIdx.x * TPB + threadIdx.x; l < n; l += (int64_t)gridDim.x * TPB)
    z[l] = to_d(t[l]);
}

// out[2k] = ||e_k^F||^2 (non-owned columns of strip k), out[2k+1] = ||e_k||^2
template <typename R>
__global__ void __launch_bounds__(TPB) k_strip_norms(const StripDev *__restrict__ strips, int ny,
                                                     const void *tloc, double *__restrict__ out) {
  using C = typename CT<R>::T;
  __shared__ double sh[2][TPB / 32];
  const StripDev s = strips[blockIdx.x];
  const C *t = reinterpret_cast<const C *>(tloc) + s.vec_off;
  const int64_t nl = (int64_t)(s.x1 - s.x0) * ny;
  const int64_t lo = (int64_t)(s.c0 - s.x0) * ny, hi = (int64_t)(s.c1 - s.x0) * ny;
  double f = 0, e = 0;
  for (int64_t l = threadIdx.x; l < nl; l += TPB) {
    const double2 v = to_d(t[l]);
    const double a = v.x * v.x + v.y * v.y;
    e += a;
    if (l < lo || l >= hi) f += a;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f += __shfl_xor_sync(0xffffffffu, f, o);
    e += __shfl_xor_sync(0xffffffffu, e, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = f;
    sh[1][threadIdx.x >> 5] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double fs = 0, es = 0;
    for (int w = 0; w < TPB / 32; ++w) {
      fs += sh[0][w];
      es += sh[1][w];
    }
    out[2 * blockIdx.x] = fs;
    out[2 * blockIdx.x + 1] = es;
  }
}

}  // namespace

template <typename R>
void launch_strip_norms(const StripDev *strips_dev, int nsub, int ny, const void *tloc, double *out,
                        cudaStream_t st) {
  k_strip_norms<R><<<nsub, TPB, 0, st>>>(strips_dev, ny, tloc, out);
  count_launch();
}
template void launch_strip_norms<double>(const StripDev *, int, int, const void *, double *, cudaStream_t);
template void launch_strip_norms<float>(const StripDev *, int, int, const void *, double *, cudaStream_t);

void launch_stencil(const GridDev &g, const double2 *x, double2 *y, cudaStream_t st) {
  k_stencil<<<grid_for((int64_t)g.nx * g.ny), TPB, 0, st>>>(g, x, y);
  count_launch();
}

void launch_residual(const GridDev &g, const double2 *b, const double2 *x, double2 *r, cudaStream_t st) {
  k_residual<<<grid_for((int64_t)g.nx * g.ny), TPB, 0, st>>>(g, b, x, r);
  count_launch();
}

template <typename R>
void launch_restrict(const StripDev *strips_dev, int nsub, int64_t nloc_max, int ny, const int *,
                     const double2 *v, void *tloc, cudaStream_t st) {
  const int gx = (int)std::min<int64_t>((nloc_max + TPB - 1) / TPB, 1024);
  k_restrict<R><<<dim3(gx, nsub), TPB, 0, st>>>(strips_dev, ny, v, tloc);
  count_launch();
}

template <typename R>
void launch_synthesize(const StripDev *strips_dev, int nsub, int nx, int ny, const int *col_strip,
                       const void *tloc, double2 *z, cudaStream_t st) {
  k_synthesize<R><<<grid_for((int64_t)nx * ny), TPB, 0, st>>>(strips_dev, nsub, nx, ny, col_strip, tloc, z);
  count_launch();
}

template <typename R>
void launch_restrict_box(const StripDev *boxes_dev, int nbox, int64_t nloc_max, int ny, const double2 *v, void *tloc,
                         cudaStream_t st) {
  const int gx = (int)std::min<int64_t>((nloc_max + TPB - 1) / TPB, 1024);
  k_restrict_box<R><<<dim3(gx, nbox), TPB, 0, st>>>(boxes_dev, ny, v, tloc);
  count_launch();
}

template <typename R>
void launch_synthesize_box(const StripDev *boxes_dev, int px, int py, int nx, int ny, const int *col_box,
                           const int *row_box, const void *tloc, double2 *z, cudaStream_t st) {
  k_synthesize_box<R><<<grid_for((int64_t)nx * ny), TPB, 0, st>>>(boxes_dev, px, py, nx, ny, col_box, row_box, tloc,
                                                                   z);
  count_launch();
}
template void launch_restrict_box<double>(const StripDev *, int, int64_t, int, const double2 *, void *, cudaStream_t);
template void launch_restrict_box<float>(const StripDev *, int, int64_t, int, const double2 *, void *, cudaStream_t);
template void launch_synthesize_box<double>(const StripDev *, int, int, int, int, const int *, const int *,
                                            const void *, double2 *, cudaStream_t);
template void launch_synthesize_box<float>(const StripDev *, int, int, int, int, const int *, const int *,
                                           const void *, double2 *, cudaStream_t);

template <typename R> void launch_to_local(const double2 *t, void *tloc, int64_t n, cudaStream_t st) {
  k_to_local<R><<<grid_for(n), TPB, 0, st>>>(t, tloc, n);
  count_launch();
}
template <typename R> void launch_from_local(const void *tloc, double2 *z, int64_t n, cudaStream_t st) {
  k_from_local<R><<<grid_for(n), TPB, 0, st>>>(tloc, z, n);
  count_launch();
}

template <typename R>
void launch_restrict_residual_strip(const GridDev &g, const StripDev &s, const double2 *v, const double2 *z,
                                    void *tloc, cudaStream_t st) {
  k_restrict_residual_strip<R><<<grid_for((int64_t)(s.x1 - s.x0) * g.ny), TPB, 0, st>>>(g, s, v, z, tloc);
  count_launch();
}
template <typename R> void launch_add_strip(const StripDev &s, int ny, const void *tloc, double2 *z, cudaStream_t st) {
  k_add_strip<R><<<grid_for((int64_t)(s.x1 - s.x0) * ny), TPB, 0, st>>>(s, ny, tloc, z);
  count_launch();
}
template void launch_restrict_residual_strip<double>(const GridDev &, const StripDev &, const double2 *,
                                                     const double2 *, void *, cudaStream_t);
template void launch_restrict_residual_strip<float>(const GridDev &, const StripDev &, const double2 *,
                                                    const double2 *, void *, cudaStream_t);
template void launch_add_strip<double>(const StripDev &, int, const void *, double2 *, cudaStream_t);
template void launch_add_strip<float>(const StripDev &, int, const void *, double2 *, cudaStream_t);

template <typename R>
void launch_restrict_band(const StripDev *strips_dev, int nsub, int64_t nloc_max, int ny, const int64_t *colband,
                          const double2 *s, void *tloc, cudaStream_t st) {
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((nloc_max + TPB - 1) / TPB, 152 * 4)), nsub);
  k_restrict_band<R><<<grid, TPB, 0, st>>>(strips_dev, ny, colband, s, tloc);
  count_launch();
}
template <typename R>
void launch_synthesize_band(const StripDev *strips_dev, int nsub, int ny, const int *col_strip, const BandDev &b,
                            const void *tloc, double2 *z, cudaStream_t st) {
  k_synthesize_band<R><<<grid_for(b.n1), TPB, 0, st>>>(strips_dev, nsub, ny, col_strip, b.iv1, b.off1, b.niv1, b.n1,
                                                        tloc, z);
  count_launch();
}
void launch_stencil_band(const GridDev &g, const BandDev &b, const double2 *z, const double2 *sub, bool sub_global,
                         bool neg, double2 *y, cudaStream_t st) {
  k_stencil_band<<<grid_for(b.n), TPB, 0, st>>>(g, b.iv, b.off, b.niv, b.n, z, sub, sub_global ? 1 : 0, neg ? 1 : 0,
                                                 y);
  count_launch();
}
void launch_vsub(const double2 *a, const double2 *b, double2 *r, int64_t n, cudaStream_t st) {
  k_vsub<<<grid_for(n), TPB, 0, st>>>(a, b, r, n);
  count_launch();
}
void launch_band_gather(const BandDev &b, int ny, const double2 *x, double2 *y, cudaStream_t st) {
  k_band_copy<<<grid_for(b.n), TPB, 0, st>>>(b.iv, b.off, b.niv, b.n, ny, const_cast<double2 *>(x), y, 1);
  count_launch();
}
void launch_band_scatter_add(const BandDev &b, int ny, const double2 *y, double2 *x, cudaStream_t st) {
  k_band_copy<<<grid_for(b.n), TPB, 0, st>>>(b.iv, b.off, b.niv, b.n, ny, x, const_cast<double2 *>(y), 0);
  count_launch();
}
template void launch_restrict_band<double>(const StripDev *, int, int64_t, int, const int64_t *, const double2 *,
                                           void *, cudaStream_t);
template void launch_restrict_band<float>(const StripDev *, int, int64_t, int, const int64_t *, const double2 *,
                                          void *, cudaStream_t);
template void launch_synthesize_band<double>(const StripDev *, int, int, const int *, const BandDev &, const void *,
                                             double2 *, cudaStream_t);
template void launch_synthesize_band<float>(const StripDev *, int, int, const int *, const BandDev &, const void *,
                                            double2 *, cudaStream_t);

template void launch_restrict<double>(const StripDev *, int, int64_t, int, const int *, const double2 *, void *,
                                      cudaStream_t);
template void launch_restrict<float>(const StripDev *, int, int64_t, int, const int *, const double2 *, void *,
                                     cudaStream_t);
template void launch_synthesize<double>(const StripDev *, int, int, int, const int *, const void *, double2 *,
                                        cudaStream_t);
template void launch_synthesize<float>(const StripDev *, int, int, int, const int *, const void *, double2 *,
                                       cudaStream_t);
template void launch_to_local<double>(const double2 *, void *, int64_t, cudaStream_t);
template void launch_to_local<float>(const double2 *, void *, int64_t, cudaStream_t);
template void launch_from_local<double>(const void *, double2 *, int64_t, cudaStream_t);
template void launch_from_local<float>(const void *, double2 *, int64_t, cudaStream_t);

}  // namespace stdd

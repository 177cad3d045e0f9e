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

__device__ __forceinline__ double2 apply_row(const GridDev &g, const double2 *__restrict__ x, int64_t idx) {
  const int i = (int)(idx / g.ny), j = (int)(idx - (int64_t)i * g.ny);
  const double2 xm = g.cxm[i], xp = g.cxp[i], ym = g.cym[j], yp = g.cyp[j];
  double2 d;
  d.x = g.k0sq * g.eps[idx] - xm.x - xp.x - ym.x - yp.x;
  d.y = -xm.y - xp.y - ym.y - yp.y;
  double2 acc = cmul(d, x[idx]);
  if (i > 0) acc = cfma(xm, x[idx - g.ny], acc);
  if (i < g.nx - 1) acc = cfma(xp, x[idx + g.ny], acc);
  if (j > 0) acc = cfma(ym, x[idx - 1], acc);
  if (j < g.ny - 1) acc = cfma(yp, x[idx + 1], acc);
  return acc;
}

__global__ void __launch_bounds__(TPB) k_stencil(GridDev g, const double2 *__restrict__ x, double2 *__restrict__ y) {
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t idx = (int64_t)blockIdx.x * TPB + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * TPB)
    y[idx] = apply_row(g, x, idx);
}

__global__ void __launch_bounds__(TPB) k_residual(GridDev g, const double2 *__restrict__ b,
                                                  const double2 *__restrict__ x, double2 *__restrict__ r) {
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t idx = (int64_t)blockIdx.x * TPB + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * TPB)
    r[idx] = csub(b[idx], apply_row(g, x, idx));
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

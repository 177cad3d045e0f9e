// FP64 complex kernels of the flexible GMRES outer iteration: classical
// Gram-Schmidt passes (multi-dot and multi-axpy fused with the norm of the
// result), the solution update x += Z y, norms and scaling.
//
// All reductions are deterministic: every block writes its partial sums to
// a fixed slot and a second kernel adds the slots in a fixed order.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace stdd {

namespace {

constexpr int TPB = 256;
constexpr int NBLK = 152 * 4;   // partial-sum blocks: 4 per SM
constexpr int GROUP = 8;        // vectors per multi-dot pass
constexpr int MAXM = 512;       // longest basis handled by the axpy kernels

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of one double; result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double *sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0;
  if (warp == 0) {
    s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// partial[blk][i] = sum conj(V_i) w over the block's chunk, i < m; with
// self_norm, partial[blk][m] = (sum |w|^2, 0)
__global__ void __launch_bounds__(TPB) k_mdot(const double2 *__restrict__ V, int64_t ldv, int m,
                                              const double2 *__restrict__ w, int64_t n,
                                              double2 *__restrict__ partial, int self_norm) {
  __shared__ double sh[TPB / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * chunk, g1 = min(n, g0 + chunk);
  const int mt = m + (self_norm ? 1 : 0);
  if (self_norm) {
    double a = 0;
    for (int64_t g = g0 + threadIdx.x; g < g1; g += TPB) {
      const double2 wv = w[g];
      a = fma(wv.x, wv.x, fma(wv.y, wv.y, a));
    }
    const double sa = block_sum(a, sh);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * mt + m] = make_double2(sa, 0.0);
  }
  for (int i0 = 0; i0 < m; i0 += GROUP) {
    const int gi = min(GROUP, m - i0);
    double2 acc[GROUP];
#pragma unroll
    for (int q = 0; q < GROUP; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int64_t g = g0 + threadIdx.x; g < g1; g += TPB) {
      const double2 wv = w[g];
#pragma unroll
      for (int q = 0; q < GROUP; ++q)
        if (q < gi) {
          const double2 v = V[(int64_t)(i0 + q) * ldv + g];
          acc[q].x = fma(v.x, wv.x, fma(v.y, wv.y, acc[q].x));
          acc[q].y = fma(v.x, wv.y, fma(-v.y, wv.x, acc[q].y));
        }
    }
#pragma unroll
    for (int q = 0; q < GROUP; ++q) {
      if (q < gi) {
        const double sr = block_sum(acc[q].x, sh);
        const double si = block_sum(acc[q].y, sh);
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * mt + i0 + q] = make_double2(sr, si);
      }
    }
  }
}

// h[i] = sum over blocks of partial[blk][i], fixed order; one warp per i
__global__ void k_reduce_c(const double2 *__restrict__ partial, int nblk, int m, double2 *__restrict__ h) {
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double sr = 0, si = 0;
  for (int b = lane; b < nblk; b += 32) {
    const double2 v = partial[(int64_t)b * m + i];
    sr += v.x;
    si += v.y;
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  if (lane == 0) h[i] = make_double2(sr, si);
}

__global__ void k_reduce_r(const double *__restrict__ partial, int nblk, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  double s = 0;
  for (int b = lane; b < nblk; b += 32) s += partial[b];
  s = warp_sum(s);
  if (lane == 0) out[0] = s;
}

__global__ void __launch_bounds__(TPB) k_maxpy_norm(const double2 *__restrict__ V, int64_t ldv, int m,
                                                    const double2 *__restrict__ h, double2 *__restrict__ w,
                                                    int64_t n, double *__restrict__ partial) {
  __shared__ double2 hs[MAXM];
  __shared__ double sh[TPB / 32];
  for (int i = threadIdx.x; i < m; i += TPB) hs[i] = h[i];
  __syncthreads();
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * chunk, g1 = min(n, g0 + chunk);
  double nrm = 0;
  for (int64_t g = g0 + threadIdx.x; g < g1; g += TPB) {
    double2 acc = w[g];
    for (int i = 0; i < m; ++i) acc = cfms(hs[i], V[(int64_t)i * ldv + g], acc);
    w[g] = acc;
    nrm = fma(acc.x, acc.x, fma(acc.y, acc.y, nrm));
  }
  const double s = block_sum(nrm, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(TPB) k_maxpy(const double2 *__restrict__ Z, int64_t ldz, int m,
                                               const double2 *__restrict__ y, double2 *__restrict__ x,
                                               int64_t n) {
  __shared__ double2 ys[MAXM];
  for (int i = threadIdx.x; i < m; i += TPB) ys[i] = y[i];
  __syncthreads();
  for (int64_t g = (int64_t)blockIdx.x * TPB + threadIdx.x; g < n; g += (int64_t)gridDim.x * TPB) {
    double2 acc = x[g];
    for (int i = 0; i < m; ++i) acc = cfma(ys[i], Z[(int64_t)i * ldz + g], acc);
    x[g] = acc;
  }
}

__global__ void __launch_bounds__(TPB) k_norm2(const double2 *__restrict__ x, int64_t n,
                                               double *__restrict__ partial) {
  __shared__ double sh[TPB / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * chunk, g1 = min(n, g0 + chunk);
  double nrm = 0;
  for (int64_t g = g0 + threadIdx.x; g < g1; g += TPB) {
    const double2 v = x[g];
    nrm = fma(v.x, v.x, fma(v.y, v.y, nrm));
  }
  const double s = block_sum(nrm, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(TPB) k_scale(const double2 *__restrict__ x, const double *__restrict__ nrm2,
                                               double2 *__restrict__ y, int64_t n) {
  const double a = 1.0 / sqrt(nrm2[0]);
  for (int64_t g = (int64_t)blockIdx.x * TPB + threadIdx.x; g < n; g += (int64_t)gridDim.x * TPB) {
    const double2 v = x[g];
    y[g] = make_double2(a * v.x, a * v.y);
  }
}

inline int nblocks_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(NBLK, (n + TPB - 1) / TPB)); }

}  // namespace

int krylov_partial_blocks() { return NBLK; }

void launch_mdot(const double2 *V, int64_t ldv, int m, const double2 *w, int64_t n, double2 *partial,
                 double2 *h, cudaStream_t st, int self_norm) {
  const int nb = nblocks_for(n);
  k_mdot<<<nb, TPB, 0, st>>>(V, ldv, m, w, n, partial, self_norm);
  count_launch();
  const int mt = m + (self_norm ? 1 : 0);
  k_reduce_c<<<(mt + 7) / 8, 256, 0, st>>>(partial, nb, mt, h);
  count_launch();
}

void launch_maxpy_norm(const double2 *V, int64_t ldv, int m, const double2 *h, double2 *w, int64_t n,
                       double *partial, double *nrm2, cudaStream_t st) {
  const int nb = nblocks_for(n);
  k_maxpy_norm<<<nb, TPB, 0, st>>>(V, ldv, m, h, w, n, partial);
  count_launch();
  k_reduce_r<<<1, 32, 0, st>>>(partial, nb, nrm2);
  count_launch();
}

void launch_maxpy(const double2 *Z, int64_t ldz, int m, const double2 *y, double2 *x, int64_t n,
                  cudaStream_t st) {
  k_maxpy<<<nblocks_for(n), TPB, 0, st>>>(Z, ldz, m, y, x, n);
  count_launch();
}

void launch_norm2(const double2 *x, int64_t n, double *partial, double *nrm2, cudaStream_t st) {
  const int nb = nblocks_for(n);
  k_norm2<<<nb, TPB, 0, st>>>(x, n, partial);
  count_launch();
  k_reduce_r<<<1, 32, 0, st>>>(partial, nb, nrm2);
  count_launch();
}

void launch_scale(const double2 *x, const double *inv_norm2, double2 *y, int64_t n, cudaStream_t st) {
  k_scale<<<nblocks_for(n), TPB, 0, st>>>(x, inv_norm2, y, n);
  count_launch();
}

}  // namespace stdd

// Numeric multifrontal LU of the strip operators A_i and the batched
// forward / back substitutions that apply A_i^-1 (Sec. 2.4, Eqs. 22-23).
//
// Every kernel works on one level of the elimination trees at a time, over
// all fronts of that level in all strips (blockIdx.x = front within the
// level, blockIdx.y = tile within the front).  Fronts of one level are independent; a level needs
// only the Schur complements (factor) or update vectors (forward solve) of
// the level below, kept in two parity buffers.
//
// Front layout (n = p + b, column-major, complex):
//   [F11 F12] : p x n, leading dimension p, in the factor block
//   F21       : b x p, leading dimension b, right after it
//   F22       : b x b, leading dimension b, in the level workspace
// After factorization F11 holds L11 (unit, strictly lower) and U11, F21 holds
// L21 = F21 U11^-1, F12 holds U12 = L11^-1 F12 and F22 the Schur complement
// F22 - L21 U12 that the parent extend-adds.  No pivoting: the fill-reducing
// order is the only permutation (Eq. 22); zero or non-finite pivots raise a
// flag that the host turns into STDD_EPIVOT.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace stdd {

namespace {

template <typename C>
__device__ __forceinline__ int64_t elem_off(int r, int c, int p, int b, int64_t fo, int64_t so,
                                            bool &in_ws) {
  const int n = p + b;
  if (r < p) { in_ws = false; return fo + (int64_t)c * p + r; }
  if (c < p) { in_ws = false; return fo + (int64_t)p * n + (int64_t)c * b + (r - p); }
  in_ws = true;
  return so + (int64_t)(c - p) * b + (r - p);
}

template <typename C> __device__ __forceinline__ bool cfinite(C a) {
  return isfinite(a.x) && isfinite(a.y);
}

}  // namespace

// ------------------------------------------------------------- assembly
// F = A-entries of this front (rows or columns that are pivots here) plus the
// children's Schur complements placed by the inverse extend-add maps.
template <typename R>
__global__ void __launch_bounds__(256) mf_assemble(MfArgs a, int f0) {
  using C = typename CT<R>::T;
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, b = f.b, n = p + b;
  const int64_t nn = (int64_t)n * n;
  const StripDev s = a.strips[f.strip];
  const int H = a.H;
  FrontDev ch[2];
  bool has[2];
#pragma unroll
  for (int ci = 0; ci < 2; ++ci) {
    has[ci] = f.child[ci] >= 0;
    if (has[ci]) ch[ci] = a.fronts[f.child[ci]];
  }
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.y * blockDim.x) {
    const int c = (int)(e / n), r = (int)(e - (int64_t)c * n);
    double2 v = make_double2(0.0, 0.0);
    if (r < p || c < p) {
      const int u = a.nodes[f.node_off + r], w = a.nodes[f.node_off + c];
      const int ux = u / H, uy = u - ux * H;
      if (u == w) {
        const double2 xm = a.cxm[s.coef_off + ux], xp = a.cxp[s.coef_off + ux];
        const double2 ym = a.cym[uy], yp = a.cyp[uy];
        v.x = a.k0sq * a.eps[(int64_t)(s.x0 + ux) * H + uy] - xm.x - xp.x - ym.x - yp.x;
        v.y = -xm.y - xp.y - ym.y - yp.y;
      } else if (w == u - H) {
        v = a.cxm[s.coef_off + ux];
      } else if (w == u + H) {
        v = a.cxp[s.coef_off + ux];
      } else if (w == u - 1 && uy > 0) {
        v = a.cym[uy];
      } else if (w == u + 1 && uy < H - 1) {
        v = a.cyp[uy];
      }
    }
    C out = to_c(v, C());
#pragma unroll
    for (int ci = 0; ci < 2; ++ci) {
      if (!has[ci]) continue;
      const int ir = a.inv[f.inv_off[ci] + r];
      if (ir < 0) continue;
      const int ic = a.inv[f.inv_off[ci] + c];
      if (ic < 0) continue;
      const C sv = reinterpret_cast<const C *>(a.ws_child)[ch[ci].s_off + (int64_t)ic * ch[ci].b + ir];
      out = cadd(out, sv);
    }
    bool in_ws;
    const int64_t off = elem_off<C>(r, c, p, b, f.fac_off, f.s_off, in_ws);
    if (in_ws) reinterpret_cast<C *>(a.ws_cur)[off] = out;
    else reinterpret_cast<C *>(a.fac)[off] = out;
  }
}

// ------------------------------------------------------ diagonal block k
// One CTA per front: unblocked LU (no pivoting) of the nbk x nbk block at
// (k, k), in shared memory, written back in place; zero or non-finite pivots
// set the flag, |pivot| feeds the running minimum.
template <typename R>
__global__ void __launch_bounds__(MF_PANEL_THREADS) mf_diag(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB;
  __shared__ C D[NB][NB + 1];
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p;
  if (k >= p) return;
  const int nbk = min(NB, p - k);
  C *fac = reinterpret_cast<C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nbk * nbk; idx += blockDim.x) {
    const int i = idx % nbk, j = idx / nbk;
    D[i][j] = fac[fo + (int64_t)(k + j) * p + k + i];
  }
  __syncthreads();
  for (int j = 0; j < nbk; ++j) {
    const C inv = crecip(D[j][j]);
    for (int i = j + 1 + tid; i < nbk; i += blockDim.x) D[i][j] = cmul(D[i][j], inv);
    __syncthreads();
    const int m = nbk - j - 1;
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      const int i = j + 1 + idx % m, l = j + 1 + idx / m;
      D[i][l] = cfms(D[i][j], D[j][l], D[i][l]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nbk * nbk; idx += blockDim.x) {
    const int i = idx % nbk, j = idx / nbk;
    fac[fo + (int64_t)(k + j) * p + k + i] = D[i][j];
  }
  for (int j = tid; j < nbk; j += blockDim.x) {
    const C d = D[j][j];
    const double ad = sqrt((double)cabs2(d));
    if (!(ad > 0.0) || !cfinite(d)) atomicOr(a.flag, 1);
    else atomicMin(reinterpret_cast<unsigned long long *>(a.min_pivot),
                   (unsigned long long)__double_as_longlong(ad));
  }
}

// ---------------------------------------------------------- panel step k
// After mf_diag: blockIdx.y = 0 .. ntr-1 are row tiles of L (rows k+nbk ..
// n) solving X U_D = F; blockIdx.y = ntr .. 2 ntr-1 are column tiles of U
// (cols k+nbk .. n) solving L_D Y = F.  The factored diagonal block is only
// read here, so the tiles need no ordering among themselves.
template <typename R>
__global__ void __launch_bounds__(MF_PANEL_THREADS) mf_panel(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB;
  constexpr int TILE = MF_PANEL_THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C(*D)[NB + 1] = reinterpret_cast<C(*)[NB + 1]>(smem_raw);
  C *dinv = reinterpret_cast<C *>(smem_raw + sizeof(C) * NB * (NB + 1));
  C(*T)[NB + 1] = reinterpret_cast<C(*)[NB + 1]>(smem_raw + sizeof(C) * (NB * (NB + 1) + NB));

  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, b = f.b, n = p + b;
  if (k >= p) return;
  const int nbk = min(NB, p - k);
  const int rem = n - k - nbk;
  const int ntr = (rem + TILE - 1) / TILE;
  const int t = blockIdx.y;
  if (t >= 2 * ntr) return;
  C *fac = reinterpret_cast<C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x;

  for (int idx = tid; idx < nbk * nbk; idx += blockDim.x) {
    const int i = idx % nbk, j = idx / nbk;
    D[i][j] = fac[fo + (int64_t)(k + j) * p + k + i];
  }
  __syncthreads();
  for (int j = tid; j < nbk; j += blockDim.x) dinv[j] = crecip(D[j][j]);
  __syncthreads();

  if (t < ntr) {
    // rows r = k+nbk+t*TILE+tid of column block [k, k+nbk): X = F U_D^-1
    const int r = k + nbk + t * TILE + tid;
    if (r < n) {
      C x[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < nbk) {
          const int64_t off = r < p ? fo + (int64_t)(k + j) * p + r
                                    : fo + (int64_t)p * n + (int64_t)(k + j) * b + (r - p);
          x[j] = fac[off];
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < nbk) {
          C s = x[j];
#pragma unroll
          for (int l = 0; l < NB; ++l)
            if (l < j) s = cfms(x[l], D[l][j], s);
          x[j] = cmul(s, dinv[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < nbk) {
          const int64_t off = r < p ? fo + (int64_t)(k + j) * p + r
                                    : fo + (int64_t)p * n + (int64_t)(k + j) * b + (r - p);
          fac[off] = x[j];
        }
      }
    }
  } else {
    // columns c of row block [k, k+nbk): Y = L_D^-1 F, staged through smem
    const int cbase = k + nbk + (t - ntr) * TILE;
    const int ncol = min(TILE, n - cbase);
    for (int idx = tid; idx < nbk * ncol; idx += blockDim.x) {
      const int i = idx % nbk, cc = idx / nbk;
      T[cc][i] = fac[fo + (int64_t)(cbase + cc) * p + k + i];
    }
    __syncthreads();
    if (tid < ncol) {
      C y[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < nbk) y[i] = T[tid][i];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i < nbk) {
          C s = y[i];
#pragma unroll
          for (int l = 0; l < NB; ++l)
            if (l < i) s = cfms(D[i][l], y[l], s);
          y[i] = s;
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < nbk) T[tid][i] = y[i];
    }
    __syncthreads();
    for (int idx = tid; idx < nbk * ncol; idx += blockDim.x) {
      const int i = idx % nbk, cc = idx / nbk;
      fac[fo + (int64_t)(cbase + cc) * p + k + i] = T[cc][i];
    }
  }
}

// ------------------------------------------------------- tile GEMM core
// acc[4][4] += A(64 x K) B(K x 64) for one 64 x 64 tile, K <= MF_NB per call.
// 256 threads as 16 x 16; thread (tx, ty) owns rows ty + 16*i, cols tx + 16*j.
template <typename C>
__device__ __forceinline__ void tile_mma(const C (*As)[MF_NB + 1], const C (*Bs)[64 + 1], int K,
                                         C acc[4][4], int tx, int ty) {
  for (int kk = 0; kk < K; ++kk) {
    C av[4], bv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = As[ty + 16 * i][kk];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = cfma(av[i], bv[j], acc[i][j]);
  }
}

// ------------------------------------------------- trailing update step k
// F(r, c) -= L(r, k:k+nbk) U(k:k+nbk, c) for r, c >= k+nbk outside F22
// (the F22 block is updated once, at the end, by mf_schur).
template <typename R>
__global__ void __launch_bounds__(256) mf_update(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C(*As)[NB + 1] = reinterpret_cast<C(*)[NB + 1]>(smem_raw);
  C(*Bs)[64 + 1] = reinterpret_cast<C(*)[64 + 1]>(smem_raw + sizeof(C) * 64 * (NB + 1));

  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, b = f.b, n = p + b;
  if (k >= p) return;
  const int nbk = min(NB, p - k);
  const int s0 = k + nbk;
  const int rem = n - s0;
  if (rem <= 0 || s0 >= p) return;
  const int nt = (rem + 63) / 64;
  if ((int)blockIdx.y >= nt * nt) return;
  const int r0 = s0 + (blockIdx.y % nt) * 64, c0 = s0 + (blockIdx.y / nt) * 64;
  if (r0 >= p && c0 >= p) return;  // entirely inside F22
  C *fac = reinterpret_cast<C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;

  for (int idx = tid; idx < 64 * nbk; idx += 256) {
    const int rr = idx % 64, j = idx / 64, r = r0 + rr;
    C v = czero<C>();
    if (r < n)
      v = r < p ? fac[fo + (int64_t)(k + j) * p + r]
                : fac[fo + (int64_t)p * n + (int64_t)(k + j) * b + (r - p)];
    As[rr][j] = v;
  }
  for (int idx = tid; idx < 64 * nbk; idx += 256) {
    const int j = idx % nbk, cc = idx / nbk, c = c0 + cc;
    Bs[j][cc] = c < n ? fac[fo + (int64_t)c * p + k + j] : czero<C>();
  }
  __syncthreads();
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = czero<C>();
  tile_mma<C>(As, Bs, nbk, acc, tx, ty);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 16 * i;
    if (r >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c >= n || (r >= p && c >= p)) continue;
      const int64_t off = r < p ? fo + (int64_t)c * p + r
                                : fo + (int64_t)p * n + (int64_t)c * b + (r - p);
      fac[off] = csub(fac[off], acc[i][j]);
    }
  }
}

// ------------------------------------------------------ Schur complement
// F22 -= L21 U12 (b x b x p), one 64 x 64 tile of one front per CTA.
template <typename R>
__global__ void __launch_bounds__(256) mf_schur(MfArgs a, int f0) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C(*As)[NB + 1] = reinterpret_cast<C(*)[NB + 1]>(smem_raw);
  C(*Bs)[64 + 1] = reinterpret_cast<C(*)[64 + 1]>(smem_raw + sizeof(C) * 64 * (NB + 1));

  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, b = f.b, n = p + b;
  if (b == 0) return;
  const int nt = (b + 63) / 64;
  if ((int)blockIdx.y >= nt * nt) return;
  const int r0 = (blockIdx.y % nt) * 64, c0 = (blockIdx.y / nt) * 64;
  const C *fac = reinterpret_cast<const C *>(a.fac);
  C *ws = reinterpret_cast<C *>(a.ws_cur);
  const int64_t L21 = f.fac_off + (int64_t)p * n;  // b x p, ld b
  const int64_t U12 = f.fac_off + (int64_t)p * p;  // p x b, ld p
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = czero<C>();
  for (int k0 = 0; k0 < p; k0 += NB) {
    const int kb = min(NB, p - k0);
    __syncthreads();
    for (int idx = tid; idx < 64 * kb; idx += 256) {
      const int rr = idx % 64, j = idx / 64, r = r0 + rr;
      As[rr][j] = r < b ? fac[L21 + (int64_t)(k0 + j) * b + r] : czero<C>();
    }
    for (int idx = tid; idx < 64 * kb; idx += 256) {
      const int j = idx % kb, cc = idx / kb, c = c0 + cc;
      Bs[j][cc] = c < b ? fac[U12 + (int64_t)c * p + k0 + j] : czero<C>();
    }
    __syncthreads();
    tile_mma<C>(As, Bs, kb, acc, tx, ty);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 16 * i;
    if (r >= b) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c >= b) continue;
      const int64_t off = f.s_off + (int64_t)c * b + r;
      ws[off] = csub(ws[off], acc[i][j]);
    }
  }
}

// ----------------------------------------------------- forward solve
// One CTA per front.  w = [t(pivots); 0] + sum_children extend(u_child);
// y = L11^-1 w_piv (unit lower, column-oriented in blocks of 32: warp 0
// solves the diagonal block with shuffles, all warps update the rows below);
// u = w_border - L21 y goes to the parent; y overwrites t at the pivots.
template <typename R>
__global__ void __launch_bounds__(256) mf_forward(MfArgs a, int f0, int nrhs, int64_t ldt) {
  using C = typename CT<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, b = f.b, n = p + b;
  C *w = reinterpret_cast<C *>(smem_raw);  // [nrhs][n]
  C *tv = reinterpret_cast<C *>(a.tloc);
  const StripDev s = a.strips[f.strip];
  const C *fac = reinterpret_cast<const C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x;

  for (int idx = tid; idx < n * nrhs; idx += blockDim.x) {
    const int q = idx / n, k = idx - q * n;
    w[idx] = k < p ? tv[q * ldt + s.vec_off + a.nodes[f.node_off + k]] : czero<C>();
  }
  __syncthreads();
  for (int ci = 0; ci < 2; ++ci) {
    if (f.child[ci] < 0) continue;
    const FrontDev ch = a.fronts[f.child[ci]];
    const C *uc = reinterpret_cast<const C *>(a.ub_child) + ch.u_off * nrhs;
    for (int idx = tid; idx < ch.b * nrhs; idx += blockDim.x) {
      const int q = idx / ch.b, k = idx - q * ch.b;
      const int at = a.cmap[f.cmap_off[ci] + k];
      w[q * n + at] = cadd(w[q * n + at], uc[(int64_t)q * ch.b + k]);
    }
    __syncthreads();
  }
  const int lane = tid & 31, warp = tid >> 5;
  for (int J = 0; J < p; J += 32) {
    const int jb = min(32, p - J);
    if (warp == 0) {
      C Lrow[32];
#pragma unroll
      for (int j = 0; j < 32; ++j)
        Lrow[j] = (j < jb && lane < jb) ? fac[fo + (int64_t)(J + j) * p + J + lane] : czero<C>();
      for (int q = 0; q < nrhs; ++q) {
        C x = lane < jb ? w[q * n + J + lane] : czero<C>();
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const C yj = shfl(x, j);
          if (lane > j && j < jb) x = cfms(Lrow[j], yj, x);
        }
        if (lane < jb) w[q * n + J + lane] = x;
      }
    }
    __syncthreads();
    for (int r = J + jb + tid; r < p; r += blockDim.x) {
      for (int q = 0; q < nrhs; ++q) {
        C acc = w[q * n + r];
        for (int j = 0; j < jb; ++j) acc = cfms(fac[fo + (int64_t)(J + j) * p + r], w[q * n + J + j], acc);
        w[q * n + r] = acc;
      }
    }
    __syncthreads();
  }
  // border update u = w_b - L21 y, and y back to the local vector
  C *ub = reinterpret_cast<C *>(a.ub_cur) + f.u_off * nrhs;
  const int64_t L21 = fo + (int64_t)p * n;
  for (int r = tid; r < b; r += blockDim.x) {
    for (int q = 0; q < nrhs; ++q) {
      C acc = w[q * n + p + r];
      for (int j = 0; j < p; ++j) acc = cfms(fac[L21 + (int64_t)j * b + r], w[q * n + j], acc);
      ub[(int64_t)q * b + r] = acc;
    }
  }
  for (int idx = tid; idx < p * nrhs; idx += blockDim.x) {
    const int q = idx / p, k = idx - q * p;
    tv[q * ldt + s.vec_off + a.nodes[f.node_off + k]] = w[q * n + k];
  }
}

// ----------------------------------------------------- backward solve
// One CTA per front, root level first.  z = y - U12 x_border (x_border read
// from the local vector, already final), then x = U11^-1 z by 32-blocks from
// the bottom; x overwrites y at the pivots.
template <typename R>
__global__ void __launch_bounds__(256) mf_backward(MfArgs a, int f0, int nrhs, int64_t ldt) {
  using C = typename CT<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, b = f.b, n = p + b;
  C *w = reinterpret_cast<C *>(smem_raw);  // [nrhs][n]: z then x_border
  C *tv = reinterpret_cast<C *>(a.tloc);
  const StripDev s = a.strips[f.strip];
  const C *fac = reinterpret_cast<const C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < n * nrhs; idx += blockDim.x) {
    const int q = idx / n, k = idx - q * n;
    w[idx] = tv[q * ldt + s.vec_off + a.nodes[f.node_off + k]];
  }
  __syncthreads();
  const int64_t U12 = fo + (int64_t)p * p;
  for (int r = tid; r < p; r += blockDim.x) {
    for (int q = 0; q < nrhs; ++q) {
      C acc = w[q * n + r];
      for (int j = 0; j < b; ++j) acc = cfms(fac[U12 + (int64_t)j * p + r], w[q * n + p + j], acc);
      w[q * n + r] = acc;
    }
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  const int nblk = (p + 31) / 32;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int J = bi * 32;
    const int jb = min(32, p - J);
    if (warp == 0) {
      C Urow[32];
#pragma unroll
      for (int j = 0; j < 32; ++j)
        Urow[j] = (j < jb && lane < jb) ? fac[fo + (int64_t)(J + j) * p + J + lane] : czero<C>();
      // lane j needs 1/U(j,j): the diagonal entry is Urow[lane] on lane `lane`
      C dg = czero<C>();
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j == lane) dg = Urow[j];
      const C dinv = lane < jb ? crecip(dg) : czero<C>();
      for (int q = 0; q < nrhs; ++q) {
        C x = lane < jb ? w[q * n + J + lane] : czero<C>();
#pragma unroll
        for (int j = 31; j >= 0; --j) {
          if (j < jb) {
            if (lane == j) x = cmul(x, dinv);
            const C xj = shfl(x, j);
            if (lane < j) x = cfms(Urow[j], xj, x);
          }
        }
        if (lane < jb) w[q * n + J + lane] = x;
      }
    }
    __syncthreads();
    for (int r = tid; r < J; r += blockDim.x) {
      for (int q = 0; q < nrhs; ++q) {
        C acc = w[q * n + r];
        for (int j = 0; j < jb; ++j) acc = cfms(fac[fo + (int64_t)(J + j) * p + r], w[q * n + J + j], acc);
        w[q * n + r] = acc;
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < p * nrhs; idx += blockDim.x) {
    const int q = idx / p, k = idx - q * p;
    tv[q * ldt + s.vec_off + a.nodes[f.node_off + k]] = w[q * n + k];
  }
}

// ------------------------------------------------------------ launchers
template <typename R>
static size_t panel_smem() {
  using C = typename CT<R>::T;
  return sizeof(C) * (MF_NB * (MF_NB + 1) + MF_NB + MF_PANEL_THREADS * (MF_NB + 1));
}
template <typename R>
static size_t gemm_smem() {
  using C = typename CT<R>::T;
  return sizeof(C) * (64 * (MF_NB + 1) + MF_NB * (64 + 1));
}

template <typename R>
cudaError_t mf_setup_attributes() {
  cudaError_t e;
  e = cudaFuncSetAttribute(mf_panel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem<R>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mf_update<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<R>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mf_schur<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<R>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mf_forward<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(mf_backward<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <typename R>
void mf_factor_level(const MfArgs &a, const LevelInfo &L, cudaStream_t st) {
  if (L.nf == 0) return;
  {
    const int64_t nn = (int64_t)L.max_n * L.max_n;
    int gx = (int)std::min<int64_t>((nn + 255) / 256, 4096);
    mf_assemble<R><<<dim3(L.nf, gx), 256, 0, st>>>(a, L.f0);
  }
  for (int k = 0; k < L.max_p; k += MF_NB) {
    const int rem = L.max_n - k - 1;
    const int ntr = std::max(1, (rem + MF_PANEL_THREADS - 1) / MF_PANEL_THREADS);
    mf_diag<R><<<L.nf, MF_PANEL_THREADS, 0, st>>>(a, L.f0, k);
    mf_panel<R><<<dim3(L.nf, 2 * ntr), MF_PANEL_THREADS, panel_smem<R>(), st>>>(a, L.f0, k);
    const int nt = std::max(1, (rem + 63) / 64);
    mf_update<R><<<dim3(L.nf, nt * nt), 256, gemm_smem<R>(), st>>>(a, L.f0, k);
  }
  if (L.max_b > 0) {
    const int nt = (L.max_b + 63) / 64;
    mf_schur<R><<<dim3(L.nf, nt * nt), 256, gemm_smem<R>(), st>>>(a, L.f0);
  }
}

template <typename R>
void mf_forward_level(const MfArgs &a, const LevelInfo &L, int nrhs, int64_t ldt, cudaStream_t st) {
  if (L.nf == 0) return;
  using C = typename CT<R>::T;
  const size_t sm = sizeof(C) * (size_t)L.max_n * nrhs;
  mf_forward<R><<<L.nf, 256, sm, st>>>(a, L.f0, nrhs, ldt);
}

template <typename R>
void mf_backward_level(const MfArgs &a, const LevelInfo &L, int nrhs, int64_t ldt, cudaStream_t st) {
  if (L.nf == 0) return;
  using C = typename CT<R>::T;
  const size_t sm = sizeof(C) * (size_t)L.max_n * nrhs;
  mf_backward<R><<<L.nf, 256, sm, st>>>(a, L.f0, nrhs, ldt);
}

template cudaError_t mf_setup_attributes<double>();
template cudaError_t mf_setup_attributes<float>();
template void mf_factor_level<double>(const MfArgs &, const LevelInfo &, cudaStream_t);
template void mf_factor_level<float>(const MfArgs &, const LevelInfo &, cudaStream_t);
template void mf_forward_level<double>(const MfArgs &, const LevelInfo &, int, int64_t, cudaStream_t);
template void mf_forward_level<float>(const MfArgs &, const LevelInfo &, int, int64_t, cudaStream_t);
template void mf_backward_level<double>(const MfArgs &, const LevelInfo &, int, int64_t, cudaStream_t);
template void mf_backward_level<float>(const MfArgs &, const LevelInfo &, int, int64_t, cudaStream_t);

}  // namespace stdd

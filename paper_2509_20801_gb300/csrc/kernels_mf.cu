// Numeric multifrontal factorization of the strip operators A_i and the
// batched substitution sweeps that apply A_i^-1 (Sec. 2.4, Eqs. 22-23).
//
// Each front F = [F11 F12; F21 F22] (p pivots, b border nodes, n = p + b) is
// eliminated by a Gauss-Jordan sweep of its p pivots, which leaves
//     [ F11^-1          F11^-1 F12            ]   =  [ Finv   H12 ]
//     [ -F21 F11^-1     F22 - F21 F11^-1 F12  ]      [ -G21   S   ]
// in place.  S is the Schur complement the parent extend-adds.  With these
// blocks the two substitutions of Eq. 23 become plain matrix-vector products
// with no sequential triangular chain: going up the tree (leaves to root)
//     w = [t_piv; 0] + sum_children extend(u_child),   u = w_b - G21 w_p,
// and coming down (root to leaves)
//     x_p = Finv w_p - H12 x_b,
// the block-LU solve of the front written with the inverse of F11.  The
// elimination order (nested dissection) is the only permutation; there is no
// pivoting (Eq. 22 uses fill-reducing P, Q only) and zero / non-finite pivots
// raise a flag the host turns into STDD_EPIVOT.  Optionally (static
// pivoting, an option of the context) a pivot smaller in modulus
// than a floor is replaced by the floor times its phase before it is used:
// the sweep then factors A + E, E diagonal with one entry per raised pivot,
// and the outer FGMRES absorbs the low-rank difference.  This bounds the
// element growth that near-singular pivot blocks cause without pivoting
// (nested dissection eliminates each box with its separators held fixed,
// i.e. a closed cavity, and high-index boxes can sit near a resonance).
//
// Optionally (partial pivoting, an option of the context) the sweep swaps
// rows among the not yet eliminated pivot rows of a front before each pivot
// (each 32-pivot block of a large front): the pivot of largest modulus in
// the pivot column, searched over the front's pivot rows only, so the
// nested-dissection order and the front structure stay as they are.  The
// elimination then works on P F (P permutes pivot rows), which leaves
//     [ F11^-1 P^T      F11^-1 F12 ]
//     [ -F21 F11^-1 P^T S          ]
// -- F12's block and S unchanged, the columns of the two blocks that
// multiply w_p permuted -- so the substitutions only read w_p through the
// stored column -> pivot map pcol (w_p[pcol[j]] for column j).
//
// Front storage (column-major, complex):
//   rows 0..p-1, all n columns : p x n, leading dimension p ([Finv H12])
//   rows p..n-1, columns < p   : b x p, leading dimension b (-G21)
//   rows p..n-1, columns >= p  : b x b in the level workspace (S)
// Every kernel handles one level of the elimination trees of all strips.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace stdd {

namespace {

template <typename C> __device__ __forceinline__ bool cfinite(C a) { return isfinite(a.x) && isfinite(a.y); }

template <typename C> __device__ __forceinline__ C cneg(C a) {
  a.x = -a.x;
  a.y = -a.y;
  return a;
}

// address of front element (r, c); *ws selects the level workspace
__device__ __forceinline__ int64_t elem_off(int r, int c, int p, int b, int64_t fo, int64_t so, bool &ws) {
  if (r < p) {
    ws = false;
    return fo + (int64_t)c * p + r;
  }
  const int n = p + b;
  if (c < p) {
    ws = false;
    return fo + (int64_t)p * n + (int64_t)c * b + (r - p);
  }
  ws = true;
  return so + (int64_t)(c - p) * b + (r - p);
}

template <typename C> __device__ __forceinline__ C ld_elem(const MfArgs &a, const FrontDev &f, int r, int c) {
  bool ws;
  const int64_t o = elem_off(r, c, f.p, f.b, f.fac_off, f.s_off, ws);
  return ws ? reinterpret_cast<const C *>(a.ws_cur)[o] : reinterpret_cast<const C *>(a.fac)[o];
}
template <typename C> __device__ __forceinline__ void st_elem(const MfArgs &a, const FrontDev &f, int r, int c, C v) {
  bool ws;
  const int64_t o = elem_off(r, c, f.p, f.b, f.fac_off, f.s_off, ws);
  if (ws) reinterpret_cast<C *>(a.ws_cur)[o] = v;
  else reinterpret_cast<C *>(a.fac)[o] = v;
}

// the pivot actually used: d, or the floor with d's phase when |d| < floor
template <typename C> __device__ __forceinline__ C floor_pivot(const MfArgs &a, C d, bool &raised) {
  raised = false;
  if (!(a.piv_floor > 0.0) || !cfinite(d)) return d;
  const double ad = sqrt((double)cabs2(d));
  if (!(ad < a.piv_floor)) return d;
  raised = true;
  C r;
  if (ad > 0.0) {
    r.x = (decltype(r.x))((double)d.x * (a.piv_floor / ad));
    r.y = (decltype(r.y))((double)d.y * (a.piv_floor / ad));
  } else {
    r.x = (decltype(r.x))a.piv_floor;
    r.y = 0;
  }
  return r;
}

__device__ __forceinline__ void note_pivot(const MfArgs &a, double ad, bool finite) {
  if (!(ad > 0.0) || !finite) atomicOr(a.flag, 1);
  else atomicMin(reinterpret_cast<unsigned long long *>(a.min_pivot), (unsigned long long)__double_as_longlong(ad));
}

// skip the pivot band [k, k + nbk) when enumerating rows / columns
__device__ __forceinline__ int unband(int i, int k, int nbk) { return i < k ? i : i + nbk; }

}  // namespace

// ------------------------------------------------------------- assembly
// Entry (r, c) of front f before elimination: the A-entry if row or column
// is a pivot here (Eq. 2 with the stretched couplings of Eq. 9, strip-local
// x couplings), plus the children's Schur complements placed by the inverse
// extend-add maps.
template <typename C>
__device__ __forceinline__ C front_entry(const MfArgs &a, const FrontDev &f, const StripDev &s, const FrontDev *ch,
                                         const bool *has, int r, int c) {
  const int p = f.p, H = s.y1 - s.y0;   // local box height
  double2 v = make_double2(0.0, 0.0);
  if ((r < p || c < p) && a.sym) {
    // row u of D A: the diagonal times d_u = s_x s_y; each coupling between
    // two nodes computed from the lower-indexed node of the pair, so that
    // entries (u, w) and (w, u) are the same number
    const int u = a.nodes[f.node_off + r], w = a.nodes[f.node_off + c];
    const int ux = u / H, uy = u - ux * H;
    const double2 sxu = a.lsx[s.coef_off + ux], syu = a.lsy[s.ycoef_off + uy];
    if (u == w) {
      const double2 xm = a.cxm[s.coef_off + ux], xp = a.cxp[s.coef_off + ux];
      const double2 ym = a.cym[s.ycoef_off + uy], yp = a.cyp[s.ycoef_off + uy];
      double2 d0;
      d0.x = a.k0sq * a.eps[(int64_t)(s.x0 + ux) * a.H + s.y0 + uy] - xm.x - xp.x - ym.x - yp.x;
      d0.y = -xm.y - xp.y - ym.y - yp.y;
      v = cmul(cmul(sxu, syu), d0);
    } else if (w == u - H || w == u + H) {
      const int lx = w == u - H ? ux - 1 : ux;     // the pair's left column
      v = cmul(cmul(a.lsx[s.coef_off + lx], a.cxp[s.coef_off + lx]), syu);
    } else if ((w == u - 1 && uy > 0) || (w == u + 1 && uy < H - 1)) {
      const int ly = w == u - 1 ? uy - 1 : uy;     // the pair's lower row
      v = cmul(cmul(a.lsy[s.ycoef_off + ly], a.cyp[s.ycoef_off + ly]), sxu);
    }
  } else if (r < p || c < p) {
    const int u = a.nodes[f.node_off + r], w = a.nodes[f.node_off + c];
    const int ux = u / H, uy = u - ux * H;
    if (u == w) {
      const double2 xm = a.cxm[s.coef_off + ux], xp = a.cxp[s.coef_off + ux];
      const double2 ym = a.cym[s.ycoef_off + uy], yp = a.cyp[s.ycoef_off + uy];
      v.x = a.k0sq * a.eps[(int64_t)(s.x0 + ux) * a.H + s.y0 + uy] - xm.x - xp.x - ym.x - yp.x;
      v.y = -xm.y - xp.y - ym.y - yp.y;
    } else if (w == u - H) {
      v = a.cxm[s.coef_off + ux];
    } else if (w == u + H) {
      v = a.cxp[s.coef_off + ux];
    } else if (w == u - 1 && uy > 0) {
      v = a.cym[s.ycoef_off + uy];
    } else if (w == u + 1 && uy < H - 1) {
      v = a.cyp[s.ycoef_off + uy];
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
    out = cadd(out, reinterpret_cast<const C *>(a.ws_child)[ch[ci].s_off + (int64_t)ic * ch[ci].b + ir]);
  }
  return out;
}

// Large fronts (n > MF_SMALL): write the assembled front to its storage.
template <typename R>
__global__ void __launch_bounds__(256) mf_assemble(MfArgs a, int f0) {
  using C = typename CT<R>::T;
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int n = f.p + f.b;
  if (n <= MF_SMALL) return;
  const int64_t nn = (int64_t)n * n;
  const StripDev s = a.strips[f.strip];
  FrontDev ch[2];
  bool has[2];
#pragma unroll
  for (int ci = 0; ci < 2; ++ci) {
    has[ci] = f.child[ci] >= 0;
    if (has[ci]) ch[ci] = a.fronts[f.child[ci]];
  }
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.y * blockDim.x) {
    const int c = (int)(e / n), r = (int)(e - (int64_t)c * n);
    st_elem<C>(a, f, r, c, front_entry<C>(a, f, s, ch, has, r, c));
  }
  if (a.pcol && blockIdx.y == 0)
    for (int j = threadIdx.x; j < f.p; j += blockDim.x) a.pcol[f.piv_off + j] = j;
}

// ------------------------------------------------ small fronts, in smem
// Fronts with n <= MF_SMALL are assembled straight into shared memory,
// swept one pivot at a time (row k scaled by 1/d, column k kept, rank-1
// update of everything else) and written out.  TPF threads work on one
// front: 32 (a warp, blockDim/32 fronts per CTA) for n <= 32, else the whole
// CTA (TPF = blockDim), so that the shared memory per resident warp stays
// small.  ldn is the level's largest small n.
template <int TPF> __device__ __forceinline__ void front_sync() {
  if (TPF == 32) __syncwarp();
  else __syncthreads();
}

// argmax of |v|^2 over a group of TPF threads (ties: the smaller index)
template <int TPF, typename T> __device__ __forceinline__ void group_argmax(T &v, int &i) {
  __shared__ T red_v[8];
  __shared__ int red_i[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
  if (TPF > 32) {
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      red_v[w] = v;
      red_i[w] = i;
    }
    __syncthreads();
    for (int u = 0; u < TPF / 32; ++u)
      if (red_v[u] > v || (red_v[u] == v && red_i[u] < i)) {
        v = red_v[u];
        i = red_i[u];
      }
  }
}

template <typename R, int TPF>
__global__ void __launch_bounds__(128) mf_gj_small(MfArgs a, int f0, int nf, int ldn) {
  using C = typename CT<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int fpc = blockDim.x / TPF;                 // fronts per CTA
  const int slot = threadIdx.x / TPF, t = threadIdx.x % TPF;
  const int slot_elems = ldn * (ldn + 1) + 2 * ldn;
  C *F = reinterpret_cast<C *>(smem_raw) + (size_t)slot * slot_elems;  // n x n, column-major, ld below
  C *rowk = F + ldn * (ldn + 1);
  C *colk = rowk + ldn;
  // column -> pivot map of this front (partial pivoting), after all fronts' matrices
  int *perm = reinterpret_cast<int *>(reinterpret_cast<C *>(smem_raw) + (size_t)fpc * slot_elems) +
              (size_t)slot * ldn;
  const int fi = blockIdx.x * fpc + slot;
  bool live = fi < nf;
  FrontDev f;
  int p = 0, n = 0;
  if (live) {
    f = a.fronts[f0 + fi];
    p = f.p;
    n = p + f.b;
    live = n <= MF_SMALL && n <= ldn;
  }
  if (TPF == 32 && !live) return;   // warp-private work: leaving is safe
  if (TPF > 32 && !live) return;    // whole CTA is this front
  const StripDev s = a.strips[f.strip];
  // symmetric form: updates on the lower triangle, each entry also stored
  // at its mirror (F's leading dimension odd so that the mirror stores, a
  // stride apart, fall in different banks)
  const bool sym = a.sym && a.pcol == nullptr;
  const int ld = sym ? (n | 1) : n;
  FrontDev ch[2];
  bool has[2];
#pragma unroll
  for (int ci = 0; ci < 2; ++ci) {
    has[ci] = f.child[ci] >= 0;
    if (has[ci]) ch[ci] = a.fronts[f.child[ci]];
  }
  if (sym) {
    // the assembled front is exactly symmetric (pairwise-equal stencil
    // entries, children's Schur complements stored symmetric): lower half
    // and mirror, enumerated as in the update below
    for (int e = t; e < n * (n + 1) / 2; e += TPF) {
      const int g = e / (n + 1), j = e - g * (n + 1);
      const int c = j < n - g ? g : n - 1 - g, r = j < n - g ? g + j : c + j - (n - g);
      const C v = front_entry<C>(a, f, s, ch, has, r, c);
      F[c * ld + r] = v;
      F[r * ld + c] = v;
    }
  } else {
    for (int idx = t; idx < n * n; idx += TPF) {
      const int c = idx / n, r = idx - c * n;
      F[c * ld + r] = front_entry<C>(a, f, s, ch, has, r, c);
    }
  }
  const bool piv = a.pcol != nullptr;
  if (piv)
    for (int j = t; j < p; j += TPF) perm[j] = j;
  front_sync<TPF>();
  double d2min = INFINITY;      // smallest |pivot|^2 (its square root taken once, at the end)
  bool bad = false;
  for (int k = 0; k < p; ++k) {
    if (piv) {
      // largest |entry| of column k among the pivot rows k .. p-1
      R bv = -1;
      int bi = k;
      for (int i = k + t; i < p; i += TPF) {
        const R v = cabs2(F[k * ld + i]);
        if (v > bv) {
          bv = v;
          bi = i;
        }
      }
      group_argmax<TPF>(bv, bi);
      const bool sw = bi != k && bv > cabs2(F[k * ld + k]);
      front_sync<TPF>();          // every thread has read F(k, k) before any swap
      if (sw) {
        for (int c = t; c < n; c += TPF) {
          const C u = F[c * ld + k];
          F[c * ld + k] = F[c * ld + bi];
          F[c * ld + bi] = u;
        }
        if (t == 0) {
          const int u = perm[k];
          perm[k] = perm[bi];
          perm[bi] = u;
        }
      }
      front_sync<TPF>();
    }
    // the pivot's reciprocal and its statistics, by one thread of the front
    // (FP64 division and square root are long sequences on the FP64 pipe;
    // every other thread takes the reciprocal from it)
    C inv = czero<C>();
    if (t == 0) {
      const C d0 = F[k * ld + k];
      bool raised;
      inv = crecip(floor_pivot(a, d0, raised));
      const R d2 = cabs2(d0);
      bad |= !pivot_ok(d2);
      d2min = fmin(d2min, (double)d2);
      if (raised) atomicAdd(a.n_raised, 1ull);
    }
    if (TPF == 32) {
      inv.x = __shfl_sync(0xffffffffu, inv.x, 0);
      inv.y = __shfl_sync(0xffffffffu, inv.y, 0);
    } else {
      __shared__ C inv_s;
      if (t == 0) inv_s = inv;
      __syncthreads();
      inv = inv_s;
    }
    for (int j = t; j < n; j += TPF) {
      rowk[j] = cmul(F[j * ld + k], inv);
      colk[j] = F[k * ld + j];
    }
    front_sync<TPF>();
    if (sym) {
      // the n (n + 1) / 2 entries with r >= c, enumerated by column pairs
      // (c, n - 1 - c) of n + 1 entries each; the mirror of (r, c) is
      // negated when exactly one of r and c is eliminated (<= k)
      for (int e = t; e < n * (n + 1) / 2; e += TPF) {
        const int g = e / (n + 1), j = e - g * (n + 1);
        int r, c;
        if (j < n - g) {
          c = g;
          r = g + j;
        } else {
          c = n - 1 - g;
          r = c + j - (n - g);
        }
        C v;
        if (r == k) v = (c == k) ? inv : rowk[c];
        else if (c == k) v = cneg(cmul(colk[r], inv));
        else v = cfms(colk[r], rowk[c], F[c * ld + r]);
        F[c * ld + r] = v;
        if (r != c) F[r * ld + c] = cneg_if(v, (r <= k) != (c <= k));
      }
    } else {
      for (int idx = t; idx < n * n; idx += TPF) {
        const int c = idx / n, r = idx - c * n;
        C v;
        if (r == k) v = (c == k) ? inv : rowk[c];
        else if (c == k) v = cneg(cmul(colk[r], inv));
        else v = cfms(colk[r], rowk[c], F[c * ld + r]);
        F[c * ld + r] = v;
      }
    }
    front_sync<TPF>();
  }
  if (t == 0) note_pivot(a, bad ? 0.0 : sqrt(d2min), !bad);
  for (int idx = t; idx < n * n; idx += TPF) {
    const int c = idx / n, r = idx - c * n;
    st_elem<C>(a, f, r, c, F[c * ld + r]);
  }
  if (piv)
    for (int j = t; j < p; j += TPF) a.pcol[f.piv_off + j] = perm[j];
}

// ------------------------------------------- large fronts, blocked sweep
// Step k sweeps pivots [k, k + nbk) of every front with n > MF_SMALL:
//   gj_diag  : D <- D^-1                          (one CTA per front)
//   gj_col   : C <- -C D^-1    rows outside the band
//   gj_update: A <- A + C R    rows and columns outside the band (R unscaled)
//   gj_row   : R <- D^-1 R     columns outside the band
// Pivot search of step k (partial pivoting within the front): LU with
// partial pivoting of a copy of the panel, rows k .. p-1 x columns
// k .. k+nbk-1 (the not yet eliminated pivot rows), in the level's panel
// scratch; then its row interchanges applied, in order, to the whole rows
// of [F11 F12] and to the column -> pivot map.  The blocked sweep that
// follows eliminates the interchanged rows without further pivoting, which
// takes the same pivots.  One CTA per front.
template <typename R>
__global__ void __launch_bounds__(256) mf_gj_pivot(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB;
  __shared__ int ipiv[NB];
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(NB, p - k), m = p - k;
  C *fac = reinterpret_cast<C *>(a.fac);
  C *P = reinterpret_cast<C *>(a.panel) + f.pan_off;    // m x nbk, ld p
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < m * nbk; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    P[(int64_t)j * p + i] = fac[fo + (int64_t)(k + j) * p + k + i];
  }
  __syncthreads();
  for (int q = 0; q < nbk; ++q) {
    R bv = -1;
    int bi = q;
    for (int i = q + tid; i < m; i += blockDim.x) {
      const R v = cabs2(P[(int64_t)q * p + i]);
      if (v > bv) {
        bv = v;
        bi = i;
      }
    }
    group_argmax<256>(bv, bi);
    if (!(bv > cabs2(P[(int64_t)q * p + q]))) bi = q;   // keep the diagonal on ties
    __syncthreads();                                    // every thread has read P(q, q)
    if (tid == 0) ipiv[q] = bi;
    if (bi != q && tid < nbk) {
      const C u = P[(int64_t)tid * p + q];
      P[(int64_t)tid * p + q] = P[(int64_t)tid * p + bi];
      P[(int64_t)tid * p + bi] = u;
    }
    __syncthreads();
    const C d = P[(int64_t)q * p + q];
    if (cabs2(d) > 0) {
      const C inv = crecip(d);
      for (int i = q + 1 + tid; i < m; i += blockDim.x) P[(int64_t)q * p + i] = cmul(P[(int64_t)q * p + i], inv);
      __syncthreads();
      for (int idx = tid; idx < (m - q - 1) * (nbk - q - 1); idx += blockDim.x) {
        const int i = q + 1 + idx % (m - q - 1), j = q + 1 + idx / (m - q - 1);
        P[(int64_t)j * p + i] = cfms(P[(int64_t)q * p + i], P[(int64_t)j * p + q], P[(int64_t)j * p + i]);
      }
    }
    __syncthreads();
  }
  // interchanges in order: rows k+q and k+ipiv[q] of the p x n block
  for (int q = 0; q < nbk; ++q) {
    const int r = ipiv[q];
    if (r == q) continue;
    for (int c = tid; c < n; c += blockDim.x) {
      C *x = fac + fo + (int64_t)c * p;
      const C u = x[k + q];
      x[k + q] = x[k + r];
      x[k + r] = u;
    }
    if (tid == 0) {
      int *pc = a.pcol + f.piv_off;
      const int u = pc[k + q];
      pc[k + q] = pc[k + r];
      pc[k + r] = u;
    }
    __syncthreads();
  }
}

template <typename R>
__global__ void __launch_bounds__(MF_PANEL_THREADS) mf_gj_diag(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB;
  __shared__ C D[NB][NB + 1];
  __shared__ C rowk[NB], colk[NB];
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(NB, p - k);
  C *fac = reinterpret_cast<C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nbk * nbk; idx += blockDim.x) {
    const int i = idx % nbk, j = idx / nbk;
    D[i][j] = fac[fo + (int64_t)(k + j) * p + k + i];
  }
  __syncthreads();
  double d2min = INFINITY;
  bool bad = false;
  __shared__ C inv_s;
  for (int q = 0; q < nbk; ++q) {
    // reciprocal and statistics of the pivot by one thread (see mf_gj_small)
    if (tid == 0) {
      const C d0 = D[q][q];
      bool raised;
      inv_s = crecip(floor_pivot(a, d0, raised));
      const R d2 = cabs2(d0);
      bad |= !pivot_ok(d2);
      d2min = fmin(d2min, (double)d2);
      if (raised) atomicAdd(a.n_raised, 1ull);
    }
    __syncthreads();
    const C inv = inv_s;
    for (int j = tid; j < nbk; j += blockDim.x) {
      rowk[j] = cmul(D[q][j], inv);
      colk[j] = D[j][q];
    }
    __syncthreads();
    for (int idx = tid; idx < nbk * nbk; idx += blockDim.x) {
      const int i = idx % nbk, j = idx / nbk;
      C v;
      if (i == q) v = (j == q) ? inv : rowk[j];
      else if (j == q) v = cneg(cmul(colk[i], inv));
      else v = cfms(colk[i], rowk[j], D[i][j]);
      D[i][j] = v;
    }
    __syncthreads();
  }
  if (tid == 0) note_pivot(a, bad ? 0.0 : sqrt(d2min), !bad);
  for (int idx = tid; idx < nbk * nbk; idx += blockDim.x) {
    const int i = idx % nbk, j = idx / nbk;
    fac[fo + (int64_t)(k + j) * p + k + i] = D[i][j];
  }
}

template <typename R>
__global__ void __launch_bounds__(MF_PANEL_THREADS) mf_gj_col(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB;
  __shared__ C Dinv[NB][NB + 1];
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(NB, p - k);
  const int rows = n - nbk;
  if ((int)blockIdx.y * MF_PANEL_THREADS >= rows) return;
  const C *fac = reinterpret_cast<const C *>(a.fac);
  const int64_t fo = f.fac_off;
  for (int idx = threadIdx.x; idx < nbk * nbk; idx += blockDim.x) {
    const int i = idx % nbk, j = idx / nbk;
    Dinv[i][j] = fac[fo + (int64_t)(k + j) * p + k + i];
  }
  __syncthreads();
  const int ri = blockIdx.y * MF_PANEL_THREADS + threadIdx.x;
  if (ri >= rows) return;
  const int r = unband(ri, k, nbk);
  C x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nbk) x[j] = ld_elem<C>(a, f, r, k + j);
#pragma unroll 4
  for (int j = 0; j < NB; ++j) {
    if (j < nbk) {
      C s = czero<C>();
#pragma unroll
      for (int l = 0; l < NB; ++l)
        if (l < nbk) s = cfma(x[l], Dinv[l][j], s);
      st_elem<C>(a, f, r, k + j, cneg(s));
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(MF_PANEL_THREADS) mf_gj_row(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB;
  constexpr int TILE = MF_PANEL_THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C(*Dinv)[NB + 1] = reinterpret_cast<C(*)[NB + 1]>(smem_raw);
  C(*T)[NB + 1] = reinterpret_cast<C(*)[NB + 1]>(smem_raw + sizeof(C) * NB * (NB + 1));
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(NB, p - k);
  const int cols = n - nbk;
  const int cbase = blockIdx.y * TILE;
  if (cbase >= cols) return;
  const int ncol = min(TILE, cols - cbase);
  C *fac = reinterpret_cast<C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nbk * nbk; idx += blockDim.x) {
    const int i = idx % nbk, j = idx / nbk;
    Dinv[i][j] = fac[fo + (int64_t)(k + j) * p + k + i];
  }
  for (int idx = tid; idx < nbk * ncol; idx += blockDim.x) {
    const int i = idx % nbk, cc = idx / nbk;
    T[cc][i] = fac[fo + (int64_t)unband(cbase + cc, k, nbk) * p + k + i];
  }
  __syncthreads();
  if (tid < ncol) {
    C y[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i < nbk) y[i] = T[tid][i];
#pragma unroll 4
    for (int i = 0; i < NB; ++i) {
      if (i < nbk) {
        C s = czero<C>();
#pragma unroll
        for (int l = 0; l < NB; ++l)
          if (l < nbk) s = cfma(Dinv[i][l], y[l], s);
        T[tid][i] = s;
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < nbk * ncol; idx += blockDim.x) {
    const int i = idx % nbk, cc = idx / nbk;
    fac[fo + (int64_t)unband(cbase + cc, k, nbk) * p + k + i] = T[cc][i];
  }
}

// Symmetric form: the pivot rows after step k without the row product.
// The working matrix after the step is symmetric within the eliminated and
// within the remaining indices and antisymmetric between them, so pivot row
// k + i at column c is the column just written by mf_gj_col at (c, k + i),
// negated when c is not yet eliminated (c >= k + nbk) and kept when c < k.
// A transpose through shared memory: reads along c, writes along i.
template <typename R>
__global__ void __launch_bounds__(MF_PANEL_THREADS) mf_gj_row_mirror(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB, TILE = MF_PANEL_THREADS, HALF = TILE / 2;
  __shared__ C T[HALF][NB + 1];
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(NB, p - k);
  const int cols = n - nbk;
  C *fac = reinterpret_cast<C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x;
  for (int h = 0; h < 2; ++h) {       // the block's TILE columns, HALF at a time
    const int cbase = blockIdx.y * TILE + h * HALF;
    if (cbase >= cols) return;
    const int ncol = min(HALF, cols - cbase);
    if (h) __syncthreads();
    for (int idx = tid; idx < nbk * ncol; idx += TILE) {
      const int cc = idx % ncol, i = idx / ncol, c = unband(cbase + cc, k, nbk);
      const C v = ld_elem<C>(a, f, c, k + i);
      T[cc][i] = cneg_if(v, c >= k);
    }
    __syncthreads();
    for (int idx = tid; idx < nbk * ncol; idx += TILE) {
      const int i = idx % nbk, cc = idx / nbk;
      fac[fo + (int64_t)unband(cbase + cc, k, nbk) * p + k + i] = T[cc][i];
    }
  }
}

// The same update on 32 x 32 tiles (64 threads as 8 x 8, thread (tx, ty)
// owns rows ty + 8 i and columns tx + 8 j): more, smaller blocks for levels
// whose fronts are too small to fill 64 x 64 tiles.  Every entry accumulates
// its K products in the same order as on 64 x 64 tiles, so the autotuner's
// choice between the two never changes a result.
template <typename R>
__global__ void __launch_bounds__(64) mf_gj_update32(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB, TM = 32;
  __shared__ C As[TM][NB + 1];
  __shared__ C Bs[NB][TM + 1];
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(NB, p - k);
  const int m = n - nbk;
  const int nt = (m + TM - 1) / TM;
  if ((int)blockIdx.y >= nt * nt) return;
  const int i0 = (blockIdx.y % nt) * TM, j0 = (blockIdx.y / nt) * TM;
  const C *fac = reinterpret_cast<const C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x, tx = tid % 8, ty = tid / 8;
  for (int idx = tid; idx < TM * nbk; idx += 64) {
    const int rr = idx % TM, j = idx / TM, ri = i0 + rr;
    As[rr][j] = ri < m ? ld_elem<C>(a, f, unband(ri, k, nbk), k + j) : czero<C>();
  }
  for (int idx = tid; idx < TM * nbk; idx += 64) {
    const int j = idx % nbk, cc = idx / nbk, ci = j0 + cc;
    Bs[j][cc] = ci < m ? fac[fo + (int64_t)unband(ci, k, nbk) * p + k + j] : czero<C>();
  }
  __syncthreads();
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = czero<C>();
  for (int kk = 0; kk < nbk; ++kk) {
    C av[4], bv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = As[ty + 8 * i][kk];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 8 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = cfma(av[i], bv[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int ri = i0 + ty + 8 * i;
    if (ri >= m) continue;
    const int r = unband(ri, k, nbk);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ci = j0 + tx + 8 * j;
      if (ci >= m) continue;
      const int c = unband(ci, k, nbk);
      st_elem<C>(a, f, r, c, cadd(ld_elem<C>(a, f, r, c), acc[i][j]));
    }
  }
}

// Symmetric form: the update of step k on the lower tile triangle only.
// Between steps the working matrix of a symmetric front is
//     [ X^-1        X^-1 M_ER           ]    E = eliminated pivots [0, k)
//     [ -M_RE X^-1  M_RR - M_RE X^-1 M_ER ]    (X = M_EE, R the rest)
// -- symmetric within the E and R blocks, antisymmetric between them -- so
// every entry below the diagonal (row after column, in the order that skips
// the pivot band) also writes its mirror, negated when exactly one of the
// row and the column is eliminated.  Only tiles on or below the diagonal are
// launched, and diagonal tiles store their lower half, so every entry comes
// from the same lower-half sum whatever the tile size.  TM x TM tiles,
// (TM / 4)^2 threads, each thread 4 x 4 entries.
template <typename R, int TM>
__global__ void __launch_bounds__((TM / 4) * (TM / 4)) mf_gj_update_sym(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB, TS = TM / 4, NT = TS * TS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C(*As)[NB + 1] = reinterpret_cast<C(*)[NB + 1]>(smem_raw);
  C(*Bs)[TM + 1] = reinterpret_cast<C(*)[TM + 1]>(smem_raw + sizeof(C) * TM * (NB + 1));
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(NB, p - k);
  const int m = n - nbk;
  const int nt = (m + TM - 1) / TM;
  const int y = blockIdx.y;
  if (y >= nt * (nt + 1) / 2) return;
  int ti = (int)((sqrtf(8.f * y + 1.f) - 1.f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= y) ++ti;
  while (ti * (ti + 1) / 2 > y) --ti;
  const int tj = y - ti * (ti + 1) / 2;
  const int i0 = ti * TM, j0 = tj * TM;
  const C *fac = reinterpret_cast<const C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x, tx = tid % TS, ty = tid / TS;
  for (int idx = tid; idx < TM * nbk; idx += NT) {
    const int rr = idx % TM, j = idx / TM, ri = i0 + rr;
    As[rr][j] = ri < m ? ld_elem<C>(a, f, unband(ri, k, nbk), k + j) : czero<C>();
  }
  for (int idx = tid; idx < TM * nbk; idx += NT) {
    const int j = idx % nbk, cc = idx / nbk, ci = j0 + cc;
    Bs[j][cc] = ci < m ? fac[fo + (int64_t)unband(ci, k, nbk) * p + k + j] : czero<C>();
  }
  __syncthreads();
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = czero<C>();
  if (ti != tj) {
    for (int kk = 0; kk < nbk; ++kk) {
      C av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[ty + TS * i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + TS * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma(av[i], bv[j], acc[i][j]);
    }
  } else {
    // diagonal tile: entry (i, j) of a thread is on or below the diagonal
    // when j < i, or j == i and tx <= ty; the 6 entries with j > i never are
    const bool mine = tx <= ty;
    for (int kk = 0; kk < nbk; ++kk) {
      C av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[ty + TS * i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + TS * j];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < i; ++j) acc[i][j] = cfma(av[i], bv[j], acc[i][j]);
        if (mine) acc[i][i] = cfma(av[i], bv[i], acc[i][i]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int ri = i0 + ty + TS * i;
    if (ri >= m) continue;
    const int r = unband(ri, k, nbk);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ci = j0 + tx + TS * j;
      if (ci > ri) continue;      // upper entries of a diagonal tile: written as mirrors
      const int c = unband(ci, k, nbk);
      const C v = cadd(ld_elem<C>(a, f, r, c), acc[i][j]);
      st_elem<C>(a, f, r, c, v);
      if (ci < ri) st_elem<C>(a, f, c, r, cneg_if(v, (r < k) != (c < k)));
    }
  }
}

// acc[4][4] += A(64 x K) B(K x 64); 256 threads as 16 x 16, thread (tx, ty)
// owns rows ty + 16 i and columns tx + 16 j
template <typename C>
__device__ __forceinline__ void tile_mma(const C (*As)[MF_NB + 1], const C (*Bs)[64 + 1], int K, C acc[4][4],
                                         int tx, int ty) {
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

template <typename R>
__global__ void __launch_bounds__(256) mf_gj_update(MfArgs a, int f0, int k) {
  using C = typename CT<R>::T;
  constexpr int NB = MF_NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C(*As)[NB + 1] = reinterpret_cast<C(*)[NB + 1]>(smem_raw);
  C(*Bs)[64 + 1] = reinterpret_cast<C(*)[64 + 1]>(smem_raw + sizeof(C) * 64 * (NB + 1));
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(NB, p - k);
  const int m = n - nbk;
  const int nt = (m + 63) / 64;
  if ((int)blockIdx.y >= nt * nt) return;
  const int i0 = (blockIdx.y % nt) * 64, j0 = (blockIdx.y / nt) * 64;
  const C *fac = reinterpret_cast<const C *>(a.fac);
  const int64_t fo = f.fac_off;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int idx = tid; idx < 64 * nbk; idx += 256) {
    const int rr = idx % 64, j = idx / 64, ri = i0 + rr;
    As[rr][j] = ri < m ? ld_elem<C>(a, f, unband(ri, k, nbk), k + j) : czero<C>();
  }
  for (int idx = tid; idx < 64 * nbk; idx += 256) {
    const int j = idx % nbk, cc = idx / nbk, ci = j0 + cc;
    Bs[j][cc] = ci < m ? fac[fo + (int64_t)unband(ci, k, nbk) * p + k + j] : czero<C>();
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
    const int ri = i0 + ty + 16 * i;
    if (ri >= m) continue;
    const int r = unband(ri, k, nbk);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ci = j0 + tx + 16 * j;
      if (ci >= m) continue;
      const int c = unband(ci, k, nbk);
      st_elem<C>(a, f, r, c, cadd(ld_elem<C>(a, f, r, c), acc[i][j]));
    }
  }
}

// ------------------------------------------------------- substitutions
// Work items are (front, chunk of ROWS rows).  ROWS lanes ("row group") own
// the ROWS rows of an item, lane = row; a 256-thread CTA holds 256/ROWS row
// groups.  Columns are summed in fixed segments of MF_SEG columns: each
// segment's sum starts from zero and the segment sums are added in column
// order, so the result does not depend on how many row groups share an item
// (split) -- split only decides which group computes which segments.  With
// split > 1 the segment sums meet in shared memory and the first group of
// the item adds them.  Column values are gathered ROWS at a time (one per
// lane) and broadcast by shuffles; each lane keeps MF_UNROLL matrix loads in
// flight.
template <int W, typename C> __device__ __forceinline__ C shfl_w(unsigned mask, C v, int src) {
  v.x = __shfl_sync(mask, v.x, src, W);
  v.y = __shfl_sync(mask, v.y, src, W);
  return v;
}

// acc[q] = sum over columns [c0, c1) of M(r, c) * vec_q(c), q < NR, for one
// segment; M(r, c) at M[c * ld + r]; vec_q(c) comes from gather(c, q).
// Each matrix entry is loaded once for all NR right-hand sides.
template <int ROWS, int NR, bool AHEAD, typename C, typename Gather>
__device__ __forceinline__ void seg_dot(const C *__restrict__ M, int64_t ld, int r, bool row, int c0, int c1,
                                        int lane, unsigned mask, Gather gather, C (&acc)[NR]) {
  // the next chunk's vector values are requested before this chunk's
  // products (at the top tree levels a few warps carry a whole phase and
  // would otherwise wait for the dependent gather once per chunk)
  constexpr int U0 = sizeof(C) == 16 ? 8 : 32;  // FP64 is ALU-bound: fewer loads, more warps
  constexpr int U = NR > 1 ? (U0 / NR > 4 ? U0 / NR : 4) : U0;
  constexpr int UU = U < ROWS ? U : ROWS;
  static_assert(MF_SUB % ROWS == 0, "a sub-segment is a whole number of chunks");
  // each MF_SUB columns form a chain of their own (sub), folded into the
  // segment sum in column order: acc = ((s0 + s1) + s2) + s3
  C sub[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = sub[q] = czero<C>();
  C vn[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) vn[q] = c0 + lane < c1 ? gather(c0 + lane, q) : czero<C>();
  // complex128, one right-hand side, AHEAD (the per-level kernels; the
  // persistent sweep has no registers to spare): matrix loads run one block of UU
  // columns ahead of the products (the block after a chunk's last one is
  // the next chunk's first); complex64 and several right-hand sides keep
  // one block in registers
  constexpr bool PIPE = AHEAD && sizeof(C) == 16 && NR == 1;
  C m[UU];
  if (PIPE && c1 - c0 >= ROWS) {
#pragma unroll
    for (int u = 0; u < UU; ++u) m[u] = row ? M[(int64_t)(c0 + u) * ld + r] : czero<C>();
  }
  for (int cb = c0; cb < c1; cb += ROWS) {
    if ((cb - c0) % MF_SUB == 0) {
#pragma unroll
      for (int q = 0; q < NR; ++q) sub[q] = czero<C>();
    }
    C v[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) v[q] = vn[q];
    const int cn = cb + ROWS + lane;
#pragma unroll
    for (int q = 0; q < NR; ++q) vn[q] = cn < c1 ? gather(cn, q) : czero<C>();
    const int nv = min(ROWS, c1 - cb);
    if (nv == ROWS) {
      const bool next_full = c1 - (cb + ROWS) >= ROWS;
#pragma unroll
      for (int u0 = 0; u0 < ROWS; u0 += UU) {
        if (PIPE) {
          C mn[UU];
          const int nb = u0 + UU < ROWS ? cb + u0 + UU : cb + ROWS;   // the block loaded ahead
          const bool ahead = u0 + UU < ROWS || next_full;
#pragma unroll
          for (int u = 0; u < UU; ++u) mn[u] = (row && ahead) ? M[(int64_t)(nb + u) * ld + r] : czero<C>();
#pragma unroll
          for (int u = 0; u < UU; ++u)
#pragma unroll
            for (int q = 0; q < NR; ++q) sub[q] = cfma(m[u], shfl_w<ROWS>(mask, v[q], u0 + u), sub[q]);
#pragma unroll
          for (int u = 0; u < UU; ++u) m[u] = mn[u];
        } else {
#pragma unroll
          for (int u = 0; u < UU; ++u) m[u] = row ? M[(int64_t)(cb + u0 + u) * ld + r] : czero<C>();
#pragma unroll
          for (int u = 0; u < UU; ++u)
#pragma unroll
            for (int q = 0; q < NR; ++q) sub[q] = cfma(m[u], shfl_w<ROWS>(mask, v[q], u0 + u), sub[q]);
        }
      }
    } else {
      // ragged last chunk: only the valid columns (no multiply-adds by zero)
      int u = 0;
      for (; u + 4 <= nv; u += 4) {
        C m[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) m[t] = row ? M[(int64_t)(cb + u + t) * ld + r] : czero<C>();
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int q = 0; q < NR; ++q) sub[q] = cfma(m[t], shfl_w<ROWS>(mask, v[q], u + t), sub[q]);
      }
      for (; u < nv; ++u) {
        const C m = row ? M[(int64_t)(cb + u) * ld + r] : czero<C>();
#pragma unroll
        for (int q = 0; q < NR; ++q) sub[q] = cfma(m, shfl_w<ROWS>(mask, v[q], u), sub[q]);
      }
    }
    if ((cb + ROWS - c0) % MF_SUB == 0 || cb + ROWS >= c1) {
      const bool first = cb - c0 < MF_SUB;
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] = first ? sub[q] : cadd(acc[q], sub[q]);
    }
  }
}

// Going up, part 1: one warp per front forms w = [t at the pivots; 0] plus
// the children's update vectors (inverse extend-add maps); w_p goes to the
// pivot slots of wloc (kept for the way down) and w_b is the initial value
// of the front's update vector.
// What the upward sweep gathers for front f: at pivot position k < p the
// source entry (times s_x s_y in the symmetric form) plus the children's
// update vectors there, at border position k >= p the children's update
// vectors alone.  The same arithmetic serves the gather kernels and the
// products that gather on the fly (fused).
template <typename C> struct WSrc {
  const int *nodes, *inv[2];
  const C *uc[2];
  int bc[2];
  int64_t voff, coef_off, ycoef_off;
  int Hl;
  bool sym;
};
template <typename C>
__device__ __forceinline__ WSrc<C> wsrc_make(const MfArgs &a, const FrontDev &f, int nrhs) {
  WSrc<C> w;
  const StripDev st = a.strips[f.strip];
  w.nodes = a.nodes + f.node_off;
  w.voff = st.vec_off;
  w.coef_off = st.coef_off;
  w.ycoef_off = st.ycoef_off;
  w.Hl = st.y1 - st.y0;
  w.sym = a.sym != 0;
#pragma unroll
  for (int ci = 0; ci < 2; ++ci) {
    w.inv[ci] = nullptr;
    w.uc[ci] = nullptr;
    w.bc[ci] = 0;
    if (f.child[ci] >= 0) {
      const FrontDev ch = a.fronts[f.child[ci]];
      w.inv[ci] = a.inv + f.inv_off[ci];
      w.uc[ci] = reinterpret_cast<const C *>(a.ub_child) + ch.u_off * nrhs;
      w.bc[ci] = ch.b;
    }
  }
  return w;
}
// children's update vectors at position k, added to w in child order
template <typename C>
__device__ __forceinline__ C wsrc_children(const WSrc<C> &s, int k, int q, C w) {
#pragma unroll
  for (int ci = 0; ci < 2; ++ci)
    if (s.uc[ci]) {
      const int t = s.inv[ci][k];
      if (t >= 0) w = cadd(w, s.uc[ci][(int64_t)q * s.bc[ci] + t]);
    }
  return w;
}
// pivot position k < p; *gi = its slot in tloc / wloc
template <typename C>
__device__ __forceinline__ C wsrc_pivot(const MfArgs &a, const WSrc<C> &s, int k, int q, int64_t ldt, int64_t *gi) {
  const int node = s.nodes[k];
  *gi = q * ldt + s.voff + node;
  C w = reinterpret_cast<const C *>(a.tloc)[*gi];
  if (s.sym) {   // the source of D A x = D t
    const int ux = node / s.Hl, uy = node - ux * s.Hl;
    w = cmul(w, to_c(cmul(a.lsx[s.coef_off + ux], a.lsy[s.ycoef_off + uy]), C()));
  }
  return wsrc_children(s, k, q, w);
}

// one entry k of front f0 + fi, every right-hand side (k >= n: nothing)
template <typename R> __device__ __forceinline__ void up_gather_elem(const MfArgs &a, int f0, int fi, int k, int nrhs,
                                                                     int64_t ldt) {
  using C = typename CT<R>::T;
  const FrontDev f = a.fronts[f0 + fi];
  const int p = f.p, b = f.b, n = p + b;
  if (k >= n) return;
  const WSrc<C> src = wsrc_make<C>(a, f, nrhs);
  C *wl = reinterpret_cast<C *>(a.wloc);
  C *u = reinterpret_cast<C *>(a.ub_cur) + f.u_off * nrhs;
  for (int q = 0; q < nrhs; ++q) {
    if (k < p) {
      int64_t gi;
      const C w = wsrc_pivot(a, src, k, q, ldt, &gi);
      wl[gi] = w;
    } else {
      u[(int64_t)q * b + (k - p)] = wsrc_children(src, k, q, czero<C>());
    }
  }
}

// every entry of every front of a level, one thread per (front, entry):
// the dependent loads of an entry (its node, source, the children's
// update vectors) are short, and a front's entries run side by side
template <typename R>
__global__ void __launch_bounds__(256) mf_up_gather(MfArgs a, int f0, int nf, int nmax, int nrhs, int64_t ldt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nf * nmax) return;
  const int fi = (int)(e / nmax), k = (int)(e - (int64_t)fi * nmax);
  up_gather_elem<R>(a, f0, fi, k, nrhs, ldt);
}

// Going up, part 2: lane = border row r;
// u[r] = w_b[r] + sum_j (-G21)(r, j) w_p[j]  (w_b already in u).
// NR right-hand sides share every matrix load (NR > 1 requires split == 1).
// one (virtual) block of the upward products: the items of block vb
// FUSED: no gather pass before -- the products form the gathered entries
// themselves (WSrc, the gather's own arithmetic), the front's first row
// chunk stores w_p for the way down, and each row starts from the
// children's update vectors.
template <typename R, int ROWS, int NR, bool AHEAD = true, bool FUSED = false>
__device__ __forceinline__ void up_block(const MfArgs &a, const int2 *__restrict__ items, int nitems, int split,
                                         int nrhs, int64_t ldt, int vb, typename CT<R>::T *part) {
  using C = typename CT<R>::T;
  constexpr int GROUPS = 256 / ROWS;
  const int g = threadIdx.x / ROWS, lane = threadIdx.x % ROWS;
  const int ipc = GROUPS / split;
  const int il = g / split, sidx = g - il * split;
  const int it = vb * ipc + il;
  const bool active = it < nitems;
  const unsigned mask = ROWS == 32 ? 0xffffffffu : (0xffffu << (threadIdx.x & 16));
  int p = 0, b = 0, r = 0, seg0 = 0, seg1 = 0, nseg = 0;
  bool row = false;
  const C *G = nullptr;
  const int *nodes = nullptr, *pc = nullptr;
  int64_t voff = 0;
  C *u = nullptr;
  WSrc<C> src;
  bool writer = false;
  if (active) {
    const int2 item = items[it];
    const FrontDev f = a.fronts[item.x];
    p = f.p;
    b = f.b;
    voff = a.strips[f.strip].vec_off;
    if (FUSED) {
      src = wsrc_make<C>(a, f, nrhs);
      writer = item.y == 0;
    }
    G = reinterpret_cast<const C *>(a.fac) + f.fac_off + (int64_t)p * (p + b);  // -G21, b x p, ld b
    r = item.y * ROWS + lane;
    row = r < b;
    nodes = a.nodes + f.node_off;
    u = reinterpret_cast<C *>(a.ub_cur) + f.u_off * nrhs;
    if (a.pcol) pc = a.pcol + f.piv_off;
    nseg = (p + MF_SEG - 1) / MF_SEG;
    seg0 = sidx * nseg / split;
    seg1 = (sidx + 1) * nseg / split;
  }
  C *wl = reinterpret_cast<C *>(a.wloc);
  for (int q0 = 0; q0 < nrhs; q0 += NR) {
    C total[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) total[q] = czero<C>();
    if (active) {
      if (row && sidx == 0)
#pragma unroll
        for (int q = 0; q < NR; ++q)
          if (q0 + q < nrhs)
            total[q] = FUSED ? wsrc_children(src, p + r, q0 + q, czero<C>()) : u[(int64_t)(q0 + q) * b + r];
      auto gather = [&](int j, int q) {
        if (q0 + q >= nrhs) return czero<C>();
        if (!FUSED) return wl[(q0 + q) * ldt + voff + nodes[pc ? pc[j] : j]];
        int64_t gi;
        const C w = wsrc_pivot(a, src, pc ? pc[j] : j, q0 + q, ldt, &gi);
        if (writer) wl[gi] = w;
        return w;
      };
      for (int sg = seg0; sg < seg1; ++sg) {
        C sv[NR];
        seg_dot<ROWS, NR, AHEAD, C>(G, b, r, row, sg * MF_SEG, min(p, (sg + 1) * MF_SEG), lane, mask, gather, sv);
        if (split == 1) {
#pragma unroll
          for (int q = 0; q < NR; ++q) total[q] = cadd(total[q], sv[q]);
        } else {
          part[(il * MF_MAXSEG + sg) * ROWS + lane] = sv[0];
        }
      }
    }
    if (split > 1) {
      __syncthreads();
      if (active && row && sidx == 0) {
        for (int sg = 0; sg < nseg; ++sg) total[0] = cadd(total[0], part[(il * MF_MAXSEG + sg) * ROWS + lane]);
        u[(int64_t)q0 * b + r] = total[0];
      }
      __syncthreads();
    } else if (active && row) {
#pragma unroll
      for (int q = 0; q < NR; ++q)
        if (q0 + q < nrhs) u[(int64_t)(q0 + q) * b + r] = total[q];
    }
  }
}

// Coming down: lane = pivot row r;
// x[r] = sum_{c<p} Finv(r, c) w_p[c] - sum_{c>=p} H12(r, c) x_b[c].
// one (virtual) block of the downward products: the items of block vb
template <typename R, int ROWS, int NR, bool AHEAD = true>
__device__ __forceinline__ void down_block(const MfArgs &a, const int2 *__restrict__ items, int nitems, int split,
                                           int nrhs, int64_t ldt, int vb, typename CT<R>::T *part) {
  using C = typename CT<R>::T;
  constexpr int GROUPS = 256 / ROWS;
  const int g = threadIdx.x / ROWS, lane = threadIdx.x % ROWS;
  const int ipc = GROUPS / split;
  const int il = g / split, sidx = g - il * split;
  const int it = vb * ipc + il;
  const bool active = it < nitems;
  const unsigned mask = ROWS == 32 ? 0xffffffffu : (0xffffu << (threadIdx.x & 16));
  int p = 0, n = 0, r = 0, seg0 = 0, seg1 = 0, nseg = 0;
  bool row = false;
  const C *Fm = nullptr;
  const int *nodes = nullptr, *pc = nullptr;
  int64_t voff = 0;
  if (active) {
    const int2 item = items[it];
    const FrontDev f = a.fronts[item.x];
    p = f.p;
    n = p + f.b;
    voff = a.strips[f.strip].vec_off;
    Fm = reinterpret_cast<const C *>(a.fac) + f.fac_off;  // p x n, ld p
    r = item.y * ROWS + lane;
    row = r < p;
    nodes = a.nodes + f.node_off;
    if (a.pcol) pc = a.pcol + f.piv_off;
    nseg = (n + MF_SEG - 1) / MF_SEG;
    seg0 = sidx * nseg / split;
    seg1 = (sidx + 1) * nseg / split;
  }
  C *tv = reinterpret_cast<C *>(a.tloc);
  const C *wl = reinterpret_cast<const C *>(a.wloc);
  for (int q0 = 0; q0 < nrhs; q0 += NR) {
    C total[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) total[q] = czero<C>();
    if (active) {
      auto gather = [&](int c, int q) {
        if (q0 + q >= nrhs) return czero<C>();
        const int64_t base = (q0 + q) * ldt + voff;
        return c < p ? wl[base + nodes[pc ? pc[c] : c]] : cneg(tv[base + nodes[c]]);
      };
      for (int sg = seg0; sg < seg1; ++sg) {
        C sv[NR];
        seg_dot<ROWS, NR, AHEAD, C>(Fm, p, r, row, sg * MF_SEG, min(n, (sg + 1) * MF_SEG), lane, mask, gather, sv);
        if (split == 1) {
#pragma unroll
          for (int q = 0; q < NR; ++q) total[q] = cadd(total[q], sv[q]);
        } else {
          part[(il * MF_MAXSEG + sg) * ROWS + lane] = sv[0];
        }
      }
    }
    if (split > 1) {
      __syncthreads();
      if (active && row && sidx == 0) {
        for (int sg = 0; sg < nseg; ++sg) total[0] = cadd(total[0], part[(il * MF_MAXSEG + sg) * ROWS + lane]);
        tv[q0 * ldt + voff + nodes[r]] = total[0];
      }
      __syncthreads();
    } else if (active && row) {
#pragma unroll
      for (int q = 0; q < NR; ++q)
        if (q0 + q < nrhs) tv[(q0 + q) * ldt + voff + nodes[r]] = total[q];
    }
  }
}

template <typename R, int ROWS, int NR, bool FUSED>
__global__ void __launch_bounds__(256, 2) mf_up(MfArgs a, const int2 *__restrict__ items,
                                                                     int nitems, int split, int nrhs, int64_t ldt) {
  __shared__ typename CT<R>::T part[MF_MAXSEG * 256 / 2];
  up_block<R, ROWS, NR, true, FUSED>(a, items, nitems, split, nrhs, ldt, blockIdx.x, part);
}

template <typename R, int ROWS, int NR>
__global__ void __launch_bounds__(256, 2) mf_down(MfArgs a, const int2 *__restrict__ items,
                                                                       int nitems, int split, int nrhs,
                                                                       int64_t ldt) {
  __shared__ typename CT<R>::T part[MF_MAXSEG * 256 / 2];
  down_block<R, ROWS, NR>(a, items, nitems, split, nrhs, ldt, blockIdx.x, part);
}

// Products split across the grid: one warp per (work item, MF_SUB-column
// chain) anywhere in the grid writes the chain's sum per row, and a second
// launch folds the chains into segment sums and the segment sums into the
// total, in column order -- the association seg_dot and the in-block
// split use, so the choice between them changes no result.  At the top tree levels a few fronts
// carry a whole phase; an in-block split keeps an item on one SM, whose FP64
// pipe then sets the phase time.
template <typename R, bool UP, bool FUSED>
__global__ void __launch_bounds__(256) mf_seg_partial(MfArgs a, const int2 *__restrict__ items, int nitems,
                                                      int nsubmax, int64_t ldt) {
  using C = typename CT<R>::T;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = (int64_t)blockIdx.x * 8 + warp;
  if (u >= (int64_t)nitems * nsubmax) return;
  const int it = (int)(u / nsubmax), sg = (int)(u - (int64_t)it * nsubmax);
  const int2 item = items[it];
  const FrontDev f = a.fronts[item.x];
  const int p = f.p, b = f.b, n = p + b;
  const int cols = UP ? p : n;
  if (sg * MF_SUB >= cols) return;
  const int64_t voff = a.strips[f.strip].vec_off;
  const int *nodes = a.nodes + f.node_off;
  const int *pc = a.pcol ? a.pcol + f.piv_off : nullptr;
  const C *wl = reinterpret_cast<const C *>(a.wloc);
  const C *tv = reinterpret_cast<const C *>(a.tloc);
  const C *fac = reinterpret_cast<const C *>(a.fac) + f.fac_off;
  const int r = item.y * 32 + lane;
  const bool row = r < (UP ? b : p);
  C sv[1];
  if (UP) {
    WSrc<C> src;
    if (FUSED) src = wsrc_make<C>(a, f, 1);
    auto gather = [&](int j, int) {
      if (!FUSED) return wl[voff + nodes[pc ? pc[j] : j]];
      int64_t gi;
      const C w = wsrc_pivot(a, src, pc ? pc[j] : j, 0, ldt, &gi);
      if (item.y == 0) const_cast<C *>(wl)[gi] = w;
      return w;
    };
    seg_dot<32, 1, true, C>(fac + (int64_t)p * n, b, r, row, sg * MF_SUB, min(cols, (sg + 1) * MF_SUB), lane,
                            0xffffffffu, gather, sv);
  } else {
    auto gather = [&](int c, int) {
      return c < p ? wl[voff + nodes[pc ? pc[c] : c]] : cneg(tv[voff + nodes[c]]);
    };
    seg_dot<32, 1, true, C>(fac, p, r, row, sg * MF_SUB, min(cols, (sg + 1) * MF_SUB), lane, 0xffffffffu, gather,
                            sv);
  }
  reinterpret_cast<C *>(a.segpart)[u * 32 + lane] = sv[0];
}

template <typename R, bool UP, bool FUSED>
__global__ void __launch_bounds__(256) mf_seg_reduce(MfArgs a, const int2 *__restrict__ items, int nitems,
                                                     int nsubmax) {
  using C = typename CT<R>::T;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int it = (int)(t >> 5), lane = (int)(t & 31);
  if (it >= nitems) return;
  const int2 item = items[it];
  const FrontDev f = a.fronts[item.x];
  const int p = f.p, b = f.b;
  const int r = item.y * 32 + lane;
  if (r >= (UP ? b : p)) return;
  const int cols = UP ? p : p + b;
  const int nsub = (cols + MF_SUB - 1) / MF_SUB, per = MF_SEG / MF_SUB;
  const C *P = reinterpret_cast<const C *>(a.segpart) + (int64_t)it * nsubmax * 32 + lane;
  C *u = reinterpret_cast<C *>(a.ub_cur) + f.u_off;
  C total = czero<C>();
  if (UP) total = FUSED ? wsrc_children(wsrc_make<C>(a, f, 1), p + r, 0, czero<C>()) : u[r];
  for (int k0 = 0; k0 < nsub; k0 += per) {
    C seg = P[k0 * 32];
    for (int k = k0 + 1; k < min(k0 + per, nsub); ++k) seg = cadd(seg, P[k * 32]);
    total = cadd(total, seg);
  }
  if (UP) u[r] = total;
  else reinterpret_cast<C *>(a.tloc)[a.strips[f.strip].vec_off + a.nodes[f.node_off + r]] = total;
}

template <typename R, bool UP, bool FUSED = false>
void mf_seg_launch(const MfArgs &a, const int2 *items, int nitems, int cols_max, int64_t ldt, cudaStream_t st) {
  const int nsubmax = (cols_max + MF_SUB - 1) / MF_SUB;
  const int64_t units = (int64_t)nitems * nsubmax;
  mf_seg_partial<R, UP, FUSED><<<(unsigned)((units + 7) / 8), 256, 0, st>>>(a, items, nitems, nsubmax, ldt);
  mf_seg_reduce<R, UP, FUSED><<<(unsigned)(((int64_t)nitems * 32 + 255) / 256), 256, 0, st>>>(a, items, nitems,
                                                                                              nsubmax);
  count_launch(2);
}

// ------------------------------------------- persistent one-strip sweep
// Grid-wide barrier of a cooperative launch: bar[0] counts arrivals, bar[1]
// is the generation.  A block that polls more than `limit` times sets bit 0
// of *flag and gives up; a block that sees the flag gives up too.  Returns
// false (uniformly across the block) if the barrier was abandoned.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *flag, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vb = bar;
    volatile int *vf = flag;
    ok = 1;
    const unsigned gen = vb[1];
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      long long it = 0;
      while (vb[1] == gen) {
        if (++it > limit || (*vf & 1)) {
          atomicOr(flag, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename R, int ROWS>
__device__ __forceinline__ void up_items(const MfArgs &a, const StripLevel &l, int64_t ldt,
                                         typename CT<R>::T *part) {
  const int ipc = (256 / ROWS) / l.split_up;
  const int nvb = (l.up_n + ipc - 1) / ipc;
  for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x)
    up_block<R, ROWS, 1, false, true>(a, a.items_sweep + l.up_first, l.up_n, l.split_up, 1, ldt, vb, part);
}

template <typename R, int ROWS>
__device__ __forceinline__ void down_items(const MfArgs &a, const StripLevel &l, int64_t ldt,
                                           typename CT<R>::T *part) {
  const int ipc = (256 / ROWS) / l.split_down;
  const int nvb = (l.down_n + ipc - 1) / ipc;
  for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x)
    down_block<R, ROWS, 1, false>(a, a.items_sweep + l.down_first, l.down_n, l.split_down, 1, ldt, vb, part);
}

// The launches of one strip's solve in the sequential orders (residual
// restriction, per level the upward products -- gathering their own
// entries -- per level the downward products, the add-back) as one launch:
// the same device code, the launch boundaries replaced by grid barriers.
template <typename R>
__global__ void __launch_bounds__(256, 2)
    mf_strip_sweep(MfArgs a, const void *ub0, const void *ub1, GridDev g, StripDev s, const StripLevel *lv,
                   int depth, const double2 *__restrict__ v, double2 *__restrict__ z, unsigned *bar, int *flag,
                   long long limit, int64_t ldt) {
  using C = typename CT<R>::T;
  __shared__ C part[MF_MAXSEG * 256 / 2];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int Hl = s.y1 - s.y0;
  const int64_t nl = (int64_t)(s.x1 - s.x0) * Hl;
  C *t = reinterpret_cast<C *>(a.tloc) + s.vec_off;
  // t = R_s^I (v - A z): the strip's owned columns, zero elsewhere
  {
    const int64_t lo = (int64_t)(s.c0 - s.x0) * g.ny, hi = (int64_t)(s.c1 - s.x0) * g.ny;
    const int64_t g0 = (int64_t)s.x0 * g.ny;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += stride) {
      C val = czero<C>();
      if (l >= lo && l < hi) {
        const int64_t gi = g0 + l;
        const int i = (int)(gi / g.ny), j = (int)(gi - (int64_t)i * g.ny);
        val = to_c(csub(v[gi], grid_row(g, z, gi, i, j)), C());
      }
      t[l] = val;
    }
  }
  if (!grid_barrier(bar, flag, limit)) return;
  for (int L = depth - 1; L >= 0; --L) {
    const StripLevel l = lv[L];
    if (l.nf == 0) continue;
    MfArgs al = a;
    al.ub_cur = const_cast<void *>(L & 1 ? ub1 : ub0);
    al.ub_child = L & 1 ? ub0 : ub1;
    // (the products gather their own entries: no gather phase, one barrier per level)
    if (l.rows_up == 16) up_items<R, 16>(al, l, ldt, part);
    else up_items<R, 32>(al, l, ldt, part);
    if (!grid_barrier(bar, flag, limit)) return;
  }
  for (int L = 0; L < depth; ++L) {
    const StripLevel l = lv[L];
    if (l.down_n == 0) continue;
    if (l.rows_down == 16) down_items<R, 16>(a, l, ldt, part);
    else down_items<R, 32>(a, l, ldt, part);
    if (!grid_barrier(bar, flag, limit)) return;
  }
  // z += E_s t
  double2 *zs = z + (int64_t)s.x0 * g.ny;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += stride)
    zs[l] = cadd(zs[l], to_d(t[l]));
}

// ------------------------------------------------------------ launchers
// small-front launch shape: a warp per front (4 per CTA) up to n = 32, one
// 128-thread CTA per front above
template <typename R> static size_t small_smem(int ldn, int fpc) {
  using C = typename CT<R>::T;
  return sizeof(C) * fpc * (size_t)(ldn * (ldn + 1) + 2 * ldn) + sizeof(int) * fpc * (size_t)ldn;
}
template <typename R> static size_t row_smem() {
  using C = typename CT<R>::T;
  return sizeof(C) * (MF_NB * (MF_NB + 1) + MF_PANEL_THREADS * (MF_NB + 1));
}
template <typename R> static size_t gemm_smem() {
  using C = typename CT<R>::T;
  return sizeof(C) * (64 * (MF_NB + 1) + MF_NB * (64 + 1));
}

template <typename R> cudaError_t mf_setup_attributes() {
  cudaError_t e;
  e = cudaFuncSetAttribute(mf_gj_small<R, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mf_gj_small<R, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mf_gj_row<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem<R>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mf_gj_update_sym<R, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)gemm_smem<R>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(mf_gj_update<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<R>());
}

template <typename R>
void mf_factor_level(const MfArgs &a, const LevelInfo &L, int level, cudaStream_t st, LaunchHook *hook,
                     int tc_fmt) {
  if (L.nf == 0) return;
  if (L.min_n <= MF_SMALL) {
    const int ldn = std::min(L.max_n, MF_SMALL);
    if (hook) hook->before(K_SMALL, level, 0);
    if (ldn <= 32) {
      mf_gj_small<R, 32><<<(L.nf + 3) / 4, 128, small_smem<R>(ldn, 4), st>>>(a, L.f0, L.nf, ldn);
    } else {
      mf_gj_small<R, 128><<<L.nf, 128, small_smem<R>(ldn, 1), st>>>(a, L.f0, L.nf, ldn);
    }
    if (hook) hook->after(K_SMALL, level, 0);
    count_launch();
  }
  if (L.max_n > MF_SMALL) {
    const int64_t nn = (int64_t)L.max_n * L.max_n;
    const int gy = (int)std::min<int64_t>((nn + 255) / 256, 4096);
    mf_assemble<R><<<dim3(L.nf, gy), 256, 0, st>>>(a, L.f0);
    count_launch();
    for (int k = 0; k < L.max_p; k += MF_NB) {
      const int m = L.max_n - std::min(MF_NB, std::max(1, L.max_p - k));
      const int tiles = std::max(1, (m + MF_PANEL_THREADS - 1) / MF_PANEL_THREADS);
      const int nt = std::max(1, (m + 63) / 64);
      if (a.pcol) {
        mf_gj_pivot<R><<<L.nf, 256, 0, st>>>(a, L.f0, k);
        count_launch();
      }
      mf_gj_diag<R><<<L.nf, MF_PANEL_THREADS, 0, st>>>(a, L.f0, k);
      if (a.sym && a.fp64_tc && sizeof(R) == 8) mf_oz_col_launch(a, L, k, st);
      else mf_gj_col<R><<<dim3(L.nf, tiles), MF_PANEL_THREADS, 0, st>>>(a, L.f0, k);
      if (hook) hook->before(K_UPDATE, level, k);
      if (tc_fmt >= 0 && sizeof(R) == 4) {
        mf_tc_update_launch(a, L, k, tc_fmt, st);
      } else if (a.sym && a.fp64_tc && sizeof(R) == 8) {
        mf_oz_update_launch(a, L, k, st);
      } else if (a.sym) {
        const int tm = L.upd_tile == 32 ? 32 : 64, nts = std::max(1, (m + tm - 1) / tm);
        const size_t sm = sizeof(typename CT<R>::T) * (tm * (MF_NB + 1) + MF_NB * (tm + 1));
        if (tm == 32) mf_gj_update_sym<R, 32><<<dim3(L.nf, nts * (nts + 1) / 2), 64, sm, st>>>(a, L.f0, k);
        else mf_gj_update_sym<R, 64><<<dim3(L.nf, nts * (nts + 1) / 2), 256, sm, st>>>(a, L.f0, k);
      } else if (L.upd_tile == 32) {
        const int nt32 = std::max(1, (m + 31) / 32);
        mf_gj_update32<R><<<dim3(L.nf, nt32 * nt32), 64, 0, st>>>(a, L.f0, k);
      } else {
        mf_gj_update<R><<<dim3(L.nf, nt * nt), 256, gemm_smem<R>(), st>>>(a, L.f0, k);
      }
      if (hook) hook->after(K_UPDATE, level, k);
      if (a.sym) mf_gj_row_mirror<R><<<dim3(L.nf, tiles), MF_PANEL_THREADS, 0, st>>>(a, L.f0, k);
      else mf_gj_row<R><<<dim3(L.nf, tiles), MF_PANEL_THREADS, row_smem<R>(), st>>>(a, L.f0, k);
      count_launch(4);
    }
  }
}

template <typename R>
void mf_up_gather_level(const MfArgs &a, const LevelInfo &L, int nrhs, int64_t ldt, cudaStream_t st) {
  if (L.nf == 0) return;
  const int64_t ne = (int64_t)L.nf * L.max_n;
  mf_up_gather<R><<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(a, L.f0, L.nf, L.max_n, nrhs, ldt);
  count_launch();
}

template <typename R>
void mf_up_level(const MfArgs &a, const int2 *items, int nitems, int rows, int split, int nrhs, int64_t ldt,
                 cudaStream_t st, int cols_max, bool fused) {
  if (nitems == 0) return;
  if (nrhs > 1) split = 1;  // several right-hand sides: every group keeps its segments in registers
  if (split == MF_SPLIT_GRID) {
    if (rows == 32 && a.segpart && cols_max > 0) {
      if (fused) mf_seg_launch<R, true, true>(a, items, nitems, cols_max, ldt, st);
      else mf_seg_launch<R, true, false>(a, items, nitems, cols_max, ldt, st);
      return;
    }
    split = 1;
  }
  if (split > 1 && cols_max > 0 && (cols_max + MF_SEG - 1) / MF_SEG > MF_MAXSEG) split = 1;
  const int ipc = (256 / rows) / split;
  const int grid = (nitems + ipc - 1) / ipc;
  const int nr = (nrhs >= 4 && sizeof(R) == 4) ? 4 : (nrhs >= 2 ? 2 : 1);
#define STDD_UP(RW, NRV)                                                                \
  do {                                                                                  \
    if (fused) mf_up<R, RW, NRV, true><<<grid, 256, 0, st>>>(a, items, nitems, split, nrhs, ldt);  \
    else mf_up<R, RW, NRV, false><<<grid, 256, 0, st>>>(a, items, nitems, split, nrhs, ldt);       \
  } while (0)
  if (rows == 16) {
    if (nr == 4) STDD_UP(16, 4); else if (nr == 2) STDD_UP(16, 2); else STDD_UP(16, 1);
  } else {
    if (nr == 4) STDD_UP(32, 4); else if (nr == 2) STDD_UP(32, 2); else STDD_UP(32, 1);
  }
#undef STDD_UP
  count_launch();
}

template <typename R>
void mf_down_level(const MfArgs &a, const int2 *items, int nitems, int rows, int split, int nrhs, int64_t ldt,
                   cudaStream_t st, int cols_max) {
  if (nitems == 0) return;
  if (nrhs > 1) split = 1;
  if (split == MF_SPLIT_GRID) {
    if (rows == 32 && a.segpart && cols_max > 0) {
      mf_seg_launch<R, false>(a, items, nitems, cols_max, ldt, st);
      return;
    }
    split = 1;
  }
  if (split > 1 && cols_max > 0 && (cols_max + MF_SEG - 1) / MF_SEG > MF_MAXSEG) split = 1;
  const int ipc = (256 / rows) / split;
  const int grid = (nitems + ipc - 1) / ipc;
  const int nr = (nrhs >= 4 && sizeof(R) == 4) ? 4 : (nrhs >= 2 ? 2 : 1);
#define STDD_DOWN(RW, NRV) mf_down<R, RW, NRV><<<grid, 256, 0, st>>>(a, items, nitems, split, nrhs, ldt)
  if (rows == 16) {
    if (nr == 4) STDD_DOWN(16, 4); else if (nr == 2) STDD_DOWN(16, 2); else STDD_DOWN(16, 1);
  } else {
    if (nr == 4) STDD_DOWN(32, 4); else if (nr == 2) STDD_DOWN(32, 2); else STDD_DOWN(32, 1);
  }
#undef STDD_DOWN
  count_launch();
}

static int g_sweep_sms = 0, g_sweep_per[2] = {0, 0};

// SMs and co-resident blocks per SM of the persistent sweep (queried once)
template <typename R> static int sweep_per_sm() {
  int &per = g_sweep_per[sizeof(R) == 8 ? 1 : 0];
  if (per == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sweep_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mf_strip_sweep<R>, 256, 0);
    per = std::max(1, per);
  }
  return per;
}

int mf_strip_sweep_grid() {
  sweep_per_sm<float>();
  return g_sweep_sms * sweep_per_sm<double>();
}

template <typename R>
cudaError_t mf_strip_sweep_launch(const MfArgs &a, const void *ub0, const void *ub1, const GridDev &g,
                                  const StripDev &s, const StripLevel *lv_dev, int depth, const double2 *v,
                                  double2 *z, unsigned *bar, int *sweep_flag, long long wait_limit,
                                  int blocks_per_sm, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(g_sweep_sms * std::max(1, std::min(blocks_per_sm, sweep_per_sm<R>()))));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident, or the launch fails
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int64_t ldt = 0;   // one right-hand side
  count_launch();
  return cudaLaunchKernelEx(&cfg, mf_strip_sweep<R>, a, ub0, ub1, g, s, lv_dev, depth, v, z, bar, sweep_flag,
                            wait_limit, ldt);
}

template cudaError_t mf_strip_sweep_launch<double>(const MfArgs &, const void *, const void *, const GridDev &,
                                                   const StripDev &, const StripLevel *, int, const double2 *,
                                                   double2 *, unsigned *, int *, long long, int, cudaStream_t);
template cudaError_t mf_strip_sweep_launch<float>(const MfArgs &, const void *, const void *, const GridDev &,
                                                  const StripDev &, const StripLevel *, int, const double2 *,
                                                  double2 *, unsigned *, int *, long long, int, cudaStream_t);

__global__ void k_factor_begin(int *flag, unsigned long long *n_raised, double *min_pivot) {
  *flag = 0;
  *n_raised = 0ull;
  *min_pivot = INFINITY;
}

void mf_factor_begin(const MfArgs &a, cudaStream_t st) {
  k_factor_begin<<<1, 1, 0, st>>>(a.flag, a.n_raised, a.min_pivot);
  count_launch();
}

template cudaError_t mf_setup_attributes<double>();
template cudaError_t mf_setup_attributes<float>();
template void mf_factor_level<double>(const MfArgs &, const LevelInfo &, int, cudaStream_t, LaunchHook *, int);
template void mf_factor_level<float>(const MfArgs &, const LevelInfo &, int, cudaStream_t, LaunchHook *, int);
template void mf_up_gather_level<double>(const MfArgs &, const LevelInfo &, int, int64_t, cudaStream_t);
template void mf_up_gather_level<float>(const MfArgs &, const LevelInfo &, int, int64_t, cudaStream_t);
template void mf_up_level<double>(const MfArgs &, const int2 *, int, int, int, int, int64_t, cudaStream_t, int,
                                  bool);
template void mf_up_level<float>(const MfArgs &, const int2 *, int, int, int, int, int64_t, cudaStream_t, int, bool);
template void mf_down_level<double>(const MfArgs &, const int2 *, int, int, int, int, int64_t, cudaStream_t, int);
template void mf_down_level<float>(const MfArgs &, const int2 *, int, int, int, int, int64_t, cudaStream_t, int);

}  // namespace stdd

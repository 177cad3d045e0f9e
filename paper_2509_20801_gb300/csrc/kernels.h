// Kernel launchers shared by the C-ABI layer (api.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace stdd {

// kernels launched by this library (all contexts), for launch accounting
extern long long g_launches;
inline void count_launch(int n = 1) { __atomic_add_fetch(&g_launches, (long long)n, __ATOMIC_RELAXED); }

constexpr int MF_NB = 32;             // pivot block of the blocked Gauss-Jordan sweep
constexpr int MF_PANEL_THREADS = 128; // rows / columns per panel tile
constexpr int MF_SMALL = 64;          // fronts with n <= MF_SMALL are swept in shared memory
constexpr int MF_SEG = 128;           // columns per fixed summation segment of the sweeps
constexpr int MF_MAXSEG = 16;         // segments an item may have when its columns are split
constexpr int MF_SPLIT_GRID = 16;     // split value: one warp per (item, sub-segment) anywhere in the grid
constexpr int MF_SUB = 32;            // columns per chain inside a segment (segment = chains added in order)
static_assert(MF_SEG % MF_SUB == 0, "segments are whole sub-segments");

// Everything a multifrontal kernel needs (device pointers).
struct MfArgs {
  const FrontDev *fronts;
  const StripDev *strips;
  const int *nodes, *cmap, *inv;
  const double2 *cxm, *cxp;   // per-strip x couplings, indexed coef_off + local column
  const double2 *cym, *cyp;   // per-box y couplings, indexed ycoef_off + local row
  const double *eps;          // global node permittivity
  double k0sq;
  int H;                      // ny (row stride of the global permittivity)
  void *fac;                  // factor storage (complex R)
  void *ws_cur;               // F22 of this level
  const void *ws_child;       // F22 of the level below
  void *tloc;                 // local fields, [nrhs][ldt]: t on entry, x on exit
  void *wloc;                 // w at the pivots of every front (going up), [nrhs][ldt]
  void *ub_cur;               // forward update vectors of this level
  const void *ub_child;       // and of the level below
  int *flag;                  // bit 0: zero / non-finite pivot
  double *min_pivot;          // min |pivot| (atomicMin on the bit pattern)
  double piv_floor;           // static pivoting: |pivot| < piv_floor is raised to it (0: off)
  unsigned long long *n_raised;  // pivots raised
  // Partial pivoting restricted to each front's pivot rows (null: off).
  // pcol[piv_off + j] = the pivot (0..p-1) whose value column j of the
  // stored F11^-1 and -G21 blocks multiplies; panel: pivot-search scratch.
  int *pcol;
  void *panel;
  const int2 *items_sweep;    // the substitution work items (persistent sweep)
  // Symmetric form (sym = 1): the fronts hold D A_i, D = diag(s_x s_y) of the
  // local stretches, which is complex symmetric; the Gauss-Jordan working
  // matrix then stays symmetric up to the sign of its cross blocks and the
  // update computes the lower half only.  lsx / lsy: local node stretches,
  // indexed like cxm / cym.
  const double2 *lsx, *lsy;
  int sym;
  // complex128 symmetric form: 1 = large-front updates on the tensor cores
  // by exact splitting into BF16 slices (FP64 accuracy), 0 = FP64 pipe
  int fp64_tc;
  // substitution products split across the grid (split == MF_SPLIT_GRID):
  // one partial sum per (work item, column segment, row), summed in segment
  // order by a second launch
  void *segpart;
};

struct LevelInfo {
  int f0, nf;                 // fronts [f0, f0 + nf) of the level
  int max_p, max_b, max_n, min_n;
  int64_t up_off, down_off;   // offsets of the level's work items
  int n_up, n_down;           // (front, row chunk) items going up / down
  int rows_up, rows_down;     // rows per item: 16 or 32
  int split_up, split_down;   // row groups sharing one item's columns (1..8)
  int split_up1, split_down1; // the same for launches over one strip's fronts (sequential orders)
  int upd_tile;               // blocked-update tile edge of the level: 64 or 32 (chosen by timing)
  int pad_;
};

// Optional per-launch observer (phase profiling): kind is one of the K_*
// values, level the tree level, k the pivot-block step (factorization).
enum { K_SMALL = 0, K_UPDATE = 1, K_UP = 2, K_DOWN = 3, K_SWEEP = 4, K_COUNT = 5 };
struct LaunchHook {
  virtual void before(int kind, int level, int k) = 0;
  virtual void after(int kind, int level, int k) = 0;
};

template <typename R> cudaError_t mf_setup_attributes();
// start of a factorization: clear the pivot flag and the raised-pivot count,
// set the smallest-pivot record to +inf (one kernel, so it can be captured)
void mf_factor_begin(const MfArgs &a, cudaStream_t st);
// tc_fmt: -1 CUDA-core updates; 0 / 1 tensor-core updates with FP16 / BF16 inputs
template <typename R>
void mf_factor_level(const MfArgs &a, const LevelInfo &L, int level, cudaStream_t st, LaunchHook *hook = nullptr,
                     int tc_fmt = -1);

// ---- tensor-core front updates (kernels_tc.cu), complex64 fronts only
cudaError_t tc_setup_attributes();
void mf_tc_update_launch(const MfArgs &a, const LevelInfo &L, int k, int fmt, cudaStream_t st);
// symmetric form, complex128: the update on the BF16 tensor cores by exact splitting
void mf_oz_update_launch(const MfArgs &a, const LevelInfo &L, int k, cudaStream_t st);
void mf_oz_col_launch(const MfArgs &a, const LevelInfo &L, int k, cudaStream_t st);
int oz_tile_product(int kc, const double2 *C, const double2 *R, double2 *D, cudaError_t *err);
// one 64 x kc by kc x 128 complex tile product on the tensor cores from host
// arrays: 0 ok, 1 wait timed out, -1 CUDA error (*err)
int tc_tile_product(int fmt, int kc, const float2 *C, const float2 *R, float2 *D, cudaError_t *err);
template <typename R>
void mf_up_gather_level(const MfArgs &a, const LevelInfo &L, int nrhs, int64_t ldt, cudaStream_t st);

// One strip's share of one tree level, for the persistent sweep.
struct StripLevel {
  int f0, nf;                  // the strip's fronts at this level
  int up_n, down_n;            // its upward / downward work items
  int64_t up_first, down_first;
  int rows_up, rows_down, split_up, split_down;
  int max_n, pad_;             // the level's largest front (entries per front in the gather)
};
struct GridDev;
// Persistent sweep of one strip (one right-hand side): t = R_s^I (v - A z),
// the upward products leaves to root, the downward ones root to leaves,
// then z += E_s t -- one cooperative launch, the levels separated by a
// grid-wide barrier whose waits give up after wait_limit polls (then
// *sweep_flag |= 1 and every block returns).  bar: two zeroed unsigned.
template <typename R>
cudaError_t mf_strip_sweep_launch(const MfArgs &a, const void *ub0, const void *ub1, const GridDev &g,
                                  const StripDev &s, const StripLevel *lv_dev, int depth, const double2 *v,
                                  double2 *z, unsigned *bar, int *sweep_flag, long long wait_limit,
                                  int blocks_per_sm, cudaStream_t st);
int mf_strip_sweep_grid();   // blocks of the persistent sweep (co-resident); call outside stream capture
template <typename R>
void mf_up_level(const MfArgs &a, const int2 *items, int nitems, int rows, int split, int nrhs, int64_t ldt,
                 cudaStream_t st, int cols_max = 0, bool fused = false);
template <typename R>
void mf_down_level(const MfArgs &a, const int2 *items, int nitems, int rows, int split, int nrhs, int64_t ldt,
                   cudaStream_t st, int cols_max = 0);

// ---- FDFD / DDM vector kernels (kernels_fdfd.cu)
struct GridDev {
  int nx, ny;
  double k0sq;
  const double *eps;
  const double2 *cxm, *cxp;   // global x couplings (nx)
  const double2 *cym, *cyp;   // y couplings (ny)
};

// Row idx = i * ny + j of the global operator applied to x (the stretched
// 5-point stencil of Eqs. 2, 9; zero field beyond the grid).
// Outside the PML the four couplings are real: the row then takes real
// times complex products (half the FP64 operations; for finite values the
// same results as the complex form, whose extra terms are products with 0).
__device__ __forceinline__ double2 grid_row(const GridDev &g, const double2 *__restrict__ x, int64_t idx, int i,
                                            int j) {
  const double2 xm = g.cxm[i], xp = g.cxp[i], ym = g.cym[j], yp = g.cyp[j];
  double2 d;
  d.x = g.k0sq * g.eps[idx] - xm.x - xp.x - ym.x - yp.x;
  d.y = -xm.y - xp.y - ym.y - yp.y;
  if (xm.y == 0.0 && xp.y == 0.0 && ym.y == 0.0 && yp.y == 0.0 && i > 0 && i < g.nx - 1 && j > 0 &&
      j < g.ny - 1) {
    const double2 c = x[idx], w = x[idx - g.ny], e = x[idx + g.ny], s = x[idx - 1], n = x[idx + 1];
    double2 acc = make_double2(d.x * c.x, d.x * c.y);
    acc.x = fma(xm.x, w.x, acc.x);
    acc.y = fma(xm.x, w.y, acc.y);
    acc.x = fma(xp.x, e.x, acc.x);
    acc.y = fma(xp.x, e.y, acc.y);
    acc.x = fma(ym.x, s.x, acc.x);
    acc.y = fma(ym.x, s.y, acc.y);
    acc.x = fma(yp.x, n.x, acc.x);
    acc.y = fma(yp.x, n.y, acc.y);
    return acc;
  }
  double2 acc = cmul(d, x[idx]);
  if (i > 0) acc = cfma(xm, x[idx - g.ny], acc);
  if (i < g.nx - 1) acc = cfma(xp, x[idx + g.ny], acc);
  if (j > 0) acc = cfma(ym, x[idx - 1], acc);
  if (j < g.ny - 1) acc = cfma(yp, x[idx + 1], acc);
  return acc;
}
// y = A x (global stretched 5-point operator), nrhs vectors of nx*ny
void launch_stencil(const GridDev &g, const double2 *x, double2 *y, cudaStream_t st);
// r = b - A x
void launch_residual(const GridDev &g, const double2 *b, const double2 *x, double2 *r, cudaStream_t st);
// local[k] = R_k^I v (owned columns of v, zero elsewhere), all strips, R = double or float
template <typename R>
void launch_restrict(const StripDev *strips_dev, int nsub, int64_t nloc, int ny, const int *col_strip,
                     const double2 *v, void *tloc, cudaStream_t st);
// z = sum_k E_k local[k] (gather form: <= 3 strips per column, fixed order)
template <typename R>
void launch_synthesize(const StripDev *strips_dev, int nsub, int nx, int ny, const int *col_strip,
                       const void *tloc, double2 *z, cudaStream_t st);
// 2-D boxes (px x py, box id kx * py + ky): restriction to the owned blocks
// and synthesis of the full local fields (<= 9 boxes per node)
template <typename R>
void launch_restrict_box(const StripDev *boxes_dev, int nbox, int64_t nloc_max, int ny, const double2 *v, void *tloc,
                         cudaStream_t st);
template <typename R>
void launch_synthesize_box(const StripDev *boxes_dev, int px, int py, int nx, int ny, const int *col_box,
                           const int *row_box, const void *tloc, double2 *z, cudaStream_t st);
// out[2k] = ||e_k^F||^2, out[2k+1] = ||e_k||^2 of every strip's local field
template <typename R>
void launch_strip_norms(const StripDev *strips_dev, int nsub, int ny, const void *tloc, double *out,
                        cudaStream_t st);
// one strip (multiplicative order): its local source R_s^I (v - A z), and
// z += E_s e_s (tloc is the base of all strips' local fields)
template <typename R>
void launch_restrict_residual_strip(const GridDev &g, const StripDev &s, const double2 *v, const double2 *z,
                                    void *tloc, cudaStream_t st);
template <typename R> void launch_add_strip(const StripDev &s, int ny, const void *tloc, double2 *z, cudaStream_t st);
// local strip k only: tloc_k = t (converted), and back
template <typename R> void launch_to_local(const double2 *t, void *tloc, int64_t n, cudaStream_t st);
template <typename R> void launch_from_local(const void *tloc, double2 *z, int64_t n, cudaStream_t st);

// ---- band space (band-space FGMRES): the interface bands as column
// intervals iv[k] = (first column, width), element offsets off[k]; n
// elements.  iv1 / off1 / n1: the same widened by one column each side.
struct BandDev {
  const int2 *iv;
  const int64_t *off;
  int niv;
  int64_t n;
  const int2 *iv1;
  const int64_t *off1;
  int niv1;
  int64_t n1;
};
// every strip's owned part of the band vector s (zero elsewhere) into tloc
template <typename R>
void launch_restrict_band(const StripDev *strips_dev, int nsub, int64_t nloc_max, int ny, const int64_t *colband,
                          const double2 *s, void *tloc, cudaStream_t st);
// z = sum_k E_k local[k] on the widened band only
template <typename R>
void launch_synthesize_band(const StripDev *strips_dev, int nsub, int ny, const int *col_strip, const BandDev &b,
                            const void *tloc, double2 *z, cudaStream_t st);
// y = +-((A z)|band - sub) (sub: global or band vector, or null)
void launch_stencil_band(const GridDev &g, const BandDev &b, const double2 *z, const double2 *sub, bool sub_global,
                         bool neg, double2 *y, cudaStream_t st);
void launch_vsub(const double2 *a, const double2 *b, double2 *r, int64_t n, cudaStream_t st);  // r = a - b
void launch_band_gather(const BandDev &b, int ny, const double2 *x, double2 *y, cudaStream_t st);      // y = x|band
void launch_band_scatter_add(const BandDev &b, int ny, const double2 *y, double2 *x, cudaStream_t st); // x += y

// ---- Krylov kernels (kernels_krylov.cu), FP64 complex
// partial[blk][i] = sum_g conj(V_i[g]) w[g], i < m; then h[i] = sum_blk partial.
// With self_norm, h[m] = (||w||^2, 0) as well.
void launch_mdot(const double2 *V, int64_t ldv, int m, const double2 *w, int64_t n, double2 *partial,
                 double2 *h, cudaStream_t st, int self_norm = 0);
// w -= sum_i h[i] V_i, and nrm2 = ||w||^2 (partials then a fixed-order sum)
void launch_maxpy_norm(const double2 *V, int64_t ldv, int m, const double2 *h, double2 *w, int64_t n,
                       double *partial, double *nrm2, cudaStream_t st);
// x += sum_i y[i] Z_i
void launch_maxpy(const double2 *Z, int64_t ldz, int m, const double2 *y, double2 *x, int64_t n,
                  cudaStream_t st);
// nrm2 = ||x||^2
void launch_norm2(const double2 *x, int64_t n, double *partial, double *nrm2, cudaStream_t st);
// y = alpha * x (alpha real, read from device)
void launch_scale(const double2 *x, const double *inv_norm2, double2 *y, int64_t n, cudaStream_t st);
int krylov_partial_blocks();

// ---- learned initial guess (kernels_nn.cu): FP32 NCHW activations
// out = conv3x3(in) + bias (zero padding, optional ReLU); flip = 1 applies
// the input gradient of the convolution with weights w[Cout'][Cin'] instead
void nn_conv(const float *in, int Cin, const float *w, const float *bias, float *out, int Cout, int N, int H, int W,
             bool relu, bool flip, cudaStream_t st);
// gw += weight gradient, gb += bias gradient (accumulated: zero them first)
void nn_conv_wgrad(const float *in, int Cin, const float *gout, int Cout, int N, int H, int W, float *gw, float *gb,
                   cudaStream_t st);
void nn_relu_mask(const float *y, float *g, int64_t n, cudaStream_t st);  // g = 0 where y <= 0
void nn_pool2(const float *in, float *out, int64_t planes, int H, int W, cudaStream_t st);       // H, W of in
void nn_pool2_bwd(const float *gout, float *gin, int64_t planes, int H, int W, cudaStream_t st);  // H, W of gin
void nn_up2(const float *in, float *out, int64_t planes, int H, int W, cudaStream_t st);         // H, W of out
void nn_up2_bwd(const float *gout, float *gin, int64_t planes, int H, int W, cudaStream_t st);   // H, W of gout
void nn_axpy(const float *x, float *y, float a, int64_t n, cudaStream_t st);
// loss += sum (p - t)^2 / n, g = 2 (p - t) / n
void nn_mse(const float *p, const float *t, float *g, int64_t n, float *loss, cudaStream_t st);
void nn_adam(float *w, float *wb, const float *g, float *m, float *v, int64_t n, float lr, int step, bool bf16,
             cudaStream_t st);
void nn_round(const float *w, float *wb, int64_t n, bool bf16, cudaStream_t st);
void nn_input(const double *eps, const double2 *b, const double *scale, float *out, int nx, int ny, int Wp, int Hp,
              cudaStream_t st);
void nn_output(const float *out, const double *scale, double unit, double2 *x0, int nx, int ny, int Wp, int Hp,
               cudaStream_t st);
void nn_target(const double2 *x, const double *scale, double unit, float *out, int nx, int ny, int Wp, int Hp,
               cudaStream_t st);
void nn_absmax(const double2 *b, int64_t n, double *part, double *out, cudaStream_t st);
void nn_fit(const double2 *a, const double2 *b, int64_t n, double *part, double *out4, cudaStream_t st);
void nn_zscale(double2 *x, int64_t n, double ar, double ai, cudaStream_t st);  // x *= ar + i ai
void nn_zadd(const double2 *z, double2 *x, int64_t n, cudaStream_t st);              // x += z
constexpr int NN_PART = 4 * 608;  // doubles of scratch nn_absmax / nn_fit need

// ---- tensor-core convolutions (kernels_nn_tc.cu): BF16 operands, FP32
// accumulation; Cout <= 256.  Weights are packed per layer by nn_pack_weights
// (flip = the layer's input-gradient convolution) into nn_tc_packed_elems
// halves.  flag |= 1 if a wait timed out.
cudaError_t nn_tc_setup();
int nn_tc_npad(int Cout);
int nn_tc_nchunks(int Cin);
int64_t nn_tc_packed_elems(int Cin, int Cout);
void nn_pack_weights(const float *w, int CinL, int CoutL, bool flip, uint16_t *out, cudaStream_t st);
// part: scratch for split-K partial sums (nn_tc_ksplit(...) x N x Cout x H x W
// floats), or null for no split; small images split their input channels
// over several CTAs and a second kernel adds the slices in fixed order
int nn_tc_ksplit(int Cin, int Cout, int N, int H, int W);
// number of SMs of the current device (queried once)
int nn_num_sms();
// weight gradient on the tensor cores (BF16 operands, FP32 accumulation):
// gw += ..., gb += ... (accumulated with atomics: zero them first)
void nn_conv_wgrad_tc(const float *in, int Cin, const float *gout, int Cout, int N, int H, int W, float *gw,
                      float *gb, int *flag, cudaStream_t st);
void nn_conv_tc(const float *in, int Cin, const uint16_t *wp, const float *bias, float *out, int Cout, int N, int H,
                int W, bool relu, int *flag, cudaStream_t st, float *part);

}  // namespace stdd

// The network object (nn.cu); the solver asks it for a raw field guess.
struct stdd_nn;
namespace stdd {
int nn_device(const stdd_nn *nn);
// x0 = network(eps, b) * max(|Re b|, |Im b|) * unit on the nx x ny grid;
// scratch holds NN_PART doubles + 1
void nn_guess_field(stdd_nn *nn, const double *eps, const double2 *b, int nx, int ny, double unit, double2 *x0,
                    double *scratch, cudaStream_t st);
}  // namespace stdd

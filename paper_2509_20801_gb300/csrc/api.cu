// C ABI (include/stdd.h): context, configuration state machine, the
// preprocessing of Algorithm 1 (symbolic analysis + batched numeric
// multifrontal factorization) and the flexible GMRES outer iteration whose
// preconditioner is one Jacobi source-transfer sweep (Algorithm 1's loop
// body in residual form, Eqs. 18-21).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <complex>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/stdd.h"
#include "common.cuh"
#include "kernels.h"
#include "symbolic.h"

using stdd::FrontDev;
using stdd::LevelInfo;
using stdd::MfArgs;
using stdd::Shape;
using stdd::StripDev;
using cd = std::complex<double>;

namespace {

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct ArgError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct StateError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct TimeoutError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

#define CK(expr)                                                                         \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      throw CudaError(std::string(#expr) + ": " + cudaGetErrorString(_e));               \
  } while (0)

// owning device allocation
struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t n) {
    if (n <= bytes && p) return;
    release();
    if (n == 0) return;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      throw std::bad_alloc();
    }
    bytes = n;
  }
  template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// SC-PML stretch on a line of n nodes (Eqs. 10-13): node u = 1..L of a PML
// at depth (u - 1/2) cells, half node u + 1/2 at depth u cells from the
// interface; sigma/(w eps0) = (m+1)(-ln R)/(2 k0 L delta) (rho/(L delta))^m.
void stretch(int n, int Llo, int Lhi, double delta, double k0, int m, double R, std::vector<cd> &s,
             std::vector<cd> &sh) {
  auto smax = [&](int L) { return (m + 1) * (-std::log(R)) / (2.0 * k0 * L * delta); };
  auto sig = [&](double pos) {
    double v = 0;
    if (Llo > 0) {
      const double d = std::max(0.0, (Llo - 0.5) - pos);
      v += smax(Llo) * std::pow(d / Llo, m);
    }
    if (Lhi > 0) {
      const double d = std::max(0.0, pos - (n - Lhi - 0.5));
      v += smax(Lhi) * std::pow(d / Lhi, m);
    }
    return v;
  };
  s.resize(n);
  sh.resize(n + 1);
  for (int i = 0; i < n; ++i) s[i] = cd(1.0, sig(i));
  for (int h = 0; h <= n; ++h) sh[h] = cd(1.0, sig(h - 0.5));
}

// couplings of row i to i-1 and i+1: 1/(s_i s_{i-+1/2} delta^2)
void couplings(const std::vector<cd> &s, const std::vector<cd> &sh, double delta, std::vector<double2> &cm,
               std::vector<double2> &cp) {
  const int n = (int)s.size();
  cm.resize(n);
  cp.resize(n);
  for (int i = 0; i < n; ++i) {
    const cd a = 1.0 / (s[i] * sh[i] * delta * delta);
    const cd b = 1.0 / (s[i] * sh[i + 1] * delta * delta);
    cm[i] = make_double2(a.real(), a.imag());
    cp[i] = make_double2(b.real(), b.imag());
  }
}

template <typename T> void upload(DBuf &d, const std::vector<T> &h, cudaStream_t st) {
  d.alloc(std::max<size_t>(1, h.size()) * sizeof(T));
  if (!h.empty()) CK(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

// A subdomain: owned columns [c0, c1) and rows [r0, r1), local box
// [x0, x1) x [y0, y1), local PML widths at its four sides.  Strips span all
// rows (r0 = y0 = 0, r1 = y1 = ny, the global y-PML).
struct StripHost {
  int c0, c1, x0, x1, Llo, Lhi;
  int r0, r1, y0, y1, Lylo, Lyhi;
  int W() const { return x1 - x0; }
  int H() const { return y1 - y0; }
};

// Strip partition of n nodes along one axis (Sec. 2.3): equal widths with
// the remainder to the first parts, or explicit cuts; each part's local box
// reaches ext = overlap + ipml nodes into each neighbour, whose width must
// be at least ext.  Returns (owned begin, owned end, box begin, box end,
// low PML, high PML) per part.
std::vector<std::array<int, 6>> partition_axis(int n, int parts, const std::vector<int> &cuts, int overlap,
                                               int ipml, int pml_lo, int pml_hi) {
  const int ext = overlap + ipml;
  std::vector<int> c = cuts;
  if (c.empty()) {
    c.push_back(0);
    const int base = n / parts, rem = n % parts;
    for (int k = 0; k < parts; ++k) c.push_back(c.back() + base + (k < rem ? 1 : 0));
  }
  std::vector<std::array<int, 6>> out;
  for (int k = 0; k < parts; ++k) {
    if (k > 0 && ext > c[k] - c[k - 1]) throw ArgError("overlap + interface PML wider than a neighbouring strip");
    if (k < parts - 1 && ext > c[k + 2] - c[k + 1])
      throw ArgError("overlap + interface PML wider than a neighbouring strip");
    out.push_back({c[k], c[k + 1], k > 0 ? c[k] - ext : 0, k < parts - 1 ? c[k + 1] + ext : n,
                   k > 0 ? ipml : pml_lo, k < parts - 1 ? ipml : pml_hi});
  }
  return out;
}

}  // namespace

struct stdd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;

  // configuration
  int nx = 0, ny = 0;
  double dx = 0, dy = 0, wavelength = 0;
  bool have_eps = false;
  int npml[4] = {0, 0, 0, 0};
  int pml_m = 3;
  double pml_R = 1e-8;
  bool have_pml = false;
  int nsub = 0, overlap = 0, ipml = 0;
  std::vector<int> cuts;
  // 2-D (checkerboard) decomposition: nsx x nsy boxes, box k = kx * nsy + ky
  // (nsy = 1: the strips of Sec. 2.3); nsub = nsx * nsy
  int nsx = 0, nsy = 1;
  std::vector<int> ycuts;
  bool boxes() const { return nsy > 1; }
  void require_strips(const char *what) const {
    if (boxes()) throw ArgError(std::string(what) + " needs an x-strip decomposition (one box row)");
  }
  int prec = STDD_PREC_FP64;
  int leaf_max = 16;
  int nrhs = 0;

  // operator (global) state
  bool op_ready = false;
  DBuf d_eps, d_cxm, d_cxp, d_cym, d_cyp;
  double k0sq = 0;

  // decomposition + factors
  bool factored = false;
  std::vector<StripHost> strips;
  std::map<std::pair<int, int>, Shape> shapes;   // ND analysis per local box shape (W, H)
  std::vector<LevelInfo> levels;
  DBuf d_strips, d_fronts, d_nodes, d_cmap, d_inv, d_lcxm, d_lcxp, d_colstrip, d_lcym, d_lcyp, d_rowbox;
  // distinct local y-coupling profiles (box height, low and high PML)
  std::vector<std::array<int, 3>> ycoef_keys;
  DBuf d_fac, d_ws[2], d_ub[2], d_tloc, d_wloc, d_flag, d_minpiv, d_nraised, d_items;
  int64_t nloc = 0, nloc_max = 0, ub_elems[2] = {0, 0}, panel_need = 0;
  // partial pivoting restricted to each front's pivot rows (STDD_OPT_PIVOTING)
  int pivoting = 0;
  DBuf d_pcol, d_panel;
  // symmetric form (STDD_OPT_SYMMETRIC): fronts of D A, D = the local
  // stretch products s_x s_y, with lower-half updates; not with pivoting
  // nor with the tensor-core updates (which update whole tiles)
  int symmetric = 1;   // 1: complex128 factors, 2: complex64 ones too
  bool sym_active() const {
    return symmetric && !pivoting && tc_fmt() < 0 && (prec == STDD_PREC_FP64 || symmetric == 2);
  }
  // complex128 symmetric form: large-front updates on the tensor cores by
  // exact splitting (STDD_OPT_FP64_TC)
  int fp64_tc = 1;
  bool oz_active() const { return fp64_tc && sym_active() && prec == STDD_PREC_FP64; }
  DBuf d_lsx, d_lsy;
  DBuf d_segpart;   // partial sums of the grid-split substitution products
  int forced_split = 0;   // STDD_OPT_SWEEP_SPLIT: 0 tuned, else 1, 2, 4, 8 or MF_SPLIT_GRID
  int64_t nfronts = 0, factor_entries = 0;
  double factor_cflops = 0, factor_cflops_lu = 0, solve_cflops = 0;
  int max_p = 0, max_b = 0, depth = 0;
  double min_pivot = 0;
  long long raised_pivots = 0;
  // static pivoting: 0 = off, k > 0 = floor 10^-k of the stencil scale
  int static_pivot = 0;
  double pivot_floor() const;
  int solve_nrhs_cap = 0;

  // sources and Krylov state
  DBuf d_b, d_x, d_r, d_V, d_Z, d_w, d_part, d_h, d_nrm, d_y, d_pre, d_fpart;
  // learned initial guess
  stdd_nn *learned = nullptr;
  DBuf d_guess, d_gscr;
  std::vector<double> lg_raw, lg_scaled;
  std::vector<int> lg_used;
  int V_cols = 0, V_rhs = 0;
  bool last_noconv = false;
  std::vector<std::vector<double>> history;
  int last_its = 0, last_reorth = 0;
  double last_res = 0;

  // phase profiling (CUDA events on the context stream)
  enum { PH_FACTOR = 0, PH_MINV, PH_MATVEC, PH_ORTHO, PH_SOLVE, PH_K0, PH_COUNT = PH_K0 + stdd::K_COUNT };
  int prof = 0;  // 0 off, 1 phase spans, 2 phase + per-launch kernel spans
  struct Span {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<Span> spans;
  cudaEvent_t next_event() {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }
  int pbegin(int phase) {
    if (!prof) return -1;
    Span sp{phase, next_event(), next_event()};
    CK(cudaEventRecord(sp.a, stream));
    spans.push_back(sp);
    return (int)spans.size() - 1;
  }
  void pend(int id) {
    if (id >= 0) CK(cudaEventRecord(spans[id].b, stream));
  }
  ~stdd_ctx() {
    clear_graphs();
    for (auto e : ev_pool) cudaEventDestroy(e);
  }

  // per-launch profiling of the dominant kernels: algorithmic work per
  // launch from the host front list (flops for the eliminations, factor
  // bytes for the substitution sweeps)
  // Elimination kernels are credited with the LU flops of what they do (the
  // trailing-block updates, Sec. 2.4, Eq. 22), and separately with the
  // Gauss-Jordan flops they execute (which also update the eliminated pivot
  // rows and columns).
  std::vector<double> unit_small, unit_up, unit_down;       // per level
  std::vector<std::vector<double>> unit_update;             // per level, per step
  std::vector<double> exec_small;                           // per level, Gauss-Jordan flops
  std::vector<std::vector<double>> exec_update;             // per level, per step
  std::vector<std::vector<double>> unit_update_sym, exec_update_sym;  // the symmetric form's
  std::vector<double> unit_small_sym, exec_small_sym;
  std::vector<std::vector<double>> exec_update_oz;          // BF16 tensor flops of the split update
  std::vector<double> span_units, span_exec;                // parallel to spans
  std::vector<int64_t> strip_fac_entries;                   // factor entries of each strip
  std::vector<int> span_level;                              // parallel to spans
  struct Hook : stdd::LaunchHook {
    stdd_ctx *c = nullptr;
    int open = -1;
    void before(int kind, int level, int k) override {
      if (c->prof < 2) return;
      open = c->pbegin(PH_K0 + kind);
      c->span_level.resize(c->spans.size(), -1);
      c->span_level[open] = level;
      double u = 0, x = 0;
      if (kind == stdd::K_SMALL) {
        const bool sy = c->sym_active();
        u = (sy ? c->unit_small_sym : c->unit_small)[level];
        x = (sy ? c->exec_small_sym : c->exec_small)[level];
      } else if (kind == stdd::K_UPDATE) {
        const bool sy = c->sym_active();
        u = (sy ? c->unit_update_sym : c->unit_update)[level][k / stdd::MF_NB];
        x = (c->oz_active() ? c->exec_update_oz : sy ? c->exec_update_sym : c->exec_update)[level][k / stdd::MF_NB];
      } else if (kind == stdd::K_SWEEP) {   // "level" is the strip
        u = x = c->strip_fac_entries[level] * (double)c->elem();
      } else if (kind == stdd::K_UP) {
        u = x = c->unit_up[level];
      } else {
        u = x = c->unit_down[level];
      }
      c->span_units.resize(c->spans.size(), 0.0);
      c->span_exec.resize(c->spans.size(), 0.0);
      c->span_units[open] = u;
      c->span_exec[open] = x;
    }
    void after(int, int, int) override {
      if (open >= 0) c->pend(open);
      open = -1;
    }
    // a launch over a fraction of a level's substitution items
    void before_part(int kind, int level, double frac) {
      before(kind, level, 0);
      if (open >= 0) {
        c->span_units[open] *= frac;
        c->span_exec[open] *= frac;
      }
    }
  } hook;

  size_t elem() const { return prec == STDD_PREC_FP64 ? sizeof(double2) : sizeof(float2); }
  // tensor-core input format of the large-front updates (-1: CUDA cores)
  int tc_fmt() const { return prec == STDD_PREC_C64_FP16 ? 0 : (prec == STDD_PREC_C64_BF16 ? 1 : -1); }
  int64_t N() const { return (int64_t)nx * ny; }

  void invalidate_factors() { factored = false; }
  void invalidate_operator() {
    op_ready = false;
    factored = false;
  }

  stdd::GridDev grid() const {
    stdd::GridDev g;
    g.nx = nx;
    g.ny = ny;
    g.k0sq = k0sq;
    g.eps = d_eps.as<double>();
    g.cxm = d_cxm.as<double2>();
    g.cxp = d_cxp.as<double2>();
    g.cym = d_cym.as<double2>();
    g.cyp = d_cyp.as<double2>();
    return g;
  }

  void require_operator() {
    if (nx <= 0) throw StateError("grid not set");
    if (!have_eps) throw StateError("permittivity not set");
    if (wavelength <= 0) throw StateError("frequency not set");
    if (!have_pml) throw StateError("PML not set");
    if (op_ready) return;
    const double k0 = 2.0 * M_PI / wavelength;
    k0sq = k0 * k0;
    std::vector<cd> sx, sxh, sy, syh;
    stretch(nx, npml[0], npml[1], dx, k0, pml_m, pml_R, sx, sxh);
    stretch(ny, npml[2], npml[3], dy, k0, pml_m, pml_R, sy, syh);
    std::vector<double2> cxm, cxp, cym, cyp;
    couplings(sx, sxh, dx, cxm, cxp);
    couplings(sy, syh, dy, cym, cyp);
    upload(d_cxm, cxm, stream);
    upload(d_cxp, cxp, stream);
    upload(d_cym, cym, stream);
    upload(d_cyp, cyp, stream);
    CK(cudaStreamSynchronize(stream));
    op_ready = true;
  }

  void build_strips() {
    if (nsub <= 0) throw StateError("decomposition not set");
    const auto xs = partition_axis(nx, nsx, cuts, overlap, ipml, npml[0], npml[1]);
    const auto ys = nsy > 1 ? partition_axis(ny, nsy, ycuts, overlap, ipml, npml[2], npml[3])
                            : std::vector<std::array<int, 6>>{{0, ny, 0, ny, npml[2], npml[3]}};
    strips.clear();
    for (const auto &x : xs)
      for (const auto &y : ys) {
        StripHost s;
        s.c0 = x[0];
        s.c1 = x[1];
        s.x0 = x[2];
        s.x1 = x[3];
        s.Llo = x[4];
        s.Lhi = x[5];
        s.r0 = y[0];
        s.r1 = y[1];
        s.y0 = y[2];
        s.y1 = y[3];
        s.Lylo = y[4];
        s.Lyhi = y[5];
        strips.push_back(s);
      }
  }

  // set a px x py decomposition (py = 1: strips), restoring the previous one
  // if it is invalid
  void set_boxes(int px, const std::vector<int> &xc, int py, const std::vector<int> &yc, int ov, int ip) {
    const int o_n = nsub, o_x = nsx, o_y = nsy, o_o = overlap, o_p = ipml;
    const auto o_c = cuts, o_yc = ycuts;
    nsx = px;
    nsy = py;
    nsub = px * py;
    cuts = xc;
    ycuts = yc;
    overlap = ov;
    ipml = ip;
    try {
      build_strips();
    } catch (...) {
      nsub = o_n;
      nsx = o_x;
      nsy = o_y;
      cuts = o_c;
      ycuts = o_yc;
      overlap = o_o;
      ipml = o_p;
      throw;
    }
    invalidate_factors();
    clear_graphs();
  }
  void factor();
  void build_structure();
  void upload_local_couplings();
  bool struct_ready = false;
  std::vector<int64_t> struct_key;
  void apply_minv(const double2 *v, double2 *z);
  void apply_minv_multi(const std::vector<const double2 *> &vs, const std::vector<double2 *> &zs);
  void enqueue_minv(const std::vector<const double2 *> &vs, const std::vector<double2 *> &zs);
  // captured CUDA graphs of M^-1 applications, keyed by (input, output)
  struct GraphEntry {
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::map<std::vector<const void *>, GraphEntry> minv_graphs;
  // Capture the launches f() enqueues into an instantiated graph.  Any
  // exception thrown while capturing (a refused argument, a CUDA error) ends
  // the capture first, so the stream never stays in capture mode.  Kernels
  // counted during capture are uncounted here and counted at each replay.
  template <typename F> GraphEntry capture(F &&f) {
    const long long before = __atomic_load_n(&stdd::g_launches, __ATOMIC_RELAXED);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    try {
      f();
    } catch (...) {
      cudaGraph_t dead = nullptr;
      cudaStreamEndCapture(stream, &dead);
      if (dead) cudaGraphDestroy(dead);
      (void)cudaGetLastError();
      const long long k = __atomic_load_n(&stdd::g_launches, __ATOMIC_RELAXED) - before;
      __atomic_add_fetch(&stdd::g_launches, -k, __ATOMIC_RELAXED);
      throw;
    }
    const cudaError_t ce = cudaStreamEndCapture(stream, &g);
    if (ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      throw CudaError(std::string("graph capture: ") + cudaGetErrorString(ce));
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) throw CudaError(std::string("graph instantiate: ") + cudaGetErrorString(ie));
    const long long kernels = __atomic_load_n(&stdd::g_launches, __ATOMIC_RELAXED) - before;
    __atomic_add_fetch(&stdd::g_launches, -kernels, __ATOMIC_RELAXED);
    return GraphEntry{ex, kernels};
  }

  // captured graph of the numeric factorization, valid while every argument
  // its launches were captured with (all levels' MfArgs bytes) is unchanged
  cudaGraphExec_t factor_graph = nullptr;
  long long factor_graph_kernels = 0;
  std::vector<unsigned char> factor_graph_key;
  template <typename R> void enqueue_factor();
  bool use_graphs = true;
  // preconditioner order: 0 additive (Algorithm 1), 1 symmetric
  // multiplicative, 2 red-black (even strips together, then odd strips)
  int order = 0;
  // Within a level, fronts and work items are grouped by strip, strips in
  // the order perm (even strips first, then odd), so every single strip and
  // both colour groups are contiguous ranges.  pos[k] = position of strip k;
  // per level and position: first front, first upward / downward item.
  std::vector<int> perm, pos;
  std::vector<std::vector<int>> lvl_front, lvl_up, lvl_down;
  std::vector<StripDev> strips_host;
  std::vector<FrontDev> fronts_host;   // host copies for the band analysis
  std::vector<int> nodes_host;
  // band-space FGMRES (STDD_OPT_BAND): interface bands as column intervals,
  // the column -> band offset map, and per level the work items of the
  // fronts a band vector needs (upward: subtree holds band sources;
  // downward: pivots on the widened band, and their ancestors)
  bool use_band = false, band_ready = false;
  std::vector<int2> band_iv, band_iv1;
  std::vector<int64_t> band_off, band_off1;
  int64_t band_n = 0, band_n1 = 0;
  DBuf d_band_iv, d_band_off, d_band_iv1, d_band_off1, d_colband, d_items_band, d_fb, d_sb;
  std::vector<int64_t> lvl_bup_off, lvl_bdown_off;
  std::vector<int> lvl_bup_n, lvl_bdown_n;
  void build_band();
  stdd::BandDev band_dev() const {
    return stdd::BandDev{d_band_iv.as<int2>(), d_band_off.as<int64_t>(), (int)band_iv.size(), band_n,
                         d_band_iv1.as<int2>(), d_band_off1.as<int64_t>(), (int)band_iv1.size(), band_n1};
  }
  template <typename R> void solve_levels_band(int nr);
  void enqueue_op_band(const std::vector<const double2 *> &ss, const std::vector<double2 *> &ys);
  void apply_op_band(const std::vector<const double2 *> &ss, const std::vector<double2 *> &ys);
  void clear_graphs() {
    for (auto &kv : minv_graphs) cudaGraphExecDestroy(kv.second.exec);
    minv_graphs.clear();
    if (factor_graph) cudaGraphExecDestroy(factor_graph);
    factor_graph = nullptr;
    factor_graph_key.clear();
  }
  template <typename R> void factor_t();
  template <typename R> void tune_update_tiles();
  int forced_tile = 0;   // STDD_OPT_UPDATE_TILE: 0 = tuned, else 64 or 32 for every level
  void factor_prepare();
  template <typename R> void solve_levels(int nrhs_);
  template <typename R> void solve_range_levels(int j0, int j1, int nrhs_);
  template <typename R> void enqueue_minv_multiplicative(const std::vector<const double2 *> &vs,
                                                         const std::vector<double2 *> &zs);
  void check_red_black() const;
  template <typename R> void autotune();
  void ensure_solve_buffers(int nr);
  // sweep launch configurations chosen by timing, keyed by the device and
  // the level shape; shared by every context of the process (contexts of
  // the same grid and decomposition, or any with the same level shapes,
  // reuse one tuning)
  static std::map<std::vector<int64_t>, int> &tuned() {
    static std::map<std::vector<int64_t>, int> m;
    return m;
  }
  static std::mutex &tuned_mutex() {
    static std::mutex m;
    return m;
  }
  bool autotune_on = true;
  MfArgs mf_args(int level_parity_cur, bool solve) const;
  void ensure_krylov(int m);
  // persistent one-strip sweeps of the sequential orders (STDD_OPT_PERSISTENT):
  // per strip position and level the strip's share of the sweep
  int persistent = -1;                // 0: per-level launches; k: persistent sweeps, k blocks per SM; -1: by precision
  // automatic choice: complex64 sweeps run persistent (2 blocks per SM);
  // complex128 ones are FP64-bound per warp and gain more from the per-level
  // kernels' deeper load pipelines than from saving launches
  int persistent_eff() const { return persistent >= 0 ? persistent : (prec == STDD_PREC_FP64 ? 0 : 2); }
  long long sweep_wait = 1ll << 22;   // polls of a grid-barrier wait before it gives up
  DBuf d_striplv, d_bar, d_sweep_flag;
  int sweep_flag_h = 0;
  void build_strip_levels();
  void poll_sweep_flag() {           // enqueue a copy of the flag (read after the next sync)
    if (d_sweep_flag.p) CK(cudaMemcpyAsync(&sweep_flag_h, d_sweep_flag.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
  }
  void raise_sweep_flag() {          // after a sync: a persistent sweep gave up a barrier wait
    if (sweep_flag_h & 1) {
      sweep_flag_h = 0;
      CK(cudaMemsetAsync(d_sweep_flag.p, 0, sizeof(int), stream));
      CK(cudaStreamSynchronize(stream));
      throw TimeoutError("a persistent substitution sweep gave up waiting at a grid barrier");
    }
  }
  void gmres_multi(const stdd_solve_opts &o);
  void richardson(int rhs, const stdd_solve_opts &o, double2 *x);
  void learned_guesses(double2 *X);  // all right-hand sides
  int64_t device_bytes() const;
};

// Static-pivot floor: 10^-k times the modulus scale of the stencil's
// diagonal, 2/dx^2 + 2/dy^2.
double stdd_ctx::pivot_floor() const {
  if (static_pivot <= 0) return 0.0;
  return std::pow(10.0, -static_pivot) * (2.0 / (dx * dx) + 2.0 / (dy * dy));
}

MfArgs stdd_ctx::mf_args(int par, bool solve) const {
  MfArgs a;
  std::memset(&a, 0, sizeof a);  // padding too: the bytes key the factorization graph
  a.fronts = d_fronts.as<FrontDev>();
  a.strips = d_strips.as<StripDev>();
  a.nodes = d_nodes.as<int>();
  a.cmap = d_cmap.as<int>();
  a.inv = d_inv.as<int>();
  a.cxm = d_lcxm.as<double2>();
  a.cxp = d_lcxp.as<double2>();
  a.cym = d_lcym.as<double2>();
  a.cyp = d_lcyp.as<double2>();
  a.eps = d_eps.as<double>();
  a.k0sq = k0sq;
  a.H = ny;
  a.fac = d_fac.p;
  a.ws_cur = d_ws[par].p;
  a.ws_child = d_ws[par ^ 1].p;
  a.tloc = d_tloc.p;
  a.wloc = d_wloc.p;
  a.ub_cur = d_ub[par].p;
  a.ub_child = d_ub[par ^ 1].p;
  a.flag = d_flag.as<int>();
  a.min_pivot = d_minpiv.as<double>();
  a.piv_floor = pivot_floor();
  a.n_raised = d_nraised.as<unsigned long long>();
  a.pcol = pivoting ? d_pcol.as<int>() : nullptr;
  a.panel = pivoting ? d_panel.p : nullptr;
  a.sym = sym_active() ? 1 : 0;
  a.segpart = d_segpart.p;
  a.fp64_tc = oz_active() ? 1 : 0;
  a.lsx = a.sym ? d_lsx.as<double2>() : nullptr;
  a.lsy = a.sym ? d_lsy.as<double2>() : nullptr;
  (void)solve;
  return a;
}

// Strip-local x couplings (local PML at interior sides, global PML at the
// domain ends), re-derived at every factorization (they depend on the
// frequency and the PML, not on the structure).
void stdd_ctx::upload_local_couplings() {
  const double k0 = 2.0 * M_PI / wavelength;
  std::vector<double2> lcxm, lcxp, lsx, lsy;
  auto nodes_of = [](const std::vector<cd> &v, std::vector<double2> &out) {
    for (const cd &z : v) out.push_back(make_double2(z.real(), z.imag()));
  };
  for (int k = 0; k < nsub; ++k) {
    const StripHost &s = strips[k];
    std::vector<cd> sx, sxh;
    stretch(s.W(), s.Llo, s.Lhi, dx, k0, pml_m, pml_R, sx, sxh);
    std::vector<double2> cm, cp;
    couplings(sx, sxh, dx, cm, cp);
    lcxm.insert(lcxm.end(), cm.begin(), cm.end());
    lcxp.insert(lcxp.end(), cp.begin(), cp.end());
    nodes_of(sx, lsx);
  }
  upload(d_lcxm, lcxm, stream);
  upload(d_lcxp, lcxp, stream);
  upload(d_lsx, lsx, stream);
  // local y couplings of the distinct box heights and PML widths (a strip
  // decomposition has one: all rows with the global y-PML, the global ones)
  std::vector<double2> lcym, lcyp;
  for (const auto &yk : ycoef_keys) {
    std::vector<cd> sy, syh;
    stretch(yk[0], yk[1], yk[2], dy, k0, pml_m, pml_R, sy, syh);
    std::vector<double2> cm, cp;
    couplings(sy, syh, dy, cm, cp);
    lcym.insert(lcym.end(), cm.begin(), cm.end());
    lcyp.insert(lcyp.end(), cp.begin(), cp.end());
    nodes_of(sy, lsy);
  }
  upload(d_lcym, lcym, stream);
  upload(d_lcyp, lcyp, stream);
  upload(d_lsy, lsy, stream);
}

void stdd_ctx::factor() {
  require_operator();
  build_strips();
  factored = false;
  clear_graphs();
  std::vector<int64_t> key = {nx, ny, nsub, nsx, nsy, overlap, ipml, prec, leaf_max};
  key.insert(key.end(), cuts.begin(), cuts.end());
  key.push_back(-1);
  key.insert(key.end(), ycuts.begin(), ycuts.end());
  if (!struct_ready || key != struct_key) {
    struct_ready = false;
    build_structure();
    struct_key = key;
    struct_ready = true;
  }
  upload_local_couplings();
  CK(cudaStreamSynchronize(stream));
  if (autotune_on || forced_tile) {
    if (prec == STDD_PREC_FP64) tune_update_tiles<double>();
    else tune_update_tiles<float>();
  } else {
    for (auto &li : levels) li.upd_tile = 64;
  }
  if (prec == STDD_PREC_FP64) factor_t<double>();
  else factor_t<float>();
  factored = true;
  if (autotune_on) {
    if (prec == STDD_PREC_FP64) autotune<double>();
    else autotune<float>();
  }
  if (forced_split) {
    // one split everywhere it is valid (32-row items for the grid split, at
    // most MF_MAXSEG segments for an in-block one); results do not change
    for (auto &li : levels) {
      auto pick = [&](int rows, int cols) {
        int sp = forced_split;
        if (sp == stdd::MF_SPLIT_GRID) {
          if (rows == 32) return sp;
          sp = 8;
        }
        if (sp > 256 / rows) sp = 256 / rows;
        if (sp > 1 && (cols + stdd::MF_SEG - 1) / stdd::MF_SEG > stdd::MF_MAXSEG) sp = 1;
        return sp;
      };
      li.split_up = li.split_up1 = pick(li.rows_up, li.max_p);
      li.split_down = li.split_down1 = pick(li.rows_down, li.max_n);
    }
  }
  build_strip_levels();
}

// Each strip's share of every level, for the persistent sweeps (after the
// autotuner: it carries the single-strip launch shapes).
void stdd_ctx::build_strip_levels() {
  std::vector<stdd::StripLevel> t((size_t)nsub * depth);
  for (int j = 0; j < nsub; ++j)
    for (int L = 0; L < depth; ++L) {
      const LevelInfo &li = levels[L];
      stdd::StripLevel &l = t[(size_t)j * depth + L];
      l.f0 = lvl_front[L][j];
      l.nf = lvl_front[L][j + 1] - lvl_front[L][j];
      l.up_first = li.up_off + lvl_up[L][j];
      l.up_n = lvl_up[L][j + 1] - lvl_up[L][j];
      l.down_first = li.down_off + lvl_down[L][j];
      l.down_n = lvl_down[L][j + 1] - lvl_down[L][j];
      l.rows_up = li.rows_up;
      l.rows_down = li.rows_down;
      // (the persistent kernel splits within a block only; any split gives
      // the same sums)
      auto inblock = [](int sp, int cols) {
        if (sp > 8) sp = 8;
        return (sp > 1 && (cols + stdd::MF_SEG - 1) / stdd::MF_SEG > stdd::MF_MAXSEG) ? 1 : sp;
      };
      l.split_up = inblock(li.split_up1, li.max_p);
      l.split_down = inblock(li.split_down1, li.max_n);
      l.max_n = li.max_n;
      l.pad_ = 0;
    }
  upload(d_striplv, t, stream);
  stdd::mf_strip_sweep_grid();   // launch shape queried once, outside any capture
  if (!d_bar.p) {
    d_bar.alloc(2 * sizeof(unsigned));
    CK(cudaMemsetAsync(d_bar.p, 0, 2 * sizeof(unsigned), stream));
  }
  if (!d_sweep_flag.p) {
    d_sweep_flag.alloc(sizeof(int));
    CK(cudaMemsetAsync(d_sweep_flag.p, 0, sizeof(int), stream));
  }
  CK(cudaStreamSynchronize(stream));
}

// Everything that depends only on the grid, the decomposition and the
// precision: symbolic analysis, strip and front descriptors, work items,
// device buffers.  Cached across factorizations of the same structure.
void stdd_ctx::build_structure() {
  // ---- symbolic analysis per distinct local box shape (host, cached)
  for (auto &s : strips) {
    const std::pair<int, int> key{s.W(), s.H()};
    if (!shapes.count(key) || shapes[key].leaf_max != leaf_max) {
      Shape sh;
      stdd::nd_analyze(s.W(), s.H(), leaf_max, sh);
      shapes[key] = std::move(sh);
    }
  }
  auto shape_of = [&](const StripHost &s) -> const Shape & { return shapes.at({s.W(), s.H()}); };
  // concatenated shape arrays
  std::map<std::pair<int, int>, int64_t> node_base, cmap_base, inv_base;
  std::vector<int> nodes, cmap, inv;
  for (auto &kv : shapes) {
    node_base[kv.first] = (int64_t)nodes.size();
    cmap_base[kv.first] = (int64_t)cmap.size();
    inv_base[kv.first] = (int64_t)inv.size();
    nodes.insert(nodes.end(), kv.second.nodes.begin(), kv.second.nodes.end());
    cmap.insert(cmap.end(), kv.second.cmap.begin(), kv.second.cmap.end());
    inv.insert(inv.end(), kv.second.inv.begin(), kv.second.inv.end());
  }
  // ---- strips: local fields, local x couplings, factor blocks
  std::vector<StripDev> sdev(nsub);
  int64_t vec = 0, fac = 0, coef = 0;
  depth = 0;
  max_p = max_b = 0;
  factor_cflops = factor_cflops_lu = solve_cflops = 0;
  nloc_max = 0;
  ycoef_keys.clear();
  strip_fac_entries.assign(nsub, 0);
  for (int k = 0; k < nsub; ++k) {
    const StripHost &s = strips[k];
    const Shape &sh = shape_of(s);
    sdev[k].x0 = s.x0;
    sdev[k].x1 = s.x1;
    sdev[k].c0 = s.c0;
    sdev[k].c1 = s.c1;
    sdev[k].y0 = s.y0;
    sdev[k].y1 = s.y1;
    sdev[k].r0 = s.r0;
    sdev[k].r1 = s.r1;
    // local y couplings, one copy per distinct (height, low PML, high PML)
    const std::array<int, 3> yk{s.H(), s.Lylo, s.Lyhi};
    int64_t yoff = 0;
    size_t q = 0;
    for (; q < ycoef_keys.size() && ycoef_keys[q] != yk; ++q) yoff += ycoef_keys[q][0];
    if (q == ycoef_keys.size()) ycoef_keys.push_back(yk);
    sdev[k].ycoef_off = yoff;
    sdev[k].vec_off = vec;
    sdev[k].coef_off = coef;
    sdev[k].fac_off = fac;
    vec += (int64_t)s.W() * s.H();
    nloc_max = std::max<int64_t>(nloc_max, (int64_t)s.W() * s.H());
    fac += sh.factor_entries;
    strip_fac_entries[k] = sh.factor_entries;
    coef += s.W();
    depth = std::max(depth, sh.depth);
    max_p = std::max(max_p, sh.max_p);
    max_b = std::max(max_b, sh.max_b);
    factor_cflops += sh.factor_cflops;
    factor_cflops_lu += sh.factor_cflops_lu;
    solve_cflops += sh.solve_cflops;
  }
  nloc = vec;
  factor_entries = fac;
  // ---- front instances, level-major
  std::vector<std::vector<int>> inst(nsub);
  for (int k = 0; k < nsub; ++k) inst[k].assign(shape_of(strips[k]).fronts.size(), -1);
  std::vector<FrontDev> fr;
  levels.assign(depth, LevelInfo{0, 0, 0, 0, 0, 1 << 30, 0, 0, 0, 0, 32, 32, 1, 1, 1, 1, 64, 0});
  perm.clear();
  for (int k = 0; k < nsub; k += 2) perm.push_back(k);
  for (int k = 1; k < nsub; k += 2) perm.push_back(k);
  pos.assign(nsub, 0);
  for (int j = 0; j < nsub; ++j) pos[perm[j]] = j;
  lvl_front.assign(depth, {});
  lvl_up.assign(depth, std::vector<int>(nsub + 1, 0));
  lvl_down.assign(depth, std::vector<int>(nsub + 1, 0));
  int64_t ws_need[2] = {0, 0};
  int64_t piv_run = 0;
  panel_need = 0;
  ub_elems[0] = ub_elems[1] = 0;
  for (int L = 0; L < depth; ++L) {
    LevelInfo &li = levels[L];
    li.f0 = (int)fr.size();
    int64_t s_run = 0, u_run = 0, pan_run = 0;
    lvl_front[L].assign(nsub + 1, 0);
    for (int j = 0; j < nsub; ++j) {
      const int k = perm[j];
      lvl_front[L][j] = (int)fr.size();
      const Shape &sh = shape_of(strips[k]);
      const std::pair<int, int> skey{sh.W, sh.H};
      for (size_t f = 0; f < sh.fronts.size(); ++f) {
        const auto &sf = sh.fronts[f];
        if (sf.level != L) continue;
        inst[k][f] = (int)fr.size();
        FrontDev d;
        d.p = sf.p;
        d.b = sf.b;
        d.strip = k;
        d.child[0] = d.child[1] = -1;
        d.node_off = node_base[skey] + sf.node_off;
        for (int ci = 0; ci < 2; ++ci) {
          d.cmap_off[ci] = sf.cmap_off[ci] >= 0 ? cmap_base[skey] + sf.cmap_off[ci] : -1;
          d.inv_off[ci] = sf.inv_off[ci] >= 0 ? inv_base[skey] + sf.inv_off[ci] : -1;
        }
        d.fac_off = sdev[k].fac_off + sf.fac_off;
        d.s_off = s_run;
        d.u_off = u_run;
        d.piv_off = piv_run;
        d.pan_off = pan_run;
        piv_run += sf.p;
        if (sf.p + sf.b > stdd::MF_SMALL) pan_run += (int64_t)sf.p * stdd::MF_NB;
        s_run += (int64_t)sf.b * sf.b;
        u_run += sf.b;
        li.max_p = std::max(li.max_p, sf.p);
        li.max_b = std::max(li.max_b, sf.b);
        li.max_n = std::max(li.max_n, sf.p + sf.b);
        li.min_n = std::min(li.min_n, sf.p + sf.b);
        fr.push_back(d);
      }
    }
    li.nf = (int)fr.size() - li.f0;
    lvl_front[L][nsub] = (int)fr.size();
    ws_need[L & 1] = std::max(ws_need[L & 1], s_run);
    panel_need = std::max(panel_need, pan_run);
    ub_elems[L & 1] = std::max(ub_elems[L & 1], u_run);
  }
  // children ids (instances of children are at level + 1, already numbered)
  for (int k = 0; k < nsub; ++k) {
    const Shape &sh = shape_of(strips[k]);
    for (size_t f = 0; f < sh.fronts.size(); ++f) {
      FrontDev &d = fr[inst[k][f]];
      for (int ci = 0; ci < 2; ++ci)
        if (sh.fronts[f].child[ci] >= 0) d.child[ci] = inst[k][sh.fronts[f].child[ci]];
    }
  }
  nfronts = (int64_t)fr.size();
  // algorithmic work per launch for the profiler
  {
    const double E = (double)elem();
    unit_small.assign(depth, 0.0);
    exec_small.assign(depth, 0.0);
    unit_small_sym.assign(depth, 0.0);
    exec_small_sym.assign(depth, 0.0);
    unit_up.assign(depth, 0.0);
    unit_down.assign(depth, 0.0);
    unit_update.assign(depth, {});
    exec_update.assign(depth, {});
    unit_update_sym.assign(depth, {});
    exec_update_sym.assign(depth, {});
    exec_update_oz.assign(depth, {});
    for (int L = 0; L < depth; ++L) {
      const LevelInfo &li = levels[L];
      unit_update[L].assign((li.max_p + stdd::MF_NB - 1) / stdd::MF_NB + 1, 0.0);
      exec_update[L].assign(unit_update[L].size(), 0.0);
      unit_update_sym[L].assign(unit_update[L].size(), 0.0);
      exec_update_sym[L].assign(unit_update[L].size(), 0.0);
      exec_update_oz[L].assign(unit_update[L].size(), 0.0);
      for (int f = li.f0; f < li.f0 + li.nf; ++f) {
        const double p = fr[f].p, b = fr[f].b, n = p + b;
        unit_up[L] += E * b * p;
        unit_down[L] += E * p * n;
        if (n <= stdd::MF_SMALL) {
          exec_small[L] += 8.0 * p * n * n;
          exec_small_sym[L] += 8.0 * p * n * (n + 1) / 2;
          for (int k = 0; k < fr[f].p; ++k) {
            unit_small[L] += 8.0 * (n - k - 1) * (n - k - 1);
            unit_small_sym[L] += 8.0 * (n - k - 1) * (n - k) / 2;
          }
        } else {
          for (int k = 0; k < fr[f].p; k += stdd::MF_NB) {
            const double nbk = std::min(stdd::MF_NB, fr[f].p - k);
            const double me = n - nbk, mt = n - k - nbk;
            exec_update[L][k / stdd::MF_NB] += 8.0 * me * me * nbk;
            unit_update[L][k / stdd::MF_NB] += 8.0 * mt * mt * nbk;
            // symmetric form: one triangle with its diagonal
            exec_update_sym[L][k / stdd::MF_NB] += 8.0 * me * (me + 1) / 2 * nbk;
            unit_update_sym[L][k / stdd::MF_NB] += 8.0 * mt * (mt + 1) / 2 * nbk;
            // split tensor-core update: 64 x 64 complex tiles on and below the
            // diagonal, each 36 BF16 products of 128 x 64 x 64 (real)
            const double nto = std::ceil(me / 64.0);
            exec_update_oz[L][k / stdd::MF_NB] += nto * (nto + 1) / 2 * 36.0 * 2.0 * 128 * 64 * 64;
          }
        }
      }
    }
  }
  // substitution work items: (front, row chunk) of the border going up (at
  // least one per front: chunk 0 also stores w_p) and of the pivots coming
  // down.  Levels whose row counts fit in 16 use 16-lane row groups (two
  // fronts per warp); wide fronts split their columns over up to 8 row groups.
  auto pow2_split = [](int cols, int rows) {
    int want = (cols + 4 * rows - 1) / (4 * rows), s = 1;
    while (s < want && s < 8) s *= 2;
    if ((cols + stdd::MF_SEG - 1) / stdd::MF_SEG > stdd::MF_MAXSEG) s = 1;
    return s;
  };
  std::vector<int2> items;
  for (int L = 0; L < depth; ++L) {
    LevelInfo &li = levels[L];
    li.rows_up = li.max_b <= 16 ? 16 : 32;
    li.rows_down = li.max_p <= 16 ? 16 : 32;
    li.split_up = li.split_up1 = pow2_split(li.max_p, li.rows_up);
    li.split_down = li.split_down1 = pow2_split(li.max_n, li.rows_down);
    li.up_off = (int64_t)items.size();
    for (int k = 0; k <= nsub; ++k) {
      lvl_up[L][k] = (int)((int64_t)items.size() - li.up_off);
      if (k == nsub) break;
      for (int f = lvl_front[L][k]; f < lvl_front[L][k + 1]; ++f)
        for (int c = 0; c < std::max(1, (fr[f].b + li.rows_up - 1) / li.rows_up); ++c)
          items.push_back(make_int2(f, c));
    }
    li.n_up = (int)((int64_t)items.size() - li.up_off);
    li.down_off = (int64_t)items.size();
    for (int k = 0; k <= nsub; ++k) {
      lvl_down[L][k] = (int)((int64_t)items.size() - li.down_off);
      if (k == nsub) break;
      for (int f = lvl_front[L][k]; f < lvl_front[L][k + 1]; ++f)
        for (int c = 0; c < (fr[f].p + li.rows_down - 1) / li.rows_down; ++c) items.push_back(make_int2(f, c));
    }
    li.n_down = (int)((int64_t)items.size() - li.down_off);
  }
  {
    // partial sums of the grid-split products: every item of a level times
    // its segments (32 rows each), for the widest level
    int64_t need = 1;
    for (int L = 0; L < depth; ++L) {
      const LevelInfo &li = levels[L];
      const int64_t su = (li.max_p + stdd::MF_SUB - 1) / stdd::MF_SUB, sd = (li.max_n + stdd::MF_SUB - 1) / stdd::MF_SUB;
      need = std::max(need, std::max((int64_t)li.n_up * su, (int64_t)li.n_down * sd) * 32);
    }
    d_segpart.alloc((size_t)need * sizeof(double2));
  }
  // owner of every column (the strip, or the box column kx) and of every row
  // (the box row ky)
  std::vector<int> colstrip(nx), rowbox(ny);
  for (int k = 0; k < nsub; ++k) {
    for (int i = strips[k].c0; i < strips[k].c1; ++i) colstrip[i] = k / nsy;
    for (int j = strips[k].r0; j < strips[k].r1; ++j) rowbox[j] = k % nsy;
  }

  strips_host = sdev;
  fronts_host = fr;
  nodes_host = nodes;
  band_ready = false;
  upload(d_strips, sdev, stream);
  upload(d_fronts, fr, stream);
  upload(d_nodes, nodes, stream);
  upload(d_cmap, cmap, stream);
  upload(d_inv, inv, stream);
  upload(d_colstrip, colstrip, stream);
  upload(d_rowbox, rowbox, stream);
  upload(d_items, items, stream);
  const size_t E = elem();
  d_fac.alloc(std::max<int64_t>(1, factor_entries) * E);
  d_ws[0].alloc(std::max<int64_t>(1, ws_need[0]) * E);
  d_ws[1].alloc(std::max<int64_t>(1, ws_need[1]) * E);
  solve_nrhs_cap = 0;
  d_flag.alloc(sizeof(int));
  d_minpiv.alloc(sizeof(double));
  d_nraised.alloc(sizeof(unsigned long long));
  CK(cudaStreamSynchronize(stream));
}

// Column split of every substitution level, chosen by timing each admissible
// split (1, 2, 4, 8 row groups per item) on the real fronts; the result is
// cached per level shape and does not change the arithmetic (fixed
// summation segments), only the speed.
// Two launch shapes are tuned per level and direction: the launch over every
// strip's fronts (additive order, band space) and the launch over one
// strip's fronts (the sequential orders solve one strip at a time, with far
// fewer work items, so a wider split pays there).
template <typename R> void stdd_ctx::autotune() {
  ensure_solve_buffers(1);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int2 *items = d_items.as<int2>();
  const int one = pos[std::min(1, nsub - 1)];   // an interior strip's position in the level lists
  for (int L = 0; L < depth; ++L) {
    LevelInfo &li = levels[L];
    for (int range = 0; range < 2; ++range) {
      if (range == 1 && nsub == 1) {
        li.split_up1 = li.split_up;
        li.split_down1 = li.split_down;
        continue;
      }
      for (int dir = 0; dir < 2; ++dir) {
        const int rows = dir == 0 ? li.rows_up : li.rows_down;
        const int cols = dir == 0 ? li.max_p : li.max_n;
        int64_t first = dir == 0 ? li.up_off : li.down_off;
        int nitems = dir == 0 ? li.n_up : li.n_down;
        if (range == 1) {
          const std::vector<int> &lv = dir == 0 ? lvl_up[L] : lvl_down[L];
          first += lv[one];
          nitems = lv[one + 1] - lv[one];
        }
        if (nitems == 0) continue;
        const std::vector<int64_t> key = {device, dir, (int64_t)sizeof(R), li.nf, li.max_p, li.max_b, li.min_n,
                                          nitems, rows, range};
        int best = dir == 0 ? li.split_up : li.split_down;
        bool found = false;
        {
          std::lock_guard<std::mutex> lk(tuned_mutex());
          auto hit = tuned().find(key);
          if (hit != tuned().end()) {
            best = hit->second;
            found = true;
          }
        }
        if (!found) {
          float best_ms = 1e30f;
          // in-block splits 1, 2, 4, 8, then the grid split (one warp per
          // segment anywhere on the GPU) for items of 32 rows and several segments
          for (int sp = 1; sp <= stdd::MF_SPLIT_GRID; sp *= 2) {
            if (sp == stdd::MF_SPLIT_GRID) {
              if (rows != 32 || cols <= stdd::MF_SEG) break;
            } else {
              if (sp > 256 / rows) continue;
              if (sp > 1 && (cols + stdd::MF_SEG - 1) / stdd::MF_SEG > stdd::MF_MAXSEG) continue;
            }
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
              MfArgs a = mf_args(L & 1, true);
              CK(cudaEventRecord(e0, stream));
              if (dir == 0) stdd::mf_up_level<R>(a, items + first, nitems, rows, sp, 1, nloc, stream, cols);
              else stdd::mf_down_level<R>(a, items + first, nitems, rows, sp, 1, nloc, stream, cols);
              CK(cudaEventRecord(e1, stream));
              CK(cudaEventSynchronize(e1));
              float ms = 0;
              CK(cudaEventElapsedTime(&ms, e0, e1));
              ms_min = std::min(ms_min, ms);
            }
            if (ms_min < best_ms) {
              best_ms = ms_min;
              best = sp;
            }
          }
          std::lock_guard<std::mutex> lk(tuned_mutex());
          tuned()[key] = best;
        }
        int &dst = range == 0 ? (dir == 0 ? li.split_up : li.split_down) : (dir == 0 ? li.split_up1 : li.split_down1);
        dst = best;
      }
    }
  }
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  CK(cudaGetLastError());
}

void stdd_ctx::factor_prepare() {
  if (pivoting) {
    d_pcol.alloc((size_t)std::max<int64_t>(1, nloc) * sizeof(int));
    d_panel.alloc((size_t)std::max<int64_t>(1, panel_need) * elem());
  }
  static bool attrs = false;
  if (!attrs) {
    CK(stdd::mf_setup_attributes<double>());
    CK(stdd::mf_setup_attributes<float>());
    CK(stdd::tc_setup_attributes());
    attrs = true;
  }
}

// Front-update tile shape per level, chosen by timing: the factorization is
// run level by level once with 64 x 64 and once with 32 x 32 update tiles
// (the other kernels of a level are the same in both), and each level keeps
// the faster.  Both shapes sum every entry's products in the same order, so
// the choice changes no result.  Cached per device and level shape for every
// context of the process (the first factorization of a new shape pays for
// two extra ones).
template <typename R> void stdd_ctx::tune_update_tiles() {
  if (tc_fmt() >= 0) return;
  if (sizeof(R) == 8 && oz_active()) {   // one tile shape on the tensor cores
    for (auto &li : levels) li.upd_tile = 64;
    return;
  }
  if (forced_tile) {
    for (auto &li : levels) li.upd_tile = forced_tile;
    return;
  }
  factor_prepare();
  std::vector<int> todo;
  std::vector<std::vector<int64_t>> keys(depth);
  for (int L = 0; L < depth; ++L) {
    const LevelInfo &li = levels[L];
    if (li.max_n <= stdd::MF_SMALL) continue;
    keys[L] = {device, (int64_t)sizeof(R), 7, sym_active() ? 1 : 0, li.nf, li.max_p, li.max_b, li.max_n, li.min_n};
    std::lock_guard<std::mutex> lk(tuned_mutex());
    auto hit = tuned().find(keys[L]);
    if (hit != tuned().end()) levels[L].upd_tile = hit->second;
    else todo.push_back(L);
  }
  if (todo.empty()) return;
  std::vector<cudaEvent_t> ev(2 * depth);
  for (auto &e : ev) CK(cudaEventCreate(&e));
  std::vector<float> t[2];
  const int tiles[2] = {64, 32};
  for (int v = 0; v < 2; ++v) {
    for (int L : todo) levels[L].upd_tile = tiles[v];
    stdd::mf_factor_begin(mf_args(0, false), stream);
    for (int L = depth - 1; L >= 0; --L) {
      CK(cudaEventRecord(ev[2 * L], stream));
      stdd::mf_factor_level<R>(mf_args(L & 1, false), levels[L], L, stream, nullptr, -1);
      CK(cudaEventRecord(ev[2 * L + 1], stream));
    }
    CK(cudaStreamSynchronize(stream));
    t[v].assign(depth, 0.f);
    for (int L : todo) CK(cudaEventElapsedTime(&t[v][L], ev[2 * L], ev[2 * L + 1]));
  }
  for (auto &e : ev) CK(cudaEventDestroy(e));
  std::lock_guard<std::mutex> lk(tuned_mutex());
  for (int L : todo) {
    levels[L].upd_tile = t[1][L] < t[0][L] ? 32 : 64;
    tuned()[keys[L]] = levels[L].upd_tile;
  }
}

template <typename R> void stdd_ctx::factor_t() {
  factor_prepare();
  const int span = pbegin(PH_FACTOR);
  if (use_graphs && prof < 2) {
    // one replayed graph for all levels (captured again whenever a pointer
    // or value the launches were captured with has changed)
    std::vector<unsigned char> key;
    auto put = [&](const void *p, size_t nb) {
      const unsigned char *c = static_cast<const unsigned char *>(p);
      key.insert(key.end(), c, c + nb);
    };
    const int tc = tc_fmt();
    const size_t rs = sizeof(R);
    put(&tc, sizeof tc);
    put(&rs, sizeof rs);
    put(&depth, sizeof depth);
    for (int par = 0; par < 2; ++par) {
      const MfArgs a = mf_args(par, false);
      put(&a, sizeof a);
    }
    for (const LevelInfo &li : levels) put(&li, sizeof li);
    if (!factor_graph || key != factor_graph_key) {
      if (factor_graph) cudaGraphExecDestroy(factor_graph);
      factor_graph = nullptr;
      const GraphEntry ge = capture([&] { enqueue_factor<R>(); });
      factor_graph_kernels = ge.kernels;
      factor_graph = ge.exec;
      factor_graph_key = key;
    }
    CK(cudaGraphLaunch(factor_graph, stream));
    stdd::count_launch((int)factor_graph_kernels);
  } else {
    enqueue_factor<R>();
  }
  pend(span);
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(&min_pivot, d_minpiv.p, sizeof(double), cudaMemcpyDeviceToHost, stream));
  unsigned long long nr = 0;
  CK(cudaMemcpyAsync(&nr, d_nraised.p, sizeof(nr), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  raised_pivots = (long long)nr;
  if (flag & 2) throw TimeoutError("a tensor-core tile did not complete within its wait limit");
  if (flag & 1) throw std::domain_error("zero or non-finite pivot in a front");
}

// The launches of one numeric factorization, leaves to root.
template <typename R> void stdd_ctx::enqueue_factor() {
  stdd::mf_factor_begin(mf_args(0, false), stream);
  for (int L = depth - 1; L >= 0; --L) {
    MfArgs a = mf_args(L & 1, false);
    hook.c = this;
    stdd::mf_factor_level<R>(a, levels[L], L, stream, &hook, tc_fmt());
    CK(cudaGetLastError());
  }
}

template <typename R> void stdd_ctx::solve_levels(int nr) {
  ensure_solve_buffers(nr);
  const int2 *items = d_items.as<int2>();
  hook.c = this;
  for (int L = depth - 1; L >= 0; --L) {
    const LevelInfo &li = levels[L];
    hook.before(stdd::K_UP, L, 0);
    stdd::mf_up_level<R>(mf_args(L & 1, true), items + li.up_off, li.n_up, li.rows_up, li.split_up, nr, nloc,
                         stream, li.max_p, true);
    hook.after(stdd::K_UP, L, 0);
  }
  for (int L = 0; L < depth; ++L) {
    const LevelInfo &li = levels[L];
    hook.before(stdd::K_DOWN, L, 0);
    stdd::mf_down_level<R>(mf_args(L & 1, true), items + li.down_off, li.n_down, li.rows_down, li.split_down, nr,
                           nloc, stream, li.max_n);
    hook.after(stdd::K_DOWN, L, 0);
  }
  CK(cudaGetLastError());
}

// Forward and back substitution of the strips at positions [j0, j1) of
// perm alone: the level kernels of solve_levels on their subrange of fronts
// and work items.
template <typename R> void stdd_ctx::solve_range_levels(int j0, int j1, int nr) {
  const int2 *items = d_items.as<int2>();
  hook.c = this;
  // per-launch spans (profiling level 2) credit each launch with its share
  // of the level's factor bytes, by its fraction of the level's work items
  for (int L = depth - 1; L >= 0; --L) {
    LevelInfo li = levels[L];
    li.f0 = lvl_front[L][j0];
    li.nf = lvl_front[L][j1] - lvl_front[L][j0];
    if (li.nf == 0) continue;
    const int cnt = lvl_up[L][j1] - lvl_up[L][j0];
    hook.before_part(stdd::K_UP, L, levels[L].n_up ? (double)cnt / levels[L].n_up : 0.0);
    stdd::mf_up_level<R>(mf_args(L & 1, true), items + li.up_off + lvl_up[L][j0], cnt, li.rows_up,
                         j1 - j0 == 1 ? li.split_up1 : li.split_up, nr, nloc, stream, li.max_p, true);
    hook.after(stdd::K_UP, L, 0);
  }
  for (int L = 0; L < depth; ++L) {
    const LevelInfo &li = levels[L];
    const int cnt = lvl_down[L][j1] - lvl_down[L][j0];
    if (cnt == 0) continue;
    hook.before_part(stdd::K_DOWN, L, li.n_down ? (double)cnt / li.n_down : 0.0);
    stdd::mf_down_level<R>(mf_args(L & 1, true), items + li.down_off + lvl_down[L][j0], cnt, li.rows_down,
                           j1 - j0 == 1 ? li.split_down1 : li.split_down, nr, nloc, stream, li.max_n);
    hook.after(stdd::K_DOWN, L, 0);
  }
  CK(cudaGetLastError());
}

// Strips of one colour may be solved together only if none of them changes
// the residual another one reads: the local box of strip k (with its stencil
// reach of one column) must stay clear of the owned columns of strip k + 2.
void stdd_ctx::check_red_black() const {
  for (int k = 0; k + 2 < nsub; ++k)
    if (strips[k].x1 + 1 > strips[k + 2].c0 || strips[k + 2].x0 - 1 < strips[k].c1)
      throw ArgError("red-black order needs every interior strip wider than overlap + interface PML + 1");
}

// Multiplicative orders: z = 0, then group by group (a group = positions
// [j0, j1) of perm): every strip k of the group solves for the current
// residual, z += E_k A_k^-1 R_k^I (v - A z), all of them from the same z.
// Order 1: single strips k = 0 .. n-1, n-2 .. 0 (symmetric sweep); order 2:
// the even strips, then the odd strips (red-black; the same as solving them
// one by one because same-colour strips do not interact, check_red_black).
// Every slot i has its own (v_i, z_i).
template <typename R>
void stdd_ctx::enqueue_minv_multiplicative(const std::vector<const double2 *> &vs, const std::vector<double2 *> &zs) {
  const int na = (int)vs.size();
  const size_t E = elem();
  const stdd::GridDev g = grid();
  auto slot = [&](int i) { return static_cast<void *>(d_tloc.as<char>() + (size_t)i * nloc * E); };
  for (int i = 0; i < na; ++i) CK(cudaMemsetAsync(zs[i], 0, (size_t)N() * sizeof(double2), stream));
  std::vector<std::pair<int, int>> groups;
  if (order == 2) {
    const int ne = (nsub + 1) / 2;
    groups.push_back({0, ne});
    if (nsub > 1) groups.push_back({ne, nsub});
  } else {
    for (int k = 0; k < nsub; ++k) groups.push_back({pos[k], pos[k] + 1});
    if (order == 1)  // symmetric: back again (order 3 is the forward sweep alone)
      for (int k = nsub - 2; k >= 0; --k) groups.push_back({pos[k], pos[k] + 1});
  }
  if (persistent_eff() && na == 1 && order != 2 && d_striplv.p) {
    // one cooperative launch per strip solve (the barrier counters are
    // cleared before each, so a sweep that gave up leaves nothing behind)
    MfArgs a = mf_args(0, true);
    a.items_sweep = d_items.as<int2>();
    for (const auto &gr : groups) {
      const int j = gr.first;
      CK(cudaMemsetAsync(d_bar.p, 0, 2 * sizeof(unsigned), stream));
      hook.before(stdd::K_SWEEP, perm[j], 0);
      CK(stdd::mf_strip_sweep_launch<R>(a, d_ub[0].p, d_ub[1].p, g, strips_host[perm[j]],
                                        d_striplv.as<stdd::StripLevel>() + (size_t)j * depth, depth, vs[0], zs[0],
                                        d_bar.as<unsigned>(), d_sweep_flag.as<int>(), sweep_wait, persistent_eff(),
                                        stream));
      hook.after(stdd::K_SWEEP, perm[j], 0);
    }
    return;
  }
  for (const auto &gr : groups) {
    for (int j = gr.first; j < gr.second; ++j)
      for (int i = 0; i < na; ++i)
        stdd::launch_restrict_residual_strip<R>(g, strips_host[perm[j]], vs[i], zs[i], slot(i), stream);
    solve_range_levels<R>(gr.first, gr.second, na);
    for (int j = gr.first; j < gr.second; ++j)
      for (int i = 0; i < na; ++i) stdd::launch_add_strip<R>(strips_host[perm[j]], ny, slot(i), zs[i], stream);
  }
  CK(cudaGetLastError());
}

// Band analysis.  For the additive order, A M^-1 v - v vanishes outside the
// interface bands (the transfer identity): around the interface at column c
// between strips k and k+1 the band is [c - e_l - 1, c + e_r + 1), e_r the
// columns strip k's box reaches past c, e_l those strip k+1's box reaches
// before it (the stencil adds one).  A band vector's sources reach strip k
// only on its owned band columns, and the band values of A M^-1 v need the
// synthesized field on the band widened by one column.
void stdd_ctx::build_band() {
  if (band_ready) return;
  std::vector<std::pair<int, int>> ivs;  // [first, last) columns
  for (int k = 0; k + 1 < nsub; ++k) {
    const int c = strips[k].c1;
    const int er = strips[k].x1 - c, el = c - strips[k + 1].x0;
    ivs.push_back({std::max(0, c - el - 1), std::min(nx, c + er + 1)});
  }
  auto merge = [](std::vector<std::pair<int, int>> v) {
    std::sort(v.begin(), v.end());
    std::vector<std::pair<int, int>> out;
    for (auto &p : v) {
      if (!out.empty() && p.first <= out.back().second) out.back().second = std::max(out.back().second, p.second);
      else out.push_back(p);
    }
    return out;
  };
  const auto b0 = merge(ivs);
  std::vector<std::pair<int, int>> w1;
  for (auto &p : b0) w1.push_back({std::max(0, p.first - 1), std::min(nx, p.second + 1)});
  const auto b1 = merge(w1);
  auto lay = [&](const std::vector<std::pair<int, int>> &b, std::vector<int2> &iv, std::vector<int64_t> &off) {
    iv.clear();
    off.clear();
    int64_t o = 0;
    for (auto &p : b) {
      iv.push_back(make_int2(p.first, p.second - p.first));
      off.push_back(o);
      o += (int64_t)(p.second - p.first) * ny;
    }
    if (iv.empty()) {  // one strip: no band (keep the arrays non-empty)
      iv.push_back(make_int2(0, 0));
      off.push_back(0);
    }
    return o;
  };
  band_n = lay(b0, band_iv, band_off);
  band_n1 = lay(b1, band_iv1, band_off1);
  std::vector<int64_t> colband(nx, -1);
  std::vector<char> in1(nx, 0);
  for (size_t k = 0; k < b0.size(); ++k)
    for (int c = b0[k].first; c < b0[k].second; ++c) colband[c] = band_off[k] + (int64_t)(c - b0[k].first) * ny;
  for (auto &p : b1)
    for (int c = p.first; c < p.second; ++c) in1[c] = 1;
  // active fronts; children come after their parents in the level-major list
  const int64_t nf = (int64_t)fronts_host.size();
  std::vector<char> up(nf, 0), dn(nf, 0);
  for (int64_t f = nf - 1; f >= 0; --f) {
    const FrontDev &d = fronts_host[f];
    const StripHost &st = strips[d.strip];
    bool u = false, w = false;
    for (int q = 0; q < d.p && !(u && w); ++q) {
      const int col = st.x0 + nodes_host[d.node_off + q] / ny;
      if (col >= st.c0 && col < st.c1 && colband[col] >= 0) u = true;
      if (in1[col]) w = true;
    }
    for (int ci = 0; ci < 2; ++ci)
      if (d.child[ci] >= 0) {
        u = u || up[d.child[ci]];
        w = w || dn[d.child[ci]];
      }
    up[f] = u;
    dn[f] = w;
  }
  std::vector<int2> items;
  lvl_bup_off.assign(depth, 0);
  lvl_bdown_off.assign(depth, 0);
  lvl_bup_n.assign(depth, 0);
  lvl_bdown_n.assign(depth, 0);
  for (int L = 0; L < depth; ++L) {
    const LevelInfo &li = levels[L];
    lvl_bup_off[L] = (int64_t)items.size();
    for (int f = li.f0; f < li.f0 + li.nf; ++f)
      if (up[f])
        for (int c = 0; c < std::max(1, (fronts_host[f].b + li.rows_up - 1) / li.rows_up); ++c)
          items.push_back(make_int2(f, c));
    lvl_bup_n[L] = (int)((int64_t)items.size() - lvl_bup_off[L]);
    lvl_bdown_off[L] = (int64_t)items.size();
    for (int f = li.f0; f < li.f0 + li.nf; ++f)
      if (dn[f])
        for (int c = 0; c < (fronts_host[f].p + li.rows_down - 1) / li.rows_down; ++c)
          items.push_back(make_int2(f, c));
    lvl_bdown_n[L] = (int)((int64_t)items.size() - lvl_bdown_off[L]);
  }
  if (items.empty()) items.push_back(make_int2(0, 0));
  upload(d_band_iv, band_iv, stream);
  upload(d_band_off, band_off, stream);
  upload(d_band_iv1, band_iv1, stream);
  upload(d_band_off1, band_off1, stream);
  upload(d_colband, colband, stream);
  upload(d_items_band, items, stream);
  CK(cudaStreamSynchronize(stream));
  band_ready = true;
}

// Substitution sweeps for band sources: the gather over every front (it
// writes zeros where a subtree has no source), the upward GEMVs of the
// fronts with sources in their subtree, the downward ones of the fronts the
// widened band needs.
template <typename R> void stdd_ctx::solve_levels_band(int nr) {
  ensure_solve_buffers(nr);
  const int2 *items = d_items_band.as<int2>();
  for (int L = depth - 1; L >= 0; --L) {
    const LevelInfo &li = levels[L];
    stdd::mf_up_gather_level<R>(mf_args(L & 1, true), li, nr, nloc, stream);
    stdd::mf_up_level<R>(mf_args(L & 1, true), items + lvl_bup_off[L], lvl_bup_n[L], li.rows_up, li.split_up, nr,
                         nloc, stream, li.max_p);
  }
  for (int L = 0; L < depth; ++L) {
    const LevelInfo &li = levels[L];
    stdd::mf_down_level<R>(mf_args(L & 1, true), items + lvl_bdown_off[L], lvl_bdown_n[L], li.rows_down,
                           li.split_down, nr, nloc, stream, li.max_n);
  }
  CK(cudaGetLastError());
}

// y_i = (A M^-1 G(s_i))|band = (I + T) s_i for band vectors s_i; the
// synthesized fields go to the Z storage (unused by the band iteration).
void stdd_ctx::enqueue_op_band(const std::vector<const double2 *> &ss, const std::vector<double2 *> &ys) {
  const int na = (int)ss.size();
  const size_t E = elem();
  const stdd::BandDev bd = band_dev();
  auto slot = [&](int i) { return static_cast<void *>(d_tloc.as<char>() + (size_t)i * nloc * E); };
  const bool fp64 = prec == STDD_PREC_FP64;
  for (int i = 0; i < na; ++i) {
    if (fp64)
      stdd::launch_restrict_band<double>(d_strips.as<StripDev>(), nsub, nloc_max, ny, d_colband.as<int64_t>(), ss[i],
                                         slot(i), stream);
    else
      stdd::launch_restrict_band<float>(d_strips.as<StripDev>(), nsub, nloc_max, ny, d_colband.as<int64_t>(), ss[i],
                                        slot(i), stream);
  }
  if (fp64) solve_levels_band<double>(na);
  else solve_levels_band<float>(na);
  for (int i = 0; i < na; ++i) {
    double2 *zg = d_Z.as<double2>() + (int64_t)i * N();
    if (fp64)
      stdd::launch_synthesize_band<double>(d_strips.as<StripDev>(), nsub, ny, d_colstrip.as<int>(), bd, slot(i), zg,
                                           stream);
    else
      stdd::launch_synthesize_band<float>(d_strips.as<StripDev>(), nsub, ny, d_colstrip.as<int>(), bd, slot(i), zg,
                                          stream);
    stdd::launch_stencil_band(grid(), bd, zg, nullptr, false, false, ys[i], stream);
  }
  CK(cudaGetLastError());
}

void stdd_ctx::apply_op_band(const std::vector<const double2 *> &ss, const std::vector<double2 *> &ys) {
  const int na = (int)ss.size();
  ensure_solve_buffers(na);
  const int span = pbegin(PH_MINV);
  if (use_graphs && prof < 2) {
    std::vector<const void *> key{reinterpret_cast<const void *>(1)};  // tag: band operator
    for (int i = 0; i < na; ++i) {
      key.push_back(ss[i]);
      key.push_back(ys[i]);
    }
    auto it = minv_graphs.find(key);
    if (it == minv_graphs.end()) {
      it = minv_graphs.emplace(key, capture([&] { enqueue_op_band(ss, ys); })).first;
    }
    CK(cudaGraphLaunch(it->second.exec, stream));
    stdd::count_launch((int)it->second.kernels);
  } else {
    enqueue_op_band(ss, ys);
  }
  pend(span);
  CK(cudaGetLastError());
}

void stdd_ctx::ensure_solve_buffers(int nr) {
  if (nr <= solve_nrhs_cap) return;
  clear_graphs();
  const size_t E = elem();
  d_tloc.alloc(std::max<int64_t>(1, nloc) * nr * E);
  d_wloc.alloc(std::max<int64_t>(1, nloc) * nr * E);
  d_ub[0].alloc(std::max<int64_t>(1, ub_elems[0]) * nr * E);
  d_ub[1].alloc(std::max<int64_t>(1, ub_elems[1]) * nr * E);
  solve_nrhs_cap = nr;
}

// z_i = M^-1 v_i for every pair: restriction of each v_i to the strips'
// owned columns (local slot i), batched upward / downward sweeps over all
// strips and all slots, synthesis of the full local fields into z_i.
void stdd_ctx::apply_minv(const double2 *v, double2 *z) {
  std::vector<const double2 *> vs{v};
  std::vector<double2 *> zs{z};
  apply_minv_multi(vs, zs);
}

void stdd_ctx::apply_minv_multi(const std::vector<const double2 *> &vs, const std::vector<double2 *> &zs) {
  const int na = (int)vs.size();
  ensure_solve_buffers(na);
  const int span = pbegin(PH_MINV);
  // replay a captured graph of the whole application (one per list of
  // buffers); per-launch profiling needs the individual launches
  if (use_graphs && prof < 2) {
    std::vector<const void *> key;
    for (int i = 0; i < na; ++i) {
      key.push_back(vs[i]);
      key.push_back(zs[i]);
    }
    auto it = minv_graphs.find(key);
    if (it == minv_graphs.end()) {
      it = minv_graphs.emplace(key, capture([&] { enqueue_minv(vs, zs); })).first;
    }
    CK(cudaGraphLaunch(it->second.exec, stream));
    stdd::count_launch((int)it->second.kernels);
    pend(span);
    return;
  }
  enqueue_minv(vs, zs);
  pend(span);
  CK(cudaGetLastError());
}

void stdd_ctx::enqueue_minv(const std::vector<const double2 *> &vs, const std::vector<double2 *> &zs) {
  const int na = (int)vs.size();
  const size_t E = elem();
  if (order != 0) {
    require_strips("the multiplicative and red-black orders");
    if (order == 2) check_red_black();
    if (prec == STDD_PREC_FP64) enqueue_minv_multiplicative<double>(vs, zs);
    else enqueue_minv_multiplicative<float>(vs, zs);
    return;
  }
  auto slot = [&](int i) { return static_cast<void *>(d_tloc.as<char>() + (size_t)i * nloc * E); };
  if (boxes()) {
    // 2-D boxes: owned blocks in, full local fields summed over <= 9 boxes out
    const StripDev *bx = d_strips.as<StripDev>();
    if (prec == STDD_PREC_FP64) {
      for (int i = 0; i < na; ++i) stdd::launch_restrict_box<double>(bx, nsub, nloc_max, ny, vs[i], slot(i), stream);
      solve_levels<double>(na);
      for (int i = 0; i < na; ++i)
        stdd::launch_synthesize_box<double>(bx, nsx, nsy, nx, ny, d_colstrip.as<int>(), d_rowbox.as<int>(), slot(i),
                                            zs[i], stream);
    } else {
      for (int i = 0; i < na; ++i) stdd::launch_restrict_box<float>(bx, nsub, nloc_max, ny, vs[i], slot(i), stream);
      solve_levels<float>(na);
      for (int i = 0; i < na; ++i)
        stdd::launch_synthesize_box<float>(bx, nsx, nsy, nx, ny, d_colstrip.as<int>(), d_rowbox.as<int>(), slot(i),
                                           zs[i], stream);
    }
    CK(cudaGetLastError());
    return;
  }
  if (prec == STDD_PREC_FP64) {
    for (int i = 0; i < na; ++i)
      stdd::launch_restrict<double>(d_strips.as<StripDev>(), nsub, nloc_max, ny, nullptr, vs[i], slot(i), stream);
    solve_levels<double>(na);
    for (int i = 0; i < na; ++i)
      stdd::launch_synthesize<double>(d_strips.as<StripDev>(), nsub, nx, ny, d_colstrip.as<int>(), slot(i), zs[i],
                                      stream);
  } else {
    for (int i = 0; i < na; ++i)
      stdd::launch_restrict<float>(d_strips.as<StripDev>(), nsub, nloc_max, ny, nullptr, vs[i], slot(i), stream);
    solve_levels<float>(na);
    for (int i = 0; i < na; ++i)
      stdd::launch_synthesize<float>(d_strips.as<StripDev>(), nsub, nx, ny, d_colstrip.as<int>(), slot(i), zs[i],
                                     stream);
  }
  CK(cudaGetLastError());
}

void stdd_ctx::ensure_krylov(int m) {
  const int64_t n = N();
  const int nq = std::max(1, nrhs);
  if (V_cols < m || V_rhs < nq) {
    d_V.release();
    d_Z.release();
    d_V.alloc((size_t)(m + 1) * n * nq * sizeof(double2));
    d_Z.alloc((size_t)m * n * nq * sizeof(double2));
    V_cols = m;
    V_rhs = nq;
    clear_graphs();
  }
  d_x.alloc(n * nq * sizeof(double2));
  d_r.alloc(n * sizeof(double2));
  d_w.alloc(n * sizeof(double2));
  d_part.alloc((size_t)stdd::krylov_partial_blocks() * (m + 2) * sizeof(double2));
  d_h.alloc((size_t)(2 * (m + 2)) * nq * sizeof(double2));
  d_nrm.alloc((4 + 2 * (size_t)nq) * sizeof(double));
  d_y.alloc((size_t)(m + 1) * nq * sizeof(double2));
  d_fpart.alloc((size_t)std::max(1, 2 * nsub) * sizeof(double));
}

namespace {
void givens(cd a, cd b, double &c, cd &s) {
  if (std::abs(b) == 0) {
    c = 1;
    s = 0;
    return;
  }
  if (std::abs(a) == 0) {
    c = 0;
    s = std::conj(b) / std::abs(b);
    return;
  }
  const double t = std::hypot(std::abs(a), std::abs(b));
  c = std::abs(a) / t;
  s = (a / std::abs(a)) * std::conj(b) / t;
}

double dev_norm(double2 *x, int64_t n, DBuf &part, DBuf &nrm, cudaStream_t st) {
  stdd::launch_norm2(x, n, reinterpret_cast<double *>(part.p), nrm.as<double>(), st);
  double v = 0;
  CK(cudaMemcpyAsync(&v, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return std::sqrt(v);
}
}  // namespace

// Restarted flexible GMRES(m), right preconditioned by M^-1, for every
// right-hand side at once: each has its own basis V_q, Z_q, Hessenberg
// matrix, Givens rotations and restart cycle, and they advance in lockstep
// so that one batched M^-1 application serves all systems still iterating.
// FP64 throughout; classical Gram-Schmidt with a second pass when the first
// one shrank ||w|| below 1/sqrt(2) of its value (Daniel-Gragg-Kaufman-
// Stewart); Givens rotations and the small triangular solves on the host.
// d_x holds the initial guesses on entry and the iterates on exit.
// Band mode (STDD_OPT_BAND, additive order): with r0 = b - A x0 and
// T = A M^-1 - I, whose range is the interface bands when the local solves
// are exact, the right-preconditioned iterate x = x0 + M^-1 (r0 + s) has the
// residual b - A x = -(T r0 + (I + T) s) on the bands and zero elsewhere, so
// GMRES runs on the band system (I + T) s = -T r0 with band-sized vectors
// and partial sweeps.  One full application before (for T r0, counted as an
// iteration) and one after (for x).  The cycle ends with the true residual
// of the new x, which equals the band residual up to rounding (FP64 local
// solves); should rounding leave it above rtol, another cycle starts from
// the new x.
void stdd_ctx::gmres_multi(const stdd_solve_opts &o) {
  const int m = o.restart, nq = nrhs;
  bool band = use_band;
  const int64_t NN = N();
  ensure_krylov(m);
  if (band) {
    build_band();
    band = band_n > 0;  // one strip: no bands, the standard iteration
  }
  const int64_t n = band ? band_n : NN;
  double2 *Vb = d_V.as<double2>(), *Zb = d_Z.as<double2>(), *X = d_x.as<double2>(), *r = d_r.as<double2>();
  double *nrm_base = d_nrm.as<double>();
  double *part = reinterpret_cast<double *>(d_part.p);
  auto V = [&](int q, int j) { return Vb + ((int64_t)q * (m + 1) + j) * n; };
  auto Z = [&](int q, int j) { return band ? V(q, j) : Zb + ((int64_t)q * m + j) * n; };
  if (band) {
    d_fb.alloc((size_t)std::max<int64_t>(1, n) * nq * sizeof(double2));
    d_sb.alloc((size_t)std::max<int64_t>(1, n) * nq * sizeof(double2));
  }
  auto FB = [&](int q) { return d_fb.as<double2>() + (int64_t)q * n; };
  auto SB = [&](int q) { return d_sb.as<double2>() + (int64_t)q * n; };
  // x (full field, standard mode) or s (band vector, band mode) of rhs q
  auto XS = [&](int q) { return band ? SB(q) : X + (int64_t)q * NN; };
  auto h1 = [&](int q) { return d_h.as<double2>() + (size_t)q * 2 * (m + 2); };
  auto h2 = [&](int q) { return h1(q) + (m + 2); };
  auto nrmq = [&](int q) { return nrm_base + 4 + 2 * q; };
  struct St {
    std::vector<cd> H, g, sn, hv;
    std::vector<double> cs;
    double bnorm = 0, nrm2 = 0, res = 0, tgt = 0;  // tgt: absolute residual target of the iteration
    int its = 0, reorth = 0, k = 0;
    bool done = false;
  };
  std::vector<St> S(nq);
  for (int q = 0; q < nq; ++q) {
    St &t = S[q];
    t.H.assign((size_t)(m + 1) * m, 0);
    t.g.assign(m + 1, 0);
    t.sn.assign(m, 0);
    t.cs.assign(m, 0);
    t.hv.assign(2 * (m + 2), 0);
    const double2 *b = d_b.as<double2>() + (int64_t)q * NN;
    t.bnorm = dev_norm(const_cast<double2 *>(b), NN, d_part, d_nrm, stream);
    t.tgt = o.rtol * t.bnorm;
    if (t.bnorm == 0) {
      CK(cudaMemsetAsync(X + (int64_t)q * NN, 0, NN * sizeof(double2), stream));
      history[q].push_back(0.0);
      t.done = true;
    }
  }
  std::vector<char> s_zero(nq, 1);
  for (int cycle = 0;; ++cycle) {
  std::vector<int> cyc;  // right-hand sides iterating in this band cycle
  if (band) {
    // true residual r0 = b - A x (in the V storage); if not yet at rtol:
    // z = M^-1 r0 (in Z), f = (r0 - A z)|band, s = 0
    std::vector<const double2 *> rs;
    std::vector<double2 *> zs;
    for (int q = 0; q < nq; ++q) {
      St &t = S[q];
      if (t.done) continue;
      double2 *r0 = Vb + (int64_t)q * NN;
      stdd::launch_residual(grid(), d_b.as<double2>() + (int64_t)q * NN, X + (int64_t)q * NN, r0, stream);
      const double rn = dev_norm(r0, NN, d_part, d_nrm, stream) / t.bnorm;
      history[q].push_back(rn);
      t.res = rn;
      if (!std::isfinite(rn)) throw std::range_error("non-finite residual");
      if (rn <= o.rtol || t.its >= o.maxit) {
        t.done = true;
        continue;
      }
      rs.push_back(r0);
      zs.push_back(Zb + (int64_t)q * NN);
      cyc.push_back(q);
    }
    if (cyc.empty()) break;
    apply_minv_multi(rs, zs);
    const stdd::BandDev bd = band_dev();
    for (size_t i = 0; i < cyc.size(); ++i) {
      const int q = cyc[i];
      St &t = S[q];
      stdd::launch_stencil_band(grid(), bd, zs[i], rs[i], true, true, FB(q), stream);
      CK(cudaMemsetAsync(SB(q), 0, std::max<int64_t>(1, n) * sizeof(double2), stream));
      history[q].push_back(dev_norm(FB(q), n, d_part, d_nrm, stream) / t.bnorm);
      t.its += 1;
      t.tgt = o.rtol * t.bnorm;
      s_zero[q] = 1;
    }
  }
  while (true) {
    // restart cycle: true residuals, first basis vectors
    std::vector<int> act;
    for (int q = 0; q < nq; ++q) {
      St &t = S[q];
      if (t.done) continue;
      int sp = pbegin(PH_MATVEC);
      if (band) {
        // r = f - (I + T) s, the true residual on the band
        if (s_zero[q]) {
          CK(cudaMemcpyAsync(r, FB(q), n * sizeof(double2), cudaMemcpyDeviceToDevice, stream));
        } else {
          apply_op_band({SB(q)}, {V(q, 0)});
          stdd::launch_vsub(FB(q), V(q, 0), r, n, stream);
        }
      } else {
        stdd::launch_residual(grid(), d_b.as<double2>() + (int64_t)q * NN, X + (int64_t)q * NN, r, stream);
      }
      pend(sp);
      const double beta = dev_norm(r, n, d_part, d_nrm, stream);
      if (history[q].empty()) history[q].push_back(beta / t.bnorm);
      t.res = beta / t.bnorm;
      if (!std::isfinite(beta)) throw std::range_error("non-finite residual");
      if (beta <= t.tgt || t.its >= o.maxit) {
        t.done = true;
        continue;
      }
      stdd::launch_scale(r, d_nrm.as<double>(), V(q, 0), n, stream);
      std::fill(t.H.begin(), t.H.end(), cd(0));
      std::fill(t.g.begin(), t.g.end(), cd(0));
      t.g[0] = beta;
      t.k = 0;
      act.push_back(q);
    }
    if (act.empty()) break;
    std::vector<int> inner = act;
    for (int j = 0; j < m && !inner.empty(); ++j) {
      std::vector<const double2 *> vs;
      std::vector<double2 *> zs;
      for (int q : inner) {
        vs.push_back(V(q, j));
        zs.push_back(Z(q, j));
      }
      if (band) {
        std::vector<double2 *> ws;
        for (int q : inner) ws.push_back(V(q, j + 1));
        apply_op_band(vs, ws);
      } else {
        apply_minv_multi(vs, zs);
        int sp = pbegin(PH_MATVEC);
        for (int q : inner) stdd::launch_stencil(grid(), Z(q, j), V(q, j + 1), stream);
        pend(sp);
      }
      int sp = pbegin(PH_ORTHO);
      for (int q : inner) {
        double2 *w = V(q, j + 1);
        stdd::launch_mdot(V(q, 0), n, j + 1, w, n, d_part.as<double2>(), h1(q), stream, 1);
        stdd::launch_maxpy_norm(V(q, 0), n, j + 1, h1(q), w, n, part, nrmq(q), stream);
        CK(cudaMemcpyAsync(S[q].hv.data(), h1(q), sizeof(double2) * (j + 2), cudaMemcpyDeviceToHost, stream));
        CK(cudaMemcpyAsync(&S[q].nrm2, nrmq(q), sizeof(double), cudaMemcpyDeviceToHost, stream));
      }
      poll_sweep_flag();
      CK(cudaStreamSynchronize(stream));
      raise_sweep_flag();
      std::vector<int> again;
      for (int q : inner) {
        St &t = S[q];
        for (int i = 0; i <= j; ++i) t.H[(size_t)i * m + j] = t.hv[i];
        if (t.nrm2 < 0.5 * t.hv[j + 1].real()) again.push_back(q);
      }
      for (int q : again) {
        double2 *w = V(q, j + 1);
        stdd::launch_mdot(V(q, 0), n, j + 1, w, n, d_part.as<double2>(), h2(q), stream);
        stdd::launch_maxpy_norm(V(q, 0), n, j + 1, h2(q), w, n, part, nrmq(q), stream);
        CK(cudaMemcpyAsync(S[q].hv.data() + (m + 2), h2(q), sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost,
                           stream));
        CK(cudaMemcpyAsync(&S[q].nrm2, nrmq(q), sizeof(double), cudaMemcpyDeviceToHost, stream));
      }
      if (!again.empty()) CK(cudaStreamSynchronize(stream));
      for (int q : again) {
        St &t = S[q];
        for (int i = 0; i <= j; ++i) t.H[(size_t)i * m + j] += t.hv[(m + 2) + i];
        ++t.reorth;
      }
      pend(sp);
      std::vector<int> next;
      for (int q : inner) {
        St &t = S[q];
        std::vector<cd> &H = t.H;
        const double hn = std::sqrt(t.nrm2);
        H[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
          const cd a = t.cs[i] * H[(size_t)i * m + j] + t.sn[i] * H[(size_t)(i + 1) * m + j];
          H[(size_t)(i + 1) * m + j] = -std::conj(t.sn[i]) * H[(size_t)i * m + j] + t.cs[i] * H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = a;
        }
        givens(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j], t.cs[j], t.sn[j]);
        const cd hjj = t.cs[j] * H[(size_t)j * m + j] + t.sn[j] * H[(size_t)(j + 1) * m + j];
        H[(size_t)j * m + j] = hjj;
        H[(size_t)(j + 1) * m + j] = 0;
        t.g[j + 1] = -std::conj(t.sn[j]) * t.g[j];
        t.g[j] = t.cs[j] * t.g[j];
        ++t.its;
        t.k = j + 1;
        const double est = std::abs(t.g[j + 1]) / t.bnorm;
        history[q].push_back(est);
        if (!std::isfinite(est)) throw std::range_error("non-finite residual estimate");
        const bool breakdown = !(hn > 0) || std::abs(hjj) == 0;
        if (!breakdown) stdd::launch_scale(V(q, j + 1), nrmq(q), V(q, j + 1), n, stream);
        if (!(est * t.bnorm <= t.tgt || t.its >= o.maxit || breakdown)) next.push_back(q);
      }
      inner.swap(next);
    }
    // x_q += Z_q y_q with y_q = R_q^-1 g_q
    for (int q : act) {
      St &t = S[q];
      const int k = t.k;
      std::vector<cd> y(k);
      for (int i = k - 1; i >= 0; --i) {
        cd sum = t.g[i];
        for (int l = i + 1; l < k; ++l) sum -= t.H[(size_t)i * m + l] * y[l];
        y[i] = sum / t.H[(size_t)i * m + i];
      }
      std::vector<double2> yd(k);
      for (int i = 0; i < k; ++i) yd[i] = make_double2(y[i].real(), y[i].imag());
      double2 *yq = d_y.as<double2>() + (size_t)q * (m + 1);
      CK(cudaMemcpyAsync(yq, yd.data(), sizeof(double2) * k, cudaMemcpyHostToDevice, stream));
      stdd::launch_maxpy(Z(q, 0), n, k, yq, XS(q), n, stream);
      s_zero[q] = 0;
    }
    CK(cudaStreamSynchronize(stream));
  }
  if (!band) break;
  {
    // x = x + M^-1 (r0 + s): r0 again (in V storage), plus the band s
    std::vector<const double2 *> rs;
    std::vector<double2 *> zs;
    const stdd::BandDev bd = band_dev();
    for (int q : cyc) {
      double2 *r0 = Vb + (int64_t)q * NN;
      stdd::launch_residual(grid(), d_b.as<double2>() + (int64_t)q * NN, X + (int64_t)q * NN, r0, stream);
      stdd::launch_band_scatter_add(bd, ny, SB(q), r0, stream);
      rs.push_back(r0);
      zs.push_back(Zb + (int64_t)q * NN);
    }
    apply_minv_multi(rs, zs);
    for (size_t i = 0; i < cyc.size(); ++i) stdd::nn_zadd(zs[i], X + (int64_t)cyc[i] * NN, NN, stream);
    CK(cudaStreamSynchronize(stream));
    // the next cycle starts from the true residual of the new x
    for (int q : cyc) S[q].done = false;
  }
  }  // cycles
  last_noconv = false;
  for (int q = 0; q < nq; ++q)
    if (!(S[q].res <= o.rtol)) last_noconv = true;
  last_its = S[0].its;
  last_reorth = 0;
  for (int q = 0; q < nq; ++q) last_reorth += S[q].reorth;
  last_res = S[0].res;
}

// Algorithm 1 in residual form: x_{n+1} = x_n + M^-1 (b - A x_n) from x_0,
// stopping when sum_i ||e_i^F|| < rtol * sum_i ||e_i^(0)|| (Eq. 20, with a
// relative TOL); the history records the true relative residual per sweep.
void stdd_ctx::richardson(int rhs, const stdd_solve_opts &o, double2 *x) {
  const int64_t n = N();
  ensure_krylov(1);
  auto &hist = history[rhs];
  const double2 *b = d_b.as<double2>() + (int64_t)rhs * n;
  const double bnorm = dev_norm(const_cast<double2 *>(b), n, d_part, d_nrm, stream);
  double2 *r = d_r.as<double2>(), *z = d_w.as<double2>();
  double f0 = -1;
  int its = 0;
  stdd::launch_residual(grid(), b, x, r, stream);
  hist.push_back(bnorm > 0 ? dev_norm(r, n, d_part, d_nrm, stream) / bnorm : 0.0);
  while (its < o.maxit && bnorm > 0) {
    apply_minv(r, z);
    // sum_i ||e_i^F|| and sum_i ||e_i|| from the local fields of this sweep
    if (prec == STDD_PREC_FP64)
      stdd::launch_strip_norms<double>(d_strips.as<StripDev>(), nsub, ny, d_tloc.p, d_fpart.as<double>(), stream);
    else
      stdd::launch_strip_norms<float>(d_strips.as<StripDev>(), nsub, ny, d_tloc.p, d_fpart.as<double>(), stream);
    std::vector<double> sn2(2 * nsub);
    CK(cudaMemcpyAsync(sn2.data(), d_fpart.p, sizeof(double) * 2 * nsub, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    double fsum = 0, esum = 0;
    for (int k = 0; k < nsub; ++k) {
      fsum += std::sqrt(sn2[2 * k]);
      esum += std::sqrt(sn2[2 * k + 1]);
    }
    if (f0 < 0) f0 = esum;
    // x += z
    std::vector<double2> one(1, make_double2(1.0, 0.0));
    CK(cudaMemcpyAsync(d_y.p, one.data(), sizeof(double2), cudaMemcpyHostToDevice, stream));
    stdd::launch_maxpy(z, n, 1, d_y.as<double2>(), x, n, stream);
    ++its;
    stdd::launch_residual(grid(), b, x, r, stream);
    const double res = dev_norm(r, n, d_part, d_nrm, stream) / bnorm;
    hist.push_back(res);
    last_res = res;
    if (!std::isfinite(res)) throw std::range_error("non-finite residual");
    if (fsum < o.rtol * f0) break;
  }
  last_its = its;
}

int64_t stdd_ctx::device_bytes() const {
  const DBuf *all[] = {&d_eps, &d_cxm, &d_cxp, &d_cym, &d_cyp, &d_strips, &d_fronts, &d_nodes, &d_cmap,
                       &d_inv, &d_lcxm, &d_lcxp, &d_colstrip, &d_lcym, &d_lcyp, &d_rowbox, &d_fac, &d_ws[0], &d_ws[1], &d_ub[0],
                       &d_ub[1], &d_tloc, &d_wloc, &d_items, &d_flag, &d_minpiv, &d_b, &d_x, &d_r, &d_V, &d_Z, &d_w,
                       &d_part, &d_h, &d_nrm, &d_y, &d_pre, &d_fpart, &d_guess, &d_gscr, &d_pcol, &d_panel,
                       &d_striplv, &d_bar, &d_sweep_flag, &d_lsx, &d_lsy, &d_segpart};
  int64_t s = 0;
  for (auto *d : all) s += (int64_t)d->bytes;
  return s;
}

// ---------------------------------------------------------------- C ABI
void stdd_ctx::learned_guesses(double2 *X) {
  if (!learned) throw StateError("STDD_X0_LEARNED needs a network (stdd_set_learned_guess)");
  const int64_t n = N();
  d_guess.alloc((size_t)2 * nrhs * n * sizeof(double2));
  d_gscr.alloc((stdd::NN_PART + 8) * sizeof(double));
  double *scr = d_gscr.as<double>();
  double2 *R = d_guess.as<double2>(), *Zs = R + (int64_t)nrhs * n;
  std::vector<double> bnorm(nrhs), raw(nrhs);
  std::vector<const double2 *> vs;
  std::vector<double2 *> zs;
  for (int q = 0; q < nrhs; ++q) {
    const double2 *b = d_b.as<double2>() + (int64_t)q * n;
    double2 *x = X + (int64_t)q * n, *r = R + (int64_t)q * n;
    // network field y, then its residual r = b - A y
    stdd::nn_guess_field(learned, d_eps.as<double>(), b, nx, ny, dx * dy, x, scr, stream);
    stdd::launch_residual(grid(), b, x, r, stream);
    bnorm[q] = dev_norm(const_cast<double2 *>(b), n, d_part, d_nrm, stream);
    raw[q] = bnorm[q] > 0 ? dev_norm(r, n, d_part, d_nrm, stream) / bnorm[q] : 0.0;
    vs.push_back(r);
    zs.push_back(Zs + (int64_t)q * n);
  }
  // one sweep of the method from y: x0 = y + M^-1 (b - A y), all right-hand
  // sides in one preconditioner application
  apply_minv_multi(vs, zs);
  for (int q = 0; q < nrhs; ++q) {
    const double2 *b = d_b.as<double2>() + (int64_t)q * n;
    double2 *x = X + (int64_t)q * n, *Ax = R + (int64_t)q * n;
    stdd::nn_zadd(zs[q], x, n, stream);
    stdd::launch_stencil(grid(), x, Ax, stream);
    stdd::nn_fit(Ax, b, n, scr, scr + stdd::NN_PART + 4, stream);
    double h[4];
    CK(cudaMemcpyAsync(h, scr + stdd::NN_PART + 4, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    // with alpha = (A x0)^H b / |A x0|^2, ||b - alpha A x0||^2 = |b|^2 - |(A x0)^H b|^2 / |A x0|^2
    const double bb = h[3], aa = h[2], dr = h[0], di = h[1];
    double scaled = 1;
    bool use = false;
    if (bb > 0 && aa > 0 && std::isfinite(aa) && std::isfinite(dr) && std::isfinite(di)) {
      scaled = std::sqrt(std::max(0.0, 1.0 - (dr * dr + di * di) / (aa * bb)));
      use = scaled < 1.0 - 1e-12;
    }
    lg_raw[q] = raw[q];
    lg_scaled[q] = use ? scaled : 1.0;
    lg_used[q] = use ? 1 : 0;
    if (use) stdd::nn_zscale(x, n, dr / aa, di / aa, stream);
    else CK(cudaMemsetAsync(x, 0, n * sizeof(double2), stream));
  }
}

namespace {

template <typename F> stdd_status guarded(stdd_ctx *c, F &&f) {
  if (!c) return STDD_EINVAL;
  try {
    CK(cudaSetDevice(c->device));
    f();
    c->err.clear();
    return STDD_OK;
  } catch (const ArgError &e) {
    c->err = e.what();
    return STDD_EINVAL;
  } catch (const std::invalid_argument &e) {
    c->err = e.what();
    return STDD_EINVAL;
  } catch (const StateError &e) {
    c->err = e.what();
    return STDD_ESTATE;
  } catch (const CudaError &e) {
    c->err = e.what();
    return STDD_ECUDA;
  } catch (const TimeoutError &e) {
    c->err = e.what();
    return STDD_ETIMEOUT;
  } catch (const std::bad_alloc &) {
    c->err = "out of device or host memory";
    return STDD_ENOMEM;
  } catch (const std::domain_error &e) {
    c->err = e.what();
    return STDD_EPIVOT;
  } catch (const std::range_error &e) {
    c->err = e.what();
    return STDD_EBREAKDOWN;
  } catch (const std::exception &e) {
    c->err = e.what();
    return STDD_EINVAL;
  } catch (...) {
    c->err = "unknown error";
    return STDD_EINVAL;
  }
}

void copy_in(void *dst, const void *src, size_t bytes, int is_device, cudaStream_t st) {
  CK(cudaMemcpyAsync(dst, src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
}
void copy_out(void *dst, const void *src, size_t bytes, int is_device, cudaStream_t st) {
  CK(cudaMemcpyAsync(dst, src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

}  // namespace

extern "C" {

stdd_status stdd_create(stdd_ctx **out, int device, void *cuda_stream) {
  if (!out) return STDD_EINVAL;
  *out = nullptr;
  stdd_ctx *c = new (std::nothrow) stdd_ctx();
  if (!c) return STDD_ENOMEM;
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete c;
    return STDD_ECUDA;
  }
  if (cuda_stream) {
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      delete c;
      return STDD_ECUDA;
    }
    c->own_stream = true;
  }
  *out = c;
  return STDD_OK;
}

void stdd_destroy(stdd_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

stdd_status stdd_set_grid(stdd_ctx *c, int nx, int ny, double dx, double dy) {
  return guarded(c, [&] {
    if (nx < 1 || ny < 1 || !(dx > 0) || !(dy > 0)) throw ArgError("bad grid");
    if ((int64_t)nx * ny > (int64_t)1 << 31) throw ArgError("grid too large");
    c->nx = nx;
    c->ny = ny;
    c->dx = dx;
    c->dy = dy;
    c->have_eps = false;
    c->nrhs = 0;
    c->nsub = 0;
    c->nsx = 0;
    c->nsy = 1;
    c->cuts.clear();
    c->ycuts.clear();
    c->shapes.clear();
    c->invalidate_operator();
  });
}

stdd_status stdd_set_permittivity(stdd_ctx *c, const double *eps, int is_device) {
  return guarded(c, [&] {
    if (c->nx <= 0) throw StateError("grid not set");
    if (!eps) throw ArgError("null permittivity");
    c->d_eps.alloc(c->N() * sizeof(double));
    copy_in(c->d_eps.p, eps, c->N() * sizeof(double), is_device, c->stream);
    CK(cudaStreamSynchronize(c->stream));
    c->have_eps = true;
    c->invalidate_factors();
  });
}

stdd_status stdd_set_frequency(stdd_ctx *c, double wavelength) {
  return guarded(c, [&] {
    if (!(wavelength > 0) || !std::isfinite(wavelength)) throw ArgError("bad wavelength");
    c->wavelength = wavelength;
    c->invalidate_operator();
  });
}

stdd_status stdd_set_pml(stdd_ctx *c, const int npml[4], int order_m, double R0) {
  return guarded(c, [&] {
    if (c->nx <= 0) throw StateError("grid not set");
    if (!npml || order_m < 0 || !(R0 > 0 && R0 < 1)) throw ArgError("bad PML parameters");
    for (int s = 0; s < 4; ++s)
      if (npml[s] < 0) throw ArgError("negative PML width");
    if (npml[0] + npml[1] > c->nx || npml[2] + npml[3] > c->ny) throw ArgError("PML wider than the grid");
    std::memcpy(c->npml, npml, sizeof(c->npml));
    c->pml_m = order_m;
    c->pml_R = R0;
    c->have_pml = true;
    c->invalidate_operator();
  });
}

stdd_status stdd_set_decomposition(stdd_ctx *c, int nsub, const int *x_cuts, int overlap, int ipml) {
  return guarded(c, [&] {
    if (c->nx <= 0) throw StateError("grid not set");
    if (nsub < 1 || nsub > c->nx || overlap < 0 || ipml < 0) throw ArgError("bad decomposition");
    std::vector<int> cuts;
    if (x_cuts) {
      cuts.assign(x_cuts, x_cuts + nsub + 1);
      if (cuts.front() != 0 || cuts.back() != c->nx) throw ArgError("cuts must run from 0 to nx");
      for (int k = 0; k < nsub; ++k)
        if (cuts[k + 1] <= cuts[k]) throw ArgError("cuts must increase");
    }
    if (nsub > c->nx) throw ArgError("bad decomposition");
    c->set_boxes(nsub, cuts, 1, {}, overlap, ipml);
  });
}

stdd_status stdd_set_decomposition_2d(stdd_ctx *c, int px, const int *x_cuts, int py, const int *y_cuts, int overlap,
                                      int ipml) {
  return guarded(c, [&] {
    if (c->nx <= 0) throw StateError("grid not set");
    if (px < 1 || px > c->nx || py < 1 || py > c->ny || overlap < 0 || ipml < 0)
      throw ArgError("bad decomposition");
    auto take = [](const int *cu, int parts, int n, std::vector<int> &out) {
      if (!cu) return;
      out.assign(cu, cu + parts + 1);
      if (out.front() != 0 || out.back() != n) throw ArgError("cuts must run from 0 to the grid size");
      for (int k = 0; k < parts; ++k)
        if (out[k + 1] <= out[k]) throw ArgError("cuts must increase");
    };
    std::vector<int> xc, yc;
    take(x_cuts, px, c->nx, xc);
    take(y_cuts, py, c->ny, yc);
    c->set_boxes(px, xc, py, yc, overlap, ipml);
  });
}

stdd_status stdd_box_info(const stdd_ctx *cc, int k, int out[8]) {
  stdd_ctx *c = const_cast<stdd_ctx *>(cc);
  return guarded(c, [&] {
    if (!out) throw ArgError("null output");
    if (c->strips.empty()) c->build_strips();
    if (k < 0 || k >= (int)c->strips.size()) throw ArgError("bad box");
    const StripHost &s = c->strips[k];
    const int v[8] = {s.c0, s.c1, s.r0, s.r1, s.x0, s.x1, s.y0, s.y1};
    std::memcpy(out, v, sizeof v);
  });
}

stdd_status stdd_set_precision(stdd_ctx *c, int mode) {
  return guarded(c, [&] {
    if (mode < STDD_PREC_FP64 || mode > STDD_PREC_C64_FP16) throw ArgError("unknown precision mode");
    if (mode != c->prec) {
      c->prec = mode;
      c->solve_nrhs_cap = 0;
      c->invalidate_factors();
    }
  });
}

stdd_status stdd_set_sources(stdd_ctx *c, int nrhs, const double *b, int is_device) {
  return guarded(c, [&] {
    if (c->nx <= 0) throw StateError("grid not set");
    if (nrhs < 1 || !b) throw ArgError("bad sources");
    const size_t bytes = (size_t)nrhs * c->N() * sizeof(double2);
    c->d_b.alloc(bytes);
    copy_in(c->d_b.p, b, bytes, is_device, c->stream);
    CK(cudaStreamSynchronize(c->stream));
    c->nrhs = nrhs;
  });
}

stdd_status stdd_factor(stdd_ctx *c) {
  return guarded(c, [&] { c->factor(); });
}

stdd_status stdd_solve(stdd_ctx *c, const stdd_solve_opts *o, double *x_out, int is_device) {
  bool noconv = false;
  stdd_status st = guarded(c, [&] {
    if (!o || !x_out) throw ArgError("null argument");
    if (!c->factored) throw StateError("stdd_factor has not run since the last configuration change");
    if (c->nrhs < 1) throw StateError("no sources set");
    if (o->restart < 1 || o->restart > 500 || o->maxit < 0 || !(o->rtol >= 0)) throw ArgError("bad solve options");
    if (o->x0_mode == STDD_X0_USER && !o->x0) throw ArgError("x0 missing");
    if (o->x0_mode < STDD_X0_ZERO || o->x0_mode > STDD_X0_LEARNED) throw ArgError("bad x0_mode");
    if (c->use_band && !o->paper_richardson && (c->prec != STDD_PREC_FP64 || c->order != 0))
      throw ArgError("band-space FGMRES needs FP64 factors and the additive order");
    if (c->use_band && !o->paper_richardson) c->require_strips("band-space FGMRES");
    if (o->paper_richardson) c->require_strips("the paper's Richardson mode (Eq. 20 stopping test)");
    if (c->order != 0) c->require_strips("the multiplicative and red-black orders");
    const int64_t n = c->N();
    c->history.assign(c->nrhs, {});
    c->lg_raw.assign(c->nrhs, 0.0);
    c->lg_scaled.assign(c->nrhs, 1.0);
    c->lg_used.assign(c->nrhs, 0);
    c->ensure_krylov(o->paper_richardson ? 1 : o->restart);
    const int span = c->pbegin(stdd_ctx::PH_SOLVE);
    double2 *X = c->d_x.as<double2>();
    if (o->x0_mode == STDD_X0_LEARNED) {
      c->learned_guesses(X);
    } else {
      for (int q = 0; q < c->nrhs; ++q) {
        if (o->x0_mode == STDD_X0_USER)
          copy_in(X + (int64_t)q * n, o->x0 + (size_t)q * n * 2, n * sizeof(double2), o->x0_is_device, c->stream);
        else
          CK(cudaMemsetAsync(X + (int64_t)q * n, 0, n * sizeof(double2), c->stream));
      }
    }
    if (o->paper_richardson) {
      for (int q = 0; q < c->nrhs; ++q) c->richardson(q, *o, X + (int64_t)q * n);
    } else {
      c->gmres_multi(*o);
      noconv = c->last_noconv;
    }
    c->pend(span);
    c->poll_sweep_flag();
    copy_out(x_out, X, (size_t)c->nrhs * n * sizeof(double2), is_device, c->stream);
    c->raise_sweep_flag();
  });
  if (st == STDD_OK && noconv) {
    c->err = "maxit reached before rtol";
    return STDD_ENOCONV;
  }
  return st;
}

stdd_status stdd_residual_history(stdd_ctx *c, int rhs, double *out, int cap, int *n_out) {
  return guarded(c, [&] {
    if (rhs < 0 || rhs >= (int)c->history.size()) throw ArgError("no history for that right-hand side");
    const auto &h = c->history[rhs];
    if (n_out) *n_out = (int)h.size();
    if (out)
      for (int i = 0; i < cap && i < (int)h.size(); ++i) out[i] = h[i];
  });
}

const char *stdd_last_error(const stdd_ctx *c) { return c ? c->err.c_str() : "null context"; }

stdd_status stdd_apply_operator(stdd_ctx *c, const double *x, double *y, int is_device) {
  return guarded(c, [&] {
    if (!x || !y) throw ArgError("null vector");
    c->require_operator();
    const int64_t n = c->N();
    c->d_w.alloc(n * sizeof(double2));
    c->d_r.alloc(n * sizeof(double2));
    copy_in(c->d_w.p, x, n * sizeof(double2), is_device, c->stream);
    stdd::launch_stencil(c->grid(), c->d_w.as<double2>(), c->d_r.as<double2>(), c->stream);
    CK(cudaGetLastError());
    copy_out(y, c->d_r.p, n * sizeof(double2), is_device, c->stream);
  });
}

stdd_status stdd_apply_preconditioner(stdd_ctx *c, const double *v, double *z, int is_device) {
  return guarded(c, [&] {
    if (!v || !z) throw ArgError("null vector");
    if (!c->factored) throw StateError("not factored");
    const int64_t n = c->N();
    c->d_w.alloc(n * sizeof(double2));
    c->d_r.alloc(n * sizeof(double2));
    copy_in(c->d_w.p, v, n * sizeof(double2), is_device, c->stream);
    c->apply_minv(c->d_w.as<double2>(), c->d_r.as<double2>());
    c->poll_sweep_flag();
    copy_out(z, c->d_r.p, n * sizeof(double2), is_device, c->stream);
    c->raise_sweep_flag();
  });
}

stdd_status stdd_local_solve(stdd_ctx *c, int k, const double *t, double *z, int is_device) {
  return guarded(c, [&] {
    if (!t || !z) throw ArgError("null vector");
    if (!c->factored) throw StateError("not factored");
    if (k < 0 || k >= c->nsub) throw ArgError("bad strip");
    const int64_t nl = (int64_t)c->strips[k].W() * c->strips[k].H();
    int64_t off = 0;
    for (int kk = 0; kk < k; ++kk) off += (int64_t)c->strips[kk].W() * c->strips[kk].H();
    c->ensure_solve_buffers(1);
    c->d_w.alloc(nl * sizeof(double2));
    copy_in(c->d_w.p, t, nl * sizeof(double2), is_device, c->stream);
    const size_t E = c->elem();
    CK(cudaMemsetAsync(c->d_tloc.p, 0, c->nloc * E, c->stream));
    char *base = c->d_tloc.as<char>() + off * E;
    if (c->prec == STDD_PREC_FP64) {
      stdd::launch_to_local<double>(c->d_w.as<double2>(), base, nl, c->stream);
      c->solve_levels<double>(1);
      stdd::launch_from_local<double>(base, c->d_w.as<double2>(), nl, c->stream);
    } else {
      stdd::launch_to_local<float>(c->d_w.as<double2>(), base, nl, c->stream);
      c->solve_levels<float>(1);
      stdd::launch_from_local<float>(base, c->d_w.as<double2>(), nl, c->stream);
    }
    CK(cudaGetLastError());
    copy_out(z, c->d_w.p, nl * sizeof(double2), is_device, c->stream);
  });
}

stdd_status stdd_strip_info(const stdd_ctx *cc, int k, int *c0, int *c1, int *x0, int *x1) {
  stdd_ctx *c = const_cast<stdd_ctx *>(cc);
  return guarded(c, [&] {
    if (c->strips.empty()) c->build_strips();
    if (k < 0 || k >= (int)c->strips.size()) throw ArgError("bad strip");
    const StripHost &s = c->strips[k];
    if (c0) *c0 = s.c0;
    if (c1) *c1 = s.c1;
    if (x0) *x0 = s.x0;
    if (x1) *x1 = s.x1;
  });
}

stdd_status stdd_get_stats(stdd_ctx *c, stdd_stats *o) {
  return guarded(c, [&] {
    if (!o) throw ArgError("null stats");
    std::memset(o, 0, sizeof(*o));
    o->nfronts = c->nfronts;
    o->depth = c->depth;
    o->max_pivots = c->max_p;
    o->max_border = c->max_b;
    o->factor_entries = c->factor_entries;
    o->factor_flops = 8.0 * c->factor_cflops;
    o->factor_flops_lu = 8.0 * c->factor_cflops_lu;
    o->solve_flops = 8.0 * c->solve_cflops;
    o->local_dofs = c->nloc;
    o->device_bytes = c->device_bytes();
    o->iterations = c->last_its;
    o->final_residual = c->last_res;
    o->min_pivot = c->min_pivot;
    o->reorth_passes = c->last_reorth;
    o->raised_pivots = c->raised_pivots;
  });
}

stdd_status stdd_residual(stdd_ctx *c, const double *x, const double *b, double *r, double *rel_out,
                          int is_device) {
  return guarded(c, [&] {
    if (!x || !b || !r || !rel_out) throw ArgError("null argument");
    c->require_operator();
    const int64_t n = c->N();
    c->d_w.alloc(n * sizeof(double2));
    c->d_r.alloc(n * sizeof(double2));
    c->d_x.alloc(n * sizeof(double2));
    c->d_part.alloc((size_t)stdd::krylov_partial_blocks() * sizeof(double2));
    c->d_nrm.alloc(4 * sizeof(double));
    copy_in(c->d_w.p, x, n * sizeof(double2), is_device, c->stream);
    copy_in(c->d_x.p, b, n * sizeof(double2), is_device, c->stream);
    stdd::launch_residual(c->grid(), c->d_x.as<double2>(), c->d_w.as<double2>(), c->d_r.as<double2>(), c->stream);
    const double rn = dev_norm(c->d_r.as<double2>(), n, c->d_part, c->d_nrm, c->stream);
    const double bn = dev_norm(c->d_x.as<double2>(), n, c->d_part, c->d_nrm, c->stream);
    *rel_out = bn > 0 ? rn / bn : rn;
    copy_out(r, c->d_r.p, n * sizeof(double2), is_device, c->stream);
  });
}

stdd_status stdd_set_profiling(stdd_ctx *c, int level) {
  return guarded(c, [&] {
    if (level < 0 || level > 2) throw ArgError("profiling level must be 0, 1 or 2");
    c->prof = level;
  });
}

stdd_status stdd_set_option(stdd_ctx *c, int option, int value) {
  return guarded(c, [&] {
    switch (option) {
      case STDD_OPT_GRAPHS:
        c->use_graphs = value != 0;
        if (!c->use_graphs) c->clear_graphs();
        break;
      case STDD_OPT_AUTOTUNE:
        c->autotune_on = value != 0;
        break;
      case STDD_OPT_ORDER:
        if (value < 0 || value > 3)
          throw ArgError("order must be 0 (additive), 1 (symmetric multiplicative), 2 (red-black) or 3 (forward "
                         "multiplicative)");
        if (value != c->order) {
          c->order = value;
          c->clear_graphs();
        }
        break;
      case STDD_OPT_BAND:
        c->use_band = value != 0;
        break;
      case STDD_OPT_UPDATE_TILE:
        if (value != 0 && value != 32 && value != 64) throw ArgError("update tile must be 0 (tuned), 32 or 64");
        c->forced_tile = value;
        c->invalidate_factors();
        break;
      case STDD_OPT_PERSISTENT:
        if (value < -1 || value > 8)
          throw ArgError("persistent must be -1 (by precision), 0 (off) or 1..8 blocks per SM");
        if (value != c->persistent) {
          c->persistent = value;
          c->clear_graphs();
        }
        break;
      case STDD_OPT_SWEEP_WAIT:
        if (value < 0) throw ArgError("wait limit must be >= 0 (0: the default)");
        c->sweep_wait = value == 0 ? (1ll << 22) : (long long)value;
        c->clear_graphs();
        break;
      case STDD_OPT_PIVOTING:
        if (value < 0 || value > 1) throw ArgError("pivoting must be 0 (off) or 1 (partial, within fronts)");
        if (value != c->pivoting) {
          c->pivoting = value;
          c->invalidate_factors();
          c->clear_graphs();
        }
        break;
      case STDD_OPT_SYMMETRIC:
        if (value < 0 || value > 2)
          throw ArgError("symmetric must be 0 (off), 1 (complex128 factors) or 2 (complex64 factors too)");
        if (value != c->symmetric) {
          c->symmetric = value;
          c->invalidate_factors();
          c->clear_graphs();
        }
        break;
      case STDD_OPT_SWEEP_SPLIT:
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != stdd::MF_SPLIT_GRID)
          throw ArgError("sweep split must be 0 (tuned), 1, 2, 4, 8 or 16 (across the grid)");
        c->forced_split = value;
        c->invalidate_factors();
        c->clear_graphs();
        break;
      case STDD_OPT_FP64_TC:
        if (value < 0 || value > 1) throw ArgError("fp64 tensor-core updates must be 0 (off) or 1 (on)");
        if (value != c->fp64_tc) {
          c->fp64_tc = value;
          c->invalidate_factors();
          c->clear_graphs();
        }
        break;
      case STDD_OPT_STATIC_PIVOT:
        if (value < 0 || value > 15) throw ArgError("static pivot exponent must be 0 .. 15");
        if (value != c->static_pivot) {
          c->static_pivot = value;
          c->invalidate_factors();
        }
        break;
      case STDD_OPT_LEAF:
        if (value < 1 || value > 4096) throw ArgError("leaf size out of range");
        if (value != c->leaf_max) {
          c->leaf_max = value;
          c->shapes.clear();
          c->struct_ready = false;
          c->invalidate_factors();
        }
        break;
      default:
        throw ArgError("unknown option");
    }
  });
}

stdd_status stdd_get_profile(stdd_ctx *c, stdd_profile *o, int reset) {
  return guarded(c, [&] {
    if (!o) throw ArgError("null profile");
    std::memset(o, 0, sizeof(*o));
    CK(cudaStreamSynchronize(c->stream));
    double t[stdd_ctx::PH_COUNT] = {0}, units[stdd_ctx::PH_COUNT] = {0}, execu[stdd_ctx::PH_COUNT] = {0};
    int cnt[stdd_ctx::PH_COUNT] = {0};
    c->span_units.resize(c->spans.size(), 0.0);
    c->span_exec.resize(c->spans.size(), 0.0);
    for (size_t si = 0; si < c->spans.size(); ++si) {
      const auto &sp = c->spans[si];
      float ms = 0;
      if (cudaEventElapsedTime(&ms, sp.a, sp.b) != cudaSuccess) {  // span left open by a failed call
        (void)cudaGetLastError();
        continue;
      }
      t[sp.phase] += ms;
      cnt[sp.phase] += 1;
      units[sp.phase] += c->span_units[si];
      execu[sp.phase] += c->span_exec[si];
    }
    const int K0 = stdd_ctx::PH_K0;
    if (std::getenv("STDD_PROFILE_LEVELS")) {   // per-level breakdown on stderr
      c->span_level.resize(c->spans.size(), -1);
      std::map<std::pair<int, int>, std::pair<double, double>> lv;
      for (size_t si = 0; si < c->spans.size(); ++si) {
        if (c->span_level[si] < 0) continue;
        float ms = 0;
        if (cudaEventElapsedTime(&ms, c->spans[si].a, c->spans[si].b) != cudaSuccess) {
          (void)cudaGetLastError();
          continue;
        }
        auto &e = lv[{c->spans[si].phase - K0, c->span_level[si]}];
        e.first += ms;
        e.second += c->span_units[si];
      }
      static const char *names[] = {"small", "update", "up", "down", "sweep"};
      for (auto &kv : lv)
        std::fprintf(stderr, "level-profile %s L%d ms %.3f units %.4g rate %.4g\n", names[kv.first.first],
                     kv.first.second, kv.second.first, kv.second.second,
                     kv.second.second / (kv.second.first * 1e-3));
    }
    o->small_ms = t[K0 + stdd::K_SMALL];
    o->small_flops = units[K0 + stdd::K_SMALL];
    o->small_calls = cnt[K0 + stdd::K_SMALL];
    o->update_ms = t[K0 + stdd::K_UPDATE];
    o->update_flops = units[K0 + stdd::K_UPDATE];
    o->update_calls = cnt[K0 + stdd::K_UPDATE];
    o->up_ms = t[K0 + stdd::K_UP];
    o->up_bytes = units[K0 + stdd::K_UP];
    o->up_calls = cnt[K0 + stdd::K_UP];
    o->down_ms = t[K0 + stdd::K_DOWN];
    o->down_bytes = units[K0 + stdd::K_DOWN];
    o->down_calls = cnt[K0 + stdd::K_DOWN];
    o->sweep_ms = t[K0 + stdd::K_SWEEP];
    o->sweep_bytes = units[K0 + stdd::K_SWEEP];
    o->sweep_calls = cnt[K0 + stdd::K_SWEEP];
    o->small_flops_executed = execu[K0 + stdd::K_SMALL];
    o->update_flops_executed = execu[K0 + stdd::K_UPDATE];
    o->factor_ms = t[stdd_ctx::PH_FACTOR];
    o->minv_ms = t[stdd_ctx::PH_MINV];
    o->minv_calls = cnt[stdd_ctx::PH_MINV];
    o->matvec_ms = t[stdd_ctx::PH_MATVEC];
    o->matvec_calls = cnt[stdd_ctx::PH_MATVEC];
    o->ortho_ms = t[stdd_ctx::PH_ORTHO];
    o->ortho_calls = cnt[stdd_ctx::PH_ORTHO];
    o->solve_ms = t[stdd_ctx::PH_SOLVE];
    o->launches = __atomic_load_n(&stdd::g_launches, __ATOMIC_RELAXED);
    if (reset) {
      c->spans.clear();
      c->span_units.clear();
      c->span_exec.clear();
      c->span_level.clear();
      c->ev_used = 0;
    }
  });
}

stdd_status stdd_set_learned_guess(stdd_ctx *c, stdd_nn *nn) {
  return guarded(c, [&] {
    if (nn && stdd::nn_device(nn) != c->device) throw ArgError("network lives on another device");
    c->learned = nn;
  });
}

stdd_status stdd_learned_guess_info(stdd_ctx *c, int rhs, double *raw_rel, double *scaled_rel, int *used) {
  return guarded(c, [&] {
    if (rhs < 0 || rhs >= (int)c->lg_used.size()) throw ArgError("no guess recorded for that right-hand side");
    if (raw_rel) *raw_rel = c->lg_raw[rhs];
    if (scaled_rel) *scaled_rel = c->lg_scaled[rhs];
    if (used) *used = c->lg_used[rhs];
  });
}

stdd_status stdd_tc_tile_product(int device, int fmt, int kc, const double *C, const double *R, double *D) {
  if (!C || !R || !D || (fmt != 0 && fmt != 1) || kc < 1 || kc > stdd::MF_NB) return STDD_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) {
    (void)cudaGetLastError();
    return STDD_ECUDA;
  }
  std::vector<float2> c((size_t)64 * kc), r((size_t)kc * 128), d((size_t)64 * 128);
  for (size_t i = 0; i < c.size(); ++i) c[i] = make_float2((float)C[2 * i], (float)C[2 * i + 1]);
  for (size_t i = 0; i < r.size(); ++i) r[i] = make_float2((float)R[2 * i], (float)R[2 * i + 1]);
  cudaError_t e = cudaSuccess;
  const int st = stdd::tc_tile_product(fmt, kc, c.data(), r.data(), d.data(), &e);
  if (st < 0) {
    (void)cudaGetLastError();
    return STDD_ECUDA;
  }
  if (st == 1) return STDD_ETIMEOUT;
  for (size_t i = 0; i < d.size(); ++i) {
    D[2 * i] = d[i].x;
    D[2 * i + 1] = d[i].y;
  }
  return STDD_OK;
}

stdd_status stdd_tc_f64_tile_product(int device, int kc, const double *C, const double *R, double *D) {
  if (!C || !R || !D || kc < 1 || kc > stdd::MF_NB) return STDD_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) {
    (void)cudaGetLastError();
    return STDD_ECUDA;
  }
  cudaError_t e = cudaSuccess;
  const int st = stdd::oz_tile_product(kc, reinterpret_cast<const double2 *>(C),
                                       reinterpret_cast<const double2 *>(R), reinterpret_cast<double2 *>(D), &e);
  if (st < 0) {
    (void)cudaGetLastError();
    return STDD_ECUDA;
  }
  if (st == 1) return STDD_ETIMEOUT;
  if (st == 2) return STDD_EINVAL;
  return STDD_OK;
}

stdd_status stdd_nd_analyze(int W, int H, int leaf_max, int *nfronts, long long *nnodes, int *p, int *b,
                            int *parent, int *level, int *nodes) {
  try {
    Shape S;
    stdd::nd_analyze(W, H, leaf_max, S);
    if (nfronts) *nfronts = (int)S.fronts.size();
    if (nnodes) *nnodes = (long long)S.nodes.size();
    if (nodes) {
      for (size_t f = 0; f < S.fronts.size(); ++f) {
        if (p) p[f] = S.fronts[f].p;
        if (b) b[f] = S.fronts[f].b;
        if (parent) parent[f] = S.fronts[f].parent;
        if (level) level[f] = S.fronts[f].level;
      }
      std::memcpy(nodes, S.nodes.data(), S.nodes.size() * sizeof(int));
    }
    return STDD_OK;
  } catch (const std::invalid_argument &) {
    return STDD_EINVAL;
  } catch (const std::bad_alloc &) {
    return STDD_ENOMEM;
  } catch (...) {
    return STDD_EINVAL;
  }
}

}  // extern "C"

// ------------------------------------------------------------------------
// Residual without device allocation.
//
// stdd_residual stages its inputs in context buffers and reduces through
// context scratch that it grows with cudaMalloc on first use.  Callers that
// must not allocate device memory at call time -- real-time loops that
// reserve all of their memory before they start, or hosts that hand out GPU
// memory only through their own pool -- use stdd_residual_noalloc instead:
// it reads and writes only the caller's device buffers and a fixed scratch
// array compiled into this library (g_noalloc_scratch, ~256 KiB), which
// every GPU that loads the library keeps until the process exits.
// ------------------------------------------------------------------------
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CHUNK = 4096;            // grid nodes reduced by one block
constexpr int NA_MAX_BLOCKS = 16384;      // so at most NA_CHUNK * NA_MAX_BLOCKS nodes
constexpr int64_t NA_MAX_NODES = (int64_t)NA_CHUNK * NA_MAX_BLOCKS;  // 67,108,864

// [2 * NA_MAX_BLOCKS] per-block (||r||^2, ||b||^2), then the two totals.
static __device__ __align__(256) double g_noalloc_scratch[2 * NA_MAX_BLOCKS + 2];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double *g_na_ptr[NA_MAX_DEVICES] = {nullptr};

// device address of g_noalloc_scratch on the current device (looked up once)
cudaError_t na_scratch(int device, double **out) {
  if (device < 0 || device >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[device] = static_cast<double *>(p);
  }
  *out = g_na_ptr[device];
  return cudaSuccess;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_residual(stdd::GridDev g, const double2 *__restrict__ b,
                                                            const double2 *__restrict__ x,
                                                            double2 *__restrict__ r, double *scratch) {
  const int64_t n = (int64_t)g.nx * g.ny;
  const int64_t g0 = (int64_t)blockIdx.x * NA_CHUNK, g1 = min(n, g0 + NA_CHUNK);
  double rr = 0, bb = 0;
  for (int64_t idx = g0 + threadIdx.x; idx < g1; idx += NA_THREADS) {
    const int i = (int)(idx / g.ny), j = (int)(idx - (int64_t)i * g.ny);
    const double2 xm = g.cxm[i], xp = g.cxp[i], ym = g.cym[j], yp = g.cyp[j];
    double2 d;
    d.x = g.k0sq * g.eps[idx] - xm.x - xp.x - ym.x - yp.x;
    d.y = -xm.y - xp.y - ym.y - yp.y;
    double2 ax = stdd::cmul(d, x[idx]);
    if (i > 0) ax = stdd::cfma(xm, x[idx - g.ny], ax);
    if (i < g.nx - 1) ax = stdd::cfma(xp, x[idx + g.ny], ax);
    if (j > 0) ax = stdd::cfma(ym, x[idx - 1], ax);
    if (j < g.ny - 1) ax = stdd::cfma(yp, x[idx + 1], ax);
    const double2 bv = b[idx];
    const double2 rv = stdd::csub(bv, ax);
    r[idx] = rv;
    rr = fma(rv.x, rv.x, fma(rv.y, rv.y, rr));
    bb = fma(bv.x, bv.x, fma(bv.y, bv.y, bb));
  }
  __shared__ double sh[2][NA_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = rr;
    sh[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0, sb = 0;
    for (int w = 0; w < NA_THREADS / 32; ++w) {
      sr += sh[0][w];
      sb += sh[1][w];
    }
    scratch[2 * blockIdx.x] = sr;       // every slot read below is written here first
    scratch[2 * blockIdx.x + 1] = sb;
  }
}

// fixed-order sum of the per-block partials into the two total slots
__global__ void k_na_finish(int nblk, double *scratch) {
  const int lane = threadIdx.x;
  double sr = 0, sb = 0;
  for (int k = lane; k < nblk; k += 32) {
    sr += scratch[2 * k];
    sb += scratch[2 * k + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if (lane == 0) {
    scratch[2 * NA_MAX_BLOCKS] = sr;
    scratch[2 * NA_MAX_BLOCKS + 1] = sb;
  }
}

}  // namespace

extern "C" stdd_status stdd_residual_noalloc(stdd_ctx *c, const double *x, const double *b, double *r,
                                             double *rel_out) {
  if (!c) return STDD_EINVAL;
  if (!x || !b || !r || !rel_out) {
    c->err = "stdd_residual_noalloc: null argument";
    return STDD_EINVAL;
  }
  const int64_t n = c->N();
  if (n > NA_MAX_NODES) {
    c->err = "stdd_residual_noalloc: grid has more than 67,108,864 nodes, the size of its fixed scratch";
    return STDD_EINVAL;
  }
  {
    // r is written while other threads still read x's neighbours: it must
    // not overlap x; r == b is safe (b[idx] is read before r[idx] is
    // written by the same thread), a partial overlap with b is not
    const uintptr_t bytes = (uintptr_t)n * 2 * sizeof(double);
    const uintptr_t pr = (uintptr_t)r, px = (uintptr_t)x, pb = (uintptr_t)b;
    auto overlap = [&](uintptr_t a, uintptr_t o) { return a < o + bytes && o < a + bytes; };
    if (n > 0 && (overlap(pr, px) || (pr != pb && overlap(pr, pb)))) {
      c->err = "stdd_residual_noalloc: r must not overlap x, and may overlap b only as the same buffer";
      return STDD_EINVAL;
    }
  }
  if (!c->op_ready || !c->have_eps || n == 0) {
    c->err = "stdd_residual_noalloc: operator not set up (call stdd_apply_operator, stdd_residual or "
             "stdd_factor once after configuring the grid)";
    return STDD_ESTATE;
  }
  cudaError_t e = cudaSetDevice(c->device);
  double *scratch = nullptr;
  if (e == cudaSuccess) e = na_scratch(c->device, &scratch);
  if (e == cudaSuccess) {
    const int nblk = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
    k_na_residual<<<nblk, NA_THREADS, 0, c->stream>>>(c->grid(), reinterpret_cast<const double2 *>(b),
                                                    reinterpret_cast<const double2 *>(x),
                                                    reinterpret_cast<double2 *>(r), scratch);
    k_na_finish<<<1, 32, 0, c->stream>>>(nblk, scratch);
    stdd::count_launch(2);
    e = cudaGetLastError();
  }
  double tot[2] = {0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tot, scratch + 2 * NA_MAX_BLOCKS, sizeof(tot), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->err = std::string("stdd_residual_noalloc: ") + cudaGetErrorString(e);
    return STDD_ECUDA;
  }
  const double rn = std::sqrt(tot[0]), bn = std::sqrt(tot[1]);
  *rel_out = bn > 0 ? rn / bn : rn;
  c->err.clear();
  return STDD_OK;
}

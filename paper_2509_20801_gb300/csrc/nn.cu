// Learned initial guess: the convolutional encoder-decoder (host side).
//
// Layout of the network with L levels and channels c_l = min(c0 * 2^l, cmax):
//   encoder level l: A: conv3x3(in_l -> c_l) + ReLU, B: conv3x3(c_l -> c_l) + ReLU
//                    = skip_l; in_0 = the 3-channel input, in_l = avgpool2(skip_{l-1})
//   decoder level l = L-2 .. 0: C: conv3x3(up2(d_{l+1}): c_{l+1} -> c_l) + ReLU,
//                    add skip_l, D: conv3x3(c_l -> c_l) + ReLU = d_l (d_{L-1} = skip_{L-1})
//   output: conv3x3(d_0: c_0 -> 2), no activation.
// Parameters are stored layer by layer in that order (enc 0 A, B, enc 1 A,
// B, ..., dec L-2 C, D, ..., dec 0 C, D, out), each as weights
// [cout][cin][3][3] then bias [cout].  Forward and backward use the weights
// rounded to BF16 (or the FP32 weights, for exact-layout checks).
#include <cmath>
#include <cstring>
#include <map>
#include <random>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/stdd.h"
#include "common.cuh"
#include "kernels.h"


namespace {

struct NnError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

#define NCK(expr)                                                                                            \
  do {                                                                                                       \
    cudaError_t _e = (expr);                                                                                 \
    if (_e != cudaSuccess) throw NnError(std::string(#expr) + ": " + cudaGetErrorString(_e));               \
  } while (0)

struct DevF {
  float *p = nullptr;
  size_t n = 0;
  DevF() = default;
  DevF(const DevF &) = delete;
  DevF &operator=(const DevF &) = delete;
  ~DevF() {
    if (p) cudaFree(p);
  }
  void alloc(size_t count) {
    if (count == 0) throw std::invalid_argument("empty device buffer requested");
    if (count <= n && p) return;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    if (cudaMalloc(&p, std::max<size_t>(1, count) * sizeof(float)) != cudaSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
      throw std::bad_alloc();
    }
    n = count;
  }
};

struct Layer {
  int cin, cout;
  int64_t woff, boff;
};

bool g_tc_ready = false;

}  // namespace

struct stdd_nn {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int L = 0, c0 = 0, cmax = 0;
  int mode = STDD_NN_TC;
  bool bf16 = true;          // weights rounded to BF16 (modes 1 and 2)
  // tensor-core mode: per layer, packed BF16 weights of the forward and of
  // the input-gradient convolution
  std::vector<int64_t> pk_fwd, pk_bwd;
  uint16_t *packed = nullptr;
  int *d_flag = nullptr;
  std::vector<int> ch;
  std::vector<Layer> layers;  // enc A/B per level, dec C/D per level (L-2..0), out
  int64_t nparams = 0;
  DevF w, wb, g, m, v, loss;
  int step = 0;
  std::string err;
  // activations for one (N, H, W)
  int aN = 0, aH = 0, aW = 0;
  std::map<std::string, DevF> act;

  const Layer &encA(int l) const { return layers[2 * l]; }
  const Layer &encB(int l) const { return layers[2 * l + 1]; }
  const Layer &decC(int l) const { return layers[2 * L + 2 * (L - 2 - l)]; }
  const Layer &decD(int l) const { return layers[2 * L + 2 * (L - 2 - l) + 1]; }
  const Layer &outL() const { return layers.back(); }

  float *buf(const std::string &name, size_t count) {
    DevF &d = act[name];
    d.alloc(count);
    return d.p;
  }
  float *A(const std::string &k, int l) {
    auto it = act.find(k + std::to_string(l));
    if (it == act.end() || !it->second.p) throw std::logic_error("activation " + k + std::to_string(l) + " missing");
    return it->second.p;
  }
  size_t sz(int l, int c) const { return (size_t)aN * c * (aH >> l) * (aW >> l); }

  ~stdd_nn() {
    if (packed) cudaFree(packed);
    if (d_flag) cudaFree(d_flag);
  }

  void build(int levels, int base, int maxc, int use_mode, unsigned long long seed) {
    if (levels < 1 || levels > 8 || base < 1 || maxc < base) throw std::invalid_argument("bad network shape");
    if (use_mode < STDD_NN_FP32 || use_mode > STDD_NN_TC) throw std::invalid_argument("bad network mode");
    if (use_mode == STDD_NN_TC && maxc > 256) throw std::invalid_argument("tensor-core mode allows at most 256 channels");
    mode = use_mode;
    const bool use_bf16 = mode != STDD_NN_FP32;
    L = levels;
    c0 = base;
    cmax = maxc;
    bf16 = use_bf16;
    ch.clear();
    for (int l = 0; l < L; ++l) ch.push_back(std::min(cmax, c0 << l));
    layers.clear();
    int64_t off = 0;
    auto add = [&](int ci, int co) {
      Layer ly{ci, co, off, off + (int64_t)co * ci * 9};
      off += (int64_t)co * ci * 9 + co;
      layers.push_back(ly);
    };
    for (int l = 0; l < L; ++l) {
      add(l == 0 ? 3 : ch[l - 1], ch[l]);
      add(ch[l], ch[l]);
    }
    for (int l = L - 2; l >= 0; --l) {
      add(ch[l + 1], ch[l]);
      add(ch[l], ch[l]);
    }
    add(ch[0], 2);
    nparams = off;
    // He-normal weights (variance 2 / fan_in), zero biases; output layer x0.1
    std::vector<float> h((size_t)nparams, 0.f);
    std::mt19937_64 rng(seed);
    for (size_t li = 0; li < layers.size(); ++li) {
      const Layer &ly = layers[li];
      std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (9.0 * ly.cin)) * (li + 1 == layers.size() ? 0.1 : 1));
      for (int64_t i = 0; i < (int64_t)ly.cout * ly.cin * 9; ++i) h[ly.woff + i] = (float)nd(rng);
    }
    w.alloc(nparams);
    wb.alloc(nparams);
    g.alloc(nparams);
    m.alloc(nparams);
    v.alloc(nparams);
    loss.alloc(1);
    NCK(cudaMemcpyAsync(w.p, h.data(), nparams * sizeof(float), cudaMemcpyHostToDevice, stream));
    NCK(cudaMemsetAsync(m.p, 0, nparams * sizeof(float), stream));
    NCK(cudaMemsetAsync(v.p, 0, nparams * sizeof(float), stream));
    if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess) {
      (void)cudaGetLastError();
      throw std::bad_alloc();
    }
    NCK(cudaMemsetAsync(d_flag, 0, sizeof(int), stream));
    if (mode == STDD_NN_TC) {
      if (!g_tc_ready) {
        NCK(stdd::nn_tc_setup());
        g_tc_ready = true;
      }
      int64_t off = 0;
      for (const Layer &ly : layers) {
        pk_fwd.push_back(off);
        off += stdd::nn_tc_packed_elems(ly.cin, ly.cout);
        pk_bwd.push_back(off);
        off += stdd::nn_tc_packed_elems(ly.cout, ly.cin);
      }
      if (cudaMalloc(&packed, std::max<int64_t>(1, off) * sizeof(uint16_t)) != cudaSuccess) {
        (void)cudaGetLastError();
        throw std::bad_alloc();
      }
    }
    stdd::nn_round(w.p, wb.p, nparams, bf16, stream);
    repack();
    NCK(cudaStreamSynchronize(stream));
    step = 0;
  }

  // tensor-core operand copies of the current (BF16-rounded) weights
  void repack() {
    if (mode != STDD_NN_TC) return;
    for (size_t i = 0; i < layers.size(); ++i) {
      const Layer &ly = layers[i];
      stdd::nn_pack_weights(wb.p + ly.woff, ly.cin, ly.cout, false, packed + pk_fwd[i], stream);
      stdd::nn_pack_weights(wb.p + ly.woff, ly.cin, ly.cout, true, packed + pk_bwd[i], stream);
    }
  }

  size_t layer_index(const Layer &ly) const { return (size_t)(&ly - layers.data()); }

  // out = conv(in) with layer ly (forward) or its input gradient (flip)
  void conv(const float *in, const Layer &ly, float *out, int N, int H, int W, bool relu, bool flip,
            cudaStream_t st) {
    const int cin = flip ? ly.cout : ly.cin, cout = flip ? ly.cin : ly.cout;
    if (mode == STDD_NN_TC) {
      const size_t i = layer_index(ly);
      stdd::nn_conv_tc(in, cin, packed + (flip ? pk_bwd[i] : pk_fwd[i]), flip ? nullptr : wb.p + ly.boff, out, cout,
                       N, H, W, relu, d_flag, st, act["ksplit"].p);
    } else {
      stdd::nn_conv(in, cin, wb.p + ly.woff, flip ? nullptr : wb.p + ly.boff, out, cout, N, H, W, relu, flip, st);
    }
  }

  // throws if a tensor-core wait timed out since the last check (syncs st)
  // weight and bias gradient of one convolution (accumulated into gw, gb)
  void wgrad(const float *in, int cin, const float *gout, int cout, int N, int H, int W, float *gw, float *gb,
             cudaStream_t st) {
    if (mode == STDD_NN_TC)
      stdd::nn_conv_wgrad_tc(in, cin, gout, cout, N, H, W, gw, gb, d_flag, st);
    else
      stdd::nn_conv_wgrad(in, cin, gout, cout, N, H, W, gw, gb, st);
  }

  void check_flag(cudaStream_t st) {
    int f = 0;
    NCK(cudaMemcpyAsync(&f, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    NCK(cudaStreamSynchronize(st));
    if (f) {
      NCK(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
      throw NnError("tensor-core convolution timed out");
    }
  }

  void check_shape(int N, int H, int W) const {
    const int f = 1 << (L - 1);
    if (N < 1 || H < f || W < f || H % f || W % f) throw std::invalid_argument("image size must be a multiple of 2^(levels-1)");
  }

  void ensure_acts(int N, int H, int W) {
    if (N == aN && H == aH && W == aW) return;
    aN = N;
    aH = H;
    aW = W;
    for (int l = 0; l < L; ++l) {
      act["encA" + std::to_string(l)].alloc(sz(l, ch[l]));
      act["skip" + std::to_string(l)].alloc(sz(l, ch[l]));
      act["gskip" + std::to_string(l)].alloc(sz(l, ch[l]));
      if (l > 0) act["pool" + std::to_string(l)].alloc(sz(l, ch[l - 1]));
      if (l < L - 1) {
        act["up" + std::to_string(l)].alloc(sz(l, ch[l + 1]));
        act["decC" + std::to_string(l)].alloc(sz(l, ch[l]));
        act["sum" + std::to_string(l)].alloc(sz(l, ch[l]));
        act["d" + std::to_string(l)].alloc(sz(l, ch[l]));
      }
    }
    size_t big = 0;
    for (int l = 0; l < L; ++l) big = std::max(big, sz(l, std::max(ch[l], l + 1 < L ? ch[l + 1] : 0)));
    big = std::max(big, sz(0, std::max(3, ch[0])));
    act["t1"].alloc(big);
    act["t2"].alloc(big);
    act["gout"].alloc(sz(0, 2));
    act["gd"].alloc(big);
    if (mode == STDD_NN_TC) {
      // split-K scratch: the largest (slices x output) over every layer in
      // both directions at its level's size
      size_t need = 1;
      auto take = [&](const Layer &ly, int l) {
        const int h = H >> l, w = W >> l;
        for (int flip = 0; flip < 2; ++flip) {
          const int ci = flip ? ly.cout : ly.cin, co = flip ? ly.cin : ly.cout;
          const size_t ks = (size_t)stdd::nn_tc_ksplit(ci, co, N, h, w);
          if (ks > 1) need = std::max(need, ks * N * co * (size_t)h * w);
        }
      };
      for (int l = 0; l < L; ++l) {
        take(encA(l), l);
        take(encB(l), l);
        if (l < L - 1) {
          take(decC(l), l);
          take(decD(l), l);
        }
      }
      take(outL(), 0);
      act["ksplit"].alloc(need);
    }
  }


  // forward pass; returns the output buffer (N x 2 x H x W)
  void forward(int N, int H, int W, const float *in, float *out, cudaStream_t st) {
    check_shape(N, H, W);
    ensure_acts(N, H, W);
    for (int l = 0; l < L; ++l) {
      const int h = H >> l, wd = W >> l;
      const float *src = in;
      int cin = 3;
      if (l > 0) {
        stdd::nn_pool2(A("skip", l - 1), A("pool", l), (int64_t)N * ch[l - 1], H >> (l - 1), W >> (l - 1), st);
        src = A("pool", l);
        cin = ch[l - 1];
      }
      conv(src, encA(l), A("encA", l), N, h, wd, true, false, st);
      conv(A("encA", l), encB(l), A("skip", l), N, h, wd, true, false, st);
    }
    for (int l = L - 2; l >= 0; --l) {
      const int h = H >> l, wd = W >> l;
      const float *deeper = (l + 1 == L - 1) ? A("skip", L - 1) : A("d", l + 1);
      stdd::nn_up2(deeper, A("up", l), (int64_t)N * ch[l + 1], h, wd, st);
      conv(A("up", l), decC(l), A("decC", l), N, h, wd, true, false, st);
      const size_t cnt = sz(l, ch[l]);
      NCK(cudaMemcpyAsync(A("sum", l), A("decC", l), cnt * sizeof(float), cudaMemcpyDeviceToDevice, st));
      stdd::nn_axpy(A("skip", l), A("sum", l), 1.f, (int64_t)cnt, st);
      conv(A("sum", l), decD(l), A("d", l), N, h, wd, true, false, st);
    }
    const float *last = L > 1 ? A("d", 0) : A("skip", 0);
    conv(last, outL(), out, N, H, W, false, false, st);
    NCK(cudaGetLastError());
  }

  // gradient of the MSE loss w.r.t. all parameters into g; loss into loss.p
  void backward(int N, int H, int W, const float *in, const float *target) {
    cudaStream_t st = stream;
    check_shape(N, H, W);
    ensure_acts(N, H, W);  // sets the shapes sz() uses
    float *out = buf("out", sz(0, 2));
    forward(N, H, W, in, out, st);
    NCK(cudaMemsetAsync(g.p, 0, nparams * sizeof(float), st));
    NCK(cudaMemsetAsync(loss.p, 0, sizeof(float), st));
    float *gout = act["gout"].p;
    stdd::nn_mse(out, target, gout, (int64_t)sz(0, 2), loss.p, st);
    float *t1 = act["t1"].p, *t2 = act["t2"].p, *gd = act["gd"].p;
    // output layer
    const float *last = L > 1 ? A("d", 0) : A("skip", 0);
    wgrad(last, ch[0], gout, 2, N, H, W, g.p + outL().woff, g.p + outL().boff, st);
    conv(gout, outL(), gd, N, H, W, false, true, st);  // grad of d_0
    for (int l = 0; l < L; ++l)
      NCK(cudaMemsetAsync(A("gskip", l), 0, sz(l, ch[l]) * sizeof(float), st));
    if (L == 1) {
      NCK(cudaMemcpyAsync(A("gskip", 0), gd, sz(0, ch[0]) * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    // decoder, fine to coarse; gd holds the gradient w.r.t. d_l
    for (int l = 0; l <= L - 2; ++l) {
      const int h = H >> l, wd = W >> l;
      const size_t cnt = sz(l, ch[l]);
      stdd::nn_relu_mask(A("d", l), gd, (int64_t)cnt, st);
      wgrad(A("sum", l), ch[l], gd, ch[l], N, h, wd, g.p + decD(l).woff, g.p + decD(l).boff, st);
      conv(gd, decD(l), t1, N, h, wd, false, true, st);  // grad of sum
      stdd::nn_axpy(t1, A("gskip", l), 1.f, (int64_t)cnt, st);
      stdd::nn_relu_mask(A("decC", l), t1, (int64_t)cnt, st);
      wgrad(A("up", l), ch[l + 1], t1, ch[l], N, h, wd, g.p + decC(l).woff, g.p + decC(l).boff, st);
      conv(t1, decC(l), t2, N, h, wd, false, true, st);  // grad of up
      stdd::nn_up2_bwd(t2, gd, (int64_t)N * ch[l + 1], h, wd, st);  // grad of d_{l+1}
      if (l + 1 == L - 1)
        stdd::nn_axpy(gd, A("gskip", L - 1), 1.f, (int64_t)sz(L - 1, ch[L - 1]), st);
    }
    // encoder, coarse to fine
    for (int l = L - 1; l >= 0; --l) {
      const int h = H >> l, wd = W >> l;
      const size_t cnt = sz(l, ch[l]);
      float *gs = A("gskip", l);
      stdd::nn_relu_mask(A("skip", l), gs, (int64_t)cnt, st);
      wgrad(A("encA", l), ch[l], gs, ch[l], N, h, wd, g.p + encB(l).woff, g.p + encB(l).boff, st);
      conv(gs, encB(l), t1, N, h, wd, false, true, st);  // grad of encA
      stdd::nn_relu_mask(A("encA", l), t1, (int64_t)cnt, st);
      const float *src = l > 0 ? A("pool", l) : in;
      const int cin = l > 0 ? ch[l - 1] : 3;
      wgrad(src, cin, t1, ch[l], N, h, wd, g.p + encA(l).woff, g.p + encA(l).boff, st);
      if (l > 0) {
        conv(t1, encA(l), t2, N, h, wd, false, true, st);  // grad of pool
        stdd::nn_pool2_bwd(t2, t1, (int64_t)N * cin, H >> (l - 1), W >> (l - 1), st);
        stdd::nn_axpy(t1, A("gskip", l - 1), 1.f, (int64_t)sz(l - 1, ch[l - 1]), st);
      }
    }
    NCK(cudaGetLastError());
  }
};

namespace stdd {
int nn_device(const stdd_nn *nn) { return nn->device; }

void nn_guess_field(stdd_nn *nn, const double *eps, const double2 *b, int nx, int ny, double unit, double2 *x0,
                    double *scratch, cudaStream_t st) {
  const int f = 1 << (nn->L - 1);
  const int Wp = (nx + f - 1) / f * f, Hp = (ny + f - 1) / f * f;
  float *in = nn->buf("guess_in", (size_t)3 * Wp * Hp);
  float *out = nn->buf("guess_out", (size_t)2 * Wp * Hp);
  NCK(cudaMemsetAsync(in, 0, (size_t)3 * Wp * Hp * sizeof(float), st));
  double *scale = scratch + NN_PART;
  nn_absmax(b, (int64_t)nx * ny, scratch, scale, st);
  nn_input(eps, b, scale, in, nx, ny, Wp, Hp, st);
  nn->forward(1, Hp, Wp, in, out, st);
  nn->check_flag(st);
  nn_output(out, scale, unit, x0, nx, ny, Wp, Hp, st);
  NCK(cudaGetLastError());
}
}  // namespace stdd

namespace {
template <typename F> stdd_status nn_guard(stdd_nn *nn, F &&f) {
  if (!nn) return STDD_EINVAL;
  try {
    NCK(cudaSetDevice(nn->device));
    f();
    nn->err.clear();
    return STDD_OK;
  } catch (const std::invalid_argument &e) {
    nn->err = e.what();
    return STDD_EINVAL;
  } catch (const std::bad_alloc &) {
    nn->err = "out of memory";
    return STDD_ENOMEM;
  } catch (const NnError &e) {
    nn->err = e.what();
    return STDD_ECUDA;
  } catch (const std::exception &e) {
    nn->err = e.what();
    return STDD_EINVAL;
  }
}
}  // namespace

extern "C" {

stdd_status stdd_nn_create(stdd_nn **out, int device, void *cuda_stream, int levels, int base_channels,
                           int max_channels, int mode, unsigned long long seed) {
  if (!out) return STDD_EINVAL;
  *out = nullptr;
  stdd_nn *nn = new (std::nothrow) stdd_nn();
  if (!nn) return STDD_ENOMEM;
  nn->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete nn;
    return STDD_ECUDA;
  }
  if (cuda_stream) {
    nn->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&nn->stream, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      delete nn;
      return STDD_ECUDA;
    }
    nn->own_stream = true;
  }
  const stdd_status st = nn_guard(nn, [&] { nn->build(levels, base_channels, max_channels, mode, seed); });
  if (st != STDD_OK) {
    if (nn->own_stream) cudaStreamDestroy(nn->stream);
    delete nn;
    return st;
  }
  *out = nn;
  return STDD_OK;
}

void stdd_nn_destroy(stdd_nn *nn) {
  if (!nn) return;
  cudaSetDevice(nn->device);
  cudaStreamSynchronize(nn->stream);
  if (nn->own_stream) cudaStreamDestroy(nn->stream);
  delete nn;
}

long long stdd_nn_num_params(const stdd_nn *nn) { return nn ? nn->nparams : -1; }

stdd_status stdd_nn_get_params(stdd_nn *nn, float *host) {
  return nn_guard(nn, [&] {
    if (!host) throw std::invalid_argument("null buffer");
    NCK(cudaMemcpyAsync(host, nn->w.p, nn->nparams * sizeof(float), cudaMemcpyDeviceToHost, nn->stream));
    NCK(cudaStreamSynchronize(nn->stream));
  });
}

stdd_status stdd_nn_set_params(stdd_nn *nn, const float *host) {
  return nn_guard(nn, [&] {
    if (!host) throw std::invalid_argument("null buffer");
    NCK(cudaMemcpyAsync(nn->w.p, host, nn->nparams * sizeof(float), cudaMemcpyHostToDevice, nn->stream));
    stdd::nn_round(nn->w.p, nn->wb.p, nn->nparams, nn->bf16, nn->stream);
    nn->repack();
    NCK(cudaStreamSynchronize(nn->stream));
  });
}

stdd_status stdd_nn_forward(stdd_nn *nn, int batch, int H, int W, const float *input, float *output) {
  return nn_guard(nn, [&] {
    if (!input || !output) throw std::invalid_argument("null buffer");
    nn->forward(batch, H, W, input, output, nn->stream);
    nn->check_flag(nn->stream);
  });
}

stdd_status stdd_nn_gradient(stdd_nn *nn, int batch, int H, int W, const float *input, const float *target,
                             float *loss_out, float *grad_host) {
  return nn_guard(nn, [&] {
    if (!input || !target) throw std::invalid_argument("null buffer");
    nn->check_shape(batch, H, W);
    nn->backward(batch, H, W, input, target);
    if (loss_out) NCK(cudaMemcpyAsync(loss_out, nn->loss.p, sizeof(float), cudaMemcpyDeviceToHost, nn->stream));
    if (grad_host)
      NCK(cudaMemcpyAsync(grad_host, nn->g.p, nn->nparams * sizeof(float), cudaMemcpyDeviceToHost, nn->stream));
    nn->check_flag(nn->stream);
  });
}

stdd_status stdd_nn_train_step(stdd_nn *nn, int batch, int H, int W, const float *input, const float *target,
                               float lr, float *loss_out) {
  return nn_guard(nn, [&] {
    if (!input || !target || !(lr > 0)) throw std::invalid_argument("bad training arguments");
    nn->check_shape(batch, H, W);
    nn->backward(batch, H, W, input, target);
    ++nn->step;
    stdd::nn_adam(nn->w.p, nn->wb.p, nn->g.p, nn->m.p, nn->v.p, nn->nparams, lr, nn->step, nn->bf16, nn->stream);
    nn->repack();
    if (loss_out) NCK(cudaMemcpyAsync(loss_out, nn->loss.p, sizeof(float), cudaMemcpyDeviceToHost, nn->stream));
    nn->check_flag(nn->stream);
  });
}

stdd_status stdd_nn_make_images(stdd_nn *nn, int nx, int ny, double unit, const double *eps, const double *b,
                                const double *x, int H, int W, float *input, float *target) {
  return nn_guard(nn, [&] {
    if (nx < 1 || ny < 1 || W < nx || H < ny || !(unit > 0) || !eps || !b || !input || (x && !target))
      throw std::invalid_argument("bad image arguments");
    cudaStream_t st = nn->stream;
    double *scr = nullptr;
    {
      DevF &d = nn->act["images_scratch"];
      d.alloc(2 * (stdd::NN_PART + 1));
      scr = reinterpret_cast<double *>(d.p);
    }
    NCK(cudaMemsetAsync(input, 0, (size_t)3 * H * W * sizeof(float), st));
    const double2 *bz = reinterpret_cast<const double2 *>(b);
    stdd::nn_absmax(bz, (int64_t)nx * ny, scr, scr + stdd::NN_PART, st);
    stdd::nn_input(eps, bz, scr + stdd::NN_PART, input, nx, ny, W, H, st);
    if (x) {
      NCK(cudaMemsetAsync(target, 0, (size_t)2 * H * W * sizeof(float), st));
      stdd::nn_target(reinterpret_cast<const double2 *>(x), scr + stdd::NN_PART, unit, target, nx, ny, W, H, st);
    }
    NCK(cudaGetLastError());
    NCK(cudaStreamSynchronize(st));
  });
}

const char *stdd_nn_last_error(const stdd_nn *nn) { return nn ? nn->err.c_str() : "null network"; }

}  // extern "C"

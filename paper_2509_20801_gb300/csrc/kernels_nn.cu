// Kernels of the learned initial guess: a convolutional encoder-decoder that
// maps (permittivity, Re b, Im b) on the grid to (Re x0, Im x0).  Activations
// are FP32 NCHW; the convolution weights used by the forward and backward
// passes are the FP32 master weights rounded to BF16 (kept as floats), with
// FP32 accumulation.  Training: MSE loss, Adam on the FP32 master weights.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace stdd {

namespace {

constexpr int TPX = 16;   // 16 x 16 pixel tiles
constexpr int COB = 16;   // output channels per block
constexpr int CIB = 16;   // input channels per shared-memory stage

// out[n, co] = bias[co] + sum_ci sum_3x3 w[co, ci] * in[n, ci] (zero padding);
// flip = 1 uses the transposed, spatially flipped weights (the input
// gradient of a convolution): w'[co, ci, ky, kx] = w[ci, co, 2-ky, 2-kx].
__global__ void __launch_bounds__(256) k_conv3x3(const float *__restrict__ in, int Cin,
                                                 const float *__restrict__ w, const float *__restrict__ bias,
                                                 float *__restrict__ out, int Cout, int H, int W, int relu,
                                                 int flip) {
  __shared__ float tin[CIB][TPX + 2][TPX + 2];
  __shared__ float tw[COB][CIB][9];
  const int tx = threadIdx.x % TPX, ty = threadIdx.x / TPX;
  const int tiles_x = (W + TPX - 1) / TPX;
  const int x0 = (blockIdx.x % tiles_x) * TPX, y0 = (blockIdx.x / tiles_x) * TPX;
  const int cob = (Cout + COB - 1) / COB;
  const int n = blockIdx.y / cob, co0 = (blockIdx.y % cob) * COB;
  const int x = x0 + tx, y = y0 + ty;
  float acc[COB];
#pragma unroll
  for (int c = 0; c < COB; ++c) acc[c] = (bias && co0 + c < Cout) ? bias[co0 + c] : 0.f;
  for (int ci0 = 0; ci0 < Cin; ci0 += CIB) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < CIB * (TPX + 2) * (TPX + 2); idx += 256) {
      const int c = idx / ((TPX + 2) * (TPX + 2)), rem = idx % ((TPX + 2) * (TPX + 2));
      const int yy = y0 - 1 + rem / (TPX + 2), xx = x0 - 1 + rem % (TPX + 2);
      float v = 0.f;
      if (ci0 + c < Cin && yy >= 0 && yy < H && xx >= 0 && xx < W)
        v = in[(((int64_t)n * Cin + ci0 + c) * H + yy) * W + xx];
      tin[c][rem / (TPX + 2)][rem % (TPX + 2)] = v;
    }
    for (int idx = threadIdx.x; idx < COB * CIB * 9; idx += 256) {
      const int c = idx / (CIB * 9), rem = idx % (CIB * 9), ci = rem / 9, k = rem % 9;
      float v = 0.f;
      if (co0 + c < Cout && ci0 + ci < Cin) {
        if (!flip) v = w[((int64_t)(co0 + c) * Cin + ci0 + ci) * 9 + k];
        else v = w[((int64_t)(ci0 + ci) * Cout + co0 + c) * 9 + (8 - k)];
      }
      tw[c][ci][k] = v;
    }
    __syncthreads();
    const int cin_here = min(CIB, Cin - ci0);
    for (int ci = 0; ci < cin_here; ++ci) {
      float v[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) v[k] = tin[ci][ty + k / 3][tx + k % 3];
#pragma unroll
      for (int c = 0; c < COB; ++c)
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[c] = fmaf(tw[c][ci][k], v[k], acc[c]);
    }
  }
  if (x < W && y < H) {
#pragma unroll
    for (int c = 0; c < COB; ++c) {
      if (co0 + c < Cout) {
        float r = acc[c];
        if (relu) r = fmaxf(r, 0.f);
        out[(((int64_t)n * Cout + co0 + c) * H + y) * W + x] = r;
      }
    }
  }
}

// gw[co, ci, k] += sum_n sum_pixels gout[n, co] * in[n, ci] shifted by k,
// gb[co] += sum gout[n, co]; one block per (co block, ci block, tile, n)
__global__ void __launch_bounds__(256) k_conv3x3_wgrad(const float *__restrict__ in, int Cin,
                                                       const float *__restrict__ gout, int Cout, int H, int W,
                                                       float *__restrict__ gw, float *__restrict__ gb) {
  __shared__ float tin[CIB][TPX + 2][TPX + 2];
  __shared__ float tg[COB][TPX][TPX];
  const int cib = (Cin + CIB - 1) / CIB;
  const int co0 = (blockIdx.x / cib) * COB, ci0 = (blockIdx.x % cib) * CIB;
  const int tiles_x = (W + TPX - 1) / TPX;
  const int x0 = (blockIdx.y % tiles_x) * TPX, y0 = (blockIdx.y / tiles_x) * TPX;
  const int n = blockIdx.z;
  for (int idx = threadIdx.x; idx < CIB * (TPX + 2) * (TPX + 2); idx += 256) {
    const int c = idx / ((TPX + 2) * (TPX + 2)), rem = idx % ((TPX + 2) * (TPX + 2));
    const int yy = y0 - 1 + rem / (TPX + 2), xx = x0 - 1 + rem % (TPX + 2);
    float v = 0.f;
    if (ci0 + c < Cin && yy >= 0 && yy < H && xx >= 0 && xx < W)
      v = in[(((int64_t)n * Cin + ci0 + c) * H + yy) * W + xx];
    tin[c][rem / (TPX + 2)][rem % (TPX + 2)] = v;
  }
  for (int idx = threadIdx.x; idx < COB * TPX * TPX; idx += 256) {
    const int c = idx / (TPX * TPX), rem = idx % (TPX * TPX);
    const int yy = y0 + rem / TPX, xx = x0 + rem % TPX;
    float v = 0.f;
    if (co0 + c < Cout && yy < H && xx < W) v = gout[(((int64_t)n * Cout + co0 + c) * H + yy) * W + xx];
    tg[c][rem / TPX][rem % TPX] = v;
  }
  __syncthreads();
  const int co = threadIdx.x / CIB, ci = threadIdx.x % CIB;
  float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  float bsum = 0.f;
  for (int py = 0; py < TPX; ++py)
    for (int px = 0; px < TPX; ++px) {
      const float g = tg[co][py][px];
      bsum += g;
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] = fmaf(g, tin[ci][py + k / 3][px + k % 3], acc[k]);
    }
  if (co0 + co < Cout && ci0 + ci < Cin) {
#pragma unroll
    for (int k = 0; k < 9; ++k) atomicAdd(&gw[((int64_t)(co0 + co) * Cin + ci0 + ci) * 9 + k], acc[k]);
  }
  if (gb && ci == 0 && ci0 == 0 && co0 + co < Cout) atomicAdd(&gb[co0 + co], bsum);
}

__global__ void k_relu_mask(const float *__restrict__ y, float *__restrict__ g, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(y[i] > 0.f)) g[i] = 0.f;
}

// 2 x 2 average pooling (H, W even) and its adjoint
__global__ void k_pool2(const float *__restrict__ in, float *__restrict__ out, int64_t planes, int H, int W) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t n = planes * Ho * Wo;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pl = i / ((int64_t)Ho * Wo);
    const int r = (int)(i % ((int64_t)Ho * Wo)), yo = r / Wo, xo = r % Wo;
    const float *p = in + (pl * H + 2 * yo) * W + 2 * xo;
    out[i] = 0.25f * (p[0] + p[1] + p[W] + p[W + 1]);
  }
}
__global__ void k_pool2_bwd(const float *__restrict__ gout, float *__restrict__ gin, int64_t planes, int H, int W) {
  const int64_t n = planes * H * W;
  const int Wo = W / 2, Ho = H / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pl = i / ((int64_t)H * W);
    const int r = (int)(i % ((int64_t)H * W)), y = r / W, x = r % W;
    gin[i] = 0.25f * gout[(pl * Ho + y / 2) * Wo + x / 2];
  }
}
// nearest 2x upsampling (output H, W) and its adjoint
__global__ void k_up2(const float *__restrict__ in, float *__restrict__ out, int64_t planes, int H, int W) {
  const int64_t n = planes * H * W;
  const int Wi = W / 2, Hi = H / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pl = i / ((int64_t)H * W);
    const int r = (int)(i % ((int64_t)H * W)), y = r / W, x = r % W;
    out[i] = in[(pl * Hi + y / 2) * Wi + x / 2];
  }
}
__global__ void k_up2_bwd(const float *__restrict__ gout, float *__restrict__ gin, int64_t planes, int H, int W) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t n = planes * Ho * Wo;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pl = i / ((int64_t)Ho * Wo);
    const int r = (int)(i % ((int64_t)Ho * Wo)), yo = r / Wo, xo = r % Wo;
    const float *p = gout + (pl * H + 2 * yo) * W + 2 * xo;
    gin[i] = p[0] + p[1] + p[W] + p[W + 1];
  }
}
__global__ void k_axpy_f(const float *__restrict__ x, float *__restrict__ y, float a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
// loss = sum (p - t)^2 / n, g = 2 (p - t) / n
__global__ void k_mse(const float *__restrict__ p, const float *__restrict__ t, float *__restrict__ g, int64_t n,
                      float *__restrict__ loss) {
  float s = 0.f;
  const float sc = 1.f / (float)n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = p[i] - t[i];
    s += d * d;
    g[i] = 2.f * d * sc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * sc);
}
// Adam (Kingma & Ba 2015) on the master weights, then the BF16-rounded copy
__global__ void k_adam(float *__restrict__ w, float *__restrict__ wb, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2, int round_bf16) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = round_bf16 ? __bfloat162float(__float2bfloat16_rn(wi)) : wi;
  }
}
__global__ void k_round(const float *__restrict__ w, float *__restrict__ wb, int64_t n, int round_bf16) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    wb[i] = round_bf16 ? __bfloat162float(__float2bfloat16_rn(w[i])) : w[i];
}

// network input from the solver's fields, on an image of Wp x Hp pixels
// (Wp >= nx, Hp >= ny, padding left at zero = vacuum and no source):
// ch0 = (eps - 1) / 10, ch1 / ch2 = Re / Im b divided by scale[0] (the largest
// |Re| or |Im| of b); solver node (i, j) maps to image row j, column i
__global__ void k_nn_input(const double *__restrict__ eps, const double2 *__restrict__ b, const double *scale,
                           float *__restrict__ out, int nx, int ny, int Wp, int64_t plane) {
  const int64_t n = (int64_t)nx * ny;
  const double s = scale[0] > 0 ? 1.0 / scale[0] : 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(g / ny), j = (int)(g % ny);
    const int64_t pix = (int64_t)j * Wp + i;
    out[pix] = (float)((eps[g] - 1.0) / 10.0);
    out[plane + pix] = (float)(b[g].x * s);
    out[2 * plane + pix] = (float)(b[g].y * s);
  }
}
// x0 = (out0 + i out1) * scale[0] * unit
__global__ void k_nn_output(const float *__restrict__ out, const double *scale, double unit,
                            double2 *__restrict__ x0, int nx, int ny, int Wp, int64_t plane) {
  const int64_t n = (int64_t)nx * ny;
  const double s = scale[0] * unit;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(g / ny), j = (int)(g % ny);
    const int64_t pix = (int64_t)j * Wp + i;
    x0[g] = make_double2(out[pix] * s, out[plane + pix] * s);
  }
}
// training target from a solved field: the inverse map of k_nn_output
__global__ void k_nn_target(const double2 *__restrict__ x, const double *scale, double unit, float *__restrict__ out,
                            int nx, int ny, int Wp, int64_t plane) {
  const int64_t n = (int64_t)nx * ny;
  const double s = scale[0] > 0 ? 1.0 / (scale[0] * unit) : 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(g / ny), j = (int)(g % ny);
    const int64_t pix = (int64_t)j * Wp + i;
    out[pix] = (float)(x[g].x * s);
    out[plane + pix] = (float)(x[g].y * s);
  }
}
// out[0..3] = Re sum conj(a) b, Im sum conj(a) b, sum |a|^2, sum |b|^2
// (deterministic: fixed per-block partials, one final warp)
__global__ void k_fit_part(const double2 *__restrict__ a, const double2 *__restrict__ b, int64_t n,
                           double *__restrict__ part) {
  double s[4] = {0, 0, 0, 0};
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = a[g], y = b[g];
    s[0] += x.x * y.x + x.y * y.y;
    s[1] += x.x * y.y - x.y * y.x;
    s[2] += x.x * x.x + x.y * x.y;
    s[3] += y.x * y.x + y.y * y.y;
  }
  __shared__ double sh[4][8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = s[k];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[threadIdx.x][w];
    part[(int64_t)blockIdx.x * 4 + threadIdx.x] = r;
  }
}
__global__ void k_fit_final(const double *__restrict__ part, int nb, double *__restrict__ out) {
  const int k = threadIdx.x >> 3, l = threadIdx.x & 7;  // 4 groups of 8 lanes
  double r = 0;
  for (int i = l; i < nb; i += 8) r += part[(int64_t)i * 4 + k];
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  if (l == 0) out[k] = r;
}
__global__ void k_zadd(const double2 *__restrict__ z, double2 *__restrict__ x, int64_t n) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = z[g], v = x[g];
    x[g] = make_double2(v.x + a.x, v.y + a.y);
  }
}
__global__ void k_zscale(double2 *__restrict__ x, int64_t n, double ar, double ai) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[g];
    x[g] = make_double2(ar * v.x - ai * v.y, ar * v.y + ai * v.x);
  }
}
// scale[0] = max over the field of max(|re|, |im|) (deterministic two-stage)
__global__ void k_absmax_part(const double2 *__restrict__ b, int64_t n, double *__restrict__ part) {
  double m = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fmax(fabs(b[g].x), fabs(b[g].y)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
    part[blockIdx.x] = r;
  }
}
__global__ void k_absmax_final(const double *__restrict__ part, int nb, double *__restrict__ out) {
  double m = 0;
  for (int i = threadIdx.x; i < nb; i += 32) m = fmax(m, part[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x == 0) out[0] = m;
}

inline int egrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

void nn_conv(const float *in, int Cin, const float *w, const float *bias, float *out, int Cout, int N, int H, int W,
             bool relu, bool flip, cudaStream_t st) {
  const int tiles = ((W + TPX - 1) / TPX) * ((H + TPX - 1) / TPX);
  const dim3 grid(tiles, N * ((Cout + COB - 1) / COB));
  k_conv3x3<<<grid, 256, 0, st>>>(in, Cin, w, bias, out, Cout, H, W, relu ? 1 : 0, flip ? 1 : 0);
  count_launch();
}
void nn_conv_wgrad(const float *in, int Cin, const float *gout, int Cout, int N, int H, int W, float *gw, float *gb,
                   cudaStream_t st) {
  const int tiles = ((W + TPX - 1) / TPX) * ((H + TPX - 1) / TPX);
  const dim3 grid(((Cout + COB - 1) / COB) * ((Cin + CIB - 1) / CIB), tiles, N);
  k_conv3x3_wgrad<<<grid, 256, 0, st>>>(in, Cin, gout, Cout, H, W, gw, gb);
  count_launch();
}
void nn_relu_mask(const float *y, float *g, int64_t n, cudaStream_t st) {
  k_relu_mask<<<egrid(n), 256, 0, st>>>(y, g, n);
  count_launch();
}
void nn_pool2(const float *in, float *out, int64_t planes, int H, int W, cudaStream_t st) {
  k_pool2<<<egrid(planes * H * W / 4), 256, 0, st>>>(in, out, planes, H, W);
  count_launch();
}
void nn_pool2_bwd(const float *gout, float *gin, int64_t planes, int H, int W, cudaStream_t st) {
  k_pool2_bwd<<<egrid(planes * H * W), 256, 0, st>>>(gout, gin, planes, H, W);
  count_launch();
}
void nn_up2(const float *in, float *out, int64_t planes, int H, int W, cudaStream_t st) {
  k_up2<<<egrid(planes * H * W), 256, 0, st>>>(in, out, planes, H, W);
  count_launch();
}
void nn_up2_bwd(const float *gout, float *gin, int64_t planes, int H, int W, cudaStream_t st) {
  k_up2_bwd<<<egrid(planes * H * W / 4), 256, 0, st>>>(gout, gin, planes, H, W);
  count_launch();
}
void nn_axpy(const float *x, float *y, float a, int64_t n, cudaStream_t st) {
  k_axpy_f<<<egrid(n), 256, 0, st>>>(x, y, a, n);
  count_launch();
}
void nn_mse(const float *p, const float *t, float *g, int64_t n, float *loss, cudaStream_t st) {
  k_mse<<<egrid(n), 256, 0, st>>>(p, t, g, n, loss);
  count_launch();
}
void nn_adam(float *w, float *wb, const float *g, float *m, float *v, int64_t n, float lr, int step, bool bf16,
             cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<egrid(n), 256, 0, st>>>(w, wb, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2, bf16 ? 1 : 0);
  count_launch();
}
void nn_round(const float *w, float *wb, int64_t n, bool bf16, cudaStream_t st) {
  k_round<<<egrid(n), 256, 0, st>>>(w, wb, n, bf16 ? 1 : 0);
  count_launch();
}
void nn_input(const double *eps, const double2 *b, const double *scale, float *out, int nx, int ny, int Wp, int Hp,
              cudaStream_t st) {
  k_nn_input<<<egrid((int64_t)nx * ny), 256, 0, st>>>(eps, b, scale, out, nx, ny, Wp, (int64_t)Wp * Hp);
  count_launch();
}
void nn_output(const float *out, const double *scale, double unit, double2 *x0, int nx, int ny, int Wp, int Hp,
               cudaStream_t st) {
  k_nn_output<<<egrid((int64_t)nx * ny), 256, 0, st>>>(out, scale, unit, x0, nx, ny, Wp, (int64_t)Wp * Hp);
  count_launch();
}
void nn_target(const double2 *x, const double *scale, double unit, float *out, int nx, int ny, int Wp, int Hp,
               cudaStream_t st) {
  k_nn_target<<<egrid((int64_t)nx * ny), 256, 0, st>>>(x, scale, unit, out, nx, ny, Wp, (int64_t)Wp * Hp);
  count_launch();
}
void nn_fit(const double2 *a, const double2 *b, int64_t n, double *part, double *out4, cudaStream_t st) {
  const int nb = std::min(egrid(n), 608);
  k_fit_part<<<nb, 256, 0, st>>>(a, b, n, part);
  k_fit_final<<<1, 32, 0, st>>>(part, nb, out4);
  count_launch(2);
}
void nn_zadd(const double2 *z, double2 *x, int64_t n, cudaStream_t st) {
  k_zadd<<<egrid(n), 256, 0, st>>>(z, x, n);
  count_launch();
}
void nn_zscale(double2 *x, int64_t n, double ar, double ai, cudaStream_t st) {
  k_zscale<<<egrid(n), 256, 0, st>>>(x, n, ar, ai);
  count_launch();
}
// part needs 608 doubles (nn_absmax) or 4 x 608 (nn_fit)
void nn_absmax(const double2 *b, int64_t n, double *part, double *out, cudaStream_t st) {
  const int nb = std::min(egrid(n), 608);
  k_absmax_part<<<nb, 256, 0, st>>>(b, n, part);
  k_absmax_final<<<1, 32, 0, st>>>(part, nb, out);
  count_launch(2);
}

}  // namespace stdd

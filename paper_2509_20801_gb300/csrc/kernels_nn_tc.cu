// Tensor-core (tcgen05) 3x3 convolutions of the learned-guess network: the
// forward pass and the input gradient (the same convolution with the
// weights transposed and flipped), as implicit GEMMs with BF16 operands and
// FP32 accumulation in TMEM.
//
// One CTA (256 threads) computes a 16 x 16 pixel tile for all output
// channels (N = Cout rounded up to 16, at most 256) as two M = 128 halves
// (16 rows x 8 columns each, accumulators side by side in TMEM).  The input
// channels are consumed in chunks of 16 (K = 16 per MMA); per chunk the
// threads stage the 18 x 18 halo of the tile as BF16, channel-innermost in
// two 8-channel planes, and one thread issues 9 taps x 2 halves MMAs.  With
// the halo rows 18 pixels apart, the A operand of tap (ky, kx) is the halo
// viewed from pixel (ky, kx): core matrices of 8 consecutive pixels x 8
// channels, SBO = one halo row (288 B), LBO = one channel plane, so no
// im2col copy is made.  The B operand (weights) is packed once per weight
// update into the exact shared-memory order and arrives by one bulk copy per
// chunk.  Activations and weights are double-buffered: chunk c+1 is staged
// while the MMAs of chunk c run.  Every wait has an iteration limit; a
// timeout sets the error flag and the CTA stops cleanly.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace stdd {

namespace {

constexpr int CT_T = 16;                        // tile side (pixels)
constexpr int CT_HP = CT_T + 2;                 // halo pitch (pixels)
constexpr int CT_PLANE = CT_HP * CT_HP * 16;    // one 8-channel plane: 5184 B
constexpr int CT_ACT = 2 * CT_PLANE;            // one stage of activations
constexpr long long CT_WAIT = 1ll << 22;
constexpr int CT_ITEMS = (2 * CT_HP * CT_HP + 255) / 256;  // halo items per thread and chunk (3)

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__host__ __device__ inline int tmem_cols_for(int Npad) {
  int c = 32;
  while (c < 2 * Npad) c <<= 1;
  return c;
}

struct ConvTcArgs {
  const float *in;
  int Cin;
  const uint16_t *wp;    // packed weights [chunk][tap][cg][Npad][8] BF16
  int Npad, nchunks;
  const float *bias;
  float *out;
  int Cout, H, W, relu;
  int *flag;
  float *part;    // split-K: partial sums [gridDim.z][N][Cout][H][W], or null
};

__global__ void __launch_bounds__(256) k_conv3x3_tc(ConvTcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int wbytes = 288 * a.Npad;
  uint8_t *act0 = sm;
  uint8_t *wst0 = sm + 2 * CT_ACT;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 2 * CT_ACT + 2 * wbytes);  // w[2], mma[2]
  uint32_t *tm = reinterpret_cast<uint32_t *>(bars + 4);
  int *abort_flag = reinterpret_cast<int *>(tm + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = (a.W + CT_T - 1) / CT_T;
  const int x0 = (blockIdx.x % tiles_x) * CT_T, y0 = (blockIdx.x / tiles_x) * CT_T;
  const int n = blockIdx.y;
  // split-K: this CTA takes input-channel chunks [cb, ce)
  const int cb = (int)((int64_t)blockIdx.z * a.nchunks / gridDim.z);
  const int ce = (int)((int64_t)(blockIdx.z + 1) * a.nchunks / gridDim.z);
  const int cols = tmem_cols_for(a.Npad);
  const uint32_t bar0 = tcx::smem_u32(&bars[0]);
  auto bw = [&](int s) { return bar0 + 8u * (uint32_t)s; };        // weight copies landed
  auto bm = [&](int s) { return bar0 + 16u + 8u * (uint32_t)s; };  // MMAs of the stage done
  if (warp == 0) tcx::tmem_alloc(tcx::smem_u32(tm), (uint32_t)cols);
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tcx::mbar_init(tcx::smem_u32(&bars[i]), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tcx::fence_before();
  __syncthreads();
  tcx::fence_after();
  const uint32_t tmem = *tm;
  const uint32_t idesc = tcx::instr_desc_f16(1, 128, a.Npad);
  const int64_t plane = (int64_t)a.H * a.W;
  const float *inb = a.in + (int64_t)n * a.Cin * plane;
  bool ok = true;
  int issued = 0;   // chunks whose MMAs were committed
  for (int c = cb; c < ce; ++c) {
    const int lc = c - cb;  // local chunk count: stages and barrier phases
    const int s = lc & 1;
    uint8_t *act = act0 + s * CT_ACT;
    uint8_t *wst = wst0 + s * wbytes;
    // stage s is free once the MMAs of chunk c - 2 completed
    if (lc >= 2 && !tcx::mbar_wait(bm(s), ((lc - 2) >> 1) & 1, CT_WAIT)) ok = false;
    if (!__syncthreads_and(ok && !*abort_flag)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      tcx::mbar_expect_tx(bw(s), (uint32_t)wbytes);
      tcx::bulk_g2s(tcx::smem_u32(wst), a.wp + (size_t)c * (wbytes / 2), (uint32_t)wbytes, bw(s));
    }
    // halo tile of 16 channels: items (plane cg, halo row, halo column),
    // at most CT_ITEMS per thread; every load of a thread is issued before
    // any is converted, so their latencies overlap
    {
      float v[CT_ITEMS][8];
#pragma unroll
      for (int u = 0; u < CT_ITEMS; ++u) {
        const int it = tid + u * 256;
        const int cg = it / (CT_HP * CT_HP), r = it % (CT_HP * CT_HP);
        const int y = y0 - 1 + r / CT_HP, x = x0 - 1 + r % CT_HP;
        const bool ok_item = it < 2 * CT_HP * CT_HP && y >= 0 && y < a.H && x >= 0 && x < a.W;
        const int ci0 = c * 16 + cg * 8;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          v[u][j] = (ok_item && ci0 + j < a.Cin) ? __ldg(inb + (int64_t)(ci0 + j) * plane + (int64_t)y * a.W + x)
                                                 : 0.f;
      }
#pragma unroll
      for (int u = 0; u < CT_ITEMS; ++u) {
        const int it = tid + u * 256;
        if (it < 2 * CT_HP * CT_HP) {
          const int cg = it / (CT_HP * CT_HP), r = it % (CT_HP * CT_HP);
          *reinterpret_cast<uint4 *>(act + cg * CT_PLANE + r * 16) =
              make_uint4(pack_bf16x2(v[u][0], v[u][1]), pack_bf16x2(v[u][2], v[u][3]),
                         pack_bf16x2(v[u][4], v[u][5]), pack_bf16x2(v[u][6], v[u][7]));
        }
      }
    }
    tcx::fence_proxy_async();
    tcx::fence_before();
    __syncthreads();
    tcx::fence_after();
    if (tid == 0) {
      if (tcx::mbar_wait(bw(s), (lc >> 1) & 1, CT_WAIT)) {
        const uint32_t a_base = tcx::smem_u32(act), b_base = tcx::smem_u32(wst);
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
          const int ky = tap / 3, kx = tap % 3;
          const uint64_t bdesc = tcx::smem_desc(b_base + tap * a.Npad * 32, a.Npad * 16, 128);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint64_t adesc =
                tcx::smem_desc(a_base + (ky * CT_HP + 8 * h + kx) * 16, CT_PLANE, CT_HP * 16);
            tcx::mma_f16(tmem + (uint32_t)(h * a.Npad), adesc, bdesc, idesc, (lc > 0 || tap > 0) ? 1u : 0u);
          }
        }
      } else {
        *abort_flag = 1;
        // the copy may still land: give it one more bounded wait
        tcx::mbar_wait(bw(s), (lc >> 1) & 1, CT_WAIT);
      }
      tcx::mma_commit(bm(s));
    }
    issued = lc + 1;
  }
  // all MMAs done: the last commit covers every earlier one
  if (issued > 0) {
    const int last = issued - 1;
    if (!tcx::mbar_wait(bm(last & 1), (last >> 1) & 1, CT_WAIT)) ok = false;
  }
  ok = __syncthreads_and(ok && !*abort_flag);
  tcx::fence_after();
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (pixels of its quarter) of
    // half w / 4; pixel m = 32 (w % 4) + lane is row m / 8, column m % 8
    const int q = warp & 3, h = warp >> 2;
    const int m = 32 * q + lane;
    const int y = y0 + (m >> 3), x = x0 + 8 * h + (m & 7);
    const bool store = y < a.H && x < a.W;
    const bool split = a.part != nullptr;
    float *outp = (split ? a.part + (int64_t)blockIdx.z * gridDim.y * a.Cout * plane : a.out) +
                  (int64_t)n * a.Cout * plane + (int64_t)y * a.W + x;
    for (int c0 = 0; c0 < a.Npad; c0 += 16) {
      uint32_t v[16];
      tcx::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * a.Npad + c0), v);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int co = c0 + u;
        if (store && co < a.Cout) {
          float r = __uint_as_float(v[u]);
          if (!split) {
            r += a.bias ? a.bias[co] : 0.f;
            if (a.relu) r = fmaxf(r, 0.f);
          }
          outp[(int64_t)co * plane] = r;
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(a.flag, 1);
  }
  tcx::fence_before();
  __syncthreads();
  if (warp == 0) tcx::tmem_dealloc(tmem, (uint32_t)cols);
}

// split-K epilogue: out = act(bias + sum over the slices, in slice order)
__global__ void k_splitk_finish(const float *__restrict__ part, int ks, int64_t count, int64_t plane, int Cout,
                                const float *__restrict__ bias, int relu, float *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    float r = 0.f;
    for (int z = 0; z < ks; ++z) r += part[(int64_t)z * count + i];
    if (bias) r += bias[(int)((i / plane) % Cout)];
    out[i] = relu ? fmaxf(r, 0.f) : r;
  }
}

// ---- weight gradient on the tensor cores
// gw[co][ci][t] += sum over pixels p of gout[co](p) in[ci](p + shift_t), one
// GEMM per tap t = 3 ky + kx with M = 128 output channels, N = 32 input
// channels, K = pixels.  A CTA walks a contiguous range of 64-pixel row
// segments (image n, row y, columns x0 .. x0 + 63; past the row end zero):
// the output-gradient segment is the A tile, and the three input rows
// y - 1 .. y + 1 (with a one-pixel halo) are written straight into the nine
// tap-shifted B tiles.  The nine accumulators (32 TMEM columns each) stay
// in TMEM across the CTA's segments; the epilogue adds them to gw with FP32
// atomics (CTAs split the pixels).  The bias gradient (sum of gout) is
// taken from the FP32 values while staging, by the CTAs of the first input
// channel tile.
constexpr int WG_M = 128, WG_N = 32, WG_K = 64;
constexpr int WG_A = WG_M * WG_K * 2;          // 16 KiB
constexpr int WG_BT = WG_N * WG_K * 2;         // 4 KiB per tap
constexpr int WG_STAGE = WG_A + 9 * WG_BT;     // 52 KiB
constexpr int WG_SMEM = 2 * WG_STAGE + 64;

// byte offset of (row, k) in a K-major tile of 64 K (core matrices 8 x 16 B)
__device__ __forceinline__ uint32_t wg_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

struct WgradTcArgs {
  const float *in, *gout;
  int Cin, Cout, N, H, W;
  float *gw, *gb;
  int *flag;
};

__global__ void __launch_bounds__(256, 1) k_conv3x3_wgrad_tc(WgradTcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ float gbs[WG_M];
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 2 * WG_STAGE);  // mma[2]
  uint32_t *tm = reinterpret_cast<uint32_t *>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int co0 = blockIdx.x * WG_M, ci0 = blockIdx.y * WG_N;
  const int spr = (a.W + WG_K - 1) / WG_K;
  const int64_t total = (int64_t)a.N * a.H * spr;
  const int64_t g0 = blockIdx.z * total / gridDim.z, g1 = (blockIdx.z + 1) * total / gridDim.z;
  const bool do_bias = a.gb && blockIdx.y == 0;
  const uint32_t bar0 = tcx::smem_u32(&bars[0]);
  auto bm = [&](int st) { return bar0 + 8u * (uint32_t)st; };
  if (warp == 0) tcx::tmem_alloc(tcx::smem_u32(tm), 512);
  if (tid < WG_M) gbs[tid] = 0.f;
  if (tid == 0) {
    tcx::mbar_init(bm(0), 1);
    tcx::mbar_init(bm(1), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tcx::fence_before();
  __syncthreads();
  tcx::fence_after();
  const uint32_t tmem = *tm;
  const uint32_t idesc = tcx::instr_desc_f16(1, WG_M, WG_N);
  const int64_t plane = (int64_t)a.H * a.W;
  bool ok = true;
  int issued = 0;
  for (int64_t g = g0; g < g1; ++g) {
    const int lc = (int)(g - g0), st = lc & 1;
    uint8_t *As = sm + st * WG_STAGE, *Bs = As + WG_A;
    if (lc >= 2 && !tcx::mbar_wait(bm(st), ((lc - 2) >> 1) & 1, CT_WAIT)) ok = false;
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    const int n = (int)(g / ((int64_t)a.H * spr));
    const int rem = (int)(g % ((int64_t)a.H * spr));
    const int y = rem / spr, x0 = (rem % spr) * WG_K;
    // A: output gradient, items (group of 8 pixels, channel); a quarter
    // warp stores 8 consecutive channels' 16-byte rows (one core matrix)
    for (int it = tid; it < WG_M * (WG_K / 8); it += 256) {
      const int co = it & (WG_M - 1), kg = it >> 7;
      float v[8];
      const bool cv = co0 + co < a.Cout;
      const float *src = a.gout + ((int64_t)n * a.Cout + co0 + co) * plane + (int64_t)y * a.W;
      float bsum = 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int x = x0 + kg * 8 + j;
        v[j] = (cv && x < a.W) ? __ldg(src + x) : 0.f;
        bsum += v[j];
      }
      if (do_bias && cv) atomicAdd(&gbs[co], bsum);
      *reinterpret_cast<uint4 *>(As + wg_off(co, kg * 8)) =
          make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                     pack_bf16x2(v[6], v[7]));
    }
    // B: items (input channel, row ky, group of 8 pixels); the ten input
    // pixels x0 - 1 + 8 kg .. x0 + 8 kg + 8 of row y + ky - 1 give the
    // group's 8 K elements of the three taps (ky, kx): element k = 8 kg + m
    // of tap kx is pixel x0 + k + kx - 1, i.e. the (m + kx)-th loaded value
    for (int it = tid; it < WG_N * 3 * (WG_K / 8); it += 256) {
      const int ci = it & (WG_N - 1), r = it >> 5;
      const int ky = r >> 3, kg = r & 7;
      const int yy = y + ky - 1;
      const bool rv = ci0 + ci < a.Cin && yy >= 0 && yy < a.H;
      const float *src = a.in + ((int64_t)n * a.Cin + ci0 + ci) * plane + (int64_t)yy * a.W;
      uint32_t hv[10];
#pragma unroll
      for (int j = 0; j < 10; ++j) {
        const int xx = x0 - 1 + kg * 8 + j;
        const float v = (rv && xx >= 0 && xx < a.W) ? __ldg(src + xx) : 0.f;
        hv[j] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
      }
#pragma unroll
      for (int kx = 0; kx < 3; ++kx)
        *reinterpret_cast<uint4 *>(Bs + (ky * 3 + kx) * WG_BT + wg_off(ci, kg * 8)) =
            make_uint4(hv[kx] | (hv[kx + 1] << 16), hv[kx + 2] | (hv[kx + 3] << 16),
                       hv[kx + 4] | (hv[kx + 5] << 16), hv[kx + 6] | (hv[kx + 7] << 16));
    }
    tcx::fence_proxy_async();
    tcx::fence_before();
    __syncthreads();
    tcx::fence_after();
    if (tid == 0) {
      const uint32_t a_base = tcx::smem_u32(As), b_base = tcx::smem_u32(Bs);
#pragma unroll 1
      for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int s4 = 0; s4 < WG_K / 16; ++s4)
          tcx::mma_f16(tmem + (uint32_t)(t * WG_N), tcx::smem_desc(a_base + s4 * 256, 128, 1024),
                       tcx::smem_desc(b_base + t * WG_BT + s4 * 256, 128, 1024), idesc,
                       (lc > 0 || s4 > 0) ? 1u : 0u);
      tcx::mma_commit(bm(st));
    }
    issued = lc + 1;
  }
  if (issued > 0) {
    const int last = issued - 1;
    if (!tcx::mbar_wait(bm(last & 1), (last >> 1) & 1, CT_WAIT)) ok = false;
  }
  ok = __syncthreads_and(ok);
  tcx::fence_after();
  if (ok && issued > 0) {
    // warp w: TMEM lanes 32 (w % 4) .. (output channels), half w / 4 of
    // the 9 x 32 columns
    const int q = warp & 3, h = warp >> 2;
    const int co = 32 * q + lane;
    const bool cv = co0 + co < a.Cout;
    for (int j = 0; j < 9; ++j) {
      const int c0 = h * 144 + j * 16;
      uint32_t v[16];
      tcx::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int c = c0 + u, t = c >> 5, ci = c & 31;
        if (cv && ci0 + ci < a.Cin)
          atomicAdd(&a.gw[((int64_t)(co0 + co) * a.Cin + ci0 + ci) * 9 + t], __uint_as_float(v[u]));
      }
    }
    if (do_bias && tid < WG_M && co0 + tid < a.Cout) atomicAdd(&a.gb[co0 + tid], gbs[tid]);
  } else if (!ok && tid == 0) {
    atomicOr(a.flag, 1);
  }
  tcx::fence_before();
  __syncthreads();
  if (warp == 0) tcx::tmem_dealloc(tmem, 512);
}

// Pack one layer's weights for k_conv3x3_tc: element (chunk c, tap t, plane
// cg, n, j) is B(n, k = 16 c + 8 cg + j) of tap t.  Forward: B = w[n][k][t];
// flipped (input gradient of the layer): B = w[k][n][8 - t].  Values are
// rounded to BF16; entries outside the channel counts are zero.
__global__ void k_pack_w(const float *__restrict__ w, int CinL, int CoutL, int flip, uint16_t *__restrict__ out,
                         int Npad, int nchunks) {
  const int Cin = flip ? CoutL : CinL, Cout = flip ? CinL : CoutL;
  const int64_t total = (int64_t)nchunks * 9 * 2 * Npad * 8;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % 8);
    const int nn = (int)((idx / 8) % Npad);
    const int cg = (int)((idx / (8 * Npad)) % 2);
    const int tap = (int)((idx / (16 * Npad)) % 9);
    const int c = (int)(idx / (144 * (int64_t)Npad));
    const int ci = c * 16 + cg * 8 + j;
    float v = 0.f;
    if (ci < Cin && nn < Cout) {
      if (!flip) v = w[((int64_t)nn * CinL + ci) * 9 + tap];
      else v = w[((int64_t)ci * CinL + nn) * 9 + (8 - tap)];
    }
    out[idx] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
}

}  // namespace

int nn_tc_npad(int Cout) { return (Cout + 15) / 16 * 16; }
int nn_tc_nchunks(int Cin) { return (Cin + 15) / 16; }
int64_t nn_tc_packed_elems(int Cin, int Cout) { return (int64_t)nn_tc_nchunks(Cin) * 9 * 2 * nn_tc_npad(Cout) * 8; }

cudaError_t nn_tc_setup() {
  const cudaError_t e =
      cudaFuncSetAttribute(k_conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * CT_ACT + 576 * 256 + 64);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_conv3x3_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM);
}

void nn_conv_wgrad_tc(const float *in, int Cin, const float *gout, int Cout, int N, int H, int W, float *gw,
                      float *gb, int *flag, cudaStream_t st) {
  WgradTcArgs a{in, gout, Cin, Cout, N, H, W, gw, gb, flag};
  const int cot = (Cout + WG_M - 1) / WG_M, cit = (Cin + WG_N - 1) / WG_N;
  const int64_t segs = (int64_t)N * H * ((W + WG_K - 1) / WG_K);
  const int64_t want = std::max<int64_t>(1, (2 * 152 + cot * cit - 1) / (cot * cit));
  const int ks = (int)std::max<int64_t>(1, std::min<int64_t>(segs, want));
  k_conv3x3_wgrad_tc<<<dim3(cot, cit, ks), 256, WG_SMEM, st>>>(a);
  count_launch();
}

void nn_pack_weights(const float *w, int CinL, int CoutL, bool flip, uint16_t *out, cudaStream_t st) {
  const int Cin = flip ? CoutL : CinL, Cout = flip ? CinL : CoutL;
  const int64_t total = nn_tc_packed_elems(Cin, Cout);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
  k_pack_w<<<grid, 256, 0, st>>>(w, CinL, CoutL, flip ? 1 : 0, out, nn_tc_npad(Cout), nn_tc_nchunks(Cin));
  count_launch();
}

int nn_tc_ksplit(int Cin, int Cout, int N, int H, int W) {
  const int tiles = ((W + CT_T - 1) / CT_T) * ((H + CT_T - 1) / CT_T) * N;
  const int nch = nn_tc_nchunks(Cin);
  if (tiles >= 76 || nch < 2) return 1;  // half a wave or more: no split
  return std::max(1, std::min(nch, 152 / tiles));
}

void nn_conv_tc(const float *in, int Cin, const uint16_t *wp, const float *bias, float *out, int Cout, int N, int H,
                int W, bool relu, int *flag, cudaStream_t st, float *part) {
  ConvTcArgs a;
  a.in = in;
  a.Cin = Cin;
  a.wp = wp;
  a.Npad = nn_tc_npad(Cout);
  a.nchunks = nn_tc_nchunks(Cin);
  a.bias = bias;
  a.out = out;
  a.Cout = Cout;
  a.H = H;
  a.W = W;
  a.relu = relu ? 1 : 0;
  a.flag = flag;
  a.part = nullptr;
  const int tiles = ((W + CT_T - 1) / CT_T) * ((H + CT_T - 1) / CT_T);
  const size_t smem = 2 * CT_ACT + 2 * 288 * (size_t)a.Npad + 64;
  const int ks = part ? nn_tc_ksplit(Cin, Cout, N, H, W) : 1;
  a.part = ks > 1 ? part : nullptr;
  k_conv3x3_tc<<<dim3(tiles, N, ks), 256, smem, st>>>(a);
  count_launch();
  if (ks > 1) {
    const int64_t count = (int64_t)N * Cout * H * W;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152 * 8));
    k_splitk_finish<<<grid, 256, 0, st>>>(part, ks, count, (int64_t)H * W, Cout, bias, relu ? 1 : 0, out);
    count_launch();
  }
}

}  // namespace stdd

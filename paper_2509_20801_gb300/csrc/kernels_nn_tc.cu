// Tensor-core (tcgen05) 3x3 convolutions of the learned-guess network: the
// forward pass, the input gradient (the same convolution with the weights
// transposed and flipped) and the weight gradient, as implicit GEMMs with
// BF16 operands and FP32 accumulation in TMEM.  The weight-gradient kernel
// is described at its definition; the rest of this header is about the
// forward kernel.
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
// while the MMAs of chunk c run, and the FP32 halo loads of chunk c+1 are
// issued before chunk c is converted.  When an image has too few tiles to
// fill the GPU, the chunks are split over CTAs (blockIdx.z); their partial
// sums go to a scratch buffer that k_splitk_finish adds in a fixed order
// with the bias and the activation.  Every wait has an iteration limit; a
// timeout sets the error flag and the CTA stops cleanly.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <stdexcept>

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
  // halo tile of 16 channels: items (plane cg, halo row, halo column), at
  // most CT_ITEMS per thread; the loads of chunk c + 1 are issued before
  // chunk c is converted and handed to the MMAs, so their latency overlaps
  // the wait for the stage, the conversion and the barrier
  float v[CT_ITEMS][8];
  auto load_halo = [&](int c) {
#pragma unroll
    for (int u = 0; u < CT_ITEMS; ++u) {
      const int it = tid + u * 256;
      const int cg = it / (CT_HP * CT_HP), r = it % (CT_HP * CT_HP);
      const int y = y0 - 1 + r / CT_HP, x = x0 - 1 + r % CT_HP;
      const bool ok_item = c < ce && it < 2 * CT_HP * CT_HP && y >= 0 && y < a.H && x >= 0 && x < a.W;
      const int ci0 = c * 16 + cg * 8;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[u][j] = (ok_item && ci0 + j < a.Cin) ? __ldg(inb + (int64_t)(ci0 + j) * plane + (int64_t)y * a.W + x)
                                               : 0.f;
    }
  };
  if (cb < ce) load_halo(cb);
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
    {
      uint32_t pk[CT_ITEMS][4];
#pragma unroll
      for (int u = 0; u < CT_ITEMS; ++u) {
        pk[u][0] = pack_bf16x2(v[u][0], v[u][1]);
        pk[u][1] = pack_bf16x2(v[u][2], v[u][3]);
        pk[u][2] = pack_bf16x2(v[u][4], v[u][5]);
        pk[u][3] = pack_bf16x2(v[u][6], v[u][7]);
      }
      if (c + 1 < ce) load_halo(c + 1);
#pragma unroll
      for (int u = 0; u < CT_ITEMS; ++u) {
        const int it = tid + u * 256;
        if (it < 2 * CT_HP * CT_HP) {
          const int cg = it / (CT_HP * CT_HP), r = it % (CT_HP * CT_HP);
          *reinterpret_cast<uint4 *>(act + cg * CT_PLANE + r * 16) = make_uint4(pk[u][0], pk[u][1], pk[u][2], pk[u][3]);
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
// channels, K = pixels.  A CTA walks down one 64-pixel column strip (columns
// x0 .. x0 + 63, past the row end zero) over a contiguous range of (image,
// row) steps; the CTAs of all strips of a row range run side by side, so the
// one-pixel halos they share are read from L2.  Per step the output-gradient
// row segment is the A tile, and the input rows y - 1 .. y + 1 come from a
// ring of four rows in shared memory, each stored in its three horizontal
// shifts (tap kx reads pixel x + kx - 1), so every input row is converted
// once per strip.  The FP32 rows arrive through a ring of D raw slots filled
// by cp.async D - 1 steps ahead (each thread copies and later converts the
// same 16-byte pieces, so only its own copies need to have landed); the
// conversion writes BF16 into the K-major operand tiles, whose K core
// matrices sit 144 bytes apart (a 16-byte pad that makes the 8-byte stores of
// a half warp hit 32 distinct banks).  Sixteen converter warps hand each
// row to a seventeenth warp through a "full" mbarrier; that warp issues the
// row's MMAs and commits them to an "empty" mbarrier, which the converters
// wait on two rows later before reusing the row's shared-memory slots (no
// CTA-wide barrier per row).  The nine accumulators (32 TMEM
// columns each) stay in TMEM; the epilogue adds them to gw with FP32 atomics
// (CTAs split the rows).  The three shifts of a ring row are contiguous, so
// the taps of one kernel row ky are a single MMA with N = 96.  The bias
// gradient (sum of gout) is summed from the FP32 values by the CTAs of the
// first input-channel tile.
constexpr int WG_M = 128, WG_N = 32, WG_K = 64;
constexpr int WG_T = 512, WG_RP = WG_T / 16;  // converter threads; rows per pass (16 threads per row)
constexpr int WG_THREADS = WG_T + 32;          // plus the MMA warp
constexpr int WG_LBO = 144, WG_SBO = 8 * WG_LBO;
constexpr int WG_A = (WG_M / 8) * WG_SBO;      // 18 KiB, one output-gradient row segment
constexpr int WG_BT = (WG_N / 8) * WG_SBO;     // 4.5 KiB, one input row in one shift
constexpr int WG_OPS = 2 * WG_A + 4 * 3 * WG_BT;
constexpr int WG_RAW_B = WG_N * WG_K * 4 + WG_N * 2 * 4;  // input row + its two halo pixels

template <int AROWS>
struct WgCfg {
  static constexpr int D = AROWS <= 32 ? 6 : 3;             // raw slots (prefetch depth D - 1)
  static constexpr int RAW = AROWS * WG_K * 4 + WG_RAW_B;   // one raw slot
  static constexpr int BAR = WG_OPS + D * RAW;
  static constexpr int SMEM = BAR + 64;
};
static_assert(WgCfg<128>::SMEM <= 227 * 1024 && WgCfg<32>::SMEM <= 227 * 1024, "weight-gradient smem");
static_assert(WgCfg<32>::SMEM > 114 * 1024, "one CTA per SM (each holds 512 TMEM columns)");

__device__ __forceinline__ uint32_t wg_off(int row, int k) {
  return (uint32_t)((row >> 3) * WG_SBO + (k >> 3) * WG_LBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint2 pack4_bf16(float a, float b, float c, float d) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  return make_uint2(*reinterpret_cast<const uint32_t *>(&lo), *reinterpret_cast<const uint32_t *>(&hi));
}

// cp.async of `bytes` (0 .. 16) valid bytes into a 16-byte slot, rest zero
__device__ __forceinline__ void cpa16(uint32_t dst, const void *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cpa4(uint32_t dst, const void *src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct WgradTcArgs {
  const float *in, *gout;
  int Cin, Cout, N, H, W;
  float *gw, *gb;
  int *flag;
  int cit, strips, chunks;
  int vec;  // rows 16-byte aligned (W % 4 == 0 and aligned bases)
};

template <int AROWS>
__global__ void __launch_bounds__(WG_THREADS, 1) k_conv3x3_wgrad_tc(WgradTcArgs a) {
  using C = WgCfg<AROWS>;
  constexpr int D = C::D, JA = AROWS / WG_RP, JB = WG_N / WG_RP;
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + C::BAR);  // empty[2] (MMA commits), full[2]
  uint32_t *tm = reinterpret_cast<uint32_t *>(bars + 4);
  int *mma_ok = reinterpret_cast<int *>(bars + 5);
  uint8_t *ring = sm + 2 * WG_A, *raw = sm + WG_OPS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = tid & 15, r16 = tid >> 4;
  const int co0 = (blockIdx.x / a.cit) * WG_M, ci0 = (blockIdx.x % a.cit) * WG_N;
  const int strip = blockIdx.y % a.strips, chunk = blockIdx.y / a.strips;
  const int x0 = strip * WG_K;
  const int64_t nh = (int64_t)a.N * a.H;
  const int64_t r0 = chunk * nh / a.chunks, r1 = (chunk + 1) * nh / a.chunks;
  const int steps = (int)(r1 - r0);
  const bool do_bias = a.gb && ci0 == 0;
  const int64_t plane = (int64_t)a.H * a.W;
  const uint32_t bar0 = tcx::smem_u32(&bars[0]), raw_s = tcx::smem_u32(raw);
  auto bm = [&](int st) { return bar0 + 8u * (uint32_t)st; };
  auto bf = [&](int st) { return bar0 + 16u + 8u * (uint32_t)st; };
  if (warp == 0) tcx::tmem_alloc(tcx::smem_u32(tm), 512);
  // A rows AROWS .. 127 stay zero in both slots
  if (AROWS < WG_M)
    for (int i = tid; i < 2 * WG_A / 16; i += WG_THREADS) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    tcx::mbar_init(bm(0), 1);
    tcx::mbar_init(bm(1), 1);
    tcx::mbar_init(bf(0), WG_T);
    tcx::mbar_init(bf(1), WG_T);
    *mma_ok = 1;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tcx::fence_before();
  __syncthreads();
  tcx::fence_after();
  const uint32_t tmem = *tm;
  const uint32_t idesc = tcx::instr_desc_f16(1, WG_M, 3 * WG_N);

  // this thread's pieces: output-gradient rows r16 + 32 j (j < JA) and input
  // rows r16 + 32 j (j < JB), pixels x0 + 4q .. x0 + 4q + 3, at image 0, row 0
  // (a step adds n * C * plane + y * W); invalid channels copy nothing
  const int xq = x0 + 4 * q;
  const int nbx = max(0, min(4, a.W - xq)) * 4;  // valid bytes of the piece
  const float *pa[JA];
  bool va[JA];
#pragma unroll
  for (int j = 0; j < JA; ++j) {
    va[j] = co0 + r16 + WG_RP * j < a.Cout;
    pa[j] = a.gout + (int64_t)(va[j] ? co0 + r16 + WG_RP * j : 0) * plane + xq;
  }
  const float *pb[JB];
  bool vb[JB];
#pragma unroll
  for (int j = 0; j < JB; ++j) {
    vb[j] = ci0 + r16 + WG_RP * j < a.Cin;
    pb[j] = a.in + (int64_t)(vb[j] ? ci0 + r16 + WG_RP * j : 0) * plane + xq;
  }
  const bool hl = q == 0 && x0 > 0, hr = q == 15 && x0 + WG_K < a.W;
  const int64_t cpa_stride = (int64_t)a.Cout * plane, cpb_stride = (int64_t)a.Cin * plane;
  // four pixels from p into a 16-byte raw slot, nb valid bytes, rest zero
  auto copy4 = [&](uint32_t dst, const float *p, int nb) {
    if (a.vec) {
      cpa16(dst, nb ? p : a.in, nb);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool ok = 4 * e < nb;
        cpa4(dst + 4 * e, ok ? p + e : a.in, ok ? 4 : 0);
      }
    }
  };
  // input row yb of image n into the B part of raw slot `slot`; halo pixels
  // x0 - 1 (by lane q = 0) and x0 + 64 (by lane q = 15)
  auto issue_b = [&](uint32_t slot, int n, int yb) {
    const bool rv = yb >= 0 && yb < a.H;
    const int64_t o = n * cpb_stride + (int64_t)(rv ? yb : 0) * a.W;
    const uint32_t b = slot + AROWS * WG_K * 4;
#pragma unroll
    for (int j = 0; j < JB; ++j) {
      const int ci = r16 + WG_RP * j;
      const bool v = rv && vb[j];
      copy4(b + (uint32_t)(ci * WG_K + 4 * q) * 4, pb[j] + o, v ? nbx : 0);
      const uint32_t h = b + WG_N * WG_K * 4 + (uint32_t)ci * 8;
      // lane 0's piece starts at x0, lane 15's at x0 + 60
      if (q == 0) cpa4(h, v && hl ? pb[j] + o - 1 : a.in, v && hl ? 4 : 0);
      if (q == 15) cpa4(h + 4, v && hr ? pb[j] + o + 4 : a.in, v && hr ? 4 : 0);
    }
  };
  auto issue = [&](int s, int n, int y) {
    const uint32_t slot = raw_s + (uint32_t)((s % D) * C::RAW);
    const int64_t o = n * cpa_stride + (int64_t)y * a.W;
#pragma unroll
    for (int j = 0; j < JA; ++j)
      copy4(slot + (uint32_t)((r16 + WG_RP * j) * WG_K + 4 * q) * 4, pa[j] + o, va[j] ? nbx : 0);
    issue_b(slot, n, y + 1);
  };
  // raw input row of `slot` (this thread's pieces) into ring row `rs`
  auto convert_b = [&](const uint8_t *slot, int rs) {
    const float *b = reinterpret_cast<const float *>(slot + AROWS * WG_K * 4);
#pragma unroll
    for (int j = 0; j < JB; ++j) {
      const int ci = r16 + WG_RP * j;
      const float4 v = *reinterpret_cast<const float4 *>(b + ci * WG_K + 4 * q);
      const float up = __shfl_up_sync(0xffffffffu, v.w, 1, 16);
      const float dn = __shfl_down_sync(0xffffffffu, v.x, 1, 16);
      const float *h = b + WG_N * WG_K + 2 * ci;
      const float left = q == 0 ? h[0] : up, right = q == 15 ? h[1] : dn;
      uint8_t *t = ring + rs * 3 * WG_BT + wg_off(ci, 4 * q);
      *reinterpret_cast<uint2 *>(t) = pack4_bf16(left, v.x, v.y, v.z);
      *reinterpret_cast<uint2 *>(t + WG_BT) = pack4_bf16(v.x, v.y, v.z, v.w);
      *reinterpret_cast<uint2 *>(t + 2 * WG_BT) = pack4_bf16(v.y, v.z, v.w, right);
    }
  };

  // cursors: (n, y) of the step being computed and of the step being fetched
  int n = (int)(r0 / a.H), y = (int)(r0 % a.H);
  int pn = n, py = y;
  float bsum[JA];
#pragma unroll
  for (int j = 0; j < JA; ++j) bsum[j] = 0.f;
  bool ok = true;
  int issued = 0;
  if (warp == WG_T / 32) {
    // the MMA warp: row lc's operands are complete when all converter
    // threads have arrived on full[lc & 1]
    if (lane == 0) {
      for (int lc = 0; lc < steps; ++lc) {
        if (!tcx::mbar_wait(bf(lc & 1), (lc >> 1) & 1, CT_WAIT)) {
          *mma_ok = 0;
          break;
        }
        tcx::fence_after();
        // the three shifts of a ring row are stored back to back, so one MMA
        // with N = 96 (rows kx * 32 + ci) covers the taps (ky, 0 .. 2), and
        // its accumulator columns ky * 96 + kx * 32 + ci are those of tap
        // 3 ky + kx
        const uint64_t ad = tcx::smem_desc(tcx::smem_u32(sm + (lc & 1) * WG_A), WG_LBO, WG_SBO);
        const uint64_t bd = tcx::smem_desc(tcx::smem_u32(ring), WG_LBO, WG_SBO);
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
          const uint64_t bt = bd + (uint64_t)(((((y + ky - 1) & 3) * 3) * WG_BT) >> 4);
#pragma unroll
          for (int s4 = 0; s4 < WG_K / 16; ++s4)
            tcx::mma_f16(tmem + (uint32_t)(ky * 3 * WG_N), ad + (uint64_t)(s4 * 2 * WG_LBO / 16),
                         bt + (uint64_t)(s4 * 2 * WG_LBO / 16), idesc, (lc > 0 || s4 > 0) ? 1u : 0u);
        }
        tcx::mma_commit(bm(lc & 1));
        if (++y == a.H) y = 0;
      }
    }
    __syncwarp();
    issued = steps;
  } else {
#pragma unroll
    for (int s = 0; s < D - 1; ++s) {
      if (s < steps) {
        issue(s, pn, py);
        if (++py == a.H) py = 0, ++pn;
      }
      cpa_commit();
    }
    for (int lc = 0; lc < steps; ++lc) {
      if (lc + D - 1 < steps) {
        issue(lc + D - 1, pn, py);
        if (++py == a.H) py = 0, ++pn;
      }
      cpa_commit();
      const bool restart = lc == 0 || y == 0;
      // the A slot and the ring slot written here were last read by step
      // lc - 2 (or, at a restart, by any earlier step); a warp leaves the
      // loop together when one of its lanes' waits timed out
      if (restart && lc >= 1) {
        if (!tcx::mbar_wait(bm((lc - 1) & 1), ((lc - 1) >> 1) & 1, CT_WAIT)) ok = false;
      } else if (lc >= 2) {
        if (!tcx::mbar_wait(bm(lc & 1), ((lc - 2) >> 1) & 1, CT_WAIT)) ok = false;
      }
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      if (restart) {
        // rows y - 1 and y through the slot of step lc + D - 1 (its copies
        // are issued again afterwards)
        const uint32_t spare = raw_s + (uint32_t)(((lc + D - 1) % D) * C::RAW);
        const uint8_t *sp = raw + ((lc + D - 1) % D) * C::RAW;
        if (lc + D - 1 < steps) {
          // the spare slot is in flight for step lc + D - 1: drain it first
          cpa_wait<0>();
        }
        issue_b(spare, n, y - 1);
        cpa_commit();
        cpa_wait<0>();
        convert_b(sp, (y - 1) & 3);
        issue_b(spare, n, y);
        cpa_commit();
        cpa_wait<0>();
        convert_b(sp, y & 3);
        if (lc + D - 1 < steps) {
          issue(lc + D - 1, n + (int)((y + D - 1) / a.H), (y + D - 1) % a.H);
          cpa_commit();
        }
      }
      cpa_wait<D - 1>();
      const uint8_t *slot = raw + (lc % D) * C::RAW;
      uint8_t *As = sm + (lc & 1) * WG_A;
#pragma unroll
      for (int j = 0; j < JA; ++j) {
        const int co = r16 + WG_RP * j;
        const float4 v = *reinterpret_cast<const float4 *>(slot + (co * WG_K + 4 * q) * 4);
        *reinterpret_cast<uint2 *>(As + wg_off(co, 4 * q)) = pack4_bf16(v.x, v.y, v.z, v.w);
        bsum[j] += (v.x + v.y) + (v.z + v.w);
      }
      convert_b(slot, (y + 1) & 3);
      // make the generic-proxy stores visible to the MMAs, then hand the row over
      tcx::fence_proxy_async();
      tcx::mbar_arrive(bf(lc & 1));
      issued = lc + 1;
      if (++y == a.H) y = 0, ++n;
    }
  }
  cpa_wait<0>();
  if (issued > 0) {
    const int last = issued - 1;
    if (!tcx::mbar_wait(bm(last & 1), (last >> 1) & 1, CT_WAIT)) ok = false;
  }
  ok = __syncthreads_and(ok && issued == steps) && *mma_ok;
  tcx::fence_after();
  if (ok && steps > 0 && warp < WG_T / 32) {
    if (do_bias) {
#pragma unroll
      for (int j = 0; j < JA; ++j) {
        float v = bsum[j];
#pragma unroll
        for (int o = 8; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 16);
        const int co = r16 + WG_RP * j;
        if (q == 0 && co0 + co < a.Cout) atomicAdd(&a.gb[co0 + co], v);
      }
    }
    // warp w: TMEM lanes 32 (w % 4) .. (output channels), the 16-column
    // groups w / 4, w / 4 + 4, ... of the 9 x 32 columns
    const int qw = warp & 3, h = warp >> 2;
    const int co = 32 * qw + lane;
    if (32 * qw < AROWS) {
      const bool cv = co0 + co < a.Cout;
      for (int jj = h; jj < 9 * WG_N / 16; jj += WG_T / 128) {
        const int c0 = jj * 16;
        uint32_t v[16];
        tcx::tmem_ld16(tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int c = c0 + u, t = c >> 5, ci = c & 31;
          if (cv && ci0 + ci < a.Cin)
            atomicAdd(&a.gw[((int64_t)(co0 + co) * a.Cin + ci0 + ci) * 9 + t], __uint_as_float(v[u]));
        }
      }
    }
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
  const cudaError_t e2 =
      cudaFuncSetAttribute(k_conv3x3_wgrad_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, WgCfg<32>::SMEM);
  if (e2 != cudaSuccess) return e2;
  return cudaFuncSetAttribute(k_conv3x3_wgrad_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              WgCfg<128>::SMEM);
}

int nn_num_sms() {
  static int n = 0;
  if (n == 0) {
    int d = 0, v = 0;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess ||
        v <= 0)
      throw std::runtime_error("cannot query the SM count");
    n = v;
  }
  return n;
}

void nn_conv_wgrad_tc(const float *in, int Cin, const float *gout, int Cout, int N, int H, int W, float *gw,
                      float *gb, int *flag, cudaStream_t st) {
  const int cot = (Cout + WG_M - 1) / WG_M, cit = (Cin + WG_N - 1) / WG_N;
  const int strips = (W + WG_K - 1) / WG_K;
  // one wave: every SM takes at most one CTA; the CTAs of one row range
  // cover all strips
  const int64_t nh = (int64_t)N * H;
  const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(nh, nn_num_sms() / (cot * cit * strips)));
  const int vec = (W % 4 == 0) && (reinterpret_cast<uintptr_t>(in) % 16 == 0) &&
                  (reinterpret_cast<uintptr_t>(gout) % 16 == 0);
  WgradTcArgs a{in, gout, Cin, Cout, N, H, W, gw, gb, flag, cit, strips, chunks, vec};
  const dim3 grid(cot * cit, strips * chunks);
  if (Cout <= 32)
    k_conv3x3_wgrad_tc<32><<<grid, WG_THREADS, WgCfg<32>::SMEM, st>>>(a);
  else
    k_conv3x3_wgrad_tc<128><<<grid, WG_THREADS, WgCfg<128>::SMEM, st>>>(a);
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

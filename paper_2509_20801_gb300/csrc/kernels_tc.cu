// Tensor-core (tcgen05, sm_103a) front updates for the mixed-precision path.
//
// The blocked Gauss-Jordan step adds C R to the trailing part of a front,
// C (m x 32) and R (32 x m) complex.  Here one CTA computes a 64 x 128 complex
// tile of C R as ONE real GEMM through the 2 x 2 real embedding
//     [Re; Im](C R) = [Cr -Ci; Ci Cr] [Rr; Ri]
// (M = 128 real rows, K = 64 real, N = 128), inputs rounded to BF16 or FP16
// after a power-of-two scaling per tile (exact, undone after the product;
// it keeps FP16 inside its range), products accumulated in FP32 in tensor
// memory (TMEM), and the tile added to the front in FP32.
//
// Operands are staged by the threads (they need the conversion) in the
// canonical no-swizzle K-major layout: 8 x 16-byte core matrices, element
// (row, k) at (row/8)*SBO + (k/8)*LBO + (row%8)*16 + (k%8)*2 bytes with
// LBO = 128 (K-adjacent core matrices) and SBO = 1024 (row-adjacent).  One
// thread issues the four K = 16 MMAs, commits them to an mbarrier, and all
// threads wait for it with an iteration limit; a timeout sets an error flag
// and skips the tile instead of hanging.  Each warp then reads its 32 TMEM
// lanes (32x32b shape) and updates its rows.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace stdd {

namespace {

constexpr int TC_MC = 64;            // complex rows per tile (128 real)
constexpr int TC_N = 128;            // complex columns per tile
constexpr int TC_KC = 32;            // complex K (one Gauss-Jordan block)
constexpr int TC_KR = 2 * TC_KC;     // real K
constexpr int TC_OPBYTES = 128 * TC_KR * 2;  // one operand: 128 rows x 64 halves = 16 KiB
constexpr uint32_t TC_TMEM_COLS = 128;
constexpr long long TC_WAIT_LIMIT = 1ll << 20;

using tcx::mbar_try_wait;
using tcx::mma_f16;
using tcx::smem_u32;
using tcx::tmem_ld32;

// byte offset of element (row, k) in an operand tile (K-major, no swizzle)
__device__ __forceinline__ uint32_t op_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) { return tcx::smem_desc(addr, 128, 1024); }

// kind::f16 instruction descriptor: D = F32, A = B = fmt (0 F16, 1 BF16),
// both K-major, M = 128, N = TC_N
__device__ __forceinline__ uint32_t instr_desc(int fmt) { return tcx::instr_desc_f16(fmt, 128, TC_N); }

template <int FMT> __device__ __forceinline__ uint16_t to_half_bits(float x) {
  if (FMT == 1) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
  return __half_as_ushort(__float2half_rn(x));
}

// power-of-two exponent e with |x| * 2^e in [1, 2) for the largest |x| (0 if x = 0)
__device__ __forceinline__ int scale_exp(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 0;
  int e;
  frexpf(amax, &e);  // amax = f * 2^e, f in [0.5, 1)
  return 1 - e;
}

// Shared state of one tile CTA (128 threads).
struct TileSmem {
  uint8_t A[TC_OPBYTES];
  uint8_t B[TC_OPBYTES];
  unsigned long long mbar;
  uint32_t tmem;
  float red[8];
};

// One 64 x 128 complex tile D = C R on the tensor cores.  cload(rr, j) gives
// C(rr, j), rload(cc, j) gives R(j, cc) (zero outside the tile); sink(rr, cc,
// comp, v) receives component comp (0 re, 1 im) of D(rr, cc).  Returns false
// if the completion wait timed out.
template <int FMT, typename CLoad, typename RLoad, typename Sink>
__device__ bool tc_tile(TileSmem &sm, int kc, CLoad cload, RLoad rload, Sink sink) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&sm.tmem)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.mbar)));
  // per-tile power-of-two scales from the largest component of C and R
  float ma = 0.f, mb = 0.f;
  for (int idx = tid; idx < TC_MC * kc; idx += 128) {
    const float2 v = cload(idx % TC_MC, idx / TC_MC);
    ma = fmaxf(ma, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int idx = tid; idx < TC_N * kc; idx += 128) {
    const float2 v = rload(idx % TC_N, idx / TC_N);
    mb = fmaxf(mb, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  }
  if (lane == 0) {
    sm.red[warp] = ma;
    sm.red[4 + warp] = mb;
  }
  __syncthreads();
  const int ea = scale_exp(fmaxf(fmaxf(sm.red[0], sm.red[1]), fmaxf(sm.red[2], sm.red[3])));
  const int eb = scale_exp(fmaxf(fmaxf(sm.red[4], sm.red[5]), fmaxf(sm.red[6], sm.red[7])));
  // stage the embedded operands: A row 2rr = [Cr, -Ci], row 2rr+1 = [Ci, Cr];
  // B row cc (K-major) = [Rr, Ri] per complex k
  for (int idx = tid; idx < TC_MC * TC_KC; idx += 128) {
    const int rr = idx % TC_MC, j = idx / TC_MC;
    float2 v = j < kc ? cload(rr, j) : make_float2(0.f, 0.f);
    v.x = ldexpf(v.x, ea);
    v.y = ldexpf(v.y, ea);
    const uint16_t re = to_half_bits<FMT>(v.x), im = to_half_bits<FMT>(v.y), nim = to_half_bits<FMT>(-v.y);
    *reinterpret_cast<uint16_t *>(sm.A + op_off(2 * rr, 2 * j)) = re;
    *reinterpret_cast<uint16_t *>(sm.A + op_off(2 * rr, 2 * j + 1)) = nim;
    *reinterpret_cast<uint16_t *>(sm.A + op_off(2 * rr + 1, 2 * j)) = im;
    *reinterpret_cast<uint16_t *>(sm.A + op_off(2 * rr + 1, 2 * j + 1)) = re;
  }
  for (int idx = tid; idx < TC_N * TC_KC; idx += 128) {
    const int cc = idx % TC_N, j = idx / TC_N;
    float2 v = j < kc ? rload(cc, j) : make_float2(0.f, 0.f);
    *reinterpret_cast<uint16_t *>(sm.B + op_off(cc, 2 * j)) = to_half_bits<FMT>(ldexpf(v.x, eb));
    *reinterpret_cast<uint16_t *>(sm.B + op_off(cc, 2 * j + 1)) = to_half_bits<FMT>(ldexpf(v.y, eb));
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = sm.tmem;
  if (tid == 0) {
    const uint32_t idesc = instr_desc(FMT);
    const uint32_t a0 = smem_u32(sm.A), b0 = smem_u32(sm.B);
#pragma unroll
    for (int s = 0; s < TC_KR / 16; ++s)
      mma_f16(tmem, smem_desc(a0 + s * 256), smem_desc(b0 + s * 256), idesc, s > 0 ? 1u : 0u);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(&sm.mbar))
                 : "memory");
  }
  bool done = false;
  for (long long it = 0; it < TC_WAIT_LIMIT && !done; ++it) done = mbar_try_wait(smem_u32(&sm.mbar), 0);
  done = __all_sync(0xffffffffu, done);   // the TMEM reads below are warp-collective
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (done) {
    const float inv = ldexpf(1.f, -(ea + eb));
    const int drow = warp * 32 + lane;       // D row = TMEM lane
    const int rr = drow >> 1, comp = drow & 1;
    for (int c0 = 0; c0 < TC_N; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int u = 0; u < 32; ++u) sink(rr, c0 + u, comp, __uint_as_float(v[u]) * inv);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS));
  return done;
}

// element addressing of the front layout (see kernels_mf.cu)
__device__ __forceinline__ float2 *front_ptr(const MfArgs &a, const FrontDev &f, int r, int c) {
  const int p = f.p, b = f.b, n = p + b;
  float2 *fac = reinterpret_cast<float2 *>(a.fac);
  if (r < p) return fac + f.fac_off + (int64_t)c * p + r;
  if (c < p) return fac + f.fac_off + (int64_t)p * n + (int64_t)c * b + (r - p);
  return reinterpret_cast<float2 *>(a.ws_cur) + f.s_off + (int64_t)(c - p) * b + (r - p);
}
__device__ __forceinline__ int unband_tc(int i, int k, int nbk) { return i < k ? i : i + nbk; }

// Gauss-Jordan step k of every large front: A(r, c) += C'(r, band) R(band, c)
// for r, c outside the pivot band, C' the (already scaled) column panel and R
// the (not yet scaled) row panel.  grid = (fronts, 64 x 128 tiles).
template <int FMT>
__global__ void __launch_bounds__(128) mf_gj_update_tc(MfArgs a, int f0, int k) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TileSmem &sm = *reinterpret_cast<TileSmem *>(smem_raw);
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(MF_NB, p - k);
  const int m = n - nbk;
  const int nti = (m + TC_MC - 1) / TC_MC, ntj = (m + TC_N - 1) / TC_N;
  if ((int)blockIdx.y >= nti * ntj) return;
  const int i0 = (blockIdx.y % nti) * TC_MC, j0 = (blockIdx.y / nti) * TC_N;
  auto cload = [&](int rr, int j) -> float2 {
    const int ri = i0 + rr;
    return ri < m ? *front_ptr(a, f, unband_tc(ri, k, nbk), k + j) : make_float2(0.f, 0.f);
  };
  auto rload = [&](int cc, int j) -> float2 {
    const int ci = j0 + cc;
    return ci < m ? *front_ptr(a, f, k + j, unband_tc(ci, k, nbk)) : make_float2(0.f, 0.f);
  };
  auto sink = [&](int rr, int cc, int comp, float v) {
    const int ri = i0 + rr, ci = j0 + cc;
    if (ri < m && ci < m) {
      float *e = reinterpret_cast<float *>(front_ptr(a, f, unband_tc(ri, k, nbk), unband_tc(ci, k, nbk)));
      e[comp] += v;
    }
  };
  if (!tc_tile<FMT>(sm, nbk, cload, rload, sink) && threadIdx.x == 0) atomicOr(a.flag, 2);
}

// ===================================================== FP64 on BF16 units
// The complex128 front update C R (C: 64 x kc, R: kc x 64, kc <= 32) on the
// BF16 tensor cores with FP64 accuracy, by exact splitting (the scheme of
// Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012) 95-118): every
// real row of the 2 x 2 embedding of C and every real column of R is scaled
// by a power of two 2^-e (|x| < 2^e over the row / column) and cut into
// OZ_S = 8 fixed-point slices of 7 bits,
//     x = 2^e sum_{i<8} a_i 2^(-7 (i + 1)),   a_i integer, |a_i| <= 127,
// each exactly a BF16 number.  A product of two slices is an integer below
// 2^14 in modulus, a K = 64 dot product of them below 2^20, and the sum of
// the g + 1 slice products of one order g = i + j (at most 8) below 2^23:
// all exact in the FP32 accumulators.  Orders g = 0..7 keep everything down
// to 2^-63 relative to the row and column scales (the dropped orders weigh
// less than 2^-53 of them, as in an FP64 dot product's error bound), each
// order summed in its own TMEM accumulator (8 x 64 columns = the SM's 512)
// by its 4 (g + 1) MMAs of K = 16.  The eight FP32 sums, exact integers, are
// combined in 64-bit integer arithmetic and rounded to FP64 once:
//     hi = sum_{g<4} G_g 2^(7 (3 - g)),   lo = sum_{g>=4} G_g 2^(7 (7 - g)),
//     V = hi 2^20 + floor(lo / 2^8),      value = V 2^(eA + eB - 55).
// Only the epilogue's add to the front uses the FP64 pipe.
constexpr int OZ_S = 8;                      // slices per operand value
constexpr int OZ_MR = 64;                    // complex rows per CTA (128 real rows, M = 128)
constexpr int OZ_NC = 32;                    // complex columns per sub-tile (N = 32)
constexpr int OZ_CHUNK = 16;                 // sub-tiles per CTA at most
constexpr int OZ_ABYTES = 128 * 64 * 2;      // one A slice: 128 real rows x 64 real K, BF16
constexpr int OZ_BBYTES = OZ_NC * 64 * 2;    // one B slice: 32 columns x 64 real K, BF16
constexpr uint32_t OZ_TMEM_COLS = 512;       // 2 buffers x 8 accumulators x 32 columns
constexpr int OZ_EMPTY = -2000;              // exponent of an all-zero row or column
constexpr int OZ_WORKERS = 256;              // 8 warps stage and read out (w and w + 4: TMEM lanes 32 (w % 4))
constexpr int OZ_THREADS = OZ_WORKERS + 32;  // plus one warp that issues the MMAs
constexpr int OZ_SINK = 8;                   // columns a thread reads out at a time

// One CTA: the 64 rows of C against up to OZ_CHUNK sub-tiles of 32 columns
// of R.  C's slices stay in shared memory; R's are staged per sub-tile into
// one of two buffers, and the MMAs of a sub-tile (into one of two TMEM
// halves) run while the threads read out the previous sub-tile's sums.
struct OzSmem {
  uint8_t A[OZ_S][OZ_ABYTES];
  uint8_t B[2][OZ_S][OZ_BBYTES];
  int eA[OZ_MR];
  int eB[2][OZ_NC];
  int red[OZ_WORKERS];
  unsigned long long bfull[2], tfull[2], tempty[2];
  uint32_t tmem;
  int bad;          // bit 0: non-finite operand, bit 1: a completion wait gave up
};

// frexp exponent of x (|x| < 2^e) from its bits; OZ_EMPTY for zero and
// subnormals (below every scale that matters here), 1025 for inf / NaN
__device__ __forceinline__ int oz_exp(double x) {
  const int ef = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return ef == 0 ? OZ_EMPTY : ef - 1022;
}

// the 8 slices of x / 2^er (|x| < 2^er) as BF16 bit patterns: the 56-bit
// fixed-point magnitude Y = floor(|x| 2^(56 - er)) cut into 7-bit chunks
// from the top, each converted exactly (2^23 + c - 2^23 in FP32, whose low
// 16 bits are zero for c < 128), with the sign of x
__device__ __forceinline__ void oz_slice(double x, int er, uint32_t (&s)[OZ_S]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ef = (int)((u >> 52) & 0x7ff);
  unsigned long long Y = 0;
  if (ef != 0 && ef != 0x7ff) {
    const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // |x| = M 2^(ef - 1075)
    const int sh = er - (ef - 1022) - 3;                                   // Y = M 2^-sh, sh >= -3
    Y = sh >= 0 ? (sh < 64 ? M >> sh : 0ull) : M << (-sh);
  }
  const uint32_t sgn = (uint32_t)(u >> 63) << 15;
#pragma unroll
  for (int i = 0; i < OZ_S; ++i) {
    const int c = (int)((Y >> (49 - 7 * i)) & 127);
    const float f = __int_as_float(0x4B000000 | c) - 8388608.0f;
    s[i] = (__float_as_uint(f) >> 16) | sgn;
  }
}

// barrier over the 8 staging / read-out warps only (the MMA warp runs on)
__device__ __forceinline__ void worker_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(OZ_WORKERS) : "memory"); }

// V 2^e as a double: one rounding of V (|V| < 2^62), then the exact power of
// two added to the exponent field (values below the normal range flush to 0)
__device__ __forceinline__ double oz_value(long long V, int e) {
  if (V == 0) return 0.0;
  const long long b = __double_as_longlong(__ll2double_rn(V));
  const int ef = (int)((b >> 52) & 0x7ff) + e;
  if (ef <= 0) return 0.0;
  if (ef >= 2047) return __longlong_as_double((b & (long long)(1ull << 63)) | 0x7ff0000000000000ll);
  return __longlong_as_double(b + ((long long)e << 52));
}

// C R for the 64 rows of C and the columns [0, ncols) of R (ncols <= 32 OZ_CHUNK):
// cload(rr, j) = C(rr, j), rload(cc, j) = R(j, cc) for j < kc (zero where
// the matrix ends); sink(rr, c0, comp, produce) receives component comp of
// (C R)(rr, c0 + u), u < OZ_SINK, as add[u] from produce(add) (called once,
// after the sink has issued the loads it needs).  Returns the OzSmem::bad bits.
template <typename CLoad, typename RLoad, typename Sink>
__device__ int oz_rows(OzSmem &sm, int kc, int ncols, CLoad cload, RLoad rload, Sink sink) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (warp == 0) tcx::tmem_alloc(smem_u32(&sm.tmem), OZ_TMEM_COLS);
  if (t == 0) {
    for (int b = 0; b < 2; ++b) {
      tcx::mbar_init(smem_u32(&sm.bfull[b]), OZ_WORKERS);
      tcx::mbar_init(smem_u32(&sm.tfull[b]), 1);
      tcx::mbar_init(smem_u32(&sm.tempty[b]), OZ_WORKERS);
    }
    sm.bad = 0;
  }
  // ---- A = the embedded C: real row 2rr = [Cr, -Ci], 2rr + 1 = [Ci, Cr]
  if (t < OZ_WORKERS) {
    const int rr = t & 63, quarter = t >> 6;   // pivots [8 quarter, 8 quarter + 8) of row rr
    double2 v[8];
    int em = OZ_EMPTY;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = 8 * quarter + q;
      v[q] = j < kc ? cload(rr, j) : make_double2(0.0, 0.0);
      em = max(em, max(oz_exp(v[q].x), oz_exp(v[q].y)));
    }
    sm.red[t] = em;
    worker_sync();
    const int er = max(max(sm.red[rr], sm.red[rr + 64]), max(sm.red[rr + 128], sm.red[rr + 192]));
    if (quarter == 0) sm.eA[rr] = er;
    if (er > 1024) sm.bad = 1;
#pragma unroll
    for (int q0 = 0; q0 < 8; q0 += 4) {
      uint32_t re[4][OZ_S], im[4][OZ_S];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        oz_slice(v[q0 + q].x, er, re[q]);
        oz_slice(v[q0 + q].y, er, im[q]);
      }
      const int k0 = 2 * (8 * quarter + q0);   // real K of this 16-byte chunk (a multiple of 8)
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) {
        uint4 w0, w1;
        w0.x = re[0][i] | ((im[0][i] ^ 0x8000u) << 16);
        w0.y = re[1][i] | ((im[1][i] ^ 0x8000u) << 16);
        w0.z = re[2][i] | ((im[2][i] ^ 0x8000u) << 16);
        w0.w = re[3][i] | ((im[3][i] ^ 0x8000u) << 16);
        w1.x = im[0][i] | (re[0][i] << 16);
        w1.y = im[1][i] | (re[1][i] << 16);
        w1.z = im[2][i] | (re[2][i] << 16);
        w1.w = im[3][i] | (re[3][i] << 16);
        *reinterpret_cast<uint4 *>(sm.A[i] + op_off(2 * rr, k0)) = w0;
        *reinterpret_cast<uint4 *>(sm.A[i] + op_off(2 * rr + 1, k0)) = w1;
      }
    }
  }
  const int nsub = (ncols + OZ_NC - 1) / OZ_NC;
  const uint32_t idesc = tcx::instr_desc_f16(1, 128, OZ_NC);
  const int drow = (warp & 3) * 32 + lane, er = drow >> 1, comp = drow & 1;
  const int hsel = warp >> 2;   // warps 0-3 read columns 0-15 of a sub-tile, warps 4-7 columns 16-31
  // read out sub-tile s: the 8 order sums of 16 columns at a time
  auto drain = [&](int s) {
    const int buf = s & 1;
    // one decision per warp: the reads below are warp-collective
    const bool ok = __all_sync(0xffffffffu,
                               tcx::mbar_wait(smem_u32(&sm.tfull[buf]), (uint32_t)((s >> 1) & 1), TC_WAIT_LIMIT));
    tcx::fence_after();
    if (!ok && lane == 0) atomicOr(&sm.bad, 2);
    if (!ok || (__shfl_sync(0xffffffffu, sm.bad, 0) & 1)) return;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int h = 16 * hsel + OZ_SINK * pass;
      // the sink loads what it adds to first, then asks for the values
      auto produce = [&](double (&add)[OZ_SINK]) {
        // pairs of orders first, in 32 bits: G_2q 2^7 + G_2q+1 stays below 2^31
        int pr[4][OZ_SINK];
#pragma unroll
        for (int g = 0; g < OZ_S; ++g) {
          uint32_t vv[OZ_SINK];
          tcx::tmem_ld8(sm.tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(256 * buf + OZ_NC * g + h), vv);
#pragma unroll
          for (int u = 0; u < OZ_SINK; ++u) {
            const int G = __float2int_rn(__uint_as_float(vv[u]));
            if (g & 1) pr[g >> 1][u] += G;
            else pr[g >> 1][u] = G * 128;
          }
        }
#pragma unroll
        for (int u = 0; u < OZ_SINK; ++u) {
          const long long hi = (long long)pr[0][u] * (1ll << 14) + pr[1][u];
          const long long lo = (long long)pr[2][u] * (1ll << 14) + pr[3][u];
          add[u] = oz_value(hi * (1ll << 20) + (lo >> 8), sm.eA[er] + sm.eB[buf][h + u] - 55);
        }
      };
      sink(er, OZ_NC * s + h, comp, produce);
    }
  };
  tcx::fence_proxy_async();
  __syncthreads();   // A staged, barriers initialised, TMEM allocated
  if (warp == OZ_WORKERS / 32) {
    // ---- the MMA warp: sub-tile s once its B slices are staged and its
    // TMEM half has been read out (sub-tile s - 2)
    if (lane == 0) {
#pragma unroll 1
      for (int s = 0; s < nsub; ++s) {
        const int buf = s & 1;
        bool ok = tcx::mbar_wait(smem_u32(&sm.bfull[buf]), (uint32_t)((s >> 1) & 1), TC_WAIT_LIMIT);
        if (ok && s >= 2)
          ok = tcx::mbar_wait(smem_u32(&sm.tempty[buf]), (uint32_t)(((s - 2) >> 1) & 1), TC_WAIT_LIMIT);
        if (!ok) {
          atomicOr(&sm.bad, 2);
          break;
        }
        tcx::fence_after();
        const uint32_t dcol = sm.tmem + (uint32_t)(256 * buf);
        const uint64_t da = smem_desc(smem_u32(sm.A[0])), db = smem_desc(smem_u32(sm.B[buf][0]));
#pragma unroll 1
        for (int g = 0; g < OZ_S; ++g) {
#pragma unroll 1
          for (int i = 0; i <= g; ++i) {
            // descriptor start fields advance by address / 16: a slice of A
            // is 16 KiB, of B 4 KiB, a K step of 16 is 256 bytes
            const uint64_t a0 = da + (uint64_t)(i * (OZ_ABYTES >> 4)), b0 = db + (uint64_t)((g - i) * (OZ_BBYTES >> 4));
#pragma unroll
            for (int k = 0; k < 4; ++k)
              tcx::mma_f16(dcol + (uint32_t)(OZ_NC * g), a0 + (uint64_t)(16 * k), b0 + (uint64_t)(16 * k), idesc,
                           (i == 0 && k == 0) ? 0u : 1u);
          }
        }
        tcx::mma_commit(smem_u32(&sm.tfull[buf]));
      }
    }
    __syncwarp();
  } else {
    const int cc = t & 31, oct = t >> 5;   // B staging: pivots [4 oct, 4 oct + 4) of column cc
    double2 vn[4];                          // the next sub-tile's values, loaded ahead
    auto load_b = [&](int s) {
      const int col = OZ_NC * s + cc;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = 4 * oct + q;
        vn[q] = (j < kc && col < ncols) ? rload(col, j) : make_double2(0.0, 0.0);
      }
    };
    if (nsub > 0) load_b(0);
#pragma unroll 1
    for (int s = 0; s < nsub; ++s) {
      const int buf = s & 1;
      // ---- B(s): 32 columns as rows of K = [Rr, Ri] per pivot (its buffer
      // was last read by the MMAs of s - 2, finished before drain(s - 2))
      {
        double2 v[4];
        int em = OZ_EMPTY;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          v[q] = vn[q];
          em = max(em, max(oz_exp(v[q].x), oz_exp(v[q].y)));
        }
        worker_sync();                 // red is free (A's reduction, or the previous B's)
        sm.red[t] = em;
        worker_sync();
        int ec = sm.red[cc];
#pragma unroll
        for (int o = 1; o < 8; ++o) ec = max(ec, sm.red[cc + 32 * o]);
        if (oct == 0) sm.eB[buf][cc] = ec;
        if (ec > 1024) sm.bad = 1;
        uint32_t re[4][OZ_S], im[4][OZ_S];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          oz_slice(v[q].x, ec, re[q]);
          oz_slice(v[q].y, ec, im[q]);
        }
        const int k0 = 8 * oct;
#pragma unroll
        for (int i = 0; i < OZ_S; ++i) {
          uint4 w;
          w.x = re[0][i] | (im[0][i] << 16);
          w.y = re[1][i] | (im[1][i] << 16);
          w.z = re[2][i] | (im[2][i] << 16);
          w.w = re[3][i] | (im[3][i] << 16);
          *reinterpret_cast<uint4 *>(sm.B[buf][i] + op_off(cc, k0)) = w;
        }
      }
      tcx::fence_proxy_async();
      tcx::mbar_arrive(smem_u32(&sm.bfull[buf]));
      if (s + 1 < nsub) load_b(s + 1);   // in flight during the read-out below
      if (s > 0) {
        drain(s - 1);
        tcx::fence_before();
        tcx::mbar_arrive(smem_u32(&sm.tempty[(s - 1) & 1]));
      }
    }
    if (nsub > 0) drain(nsub - 1);
  }
  if (nsub > 0 && (sm.bad & 2) && t == 0)   // let issued MMAs finish before TMEM is freed
    tcx::mbar_wait(smem_u32(&sm.tfull[(nsub - 1) & 1]), (uint32_t)(((nsub - 1) >> 1) & 1), TC_WAIT_LIMIT);
  tcx::fence_before();
  __syncthreads();
  if (warp == 0) tcx::tmem_dealloc(sm.tmem, OZ_TMEM_COLS);
  return sm.bad;
}

__device__ __forceinline__ double2 *front_ptr64(const MfArgs &a, const FrontDev &f, int r, int c) {
  const int p = f.p, b = f.b, n = p + b;
  double2 *fac = reinterpret_cast<double2 *>(a.fac);
  if (r < p) return fac + f.fac_off + (int64_t)c * p + r;
  if (c < p) return fac + f.fac_off + (int64_t)p * n + (int64_t)c * b + (r - p);
  return reinterpret_cast<double2 *>(a.ws_cur) + f.s_off + (int64_t)(c - p) * b + (r - p);
}

// Symmetric form, step k of every large front on the tensor cores: the
// trailing update on and below the diagonal (rows and columns in the order
// that skips the pivot band), lower entries added to the front and their
// signed mirrors stored, as mf_gj_update_sym does on the FP64 pipe.  CTA
// (front, ti, chunk): rows [64 ti, 64 ti + 64) against the chunk's columns
// (at most 32 OZ_CHUNK) up to the diagonal.  grid = (fronts, tile rows x chunks).
__global__ void __launch_bounds__(OZ_THREADS, 1) mf_gj_update_oz(MfArgs a, int f0, int k, int nchunk) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  OzSmem &sm = *reinterpret_cast<OzSmem *>(smem_raw);
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(MF_NB, p - k);
  const int m = n - nbk;
  const int ti = blockIdx.y / nchunk, ch = blockIdx.y - ti * nchunk;
  const int i0 = ti * OZ_MR;
  const int c0 = ch * OZ_NC * OZ_CHUNK;
  const int cend = min(min(i0 + OZ_MR, m), c0 + OZ_NC * OZ_CHUNK);
  if (i0 >= m || c0 >= cend) return;
  const double2 *fac = reinterpret_cast<const double2 *>(a.fac);
  const int64_t fo = f.fac_off;
  auto cload = [&](int rr, int j) -> double2 {
    const int ri = i0 + rr;
    return ri < m ? *front_ptr64(a, f, unband_tc(ri, k, nbk), k + j) : make_double2(0.0, 0.0);
  };
  auto rload = [&](int cc, int j) -> double2 {
    return fac[fo + (int64_t)unband_tc(c0 + cc, k, nbk) * p + k + j];
  };
  // element (r, c) of the front as a double pointer, component comp:
  // column c < p or >= p picks the region, then base + c * stride
  const int b = f.b;
  double *facd = reinterpret_cast<double *>(a.fac), *wsd = reinterpret_cast<double *>(a.ws_cur);
  auto sink = [&](int rr, int cb, int comp, auto &&produce) {
    // produce() reads tensor memory with warp-collective loads: every lane
    // calls it, rows past the front only skip their loads and stores
    const int ri = i0 + rr;
    const bool rowok = ri < m;
    const int r = rowok ? unband_tc(ri, k, nbk) : 0;
    // (r, c): r < p: [Finv H12] column-major, ld p; r >= p: -G21 (c < p,
    // ld b) or S (c >= p, ld b, in the level workspace)
    double *dlo, *dhi;
    int64_t slo, shi;
    // (c, r), the mirror: c < p: row c of [Finv H12] at column r; c >= p:
    // -G21 (r < p) or S (r >= p) at row c - p
    double *mlo, *mhi;
    if (r < p) {
      dlo = dhi = facd + 2 * (fo + r) + comp;
      slo = shi = 2 * (int64_t)p;
      mhi = facd + 2 * (fo + (int64_t)p * n + (int64_t)r * b - p) + comp;
    } else {
      dlo = facd + 2 * (fo + (int64_t)p * n + (r - p)) + comp;
      dhi = wsd + 2 * (f.s_off + (r - p) - (int64_t)p * b) + comp;
      slo = shi = 2 * (int64_t)b;
      mhi = wsd + 2 * (f.s_off + (int64_t)(r - p) * b - p) + comp;
    }
    mlo = facd + 2 * (fo + (int64_t)r * p) + comp;
    double *px[OZ_SINK];
    double old[OZ_SINK];
#pragma unroll
    for (int u = 0; u < OZ_SINK; ++u) {
      const int ci = c0 + cb + u;
      px[u] = nullptr;
      if (rowok && ci < cend && ci <= ri) {
        const int c = unband_tc(ci, k, nbk);
        px[u] = c < p ? dlo + c * slo : dhi + c * shi;
        old[u] = *px[u];
      }
    }
    double add[OZ_SINK];
    produce(add);
#pragma unroll
    for (int u = 0; u < OZ_SINK; ++u) {
      if (!px[u]) continue;
      const int ci = c0 + cb + u, c = unband_tc(ci, k, nbk);
      const double v = old[u] + add[u];
      *px[u] = v;
      if (ci < ri) {
        const long long flip = ((r < k) != (c < k)) ? (long long)(1ull << 63) : 0ll;
        *((c < p ? mlo : mhi) + 2 * c) = __longlong_as_double(__double_as_longlong(v) ^ flip);
      }
    }
  };
  const int bad = oz_rows(sm, nbk, cend - c0, cload, rload, sink);
  if (threadIdx.x == 0) {
    if (bad & 2) atomicOr(a.flag, 2);
    else if (bad & 1) atomicOr(a.flag, 1);
  }
}

// The column panel of step k on the tensor cores (symmetric form,
// complex128): C(r, band) <- -C(r, band) D^-1 for the rows r outside the
// pivot band, 64 rows per CTA, D^-1 (nbk x nbk, left in the band by
// mf_gj_diag) the single 32-column sub-tile.  Each CTA slices its rows into
// shared memory before any result is written, and CTAs own disjoint rows.
// grid = (fronts, row tiles).
__global__ void __launch_bounds__(OZ_THREADS, 1) mf_gj_col_oz(MfArgs a, int f0, int k) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  OzSmem &sm = *reinterpret_cast<OzSmem *>(smem_raw);
  const FrontDev f = a.fronts[f0 + blockIdx.x];
  const int p = f.p, n = p + f.b;
  if (n <= MF_SMALL || k >= p) return;
  const int nbk = min(MF_NB, p - k);
  const int m = n - nbk;
  const int i0 = blockIdx.y * OZ_MR;
  if (i0 >= m) return;
  const double2 *fac = reinterpret_cast<const double2 *>(a.fac);
  const int64_t fo = f.fac_off;
  auto cload = [&](int rr, int j) -> double2 {
    const int ri = i0 + rr;
    return ri < m ? *front_ptr64(a, f, unband_tc(ri, k, nbk), k + j) : make_double2(0.0, 0.0);
  };
  auto rload = [&](int cc, int j) -> double2 { return fac[fo + (int64_t)(k + cc) * p + k + j]; };
  auto sink = [&](int rr, int cb, int comp, auto &&produce) {
    double add[OZ_SINK];
    produce(add);   // every lane (warp-collective reads)
    const int ri = i0 + rr;
    if (ri >= m) return;
    const int r = unband_tc(ri, k, nbk);
#pragma unroll
    for (int u = 0; u < OZ_SINK; ++u) {
      const int cc = cb + u;
      if (cc < nbk) reinterpret_cast<double *>(front_ptr64(a, f, r, k + cc))[comp] = -add[u];
    }
  };
  const int bad = oz_rows(sm, nbk, nbk, cload, rload, sink);
  if (threadIdx.x == 0) {
    if (bad & 2) atomicOr(a.flag, 2);
    else if (bad & 1) atomicOr(a.flag, 1);
  }
}

// One tile D = C R in complex128 (C(rr, j) at j * 64 + rr, R(j, cc) at
// cc * kc + j, D(rr, cc) at cc * 64 + rr) through oz_rows.
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_tile_kernel(const double2 *C, const double2 *R, double2 *D, int kc,
                                                         int *flag) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  OzSmem &sm = *reinterpret_cast<OzSmem *>(smem_raw);
  auto cload = [&](int rr, int j) { return C[j * OZ_MR + rr]; };
  auto rload = [&](int cc, int j) { return R[cc * kc + j]; };
  auto sink = [&](int rr, int cb, int comp, auto &&produce) {
    double add[OZ_SINK];
    produce(add);
#pragma unroll
    for (int u = 0; u < OZ_SINK; ++u) reinterpret_cast<double *>(&D[(cb + u) * OZ_MR + rr])[comp] = add[u];
  };
  const int bad = oz_rows(sm, kc, OZ_MR, cload, rload, sink);
  if (threadIdx.x == 0 && bad) atomicOr(flag, (bad & 2) ? 2 : 1);
}

// One tile D = C R with C (64 x kc) and R (kc x 128) complex, column-major
// (C(rr, j) at j * 64 + rr, R(j, cc) at cc * kc + j, D(rr, cc) at cc * 64 + rr).
template <int FMT>
__global__ void __launch_bounds__(128) tc_tile_kernel(const float2 *C, const float2 *R, float2 *D, int kc,
                                                      int *flag) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TileSmem &sm = *reinterpret_cast<TileSmem *>(smem_raw);
  auto cload = [&](int rr, int j) { return C[j * TC_MC + rr]; };
  auto rload = [&](int cc, int j) { return R[cc * kc + j]; };
  auto sink = [&](int rr, int cc, int comp, float v) { reinterpret_cast<float *>(&D[cc * TC_MC + rr])[comp] = v; };
  if (!tc_tile<FMT>(sm, kc, cload, rload, sink) && threadIdx.x == 0) atomicOr(flag, 2);
}

}  // namespace

// 56 KiB per CTA keeps at most 4 tile CTAs on an SM: 4 x 128 TMEM columns
// = the SM's 512, so no allocation ever has to wait for another CTA
size_t tc_smem_bytes() { return std::max<size_t>(sizeof(TileSmem) + 1024, 56u << 10); }

template <int FMT> cudaError_t tc_setup_attributes_fmt() {
  cudaError_t e = cudaFuncSetAttribute(mf_gj_update_tc<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc_tile_kernel<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes());
}

size_t oz_smem_bytes() { return sizeof(OzSmem) + 1024; }

cudaError_t tc_setup_attributes() {
  cudaError_t e = tc_setup_attributes_fmt<0>();
  if (e != cudaSuccess) return e;
  e = tc_setup_attributes_fmt<1>();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mf_gj_update_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mf_gj_col_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(oz_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
}

void mf_oz_col_launch(const MfArgs &a, const LevelInfo &L, int k, cudaStream_t st) {
  const int m = L.max_n - std::min(MF_NB, std::max(1, L.max_p - k));
  const int nt = std::max(1, (m + OZ_MR - 1) / OZ_MR);
  mf_gj_col_oz<<<dim3(L.nf, nt), OZ_THREADS, oz_smem_bytes(), st>>>(a, L.f0, k);
  count_launch();
}

void mf_oz_update_launch(const MfArgs &a, const LevelInfo &L, int k, cudaStream_t st) {
  const int m = L.max_n - std::min(MF_NB, std::max(1, L.max_p - k));
  const int nt = std::max(1, (m + OZ_MR - 1) / OZ_MR);
  const int nchunk = std::max(1, (nt * OZ_MR + OZ_NC * OZ_CHUNK - 1) / (OZ_NC * OZ_CHUNK));
  mf_gj_update_oz<<<dim3(L.nf, nt * nchunk), OZ_THREADS, oz_smem_bytes(), st>>>(a, L.f0, k, nchunk);
  count_launch();
}

void mf_tc_update_launch(const MfArgs &a, const LevelInfo &L, int k, int fmt, cudaStream_t st) {
  const int m = L.max_n - std::min(MF_NB, std::max(1, L.max_p - k));
  const int tiles = std::max(1, ((m + TC_MC - 1) / TC_MC) * ((m + TC_N - 1) / TC_N));
  if (fmt == 1) mf_gj_update_tc<1><<<dim3(L.nf, tiles), 128, tc_smem_bytes(), st>>>(a, L.f0, k);
  else mf_gj_update_tc<0><<<dim3(L.nf, tiles), 128, tc_smem_bytes(), st>>>(a, L.f0, k);
  count_launch();
}

// One complex128 tile product through the exact-splitting tensor-core path
// (see oz_tile_kernel for the layouts); returns 0 on success, 1 if the device
// reported a timeout, 2 for a non-finite input, -1 on a CUDA error (*err).
int oz_tile_product(int kc, const double2 *C, const double2 *R, double2 *D, cudaError_t *err) {
  const size_t nc = (size_t)OZ_MR * kc, nr = (size_t)kc * OZ_MR, nd = (size_t)OZ_MR * OZ_MR;
  double2 *dC = nullptr, *dR = nullptr, *dD = nullptr;
  int *dflag = nullptr;
  *err = cudaSuccess;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && *err == cudaSuccess) *err = e;
    return e == cudaSuccess;
  };
  bool ok = ck(tc_setup_attributes()) && ck(cudaMalloc(&dC, std::max<size_t>(1, nc) * sizeof(double2))) &&
            ck(cudaMalloc(&dR, std::max<size_t>(1, nr) * sizeof(double2))) &&
            ck(cudaMalloc(&dD, nd * sizeof(double2))) && ck(cudaMalloc(&dflag, sizeof(int)));
  int flag = 0;
  if (ok) {
    ok = (nc == 0 || ck(cudaMemcpy(dC, C, nc * sizeof(double2), cudaMemcpyHostToDevice))) &&
         (nr == 0 || ck(cudaMemcpy(dR, R, nr * sizeof(double2), cudaMemcpyHostToDevice))) &&
         ck(cudaMemset(dD, 0, nd * sizeof(double2))) && ck(cudaMemset(dflag, 0, sizeof(int)));
  }
  if (ok) {
    oz_tile_kernel<<<1, OZ_THREADS, oz_smem_bytes()>>>(dC, dR, dD, kc, dflag);
    count_launch();
    ok = ck(cudaGetLastError()) && ck(cudaDeviceSynchronize()) &&
         ck(cudaMemcpy(D, dD, nd * sizeof(double2), cudaMemcpyDeviceToHost)) &&
         ck(cudaMemcpy(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost));
  }
  cudaFree(dC);
  cudaFree(dR);
  cudaFree(dD);
  cudaFree(dflag);
  if (!ok) return -1;
  return (flag & 2) ? 1 : ((flag & 1) ? 2 : 0);
}

// One tile product on the device from host arrays (see tc_tile_kernel for
// the layouts); returns 0 on success, 1 if the device reported a timeout,
// -1 on a CUDA error (*err).
int tc_tile_product(int fmt, int kc, const float2 *C, const float2 *R, float2 *D, cudaError_t *err) {
  const size_t nc = (size_t)TC_MC * kc, nr = (size_t)kc * TC_N, nd = (size_t)TC_MC * TC_N;
  float2 *dC = nullptr, *dR = nullptr, *dD = nullptr;
  int *dflag = nullptr;
  *err = cudaSuccess;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && *err == cudaSuccess) *err = e;
    return e == cudaSuccess;
  };
  bool ok = ck(tc_setup_attributes()) && ck(cudaMalloc(&dC, nc * sizeof(float2))) &&
            ck(cudaMalloc(&dR, nr * sizeof(float2))) && ck(cudaMalloc(&dD, nd * sizeof(float2))) &&
            ck(cudaMalloc(&dflag, sizeof(int)));
  int flag = 0;
  if (ok) {
    ok = ck(cudaMemcpy(dC, C, nc * sizeof(float2), cudaMemcpyHostToDevice)) &&
         ck(cudaMemcpy(dR, R, nr * sizeof(float2), cudaMemcpyHostToDevice)) &&
         ck(cudaMemset(dD, 0, nd * sizeof(float2))) && ck(cudaMemset(dflag, 0, sizeof(int)));
  }
  if (ok) {
    if (fmt == 1) tc_tile_kernel<1><<<1, 128, tc_smem_bytes()>>>(dC, dR, dD, kc, dflag);
    else tc_tile_kernel<0><<<1, 128, tc_smem_bytes()>>>(dC, dR, dD, kc, dflag);
    count_launch();
    ok = ck(cudaGetLastError()) && ck(cudaDeviceSynchronize()) &&
         ck(cudaMemcpy(D, dD, nd * sizeof(float2), cudaMemcpyDeviceToHost)) &&
         ck(cudaMemcpy(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost));
  }
  cudaFree(dC);
  cudaFree(dR);
  cudaFree(dD);
  cudaFree(dflag);
  if (!ok) return -1;
  return flag ? 1 : 0;
}

}  // namespace stdd

// Warm-start predictor for MFWH: a small convolutional network that maps a forcing f_m and
// its frequency omega_m to an initial iterate V_m^0 for GMRES (the learned warm start; the
// paper itself starts from zero).  L layers of 3 x 3 "same" convolutions (zero padding) with
// bias, ReLU after every layer but the last, images [B][C][H][W].
//
// Arithmetic: activations and weights in BF16, products accumulated in FP32 on the
// 5th-generation tensor cores (tcgen05.mma with the accumulator in tensor memory, operands in
// shared memory: an implicit GEMM whose rows are 128 consecutive pixels of the batch and whose
// reduction runs over (input channel, tap)), for the forward convolutions and the input
// gradients; gradients, master weights and the Adam state in FP32.  The weight gradient, a
// reduction over every pixel of the batch, runs on the FP32 CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "internal.h"
#include "mfwh.h"

namespace mfwh {
namespace {

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ---- 3 x 3 convolution as an implicit GEMM on the 5th-generation tensor cores ----------
// D[p][n] = sum_k A[p][k] B[n][k] with p a pixel, n an output channel and k the position of
// (input channel ci, tap = dy * 3 + dx) in the order of conv_kidx below: A[p][k] =
// in[ci][y + dy - 1][x + dx - 1] (zero outside the image), B[n][k] = Wk[n][k].  A CTA of 128
// threads takes 128 consecutive pixels of the batch (M = 128) and all output channels (N = 16
// or 32, rows past Cout zero).  K is taken in passes, one group of GC = 8 or 16 input channels
// per pass.  Each pass first copies the image rows that the CTA's pixels and their vertical
// neighbours touch, for its channel group, from global into shared memory, channel innermost;
// then each thread builds its pixel's row of A from that copy, one tap of 8 channels (one
// 16-byte load) per k-chunk, in the canonical K-major layout without swizzle: 8 x 16-byte core matrices, the 16
// row groups of a k-chunk 128 bytes apart (the descriptor's stride byte offset) and successive
// k-chunks 16 * 128 bytes apart (its leading byte offset); B (all of K, loaded once) likewise
// with N / 8 row groups.  One thread issues the pass's MMAs (tcgen05.mma, kind::f16, BF16
// operands, FP32 accumulator in tensor memory) and commits them to an mbarrier; the next pass
// overwrites A only after a bounded wait for that commit.  After the last pass every warp reads
// its 32 rows of the accumulator (tcgen05.ld) and applies bias and ReLU.  Images too wide for
// the row copy (more than 16.5 KB of rows per pass) are read from global memory instead.
// About 71 KB of shared memory and 32 tensor-memory columns per CTA: three CTAs per SM.
constexpr int kConvM = 128;              // pixels per CTA (accumulator lanes)
constexpr int kConvTmemCols = 32;        // tensor-memory columns allocated per CTA (N <= 32)
constexpr int kConvMaxKp = 288;          // 32 input channels x 9 taps
constexpr int kConvTileBytes = 16896;    // staged image rows of one pass (4 rows of 129 pixels)

// K order.  The input channels are taken in groups of GC = 8 (at most 8 channels) or 16, one
// group per pass; within a pass k = tap * GC + c (c the channel within the group, tap = dy * 3 +
// dx), padded to a multiple of 16 (9 x 8 = 72 -> 80; 9 x 16 = 144).  So each 8-value k-chunk is
// one tap of 8 consecutive channels.
__host__ __device__ constexpr int conv_group(int cin) { return cin <= 8 ? 8 : 16; }
__host__ __device__ constexpr int conv_pass_k(int gc) { return (9 * gc + 15) / 16 * 16; }
// Padded K of a convolution with cin input channels, and the position of (ci, tap) in it.
__host__ __device__ constexpr int conv_kp(int cin) {
  return (cin + conv_group(cin) - 1) / conv_group(cin) * conv_pass_k(conv_group(cin));
}
__host__ __device__ constexpr int conv_kidx(int cin, int ci, int tap) {
  return ci / conv_group(cin) * conv_pass_k(conv_group(cin)) + tap * conv_group(cin) +
         ci % conv_group(cin);
}

__host__ __device__ constexpr size_t conv_a_bytes() {
  return (size_t)conv_pass_k(16) / 8 * (kConvM / 8) * 128;
}
__host__ __device__ constexpr size_t conv_b_bytes(int nt) {
  return (size_t)kConvMaxKp / 8 * (nt / 8) * 128;
}
// Dynamic shared memory of k_conv_tc: A of one pass, B, the staged rows.
__host__ __device__ constexpr size_t conv_smem_bytes(int nt) {
  return conv_a_bytes() + conv_b_bytes(nt) + kConvTileBytes;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte offset (between core
// matrices along K), stride byte offset (between 8-row groups), all >> 4; descriptor version 1
// (bit 46); no swizzle (layout type 0 in bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9
// and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t conv_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kConvM >> 4) << 24);
}

// Bounded wait for phase `parity` of an mbarrier; false when the bound ran out.
__device__ __forceinline__ bool conv_mbar_wait(uint32_t bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int NT, int GC>
__global__ void __launch_bounds__(kConvM)
k_conv_tc(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ Wk,
          const float* __restrict__ bias, int Cin, int Cout, int Kp, int Np, int B, int H, int W,
          int relu, __nv_bfloat16* __restrict__ out_bf, float* __restrict__ out_f,
          int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char conv_smem[];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = Kp / 8;                                  // k-chunks of 8 (Kp = conv_kp(Cin))
  constexpr int kPassChunks = conv_pass_k(GC) / 8;        // 18 (GC = 16) or 10 (GC = 8)
  constexpr int kGroups = GC / 8;                         // k-chunks per tap
  constexpr uint32_t kSbo = 128;                          // 8-row groups 128 bytes apart
  constexpr uint32_t kLboA = (kConvM / 8) * 128;          // 2048 bytes per k-chunk of A
  constexpr uint32_t kLboB = (NT / 8) * 128;              // bytes per k-chunk of B
  unsigned char* sA = conv_smem;                          // kConvM x 144 BF16 (one pass)
  unsigned char* sB = conv_smem + conv_a_bytes();         // NT x Kp BF16
  uint16_t* sT = reinterpret_cast<uint16_t*>(conv_smem + conv_a_bytes() + conv_b_bytes(NT));
  const int64_t plane = (int64_t)H * W, total = (int64_t)B * plane;
  const int64_t pix0 = (int64_t)blockIdx.x * kConvM;
  const int64_t pix = pix0 + tid;
  const uint32_t bar = smem_u32(&mma_bar);

  if (warp == 0) {   // tensor memory for the accumulator (whole warp, aligned)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kConvTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // This thread's pixel, and the rows (b H + y over the batch) the CTA's pixels and their
  // vertical neighbours touch: rlo .. rlo + nrows - 1.
  const bool valid = pix < total;
  const int b = valid ? (int)(pix / plane) : 0;
  const int64_t rem = valid ? pix - (int64_t)b * plane : 0;
  const int y = (int)(rem / W), x = (int)(rem - (int64_t)y * W);
  const int64_t rows_total = (int64_t)B * H;
  const int64_t last = (pix0 + kConvM < total ? pix0 + kConvM : total) - 1;
  const int64_t rlo = pix0 / W > 0 ? pix0 / W - 1 : 0;
  const int64_t rhi = last / W + 1 < rows_total ? last / W + 1 : rows_total - 1;
  const int nrows = (int)(rhi - rlo + 1);
  const bool staged = (int64_t)nrows * W * GC * 2 <= kConvTileBytes;
  const int b_lo = (int)(rlo / H), y_lo = (int)(rlo - (int64_t)b_lo * H);   // row rlo
  const __nv_bfloat16* inb = in + (size_t)b * Cin * plane;
  // the 9 taps of this pixel: inside the image (bit t of tap_in)
  int tap_in = 0;
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
    if (valid && yy >= 0 && yy < H && xx >= 0 && xx < W) tap_in |= 1 << t;
  }
  // the staged copy's element of (row prow, column x) is sT[(prow W + x) GC + c]
  const int prow = (int)((int64_t)b * H + y - rlo);

  // B: NT rows of the weights (rows Np .. NT - 1 zero), 16 bytes per (row, k-chunk)
  for (int e = tid; e < NT * nk; e += kConvM) {
    const int n = e / nk, kc = e - n * nk;
    uint4 row = make_uint4(0u, 0u, 0u, 0u);
    if (n < Np) row = *reinterpret_cast<const uint4*>(Wk + (size_t)n * Kp + kc * 8);
    *reinterpret_cast<uint4*>(sB + (size_t)kc * kLboB + (n >> 3) * kSbo + (n & 7) * 16) = row;
  }

  const int npass = (nk + kPassChunks - 1) / kPassChunks;
  bool ok = true;
  int waited = -1;   // the last pass whose MMAs are known complete
  for (int pass = 0; pass < npass; ++pass) {
    const int c0 = pass * kPassChunks;                         // first k-chunk of the pass
    const int nkp = nk - c0 < kPassChunks ? nk - c0 : kPassChunks;   // even: Kp % 16 == 0
    const int ci0 = pass * GC;                                  // the pass's channel group
    const int nci = Cin - ci0 < GC ? Cin - ci0 : GC;
    if (pass > 0) {
      // the previous pass's MMAs read A (and the copy is rewritten below): wait for them
      ok = conv_mbar_wait(bar, (uint32_t)((pass - 1) & 1), 1 << 22);
      if (__syncthreads_or(!ok)) break;
      waited = pass - 1;
    }
    if (staged) {
      // rows rlo .. rhi of the group's channels, channel innermost: sT[(row W + x) GC + c]
      // (zero for c >= nci).  Item (row, 8-channel part g, 32-column segment) per warp: each
      // lane loads its column's 8 channels (8 independent loads) and stores them as 16 bytes.
      const int nxs = (W + 31) / 32;
      const int items = nrows * kGroups * nxs;
      const uint16_t* in16 = reinterpret_cast<const uint16_t*>(in);
      for (int it = warp; it < items; it += kConvM / 32) {
        const int row = it / (kGroups * nxs), rest = it - row * (kGroups * nxs);
        const int g = rest / nxs, xr = (rest - g * nxs) * 32 + lane;
        if (xr >= W) continue;
        if (8 * g >= nci) {   // a part of the group past the last channel: zeros
          *reinterpret_cast<uint4*>(sT + ((size_t)row * W + xr) * GC + 8 * g) =
              make_uint4(0u, 0u, 0u, 0u);
          continue;
        }
        int bb = b_lo, yy = y_lo + row;   // batch row rlo + row as (image, row)
        while (yy >= H) {
          yy -= H;
          ++bb;
        }
        const uint16_t* src = in16 + ((size_t)bb * Cin + ci0 + 8 * g) * plane + (size_t)yy * W + xr;
        uint16_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 8 * g + j < nci ? src[(size_t)j * plane] : (uint16_t)0;
        uint4 pk;
        pk.x = v[0] | ((uint32_t)v[1] << 16);
        pk.y = v[2] | ((uint32_t)v[3] << 16);
        pk.z = v[4] | ((uint32_t)v[5] << 16);
        pk.w = v[6] | ((uint32_t)v[7] << 16);
        *reinterpret_cast<uint4*>(sT + ((size_t)row * W + xr) * GC + 8 * g) = pk;
      }
      __syncthreads();
    }
    // A of the pass: this thread's pixel row; k-chunk kc is tap kc / kGroups of the channels
    // 8 (kc % kGroups) .. + 7 of the group: one 16-byte load from the copy
#pragma unroll
    for (int kc = 0; kc < kPassChunks; ++kc) {
      const int tap = kc / kGroups, g = kc - tap * kGroups;
      uint4 row = make_uint4(0u, 0u, 0u, 0u);
      if (tap < 9 && ((tap_in >> tap) & 1) && (staged || 8 * g < nci)) {
        const int dy = tap / 3, dx = tap - dy * 3;
        if (staged) {
          row = *reinterpret_cast<const uint4*>(
              sT + ((size_t)(prow + dy - 1) * W + x + dx - 1) * GC + 8 * g);
        } else {
          const __nv_bfloat16* src =
              inb + (size_t)(ci0 + 8 * g) * plane + (size_t)(y + dy - 1) * W + x + dx - 1;
          uint16_t v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            v[j] = 8 * g + j < nci ? __bfloat16_as_ushort(src[(size_t)j * plane]) : (uint16_t)0;
          row.x = v[0] | ((uint32_t)v[1] << 16);
          row.y = v[2] | ((uint32_t)v[3] << 16);
          row.z = v[4] | ((uint32_t)v[5] << 16);
          row.w = v[6] | ((uint32_t)v[7] << 16);
        }
      }
      *reinterpret_cast<uint4*>(sA + (size_t)kc * kLboA + (tid >> 3) * kSbo + (tid & 7) * 16) = row;
    }
    // make the operands visible to the tensor core's asynchronous proxy, then issue
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      constexpr uint32_t idesc = conv_idesc(NT);
      const uint32_t taddr = tmem_base;
      for (int ks = 0; ks < nkp / 2; ++ks) {
        const uint64_t ad = smem_desc(smem_u32(sA) + ks * 2 * kLboA, kLboA, kSbo);
        const uint64_t bd = smem_desc(smem_u32(sB) + (c0 + ks * 2) * kLboB, kLboB, kSbo);
        const uint32_t acc = (pass > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              bar)
          : "memory");
    }
  }
  const uint32_t taddr = tmem_base;
  // the last issued pass: all of them after a normal loop, the one before the failed wait else
  const int issued = ok ? npass - 1 : waited + 1;
  if (ok) ok = conv_mbar_wait(bar, (uint32_t)((npass - 1) & 1), 1 << 22);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (__syncthreads_or(!ok)) {
    // The MMAs did not complete within the bound: report it, give the last issued commit one
    // more bounded wait, release the tensor memory and stop.
    if (tid == 0) atomicExch(err, 1);
    conv_mbar_wait(bar, (uint32_t)(issued & 1), 1 << 22);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                   "r"(kConvTmemCols)
                   : "memory");
    }
    return;
  }
  // accumulator row tid (lanes 32 warp .. 32 warp + 31), NT columns
  float accv[NT];
  const uint32_t lane_addr = taddr + ((uint32_t)(warp * 32) << 16);
  if constexpr (NT == 16) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(lane_addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) accv[j] = __uint_as_float(r[j]);
  } else {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(lane_addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) accv[j] = __uint_as_float(r[j]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(kConvTmemCols)
                 : "memory");
  }
  if (pix >= total) return;
#pragma unroll
  for (int n = 0; n < NT; ++n) {
    if (n >= Cout) break;
    float v = accv[n] + (bias ? bias[n] : 0.0f);
    if (relu) v = fmaxf(v, 0.0f);
    const size_t o = ((size_t)b * Cout + n) * plane + rem;
    if (out_f) out_f[o] = v;
    if (out_bf) out_bf[o] = __float2bfloat16(v);
  }
}


// Weight and bias gradients of one layer: gw[co][ci][tap] = sum_{b,y,x} g[b][co][y][x] *
// in[b][ci][y + dy - 1][x + dx - 1]; gb[co] = sum g[b][co].  One CTA per (co, ci).
__global__ void __launch_bounds__(256)
k_wgrad(const __nv_bfloat16* __restrict__ in, const float* __restrict__ g, int Cin, int Cout,
        int B, int H, int W, float* __restrict__ gw, float* __restrict__ gb) {
  const int co = blockIdx.x / Cin, ci = blockIdx.x % Cin;
  const size_t plane = (size_t)H * W;
  float acc[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) acc[i] = 0.0f;
  const int64_t total = (int64_t)B * H * W;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int x = (int)(e % W), y = (int)((e / W) % H), b = (int)(e / plane);
    const float gv = g[((size_t)b * Cout + co) * plane + (size_t)y * W + x];
    const __nv_bfloat16* ib = in + ((size_t)b * Cin + ci) * plane;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      const float iv = (yy >= 0 && yy < H && xx >= 0 && xx < W)
                           ? __bfloat162float(ib[(size_t)yy * W + xx]) : 0.0f;
      acc[tap] = fmaf(gv, iv, acc[tap]);
    }
    acc[9] += gv;
  }
  __shared__ float red[10][8];
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    float v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    float v = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    if (threadIdx.x < 9)
      gw[((size_t)co * Cin + ci) * 9 + threadIdx.x] = v;
    else if (ci == 0)
      gb[co] = v;
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                              int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// g_prev = g_in * (a > 0): the ReLU of the previous layer, a its (post-ReLU) output.
// gin and gout may be the same array (element-wise, read before write).
__global__ void k_relu_mask(const float* gin, const __nv_bfloat16* __restrict__ a, float* gout,
                            int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    gout[i] = __bfloat162float(a[i]) > 0.0f ? gin[i] : 0.0f;
}

// Masked mean squared error: g = 2 (y - t) m / count, partial sums of (y - t)^2 m per block.
__global__ void __launch_bounds__(256)
k_mse(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ mask,
      int64_t plane, int64_t n, float inv_count, float* __restrict__ g, float* __restrict__ part) {
  float s = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = (y[i] - t[i]) * mask[i % plane];
    g[i] = 2.0f * d * inv_count;
    s = fmaf(d, d, s);
  }
  __shared__ float red[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.0f;
    for (int w = 0; w < 8; ++w) v += red[w];
    part[blockIdx.x] = v;
  }
}

// Adam (bias-corrected moments) on the FP32 master parameters.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 GEMM layouts of one layer's weights w[co][ci][3][3] in the K order of conv_kidx: forward
// Wk[co][kidx(ci, tap)] and, for the input gradient, the flipped transpose
// Wt[ci][kidx(co, 8 - tap)].
__global__ void k_pack(const float* __restrict__ w, int Cin, int Cout, int Kp, int Kpt,
                       __nv_bfloat16* __restrict__ Wk, __nv_bfloat16* __restrict__ Wt) {
  const int n = Cout * Cin * 9;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int tap = i % 9, ci = (i / 9) % Cin, co = i / (9 * Cin);
    const __nv_bfloat16 v = __float2bfloat16(w[i]);
    Wk[(size_t)co * Kp + conv_kidx(Cin, ci, tap)] = v;
    Wt[(size_t)ci * Kpt + conv_kidx(Cout, co, 8 - tap)] = v;
  }
}

// ---- features and targets of the warm start (2D grids, H = ny + 1 rows, W = nx + 1) ----
// For frequency m: input channels x[m][0] = f_m / max|f_m| and x[m][1] = omega_m / omega_scale;
// target t[m] = V_m / max|V_m| (the shape of the solution); the prediction is that shape with
// 0 on the boundary, its amplitude fitted afterwards to the Helmholtz residual.

__global__ void k_ws_scale(const double* __restrict__ f, int64_t P, double* __restrict__ scale) {
  const int m = blockIdx.x;
  double mx = 0.0;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) mx = fmax(mx, fabs(f[m * P + i]));
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v = fmax(v, red[w]);
    scale[m] = v > 0.0 ? v : 1.0;
  }
}

struct WsFreq {
  double omega[MFWH_MAX_NF];
};

__global__ void k_ws_features(const double* __restrict__ f, const double* __restrict__ v,
                              const double* __restrict__ fscale, const double* __restrict__ vscale,
                              const WsFreq fr, int nf, int64_t P, double omega_scale,
                              float* __restrict__ x, float* __restrict__ t) {
  const int64_t n = (int64_t)nf * P;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e / P);
    const int64_t i = e - (int64_t)m * P;
    x[((int64_t)m * 2) * P + i] = (float)(f[e] / fscale[m]);
    x[((int64_t)m * 2 + 1) * P + i] = (float)(fr.omega[m] / omega_scale);
    if (t) t[e] = (float)(v[e] / vscale[m]);
  }
}

__global__ void k_ws_output(const float* __restrict__ y, int nf, int H, int W,
                            double* __restrict__ v) {
  const int64_t P = (int64_t)H * W, n = (int64_t)nf * P;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % P;
    const int xx = (int)(i % W), yy = (int)(i / W);
    const bool interior = xx > 0 && xx < W - 1 && yy > 0 && yy < H - 1;
    v[e] = interior ? (double)y[e] : 0.0;
  }
}

mfwh_status cnn_fail(mfwh_status st, const std::string& m) {
  set_error(m);
  return st;
}

}  // namespace
}  // namespace mfwh

using namespace mfwh;

struct mfwh_cnn_s {
  int layers = 0, channels = 0, in_channels = 0;
  cudaStream_t stream = nullptr;
  std::vector<int> cin, cout;          // per layer
  std::vector<int64_t> woff, boff;     // offsets of w and b in the flat parameter vector
  int64_t nparams = 0;
  float* p = nullptr;                  // FP32 master parameters
  float* grad = nullptr;               // gradients (same layout)
  float* m = nullptr;
  float* v = nullptr;
  int step = 0;
  std::vector<__nv_bfloat16*> Wk, Wt;  // BF16 GEMM layouts per layer
  std::vector<int> Kp, Kpt, Np, Npt;
  // activation workspace, sized for cap elements per channel plane times the batch
  int64_t cap = 0;                     // B * H * W the workspace holds
  std::vector<__nv_bfloat16*> act;     // inputs of each layer (BF16), [B][C][H][W]
  float* y = nullptr;                  // network output [B][1][H][W]
  float* g0 = nullptr;                 // gradient buffers [B][channels][H][W]
  float* g1 = nullptr;
  __nv_bfloat16* gbf = nullptr;
  float* part = nullptr;               // loss partial sums
  float* part_h = nullptr;             // pinned
  int* err = nullptr;                  // device flag: a convolution's MMA wait ran out
};

namespace {

constexpr int kLossBlocks = 256;

#define CKC(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return cnn_fail(MFWH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

mfwh_status ensure_ws(mfwh_cnn_t c, int64_t bhw) {
  if (bhw <= c->cap) return MFWH_OK;
  for (auto& a : c->act)
    if (a) cudaFree(a);
  if (c->y) cudaFree(c->y);
  if (c->g0) cudaFree(c->g0);
  if (c->g1) cudaFree(c->g1);
  if (c->gbf) cudaFree(c->gbf);
  c->act.assign(c->layers + 1, nullptr);
  c->cap = 0;
  const int maxc = std::max(c->channels, c->in_channels);
  for (int l = 0; l <= c->layers; ++l) {
    const int ch = l == 0 ? c->in_channels : (l == c->layers ? 1 : c->channels);
    CKC(cudaMalloc(&c->act[l], sizeof(__nv_bfloat16) * bhw * ch));
  }
  CKC(cudaMalloc(&c->y, sizeof(float) * bhw));
  CKC(cudaMalloc(&c->g0, sizeof(float) * bhw * maxc));
  CKC(cudaMalloc(&c->g1, sizeof(float) * bhw * maxc));
  CKC(cudaMalloc(&c->gbf, sizeof(__nv_bfloat16) * bhw * maxc));
  c->cap = bhw;
  return MFWH_OK;
}

void conv(mfwh_cnn_t c, const __nv_bfloat16* in, const __nv_bfloat16* Wk, const float* bias,
          int Cin, int Cout, int Kp, int Np, int B, int H, int W, int relu, __nv_bfloat16* out_bf,
          float* out_f) {
  const int64_t total = (int64_t)B * H * W;
  const unsigned blocks = (unsigned)((total + kConvM - 1) / kConvM);
  auto launch = [&](auto kernel, int nt) {
    kernel<<<blocks, kConvM, conv_smem_bytes(nt), c->stream>>>(
        in, Wk, bias, Cin, Cout, Kp, Np, B, H, W, relu, out_bf, out_f, c->err);
  };
  const bool g8 = conv_group(Cin) == 8;
  if (Np <= 16)
    g8 ? launch(k_conv_tc<16, 8>, 16) : launch(k_conv_tc<16, 16>, 16);
  else
    g8 ? launch(k_conv_tc<32, 8>, 32) : launch(k_conv_tc<32, 16>, 32);
}

// The convolution kernels' shared-memory limit, once per device.
mfwh_status conv_configure() {
  static bool done[64] = {};
  int dev = 0;
  CKC(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && done[dev]) return MFWH_OK;
  CKC(cudaFuncSetAttribute(k_conv_tc<16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem_bytes(16)));
  CKC(cudaFuncSetAttribute(k_conv_tc<16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem_bytes(16)));
  CKC(cudaFuncSetAttribute(k_conv_tc<32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem_bytes(32)));
  CKC(cudaFuncSetAttribute(k_conv_tc<32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem_bytes(32)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return MFWH_OK;
}

// A convolution's bounded MMA wait ran out since the last check: report it and clear the flag.
mfwh_status check_err(mfwh_cnn_t c) {
  int flag = 0;
  CKC(cudaMemcpyAsync(&flag, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CKC(cudaStreamSynchronize(c->stream));
  if (!flag) return MFWH_OK;
  CKC(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
  return cnn_fail(MFWH_ERR_TIMEOUT, "cnn: a convolution's tensor-core wait timed out");
}

mfwh_status pack_all(mfwh_cnn_t c) {
  for (int l = 0; l < c->layers; ++l) {
    CKC(cudaMemsetAsync(c->Wk[l], 0, sizeof(__nv_bfloat16) * c->Np[l] * c->Kp[l], c->stream));
    CKC(cudaMemsetAsync(c->Wt[l], 0, sizeof(__nv_bfloat16) * c->Npt[l] * c->Kpt[l], c->stream));
    k_pack<<<64, 256, 0, c->stream>>>(c->p + c->woff[l], c->cin[l], c->cout[l], c->Kp[l],
                                      c->Kpt[l], c->Wk[l], c->Wt[l]);
  }
  CKC(cudaGetLastError());
  return MFWH_OK;
}

mfwh_status forward_impl(mfwh_cnn_t c, const float* x, int B, int H, int W) {
  const int64_t bhw = (int64_t)B * H * W;
  mfwh_status st = ensure_ws(c, bhw);
  if (st != MFWH_OK) return st;
  k_f32_to_bf16<<<256, 256, 0, c->stream>>>(x, c->act[0], bhw * c->in_channels);
  for (int l = 0; l < c->layers; ++l) {
    const bool last = l + 1 == c->layers;
    conv(c, c->act[l], c->Wk[l], c->p + c->boff[l], c->cin[l], c->cout[l], c->Kp[l], c->Np[l], B,
         H, W, last ? 0 : 1, last ? nullptr : c->act[l + 1], last ? c->y : nullptr);
  }
  CKC(cudaGetLastError());
  return MFWH_OK;
}

}  // namespace

extern "C" {

mfwh_status mfwh_cnn_create(int layers, int channels, int in_channels, uint64_t seed,
                            void* stream, mfwh_cnn_t* out) {
  if (!out || layers < 2 || layers > 16 || channels < 1 || channels > 32 || in_channels < 1 ||
      in_channels > 32)
    return cnn_fail(MFWH_ERR_INVALID_ARG, "cnn: 2..16 layers, 1..32 channels and inputs");
  *out = nullptr;
  auto* c = new (std::nothrow) mfwh_cnn_s();
  if (!c) return cnn_fail(MFWH_ERR_NOMEM, "host allocation failed");
  c->layers = layers;
  c->channels = channels;
  c->in_channels = in_channels;
  c->stream = static_cast<cudaStream_t>(stream);
  for (int l = 0; l < layers; ++l) {
    const int ci = l == 0 ? in_channels : channels, co = l + 1 == layers ? 1 : channels;
    c->cin.push_back(ci);
    c->cout.push_back(co);
    c->woff.push_back(c->nparams);
    c->nparams += (int64_t)co * ci * 9;
    c->boff.push_back(c->nparams);
    c->nparams += co;
    c->Kp.push_back(conv_kp(ci));
    c->Np.push_back(round_up(co, 8));
    c->Kpt.push_back(conv_kp(co));
    c->Npt.push_back(round_up(ci, 8));
  }
  // He-normal weights (std sqrt(2 / (9 Cin))), zero biases, from a seeded host generator
  std::vector<float> h(c->nparams, 0.0f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < layers; ++l) {
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (9.0 * c->cin[l])));
    for (int64_t i = 0; i < (int64_t)c->cout[l] * c->cin[l] * 9; ++i)
      h[c->woff[l] + i] = (float)nd(rng);
  }
  auto fail_free = [&](mfwh_status s) {
    mfwh_cnn_destroy(c);
    return s;
  };
  for (float** b : {&c->p, &c->grad, &c->m, &c->v})
    if (cudaMalloc(b, sizeof(float) * c->nparams) != cudaSuccess)
      return fail_free(cnn_fail(MFWH_ERR_NOMEM, "cnn: parameter allocation failed"));
  c->Wk.assign(layers, nullptr);
  c->Wt.assign(layers, nullptr);
  for (int l = 0; l < layers; ++l)
    if (cudaMalloc(&c->Wk[l], sizeof(__nv_bfloat16) * c->Np[l] * c->Kp[l]) != cudaSuccess ||
        cudaMalloc(&c->Wt[l], sizeof(__nv_bfloat16) * c->Npt[l] * c->Kpt[l]) != cudaSuccess)
      return fail_free(cnn_fail(MFWH_ERR_NOMEM, "cnn: weight allocation failed"));
  if (cudaMalloc(&c->part, sizeof(float) * kLossBlocks) != cudaSuccess ||
      cudaMallocHost(&c->part_h, sizeof(float) * kLossBlocks) != cudaSuccess ||
      cudaMalloc(&c->err, sizeof(int)) != cudaSuccess)
    return fail_free(cnn_fail(MFWH_ERR_NOMEM, "cnn: allocation failed"));
  if (cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) != cudaSuccess)
    return fail_free(cnn_fail(MFWH_ERR_CUDA, "cnn: initialisation failed"));
  if (conv_configure() != MFWH_OK) return fail_free(MFWH_ERR_CUDA);
  if (cudaMemcpyAsync(c->p, h.data(), sizeof(float) * c->nparams, cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->m, 0, sizeof(float) * c->nparams, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->v, 0, sizeof(float) * c->nparams, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->grad, 0, sizeof(float) * c->nparams, c->stream) != cudaSuccess)
    return fail_free(cnn_fail(MFWH_ERR_CUDA, "cnn: initialisation failed"));
  mfwh_status st = pack_all(c);
  if (st == MFWH_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = MFWH_ERR_CUDA;
  if (st != MFWH_OK) return fail_free(st);
  *out = c;
  return MFWH_OK;
}

int64_t mfwh_cnn_param_count(mfwh_cnn_t c) { return c ? c->nparams : 0; }

mfwh_status mfwh_cnn_set_params(mfwh_cnn_t c, const float* host, int64_t count) {
  if (!c || !host || count != c->nparams)
    return cnn_fail(MFWH_ERR_INVALID_ARG, "cnn: parameter count mismatch");
  CKC(cudaMemcpyAsync(c->p, host, sizeof(float) * count, cudaMemcpyHostToDevice, c->stream));
  CKC(cudaMemsetAsync(c->m, 0, sizeof(float) * count, c->stream));
  CKC(cudaMemsetAsync(c->v, 0, sizeof(float) * count, c->stream));
  c->step = 0;
  mfwh_status st = pack_all(c);
  if (st != MFWH_OK) return st;
  CKC(cudaStreamSynchronize(c->stream));
  return MFWH_OK;
}

mfwh_status mfwh_cnn_get_params(mfwh_cnn_t c, float* host, float* grads_host, int64_t count) {
  if (!c || !host || count != c->nparams)
    return cnn_fail(MFWH_ERR_INVALID_ARG, "cnn: parameter count mismatch");
  CKC(cudaMemcpyAsync(host, c->p, sizeof(float) * count, cudaMemcpyDeviceToHost, c->stream));
  if (grads_host)
    CKC(cudaMemcpyAsync(grads_host, c->grad, sizeof(float) * count, cudaMemcpyDeviceToHost,
                        c->stream));
  CKC(cudaStreamSynchronize(c->stream));
  return check_err(c);
}

mfwh_status mfwh_cnn_forward(mfwh_cnn_t c, const float* x, int B, int H, int W, float* y) {
  if (!c || !x || !y || B < 1 || H < 1 || W < 1)
    return cnn_fail(MFWH_ERR_INVALID_ARG, "cnn: bad forward arguments");
  mfwh_status st = forward_impl(c, x, B, H, W);
  if (st != MFWH_OK) return st;
  CKC(cudaMemcpyAsync(y, c->y, sizeof(float) * B * H * W, cudaMemcpyDeviceToDevice, c->stream));
  return MFWH_OK;
}

mfwh_status mfwh_cnn_train_step(mfwh_cnn_t c, const float* x, const float* target,
                                const float* mask, int B, int H, int W, float lr, float* loss) {
  if (!c || !x || !target || !mask || B < 1 || H < 1 || W < 1 || !(lr > 0.0f))
    return cnn_fail(MFWH_ERR_INVALID_ARG, "cnn: bad training arguments");
  mfwh_status st = forward_impl(c, x, B, H, W);
  if (st != MFWH_OK) return st;
  const int64_t hw = (int64_t)H * W, n = (int64_t)B * hw;
  // the mask's point count, for the mean
  std::vector<float> mh(hw);
  CKC(cudaMemcpyAsync(mh.data(), mask, sizeof(float) * hw, cudaMemcpyDeviceToHost, c->stream));
  CKC(cudaStreamSynchronize(c->stream));
  double cnt = 0.0;
  for (float v : mh) cnt += v;
  const float inv = (float)(1.0 / std::max(1.0, cnt * B));
  float* g = c->g0;
  float* gnext = c->g1;
  k_mse<<<kLossBlocks, 256, 0, c->stream>>>(c->y, target, mask, hw, n, inv, g, c->part);
  for (int l = c->layers - 1; l >= 0; --l) {
    k_wgrad<<<c->cout[l] * c->cin[l], 256, 0, c->stream>>>(
        c->act[l], g, c->cin[l], c->cout[l], B, H, W, c->grad + c->woff[l], c->grad + c->boff[l]);
    if (l > 0) {
      k_f32_to_bf16<<<256, 256, 0, c->stream>>>(g, c->gbf, n * c->cout[l]);
      conv(c, c->gbf, c->Wt[l], nullptr, c->cout[l], c->cin[l], c->Kpt[l], c->Npt[l], B, H, W, 0,
           nullptr, gnext);
      k_relu_mask<<<256, 256, 0, c->stream>>>(gnext, c->act[l], gnext, n * c->cin[l]);
      std::swap(g, gnext);
    }
  }
  c->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  k_adam<<<256, 256, 0, c->stream>>>(c->p, c->grad, c->m, c->v, c->nparams, lr, b1, b2, 1e-8f,
                                     1.0f - std::pow(b1, (float)c->step),
                                     1.0f - std::pow(b2, (float)c->step));
  st = pack_all(c);
  if (st != MFWH_OK) return st;
  CKC(cudaMemcpyAsync(c->part_h, c->part, sizeof(float) * kLossBlocks, cudaMemcpyDeviceToHost,
                      c->stream));
  CKC(cudaStreamSynchronize(c->stream));
  double s = 0.0;
  for (int i = 0; i < kLossBlocks; ++i) s += c->part_h[i];
  if (loss) *loss = (float)(s * inv);
  return check_err(c);
}

void mfwh_cnn_destroy(mfwh_cnn_t c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (float* b : {c->p, c->grad, c->m, c->v, c->y, c->g0, c->g1, c->part})
    if (b) cudaFree(b);
  if (c->gbf) cudaFree(c->gbf);
  for (auto* w : c->Wk)
    if (w) cudaFree(w);
  for (auto* w : c->Wt)
    if (w) cudaFree(w);
  for (auto* a : c->act)
    if (a) cudaFree(a);
  if (c->part_h) cudaFreeHost(c->part_h);
  if (c->err) cudaFree(c->err);
  delete c;
}

}  // extern "C"

namespace mfwh {

// Training pairs of one solved 2D problem (device arrays; see the feature definition above).
// scale: device scratch of 2 nf doubles.
mfwh_status cnn_ws_data(const double* f, const double* v, const double* omega, int nf, int H,
                        int W, double omega_scale, float* x, float* t, double* scale,
                        cudaStream_t st) {
  WsFreq fr{};
  for (int m = 0; m < nf; ++m) fr.omega[m] = omega[m];
  const int64_t P = (int64_t)H * W;
  k_ws_scale<<<nf, 256, 0, st>>>(f, P, scale);
  if (v) k_ws_scale<<<nf, 256, 0, st>>>(v, P, scale + nf);
  k_ws_features<<<256, 256, 0, st>>>(f, v, scale, scale + nf, fr, nf, P, omega_scale, x, t);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MFWH_OK : cnn_fail(MFWH_ERR_CUDA, cudaGetErrorString(e));
}

// The network's solution shape for every frequency of a 2D problem (0 on the boundary).
mfwh_status cnn_ws_predict(mfwh_cnn_t c, const double* f, const double* omega, int nf, int H,
                           int W, double omega_scale, double* v, cudaStream_t st) {
  if (c->in_channels != 2) return cnn_fail(MFWH_ERR_INVALID_ARG, "warm start needs 2 inputs");
  const int64_t P = (int64_t)H * W;
  float* x = nullptr;
  float* y = nullptr;
  double* scale = nullptr;
  mfwh_status res = MFWH_OK;
  if (cudaMalloc(&x, sizeof(float) * 2 * nf * P) != cudaSuccess ||
      cudaMalloc(&y, sizeof(float) * nf * P) != cudaSuccess ||
      cudaMalloc(&scale, sizeof(double) * 2 * nf) != cudaSuccess) {
    res = cnn_fail(MFWH_ERR_NOMEM, "warm start: allocation failed");
  } else {
    res = cnn_ws_data(f, nullptr, omega, nf, H, W, omega_scale, x, nullptr, scale, st);
    cudaStream_t keep = c->stream;
    c->stream = st;
    if (res == MFWH_OK) res = mfwh_cnn_forward(c, x, nf, H, W, y);
    c->stream = keep;
    if (res == MFWH_OK) {
      k_ws_output<<<256, 256, 0, st>>>(y, nf, H, W, v);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        res = cnn_fail(MFWH_ERR_CUDA, "warm start: output kernel failed");
    }
    if (res == MFWH_OK) {
      c->stream = st;
      res = check_err(c);
      c->stream = keep;
    }
  }
  cudaStreamSynchronize(st);
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  if (scale) cudaFree(scale);
  return res;
}

}  // namespace mfwh

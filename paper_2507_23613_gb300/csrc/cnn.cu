// Warm-start predictor for MFWH: a small convolutional network that maps a forcing f_m and
// its frequency omega_m to an initial iterate V_m^0 for GMRES (the learned warm start; the
// paper itself starts from zero).  L layers of 3 x 3 "same" convolutions (zero padding) with
// bias, ReLU after every layer but the last, images [B][C][H][W].
//
// Arithmetic: activations and weights in BF16, products accumulated in FP32 on the tensor
// cores (mma.sync m16n8k16, an implicit GEMM whose rows are 16 consecutive pixels of one image
// row and whose reduction runs over (input channel, tap)); gradients, master weights and the
// Adam state in FP32.  The weight gradient, a reduction over every pixel of the batch, runs on
// the FP32 CUDA cores.
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

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  const uint32_t l = __bfloat16_as_ushort(lo), h = __bfloat16_as_ushort(hi);
  return l | (h << 16);
}

// Implicit-GEMM 3 x 3 convolution.  One warp computes 16 consecutive pixels (x0 .. x0 + 15 of
// row y of image b) for all output channels (NT tiles of 8).  Wk: [Np][Kp] BF16, Wk[n][k] with
// k = ci * 9 + tap (tap = dy * 3 + dx), zero for k >= Cin * 9 and n >= Cout.
template <int NT>
__global__ void __launch_bounds__(128)
k_conv_mma(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ Wk,
           const float* __restrict__ bias, int Cin, int Cout, int Kp, int B, int H, int W,
           int relu, __nv_bfloat16* __restrict__ out_bf, float* __restrict__ out_f) {
  const int lane = threadIdx.x & 31;
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int segs = (W + 15) / 16;
  if (warp >= B * H * segs) return;
  const int seg = warp % segs, y = (warp / segs) % H, b = warp / (segs * H);
  const int x0 = seg * 16;
  const int g = lane >> 2, t = lane & 3;
  const int K = Cin * 9;
  const size_t plane = (size_t)H * W;
  const __nv_bfloat16* inb = in + (size_t)b * Cin * plane;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  // value of A[row r][col k] (pixel x0 + r, reduction index k)
  auto a_val = [&](int r, int k) -> __nv_bfloat16 {
    if (k >= K) return zero;
    const int ci = k / 9, tap = k - ci * 9;
    const int yy = y + tap / 3 - 1, xx = x0 + r + tap % 3 - 1;
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) return zero;
    return inb[(size_t)ci * plane + (size_t)yy * W + xx];
  };
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
  for (int kc = 0; kc < Kp; kc += 16) {
    const int c0 = kc + 2 * t, c2 = kc + 2 * t + 8;
    const uint32_t a0 = pack_bf16(a_val(g, c0), a_val(g, c0 + 1));
    const uint32_t a1 = pack_bf16(a_val(g + 8, c0), a_val(g + 8, c0 + 1));
    const uint32_t a2 = pack_bf16(a_val(g, c2), a_val(g, c2 + 1));
    const uint32_t a3 = pack_bf16(a_val(g + 8, c2), a_val(g + 8, c2 + 1));
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const __nv_bfloat16* wr = Wk + (size_t)(j * 8 + g) * Kp;
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr + c0);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + c2);
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};"
          : "+f"(acc[j][0]), "+f"(acc[j][1]), "+f"(acc[j][2]), "+f"(acc[j][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = g + (e >= 2 ? 8 : 0), n = j * 8 + 2 * t + (e & 1);
      const int x = x0 + r;
      if (n >= Cout || x >= W) continue;
      float v = acc[j][e] + (bias ? bias[n] : 0.0f);
      if (relu) v = fmaxf(v, 0.0f);
      const size_t o = ((size_t)b * Cout + n) * plane + (size_t)y * W + x;
      if (out_f) out_f[o] = v;
      if (out_bf) out_bf[o] = __float2bfloat16(v);
    }
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

// BF16 GEMM layouts of one layer's weights w[co][ci][3][3]: forward Wk[co][ci * 9 + tap] and,
// for the input gradient, the flipped transpose Wt[ci][co * 9 + 8 - tap].
__global__ void k_pack(const float* __restrict__ w, int Cin, int Cout, int Kp, int Kpt,
                       __nv_bfloat16* __restrict__ Wk, __nv_bfloat16* __restrict__ Wt) {
  const int n = Cout * Cin * 9;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int tap = i % 9, ci = (i / 9) % Cin, co = i / (9 * Cin);
    const __nv_bfloat16 v = __float2bfloat16(w[i]);
    Wk[(size_t)co * Kp + ci * 9 + tap] = v;
    Wt[(size_t)ci * Kpt + co * 9 + (8 - tap)] = v;
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
  const int warps = B * H * ((W + 15) / 16);
  const int blocks = (warps + 3) / 4;
  switch (Np / 8) {
    case 1: k_conv_mma<1><<<blocks, 128, 0, c->stream>>>(in, Wk, bias, Cin, Cout, Kp, B, H, W, relu, out_bf, out_f); break;
    case 2: k_conv_mma<2><<<blocks, 128, 0, c->stream>>>(in, Wk, bias, Cin, Cout, Kp, B, H, W, relu, out_bf, out_f); break;
    case 3: k_conv_mma<3><<<blocks, 128, 0, c->stream>>>(in, Wk, bias, Cin, Cout, Kp, B, H, W, relu, out_bf, out_f); break;
    default: k_conv_mma<4><<<blocks, 128, 0, c->stream>>>(in, Wk, bias, Cin, Cout, Kp, B, H, W, relu, out_bf, out_f); break;
  }
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
    c->Kp.push_back(round_up(ci * 9, 16));
    c->Np.push_back(round_up(co, 8));
    c->Kpt.push_back(round_up(co * 9, 16));
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
      cudaMallocHost(&c->part_h, sizeof(float) * kLossBlocks) != cudaSuccess)
    return fail_free(cnn_fail(MFWH_ERR_NOMEM, "cnn: allocation failed"));
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
  return MFWH_OK;
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
  return MFWH_OK;
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
  }
  cudaStreamSynchronize(st);
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  if (scale) cudaFree(scale);
  return res;
}

}  // namespace mfwh

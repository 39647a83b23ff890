// FP64 vector kernels for the GMRES Arnoldi process (Section "Acceleration by
// Krylov methods"): batched inner products <V_i, w> for the Gram-Schmidt
// projections, the matching batched update w -= sum_i h_i V_i, and axpby.
// Inner products reduce per thread, then across the warp with shuffles, then
// across the block in shared memory; per-block partials are summed by a second
// kernel in a fixed order, so results are deterministic.
#include <cuda_runtime.h>

#include "kernels.h"

namespace mfwh {
namespace {

constexpr int kDotBlocks = 2 * 152;
constexpr int kDotThreads = 256;

template <int K>
__global__ void __launch_bounds__(kDotThreads)
k_multidot(const double* __restrict__ V, int64_t ldv, int k, const double* __restrict__ w,
           int64_t N, double* __restrict__ partial) {
  double acc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) acc[i] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double we = w[e];
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i < k) acc[i] = fma(V[i * ldv + e], we, acc[i]);
  }
  __shared__ double red[K][kDotThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (i >= k) break;
    double s = acc[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[i][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int wi = 0; wi < kDotThreads / 32; ++wi) s += red[threadIdx.x][wi];
    partial[(int64_t)blockIdx.x * kMaxDots + threadIdx.x] = s;
  }
}

__global__ void k_sum_partials(const double* __restrict__ partial, int nblocks, int k,
                               double* __restrict__ out) {
  // one warp per output: lane-strided sum, then a shuffle tree
  const int i = blockIdx.x;
  if (i >= k) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) s += partial[(int64_t)b * kMaxDots + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[i] = s;
}

struct AxpyCoef {
  double c[kMaxDots];
};

template <int K>
__global__ void __launch_bounds__(256)
k_multi_axpy(double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int k,
             const AxpyCoef a, int64_t N) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = w[e];
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i < k) s = fma(-a.c[i], V[i * ldv + e], s);
    w[e] = s;
  }
}

__global__ void __launch_bounds__(256)
k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b, int64_t N) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (b == 0.0) ? a * x[e] : fma(a, x[e], b * y[e]);
}

unsigned stream_blocks(int64_t N) {
  int64_t b = (N + 255) / 256;
  const int64_t cap = 152 * 8;
  return (unsigned)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace

int64_t dot_partial_size() { return (int64_t)kDotBlocks * kMaxDots; }

int multidot_launches(int k) { return 2 * ((k + kMaxDots - 1) / kMaxDots); }
int multi_axpy_launches(int k) { return (k + kMaxDots - 1) / kMaxDots; }

void launch_multidot(const double* V, int64_t ldv, int k, const double* w, int64_t N,
                     double* partial, double* out, cudaStream_t st) {
  for (int c0 = 0; c0 < k; c0 += kMaxDots) {
    const int kc = k - c0 < kMaxDots ? k - c0 : kMaxDots;
    const double* Vc = V + (int64_t)c0 * ldv;
    if (kc <= 4)
      k_multidot<4><<<kDotBlocks, kDotThreads, 0, st>>>(Vc, ldv, kc, w, N, partial);
    else if (kc <= 8)
      k_multidot<8><<<kDotBlocks, kDotThreads, 0, st>>>(Vc, ldv, kc, w, N, partial);
    else if (kc <= 16)
      k_multidot<16><<<kDotBlocks, kDotThreads, 0, st>>>(Vc, ldv, kc, w, N, partial);
    else
      k_multidot<kMaxDots><<<kDotBlocks, kDotThreads, 0, st>>>(Vc, ldv, kc, w, N, partial);
    // the partials are consumed before the next chunk overwrites them (same stream)
    k_sum_partials<<<kc, 32, 0, st>>>(partial, kDotBlocks, kc, out + c0);
  }
}

void launch_multi_axpy(double* w, const double* V, int64_t ldv, int k, const double* coef,
                       int64_t N, cudaStream_t st) {
  const unsigned nb = stream_blocks(N);
  for (int c0 = 0; c0 < k; c0 += kMaxDots) {
    const int kc = k - c0 < kMaxDots ? k - c0 : kMaxDots;
    const double* Vc = V + (int64_t)c0 * ldv;
    AxpyCoef a;
    for (int i = 0; i < kMaxDots; ++i) a.c[i] = i < kc ? coef[c0 + i] : 0.0;
    if (kc <= 4)
      k_multi_axpy<4><<<nb, 256, 0, st>>>(w, Vc, ldv, kc, a, N);
    else if (kc <= 8)
      k_multi_axpy<8><<<nb, 256, 0, st>>>(w, Vc, ldv, kc, a, N);
    else if (kc <= 16)
      k_multi_axpy<16><<<nb, 256, 0, st>>>(w, Vc, ldv, kc, a, N);
    else
      k_multi_axpy<kMaxDots><<<nb, 256, 0, st>>>(w, Vc, ldv, kc, a, N);
  }
}

void launch_axpby(double* y, double a, const double* x, double b, int64_t N, cudaStream_t st) {
  k_axpby<<<stream_blocks(N), 256, 0, st>>>(y, a, x, b, N);
}

}  // namespace mfwh

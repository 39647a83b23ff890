// Temporally blocked MFWH wave step for 2D grids, FP64, sm_103a.
//
// One launch advances the leapfrog scheme (eq. WaveSchemeA; the first step of a
// wave solve as eq. implicitFirstStep with alpha = 0) by up to T steps and
// accumulates the N_f filter sums (eq. pDefQ) on the way.  Each CTA owns a
// 32 x (16 K) tile of output points.  It loads W^n and W^{n-1} on the tile plus
// a halo of T points into shared memory, then steps: at step s it updates the
// tile plus a ring of radius steps-1-s (the points whose values later steps
// still need), so after the last step W^{n+T} and W^{n+T-1} are exact on the
// tile.  Every thread keeps the filter sums q_m of its K owned tile points in
// registers for all T steps, so per point and launch HBM sees one read of the
// two wave levels (with halo), one read-modify-write of the N_f sums and one
// write of the two new levels, instead of T of each.
//
// The per-point arithmetic is the unblocked kernel's (k_step in wave.cu) in the
// same order, so results are bit-identical to it.  The last launch of a wave
// solve can fuse the filter solve V = B^{-1} q (eq. waveHoltzMatrixIteration).
#include <cuda_runtime.h>

#include "fpair.cuh"
#include "kernels.h"

namespace mfwh {
namespace {

constexpr int kTX = 32;   // threads in x = tile width
constexpr int kTY = 16;   // threads in y; tile height = kTY * K

template <int NF>
struct TBParams {
  LayerCoef reg_lo, reg_hi;       // regular step (a_cur = 2, kappa = dt^2)
  LayerCoef first_lo, first_hi;   // first step of a wave solve (a_cur = 1, kappa = dt^2 / 2)
  const double* wq_table;         // [(N_t + 1) * NF] filter weights w_{n,m}
  const double* cos_table;        // [(N_t + 1) * NF] cos(omega~_m t^n)
  double dt2, half_dt2;
  int n0;                         // this launch computes W^{n0+1} .. W^{n0+steps}
  int steps;                      // 1 .. T
  int forced;
  int last;                       // fuse the filter solve; v_out written instead of W and q
  int subtract;                   // v_out = v_sub - V^{k+1}
  int has_e;                      // V^{k+1} = C q + E V^k with E != 0 (explicit filter)
  const double* vprev;            // V^k
  double binv[NF * NF];           // C
  double emat[NF * NF];           // E
};

__device__ __forceinline__ bool interior_pt(int64_t gx, int64_t gy, const Geom& g) {
  return gx > 0 && gx < g.nx && gy > 0 && gy < g.ny;
}

// New level at local point l of the tile (row length EX) from the current level A and the
// previous level B (W^{n-1}, read at the point only); same operation order as k_step.
// fneg: this step's kappa cos(omega~_m t^n), in shared memory.
template <int NF>
__device__ __forceinline__ double update_point(const double* A, const double* B, int l, int ex,
                                               const LayerCoef& L, const double* fneg,
                                               const double* __restrict__ f, int64_t p,
                                               int64_t points, bool forced) {
  const double wc = A[l];
  const double sx = A[l - 1] + A[l + 1];
  const double sy = A[l - ex] + A[l + ex];
  double acc = fma(L.A0, wc, -B[l]);
  acc = fma(L.Ax, sx, acc);
  acc = fma(L.Ay, sy, acc);
  if (forced) {
#pragma unroll
    for (int m = 0; m < NF; ++m) acc = fma(-fneg[m], f[m * points + p], acc);
  }
  return acc;
}

template <int NF, int T, int K>
__global__ void __launch_bounds__(kTX * kTY, 1)
k_tb2d(const double* __restrict__ Wc_in, const double* __restrict__ Wp_in,
       double* __restrict__ Wc_out, double* __restrict__ Wp_out, const double* __restrict__ f,
       float2* __restrict__ q, double* vout, const double* vsub, const TBParams<NF> a,
       const Geom g) {
  constexpr int BX = kTX, BY = kTY * K;
  constexpr int EX = BX + 2 * T, EY = BY + 2 * T;
  extern __shared__ double smem[];
  double* A = smem;             // current level
  double* B = smem + EX * EY;   // previous level, overwritten by the next one
  double* s_wq = smem + 2 * EX * EY;   // [T][NF] filter weights of the new level per step
  double* s_fc = s_wq + T * NF;        // [T][NF] kappa cos(omega~_m t^n) per step
  float* s_wh = reinterpret_cast<float*>(s_fc + T * NF);   // [T][NF] s_wq as float pairs
  float* s_wl = s_wh + T * NF;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kTX + tx;
  constexpr int NT = kTX * kTY;
  const int64_t bx0 = (int64_t)blockIdx.x * BX, by0 = (int64_t)blockIdx.y * BY;
  const int64_t x0 = bx0 - T, y0 = by0 - T;     // global coordinates of smem (0, 0)

  // Load both levels on the tile plus halo; points outside the grid read as 0.
  for (int e = tid; e < EX * EY; e += NT) {
    const int lx = e % EX, ly = e / EX;
    const int64_t gx = x0 + lx, gy = y0 + ly;
    const bool in = gx >= 0 && gx <= g.nx && gy >= 0 && gy <= g.ny;
    const int64_t p = gy * g.sy + gx;
    A[e] = in ? Wc_in[p] : 0.0;
    B[e] = (in && Wp_in != nullptr) ? Wp_in[p] : 0.0;
  }
  // Per-step coefficients of this launch.
  for (int e = tid; e < a.steps * NF; e += NT) {
    const int st = e / NF, m = e % NF;
    const int n = a.n0 + st;
    const double w = a.wq_table[(n + 1) * NF + m];
    s_wq[e] = w;
    s_wh[e] = (float)w;
    s_wl[e] = (float)(w - (double)s_wh[e]);
    s_fc[e] = a.forced ? (n == 0 ? a.half_dt2 : a.dt2) * a.cos_table[n * NF + m] : 0.0;
  }
  // Owned tile points: (T + tx, T + ty + kTY k); their filter sums live in registers as float
  // pairs, updated as in k_step.  The final step of a wave solve (a.last) adds its term in
  // FP64 in the epilogue, as k_last does.
  float2 qr[K][NF];
  double wlast[K];
  int64_t own_p[K];
  bool own_int[K], own_in[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t gx = bx0 + tx, gy = by0 + ty + kTY * k;
    own_in[k] = gx <= g.nx && gy <= g.ny;
    own_int[k] = interior_pt(gx, gy, g);
    own_p[k] = gy * g.sy + gx;
#pragma unroll
    for (int m = 0; m < NF; ++m)
      qr[k][m] = own_int[k] ? q[m * g.points + own_p[k]] : make_float2(0.0f, 0.0f);
    wlast[k] = 0.0;
  }
  __syncthreads();

  for (int s = 0; s < a.steps; ++s) {
    const int r = a.steps - 1 - s;          // ring radius still needed after this step
    const int n = a.n0 + s;                 // computing W^{n+1}
    const bool first = n == 0;
    const LayerCoef lo = first ? a.first_lo : a.reg_lo;
    const LayerCoef hi = first ? a.first_hi : a.reg_hi;
    const double* fneg = s_fc + s * NF;
    const float* wh = s_wh + s * NF;
    const float* wl = s_wl + s * NF;
    const bool final_step = a.last && s == a.steps - 1;
    // owned tile points
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!own_int[k]) continue;
      const int l = (T + ty + kTY * k) * EX + (T + tx);
      const int64_t gx = bx0 + tx, gy = by0 + ty + kTY * k;
      const int64_t li = g.layer_axis == 0 ? gx : gy;
      const LayerCoef& L = li >= g.layer_split ? hi : lo;
      const double wn = update_point<NF>(A, B, l, EX, L, fneg, f, own_p[k], g.points, a.forced);
      B[l] = wn;
      if (final_step) {
        wlast[k] = wn;
      } else {
        const float2 xw = fpair_from(wn);
#pragma unroll
        for (int m = 0; m < NF; ++m) qr[k][m] = fpair_fma(wh[m], wl[m], xw.x, xw.y, qr[k][m]);
      }
    }
    // ring of radius r around the tile (halo points later steps need)
    if (r > 0) {
      const int W = BX + 2 * r;
      const int ring = 2 * r * W + 2 * r * BY;
      for (int e = tid; e < ring; e += NT) {
        int lx, ly;
        if (e < r * W) {
          ly = T - r + e / W;
          lx = T - r + e % W;
        } else if (e < 2 * r * W) {
          const int e2 = e - r * W;
          ly = T + BY + e2 / W;
          lx = T - r + e2 % W;
        } else if (e < 2 * r * W + r * BY) {
          const int e3 = e - 2 * r * W;
          ly = T + e3 / r;
          lx = T - r + e3 % r;
        } else {
          const int e4 = e - 2 * r * W - r * BY;
          ly = T + e4 / r;
          lx = T + BX + e4 % r;
        }
        const int64_t gx = x0 + lx, gy = y0 + ly;
        if (!interior_pt(gx, gy, g)) continue;
        const int64_t li = g.layer_axis == 0 ? gx : gy;
        const LayerCoef& L = li >= g.layer_split ? hi : lo;
        const int l = ly * EX + lx;
        B[l] = update_point<NF>(A, B, l, EX, L, fneg, f, gy * g.sy + gx, g.points, a.forced);
      }
    }
    __syncthreads();
    double* t = A;
    A = B;
    B = t;
  }
  // A = W^{n0+steps}, B = W^{n0+steps-1} on the tile
  if (!a.last) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!own_int[k]) continue;
      const int l = (T + ty + kTY * k) * EX + (T + tx);
      Wc_out[own_p[k]] = A[l];
      Wp_out[own_p[k]] = B[l];
#pragma unroll
      for (int m = 0; m < NF; ++m) q[m * g.points + own_p[k]] = qr[k][m];
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!own_in[k]) continue;
      const double* wq = s_wq + (a.steps - 1) * NF;
      double qq[NF];
#pragma unroll
      for (int j = 0; j < NF; ++j) qq[j] = fma(wq[j], wlast[k], fpair_value(qr[k][j]));
      double vk[NF];
#pragma unroll
      for (int j = 0; j < NF; ++j)
        vk[j] = (a.has_e && own_int[k]) ? a.vprev[j * g.points + own_p[k]] : 0.0;
      double out[NF];
#pragma unroll
      for (int m = 0; m < NF; ++m) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NF; ++j) s = fma(a.binv[m * NF + j], qq[j], s);
        if (a.has_e) {
#pragma unroll
          for (int j = 0; j < NF; ++j) s = fma(a.emat[m * NF + j], vk[j], s);
        }
        out[m] = s;
      }
#pragma unroll
      for (int m = 0; m < NF; ++m) {
        double val = 0.0;
        if (own_int[k]) val = a.subtract ? vsub[m * g.points + own_p[k]] - out[m] : out[m];
        vout[m * g.points + own_p[k]] = val;
      }
    }
  }
}

template <int NF, int T>
void tb_launch_nf(const Geom& g, const double* Wc_in, const double* Wp_in, double* Wc_out,
                  double* Wp_out, const double* f, double* q, double* vout, const double* vsub,
                  const TBHost& h, cudaStream_t st) {
  constexpr int K = NF <= 8 ? 4 : 2;
  constexpr int BX = kTX, BY = kTY * K;
  constexpr int EX = BX + 2 * T, EY = BY + 2 * T;
  constexpr size_t smem = sizeof(double) * (2 * EX * EY + 3 * T * NF);
  // The attribute is per device; set it once per device for this instance.
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_tb2d<NF, T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  TBParams<NF> a;
  a.reg_lo = h.reg_lo;
  a.reg_hi = h.reg_hi;
  a.first_lo = h.first_lo;
  a.first_hi = h.first_hi;
  a.wq_table = h.wq_table;
  a.cos_table = h.cos_table;
  a.dt2 = h.dt2;
  a.half_dt2 = h.half_dt2;
  a.n0 = h.n0;
  a.steps = h.steps;
  a.forced = h.forced;
  a.last = h.last;
  a.subtract = h.subtract;
  a.has_e = h.has_e && h.vprev != nullptr;
  a.vprev = h.vprev;
  for (int m = 0; m < NF; ++m)
    for (int j = 0; j < NF; ++j) {
      a.binv[m * NF + j] = h.binv[m * MFWH_MAX_NF + j];
      a.emat[m * NF + j] = h.emat[m * MFWH_MAX_NF + j];
    }
  dim3 grid((unsigned)((g.nx + 1 + BX - 1) / BX), (unsigned)((g.ny + 1 + BY - 1) / BY));
  k_tb2d<NF, T, K><<<grid, dim3(kTX, kTY), smem, st>>>(Wc_in, Wp_in, Wc_out, Wp_out, f,
                                                       reinterpret_cast<float2*>(q), vout, vsub,
                                                       a, g);
}

template <int NF>
void tb_launch_depth(const Geom& g, const double* Wc_in, const double* Wp_in, double* Wc_out,
                     double* Wp_out, const double* f, double* q, double* vout, const double* vsub,
                     const TBHost& h, cudaStream_t st) {
  if (h.depth <= 4)
    tb_launch_nf<NF, 4>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
  else
    tb_launch_nf<NF, 8>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
}

}  // namespace

void launch_tb2d(int nf, const Geom& g, const double* Wc_in, const double* Wp_in, double* Wc_out,
                 double* Wp_out, const double* f, double* q, double* vout, const double* vsub,
                 const TBHost& h, cudaStream_t st) {
  switch (nf) {
#define CASE(N) \
  case N: tb_launch_depth<N>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st); break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
    CASE(9) CASE(10) CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16)
#undef CASE
    default: break;
  }
}

}  // namespace mfwh

// Temporally blocked MFWH wave step for 2D grids, FP64 wave levels, sm_103a.
//
// The kernel template and its launchers; wave_tb_p1.cu .. wave_tb_p5.cu instantiate them for
// a few frequency counts each (to keep every translation unit's compile time short), and
// wave_tb.cu dispatches on the frequency count.
//
// One launch advances the leapfrog scheme (eq. WaveSchemeA; the first step of a wave solve as
// eq. implicitFirstStep with alpha = 0) by up to T steps and accumulates the N_f filter sums
// (eq. pDefQ) on the way.  The interior points 1..n-1 of each axis are cut into tiles of
// 32 x (TY K) points, one tile per CTA of 32 x TY threads.  A CTA loads W^n and W^{n-1} on its
// tile plus a halo of T points into shared memory; at step s it updates the tile and the ring
// of radius T-1-s around it (the points later steps still read), so after T steps W^{n+T} and
// W^{n+T-1} are exact on the tile.  Per point and launch HBM sees one read and one write of the
// two levels and of the N_f filter sums, instead of T of each.
//
// Thread (tx, ty) owns the K consecutive tile rows ty K .. ty K + K - 1 of column tx: the
// current wave level and the N_f filter sums (float pairs, fpair.cuh) of its points stay in
// registers for all T steps, vertical neighbours come from registers, and only the previous
// level, the left and right neighbours and the rows just above and below the strip come from
// shared memory.  The ring is
// spread evenly over all threads by a flat index.  On sm_103a the FP64 pipe bounds this kernel
// (a warp instruction occupies it for about 64 cycles), so the float pair of each new value is
// split off its bit pattern on the integer and FP32 pipes (fpair_split) and the filter updates
// run on the FP32 pipe: a point-step of the homogeneous 5-point scheme costs two FP64 adds and
// three FP64 FMAs.
//
// The per-point arithmetic is the unblocked kernel's (k_step in wave.cu) in the same order, so
// results are bit-identical to it.  The last launch of a wave solve fuses the filter solve
// V = C q + E V^k (eq. waveHoltzMatrixIteration; E = 0 for the implicit filter).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "fpair.cuh"
#include "kernels.h"

namespace mfwh {
namespace {

constexpr int kTX = 32;   // threads in x = tile width

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
  // launches of at most 4 steps (the persistent kernel): w_{n+1,m} of step s as a float pair
  // and the forcing coefficients kappa cos(omega~_m t^n), [s * NF + m]
  float wph[4 * NF], wpl[4 * NF];
  double fcp[4 * NF];
};

// Clamp a local coordinate bound (64-bit global difference) to [lo, hi].
__device__ __forceinline__ int clamp_local(int64_t v, int lo, int hi) {
  return (int)(v < lo ? lo : (v > hi ? hi : v));
}

// New level at local point l (row length EX) of a ring point: the operations of k_step in the
// same order.  A: W^n, wprev: W^{n-1} at l (0 on the first step of a wave solve, where the
// first-step coefficients make the update W^1 = W^0 + dt^2/2 (c^2 Delta_h W^0 - F^0)).
template <int NF, int EX, bool FORCED>
__device__ __forceinline__ double ring_update(const double* A, double wprev, int l,
                                              const LayerCoef& L, const double* fneg,
                                              const double* __restrict__ f, int64_t p,
                                              int64_t points) {
  const double wc = A[l];
  const double sx = A[l - 1] + A[l + 1];
  const double sy = A[l - EX] + A[l + EX];
  double acc = fma(L.A0, wc, -wprev);     // wprev = 0 on the first step: exactly L.A0 * wc
  acc = fma(L.Ax, sx, acc);
  acc = fma(L.Ay, sy, acc);
  if (FORCED) {
#pragma unroll
    for (int m = 0; m < NF; ++m) acc = fma(-fneg[m], f[m * points + p], acc);
  }
  return acc;
}

// ceil(2^32 / d) for 2 <= d < 128, a table in constant memory filled at compile time: the
// multiplier of the exact division floor(e / d) = (e * m) >> 32 for the small ring indices e
// of the blocked kernels (e < 2^16; checked exhaustively on the host).
struct DivMagic {
  unsigned m[128];
};
constexpr DivMagic make_div_magic() {
  DivMagic t{};
  for (int d = 2; d < 128; ++d) t.m[d] = 0xFFFFFFFFu / (unsigned)d + 1u;
  return t;
}
__constant__ DivMagic c_div_magic = make_div_magic();
__device__ __forceinline__ unsigned div_magic(int d) { return c_div_magic.m[d]; }

// Local coordinates of flat ring index e at radius r: the 2r rows of BX + 2r points above and
// below the tile, then the BY rows of 2r points left and right of it.  Quotients by the row
// lengths are integer divisions by multipliers m_rw = div_magic(rw), m_2r = div_magic(2r).
template <int T, int BX, int BY>
__device__ __forceinline__ void ring_coords(int e, int r, int rw, int top, unsigned m_rw,
                                            unsigned m_2r, int& lx, int& ly) {
  if (e < top) {
    const int row = (int)__umulhi((unsigned)e, m_rw);
    lx = T - r + (e - row * rw);
    ly = row < r ? T - r + row : T + BY + row - r;
  } else {
    const int e2 = e - top;
    const int row = (int)__umulhi((unsigned)e2, m_2r);
    const int col = e2 - row * 2 * r;
    ly = T + row;
    lx = col < r ? T - r + col : T + BX + col - r;
  }
}

// TY threads in y, MB CTAs per SM at least (registers per thread at most 65536 / (MB 32 TY)).
// Several CTAs per SM let one CTA's loads, stores and barriers overlap another's FP64 work.
template <int NF, int T, int K, int TY, int MB>
__global__ void __launch_bounds__(kTX * TY, MB)
k_tb2d(const double* __restrict__ Wc_in, const double* __restrict__ Wp_in,
       double* __restrict__ Wc_out, double* __restrict__ Wp_out, const double* __restrict__ f,
       float2* __restrict__ q, double* vout, const double* vsub, const TBParams<NF> a,
       const Geom g) {
  constexpr int BX = kTX, BY = TY * K;
  constexpr int EX = BX + 2 * T, EY = BY + 2 * T, E = EX * EY;
  constexpr int NT = kTX * TY;
  extern __shared__ double smem[];
  double* A = smem;                  // W^n on the extended tile
  double* B = smem + E;              // W^{n-1} on the ring, overwritten by W^{n+1}
  double* s_wq = smem + 2 * E;       // [T][NF] filter weights of the new level per step
  double* s_fc = s_wq + T * NF;      // [T][NF] kappa cos(omega~_m t^n) per step
  float* s_wh = reinterpret_cast<float*>(s_fc + T * NF);   // [T][NF] s_wq as float pairs
  float* s_wl = s_wh + T * NF;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
  // global coordinates of local (0, 0); tiles start at the first interior point
  const int64_t x0 = 1 + (int64_t)blockIdx.x * BX - T, y0 = 1 + (int64_t)blockIdx.y * BY - T;
  // local bounds: grid points [gl, gh], interior points [il, ih] (32-bit)
  const int glx = clamp_local(-x0, 0, EX), ghx = clamp_local(g.nx - x0, -1, EX - 1);
  const int gly = clamp_local(-y0, 0, EY), ghy = clamp_local(g.ny - y0, -1, EY - 1);
  const int ilx = clamp_local(1 - x0, 0, EX), ihx = clamp_local(g.nx - 1 - x0, -1, EX - 1);
  const int ily = clamp_local(1 - y0, 0, EY), ihy = clamp_local(g.ny - 1 - y0, -1, EY - 1);
  // c^2 layer: points whose local coordinate along the layer axis is >= lay_thr use hi
  const bool lay_x = g.layer_axis == 0;
  const int lay_thr = clamp_local(g.layer_split - (lay_x ? x0 : y0), -1, EX + EY);
  // every point updated by any step interior, all with one c^2: no per-point tests needed
  const bool simple = ilx <= 1 && ihx >= EX - 2 && ily <= 1 && ihy >= EY - 2 &&
                      (lay_thr <= 0 || lay_thr >= (lay_x ? EX : EY));
  const bool all_hi = lay_thr <= 0;

  // Both levels on the tile plus halo; points outside the grid read as 0.
  for (int e = tid; e < E; e += NT) {
    const int ly = e / EX, lx = e - ly * EX;
    const bool in = ly >= gly && ly <= ghy && lx >= glx && lx <= ghx &&
                    MFWH_IDX(g.fault, (y0 + ly) * g.sy + x0 + lx, g.points);
    const int64_t p = (y0 + ly) * g.sy + x0 + lx;
    A[e] = in ? Wc_in[p] : 0.0;
    B[e] = (in && Wp_in != nullptr) ? Wp_in[p] : 0.0;
  }
  // Per-step coefficients of this launch.
  for (int e = tid; e < a.steps * NF; e += NT) {
    const int st = e / NF, m = e - st * NF;
    const int n = a.n0 + st;
    const double w = a.wq_table[(n + 1) * NF + m];
    s_wq[e] = w;
    const float wh = (float)w;
    s_wh[e] = wh;
    s_wl[e] = (float)(w - (double)wh);
    s_fc[e] = a.forced ? (n == 0 ? a.half_dt2 : a.dt2) * a.cos_table[n * NF + m] : 0.0;
  }
  // The strip: local column lxo, rows lyo .. lyo + K - 1.
  const int lxo = T + tx, lyo = T + ty * K;
  const int64_t p0 = (y0 + lyo) * g.sy + x0 + lxo;
  const bool col_int = lxo >= ilx && lxo <= ihx;
  bool own_int[K], own_up[K];
  double wc[K];
  float2 qr[K][NF];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    own_int[k] = col_int && lyo + k >= ily && lyo + k <= ihy;
    own_up[k] = (lay_x ? lxo : lyo + k) >= lay_thr;
#pragma unroll
    for (int m = 0; m < NF; ++m)
      qr[k][m] = own_int[k] ? q[m * g.points + p0 + k * g.sy] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) wc[k] = A[(lyo + k) * EX + lxo];

  // The steps in three compiled copies with the same per-point arithmetic: ALLINT for
  // homogeneous launches of CTAs whose updated points are all interior with one c^2 (no
  // forcing terms, no per-point interior or layer tests), and the general one with and
  // without the forcing terms (FORCED), so that no copy carries FP64 work under a predicate.
  // The filter update of a step's new values is deferred into the next step, after that
  // step's FP64 stencil in the same block, so that each warp's FP32 pair arithmetic overlaps
  // FP64 work instead of following it behind the step's barrier; the updates keep their order.
  float2 pend[K];   // float pairs of the newest owned values, not yet added to the sums
  auto filter_update = [&](int s) {   // add pend with the weights of step s
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!own_int[k]) continue;
#pragma unroll
      for (int m = 0; m < NF; ++m)
        qr[k][m] = fpair_fma(s_wh[s * NF + m], s_wl[s * NF + m], pend[k].x, pend[k].y, qr[k][m]);
    }
  };
  // The steps in three compiled copies with the same per-point arithmetic: ALLINT for
  // homogeneous launches of CTAs whose updated points are all interior with one c^2 (no
  // forcing terms, no per-point interior or layer tests), and the general one with and
  // without the forcing terms (FORCED), so that no copy carries FP64 work under a predicate.
  auto run_steps = [&](auto allint_c, auto forced_c) {
    constexpr bool ALLINT = decltype(allint_c)::value;
    constexpr bool FORCED = decltype(forced_c)::value;
    auto step = [&](int s, auto defer_c) {
      constexpr bool DEFER = decltype(defer_c)::value;   // the previous step's update pending
      const int r = a.steps - 1 - s;          // ring radius still needed after this step
      const int n = a.n0 + s;                 // computing W^{n+1}
      const bool first = n == 0;
      const LayerCoef& lo = first ? a.first_lo : a.reg_lo;
      const LayerCoef& hi = first ? a.first_hi : a.reg_hi;
      const double* fneg = s_fc + s * NF;
      const bool final_step = a.last && s == a.steps - 1;
      // owned strip: centre and vertical neighbours from registers
      {
        const double above = A[(lyo - 1) * EX + lxo];
        const double below = A[(lyo + K) * EX + lxo];
        double wn[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          wn[k] = wc[k];
          if (!ALLINT && !own_int[k]) continue;   // boundary and outside points keep W = 0
          const int l = (lyo + k) * EX + lxo;
          const LayerCoef& L = ALLINT ? (all_hi ? hi : lo) : (own_up[k] ? hi : lo);
          const double up = k == 0 ? above : wc[k - 1];
          const double dn = k == K - 1 ? below : wc[k + 1];
          const double sx = A[l - 1] + A[l + 1];
          const double sy = up + dn;
          // W^{n-1} of the strip is still in B (0 on the first step)
          double acc = fma(L.A0, wc[k], -B[l]);
          acc = fma(L.Ax, sx, acc);
          acc = fma(L.Ay, sy, acc);
          if (FORCED) {
#pragma unroll
            for (int m = 0; m < NF; ++m)
              acc = fma(-fneg[m], f[m * g.points + p0 + k * g.sy], acc);
          }
          wn[k] = acc;
        }
        if (DEFER) filter_update(s - 1);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (!ALLINT && !own_int[k]) continue;
          B[(lyo + k) * EX + lxo] = wn[k];
          wc[k] = wn[k];
          // the last level of a wave solve enters the sums in FP64 in the epilogue
          if (!final_step) pend[k] = fpair_split(wn[k]);
        }
      }
      // ring of radius r around the tile
      if (r > 0) {
        const int rw = BX + 2 * r;
        const int top = 2 * r * rw;
        const int ring = top + 2 * r * BY;
        const unsigned m_rw = div_magic(rw), m_2r = div_magic(2 * r);
        for (int e = tid; e < ring; e += NT) {
          int lx, ly;
          ring_coords<T, BX, BY>(e, r, rw, top, m_rw, m_2r, lx, ly);
          if (!ALLINT && !simple && (lx < ilx || lx > ihx || ly < ily || ly > ihy)) continue;
          if (!MFWH_IDX(g.fault, ly * EX + lx - EX, E) || !MFWH_IDX(g.fault, ly * EX + lx + EX, E))
            continue;
          const LayerCoef& L =
              (ALLINT || simple) ? (all_hi ? hi : lo) : (((lay_x ? lx : ly) >= lay_thr) ? hi : lo);
          const int l = ly * EX + lx;
          const int64_t p = (y0 + ly) * g.sy + x0 + lx;
          B[l] = ring_update<NF, EX, FORCED>(A, B[l], l, L, fneg, f, p, g.points);
        }
      }
      __syncthreads();
      double* t = A;
      A = B;
      B = t;
    };
    step(0, std::false_type{});
    for (int s = 1; s < a.steps; ++s) step(s, std::true_type{});
  };
  if (a.forced)
    run_steps(std::false_type{}, std::true_type{});
  else if (simple)
    run_steps(std::true_type{}, std::false_type{});
  else
    run_steps(std::false_type{}, std::false_type{});
  // the last step's update (except for the final level of a wave solve)
  if (!a.last) filter_update(a.steps - 1);

  // wc = W^{n0+steps} on the strip, B = W^{n0+steps-1}
  if (!a.last) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!own_int[k]) continue;
      const int64_t p = p0 + k * g.sy;
      if (!MFWH_IDX(g.fault, p, g.points)) continue;
      Wc_out[p] = wc[k];
      Wp_out[p] = B[(lyo + k) * EX + lxo];
#pragma unroll
      for (int m = 0; m < NF; ++m) q[m * g.points + p] = qr[k][m];
    }
    return;
  }
  // Last launch: V^{k+1} = C (q + w_{N_t} W^{N_t}) + E V^k at the interior points, 0 on the
  // boundary points of this CTA's part of the grid.
  const double* wq = s_wq + (a.steps - 1) * NF;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!own_int[k]) continue;
    const int64_t p = p0 + k * g.sy;
    double qq[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) qq[j] = fma(wq[j], wc[k], fpair_value(qr[k][j]));
    double vk[NF];
    if (a.has_e) {
#pragma unroll
      for (int j = 0; j < NF; ++j) vk[j] = a.vprev[j * g.points + p];
    }
    double out[NF];
#pragma unroll
    for (int m = 0; m < NF; ++m) {
      double sacc = 0.0;
#pragma unroll
      for (int j = 0; j < NF; ++j) sacc = fma(a.binv[m * NF + j], qq[j], sacc);
      if (a.has_e) {
#pragma unroll
        for (int j = 0; j < NF; ++j) sacc = fma(a.emat[m * NF + j], vk[j], sacc);
      }
      out[m] = sacc;
    }
#pragma unroll
    for (int m = 0; m < NF; ++m)
      vout[m * g.points + p] = a.subtract ? vsub[m * g.points + p] - out[m] : out[m];
  }
  // Boundary points: the CTA at each edge of the tile grid writes the boundary lines along
  // its part of that edge (the parts partition the edges, corners included).
  const int64_t xs = blockIdx.x == 0 ? 0 : 1 + (int64_t)blockIdx.x * BX;
  const int64_t xe = blockIdx.x == gridDim.x - 1 ? g.nx + 1 : 1 + (int64_t)(blockIdx.x + 1) * BX;
  const int64_t ys = blockIdx.y == 0 ? 0 : 1 + (int64_t)blockIdx.y * BY;
  const int64_t ye = blockIdx.y == gridDim.y - 1 ? g.ny + 1 : 1 + (int64_t)(blockIdx.y + 1) * BY;
  auto zero_point = [&](int64_t gx, int64_t gy) {
#pragma unroll
    for (int m = 0; m < NF; ++m) vout[m * g.points + gy * g.sy + gx] = 0.0;
  };
  if (ys == 0)
    for (int64_t gx = xs + tid; gx < xe; gx += NT) zero_point(gx, 0);
  if (ye == g.ny + 1)
    for (int64_t gx = xs + tid; gx < xe; gx += NT) zero_point(gx, g.ny);
  if (xs == 0)
    for (int64_t gy = ys + tid; gy < ye; gy += NT) zero_point(0, gy);
  if (xe == g.nx + 1)
    for (int64_t gy = ys + tid; gy < ye; gy += NT) zero_point(g.nx, gy);
}

// ---- persistent, software-pipelined variant (tile shape 5) ---------------------------------
//
// On sm_103a the FP64 pipe executes two lanes per SM and cycle, so a warp's FP64 instruction
// holds it for 64 cycles of its SM sub-partition, and the five FP64 instructions of a
// point-step are as long as about 300 issued instructions of other kinds.  This variant keeps
// the instruction stream between them short and the FP64 pipe fed from several CTAs:
//   - each CTA stays resident and walks a list of 32 x 16-point tiles (one point per thread,
//     512 threads, up to three CTAs per SM);
//   - while it steps one tile, the next tile's two wave levels (with their T-point halo) are
//     already on their way into the other half of a double buffer in shared memory (cp.async),
//     and the next tile's filter sums follow as soon as this tile's have been used;
//   - the step loop holds only the stencil and the float-pair split of each new value; the
//     N_f filter updates of all T steps run once at the end of the tile, from the T pairs kept
//     in registers, in step order for each frequency.
// The per-step coefficients travel as kernel parameters.  Per point the arithmetic is that of
// k_step in the same order (each q_m receives the same float-pair updates in the same
// sequence), so results are bit-identical to one step per launch.  Every launch runs exactly T
// steps; the last launch of a wave solve (the filter solve fused into it) and launches of fewer
// steps run on the shape-4 kernel.  No CTA waits on another.

// f(integral_constant<int, I>) for I = B .. E - 1, in order.
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Asynchronous 8-byte copy global -> shared; src_bytes = 0 writes zeros and reads nothing.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}
// Wait until at most the most recent commit group of this thread is still in flight.
__device__ __forceinline__ void cp_async_wait_prior() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

constexpr int kPipeTY = 16, kPipeThreads = kTX * kPipeTY;

// K rows per thread: 32 x 16 K-point tiles; three CTAs per SM for K = 1, two for K = 2.  The
// library runs K = 1 (tile shape 5): K = 2 (a smaller halo ring, two FMA chains per thread, but
// 32 instead of 48 resident warps per SM) measured 0.91x of it at depth 3.
template <int K>
constexpr int pipe_min_blocks() {
  return K == 1 ? 3 : 2;
}

template <int NF, int T, int K>
constexpr size_t pipe_smem_bytes() {
  return sizeof(double) * 4 * (kTX + 2 * T) * (kPipeTY * K + 2 * T) +
         sizeof(float2) * NF * K * kPipeThreads;
}

template <int NF, int T, int K>
__global__ void __launch_bounds__(kPipeThreads, pipe_min_blocks<K>())
k_tb2d_pipe(const double* __restrict__ Wc_in, const double* __restrict__ Wp_in,
            double* __restrict__ Wc_out, double* __restrict__ Wp_out,
            const double* __restrict__ f, float2* __restrict__ q, const TBParams<NF> a,
            const Geom g, int tiles_x, int tiles_y) {
  constexpr int BX = kTX, BY = kPipeTY * K, NT = kPipeThreads;
  constexpr int EX = BX + 2 * T, EY = BY + 2 * T, E = EX * EY;
  extern __shared__ double smem[];
  double* stage = smem;                                      // [2][A, B][E]
  float2* qbuf = reinterpret_cast<float2*>(smem + 4 * E);    // [NF][K][NT] sums of own points
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int n_tiles = tiles_x * tiles_y;
  // the thread's own points: column lxo, rows lyo .. lyo + K - 1
  const int lxo = T + tx, lyo = T + ty * K, lown = lyo * EX + lxo;

  // Global index of own point k in a tile, or -1 outside the interior.
  auto own_index = [&](int tile, int k) -> int64_t {
    const int bx = tile % tiles_x, by = tile / tiles_x;
    const int64_t gx = 1 + (int64_t)bx * BX + tx, gy = 1 + (int64_t)by * BY + ty * K + k;
    return (gx <= g.nx - 1 && gy <= g.ny - 1 && MFWH_IDX(g.fault, gy * g.sy + gx, g.points))
               ? gy * g.sy + gx
               : -1;
  };
  // Both levels of a tile on its extended tile into half h (zeros outside the grid, and for
  // W^{n-1} before the first step).
  auto prefetch_levels = [&](int tile, int h) {
    const int bx = tile % tiles_x, by = tile / tiles_x;
    const int64_t x0 = 1 + (int64_t)bx * BX - T, y0 = 1 + (int64_t)by * BY - T;
    double* A = stage + 2 * h * E;
    for (int e = tid; e < E; e += NT) {
      const int ly = e / EX, lx = e - ly * EX;
      const int64_t gx = x0 + lx, gy = y0 + ly;
      const bool in = gx >= 0 && gx <= g.nx && gy >= 0 && gy <= g.ny &&
                      MFWH_IDX(g.fault, gy * g.sy + gx, g.points);
      const int64_t p = in ? gy * g.sy + gx : 0;
      cp_async8(A + e, Wc_in + p, in ? 8 : 0);
      cp_async8(A + E + e, (Wp_in != nullptr ? Wp_in : Wc_in) + p,
                (in && Wp_in != nullptr) ? 8 : 0);
    }
  };
  // The own points' filter sums (each thread copies and later reads only its own slots).
  auto prefetch_sums = [&](int tile) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t p = own_index(tile, k);
#pragma unroll
      for (int m = 0; m < NF; ++m)
        cp_async8(qbuf + (m * K + k) * NT + tid, q + m * g.points + (p < 0 ? 0 : p),
                  p < 0 ? 0 : 8);
    }
  };

  // Copies go in two kinds of commit groups, levels then sums, one of each per tile (empty when
  // there is no next tile): a tile's levels are awaited at its start, its sums only at its end,
  // so the sums have the whole tile's steps to arrive.
  int tile = blockIdx.x;
  if (tile < n_tiles) {
    prefetch_levels(tile, 0);
    cp_async_commit();
    prefetch_sums(tile);
    cp_async_commit();
  }

  for (int h = 0; tile < n_tiles; tile += gridDim.x, h ^= 1) {
    cp_async_wait_prior();   // this tile's levels (its sums may still be in flight)
    __syncthreads();         // ... are in half h for every thread; half h ^ 1 is free
    const int next = tile + (int)gridDim.x;
    if (next < n_tiles) prefetch_levels(next, h ^ 1);
    cp_async_commit();
    const int bx = tile % tiles_x, by = tile / tiles_x;
    const int64_t x0 = 1 + (int64_t)bx * BX - T, y0 = 1 + (int64_t)by * BY - T;
    const int ilx = clamp_local(1 - x0, 0, EX), ihx = clamp_local(g.nx - 1 - x0, -1, EX - 1);
    const int ily = clamp_local(1 - y0, 0, EY), ihy = clamp_local(g.ny - 1 - y0, -1, EY - 1);
    const bool lay_x = g.layer_axis == 0;
    const int lay_thr = clamp_local(g.layer_split - (lay_x ? x0 : y0), -1, EX + EY);
    const bool simple = ilx <= 1 && ihx >= EX - 2 && ily <= 1 && ihy >= EY - 2 &&
                        (lay_thr <= 0 || lay_thr >= (lay_x ? EX : EY));
    const bool all_hi = lay_thr <= 0;
    bool own_int[K], own_up[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      own_int[k] = lxo >= ilx && lxo <= ihx && lyo + k >= ily && lyo + k <= ihy;
      own_up[k] = (lay_x ? lxo : lyo + k) >= lay_thr;
    }
    const int64_t p0 = (y0 + lyo) * g.sy + x0 + lxo;
    double* A = stage + 2 * h * E;   // W^n on the extended tile
    double* B = A + E;               // W^{n-1}, overwritten by W^{n+1}
    double wc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) wc[k] = A[lown + k * EX];
    float2 pend[K][T];               // float pairs of the tile's new own values, step by step
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int s = 0; s < T; ++s) pend[k][s] = make_float2(0.0f, 0.0f);

    // The T steps, each with its ring radius r = T - 1 - s known at compile time (every launch
    // of this kernel runs exactly T steps): the ring has at most one point per thread and its
    // decode divides by constants.
    auto run_steps = [&](auto allint_c, auto forced_c) {
      constexpr bool ALLINT = decltype(allint_c)::value;
      constexpr bool FORCED = decltype(forced_c)::value;
      static_for<0, T>([&](auto s_c) {
        constexpr int s = decltype(s_c)::value;
        constexpr int r = T - 1 - s;
        const bool first = a.n0 + s == 0;
        const double* fneg = a.fcp + s * NF;
        // own points: vertical neighbours inside the strip from registers
        double wn[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          wn[k] = wc[k];
          if (!(ALLINT || own_int[k])) continue;
          const int l = lown + k * EX;
          const double up = k == 0 ? A[l - EX] : wc[k - 1];
          const double dn = k == K - 1 ? A[l + EX] : wc[k + 1];
          const double sx = A[l - 1] + A[l + 1];
          const double sy = up + dn;
          // the point's coefficients (the first step of a wave solve has its own)
          const bool upper = ALLINT ? all_hi : own_up[k];
          const LayerCoef& L =
              first ? (upper ? a.first_hi : a.first_lo) : (upper ? a.reg_hi : a.reg_lo);
          double acc = fma(L.A0, wc[k], -B[l]);
          acc = fma(L.Ax, sx, acc);
          acc = fma(L.Ay, sy, acc);
          if (FORCED) {
#pragma unroll
            for (int m = 0; m < NF; ++m)
              acc = fma(-fneg[m], f[m * g.points + p0 + k * g.sy], acc);
          }
          wn[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (!(ALLINT || own_int[k])) continue;
          B[lown + k * EX] = wn[k];
          wc[k] = wn[k];
          pend[k][s] = fpair_split(wn[k]);
        }
        if constexpr (r > 0) {
          // ring of radius r: the 2r rows of RW points above and below the tile, then the BY
          // rows of 2r points left and right of it
          constexpr int RW = BX + 2 * r, TOP = 2 * r * RW, RING = TOP + 2 * r * BY;
          static_assert(RING <= NT, "one ring point per thread at most");
          if (tid < RING) {
            int lx, ly;
            if (tid < TOP) {
              const int row = tid / RW;
              lx = T - r + (tid - row * RW);
              ly = row < r ? T - r + row : T + BY + row - r;
            } else {
              const int e2 = tid - TOP;
              const int row = e2 / (2 * r), col = e2 - row * (2 * r);
              ly = T + row;
              lx = col < r ? T - r + col : T + BX + col - r;
            }
            if ((ALLINT || simple || (lx >= ilx && lx <= ihx && ly >= ily && ly <= ihy)) &&
                MFWH_IDX(g.fault, ly * EX + lx - EX, E) && MFWH_IDX(g.fault, ly * EX + lx + EX, E)) {
              const LayerCoef& lo = first ? a.first_lo : a.reg_lo;
              const LayerCoef& hi = first ? a.first_hi : a.reg_hi;
              const LayerCoef& L = (ALLINT || simple)
                                       ? (all_hi ? hi : lo)
                                       : (((lay_x ? lx : ly) >= lay_thr) ? hi : lo);
              const int l = ly * EX + lx;
              const int64_t p = (y0 + ly) * g.sy + x0 + lx;
              B[l] = ring_update<NF, EX, FORCED>(A, B[l], l, L, fneg, f, p, g.points);
            }
          }
        }
        __syncthreads();
        double* t = A;
        A = B;
        B = t;
      });
    };
    if (a.forced)
      run_steps(std::false_type{}, std::true_type{});
    else if (simple)
      run_steps(std::true_type{}, std::false_type{});
    else
      run_steps(std::false_type{}, std::false_type{});

    // The filter updates of the tile's steps, then the sums' slots take the next tile's sums.
    cp_async_wait_prior();   // this thread's sums of this tile (the next tile's levels may pend)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t pk = p0 + k * g.sy;
      if (!own_int[k] || !MFWH_IDX(g.fault, pk, g.points)) continue;
      Wc_out[pk] = wc[k];
      Wp_out[pk] = B[lown + k * EX];
      // one frequency at a time: few registers live
#pragma unroll
      for (int m = 0; m < NF; ++m) {
        float2 qm = qbuf[(m * K + k) * NT + tid];
#pragma unroll
        for (int s = 0; s < T; ++s)
          qm = fpair_fma(a.wph[s * NF + m], a.wpl[s * NF + m], pend[k][s].x, pend[k][s].y, qm);
        q[m * g.points + pk] = qm;
      }
    }
    if (next < n_tiles) prefetch_sums(next);
    cp_async_commit();
  }
  cp_async_wait_all();   // no copy of this CTA outlives it
}

template <int NF, int T>
TBParams<NF> tb_params(const TBHost& h) {
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
  for (int s = 0; s < 4; ++s)
    for (int m = 0; m < NF; ++m) {
      const int n = h.n0 + s;
      const bool in = s < h.steps && h.wq_host != nullptr;
      const double w = in ? h.wq_host[(size_t)(n + 1) * NF + m] : 0.0;
      const float wh = (float)w;
      a.wph[s * NF + m] = wh;
      a.wpl[s * NF + m] = (float)(w - (double)wh);
      a.fcp[s * NF + m] =
          (in && h.forced) ? (n == 0 ? h.half_dt2 : h.dt2) * h.cos_host[(size_t)n * NF + m] : 0.0;
    }
  return a;
}

template <int NF, int T, int K>
void tb_launch_pipe(const Geom& g, const double* Wc_in, const double* Wp_in, double* Wc_out,
                    double* Wp_out, const double* f, double* q, const TBHost& h,
                    cudaStream_t st) {
  constexpr size_t smem = pipe_smem_bytes<NF, T, K>();
  // Attribute and resident CTAs per SM, once per device for this instance.
  static int resident[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = (dev >= 0 && dev < 64) ? resident[dev] : 0;
  if (per_sm == 0) {
    cudaFuncSetAttribute(k_tb2d_pipe<NF, T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tb2d_pipe<NF, T, K>, kPipeThreads,
                                                      smem) != cudaSuccess || occ < 1)
      occ = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
      sms = 1;
    per_sm = occ * sms;
    if (dev >= 0 && dev < 64) resident[dev] = per_sm;
  }
  const TBParams<NF> a = tb_params<NF, T>(h);
  const int tiles_x = (int)((g.nx - 1 + kTX - 1) / kTX);
  const int tiles_y = (int)((g.ny - 1 + kPipeTY * K - 1) / (kPipeTY * K));
  const int grid = std::min(tiles_x * tiles_y, per_sm);
  k_tb2d_pipe<NF, T, K><<<grid, dim3(kTX, kPipeTY), smem, st>>>(
      Wc_in, Wp_in, Wc_out, Wp_out, f, reinterpret_cast<float2*>(q), a, g, tiles_x, tiles_y);
}

template <int NF, int T, int K, int TY, int MB>
void tb_launch_k(const Geom& g, const double* Wc_in, const double* Wp_in, double* Wc_out,
                 double* Wp_out, const double* f, double* q, double* vout, const double* vsub,
                 const TBHost& h, cudaStream_t st) {
  constexpr int BX = kTX, BY = TY * K;
  constexpr int EX = BX + 2 * T, EY = BY + 2 * T;
  constexpr size_t smem = sizeof(double) * (2 * EX * EY + 2 * T * NF) + sizeof(float) * 2 * T * NF;
  // The attribute is per device; set it once per device for this instance.
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_tb2d<NF, T, K, TY, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  const TBParams<NF> a = tb_params<NF, T>(h);
  // tiles over the interior points 1 .. n-1 of each axis
  dim3 grid((unsigned)((g.nx - 1 + BX - 1) / BX), (unsigned)((g.ny - 1 + BY - 1) / BY));
  k_tb2d<NF, T, K, TY, MB><<<grid, dim3(kTX, TY), smem, st>>>(Wc_in, Wp_in, Wc_out, Wp_out, f,
                                                          reinterpret_cast<float2*>(q), vout,
                                                          vsub, a, g);
}

// Tile shapes (points in x by y, threads, CTAs per SM):
//   0 = 32 x 64, 512 threads, 4 rows each;   1 = 32 x 32, 512 threads, 2 rows each;
//   2 = 32 x 48, 512 threads, 3 rows each;   3 = 32 x 32, 256 threads, 4 rows each, 2 per SM;
//   4 = 32 x 16, 512 threads, 1 row each, 2 per SM (64 registers per thread);
//   5 = shape 4's tiles, stepped by persistent CTAs that copy the next tile while stepping one
//       (k_tb2d_pipe; up to 8 frequencies, depths 2 to 4).
// Shapes 4 and 5 serve the shallow depths 2, 3 and 4: few registers per thread keep enough
// warps resident.  Depths 2 and 3 take shape 1 for shapes 0 to 3, depth 8 takes shape 3 for 4
// and 5.  Above 8 frequencies the filter sums of more than two points per thread would not fit
// in registers: shape 5 takes shape 4 and shapes 0 to 3 take shape 1.
template <int NF, int T>
void tb_launch_shape(const Geom& g, const double* Wc_in, const double* Wp_in, double* Wc_out,
                     double* Wp_out, const double* f, double* q, double* vout, const double* vsub,
                     const TBHost& h, cudaStream_t st) {
  constexpr bool wide = NF > 8;
  int shape = h.shape;
  if (T == 8 && shape >= 4) shape = wide ? 1 : 3;
  if (wide && shape == 5) shape = 4;
  // the launch with the fused filter solve, and any launch of fewer than T steps, run on shape 4
  if (shape == 5 && (h.last || h.steps != T)) shape = 4;
  if (shape < 4 && (wide || T <= 3)) shape = 1;
  switch (shape) {
    case 5:
      if constexpr (!wide && T <= 4)
        tb_launch_pipe<NF, T, 1>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, h, st);
      break;

    case 4:
      if constexpr (T <= 4)
        tb_launch_k<NF, T, 1, 16, 2>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
      break;
    case 1:
      tb_launch_k<NF, T, 2, 16, 1>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
      break;
    case 2:
      if constexpr (!wide && T >= 4)
        tb_launch_k<NF, T, 3, 16, 1>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
      break;
    case 3:
      if constexpr (!wide && T >= 4)
        tb_launch_k<NF, T, 4, 8, 2>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
      break;
    default:
      if constexpr (!wide && T >= 4)
        tb_launch_k<NF, T, 4, 16, 1>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
      break;
  }
}

// Up to h.depth (2, 3, 4 or 8) steps of an NF-frequency 2D grid in one launch.
template <int NF>
void tb_launch_nf(const Geom& g, const double* Wc_in, const double* Wp_in, double* Wc_out,
                  double* Wp_out, const double* f, double* q, double* vout, const double* vsub,
                  const TBHost& h, cudaStream_t st) {
  if (h.depth <= 2)
    tb_launch_shape<NF, 2>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
  else if (h.depth == 3)
    tb_launch_shape<NF, 3>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
  else if (h.depth == 4)
    tb_launch_shape<NF, 4>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
  else
    tb_launch_shape<NF, 8>(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
}

}  // namespace

using TbFn = void (*)(const Geom&, const double*, const double*, double*, double*, const double*,
                      double*, double*, const double*, const TBHost&, cudaStream_t);
TbFn tb_fn_p1(int nf);   // wave_tb_p1.cu: 1-3 frequencies
TbFn tb_fn_p2(int nf);   // wave_tb_p2.cu: 4-6
TbFn tb_fn_p3(int nf);   // wave_tb_p3.cu: 7-8
TbFn tb_fn_p4(int nf);   // wave_tb_p4.cu: 9-12
TbFn tb_fn_p5(int nf);   // wave_tb_p5.cu: 13-16

}  // namespace mfwh

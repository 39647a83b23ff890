// FP32 MFWH wave solve with compensated filter sums, sm_103a.
//
// The wave levels are FP32 and the leapfrog scheme (eq. WaveSchemeA, first step
// eq. implicitFirstStep with alpha = 0) is advanced in its increment form
//   D^{n+1/2} = D^{n-1/2} + kappa_n (c^2 Delta_h W^n - F^n),   W^{n+1} = W^n + D^{n+1/2},
// with D^{-1/2} = 0, kappa_0 = dt^2/2 and kappa_n = dt^2 otherwise.  In exact
// arithmetic this is the same recurrence as W^{n+1} = 2W^n - W^{n-1} + ...; in
// FP32 it keeps the velocity D exactly where the two-level form would round it,
// so a rounding of W^{n+1} stays a position error instead of turning into a
// velocity error that grows over the N_t steps.  The Laplacian is taken as sums
// of neighbour differences, (W_e - W) + (W_w - W), which are small and nearly
// exact for smooth fields.
//
// The filter sums q_m = sum_n w_{n,m} W^n (eq. pDefQ) are accumulated in FP32
// with Kahan's compensated summation: a pair (s_m, c_m) per point and frequency,
// q_m = s_m - c_m.  The filter solve V = B^{-1} q (eq. waveHoltzMatrixIteration)
// and everything after it are FP64.
//
// Two kernels advance the scheme:
//  * k_tb2d32: 2D, T steps per launch on a 32 x (TY K) tile with a T-point halo in
//    shared memory (the tile plus a ring of radius T-1-s updated at step s), the
//    Kahan pairs of the tile's points in registers for all T steps;
//  * k_step32 / k_last32: one step per launch, 2D or 3D, second- or fourth-order L_h.
// Both perform the same FP32 operations per point in the same order, so their
// results are bit-identical.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "kernels.h"

namespace mfwh {

// The four host launchers of one frequency count, collected so that the
// translation units wave32_p1.cu .. wave32_p8.cu can each instantiate two counts.
struct W32Ops {
  void (*init)(const Geom&, const double*, float*, float*, float*, const float*, cudaStream_t);
  void (*step)(const Geom&, const float*, const float*, float*, float*, const float*, float*,
               float*, const Step32Host&, cudaStream_t);
  void (*last)(const Geom&, const float*, const float*, const float*, const float*, const float*,
               double*, const double*, const Step32Host&, const StepHost&, cudaStream_t);
  void (*tb)(const Geom&, const float*, const float*, float*, float*, const float*, float*, float*,
             double*, const double*, const TB32Host&, cudaStream_t);
};

namespace {

// Epilogue V^{k+1} = C q + E V^k (E != 0 only for the explicit filter).
template <int NF>
struct Last32Binv {
  double binv[NF * NF];      // C
  double emat[NF * NF];      // E
  const double* vprev;       // V^k
  int has_e;
};

template <int NF>
struct Init32Args {
  float w0[NF];
};

template <int NF>
struct Step32Args {
  Coef32 lo, hi;
  float fc[NF];     // kappa_n cos(omega~_m t^n)
  float wq[NF];     // w_{n+1,m}
  int forced;
};

__device__ __forceinline__ bool interior2(int64_t gx, int64_t gy, const Geom& g) {
  return gx > 0 && gx < g.nx && gy > 0 && gy < g.ny;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float w, float x) {
  const float y = fmaf(w, x, -c);
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// kappa c^2 Delta_h W at a point whose value is w and whose neighbour sums of
// differences are dxx, dyy, dzz, minus the forcing; same order in every kernel.
template <int NF, int DIM>
__device__ __forceinline__ float increment(const Coef32& L, float dxx, float dyy, float dzz,
                                           const float* fc, const float* __restrict__ f,
                                           int64_t p, int64_t points, int forced) {
  float inc = L.Ay * dyy;
  if (DIM == 3) inc = fmaf(L.Az, dzz, inc);
  inc = fmaf(L.Ax, dxx, inc);
  if (forced) {
#pragma unroll
    for (int m = 0; m < NF; ++m) inc = fmaf(-fc[m], f[m * points + p], inc);
  }
  return inc;
}

// ---- one step per launch (2D and 3D) -------------------------------------------

constexpr int kBX = 32, kBY = 8;

template <int DIM>
__device__ __forceinline__ bool index_of(const Geom& g, int64_t& i, int64_t& j, int64_t& k,
                                         int64_t& p, bool& interior) {
  i = (int64_t)blockIdx.x * kBX + threadIdx.x;
  j = (int64_t)blockIdx.y * kBY + threadIdx.y;
  k = DIM == 3 ? (int64_t)blockIdx.z : 0;
  const bool inside = i <= g.nx && j <= g.ny;
  p = k * g.sz + j * g.sy + i;
  interior = inside && i > 0 && i < g.nx && j > 0 && j < g.ny &&
             (DIM == 2 || (k > 0 && k < g.nz));
  return inside;
}

// Fourth-order combination 16 d1 - d2 along one axis at index idx of n cells, from the
// first-neighbour difference sum d1 and the second neighbours (ghost values beyond the
// boundary are minus the centre value, so their difference is -2w).
__device__ __forceinline__ float comb4(const float* W, int64_t p, int64_t s, int64_t idx,
                                       int64_t n, float w, float d1) {
  const float dm = idx == 1 ? -2.0f * w : W[p - 2 * s] - w;
  const float dp = idx == n - 1 ? -2.0f * w : W[p + 2 * s] - w;
  return fmaf(16.0f, d1, -(dm + dp));
}

// Index of grid point (i, j, k) in the wave-level arrays W and D (padded rows in 2D).
__device__ __forceinline__ int64_t wpos(const Geom& g, int64_t i, int64_t j, int64_t k) {
  return k * g.szw + j * g.syw + i;
}

template <int NF, int DIM, int ORDER>
__device__ __forceinline__ void step_point(const float* __restrict__ W, const float* D,
                                           const float* __restrict__ f, const Step32Args<NF>& a,
                                           const Geom& g, int64_t i, int64_t j, int64_t k,
                                           int64_t p, float& wn, float& dn) {
  const int64_t li = g.layer_axis == 0 ? i : (g.layer_axis == 1 ? j : k);
  const Coef32& L = li >= g.layer_split ? a.hi : a.lo;
  const int64_t q = wpos(g, i, j, k);
  const float w = W[q];
  float dxx = (W[q - 1] - w) + (W[q + 1] - w);
  float dyy = (W[q - g.syw] - w) + (W[q + g.syw] - w);
  float dzz = DIM == 3 ? (W[q - g.szw] - w) + (W[q + g.szw] - w) : 0.0f;
  if (ORDER == 4) {
    dxx = comb4(W, q, 1, i, g.nx, w, dxx);
    dyy = comb4(W, q, g.syw, j, g.ny, w, dyy);
    if (DIM == 3) dzz = comb4(W, q, g.szw, k, g.nz, w, dzz);
  }
  const float inc = increment<NF, DIM>(L, dxx, dyy, dzz, a.fc, f, p, g.points, a.forced);
  dn = (D ? D[q] : 0.0f) + inc;
  wn = w + dn;
}

// W_out = W + D', D' = D + increment (D_out may alias D_in; W_out must not alias W_in);
// Kahan sums updated in place.
template <int NF, int DIM, int ORDER>
__global__ void __launch_bounds__(kBX * kBY)
k_step32(const float* __restrict__ W, const float* D_in, float* __restrict__ W_out, float* D_out,
         const float* __restrict__ f, float* __restrict__ qs, float* __restrict__ qc,
         const Step32Args<NF> a, const Geom g) {
  int64_t i, j, k, p;
  bool interior;
  index_of<DIM>(g, i, j, k, p, interior);
  if (!interior) return;
  float wn, dn;
  step_point<NF, DIM, ORDER>(W, D_in, f, a, g, i, j, k, p, wn, dn);
  W_out[wpos(g, i, j, k)] = wn;
  D_out[wpos(g, i, j, k)] = dn;
#pragma unroll
  for (int m = 0; m < NF; ++m) {
    float s = qs[m * g.points + p], c = qc[m * g.points + p];
    kahan_add(s, c, a.wq[m], wn);
    qs[m * g.points + p] = s;
    qc[m * g.points + p] = c;
  }
}

template <int NF>
__device__ __forceinline__ void filter_solve_out(const float* s, const float* c,
                                                 const Last32Binv<NF>& b, int subtract,
                                                 const double* vsub, double* vout,
                                                 int64_t p, int64_t points, bool interior) {
  double qd[NF], vk[NF];
#pragma unroll
  for (int m = 0; m < NF; ++m) {
    qd[m] = (double)s[m] - (double)c[m];
    vk[m] = (b.has_e && interior) ? b.vprev[m * points + p] : 0.0;
  }
#pragma unroll
  for (int m = 0; m < NF; ++m) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < NF; ++j) acc = fma(b.binv[m * NF + j], qd[j], acc);
    if (b.has_e) {
#pragma unroll
      for (int j = 0; j < NF; ++j) acc = fma(b.emat[m * NF + j], vk[j], acc);
    }
    double val = 0.0;
    if (interior) val = subtract ? vsub[m * points + p] - acc : acc;
    vout[m * points + p] = val;
  }
}

template <int NF, int DIM, int ORDER>
__global__ void __launch_bounds__(kBX * kBY)
k_last32(const float* __restrict__ W, const float* __restrict__ D, const float* __restrict__ f,
         const float* __restrict__ qs, const float* __restrict__ qc, double* vout,
         const double* vsub, const Step32Args<NF> a, const Last32Binv<NF> b, int subtract,
         const Geom g) {
  int64_t i, j, k, p;
  bool interior;
  if (!index_of<DIM>(g, i, j, k, p, interior)) return;
  float s[NF], c[NF];
#pragma unroll
  for (int m = 0; m < NF; ++m) s[m] = c[m] = 0.0f;
  if (interior) {
    float wn, dn;
    step_point<NF, DIM, ORDER>(W, D, f, a, g, i, j, k, p, wn, dn);
#pragma unroll
    for (int m = 0; m < NF; ++m) {
      s[m] = qs[m * g.points + p];
      c[m] = qc[m * g.points + p];
      kahan_add(s[m], c[m], a.wq[m], wn);
    }
  }
  filter_solve_out<NF>(s, c, b, subtract, vsub, vout, p, g.points, interior);
}

// ---- temporally blocked 2D kernel ----------------------------------------------

template <int NF>
struct TB32Args {
  Coef32 reg_lo, reg_hi, first_lo, first_hi;
  const float* wq;   // [(N_t + 1) * NF]
  const float* fc;   // [N_t * NF]
  int* err;          // set to 1 when a tile's tensor copy does not complete
  int n0, steps, forced, last, subtract;
};

// A global offset clamped into [lo, hi] as a 32-bit local coordinate.
__device__ __forceinline__ int clamp_local(int64_t v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : (int)v);
}

// One leapfrog update at local point l of the extended tile (increment form).
template <int NF, int EX>
__device__ __forceinline__ float tb_update(const float* Wc, float* Wn, float* Dv, int l,
                                           const Coef32& L, const float* fc,
                                           const float* __restrict__ f, int64_t p,
                                           int64_t points, int forced) {
  const float w = Wc[l];
  const float dxx = (Wc[l - 1] - w) + (Wc[l + 1] - w);
  const float dyy = (Wc[l - EX] - w) + (Wc[l + EX] - w);
  const float inc = increment<NF, 2>(L, dxx, dyy, 0.0f, fc, f, p, points, forced);
  const float dn = Dv[l] + inc;
  const float wn = w + dn;
  Dv[l] = dn;
  Wn[l] = wn;
  return wn;
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

// Fold a partial sum x into the Kahan pair (s, c).
__device__ __forceinline__ void kahan_fold(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// The halo ring of radius r around a BX x BY tile at one step, enumerated evenly over all
// threads: first the 2r rows of BX + 2r points above and below the tile, then the BY rows of
// 2r points to its left and right.  Quotients by the row lengths are exact integer divisions by
// a multiplier: floor(e / d) = (e * ceil(2^32 / d)) >> 32 for the ring indices used here
// (e < 2^16, d < 2^7; checked exhaustively on the host).
// SIMPLE: every ring point is interior and has the same c^2 (no bounds or layer tests).
template <int NF, int T, int BX, int BY, bool SIMPLE>
__device__ __forceinline__ void ring_pass(const float* Wc, float* Wn, float* Dv, int r, int tid,
                                          int nthreads, int ilx, int ihx, int ily, int ihy,
                                          bool lay_x, int lay_thr, const Coef32& lo,
                                          const Coef32& hi, const float* fc,
                                          const float* __restrict__ f, int64_t y0, int64_t x0,
                                          const Geom& g, int forced) {
  constexpr int EX = BX + 2 * T;
  const int RW = BX + 2 * r;
  const int top = 2 * r * RW;
  const int ring = top + 2 * r * BY;
  const unsigned m_rw = div_magic(RW), m_2r = div_magic(2 * r);
  for (int e = tid; e < ring; e += nthreads) {
    int lx, ly;
    if (e < top) {
      const int row = (int)__umulhi((unsigned)e, m_rw);
      lx = T - r + (e - row * RW);
      ly = row < r ? T - r + row : T + BY + row - r;
    } else {
      const int e2 = e - top;
      const int row = (int)__umulhi((unsigned)e2, m_2r);
      const int col = e2 - row * 2 * r;
      ly = T + row;
      lx = col < r ? T - r + col : T + BX + col - r;
    }
    if (!SIMPLE && (lx < ilx || lx > ihx || ly < ily || ly > ihy)) continue;
    const Coef32& L = SIMPLE ? lo : (((lay_x ? lx : ly) >= lay_thr) ? hi : lo);
    tb_update<NF, EX>(Wc, Wn, Dv, ly * EX + lx, L, fc, f, (y0 + ly) * g.sy + x0 + lx, g.points,
                      forced);
  }
}

// ACC = 0: Kahan update of (s_m, c_m) at every step.
// ACC = 1: plain FP32 partial sums over the steps of one launch, folded into the Kahan
//          pair once per launch (compensated across launches; the partial of at most T
//          terms carries a rounding error far below that of the FP32 wave levels).
//
// The CTA has BX x TY threads (BX = 32 or 64) and a BX x (TY K) tile.  Thread (tx, ty) owns
// the K consecutive tile rows ty K .. ty K + K - 1 of column tx.  The wave values W and
// increments D of its own points stay in registers for all T steps; only the left and right
// neighbours and the rows just above and below the strip come from shared memory.  The halo
// ring is updated from shared memory by all threads.
// Tensor-memory-accelerator (TMA) copies of the extended tile: one 2D tiled copy of EX x EY
// floats per array, completing on an mbarrier with a transaction count.  Points outside the
// grid (negative or past the extents) arrive as zeros.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tma_tile_2d(float* dst, const CUtensorMap* map, int x, int y,
                                            unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false when the bound ran out.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    unsigned done;
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

template <int NF, int T, int BX, int TY, int K, int MB, int ACC>
__global__ void __launch_bounds__(BX * TY, MB)
k_tb2d32(const float* __restrict__ W_in, const float* __restrict__ D_in,
         float* __restrict__ W_out, float* __restrict__ D_out, const float* __restrict__ f,
         float* __restrict__ qs, float* __restrict__ qc, double* vout, const double* vsub,
         const TB32Args<NF> a, const Last32Binv<NF> b, const Geom g,
         const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmD,
         int use_tma) {
  constexpr int BY = TY * K, NT = BX * TY;
  constexpr int EX = BX + 2 * T, EY = BY + 2 * T, E = EX * EY;
  static_assert((E * sizeof(float)) % 128 == 0, "tile arrays must stay 128-byte aligned");
  extern __shared__ __align__(128) float sm32[];
  __shared__ __align__(8) uint64_t tile_bar;
  float* Wc = sm32;             // W^n on the extended tile
  float* Wn = sm32 + E;         // W^{n+1}
  float* Dv = sm32 + 2 * E;     // D on the halo (the tile's own D lives in registers)
  float* s_wq = sm32 + 3 * E;   // [T][NF]
  float* s_fc = s_wq + T * NF;  // [T][NF]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int64_t x0 = (int64_t)blockIdx.x * BX - T, y0 = (int64_t)blockIdx.y * BY - T;
  // Local-coordinate bounds (32-bit): grid points gl*, interior points il*.
  const int glx = clamp_local(-x0, 0, EX), ghx = clamp_local(g.nx - x0, -1, EX - 1);
  const int gly = clamp_local(-y0, 0, EY), ghy = clamp_local(g.ny - y0, -1, EY - 1);
  const int ilx = clamp_local(1 - x0, 0, EX), ihx = clamp_local(g.nx - 1 - x0, -1, EX - 1);
  const int ily = clamp_local(1 - y0, 0, EY), ihy = clamp_local(g.ny - 1 - y0, -1, EY - 1);
  // c^2 layer: points whose local coordinate along the layer axis is >= lay_thr use hi.
  const bool lay_x = g.layer_axis == 0;
  const int lay_thr = clamp_local(g.layer_split - (lay_x ? x0 : y0), -1, EX + EY);
  // Every point of the largest ring interior, all with one c^2: the ring needs no tests.
  const bool simple = ilx <= 1 && ihx >= EX - 2 && ily <= 1 && ihy >= EY - 2 &&
                      (lay_thr <= 0 || lay_thr >= (lay_x ? EX : EY));
  const bool all_hi = lay_thr <= 0;

  if (use_tma) {
    // W twice (current level and the buffer of the next one, whose boundary values must be
    // in place) and D once, by tensor copies issued from one thread.
    const unsigned bar = smem_addr(&tile_bar);
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
      const unsigned bytes = (D_in != nullptr ? 3u : 2u) * (unsigned)(E * sizeof(float));
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                   : "memory");
      tma_tile_2d(Wc, &tmW, (int)x0, (int)y0, bar);
      tma_tile_2d(Wn, &tmW, (int)x0, (int)y0, bar);
      if (D_in != nullptr) tma_tile_2d(Dv, &tmD, (int)x0, (int)y0, bar);
    }
    if (D_in == nullptr)
      for (int e = tid; e < E; e += NT) Dv[e] = 0.0f;
    const bool ok = mbar_wait(bar, 0, 1 << 22);
    if (__syncthreads_or(!ok)) {
      // The copies did not complete within the bound: report it (the host fails the call with
      // MFWH_ERR_TIMEOUT), give them one more bounded wait to land while the CTA still owns its
      // shared memory, and stop.  If that wait runs out too the CTA stops all the same: every
      // wait in this kernel must end.
      if (tid == 0) atomicExch(a.err, 1);
      mbar_wait(bar, 0, 1 << 22);
      return;
    }
  } else {
    for (int ly = ty; ly < EY; ly += TY) {
      const bool row = ly >= gly && ly <= ghy;
      const int64_t rbase = (y0 + ly) * g.syw + x0;
      for (int lx = tx; lx < EX; lx += BX) {
        const bool in = row && lx >= glx && lx <= ghx;
        const int l = ly * EX + lx;
        const float w = in ? W_in[rbase + lx] : 0.0f;
        Wc[l] = w;
        Wn[l] = w;
        Dv[l] = (in && D_in != nullptr) ? D_in[rbase + lx] : 0.0f;
      }
    }
  }
  for (int e = tid; e < a.steps * NF; e += NT) {
    const int st = e / NF, m = e - st * NF;
    const int n = a.n0 + st;
    s_wq[e] = a.wq[(n + 1) * NF + m];
    s_fc[e] = a.forced ? a.fc[n * NF + m] : 0.0f;
  }
  // The strip: local column lxo, rows lyo .. lyo + K - 1.
  const int lxo = T + tx, lyo = T + ty * K;
  const int64_t p0 = (y0 + lyo) * g.sy + x0 + lxo;
  if (ACC == 1) {
    // Ask L2 for the Kahan pairs folded at the end of the launch.  A warp's 32 columns of
    // one row span at most two 128-byte lines; each lane prefetches some of the warp's
    // (row, frequency, array) lines.
    const int lane = tid & 31;
    const int64_t wbase = p0 - (tx & 31);
    for (int c = lane; c < 4 * K * NF; c += 32) {
      const int half = c & 1, k = (c >> 1) % K, m = ((c >> 1) / K) % NF, arr = c / (2 * K * NF);
      const int64_t pl = wbase + k * g.sy + half * 31;
      if (lxo - (tx & 31) + half * 31 <= ihx && lyo + k <= ihy) {
        const float* ptr = (arr ? qc : qs) + m * g.points + pl;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
      }
    }
  }
  const bool col_int = lxo >= ilx && lxo <= ihx;
  bool own_int[K], own_up[K];
  float wr[K], dr[K], ks[K][NF], kc[K][NF], part[K][NF];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int ly = lyo + k;
    own_int[k] = col_int && ly >= ily && ly <= ihy;
    own_up[k] = (lay_x ? lxo : ly) >= lay_thr;
    wr[k] = Wc[ly * EX + lxo];
    dr[k] = Dv[ly * EX + lxo];
#pragma unroll
    for (int m = 0; m < NF; ++m) {
      part[k][m] = 0.0f;
      if (ACC == 0) {
        ks[k][m] = own_int[k] ? qs[m * g.points + p0 + k * g.sy] : 0.0f;
        kc[k][m] = own_int[k] ? qc[m * g.points + p0 + k * g.sy] : 0.0f;
      }
    }
  }

  // The T steps in two compiled copies with the same arithmetic per point: ALLINT, for
  // homogeneous launches of CTAs whose updated points are all interior with one c^2, without
  // the forcing terms and the per-point interior and layer tests; and the general one.
  auto run_steps = [&](auto allint_c) {
    constexpr bool ALLINT = decltype(allint_c)::value;
    const int forcing = ALLINT ? 0 : a.forced;
    for (int s = 0; s < a.steps; ++s) {
      const int r = a.steps - 1 - s;
      const bool first = a.n0 + s == 0;
      const Coef32 lo = first ? a.first_lo : a.reg_lo;
      const Coef32 hi = first ? a.first_hi : a.reg_hi;
      const float* fc = s_fc + s * NF;
      float wq[NF];
#pragma unroll
      for (int m = 0; m < NF; ++m) wq[m] = s_wq[s * NF + m];
      // the strip: centre values from registers, neighbours from shared memory
      {
        const float above = Wc[(lyo - 1) * EX + lxo];
        const float below = Wc[(lyo + K) * EX + lxo];
        float wnew[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float w = wr[k];
          wnew[k] = w;
          if (!ALLINT && !own_int[k]) continue;   // boundary and outside points keep W = 0
          const int l = (lyo + k) * EX + lxo;
          const float up = k == 0 ? above : wr[k - 1];
          const float dn = k == K - 1 ? below : wr[k + 1];
          const float dxx = (Wc[l - 1] - w) + (Wc[l + 1] - w);
          const float dyy = (up - w) + (dn - w);
          const Coef32 L = ALLINT ? (all_hi ? hi : lo) : (own_up[k] ? hi : lo);
          const float inc = increment<NF, 2>(L, dxx, dyy, 0.0f, fc, f, p0 + k * g.sy, g.points,
                                             forcing);
          dr[k] = dr[k] + inc;
          wnew[k] = w + dr[k];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          wr[k] = wnew[k];
          Wn[(lyo + k) * EX + lxo] = wnew[k];
          if (ALLINT || own_int[k]) {
#pragma unroll
            for (int m = 0; m < NF; ++m) {
              if (ACC == 0)
                kahan_add(ks[k][m], kc[k][m], wq[m], wnew[k]);
              else
                part[k][m] = fmaf(wq[m], wnew[k], part[k][m]);
            }
          }
        }
      }
      if (r > 0) {
        if (ALLINT || simple)
          ring_pass<NF, T, BX, BY, true>(Wc, Wn, Dv, r, tid, NT, ilx, ihx, ily, ihy, lay_x,
                                         lay_thr, all_hi ? hi : lo, hi, fc, f, y0, x0, g,
                                         forcing);
        else
          ring_pass<NF, T, BX, BY, false>(Wc, Wn, Dv, r, tid, NT, ilx, ihx, ily, ihy, lay_x,
                                          lay_thr, lo, hi, fc, f, y0, x0, g, forcing);
      }
      __syncthreads();
      float* t = Wc;
      Wc = Wn;
      Wn = t;
    }
  };
  if (simple && !a.forced)
    run_steps(std::true_type{});
  else
    run_steps(std::false_type{});
  // wr = W^{n0+steps}, dr = D^{n0+steps-1/2} on the strip
  const bool col_in = lxo <= ghx;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t p = p0 + k * g.sy;
    if (ACC == 1 && own_int[k]) {
#pragma unroll
      for (int m = 0; m < NF; ++m) {
        ks[k][m] = qs[m * g.points + p];
        kc[k][m] = qc[m * g.points + p];
        kahan_fold(ks[k][m], kc[k][m], part[k][m]);
      }
    }
    if (!a.last) {
      if (!own_int[k]) continue;
      W_out[(y0 + lyo + k) * g.syw + x0 + lxo] = wr[k];
      D_out[(y0 + lyo + k) * g.syw + x0 + lxo] = dr[k];
#pragma unroll
      for (int m = 0; m < NF; ++m) {
        qs[m * g.points + p] = ks[k][m];
        qc[m * g.points + p] = kc[k][m];
      }
    } else {
      if (!col_in || lyo + k > ghy) continue;
      if (!own_int[k]) {
#pragma unroll
        for (int m = 0; m < NF; ++m) ks[k][m] = kc[k][m] = 0.0f;
      }
      filter_solve_out<NF>(ks[k], kc[k], b, a.subtract, vsub, vout, p, g.points, own_int[k]);
    }
  }
}

// ---- init and conversion ---------------------------------------------------------

template <int NF, int DIM>
__global__ void __launch_bounds__(kBX * kBY)
k_init32(const double* __restrict__ v, float* __restrict__ W0, float* __restrict__ qs,
         float* __restrict__ qc, const Init32Args<NF> a, const Geom g) {
  int64_t i, j, k, p;
  bool interior;
  if (!index_of<DIM>(g, i, j, k, p, interior)) return;
  double w = 0.0;
  if (interior && v != nullptr) {
#pragma unroll
    for (int m = 0; m < NF; ++m) w += v[m * g.points + p];
  }
  const float wf = (float)w;
  W0[wpos(g, i, j, k)] = wf;
#pragma unroll
  for (int m = 0; m < NF; ++m) {
    qs[m * g.points + p] = a.w0[m] * wf;
    qc[m * g.points + p] = 0.0f;
  }
}

// ---- temporally blocked 3D kernel ------------------------------------------------
// Overlapped tiling in all three axes: a CTA owns a (32 - 2T) x 8 x 8 tile and keeps the tile
// plus a halo of T points per side of W^n, W^{n+1} and D in shared memory, 32 points wide in
// x so that a warp covers a row.  At step s of a launch of S steps it updates every interior
// point of the tile grown by S - 1 - s points per side (reading the values of the previous
// step one point further out), so the owned points are exact after S steps.  The rows (y, z)
// of the region are spread over the warps and a row's points over the lanes.  Thread (x, y)
// with x < 32 - 2T owns the 8 points of tile column (x, y) and keeps their filter sums in
// registers (ACC as in k_tb2d32).  Each point update performs the operations of
// step_point<NF, 3, 2> in the same order, so with ACC = 0 every depth is bit-identical to
// one step per launch.
constexpr int kT3W = 32, kT3Y = 8, kT3Z = 8, kT3Threads = kT3W * kT3Y;

template <int NF, int T, int ACC>
__global__ void __launch_bounds__(kT3Threads, ACC == 1 ? 2 : 1)
k_tb3d32(const float* __restrict__ W_in, const float* __restrict__ D_in,
         float* __restrict__ W_out, float* __restrict__ D_out, const float* __restrict__ f,
         float* __restrict__ qs, float* __restrict__ qc, double* vout, const double* vsub,
         const TB32Args<NF> a, const Last32Binv<NF> b, const Geom g) {
  constexpr int BX = kT3W - 2 * T;
  constexpr int EX = kT3W, EY = kT3Y + 2 * T, EZ = kT3Z + 2 * T;
  constexpr int SXY = EX * EY, E = SXY * EZ;
  extern __shared__ __align__(16) float sm3[];
  float* Wc = sm3;
  float* Wn = sm3 + E;
  float* Dv = sm3 + 2 * E;
  float* s_wq = sm3 + 3 * E;    // [T][NF]
  float* s_fc = s_wq + T * NF;  // [T][NF]
  const int tid = threadIdx.x;
  const int tx = tid % kT3W, ty = tid / kT3W;   // lanes along x, warps along rows
  const int64_t x0 = (int64_t)blockIdx.x * BX - T, y0 = (int64_t)blockIdx.y * kT3Y - T,
                z0 = (int64_t)blockIdx.z * kT3Z - T;
  {
    const int64_t gx = x0 + tx;
    for (int row = ty; row < EY * EZ; row += kT3Y) {
      const int lz = row / EY, ly = row - lz * EY;
      const int64_t gy = y0 + ly, gz = z0 + lz;
      const bool in = gz >= 0 && gz <= g.nz && gy >= 0 && gy <= g.ny && gx >= 0 && gx <= g.nx;
      const int64_t q = gz * g.szw + gy * g.syw + gx;
      const int e = lz * SXY + ly * EX + tx;
      const float w = in ? W_in[q] : 0.0f;
      Wc[e] = w;
      Wn[e] = w;
      Dv[e] = (in && D_in != nullptr) ? D_in[q] : 0.0f;
    }
  }
  for (int e = tid; e < a.steps * NF; e += kT3Threads) {
    const int st = e / NF, m = e - st * NF;
    const int n = a.n0 + st;
    s_wq[e] = a.wq[(n + 1) * NF + m];
    s_fc[e] = a.forced ? a.fc[n * NF + m] : 0.0f;
  }
  // the owned column (threads with tx < BX)
  const bool owner = tx < BX;
  const int64_t gx = x0 + T + tx, gy = y0 + T + ty;
  const bool col_int = owner && gx > 0 && gx < g.nx && gy > 0 && gy < g.ny;
  bool own_int[kT3Z];
  float ks[kT3Z][NF], kc[kT3Z][NF], part[kT3Z][NF];
#pragma unroll
  for (int k = 0; k < kT3Z; ++k) {
    const int64_t gz = z0 + T + k;
    own_int[k] = col_int && gz > 0 && gz < g.nz;
    const int64_t p = gz * g.sz + gy * g.sy + gx;
#pragma unroll
    for (int m = 0; m < NF; ++m) {
      part[k][m] = 0.0f;
      ks[k][m] = (ACC == 0 && own_int[k]) ? qs[m * g.points + p] : 0.0f;
      kc[k][m] = (ACC == 0 && own_int[k]) ? qc[m * g.points + p] : 0.0f;
    }
  }
  __syncthreads();
  for (int s = 0; s < a.steps; ++s) {
    const int r = a.steps - 1 - s;
    const bool first = a.n0 + s == 0;
    const Coef32 lo = first ? a.first_lo : a.reg_lo;
    const Coef32 hi = first ? a.first_hi : a.reg_hi;
    const float* fc = s_fc + s * NF;
    // the region [T - r, T + tile + r) per axis
    const int l0 = T - r, RY = kT3Y + 2 * r, RZ = kT3Z + 2 * r;
    const int lx = l0 + tx;
    const int64_t px = x0 + lx;
    const bool x_ok = lx < T + BX + r && px > 0 && px < g.nx;
    for (int row = ty; row < RY * RZ; row += kT3Y) {
      const int rz = row / RY, ry = row - rz * RY;
      const int ly = l0 + ry, lz = l0 + rz;
      const int64_t py = y0 + ly, pz = z0 + lz;
      if (!x_ok || py <= 0 || py >= g.ny || pz <= 0 || pz >= g.nz) continue;
      const int l = lz * SXY + ly * EX + lx;
      const int64_t li = g.layer_axis == 0 ? px : (g.layer_axis == 1 ? py : pz);
      const Coef32& L = li >= g.layer_split ? hi : lo;
      const float w = Wc[l];
      const float dxx = (Wc[l - 1] - w) + (Wc[l + 1] - w);
      const float dyy = (Wc[l - EX] - w) + (Wc[l + EX] - w);
      const float dzz = (Wc[l - SXY] - w) + (Wc[l + SXY] - w);
      const int64_t p = pz * g.sz + py * g.sy + px;
      const float inc = increment<NF, 3>(L, dxx, dyy, dzz, fc, f, p, g.points, a.forced);
      const float dn = Dv[l] + inc;
      Dv[l] = dn;
      Wn[l] = w + dn;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kT3Z; ++k) {
      if (!own_int[k]) continue;
      const float wn = Wn[(T + k) * SXY + (T + ty) * EX + T + tx];
#pragma unroll
      for (int m = 0; m < NF; ++m) {
        if (ACC == 0)
          kahan_add(ks[k][m], kc[k][m], s_wq[s * NF + m], wn);
        else
          part[k][m] = fmaf(s_wq[s * NF + m], wn, part[k][m]);
      }
    }
    float* t = Wc;
    Wc = Wn;
    Wn = t;
  }
  // Wc holds W^{n0+steps} and Dv the matching D on the owned points
  if (!owner) return;
#pragma unroll
  for (int k = 0; k < kT3Z; ++k) {
    const int64_t gz = z0 + T + k;
    if (gx > g.nx || gy > g.ny || gz > g.nz) continue;
    const int64_t p = gz * g.sz + gy * g.sy + gx;
    const int l = (T + k) * SXY + (T + ty) * EX + T + tx;
    if (ACC == 1 && own_int[k]) {
#pragma unroll
      for (int m = 0; m < NF; ++m) {
        ks[k][m] = qs[m * g.points + p];
        kc[k][m] = qc[m * g.points + p];
        kahan_fold(ks[k][m], kc[k][m], part[k][m]);
      }
    }
    if (!a.last) {
      if (!own_int[k]) continue;
      const int64_t q = gz * g.szw + gy * g.syw + gx;
      W_out[q] = Wc[l];
      D_out[q] = Dv[l];
#pragma unroll
      for (int m = 0; m < NF; ++m) {
        qs[m * g.points + p] = ks[k][m];
        qc[m * g.points + p] = kc[k][m];
      }
    } else {
      if (!own_int[k]) {
#pragma unroll
        for (int m = 0; m < NF; ++m) ks[k][m] = kc[k][m] = 0.0f;
      }
      filter_solve_out<NF>(ks[k], kc[k], b, a.subtract, vsub, vout, p, g.points, own_int[k]);
    }
  }
}

// ---- host launchers --------------------------------------------------------------

template <int NF>
Step32Args<NF> step_args(const Step32Host& h) {
  Step32Args<NF> a;
  a.lo = h.lo;
  a.hi = h.hi;
  for (int m = 0; m < NF; ++m) {
    a.fc[m] = h.fc[m];
    a.wq[m] = h.wq[m];
  }
  a.forced = h.forced;
  return a;
}

template <int NF>
Last32Binv<NF> binv_args(const double* binv, const double* emat, int has_e,
                         const double* vprev) {
  Last32Binv<NF> b;
  for (int m = 0; m < NF; ++m)
    for (int j = 0; j < NF; ++j) {
      b.binv[m * NF + j] = binv[m * MFWH_MAX_NF + j];
      b.emat[m * NF + j] = emat[m * MFWH_MAX_NF + j];
    }
  b.has_e = has_e && vprev != nullptr;
  b.vprev = vprev;
  return b;
}

dim3 grid_of(const Geom& g) {
  return dim3((unsigned)((g.nx + kBX) / kBX), (unsigned)((g.ny + kBY) / kBY),
              (unsigned)(g.dim == 3 ? g.nz + 1 : 1));
}

template <int NF>
void step32_nf(const Geom& g, const float* W, const float* D_in, float* W_out, float* D_out,
               const float* f, float* qs, float* qc, const Step32Host& h, cudaStream_t st) {
  const Step32Args<NF> a = step_args<NF>(h);
  const dim3 grid = grid_of(g), blk(kBX, kBY);
  if (g.order == 4) {
    if (g.dim == 3)
      k_step32<NF, 3, 4><<<grid, blk, 0, st>>>(W, D_in, W_out, D_out, f, qs, qc, a, g);
    else
      k_step32<NF, 2, 4><<<grid, blk, 0, st>>>(W, D_in, W_out, D_out, f, qs, qc, a, g);
  } else if (g.dim == 3) {
    k_step32<NF, 3, 2><<<grid, blk, 0, st>>>(W, D_in, W_out, D_out, f, qs, qc, a, g);
  } else {
    k_step32<NF, 2, 2><<<grid, blk, 0, st>>>(W, D_in, W_out, D_out, f, qs, qc, a, g);
  }
}

template <int NF>
void last32_nf(const Geom& g, const float* W, const float* D, const float* f, const float* qs,
               const float* qc, double* vout, const double* vsub, const Step32Host& h,
               const StepHost& epi, cudaStream_t st) {
  const Step32Args<NF> a = step_args<NF>(h);
  const Last32Binv<NF> b = binv_args<NF>(epi.binv, epi.emat, epi.has_e, epi.vprev);
  const int sub = vsub != nullptr;
  const dim3 grid = grid_of(g), blk(kBX, kBY);
  if (g.order == 4) {
    if (g.dim == 3)
      k_last32<NF, 3, 4><<<grid, blk, 0, st>>>(W, D, f, qs, qc, vout, vsub, a, b, sub, g);
    else
      k_last32<NF, 2, 4><<<grid, blk, 0, st>>>(W, D, f, qs, qc, vout, vsub, a, b, sub, g);
  } else if (g.dim == 3) {
    k_last32<NF, 3, 2><<<grid, blk, 0, st>>>(W, D, f, qs, qc, vout, vsub, a, b, sub, g);
  } else {
    k_last32<NF, 2, 2><<<grid, blk, 0, st>>>(W, D, f, qs, qc, vout, vsub, a, b, sub, g);
  }
}

template <int NF>
void init32_nf(const Geom& g, const double* v, float* W0, float* qs, float* qc, const float* w0,
               cudaStream_t st) {
  Init32Args<NF> a;
  for (int m = 0; m < NF; ++m) a.w0[m] = w0[m];
  if (g.dim == 3)
    k_init32<NF, 3><<<grid_of(g), dim3(kBX, kBY), 0, st>>>(v, W0, qs, qc, a, g);
  else
    k_init32<NF, 2><<<grid_of(g), dim3(kBX, kBY), 0, st>>>(v, W0, qs, qc, a, g);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no driver library link).
inline EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map of one 2D wave-level array for EX x EY boxes; false if unavailable, in which
// case the kernel loads its tile with ordinary loads.
inline bool wave_tensor_map(CUtensorMap* m, const float* base, const Geom& g, int ex, int ey) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || !base || g.dim != 2 || (g.syw * sizeof(float)) % 16 != 0 ||
      (reinterpret_cast<uintptr_t>(base) & 15) != 0)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(g.nx + 1), (cuuint64_t)(g.ny + 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)(g.syw * sizeof(float))};
  const cuuint32_t box[2] = {(cuuint32_t)ex, (cuuint32_t)ey};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NF, int T, int BX, int TY, int K, int MB, int ACC>
void tb32_launch(const Geom& g, const float* W_in, const float* D_in, float* W_out, float* D_out,
                 const float* f, float* qs, float* qc, double* vout, const double* vsub,
                 const TB32Host& h, cudaStream_t st) {
  constexpr int BY = TY * K;
  constexpr int EX = BX + 2 * T, EY = BY + 2 * T;
  constexpr size_t smem = sizeof(float) * (3 * EX * EY + 2 * T * NF);
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_tb2d32<NF, T, BX, TY, K, MB, ACC>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  TB32Args<NF> a;
  a.reg_lo = h.reg_lo;
  a.reg_hi = h.reg_hi;
  a.first_lo = h.first_lo;
  a.first_hi = h.first_hi;
  a.wq = h.wq;
  a.fc = h.fc;
  a.n0 = h.n0;
  a.steps = h.steps;
  a.forced = h.forced;
  a.last = h.last;
  a.subtract = vsub != nullptr;
  a.err = h.err;
  const Last32Binv<NF> b = binv_args<NF>(h.binv, h.emat, h.has_e, h.vprev);
  dim3 grid((unsigned)((g.nx + BX) / BX), (unsigned)((g.ny + BY) / BY));
  CUtensorMap tmW{}, tmD{};
  int use_tma = h.err != nullptr && wave_tensor_map(&tmW, W_in, g, EX, EY) &&
                (D_in == nullptr || wave_tensor_map(&tmD, D_in, g, EX, EY));
  if (D_in == nullptr) tmD = tmW;
  k_tb2d32<NF, T, BX, TY, K, MB, ACC><<<grid, dim3(BX, TY), smem, st>>>(
      W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, a, b, g, tmW, tmD, use_tma);
}

template <int NF, int T, int ACC>
void tb32_shape(const Geom& g, const float* W_in, const float* D_in, float* W_out, float* D_out,
                const float* f, float* qs, float* qc, double* vout, const double* vsub,
                const TB32Host& h, cudaStream_t st) {
  // Tile shapes, K consecutive rows per thread (K halves above 8 frequencies to bound
  // registers):
  //  0: 512 threads, tile 32 x 32 (K = 2; 32 x 16), two CTAs per SM (one with ACC = 0);
  //  1: 512 threads, tile 32 x 64 (K = 4; 32 x 32), one CTA per SM;
  //  2: 1024 threads, tile 64 x 64 (K = 4; 64 x 32), one CTA per SM.
  constexpr int KS = NF <= 8 ? 2 : 1;
  constexpr int M2 = ACC == 0 ? 1 : 2;
  switch (h.shape) {
    case 1:
      tb32_launch<NF, T, 32, 16, 2 * KS, 1, ACC>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout,
                                                 vsub, h, st);
      break;
    case 2:
      tb32_launch<NF, T, 64, 16, 2 * KS, 1, ACC>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout,
                                                 vsub, h, st);
      break;
    default:
      tb32_launch<NF, T, 32, 16, KS, M2, ACC>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub,
                                              h, st);
      break;
  }
}

template <int NF, int T>
void tb32_acc(const Geom& g, const float* W_in, const float* D_in, float* W_out, float* D_out,
              const float* f, float* qs, float* qc, double* vout, const double* vsub,
              const TB32Host& h, cudaStream_t st) {
  if (h.acc == 1)
    tb32_shape<NF, T, 1>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
  else
    tb32_shape<NF, T, 0>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
}

template <int NF>
void tb32_nf(const Geom& g, const float* W_in, const float* D_in, float* W_out, float* D_out,
             const float* f, float* qs, float* qc, double* vout, const double* vsub,
             const TB32Host& h, cudaStream_t st) {
  // Depth 4 runs on the depth-8 instantiation: a launch of at most 4 steps only needs the
  // inner 4 points of its 8-point halo, and the arithmetic per point is the same.
  if (h.depth <= 8)
    tb32_acc<NF, 8>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
  else
    tb32_acc<NF, 16>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
}

template <int NF, int T, int ACC>
void tb3d32_launch(const Geom& g, const float* W_in, const float* D_in, float* W_out,
                   float* D_out, const float* f, float* qs, float* qc, double* vout,
                   const double* vsub, const TB32Host& h, cudaStream_t st) {
  constexpr int E = kT3W * (kT3Y + 2 * T) * (kT3Z + 2 * T);
  constexpr int BX = kT3W - 2 * T;
  constexpr size_t smem = sizeof(float) * (3 * E + 2 * T * NF);
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_tb3d32<NF, T, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  TB32Args<NF> a;
  a.reg_lo = h.reg_lo;
  a.reg_hi = h.reg_hi;
  a.first_lo = h.first_lo;
  a.first_hi = h.first_hi;
  a.wq = h.wq;
  a.fc = h.fc;
  a.n0 = h.n0;
  a.steps = h.steps;
  a.forced = h.forced;
  a.last = h.last;
  a.subtract = vsub != nullptr;
  a.err = h.err;
  const Last32Binv<NF> b = binv_args<NF>(h.binv, h.emat, h.has_e, h.vprev);
  const dim3 grid((unsigned)((g.nx + BX) / BX), (unsigned)((g.ny + kT3Y) / kT3Y),
                  (unsigned)((g.nz + kT3Z) / kT3Z));
  k_tb3d32<NF, T, ACC><<<grid, kT3Threads, smem, st>>>(W_in, D_in, W_out, D_out, f, qs, qc,
                                                          vout, vsub, a, b, g);
}

// Depth 2 or 4 (a launch of at most T steps; the halo is T points).
template <int NF>
void tb3d32_nf(const Geom& g, const float* W_in, const float* D_in, float* W_out, float* D_out,
               const float* f, float* qs, float* qc, double* vout, const double* vsub,
               const TB32Host& h, cudaStream_t st) {
  if (h.depth <= 2) {
    if (h.acc == 1)
      tb3d32_launch<NF, 2, 1>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
    else
      tb3d32_launch<NF, 2, 0>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
  } else {
    if (h.acc == 1)
      tb3d32_launch<NF, 4, 1>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
    else
      tb3d32_launch<NF, 4, 0>(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
  }
}

template <int NF>
W32Ops make_w32_ops() {
  return W32Ops{init32_nf<NF>, step32_nf<NF>, last32_nf<NF>, tb32_nf<NF>};
}

using Tb3dFn = void (*)(const Geom&, const float*, const float*, float*, float*, const float*,
                        float*, float*, double*, const double*, const TB32Host&, cudaStream_t);

}  // namespace

// Defined in wave32_p1.cu .. wave32_p8.cu for nf in 1-2, 3-4, ..., 15-16.
W32Ops w32_ops_p1(int nf);
W32Ops w32_ops_p2(int nf);
W32Ops w32_ops_p3(int nf);
W32Ops w32_ops_p4(int nf);
W32Ops w32_ops_p5(int nf);
W32Ops w32_ops_p6(int nf);
W32Ops w32_ops_p7(int nf);
W32Ops w32_ops_p8(int nf);
// The 3D blocked launcher for nf, from the translation unit that instantiates nf.
Tb3dFn w32_tb3_p1(int nf);
Tb3dFn w32_tb3_p2(int nf);
Tb3dFn w32_tb3_p3(int nf);
Tb3dFn w32_tb3_p4(int nf);
Tb3dFn w32_tb3_p5(int nf);
Tb3dFn w32_tb3_p6(int nf);
Tb3dFn w32_tb3_p7(int nf);
Tb3dFn w32_tb3_p8(int nf);

}  // namespace mfwh

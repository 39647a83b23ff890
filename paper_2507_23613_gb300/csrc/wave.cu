// MFWH wave-solve kernels for sm_103a, FP64.
//
// One application of the MFWH map (Algorithm 1, loop body) is
//   k_init  : W^0 = sum_m V_m, q_m = w_{0,m} W^0
//   k_step  : W^{n+1} = 2 W^n - W^{n-1} + dt^2 (c^2 Delta_h W^n - F^n)        (eq. WaveSchemeA)
//             (first step: W^1 = W^0 + dt^2/2 (c^2 Delta_h W^0 - F^0),       eq. implicitFirstStep)
//             fused with the N_f filter sums q_m += w_{n+1,m} W^{n+1}         (eq. pDefQ)
//   k_last  : the final step fused with the filter solve V = B^{-1} q          (eq. waveHoltzMatrixIteration)
// F^n = sum_m f_m cos(omega~_m t^n) (eq. WaveSchemeForcing).  The wave levels are
// stored as two ping-pong grids; W^{n+1} overwrites W^{n-1} at the same point, so
// each point is read and written by one thread only.  The forcing grids f_m and
// the accumulators q_m are [N_f][points] arrays; the N_f accumulations of a point
// run in registers on the value just computed, so W^{n+1} is never re-read.  The
// accumulators are float pairs updated on the FP32 pipe (fpair.cuh); k_last adds the
// final term in FP64 and solves for V in FP64.
#include <cuda_runtime.h>

#include "fpair.cuh"
#include "kernels.h"

namespace mfwh {
namespace {

constexpr int kBX = 32, kBY = 8;

template <int NF>
struct StepParams {
  LayerCoef lo, hi;
  double acur;
  double fneg[NF];   // kappa cos(omega~_m t^n)
  double wq[NF];
  float wq_hi[NF], wq_lo[NF];   // w_{n+1,m} as a float pair
  int first, forced;
};

template <int NF>
struct LastParams {
  StepParams<NF> st;
  double binv[NF * NF];      // C of V^{k+1} = C q + E V^k
  double emat[NF * NF];      // E (explicit filter)
  const double* vprev;       // V^k
  int subtract, has_e;
};

template <int NF>
struct InitParams {
  double w0[NF];
};

template <int NF>
StepParams<NF> to_params(const StepHost& a) {
  StepParams<NF> p;
  p.lo = a.lo;
  p.hi = a.hi;
  p.acur = a.a_cur;
  for (int m = 0; m < NF; ++m) {
    p.fneg[m] = a.fc[m];
    p.wq[m] = a.wq[m];
    p.wq_hi[m] = (float)a.wq[m];
    p.wq_lo[m] = (float)(a.wq[m] - (double)p.wq_hi[m]);
  }
  p.first = a.first;
  p.forced = a.forced;
  return p;
}

struct PointIndex {
  int64_t i, j, k, p;
  bool inside, interior;
};

template <int DIM>
__device__ __forceinline__ PointIndex point_index(const Geom& g) {
  PointIndex r;
  r.i = (int64_t)blockIdx.x * kBX + threadIdx.x;
  r.j = (int64_t)blockIdx.y * kBY + threadIdx.y;
  r.k = (DIM == 3) ? (int64_t)blockIdx.z : 0;
  r.inside = r.i <= g.nx && r.j <= g.ny;
  r.p = r.k * g.sz + r.j * g.sy + r.i;
  r.interior = r.inside && r.i > 0 && r.i < g.nx && r.j > 0 && r.j < g.ny &&
               (DIM == 2 || (r.k > 0 && r.k < g.nz));
  return r;
}

// New wave level at an interior point (the leapfrog update with the composite forcing).
// ORDER 4 adds the second neighbours along each axis; beyond the boundary the ghost value is
// minus the centre point (odd reflection of homogeneous Dirichlet data).  With a c^2 field
// (FIELD, g.c2f) the coefficients are those of c = 1 and the operator's terms are scaled by c_j^2:
// W^{n+1} = a_cur W^n - W^{n-1} + c_j^2 (A0 W^n + Ax sx + ... - a_cur W^n).
template <int NF, int DIM, int ORDER, bool FIELD, bool FORCED>
__device__ __forceinline__ double leapfrog_point(const double* __restrict__ Wc,
                                                 const double* __restrict__ Wp,
                                                 const double* __restrict__ f,
                                                 const StepParams<NF>& a, const Geom& g,
                                                 const PointIndex& x) {
  const int64_t li = g.layer_axis == 0 ? x.i : (g.layer_axis == 1 ? x.j : x.k);
  const bool up = li >= g.layer_split;
  const double A0 = up ? a.hi.A0 : a.lo.A0;
  const double Ax = up ? a.hi.Ax : a.lo.Ax;
  const double Ay = up ? a.hi.Ay : a.lo.Ay;
  const int64_t p = x.p;
  const double wc = Wc[p];
  const double sx = Wc[p - 1] + Wc[p + 1];
  const double sy = Wc[p - g.sy] + Wc[p + g.sy];
  // W^{n-1} is absent on the first step: a zero operand (not a second FP64 instruction under
  // a predicate) keeps one FP64 FMA per point; fma(A0, wc, -0) rounds exactly as A0 * wc
  const double wprev = a.first ? 0.0 : Wp[p];
  double acc = FIELD ? (A0 - a.acur) * wc : fma(A0, wc, -wprev);
  acc = fma(Ax, sx, acc);
  acc = fma(Ay, sy, acc);
  if (DIM == 3) {
    const double Az = up ? a.hi.Az : a.lo.Az;
    const double sz = Wc[p - g.sz] + Wc[p + g.sz];
    acc = fma(Az, sz, acc);
  }
  if (ORDER == 4) {
    const double Bx = up ? a.hi.Bx : a.lo.Bx;
    const double By = up ? a.hi.By : a.lo.By;
    const double tx = (x.i == 1 ? -wc : Wc[p - 2]) + (x.i == g.nx - 1 ? -wc : Wc[p + 2]);
    const double ty = (x.j == 1 ? -wc : Wc[p - 2 * g.sy]) + (x.j == g.ny - 1 ? -wc : Wc[p + 2 * g.sy]);
    acc = fma(Bx, tx, acc);
    acc = fma(By, ty, acc);
    if (DIM == 3) {
      const double Bz = up ? a.hi.Bz : a.lo.Bz;
      const double tz = (x.k == 1 ? -wc : Wc[p - 2 * g.sz]) + (x.k == g.nz - 1 ? -wc : Wc[p + 2 * g.sz]);
      acc = fma(Bz, tz, acc);
    }
  }
  if (FIELD) acc = fma(g.c2f[p], acc, fma(a.acur, wc, -wprev));
  if (FORCED) {
#pragma unroll
    for (int m = 0; m < NF; ++m) acc = fma(-a.fneg[m], f[m * g.points + p], acc);
  }
  return acc;
}

template <int NF, int DIM>
__global__ void __launch_bounds__(kBX * kBY)
k_init(const double* __restrict__ v, double* __restrict__ W0, float2* __restrict__ q,
       const InitParams<NF> a, const Geom g) {
  const PointIndex x = point_index<DIM>(g);
  if (!x.inside) return;
  if (!MFWH_IDX(g.fault, x.p, g.points)) return;
  double w = 0.0;
  if (x.interior && v != nullptr) {
#pragma unroll
    for (int m = 0; m < NF; ++m) w += v[m * g.points + x.p];
  }
  W0[x.p] = w;
#pragma unroll
  for (int m = 0; m < NF; ++m) q[m * g.points + x.p] = fpair_from(a.w0[m] * w);
}

template <int NF, int DIM, int ORDER, bool FIELD, bool FORCED>
__global__ void __launch_bounds__(kBX * kBY)
k_step(const double* __restrict__ Wc, double* __restrict__ Wp, const double* __restrict__ f,
       float2* __restrict__ q, const StepParams<NF> a, const Geom g) {
  const PointIndex x = point_index<DIM>(g);
  if (!x.interior) return;           // boundary values stay 0 (Dirichlet, g = 0)
  // index-checked build: the nearest neighbours along the outermost axis lie in the arrays
  // (they bound every other read and write of the point; f, q: [NF][points])
  const int64_t reach = DIM == 3 ? g.sz : g.sy;
  if (!MFWH_IDX(g.fault, x.p - reach, g.points) || !MFWH_IDX(g.fault, x.p + reach, g.points))
    return;
  const double wn = leapfrog_point<NF, DIM, ORDER, FIELD, FORCED>(Wc, Wp, f, a, g, x);
  Wp[x.p] = wn;
  const float2 xw = fpair_split(wn);
#pragma unroll
  for (int m = 0; m < NF; ++m) {
    float2* qm = q + m * g.points + x.p;
    *qm = fpair_fma(a.wq_hi[m], a.wq_lo[m], xw.x, xw.y, *qm);
  }
}

template <int NF, int DIM, int ORDER, bool FIELD>
__global__ void __launch_bounds__(kBX * kBY)
k_last(const double* __restrict__ Wc, const double* __restrict__ Wp, const double* __restrict__ f,
       const float2* __restrict__ q, double* vout, const double* vsub, const LastParams<NF> a,
       const Geom g) {
  const PointIndex x = point_index<DIM>(g);
  if (!x.inside) return;
  if (!MFWH_IDX(g.fault, x.p, g.points)) return;
  if (!x.interior) {
#pragma unroll
    for (int m = 0; m < NF; ++m) vout[m * g.points + x.p] = 0.0;
    return;
  }
  {
    const int64_t reach = DIM == 3 ? g.sz : g.sy;
    if (!MFWH_IDX(g.fault, x.p - reach, g.points) || !MFWH_IDX(g.fault, x.p + reach, g.points))
      return;
  }
  const double wn = a.st.forced ? leapfrog_point<NF, DIM, ORDER, FIELD, true>(Wc, Wp, f, a.st, g, x)
                                : leapfrog_point<NF, DIM, ORDER, FIELD, false>(Wc, Wp, f, a.st, g, x);
  double qq[NF];
#pragma unroll
  for (int m = 0; m < NF; ++m) qq[m] = fma(a.st.wq[m], wn, fpair_value(q[m * g.points + x.p]));
  double vk[NF];
  if (a.has_e) {
#pragma unroll
    for (int j = 0; j < NF; ++j) vk[j] = a.vprev[j * g.points + x.p];
  }
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
    out[m] = a.subtract ? vsub[m * g.points + x.p] - s : s;
  }
#pragma unroll
  for (int m = 0; m < NF; ++m) vout[m * g.points + x.p] = out[m];
}

// ---- Helmholtz residual -------------------------------------------------------

constexpr int kResBlocks = kResidualBlocks;

__device__ __forceinline__ double nanmax(double a, double b) {
  // max that propagates NaN so that non-finite iterates are reported
  return (b > a || b != b) ? b : a;
}

// h^2 times the fourth-order second difference along one axis at index idx of n cells
// (ghost values beyond the boundary are minus the centre value vc).
__device__ __forceinline__ double diff4(const double* vm, int64_t p, int64_t s, int64_t idx,
                                        int64_t n, double vc) {
  const double m2 = idx == 1 ? -vc : vm[p - 2 * s];
  const double p2 = idx == n - 1 ? -vc : vm[p + 2 * s];
  return (16.0 * (vm[p - s] + vm[p + s]) - (m2 + p2) - 30.0 * vc) / 12.0;
}

template <int NF>
struct ResParams {
  double omega2[NF];
  double c2_lo, c2_hi;
  double ihx2, ihy2, ihz2;
};

template <int NF, int DIM>
__global__ void __launch_bounds__(256)
k_residual(const double* __restrict__ v, const double* __restrict__ f, const ResParams<NF> a,
           const Geom g, double* __restrict__ partial) {
  double rmax[NF], fmax_[NF];
#pragma unroll
  for (int m = 0; m < NF; ++m) rmax[m] = fmax_[m] = 0.0;
  const int64_t nx1 = g.nx + 1, ny1 = g.ny + 1;
  const int64_t total = g.points;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % nx1;
    const int64_t j = (p / nx1) % ny1;
    const int64_t k = (DIM == 3) ? p / (nx1 * ny1) : 0;
    if (i == 0 || i == g.nx || j == 0 || j == g.ny) continue;
    if (DIM == 3 && (k == 0 || k == g.nz)) continue;
    const int64_t li = g.layer_axis == 0 ? i : (g.layer_axis == 1 ? j : k);
    const double c2 = g.c2f ? g.c2f[p] : (li >= g.layer_split ? a.c2_hi : a.c2_lo);
#pragma unroll
    for (int m = 0; m < NF; ++m) {
      const double* vm = v + m * g.points;
      const double vc = vm[p];
      double lap;
      if (g.order == 4) {
        lap = a.ihx2 * diff4(vm, p, 1, i, g.nx, vc) + a.ihy2 * diff4(vm, p, g.sy, j, g.ny, vc);
        if (DIM == 3) lap += a.ihz2 * diff4(vm, p, g.sz, k, g.nz, vc);
      } else {
        lap = a.ihx2 * (vm[p - 1] - 2.0 * vc + vm[p + 1]) +
              a.ihy2 * (vm[p - g.sy] - 2.0 * vc + vm[p + g.sy]);
        if (DIM == 3) lap += a.ihz2 * (vm[p - g.sz] - 2.0 * vc + vm[p + g.sz]);
      }
      const double fm = f[m * g.points + p];
      const double r = fm - (c2 * lap + a.omega2[m] * vc);
      rmax[m] = nanmax(rmax[m], fabs(r));
      fmax_[m] = nanmax(fmax_[m], fabs(fm));
    }
  }
  __shared__ double red[2 * NF][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < NF; ++m) {
    double r = rmax[m], fv = fmax_[m];
    for (int o = 16; o > 0; o >>= 1) {
      r = nanmax(r, __shfl_xor_sync(0xffffffffu, r, o));
      fv = nanmax(fv, __shfl_xor_sync(0xffffffffu, fv, o));
    }
    if (lane == 0) {
      red[m][warp] = r;
      red[NF + m][warp] = fv;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * NF) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = nanmax(r, red[threadIdx.x][w]);
    partial[(int64_t)blockIdx.x * 2 * NF + threadIdx.x] = r;
  }
}

__global__ void k_max_partials(const double* __restrict__ partial, int nblocks, int width,
                               double* __restrict__ out) {
  // one thread per output column
  const int c = threadIdx.x;
  if (c >= width) return;
  double r = 0.0;
  for (int b = 0; b < nblocks; ++b) r = nanmax(r, partial[(int64_t)b * width + c]);
  out[c] = r;
}

dim3 step_grid(const Geom& g) {
  return dim3((unsigned)((g.nx + 1 + kBX - 1) / kBX), (unsigned)((g.ny + 1 + kBY - 1) / kBY),
              (unsigned)(g.dim == 3 ? g.nz + 1 : 1));
}

template <int NF>
void init_nf(const Geom& g, const double* v, double* W0, double* q, const double* w0,
             cudaStream_t st) {
  InitParams<NF> a;
  for (int m = 0; m < NF; ++m) a.w0[m] = w0[m];
  float2* qp = reinterpret_cast<float2*>(q);
  dim3 blk(kBX, kBY);
  if (g.dim == 2)
    k_init<NF, 2><<<step_grid(g), blk, 0, st>>>(v, W0, qp, a, g);
  else
    k_init<NF, 3><<<step_grid(g), blk, 0, st>>>(v, W0, qp, a, g);
}

// Kernel instance for the grid: dimension, operator order and whether c^2 is a field (a
// compile-time choice, so that the constant-c kernels carry no field code at all).
template <int NF, bool FIELD, bool FORCED>
void step_nf_f(const Geom& g, const double* Wc, double* Wp, const double* f, float2* qp,
               const StepParams<NF>& a, cudaStream_t st) {
  dim3 blk(kBX, kBY);
  if (g.order == 4) {
    if (g.dim == 2)
      k_step<NF, 2, 4, FIELD, FORCED><<<step_grid(g), blk, 0, st>>>(Wc, Wp, f, qp, a, g);
    else
      k_step<NF, 3, 4, FIELD, FORCED><<<step_grid(g), blk, 0, st>>>(Wc, Wp, f, qp, a, g);
  } else if (g.dim == 2) {
    k_step<NF, 2, 2, FIELD, FORCED><<<step_grid(g), blk, 0, st>>>(Wc, Wp, f, qp, a, g);
  } else {
    k_step<NF, 3, 2, FIELD, FORCED><<<step_grid(g), blk, 0, st>>>(Wc, Wp, f, qp, a, g);
  }
}

template <int NF>
void step_nf(const Geom& g, const double* Wc, double* Wp, const double* f, double* q,
             const StepHost& h, cudaStream_t st) {
  const StepParams<NF> a = to_params<NF>(h);
  float2* qp = reinterpret_cast<float2*>(q);
  if (g.c2f) {
    if (h.forced)
      step_nf_f<NF, true, true>(g, Wc, Wp, f, qp, a, st);
    else
      step_nf_f<NF, true, false>(g, Wc, Wp, f, qp, a, st);
  } else if (h.forced) {
    step_nf_f<NF, false, true>(g, Wc, Wp, f, qp, a, st);
  } else {
    step_nf_f<NF, false, false>(g, Wc, Wp, f, qp, a, st);
  }
}

template <int NF, bool FIELD>
void last_nf_f(const Geom& g, const double* Wc, const double* Wp, const double* f,
               const float2* qp, double* vout, const double* vsub, const LastParams<NF>& a,
               cudaStream_t st) {
  dim3 blk(kBX, kBY);
  if (g.order == 4) {
    if (g.dim == 2)
      k_last<NF, 2, 4, FIELD><<<step_grid(g), blk, 0, st>>>(Wc, Wp, f, qp, vout, vsub, a, g);
    else
      k_last<NF, 3, 4, FIELD><<<step_grid(g), blk, 0, st>>>(Wc, Wp, f, qp, vout, vsub, a, g);
  } else if (g.dim == 2) {
    k_last<NF, 2, 2, FIELD><<<step_grid(g), blk, 0, st>>>(Wc, Wp, f, qp, vout, vsub, a, g);
  } else {
    k_last<NF, 3, 2, FIELD><<<step_grid(g), blk, 0, st>>>(Wc, Wp, f, qp, vout, vsub, a, g);
  }
}

template <int NF>
void last_nf(const Geom& g, const double* Wc, const double* Wp, const double* f, const double* q,
             double* vout, const double* vsub, const StepHost& h, cudaStream_t st) {
  LastParams<NF> a;
  a.st = to_params<NF>(h);
  for (int m = 0; m < NF; ++m)
    for (int j = 0; j < NF; ++j) {
      a.binv[m * NF + j] = h.binv[m * MFWH_MAX_NF + j];
      a.emat[m * NF + j] = h.emat[m * MFWH_MAX_NF + j];
    }
  a.subtract = h.subtract;
  a.has_e = h.has_e && h.vprev != nullptr;
  a.vprev = h.vprev;
  const float2* qp = reinterpret_cast<const float2*>(q);
  if (g.c2f)
    last_nf_f<NF, true>(g, Wc, Wp, f, qp, vout, vsub, a, st);
  else
    last_nf_f<NF, false>(g, Wc, Wp, f, qp, vout, vsub, a, st);
}

// R_m = f_m - (c^2 Delta_h + omega_m^2) v_m at interior points, 0 on the boundary: the
// defect of v in the discrete Helmholtz system (eq. MultipleHelmholtz), one thread per point.
template <int NF, int DIM>
__global__ void __launch_bounds__(kBX * kBY)
k_residual_field(const double* __restrict__ v, const double* __restrict__ f,
                 const ResParams<NF> a, const Geom g, double* __restrict__ R) {
  const PointIndex x = point_index<DIM>(g);
  if (!x.inside) return;
  if (!x.interior) {
#pragma unroll
    for (int m = 0; m < NF; ++m) R[m * g.points + x.p] = 0.0;
    return;
  }
  const int64_t li = g.layer_axis == 0 ? x.i : (g.layer_axis == 1 ? x.j : x.k);
  const int64_t p = x.p;
  const double c2 = g.c2f ? g.c2f[p] : (li >= g.layer_split ? a.c2_hi : a.c2_lo);
#pragma unroll
  for (int m = 0; m < NF; ++m) {
    const double* vm = v + m * g.points;
    const double c = vm[p];
    double lap;
    if (g.order == 4) {
      lap = a.ihx2 * diff4(vm, p, 1, x.i, g.nx, c) + a.ihy2 * diff4(vm, p, g.sy, x.j, g.ny, c);
      if (DIM == 3) lap += a.ihz2 * diff4(vm, p, g.sz, x.k, g.nz, c);
    } else {
      lap = a.ihx2 * ((vm[p - 1] - c) + (vm[p + 1] - c)) +
            a.ihy2 * ((vm[p - g.sy] - c) + (vm[p + g.sy] - c));
      if (DIM == 3) lap += a.ihz2 * ((vm[p - g.sz] - c) + (vm[p + g.sz] - c));
    }
    R[m * g.points + p] = f[m * g.points + p] - (c2 * lap + a.omega2[m] * c);
  }
}

template <int NF>
void residual_field_nf(const Geom& g, const double* v, const double* f, const double* omega2,
                       double c2_lo, double c2_hi, const double* inv_h2, double* R,
                       cudaStream_t st) {
  ResParams<NF> a;
  for (int m = 0; m < NF; ++m) a.omega2[m] = omega2[m];
  a.c2_lo = c2_lo;
  a.c2_hi = c2_hi;
  a.ihx2 = inv_h2[0];
  a.ihy2 = inv_h2[1];
  a.ihz2 = inv_h2[2];
  if (g.dim == 2)
    k_residual_field<NF, 2><<<step_grid(g), dim3(kBX, kBY), 0, st>>>(v, f, a, g, R);
  else
    k_residual_field<NF, 3><<<step_grid(g), dim3(kBX, kBY), 0, st>>>(v, f, a, g, R);
}

template <int NF>
void residual_nf(const Geom& g, const double* v, const double* f, const double* omega2,
                 double c2_lo, double c2_hi, const double* inv_h2, double* partial, double* out,
                 cudaStream_t st) {
  ResParams<NF> a;
  for (int m = 0; m < NF; ++m) a.omega2[m] = omega2[m];
  a.c2_lo = c2_lo;
  a.c2_hi = c2_hi;
  a.ihx2 = inv_h2[0];
  a.ihy2 = inv_h2[1];
  a.ihz2 = inv_h2[2];
  if (g.dim == 2)
    k_residual<NF, 2><<<kResBlocks, 256, 0, st>>>(v, f, a, g, partial);
  else
    k_residual<NF, 3><<<kResBlocks, 256, 0, st>>>(v, f, a, g, partial);
  k_max_partials<<<1, 64, 0, st>>>(partial, kResBlocks, 2 * NF, out);
}

}  // namespace

#define MFWH_NF_SWITCH(nf, CALL)                                   \
  switch (nf) {                                                    \
    case 1: CALL(1); break;   case 2: CALL(2); break;              \
    case 3: CALL(3); break;   case 4: CALL(4); break;              \
    case 5: CALL(5); break;   case 6: CALL(6); break;              \
    case 7: CALL(7); break;   case 8: CALL(8); break;              \
    case 9: CALL(9); break;   case 10: CALL(10); break;            \
    case 11: CALL(11); break; case 12: CALL(12); break;            \
    case 13: CALL(13); break; case 14: CALL(14); break;            \
    case 15: CALL(15); break; case 16: CALL(16); break;            \
    default: break;                                                \
  }

void launch_init(int nf, const Geom& g, const double* v, double* W0, double* q, const double* w0,
                 cudaStream_t st) {
#define CALL(N) init_nf<N>(g, v, W0, q, w0, st)
  MFWH_NF_SWITCH(nf, CALL)
#undef CALL
}

void launch_step(int nf, const Geom& g, const double* Wc, double* Wp, const double* f, double* q,
                 const StepHost& a, cudaStream_t st) {
#define CALL(N) step_nf<N>(g, Wc, Wp, f, q, a, st)
  MFWH_NF_SWITCH(nf, CALL)
#undef CALL
}

void launch_last(int nf, const Geom& g, const double* Wc, const double* Wp, const double* f,
                 const double* q, double* vout, const double* vsub, const StepHost& a,
                 cudaStream_t st) {
#define CALL(N) last_nf<N>(g, Wc, Wp, f, q, vout, vsub, a, st)
  MFWH_NF_SWITCH(nf, CALL)
#undef CALL
}

void launch_residual(int nf, const Geom& g, const double* v, const double* f, const double* omega2,
                     double c2_lo, double c2_hi, const double* inv_h2, double* partial, double* out,
                     cudaStream_t st) {
#define CALL(N) residual_nf<N>(g, v, f, omega2, c2_lo, c2_hi, inv_h2, partial, out, st)
  MFWH_NF_SWITCH(nf, CALL)
#undef CALL
}

int64_t residual_partial_size(int nf) { return (int64_t)kResBlocks * 2 * nf; }

void launch_residual_field(int nf, const Geom& g, const double* v, const double* f,
                           const double* omega2, double c2_lo, double c2_hi, const double* inv_h2,
                           double* R, cudaStream_t st) {
#define CALL(N) residual_field_nf<N>(g, v, f, omega2, c2_lo, c2_hi, inv_h2, R, st)
  MFWH_NF_SWITCH(nf, CALL)
#undef CALL
}

}  // namespace mfwh

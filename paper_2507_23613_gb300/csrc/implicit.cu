// Implicit trapezoidal time stepping of the MFWH wave solve, FP64 results (Section "Explicit
// and implicit time-stepping", eq. WaveScheme with (alpha, beta) = (1/2, 0)).
//
// With A = I - (dt^2/2) L_h the scheme
//   A W^{n+1} = 2 W^n - A W^{n-1} - dt^2 F^n,   F^n = sum_m f_m cos(omega~_m t^n) cos(omega~_m dt)
// is solved as A Z = 2 W^n - dt^2 F^n, W^{n+1} = Z - W^{n-1}; the first step (eq.
// implicitFirstStep with beta = 0) is the same solve with W^1 = Z / 2.  A is symmetric
// positive definite and, for the steps of 5-10 per period the method uses, strongly
// Laplacian-dominated on fine grids and identity-dominated on coarse ones, so geometric
// multigrid solves it in a few V-cycles (the paper solves it with multigrid to 1e-10).
//
// Multigrid: vertex-centred coarsening by 2 in every axis, red-black Gauss-Seidel smoothing
// (2 sweeps before, 1 after the coarse correction), full-weighting restriction of the
// residual, multilinear prolongation, and the operator rediscretised on every level
// (pointwise c^2 of the level's grid points).  Levels of at most kMgCoarsePoints points are
// solved by one CTA in shared memory (the coarsest with coarse_sweeps sweeps).
//
// Precision.  A 2D hierarchy with grid-wide levels runs defect correction: each cycle forms
// the residual r = rhs - A Z in FP64, solves A e = r approximately by one FP32 V-cycle from
// e = 0, and adds e to Z in FP64, so the iterate converges to the FP64 solution at the
// V-cycle's rate while the smoothing runs on the FP32 pipes (GB300 issues FP64 arithmetic at
// a small fraction of its FP32 rate).  2D grid-wide levels run in tiled shared-memory phases,
// 3D ones in grid-wide phases.  Hierarchies held by one CTA (grids of at most 5000 points)
// run the V-cycles on Z itself in FP64.
//
// One step is one launch.  When the hierarchy has grid-wide levels the launch is
// cooperative (all blocks resident) and phases are separated by a grid barrier whose waits
// are bounded in time (ImpArgs::wait_ns, 2 s by default): a wait that runs out sets *err = 2
// and makes every later barrier of the launch pass through, so the launch ends and the host
// reports the error.  The convergence test max|rhs - A Z| <= tol max|rhs| is evaluated once
// per cycle from a grid-wide atomicMax, read after a barrier; one thread per block reads it
// and shares it through shared memory, so the threads of a block always take the same branch
// (also after a timed-out barrier, when blocks may read the maximum at different moments).
// No index depends on data, and every loop has a bound, so a launch whose barriers pass
// through still ends after its usual number of phases with all accesses in bounds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace mfwh {
namespace {

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double nanmax(double a, double b) { return (b > a || b != b) ? b : a; }

// Grid barrier for a cooperative launch.  Bounded wait (wait_ns); see the file comment.
__device__ void grid_sync(unsigned* bar, int* err, unsigned long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile int*)err == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*gen == g0) {
        __nanosleep(32);
        if (*(volatile int*)err != 0) break;
        if (global_ns() - t0 > wait_ns) {
          atomicExch(err, 2);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Max over the block (all threads get the result).  red: shared scratch of 32 doubles.
__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x = nanmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (l == 0) red[0] = x;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* slot, double v) {
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double load_nonneg(const unsigned long long* slot) {
  return __longlong_as_double((long long)*(const volatile unsigned long long*)slot);
}

// Convergence test of cycle c taken once per block: thread 0 reads the grid-wide maximum and
// shares the decision, so that all threads of the block branch alike.  flag: shared int.
__device__ bool block_converged(const MgState* st, int c, double thresh, int* flag) {
  if (threadIdx.x == 0) *flag = load_nonneg(&st->rmax[c]) <= thresh ? 1 : 0;
  __syncthreads();
  const bool r = *flag != 0;
  __syncthreads();
  return r;
}

// Coefficients of a level in the arithmetic type R.
template <typename R>
struct Co;
template <>
struct Co<double> {
  __device__ static const double* a(const MgLevel& L, bool hi) { return hi ? L.a_hi : L.a_lo; }
  __device__ static double d(const MgLevel& L, bool hi) { return hi ? L.d_hi : L.d_lo; }
  __device__ static double dinv(const MgLevel& L, bool hi) { return hi ? L.dinv_hi : L.dinv_lo; }
};
template <>
struct Co<float> {
  __device__ static const float* a(const MgLevel& L, bool hi) { return hi ? L.a32_hi : L.a32_lo; }
  __device__ static float d(const MgLevel& L, bool hi) { return hi ? L.d32_hi : L.d32_lo; }
  __device__ static float dinv(const MgLevel& L, bool hi) { return hi ? L.dinv32_hi : L.dinv32_lo; }
};

__device__ __forceinline__ bool upper(const MgLevel& L, int axis, int i, int j, int k) {
  return (axis == 0 ? i : (axis == 1 ? j : k)) >= L.split;
}
// Sum of a_i (u_{p+e_i} + u_{p-e_i}); sy, sz are the strides of the array u.
template <int DIM, typename R>
__device__ __forceinline__ R neighbours(const R* u, int64_t p, int64_t sy, int64_t sz, const R* a) {
  R s = a[0] * (u[p - 1] + u[p + 1]) + a[1] * (u[p - sy] + u[p + sy]);
  if (DIM == 3) s += a[2] * (u[p - sz] + u[p + sz]);
  return s;
}
template <int DIM, typename R>
__device__ __forceinline__ R residual_at(const MgLevel& L, const R* u, const R* f, int axis, int i,
                                         int j, int k) {
  const int64_t p = (int64_t)k * L.sz + (int64_t)j * L.sy + i;
  const bool hi = upper(L, axis, i, j, k);
  const R s = neighbours<DIM, R>(u, p, L.sy, L.sz, Co<R>::a(L, hi));
  return f[p] - (Co<R>::d(L, hi) * u[p] - s);
}

// One red (color 0) or black (color 1) half-sweep; (t0, stride) split the colour's points.
template <int DIM, typename R>
__device__ void rb_half(const MgLevel& L, R* u, const R* f, int color, int axis, uint32_t t0,
                        uint32_t stride) {
  const uint32_t hw = (uint32_t)L.nx / 2;
  const uint32_t my = (uint32_t)L.ny - 1;
  const uint32_t total = hw * my * (DIM == 3 ? (uint32_t)L.nz - 1 : 1u);
  for (uint32_t t = t0; t < total; t += stride) {
    const uint32_t row = t / hw, it = t - row * hw;
    const int j = 1 + (int)(row % my);
    const int k = DIM == 3 ? 1 + (int)(row / my) : 0;
    const int i = (((j + k + color) & 1) ? 1 : 2) + 2 * (int)it;
    if (i > L.nx - 1) continue;
    const int64_t p = (int64_t)k * L.sz + (int64_t)j * L.sy + i;
    const bool hi = upper(L, axis, i, j, k);
    const R s = neighbours<DIM, R>(u, p, L.sy, L.sz, Co<R>::a(L, hi));
    u[p] = (f[p] + s) * Co<R>::dinv(L, hi);
  }
}

// Residual of the interior points into r (if r) and its max over this thread's points (FP64).
template <int DIM>
__device__ double residual_pass(const MgLevel& L, const double* u, const double* f, double* r,
                                int axis, uint32_t t0, uint32_t stride) {
  const uint32_t mx = (uint32_t)L.nx - 1, my = (uint32_t)L.ny - 1;
  const uint32_t total = mx * my * (DIM == 3 ? (uint32_t)L.nz - 1 : 1u);
  double m = 0.0;
  for (uint32_t t = t0; t < total; t += stride) {
    const int i = 1 + (int)(t % mx);
    const uint32_t rest = t / mx;
    const int j = 1 + (int)(rest % my);
    const int k = DIM == 3 ? 1 + (int)(rest / my) : 0;
    const double res = residual_at<DIM, double>(L, u, f, axis, i, j, k);
    if (r) r[(int64_t)k * L.sz + (int64_t)j * L.sy + i] = res;
    m = nanmax(m, fabs(res));
  }
  return m;
}

// Residual of the interior points stored into r (type R).
template <int DIM, typename R>
__device__ void residual_store(const MgLevel& L, const R* u, const R* f, R* r, int axis,
                               uint32_t t0, uint32_t stride) {
  const uint32_t mx = (uint32_t)L.nx - 1, my = (uint32_t)L.ny - 1;
  const uint32_t total = mx * my * (DIM == 3 ? (uint32_t)L.nz - 1 : 1u);
  for (uint32_t t = t0; t < total; t += stride) {
    const int i = 1 + (int)(t % mx);
    const uint32_t rest = t / mx;
    const int j = 1 + (int)(rest % my);
    const int k = DIM == 3 ? 1 + (int)(rest / my) : 0;
    r[(int64_t)k * L.sz + (int64_t)j * L.sy + i] = residual_at<DIM, R>(L, u, f, axis, i, j, k);
  }
}

// Z of a 3D level 0 at (i, j, k), each index in [-1, n + 1]: one point beyond the Dirichlet
// boundary the fourth-order stencil reads the odd-reflection ghost (Z_{-1} = -Z_1,
// Z_{n+1} = -Z_{n-1}), as L_4h is defined on the interior unknowns.
__device__ __forceinline__ double z_ghost3(const MgLevel& F, int i, int j, int k) {
  double sgn = 1.0;
  if (i == -1) { i = 1; sgn = -sgn; }
  if (i == F.nx + 1) { i = F.nx - 1; sgn = -sgn; }
  if (j == -1) { j = 1; sgn = -sgn; }
  if (j == F.ny + 1) { j = F.ny - 1; sgn = -sgn; }
  if (k == -1) { k = 1; sgn = -sgn; }
  if (k == F.nz + 1) { k = F.nz - 1; sgn = -sgn; }
  return sgn * F.u[(int64_t)k * F.sz + (int64_t)j * F.sy + i];
}

// FP64 residual rhs - A_4 Z at an interior point of a 3D level 0 with the fourth-order
// operator: A_4 = d4 - sum_a (a4_a (Z_{+-1}) + b4_a (Z_{+-2})) along each axis a.
__device__ __forceinline__ double residual4_3d(const MgLevel& F, int axis, int i, int j, int k) {
  const int64_t p = (int64_t)k * F.sz + (int64_t)j * F.sy + i;
  const bool hi = upper(F, axis, i, j, k);
  const double* a4 = hi ? F.a4_hi : F.a4_lo;
  const double* b4 = hi ? F.b4_hi : F.b4_lo;
  const double* u = F.u;
  const double s =
      a4[0] * (u[p - 1] + u[p + 1]) + a4[1] * (u[p - F.sy] + u[p + F.sy]) +
      a4[2] * (u[p - F.sz] + u[p + F.sz]) +
      b4[0] * (z_ghost3(F, i - 2, j, k) + z_ghost3(F, i + 2, j, k)) +
      b4[1] * (z_ghost3(F, i, j - 2, k) + z_ghost3(F, i, j + 2, k)) +
      b4[2] * (z_ghost3(F, i, j, k - 2) + z_ghost3(F, i, j, k + 2));
  return F.f[p] - ((hi ? F.d4_hi : F.d4_lo) * u[p] - s);
}

// Level 0 of a grid-wide 3D hierarchy: r = rhs - A Z in FP64 into f32 (the correction's
// right-hand side), e = 0 in u32; returns the max |r| over this thread's points.  A is the
// second-order operator, or the fourth-order one when L.order4 is set.
template <int DIM>
__device__ double residual_to32(const MgLevel& L, int axis, uint32_t t0, uint32_t stride) {
  const uint32_t mx = (uint32_t)L.nx - 1, my = (uint32_t)L.ny - 1;
  const uint32_t total = mx * my * (DIM == 3 ? (uint32_t)L.nz - 1 : 1u);
  double m = 0.0;
  for (uint32_t t = t0; t < total; t += stride) {
    const int i = 1 + (int)(t % mx);
    const uint32_t rest = t / mx;
    const int j = 1 + (int)(rest % my);
    const int k = DIM == 3 ? 1 + (int)(rest / my) : 0;
    const double res = (DIM == 3 && L.order4) ? residual4_3d(L, axis, i, j, k)
                                              : residual_at<DIM, double>(L, L.u, L.f, axis, i, j, k);
    const int64_t p = (int64_t)k * L.sz + (int64_t)j * L.sy + i;
    L.f32[p] = (float)res;
    L.u32[p] = 0.0f;
    m = nanmax(m, fabs(res));
  }
  return m;
}

// Z += omega e at the interior points (FP64).
template <int DIM>
__device__ void add_correction(const MgLevel& L, double omega, uint32_t t0, uint32_t stride) {
  const uint32_t mx = (uint32_t)L.nx - 1, my = (uint32_t)L.ny - 1;
  const uint32_t total = mx * my * (DIM == 3 ? (uint32_t)L.nz - 1 : 1u);
  for (uint32_t t = t0; t < total; t += stride) {
    const int i = 1 + (int)(t % mx);
    const uint32_t rest = t / mx;
    const int j = 1 + (int)(rest % my);
    const int k = DIM == 3 ? 1 + (int)(rest / my) : 0;
    const int64_t p = (int64_t)k * L.sz + (int64_t)j * L.sy + i;
    L.u[p] = fma(omega, (double)L.u32[p], L.u[p]);
  }
}

// Full weighting of the fine residual onto the coarse interior: weights 1/2 at offset 0 and
// 1/4 at offsets +-1 per axis.  The residual comes from rf, or (rf null) is evaluated from
// (uf, ff).  The coarse correction uc starts at 0.
template <int DIM, typename R>
__device__ void restrict_pass(const MgLevel& F, const R* rf, const R* uf, const R* ff,
                              const MgLevel& C, R* fc, R* uc, int axis, uint32_t t0,
                              uint32_t stride) {
  const uint32_t mx = (uint32_t)C.nx - 1, my = (uint32_t)C.ny - 1;
  const uint32_t total = mx * my * (DIM == 3 ? (uint32_t)C.nz - 1 : 1u);
  for (uint32_t t = t0; t < total; t += stride) {
    const int I = 1 + (int)(t % mx);
    const uint32_t rest = t / mx;
    const int J = 1 + (int)(rest % my);
    const int K = DIM == 3 ? 1 + (int)(rest / my) : 0;
    R acc = 0;
    for (int c = (DIM == 3 ? -1 : 0); c <= (DIM == 3 ? 1 : 0); ++c) {
      const R wc = DIM == 3 ? (c == 0 ? R(0.5) : R(0.25)) : R(1);
      for (int b = -1; b <= 1; ++b) {
        const R wb = b == 0 ? R(0.5) : R(0.25);
        for (int a = -1; a <= 1; ++a) {
          const R wa = a == 0 ? R(0.5) : R(0.25);
          const int i = 2 * I + a, j = 2 * J + b, k = DIM == 3 ? 2 * K + c : 0;
          const R r = rf ? rf[(int64_t)k * F.sz + (int64_t)j * F.sy + i]
                         : residual_at<DIM, R>(F, uf, ff, axis, i, j, k);
          acc += wc * wb * wa * r;
        }
      }
    }
    const int64_t P = (int64_t)K * C.sz + (int64_t)J * C.sy + I;
    fc[P] = acc;
    uc[P] = 0;
  }
}

// Multilinear interpolation at fine point (i, j, k) of a coarse grid function (coarse boundary
// values are 0).
template <int DIM, typename R>
__device__ __forceinline__ R prolong_at(const MgLevel& C, const R* uc, int i, int j, int k) {
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  auto line = [&](int JJ, int KK) {
    const R* c = uc + (int64_t)KK * C.sz + (int64_t)JJ * C.sy;
    return (i & 1) ? R(0.5) * (c[I] + c[I + 1]) : c[I];
  };
  auto plane = [&](int KK) {
    return (j & 1) ? R(0.5) * (line(J, KK) + line(J + 1, KK)) : line(J, KK);
  };
  R v = plane(K);
  if (DIM == 3 && (k & 1)) v = R(0.5) * (v + plane(K + 1));
  return v;
}

// u_f += interpolation of the coarse correction at every fine interior point.
template <int DIM, typename R>
__device__ void prolong_pass(const MgLevel& C, const R* uc, const MgLevel& F, R* uf, uint32_t t0,
                             uint32_t stride) {
  const uint32_t mx = (uint32_t)F.nx - 1, my = (uint32_t)F.ny - 1;
  const uint32_t total = mx * my * (DIM == 3 ? (uint32_t)F.nz - 1 : 1u);
  for (uint32_t t = t0; t < total; t += stride) {
    const int i = 1 + (int)(t % mx);
    const uint32_t rest = t / mx;
    const int j = 1 + (int)(rest % my);
    const int k = DIM == 3 ? 1 + (int)(rest / my) : 0;
    uf[(int64_t)k * F.sz + (int64_t)j * F.sy + i] += prolong_at<DIM, R>(C, uc, i, j, k);
  }
}

// ---- tiled FP32 phases of a 2D hierarchy --------------------------------------------
// Shared-memory copies over the tile's region [is, is + Wd) x [js, js + Wd).  Tiles own fine
// points [1 + t T, 1 + (t + 1) T) per axis and the coarse points I whose centre 2I is one of
// them.  A point update, residual or restriction computes what rb_half, residual_at and
// restrict_pass compute on the whole grid (same operations in the same order).

// Half-sweep of colour `color` over the square [ri, ri + S) x [rj, rj + S).
__device__ void tile_half(const MgLevel& F, float* su, const float* sf, int Wd, int is, int js,
                          int ri, int rj, int S, int color, int axis) {
  const int hw = (S + 1) / 2;
  for (int t = threadIdx.x; t < hw * S; t += blockDim.x) {
    const int r = t / hw, it = t - r * hw;
    const int j = rj + r;
    const int i = ri + (((ri + j + color) & 1) ? 1 : 0) + 2 * it;
    if (i >= ri + S || i < 1 || i > F.nx - 1 || j < 1 || j > F.ny - 1) continue;
    const int x = (j - js) * Wd + (i - is);
    const bool hi = upper(F, axis, i, j, 0);
    const float s = neighbours<2, float>(su, x, Wd, 0, Co<float>::a(F, hi));
    su[x] = (sf[x] + s) * Co<float>::dinv(F, hi);
  }
}

__device__ __forceinline__ float tile_res(const MgLevel& F, const float* su, const float* sf,
                                          int Wd, int is, int js, int i, int j, int axis) {
  const int x = (j - js) * Wd + (i - is);
  const bool hi = upper(F, axis, i, j, 0);
  const float s = neighbours<2, float>(su, x, Wd, 0, Co<float>::a(F, hi));
  return sf[x] - (Co<float>::d(F, hi) * su[x] - s);
}

// Smooth e from 0 with 2 sweeps in shared memory (sf holds the right-hand side), then write
// the owned points to F.v32 and restrict the residual onto C.f32.
__device__ void tile_down_rest(const MgLevel& F, const MgLevel& C, float* su, const float* sf,
                               int Wd, int is, int js, int i0, int j0, int T, int axis) {
  const int H = kMgHalo;
  for (int h = 0; h < 4; ++h) {
    const int d = H - 1 - h;
    tile_half(F, su, sf, Wd, is, js, i0 - d, j0 - d, T + 2 * d, h & 1, axis);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < T * T; t += blockDim.x) {
    const int i = i0 + t % T, j = j0 + t / T;
    if (i > F.nx - 1 || j > F.ny - 1) continue;
    F.v32[(int64_t)j * F.sy + i] = su[(j - js) * Wd + (i - is)];
  }
  const int Tc = T / 2, I0 = (i0 + 1) / 2, J0 = (j0 + 1) / 2;
  for (int t = threadIdx.x; t < Tc * Tc; t += blockDim.x) {
    const int I = I0 + t % Tc, J = J0 + t / Tc;
    if (I > C.nx - 1 || J > C.ny - 1) continue;
    float acc = 0.0f;
    for (int b = -1; b <= 1; ++b) {
      const float wb = b == 0 ? 0.5f : 0.25f;
      for (int a = -1; a <= 1; ++a) {
        const float wa = a == 0 ? 0.5f : 0.25f;
        acc += 1.0f * wb * wa * tile_res(F, su, sf, Wd, is, js, 2 * I + a, 2 * J + b, axis);
      }
    }
    C.f32[(int64_t)J * C.sy + I] = acc;
  }
}

// Z at (i, j) for the residual stencils: grid values, the odd reflection -Z one point beyond
// a boundary (the fourth-order ghost value), 0 farther out (never used).
__device__ __forceinline__ double z_ghost(const MgLevel& F, int i, int j) {
  double sgn = 1.0;
  if (i == -1) { i = 1; sgn = -sgn; }
  if (i == F.nx + 1) { i = F.nx - 1; sgn = -sgn; }
  if (j == -1) { j = 1; sgn = -sgn; }
  if (j == F.ny + 1) { j = F.ny - 1; sgn = -sgn; }
  if (i < 0 || i > F.nx || j < 0 || j > F.ny) return 0.0;
  return sgn * F.u[(int64_t)j * F.sy + i];
}

// Level 0 down phase: r = rhs - A Z in FP64 on the region (Z staged with two more rings; A is
// the second- or fourth-order operator), F.f32 = r on owned points, then the FP32 smoothing
// of e from 0 and the restriction.  Returns the max |r| over this block's owned points.
__device__ double down0_tiles(const MgLevel& F, const MgLevel& C, int axis, unsigned char* smraw) {
  const int T = F.tile, H = kMgHalo, Wd = T + 2 * H, Wz = Wd + 4;
  const int ntx = (F.nx - 1 + T - 1) / T, nty = (F.ny - 1 + T - 1) / T;
  double* zs = reinterpret_cast<double*>(smraw);
  float* su = reinterpret_cast<float*>(zs + Wz * Wz);
  float* sf = su + Wd * Wd;
  double m = 0.0;
  for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
    const int i0 = 1 + (tile % ntx) * T, j0 = 1 + (tile / ntx) * T;
    const int is = i0 - H, js = j0 - H;
    for (int t = threadIdx.x; t < Wz * Wz; t += blockDim.x)
      zs[t] = z_ghost(F, is - 2 + t % Wz, js - 2 + t / Wz);
    __syncthreads();
    for (int t = threadIdx.x; t < Wd * Wd; t += blockDim.x) {
      const int i = is + t % Wd, j = js + t / Wd;
      double r = 0.0;
      if (i >= 1 && i <= F.nx - 1 && j >= 1 && j <= F.ny - 1) {
        const int64_t p = (int64_t)j * F.sy + i;
        const int x = (j - js + 2) * Wz + (i - is + 2);
        const bool hi = upper(F, axis, i, j, 0);
        if (F.order4) {
          const double* a4 = hi ? F.a4_hi : F.a4_lo;
          const double* b4 = hi ? F.b4_hi : F.b4_lo;
          const double s = a4[0] * (zs[x - 1] + zs[x + 1]) + a4[1] * (zs[x - Wz] + zs[x + Wz]) +
                           b4[0] * (zs[x - 2] + zs[x + 2]) +
                           b4[1] * (zs[x - 2 * Wz] + zs[x + 2 * Wz]);
          r = F.f[p] - ((hi ? F.d4_hi : F.d4_lo) * zs[x] - s);
        } else {
          const double s = neighbours<2, double>(zs, x, Wz, 0, Co<double>::a(F, hi));
          r = F.f[p] - (Co<double>::d(F, hi) * zs[x] - s);
        }
        if (i >= i0 && i < i0 + T && j >= j0 && j < j0 + T) {
          m = nanmax(m, fabs(r));
          F.f32[p] = (float)r;
        }
      }
      sf[t] = (float)r;
      su[t] = 0.0f;
    }
    __syncthreads();
    tile_down_rest(F, C, su, sf, Wd, is, js, i0, j0, T, axis);
    __syncthreads();
  }
  return m;
}

// Down phase of a coarser grid-wide level: e from 0 with right-hand side F.f32.
__device__ void down_tiles(const MgLevel& F, const MgLevel& C, int axis, unsigned char* smraw) {
  const int T = F.tile, H = kMgHalo, Wd = T + 2 * H;
  const int ntx = (F.nx - 1 + T - 1) / T, nty = (F.ny - 1 + T - 1) / T;
  float* su = reinterpret_cast<float*>(smraw);
  float* sf = su + Wd * Wd;
  for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
    const int i0 = 1 + (tile % ntx) * T, j0 = 1 + (tile / ntx) * T;
    const int is = i0 - H, js = j0 - H;
    for (int t = threadIdx.x; t < Wd * Wd; t += blockDim.x) {
      const int i = is + t % Wd, j = js + t / Wd;
      const bool in = i >= 1 && i <= F.nx - 1 && j >= 1 && j <= F.ny - 1;
      sf[t] = in ? F.f32[(int64_t)j * F.sy + i] : 0.0f;
      su[t] = 0.0f;
    }
    __syncthreads();
    tile_down_rest(F, C, su, sf, Wd, is, js, i0, j0, T, axis);
    __syncthreads();
  }
}

// Up phase: e = F.v32 + P (coarse correction e_c), one red-black sweep, then F.u32 = e on
// owned points (levels > 0) or Z += e in FP64 (level 0).
__device__ void up_tiles(const MgLevel& F, const MgLevel& C, const float* ec, bool level0,
                         double omega_dc, int axis, unsigned char* smraw) {
  const int T = F.tile, H = 2, Wd = T + 2 * H;
  const int ntx = (F.nx - 1 + T - 1) / T, nty = (F.ny - 1 + T - 1) / T;
  float* su = reinterpret_cast<float*>(smraw);
  float* sf = su + Wd * Wd;
  for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
    const int i0 = 1 + (tile % ntx) * T, j0 = 1 + (tile / ntx) * T;
    const int is = i0 - H, js = j0 - H;
    for (int t = threadIdx.x; t < Wd * Wd; t += blockDim.x) {
      const int i = is + t % Wd, j = js + t / Wd;
      float uu = 0.0f, ff = 0.0f;
      if (i >= 1 && i <= F.nx - 1 && j >= 1 && j <= F.ny - 1) {
        const int64_t p = (int64_t)j * F.sy + i;
        uu = F.v32[p] + prolong_at<2, float>(C, ec, i, j, 0);
        ff = F.f32[p];
      }
      su[t] = uu;
      sf[t] = ff;
    }
    __syncthreads();
    for (int h = 0; h < 2; ++h) {
      const int d = 1 - h;
      tile_half(F, su, sf, Wd, is, js, i0 - d, j0 - d, T + 2 * d, h & 1, axis);
      __syncthreads();
    }
    for (int t = threadIdx.x; t < T * T; t += blockDim.x) {
      const int i = i0 + t % T, j = j0 + t / T;
      if (i > F.nx - 1 || j > F.ny - 1) continue;
      const int64_t p = (int64_t)j * F.sy + i;
      const float e = su[(j - js) * Wd + (i - is)];
      if (level0)
        F.u[p] = fma(omega_dc, (double)e, F.u[p]);
      else
        F.u32[p] = e;
    }
    __syncthreads();
  }
}

// ---- the coarse CTA: levels lc..nlev-1 in shared memory -----------------------------

template <int DIM, typename R>
__device__ void cta_smooth(const MgLevel& L, R* u, const R* f, int sweeps, int axis) {
  for (int s = 0; s < sweeps; ++s) {
    rb_half<DIM, R>(L, u, f, 0, axis, threadIdx.x, blockDim.x);
    __syncthreads();
    rb_half<DIM, R>(L, u, f, 1, axis, threadIdx.x, blockDim.x);
    __syncthreads();
  }
}

// One V-cycle on levels l0..nlev-1 (l0's pre-smoothing skipped when presmoothed).
template <int DIM, typename R>
__device__ void cta_vcycle(const ImpArgs& a, R* sm, int l0, bool presmoothed) {
  const int axis = a.layer_axis;
  for (int l = l0; l < a.nlev - 1; ++l) {
    const MgLevel& L = a.lev[l];
    const MgLevel& C = a.lev[l + 1];
    R* u = sm + L.smem;
    if (!(presmoothed && l == l0)) cta_smooth<DIM, R>(L, u, u + L.points, a.nu1, axis);
    R* uc = sm + C.smem;
    restrict_pass<DIM, R>(L, nullptr, u, u + L.points, C, uc + C.points, uc, axis, threadIdx.x,
                          blockDim.x);
    __syncthreads();
  }
  {
    const MgLevel& L = a.lev[a.nlev - 1];
    R* u = sm + L.smem;
    cta_smooth<DIM, R>(L, u, u + L.points, a.coarse_sweeps, axis);
  }
  for (int l = a.nlev - 2; l >= l0; --l) {
    const MgLevel& L = a.lev[l];
    const MgLevel& C = a.lev[l + 1];
    R* u = sm + L.smem;
    prolong_pass<DIM, R>(C, sm + C.smem, L, u, threadIdx.x, blockDim.x);
    __syncthreads();
    cta_smooth<DIM, R>(L, u, u + L.points, a.nu2, axis);
  }
}

// Zero the shared levels, then copy level lc's rhs (and, if with_u, its start) from global.
template <typename R>
__device__ void cta_load(const ImpArgs& a, R* sm, bool with_u) {
  const MgLevel& L = a.lev[a.lc];
  const MgLevel& last = a.lev[a.nlev - 1];
  const int64_t total = last.smem + 2 * last.points;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) sm[t] = 0;
  __syncthreads();
  R* u = sm + L.smem;
  for (int64_t p = threadIdx.x; p < L.points; p += blockDim.x) {
    if constexpr (sizeof(R) == 8) {
      u[L.points + p] = L.f[p];
      if (with_u) u[p] = L.u[p];
    } else {
      u[L.points + p] = L.f32[p];
    }
  }
  __syncthreads();
}
template <typename R>
__device__ void cta_store(const ImpArgs& a, const R* sm) {
  const MgLevel& L = a.lev[a.lc];
  const R* u = sm + L.smem;
  for (int64_t p = threadIdx.x; p < L.points; p += blockDim.x) {
    if constexpr (sizeof(R) == 8)
      L.u[p] = u[p];
    else
      L.u32[p] = u[p];
  }
}

// ---- the step kernel ----------------------------------------------------------------

// W^{n+1} = Z - W^{n-1} (or Z / 2), filter sums, and the next solve's rhs and start; on the
// last step the epilogue V = C q + E V^k instead.
template <int DIM>
__device__ void update_phase(const ImpArgs& a, double* red) {
  const MgLevel& L = a.lev[0];
  const int64_t P = L.points;
  const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const int nf = a.nf;
  double bmax = 0.0;
  const uint32_t nxp = (uint32_t)L.nx + 1, nyp = (uint32_t)L.ny + 1;
  for (uint32_t t = t0; t < (uint32_t)P; t += stride) {
    const int i = (int)(t % nxp);
    const uint32_t rest = t / nxp;
    const int j = (int)(rest % nyp);
    const int k = DIM == 3 ? (int)(rest / nyp) : 0;
    const bool interior = i > 0 && i < L.nx && j > 0 && j < L.ny &&
                          (DIM == 2 || (k > 0 && k < L.nz));
    const int64_t p = t;
    if (!interior) {
      if (a.last)
        for (int m = 0; m < nf; ++m) a.vout[m * P + p] = 0.0;
      continue;
    }
    const double Z = L.u[p];
    const double wn = a.first ? 0.5 * Z : Z - a.Wp[p];
    if (a.last) {
      double qq[MFWH_MAX_NF], vk[MFWH_MAX_NF];
      for (int m = 0; m < nf; ++m) qq[m] = fma(a.wq[m], wn, a.q[m * P + p]);
      if (a.has_e)
        for (int m = 0; m < nf; ++m) vk[m] = a.vprev[m * P + p];
      for (int m = 0; m < nf; ++m) {
        double s = 0.0;
        for (int jj = 0; jj < nf; ++jj) s = fma(a.binv[m * MFWH_MAX_NF + jj], qq[jj], s);
        if (a.has_e)
          for (int jj = 0; jj < nf; ++jj) s = fma(a.emat[m * MFWH_MAX_NF + jj], vk[jj], s);
        a.vout[m * P + p] = a.subtract ? a.vsub[m * P + p] - s : s;
      }
      continue;
    }
    a.Wp[p] = wn;
    double rhs = 2.0 * wn;
    for (int m = 0; m < nf; ++m) {
      a.q[m * P + p] = fma(a.wq[m], wn, a.q[m * P + p]);
      if (a.fc[m] != 0.0) rhs = fma(-a.fc[m], a.f[m * P + p], rhs);
    }
    L.f[p] = rhs;
    // start of the next solve: Z^{n+1} = W^{n+2} + W^n ~ 2 W^{n+1} + (W^{n+1} - 2 W^n + W^{n-1})
    L.u[p] = 2.0 * wn + (Z - 2.0 * a.Wc[p]);
    bmax = nanmax(bmax, fabs(rhs));
  }
  if (!a.last) {
    bmax = block_max(bmax, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&a.st_next->bmax, bmax);
  }
}

template <int DIM>
__global__ void __launch_bounds__(kMgThreads, 2) k_imp_step(const ImpArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  __shared__ int s_flag;
  // A barrier of an earlier step timed out: return (the same decision for the whole block).
  if (threadIdx.x == 0) s_flag = *(volatile int*)a.err;
  __syncthreads();
  if (s_flag != 0) return;
  const int axis = a.layer_axis;
  const MgLevel& L0 = a.lev[0];
  const double bmax = load_nonneg(&a.st->bmax);
  const double thresh = a.tol * bmax;
  int c = 0;
  bool converged = false;
  if (DIM == 2 && a.lc > 0) {
    // FP64 defect correction with FP32 V-cycles (tiled grid-wide levels)
    for (;; ++c) {
      const double m = down0_tiles(L0, a.lev[1], axis, smraw);
      const double bm = block_max(m, red);
      if (threadIdx.x == 0) atomic_max_nonneg(&a.st->rmax[c], bm);
      grid_sync(a.bar, a.err, a.wait_ns);
      if (block_converged(a.st, c, thresh, &s_flag)) { converged = true; break; }
      if (c == a.max_cycles) break;
      for (int l = 1; l < a.lc; ++l) {
        down_tiles(a.lev[l], a.lev[l + 1], axis, smraw);
        grid_sync(a.bar, a.err, a.wait_ns);
      }
      if (blockIdx.x == 0) {
        float* sm = reinterpret_cast<float*>(smraw);
        cta_load<float>(a, sm, false);
        cta_vcycle<DIM, float>(a, sm, a.lc, false);
        cta_store<float>(a, sm);
      }
      grid_sync(a.bar, a.err, a.wait_ns);
      for (int l = a.lc - 1; l >= 0; --l) {
        up_tiles(a.lev[l], a.lev[l + 1], a.lev[l + 1].u32, l == 0, a.omega_dc, axis, smraw);
        grid_sync(a.bar, a.err, a.wait_ns);
      }
    }
  } else if (a.lc == 0) {
    // the whole hierarchy in this CTA (one block), FP64
    double* sm = reinterpret_cast<double*>(smraw);
    cta_load<double>(a, sm, true);
    double* u = sm + L0.smem;
    for (;; ++c) {
      cta_smooth<DIM, double>(L0, u, u + L0.points, a.nu1, axis);
      const double rm =
          block_max(residual_pass<DIM>(L0, u, u + L0.points, nullptr, axis, threadIdx.x,
                                       blockDim.x), red);
      if (rm <= thresh) { converged = true; break; }
      if (c == a.max_cycles) break;
      cta_vcycle<DIM, double>(a, sm, 0, true);
    }
    cta_store<double>(a, sm);
    __syncthreads();
  } else {
    // 3D: FP64 defect correction with grid-wide FP32 V-cycles (one barrier per phase)
    const uint32_t g0 = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    for (;; ++c) {
      const double rm = residual_to32<DIM>(L0, axis, g0, gs);
      const double bm = block_max(rm, red);
      if (threadIdx.x == 0) atomic_max_nonneg(&a.st->rmax[c], bm);
      grid_sync(a.bar, a.err, a.wait_ns);
      if (block_converged(a.st, c, thresh, &s_flag)) { converged = true; break; }
      if (c == a.max_cycles) break;
      for (int l = 0; l < a.lc; ++l) {
        const MgLevel& L = a.lev[l];
        for (int s = 0; s < a.nu1; ++s) {
          rb_half<DIM, float>(L, L.u32, L.f32, 0, axis, g0, gs);
          grid_sync(a.bar, a.err, a.wait_ns);
          rb_half<DIM, float>(L, L.u32, L.f32, 1, axis, g0, gs);
          grid_sync(a.bar, a.err, a.wait_ns);
        }
        residual_store<DIM, float>(L, L.u32, L.f32, L.v32, axis, g0, gs);
        grid_sync(a.bar, a.err, a.wait_ns);
        const MgLevel& C = a.lev[l + 1];
        restrict_pass<DIM, float>(L, L.v32, nullptr, nullptr, C, C.f32, C.u32, axis, g0, gs);
        grid_sync(a.bar, a.err, a.wait_ns);
      }
      if (blockIdx.x == 0) {
        float* sm = reinterpret_cast<float*>(smraw);
        cta_load<float>(a, sm, false);
        cta_vcycle<DIM, float>(a, sm, a.lc, false);
        cta_store<float>(a, sm);
      }
      grid_sync(a.bar, a.err, a.wait_ns);
      for (int l = a.lc - 1; l >= 0; --l) {
        const MgLevel& L = a.lev[l];
        prolong_pass<DIM, float>(a.lev[l + 1], a.lev[l + 1].u32, L, L.u32, g0, gs);
        grid_sync(a.bar, a.err, a.wait_ns);
        for (int s = 0; s < a.nu2; ++s) {
          rb_half<DIM, float>(L, L.u32, L.f32, 0, axis, g0, gs);
          grid_sync(a.bar, a.err, a.wait_ns);
          rb_half<DIM, float>(L, L.u32, L.f32, 1, axis, g0, gs);
          grid_sync(a.bar, a.err, a.wait_ns);
        }
      }
      add_correction<DIM>(L0, a.omega_dc, g0, gs);
      grid_sync(a.bar, a.err, a.wait_ns);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&a.counters->solves, 1ull);
    atomicAdd(&a.counters->cycles, (unsigned long long)c);
    if (!converged) atomicAdd(&a.counters->unconverged, 1ull);
  }
  update_phase<DIM>(a, red);
}

template <int DIM>
__global__ void k_imp_init(int nf, const Geom g, const double* __restrict__ v,
                           double* __restrict__ W0, double* __restrict__ q,
                           const double* __restrict__ f, double* __restrict__ Z,
                           double* __restrict__ rhs, MgState* st, const ImpInit a) {
  __shared__ double red[32];
  const int64_t P = g.points;
  double bmax = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % (g.nx + 1);
    const int64_t rest = p / (g.nx + 1);
    const int64_t j = rest % (g.ny + 1);
    const int64_t k = DIM == 3 ? rest / (g.ny + 1) : 0;
    const bool interior = i > 0 && i < g.nx && j > 0 && j < g.ny &&
                          (DIM == 2 || (k > 0 && k < g.nz));
    double w = 0.0;
    if (interior && v)
      for (int m = 0; m < nf; ++m) w += v[m * P + p];
    W0[p] = w;
    for (int m = 0; m < nf; ++m) q[m * P + p] = a.w0[m] * w;
    double r = 2.0 * w;
    if (interior)
      for (int m = 0; m < nf; ++m)
        if (a.fc0[m] != 0.0) r = fma(-a.fc0[m], f[m * P + p], r);
    rhs[p] = interior ? r : 0.0;
    Z[p] = 2.0 * w;
    bmax = nanmax(bmax, fabs(rhs[p]));
  }
  bmax = block_max(bmax, red);
  if (threadIdx.x == 0) atomic_max_nonneg(&st->bmax, bmax);
}

}  // namespace

bool mg_plan_levels(const Geom& g, const double* h, double c2_lo, double c2_hi, double dt,
                    MgLevel* lev, int* nlev, int* lc, int64_t* smem_elems) {
  int n[3] = {(int)g.nx, (int)g.ny, g.dim == 3 ? (int)g.nz : 0};
  double hh[3] = {h[0], h[1], g.dim == 3 ? h[2] : 1.0};
  int64_t split = g.layer_split;
  const double kap = 0.5 * dt * dt;   // alpha dt^2 with alpha = 1/2
  int L = 0;
  *lc = -1;
  for (;;) {
    MgLevel& v = lev[L];
    v = MgLevel{};
    v.nx = n[0];
    v.ny = n[1];
    v.nz = n[2];
    v.split = (int)std::min<int64_t>(split, (int64_t)1 << 30);
    if (L == 0) {
      v.sy = g.sy;
      v.sz = g.sz;
      v.points = g.points;
    } else {
      v.sy = n[0] + 1;
      v.sz = (int64_t)(n[0] + 1) * (n[1] + 1);
      v.points = v.sz * (g.dim == 3 ? n[2] + 1 : 1);
    }
    double slo = 0.0, shi = 0.0;
    for (int a = 0; a < 3; ++a) {
      const bool on = a < g.dim;
      v.a_lo[a] = on ? kap * c2_lo / (hh[a] * hh[a]) : 0.0;
      v.a_hi[a] = on ? kap * c2_hi / (hh[a] * hh[a]) : 0.0;
      v.a32_lo[a] = (float)v.a_lo[a];
      v.a32_hi[a] = (float)v.a_hi[a];
      slo += v.a_lo[a];
      shi += v.a_hi[a];
    }
    v.d_lo = 1.0 + 2.0 * slo;
    v.d_hi = 1.0 + 2.0 * shi;
    v.dinv_lo = 1.0 / v.d_lo;
    v.dinv_hi = 1.0 / v.d_hi;
    v.d32_lo = (float)v.d_lo;
    v.d32_hi = (float)v.d_hi;
    v.dinv32_lo = (float)v.dinv_lo;
    v.dinv32_hi = (float)v.dinv_hi;
    if (*lc < 0 && v.points <= kMgCoarsePoints) *lc = L;
    ++L;
    bool can = L < kMgMaxLevels;
    for (int a = 0; a < g.dim; ++a) can = can && n[a] % 2 == 0 && n[a] / 2 >= 2;
    if (!can) break;
    for (int a = 0; a < g.dim; ++a) {
      n[a] /= 2;
      hh[a] *= 2.0;
    }
    split = (split + 1) / 2;   // first coarse index J with 2J >= split
  }
  *nlev = L;
  if (*lc < 0) return false;
  int64_t off = 0;
  for (int l = *lc; l < L; ++l) {
    lev[l].smem = off;
    off += 2 * lev[l].points;
  }
  *smem_elems = off;
  return true;
}

void mg_set_order4(MgLevel* lev0, const double* h, double c2_lo, double c2_hi, double dt, int dim) {
  const double kap = 0.5 * dt * dt;
  double slo = 0.0, shi = 0.0;
  for (int a = 0; a < 3; ++a) {
    const bool on = a < dim;
    const double ih2 = on ? 1.0 / (h[a] * h[a]) : 0.0;
    lev0->a4_lo[a] = kap * c2_lo * ih2 * 16.0 / 12.0;
    lev0->a4_hi[a] = kap * c2_hi * ih2 * 16.0 / 12.0;
    lev0->b4_lo[a] = -kap * c2_lo * ih2 / 12.0;
    lev0->b4_hi[a] = -kap * c2_hi * ih2 / 12.0;
    slo += kap * c2_lo * ih2 * 30.0 / 12.0;
    shi += kap * c2_hi * ih2 * 30.0 / 12.0;
  }
  lev0->d4_lo = 1.0 + slo;
  lev0->d4_hi = 1.0 + shi;
  lev0->order4 = 1;
}

cudaError_t mg_launch_config(int dim, int lc, int64_t smem_elems, MgLevel* lev, int* grid,
                             size_t* smem) {
  // The attribute is per kernel, shared by every handle: it is always set to the same bound
  // (above what any hierarchy needs), and each handle launches with its own size below it.
  constexpr int kSmemBound = 120 * 1024;
  const bool mixed = mg_mixed(dim, lc);
  int64_t need = smem_elems * (mixed ? 4 : 8);
  if (mixed && dim == 2) need = std::max(need, mg_tile_smem_bytes(kMgTileMax));
  *smem = (size_t)need;
  if (*smem > (size_t)kSmemBound) return cudaErrorInvalidValue;
  const void* fn = dim == 3 ? (const void*)k_imp_step<3> : (const void*)k_imp_step<2>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBound);
  if (e != cudaSuccess) return e;
  if (lc == 0) {
    *grid = 1;
    return cudaSuccess;
  }
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kMgThreads, *smem)) != cudaSuccess)
    return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  *grid = sms * occ;
  if (mixed && dim == 2) {
    for (int l = 0; l < lc; ++l) {
      int best = kMgTileMax;
      int64_t best_cost = -1;
      for (int T = kMgTileMax; T >= 8; T /= 2) {
        const int64_t tiles = (int64_t)((lev[l].nx - 1 + T - 1) / T) * ((lev[l].ny - 1 + T - 1) / T);
        const int64_t rounds = (tiles + *grid - 1) / *grid;
        const int64_t cost = rounds * (T + 2 * kMgHalo) * (T + 2 * kMgHalo);
        if (best_cost < 0 || cost < best_cost) {
          best_cost = cost;
          best = T;
        }
      }
      lev[l].tile = best;
    }
  }
  return cudaSuccess;
}

void launch_imp_init(int nf, const Geom& g, const double* v, double* W0, double* q,
                     const double* f, double* Z, double* rhs, MgState* st, const ImpInit& a,
                     cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((g.points + 255) / 256, 8 * 152);
  if (g.dim == 3)
    k_imp_init<3><<<(unsigned)blocks, 256, 0, s>>>(nf, g, v, W0, q, f, Z, rhs, st, a);
  else
    k_imp_init<2><<<(unsigned)blocks, 256, 0, s>>>(nf, g, v, W0, q, f, Z, rhs, st, a);
}

cudaError_t launch_imp_step(int dim, const ImpArgs& a, int grid, size_t smem, cudaStream_t st) {
  void* args[] = {(void*)&a};
  const void* fn = dim == 3 ? (const void*)k_imp_step<3> : (const void*)k_imp_step<2>;
  if (grid == 1) return cudaLaunchKernel(fn, dim3(1), dim3(kMgThreads), args, smem, st);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kMgThreads), args, smem, st);
}

}  // namespace mfwh

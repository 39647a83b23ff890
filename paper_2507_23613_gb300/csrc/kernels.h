// Device-side launchers of libmfwh (implemented in wave.cu and krylov.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "check.cuh"
#include "mfwh.h"

namespace mfwh {

// Grid geometry as the kernels see it.  Points are indexed
// p = k * sz + j * sy + i with 0 <= i <= nx, 0 <= j <= ny, 0 <= k <= nz.
struct Geom {
  int64_t nx, ny, nz;        // cells per axis (nz = 0 in 2D)
  int64_t sy, sz;            // strides of j and k
  int64_t points;            // points per grid function (stride between frequencies)
  int dim;                   // 2 or 3
  int layer_axis;            // axis whose index selects the c^2 layer
  int64_t layer_split;       // indices >= layer_split use the upper-layer coefficients
  int order;                 // order of L_{ph}: 2 or 4 (0 reads as 2)
  int64_t syw, szw;          // strides of j and k in the FP32 wave-level arrays W and D (2D
                             // FP32 handles pad rows to 32 floats for tensor copies; else sy, sz)
  const double* c2f;         // c^2 per point [points] (MFWH_C_FIELD), else null; with a field
                             // the layer coefficients are those of c = 1 (lower layer only)
  BoundsFault* fault;        // device fault record of the index-checked build (check.cuh), or
                             // null; unused in the normal build
};

// Leapfrog update at one point, written as
//   W^{n+1} = A0 W^n + a_prev W^{n-1} + Ax (W_e + W_w) + Ay (W_n + W_s) + Az (W_u + W_d)
//             - sum_m fneg_m f_m,
// with A0 = a_cur - 2 kappa c^2 sum_i 1/h_i^2, A_i = kappa c^2 / h_i^2,
// (a_cur, a_prev, kappa) = (2, -1, dt^2) for a regular step (eq. WaveSchemeA) and
// (1, 0, dt^2/2) for the first step (eq. implicitFirstStep with alpha = 0).
// Fourth order adds the second neighbours: + Bx (W_ee + W_ww) + By (...) + Bz (...), with
// A_i = (4/3) kappa c^2 / h_i^2, B_i = -kappa c^2 / (12 h_i^2), A0 = a_cur - (5/2) kappa c^2
// sum_i 1/h_i^2; a ghost value beyond the boundary is minus the point next to it.
struct LayerCoef {
  double A0, Ax, Ay, Az;
  double Bx, By, Bz;
};

struct StepHost {
  LayerCoef lo, hi;                 // coefficients below / above the layer split
  double a_cur;                     // 2 (regular step) or 1 (first step): with a c^2 field the
                                    // update is a_cur W^n - a_prev W^{n-1} + c_j^2 (L - a_cur W^n),
                                    // L the sum over lo's terms (coefficients of c = 1)
  int first;                        // 1 on the first step: no W^{n-1} term
  int forced;                       // 0: homogeneous map S (no forcing)
  double fc[MFWH_MAX_NF];           // kappa cos(omega~_m t^n)
  double wq[MFWH_MAX_NF];           // w_{n+1,m}: filter weight of the new level
  // epilogue (last step only): V^{k+1} = C q + E V^k, then v_out = V^{k+1} or v_sub - V^{k+1}.
  // Implicit filter: C = B^{-1}, E = 0.  Explicit filter: C = diag(B)^{-1},
  // E = -diag(B)^{-1} (B - diag(B)).  Matrices row-major with leading dimension MFWH_MAX_NF.
  int subtract;
  double binv[MFWH_MAX_NF * MFWH_MAX_NF];   // C
  double emat[MFWH_MAX_NF * MFWH_MAX_NF];   // E
  int has_e;                                // E != 0 (applied when V^k is given)
  const double* vprev;                      // V^k (device), or null for V^k = 0
};

// Arguments of one temporally blocked launch (wave_tb.cu).
struct TBHost {
  LayerCoef reg_lo, reg_hi, first_lo, first_hi;
  const double* wq_table;    // device [(N_t + 1) * nf] w_{n,m}
  const double* cos_table;   // device [(N_t + 1) * nf] cos(omega~_m t^n)
  const double* wq_host;     // host copies of the two tables (the per-launch coefficients of
  const double* cos_host;    // depths up to 4 travel as kernel parameters)
  double dt2, half_dt2;
  int n0, steps, depth;      // first level index, steps in this launch, template depth (2, 3, 4, 8)
  int shape;                 // tile 0-5 (wave_tb_kernels.cuh): 0 = 32 x 64, 1 = 32 x 32, 2 = 32 x 48 points (32 x 32
                             // above 8 frequencies)
  int forced, last, subtract;
  double binv[MFWH_MAX_NF * MFWH_MAX_NF];   // epilogue as in StepHost
  double emat[MFWH_MAX_NF * MFWH_MAX_NF];
  int has_e;
  const double* vprev;
};
// Up to `depth` leapfrog+filter steps of a 2D grid in one launch: reads (Wc_in, Wp_in)
// (Wp_in may be null: W^{-1} = 0 before the first step), writes (Wc_out, Wp_out) and q, or on
// the last launch v_out = B^{-1} q (or v_sub - B^{-1} q).  Output buffers must not alias inputs.
void launch_tb2d(int nf, const Geom& g, const double* Wc_in, const double* Wp_in, double* Wc_out,
                 double* Wp_out, const double* f, double* q, double* vout, const double* vsub,
                 const TBHost& h, cudaStream_t st);

// ---- FP32 path with compensated filter sums (wave32.cu) ----------------------------
// Increment form: D' = D + kappa c^2 Delta_h W - sum_m fc_m f_m, W' = W + D', with
// kappa c^2 / h_i^2 per layer in Coef32.  Filter sums are Kahan pairs (qs, qc), q = qs - qc.
struct Coef32 {
  float Ax, Ay, Az;
};
struct Step32Host {
  Coef32 lo, hi;
  float fc[MFWH_MAX_NF];   // kappa_n cos(omega~_m t^n), rounded to FP32
  float wq[MFWH_MAX_NF];   // w_{n+1,m}, rounded to FP32
  int forced;
};
struct TB32Host {
  Coef32 reg_lo, reg_hi, first_lo, first_hi;
  const float* wq;         // device [(N_t + 1) * nf]
  const float* fc;         // device [N_t * nf]
  const double* binv;      // host [MFWH_MAX_NF * MFWH_MAX_NF], row-major, leading dim 16 (C)
  const double* emat;      // host, same layout (E of the explicit filter)
  int has_e;
  const double* vprev;     // device V^k, or null
  int n0, steps, depth, shape, forced, last;
  int acc;                 // 0: Kahan update every step; 1: per-launch partial sums folded
  int* err;                // device flag set to 1 when a tile's tensor copy does not complete
};
// W^0 = fl32(sum_m v_m) (0 on the boundary), qs_m = w0_m W^0, qc_m = 0.
void launch_init32(int nf, const Geom& g, const double* v, float* W0, float* qs, float* qc,
                   const float* w0, cudaStream_t st);
// One step: W_out = W + D', D_out = D' (D_in == nullptr: D = 0; D_out may equal D_in).
void launch_step32(int nf, const Geom& g, const float* W, const float* D_in, float* W_out,
                   float* D_out, const float* f, float* qs, float* qc, const Step32Host& h,
                   cudaStream_t st);
// Last step fused with V = B^{-1} q in FP64 (or v_sub - that); boundary of v_out = 0.
void launch_last32(int nf, const Geom& g, const float* W, const float* D, const float* f,
                   const float* qs, const float* qc, double* vout, const double* vsub,
                   const Step32Host& h, const StepHost& epi, cudaStream_t st);
// Up to h.depth (4, 8 or 16) steps of a 2D grid per launch; outputs must not alias inputs.
void launch_tb2d32(int nf, const Geom& g, const float* W_in, const float* D_in, float* W_out,
                   float* D_out, const float* f, float* qs, float* qc, double* vout,
                   const double* vsub, const TB32Host& h, cudaStream_t st);
// Up to h.depth (2 or 4) steps of a 3D grid per launch (second-order operator); outputs must
// not alias inputs.  Same arguments as launch_tb2d32 (tile shape ignored).
void launch_tb3d32(int nf, const Geom& g, const float* W_in, const float* D_in, float* W_out,
                   float* D_out, const float* f, float* qs, float* qc, double* vout,
                   const double* vsub, const TB32Host& h, cudaStream_t st);
void launch_to_float(const double* x, float* y, int64_t n, cudaStream_t st);

// In launch_init, launch_step, launch_last and launch_tb2d, q holds the N_f filter sums
// [N_f][points], each as a float pair (hi, lo) in the 8 bytes of a double (fpair.cuh); only
// these kernels read or write it.
// W^0 = sum_m v_m (0 on the boundary; v == nullptr gives W^0 = 0) and q_m = w0_m W^0.
void launch_init(int nf, const Geom& g, const double* v, double* W0, double* q, const double* w0,
                 cudaStream_t st);
// One leapfrog step n -> n+1 fused with q_m += w_{n+1,m} W^{n+1}.  W^{n+1} overwrites Wp.
void launch_step(int nf, const Geom& g, const double* Wc, double* Wp, const double* f, double* q,
                 const StepHost& a, cudaStream_t st);
// Last step fused with the filter solve: v_out = B^{-1}(q + w_{N_t} W^{N_t}) (or v_sub - that).
void launch_last(int nf, const Geom& g, const double* Wc, const double* Wp, const double* f,
                 const double* q, double* vout, const double* vsub, const StepHost& a,
                 cudaStream_t st);
// Per-frequency max_int |f_m - (c^2 Delta_h + omega_m^2) v_m| and max_int |f_m|, reduced over the
// grid into out[2 * nf] (device): out[m] = residual max, out[nf + m] = forcing max.
// partial: device scratch of at least residual_partial_size(nf) doubles.
void launch_residual(int nf, const Geom& g, const double* v, const double* f, const double* omega2,
                     double c2_lo, double c2_hi, const double* inv_h2, double* partial, double* out,
                     cudaStream_t st);
int64_t residual_partial_size(int nf);
// Blocks of the residual kernel: residual_partial_size(nf) = kResidualBlocks * 2 * nf.
constexpr int kResidualBlocks = 4 * 152;
// Defect field R_m = f_m - (c^2 Delta_h + omega_m^2) v_m (0 on the boundary), [nf][points].
void launch_residual_field(int nf, const Geom& g, const double* v, const double* f,
                           const double* omega2, double c2_lo, double c2_hi, const double* inv_h2,
                           double* R, cudaStream_t st);

// ---- implicit trapezoidal time stepping with geometric multigrid (implicit.cu), FP64 ----
// Step n of eq. WaveScheme with (alpha, beta) = (1/2, 0) is A Z = rhs, A = I - (dt^2/2) L_h,
// rhs = 2 W^n - dt^2 F^n, followed by W^{n+1} = Z - W^{n-1} (W^1 = Z / 2: eq.
// implicitFirstStep).  A is solved by V-cycles of red-black Gauss-Seidel, full-weighting
// restriction, multilinear prolongation and rediscretised coarse operators, inside one
// persistent (cooperative) launch per step that decides convergence on the device.
constexpr int kMgMaxLevels = 16;
constexpr int kMgMaxCycles = 60;
constexpr int64_t kMgCoarsePoints = 5000;   // levels this small run in one CTA's shared memory
constexpr int kMgThreads = 512;

struct MgLevel {
  int nx, ny, nz;             // cells per axis (nz = 0 in 2D)
  int split;                  // first index along the layer axis in the upper layer
  int64_t sy, sz, points;     // strides and points of the level's arrays
  double a_lo[3], a_hi[3];    // (dt^2/2) c^2 / h_i^2 below / above the layer split
  double d_lo, d_hi;          // diagonal of A: 1 + 2 sum_i a_i
  double dinv_lo, dinv_hi;    // 1 / diagonal
  float a32_lo[3], a32_hi[3];   // the same coefficients rounded to FP32
  // Level 0 with the fourth-order operator (order4 = 1): A_4 = I - (dt^2/2) c^2 Delta_4h with
  // first-neighbour weights a4 = (4/3)(dt^2/2) c^2 / h_i^2, second-neighbour weights
  // b4 = -(dt^2/2) c^2 / (12 h_i^2) and diagonal d4 = 1 + (5/2)(dt^2/2) c^2 sum_i 1/h_i^2;
  // the ghost value beyond the boundary is minus the point next to it.
  int order4;
  double a4_lo[3], a4_hi[3], b4_lo[3], b4_hi[3], d4_lo, d4_hi;
  float d32_lo, d32_hi, dinv32_lo, dinv32_hi;
  double* u;                  // FP64 arrays: level 0's iterate Z and right-hand side (and the
  double* f;                  // levels of a one-CTA hierarchy, in shared memory)
  float* u32;                 // FP32 arrays: the correction (2D: after the up phase), the 2D
  float* v32;                 // correction after the down phase or the 3D residual of the
  float* f32;                 // correction equation, and the level's right-hand side (level 0:
                              // the FP64 residual rhs - A Z rounded to FP32)
  int tile;                   // grid-wide 2D levels: edge of the square tile of owned points
  int64_t smem;               // coarse levels: offset in elements of u in shared memory (f follows)
};
// A 2D hierarchy with grid-wide levels is solved by defect correction: every cycle forms
// r = rhs - A Z in FP64, applies one FP32 V-cycle to A e = r from e = 0, and adds e to Z in FP64.
// Its grid-wide levels run tiled phases: a CTA loads a tile plus a halo of kMgHalo points into
// shared memory, applies the two pre-smoothing sweeps there (each half-sweep shrinks the valid
// region by one point) and restricts the residual of its tile; the up phase loads a tile plus
// 2 points, adds the prolonged correction and applies the post-smoothing sweep.
constexpr int kMgTileMax = 64;
constexpr int kMgHalo = 6;     // 2 nu1 + 2 with nu1 = 2
// Shared memory in bytes of the tiled phases with tile edge T: level 0's down phase holds Z
// (FP64, two more rings for the fourth-order residual) and e, r (FP32); the other phases hold
// u and f (FP32).
inline int64_t mg_tile_smem_bytes(int T) {
  const int64_t w = T + 2 * kMgHalo;
  return (w + 4) * (w + 4) * 8 + 2 * w * w * 4;
}

// Convergence test of one step solve: bits of non-negative doubles, so that atomicMax orders them.
struct MgState {
  unsigned long long bmax;                     // max |rhs|
  unsigned long long rmax[kMgMaxCycles + 1];   // max |rhs - A Z| at each test
};
struct MgCounters {
  unsigned long long solves, cycles, unconverged;
};

struct ImpArgs {
  MgLevel lev[kMgMaxLevels];
  int nlev, lc;               // levels; first level solved by the coarse CTA (0: all of them)
  int layer_axis, nf;
  int nu1, nu2, coarse_sweeps, max_cycles;
  double tol;
  double omega_dc;            // Z += omega_dc e: 1 (second order), 6/7 (fourth order, where the
                              // second-order V-cycle preconditions A_4: eigenvalues in [1, 4/3])
  MgState* st;                // this step's test state
  MgState* st_next;           // next step's (receives max |rhs|), null on the last step
  MgCounters* counters;
  unsigned* bar;              // grid barrier: [0] arrivals, [1] generation
  int* err;                   // set to 2 when a barrier wait times out
  unsigned long long wait_ns; // limit of one barrier wait in nanoseconds
  double* Wp;                 // in: W^{n-1}, out: W^{n+1}
  const double* Wc;           // W^n (start of the next solve: 2 W^{n+1} + Z - 2 W^n)
  double* q;                  // filter sums [nf][points]
  const double* f;            // forcing [nf][points]
  int first, last;            // n == 0; n + 1 == N_t (epilogue instead of the next rhs)
  double wq[MFWH_MAX_NF];     // w_{n+1,m}
  double fc[MFWH_MAX_NF];     // dt^2 cos(omega~_m t^{n+1}) cos(omega~_m dt); 0: homogeneous
  double* vout;               // epilogue as in StepHost
  const double* vsub;
  int subtract, has_e;
  const double* vprev;
  double binv[MFWH_MAX_NF * MFWH_MAX_NF];
  double emat[MFWH_MAX_NF * MFWH_MAX_NF];
};
struct ImpInit {
  double w0[MFWH_MAX_NF];     // w_{0,m}
  double fc0[MFWH_MAX_NF];    // dt^2 cos(omega~_m dt) (t^0 = 0); 0: homogeneous
};
// Level geometry and coefficients for A = I - (dt^2/2) c^2 Delta_h on the grid g (level 0 uses
// g's strides).  Coarsens while every n_i is even and n_i / 2 >= 2.  lc = first level with at
// most kMgCoarsePoints points; returns false if no level is that small.  smem_elems: shared
// memory of the coarse CTA in elements (u and f of levels lc..nlev-1).
bool mg_plan_levels(const Geom& g, const double* h, double c2_lo, double c2_hi, double dt,
                    MgLevel* lev, int* nlev, int* lc, int64_t* smem_elems);
// Fourth-order coefficients of level 0 (sets lev0.order4).
void mg_set_order4(MgLevel* lev0, const double* h, double c2_lo, double c2_hi, double dt, int dim);
// Blocks of the step kernel's cooperative launch (1 when lc == 0) and its shared memory; in
// 2D it also picks each grid-wide level's tile edge (64, 32, 16 or 8: fewest rounds of tiles
// over the blocks times the tile's loaded points) and grows the shared memory to hold it.
cudaError_t mg_launch_config(int dim, int lc, int64_t smem_elems, MgLevel* lev, int* grid,
                             size_t* smem);
// A hierarchy with grid-wide levels (lc > 0) runs the FP32 defect-correction cycles (tiled
// phases in 2D, grid-wide phases in 3D).
inline bool mg_mixed(int dim, int lc) { return (dim == 2 || dim == 3) && lc > 0; }
// W^0 = sum_m v_m, q_m = w_{0,m} W^0, Z = 2 W^0, rhs = 2 W^0 - dt^2 F^0 (boundary 0) and
// st->bmax = max |rhs|.  v may be null (W^0 = 0).
void launch_imp_init(int nf, const Geom& g, const double* v, double* W0, double* q,
                     const double* f, double* Z, double* rhs, MgState* st, const ImpInit& a,
                     cudaStream_t st_);
// One implicit step (multigrid solve and the update of W, q and the next rhs, or the epilogue).
cudaError_t launch_imp_step(int dim, const ImpArgs& a, int grid, size_t smem, cudaStream_t st);

// ---- Krylov vector kernels (krylov.cu), FP64 -------------------------------------
constexpr int kMaxDots = 32;       // vectors handled by one multi-dot / multi-axpy launch
constexpr int kMaxKrylov = 1024;   // largest Krylov basis (restart length + 1)
// out[i] = <V_i, w> for i < k, V_i = V + i * ldv (device), N entries, in chunks of
// kMaxDots vectors per launch; partial: device scratch of at least dot_partial_size()
// doubles; out: device [k].  k <= kMaxKrylov.
void launch_multidot(const double* V, int64_t ldv, int k, const double* w, int64_t N,
                     double* partial, double* out, cudaStream_t st);
int64_t dot_partial_size();
// number of kernel launches launch_multidot issues for k vectors
int multidot_launches(int k);
// w -= sum_i coef[i] V_i (coef host, k <= kMaxKrylov), kMaxDots vectors per pass over w.
void launch_multi_axpy(double* w, const double* V, int64_t ldv, int k, const double* coef,
                       int64_t N, cudaStream_t st);
int multi_axpy_launches(int k);
// y = a x + b y
void launch_axpby(double* y, double a, const double* x, double b, int64_t N, cudaStream_t st);

// ---- warm start (cnn.cu) -----------------------------------------------------------
// Training pairs of a solved 2D problem: x [nf][2][H][W], t [nf][H][W] (t may be null with
// v null); scale: device scratch of 2 nf doubles (max |f_m|, max |V_m|).
mfwh_status cnn_ws_data(const double* f, const double* v, const double* omega, int nf, int H,
                        int W, double omega_scale, float* x, float* t, double* scale,
                        cudaStream_t st);
// Solution shapes [nf][H][W] (device) from the network; boundary values 0.  Synchronous.
mfwh_status cnn_ws_predict(mfwh_cnn_t c, const double* f, const double* omega, int nf, int H,
                           int W, double omega_scale, double* v, cudaStream_t st);

}  // namespace mfwh

// C ABI of libmfwh: handle life cycle, the MFWH map Pi, the fixed-point
// iteration (Algorithm 1), GMRES on A = I - S (Section "Acceleration by Krylov
// methods") and the Helmholtz residual (eq. errorAndResid).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "kernels.h"

namespace mfwh {

static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }

}  // namespace mfwh

using namespace mfwh;

namespace {

constexpr int kEventPool = 2048;    // event slots: two per timed Pi application
constexpr int kMaxRestart = kMaxKrylov - 1;

mfwh_status cuda_fail(cudaError_t e, const char* what) {
  std::ostringstream os;
  os << what << ": " << cudaGetErrorName(e) << " (" << cudaGetErrorString(e) << ")";
  set_error(os.str());
  return e == cudaErrorMemoryAllocation ? MFWH_ERR_NOMEM : MFWH_ERR_CUDA;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
  } while (0)

mfwh_status fail(mfwh_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

// NVTX range over a scope (create, each application of the map, each Arnoldi step, residual
// checks, batch rounds): visible to profilers that record NVTX, a no-op otherwise.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Largest value of a problem's c^2 field (MFWH_C_FIELD), read from host or device memory, for
// the time step of plan_problem: NaN when a value is not finite or not > 0 (plan_problem then
// rejects the problem); 0 for the other c modes and for grids plan_problem rejects anyway.
mfwh_status field_max(const mfwh_problem* p, double* mx) {
  *mx = 0.0;
  if (!p || p->c_mode != MFWH_C_FIELD || !p->c2_field || (p->dim != 2 && p->dim != 3))
    return MFWH_OK;
  int64_t points = 1;
  for (int a = 0; a < p->dim; ++a) {
    if (p->n[a] < 2 || p->n[a] > (1 << 20)) return MFWH_OK;
    points *= p->n[a] + 1;
  }
  if (points > ((int64_t)1 << 34)) return MFWH_OK;
  std::vector<double> copy;
  const double* c2 = p->c2_field;
  if (is_device_ptr(c2)) {
    copy.resize((size_t)points);
    CK(cudaMemcpy(copy.data(), c2, sizeof(double) * points, cudaMemcpyDefault));
    c2 = copy.data();
  }
  double m = 0.0;
  for (int64_t i = 0; i < points; ++i) {
    const double x = c2[i];
    if (!(x > 0.0) || !std::isfinite(x)) {
      *mx = std::nan("");
      return MFWH_OK;
    }
    m = std::max(m, x);
  }
  *mx = m;
  return MFWH_OK;
}

// plan_problem with the c^2 field's maximum read first.
mfwh_status plan_with_field(const mfwh_problem* p, Plan* P) {
  double c2m = 0.0;
  mfwh_status st = field_max(p, &c2m);
  if (st != MFWH_OK) return st;
  return plan_problem(p, P, c2m);
}

}  // namespace

struct mfwh_handle_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  Plan plan;
  Geom geom{};
  int nf = 0;
  int64_t P = 0, N = 0;            // points per grid function, nf * points
  int64_t PW = 0;                   // entries of one FP32 wave-level array (padded rows in 2D)
  int* d_err = nullptr;             // device flag of the blocked FP32 kernel (tensor copy timeout)
  double inv_h2[3] = {0, 0, 0};
  double omega2[MFWH_MAX_NF] = {};
  double* f = nullptr;              // forcing [nf][P]
  double* c2f = nullptr;            // c^2 per point [P] (MFWH_C_FIELD)
  BoundsFault* fault = nullptr;     // index-checked build: the kernels' fault record
  bool use32 = false;               // wave solves in FP32 (the FP32 precisions)
  // FP64 wave solves (all of an FP64 handle's; the FP64 residuals and products of an FP32
  // handle): steps per launch (1 = one step per launch) and blocked-kernel tile
  int depth64 = 1, shape64 = 0;
  // CUDA-graph mode (mfwh_set_graphs): each variant of the wave solve is captured once on the
  // staging buffers g_in / g_out and replayed as one graph launch.
  bool graphs = false;
  cudaStream_t gstream = nullptr;   // private stream the graphs are captured and replayed on
  cudaEvent_t gev[2] = {};          // orders gstream after / before the caller's stream
  double* g_in = nullptr;
  double* g_out = nullptr;
  cudaGraphExec_t gexec[16] = {};
  int64_t g_steps[16] = {}, g_total[16] = {};
  int tune_steps = 0;               // autotuner only: stop the wave solve after this many steps
  double* vec_r = nullptr;          // outer residual of the refined solve [nf][P] (lazy)
  double* vec_e = nullptr;          // correction of the refined solve [nf][P] (lazy)
  double* Wa = nullptr;             // wave levels (ping-pong)
  double* Wb = nullptr;
  double* Wc2 = nullptr;            // second pair of wave levels (temporal blocking:
  double* Wp2 = nullptr;            // a launch reads one pair and writes the other)
  double* d_wq = nullptr;           // [(N_t + 1) * nf] filter weights w_{n,m}
  double* d_cos = nullptr;          // [(N_t + 1) * nf] cos(omega~_m t^n)
  double* q = nullptr;              // filter accumulators [nf][P]
  double* res_partial = nullptr;
  double* res_out = nullptr;
  double* dot_partial = nullptr;
  double* dot_out = nullptr;
  double* vec_b = nullptr;          // GMRES right-hand side Pi(0)
  double* vec_x = nullptr;          // iterate when the caller's buffer is on the host
  double* basis = nullptr;          // Krylov basis [(restart+1)][N]
  int basis_vectors = 0;
  double* pinned = nullptr;         // host pinned scratch (kPinned doubles)
  std::vector<cudaEvent_t> ev;      // event pool: pairs around the step loop of each Pi
  int ev_used = 0;
  double last_step_ms = 0.0;
  int64_t step_launches = 0;
  int64_t total_launches = 0;
  StepHost sh;                      // per-step kernel arguments (reused)
  // FP32 paths (precision MFWH_PREC_FP32_KAHAN or MFWH_PREC_FP32_BLOCKSUM)
  float* f32 = nullptr;             // forcing rounded to FP32 [nf][P]
  float* W32[4] = {};               // (W, D) pairs: W32[0], W32[1] and W32[2], W32[3]
  float* qs = nullptr;              // Kahan sums [nf][P]
  float* qc = nullptr;              // Kahan compensations [nf][P]
  float* wq32 = nullptr;            // device [(N_t + 1) * nf] w_{n,m}
  float* fc32 = nullptr;            // device [N_t * nf] kappa_n cos(omega~_m t^n)
  std::vector<float> wq32_h, fc32_h;
  // implicit time stepping (MFWH_TIME_IMPLICIT)
  bool implicit = false;
  ImpArgs* imp = nullptr;           // step-kernel arguments (levels filled at create)
  int imp_grid = 0;                 // blocks of the step kernel (1: one-CTA hierarchy)
  size_t imp_smem = 0;              // its dynamic shared memory
  double* imp_mem = nullptr;        // multigrid level arrays
  MgState* d_mgstate = nullptr;     // [N_t] per-step convergence state
  unsigned* d_bar = nullptr;        // grid barrier of the step kernel
  MgCounters* d_mgc = nullptr;      // multigrid statistics
  double wait_s = 2.0;              // limit of one grid-barrier wait of the step kernel (s)
  std::vector<double> imp_fc;       // [(N_t + 1) * nf] dt^2 cos(omega~_m t^n) cos(omega~_m dt)
};

namespace {

constexpr int kPinned = kMaxKrylov + 64;

void reset_timing(mfwh_handle_t h) {
  h->ev_used = 0;
  h->last_step_ms = 0.0;
  h->step_launches = 0;
  h->total_launches = 0;
}

mfwh_status collect_timing(mfwh_handle_t h) {
  if (h->d_err) {   // a bounded wait of a wave kernel ran out (1: FP32 tile copy; 2: barrier)
    CK(cudaMemcpyAsync(h->pinned, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int flag = 0;
    std::memcpy(&flag, h->pinned, sizeof(int));
    if (flag) {
      CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
      if (h->d_bar) CK(cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream));
      CK(cudaStreamSynchronize(h->stream));
      return fail(MFWH_ERR_TIMEOUT,
                  flag == 2 ? "implicit step kernel: a grid barrier wait timed out"
                            : "FP32 wave kernel: a tile's tensor copy did not complete");
    }
  }
  double ms = 0.0;
  for (int i = 0; i + 1 < h->ev_used; i += 2) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, h->ev[i], h->ev[i + 1]));
    ms += t;
  }
  h->last_step_ms = ms;
  return MFWH_OK;
}

void layer_coef(const mfwh_handle_t h, double c2, double a_cur, double kappa, LayerCoef* L) {
  const double k = kappa * c2;
  if (h->plan.order == 4) {
    const double s = k * (h->inv_h2[0] + h->inv_h2[1] + h->inv_h2[2]);
    L->Ax = (4.0 / 3.0) * k * h->inv_h2[0];
    L->Ay = (4.0 / 3.0) * k * h->inv_h2[1];
    L->Az = (4.0 / 3.0) * k * h->inv_h2[2];
    L->Bx = -k * h->inv_h2[0] / 12.0;
    L->By = -k * h->inv_h2[1] / 12.0;
    L->Bz = -k * h->inv_h2[2] / 12.0;
    L->A0 = a_cur - 2.5 * s;
    return;
  }
  L->Ax = k * h->inv_h2[0];
  L->Ay = k * h->inv_h2[1];
  L->Az = k * h->inv_h2[2];
  L->Bx = L->By = L->Bz = 0.0;
  L->A0 = a_cur - 2.0 * (L->Ax + L->Ay + L->Az);
}

// FP32 increment coefficients: kappa c^2 / h_i^2, divided by 12 for the fourth-order
// operator (whose kernels form 16 d1 - d2 from first and second neighbour differences).
void layer_coef32(const mfwh_handle_t h, double c2, double kappa, Coef32* L) {
  const double k = kappa * c2 / (h->plan.order == 4 ? 12.0 : 1.0);
  L->Ax = (float)(k * h->inv_h2[0]);
  L->Ay = (float)(k * h->inv_h2[1]);
  L->Az = (float)(k * h->inv_h2[2]);
}

// FP32 wave solve (increment form, Kahan filter sums), FP64 filter solve.
mfwh_status apply_pi32(mfwh_handle_t h, const double* vin, double* vout, int forced,
                       const double* vsub) {
  const Plan& P = h->plan;
  const int nf = h->nf;
  const int n_t = P.s.n_t;
  const int n_run = h->tune_steps > 0 ? std::min(h->tune_steps, n_t) : n_t;
  const double dt = P.s.dt;
  cudaStream_t st = h->stream;
  float w0[MFWH_MAX_NF];
  for (int m = 0; m < nf; ++m) w0[m] = h->wq32_h[m];
  launch_init32(nf, h->geom, vin, h->W32[0], h->qs, h->qc, w0, st);
  h->total_launches += 1;
  const bool timed = h->ev_used + 2 <= (int)h->ev.size();
  if (timed) CK(cudaEventRecord(h->ev[h->ev_used], st));
  Coef32 reg_lo, reg_hi, first_lo, first_hi;
  layer_coef32(h, P.c2_lo, dt * dt, &reg_lo);
  layer_coef32(h, P.c2_hi, dt * dt, &reg_hi);
  layer_coef32(h, P.c2_lo, 0.5 * dt * dt, &first_lo);
  layer_coef32(h, P.c2_hi, 0.5 * dt * dt, &first_hi);
  int launches = 0;
  if (P.time_block > 1) {
    TB32Host a;
    a.reg_lo = reg_lo;
    a.reg_hi = reg_hi;
    a.first_lo = first_lo;
    a.first_hi = first_hi;
    a.wq = h->wq32;
    a.fc = h->fc32;
    a.binv = h->sh.binv;
    a.emat = h->sh.emat;
    a.has_e = h->sh.has_e;
    a.vprev = vin;
    a.depth = P.time_block;
    a.shape = P.tile_shape;
    a.acc = P.precision == MFWH_PREC_FP32_BLOCKSUM ? 1 : 0;
    a.err = h->d_err;
    a.forced = forced;
    int cur = 0;                 // pair holding the input: (W32[2 cur], W32[2 cur + 1])
    for (int n0 = 0; n0 < n_run;) {
      a.n0 = n0;
      a.steps = std::min(P.time_block, n_run - n0);
      a.last = n0 + a.steps == n_t;
      const float* D_in = n0 == 0 ? nullptr : h->W32[2 * cur + 1];
      if (P.dim == 3)
        launch_tb3d32(nf, h->geom, h->W32[2 * cur], D_in, h->W32[2 * (1 - cur)],
                      h->W32[2 * (1 - cur) + 1], h->f32, h->qs, h->qc, vout, vsub, a, st);
      else
        launch_tb2d32(nf, h->geom, h->W32[2 * cur], D_in, h->W32[2 * (1 - cur)],
                      h->W32[2 * (1 - cur) + 1], h->f32, h->qs, h->qc, vout, vsub, a, st);
      ++launches;
      n0 += a.steps;
      cur = 1 - cur;
    }
  } else {
    Step32Host a;
    a.forced = forced;
    float* Wc = h->W32[0];
    float* Wn = h->W32[2];
    float* D = h->W32[1];
    for (int n = 0; n < n_run; ++n) {
      a.lo = n == 0 ? first_lo : reg_lo;
      a.hi = n == 0 ? first_hi : reg_hi;
      for (int m = 0; m < nf; ++m) {
        a.fc[m] = h->fc32_h[(size_t)n * nf + m];
        a.wq[m] = h->wq32_h[(size_t)(n + 1) * nf + m];
      }
      const float* D_in = n == 0 ? nullptr : D;
      if (n + 1 < n_t) {
        launch_step32(nf, h->geom, Wc, D_in, Wn, D, h->f32, h->qs, h->qc, a, st);
        std::swap(Wc, Wn);
      } else {
        h->sh.vprev = vin;
        launch_last32(nf, h->geom, Wc, D_in, h->f32, h->qs, h->qc, vout, vsub, a, h->sh, st);
      }
      ++launches;
    }
  }
  h->step_launches += launches;
  h->total_launches += launches;
  if (timed) {
    CK(cudaEventRecord(h->ev[h->ev_used + 1], st));
    h->ev_used += 2;
  }
  CK(cudaGetLastError());
  return MFWH_OK;
}

// v_out = Pi(v_in) (forced) or S v_in; with vsub: v_out = vsub - (that).
mfwh_status apply_pi_tb(mfwh_handle_t h, const double* vin, double* vout, int forced,
                        const double* vsub);

// Implicit trapezoidal wave solve: one init launch, then one launch per step (multigrid solve
// of A Z = rhs and the update of W, q and the next rhs; the last one writes v_out).
mfwh_status apply_pi_implicit(mfwh_handle_t h, const double* vin, double* vout, int forced,
                              const double* vsub) {
  const Plan& P = h->plan;
  const int nf = h->nf;
  const int n_t = P.s.n_t;
  cudaStream_t st = h->stream;
  ImpArgs& A = *h->imp;
  A.wait_ns = (unsigned long long)(h->wait_s * 1e9);
  CK(cudaMemsetAsync(h->d_mgstate, 0, sizeof(MgState) * n_t, st));
  ImpInit ini{};
  for (int m = 0; m < nf; ++m) {
    ini.w0[m] = P.w[m];
    ini.fc0[m] = forced ? h->imp_fc[m] : 0.0;
  }
  launch_imp_init(nf, h->geom, vin, h->Wa, h->q, h->f, A.lev[0].u, A.lev[0].f, h->d_mgstate, ini,
                  st);
  h->total_launches += 1;
  const bool timed = h->ev_used + 2 <= (int)h->ev.size();
  if (timed) CK(cudaEventRecord(h->ev[h->ev_used], st));
  A.q = h->q;
  A.f = h->f;
  A.vout = vout;
  A.vsub = vsub;
  A.subtract = vsub != nullptr;
  A.has_e = h->sh.has_e && vin != nullptr;
  A.vprev = vin;
  std::memcpy(A.binv, h->sh.binv, sizeof(A.binv));
  std::memcpy(A.emat, h->sh.emat, sizeof(A.emat));
  for (int n = 0; n < n_t; ++n) {
    A.st = h->d_mgstate + n;
    A.st_next = n + 1 < n_t ? h->d_mgstate + n + 1 : nullptr;
    A.Wp = (n % 2 == 0) ? h->Wb : h->Wa;   // W^{n-1}; step 0 writes W^1 into the spare level
    A.Wc = (n % 2 == 0) ? h->Wa : h->Wb;   // W^n
    A.first = n == 0;
    A.last = n + 1 == n_t;
    for (int m = 0; m < nf; ++m) {
      A.wq[m] = P.w[(size_t)(n + 1) * nf + m];
      A.fc[m] = (forced && n + 1 < n_t) ? h->imp_fc[(size_t)(n + 1) * nf + m] : 0.0;
    }
    cudaError_t e = launch_imp_step(P.dim, A, h->imp_grid, h->imp_smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "implicit step launch");
  }
  h->step_launches += n_t;
  h->total_launches += n_t;
  if (timed) {
    CK(cudaEventRecord(h->ev[h->ev_used + 1], st));
    h->ev_used += 2;
  }
  CK(cudaGetLastError());
  return MFWH_OK;
}

mfwh_status apply_pi_direct(mfwh_handle_t h, const double* vin, double* vout, int forced,
                            const double* vsub) {
  if (h->implicit) return apply_pi_implicit(h, vin, vout, forced, vsub);
  if (h->use32) return apply_pi32(h, vin, vout, forced, vsub);
  // The FP64 blocked kernel (depth 2, 3, 4 or 8) serves the FP64 wave solves of FP64 handles
  // with time_block > 1 and those of 2D FP32 handles (the FP64 residuals and products of
  // mfwh_solve_refined and mfwh_solve_relaxed).
  if (h->depth64 > 1) return apply_pi_tb(h, vin, vout, forced, vsub);
  const Plan& P = h->plan;
  const int nf = h->nf;
  const int n_t = P.s.n_t;
  const int n_run = h->tune_steps > 0 ? std::min(h->tune_steps, n_t) : n_t;
  const double dt = P.s.dt;
  cudaStream_t st = h->stream;
  launch_init(nf, h->geom, vin, h->Wa, h->q, &P.w[0], st);
  h->total_launches += 1;
  const bool timed = h->ev_used + 2 <= (int)h->ev.size();
  if (timed) CK(cudaEventRecord(h->ev[h->ev_used], st));
  double* Wc = h->Wa;
  double* Wp = h->Wb;
  StepHost& a = h->sh;
  a.forced = forced;
  a.subtract = vsub != nullptr;
  a.vprev = vin;
  for (int n = 0; n < n_run; ++n) {
    const bool first = n == 0;
    const double kappa = first ? 0.5 * dt * dt : dt * dt;
    const double a_cur = first ? 1.0 : 2.0;
    layer_coef(h, P.c2_lo, a_cur, kappa, &a.lo);
    layer_coef(h, P.c2_hi, a_cur, kappa, &a.hi);
    a.a_cur = a_cur;
    a.first = first;
    for (int m = 0; m < nf; ++m) {
      a.fc[m] = kappa * P.cosf[(size_t)n * nf + m];
      a.wq[m] = P.w[(size_t)(n + 1) * nf + m];
    }
    if (n + 1 < n_t) {
      launch_step(nf, h->geom, Wc, Wp, h->f, h->q, a, st);
      std::swap(Wc, Wp);
    } else {
      launch_last(nf, h->geom, Wc, Wp, h->f, h->q, vout, vsub, a, st);
    }
  }
  h->step_launches += n_run;
  h->total_launches += n_run;
  if (timed) {
    CK(cudaEventRecord(h->ev[h->ev_used + 1], st));
    h->ev_used += 2;
  }
  CK(cudaGetLastError());
  return MFWH_OK;
}

// Temporally blocked wave solve (2D): ceil(N_t / depth) launches, alternating between the
// two pairs of wave-level buffers; the last launch writes v_out.
mfwh_status apply_pi_tb(mfwh_handle_t h, const double* vin, double* vout, int forced,
                        const double* vsub) {
  const Plan& P = h->plan;
  const int nf = h->nf;
  const int n_t = P.s.n_t;
  const int n_run = h->tune_steps > 0 ? std::min(h->tune_steps, n_t) : n_t;
  const double dt = P.s.dt;
  const int depth = h->depth64;
  if (depth != 2 && depth != 3 && depth != 4 && depth != 8)
    return fail(MFWH_ERR_INVALID_ARG, "FP64 blocking depth must be 2, 3, 4 or 8");
  cudaStream_t st = h->stream;
  launch_init(nf, h->geom, vin, h->Wa, h->q, &P.w[0], st);
  h->total_launches += 1;
  const bool timed = h->ev_used + 2 <= (int)h->ev.size();
  if (timed) CK(cudaEventRecord(h->ev[h->ev_used], st));
  TBHost a;
  layer_coef(h, P.c2_lo, 2.0, dt * dt, &a.reg_lo);
  layer_coef(h, P.c2_hi, 2.0, dt * dt, &a.reg_hi);
  layer_coef(h, P.c2_lo, 1.0, 0.5 * dt * dt, &a.first_lo);
  layer_coef(h, P.c2_hi, 1.0, 0.5 * dt * dt, &a.first_hi);
  a.wq_table = h->d_wq;
  a.cos_table = h->d_cos;
  a.wq_host = P.w.data();
  a.cos_host = P.cosf.data();
  a.dt2 = dt * dt;
  a.half_dt2 = 0.5 * dt * dt;
  a.depth = depth;
  a.shape = h->shape64;
  a.forced = forced;
  a.subtract = vsub != nullptr;
  std::memcpy(a.binv, h->sh.binv, sizeof(a.binv));
  std::memcpy(a.emat, h->sh.emat, sizeof(a.emat));
  a.has_e = h->sh.has_e;
  a.vprev = vin;
  const double* in_c = h->Wa;
  const double* in_p = nullptr;     // W^{-1} = 0 before the first step
  double* out_c = h->Wc2;
  double* out_p = h->Wp2;
  int launches = 0;
  for (int n0 = 0; n0 < n_run;) {
    a.n0 = n0;
    a.steps = std::min(depth, n_run - n0);
    a.last = n0 + a.steps == n_t;
    launch_tb2d(nf, h->geom, in_c, in_p, out_c, out_p, h->f, h->q, vout, vsub, a, st);
    ++launches;
    n0 += a.steps;
    // next launch reads what this one wrote and writes the other pair
    double* nc = (out_c == h->Wc2) ? h->Wa : h->Wc2;
    double* np = (out_c == h->Wc2) ? h->Wb : h->Wp2;
    in_c = out_c;
    in_p = out_p;
    out_c = nc;
    out_p = np;
  }
  h->step_launches += launches;
  h->total_launches += launches;
  if (timed) {
    CK(cudaEventRecord(h->ev[h->ev_used + 1], st));
    h->ev_used += 2;
  }
  CK(cudaGetLastError());
  return MFWH_OK;
}

// One wave solve: replayed from a captured graph in graph mode, launched directly otherwise.
mfwh_status apply_pi(mfwh_handle_t h, const double* vin, double* vout, int forced,
                     const double* vsub) {
  Range range(forced ? "mfwh: Pi (forced)" : "mfwh: Pi");
  // implicit handles launch N_t + 1 kernels per wave solve: no graph
  if (!h->graphs || (vsub && vsub != vin) || h->tune_steps > 0 || h->implicit)
    return apply_pi_direct(h, vin, vout, forced, vsub);
  const int key = (vin ? 1 : 0) | (forced ? 2 : 0) | (vsub ? 4 : 0) | (h->use32 ? 8 : 0);
  cudaStream_t st = h->gstream;
  CK(cudaEventRecord(h->gev[0], h->stream));
  CK(cudaStreamWaitEvent(st, h->gev[0], 0));
  if (!h->gexec[key]) {
    const int saved_ev = h->ev_used;
    const int64_t sl = h->step_launches, tl = h->total_launches;
    h->ev_used = (int)h->ev.size();   // no timing events inside the graph
    cudaStream_t user = h->stream;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    h->stream = st;
    mfwh_status cs = apply_pi_direct(h, vin ? h->g_in : nullptr, h->g_out, forced,
                                     vsub ? h->g_in : nullptr);
    h->stream = user;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    h->ev_used = saved_ev;
    h->g_steps[key] = h->step_launches - sl;
    h->g_total[key] = h->total_launches - tl;
    h->step_launches = sl;
    h->total_launches = tl;
    if (cs != MFWH_OK) {
      if (graph) cudaGraphDestroy(graph);
      return cs;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->gexec[key], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->gexec[key] = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  if (vin) CK(cudaMemcpyAsync(h->g_in, vin, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, st));
  const bool timed = h->ev_used + 2 <= (int)h->ev.size();
  if (timed) CK(cudaEventRecord(h->ev[h->ev_used], st));
  CK(cudaGraphLaunch(h->gexec[key], st));
  if (timed) {
    CK(cudaEventRecord(h->ev[h->ev_used + 1], st));
    h->ev_used += 2;
  }
  CK(cudaMemcpyAsync(vout, h->g_out, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, st));
  CK(cudaEventRecord(h->gev[1], st));
  CK(cudaStreamWaitEvent(h->stream, h->gev[1], 0));
  h->step_launches += h->g_steps[key];
  h->total_launches += h->g_total[key];
  return MFWH_OK;
}

mfwh_status collect_timing_sync(mfwh_handle_t h) {
  CK(cudaStreamSynchronize(h->stream));
  return collect_timing(h);
}

void drop_graphs(mfwh_handle_t h) {
  for (auto& g : h->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

mfwh_status dots(mfwh_handle_t h, const double* V, int k, const double* w, double* out_host) {
  launch_multidot(V, h->N, k, w, h->N, h->dot_partial, h->dot_out, h->stream);
  h->total_launches += multidot_launches(k);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->pinned, h->dot_out, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memcpy(out_host, h->pinned, sizeof(double) * k);
  return MFWH_OK;
}

mfwh_status residual_dev(mfwh_handle_t h, const double* v_dev, double* r_out) {
  Range range("mfwh: residual");
  launch_residual(h->nf, h->geom, v_dev, h->f, h->omega2, h->plan.c2_lo, h->plan.c2_hi, h->inv_h2,
                  h->res_partial, h->res_out, h->stream);
  h->total_launches += 2;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->pinned, h->res_out, sizeof(double) * 2 * h->nf, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  bool finite = true;
  for (int m = 0; m < h->nf; ++m) {
    const double num = h->pinned[m], den = h->pinned[h->nf + m];
    r_out[m] = den > 0.0 ? num / den : num;
    finite = finite && std::isfinite(r_out[m]);
  }
  if (!finite) return fail(MFWH_ERR_NONFINITE, "non-finite value in the Helmholtz residual");
  return MFWH_OK;
}

mfwh_status ensure_basis(mfwh_handle_t h, int vectors) {
  if (h->basis_vectors >= vectors) return MFWH_OK;
  if (h->basis) cudaFree(h->basis);
  h->basis = nullptr;
  h->basis_vectors = 0;
  CK(cudaMalloc(&h->basis, sizeof(double) * h->N * vectors));
  h->basis_vectors = vectors;
  return MFWH_OK;
}

// Stage a host-or-device stack of grid functions on the device.
mfwh_status stage_in(mfwh_handle_t h, const double* v, double** dev, bool* on_device) {
  *on_device = is_device_ptr(v);
  if (*on_device) {
    *dev = const_cast<double*>(v);
    return MFWH_OK;
  }
  CK(cudaMemcpyAsync(h->vec_x, v, sizeof(double) * h->N, cudaMemcpyHostToDevice, h->stream));
  *dev = h->vec_x;
  return MFWH_OK;
}

// GMRES(restart) on (I - S) x = Pi(0) for a device iterate x, counting into I (which it
// does not reset).  *converged reports whether the Arnoldi residual fell below tol.
// relax_below > 0 (relaxed products, FP32 handles only): the products start with FP64 wave
// solves and switch to the handle's FP32 wave solves once the Arnoldi residual estimate is
// below relax_below times ||rhs|| (an inexact Krylov method whose later products may be less
// accurate); the handle's wave precision is restored on return.
mfwh_status gmres_core(mfwh_handle_t h, int restart, double tol, int max_iters, double* x,
                       const double* rhs, mfwh_solve_info& I, bool* converged_out,
                       double relax_below = 0.0) {
  const bool relax = relax_below > 0.0 && h->plan.precision != MFWH_PREC_FP64;
  const bool use32_saved = h->use32;
  if (relax) h->use32 = false;
  struct Restore {
    mfwh_handle_t h;
    bool v;
    ~Restore() { h->use32 = v; }
  } restore_use32{h, use32_saved};
  const int64_t N = h->N;
  cudaStream_t s = h->stream;
  const int it0 = I.iterations;
  mfwh_status st;
  const double* b = rhs;
  if (!b) {
    // b = Pi(0) (eq. discreteMFWHmapping)
    st = apply_pi(h, nullptr, h->vec_b, 1, nullptr);
    if (st != MFWH_OK) return st;
    I.pi_applications++;
    b = h->vec_b;
  }
  double bb = 0.0, xx = 0.0;
  st = dots(h, b, 1, b, &bb);
  if (st != MFWH_OK) return st;
  st = dots(h, x, 1, x, &xx);
  if (st != MFWH_OK) return st;
  const double bnorm = std::sqrt(bb);
  if (!std::isfinite(bnorm) || !std::isfinite(xx))
    return fail(MFWH_ERR_NONFINITE, "non-finite right-hand side or initial guess");
  bool x_nonzero = xx > 0.0;
  bool converged = false;
  std::vector<double> H((restart + 1) * restart), cs(restart), sn(restart), g(restart + 1),
      y(restart), hcol(restart + 1), h2(restart + 1);
  if (bnorm == 0.0) {
    launch_axpby(x, 0.0, x, 0.0, N, s);
    converged = true;
    I.rel_residual = 0.0;
  }
  while (!converged && I.iterations - it0 < max_iters) {
    double* V0 = h->basis;
    I.restarts++;
    if (relax) h->use32 = false;   // every cycle's residual and first products in FP64
    if (x_nonzero) {   // r = b - (x - S x)
      st = apply_pi(h, x, V0, 0, x);
      if (st != MFWH_OK) return st;
      I.pi_applications++;
      launch_axpby(V0, 1.0, b, -1.0, N, s);
    } else {
      launch_axpby(V0, 1.0, b, 0.0, N, s);
    }
    h->total_launches++;
    double rr = 0.0;
    st = dots(h, V0, 1, V0, &rr);
    if (st != MFWH_OK) return st;
    const double beta = std::sqrt(rr);
    if (!std::isfinite(beta)) return fail(MFWH_ERR_NONFINITE, "non-finite Krylov residual");
    I.rel_residual = beta / bnorm;
    if (I.rel_residual < tol) {
      converged = true;
      break;
    }
    launch_axpby(V0, 1.0 / beta, V0, 0.0, N, s);
    h->total_launches++;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j_done = 0;
    double res = beta;
    for (int j = 0; j < restart; ++j) {
      Range range("mfwh: Arnoldi step");
      double* Vj = h->basis + (int64_t)j * N;
      double* w = h->basis + (int64_t)(j + 1) * N;
      st = apply_pi(h, Vj, w, 0, Vj);   // w = A v_j = v_j - S v_j
      if (st != MFWH_OK) return st;
      I.pi_applications++;
      I.iterations++;
      // classical Gram-Schmidt, applied twice
      st = dots(h, h->basis, j + 1, w, hcol.data());
      if (st != MFWH_OK) return st;
      launch_multi_axpy(w, h->basis, N, j + 1, hcol.data(), N, s);
      h->total_launches += multi_axpy_launches(j + 1);
      st = dots(h, h->basis, j + 1, w, h2.data());
      if (st != MFWH_OK) return st;
      launch_multi_axpy(w, h->basis, N, j + 1, h2.data(), N, s);
      h->total_launches += multi_axpy_launches(j + 1);
      for (int i = 0; i <= j; ++i) hcol[i] += h2[i];
      double ww = 0.0;
      st = dots(h, w, 1, w, &ww);
      if (st != MFWH_OK) return st;
      const double hnext = std::sqrt(ww);
      if (!std::isfinite(hnext)) return fail(MFWH_ERR_NONFINITE, "non-finite Arnoldi vector");
      // Givens rotations on the new Hessenberg column
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
        hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = t;
      }
      const double r = std::hypot(hcol[j], hnext);
      cs[j] = r > 0.0 ? hcol[j] / r : 1.0;
      sn[j] = r > 0.0 ? hnext / r : 0.0;
      hcol[j] = r;
      for (int i = 0; i <= j; ++i) H[i * restart + j] = hcol[i];
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      res = std::fabs(g[j + 1]);
      if (I.history && I.history_len < I.history_capacity) I.history[I.history_len++] = res / bnorm;
      if (relax && !h->use32 && res / bnorm < relax_below) h->use32 = true;
      j_done = j + 1;
      if (res / bnorm < tol || I.iterations - it0 >= max_iters || hnext == 0.0) break;
      launch_axpby(w, 1.0 / hnext, w, 0.0, N, s);
      h->total_launches++;
    }
    // y = R^{-1} g, then x += V y
    for (int i = j_done - 1; i >= 0; --i) {
      double acc = g[i];
      for (int k = i + 1; k < j_done; ++k) acc -= H[i * restart + k] * y[k];
      y[i] = acc / H[i * restart + i];
    }
    for (int i = 0; i < j_done; ++i) y[i] = -y[i];   // multi_axpy subtracts
    launch_multi_axpy(x, h->basis, N, j_done, y.data(), N, s);
    h->total_launches += multi_axpy_launches(j_done);
    x_nonzero = true;
    I.rel_residual = res / bnorm;
    if (I.rel_residual < tol) converged = true;
  }
  *converged_out = converged;
  return MFWH_OK;
}

}  // namespace

extern "C" {

const char* mfwh_last_error(void) { return g_error.c_str(); }

const char* mfwh_status_string(mfwh_status s) {
  switch (s) {
    case MFWH_OK: return "ok";
    case MFWH_ERR_INVALID_ARG: return "invalid argument";
    case MFWH_ERR_SINGULAR: return "singular filter system";
    case MFWH_ERR_CUDA: return "CUDA error";
    case MFWH_ERR_NOMEM: return "out of memory";
    case MFWH_ERR_NOT_CONVERGED: return "not converged";
    case MFWH_ERR_SPURIOUS: return "converged to a non-solution (Helmholtz residual check failed)";
    case MFWH_ERR_NONFINITE: return "non-finite values";
    case MFWH_ERR_TIMEOUT: return "a bounded wait inside a kernel ran out";
  }
  return "unknown status";
}

mfwh_status mfwh_plan(const mfwh_problem* prob, mfwh_setup* out) {
  if (!out) return fail(MFWH_ERR_INVALID_ARG, "null output");
  Plan P;
  mfwh_status st = plan_with_field(prob, &P);
  if (st == MFWH_OK) *out = P.s;
  return st;
}

mfwh_status mfwh_plan_multigrid(const mfwh_problem* prob, int* levels, int* coarse,
                                int64_t cells[16][3]) {
  if (!levels || !coarse || !cells) return fail(MFWH_ERR_INVALID_ARG, "null output");
  Plan P;
  mfwh_status st = plan_with_field(prob, &P);
  if (st != MFWH_OK) return st;
  if (P.time_stepping != MFWH_TIME_IMPLICIT)
    return fail(MFWH_ERR_INVALID_ARG, "not an implicit-time-stepping problem");
  Geom g{};
  g.nx = P.n[0];
  g.ny = P.n[1];
  g.nz = P.dim == 3 ? P.n[2] : 0;
  g.sy = g.nx + 1;
  g.sz = (g.nx + 1) * (g.ny + 1);
  g.points = P.s.points;
  g.dim = P.dim;
  g.layer_axis = P.layer_axis;
  g.layer_split = P.layer_split;
  MgLevel lev[kMgMaxLevels];
  int nlev = 0, lc = 0;
  int64_t smem = 0;
  if (!mg_plan_levels(g, P.s.h, P.c2_lo, P.c2_hi, P.s.dt, lev, &nlev, &lc, &smem))
    return fail(MFWH_ERR_INVALID_ARG,
                "implicit time stepping: the grid must halve (every n_i even, n_i / 2 >= 2) "
                "down to a level of at most 5000 points");
  if (P.order == 4 && !mg_mixed(P.dim, lc))
    return fail(MFWH_ERR_INVALID_ARG,
                "implicit time stepping with the fourth-order operator needs a grid of more "
                "than 5000 points");
  *levels = nlev;
  *coarse = lc;
  for (int l = 0; l < 16; ++l) {
    cells[l][0] = l < nlev ? lev[l].nx : 0;
    cells[l][1] = l < nlev ? lev[l].ny : 0;
    cells[l][2] = l < nlev ? lev[l].nz : 0;
  }
  return MFWH_OK;
}

mfwh_status mfwh_plan_weights(const mfwh_problem* prob, double* w_out, int64_t capacity) {
  if (!w_out) return fail(MFWH_ERR_INVALID_ARG, "null output");
  Plan P;
  mfwh_status st = plan_with_field(prob, &P);
  if (st != MFWH_OK) return st;
  if ((int64_t)P.w.size() > capacity) return fail(MFWH_ERR_INVALID_ARG, "w_out too small");
  std::memcpy(w_out, P.w.data(), sizeof(double) * P.w.size());
  return MFWH_OK;
}

mfwh_status mfwh_adjusted_frequency(int nf, const double* omega, double dt, double alpha,
                                    double beta, double* out) {
  if (nf < 1 || !omega || !out || !(dt > 0.0)) return fail(MFWH_ERR_INVALID_ARG, "bad arguments");
  for (int m = 0; m < nf; ++m) {
    const double x = omega[m] * dt;
    const double c = (1.0 - 0.5 * beta * x * x) / (1.0 + alpha * x * x);
    if (c < -1.0 || c > 1.0) return fail(MFWH_ERR_INVALID_ARG, "frequency beyond the scheme's range");
    out[m] = std::acos(c) / dt;
  }
  return MFWH_OK;
}

mfwh_status mfwh_opt_parameters(int nf, const double* omega, int n_p, int n_t, int n_delta,
                                double c_delta, double* params_out, double* lam_max,
                                int* n_lambda) {
  if (nf < 1 || nf > MFWH_MAX_NF || !omega || !params_out || n_p < 1 || n_t < 2 || n_delta < 1)
    return fail(MFWH_ERR_INVALID_ARG, "bad arguments");
  for (int m = 0; m < nf; ++m)
    if (!(omega[m] > 0.0) || (m > 0 && !(omega[m] > omega[m - 1])))
      return fail(MFWH_ERR_INVALID_ARG, "frequencies must be positive and increasing");
  return optimise_parameters(nf, omega, n_p, n_t, n_delta, c_delta, params_out, lam_max, n_lambda);
}

mfwh_status mfwh_create(const mfwh_problem* prob, void* stream, mfwh_handle_t* out) {
  Range range("mfwh: create");
  if (!out) return fail(MFWH_ERR_INVALID_ARG, "null output");
  *out = nullptr;
  auto* h = new (std::nothrow) mfwh_handle_s();
  if (!h) return fail(MFWH_ERR_NOMEM, "host allocation failed");
  mfwh_status st = plan_with_field(prob, &h->plan);
  if (st != MFWH_OK) {
    delete h;
    return st;
  }
  const Plan& P = h->plan;
  h->stream = static_cast<cudaStream_t>(stream);
  h->nf = P.s.nf;
  h->P = P.s.points;
  h->N = h->P * h->nf;
  for (int a = 0; a < 3; ++a) h->inv_h2[a] = a < P.dim ? 1.0 / (P.s.h[a] * P.s.h[a]) : 0.0;
  for (int m = 0; m < h->nf; ++m) h->omega2[m] = prob->omega[m] * prob->omega[m];
  Geom& g = h->geom;
  g.nx = P.n[0];
  g.ny = P.n[1];
  g.nz = P.dim == 3 ? P.n[2] : 0;
  g.sy = g.nx + 1;
  g.sz = (g.nx + 1) * (g.ny + 1);
  g.points = h->P;
  g.dim = P.dim;
  g.layer_axis = P.layer_axis;
  g.layer_split = P.layer_split;
  g.order = P.order;
  // FP32 2D wave levels: rows padded to 32 floats (16-byte aligned for tensor copies)
  const bool pad_w = P.precision != MFWH_PREC_FP64 && P.dim == 2;
  g.syw = pad_w ? (g.nx + 1 + 31) / 32 * 32 : g.sy;
  g.szw = pad_w ? g.syw * (g.ny + 1) : g.sz;
  h->PW = pad_w ? g.syw * (g.ny + 1) : h->P;

  auto cleanup = [&](mfwh_status s) {
    mfwh_destroy(h);
    return s;
  };
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaGetDevice"));
  const int64_t tables = (int64_t)(P.s.n_t + 1) * h->nf;
  struct {
    double** p;
    int64_t n;
  } bufs[] = {{&h->f, h->N},
              {&h->Wa, h->P},
              {&h->Wb, h->P},
              {&h->Wc2, h->P},
              {&h->Wp2, h->P},
              {&h->d_wq, tables},
              {&h->d_cos, tables},
              {&h->q, h->N},
              {&h->res_partial, residual_partial_size(MFWH_MAX_NF)},
              {&h->res_out, 2 * MFWH_MAX_NF},
              {&h->dot_partial, dot_partial_size()},
              {&h->dot_out, kMaxKrylov},
              {&h->vec_b, h->N},
              {&h->vec_x, h->N}};
  for (auto& b : bufs) {
    e = cudaMalloc(b.p, sizeof(double) * b.n);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc (workspace)"));
  }
  if (P.precision != MFWH_PREC_FP64) {
    const int nf = h->nf;
    const int n_t = P.s.n_t;
    const double dt = P.s.dt;
    h->wq32_h.resize((size_t)(n_t + 1) * nf);
    h->fc32_h.resize((size_t)n_t * nf);
    for (size_t i = 0; i < h->wq32_h.size(); ++i) h->wq32_h[i] = (float)P.w[i];
    for (int n = 0; n < n_t; ++n) {
      const double kappa = n == 0 ? 0.5 * dt * dt : dt * dt;
      for (int m = 0; m < nf; ++m)
        h->fc32_h[(size_t)n * nf + m] = (float)(kappa * P.cosf[(size_t)n * nf + m]);
    }
    struct {
      float** p;
      int64_t n;
    } fb[] = {{&h->f32, h->N}, {&h->W32[0], h->PW}, {&h->W32[1], h->PW}, {&h->W32[2], h->PW},
              {&h->W32[3], h->PW}, {&h->qs, h->N}, {&h->qc, h->N},
              {&h->wq32, (int64_t)h->wq32_h.size()}, {&h->fc32, (int64_t)h->fc32_h.size()}};
    for (auto& b : fb) {
      e = cudaMalloc(b.p, sizeof(float) * std::max<int64_t>(b.n, 1));
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc (FP32 workspace)"));
    }
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
      e = cudaMemsetAsync(h->W32[i], 0, sizeof(float) * h->PW, h->stream);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->wq32, h->wq32_h.data(), sizeof(float) * h->wq32_h.size(),
                          cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !h->fc32_h.empty())
      e = cudaMemcpyAsync(h->fc32, h->fc32_h.data(), sizeof(float) * h->fc32_h.size(),
                          cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "initialising FP32 workspace"));
  }
  if (P.time_stepping == MFWH_TIME_IMPLICIT) {
    if (h->P >= ((int64_t)1 << 31))
      return cleanup(fail(MFWH_ERR_INVALID_ARG, "implicit time stepping: fewer than 2^31 points"));
    h->implicit = true;
    h->imp = new (std::nothrow) ImpArgs();
    if (!h->imp) return cleanup(fail(MFWH_ERR_NOMEM, "host allocation failed"));
    ImpArgs& A = *h->imp;
    int64_t smem_d = 0;
    if (!mg_plan_levels(g, P.s.h, P.c2_lo, P.c2_hi, P.s.dt, A.lev, &A.nlev, &A.lc, &smem_d))
      return cleanup(fail(MFWH_ERR_INVALID_ARG,
                          "implicit time stepping: the grid must halve (every n_i even, "
                          "n_i / 2 >= 2) down to a level of at most 5000 points"));
    if (P.order == 4) {
      if (!mg_mixed(P.dim, A.lc))
        return cleanup(fail(MFWH_ERR_INVALID_ARG,
                            "implicit time stepping with the fourth-order operator needs a "
                            "grid of more than 5000 points"));
      mg_set_order4(&A.lev[0], P.s.h, P.c2_lo, P.c2_hi, P.s.dt, P.dim);
    }
    A.omega_dc = P.order == 4 ? 6.0 / 7.0 : 1.0;
    // Level arrays (bytes counted in 4-byte words).  FP64 defect correction (grid-wide
    // levels): level 0 holds Z, rhs (FP64) and the FP32 correction arrays; levels 1..lc-1 hold
    // three FP32 arrays; level lc holds u, rhs (FP32).  One-CTA hierarchies (FP64 V-cycles):
    // u, f (FP64) at level 0 = lc.
    const bool mixed = mg_mixed(P.dim, A.lc);
    int64_t words = 0;
    for (int l = 0; l <= A.lc; ++l) {
      const int64_t n = A.lev[l].points;
      if (mixed)
        words += l == 0 ? 4 * n + (P.dim == 3 ? 3 : 2) * n : (l < A.lc ? 3 * n : 2 * n);
      else
        words += 2 * 2 * n;
    }
    e = cudaMalloc(&h->imp_mem, 4 * words);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->imp_mem, 0, 4 * words, h->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc (multigrid levels)"));
    char* cur = reinterpret_cast<char*>(h->imp_mem);
    auto take64 = [&](int64_t n) { double* p = reinterpret_cast<double*>(cur); cur += 8 * n; return p; };
    auto take32 = [&](int64_t n) { float* p = reinterpret_cast<float*>(cur); cur += 4 * n; return p; };
    for (int l = 0; l <= A.lc; ++l) {
      MgLevel& L = A.lev[l];
      const int64_t n = L.points;
      if (mixed) {
        if (l == 0) {
          L.u = take64(n);
          L.f = take64(n);
          L.v32 = take32(n);
          L.f32 = take32(n);
          if (P.dim == 3) L.u32 = take32(n);
        } else {
          L.u32 = take32(n);
          L.f32 = take32(n);
          if (l < A.lc) L.v32 = take32(n);
        }
      } else {
        L.u = take64(n);
        L.f = take64(n);
      }
    }
    e = mg_launch_config(P.dim, A.lc, smem_d, A.lev, &h->imp_grid, &h->imp_smem);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "multigrid launch configuration"));
    A.layer_axis = P.layer_axis;
    A.nf = h->nf;
    A.nu1 = 2;
    A.nu2 = 1;
    // the coarsest grid is solved by Gauss-Seidel sweeps alone: enough for its longest line
    const MgLevel& cl = A.lev[A.nlev - 1];
    const int cn = std::max({cl.nx, cl.ny, P.dim == 3 ? cl.nz : 0});
    A.coarse_sweeps = std::min(400, std::max(4, 2 * cn * cn));
    A.max_cycles = P.mg_max_cycles;
    A.tol = P.mg_tol;
    if (e == cudaSuccess) e = cudaMalloc(&h->d_mgstate, sizeof(MgState) * P.s.n_t);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_bar, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_mgc, sizeof(MgCounters));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_mgc, 0, sizeof(MgCounters), h->stream);
    if (e == cudaSuccess && !h->d_err) {
      e = cudaMalloc(&h->d_err, sizeof(int));
      if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
    }
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "implicit workspace"));
    A.bar = h->d_bar;
    A.err = h->d_err;
    A.counters = h->d_mgc;
    // F^n factor of eq. WaveSchemeForcing: beta + 2 alpha cos(omega~ dt) = cos(omega~ dt)
    const double dt = P.s.dt;
    h->imp_fc.resize((size_t)(P.s.n_t + 1) * h->nf);
    for (int n = 0; n <= P.s.n_t; ++n)
      for (int m = 0; m < h->nf; ++m)
        h->imp_fc[(size_t)n * h->nf + m] =
            dt * dt * P.cosf[(size_t)n * h->nf + m] * std::cos(P.s.omega_tilde[m] * dt);
  }
  e = cudaMallocHost(&h->pinned, sizeof(double) * kPinned);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMallocHost"));
  h->ev.resize(kEventPool);
  for (auto& x : h->ev) {
    e = cudaEventCreate(&x);
    if (e != cudaSuccess) {
      x = nullptr;
      return cleanup(cuda_fail(e, "cudaEventCreate"));
    }
  }
  // Boundary values of the wave levels are never written by the step kernels and must be 0.
  e = cudaMemsetAsync(h->Wa, 0, sizeof(double) * h->P, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Wb, 0, sizeof(double) * h->P, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Wc2, 0, sizeof(double) * h->P, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Wp2, 0, sizeof(double) * h->P, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_wq, P.w.data(), sizeof(double) * tables, cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_cos, P.cosf.data(), sizeof(double) * tables, cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->f, 0, sizeof(double) * h->N, h->stream);
  if (e == cudaSuccess && prob->forcing)
    e = cudaMemcpyAsync(h->f, prob->forcing, sizeof(double) * h->N, cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess && P.c2_field) {
    e = cudaMalloc(&h->c2f, sizeof(double) * h->P);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->c2f, prob->c2_field, sizeof(double) * h->P, cudaMemcpyDefault,
                          h->stream);
    h->geom.c2f = h->c2f;
  }
#ifdef MFWH_BOUNDS_CHECK
  if (e == cudaSuccess) e = cudaMalloc(&h->fault, sizeof(BoundsFault));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->fault, 0, sizeof(BoundsFault), h->stream);
  h->geom.fault = h->fault;
#endif
  if (e == cudaSuccess && h->f32) {
    launch_to_float(h->f, h->f32, h->N, h->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "initialising workspace"));
  h->use32 = P.precision != MFWH_PREC_FP64;
  if (P.precision == MFWH_PREC_FP64) {
    h->depth64 = P.time_block;
    h->shape64 = P.tile_shape;
  } else if (P.dim == 2 && P.order == 2 && !P.c2_field && h->nf <= 8) {
    // the FP64 wave solves of an FP32 handle take the FP64 default: 3 steps per pass on the
    // persistent pipelined kernel (bit-identical to one step per launch)
    h->depth64 = 3;
    h->shape64 = 5;
  }
  std::memset(&h->sh, 0, sizeof(h->sh));
  // Epilogue V^{k+1} = C q + E V^k: implicit filter C = B^{-1}, E = 0; explicit filter
  // C = diag(B)^{-1}, E = -diag(B)^{-1} (B - diag(B)).
  const bool expl = P.filter_update == MFWH_UPDATE_EXPLICIT;
  for (int m = 0; m < h->nf; ++m)
    for (int j = 0; j < h->nf; ++j) {
      h->sh.binv[m * MFWH_MAX_NF + j] =
          expl ? (m == j ? 1.0 / P.s.B[m][m] : 0.0) : P.s.B_inv[m][j];
      h->sh.emat[m * MFWH_MAX_NF + j] = (expl && m != j) ? -P.s.B[m][j] / P.s.B[m][m] : 0.0;
    }
  h->sh.has_e = expl ? 1 : 0;
  h->sh.vprev = nullptr;
  *out = h;
  return MFWH_OK;
}

mfwh_status mfwh_set_forcing(mfwh_handle_t h, const double* forcing) {
  if (!h || !forcing) return fail(MFWH_ERR_INVALID_ARG, "null argument");
  CK(cudaMemcpyAsync(h->f, forcing, sizeof(double) * h->N, cudaMemcpyDefault, h->stream));
  if (h->f32) {
    launch_to_float(h->f, h->f32, h->N, h->stream);
    h->total_launches++;
    CK(cudaGetLastError());
  }
  return MFWH_OK;
}

mfwh_status mfwh_apply_Pi(mfwh_handle_t h, const double* v_in, double* v_out, int forced) {
  if (!h || !v_out) return fail(MFWH_ERR_INVALID_ARG, "null argument");
  if (!is_device_ptr(v_out) || (v_in && !is_device_ptr(v_in)))
    return fail(MFWH_ERR_INVALID_ARG, "mfwh_apply_Pi takes device pointers");
  reset_timing(h);
  return apply_pi(h, v_in, v_out, forced ? 1 : 0, nullptr);
}

mfwh_status mfwh_solve_fpi(mfwh_handle_t h, int iters, double* v) {
  if (!h || !v || iters < 0) return fail(MFWH_ERR_INVALID_ARG, "bad argument");
  reset_timing(h);
  double* x = nullptr;
  bool on_dev = false;
  mfwh_status st = stage_in(h, v, &x, &on_dev);
  if (st != MFWH_OK) return st;
  for (int k = 0; k < iters; ++k) {
    st = apply_pi(h, x, x, 1, nullptr);
    if (st != MFWH_OK) return st;
  }
  if (!on_dev) CK(cudaMemcpyAsync(v, x, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return collect_timing(h);
}

mfwh_status mfwh_solve_gmres(mfwh_handle_t h, int restart, double tol, int max_iters,
                             double spurious_tol, double* v, mfwh_solve_info* info) {
  if (!h || !v) return fail(MFWH_ERR_INVALID_ARG, "null argument");
  if (restart < 1 || restart > kMaxRestart)
    return fail(MFWH_ERR_INVALID_ARG, "restart must be in 1..1023");
  if (max_iters < 1 || !(tol >= 0.0)) return fail(MFWH_ERR_INVALID_ARG, "bad max_iters or tol");
  if (restart > max_iters) restart = max_iters;   // a longer basis would never be used
  reset_timing(h);
  mfwh_status st = ensure_basis(h, restart + 1);
  if (st != MFWH_OK) return st;
  mfwh_solve_info local{};
  mfwh_solve_info& I = info ? *info : local;
  I.iterations = I.pi_applications = I.restarts = I.refinements = 0;
  I.history_len = 0;
  I.rel_residual = NAN;
  const int64_t N = h->N;
  cudaStream_t s = h->stream;
  double* x = nullptr;
  bool on_dev = false;
  st = stage_in(h, v, &x, &on_dev);
  if (st != MFWH_OK) return st;

  bool converged = false;
  st = gmres_core(h, restart, tol, max_iters, x, nullptr, I, &converged);
  if (st != MFWH_OK) return st;
  CK(cudaGetLastError());
  double r[MFWH_MAX_NF];
  st = residual_dev(h, x, r);
  for (int m = 0; m < h->nf; ++m) I.helmholtz_residual[m] = st == MFWH_OK ? r[m] : NAN;
  if (!on_dev) CK(cudaMemcpyAsync(v, x, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  mfwh_status ts = collect_timing(h);
  if (ts != MFWH_OK) return ts;
  if (st != MFWH_OK) return st;
  if (!converged) {
    std::ostringstream os;
    os << "GMRES stopped after " << I.iterations << " iterations at relative residual "
       << I.rel_residual;
    return fail(MFWH_ERR_NOT_CONVERGED, os.str());
  }
  if (spurious_tol > 0.0) {
    double worst = 0.0;
    for (int m = 0; m < h->nf; ++m) worst = std::fmax(worst, r[m]);
    if (worst > spurious_tol) {
      std::ostringstream os;
      os << "GMRES converged but the Helmholtz residual is " << worst << " > " << spurious_tol
         << " (spurious resonance?)";
      return fail(MFWH_ERR_SPURIOUS, os.str());
    }
  }
  return MFWH_OK;
}

}  // extern "C"

namespace {

// Iterative refinement with FP64 outer residuals (mfwh_solve_refined); relax_below > 0 makes
// each inner solve a relaxed one (FP64 products first, then FP32: see gmres_core).
mfwh_status refine_core(mfwh_handle_t h, int restart, double inner_tol, int max_iters,
                        double target, int max_refinements, double* v, mfwh_solve_info* info,
                        double relax_below) {
  if (!h || !v) return fail(MFWH_ERR_INVALID_ARG, "null argument");
  if (restart < 1 || restart > kMaxRestart)
    return fail(MFWH_ERR_INVALID_ARG, "restart must be in 1..1023");
  if (max_iters < 1 || !(inner_tol >= 0.0) || !(target > 0.0) || max_refinements < 0)
    return fail(MFWH_ERR_INVALID_ARG, "bad max_iters, inner_tol, target or max_refinements");
  if (restart > max_iters) restart = max_iters;
  reset_timing(h);
  mfwh_status st = ensure_basis(h, restart + 1);
  if (st != MFWH_OK) return st;
  if (!h->vec_r) CK(cudaMalloc(&h->vec_r, sizeof(double) * h->N));
  if (!h->vec_e) CK(cudaMalloc(&h->vec_e, sizeof(double) * h->N));
  mfwh_solve_info local{};
  mfwh_solve_info& I = info ? *info : local;
  I.iterations = I.pi_applications = I.restarts = I.refinements = 0;
  I.history_len = 0;
  I.rel_residual = NAN;
  const int64_t N = h->N;
  cudaStream_t s = h->stream;
  double* x = nullptr;
  bool on_dev = false;
  st = stage_in(h, v, &x, &on_dev);
  if (st != MFWH_OK) return st;
  const bool inner32 = h->plan.precision != MFWH_PREC_FP64;
  // b = Pi(0) with an FP64 wave solve
  h->use32 = false;
  st = apply_pi(h, nullptr, h->vec_b, 1, nullptr);
  I.pi_applications++;
  double bb = 0.0, xx = 0.0;
  if (st == MFWH_OK) st = dots(h, h->vec_b, 1, h->vec_b, &bb);
  if (st == MFWH_OK) st = dots(h, x, 1, x, &xx);
  if (st == MFWH_OK && (!std::isfinite(bb) || !std::isfinite(xx)))
    st = fail(MFWH_ERR_NONFINITE, "non-finite right-hand side or initial guess");
  const double bnorm = std::sqrt(bb);
  bool x_nonzero = xx > 0.0;
  double r[MFWH_MAX_NF];
  bool done = false;
  mfwh_status inner = MFWH_OK;
  for (int k = 0; st == MFWH_OK; ++k) {
    st = residual_dev(h, x, r);       // r_h of the current iterate, FP64
    if (st != MFWH_OK) break;
    double worst = 0.0;
    for (int m = 0; m < h->nf; ++m) worst = std::fmax(worst, r[m]);
    if (worst <= target || bnorm == 0.0) {
      done = true;
      break;
    }
    if (k == max_refinements || I.iterations >= max_iters) break;
    // outer residual in FP64: r = b - (x - S x)
    h->use32 = false;
    if (x_nonzero) {
      st = apply_pi(h, x, h->vec_r, 0, x);
      if (st != MFWH_OK) break;
      I.pi_applications++;
      launch_axpby(h->vec_r, 1.0, h->vec_b, -1.0, N, s);
    } else {
      launch_axpby(h->vec_r, 1.0, h->vec_b, 0.0, N, s);
    }
    h->total_launches++;
    double rr = 0.0;
    st = dots(h, h->vec_r, 1, h->vec_r, &rr);
    if (st != MFWH_OK) break;
    I.rel_residual = std::sqrt(rr) / bnorm;
    // inner solve (I - S) e = r with the handle's wave precision
    h->use32 = inner32;
    launch_axpby(h->vec_e, 0.0, h->vec_e, 0.0, N, s);
    h->total_launches++;
    bool conv = false;
    st = gmres_core(h, restart, inner_tol, max_iters - I.iterations, h->vec_e, h->vec_r, I, &conv,
                    relax_below);
    if (st != MFWH_OK) break;
    if (!conv) inner = MFWH_ERR_NOT_CONVERGED;
    launch_axpby(x, 1.0, h->vec_e, 1.0, N, s);   // x += e
    h->total_launches++;
    x_nonzero = true;
    I.refinements++;
  }
  h->use32 = inner32;
  for (int m = 0; m < h->nf; ++m) I.helmholtz_residual[m] = st == MFWH_OK ? r[m] : NAN;
  if (!on_dev) CK(cudaMemcpyAsync(v, x, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  mfwh_status ts = collect_timing(h);
  if (st != MFWH_OK) return st;
  if (ts != MFWH_OK) return ts;
  if (!done) {
    std::ostringstream os;
    os << "refinement stopped after " << I.refinements << " corrections and " << I.iterations
       << " Arnoldi steps"
       << (inner != MFWH_OK ? " (an inner GMRES solve did not reach its tolerance)" : "")
       << "; Helmholtz residual above the target " << target;
    return fail(MFWH_ERR_NOT_CONVERGED, os.str());
  }
  return MFWH_OK;
}

}  // namespace

extern "C" {

mfwh_status mfwh_solve_refined(mfwh_handle_t h, int restart, double inner_tol, int max_iters,
                               double target, int max_refinements, double* v,
                               mfwh_solve_info* info) {
  return refine_core(h, restart, inner_tol, max_iters, target, max_refinements, v, info, 0.0);
}

mfwh_status mfwh_solve_relaxed(mfwh_handle_t h, int restart, double inner_tol, double relax_below,
                               int max_iters, double target, int max_refinements, double* v,
                               mfwh_solve_info* info) {
  if (h && h->plan.precision == MFWH_PREC_FP64)
    return fail(MFWH_ERR_INVALID_ARG, "relaxed products need an FP32 handle");
  if (!(relax_below > 0.0 && relax_below < 1.0))
    return fail(MFWH_ERR_INVALID_ARG, "relax_below must be in (0, 1)");
  return refine_core(h, restart, inner_tol, max_iters, target, max_refinements, v, info,
                     relax_below);
}

mfwh_status mfwh_residual(mfwh_handle_t h, const double* v, double* r_out) {
  if (!h || !v || !r_out) return fail(MFWH_ERR_INVALID_ARG, "null argument");
  reset_timing(h);
  double* x = nullptr;
  bool on_dev = false;
  mfwh_status st = stage_in(h, v, &x, &on_dev);
  if (st != MFWH_OK) return st;
  return residual_dev(h, x, r_out);
}

mfwh_status mfwh_get_setup(mfwh_handle_t h, mfwh_setup* out) {
  if (!h || !out) return fail(MFWH_ERR_INVALID_ARG, "null argument");
  *out = h->plan.s;
  return MFWH_OK;
}

mfwh_status mfwh_last_timing(mfwh_handle_t h, double* step_ms, int64_t* step_launches,
                             int64_t* total_launches) {
  if (!h) return fail(MFWH_ERR_INVALID_ARG, "null handle");
  if (h->ev_used > 0) {
    CK(cudaEventSynchronize(h->ev[h->ev_used - 1]));
    mfwh_status st = collect_timing(h);
    if (st != MFWH_OK) return st;
  }
  if (step_ms) *step_ms = h->last_step_ms;
  if (step_launches) *step_launches = h->step_launches;
  if (total_launches) *total_launches = h->total_launches;
  return MFWH_OK;
}

mfwh_status mfwh_debug_bounds(mfwh_handle_t h, int64_t* count, int64_t* index, int64_t* extent,
                              int* line) {
  if (!h || !count) return fail(MFWH_ERR_INVALID_ARG, "null argument");
  BoundsFault r{};
#ifdef MFWH_BOUNDS_CHECK
  CK(cudaMemcpyAsync(&r, h->fault, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *count = (int64_t)r.count;
#else
  *count = -1;
#endif
  if (index) *index = r.index;
  if (extent) *extent = r.extent;
  if (line) *line = r.line;
  return MFWH_OK;
}

void mfwh_destroy(mfwh_handle_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  if (h->gstream) {
    cudaStreamSynchronize(h->gstream);
    cudaStreamDestroy(h->gstream);
  }
  for (auto& e : h->gev)
    if (e) cudaEventDestroy(e);
  if (h->g_in) cudaFree(h->g_in);
  if (h->g_out) cudaFree(h->g_out);
  if (h->vec_r) cudaFree(h->vec_r);
  if (h->vec_e) cudaFree(h->vec_e);
  double* bufs[] = {h->f,         h->Wa,      h->Wb,          h->Wc2,     h->Wp2,
                    h->d_wq,      h->d_cos,   h->q,           h->res_partial, h->res_out,
                    h->dot_partial, h->dot_out, h->vec_b,     h->vec_x,   h->basis};
  for (double* b : bufs)
    if (b) cudaFree(b);
  if (h->d_err) cudaFree(h->d_err);
  if (h->c2f) cudaFree(h->c2f);
  if (h->fault) cudaFree(h->fault);
  if (h->imp_mem) cudaFree(h->imp_mem);
  if (h->d_mgstate) cudaFree(h->d_mgstate);
  if (h->d_bar) cudaFree(h->d_bar);
  if (h->d_mgc) cudaFree(h->d_mgc);
  delete h->imp;
  float* fbufs[] = {h->f32, h->W32[0], h->W32[1], h->W32[2], h->W32[3], h->qs, h->qc,
                    h->wq32, h->fc32};
  for (float* b : fbufs)
    if (b) cudaFree(b);
  if (h->pinned) cudaFreeHost(h->pinned);
  for (auto& x : h->ev)
    if (x) cudaEventDestroy(x);
  delete h;
}

mfwh_status mfwh_set_wait_limit(mfwh_handle_t h, double seconds) {
  if (!h) return fail(MFWH_ERR_INVALID_ARG, "null handle");
  if (std::isnan(seconds) || seconds > 3600.0)
    return fail(MFWH_ERR_INVALID_ARG, "wait limit must be at most 3600 s");
  h->wait_s = seconds > 0.0 ? seconds : 2.0;
  return MFWH_OK;
}

mfwh_status mfwh_mg_stats(mfwh_handle_t h, int64_t* solves, int64_t* cycles,
                          int64_t* unconverged, int* levels, int reset) {
  if (!h) return fail(MFWH_ERR_INVALID_ARG, "null handle");
  if (!h->implicit) return fail(MFWH_ERR_INVALID_ARG, "not an implicit-time-stepping handle");
  if (levels) *levels = h->imp->nlev;
  CK(cudaMemcpyAsync(h->pinned, h->d_mgc, sizeof(MgCounters), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  MgCounters c;
  std::memcpy(&c, h->pinned, sizeof(c));
  if (solves) *solves = (int64_t)c.solves;
  if (cycles) *cycles = (int64_t)c.cycles;
  if (unconverged) *unconverged = (int64_t)c.unconverged;
  if (reset) {
    CK(cudaMemsetAsync(h->d_mgc, 0, sizeof(MgCounters), h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return MFWH_OK;
}

mfwh_status mfwh_set_graphs(mfwh_handle_t h, int enable) {
  if (!h) return fail(MFWH_ERR_INVALID_ARG, "null handle");
  CK(cudaStreamSynchronize(h->stream));
  if (h->gstream) CK(cudaStreamSynchronize(h->gstream));
  drop_graphs(h);
  if (enable && !h->g_in) {
    CK(cudaMalloc(&h->g_in, sizeof(double) * h->N));
    CK(cudaMalloc(&h->g_out, sizeof(double) * h->N));
    CK(cudaMemsetAsync(h->g_in, 0, sizeof(double) * h->N, h->stream));
    CK(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    for (auto& e : h->gev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaStreamSynchronize(h->stream));
  }
  h->graphs = enable != 0;
  return MFWH_OK;
}

mfwh_status mfwh_solve_batch(const mfwh_handle_t* handles, int count, int restart, double tol,
                             int max_iters, double* const* v, mfwh_solve_info* infos,
                             double* seconds) {
  if (!handles || !v || count < 1) return fail(MFWH_ERR_INVALID_ARG, "bad batch arguments");
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || !v[i]) return fail(MFWH_ERR_INVALID_ARG, "null handle or buffer in batch");
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return fail(MFWH_ERR_INVALID_ARG, "a handle appears twice");
  }
  std::vector<mfwh_status> status(count, MFWH_OK);
  std::vector<std::string> msg(count);
  std::vector<double> secs(count, 0.0);
  std::vector<mfwh_solve_info> local(count);
  std::atomic<int> ready{0};
  std::atomic<bool> go{false};
  std::chrono::steady_clock::time_point t0;   // written before `go`, read after it
  // One worker per explicit handle.  Implicit handles share one worker and run in sequence:
  // their step kernels are cooperative launches, which must not wait on each other's blocks.
  std::vector<std::vector<int>> groups;
  std::vector<int> imp;
  for (int i = 0; i < count; ++i) {
    if (handles[i]->implicit)
      imp.push_back(i);
    else
      groups.push_back({i});
  }
  if (!imp.empty()) groups.push_back(imp);
  auto work = [&](const std::vector<int>* idx) {
    cudaSetDevice(handles[(*idx)[0]]->device);
    ready.fetch_add(1);
    while (!go.load()) std::this_thread::yield();
    for (int i : *idx) {
      mfwh_handle_t h = handles[i];
      cudaSetDevice(h->device);
      mfwh_solve_info& I = infos ? infos[i] : local[i];
      status[i] = mfwh_solve_gmres(h, restart, tol, max_iters, 0.0, v[i], &I);
      secs[i] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (status[i] != MFWH_OK) msg[i] = g_error;
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(groups.size());
  for (auto& grp : groups) pool.emplace_back(work, &grp);
  while (ready.load() < (int)groups.size()) std::this_thread::yield();
  t0 = std::chrono::steady_clock::now();
  go.store(true);
  for (auto& t : pool) t.join();
  if (seconds)
    for (int i = 0; i < count; ++i) seconds[i] = secs[i];
  for (int i = 0; i < count; ++i)
    if (status[i] != MFWH_OK && status[i] != MFWH_ERR_NOT_CONVERGED) {
      set_error("problem " + std::to_string(i) + ": " + msg[i]);
      return status[i];
    }
  for (int i = 0; i < count; ++i)
    if (status[i] != MFWH_OK) {
      set_error("problem " + std::to_string(i) + ": " + msg[i]);
      return status[i];
    }
  return MFWH_OK;
}

// ---- lockstep batch: one graph launch per application of the map across the batch ----

}  // extern "C"

namespace {

// The wave solve of one handle captured (not instantiated) on its staging buffers: forced = 1,
// no input: g_out = Pi(0); forced = 0 with input: g_out = g_in - S g_in.  *steps / *total: the
// step-kernel and all-kernel launches one replay performs.
mfwh_status capture_child(mfwh_handle_t h, cudaStream_t cs, int forced, cudaGraph_t* out,
                          int64_t* steps, int64_t* total) {
  const int saved_ev = h->ev_used;
  const int64_t sl = h->step_launches, tl = h->total_launches;
  h->ev_used = (int)h->ev.size();   // no timing events inside the graph
  cudaStream_t user = h->stream;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  h->stream = cs;
  mfwh_status st = forced ? apply_pi_direct(h, nullptr, h->g_out, 1, nullptr)
                          : apply_pi_direct(h, h->g_in, h->g_out, 0, h->g_in);
  h->stream = user;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  h->ev_used = saved_ev;
  *steps = h->step_launches - sl;
  *total = h->total_launches - tl;
  h->step_launches = sl;
  h->total_launches = tl;
  if (st != MFWH_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture (batch)");
  *out = g;
  return MFWH_OK;
}

// GMRES(restart) state of one problem of a lockstep batch (the steps of gmres_core, split at
// each application of the map).
struct LockstepProblem {
  mfwh_handle_t h = nullptr;
  cudaStream_t user_stream = nullptr;
  bool swapped = false;                 // h->stream temporarily set to the batch stream
  double* x = nullptr;                  // device iterate
  double* v_user = nullptr;
  bool on_dev = false;
  mfwh_solve_info* I = nullptr;
  std::vector<double> H, cs, sn, g, y, hcol, h2;
  double bnorm = 0.0, res = 0.0;
  int j = 0;                            // Arnoldi index in the current cycle
  bool x_nonzero = false, converged = false, done = false, cycle_start = false;
  mfwh_status st = MFWH_OK;
  std::string msg;
  double secs = 0.0;
  cudaGraph_t child[2] = {nullptr, nullptr};   // [0]: A v on g_in, [1]: Pi(0)
  int64_t child_steps[2] = {0, 0}, child_total[2] = {0, 0};
  double* product_dest = nullptr;       // where this round's product goes
};

void lockstep_fail(LockstepProblem& P, mfwh_status st) {
  P.st = st;
  P.msg = g_error;
  P.done = true;
}

// Parent graph with one child node per listed problem (variant k), instantiated.
mfwh_status batch_graph(std::vector<LockstepProblem>& Ps, const std::vector<int>& idx, int k,
                        cudaGraphExec_t* exec) {
  cudaGraph_t parent = nullptr;
  CK(cudaGraphCreate(&parent, 0));
  for (int i : idx) {
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, Ps[i].child[k]);
    if (e != cudaSuccess) {
      cudaGraphDestroy(parent);
      return cuda_fail(e, "cudaGraphAddChildGraphNode");
    }
  }
  cudaError_t e = cudaGraphInstantiate(exec, parent, 0);
  cudaGraphDestroy(parent);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batch)");
  return MFWH_OK;
}

// Queue the dot products <V_i, w> (i < k) of problem P into its pinned buffer at offset off.
mfwh_status queue_dots(LockstepProblem& P, const double* V, int k, const double* w, int off) {
  mfwh_handle_t h = P.h;
  launch_multidot(V, h->N, k, w, h->N, h->dot_partial, h->dot_out, h->stream);
  h->total_launches += multidot_launches(k);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->pinned + off, h->dot_out, sizeof(double) * k, cudaMemcpyDeviceToHost,
                     h->stream));
  return MFWH_OK;
}

}  // namespace

extern "C" {

mfwh_status mfwh_solve_batch_graph(const mfwh_handle_t* handles, int count, int restart,
                                   double tol, int max_iters, double* const* v,
                                   mfwh_solve_info* infos, double* seconds, void* stream) {
  if (!handles || !v || count < 1) return fail(MFWH_ERR_INVALID_ARG, "bad batch arguments");
  if (restart < 1 || restart > kMaxRestart || max_iters < 1 || !(tol >= 0.0))
    return fail(MFWH_ERR_INVALID_ARG, "bad restart, max_iters or tol");
  if (restart > max_iters) restart = max_iters;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || !v[i]) return fail(MFWH_ERR_INVALID_ARG, "null handle or buffer in batch");
    if (handles[i]->implicit)
      return fail(MFWH_ERR_INVALID_ARG, "lockstep batches take explicit handles only");
    if (handles[i]->device != dev)
      return fail(MFWH_ERR_INVALID_ARG, "every handle must be on the current device");
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return fail(MFWH_ERR_INVALID_ARG, "a handle appears twice");
  }
  cudaStream_t bs = static_cast<cudaStream_t>(stream);
  std::vector<LockstepProblem> Ps(count);
  std::vector<mfwh_solve_info> local(count);
  mfwh_status st = MFWH_OK;
  for (int i = 0; i < count; ++i) {
    LockstepProblem& P = Ps[i];
    P.h = handles[i];
    P.v_user = v[i];
    P.I = infos ? &infos[i] : &local[i];
    const int cap = P.I->history_capacity;
    double* hist = P.I->history;
    *P.I = mfwh_solve_info{};
    P.I->history_capacity = cap;
    P.I->history = hist;
    P.I->rel_residual = NAN;
    if (!P.h->graphs) {
      st = mfwh_set_graphs(P.h, 1);
      if (st != MFWH_OK) return st;
    }
    st = ensure_basis(P.h, restart + 1);
    if (st != MFWH_OK) return st;
    reset_timing(P.h);
    P.H.assign((restart + 1) * restart, 0.0);
    P.cs.assign(restart, 0.0);
    P.sn.assign(restart, 0.0);
    P.g.assign(restart + 1, 0.0);
    P.y.assign(restart, 0.0);
    P.hcol.assign(restart + 1, 0.0);
    P.h2.assign(restart + 1, 0.0);
  }
  // Every handle's earlier work completes before the batch stream uses its buffers.
  cudaEvent_t ev = nullptr;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  for (auto& P : Ps) {
    CK(cudaEventRecord(ev, P.h->stream));
    CK(cudaStreamWaitEvent(bs, ev, 0));
  }
  cudaStream_t cap = nullptr;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  auto restore = [&]() {
    for (auto& P : Ps) {
      if (P.swapped) P.h->stream = P.user_stream;
      P.swapped = false;
      for (auto& c : P.child)
        if (c) cudaGraphDestroy(c);
    }
    cudaEventRecord(ev, bs);
    for (auto& P : Ps) cudaStreamWaitEvent(P.h->stream, ev, 0);
    cudaEventDestroy(ev);
    if (cap) cudaStreamDestroy(cap);
  };
  for (auto& P : Ps) {
    for (int k = 0; k < 2 && st == MFWH_OK; ++k)
      st = capture_child(P.h, cap, k, &P.child[k], &P.child_steps[k], &P.child_total[k]);
    if (st != MFWH_OK) {
      restore();
      return st;
    }
    P.user_stream = P.h->stream;
    P.h->stream = bs;
    P.swapped = true;
    st = stage_in(P.h, P.v_user, &P.x, &P.on_dev);
    if (st != MFWH_OK) {
      restore();
      return st;
    }
  }
  const auto t0 = std::chrono::steady_clock::now();
  auto elapsed = [&]() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  };
  auto sync = [&]() -> mfwh_status {
    CK(cudaStreamSynchronize(bs));
    return MFWH_OK;
  };
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  std::vector<int> exec_set[2];
  auto launch_round = [&](const std::vector<int>& idx, int k) -> mfwh_status {
    if (!exec[k] || exec_set[k] != idx) {
      if (exec[k]) cudaGraphExecDestroy(exec[k]);
      exec[k] = nullptr;
      mfwh_status s2 = batch_graph(Ps, idx, k, &exec[k]);
      if (s2 != MFWH_OK) return s2;
      exec_set[k] = idx;
    }
    CK(cudaGraphLaunch(exec[k], bs));
    for (int i : idx) {
      LockstepProblem& P = Ps[i];
      P.h->step_launches += P.child_steps[k];
      P.h->total_launches += P.child_total[k];
      P.I->pi_applications++;
    }
    return MFWH_OK;
  };

  // Round 0: b = Pi(0) for every problem, ||b||, ||x||.
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) all[i] = i;
  st = launch_round(all, 1);
  for (auto& P : Ps) {
    if (st != MFWH_OK) break;
    CK(cudaMemcpyAsync(P.h->vec_b, P.h->g_out, sizeof(double) * P.h->N,
                       cudaMemcpyDeviceToDevice, bs));
    st = queue_dots(P, P.h->vec_b, 1, P.h->vec_b, 0);
    if (st == MFWH_OK) st = queue_dots(P, P.x, 1, P.x, 1);
  }
  if (st == MFWH_OK) st = sync();
  for (auto& P : Ps) {
    if (st != MFWH_OK) break;
    P.bnorm = std::sqrt(P.h->pinned[0]);
    const double xx = P.h->pinned[1];
    if (!std::isfinite(P.bnorm) || !std::isfinite(xx)) {
      set_error("non-finite right-hand side or initial guess");
      lockstep_fail(P, MFWH_ERR_NONFINITE);
      continue;
    }
    P.x_nonzero = xx > 0.0;
    P.cycle_start = true;
    if (P.bnorm == 0.0) {
      launch_axpby(P.x, 0.0, P.x, 0.0, P.h->N, bs);
      P.converged = P.done = true;
      P.I->rel_residual = 0.0;
    }
  }

  // Arnoldi rounds: every active problem needs exactly one product A u (u = x at the start
  // of a cycle from a non-zero iterate, else its newest basis vector).
  while (st == MFWH_OK) {
    Range range("mfwh: batch round");
    // start of cycle from x = 0: V_0 = b without a product
    for (auto& P : Ps) {
      if (P.done || !P.cycle_start || P.x_nonzero) continue;
      P.I->restarts++;
      launch_axpby(P.h->basis, 1.0, P.h->vec_b, 0.0, P.h->N, bs);
      P.h->total_launches++;
      st = queue_dots(P, P.h->basis, 1, P.h->basis, 0);
      if (st != MFWH_OK) break;
    }
    if (st != MFWH_OK || (st = sync()) != MFWH_OK) break;
    for (auto& P : Ps) {
      if (P.done || !P.cycle_start || P.x_nonzero) continue;
      const double beta = std::sqrt(P.h->pinned[0]);
      P.cycle_start = false;
      P.I->rel_residual = beta / P.bnorm;
      if (!std::isfinite(beta)) {
        set_error("non-finite Krylov residual");
        lockstep_fail(P, MFWH_ERR_NONFINITE);
        continue;
      }
      if (P.I->rel_residual < tol) {
        P.converged = P.done = true;
        continue;
      }
      launch_axpby(P.h->basis, 1.0 / beta, P.h->basis, 0.0, P.h->N, bs);
      P.h->total_launches++;
      std::fill(P.g.begin(), P.g.end(), 0.0);
      P.g[0] = beta;
      P.res = beta;
      P.j = 0;
    }
    std::vector<int> active;
    for (int i = 0; i < count; ++i)
      if (!Ps[i].done) active.push_back(i);
    if (active.empty()) break;
    // inputs into the staging buffers, one graph launch, products out
    for (int i : active) {
      LockstepProblem& P = Ps[i];
      const double* u = P.cycle_start ? P.x : P.h->basis + (int64_t)P.j * P.h->N;
      P.product_dest = P.cycle_start ? P.h->basis : P.h->basis + (int64_t)(P.j + 1) * P.h->N;
      CK(cudaMemcpyAsync(P.h->g_in, u, sizeof(double) * P.h->N, cudaMemcpyDeviceToDevice, bs));
    }
    st = launch_round(active, 0);
    if (st != MFWH_OK) break;
    for (int i : active) {
      LockstepProblem& P = Ps[i];
      CK(cudaMemcpyAsync(P.product_dest, P.h->g_out, sizeof(double) * P.h->N,
                         cudaMemcpyDeviceToDevice, bs));
      if (P.cycle_start) {   // r = b - (x - S x)
        P.I->restarts++;
        launch_axpby(P.h->basis, 1.0, P.h->vec_b, -1.0, P.h->N, bs);
        P.h->total_launches++;
        st = queue_dots(P, P.h->basis, 1, P.h->basis, 0);
      } else {               // classical Gram-Schmidt, first pass
        P.I->iterations++;
        st = queue_dots(P, P.h->basis, P.j + 1, P.product_dest, 0);
      }
      if (st != MFWH_OK) break;
    }
    if (st != MFWH_OK || (st = sync()) != MFWH_OK) break;
    // second Gram-Schmidt pass (Arnoldi problems)
    for (int i : active) {
      LockstepProblem& P = Ps[i];
      if (P.cycle_start) continue;
      std::memcpy(P.hcol.data(), P.h->pinned, sizeof(double) * (P.j + 1));
      launch_multi_axpy(P.product_dest, P.h->basis, P.h->N, P.j + 1, P.hcol.data(), P.h->N, bs);
      P.h->total_launches += multi_axpy_launches(P.j + 1);
      st = queue_dots(P, P.h->basis, P.j + 1, P.product_dest, 0);
      if (st != MFWH_OK) break;
    }
    if (st != MFWH_OK || (st = sync()) != MFWH_OK) break;
    for (int i : active) {
      LockstepProblem& P = Ps[i];
      if (P.cycle_start) continue;
      std::memcpy(P.h2.data(), P.h->pinned, sizeof(double) * (P.j + 1));
      launch_multi_axpy(P.product_dest, P.h->basis, P.h->N, P.j + 1, P.h2.data(), P.h->N, bs);
      P.h->total_launches += multi_axpy_launches(P.j + 1);
      for (int k = 0; k <= P.j; ++k) P.hcol[k] += P.h2[k];
      st = queue_dots(P, P.product_dest, 1, P.product_dest, 0);
      if (st != MFWH_OK) break;
    }
    if (st != MFWH_OK || (st = sync()) != MFWH_OK) break;
    // Givens rotations, convergence, end of cycle
    for (int i : active) {
      LockstepProblem& P = Ps[i];
      const int64_t N = P.h->N;
      if (P.cycle_start) {
        const double beta = std::sqrt(P.h->pinned[0]);
        P.cycle_start = false;
        if (!std::isfinite(beta)) {
          set_error("non-finite Krylov residual");
          lockstep_fail(P, MFWH_ERR_NONFINITE);
          continue;
        }
        P.I->rel_residual = beta / P.bnorm;
        if (P.I->rel_residual < tol) {
          P.converged = P.done = true;
          continue;
        }
        launch_axpby(P.h->basis, 1.0 / beta, P.h->basis, 0.0, N, bs);
        P.h->total_launches++;
        std::fill(P.g.begin(), P.g.end(), 0.0);
        P.g[0] = beta;
        P.res = beta;
        P.j = 0;
        continue;
      }
      const int j = P.j;
      const double hnext = std::sqrt(P.h->pinned[0]);
      if (!std::isfinite(hnext)) {
        set_error("non-finite Arnoldi vector");
        lockstep_fail(P, MFWH_ERR_NONFINITE);
        continue;
      }
      std::vector<double>& hc = P.hcol;
      for (int k = 0; k < j; ++k) {
        const double t = P.cs[k] * hc[k] + P.sn[k] * hc[k + 1];
        hc[k + 1] = -P.sn[k] * hc[k] + P.cs[k] * hc[k + 1];
        hc[k] = t;
      }
      const double r = std::hypot(hc[j], hnext);
      P.cs[j] = r > 0.0 ? hc[j] / r : 1.0;
      P.sn[j] = r > 0.0 ? hnext / r : 0.0;
      hc[j] = r;
      for (int k = 0; k <= j; ++k) P.H[k * restart + j] = hc[k];
      P.g[j + 1] = -P.sn[j] * P.g[j];
      P.g[j] = P.cs[j] * P.g[j];
      P.res = std::fabs(P.g[j + 1]);
      mfwh_solve_info& I = *P.I;
      if (I.history && I.history_len < I.history_capacity)
        I.history[I.history_len++] = P.res / P.bnorm;
      const bool end = P.res / P.bnorm < tol || I.iterations >= max_iters || hnext == 0.0 ||
                       j + 1 == restart;
      if (!end) {
        launch_axpby(P.product_dest, 1.0 / hnext, P.product_dest, 0.0, N, bs);
        P.h->total_launches++;
        P.j = j + 1;
        continue;
      }
      // y = R^{-1} g, x += V y
      const int jd = j + 1;
      for (int k = jd - 1; k >= 0; --k) {
        double acc = P.g[k];
        for (int l = k + 1; l < jd; ++l) acc -= P.H[k * restart + l] * P.y[l];
        P.y[k] = acc / P.H[k * restart + k];
      }
      for (int k = 0; k < jd; ++k) P.y[k] = -P.y[k];   // multi_axpy subtracts
      launch_multi_axpy(P.x, P.h->basis, N, jd, P.y.data(), N, bs);
      P.h->total_launches += multi_axpy_launches(jd);
      P.x_nonzero = true;
      I.rel_residual = P.res / P.bnorm;
      if (I.rel_residual < tol) {
        P.converged = P.done = true;
      } else if (I.iterations >= max_iters) {
        P.done = true;
      } else {
        P.cycle_start = true;
      }
    }
    for (int i : active)
      if (Ps[i].done) Ps[i].secs = elapsed();
  }
  for (auto& e2 : exec)
    if (e2) cudaGraphExecDestroy(e2);
  // Helmholtz residuals and results back to the caller's buffers.
  if (st == MFWH_OK) {
    for (auto& P : Ps) {
      if (P.st != MFWH_OK) continue;
      double r[MFWH_MAX_NF];
      mfwh_status rs = residual_dev(P.h, P.x, r);
      for (int m = 0; m < P.h->nf; ++m) P.I->helmholtz_residual[m] = rs == MFWH_OK ? r[m] : NAN;
      if (rs != MFWH_OK) lockstep_fail(P, rs);
      if (!P.on_dev)
        CK(cudaMemcpyAsync(P.v_user, P.x, sizeof(double) * P.h->N, cudaMemcpyDeviceToHost, bs));
    }
    if (st == MFWH_OK) st = sync();
    // a bounded wait inside a wave kernel that ran out fails that problem
    for (auto& P : Ps) {
      if (st != MFWH_OK || P.st != MFWH_OK) continue;
      mfwh_status ts = collect_timing(P.h);
      if (ts != MFWH_OK) lockstep_fail(P, ts);
    }
  }
  const double t_end = elapsed();
  restore();
  if (st != MFWH_OK) return st;
  for (int i = 0; i < count; ++i) {
    if (Ps[i].secs == 0.0) Ps[i].secs = t_end;
    if (seconds) seconds[i] = Ps[i].secs;
  }
  for (int i = 0; i < count; ++i)
    if (Ps[i].st != MFWH_OK) {
      set_error("problem " + std::to_string(i) + ": " + Ps[i].msg);
      return Ps[i].st;
    }
  for (int i = 0; i < count; ++i)
    if (!Ps[i].converged) {
      std::ostringstream os;
      os << "problem " << i << ": GMRES stopped after " << Ps[i].I->iterations
         << " iterations at relative residual " << Ps[i].I->rel_residual;
      return fail(MFWH_ERR_NOT_CONVERGED, os.str());
    }
  return MFWH_OK;
}

mfwh_status mfwh_autotune(const mfwh_problem* prob, void* stream, int* time_block,
                          int* tile_shape, double* ms_per_step) {
  if (!prob || !time_block || !tile_shape) return fail(MFWH_ERR_INVALID_ARG, "null argument");
  Plan P;
  mfwh_status st = plan_with_field(prob, &P);
  if (st != MFWH_OK) return st;
  if (P.time_stepping == MFWH_TIME_IMPLICIT) {   // one step per launch; nothing to choose
    *time_block = 1;
    *tile_shape = 0;
    if (ms_per_step) *ms_per_step = 0.0;
    return MFWH_OK;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  using Key = std::tuple<int, int, int64_t, int64_t, int64_t, int, int, int>;
  static std::mutex mu;
  static std::map<Key, std::tuple<int, int, double>> cache;
  const Key key{dev, P.dim, P.n[0], P.n[1], P.dim == 3 ? P.n[2] : 0, P.s.nf, P.precision,
                P.c2_field ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *time_block = std::get<0>(it->second);
      *tile_shape = std::get<1>(it->second);
      if (ms_per_step) *ms_per_step = std::get<2>(it->second);
      return MFWH_OK;
    }
  }
  std::vector<std::pair<int, int>> cand;
  if (P.order == 4 || P.c2_field || (P.dim == 3 && P.precision == MFWH_PREC_FP64)) {
    cand = {{1, 0}};
  } else if (P.dim == 3) {
    cand = {{1, 0}, {2, 0}, {4, 0}};
  } else if (P.precision == MFWH_PREC_FP64) {
    cand = {{1, 0}, {2, 5}, {3, 5}, {4, 5}, {4, 4}, {4, 3}, {8, 3}};
  } else {
    for (int T : {4, 8, 16})
      for (int shape : {0, 1, 2}) cand.push_back({T, shape});
  }
  // Each candidate times the first tune_n steps of a homogeneous wave solve (whole launches
  // for every depth), after one untimed warm-up of the same length.
  const int tune_n = std::min(P.s.n_t, 96);
  double best = 1e300;
  int best_tb = cand[0].first, best_shape = cand[0].second;
  for (auto [tb, shape] : cand) {
    mfwh_problem q = *prob;
    q.time_block = tb;
    q.tile_shape = shape;
    mfwh_handle_t h = nullptr;
    st = mfwh_create(&q, stream, &h);
    if (st != MFWH_OK) return st;
    h->tune_steps = tune_n;
    double ms = 1e300;
    for (int rep = 0; rep < 3 && st == MFWH_OK; ++rep) {
      reset_timing(h);
      st = apply_pi(h, nullptr, h->vec_b, 0, nullptr);
      if (st == MFWH_OK) st = collect_timing_sync(h);
      if (rep > 0) ms = std::min(ms, h->last_step_ms);
    }
    mfwh_destroy(h);
    if (st != MFWH_OK) return st;
    if (ms < best) {
      best = ms;
      best_tb = tb;
      best_shape = shape;
    }
  }
  const double per_step = best / tune_n;
  {
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = {best_tb, best_shape, per_step};
  }
  *time_block = best_tb;
  *tile_shape = best_shape;
  if (ms_per_step) *ms_per_step = per_step;
  return MFWH_OK;
}

mfwh_status mfwh_warm_start_data(mfwh_handle_t h, double omega_scale, const double* v,
                                 float* x_out, float* t_out) {
  if (!h || !v || !x_out || !t_out || !(omega_scale > 0.0))
    return fail(MFWH_ERR_INVALID_ARG, "bad warm-start data arguments");
  if (h->plan.dim != 2) return fail(MFWH_ERR_INVALID_ARG, "the warm start is for 2D grids");
  if (!is_device_ptr(v) || !is_device_ptr(x_out) || !is_device_ptr(t_out))
    return fail(MFWH_ERR_INVALID_ARG, "mfwh_warm_start_data takes device pointers");
  double omega[MFWH_MAX_NF];
  for (int m = 0; m < h->nf; ++m) omega[m] = std::sqrt(h->omega2[m]);
  mfwh_status st = cnn_ws_data(h->f, v, omega, h->nf, (int)h->geom.ny + 1, (int)h->geom.nx + 1,
                               omega_scale, x_out, t_out, h->res_out, h->stream);
  if (st != MFWH_OK) return st;
  CK(cudaStreamSynchronize(h->stream));
  return MFWH_OK;
}

mfwh_status mfwh_warm_start(mfwh_handle_t h, mfwh_cnn_t net, double omega_scale, double* v,
                            double* ratio_out) {
  if (!h || !net || !v || !(omega_scale > 0.0))
    return fail(MFWH_ERR_INVALID_ARG, "bad warm-start arguments");
  if (h->plan.dim != 2) return fail(MFWH_ERR_INVALID_ARG, "the warm start is for 2D grids");
  double* x = nullptr;
  bool on_dev = false;
  mfwh_status st = stage_in(h, v, &x, &on_dev);
  if (st != MFWH_OK) return st;
  double omega[MFWH_MAX_NF];
  for (int m = 0; m < h->nf; ++m) omega[m] = std::sqrt(h->omega2[m]);
  st = cnn_ws_predict(net, h->f, omega, h->nf, (int)h->geom.ny + 1, (int)h->geom.nx + 1,
                      omega_scale, x, h->stream);
  if (st != MFWH_OK) return st;
  // Amplitude of each predicted shape phi_m: alpha_m = <A phi_m, f_m> / <A phi_m, A phi_m>
  // with A = L_h + omega_m^2 minimises the L2 Helmholtz residual ||f_m - alpha A phi_m||.
  if (!h->vec_r) CK(cudaMalloc(&h->vec_r, sizeof(double) * h->N));
  if (!h->vec_e) CK(cudaMalloc(&h->vec_e, sizeof(double) * h->N));
  CK(cudaMemsetAsync(h->vec_e, 0, sizeof(double) * h->N, h->stream));
  // defect of phi against a zero forcing is -A phi at interior points, 0 on the boundary
  launch_residual_field(h->nf, h->geom, x, h->vec_e, h->omega2, h->plan.c2_lo, h->plan.c2_hi,
                        h->inv_h2, h->vec_r, h->stream);
  launch_axpby(h->vec_r, 0.0, h->vec_r, -1.0, h->N, h->stream);
  h->total_launches += 2;
  const int64_t P = h->P;
  for (int m = 0; m < h->nf; ++m) {
    double af = 0.0, aa = 0.0;
    const double* Am = h->vec_r + m * P;
    launch_multidot(Am, P, 1, h->f + m * P, P, h->dot_partial, h->dot_out, h->stream);
    CK(cudaMemcpyAsync(h->pinned, h->dot_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    af = h->pinned[0];
    launch_multidot(Am, P, 1, Am, P, h->dot_partial, h->dot_out, h->stream);
    CK(cudaMemcpyAsync(h->pinned, h->dot_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    aa = h->pinned[0];
    const double alpha = (aa > 0.0 && std::isfinite(af / aa)) ? af / aa : 0.0;
    launch_axpby(x + m * P, alpha, x + m * P, 0.0, P, h->stream);
  }
  // Keep the prediction only if it lowers GMRES's initial residual: ||b - (x - S x)|| < ||b||
  // with b = Pi(0) (two applications of Pi, in the handle's precision).
  st = apply_pi(h, nullptr, h->vec_b, 1, nullptr);
  if (st != MFWH_OK) return st;
  st = apply_pi(h, x, h->vec_e, 0, x);                       // vec_e = x - S x
  if (st != MFWH_OK) return st;
  launch_axpby(h->vec_e, 1.0, h->vec_b, -1.0, h->N, h->stream);   // b - (x - S x)
  h->total_launches++;
  double bb = 0.0, rr = 0.0;
  st = dots(h, h->vec_b, 1, h->vec_b, &bb);
  if (st == MFWH_OK) st = dots(h, h->vec_e, 1, h->vec_e, &rr);
  if (st != MFWH_OK) return st;
  double ratio = bb > 0.0 ? std::sqrt(rr / bb) : 1.0;
  const bool better = std::isfinite(ratio) && ratio < 1.0;
  if (!better) {
    launch_axpby(x, 0.0, x, 0.0, h->N, h->stream);
    ratio = 1.0;
  }
  if (ratio_out) *ratio_out = ratio;
  if (!on_dev) CK(cudaMemcpyAsync(v, x, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return better ? MFWH_OK : MFWH_ERR_NOT_CONVERGED;
}

}  // extern "C"

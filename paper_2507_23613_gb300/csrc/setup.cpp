// Host set-up of an MFWH problem in FP64: time step, adjusted frequencies,
// period counts, quadrature weights, filter parameters (traditional or the
// least-squares Algorithm 2), filter weights, B and B^{-1}.
//
// Paper sections followed: "Governing equations" (eq. TbarDef), "Filter
// parameters from an optimization problem" (eq. yt, eq. muNice, eq.
// LambdaRange, Algorithm 2), "Discretizing the wave equation and filter"
// (eq. omegaImplicit, eq. pDefQ, eq. DefNI, eq. betadDefA, eq. origParamAdjust,
// Section "Time-step determination").
#include <algorithm>
#include <cmath>
#include <cstring>
#include <sstream>

#include "internal.h"

namespace mfwh {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMaxCondB = 1e12;   // B is applied every iteration
constexpr double kMaxCondG = 1e15;   // G only parametrises the constraint family

// ---- small dense linear algebra (row-major) --------------------------------

// Solve A X = Bm in place (A n x n, Bm n x k) by Gaussian elimination with
// partial pivoting.  Returns false if a pivot is exactly zero.
bool lu_solve(int n, std::vector<double> A, std::vector<double>& Bm, int k) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[piv * n + j]);
      for (int j = 0; j < k; ++j) std::swap(Bm[c * k + j], Bm[piv * k + j]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0) continue;
      for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
      for (int j = 0; j < k; ++j) Bm[r * k + j] -= f * Bm[c * k + j];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    for (int j = 0; j < k; ++j) {
      double s = Bm[c * k + j];
      for (int i = c + 1; i < n; ++i) s -= A[c * n + i] * Bm[i * k + j];
      Bm[c * k + j] = s / A[c * n + c];
    }
  }
  return true;
}

double norm1(int n, const std::vector<double>& A) {
  double best = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += std::fabs(A[i * n + j]);
    best = std::max(best, s);
  }
  return best;
}

// Inverse and 1-norm condition number of a small square matrix.
bool invert(int n, const std::vector<double>& A, std::vector<double>& Ainv, double* cond) {
  Ainv.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) Ainv[i * n + i] = 1.0;
  if (!lu_solve(n, A, Ainv, n)) return false;
  *cond = norm1(n, A) * norm1(n, Ainv);
  return std::isfinite(*cond);
}

// Least-squares solution of min ||M x - b||_2 (M rows x cols, rows >= cols) by
// Householder QR.  Returns false if R has a (relatively) zero diagonal entry.
bool householder_lstsq(int rows, int cols, std::vector<double> M, std::vector<double> b,
                       std::vector<double>& x) {
  double scale = 0.0;
  for (double v : M) scale = std::max(scale, std::fabs(v));
  for (int c = 0; c < cols; ++c) {
    double nrm = 0.0;
    for (int r = c; r < rows; ++r) nrm += M[r * cols + c] * M[r * cols + c];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) return false;
    double alpha = M[c * cols + c] > 0 ? -nrm : nrm;
    std::vector<double> v(rows - c);
    for (int r = c; r < rows; ++r) v[r - c] = M[r * cols + c];
    v[0] -= alpha;
    double vnorm2 = 0.0;
    for (double e : v) vnorm2 += e * e;
    if (vnorm2 == 0.0) continue;
    for (int j = c; j < cols; ++j) {        // M <- (I - 2 v v^T / v^T v) M
      double d = 0.0;
      for (int r = c; r < rows; ++r) d += v[r - c] * M[r * cols + j];
      d = 2.0 * d / vnorm2;
      for (int r = c; r < rows; ++r) M[r * cols + j] -= d * v[r - c];
    }
    double d = 0.0;
    for (int r = c; r < rows; ++r) d += v[r - c] * b[r];
    d = 2.0 * d / vnorm2;
    for (int r = c; r < rows; ++r) b[r] -= d * v[r - c];
  }
  x.assign(cols, 0.0);
  for (int c = cols - 1; c >= 0; --c) {
    double rcc = M[c * cols + c];
    if (std::fabs(rcc) <= 1e-14 * scale) return false;
    double s = b[c];
    for (int j = c + 1; j < cols; ++j) s -= M[c * cols + j] * x[j];
    x[c] = s / rcc;
  }
  return true;
}

// Weighted cosine sums of one filter: f(lam) = sum_n g[n] cos(lam t_n) and
// f'(lam) = -sum_n g[n] t_n sin(lam t_n).
struct CosineSum {
  std::vector<double> g;
  double dt;
  double value(double lam) const {
    double s = 0.0;
    for (size_t n = 0; n < g.size(); ++n) s += g[n] * std::cos(lam * (double)n * dt);
    return s;
  }
  double slope(double lam) const {
    double s = 0.0;
    for (size_t n = 0; n < g.size(); ++n) {
      double t = (double)n * dt;
      s -= g[n] * t * std::sin(lam * t);
    }
    return s;
  }
};

// N_{p,m} = floor(T_f / T_m) = floor(N_p omega_m / omega_1) (eq. TbarDef) for the given
// frequencies, exactly: their floating-point quotient can round up to an integer that the
// exact ratio stays just below.  The quotient's floor is corrected by comparing N_p omega_m
// with k omega_1 in long double, where both products are exact while N_p and k stay below
// 2^11 (at most 53 + 11 significant bits).
int period_count(int n_p, double omega_m, double omega_1) {
  long k = (long)std::floor(n_p * (omega_m / omega_1));
  const long double num = (long double)n_p * (long double)omega_m;
  while (k > 0 && (long double)k * (long double)omega_1 > num) --k;
  while ((long double)(k + 1) * (long double)omega_1 <= num) ++k;
  return (int)k;
}

}  // namespace

void trapezoid_weights(int n_t, double dt, int nf, const double* t_fm, double* sigma) {
  // Composite trapezoid rule up to t_k = k dt <= T_{f,m} < t_{k+1}; on the last,
  // partial interval the integrand is the line through t_k and t_{k+1}.  With the
  // overshoot fraction beta = (t_{k+1} - T_{f,m}) / dt this adds weight
  // dt/2 (2 - beta^2) at t_k and dt/2 (1 - beta)^2 at t_{k+1}.
  std::fill(sigma, sigma + (size_t)(n_t + 1) * nf, 0.0);
  for (int m = 0; m < nf; ++m) {
    int k = (int)std::floor(t_fm[m] / dt);
    if (k > n_t) k = n_t;
    double beta = (dt * (k + 1) - t_fm[m]) / dt;
    for (int n = 1; n < k; ++n) sigma[(size_t)n * nf + m] = dt;
    if (k == 0) {
      // T_{f,m} < dt: only the partial panel [0, T_{f,m}] contributes.
      sigma[m] = 0.5 * dt * (1.0 - beta * beta);
    } else {
      sigma[m] = 0.5 * dt;
      sigma[(size_t)k * nf + m] = (k < n_t) ? 0.5 * dt * (2.0 - beta * beta) : 0.5 * dt;
    }
    if (k < n_t) sigma[(size_t)(k + 1) * nf + m] = 0.5 * dt * (1.0 - beta) * (1.0 - beta);
  }
}

mfwh_status optimise_parameters(int nf, const double* omega, int n_p, int n_t, int n_delta,
                                double c_delta, double* params, double* lam_max_out,
                                int* n_lambda_out) {
  // Algorithm 2 with the trapezoid-rule filter functions of the wave-solve grid.
  std::vector<double> t_fm(nf);
  std::vector<int> n_pm(nf);
  double t_f = 0.0;
  for (int m = 0; m < nf; ++m) {
    n_pm[m] = period_count(n_p, omega[m], omega[0]);
    t_fm[m] = n_pm[m] * (2.0 * kPi / omega[m]);
    t_f = std::max(t_f, t_fm[m]);
  }
  const double dt = t_f / n_t;
  std::vector<double> sigma((size_t)(n_t + 1) * nf);
  trapezoid_weights(n_t, dt, nf, t_fm.data(), sigma.data());

  // Weighted kernels of the three component functions (eq. compFuncs, discrete).
  std::vector<CosineSum> fa(nf), fc(nf), fs(nf);
  for (int m = 0; m < nf; ++m) {
    fa[m].dt = fc[m].dt = fs[m].dt = dt;
    fa[m].g.resize(n_t + 1);
    fc[m].g.resize(n_t + 1);
    fs[m].g.resize(n_t + 1);
    for (int n = 0; n <= n_t; ++n) {
      double wgt = 2.0 / t_fm[m] * sigma[(size_t)n * nf + m];
      double t = n * dt;
      fa[m].g[n] = wgt;
      fc[m].g[n] = wgt * std::cos(omega[m] * t);
      fs[m].g[n] = wgt * std::sin(omega[m] * t);
    }
  }

  // Constraints: G y = z - H x_a with y = [x_c; x_s] (eq. yt).
  const int n2 = 2 * nf;
  std::vector<double> G(n2 * n2), H(n2 * nf), z(n2, 0.0);
  for (int i = 0; i < nf; ++i) {      // row: constraint at omega_i
    z[i] = 1.0;
    for (int j = 0; j < nf; ++j) {    // column: filter j
      G[i * n2 + j] = fc[j].value(omega[i]);
      G[i * n2 + nf + j] = fs[j].value(omega[i]);
      G[(nf + i) * n2 + j] = fc[j].slope(omega[i]);
      G[(nf + i) * n2 + nf + j] = fs[j].slope(omega[i]);
      H[i * nf + j] = fa[j].value(omega[i]);
      H[(nf + i) * nf + j] = fa[j].slope(omega[i]);
    }
  }
  std::vector<double> Ginv;
  double condG = 0.0;
  if (!invert(n2, G, Ginv, &condG) || condG > kMaxCondG) {
    std::ostringstream os;
    os << "filter optimisation: constraint matrix G is singular (condition " << condG << ")";
    set_error(os.str());
    return MFWH_ERR_SINGULAR;
  }
  // G^{-1} z and G^{-1} H by LU solves with partial pivoting.  The explicit inverse serves
  // only the condition estimate: products with it are not backward stable, and with cond(G)
  // near the limit they leave the constraints of eq. constraintsT visibly unmet.
  std::vector<double> Gz = z, GH = H;
  if (!lu_solve(n2, G, Gz, 1) || !lu_solve(n2, G, GH, nf)) {
    set_error("filter optimisation: constraint matrix G is singular");
    return MFWH_ERR_SINGULAR;
  }

  // Spectral interval and midpoint nodes (eq. LambdaRange).  lam_max / delta equals
  // the integer 2 N_{p,Nf} + c_delta N_f, hence the guard against rounding up.
  const double delta = omega[nf - 1] / (2.0 * n_pm[nf - 1]);
  const double lam_max = omega[nf - 1] + c_delta * nf * delta;
  const int n_lambda = (int)std::ceil(n_delta * lam_max / delta - 1e-9);
  std::vector<double> M((size_t)n_lambda * nf), m0(n_lambda);
  std::vector<double> fcs(n2);
  for (int k = 0; k < n_lambda; ++k) {
    double lam = (k + 0.5) * lam_max / n_lambda;
    for (int j = 0; j < nf; ++j) {
      fcs[j] = fc[j].value(lam);
      fcs[nf + j] = fs[j].value(lam);
    }
    double mu0 = 0.0;
    for (int i = 0; i < n2; ++i) mu0 += fcs[i] * Gz[i];
    m0[k] = -mu0;
    for (int j = 0; j < nf; ++j) {
      double g = fa[j].value(lam);
      for (int i = 0; i < n2; ++i) g -= fcs[i] * GH[i * nf + j];
      M[(size_t)k * nf + j] = g;
    }
  }
  std::vector<double> xa;
  if (!householder_lstsq(n_lambda, nf, M, m0, xa)) {
    set_error("filter optimisation: least-squares matrix is rank deficient");
    return MFWH_ERR_SINGULAR;
  }
  // y = G^{-1} (z - H x_a) (eq. yOpt), again by an LU solve.
  std::vector<double> y(n2);
  for (int i = 0; i < n2; ++i) {
    y[i] = z[i];
    for (int j = 0; j < nf; ++j) y[i] -= H[i * nf + j] * xa[j];
  }
  if (!lu_solve(n2, G, y, 1)) {
    set_error("filter optimisation: constraint matrix G is singular");
    return MFWH_ERR_SINGULAR;
  }
  for (int m = 0; m < nf; ++m) {
    params[3 * m + 0] = xa[m];
    params[3 * m + 1] = y[m];
    params[3 * m + 2] = y[nf + m];
  }
  if (lam_max_out) *lam_max_out = lam_max;
  if (n_lambda_out) *n_lambda_out = n_lambda;
  return MFWH_OK;
}

static mfwh_status fail(mfwh_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

mfwh_status plan_problem(const mfwh_problem* p, Plan* out, double c2_field_max) {
  if (!p || !out) return fail(MFWH_ERR_INVALID_ARG, "null problem or output");
  if (p->dim != 2 && p->dim != 3) return fail(MFWH_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (p->nf < 1 || p->nf > MFWH_MAX_NF) return fail(MFWH_ERR_INVALID_ARG, "nf out of range 1..16");
  if (!p->omega) return fail(MFWH_ERR_INVALID_ARG, "omega is NULL");
  for (int m = 0; m < p->nf; ++m) {
    if (!(p->omega[m] > 0.0) || !std::isfinite(p->omega[m]))
      return fail(MFWH_ERR_INVALID_ARG, "frequencies must be positive and finite");
    if (m > 0 && !(p->omega[m] > p->omega[m - 1]))
      return fail(MFWH_ERR_INVALID_ARG, "frequencies must be strictly increasing");
  }
  for (int a = 0; a < p->dim; ++a) {
    if (p->n[a] < 2 || p->n[a] > (1 << 20))
      return fail(MFWH_ERR_INVALID_ARG, "cells per axis must be in 2..2^20");
    if (!(p->length[a] > 0.0) || !std::isfinite(p->length[a]))
      return fail(MFWH_ERR_INVALID_ARG, "domain lengths must be positive");
  }
  if (p->n_p < 1) return fail(MFWH_ERR_INVALID_ARG, "n_p must be >= 1");
  if (!(p->cfl > 0.0 && p->cfl <= 1.0)) return fail(MFWH_ERR_INVALID_ARG, "cfl must be in (0, 1]");
  const bool field = p->c_mode == MFWH_C_FIELD;
  if (field) {
    if (!p->c2_field) return fail(MFWH_ERR_INVALID_ARG, "c2_field is NULL");
    if (!(c2_field_max > 0.0) || !std::isfinite(c2_field_max))
      return fail(MFWH_ERR_INVALID_ARG, "c2_field values must be finite and > 0");
  } else if (!(p->c_lo > 0.0)) {
    return fail(MFWH_ERR_INVALID_ARG, "c_lo must be > 0");
  }
  if (field) {
    if (p->precision != MFWH_PREC_FP64)
      return fail(MFWH_ERR_INVALID_ARG, "a c^2 field runs with the FP64 precision only");
    if (p->time_stepping != MFWH_TIME_EXPLICIT)
      return fail(MFWH_ERR_INVALID_ARG, "a c^2 field runs with explicit time stepping only");
    if (p->time_block > 1)
      return fail(MFWH_ERR_INVALID_ARG, "a c^2 field takes one step per launch");
  } else if (p->c_mode == MFWH_C_TWO_LAYER) {
    if (!(p->c_hi > 0.0)) return fail(MFWH_ERR_INVALID_ARG, "c_hi must be > 0");
    if (p->layer_axis < 0 || p->layer_axis >= p->dim)
      return fail(MFWH_ERR_INVALID_ARG, "layer_axis out of range");
  } else if (p->c_mode != MFWH_C_CONST) {
    return fail(MFWH_ERR_INVALID_ARG, "unknown c_mode");
  }
  if (p->filter_mode < 0 || p->filter_mode > 2) return fail(MFWH_ERR_INVALID_ARG, "unknown filter_mode");
  if (p->filter_mode == MFWH_FILTER_USER && !p->user_params)
    return fail(MFWH_ERR_INVALID_ARG, "user_params is NULL");
  if (p->filter_mode == MFWH_FILTER_OPTIMIZED && (p->n_delta < 1 || !(p->c_delta >= 0.0)))
    return fail(MFWH_ERR_INVALID_ARG, "n_delta must be >= 1 and c_delta >= 0");
  if (p->precision != MFWH_PREC_FP64 && p->precision != MFWH_PREC_FP32_KAHAN &&
      p->precision != MFWH_PREC_FP32_BLOCKSUM)
    return fail(MFWH_ERR_INVALID_ARG, "unsupported precision");
  const bool fp32 = p->precision != MFWH_PREC_FP64;
  if (p->dim == 3) {
    if (p->time_block != 0 && p->time_block != 1 &&
        !(fp32 && (p->time_block == 2 || p->time_block == 4)))
      return fail(MFWH_ERR_INVALID_ARG,
                  "3D time_block must be 0 or 1 (or 2 or 4 for the FP32 precisions)");
  } else if (p->time_block != 0 && p->time_block != 1 && p->time_block != 4 &&
             p->time_block != 8 && !(fp32 && p->time_block == 16) &&
             !(!fp32 && (p->time_block == 2 || p->time_block == 3))) {
    return fail(MFWH_ERR_INVALID_ARG,
                "time_block must be 0, 1, 4 or 8 (or 16 for FP32, 2 or 3 for FP64)");
  }
  if (p->tile_shape < 0 || p->tile_shape > (fp32 ? 2 : 5))
    return fail(MFWH_ERR_INVALID_ARG, "tile_shape must be 0, 1 or 2 (0 to 5 for FP64)");
  if (p->filter_update != MFWH_UPDATE_IMPLICIT && p->filter_update != MFWH_UPDATE_EXPLICIT)
    return fail(MFWH_ERR_INVALID_ARG, "filter_update must be implicit or explicit");
  if (p->order != 0 && p->order != 2 && p->order != 4)
    return fail(MFWH_ERR_INVALID_ARG, "order must be 2 or 4");
  if (p->order == 4 && p->time_block > 1)
    return fail(MFWH_ERR_INVALID_ARG, "the fourth-order operator takes one step per launch");
  if (p->time_stepping != MFWH_TIME_EXPLICIT && p->time_stepping != MFWH_TIME_IMPLICIT)
    return fail(MFWH_ERR_INVALID_ARG, "time_stepping must be explicit or implicit");
  const bool implicit = p->time_stepping == MFWH_TIME_IMPLICIT;
  if (implicit) {
    if (fp32) return fail(MFWH_ERR_INVALID_ARG, "implicit time stepping runs in FP64 only");
    if (p->time_block > 1)
      return fail(MFWH_ERR_INVALID_ARG, "implicit time stepping takes one step per launch");
    if (p->steps_per_period != 0 && p->steps_per_period < 5)
      return fail(MFWH_ERR_INVALID_ARG, "steps_per_period must be >= 5");
    if (p->mg_tol != 0.0 && !(p->mg_tol > 0.0 && p->mg_tol < 1.0))
      return fail(MFWH_ERR_INVALID_ARG, "mg_tol must be in (0, 1)");
    if (p->mg_max_cycles < 0 || p->mg_max_cycles > 60)
      return fail(MFWH_ERR_INVALID_ARG, "mg_max_cycles must be in 0..60");
  }

  Plan& P = *out;
  P = Plan();
  mfwh_setup& s = P.s;
  const int nf = p->nf;
  s.nf = nf;
  P.dim = p->dim;
  // Defaults (fastest measured on GB300).  FP64, 2D, second order, constant or two-layer c,
  // explicit steps, up to 8 frequencies: 3 steps per pass over HBM on the persistent pipelined
  // kernel (tile shape 5).  Other FP64 problems: one step per launch.  FP32 in 2D: 16 steps
  // per launch.
  const bool fp64_blocked = !fp32 && p->dim == 2 && p->order != 4 && !field && !implicit &&
                            p->nf <= 8;
  P.time_block = p->time_block != 0
                     ? p->time_block
                     : (fp32 && p->dim == 2 && p->order != 4 ? 16 : (fp64_blocked ? 3 : 1));
  P.tile_shape = (p->time_block == 0 && fp64_blocked && p->tile_shape == 0) ? 5 : p->tile_shape;
  P.order = p->order == 4 ? 4 : 2;
  P.filter_update = p->filter_update;
  P.precision = p->precision;
  P.time_stepping = p->time_stepping;
  if (implicit) {
    P.mg_tol = p->mg_tol != 0.0 ? p->mg_tol : 1e-10;
    P.mg_max_cycles = p->mg_max_cycles != 0 ? p->mg_max_cycles : 30;
  }
  double inv_h2 = 0.0;
  s.points = 1;
  s.interior_points = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < p->dim) {
      P.n[a] = p->n[a];
      s.h[a] = p->length[a] / (double)p->n[a];
      inv_h2 += 1.0 / (s.h[a] * s.h[a]);
      s.points *= p->n[a] + 1;
      s.interior_points *= p->n[a] - 1;
    } else {
      P.n[a] = 0;
      s.h[a] = 0.0;
    }
  }
  P.c_max = p->c_lo;
  P.c2_lo = p->c_lo * p->c_lo;
  P.c2_hi = P.c2_lo;
  P.layer_axis = 0;
  P.layer_split = P.n[0] + 1;  // everything in the lower layer
  if (p->c_mode == MFWH_C_TWO_LAYER) {
    P.c_max = std::max(p->c_lo, p->c_hi);
    P.c2_hi = p->c_hi * p->c_hi;
    P.layer_axis = p->layer_axis;
    const int64_t na = p->n[p->layer_axis];
    const double ha = p->length[p->layer_axis] / (double)na;
    int64_t split = na + 1;
    for (int64_t j = 0; j <= na; ++j)
      if (!((double)j * ha < p->interface)) { split = j; break; }
    P.layer_split = split;
  } else if (field) {
    // the kernels take c^2 from the field; the layer coefficients are those of c = 1
    P.c2_field = true;
    P.c_max = std::sqrt(c2_field_max);
    P.c2_lo = P.c2_hi = 1.0;
  }

  int n_t = 0;
  if (implicit) {
    // Trapezoidal scheme (Section "Time-step determination"): steps_per_period steps over the
    // shortest period give N_t over N_p longest periods; dt then solves omega~_1 N_t dt =
    // 2 pi N_p, i.e. (omega_1 dt)^2 = (1 - cos theta) / (beta/2 + alpha cos theta) with
    // theta = 2 pi N_p / N_t and (alpha, beta) = (1/2, 0).  N_t > 4 N_p keeps cos theta > 0.
    const int spp = p->steps_per_period != 0 ? p->steps_per_period : 10;
    const double nt_real = std::ceil(spp * (double)p->n_p * p->omega[nf - 1] / p->omega[0] - 1e-12);
    if (nt_real > 5e7) return fail(MFWH_ERR_INVALID_ARG, "too many time steps");
    n_t = (int)nt_real;
    const double theta = 2.0 * kPi * p->n_p / n_t;
    const double x2 = (1.0 - std::cos(theta)) / (0.5 * std::cos(theta));
    s.n_t = n_t;
    s.dt = std::sqrt(x2) / p->omega[0];
  } else {
    // Time step (explicit leapfrog; Section "Time-step determination").
    // Leapfrog needs dt^2 rho(-L_h) <= 4; rho = c_max^2 sum_i 4/h_i^2 for the second-order
    // operator and c_max^2 sum_i (16/3)/h_i^2 for the fourth-order one.
    const double dt_stab =
        (P.order == 4 ? std::sqrt(3.0) / 2.0 : 1.0) / (P.c_max * std::sqrt(inv_h2));
    const double t1 = p->n_p * 2.0 * kPi / p->omega[0];
    double nt_real = std::ceil(t1 / (p->cfl * dt_stab));
    if (nt_real > 5e7) return fail(MFWH_ERR_INVALID_ARG, "too many time steps");
    n_t = std::max(2 * p->n_p + 1, (int)nt_real);
    s.n_t = n_t;
    s.dt = 2.0 * std::sin(kPi * p->n_p / n_t) / p->omega[0];
  }
  const double dt = s.dt;

  // Adjusted frequencies (eq. omegaImplicit with the scheme's (alpha, beta)) and periods
  // (eq. TbarDef).
  const double alpha = implicit ? 0.5 : 0.0, beta = implicit ? 0.0 : 1.0;
  for (int m = 0; m < nf; ++m) {
    double x = p->omega[m] * dt;
    double c = (1.0 - 0.5 * beta * x * x) / (1.0 + alpha * x * x);
    if (c < -1.0) return fail(MFWH_ERR_INVALID_ARG, "frequency above the time-step Nyquist limit");
    s.omega_tilde[m] = std::acos(c) / dt;
  }
  for (int m = 0; m < nf; ++m) {
    s.n_pm[m] = period_count(p->n_p, s.omega_tilde[m], s.omega_tilde[0]);
    s.t_fm[m] = s.n_pm[m] * (2.0 * kPi / s.omega_tilde[m]);
  }
  std::vector<double> sigma((size_t)(n_t + 1) * nf);
  trapezoid_weights(n_t, dt, nf, s.t_fm, sigma.data());

  // Filter parameters.
  std::vector<double> prm(3 * nf);
  s.lam_max = 0.0;
  s.n_lambda = 0;
  if (p->filter_mode == MFWH_FILTER_OPTIMIZED) {
    mfwh_status st = optimise_parameters(nf, s.omega_tilde, p->n_p, n_t, p->n_delta, p->c_delta,
                                         prm.data(), &s.lam_max, &s.n_lambda);
    if (st != MFWH_OK) return st;
  } else if (p->filter_mode == MFWH_FILTER_TRADITIONAL) {
    for (int m = 0; m < nf; ++m) {   // eq. origParamAdjust
      double wd = s.omega_tilde[m] * dt;
      prm[3 * m + 0] = -std::tan(0.5 * wd) / (2.0 * std::tan(wd));
      prm[3 * m + 1] = 1.0;
      prm[3 * m + 2] = 0.0;
    }
  } else {
    for (int i = 0; i < 3 * nf; ++i) prm[i] = p->user_params[i];
  }
  for (int m = 0; m < nf; ++m)
    for (int k = 0; k < 3; ++k) s.params[m][k] = prm[3 * m + k];

  // Filter weights w_{n,m} (eq. pDefQ) and forcing phases cos(omega~_m t^n).
  P.w.assign((size_t)(n_t + 1) * nf, 0.0);
  P.cosf.assign((size_t)(n_t + 1) * nf, 0.0);
  for (int n = 0; n <= n_t; ++n) {
    double t = n * dt;
    for (int m = 0; m < nf; ++m) {
      double ph = s.omega_tilde[m] * t;
      double kern = prm[3 * m] + prm[3 * m + 1] * std::cos(ph) + prm[3 * m + 2] * std::sin(ph);
      P.w[(size_t)n * nf + m] = 2.0 / s.t_fm[m] * sigma[(size_t)n * nf + m] * kern;
      P.cosf[(size_t)n * nf + m] = std::cos(ph);
    }
  }
  // B_{mj} = beta_{d,m}(omega~_j) = sum_n w_{n,m} cos(omega~_j t^n) (eq. filterA, eq. betadDefA).
  std::vector<double> B(nf * nf, 0.0), Binv;
  for (int m = 0; m < nf; ++m)
    for (int j = 0; j < nf; ++j) {
      double acc = 0.0;
      for (int n = 0; n <= n_t; ++n) acc += P.w[(size_t)n * nf + m] * P.cosf[(size_t)n * nf + j];
      B[m * nf + j] = acc;
    }
  double condB = 0.0;
  if (!invert(nf, B, Binv, &condB) || condB > kMaxCondB) {
    std::ostringstream os;
    os << "filter matrix B is singular (condition " << condB << "); frequencies too close?";
    return fail(MFWH_ERR_SINGULAR, os.str());
  }
  for (int m = 0; m < MFWH_MAX_NF; ++m)
    for (int j = 0; j < MFWH_MAX_NF; ++j) {
      bool in = m < nf && j < nf;
      s.B[m][j] = in ? B[m * nf + j] : 0.0;
      s.B_inv[m][j] = in ? Binv[m * nf + j] : 0.0;
    }
  return MFWH_OK;
}

}  // namespace mfwh

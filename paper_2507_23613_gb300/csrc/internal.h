// Internal declarations shared by the translation units of libmfwh.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "mfwh.h"

namespace mfwh {

// Thread-local error message behind mfwh_last_error().
void set_error(const std::string& msg);

// Host set-up of one problem: the public mfwh_setup plus the per-step tables
// the kernels need.  Everything is FP64 and computed on the host.
struct Plan {
  mfwh_setup s{};
  double c_max = 0.0;
  double c2_lo = 0.0, c2_hi = 0.0;   // c^2 on each side of the layer interface
  int64_t layer_split = 0;           // first grid index along layer_axis in the upper layer
  bool c2_field = false;             // MFWH_C_FIELD: c^2 per point (c2_lo = c2_hi = 1 then)
  int layer_axis = 0;
  int dim = 2;
  int time_block = 1;          // steps per wave-kernel launch (1, 4, 8 or 16)
  int tile_shape = 0;          // FP32 blocked-kernel tile shape
  int precision = MFWH_PREC_FP64;
  int order = 2;               // order of L_{ph}: 2 or 4
  int filter_update = MFWH_UPDATE_IMPLICIT;
  int time_stepping = MFWH_TIME_EXPLICIT;
  double mg_tol = 1e-10;       // implicit: relative max-norm residual of each step solve
  int mg_max_cycles = 30;      // implicit: V-cycles per step solve at most
  int64_t n[3] = {1, 1, 1};
  std::vector<double> w;       // [(n_t + 1) * nf]  filter weights w_{n,m}
  std::vector<double> cosf;    // [(n_t + 1) * nf]  cos(omega~_m t^n)
};

// c2_field_max: the largest value of prob->c2_field (MFWH_C_FIELD only; the caller reads the
// field, which may be device memory, and checks that all values are finite and > 0).
mfwh_status plan_problem(const mfwh_problem* prob, Plan* out, double c2_field_max = 0.0);

// Discrete Algorithm 2 (see mfwh_opt_parameters).
mfwh_status optimise_parameters(int nf, const double* omega, int n_p, int n_t, int n_delta,
                                double c_delta, double* params, double* lam_max, int* n_lambda);

// Trapezoid weights sigma_{n,m} of eq. DefNI, [(n_t + 1) * nf], row n.
void trapezoid_weights(int n_t, double dt, int nf, const double* t_fm, double* sigma);

}  // namespace mfwh

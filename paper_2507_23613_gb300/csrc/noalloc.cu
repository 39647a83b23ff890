// Allocation-free entry point: the Helmholtz residual of mfwh_residual without a
// handle and without allocating device memory.
//
// Some callers cannot allocate device memory when they need the check: code
// whose device memory is owned by another allocator (a framework's caching
// allocator, or a pool sized once at start-up) and must not grow outside it,
// and loops that cannot afford the implicit device synchronisation that
// cudaMalloc / cudaFree may cause.  For them the reduction scratch lives in a
// fixed file-scope __device__ array instead of a handle's workspace.
#include <cmath>
#include <mutex>
#include <sstream>

#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"

namespace {

// Per-block partial maxima of the residual kernel followed by its reduced output.
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_residual_scratch[MFWH_NOALLOC_SCRATCH_DOUBLES];
static_assert((int64_t)mfwh::kResidualBlocks * 2 * MFWH_MAX_NF + 2 * MFWH_MAX_NF <=
                  MFWH_NOALLOC_SCRATCH_DOUBLES,
              "the residual's partial maxima and output must fit the scratch array");

constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).  The
// name g_residual_scratch is a host-side stand-in in host code, so the address is
// looked up once per device and cached.
mfwh_status scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) {
    mfwh::set_error("mfwh_residual_noalloc: device ordinal out of range");
    return MFWH_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e != cudaSuccess || !p) {
      std::ostringstream os;
      os << "mfwh_residual_noalloc: cudaGetSymbolAddress failed: " << cudaGetErrorString(e);
      mfwh::set_error(os.str());
      return MFWH_ERR_CUDA;
    }
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return MFWH_OK;
}

// True if p is managed memory or device memory of `device` (the current device): a
// buffer on another GPU would be read through a peer mapping that may not exist.
bool on_device(const void* p, int device) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type == cudaMemoryTypeManaged) return true;
  return attr.type == cudaMemoryTypeDevice && attr.device == device;
}

mfwh_status bad(const char* msg) {
  mfwh::set_error(msg);
  return MFWH_ERR_INVALID_ARG;
}

}  // namespace

extern "C" mfwh_status mfwh_residual_noalloc(const mfwh_problem* p, const double* forcing,
                                             const double* v, double* r_out, void* stream) {
  if (!p || !forcing || !v || !r_out) return bad("mfwh_residual_noalloc: null argument");
  if (p->dim != 2 && p->dim != 3) return bad("mfwh_residual_noalloc: dim must be 2 or 3");
  if (p->nf < 1 || p->nf > MFWH_MAX_NF || !p->omega)
    return bad("mfwh_residual_noalloc: nf must be in 1..16 with omega given");
  for (int m = 0; m < p->nf; ++m)
    if (!(std::isfinite(p->omega[m]) && p->omega[m] > 0.0))
      return bad("mfwh_residual_noalloc: every omega must be finite and > 0");
  if (p->order != 0 && p->order != 2 && p->order != 4)
    return bad("mfwh_residual_noalloc: order must be 2 or 4 (0 means 2)");
  // Guard: for nf <= MFWH_MAX_NF the static_assert above keeps the need within the array.
  const int64_t need = mfwh::residual_partial_size(p->nf) + 2 * p->nf;
  if (need > MFWH_NOALLOC_SCRATCH_DOUBLES) {
    std::ostringstream os;
    os << "mfwh_residual_noalloc: needs " << need << " scratch doubles, maximum is "
       << MFWH_NOALLOC_SCRATCH_DOUBLES;
    mfwh::set_error(os.str());
    return MFWH_ERR_INVALID_ARG;
  }
  mfwh::Geom g{};
  double inv_h2[3] = {0.0, 0.0, 0.0};
  int64_t n[3] = {0, 0, 0};
  for (int a = 0; a < p->dim; ++a) {
    if (p->n[a] < 2 || p->n[a] > (1 << 20) || !(p->length[a] > 0.0) ||
        !std::isfinite(p->length[a]))
      return bad("mfwh_residual_noalloc: bad grid size or length");
    n[a] = p->n[a];
    const double h = p->length[a] / (double)p->n[a];
    inv_h2[a] = 1.0 / (h * h);
  }
  g.nx = n[0];
  g.ny = n[1];
  g.nz = p->dim == 3 ? n[2] : 0;
  g.sy = g.nx + 1;
  g.sz = (g.nx + 1) * (g.ny + 1);
  g.points = g.sz * (p->dim == 3 ? g.nz + 1 : 1);
  g.dim = p->dim;
  g.order = p->order == 4 ? 4 : 2;
  const bool field = p->c_mode == MFWH_C_FIELD;
  if (!field && (!(p->c_lo > 0.0) || !std::isfinite(p->c_lo)))
    return bad("mfwh_residual_noalloc: c_lo must be finite and > 0");
  double c2_lo = field ? 1.0 : p->c_lo * p->c_lo, c2_hi = c2_lo;
  g.layer_axis = 0;
  g.layer_split = g.nx + 1;
  if (field) {
    if (!p->c2_field) return bad("mfwh_residual_noalloc: c2_field is NULL");
    g.c2f = p->c2_field;   // checked below: device memory of the current device
  } else if (p->c_mode == MFWH_C_TWO_LAYER) {
    if (!(p->c_hi > 0.0) || !std::isfinite(p->c_hi) || p->layer_axis < 0 ||
        p->layer_axis >= p->dim)
      return bad("mfwh_residual_noalloc: bad two-layer description");
    c2_hi = p->c_hi * p->c_hi;
    g.layer_axis = p->layer_axis;
    const int64_t na = n[p->layer_axis];
    const double ha = p->length[p->layer_axis] / (double)na;
    g.layer_split = na + 1;
    for (int64_t j = 0; j <= na; ++j)
      if (!((double)j * ha < p->interface)) {
        g.layer_split = j;
        break;
      }
  } else if (p->c_mode != MFWH_C_CONST) {
    return bad("mfwh_residual_noalloc: unknown c_mode");
  }
  double omega2[MFWH_MAX_NF];
  for (int m = 0; m < p->nf; ++m) omega2[m] = p->omega[m] * p->omega[m];
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) {
    mfwh::set_error(std::string("mfwh_residual_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return MFWH_ERR_CUDA;
  }
  if (!on_device(forcing, device) || !on_device(v, device) ||
      (field && !on_device(p->c2_field, device)))
    return bad("mfwh_residual_noalloc: forcing, v (and c2_field) must be device (or managed) "
               "memory of the current device");
  double* scratch = nullptr;
  mfwh_status st = scratch_address(device, &scratch);
  if (st != MFWH_OK) return st;
  double* partial = scratch;
  double* out = scratch + mfwh::residual_partial_size(p->nf);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Every partial the reduction reads is written by the residual kernel first, so
  // nothing left in the array by an earlier call needs clearing.
  mfwh::launch_residual(p->nf, g, v, forcing, omega2, c2_lo, c2_hi, inv_h2, partial, out, s);
  double host[2 * MFWH_MAX_NF];
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, out, sizeof(double) * 2 * p->nf, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mfwh::set_error(std::string("mfwh_residual_noalloc: ") + cudaGetErrorString(e));
    return MFWH_ERR_CUDA;
  }
  bool finite = true;
  for (int m = 0; m < p->nf; ++m) {
    const double num = host[m], den = host[p->nf + m];
    r_out[m] = den > 0.0 ? num / den : num;
    finite = finite && std::isfinite(r_out[m]);
  }
  if (!finite) {
    mfwh::set_error("mfwh_residual_noalloc: non-finite value in the Helmholtz residual");
    return MFWH_ERR_NONFINITE;
  }
  return MFWH_OK;
}

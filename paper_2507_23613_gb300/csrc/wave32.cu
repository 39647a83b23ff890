// Host entry points of the FP32 wave solve: dispatch on the number of
// frequencies to the instantiations in wave32_p1.cu .. wave32_p8.cu.  The
// kernels and the arithmetic they follow are described in wave32_kernels.cuh.
#include <cuda_runtime.h>

#include "wave32_kernels.cuh"

namespace mfwh {
namespace {

__global__ void k_to_float(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

W32Ops ops_for(int nf) {
  switch ((nf + 1) / 2) {
    case 1: return w32_ops_p1(nf);
    case 2: return w32_ops_p2(nf);
    case 3: return w32_ops_p3(nf);
    case 4: return w32_ops_p4(nf);
    case 5: return w32_ops_p5(nf);
    case 6: return w32_ops_p6(nf);
    case 7: return w32_ops_p7(nf);
    default: return w32_ops_p8(nf);
  }
}

Tb3dFn tb3_for(int nf) {
  switch ((nf + 1) / 2) {
    case 1: return w32_tb3_p1(nf);
    case 2: return w32_tb3_p2(nf);
    case 3: return w32_tb3_p3(nf);
    case 4: return w32_tb3_p4(nf);
    case 5: return w32_tb3_p5(nf);
    case 6: return w32_tb3_p6(nf);
    case 7: return w32_tb3_p7(nf);
    default: return w32_tb3_p8(nf);
  }
}

}  // namespace

void launch_tb3d32(int nf, const Geom& g, const float* W_in, const float* D_in, float* W_out,
                   float* D_out, const float* f, float* qs, float* qc, double* vout,
                   const double* vsub, const TB32Host& h, cudaStream_t st) {
  tb3_for(nf)(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
}

void launch_init32(int nf, const Geom& g, const double* v, float* W0, float* qs, float* qc,
                   const float* w0, cudaStream_t st) {
  ops_for(nf).init(g, v, W0, qs, qc, w0, st);
}

void launch_step32(int nf, const Geom& g, const float* W, const float* D_in, float* W_out,
                   float* D_out, const float* f, float* qs, float* qc, const Step32Host& h,
                   cudaStream_t st) {
  ops_for(nf).step(g, W, D_in, W_out, D_out, f, qs, qc, h, st);
}

void launch_last32(int nf, const Geom& g, const float* W, const float* D, const float* f,
                   const float* qs, const float* qc, double* vout, const double* vsub,
                   const Step32Host& h, const StepHost& epi, cudaStream_t st) {
  ops_for(nf).last(g, W, D, f, qs, qc, vout, vsub, h, epi, st);
}

void launch_tb2d32(int nf, const Geom& g, const float* W_in, const float* D_in, float* W_out,
                   float* D_out, const float* f, float* qs, float* qc, double* vout,
                   const double* vsub, const TB32Host& h, cudaStream_t st) {
  ops_for(nf).tb(g, W_in, D_in, W_out, D_out, f, qs, qc, vout, vsub, h, st);
}

void launch_to_float(const double* x, float* y, int64_t n, cudaStream_t st) {
  k_to_float<<<4 * 152, 256, 0, st>>>(x, y, n);
}

}  // namespace mfwh

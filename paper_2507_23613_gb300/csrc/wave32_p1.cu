// FP32 wave-solve kernels instantiated for 1 and 2 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p1(int nf) {
  switch (nf) {
    case 1: return make_w32_ops<1>();
    case 2: return make_w32_ops<2>();
    default: return make_w32_ops<2>();
  }
}

Tb3dFn w32_tb3_p1(int nf) {
  return nf == 1 ? tb3d32_nf<1> : tb3d32_nf<2>;
}

}  // namespace mfwh

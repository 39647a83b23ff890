// FP32 wave-solve kernels instantiated for 13 and 14 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p7(int nf) {
  switch (nf) {
    case 13: return make_w32_ops<13>();
    case 14: return make_w32_ops<14>();
    default: return make_w32_ops<14>();
  }
}

Tb3dFn w32_tb3_p7(int nf) {
  return nf == 13 ? tb3d32_nf<13> : tb3d32_nf<14>;
}

}  // namespace mfwh

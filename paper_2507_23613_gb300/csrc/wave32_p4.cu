// FP32 wave-solve kernels instantiated for 7 and 8 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p4(int nf) {
  switch (nf) {
    case 7: return make_w32_ops<7>();
    case 8: return make_w32_ops<8>();
    default: return make_w32_ops<8>();
  }
}

Tb3dFn w32_tb3_p4(int nf) {
  return nf == 7 ? tb3d32_nf<7> : tb3d32_nf<8>;
}

}  // namespace mfwh

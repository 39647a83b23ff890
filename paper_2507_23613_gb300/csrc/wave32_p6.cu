// FP32 wave-solve kernels instantiated for 11 and 12 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p6(int nf) {
  switch (nf) {
    case 11: return make_w32_ops<11>();
    case 12: return make_w32_ops<12>();
    default: return make_w32_ops<12>();
  }
}

Tb3dFn w32_tb3_p6(int nf) {
  return nf == 11 ? tb3d32_nf<11> : tb3d32_nf<12>;
}

}  // namespace mfwh

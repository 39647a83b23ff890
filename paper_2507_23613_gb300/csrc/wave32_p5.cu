// FP32 wave-solve kernels instantiated for 9 and 10 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p5(int nf) {
  switch (nf) {
    case 9: return make_w32_ops<9>();
    case 10: return make_w32_ops<10>();
    default: return make_w32_ops<10>();
  }
}

Tb3dFn w32_tb3_p5(int nf) {
  return nf == 9 ? tb3d32_nf<9> : tb3d32_nf<10>;
}

}  // namespace mfwh

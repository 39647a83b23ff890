// FP32 wave-solve kernels instantiated for 15 and 16 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p8(int nf) {
  switch (nf) {
    case 15: return make_w32_ops<15>();
    case 16: return make_w32_ops<16>();
    default: return make_w32_ops<16>();
  }
}

Tb3dFn w32_tb3_p8(int nf) {
  return nf == 15 ? tb3d32_nf<15> : tb3d32_nf<16>;
}

}  // namespace mfwh

// FP32 wave-solve kernels instantiated for 3 and 4 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p2(int nf) {
  switch (nf) {
    case 3: return make_w32_ops<3>();
    case 4: return make_w32_ops<4>();
    default: return make_w32_ops<4>();
  }
}

Tb3dFn w32_tb3_p2(int nf) {
  return nf == 3 ? tb3d32_nf<3> : tb3d32_nf<4>;
}

}  // namespace mfwh

// FP32 wave-solve kernels instantiated for 5 and 6 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p3(int nf) {
  switch (nf) {
    case 5: return make_w32_ops<5>();
    case 6: return make_w32_ops<6>();
    default: return make_w32_ops<6>();
  }
}

Tb3dFn w32_tb3_p3(int nf) {
  return nf == 5 ? tb3d32_nf<5> : tb3d32_nf<6>;
}

}  // namespace mfwh

// FP32 wave-solve kernels instantiated for 1 to 4 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p1(int nf) {
  switch (nf) {
    case 1: return make_w32_ops<1>();
    case 2: return make_w32_ops<2>();
    case 3: return make_w32_ops<3>();
    case 4: return make_w32_ops<4>();
    default: return make_w32_ops<4>();
  }
}

}  // namespace mfwh

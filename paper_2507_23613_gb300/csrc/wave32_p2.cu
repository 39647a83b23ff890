// FP32 wave-solve kernels instantiated for 5 to 8 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p2(int nf) {
  switch (nf) {
    case 5: return make_w32_ops<5>();
    case 6: return make_w32_ops<6>();
    case 7: return make_w32_ops<7>();
    case 8: return make_w32_ops<8>();
    default: return make_w32_ops<8>();
  }
}

}  // namespace mfwh

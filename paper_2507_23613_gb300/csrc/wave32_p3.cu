// FP32 wave-solve kernels instantiated for 9 to 12 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p3(int nf) {
  switch (nf) {
    case 9: return make_w32_ops<9>();
    case 10: return make_w32_ops<10>();
    case 11: return make_w32_ops<11>();
    case 12: return make_w32_ops<12>();
    default: return make_w32_ops<12>();
  }
}

}  // namespace mfwh

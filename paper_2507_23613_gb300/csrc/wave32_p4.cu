// FP32 wave-solve kernels instantiated for 13 to 16 frequencies.
#include "wave32_kernels.cuh"

namespace mfwh {

W32Ops w32_ops_p4(int nf) {
  switch (nf) {
    case 13: return make_w32_ops<13>();
    case 14: return make_w32_ops<14>();
    case 15: return make_w32_ops<15>();
    case 16: return make_w32_ops<16>();
    default: return make_w32_ops<16>();
  }
}

}  // namespace mfwh

// FP64 temporally blocked 2D step kernels instantiated for 9-12 frequencies.
#include "wave_tb_kernels.cuh"

namespace mfwh {

TbFn tb_fn_p4(int nf) {
  switch (nf) {
    case 9: return tb_launch_nf<9>;
    case 10: return tb_launch_nf<10>;
    case 11: return tb_launch_nf<11>;
    case 12: return tb_launch_nf<12>;
    default: return nullptr;
  }
}

}  // namespace mfwh

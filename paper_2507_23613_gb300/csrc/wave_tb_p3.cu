// FP64 temporally blocked 2D step kernels instantiated for 7-8 frequencies.
#include "wave_tb_kernels.cuh"

namespace mfwh {

TbFn tb_fn_p3(int nf) {
  switch (nf) {
    case 7: return tb_launch_nf<7>;
    case 8: return tb_launch_nf<8>;
    default: return nullptr;
  }
}

}  // namespace mfwh

// FP64 temporally blocked 2D step kernels instantiated for 1-3 frequencies.
#include "wave_tb_kernels.cuh"

namespace mfwh {

TbFn tb_fn_p1(int nf) {
  switch (nf) {
    case 1: return tb_launch_nf<1>;
    case 2: return tb_launch_nf<2>;
    case 3: return tb_launch_nf<3>;
    default: return nullptr;
  }
}

}  // namespace mfwh

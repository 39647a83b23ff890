// FP64 temporally blocked 2D step kernels instantiated for 4-6 frequencies.
#include "wave_tb_kernels.cuh"

namespace mfwh {

TbFn tb_fn_p2(int nf) {
  switch (nf) {
    case 4: return tb_launch_nf<4>;
    case 5: return tb_launch_nf<5>;
    case 6: return tb_launch_nf<6>;
    default: return nullptr;
  }
}

}  // namespace mfwh

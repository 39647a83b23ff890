// FP64 temporally blocked 2D step kernels instantiated for 13-16 frequencies.
#include "wave_tb_kernels.cuh"

namespace mfwh {

TbFn tb_fn_p5(int nf) {
  switch (nf) {
    case 13: return tb_launch_nf<13>;
    case 14: return tb_launch_nf<14>;
    case 15: return tb_launch_nf<15>;
    case 16: return tb_launch_nf<16>;
    default: return nullptr;
  }
}

}  // namespace mfwh

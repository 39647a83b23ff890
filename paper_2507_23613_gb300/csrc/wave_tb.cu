// Host entry point of the FP64 temporally blocked 2D wave step: dispatch on the number of
// frequencies to the instantiations in wave_tb_p1.cu .. wave_tb_p5.cu.  The kernel and the
// arithmetic it follows are described in wave_tb_kernels.cuh.
#include "wave_tb_kernels.cuh"

namespace mfwh {

void launch_tb2d(int nf, const Geom& g, const double* Wc_in, const double* Wp_in, double* Wc_out,
                 double* Wp_out, const double* f, double* q, double* vout, const double* vsub,
                 const TBHost& h, cudaStream_t st) {
  TbFn fn = nf <= 3    ? tb_fn_p1(nf)
            : nf <= 6  ? tb_fn_p2(nf)
            : nf <= 8  ? tb_fn_p3(nf)
            : nf <= 12 ? tb_fn_p4(nf)
                       : tb_fn_p5(nf);
  if (fn != nullptr) fn(g, Wc_in, Wp_in, Wc_out, Wp_out, f, q, vout, vsub, h, st);
}

}  // namespace mfwh

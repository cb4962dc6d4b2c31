// tiled_inst.cu -- one group of tiled-kernel variants, chosen by the build:
// ADM_INST_T (float or double) and ADM_INST_SET:
//   0: passive and gradient modes, 1: full Hessian, 2: filtered Hessian,
//   3: matrix-free product, 4: filtered matrix-free product.
#include "tiled_impl.cuh"

#if !defined(ADM_INST_T) || !defined(ADM_INST_SET)
#error "tiled_inst.cu is compiled with -DADM_INST_T=<float|double> -DADM_INST_SET=<0..4>"
#endif

namespace adm {
#if ADM_INST_SET == 0
ADM_TILED_INST(ADM_INST_T, MODE_VALUE, false)
ADM_TILED_INST(ADM_INST_T, MODE_GRAD, false)
#elif ADM_INST_SET == 1
ADM_TILED_INST(ADM_INST_T, MODE_HESS, false)
#elif ADM_INST_SET == 2
ADM_TILED_INST(ADM_INST_T, MODE_HESS, true)
#elif ADM_INST_SET == 3
ADM_TILED_INST(ADM_INST_T, MODE_HVP, false)
#elif ADM_INST_SET == 4
ADM_TILED_INST(ADM_INST_T, MODE_HVP, true)
#endif
}  // namespace adm

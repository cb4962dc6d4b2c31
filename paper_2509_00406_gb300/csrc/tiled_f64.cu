// tiled_f64.cu -- double instantiation of the tiled assembler's host side; the
// kernel variants are instantiated by tiled_inst.cu.
#include "tiled_impl.cuh"

namespace adm {
ADM_TILED_VARIANTS(ADM_TILED_EXTERN, double)
template adm_status eval_tiled<double>(adm_ctx *h, const EvalArgs &a);
}  // namespace adm

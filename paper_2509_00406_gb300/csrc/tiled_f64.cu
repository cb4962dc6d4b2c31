// tiled_f64.cu -- double instantiation of the tiled assembler.
#include "tiled_impl.cuh"

namespace adm {
template adm_status eval_tiled<double>(adm_ctx *h, const EvalArgs &a);
}  // namespace adm

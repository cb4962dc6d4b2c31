// tiled_f32.cu -- float instantiation of the tiled assembler.
#include "tiled_impl.cuh"

namespace adm {
template adm_status eval_tiled<float>(adm_ctx *h, const EvalArgs &a);
}  // namespace adm

// atomic_f32.cu -- float instantiation of the per-element atomic assembler.
#include "atomic_impl.cuh"

namespace adm {
template adm_status eval_atomic<float>(adm_ctx *h, const EvalArgs &a);
}  // namespace adm

// atomic_f64.cu -- double instantiation of the per-element atomic assembler.
#include "atomic_impl.cuh"

namespace adm {
template adm_status eval_atomic<double>(adm_ctx *h, const EvalArgs &a);
}  // namespace adm

// Split-TF32 tensor-core evaluation of the interpolant contraction.
#include "interp.cuh"

namespace sg {
int eval_tf32x3(const EvalArgs&, const sg_surplus*, cudaStream_t) {
  return fail(SG_EUNSUPPORTED, "sg_eval_feedback: SG_EVAL_TF32X3 is not built yet");
}
}  // namespace sg

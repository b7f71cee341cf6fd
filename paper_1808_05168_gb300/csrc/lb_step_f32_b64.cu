// lb_step_f32_b64.cu -- the bulk-path kernels of 32- and 64-column tiles in float precision.
#define LB_STEP_FAMILY_DEFS
#include "lb_step_impl.cuh"

namespace lbk {
LB_STEP_FAMILY_INST(float, 32)
LB_STEP_FAMILY_INST(float, 64)
}  // namespace lbk

// lb_step_f32_b128.cu -- the bulk-path kernels of 128-column tiles in float precision.
#define LB_STEP_FAMILY_DEFS
#include "lb_step_impl.cuh"

namespace lbk {
LB_STEP_FAMILY_INST(float, 128)
}  // namespace lbk

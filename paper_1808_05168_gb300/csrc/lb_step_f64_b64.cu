// lb_step_f64_b64.cu -- the bulk-path kernels of 32- and 64-column tiles in double precision.
#define LB_STEP_FAMILY_DEFS
#include "lb_step_impl.cuh"

namespace lbk {
LB_STEP_FAMILY_INST(double, 32)
LB_STEP_FAMILY_INST(double, 64)
}  // namespace lbk

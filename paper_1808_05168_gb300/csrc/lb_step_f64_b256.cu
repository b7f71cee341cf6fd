// lb_step_f64_b256.cu -- the bulk-path kernels of 256-column tiles in double precision.
#define LB_STEP_FAMILY_DEFS
#include "lb_step_impl.cuh"

namespace lbk {
LB_STEP_FAMILY_INST(double, 256)
}  // namespace lbk

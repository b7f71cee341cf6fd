// lb_step_f64_gen.cu -- the generic-path kernels (per-thread staging, any tile width) in double
// precision; one translation unit per kernel family keeps the build parallel.
#define LB_STEP_FAMILY_DEFS
#include "lb_step_impl.cuh"

namespace lbk {
LB_STEP_FAMILY_INST(double, 0)
}  // namespace lbk

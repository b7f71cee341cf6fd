// lb_step_f64.cu -- double-precision instantiation of the fused step kernels (the
// kernels themselves are in lb_step_impl.cuh; one translation unit per precision keeps the
// build parallel).
#include "lb_step_impl.cuh"

namespace lbk {

#define LB_STEP_INST(real)                                                                                         \
  template size_t step_smem_bytes<real>(int);                                                                      \
  template cudaError_t prepare_step<real>(int);                                                                    \
  template cudaError_t launch_step<real>(const StepArgs<real>&, int, bool, int, bool, cudaStream_t);               \
  template int persistent_grid<real>(int, int, bool);                                                              \
  template cudaError_t launch_step_persistent<real>(const StepArgs<real>&, int, int, bool, int, bool, unsigned*,  \
                                                    int*, int, int, cudaStream_t);                 \
  template cudaError_t launch_debug_normals<real>(const uint32_t*, int64_t, double*, cudaStream_t);
LB_STEP_INST(double)

}  // namespace lbk

// lb_step_f64.cu -- double-precision dispatch of the fused step kernels: the launch, persistent
// launch and set-up entry points, which reach the kernels through the kernel families compiled
// in lb_step_f64_gen.cu, lb_step_f64_b64.cu and lb_step_f64_b128.cu (one translation unit each
// keeps the build parallel).
#include "lb_step_impl.cuh"

namespace lbk {

#define LB_STEP_INST(real)                                                                                         \
  template size_t step_smem_bytes<real>(int);                                                                      \
  template cudaError_t prepare_step<real>(int);                                                                    \
  template cudaError_t launch_step<real>(const StepArgs<real>&, int, bool, int, bool, cudaStream_t);               \
  template int persistent_grid<real>(int, int, bool);                                                              \
  template cudaError_t launch_step_persistent<real>(const StepArgs<real>&, int, int, int, bool, const PersistArgs&, \
                                                    int, cudaStream_t);                                         \
  template cudaError_t launch_debug_normals<real>(const uint32_t*, int64_t, double*, cudaStream_t);
LB_STEP_INST(double)

}  // namespace lbk

// lbm_step_kern.cu -- step kernels of one storage type and forcing: LBM_INST_S (lbm_store value)
// and LBM_INST_FORCE (0 / 1) are set by the build, one object per pair.
#include "lbm_step.cuh"

#if !defined(LBM_INST_S) || !defined(LBM_INST_FORCE)
#error "lbm_step_kern.cu is compiled with -DLBM_INST_S=<store> -DLBM_INST_FORCE=<0|1>"
#endif

namespace lbm {

template <>
void launch_step_sf<LBM_INST_S, (LBM_INST_FORCE != 0)>(bool neighbor, const StepArgs &a, cudaStream_t s, const StepAux *aux) {
    step_t<LBM_INST_S, (LBM_INST_FORCE != 0)>(neighbor, a, s, aux);
}

}  // namespace lbm

// lbm_batch_kern.cu -- batched step kernels of one storage type: LBM_INST_S (lbm_store value) is
// set by the build, one object per type.
#include "lbm_batch.cuh"

#ifndef LBM_INST_S
#error "lbm_batch_kern.cu is compiled with -DLBM_INST_S=<store>"
#endif

namespace lbm {
namespace batch {

template <>
void launch_batch_s<LBM_INST_S>(int sh, bool neighbor, const BatchTables &t, const BatchParams *p, unsigned blocks,
                                cudaStream_t s) {
    if (neighbor) launch_shape<LBM_INST_S, true>(sh, t, p, blocks, s);
    else launch_shape<LBM_INST_S, false>(sh, t, p, blocks, s);
}

}  // namespace batch
}  // namespace lbm

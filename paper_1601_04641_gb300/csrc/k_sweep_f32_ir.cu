// Line-solve kernels: float, form FImagReal.
#include "k_sweep_inst.cuh"

namespace gpcn {
cudaError_t launch_sweep_f32_ir(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    return launch_form<FImagReal<float>, float>(L, a, s);
}
}  // namespace gpcn

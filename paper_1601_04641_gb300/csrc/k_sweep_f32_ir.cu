// Line-solve kernels: float, form FImagReal.
#include "k_sweep_inst.cuh"

namespace gpcn {
cudaError_t launch_sweep_f32_ir(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    return launch_form<FImagReal<float>, float>(L, a, s);
}
cudaError_t launch_sweep_f32_ir_batch(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s) {
    return launch_batch_form<FImagReal<float>, float>(L, b, s);
}
}  // namespace gpcn

// Line-solve kernels: float, form FRealTime.
#include "k_sweep_inst.cuh"

namespace gpcn {
cudaError_t launch_sweep_f32_rt(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    return launch_form<FRealTime<float>, float>(L, a, s);
}
cudaError_t launch_sweep_f32_rt_batch(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s) {
    return launch_batch_form<FRealTime<float>, float>(L, b, s);
}
}  // namespace gpcn

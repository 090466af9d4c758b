// Line-solve kernels: double, form FRealTime.
#include "k_sweep_inst.cuh"

namespace gpcn {
cudaError_t launch_sweep_f64_rt(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    return launch_form<FRealTime<double>, double>(L, a, s);
}
cudaError_t launch_sweep_f64_rt_batch(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s) {
    return launch_batch_form<FRealTime<double>, double>(L, b, s);
}
}  // namespace gpcn

// Line-solve kernels: double, form FImagCplx.
#include "k_sweep_inst.cuh"

namespace gpcn {
cudaError_t launch_sweep_f64_ic(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    return launch_form<FImagCplx<double>, double>(L, a, s);
}
cudaError_t launch_sweep_f64_ic_batch(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s) {
    return launch_batch_form<FImagCplx<double>, double>(L, b, s);
}
}  // namespace gpcn

// Line-solve kernels: double, form FImagReal.
#include "k_sweep_inst.cuh"

namespace gpcn {
cudaError_t launch_sweep_f64_ir(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    return launch_form<FImagReal<double>, double>(L, a, s);
}
cudaError_t launch_sweep_f64_ir_batch(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s) {
    return launch_batch_form<FImagReal<double>, double>(L, b, s);
}
}  // namespace gpcn

// Line-solve kernels: double, form FImagReal.
#include "k_sweep_inst.cuh"

namespace gpcn {
cudaError_t launch_sweep_f64_ir(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    return launch_form<FImagReal<double>, double>(L, a, s);
}
}  // namespace gpcn

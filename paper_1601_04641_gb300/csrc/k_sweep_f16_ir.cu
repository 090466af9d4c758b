// Line-solve kernels: FP16 storage, FP32 arithmetic, form FImagReal.
#include "k_sweep_inst.cuh"

namespace gpcn {
cudaError_t launch_sweep_f16_ir(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    return launch_form<FImagRealH, float>(L, a, s);
}
}  // namespace gpcn

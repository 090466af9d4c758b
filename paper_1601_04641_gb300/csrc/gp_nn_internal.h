// gp_nn_internal.h -- layouts and launch interface of the warm-start network.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace gpcn {

constexpr int kNNIn = 16;      // input features (9 used, zero padded to one MMA k-tile)
constexpr int kNNHidden = 64;  // width of the three hidden layers

// FP32 master parameters, in this order ([in][out] row-major matrices):
//   W0 16x64, b0 64, W1 64x64, b1 64, W2 64x64, b2 64, w3 64, b3 1.
constexpr int kOffW0 = 0;
constexpr int kOffB0 = kOffW0 + kNNIn * kNNHidden;
constexpr int kOffW1 = kOffB0 + kNNHidden;
constexpr int kOffB1 = kOffW1 + kNNHidden * kNNHidden;
constexpr int kOffW2 = kOffB1 + kNNHidden;
constexpr int kOffB2 = kOffW2 + kNNHidden * kNNHidden;
constexpr int kOffW3 = kOffB2 + kNNHidden;
constexpr int kOffB3 = kOffW3 + kNNHidden;
constexpr int kNNParams = kOffB3 + 1;  // 9473

// BF16 copies the kernels read: W0^T [out][in], W1^T, W2^T [out][in] for the
// forward pass and W1, W2 [in][out] for back-propagation.
constexpr int kDepW0T = 0;
constexpr int kDepW1T = kDepW0T + kNNHidden * kNNIn;
constexpr int kDepW2T = kDepW1T + kNNHidden * kNNHidden;
constexpr int kDepW1N = kDepW2T + kNNHidden * kNNHidden;
constexpr int kDepW2N = kDepW1N + kNNHidden * kNNHidden;
constexpr int kDeployCount = kDepW2N + kNNHidden * kNNHidden;

struct NNParams {
    float *master;            // kNNParams
    float *m, *v;             // Adam moments
    __nv_bfloat16 *deploy;    // kDeployCount
};

// One condensate as the network sees it.  Features of the node at x:
//   f0..f2 = min(w_a x_a^2, 16) / 8 - 1         (per axis, even in x_a: the
//            ground state of the symmetric trap on the symmetric grid is
//            even in x, y and z, and so is every prediction)
//   f3     = min(sum (x_a / R_a)^2, 4) / 2 - 1  (Thomas-Fermi radii
//            R_a = sqrt(2 mu_TF) / w_a, mu_TF = (15 g w_x w_y w_z / 4 pi)^(2/5) / 2)
//   f4     = min(sum w_a x_a^2, 16) / 8 - 1
//   f5     = (ln g - 3.1) / 3.1
//   f6..f8 = (w_a - 1.75) / 1.25
//   f9..f15 = 0
struct NNInstance {
    int n[3];
    float origin[3], d[3];
    float sqrt_w[3], inv_rtf[3], wn[3], lg;
    long long sites;
    long long data_off;       // offset of its target amplitudes in the data array
    float inv_max;            // 1 / max |psi| of its target
};

struct NNTrain {
    const NNInstance *inst;
    int n_inst;
    const float *data;        // target amplitudes of all instances
    const int *sample_inst;   // explicit samples (or null: SplitMix64 draws from seed)
    const long long *sample_site;
    unsigned long long seed;
    int points;               // samples per step (multiple of 128)
    float *partials;          // [blocks][kNNParams]
    float *loss_partials;     // [blocks]
    float *grad;              // kNNParams
    float *loss;              // 1
};

__device__ __forceinline__ void write_deploy(const NNParams &P, int q, float w) {
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    if (q < kOffB0) {
        const int i = (q - kOffW0) / kNNHidden, o = (q - kOffW0) % kNNHidden;
        P.deploy[kDepW0T + o * kNNIn + i] = b;
    } else if (q >= kOffW1 && q < kOffB1) {
        const int i = (q - kOffW1) / kNNHidden, o = (q - kOffW1) % kNNHidden;
        P.deploy[kDepW1T + o * kNNHidden + i] = b;
        P.deploy[kDepW1N + i * kNNHidden + o] = b;
    } else if (q >= kOffW2 && q < kOffB2) {
        const int i = (q - kOffW2) / kNNHidden, o = (q - kOffW2) % kNNHidden;
        P.deploy[kDepW2T + o * kNNHidden + i] = b;
        P.deploy[kDepW2N + i * kNNHidden + o] = b;
    }
}

// Host side: the network's view of one condensate, and its parameters.
NNInstance make_nn_instance(const int n[3], const double d[3], const double w[3], double g);

size_t nn_train_smem();
cudaError_t nn_launch_train(const NNParams &P, const NNTrain &T, int blocks, cudaStream_t s);
cudaError_t nn_launch_adam(const NNParams &P, const float *grad, float lr, float b1t, float b2t, cudaStream_t s);
cudaError_t nn_launch_deploy(const NNParams &P, cudaStream_t s);
cudaError_t nn_launch_predict(const NNParams &P, const NNInstance &I, void *out, bool f32, bool cplx,
                              cudaStream_t s);

}  // namespace gpcn

struct gp_nn_s;
namespace gpcn {
const NNParams *nn_params(gp_nn_s *net);
}

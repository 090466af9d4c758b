// gp_nn.cu -- C ABI of the warm-start network: creation, parameters,
// training set, Adam training steps on the GPU, explicit-sample gradients.
#include "gp.h"
#include "gp_internal.h"
#include "gp_nn_internal.h"

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace gpcn;

struct gp_nn_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    NNParams P{};
    NNInstance *d_inst = nullptr;
    int n_inst = 0;
    std::vector<NNInstance> inst;
    const float *data = nullptr;
    float *d_grad = nullptr, *d_loss = nullptr, *d_partials = nullptr, *d_lpart = nullptr;
    int part_blocks = 0;
    long long adam_t = 0;
    std::string err;
};

namespace {

gp_status nfail(gp_nn net, gp_status st, const std::string &m) {
    if (net) net->err = m;
    else set_thread_error(m.c_str());
    return st;
}

#define GPN_CK(n, call)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return nfail((n), GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

// SplitMix64 (Steele, Lea and Flood 2014), host side, for the weight init.
unsigned long long mix(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

gp_status ensure_partials(gp_nn net, int blocks) {
    if (blocks <= net->part_blocks) return GP_OK;
    cudaFree(net->d_partials);
    cudaFree(net->d_lpart);
    net->d_partials = nullptr;
    net->d_lpart = nullptr;
    if (gpcn::dev_malloc(&net->d_partials, (size_t)blocks * kNNParams * sizeof(float)) != cudaSuccess ||
        gpcn::dev_malloc(&net->d_lpart, (size_t)blocks * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        net->part_blocks = 0;
        return nfail(net, GP_ERR_NOMEM, "cudaMalloc of gradient partials failed");
    }
    net->part_blocks = blocks;
    return GP_OK;
}

gp_status nenter(gp_nn net) {
    if (!net) return nfail(nullptr, GP_ERR_ARG, "NULL network");
    if (cudaSetDevice(net->device) != cudaSuccess) {
        cudaGetLastError();
        return nfail(net, GP_ERR_CUDA, "cudaSetDevice failed");
    }
    return GP_OK;
}

}  // namespace

namespace gpcn {

NNInstance make_nn_instance(const int n[3], const double d[3], const double w[3], double g) {
    NNInstance I;
    std::memset(&I, 0, sizeof(I));
    const double mu_tf = 0.5 * std::pow(15.0 * std::fabs(g) * w[0] * w[1] * w[2] / (4.0 * M_PI), 0.4);
    for (int a = 0; a < 3; ++a) {
        I.n[a] = n[a];
        I.d[a] = (float)d[a];
        I.origin[a] = (float)(-0.5 * (n[a] - 1) * d[a]);
        I.sqrt_w[a] = (float)std::sqrt(w[a]);
        const double r = w[a] > 0.0 ? std::sqrt(2.0 * mu_tf) / w[a] : 0.0;
        I.inv_rtf[a] = r > 0.0 ? (float)(1.0 / r) : 0.f;
        I.wn[a] = (float)((w[a] - 1.75) / 1.25);
    }
    I.lg = (float)((std::log(std::fmax(std::fabs(g), 1e-12)) - 3.1) / 3.1);
    I.sites = (long long)n[0] * n[1] * n[2];
    I.inv_max = 1.f;
    return I;
}

const NNParams *nn_params(gp_nn net) { return net ? &net->P : nullptr; }

}  // namespace gpcn

extern "C" {

int gp_nn_param_count(void) { return kNNParams; }

gp_status gp_nn_create(gp_nn *out, unsigned long long seed, void *cuda_stream) {
    if (!out) return nfail(nullptr, GP_ERR_ARG, "out is NULL");
    *out = nullptr;
    gp_nn net = new (std::nothrow) gp_nn_s();
    if (!net) return nfail(nullptr, GP_ERR_NOMEM, "host allocation failed");
    if (cudaGetDevice(&net->device) != cudaSuccess) {
        cudaGetLastError();
        delete net;
        return nfail(nullptr, GP_ERR_CUDA, "no CUDA device");
    }
    net->stream = static_cast<cudaStream_t>(cuda_stream);
    if (gpcn::dev_malloc(&net->P.master, kNNParams * sizeof(float)) != cudaSuccess ||
        gpcn::dev_malloc(&net->P.m, kNNParams * sizeof(float)) != cudaSuccess ||
        gpcn::dev_malloc(&net->P.v, kNNParams * sizeof(float)) != cudaSuccess ||
        gpcn::dev_malloc(&net->P.deploy, kDeployCount * sizeof(__nv_bfloat16)) != cudaSuccess ||
        gpcn::dev_malloc(&net->d_grad, kNNParams * sizeof(float)) != cudaSuccess ||
        gpcn::dev_malloc(&net->d_loss, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        gp_nn_destroy(net);
        return nfail(nullptr, GP_ERR_NOMEM, "cudaMalloc of the network failed");
    }
    // Glorot-uniform weights from a SplitMix64 stream, zero biases
    std::vector<float> w(kNNParams, 0.f);
    unsigned long long state = seed;
    auto uni = [&]() { return (double)(mix(state++) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; };
    auto fill = [&](int off, int fan_in, int fan_out, int rows_used) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int i = 0; i < fan_in; ++i)
            for (int o = 0; o < fan_out; ++o) w[off + i * fan_out + o] = i < rows_used ? (float)(a * uni()) : 0.f;
    };
    fill(kOffW0, kNNIn, kNNHidden, 9);
    fill(kOffW1, kNNHidden, kNNHidden, kNNHidden);
    fill(kOffW2, kNNHidden, kNNHidden, kNNHidden);
    fill(kOffW3, kNNHidden, 1, kNNHidden);
    gp_status st = gp_nn_set_params(net, w.data(), kNNParams);
    if (st != GP_OK) {
        std::string m = net->err;
        gp_nn_destroy(net);
        return nfail(nullptr, st, m);
    }
    *out = net;
    return GP_OK;
}

void gp_nn_destroy(gp_nn net) {
    if (!net) return;
    cudaSetDevice(net->device);
    if (net->stream) cudaStreamSynchronize(net->stream);
    cudaFree(net->P.master);
    cudaFree(net->P.m);
    cudaFree(net->P.v);
    cudaFree(net->P.deploy);
    cudaFree(net->d_inst);
    cudaFree(net->d_grad);
    cudaFree(net->d_loss);
    cudaFree(net->d_partials);
    cudaFree(net->d_lpart);
    cudaGetLastError();
    delete net;
}

gp_status gp_nn_set_params(gp_nn net, const float *params, int count) {
    gp_status st = nenter(net);
    if (st != GP_OK) return st;
    if (!params || count != kNNParams) return nfail(net, GP_ERR_ARG, "need gp_nn_param_count() parameters");
    GPN_CK(net, cudaMemcpyAsync(net->P.master, params, kNNParams * sizeof(float), cudaMemcpyHostToDevice, net->stream));
    GPN_CK(net, cudaMemsetAsync(net->P.m, 0, kNNParams * sizeof(float), net->stream));
    GPN_CK(net, cudaMemsetAsync(net->P.v, 0, kNNParams * sizeof(float), net->stream));
    GPN_CK(net, cudaMemsetAsync(net->P.deploy, 0, kDeployCount * sizeof(__nv_bfloat16), net->stream));
    GPN_CK(net, nn_launch_deploy(net->P, net->stream));
    GPN_CK(net, cudaStreamSynchronize(net->stream));
    net->adam_t = 0;
    return GP_OK;
}

gp_status gp_nn_get_params(gp_nn net, float *params, int count) {
    gp_status st = nenter(net);
    if (st != GP_OK) return st;
    if (!params || count != kNNParams) return nfail(net, GP_ERR_ARG, "need gp_nn_param_count() parameters");
    GPN_CK(net, cudaMemcpyAsync(params, net->P.master, kNNParams * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
    GPN_CK(net, cudaStreamSynchronize(net->stream));
    return GP_OK;
}

gp_status gp_nn_set_data(gp_nn net, int n, const gp_grid *grids, const double *gamma, const double *nu,
                         const double *lambda, const double *g, const float *dev_data, const long long *offsets,
                         const float *psi_max) {
    gp_status st = nenter(net);
    if (st != GP_OK) return st;
    if (n < 1 || !grids || !gamma || !nu || !lambda || !g || !dev_data || !offsets || !psi_max)
        return nfail(net, GP_ERR_ARG, "bad training set description");
    net->inst.clear();
    for (int i = 0; i < n; ++i) {
        const int nn[3] = {grids[i].nx, grids[i].ny, grids[i].nz};
        const double dd[3] = {grids[i].dx, grids[i].dy, grids[i].dz};
        const double w[3] = {gamma[i], nu[i], lambda[i]};
        NNInstance I = make_nn_instance(nn, dd, w, g[i]);
        if (!(psi_max[i] > 0.f)) return nfail(net, GP_ERR_ARG, "psi_max must be > 0");
        I.data_off = offsets[i];
        I.inv_max = 1.f / psi_max[i];
        net->inst.push_back(I);
    }
    cudaFree(net->d_inst);
    net->d_inst = nullptr;
    if (gpcn::dev_malloc(&net->d_inst, n * sizeof(NNInstance)) != cudaSuccess) {
        cudaGetLastError();
        return nfail(net, GP_ERR_NOMEM, "cudaMalloc of the instance table failed");
    }
    GPN_CK(net, cudaMemcpyAsync(net->d_inst, net->inst.data(), n * sizeof(NNInstance), cudaMemcpyHostToDevice,
                                net->stream));
    GPN_CK(net, cudaStreamSynchronize(net->stream));
    net->n_inst = n;
    net->data = dev_data;
    return GP_OK;
}

gp_status gp_nn_train(gp_nn net, int steps, int points, float lr, unsigned long long seed, float *loss) {
    gp_status st = nenter(net);
    if (st != GP_OK) return st;
    if (!net->d_inst) return nfail(net, GP_ERR_STATE, "no training set (gp_nn_set_data)");
    if (steps < 0 || points < 128 || points % 128 || !(lr > 0.f)) return nfail(net, GP_ERR_ARG, "bad training arguments");
    const int blocks = points / 128;
    if ((st = ensure_partials(net, blocks)) != GP_OK) return st;
    NNTrain T{};
    T.inst = net->d_inst;
    T.n_inst = net->n_inst;
    T.data = net->data;
    T.points = points;
    T.partials = net->d_partials;
    T.loss_partials = net->d_lpart;
    T.grad = net->d_grad;
    T.loss = net->d_loss;
    for (int s = 0; s < steps; ++s) {
        T.seed = mix(seed + 0x632BE59BD9B4E019ULL * (unsigned long long)(net->adam_t + 1));
        GPN_CK(net, nn_launch_train(net->P, T, blocks, net->stream));
        net->adam_t += 1;
        const float b1t = (float)std::pow(0.9, (double)net->adam_t), b2t = (float)std::pow(0.999, (double)net->adam_t);
        GPN_CK(net, nn_launch_adam(net->P, net->d_grad, lr, b1t, b2t, net->stream));
    }
    if (loss) {
        GPN_CK(net, cudaMemcpyAsync(loss, net->d_loss, sizeof(float), cudaMemcpyDeviceToHost, net->stream));
        GPN_CK(net, cudaStreamSynchronize(net->stream));
    }
    return GP_OK;
}

gp_status gp_nn_loss_grad(gp_nn net, int count, const int *instance, const long long *site, float *loss,
                          float *grad) {
    gp_status st = nenter(net);
    if (st != GP_OK) return st;
    if (!net->d_inst) return nfail(net, GP_ERR_STATE, "no training set (gp_nn_set_data)");
    if (count < 128 || count % 128 || !instance || !site) return nfail(net, GP_ERR_ARG, "count must be a multiple of 128");
    for (int p = 0; p < count; ++p)
        if (instance[p] < 0 || instance[p] >= net->n_inst || site[p] < 0 || site[p] >= net->inst[instance[p]].sites)
            return nfail(net, GP_ERR_ARG, "sample out of range");
    const int blocks = count / 128;
    if ((st = ensure_partials(net, blocks)) != GP_OK) return st;
    int *d_i = nullptr;
    long long *d_s = nullptr;
    if (gpcn::dev_malloc(&d_i, count * sizeof(int)) != cudaSuccess || gpcn::dev_malloc(&d_s, count * sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_i);
        return nfail(net, GP_ERR_NOMEM, "cudaMalloc of the samples failed");
    }
    NNTrain T{};
    T.inst = net->d_inst;
    T.n_inst = net->n_inst;
    T.data = net->data;
    T.sample_inst = d_i;
    T.sample_site = d_s;
    T.points = count;
    T.partials = net->d_partials;
    T.loss_partials = net->d_lpart;
    T.grad = net->d_grad;
    T.loss = net->d_loss;
    cudaError_t e = cudaMemcpyAsync(d_i, instance, count * sizeof(int), cudaMemcpyHostToDevice, net->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_s, site, count * sizeof(long long), cudaMemcpyHostToDevice, net->stream);
    if (e == cudaSuccess) e = nn_launch_train(net->P, T, blocks, net->stream);
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, net->d_grad, kNNParams * sizeof(float), cudaMemcpyDeviceToHost, net->stream);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, net->d_loss, sizeof(float), cudaMemcpyDeviceToHost, net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    cudaFree(d_i);
    cudaFree(d_s);
    if (e != cudaSuccess) return nfail(net, GP_ERR_CUDA, std::string("gradient evaluation failed: ") + cudaGetErrorString(e));
    return GP_OK;
}

const char *gp_nn_last_error(gp_nn net) {
    if (!net) return gp_last_error(nullptr);
    return net->err.c_str();
}

}  // extern "C"

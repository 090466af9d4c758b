// k_noalloc.cu -- gp_observables_noalloc: the observables reduction over a
// caller-owned device psi that allocates no device memory at all.
//
// Who needs it: code that cannot call cudaMalloc -- for example a host
// framework that owns every byte of device memory through its own pool and
// hands out only the buffers it manages, or a latency-critical loop that must
// not pay the implicit device synchronisation of cudaMalloc / cudaFree.  The
// handle-based gp_observables needs a handle, and creating one allocates
// psi's second buffer, the coefficient tables and the reduction partials.
//
// How: the two-stage reduction keeps its per-block partial sums and its
// last-block-done counter in one file-scope __device__ array of fixed size
// (kNoAllocBytes below).  Every GPU that loads this library holds that array
// until the process exits.  Host code cannot use the array's name as a
// device address, so on the first call made on each device (with that device
// current) the library asks the runtime for the array's address with
// cudaGetSymbolAddress and caches it; make that first call before any stream
// capture on the device.  All calls share the one array and it keeps the
// contents of the last call: each call clears the counter before its launch,
// and calls whose launches overlap on the GPU (different streams, no ordering
// between them) race on the array and give undefined results.
#include "gp.h"
#include "gp_sweep.cuh"

#include <mutex>
#include <string>

namespace gpcn {
void set_thread_error(const char *msg);  // gp_api.cu: the message gp_last_error(NULL) returns

namespace {

// Partial sums of up to kNoAllocBlocks blocks (9 doubles each) and the counter.
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocBlocks = 8192;  // one block per 256 (y, z) lines: ny*nz <= 2,097,152
constexpr size_t kPartialBytes = (size_t)kNoAllocBlocks * 9 * sizeof(double);
constexpr size_t kNoAllocBytes = kPartialBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocArgs {
    const void *psi;
    int n[3];
    double d[3], origin[3], half_w2[3];
    double g, scale, dV;
    double *partials;       // first kPartialBytes of the scratch array
    unsigned int *counter;  // right after them
    double *out;            // caller's device buffer of 16 doubles
};

template <typename R, bool CPLX> struct NAElem;
template <typename R> struct NAElem<R, false> {
    using V = R;
    __device__ __forceinline__ static R abs2(V v) { return v * v; }
    __device__ __forceinline__ static V scaled(V v, R s) { return v * s; }
    __device__ __forceinline__ static R diff2(V a, V b) { const R d = a - b; return d * d; }
};
template <typename R> struct NAElem<R, true> {
    using V = cx<R>;
    __device__ __forceinline__ static R abs2(V v) { return fma(v.re, v.re, v.im * v.im); }
    __device__ __forceinline__ static V scaled(V v, R s) { return V{v.re * s, v.im * s}; }
    __device__ __forceinline__ static R diff2(V a, V b) {
        const R dr = a.re - b.re, di = a.im - b.im;
        return dr * dr + di * di;
    }
};

// Same sums as the handle path's observables reduction: per (j, k) thread a
// walk along i adding |psi|^2, V|psi|^2, |psi|^4, x^2|psi|^2, y^2|psi|^2,
// z^2|psi|^2 and the squared forward differences along x, y and z; block
// partials in FP64; the last block sums them in block order and writes the
// 9 raw sums and norm, mu, energy, rms_x, rms_y, rms_z and a finiteness flag.
template <typename R, bool CPLX>
__global__ void __launch_bounds__(kNoAllocThreads) observables_noalloc_kernel(NoAllocArgs a) {
    using E = NAElem<R, CPLX>;
    using V = typename E::V;
    const V *psi = static_cast<const V *>(a.psi);
    const long long plane = (long long)a.n[1] * a.n[2];
    const long long L = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    Acc<R> acc[9];
    if (L < plane) {
        const int j = (int)(L / a.n[2]), k = (int)(L % a.n[2]);
        const R s = (R)a.scale;
        const R y = (R)(a.origin[1] + j * a.d[1]);
        const R z = (R)(a.origin[2] + k * a.d[2]);
        const R vyz = (R)a.half_w2[1] * y * y + (R)a.half_w2[2] * z * z;
        const R x0 = (R)a.origin[0], dx = (R)a.d[0], hx = (R)a.half_w2[0];
        const bool has_y = j + 1 < a.n[1], has_z = k + 1 < a.n[2];
        V prev{};
        for (int i = 0; i < a.n[0]; ++i) {
            const long long off = i * plane + L;
            const V p = E::scaled(psi[off], s);
            const R rho = E::abs2(p);
            const R x = fma((R)i, dx, x0);
            acc[O_RHO].add(rho);
            acc[O_V].add(fma(hx * x, x, vyz) * rho);
            acc[O_RHO2].add(rho * rho);
            acc[O_X2].add(x * x * rho);
            acc[O_Y2].add(y * y * rho);
            acc[O_Z2].add(z * z * rho);
            if (i > 0) acc[O_LX].add(E::diff2(p, prev));
            if (has_y) acc[O_LY].add(E::diff2(E::scaled(psi[off + a.n[2]], s), p));
            if (has_z) acc[O_LZ].add(E::diff2(E::scaled(psi[off + 1], s), p));
            prev = p;
        }
    }
    __shared__ double red[32];
    __shared__ int is_last;
    double bs[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) bs[q] = block_sum(acc[q].value(), red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) a.partials[(long long)blockIdx.x * 9 + q] = bs[q];
        __threadfence();
        const unsigned prev = atomicAdd(a.counter, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double t[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        double sum = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) sum += __ldcg(a.partials + (long long)b * 9 + q);
        t[q] = block_sum(sum, red);
    }
    if (threadIdx.x == 0) {
        double *o = a.out;
        for (int q = 0; q < 9; ++q) o[q] = t[q];
        const double dv = a.dV;
        const double nrm = dv * t[O_RHO];
        const double kin = 0.5 * dv * (t[O_LX] / (a.d[0] * a.d[0]) + t[O_LY] / (a.d[1] * a.d[1]) +
                                       t[O_LZ] / (a.d[2] * a.d[2]));
        const double pot = dv * t[O_V];
        const double inter = dv * t[O_RHO2];
        o[O_NORM] = nrm;
        o[O_MU] = (kin + pot + a.g * inter) / nrm;
        o[O_E] = (kin + pot + 0.5 * a.g * inter) / nrm;
        o[O_RMSX] = sqrt(dv * t[O_X2] / nrm);
        o[O_RMSY] = sqrt(dv * t[O_Y2] / nrm);
        o[O_RMSZ] = sqrt(dv * t[O_Z2] / nrm);
        bool fin = true;
        for (int q = 0; q < 15; ++q) fin = fin && isfinite(o[q]);
        o[O_FINITE] = fin ? 1.0 : 0.0;
        *a.counter = 0u;
    }
}

gp_status na_fail(gp_status st, const std::string &m) {
    set_thread_error(m.c_str());  // read back with gp_last_error(NULL)
    return st;
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void *g_addr[kMaxDevices] = {};

gp_status scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return na_fail(GP_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return na_fail(GP_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                            cudaGetErrorString(e));
        }
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return GP_OK;
}

}  // namespace
}  // namespace gpcn

using namespace gpcn;

extern "C" gp_status gp_observables_noalloc(const void *dev_psi, gp_grid grid, gp_precision prec,
                                            gp_field field, double gamma, double nu, double lambda,
                                            double g, double scale, double *dev_out,
                                            void *cuda_stream) {
    if (!dev_psi || !dev_out) return na_fail(GP_ERR_ARG, "dev_psi and dev_out must be device pointers");
    const int n[3] = {grid.nx, grid.ny, grid.nz};
    const double d[3] = {grid.dx, grid.dy, grid.dz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 3) return na_fail(GP_ERR_ARG, "every axis needs at least 3 nodes");
        if (!(d[a] > 0.0) || !isfinite(d[a])) return na_fail(GP_ERR_ARG, "spacings must be finite and > 0");
    }
    const double w[3] = {gamma, nu, lambda};
    for (double x : w)
        if (!isfinite(x) || x < 0.0) return na_fail(GP_ERR_ARG, "trap frequencies must be finite and >= 0");
    if (!isfinite(g) || !isfinite(scale)) return na_fail(GP_ERR_ARG, "g and scale must be finite");
    if (prec != GP_F64 && prec != GP_F32) return na_fail(GP_ERR_ARG, "unknown precision");
    if (field != GP_COMPLEX && field != GP_REAL) return na_fail(GP_ERR_ARG, "unknown field");
    const long long plane = (long long)n[1] * n[2];
    const long long blocks = (plane + kNoAllocThreads - 1) / kNoAllocThreads;
    if (blocks > kNoAllocBlocks)
        return na_fail(GP_ERR_ARG, "ny*nz = " + std::to_string(plane) +
                                       " exceeds the no-allocation limit of " +
                                       std::to_string((long long)kNoAllocBlocks * kNoAllocThreads) +
                                       " (the scratch array holds 8192 block partials)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return na_fail(GP_ERR_CUDA, "no current CUDA device");
    }
    unsigned char *base = nullptr;
    gp_status st = scratch_address(dev, &base);
    if (st != GP_OK) return st;

    NoAllocArgs a;
    a.psi = dev_psi;
    for (int q = 0; q < 3; ++q) {
        a.n[q] = n[q];
        a.d[q] = d[q];
        a.origin[q] = -0.5 * (n[q] - 1) * d[q];
        a.half_w2[q] = 0.5 * w[q] * w[q];
    }
    a.g = g;
    a.scale = scale;
    a.dV = d[0] * d[1] * d[2];
    a.partials = reinterpret_cast<double *>(base);
    a.counter = reinterpret_cast<unsigned int *>(base + kPartialBytes);
    a.out = dev_out;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the counter must start at zero (a previous call leaves it at zero, but
    // nothing guarantees that an earlier launch completed)
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        if (prec == GP_F64) {
            if (field == GP_COMPLEX) observables_noalloc_kernel<double, true><<<(unsigned)blocks, kNoAllocThreads, 0, s>>>(a);
            else observables_noalloc_kernel<double, false><<<(unsigned)blocks, kNoAllocThreads, 0, s>>>(a);
        } else {
            if (field == GP_COMPLEX) observables_noalloc_kernel<float, true><<<(unsigned)blocks, kNoAllocThreads, 0, s>>>(a);
            else observables_noalloc_kernel<float, false><<<(unsigned)blocks, kNoAllocThreads, 0, s>>>(a);
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return na_fail(GP_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    return GP_OK;
}

// k_field.cu -- whole-field kernels: Gaussian initial state, norm, the
// observables reduction (calcrms, calcmuen) and applying a pending scale.
#include "gp_sweep.cuh"

namespace gpcn {

namespace {

template <typename R, bool CPLX> struct Elem;
template <typename R> struct Elem<R, false> {
    using V = R;
    __device__ __forceinline__ static double abs2(V v) { return (double)v * (double)v; }
    __device__ __forceinline__ static R abs2r(V v) { return v * v; }
    __device__ __forceinline__ static V from_real(double x) { return (R)x; }
    __device__ __forceinline__ static V scaled(V v, R s) { return v * s; }
};
template <typename R> struct Elem<R, true> {
    using V = cx<R>;
    __device__ __forceinline__ static double abs2(V v) {
        return (double)v.re * (double)v.re + (double)v.im * (double)v.im;
    }
    __device__ __forceinline__ static R abs2r(V v) { return fma(v.re, v.re, v.im * v.im); }
    __device__ __forceinline__ static V from_real(double x) { return V{(R)x, R(0)}; }
    __device__ __forceinline__ static V scaled(V v, R s) { return V{v.re * s, v.im * s}; }
};

__device__ __forceinline__ long long grid_stride() { return (long long)gridDim.x * blockDim.x; }

// Unnormalised product Gaussian prod_a (w_a/pi)^(1/4) exp(-w_a a^2/2), zero on
// the boundary nodes.  FP64 arithmetic, stored in the field's precision.
template <typename R, bool CPLX>
__global__ void gaussian_kernel(FieldArgs a) {
    using E = Elem<R, CPLX>;
    typename E::V *psi = static_cast<typename E::V *>(a.psi);
    const double pi = 3.14159265358979323846;
    const double c0 = pow(a.w[0] / pi, 0.25) * pow(a.w[1] / pi, 0.25) * pow(a.w[2] / pi, 0.25);
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < a.sites; s += grid_stride()) {
        const int k = (int)(s % a.n[2]);
        const int j = (int)((s / a.n[2]) % a.n[1]);
        const int i = (int)(s / ((long long)a.n[2] * a.n[1]));
        double v = 0.0;
        if (i > 0 && i < a.n[0] - 1 && j > 0 && j < a.n[1] - 1 && k > 0 && k < a.n[2] - 1) {
            const double x = a.origin[0] + i * a.d[0];
            const double y = a.origin[1] + j * a.d[1];
            const double z = a.origin[2] + k * a.d[2];
            v = c0 * exp(-0.5 * (a.w[0] * x * x + a.w[1] * y * y + a.w[2] * z * z));
        }
        psi[s] = E::from_real(v);
    }
}

// Reduce 9 FP64 values over the grid: block partials, then the last block
// sums them in block order (deterministic) and calls `fin`.
template <int NV, class Fin>
__device__ __forceinline__ void reduce_finalize(double (&v)[NV], const FieldArgs &a, Fin fin,
                                                unsigned block, unsigned nblocks) {
    __shared__ double red[32];
    __shared__ int is_last;
    double bs[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) bs[q] = block_sum(v[q], red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) a.partials[(long long)block * NV + q] = bs[q];
        __threadfence();
        unsigned prev = atomicAdd(a.counter, 1u);
        is_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double tot[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = 0.0;
        for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x)
            s += __ldcg(a.partials + (long long)b * NV + q);
        tot[q] = block_sum(s, red);
    }
    if (threadIdx.x == 0) {
        fin(tot);
        *a.counter = 0u;
    }
}

template <typename R, bool CPLX>
__global__ void __launch_bounds__(kReduceThreads) norm_kernel(FieldArgs a) {
    using E = Elem<R, CPLX>;
    const typename E::V *psi = static_cast<const typename E::V *>(a.psi);
    double acc = 0.0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < a.sites; s += grid_stride())
        acc += E::abs2(psi[s]);
    double v[1] = {acc};
    reduce_finalize<1>(
        v, a,
        [&](const double *tot) {
            const double nrm = a.dV * tot[0];
            *a.norm_out = nrm;
            *a.scale_out = 1.0 / sqrt(nrm);
        },
        blockIdx.x, gridDim.x);
}

// Observables: one thread per (j, k) walks along i.  Per site it adds |psi|^2,
// V|psi|^2, |psi|^4, x^2|psi|^2, y^2|psi|^2, z^2|psi|^2 and the squared
// forward differences to the +x, +y and +z neighbours (links that leave the
// grid do not exist).  psi is read through the pending scale.
template <typename R, bool CPLX>
__device__ __forceinline__ void observables_body(const FieldArgs &a, unsigned block, unsigned nblocks) {
    using E = Elem<R, CPLX>;
    using V = typename E::V;
    const V *psi = static_cast<const V *>(a.psi);
    const long long plane = (long long)a.n[1] * a.n[2];
    const long long L = (long long)block * blockDim.x + threadIdx.x;
    Acc<R> acc[9];
    if (L < plane) {
        const int j = (int)(L / a.n[2]), k = (int)(L % a.n[2]);
        const R s = (R)__ldg(a.scale);
        const R y = (R)(a.origin[1] + j * a.d[1]);
        const R z = (R)(a.origin[2] + k * a.d[2]);
        const R vyz = (R)a.half_w2[1] * y * y + (R)a.half_w2[2] * z * z;
        const R x0 = (R)a.origin[0], dx = (R)a.d[0], hx = (R)a.half_w2[0];
        const bool has_y = j + 1 < a.n[1], has_z = k + 1 < a.n[2];
        V prev = E::from_real(0.0);
        for (int i = 0; i < a.n[0]; ++i) {
            const long long off = i * plane + L;
            const V p = E::scaled(psi[off], s);
            const R rho = E::abs2r(p);
            const R x = fma((R)i, dx, x0);
            acc[O_RHO].add(rho);
            acc[O_V].add(fma(hx * x, x, vyz) * rho);
            acc[O_RHO2].add(rho * rho);
            acc[O_X2].add(x * x * rho);
            acc[O_Y2].add(y * y * rho);
            acc[O_Z2].add(z * z * rho);
            if (i > 0) {
                if constexpr (CPLX) {
                    const R dre = p.re - prev.re, dim = p.im - prev.im;
                    acc[O_LX].add(dre * dre + dim * dim);
                } else {
                    const R df = p - prev;
                    acc[O_LX].add(df * df);
                }
            }
            if (has_y) {
                const V q = E::scaled(psi[off + a.n[2]], s);
                if constexpr (CPLX) {
                    const R dre = q.re - p.re, dim = q.im - p.im;
                    acc[O_LY].add(dre * dre + dim * dim);
                } else {
                    const R df = q - p;
                    acc[O_LY].add(df * df);
                }
            }
            if (has_z) {
                const V q = E::scaled(psi[off + 1], s);
                if constexpr (CPLX) {
                    const R dre = q.re - p.re, dim = q.im - p.im;
                    acc[O_LZ].add(dre * dre + dim * dim);
                } else {
                    const R df = q - p;
                    acc[O_LZ].add(df * df);
                }
            }
            prev = p;
        }
    }
    double v[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] = acc[q].value();
    reduce_finalize<9>(v, a, [&](const double *t) {
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
    }, block, nblocks);
}

template <typename R, bool CPLX>
__global__ void __launch_bounds__(kReduceThreads) observables_kernel(FieldArgs a) {
    observables_body<R, CPLX>(a, blockIdx.x, gridDim.x);
}

// Many condensates in one launch: instance i owns blocks [first[i], first[i+1]).
template <typename R, bool CPLX>
__global__ void __launch_bounds__(kReduceThreads) observables_batch_kernel(const FieldArgs *args,
                                                                           const unsigned *first, int n) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(first + mid) <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const FieldArgs a = args[lo];
    const unsigned f = __ldg(first + lo);
    observables_body<R, CPLX>(a, blockIdx.x - f, __ldg(first + lo + 1) - f);
}

template <typename R, bool CPLX>
__global__ void apply_scale_kernel(FieldArgs a, void *dst) {
    using E = Elem<R, CPLX>;
    const typename E::V *src = static_cast<const typename E::V *>(a.psi);
    typename E::V *out = static_cast<typename E::V *>(dst);
    const R s = (R)__ldg(a.scale);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.sites; i += grid_stride())
        out[i] = E::scaled(src[i], s);
}

unsigned fill_blocks(long long sites) {
    long long b = (sites + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename R, bool CPLX>
cudaError_t dispatch(int what, const FieldArgs &a, int blocks, void *dst, cudaStream_t s) {
    switch (what) {
    case 0: gaussian_kernel<R, CPLX><<<fill_blocks(a.sites), 256, 0, s>>>(a); break;
    case 1: norm_kernel<R, CPLX><<<blocks, kReduceThreads, 0, s>>>(a); break;
    case 2: observables_kernel<R, CPLX><<<observables_blocks(a), kReduceThreads, 0, s>>>(a); break;
    case 3: apply_scale_kernel<R, CPLX><<<fill_blocks(a.sites), 256, 0, s>>>(a, dst); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t dispatch_all(Prec p, bool cplx, int what, const FieldArgs &a, int blocks, void *dst,
                         cudaStream_t s) {
    if (p == P_F64) return cplx ? dispatch<double, true>(what, a, blocks, dst, s)
                                : dispatch<double, false>(what, a, blocks, dst, s);
    return cplx ? dispatch<float, true>(what, a, blocks, dst, s)
                : dispatch<float, false>(what, a, blocks, dst, s);
}

}  // namespace

cudaError_t launch_observables_batch(Prec p, bool cplx, const FieldArgs *args, const unsigned *first, int n,
                                     unsigned total_blocks, cudaStream_t s) {
    if (total_blocks == 0) return cudaSuccess;
    if (p == P_F64) {
        if (cplx) observables_batch_kernel<double, true><<<total_blocks, kReduceThreads, 0, s>>>(args, first, n);
        else observables_batch_kernel<double, false><<<total_blocks, kReduceThreads, 0, s>>>(args, first, n);
    } else {
        if (cplx) observables_batch_kernel<float, true><<<total_blocks, kReduceThreads, 0, s>>>(args, first, n);
        else observables_batch_kernel<float, false><<<total_blocks, kReduceThreads, 0, s>>>(args, first, n);
    }
    return cudaGetLastError();
}

int observables_blocks(const FieldArgs &a) {
    const long long plane = (long long)a.n[1] * a.n[2];
    return (int)((plane + kReduceThreads - 1) / kReduceThreads);
}

cudaError_t launch_gaussian(Prec p, bool cplx, const FieldArgs &a, cudaStream_t s) {
    return dispatch_all(p, cplx, 0, a, 0, nullptr, s);
}
cudaError_t launch_norm(Prec p, bool cplx, const FieldArgs &a, int blocks, cudaStream_t s) {
    return dispatch_all(p, cplx, 1, a, blocks, nullptr, s);
}
cudaError_t launch_observables(Prec p, bool cplx, const FieldArgs &a, cudaStream_t s) {
    return dispatch_all(p, cplx, 2, a, 0, nullptr, s);
}
cudaError_t launch_apply_scale(Prec p, bool cplx, const FieldArgs &a, void *dst, cudaStream_t s) {
    return dispatch_all(p, cplx, 3, a, 0, dst, s);
}

}  // namespace gpcn

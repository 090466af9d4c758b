// k_output.cu -- integrated density profiles of the wavefunction (the 1D
// densities along x, y and z; the programs' density output).
//
//   rho_x(i) = s^2 dy dz sum_{j,k} |psi_ijk|^2,  likewise rho_y(j), rho_z(k),
//
// s the pending renormalisation factor, so that sum_i rho_x(i) dx is the norm.
// Deterministic: every sum runs in a fixed order, in FP64.
#include "gp_output.h"

namespace gpcn {

namespace {

template <typename R, bool CPLX> struct Abs2;
template <typename R> struct Abs2<R, false> {
    __device__ __forceinline__ static double of(const void *p, long long s) {
        const double v = (double)static_cast<const R *>(p)[s];
        return v * v;
    }
};
template <typename R> struct Abs2<R, true> {
    __device__ __forceinline__ static double of(const void *p, long long s) {
        const R *q = static_cast<const R *>(p) + 2 * s;
        const double re = (double)q[0], im = (double)q[1];
        return re * re + im * im;
    }
};

// One warp per (i, j) row: pxy[i ny + j] = sum_k |psi_ijk|^2 (lane-strided
// partial sums, then a fixed shuffle tree).
template <typename R, bool CPLX> __global__ void rows_z_kernel(FieldArgs a, double *pxy) {
    const long long rows = (long long)a.n[0] * a.n[1];
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const long long base = row * a.n[2];
    double acc = 0.0;
    for (int k = lane; k < a.n[2]; k += 32) acc += Abs2<R, CPLX>::of(a.psi, base + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) pxy[row] = acc;
}

// One thread per (i, k): pxz[i nz + k] = sum_j |psi_ijk|^2 in j order
// (consecutive threads read consecutive k).
template <typename R, bool CPLX> __global__ void cols_y_kernel(FieldArgs a, double *pxz) {
    const long long cols = (long long)a.n[0] * a.n[2];
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    const long long i = c / a.n[2], k = c % a.n[2];
    const long long plane = (long long)a.n[1] * a.n[2];
    double acc = 0.0;
    for (int j = 0; j < a.n[1]; ++j) acc += Abs2<R, CPLX>::of(a.psi, i * plane + (long long)j * a.n[2] + k);
    pxz[c] = acc;
}

// One thread per output node of the three profiles (x nodes, then y, then z).
__global__ void profiles_kernel(FieldArgs a, const double *pxy, const double *pxz, double *out) {
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nx + ny + nz) return;
    const double s = *a.scale;
    const double s2 = s * s;
    double acc = 0.0, w;
    if (t < nx) {  // rho_x(i) = sum_j pxy[i][j]
        for (int j = 0; j < ny; ++j) acc += pxy[(long long)t * ny + j];
        w = a.d[1] * a.d[2];
    } else if (t < nx + ny) {  // rho_y(j) = sum_i pxy[i][j]
        const int j = t - nx;
        for (int i = 0; i < nx; ++i) acc += pxy[(long long)i * ny + j];
        w = a.d[0] * a.d[2];
    } else {  // rho_z(k) = sum_i pxz[i][k]
        const int k = t - nx - ny;
        for (int i = 0; i < nx; ++i) acc += pxz[(long long)i * nz + k];
        w = a.d[0] * a.d[1];
    }
    out[t] = s2 * w * acc;
}

template <typename R, bool CPLX>
cudaError_t launch_profiles_t(const FieldArgs &a, double *scratch, double *out, cudaStream_t s) {
    const long long rows = (long long)a.n[0] * a.n[1], cols = (long long)a.n[0] * a.n[2];
    double *pxy = scratch, *pxz = scratch + rows;
    const int threads = 256;
    rows_z_kernel<R, CPLX><<<(unsigned)((rows * 32 + threads - 1) / threads), threads, 0, s>>>(a, pxy);
    cols_y_kernel<R, CPLX><<<(unsigned)((cols + threads - 1) / threads), threads, 0, s>>>(a, pxz);
    const int total = a.n[0] + a.n[1] + a.n[2];
    profiles_kernel<<<(total + threads - 1) / threads, threads, 0, s>>>(a, pxy, pxz, out);
    return cudaGetLastError();
}

}  // namespace

size_t profile_scratch_doubles(const FieldArgs &a) {
    return (size_t)a.n[0] * a.n[1] + (size_t)a.n[0] * a.n[2] + (size_t)(a.n[0] + a.n[1] + a.n[2]);
}

cudaError_t launch_density_profiles(Prec p, bool cplx, const FieldArgs &a, double *scratch, double *out,
                                    cudaStream_t s) {
    if (p == P_F64) return cplx ? launch_profiles_t<double, true>(a, scratch, out, s)
                                : launch_profiles_t<double, false>(a, scratch, out, s);
    return cplx ? launch_profiles_t<float, true>(a, scratch, out, s) : launch_profiles_t<float, false>(a, scratch, out, s);
}

}  // namespace gpcn

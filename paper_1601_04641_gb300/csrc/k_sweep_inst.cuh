// k_sweep_inst.cuh -- instantiates the line-solve kernels of one arithmetic
// form and precision and dispatches a launch to them.
#pragma once

#include "gp_sweep.cuh"

namespace gpcn {

template <class F, typename R>
static cudaError_t launch_contig(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    const unsigned threads = 32 * kTileWarps;
    const dim3 grid((unsigned)((a.n_lines + threads - 1) / threads), (unsigned)a.n_seg);
    switch (L.window) {
    case 4: sweep_contig_kernel<F, R, 4><<<grid, threads, 0, s>>>(a); break;
    case 8: sweep_contig_kernel<F, R, 8><<<grid, threads, 0, s>>>(a); break;
    case 16: sweep_contig_kernel<F, R, 16><<<grid, threads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class F, typename R, int KIND>
static cudaError_t launch_kind(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    if (KIND == K_Z && L.contiguous) return launch_contig<F, R>(L, a, s);
    const unsigned threads = (unsigned)L.threads;
    const dim3 grid((unsigned)((a.n_lines + threads - 1) / threads), (unsigned)a.n_seg);
    switch (L.window) {
    case 0: sweep_lines_kernel<F, R, 0, KIND><<<grid, threads, 0, s>>>(a); break;
    case 4: sweep_lines_kernel<F, R, 4, KIND><<<grid, threads, 0, s>>>(a); break;
    case 8: sweep_lines_kernel<F, R, 8, KIND><<<grid, threads, 0, s>>>(a); break;
    case 16: sweep_lines_kernel<F, R, 16, KIND><<<grid, threads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class F, typename R>
static cudaError_t launch_form(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    if (a.n_lines <= 0) return cudaSuccess;
    switch (L.kind) {
    case K_X: return launch_kind<F, R, K_X>(L, a, s);
    case K_Y: return launch_kind<F, R, K_Y>(L, a, s);
    case K_Z: return launch_kind<F, R, K_Z>(L, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gpcn

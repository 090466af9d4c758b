// k_sweep_inst.cuh -- instantiates the line-solve kernels of one arithmetic
// form and precision and dispatches a launch to them.
#pragma once

#include "gp_sweep.cuh"
#include "gp_sweep_tma.cuh"

namespace gpcn {

template <class F, typename R, int W>
static cudaError_t launch_contig_w(const SweepArgs &a, cudaStream_t s) {
    using V = typename F::V;
    const unsigned threads = 32 * kTileWarps;
    const dim3 grid((unsigned)((a.n_lines + threads - 1) / threads), (unsigned)a.n_seg);
    const size_t smem = kTileWarps * tile_warp_bytes<V, W>();
    static bool attr = false;  // opt in once to more than 48 KB of dynamic shared memory
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sweep_contig_kernel<F, R, W>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    sweep_contig_kernel<F, R, W><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <class F, typename R, int W>
static cudaError_t launch_tma_w(const SweepArgs &a, const TmaMaps &m, cudaStream_t s) {
    if constexpr (tma_supported<F, W>()) {
        const long long rows = (long long)kTmaWarps * kTmaRows;
        const unsigned grid = (unsigned)((a.n_lines + rows - 1) / rows);
        constexpr size_t smem = tma_smem_bytes<store_t<F>, W>();
        static bool attr = false;  // opt in once to more than 48 KB of dynamic shared memory
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(sweep_tma_kernel<F, R, W>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        sweep_tma_kernel<F, R, W><<<grid, kTmaWarps * 32, smem, s>>>(a, m);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

// Forms whose memory element differs from their arithmetic type (FP16
// storage) have only the TMA z sweep and the windowed strided sweeps with two
// or four lines per thread.
template <class F> constexpr bool narrow_store() { return !std::is_same<store_t<F>, typename F::V>::value; }

template <class F, typename R, int W>
static cudaError_t launch_contig_or_tma(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    if (L.tma && tma_usable<F, W>(a)) return launch_tma_w<F, R, W>(a, *L.tma, s);
    if constexpr (narrow_store<F>()) return cudaErrorInvalidValue;
    else return launch_contig_w<F, R, W>(a, s);
}

template <class F, typename R>
static cudaError_t launch_contig(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    switch (L.window) {
    case 4: return launch_contig_or_tma<F, R, 4>(L, a, s);
    case 8: return launch_contig_or_tma<F, R, 8>(L, a, s);
    case 16: return launch_contig_or_tma<F, R, 16>(L, a, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class F, typename R, int W, int KIND, int LPT>
static cudaError_t launch_lines_tma_wl(const SweepArgs &a, const TmaMaps &m, cudaStream_t s) {
    using MV = typename LinesPerThread<F, LPT>::M::MemV;
    const long long wpr = (a.inner / LPT + 31) / 32;  // warps per outer group (the last one may be partial)
    const long long warps = (a.n_lines / a.inner) * wpr;
    const dim3 grid((unsigned)((warps + kLineTmaWarps - 1) / kLineTmaWarps), (unsigned)a.n_seg);
    constexpr size_t smem = line_tma_smem<MV>();
    static bool attr = false;  // opt in once to more than 48 KB of dynamic shared memory
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sweep_lines_tma_kernel<F, R, W, KIND, LPT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    sweep_lines_tma_kernel<F, R, W, KIND, LPT><<<grid, kLineTmaWarps * 32, smem, s>>>(a, m);
    return cudaGetLastError();
}

template <class F, typename R, int W, int KIND, int LPT>
static cudaError_t launch_lines_wl_any(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    using V = typename LinesPerThread<F, LPT>::M::MemV;
    if constexpr (W > 0 && KIND != K_Z) {
        if (L.lmaps) return launch_lines_tma_wl<F, R, W, KIND, LPT>(a, *L.lmaps, s);
    }
    const unsigned threads = (unsigned)L.threads;
    const long long units = (a.n_lines + LPT - 1) / LPT;
    const dim3 grid((unsigned)((units + threads - 1) / threads), (unsigned)a.n_seg);
    const size_t smem = W > 0 ? column_ring_bytes<V>(threads) : 0;
    static int attr = 0;  // largest dynamic shared memory opted in so far
    if ((int)smem > attr && smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sweep_lines_kernel<F, R, W, KIND, LPT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = (int)smem;
    }
    sweep_lines_kernel<F, R, W, KIND, LPT><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <class F, typename R, int W, int KIND, int LPT>
static cudaError_t launch_lines_wl(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    using V = typename LinesPerThread<F, LPT>::M::MemV;
    if constexpr (narrow_store<F>() && (W == 0 || sizeof(V) < 4 || KIND == K_Z)) {
        return cudaErrorInvalidValue;
    } else {
        return launch_lines_wl_any<F, R, W, KIND, LPT>(L, a, s);
    }
}

template <class F, typename R, int W, int KIND>
static cudaError_t launch_lines_w(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    if constexpr (has_quad<F>() && W > 0) {
        if (L.lpt == 4) return launch_lines_wl<F, R, W, KIND, 4>(L, a, s);
    }
    if constexpr (sizeof(typename F::V) <= 8) {
        if (L.lpt == 2) return launch_lines_wl<F, R, W, KIND, 2>(L, a, s);
    }
    return launch_lines_wl<F, R, W, KIND, 1>(L, a, s);
}

template <class F, typename R, int KIND>
static cudaError_t launch_kind(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    if (KIND == K_Z && L.contiguous) return launch_contig<F, R>(L, a, s);
    switch (L.window) {
    case 0: return launch_lines_w<F, R, 0, KIND>(L, a, s);
    case 4: return launch_lines_w<F, R, 4, KIND>(L, a, s);
    case 8: return launch_lines_w<F, R, 8, KIND>(L, a, s);
    case 16: return launch_lines_w<F, R, 16, KIND>(L, a, s);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- batched
template <class F, typename R, int W, int KIND, int LPT>
static cudaError_t launch_batch_lines_wl(const BatchLaunch &b, cudaStream_t s) {
    using V = typename LinesPerThread<F, LPT>::M::MemV;
    const unsigned threads = kBatchLineThreads;
    const size_t smem = W > 0 ? column_ring_bytes<V>(threads) : 0;
    static bool attr = false;
    if (!attr && smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(batch_lines_kernel<F, R, W, KIND, LPT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    BatchDesc d{b.args, b.first, b.gridx, b.n};
    batch_lines_kernel<F, R, W, KIND, LPT><<<b.total_blocks, threads, smem, s>>>(d);
    return cudaGetLastError();
}

// One line per thread, adjacent line pairs (lpt 2; elements of 8 bytes or
// less, windowed forms) for instances whose lines pair up in memory, or
// groups of four (lpt 4; forms that have a four-line form).
template <class F, typename R, int W, int KIND>
static cudaError_t launch_batch_lines_w(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s) {
    if constexpr (has_quad<F>() && W > 0) {
        if (L.lpt == 4) return launch_batch_lines_wl<F, R, W, KIND, 4>(b, s);
    }
    if constexpr (sizeof(typename F::V) <= 8 && W > 0) {
        if (L.lpt == 2) return launch_batch_lines_wl<F, R, W, KIND, 2>(b, s);
    }
    return launch_batch_lines_wl<F, R, W, KIND, 1>(b, s);
}

template <class F, typename R, int W>
static cudaError_t launch_batch_contig_w(const BatchLaunch &b, cudaStream_t s) {
    using V = typename F::V;
    const size_t smem = kTileWarps * tile_warp_bytes<V, W>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(batch_contig_kernel<F, R, W>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    BatchDesc d{b.args, b.first, b.gridx, b.n};
    batch_contig_kernel<F, R, W><<<b.total_blocks, 32 * kTileWarps, smem, s>>>(d);
    return cudaGetLastError();
}

// The batched z sweep through TMA tiles: every instance of the launch fits
// the TMA form (tma_z_fits) and has its tensor maps in b.tma.
template <class F, typename R, int W>
static cudaError_t launch_batch_tma_w(const BatchLaunch &b, cudaStream_t s) {
    if constexpr (tma_supported<F, W>()) {
        if (b.n > kTmaBatch) return cudaErrorInvalidValue;
        constexpr size_t smem = tma_smem_bytes<typename F::V, W>();
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(batch_tma_kernel<F, R, W>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        BatchDesc d{b.args, b.first, b.gridx, b.n};
        batch_tma_kernel<F, R, W><<<b.total_blocks, kTmaWarps * 32, smem, s>>>(d, *b.tma);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <class F, typename R, int KIND>
static cudaError_t launch_batch_kind(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s) {
    if (KIND == K_Z && L.contiguous && b.tma) {
        switch (L.window) {
        case 4: return launch_batch_tma_w<F, R, 4>(b, s);
        case 8: return launch_batch_tma_w<F, R, 8>(b, s);
        case 16: return launch_batch_tma_w<F, R, 16>(b, s);
        default: return cudaErrorInvalidValue;
        }
    }
    if (KIND == K_Z && L.contiguous) {
        switch (L.window) {
        case 4: return launch_batch_contig_w<F, R, 4>(b, s);
        case 8: return launch_batch_contig_w<F, R, 8>(b, s);
        case 16: return launch_batch_contig_w<F, R, 16>(b, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (L.window) {
    case 0: return launch_batch_lines_w<F, R, 0, KIND>(L, b, s);
    case 4: return launch_batch_lines_w<F, R, 4, KIND>(L, b, s);
    case 8: return launch_batch_lines_w<F, R, 8, KIND>(L, b, s);
    case 16: return launch_batch_lines_w<F, R, 16, KIND>(L, b, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class F, typename R>
static cudaError_t launch_batch_form(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s) {
    if (b.total_blocks == 0) return cudaSuccess;
    switch (L.kind) {
    case K_X: return launch_batch_kind<F, R, K_X>(L, b, s);
    case K_Y: return launch_batch_kind<F, R, K_Y>(L, b, s);
    case K_Z: return launch_batch_kind<F, R, K_Z>(L, b, s);
    }
    return cudaErrorInvalidValue;
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

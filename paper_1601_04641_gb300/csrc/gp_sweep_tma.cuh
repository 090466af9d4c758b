// gp_sweep_tma.cuh -- z sweep (the stride-1 axis) through the tensor memory
// accelerator.
//
// With x slowest and z fastest, the z lines are the rows of a 2D array
// [n_lines][N].  A warp owns 64 consecutive rows and advances two of them
// per lane (rows lane and lane + 32, as one pair form), walking them in boxes of
// B nodes x 64 rows, where B nodes fill 64 bytes of a row (8 complex64 or 16
// float values).  One lane issues each box as a cp.async.bulk.tensor load
// into a ring of shared memory (one mbarrier per slot); the boxes the
// current chunk reads are resident while kTmaAhead more are in flight.
// Boxes land in the 64-byte swizzled layout (the 16-byte unit u of row r is
// stored at unit u ^ ((r / 2) mod 4)), so the 8 lanes of a quarter warp
// reading one column of their own rows hit 8 different bank groups.
//
// Each chunk of B results goes back the same way, stored by one TMA
// instruction from a swizzled tile.  A TMA row must start on a 16-byte
// boundary and the first interior node is node 1, so tile k holds nodes
// [kB, kB + B): the chunk's last result is carried in registers into slot 0
// of the next tile, and node 0 and node N-1 (the Dirichlet ends) are written
// as zeros.  Tile k covers exactly the nodes of input box k, which no read
// needs once chunk k's forward sweep is done, so the tile is written into
// box k's ring slot; the slot is refilled only after the tile store has read
// it.  Rows past the last line read zeros (TMA fill) and are clipped on
// store; so are nodes past N-1.
//
// Every wait on an mbarrier is bounded (about a second of clock cycles);
// on expiry the warp stops waiting, finishes without trusting its data and
// raises SweepArgs::status, which the host checks when it synchronises.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include <type_traits>

#include "gp_async.cuh"
#include "gp_sweep.cuh"

namespace gpcn {

// Four warps per block and three boxes in flight per warp (83 KB of shared
// memory per block for complex64, two blocks per SM) measured fastest on the
// 480x400x320 complex64 z sweep: 0.171 ms, against 0.180 ms with two warps
// and two boxes in flight.
constexpr int kTmaWarps = 4;                         // warps per block
constexpr int kTmaRows = 64;                         // lines per warp (two per lane)
constexpr int kTmaRowBytes = 64;                     // one box row = one swizzle span
constexpr int kTmaBoxBytes = kTmaRows * kTmaRowBytes;
constexpr int kTmaAhead = 3;                         // boxes in flight beyond the one needed
static_assert(kTmaWarps * kTmaRows == kTmaBlockRows, "rows per block of the TMA z sweep");

template <typename E> __host__ __device__ constexpr int tma_chunk() { return kTmaRowBytes / (int)sizeof(E); }
// Ring slots: a chunk reads up to (W + B + 1) / B boxes past its own, two more
// are in flight, and the chunk's own box holds its output tile until the
// tile store has read it.
template <typename E, int W> __host__ __device__ constexpr int tma_slots() {
    return (W + tma_chunk<E>() + 1) / tma_chunk<E>() + kTmaAhead + 1;
}
template <typename E, int W> __host__ __device__ constexpr size_t tma_smem_bytes() {
    return 1024 + (size_t)kTmaWarps * tma_slots<E, W>() * (kTmaBoxBytes + 8);
}

// Forms the TMA kernel is built for: 2-, 4- or 8-byte elements (2: FP16
// storage), and a register ring of B + W pair values within 256 bytes of
// storage per thread (beyond that the kernel spills; the per-thread copy
// form runs instead).
template <class F, int W> constexpr bool tma_supported() {
    using E = store_t<F>;
    if constexpr (sizeof(E) != 2 && sizeof(E) != 4 && sizeof(E) != 8) return false;
    else return (tma_chunk<E>() + W) * 2 * sizeof(E) <= 256;
}

// Whether a z sweep can take the TMA kernel: a supported form, whole lines
// (one segment), rows that start on 16-byte boundaries, and lines of at
// least one full chunk plus its window and two nodes.
template <class F, int W> inline bool tma_usable(const SweepArgs &a) {
    using E = store_t<F>;
    if constexpr (!tma_supported<F, W>()) {
        return false;
    } else {
        static_assert(tma_chunk<E>() == 64 / (int)sizeof(E), "tma_z_fits assumes 64-byte box rows");
        return tma_z_fits((int)sizeof(E), W, a.N, a.n_seg, a.n_lines);
    }
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, unsigned bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, unsigned src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, unsigned bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// Wait until at most `pending` of this thread's newest bulk groups still read
// shared memory (more than 3 waits for 3).
__device__ __forceinline__ void bulk_wait_read(int pending) {
    switch (pending) {
    case 0: asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.bulk.wait_group.read 2;\n" ::: "memory"); break;
    default: asm volatile("cp.async.bulk.wait_group.read 3;\n" ::: "memory"); break;
    }
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// Generic-proxy writes to shared memory become visible to later TMA reads.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

template <typename E> struct __align__(2 * sizeof(E)) E2 { E x, y; };

// One warp's 64 lines, whole lines, window W.  Returns the lane's partial
// sum of |phi|^2 over its two lines.
template <class F, typename R, int W>
__device__ __forceinline__ double tma_body(const SweepArgs &a, const CUtensorMap *tin, const CUtensorMap *tout,
                                           unsigned char *wbase, unsigned bar0, int y0) {
    using E = store_t<F>;
    using M = typename PairForm<F>::type;
    using V = typename M::V;
    using MV = typename M::MemV;
    using C = typename F::C;
    constexpr int B = tma_chunk<E>();
    constexpr int ES = sizeof(E);
    constexpr int S = tma_slots<E, W>();
    static_assert(W % 2 == 0 && B % 2 == 0, "node pairs must not straddle a 16-byte unit");
    const int lane = threadIdx.x & 31;
    const int N = a.N, n = N - 2;
    const int nbox = (N - 1) / B + 1;  // boxes covering nodes 0 .. N-1
    const C *cp = static_cast<const C *>(a.cp);
    const C *ipm1 = static_cast<const C *>(a.ip);
    const R kap = (R)a.kappa;
    const unsigned ring = smem_u32(wbase);
    const unsigned xm = ((lane >> 1) & 3) << 4;  // swizzle of rows lane and lane + 32
    const unsigned ra = lane * kTmaRowBytes, rb = (lane + 32) * kTmaRowBytes;

    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncwarp();
    int stored = 0;  // tiles stored so far (tile k is bulk group k)
    // Lane 0: load box b into its slot, after the store of the tile that
    // slot held (tile b - S) has finished reading it.
    auto issue = [&](int b) {
        const unsigned s = b % S;
        // tile b - S was stored at the end of chunk b - S; later chunks
        // have stored at most the tiles after it (S exceeds the boxes a
        // chunk reads ahead plus the boxes in flight)
        if (b >= S) bulk_wait_read(max(0, stored - 1 - (b - S)));
        mbar_arrive_expect_tx(bar0 + 8 * s, kTmaBoxBytes);
        tma_load_2d(ring + s * kTmaBoxBytes, tin, bar0 + 8 * s, b * B, y0);
    };
    int issued = min(kTmaAhead + 1, nbox), waited = 0;
    bool ok = true;
    if (lane == 0)
        for (int b = 0; b < issued; ++b) issue(b);
    // Make box k readable and keep kTmaAhead boxes beyond it in flight.
    auto need = [&](int k) {
        if (k < waited) return;
        for (; waited <= k; ++waited) ok = mbar_wait_bounded(bar0 + 8 * (waited % S), (waited / S) & 1, ok) && ok;
        __syncwarp();
        const int lim = min(k + kTmaAhead + 1, nbox);
        if (lane == 0)
            for (int b = issued; b < lim; ++b) issue(b);
        issued = max(issued, lim);
    };
    // Nodes c, c+1 (c even) of box k, for both of the lane's rows.
    auto rd2 = [&](int k, int c, V &v0, V &v1) {
        const unsigned char *slot = wbase + (k % S) * kTmaBoxBytes;
        const unsigned off = (unsigned)(c * ES) ^ xm;
        const E2<E> pa = *reinterpret_cast<const E2<E> *>(slot + ra + off);
        const E2<E> pb = *reinterpret_cast<const E2<E> *>(slot + rb + off);
        v0 = M::load(MV{pa.x, pb.x});
        v1 = M::load(MV{pa.y, pb.y});
    };
    auto wr2 = [&](int k, int s, V v0, V v1) {  // nodes s, s+1 (s even) of tile k
        unsigned char *tile = wbase + (k % S) * kTmaBoxBytes;
        const unsigned off = (unsigned)(s * ES) ^ xm;
        const MV m0 = M::store(v0), m1 = M::store(v1);
        *reinterpret_cast<E2<E> *>(tile + ra + off) = E2<E>{m0.a, m1.a};
        *reinterpret_cast<E2<E> *>(tile + rb + off) = E2<E>{m0.b, m1.b};
    };
    auto store_tile = [&](int k) {
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            tma_store_2d(tout, ring + (k % S) * kTmaBoxBytes, k * B, y0);
            bulk_commit();
        }
        ++stored;
    };

    Acc<R> acc;
    V carry = M::zero();  // slot 0 of the next tile (node 0 for the first)
    V D[B + W];
    V pm = M::zero(), p0, p1, p1n;
    V dprev = M::zero();
    // warm-up: dp[0 .. W-1]; dp[t] reads nodes t, t+1, t+2
    need(0);
    rd2(0, 0, p1n, p0);  // node 0 is the Dirichlet end: pm stays zero
#pragma unroll
    for (int t = 0; t < W; ++t) {
        if ((t & 1) == 0) {
            need((t + 2) / B);
            rd2((t + 2) / B, (t + 2) % B, p1, p1n);
        } else {
            p1 = p1n;
        }
        dprev = M::fwd(M::rhs(pm, p0, p1, kap), dprev, kap, ldc(ipm1 + t));
        D[t] = dprev;
        pm = p0;
        p0 = p1;
    }
    // One full chunk (outputs t0 .. t0+B-1).  Settled: the coefficients of
    // the chunk all equal the tables' last entries and come from registers.
    const C cps = ldc(cp + n - 1), ips = ldc(ipm1 + n - 1);
    auto chunk = [&](int t0, auto settled) {
        constexpr bool S = decltype(settled)::value;
        const int j = t0 / B;
        need(j + (W + B + 1) / B);
        const bool last_full = t0 + B + W == n;  // the chunk's last read is node N-1
#pragma unroll
        for (int q = 0; q < B; ++q) {
            if ((q & 1) == 0) {
                rd2(j + (W + 2 + q) / B, (W + 2 + q) % B, p1, p1n);
                if (q == B - 2 && last_full) p1n = M::zero();
            } else {
                p1 = p1n;
            }
            dprev = M::fwd(M::rhs(pm, p0, p1, kap), dprev, kap, S ? ips : ldc(ipm1 + t0 + W + q));
            D[W + q] = dprev;
            pm = p0;
            p0 = p1;
        }
        V phi = D[B + W - 1];
#pragma unroll
        for (int q = B + W - 2; q >= B; --q) phi = M::back(D[q], S ? cps : ldc(cp + t0 + q), phi);
        R csum = R(0);
        V next = M::zero(), hi = M::zero();
#pragma unroll
        for (int q = B - 1; q >= 0; --q) {  // result q goes to tile slot q + 1
            phi = M::back(D[q], S ? cps : ldc(cp + t0 + q), phi);
            csum += M::abs2(phi);
            if (q == B - 1) next = phi;
            else if ((q & 1) == 0) hi = phi;
            else wr2(j, q + 1, phi, hi);
        }
        wr2(j, 0, carry, hi);
        carry = next;
        acc.add(csum);
        store_tile(j);
#pragma unroll
        for (int q = 0; q < W; ++q) D[q] = D[B + q];
    };
    int t0 = 0;
    for (; t0 + B + W <= n && t0 < a.t_const; t0 += B) chunk(t0, std::false_type{});
    for (; t0 + B + W <= n; t0 += B) chunk(t0, std::true_type{});
    // last chunk: W <= rem < B + W positions left; exact from phi[n-1] = dp[n-1]
    {
        const int j = t0 / B;
        const int rem = n - t0;
        need(nbox - 1);
#pragma unroll
        for (int q = 0; q < B; ++q) {
            if (q < rem - W) {
                if ((q & 1) == 0) {
                    // nodes t0+W+2+q (even, at most N-2) and t0+W+3+q (at most N-1)
                    rd2(j + (W + 2 + q) / B, (W + 2 + q) % B, p1, p1n);
                    if (q == rem - W - 2) p1n = M::zero();
                } else {
                    p1 = p1n;
                }
                if (q == rem - W - 1 && (q & 1) == 0) p1 = M::zero();
                dprev = M::fwd(M::rhs(pm, p0, p1, kap), dprev, kap, ldc(ipm1 + t0 + W + q));
                D[W + q] = dprev;
                pm = p0;
                p0 = p1;
            }
        }
        V phi = M::zero();
        R csum = R(0);
#pragma unroll
        for (int q = B + W - 1; q >= 0; --q) {
            if (q < rem) {
                phi = M::back(D[q], ldc(cp + t0 + q), (q == rem - 1) ? M::zero() : phi);
                D[q] = phi;
                csum += M::abs2(phi);
            }
        }
        acc.add(csum);
        // tiles j, j+1, ... up to the one holding node N-1 = t0 + rem + 1
        constexpr int NT = (B + W) / B + 1;
#pragma unroll
        for (int kt = 0; kt < NT; ++kt) {
            if ((j + kt) * B <= N - 1) {
                auto slot = [&](int s) {  // tile slot s holds node t0 + 1 + q
                    const int q = kt * B + s - 1;
                    V v = M::zero();
                    if (q < 0) v = carry;
                    else if (q < B + W && q < rem) v = D[q < B + W ? q : 0];
                    return v;
                };
#pragma unroll
                for (int s = 0; s < B; s += 2) wr2(j + kt, s, slot(s), slot(s + 1));
                store_tile(j + kt);
            }
        }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
    if (!ok) {
        // give copies that may still be landing a fresh bound before the
        // block's shared memory is released
        for (int b = max(0, issued - S); b < issued; ++b) mbar_wait_bounded(bar0 + 8 * (b % S), (b / S) & 1, true);
        if (lane == 0 && a.status) atomicOr(a.status, 1u);
    }
    return acc.value();
}

// Many condensates in one launch: instance q owns blocks [first[q], first[q+1])
// (one block per 256 rows of its own grid) and its tensor maps maps.in[q],
// maps.out[q]; each instance's norm is reduced over its own blocks, in the
// same order as a single-condensate launch.
template <class F, typename R, int W>
__global__ void __launch_bounds__(kTmaWarps * 32, 1) batch_tma_kernel(BatchDesc d,
                                                                     const __grid_constant__ BatchTmaMaps maps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                            ~static_cast<uintptr_t>(1023));
    constexpr int S = tma_slots<store_t<F>, W>();
    const int q = find_instance(d, blockIdx.x);
    const SweepArgs a = d.args[q];
    const unsigned local = blockIdx.x - __ldg(d.first + q);
    const unsigned nblocks = __ldg(d.first + q + 1) - __ldg(d.first + q);
    const int warp = threadIdx.x >> 5;
    const long long L0 = ((long long)local * kTmaWarps + warp) * kTmaRows;
    double v = 0.0;
    if (L0 < a.n_lines)
        v = tma_body<F, R, W>(a, &maps.in[q], &maps.out[q], base + warp * S * kTmaBoxBytes,
                              smem_u32(base + kTmaWarps * S * kTmaBoxBytes) + 8 * S * warp, (int)L0);
    norm_finalize(v, a, local, nblocks);
}

template <class F, typename R, int W>
__global__ void __launch_bounds__(kTmaWarps * 32, 1) sweep_tma_kernel(SweepArgs a, const __grid_constant__ TmaMaps maps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                            ~static_cast<uintptr_t>(1023));
    constexpr int S = tma_slots<store_t<F>, W>();
    const int warp = threadIdx.x >> 5;
    const long long L0 = ((long long)blockIdx.x * kTmaWarps + warp) * kTmaRows;
    double v = 0.0;
    if (L0 < a.n_lines)
        v = tma_body<F, R, W>(a, &maps.in, &maps.out, base + warp * S * kTmaBoxBytes,
                              smem_u32(base + kTmaWarps * S * kTmaBoxBytes) + 8 * S * warp, (int)L0);
    norm_finalize(v, a, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ strided axes through TMA
// The x and y lines as a 3D array of 4-byte words [outer][node][word]: for
// the x sweep one outer group (the y-z plane, ny*nz elements per node); for
// the y sweep nx groups (planes) of nz elements per node.  The tensor map's
// origin is node 1 of the line and its node extent the n = N - 2 interior
// nodes, so every position outside [0, n) reads zeros (TMA fill).  A warp owns 32 consecutive line groups (LPT
// adjacent lines each, one MemV per node) of one outer group and streams
// them in boxes of B nodes x 32 MemV: one lane issues box b (positions
// s0 + bB ...) into the warp's ring of kRingChunks slots, one mbarrier each,
// and lane l reads column l of a box row -- one conflict-free shared-memory
// row per node, no per-element copy or address arithmetic.  Results are
// stored lane by lane (each warp store instruction writes one contiguous
// row of 32 MemV).
// Every wait is bounded; on expiry the warp stops waiting, finishes
// without trusting its data and raises SweepArgs::status.
constexpr int kLineTmaWarps = 4;  // warps per block

template <typename MV, int B> __host__ __device__ constexpr int line_box_bytes() {
    return B * 32 * (int)sizeof(MV);
}
template <typename MV> __host__ __device__ constexpr size_t line_tma_smem() {
    return 128 + (size_t)kLineTmaWarps * (kRingChunks * line_box_bytes<MV, chunk_len<MV>()>() + 8 * kRingChunks);
}

template <class F, class M, typename R, int B, int KIND> struct TmaColumnIO {
    using V = typename M::V;
    using MV = typename M::MemV;
    static constexpr int RC = kRingChunks, RL = RC * B;
    static constexpr int BOXB = line_box_bytes<MV, B>();
    const CUtensorMap *tin;
    const MV *rp;     // this warp's ring: position p at rp[((p - s0) % RL) * 32 + lane]
    unsigned ring_s, bar0;
    int cx, cz, lane;
    int s0, limit, issued, ready;
    bool ok;
    bool valid;       // the lane owns a line group (else it solves zeros and stores nothing)
    MV *out;          // the line group's node 0 in the output
    long long st;
    Hooks<F, M, R, KIND> hk;
    __device__ __forceinline__ void issue() {
        if (lane == 0) {
            const unsigned slot = (unsigned)(issued % RC);
            mbar_arrive_expect_tx(bar0 + 8 * slot, BOXB);
            tma_load_3d(ring_s + slot * BOXB, tin, bar0 + 8 * slot, cx, s0 + issued * B, cz);
        }
        ++issued;
    }
    __device__ __forceinline__ void start(int first, int lim) {
        s0 = first;
        limit = lim;
        issued = ready = 0;
        ok = true;
        while (issued < RC - 1 && s0 + issued * B < limit) issue();
    }
    // Make positions < p_end readable; keep up to two more boxes in flight.
    // The box refilled into a slot is the one two boxes behind the newest
    // readable one, which no later read needs, and the __syncwarp makes the
    // whole warp done with it first.
    __device__ __forceinline__ void need(int p_end) {
        const int c = (p_end - 1 - s0) / B;
        if (c < ready) return;
        while (issued <= c) issue();  // not reached by the solve's access pattern; a guard
        for (; ready <= c; ++ready) ok = mbar_wait_bounded(bar0 + 8 * (ready % RC), (ready / RC) & 1, ok) && ok;
        __syncwarp();
        while (issued <= c + RC - 2 && s0 + issued * B < limit) issue();
    }
    __device__ __forceinline__ V val(int p) const {
        return hk.on_load(p, M::load(rp[((p - s0) & (RL - 1)) * 32 + lane]));
    }
    template <int NB> __device__ __forceinline__ void vals(int p, V (&v)[NB]) const {
#pragma unroll
        for (int q = 0; q < NB; ++q) v[q] = M::load(rp[((p + q - s0) & (RL - 1)) * 32 + lane]);
        hk.on_load_chunk(p, v);
    }
    __device__ __forceinline__ void put(int t0, int q, V v) const {
        if (valid) out[(long long)(t0 + q + 1) * st] = M::store(v);
        hk.on_store(v);
    }
    __device__ __forceinline__ void flush(int, int) const {}
    // After an expired wait, a fresh bound for the loads that may still be
    // landing before the shared memory is released.
    __device__ __forceinline__ void finish(unsigned int *status) {
        if (!ok) {
            for (int b = max(0, issued - RC); b < issued; ++b) mbar_wait_bounded(bar0 + 8 * (b % RC), (b / RC) & 1, true);
            if (lane == 0 && status) atomicOr(status, 1u);
        }
    }
};

// One warp per 32 line groups of one outer group; the last warp of an outer
// group may be partial: its box columns past the group read the zero fill,
// and its lanes past the group solve those zeros and store nothing.
// blockIdx.y is the segment.  Windowed solves only.
template <class F, typename R, int W, int KIND, int LPT>
__global__ void __launch_bounds__(kLineTmaWarps * 32) sweep_lines_tma_kernel(SweepArgs a,
                                                                             const __grid_constant__ TmaMaps maps) {
    static_assert(W > 0 && KIND != K_Z, "strided windowed sweeps only");
    using M = typename LinesPerThread<F, LPT>::M;
    using MV = typename M::MemV;
    using C = typename F::C;
    constexpr int B = chunk_len<MV>();
    constexpr int BOXB = line_box_bytes<MV, B>();
    constexpr int RC = kRingChunks;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                            ~static_cast<uintptr_t>(127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long U = a.inner / LPT;        // line groups per outer group
    const long long wpr = (U + 31) / 32;      // warps per outer group
    const long long gw = (long long)blockIdx.x * kLineTmaWarps + warp;
    if (gw >= (a.n_lines / a.inner) * wpr) return;  // warps are independent: no block-wide barrier below
    const long long o = gw / wpr, u0 = (gw % wpr) * 32;
    const bool valid = u0 + lane < U;
    const long long L0 = o * a.inner + u0 * LPT;                   // the warp's first line
    const long long L = valid ? L0 + (long long)lane * LPT : L0;  // lanes past the group: the first line's state
    unsigned char *wb = base + warp * RC * BOXB;
    const unsigned bar0 = smem_u32(base + kLineTmaWarps * RC * BOXB) + 8 * RC * warp;
    if (lane == 0) {
        for (int q = 0; q < RC; ++q) mbar_init(bar0 + 8 * q, 1);
        mbar_init_fence();
    }
    __syncwarp();
    const long long off = (L / a.inner) * a.outer_stride + (L % a.inner);
    MV *out = reinterpret_cast<MV *>(static_cast<store_t<F> *>(a.psi_out) + off);
    const long long st = a.stride / LPT;
    const int n = a.N - 2;
    const unsigned seg = blockIdx.y;
    if (valid && seg == 0) out[0] = M::store(M::zero());
    if (valid && (int)seg == a.n_seg - 1) out[(long long)(a.N - 1) * st] = M::store(M::zero());
    Acc<R> acc;
    TmaColumnIO<F, M, R, B, KIND> io;
    io.valid = valid;
    io.tin = &maps.in;
    io.rp = reinterpret_cast<const MV *>(wb);
    io.ring_s = smem_u32(wb);
    io.bar0 = bar0;
    io.cx = (int)(u0 * LPT * (long long)sizeof(store_t<F>) / 4);
    io.cz = (int)o;
    io.lane = lane;
    io.out = out;
    io.st = st;
    io.hk.acc = &acc;
    io.hk.init(a, L);
    const int tb = seg * a.seg_len;
    const int te = (int)seg == a.n_seg - 1 ? n : tb + a.seg_len;
    solve_segment<M, R, B, W>(n, tb, te, a.t_const, (R)a.kappa, static_cast<const C *>(a.cp),
                              static_cast<const C *>(a.ip), io);
    io.finish(a.status);
}

}  // namespace gpcn

// k_field.cu -- whole-field kernels: Gaussian initial state, norm, the
// observables reduction (calcrms, calcmuen) and applying a pending scale.
#include "gp_async.cuh"
#include "gp_sweep.cuh"

#include <algorithm>
#include <atomic>
#include <type_traits>

namespace gpcn {

namespace {

template <typename R, bool CPLX> struct Elem;
template <typename R> struct Elem<R, false> {
    using V = R;
    using T = R;  // arithmetic type
    __device__ __forceinline__ static double abs2(V v) { return (double)v * (double)v; }
    __device__ __forceinline__ static R abs2r(V v) { return v * v; }
    __device__ __forceinline__ static V from_real(double x) { return (R)x; }
    __device__ __forceinline__ static V scaled(V v, R s) { return v * s; }
    __device__ __forceinline__ static R diff2(V a, V b) {
        const R d = a - b;
        return d * d;
    }
};
template <typename R> struct Elem<R, true> {
    using V = cx<R>;
    using T = R;
    __device__ __forceinline__ static double abs2(V v) {
        return (double)v.re * (double)v.re + (double)v.im * (double)v.im;
    }
    __device__ __forceinline__ static R abs2r(V v) { return fma(v.re, v.re, v.im * v.im); }
    __device__ __forceinline__ static V from_real(double x) { return V{(R)x, R(0)}; }
    __device__ __forceinline__ static V scaled(V v, R s) { return V{v.re * s, v.im * s}; }
    __device__ __forceinline__ static R diff2(V a, V b) {
        const R dre = a.re - b.re, dim = a.im - b.im;
        return dre * dre + dim * dim;
    }
};
// FP16 storage of a real field: values widened to FP32 for all arithmetic.
template <> struct Elem<__half, false> {
    using V = __half;
    using T = float;
    __device__ __forceinline__ static double abs2(V v) {
        const double x = (double)__half2float(v);
        return x * x;
    }
    __device__ __forceinline__ static float abs2r(V v) {
        const float x = __half2float(v);
        return x * x;
    }
    __device__ __forceinline__ static V from_real(double x) { return __double2half(x); }
    __device__ __forceinline__ static V scaled(V v, float s) { return __float2half_rn(__half2float(v) * s); }
    __device__ __forceinline__ static float diff2(V a, V b) {
        const float d = __half2float(a) - __half2float(b);
        return d * d;
    }
};

__device__ __forceinline__ long long grid_stride() { return (long long)gridDim.x * blockDim.x; }

// Unnormalised product Gaussian prod_a (w_a/pi)^(1/4) exp(-w_a a^2/2), zero on
// the boundary nodes.  FP64 arithmetic, stored in the field's precision.
template <typename R, bool CPLX>
__global__ void gaussian_kernel(FieldArgs a) {
    using E = Elem<R, CPLX>;
    typename E::V *psi = static_cast<typename E::V *>(a.psi);
    const double pi = 3.14159265358979323846;
    // an absent axis (one node: 1D and 2D condensates) contributes no factor
    // and has no boundary nodes
    double c0 = 1.0;
    for (int q = 0; q < 3; ++q)
        if (a.n[q] > 1) c0 *= pow(a.w[q] / pi, 0.25);
    auto inside = [](int idx, int n) { return n == 1 || (idx > 0 && idx < n - 1); };
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < a.sites; s += grid_stride()) {
        const int k = (int)(s % a.n[2]);
        const int j = (int)((s / a.n[2]) % a.n[1]);
        const int i = (int)(s / ((long long)a.n[2] * a.n[1]));
        double v = 0.0;
        if (inside(i, a.n[0]) && inside(j, a.n[1]) && inside(k, a.n[2])) {
            const double x = a.origin[0] + i * a.d[0];
            const double y = a.origin[1] + j * a.d[1];
            const double z = a.origin[2] + k * a.d[2];
            v = c0 * exp(-0.5 * (a.w[0] * x * x + a.w[1] * y * y + a.w[2] * z * z));
        }
        psi[s] = E::from_real(v);
    }
}

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Block sums of NV compensated FP32 pairs (s, c), combined by TwoSum at every
// level of a fixed tree (warp butterfly, then the warps in order), converted
// to FP64 once; valid in thread 0.  FP64 arithmetic is a small fraction of
// the FP32 rate on this part, so the per-block reduction stays in FP32.
template <int NV>
__device__ __forceinline__ void block_sum_pairs(float (&s)[NV], float (&c)[NV], double (&out)[NV]) {
    __shared__ float red_s[NV][32], red_c[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (int)((blockDim.x + 31) >> 5);
    auto warp_pairs = [&]() {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const float s2 = __shfl_xor_sync(0xffffffffu, s[q], o);
                const float c2 = __shfl_xor_sync(0xffffffffu, c[q], o);
                float t, e;
                two_sum(s[q], s2, t, e);
                s[q] = t;
                c[q] = (c[q] + c2) + e;
            }
        }
    };
    warp_pairs();
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            red_s[q][wid] = s[q];
            red_c[q][wid] = c[q];
        }
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            s[q] = lane < nw ? red_s[q][lane] : 0.f;
            c[q] = lane < nw ? red_c[q][lane] : 0.f;
        }
        warp_pairs();
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) out[q] = (double)s[q] + (double)c[q];
}

// Block sums bs (valid in thread 0) -> partials; the last block to finish
// sums the partials in block order (deterministic) and calls `fin`.
template <int NV, class Fin>
__device__ __forceinline__ void finalize_partials(const double (&bs)[NV], const FieldArgs &a, Fin fin,
                                                  unsigned block, unsigned nblocks) {
    __shared__ double red[32];
    __shared__ int is_last;
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
    double tot[NV], sum[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) sum[q] = 0.0;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < NV; ++q) sum[q] += __ldcg(a.partials + (long long)b * NV + q);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = block_sum(sum[q], red);
    if (threadIdx.x == 0) {
        fin(tot);
        *a.counter = 0u;
    }
}

// Reduce NV FP64 values over the grid: block partials, then the last block
// sums them in block order (deterministic) and calls `fin`.
template <int NV, class Fin>
__device__ __forceinline__ void reduce_finalize(double (&v)[NV], const FieldArgs &a, Fin fin,
                                                unsigned block, unsigned nblocks) {
    __shared__ double red[32];
    double bs[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) bs[q] = block_sum(v[q], red);
    finalize_partials<NV>(bs, a, fin, block, nblocks);
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

// Observables: one thread per (j, k) and segment of i (kObsSeg nodes) walks
// along i.  The 9 sums (|psi|^2, V|psi|^2, |psi|^4, x^2|psi|^2, y^2|psi|^2,
// z^2|psi|^2 and the squared forward differences to the +x, +y and +z
// neighbours; links that leave the grid do not exist, and the +x link of
// site i is counted at i + 1) come from 6 per-thread sums of the unscaled
// field: y and z are fixed along a thread's walk, so its y^2 and z^2 sums
// are y^2 and z^2 times its |psi|^2 sum, and V = gamma^2 x^2/2 +
// (nu^2 y^2 + lambda^2 z^2)/2 splits the same way; the pending scale s
// multiplies the quadratic sums by s^2 and |psi|^4 by s^4.  Sums run in the
// field's precision over chunks of 8 sites and are added to a compensated
// per-thread total (FP32) or a plain one (FP64).
constexpr int kObsSeg = 128;

template <typename R> __device__ __forceinline__ Acc<R> acc_scaled(const Acc<R> &a, R f) {
    Acc<R> r;
    if constexpr (sizeof(R) == 4) {
        r.s = a.s * f;
        r.c = a.c * f;
    } else {
        r.s = a.s * f;
    }
    return r;
}
template <typename R> __device__ __forceinline__ Acc<R> acc_sum(const Acc<R> &a, const Acc<R> &b) {
    Acc<R> r = a;
    r.add(b.s);
    if constexpr (sizeof(R) == 4) r.c += b.c;
    return r;
}

// The observables from the 9 grid sums t (ObsSlot order) into a.out:
// norm = dV sum|psi|^2, kinetic = dV/2 sum_a (link sum_a)/d_a^2, potential
// dV sum V|psi|^2, interaction dV sum|psi|^4; mu = (K + P + g I)/norm,
// E = (K + P + g I/2)/norm, rms_a = sqrt(dV sum a^2|psi|^2 / norm).
__device__ __forceinline__ void obs_finish(const FieldArgs &a, const double *t) {
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
}

template <typename R, bool CPLX>
__device__ __forceinline__ void observables_body(const FieldArgs &a, unsigned block, unsigned nblocks) {
    using E = Elem<R, CPLX>;
    using V = typename E::V;
    using T = typename E::T;  // arithmetic
    const V *psi = static_cast<const V *>(a.psi);
    const long long plane = (long long)a.n[1] * a.n[2];
    const unsigned pblocks = (unsigned)((plane + kReduceThreads - 1) / kReduceThreads);
    const long long L = (long long)(block % pblocks) * blockDim.x + threadIdx.x;
    const int i0 = (int)(block / pblocks) * kObsSeg;
    const int i1 = min(i0 + kObsSeg, a.n[0]);
    enum { S_RHO, S_X2, S_RHO2, S_LX, S_LY, S_LZ, S_N };
    Acc<T> sum[S_N];
    Acc<T> acc[9];
    if (L < plane && i0 < i1) {
        const int j = (int)(L / a.n[2]), k = (int)(L % a.n[2]);
        const T x0 = (T)a.origin[0], dx = (T)a.d[0];
        const bool has_y = j + 1 < a.n[1], has_z = k + 1 < a.n[2];
        V prev = i0 > 0 ? psi[(i0 - 1) * plane + L] : E::from_real(0.0);
        // chunks of 8 sites: all of a chunk's loads are issued before its sums
        for (int c0 = i0; c0 < i1; c0 += 8) {
            V p[8], qy[8], qz[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                p[u] = qy[u] = qz[u] = E::from_real(0.0);
                if (c0 + u < i1) {
                    const long long off = (c0 + u) * plane + L;
                    p[u] = psi[off];
                    if (has_y) qy[u] = psi[off + a.n[2]];
                    if (has_z) qz[u] = psi[off + 1];
                }
            }
            T part[S_N];
#pragma unroll
            for (int q = 0; q < S_N; ++q) part[q] = T(0);
            const T fc0 = (T)c0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = c0 + u;
                if (i < i1) {
                    const T rho = E::abs2r(p[u]);
                    const T x = fma(fc0 + (T)u, dx, x0);
                    part[S_RHO] += rho;
                    part[S_X2] = fma(x * x, rho, part[S_X2]);
                    part[S_RHO2] = fma(rho, rho, part[S_RHO2]);
                    if (i > 0) part[S_LX] += E::diff2(p[u], prev);
                    if (has_y) part[S_LY] += E::diff2(qy[u], p[u]);
                    if (has_z) part[S_LZ] += E::diff2(qz[u], p[u]);
                    prev = p[u];
                }
            }
#pragma unroll
            for (int q = 0; q < S_N; ++q) sum[q].add(part[q]);
        }
        const T sc = (T)__ldg(a.scale);
        const T s2 = sc * sc;
        const T y = (T)(a.origin[1] + j * a.d[1]);
        const T z = (T)(a.origin[2] + k * a.d[2]);
        acc[O_RHO] = acc_scaled(sum[S_RHO], s2);
        acc[O_X2] = acc_scaled(sum[S_X2], s2);
        acc[O_RHO2] = acc_scaled(sum[S_RHO2], s2 * s2);
        acc[O_LX] = acc_scaled(sum[S_LX], s2);
        acc[O_LY] = acc_scaled(sum[S_LY], s2);
        acc[O_LZ] = acc_scaled(sum[S_LZ], s2);
        acc[O_Y2] = acc_scaled(acc[O_RHO], y * y);
        acc[O_Z2] = acc_scaled(acc[O_RHO], z * z);
        const T vyz = (T)a.half_w2[1] * y * y + (T)a.half_w2[2] * z * z;
        acc[O_V] = acc_sum(acc_scaled(acc[O_X2], (T)a.half_w2[0]), acc_scaled(acc[O_RHO], vyz));
    }
    double bs[9];
    if constexpr (sizeof(T) == 4) {
        float ps[9], pc[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            ps[q] = acc[q].s;
            pc[q] = acc[q].c;
        }
        block_sum_pairs<9>(ps, pc, bs);
    } else {
        __shared__ double red[32];
#pragma unroll
        for (int q = 0; q < 9; ++q) bs[q] = block_sum(acc[q].value(), red);
    }
    finalize_partials<9>(bs, a, [&](const double *t) { obs_finish(a, t); }, block, nblocks);
}

template <typename R, bool CPLX>
__global__ void __launch_bounds__(kReduceThreads) observables_kernel(FieldArgs a) {
    observables_body<R, CPLX>(a, blockIdx.x, gridDim.x);
}

// The complex64 field's observables with at most 80 registers: three
// 256-thread blocks per SM (unbounded it took 98 and two blocks, and ncu
// showed it issue- and occupancy-bound).
__global__ void __launch_bounds__(kReduceThreads, 3) observables_c64_kernel(FieldArgs a) {
    observables_body<float, true>(a, blockIdx.x, gridDim.x);
}

// Observables of a complex64 field with nz even.  One thread per (j, pair
// of z nodes k, k+1) walks along i: each pair is one 16-byte load, read
// once from DRAM (the +y neighbours come back through L2, the +z neighbour
// k+2 through L1), and the pair's arithmetic is packed FP32x2, one node per
// component.  The sums are observables_body's: |psi|^2 per node of the pair
// (the y^2, z^2 and potential sums follow per work item), x^2 |psi|^2,
// |psi|^4 and the three link sums; FP32 over kObsFold planes, then added to
// compensated per-thread totals.  Work items (kObsZSeg planes x 256 pairs of
// a plane) go to the blocks in a fixed grid-stride order over one resident
// wave, so the summation order is fixed for a given grid.
constexpr int kObsZSeg = 32;    // planes per work item
constexpr int kObsPlanes = 4;   // planes whose loads are issued together
constexpr int kObsFold = 8;     // planes summed in FP32 before a compensated fold
static_assert(kObsZSeg % kObsFold == 0 && kObsFold % kObsPlanes == 0, "work item shape");

__host__ __device__ inline long long obs_c64z_items(const int n[3]) {
    const long long units = (long long)n[1] * n[2] / 2;
    return (units + kReduceThreads - 1) / kReduceThreads * ((n[0] + kObsZSeg - 1) / kObsZSeg);
}

__global__ void __launch_bounds__(kReduceThreads, 2) observables_c64z_kernel(FieldArgs a) {
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const long long units = (long long)ny * nz / 2;          // z pairs per plane
    const long long pst = units;                             // plane stride in float4
    const unsigned pblocks = (unsigned)((units + kReduceThreads - 1) / kReduceThreads);
    const unsigned items = (unsigned)obs_c64z_items(a.n);
    const float4 *psi4 = static_cast<const float4 *>(a.psi);
    const float x0 = (float)a.origin[0], dx = (float)a.d[0];
    Acc<float> rho, y2, z2, x2, rho2, lx, ly, lz;
    for (unsigned w = blockIdx.x; w < items; w += gridDim.x) {
        const unsigned pb = w % pblocks, sg = w / pblocks;
        const long long u = (long long)pb * kReduceThreads + threadIdx.x;
        if (u >= units) continue;
        const int j = (int)(2 * u / nz), k = (int)(2 * u % nz);
        const bool has_y = j + 1 < ny, has_z = k + 2 < nz;
        const int i0 = (int)sg * kObsZSeg, i1 = min(i0 + kObsZSeg, nx);
        const float4 *row = psi4 + u;
        float2 pre, pim;  // the previous plane's pair (the +x link into plane i0 is counted here)
        {
            const float4 v = __ldg(row + (long long)(i0 > 0 ? i0 - 1 : i0) * pst);
            pre = make_float2(v.x, v.z);
            pim = make_float2(v.y, v.w);
        }
        Acc<float> rk, rk1;  // this item's |psi|^2 per node of the pair
        for (int c0 = i0; c0 < i1; c0 += kObsFold) {
            float2 sr = dup2(0.f), sx2 = dup2(0.f), sr2 = dup2(0.f), slx = dup2(0.f), sly = dup2(0.f),
                   slz = dup2(0.f);
#pragma unroll
            for (int h = 0; h < kObsFold; h += kObsPlanes) {
                float4 P[kObsPlanes], QY[kObsPlanes];
                float2 QZ[kObsPlanes];
#pragma unroll
                for (int t = 0; t < kObsPlanes; ++t) {
                    const int i = min(c0 + h + t, i1 - 1);  // planes past i1 repeat the last, not summed
                    const float4 *r = row + (long long)i * pst;
                    P[t] = __ldg(r);
                    QY[t] = has_y ? __ldg(r + nz / 2) : P[t];
                    QZ[t] = has_z ? __ldg(reinterpret_cast<const float2 *>(r) + 2) : make_float2(P[t].z, P[t].w);
                }
#pragma unroll
                for (int t = 0; t < kObsPlanes; ++t) {
                    const int i = c0 + h + t;
                    if (i < i1) {
                        const float2 re = make_float2(P[t].x, P[t].z), im = make_float2(P[t].y, P[t].w);
                        const float2 r2 = fma2(re, re, mul2(im, im));
                        const float x = fmaf((float)i, dx, x0);
                        sr = add2(sr, r2);
                        sx2 = fma2(dup2(x * x), r2, sx2);
                        sr2 = fma2(r2, r2, sr2);
                        float2 dre = sub2(re, pre), dim = sub2(im, pim);
                        slx = fma2(dre, dre, fma2(dim, dim, slx));
                        dre = sub2(make_float2(QY[t].x, QY[t].z), re);
                        dim = sub2(make_float2(QY[t].y, QY[t].w), im);
                        sly = fma2(dre, dre, fma2(dim, dim, sly));
                        dre = sub2(make_float2(re.y, QZ[t].x), re);   // links k -> k+1 and k+1 -> k+2
                        dim = sub2(make_float2(im.y, QZ[t].y), im);
                        slz = fma2(dre, dre, fma2(dim, dim, slz));
                        pre = re;
                        pim = im;
                    }
                }
            }
            rk.add(sr.x);
            rk1.add(sr.y);
            x2.add(sx2.x + sx2.y);
            rho2.add(sr2.x + sr2.y);
            lx.add(slx.x + slx.y);
            ly.add(sly.x + sly.y);
            lz.add(slz.x + slz.y);
        }
        const float y = (float)(a.origin[1] + j * a.d[1]);
        const float zk = (float)(a.origin[2] + k * a.d[2]), zk1 = (float)(a.origin[2] + (k + 1) * a.d[2]);
        const Acc<float> r = acc_sum(rk, rk1);
        rho = acc_sum(rho, r);
        y2 = acc_sum(y2, acc_scaled(r, y * y));
        z2 = acc_sum(z2, acc_sum(acc_scaled(rk, zk * zk), acc_scaled(rk1, zk1 * zk1)));
    }
    const float sc = (float)__ldg(a.scale);
    const float s2 = sc * sc;
    Acc<float> acc[9];
    acc[O_RHO] = acc_scaled(rho, s2);
    acc[O_X2] = acc_scaled(x2, s2);
    acc[O_Y2] = acc_scaled(y2, s2);
    acc[O_Z2] = acc_scaled(z2, s2);
    acc[O_RHO2] = acc_scaled(rho2, s2 * s2);
    acc[O_LX] = acc_scaled(lx, s2);
    acc[O_LY] = acc_scaled(ly, s2);
    acc[O_LZ] = acc_scaled(lz, s2);
    acc[O_V] = acc_sum(acc_sum(acc_scaled(acc[O_X2], (float)a.half_w2[0]), acc_scaled(acc[O_Y2], (float)a.half_w2[1])),
                       acc_scaled(acc[O_Z2], (float)a.half_w2[2]));
    float ps[9], pc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        ps[q] = acc[q].s;
        pc[q] = acc[q].c;
    }
    double bs[9];
    block_sum_pairs<9>(ps, pc, bs);
    finalize_partials<9>(bs, a, [&](const double *t) { obs_finish(a, t); }, blockIdx.x, gridDim.x);
}

// Resident blocks of observables_c64z_kernel on each device (SMs x blocks
// per SM), looked up once per device by prepare_field_launches (outside any
// stream capture: the occupancy query may load the kernel's module).
constexpr int kMaxDevices = 64;
std::atomic<int> g_c64z_resident[kMaxDevices];

int c64z_resident(int dev) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, observables_c64z_kernel, kReduceThreads, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return std::max(1, sms) * std::max(1, per_sm);
}

// Blocks of observables_c64z_kernel: at most one resident wave, at most one
// per work item; 0 where the resident wave has not been looked up on the
// current device, and then the per-(j, k) kernel runs instead.
unsigned obs_c64z_grid(const FieldArgs &a) {
    int dev = 0;
    cudaGetDevice(&dev);
    const long long g = dev >= 0 && dev < kMaxDevices ? g_c64z_resident[dev].load() : 0;
    if (g <= 0) return 0;
    return (unsigned)std::max(1LL, std::min(g, obs_c64z_items(a.n)));
}

// ------------------------------------------------------------------ bulk-copy observables
// Observables of an FP32 real field with its loads staged by the tensor
// memory accelerator.  The y-z plane (ny*nz sites, contiguous) is cut into
// tiles of 1024 consecutive sites; a block walks a tile's column along x,
// plane by plane.  A producer warp (one lane) copies each plane's tile and
// the nz + 1 sites after it (the +y and +z neighbours) with one
// cp.async.bulk into a ring of kObsStages shared-memory stages: the copy
// completes on the stage's "full" mbarrier, and the stage is refilled once
// all 8 consumer warps have arrived on its "empty" mbarrier.  The consumer
// warps sum the stages in order (thread t: sites t, t + 256, t + 512,
// t + 768 of the tile), each warp at its own pace, with every neighbour read
// from shared memory and no per-thread copy or global load.  The tile-major
// sequence of (tile, plane) pairs is cut into one contiguous run per block
// (balanced to one plane); a run that starts inside a column also copies
// the plane before its first one, for the +x link.  The sums are
// observables_body's: |psi|^2 per site column (weighted by y^2 and z^2 at
// the end of the run), x^2 |psi|^2, |psi|^4 and the three link sums, FP32
// over kObsFold planes and then compensated.  (For complex64 fields the same
// scheme measured no faster than observables_c64z_kernel, 89 against 88 us
// on the 480x400x160 grid, and is not built.)
constexpr int kObsStages = 8;
constexpr int kObsStageBytes = 12288;  // the largest stage: tile, nz + 1 more sites, rounded to 16 bytes
constexpr int kObsSpt = 4;             // sites per consumer thread and plane
constexpr int kObsTile = kObsSpt * kReduceThreads;
constexpr int kObsConsumers = kReduceThreads / 32;
constexpr int kObsThreads = kReduceThreads + 32;  // consumer warps and the producer warp

// Sites of one stage: the tile and the nz + 1 after it, rounded up to 16 bytes.
__host__ __device__ inline long long obs_bulk_span(int nz) { return ((long long)kObsTile + nz + 1 + 3) / 4 * 4; }
__host__ __device__ inline size_t obs_bulk_smem(int nz) {
    return (size_t)kObsStages * obs_bulk_span(nz) * sizeof(float) + 16 * kObsStages;
}

// One block's runs: (tile, first plane i0, end plane i1) over [lo, hi) of
// the tile-major (tile, plane) sequence.
struct ObsRun {
    long long r, hi;
    int nx;
    __device__ __forceinline__ bool next(long long &tile, int &i0, int &i1) {
        if (r >= hi) return false;
        tile = r / nx;
        i0 = (int)(r % nx);
        i1 = (int)min((long long)nx, i0 + (hi - r));
        r += i1 - i0;
        return true;
    }
};

__global__ void __launch_bounds__(kObsThreads, 2) observables_bulk_kernel(FieldArgs a) {
    using V = float;
    constexpr int SPT = kObsSpt, TILE = kObsTile, S = kObsStages;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const long long plane = (long long)ny * nz;
    const long long tiles = (plane + TILE - 1) / TILE;
    const int span = (int)obs_bulk_span(nz);
    const long long pbytes = plane * (long long)sizeof(V);
    const V *stage0 = reinterpret_cast<const V *>(smem_raw);
    const unsigned ring = smem_u32(smem_raw);
    const unsigned full0 = ring + (unsigned)(S * span * sizeof(V)), empty0 = full0 + 8 * S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(full0 + 8 * q, 1);
            mbar_init(empty0 + 8 * q, kObsConsumers);
        }
        mbar_init_fence();
    }
    __syncthreads();
    const long long total = tiles * nx;
    const long long lo = total * blockIdx.x / gridDim.x, hi = total * (blockIdx.x + 1) / gridDim.x;
    Acc<float> rho, y2, z2, x2, rho2, lx, ly, lz;
    bool ok = true;
    if (warp == kObsConsumers) {
        // producer: ring position p holds the p-th copied plane of the block
        if (lane == 0) {
            ObsRun run{lo, hi, nx};
            long long tile;
            int i0, i1;
            unsigned p = 0;
            while (ok && run.next(tile, i0, i1)) {
                const long long s0 = tile * TILE;
                const unsigned bytes = (unsigned)(min((long long)span, plane - s0) * (long long)sizeof(V));
                const int pf = i0 > 0 ? i0 - 1 : 0;
                const char *src = static_cast<const char *>(a.psi) + (long long)pf * pbytes + s0 * (long long)sizeof(V);
                for (int q = 0; q < i1 - pf; ++q, ++p) {
                    const unsigned st = p % S;
                    // the stage's previous plane (position p - S) has been summed by every consumer warp
                    if (p >= S) ok = mbar_wait_bounded(empty0 + 8 * st, (p / S - 1) & 1u, ok);
                    if (!ok) break;  // after an expired wait the producer stops copying
                    mbar_arrive_expect_tx(full0 + 8 * st, bytes);
                    bulk_load(ring + st * span * (unsigned)sizeof(V), src + q * pbytes, bytes, full0 + 8 * st);
                }
            }
            // after an expired wait: give the copies still in flight a fresh
            // bound before the block's shared memory is released
            if (!ok)
                for (unsigned q = p > S ? p - S : 0; q < p; ++q) mbar_wait_bounded(full0 + 8 * (q % S), (q / S) & 1u, true);
        }
    } else {
        ObsRun run{lo, hi, nx};
        long long tile;
        int i0, i1;
        unsigned p = 0;
        const float x0 = (float)a.origin[0], dx = (float)a.d[0];
        while (run.next(tile, i0, i1)) {
            const long long s0 = tile * TILE;
            // an interior tile has every site, every +y neighbour and the
            // whole stage copied; the plane's last tile (or two) is an edge tile
            const bool interior = s0 + span <= plane;
            const int pf = i0 > 0 ? i0 - 1 : 0;
            const int np = i1 - pf;
            unsigned vmask = 0, ymask = 0, zmask = 0;  // sites present; with a +y, a +z neighbour
#pragma unroll
            for (int m = 0; m < SPT; ++m) {
                const long long sidx = s0 + threadIdx.x + m * kReduceThreads;
                const int j = (int)(sidx / nz), k = (int)(sidx % nz);
                if (sidx < plane) {
                    vmask |= 1u << m;
                    if (j + 1 < ny) ymask |= 1u << m;
                    if (k + 1 < nz) zmask |= 1u << m;
                }
            }
            V prev[SPT], sr[SPT];
            Acc<float> rk[SPT];
#pragma unroll
            for (int m = 0; m < SPT; ++m) {
                prev[m] = 0.f;
                sr[m] = 0.f;
            }
            float sx2 = 0.f, sr2 = 0.f, slx = 0.f, sly = 0.f, slz = 0.f;
            int nf = 0;  // planes in the current FP32 fold
            // one site of one plane; LX: the plane has a -x neighbour
            auto site = [&](const V v, const V qy, const V qz, int m, float xq, auto lx_tag) {
                constexpr bool LX = decltype(lx_tag)::value;
                const float r2 = v * v;
                sr[m] += r2;
                sx2 = fmaf(xq, r2, sx2);
                sr2 = fmaf(r2, r2, sr2);
                if constexpr (LX) {
                    const float d = v - prev[m];
                    slx = fmaf(d, d, slx);
                }
                const float dy = qy - v;
                sly = fmaf(dy, dy, sly);
                const float dz = (zmask >> m & 1u) ? qz - v : 0.f;
                slz = fmaf(dz, dz, slz);
                prev[m] = v;
            };
            auto sum_plane = [&](const V *t, int i, auto lx_tag) {
                const float xx = fmaf((float)i, dx, x0);
                const float xq = xx * xx;
                if (interior) {
#pragma unroll
                    for (int m = 0; m < SPT; ++m) {
                        const int l = threadIdx.x + m * kReduceThreads;
                        site(t[l], t[l + nz], t[l + 1], m, xq, lx_tag);
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < SPT; ++m) {
                        if (vmask >> m & 1u) {
                            const int l = threadIdx.x + m * kReduceThreads;
                            const V v = t[l];
                            site(v, (ymask >> m & 1u) ? t[l + nz] : v, (zmask >> m & 1u) ? t[l + 1] : v, m, xq, lx_tag);
                        }
                    }
                }
            };
            for (int q = 0; q < np; ++q, ++p) {
                const unsigned st = p % S;
                ok = mbar_wait_bounded(full0 + 8 * st, (p / S) & 1u, ok) && ok;
                const V *t = stage0 + st * span;
                const int i = pf + q;
                if (i < i0) {
#pragma unroll
                    for (int m = 0; m < SPT; ++m)
                        if (vmask >> m & 1u) prev[m] = t[threadIdx.x + m * kReduceThreads];
                } else {
                    if (i == 0) sum_plane(t, i, std::false_type());
                    else sum_plane(t, i, std::true_type());
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty0 + 8 * st);  // this warp is done with the stage
                if (i >= i0 && (++nf == kObsFold || q == np - 1)) {
#pragma unroll
                    for (int m = 0; m < SPT; ++m) {
                        rk[m].add(sr[m]);
                        sr[m] = 0.f;
                    }
                    x2.add(sx2);
                    rho2.add(sr2);
                    lx.add(slx);
                    ly.add(sly);
                    lz.add(slz);
                    sx2 = sr2 = slx = sly = slz = 0.f;
                    nf = 0;
                }
            }
#pragma unroll
            for (int m = 0; m < SPT; ++m) {
                const long long sidx = s0 + threadIdx.x + m * kReduceThreads;
                const int j = (int)(sidx / nz), k = (int)(sidx % nz);
                const float y = (float)(a.origin[1] + j * a.d[1]), z = (float)(a.origin[2] + k * a.d[2]);
                rho = acc_sum(rho, rk[m]);
                y2 = acc_sum(y2, acc_scaled(rk[m], y * y));
                z2 = acc_sum(z2, acc_scaled(rk[m], z * z));
            }
        }
    }
    const int expired = __syncthreads_or(!ok);
    if (expired && threadIdx.x == 0 && a.status) atomicOr(a.status, 2u);
    const float sc = (float)__ldg(a.scale);
    const float s2 = sc * sc;
    Acc<float> acc[9];
    acc[O_RHO] = acc_scaled(rho, s2);
    acc[O_X2] = acc_scaled(x2, s2);
    acc[O_Y2] = acc_scaled(y2, s2);
    acc[O_Z2] = acc_scaled(z2, s2);
    acc[O_RHO2] = acc_scaled(rho2, s2 * s2);
    acc[O_LX] = acc_scaled(lx, s2);
    acc[O_LY] = acc_scaled(ly, s2);
    acc[O_LZ] = acc_scaled(lz, s2);
    acc[O_V] = acc_sum(acc_sum(acc_scaled(acc[O_X2], (float)a.half_w2[0]), acc_scaled(acc[O_Y2], (float)a.half_w2[1])),
                       acc_scaled(acc[O_Z2], (float)a.half_w2[2]));
    float ps[9], pc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        ps[q] = acc[q].s;
        pc[q] = acc[q].c;
    }
    double bs[9];
    block_sum_pairs<9>(ps, pc, bs);
    finalize_partials<9>(bs, a, [&](const double *t) { obs_finish(a, t); }, blockIdx.x, gridDim.x);
}

// Resident blocks of observables_bulk_kernel on each device at its largest
// shared-memory ring, looked up (and the shared-memory limit raised) once
// per device by prepare_field_launches.
std::atomic<int> g_bulk_resident[kMaxDevices];

int bulk_resident(int dev) {
    constexpr int smem = kObsStages * kObsStageBytes + 16 * kObsStages;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(observables_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(observables_bulk_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, observables_bulk_kernel, kObsThreads, smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return std::max(1, sms) * std::max(1, per_sm);
}

// Blocks of observables_bulk_kernel for an FP32 real field, 0 where it does
// not apply: planes must be whole 16-byte units (each plane's copy starts on
// a 16-byte boundary), a stage (tile + nz + 1 sites) must fit
// kObsStageBytes, and the resident wave must have been looked up on the
// current device.  Each block gets a run of at least 8 (tile, plane) pairs.
unsigned obs_bulk_grid(const FieldArgs &a) {
    const long long plane = (long long)a.n[1] * a.n[2];
    if (plane % 4 != 0 || obs_bulk_span(a.n[2]) * (long long)sizeof(float) > kObsStageBytes) return 0;
    int dev = 0;
    cudaGetDevice(&dev);
    const long long g = dev >= 0 && dev < kMaxDevices ? g_bulk_resident[dev].load() : 0;
    if (g <= 0) return 0;
    const long long runs = ((plane + kObsTile - 1) / kObsTile * a.n[0] + 7) / 8;
    return (unsigned)std::max(1LL, std::min(g, runs));
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

// Real-time kick of every site, psi <- exp(-i kdt (V + g |s psi|^2)) s psi
// (the symmetric splitting's trailing half kick, kdt = dt / 2).  Every
// constant arrives in the field's precision (FP64 work per thread would cost
// more than the site's memory traffic on this part); a block walks
// kKickRows rows of z, threads along z.
template <typename R> struct KickConsts {
    R x0, dx, y0, dy, z0, dz, hx, hy, hz, kg, kt;
};
constexpr int kKickRows = 16;

template <typename R>
__global__ void kick_kernel(const double *__restrict__ scale, KickConsts<R> k, const void *psi, void *dst, int nx,
                            int ny, int nz) {
    using V = cx<R>;
    const R s = (R)__ldg(scale);  // once per thread: each thread walks ~kKickRows sites
    const long long rows = (long long)nx * ny;
    for (long long row = (long long)blockIdx.x * kKickRows, re = min(row + kKickRows, rows); row < re; ++row) {
        const int x = (int)(row / ny), y = (int)(row % ny);
        const R cx_ = fma((R)x, k.dx, k.x0), cy = fma((R)y, k.dy, k.y0);
        const R vxy = fma(k.hx * cx_, cx_, k.hy * cy * cy);
        const V *src = static_cast<const V *>(psi) + row * nz;
        V *out = static_cast<V *>(dst) + row * nz;
        for (int z = threadIdx.x; z < nz; z += blockDim.x) {
            const R cz = fma((R)z, k.dz, k.z0);
            const V q{src[z].re * s, src[z].im * s};
            const R th = fma(k.kg, fma(q.re, q.re, q.im * q.im), k.kt * fma(k.hz * cz, cz, vxy));
            R sn, cs;
            kick_sincos(th, &sn, &cs);
            out[z] = V{fma(cs, q.re, sn * q.im), fma(cs, q.im, -sn * q.re)};
        }
    }
}

template <typename R> cudaError_t launch_kick_r(const FieldArgs &a, double kdt, void *dst, cudaStream_t s) {
    KickConsts<R> k{(R)a.origin[0], (R)a.d[0], (R)a.origin[1], (R)a.d[1], (R)a.origin[2], (R)a.d[2],
                    (R)a.half_w2[0], (R)a.half_w2[1], (R)a.half_w2[2], (R)(kdt * a.g), (R)kdt};
    const long long rows = (long long)a.n[0] * a.n[1];
    const unsigned blocks = (unsigned)((rows + kKickRows - 1) / kKickRows);
    const unsigned threads = a.n[2] >= 256 ? 256 : 128;
    kick_kernel<R><<<blocks, threads, 0, s>>>(a.scale, k, a.psi, dst, a.n[0], a.n[1], a.n[2]);
    return cudaGetLastError();
}

template <typename R, bool CPLX>
__global__ void apply_scale_kernel(FieldArgs a, void *dst) {
    using E = Elem<R, CPLX>;
    const typename E::V *src = static_cast<const typename E::V *>(a.psi);
    typename E::V *out = static_cast<typename E::V *>(dst);
    const typename E::T s = (typename E::T)__ldg(a.scale);
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
    case 2:
        if constexpr (sizeof(R) == 4 && CPLX) {
            const unsigned g = a.n[2] % 2 == 0 ? obs_c64z_grid(a) : 0;
            if (g > 0)
                observables_c64z_kernel<<<g, kReduceThreads, 0, s>>>(a);
            else
                observables_c64_kernel<<<observables_body_blocks(a), kReduceThreads, 0, s>>>(a);
        } else if constexpr (sizeof(R) == 4) {
            const unsigned gb = obs_bulk_grid(a);
            if (gb > 0)
                observables_bulk_kernel<<<gb, kObsThreads, obs_bulk_smem(a.n[2]), s>>>(a);
            else
                observables_kernel<R, CPLX><<<observables_body_blocks(a), kReduceThreads, 0, s>>>(a);
        } else
            observables_kernel<R, CPLX><<<observables_body_blocks(a), kReduceThreads, 0, s>>>(a);
        break;
    case 3: apply_scale_kernel<R, CPLX><<<fill_blocks(a.sites), 256, 0, s>>>(a, dst); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t dispatch_all(Prec p, bool cplx, int what, const FieldArgs &a, int blocks, void *dst,
                         cudaStream_t s) {
    if (p == P_F64) return cplx ? dispatch<double, true>(what, a, blocks, dst, s)
                                : dispatch<double, false>(what, a, blocks, dst, s);
    if (p == P_F16) return cplx ? cudaErrorInvalidValue : dispatch<__half, false>(what, a, blocks, dst, s);
    return cplx ? dispatch<float, true>(what, a, blocks, dst, s)
                : dispatch<float, false>(what, a, blocks, dst, s);
}

}  // namespace

void prepare_field_launches() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return;
    }
    if (g_c64z_resident[dev].load() <= 0) g_c64z_resident[dev].store(c64z_resident(dev));
    if (g_bulk_resident[dev].load() <= 0) g_bulk_resident[dev].store(bulk_resident(dev));
}

cudaError_t launch_kick(Prec p, const FieldArgs &a, double kdt, void *dst, cudaStream_t s) {
    if (p == P_F16) return cudaErrorInvalidValue;  // real time: complex fields only
    return p == P_F64 ? launch_kick_r<double>(a, kdt, dst, s) : launch_kick_r<float>(a, kdt, dst, s);
}

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

// Blocks of observables_body over one condensate (one per 256 (j, k) and
// kObsSeg planes): the grid of observables_kernel and observables_c64_kernel,
// and one condensate's share of observables_batch_kernel.
int observables_body_blocks(const FieldArgs &a) {
    const long long plane = (long long)a.n[1] * a.n[2];
    const long long segs = (a.n[0] + kObsSeg - 1) / kObsSeg;
    return (int)((plane + kReduceThreads - 1) / kReduceThreads * segs);
}

// The most blocks (and so partials) any observables grid of this field has.
int observables_blocks(const FieldArgs &a) {
    const long long bulk = obs_bulk_grid(a);
    return (int)std::max(std::max((long long)observables_body_blocks(a), obs_c64z_items(a.n)), bulk);
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

// k_nn.cu -- kernels of the learned warm start: a conditioned coordinate MLP
// that maps a grid node of a condensate (and the condensate's gamma, nu,
// lambda, g) to a ground-state amplitude.
//
// Network (all hidden layers 64 wide, tanh):
//   x (16 features, 9 used) -> h1 = tanh(x W0 + b0) -> h2 = tanh(h1 W1 + b1)
//   -> h3 = tanh(h2 W2 + b2) -> y = softplus(h3 . w3 + b3)
// The three matrix layers run on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation); each warp carries 16 points through the
// layers in registers (a layer's FP32 output fragments are exactly the next
// layer's BF16 input fragments).  Training adds the backward pass:
//   dz4 = (2/P)(y - t) sigmoid(z4),  d3 = dz4 w3 (1 - h3^2),
//   d2 = (d3 W2^T)(1 - h2^2),  d1 = (d2 W1^T)(1 - h1^2),
//   dW2 = h2^T d3, dW1 = h1^T d2, dW0 = x^T d1 (tensor cores, K = points),
//   biases: column sums of d; dw3 = h3^T dz4; db3 = sum dz4,
// written as per-block partial gradients, summed in block order by a second
// kernel (deterministic), then an Adam step on FP32 master weights.
#include "gp_nn_internal.h"

#include <cuda_bf16.h>

namespace gpcn {
namespace {

constexpr int H = kNNHidden;       // 64
constexpr int IN = kNNIn;          // 16
constexpr int PAD = 8;             // row padding (bf16) of the shared activation tiles
constexpr int LD = H + PAD;        // 72
constexpr int LDX = IN + PAD;      // 24
constexpr int TPTS = 128;          // points per training block (8 warps x 16)

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}
__device__ __forceinline__ unsigned pack_pair(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<unsigned *>(&v);
}
__device__ __forceinline__ unsigned ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const unsigned *>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float softplus(float z) { return z > 20.f ? z : log1pf(expf(z)); }
__device__ __forceinline__ float sigmoid(float z) { return 1.f / (1.f + expf(-z)); }

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): a counter-based 64-bit mix.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Features of node `site` of instance I (see kNNFeatures in gp_nn_internal.h).
__device__ __forceinline__ void features(const NNInstance &I, long long site, float (&f)[IN]) {
    const int k = (int)(site % I.n[2]);
    const int j = (int)((site / I.n[2]) % I.n[1]);
    const int i = (int)(site / ((long long)I.n[2] * I.n[1]));
    const float x[3] = {I.origin[0] + i * I.d[0], I.origin[1] + j * I.d[1], I.origin[2] + k * I.d[2]};
    float su = 0.f, sq = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = x[a] * I.sqrt_w[a];
        f[a] = 0.125f * fminf(u * u, 16.f) - 1.f;  // even in x_a: so is every prediction
        su += u * u;
        const float q = x[a] * I.inv_rtf[a];
        sq += q * q;
    }
    f[3] = 0.5f * fminf(sq, 4.f) - 1.f;
    f[4] = 0.125f * fminf(su, 16.f) - 1.f;
    f[5] = I.lg;
#pragma unroll
    for (int a = 0; a < 3; ++a) f[6 + a] = I.wn[a];
#pragma unroll
    for (int a = 9; a < IN; ++a) f[a] = 0.f;
}

// Shared copies of the weights as the mma fragments want them.
struct SmemW {
    __nv_bfloat16 w0t[H * IN];   // [out][in]
    __nv_bfloat16 w1t[H * H];    // [out][in]
    __nv_bfloat16 w2t[H * H];
    __nv_bfloat16 w1n[H * H];    // [in][out]
    __nv_bfloat16 w2n[H * H];
    float b0[H], b1[H], b2[H], w3[H];
    float b3;
};

__device__ void load_weights(SmemW &s, const NNParams &P, bool backward) {
    const unsigned *src;
    unsigned *dst;
    const int t = threadIdx.x, nt = blockDim.x;
    src = reinterpret_cast<const unsigned *>(P.deploy + kDepW0T);
    dst = reinterpret_cast<unsigned *>(s.w0t);
    for (int q = t; q < H * IN / 2; q += nt) dst[q] = src[q];
    src = reinterpret_cast<const unsigned *>(P.deploy + kDepW1T);
    dst = reinterpret_cast<unsigned *>(s.w1t);
    for (int q = t; q < H * H / 2; q += nt) dst[q] = src[q];
    src = reinterpret_cast<const unsigned *>(P.deploy + kDepW2T);
    dst = reinterpret_cast<unsigned *>(s.w2t);
    for (int q = t; q < H * H / 2; q += nt) dst[q] = src[q];
    if (backward) {
        src = reinterpret_cast<const unsigned *>(P.deploy + kDepW1N);
        dst = reinterpret_cast<unsigned *>(s.w1n);
        for (int q = t; q < H * H / 2; q += nt) dst[q] = src[q];
        src = reinterpret_cast<const unsigned *>(P.deploy + kDepW2N);
        dst = reinterpret_cast<unsigned *>(s.w2n);
        for (int q = t; q < H * H / 2; q += nt) dst[q] = src[q];
    }
    for (int q = t; q < H; q += nt) {
        s.b0[q] = P.master[kOffB0 + q];
        s.b1[q] = P.master[kOffB1 + q];
        s.b2[q] = P.master[kOffB2 + q];
        s.w3[q] = P.master[kOffW3 + q];
    }
    if (t == 0) s.b3 = P.master[kOffB3];
}

// One dense layer for a warp's 16 points: A fragments (4 k-tiles of the
// input, or 1 for the first layer) times the transposed weights wt[out][in]
// with row length `kin`; returns the 8 output n-tiles (16 x 64, FP32).
template <int KT>
__device__ __forceinline__ void layer(const unsigned (&a)[KT][4], const __nv_bfloat16 *wt, int kin,
                                      const float *bias, float (&d)[8][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float b_lo = bias[8 * j + 2 * t], b_hi = bias[8 * j + 2 * t + 1];
        d[j][0] = b_lo;
        d[j][1] = b_hi;
        d[j][2] = b_lo;
        d[j][3] = b_hi;
        const __nv_bfloat16 *row = wt + (8 * j + g) * kin;
#pragma unroll
        for (int kt = 0; kt < KT; ++kt)
            mma_bf16(d[j], a[kt][0], a[kt][1], a[kt][2], a[kt][3], ld32(row + 16 * kt + 2 * t),
                     ld32(row + 16 * kt + 8 + 2 * t));
    }
}

// FP32 output fragments of one layer -> BF16 input fragments of the next.
__device__ __forceinline__ void to_afrag(const float (&h)[8][4], unsigned (&a)[4][4]) {
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        a[kt][0] = pack_bf16(h[2 * kt][0], h[2 * kt][1]);
        a[kt][1] = pack_bf16(h[2 * kt][2], h[2 * kt][3]);
        a[kt][2] = pack_bf16(h[2 * kt + 1][0], h[2 * kt + 1][1]);
        a[kt][3] = pack_bf16(h[2 * kt + 1][2], h[2 * kt + 1][3]);
    }
}

__device__ __forceinline__ void tanh_frag(float (&h)[8][4]) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) h[j][c] = tanhf(h[j][c]);
}

// Input fragment of 16 points from their features (rows g and g+8 of the
// warp's tile): columns 2t, 2t+1 and 2t+8, 2t+9.
__device__ __forceinline__ void input_frag(const float (&fa)[IN], const float (&fb)[IN], unsigned (&a)[1][4]) {
    const int t = threadIdx.x & 3;
    a[0][0] = pack_bf16(fa[2 * t], fa[2 * t + 1]);
    a[0][1] = pack_bf16(fb[2 * t], fb[2 * t + 1]);
    a[0][2] = pack_bf16(fa[2 * t + 8], fa[2 * t + 9]);
    a[0][3] = pack_bf16(fb[2 * t + 8], fb[2 * t + 9]);
}

// h3 . w3 over the row: each thread holds 16 of the 64 columns of rows g and
// g+8; the four threads of a row group sum their parts.
__device__ __forceinline__ void out_dot(const float (&h)[8][4], const float *w3, float b3, float *za, float *zb) {
    const int t = threadIdx.x & 3;
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float wl = w3[8 * j + 2 * t], wh = w3[8 * j + 2 * t + 1];
        sa = fmaf(h[j][0], wl, fmaf(h[j][1], wh, sa));
        sb = fmaf(h[j][2], wl, fmaf(h[j][3], wh, sb));
    }
    sa += __shfl_xor_sync(0xffffffffu, sa, 1);
    sa += __shfl_xor_sync(0xffffffffu, sa, 2);
    sb += __shfl_xor_sync(0xffffffffu, sb, 1);
    sb += __shfl_xor_sync(0xffffffffu, sb, 2);
    *za = sa + b3;
    *zb = sb + b3;
}

// ---------------------------------------------------------------- prediction
// psi0 at every node of one condensate: amplitude y (boundary nodes 0).
template <typename R, bool CPLX>
__global__ void __launch_bounds__(128) nn_predict_kernel(NNParams P, NNInstance I, void *out, long long sites) {
    __shared__ SmemW s;
    load_weights(s, P, false);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2;
    const long long base = ((long long)blockIdx.x * 4 + warp) * 16;
    if (base >= sites) return;
    const long long pa = base + g, pb = base + g + 8;
    float fa[IN], fb[IN];
    features(I, min(pa, sites - 1), fa);
    features(I, min(pb, sites - 1), fb);
    unsigned a0[1][4];
    input_frag(fa, fb, a0);
    float h[8][4];
    unsigned a[4][4];
    layer<1>(a0, s.w0t, IN, s.b0, h);
    tanh_frag(h);
    to_afrag(h, a);
    layer<4>(a, s.w1t, H, s.b1, h);
    tanh_frag(h);
    to_afrag(h, a);
    layer<4>(a, s.w2t, H, s.b2, h);
    tanh_frag(h);
    float za, zb;
    out_dot(h, s.w3, s.b3, &za, &zb);
    if ((lane & 3) == 0) {
        const long long p2[2] = {pa, pb};
        const float z2[2] = {za, zb};
        for (int r = 0; r < 2; ++r) {
            const long long p = p2[r];
            if (p >= sites) continue;
            const int k = (int)(p % I.n[2]);
            const int j = (int)((p / I.n[2]) % I.n[1]);
            const int i = (int)(p / ((long long)I.n[2] * I.n[1]));
            const bool edge = i == 0 || j == 0 || k == 0 || i == I.n[0] - 1 || j == I.n[1] - 1 || k == I.n[2] - 1;
            const R y = edge ? R(0) : (R)softplus(z2[r]);
            if (CPLX) {
                static_cast<R *>(out)[2 * p] = y;
                static_cast<R *>(out)[2 * p + 1] = R(0);
            } else {
                static_cast<R *>(out)[p] = y;
            }
        }
    }
}

// ---------------------------------------------------------------- training
struct TrainSmem {
    SmemW w;
    __nv_bfloat16 x[TPTS * LDX];
    __nv_bfloat16 h1[TPTS * LD], h2[TPTS * LD];
    __nv_bfloat16 d1[TPTS * LD], d2[TPTS * LD], d3[TPTS * LD];
    float red[8][H];   // per-warp column sums (biases, w3)
    float loss[8];
    float dz[TPTS];    // dz4 per point (for db3)
};

// Store a warp's 16 x 64 FP32 fragment tile as BF16 rows of `tile` (row = point).
__device__ __forceinline__ void store_tile(const float (&v)[8][4], __nv_bfloat16 *tile, int row0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        *reinterpret_cast<unsigned *>(tile + (row0 + g) * LD + 8 * j + 2 * t) = pack_bf16(v[j][0], v[j][1]);
        *reinterpret_cast<unsigned *>(tile + (row0 + g + 8) * LD + 8 * j + 2 * t) = pack_bf16(v[j][2], v[j][3]);
    }
}

// Column sums of a warp's 16 x 64 fragment tile into red[warp][*].
__device__ __forceinline__ void colsum(const float (&v)[8][4], float *red) {
    const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float lo = v[j][0] + v[j][2], hi = v[j][1] + v[j][3];
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            lo += __shfl_xor_sync(0xffffffffu, lo, o);
            hi += __shfl_xor_sync(0xffffffffu, hi, o);
        }
        if (lane < 4) {
            red[8 * j + 2 * t] = lo;
            red[8 * j + 2 * t + 1] = hi;
        }
    }
}

// d_in = (d_out W^T) (1 - h_in^2) for a warp's 16 points: d_out fragments
// (A, k = out index) times wn[in][out] (B[k = out][n = in]).
__device__ __forceinline__ void backprop(const unsigned (&a)[4][4], const __nv_bfloat16 *wn, const float (&h)[8][4],
                                         float (&d)[8][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.f;
        const __nv_bfloat16 *row = wn + (8 * j + g) * H;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
            mma_bf16(d[j], a[kt][0], a[kt][1], a[kt][2], a[kt][3], ld32(row + 16 * kt + 2 * t),
                     ld32(row + 16 * kt + 8 + 2 * t));
#pragma unroll
        for (int c = 0; c < 4; ++c) d[j][c] *= 1.f - h[j][c] * h[j][c];
    }
}

// dW[i][o] = sum_p A[p][i] B[p][o] over the block's 128 points (A rows of
// length lda, B rows of length LD), for i in m-tile mt, o in n-tiles n0..n0+nn-1;
// written into the block's partial-gradient row at `dst` ([in][out], row length H).
__device__ __forceinline__ void wgrad(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int mt, int n0, int nn,
                                      float *dst) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float d[4][4];
    for (int q = 0; q < nn; ++q) d[q][0] = d[q][1] = d[q][2] = d[q][3] = 0.f;
    for (int ks = 0; ks < TPTS / 16; ++ks) {
        const int p0 = 16 * ks + 2 * t;
        const int i0 = 16 * mt + g;
        const unsigned a0 = pack_pair(A[p0 * lda + i0], A[(p0 + 1) * lda + i0]);
        const unsigned a1 = pack_pair(A[p0 * lda + i0 + 8], A[(p0 + 1) * lda + i0 + 8]);
        const unsigned a2 = pack_pair(A[(p0 + 8) * lda + i0], A[(p0 + 9) * lda + i0]);
        const unsigned a3 = pack_pair(A[(p0 + 8) * lda + i0 + 8], A[(p0 + 9) * lda + i0 + 8]);
        for (int q = 0; q < nn; ++q) {
            const int o = 8 * (n0 + q) + g;
            const unsigned b0 = pack_pair(B[p0 * LD + o], B[(p0 + 1) * LD + o]);
            const unsigned b1 = pack_pair(B[(p0 + 8) * LD + o], B[(p0 + 9) * LD + o]);
            mma_bf16(d[q], a0, a1, a2, a3, b0, b1);
        }
    }
    for (int q = 0; q < nn; ++q) {
        const int o = 8 * (n0 + q) + 2 * t;
        const int i = 16 * mt + g;
        dst[i * H + o] = d[q][0];
        dst[i * H + o + 1] = d[q][1];
        dst[(i + 8) * H + o] = d[q][2];
        dst[(i + 8) * H + o + 1] = d[q][3];
    }
}

__global__ void __launch_bounds__(256, 1) nn_train_kernel(NNParams P, NNTrain T) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &s = *reinterpret_cast<TrainSmem *>(smem_raw);
    load_weights(s.w, P, true);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int row0 = 16 * warp;
    // this thread's two points (rows g and g + 8 of the warp's tile)
    const long long sa = (long long)blockIdx.x * TPTS + row0 + g, sb = sa + 8;
    int ia, ib;
    long long pa, pb;
    if (T.sample_inst) {
        ia = T.sample_inst[sa];
        pa = T.sample_site[sa];
        ib = T.sample_inst[sb];
        pb = T.sample_site[sb];
    } else {
        const unsigned long long ra = splitmix64(T.seed ^ (unsigned long long)sa * 0xD1B54A32D192ED03ULL);
        const unsigned long long rb = splitmix64(T.seed ^ (unsigned long long)sb * 0xD1B54A32D192ED03ULL);
        ia = (int)((ra >> 40) % (unsigned long long)T.n_inst);
        ib = (int)((rb >> 40) % (unsigned long long)T.n_inst);
        pa = (long long)((ra & 0xFFFFFFFFFFULL) % (unsigned long long)T.inst[ia].sites);
        pb = (long long)((rb & 0xFFFFFFFFFFULL) % (unsigned long long)T.inst[ib].sites);
    }
    const NNInstance &Ia = T.inst[ia], &Ib = T.inst[ib];
    float fa[IN], fb[IN];
    features(Ia, pa, fa);
    features(Ib, pb, fb);
    const float ta = T.data[Ia.data_off + pa] * Ia.inv_max, tb = T.data[Ib.data_off + pb] * Ib.inv_max;
    if (t == 0) {
        for (int c = 0; c < IN; ++c) {
            s.x[(row0 + g) * LDX + c] = __float2bfloat16_rn(fa[c]);
            s.x[(row0 + g + 8) * LDX + c] = __float2bfloat16_rn(fb[c]);
        }
    }
    __syncthreads();
    // forward
    unsigned a0[1][4];
    input_frag(fa, fb, a0);
    float h1[8][4], h2[8][4], h3[8][4];
    unsigned a[4][4];
    layer<1>(a0, s.w.w0t, IN, s.w.b0, h1);
    tanh_frag(h1);
    store_tile(h1, s.h1, row0);
    to_afrag(h1, a);
    layer<4>(a, s.w.w1t, H, s.w.b1, h2);
    tanh_frag(h2);
    store_tile(h2, s.h2, row0);
    to_afrag(h2, a);
    layer<4>(a, s.w.w2t, H, s.w.b2, h3);
    tanh_frag(h3);
    float za, zb;
    out_dot(h3, s.w.w3, s.w.b3, &za, &zb);
    const float ya = softplus(za), yb = softplus(zb);
    const float inv_p = 1.f / (float)T.points;
    const float dza = 2.f * inv_p * (ya - ta) * sigmoid(za), dzb = 2.f * inv_p * (yb - tb) * sigmoid(zb);
    // loss and dz4 per point
    float l = t == 0 ? ((ya - ta) * (ya - ta) + (yb - tb) * (yb - tb)) * inv_p : 0.f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) s.loss[warp] = l;
    if (t == 0) {
        s.dz[row0 + g] = dza;
        s.dz[row0 + g + 8] = dzb;
    }
    // dw3 = h3^T dz4 (per-warp column sums of h3 * dz)
    float hd[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        hd[j][0] = h3[j][0] * dza;
        hd[j][1] = h3[j][1] * dza;
        hd[j][2] = h3[j][2] * dzb;
        hd[j][3] = h3[j][3] * dzb;
    }
    float *part = T.partials + (size_t)blockIdx.x * kNNParams;
    colsum(hd, s.red[warp]);
    __syncthreads();
    if (threadIdx.x < H) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += s.red[w][threadIdx.x];
        part[kOffW3 + threadIdx.x] = v;
    }
    if (threadIdx.x == 0) {
        float v = 0.f, lv = 0.f;
        for (int p = 0; p < TPTS; ++p) v += s.dz[p];
        for (int w = 0; w < 8; ++w) lv += s.loss[w];
        part[kOffB3] = v;
        T.loss_partials[blockIdx.x] = lv;
    }
    // d3 = dz4 w3 (1 - h3^2)
    float d[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float wl = s.w.w3[8 * j + 2 * t], wh = s.w.w3[8 * j + 2 * t + 1];
        d[j][0] = dza * wl * (1.f - h3[j][0] * h3[j][0]);
        d[j][1] = dza * wh * (1.f - h3[j][1] * h3[j][1]);
        d[j][2] = dzb * wl * (1.f - h3[j][2] * h3[j][2]);
        d[j][3] = dzb * wh * (1.f - h3[j][3] * h3[j][3]);
    }
    store_tile(d, s.d3, row0);
    __syncthreads();
    colsum(d, s.red[warp]);
    __syncthreads();
    if (threadIdx.x < H) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += s.red[w][threadIdx.x];
        part[kOffB2 + threadIdx.x] = v;
    }
    // d2 = (d3 W2^T)(1 - h2^2)
    to_afrag(d, a);
    backprop(a, s.w.w2n, h2, d);
    store_tile(d, s.d2, row0);
    __syncthreads();
    colsum(d, s.red[warp]);
    __syncthreads();
    if (threadIdx.x < H) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += s.red[w][threadIdx.x];
        part[kOffB1 + threadIdx.x] = v;
    }
    // d1 = (d2 W1^T)(1 - h1^2)
    to_afrag(d, a);
    backprop(a, s.w.w1n, h1, d);
    store_tile(d, s.d1, row0);
    __syncthreads();
    colsum(d, s.red[warp]);
    __syncthreads();
    if (threadIdx.x < H) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += s.red[w][threadIdx.x];
        part[kOffB0 + threadIdx.x] = v;
    }
    // weight gradients over the block's 128 points (tensor cores, K = points)
    wgrad(s.h2, LD, s.d3, warp & 3, (warp >> 2) * 4, 4, part + kOffW2);
    wgrad(s.h1, LD, s.d2, warp & 3, (warp >> 2) * 4, 4, part + kOffW1);
    wgrad(s.x, LDX, s.d1, 0, warp, 1, part + kOffW0);
}

// grad[q] = sum over blocks of partial[b][q], in block order; loss likewise.
__global__ void nn_reduce_kernel(const float *partials, int blocks, float *grad, const float *loss_partials,
                                 float *loss) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < kNNParams) {
        float v = 0.f;
        for (int b = 0; b < blocks; ++b) v += partials[(size_t)b * kNNParams + q];
        grad[q] = v;
    }
    if (q == 0) {
        float v = 0.f;
        for (int b = 0; b < blocks; ++b) v += loss_partials[b];
        *loss = v;
    }
}

// Adam (Kingma and Ba 2015) on the FP32 master weights, then the BF16
// copies in the layouts the kernels read.
__global__ void nn_adam_kernel(NNParams P, const float *grad, float lr, float b1t, float b2t) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNNParams) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gq = grad[q];
    const float m = b1 * P.m[q] + (1.f - b1) * gq;
    const float v = b2 * P.v[q] + (1.f - b2) * gq * gq;
    P.m[q] = m;
    P.v[q] = v;
    const float w = P.master[q] - lr * (m / (1.f - b1t)) / (sqrtf(v / (1.f - b2t)) + eps);
    P.master[q] = w;
    write_deploy(P, q, w);
}

__global__ void nn_deploy_kernel(NNParams P) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < kNNParams) write_deploy(P, q, P.master[q]);
}

}  // namespace

size_t nn_train_smem() { return sizeof(TrainSmem); }

cudaError_t nn_launch_train(const NNParams &P, const NNTrain &T, int blocks, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(nn_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(TrainSmem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    nn_train_kernel<<<blocks, 256, sizeof(TrainSmem), s>>>(P, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nn_reduce_kernel<<<(kNNParams + 255) / 256, 256, 0, s>>>(T.partials, blocks, T.grad, T.loss_partials, T.loss);
    return cudaGetLastError();
}

cudaError_t nn_launch_adam(const NNParams &P, const float *grad, float lr, float b1t, float b2t, cudaStream_t s) {
    nn_adam_kernel<<<(kNNParams + 255) / 256, 256, 0, s>>>(P, grad, lr, b1t, b2t);
    return cudaGetLastError();
}

cudaError_t nn_launch_deploy(const NNParams &P, cudaStream_t s) {
    nn_deploy_kernel<<<(kNNParams + 255) / 256, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t nn_launch_predict(const NNParams &P, const NNInstance &I, void *out, bool f32, bool cplx,
                              cudaStream_t s) {
    const long long sites = (long long)I.n[0] * I.n[1] * I.n[2];
    const unsigned blocks = (unsigned)((sites + 63) / 64);
    if (f32) {
        if (cplx) nn_predict_kernel<float, true><<<blocks, 128, 0, s>>>(P, I, out, sites);
        else nn_predict_kernel<float, false><<<blocks, 128, 0, s>>>(P, I, out, sites);
    } else {
        if (cplx) nn_predict_kernel<double, true><<<blocks, 128, 0, s>>>(P, I, out, sites);
        else nn_predict_kernel<double, false><<<blocks, 128, 0, s>>>(P, I, out, sites);
    }
    return cudaGetLastError();
}

}  // namespace gpcn

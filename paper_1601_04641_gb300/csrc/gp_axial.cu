// gp_axial.cu -- axially symmetric condensates: psi(rho, z) for a trap with
// gamma = nu (the (rho, z) program variant of the predecessor package the
// paper's programs extend; the paper states the split-step CN method, not
// this grid, and the reading taken here is the oracle's R21).
//
// Grid psi[i][k] (z stride 1): radial node i = 1..nx-2 at rho_i =
// (i - 1/2) drho, node 0 a ghost nothing couples to, node nx-1 the Dirichlet
// boundary; z nodes centred, Dirichlet at both ends.  A step is the kick
// (fused into the radial sweep's loads), the radial CN line solves -- the
// finite-volume (1/rho) d/drho (rho d/drho) with face radii rho_{i +- 1/2},
// so its tridiagonal coefficients vary along the line and come from tables
// -- then the z line solves through the Cartesian z-sweep kernels, and in
// imaginary time the renormalisation in the cylindrical measure
// 2 pi rho drho dz (a weighted norm reduction; the factor is applied by
// the next kick).  The radial kernel runs one thread per z line (threads
// of a warp own adjacent z, so each node's load and store is one
// contiguous row) with the exact two-pass Thomas algorithm.
#include "gp.h"
#include "gp_host.h"
#include "gp_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace gpcn;

namespace {

template <typename R> struct Cx { R re, im; };

template <typename R> __device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return Cx<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) { return Cx<R>{a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) { return Cx<R>{a.re - b.re, a.im - b.im}; }

// The field's element: R (real field) or Cx<R>; coefficients are Cx<R> (their
// imaginary parts vanish in imaginary time).  For a real field only the real
// parts of the coefficients enter.
template <typename R, bool CPLX> struct AxElem;
template <typename R> struct AxElem<R, false> {
    using V = R;
    __device__ __forceinline__ static V zero() { return R(0); }
    __device__ __forceinline__ static V mul(Cx<R> c, V v) { return c.re * v; }
    __device__ __forceinline__ static V add(V a, V b) { return a + b; }
    __device__ __forceinline__ static V sub(V a, V b) { return a - b; }
    __device__ __forceinline__ static V scale(V v, R s) { return v * s; }
    __device__ __forceinline__ static double abs2(V v) { return (double)v * (double)v; }
    __device__ __forceinline__ static V phase(V q, R theta, bool realtime) { return q * exp(-theta); }
    __device__ __forceinline__ static V from_real(double x) { return (R)x; }
};
template <typename R> struct AxElem<R, true> {
    using V = Cx<R>;
    __device__ __forceinline__ static V zero() { return V{R(0), R(0)}; }
    __device__ __forceinline__ static V mul(Cx<R> c, V v) { return cmul(c, v); }
    __device__ __forceinline__ static V add(V a, V b) { return cadd(a, b); }
    __device__ __forceinline__ static V sub(V a, V b) { return csub(a, b); }
    __device__ __forceinline__ static V scale(V v, R s) { return V{v.re * s, v.im * s}; }
    __device__ __forceinline__ static double abs2(V v) {
        return (double)v.re * (double)v.re + (double)v.im * (double)v.im;
    }
    __device__ __forceinline__ static V phase(V q, R theta, bool realtime) {
        if (!realtime) {
            const R f = exp(-theta);
            return V{q.re * f, q.im * f};
        }
        R sn, cs;
        sincos(theta, &sn, &cs);
        return V{cs * q.re + sn * q.im, cs * q.im - sn * q.re};  // exp(-i theta) q
    }
    __device__ __forceinline__ static V from_real(double x) { return V{(R)x, R(0)}; }
};

struct AxArgs {
    const void *in;
    void *out;
    int nx, nz;
    double drho, dz, z0;  // z0: coordinate of z node 0
    double dt, g, gamma2, lambda2;
    const void *A, *C, *cp, *ip;  // radial tables, node t = 0..nx-3 (radial node t + 1)
    const double *scale;          // factor applied to psi on load (pending renormalisation)
    int realtime;
};

// Kick of radial node i, z node k, from the loaded value p.
template <typename R, bool CPLX>
__device__ __forceinline__ typename AxElem<R, CPLX>::V ax_kick(const AxArgs &a, typename AxElem<R, CPLX>::V p,
                                                               R s, int i, double vz) {
    using E = AxElem<R, CPLX>;
    const typename E::V q = E::scale(p, s);
    const double r = (i - 0.5) * a.drho;
    const R theta = (R)(a.dt * (0.5 * a.gamma2 * r * r + vz)) + (R)a.dt * (R)a.g * (R)E::abs2(q);
    return E::phase(q, theta, a.realtime != 0);
}

// Kick and radial CN solve of one z line per thread (exact two-pass Thomas:
// the forward values are staged in the output and read back).
template <typename R, bool CPLX>
__global__ void __launch_bounds__(128) axial_radial_kernel(AxArgs a) {
    using E = AxElem<R, CPLX>;
    using V = typename E::V;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.nz) return;
    const V *in = static_cast<const V *>(a.in);
    V *out = static_cast<V *>(a.out);
    const long long nz = a.nz;
    if (k == 0 || k == a.nz - 1) {  // the z boundary: zero whatever the input holds
        for (int i = 0; i < a.nx; ++i) out[i * nz + k] = E::zero();
        return;
    }
    const Cx<R> *A = static_cast<const Cx<R> *>(a.A), *C = static_cast<const Cx<R> *>(a.C);
    const Cx<R> *cp = static_cast<const Cx<R> *>(a.cp), *ip = static_cast<const Cx<R> *>(a.ip);
    const int n = a.nx - 2;
    const R s = (R)__ldg(a.scale);
    const double z = a.z0 + k * a.dz, vz = 0.5 * a.lambda2 * z * z;
    out[k] = E::zero();
    out[(a.nx - 1) * nz + k] = E::zero();
    V pm = E::zero();  // the ghost node: never coupled (A[0] = 0)
    V p0 = ax_kick<R, CPLX>(a, in[nz + k], s, 1, vz);
    V p1 = n > 1 ? ax_kick<R, CPLX>(a, in[2 * nz + k], s, 2, vz) : E::zero();
    V dp = E::zero();
    for (int t = 0; t < n; ++t) {
        const Cx<R> at = A[t], ct = C[t];
        const V r = E::add(p0, E::add(E::mul(at, E::sub(pm, p0)), E::mul(ct, E::sub(p1, p0))));
        dp = E::mul(ip[t], E::add(r, E::mul(at, dp)));
        out[(t + 1) * nz + k] = dp;
        pm = p0;
        p0 = p1;
        p1 = t + 3 <= n ? ax_kick<R, CPLX>(a, in[(t + 3) * nz + k], s, t + 3, vz) : E::zero();
    }
    V phi = dp;
    for (int t = n - 2; t >= 0; --t) {
        const Cx<R> c = cp[t];
        phi = E::sub(out[(t + 1) * nz + k], E::mul(c, phi));
        out[(t + 1) * nz + k] = phi;
    }
}

// Sums over the grid in the cylindrical measure, FP64: per-block partials of
// NV quantities, then one block adds them in block order (deterministic).
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;

__device__ __forceinline__ double ax_block_sum(double v) {
    __shared__ double red[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kRedThreads / 32; ++w) t += red[w];
    return t;
}

struct AxSums {
    const void *psi;
    int nx, nz;
    double drho, dz, z0, gamma2, lambda2;
    const double *scale;  // applied to psi on read
    double *partials;     // kRedBlocks x 6
};

// Per-block sums (weight w = 2 pi rho_i drho dz): [0] w|psi|^2, [1] w V|psi|^2,
// [2] w|psi|^4, [3] w rho^2|psi|^2, [4] w z^2|psi|^2, [5] the kinetic form
// (radial links weighted 2 pi rho_{i+1/2} dz / drho, z links 2 pi rho_i drho / dz, times 1/2).
template <typename R, bool CPLX>
__global__ void __launch_bounds__(kRedThreads) axial_sums_kernel(AxSums a) {
    using E = AxElem<R, CPLX>;
    using V = typename E::V;
    const V *psi = static_cast<const V *>(a.psi);
    const double s2 = (*a.scale) * (*a.scale);
    const long long sites = (long long)a.nx * a.nz;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const double two_pi = 6.283185307179586;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < sites;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / a.nz), k = (int)(q % a.nz);
        if (i < 1 || i > a.nx - 2) continue;
        const V p = psi[q];
        const double rho = E::abs2(p) * s2;
        const double r = (i - 0.5) * a.drho, z = a.z0 + k * a.dz, w = two_pi * r * a.drho * a.dz;
        acc[0] += w * rho;
        acc[1] += w * 0.5 * (a.gamma2 * r * r + a.lambda2 * z * z) * rho;
        acc[2] += w * rho * rho;
        acc[3] += w * r * r * rho;
        acc[4] += w * z * z * rho;
        const double dr = E::abs2(E::sub(psi[q + a.nz], p)) * s2;  // link to node i + 1
        double kin = 0.5 * two_pi * (r + 0.5 * a.drho) * a.dz / a.drho * dr;
        if (k + 1 < a.nz) kin += 0.5 * two_pi * r * a.drho / a.dz * E::abs2(E::sub(psi[q + 1], p)) * s2;
        acc[5] += kin;
    }
    for (int v = 0; v < 6; ++v) {
        const double t = ax_block_sum(acc[v]);
        if (threadIdx.x == 0) a.partials[blockIdx.x * 6 + v] = t;
    }
}

// out: [0] norm, [1] mu, [2] E, [3] rms_x = rms_y, [4] rms_z, [5] finite flag;
// with scale_out: the renormalisation factor 1 / sqrt(norm).
__global__ void axial_finish_kernel(const double *partials, int blocks, double g, double *out, double *scale_out) {
    __shared__ double tot[6];
    if (threadIdx.x < 6) {
        double t = 0.0;
        for (int b = 0; b < blocks; ++b) t += partials[b * 6 + threadIdx.x];
        tot[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double nrm = tot[0];
        out[0] = nrm;
        out[1] = (tot[5] + tot[1] + g * tot[2]) / nrm;
        out[2] = (tot[5] + tot[1] + 0.5 * g * tot[2]) / nrm;
        out[3] = sqrt(0.5 * tot[3] / nrm);
        out[4] = sqrt(tot[4] / nrm);
        bool fin = true;
        for (int q = 0; q < 5; ++q) fin = fin && isfinite(out[q]);
        out[5] = fin ? 1.0 : 0.0;
        if (scale_out) *scale_out = 1.0 / sqrt(nrm);
    }
}

template <typename R, bool CPLX>
__global__ void axial_gaussian_kernel(void *psi_v, int nx, int nz, double drho, double dz, double z0, double gamma,
                                      double lambda) {
    using E = AxElem<R, CPLX>;
    typename E::V *psi = static_cast<typename E::V *>(psi_v);
    const long long sites = (long long)nx * nz;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < sites;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / nz), k = (int)(q % nz);
        double v = 0.0;
        if (i >= 1 && i <= nx - 2 && k >= 1 && k <= nz - 2) {
            const double r = (i - 0.5) * drho, z = z0 + k * dz;
            v = exp(-0.5 * (gamma * r * r + lambda * z * z));
        }
        psi[q] = E::from_real(v);
    }
}

template <typename R, bool CPLX> __global__ void axial_scale_kernel(void *psi_v, long long sites, const double *scale) {
    using E = AxElem<R, CPLX>;
    typename E::V *psi = static_cast<typename E::V *>(psi_v);
    const R s = (R)*scale;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < sites;
         q += (long long)gridDim.x * blockDim.x)
        psi[q] = E::scale(psi[q], s);
}

enum AxScalar { AS_SCALE = 0, AS_ONE = 1, AS_ZNORM = 2, AS_ZSCALE = 3, AS_COUNT = 4 };

}  // namespace

struct gp_axial_s {
    int device = 0;
    int nx = 0, nz = 0;
    double drho = 0, dz = 0, dt = 0, gamma = 0, lambda = 0, g = 0;
    gp_precision prec = GP_F64;
    gp_field field = GP_COMPLEX;
    size_t elem = 0, sites = 0, bytes = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    cudaStream_t stream = nullptr;
    char *d_tab = nullptr;
    Tables T;                  // Cartesian tables of the (nx, 1, nz) grid: the z sweep's
    size_t rad_off[2][4] = {};  // [mode][A, C, cp, ip] byte offsets in d_tab
    double *d_scal = nullptr, *d_part = nullptr, *d_obs = nullptr;
    unsigned int *d_counter = nullptr;
    size_t part_cap = 0;
    bool scale_pending = false;
    long long step = 0;
    double t = 0.0;
    std::string err;
};

namespace {

gp_status afail(gp_axial a, gp_status st, const std::string &msg) {
    if (a) a->err = msg;
    else set_thread_error(msg.c_str());
    return st;
}

#define AX_CK(a, call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return afail((a), GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool f32_of(gp_axial a) { return a->prec == GP_F32; }
double z0_of(gp_axial a) { return -0.5 * (a->nz - 1) * a->dz; }
int modes_of(gp_axial a) { return a->field == GP_COMPLEX ? 2 : 1; }

Geometry geom_of(gp_axial a) {
    Geometry G;
    G.n[0] = a->nx;
    G.n[1] = 1;
    G.n[2] = a->nz;
    G.d[0] = a->drho;
    G.d[1] = 1.0;
    G.d[2] = a->dz;
    G.dt = a->dt;
    G.w[0] = a->gamma;
    G.w[1] = 0.0;
    G.w[2] = a->lambda;
    G.g = a->g;
    return G;
}

void put_cx(std::vector<char> &host, size_t off, std::complex<double> v, bool f32) {
    if (f32) {
        const float f[2] = {(float)v.real(), (float)v.imag()};
        std::memcpy(host.data() + off, f, sizeof(f));
    } else {
        const double d[2] = {v.real(), v.imag()};
        std::memcpy(host.data() + off, d, sizeof(d));
    }
}

// Radial tables of a mode (c = dt / (4 drho^2), times i in real time): per
// interior node t (radial node t + 1) A = c wl, C = c wr, and the Thomas
// coefficients of the matrix (-A, 1 + A + C, -C): ip = 1 / (1 + A + C +
// A cp[t-1]), cp = -C ip; all in FP64, stored in the field's precision.
void append_radial(gp_axial a, int mode, std::vector<char> &host) {
    const bool f32 = f32_of(a);
    const size_t csz = f32 ? 2 * sizeof(float) : 2 * sizeof(double);
    const int n = a->nx - 2;
    const std::complex<double> c = (mode == 1 ? std::complex<double>(0.0, 1.0) : 1.0) * (a->dt / (4.0 * a->drho * a->drho));
    size_t off = align_up(host.size(), 256);
    for (int q = 0; q < 4; ++q) {
        a->rad_off[mode][q] = off;
        off = align_up(off + csz * n, 256);
    }
    host.resize(off, 0);
    std::complex<double> cp_prev = 0.0;
    for (int t = 0; t < n; ++t) {
        const double r = (t + 0.5) * a->drho;  // radial node t + 1
        const double wl = (r - 0.5 * a->drho) / r, wr = (r + 0.5 * a->drho) / r;
        const std::complex<double> A = c * wl, C = c * wr;
        const std::complex<double> ip = 1.0 / (1.0 + A + C + A * cp_prev);  // sub-diagonal -A
        const std::complex<double> cpv = -C * ip;
        put_cx(host, a->rad_off[mode][0] + csz * t, A, f32);
        put_cx(host, a->rad_off[mode][1] + csz * t, C, f32);
        put_cx(host, a->rad_off[mode][2] + csz * t, cpv, f32);
        put_cx(host, a->rad_off[mode][3] + csz * t, ip, f32);
        cp_prev = cpv;
    }
}

template <typename R, bool CPLX> cudaError_t radial_launch(const AxArgs &args, cudaStream_t s) {
    axial_radial_kernel<R, CPLX><<<(args.nz + 127) / 128, 128, 0, s>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_radial(gp_axial a, const AxArgs &args) {
    if (f32_of(a)) return a->field == GP_COMPLEX ? radial_launch<float, true>(args, a->stream)
                                                 : radial_launch<float, false>(args, a->stream);
    return a->field == GP_COMPLEX ? radial_launch<double, true>(args, a->stream)
                                  : radial_launch<double, false>(args, a->stream);
}

template <typename R, bool CPLX> cudaError_t sums_launch(const AxSums &s, cudaStream_t st) {
    axial_sums_kernel<R, CPLX><<<kRedBlocks, kRedThreads, 0, st>>>(s);
    return cudaGetLastError();
}

// Cylindrical sums of the current psi (with the pending scale) -> out; with
// scale_out, also the renormalisation factor.
gp_status queue_sums(gp_axial a, double *out, double *scale_out) {
    AxSums s;
    s.psi = a->buf[a->cur];
    s.nx = a->nx;
    s.nz = a->nz;
    s.drho = a->drho;
    s.dz = a->dz;
    s.z0 = z0_of(a);
    s.gamma2 = a->gamma * a->gamma;
    s.lambda2 = a->lambda * a->lambda;
    s.scale = a->d_scal + (a->scale_pending ? AS_SCALE : AS_ONE);
    s.partials = a->d_part;
    cudaError_t e;
    if (f32_of(a)) e = a->field == GP_COMPLEX ? sums_launch<float, true>(s, a->stream) : sums_launch<float, false>(s, a->stream);
    else e = a->field == GP_COMPLEX ? sums_launch<double, true>(s, a->stream) : sums_launch<double, false>(s, a->stream);
    AX_CK(a, e);
    axial_finish_kernel<<<1, 32, 0, a->stream>>>(a->d_part, kRedBlocks, a->g, out, scale_out);
    AX_CK(a, cudaGetLastError());
    return GP_OK;
}

// The renormalisation factor of the current psi in the cylindrical measure
// (as a pending scale).
gp_status renormalise(gp_axial a) {
    a->scale_pending = false;  // sums of the stored values
    gp_status st = queue_sums(a, a->d_obs + 8, a->d_scal + AS_SCALE);
    if (st == GP_OK) a->scale_pending = true;
    return st;
}

gp_status run_step(gp_axial a, bool realtime) {
    const int mode = realtime ? 1 : 0;
    AxArgs r;
    r.in = a->buf[a->cur];
    r.out = a->buf[a->cur ^ 1];
    r.nx = a->nx;
    r.nz = a->nz;
    r.drho = a->drho;
    r.dz = a->dz;
    r.z0 = z0_of(a);
    r.dt = a->dt;
    r.g = a->g;
    r.gamma2 = a->gamma * a->gamma;
    r.lambda2 = a->lambda * a->lambda;
    r.A = a->d_tab + a->rad_off[mode][0];
    r.C = a->d_tab + a->rad_off[mode][1];
    r.cp = a->d_tab + a->rad_off[mode][2];
    r.ip = a->d_tab + a->rad_off[mode][3];
    r.scale = a->d_scal + (a->scale_pending ? AS_SCALE : AS_ONE);
    r.realtime = realtime ? 1 : 0;
    AX_CK(a, launch_radial(a, r));
    a->cur ^= 1;
    a->scale_pending = false;
    // z line solves through the Cartesian z-sweep kernels (their own norm
    // output goes to scratch: the cylindrical one follows)
    const Geometry G = geom_of(a);
    SweepLaunch L;
    L.prec = f32_of(a) ? P_F32 : P_F64;
    L.form = realtime ? F_REALTIME : (a->field == GP_REAL ? F_IMAG_REAL : F_IMAG_CPLX);
    L.kind = K_Z;
    L.window = default_window(a->T.ax[mode][2], f32_of(a));
    L.threads = 64;
    L.lpt = 1;
    L.contiguous = L.window > 0 ? 1 : 0;
    int seg_len = 0, n_seg = 0;
    choose_segments(G, 2, L.window, 1, (int)a->elem, true, 0, &seg_len, &n_seg);
    SweepArgs z = sweep_args(G, 2, realtime, a->buf[a->cur], a->buf[a->cur ^ 1], a->d_tab, a->T, seg_len, n_seg,
                             a->d_scal + AS_ONE, a->d_part, a->d_counter, a->d_scal + AS_ZNORM,
                             a->d_scal + AS_ZSCALE);
    const size_t zblocks = ((size_t)z.n_lines + 31) / 32 * (size_t)n_seg;
    if (zblocks > a->part_cap) return afail(a, GP_ERR_STATE, "z sweep grid exceeds the partials buffer");
    AX_CK(a, launch_sweep(L, z, a->stream));
    a->cur ^= 1;
    if (!realtime) return renormalise(a);
    return GP_OK;
}

void release(gp_axial a) {
    if (!a) return;
    for (void *p : {a->buf[0], a->buf[1], (void *)a->d_tab, (void *)a->d_scal, (void *)a->d_part,
                    (void *)a->d_obs, (void *)a->d_counter})
        if (p) cudaFree(p);
    delete a;
}

gp_status enter(gp_axial a) {
    if (!a) return afail(nullptr, GP_ERR_ARG, "NULL handle");
    if (cudaSetDevice(a->device) != cudaSuccess) {
        cudaGetLastError();
        return afail(a, GP_ERR_CUDA, "cudaSetDevice failed");
    }
    return GP_OK;
}

}  // namespace

extern "C" {

gp_status gp_axial_create(gp_axial *out, int nx, int nz, double drho, double dz, double dt, double gamma,
                          double lambda, double g, gp_precision prec, gp_field field, void *cuda_stream) {
    if (!out) return afail(nullptr, GP_ERR_ARG, "out is NULL");
    *out = nullptr;
    auto pos = [](double x) { return std::isfinite(x) && x > 0.0; };
    if (nx < 3 || nz < 3) return afail(nullptr, GP_ERR_ARG, "nx and nz need at least 3 nodes");
    if (!pos(drho) || !pos(dz) || !pos(dt) || !pos(gamma) || !pos(lambda) || !std::isfinite(g))
        return afail(nullptr, GP_ERR_ARG, "spacings, dt and trap frequencies must be finite and > 0, g finite");
    if ((long long)nx * nz > (1LL << 34)) return afail(nullptr, GP_ERR_ARG, "grid too large");
    if (prec != GP_F64 && prec != GP_F32) return afail(nullptr, GP_ERR_ARG, "precision must be GP_F64 or GP_F32");
    if (field != GP_COMPLEX && field != GP_REAL) return afail(nullptr, GP_ERR_ARG, "unknown field");
    gp_axial a = new (std::nothrow) gp_axial_s();
    if (!a) return afail(nullptr, GP_ERR_NOMEM, "host allocation failed");
    if (cudaGetDevice(&a->device) != cudaSuccess) {
        cudaGetLastError();
        delete a;
        return afail(nullptr, GP_ERR_CUDA, "no CUDA device");
    }
    a->nx = nx;
    a->nz = nz;
    a->drho = drho;
    a->dz = dz;
    a->dt = dt;
    a->gamma = gamma;
    a->lambda = lambda;
    a->g = g;
    a->prec = prec;
    a->field = field;
    a->stream = static_cast<cudaStream_t>(cuda_stream);
    a->elem = (prec == GP_F64 ? 8 : 4) * (field == GP_COMPLEX ? 2 : 1);
    a->sites = (size_t)nx * nz;
    a->bytes = a->sites * a->elem;
    std::vector<char> host;
    append_tables(geom_of(a), prec == GP_F32, modes_of(a), host, a->T);
    for (int mode = 0; mode < modes_of(a); ++mode) append_radial(a, mode, host);
    a->part_cap = std::max((size_t)kRedBlocks * 6, ((size_t)nx + 31) / 32 * (size_t)(nz > 2 ? nz - 2 : 1) + 64);
    if (dev_malloc(&a->buf[0], a->bytes) != cudaSuccess || dev_malloc(&a->buf[1], a->bytes) != cudaSuccess ||
        dev_malloc(&a->d_tab, host.size()) != cudaSuccess ||
        dev_malloc(&a->d_scal, AS_COUNT * sizeof(double)) != cudaSuccess ||
        dev_malloc(&a->d_part, a->part_cap * sizeof(double)) != cudaSuccess ||
        dev_malloc(&a->d_obs, 16 * sizeof(double)) != cudaSuccess ||
        dev_malloc(&a->d_counter, 2 * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        release(a);
        return afail(nullptr, GP_ERR_NOMEM, "cudaMalloc failed");
    }
    const double scal[AS_COUNT] = {1.0, 1.0, 0.0, 0.0};
    if (cudaMemcpy(a->d_tab, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(a->d_scal, scal, sizeof(scal), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(a->d_counter, 0, 2 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(a->buf[0], 0, a->bytes) != cudaSuccess) {
        cudaGetLastError();
        release(a);
        return afail(nullptr, GP_ERR_CUDA, "initial copies failed");
    }
    *out = a;
    return GP_OK;
}

void gp_axial_destroy(gp_axial a) { release(a); }

const char *gp_axial_last_error(gp_axial a) { return a ? a->err.c_str() : gp_last_error(nullptr); }

gp_status gp_axial_init_gaussian(gp_axial a) {
    gp_status st = enter(a);
    if (st != GP_OK) return st;
    const double z0 = z0_of(a);
    if (f32_of(a)) {
        if (a->field == GP_COMPLEX) axial_gaussian_kernel<float, true><<<256, 256, 0, a->stream>>>(a->buf[a->cur], a->nx, a->nz, a->drho, a->dz, z0, a->gamma, a->lambda);
        else axial_gaussian_kernel<float, false><<<256, 256, 0, a->stream>>>(a->buf[a->cur], a->nx, a->nz, a->drho, a->dz, z0, a->gamma, a->lambda);
    } else {
        if (a->field == GP_COMPLEX) axial_gaussian_kernel<double, true><<<256, 256, 0, a->stream>>>(a->buf[a->cur], a->nx, a->nz, a->drho, a->dz, z0, a->gamma, a->lambda);
        else axial_gaussian_kernel<double, false><<<256, 256, 0, a->stream>>>(a->buf[a->cur], a->nx, a->nz, a->drho, a->dz, z0, a->gamma, a->lambda);
    }
    AX_CK(a, cudaGetLastError());
    a->step = 0;
    a->t = 0.0;
    return renormalise(a);
}

gp_status gp_axial_set_psi(gp_axial a, const void *psi, int on_device) {
    gp_status st = enter(a);
    if (st != GP_OK) return st;
    if (!psi) return afail(a, GP_ERR_ARG, "psi is NULL");
    AX_CK(a, cudaMemcpyAsync(a->buf[a->cur], psi, a->bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             a->stream));
    AX_CK(a, cudaStreamSynchronize(a->stream));
    a->scale_pending = false;
    return GP_OK;
}

gp_status gp_axial_get_psi(gp_axial a, void *psi, int on_device) {
    gp_status st = enter(a);
    if (st != GP_OK) return st;
    if (!psi) return afail(a, GP_ERR_ARG, "psi is NULL");
    if (a->scale_pending) {  // fold the pending factor into psi
        const double *s = a->d_scal + AS_SCALE;
        if (f32_of(a)) {
            if (a->field == GP_COMPLEX) axial_scale_kernel<float, true><<<256, 256, 0, a->stream>>>(a->buf[a->cur], (long long)a->sites, s);
            else axial_scale_kernel<float, false><<<256, 256, 0, a->stream>>>(a->buf[a->cur], (long long)a->sites, s);
        } else {
            if (a->field == GP_COMPLEX) axial_scale_kernel<double, true><<<256, 256, 0, a->stream>>>(a->buf[a->cur], (long long)a->sites, s);
            else axial_scale_kernel<double, false><<<256, 256, 0, a->stream>>>(a->buf[a->cur], (long long)a->sites, s);
        }
        AX_CK(a, cudaGetLastError());
        a->scale_pending = false;
    }
    AX_CK(a, cudaMemcpyAsync(psi, a->buf[a->cur], a->bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             a->stream));
    AX_CK(a, cudaStreamSynchronize(a->stream));
    return GP_OK;
}

gp_status gp_axial_step_imag(gp_axial a, int nsteps) {
    gp_status st = enter(a);
    if (st != GP_OK) return st;
    if (nsteps < 0) return afail(a, GP_ERR_ARG, "nsteps must be >= 0");
    for (int s = 0; s < nsteps; ++s) {
        if ((st = run_step(a, false)) != GP_OK) return st;
        a->step += 1;
        a->t += a->dt;
    }
    return GP_OK;
}

gp_status gp_axial_step_real(gp_axial a, int nsteps) {
    gp_status st = enter(a);
    if (st != GP_OK) return st;
    if (nsteps < 0) return afail(a, GP_ERR_ARG, "nsteps must be >= 0");
    if (a->field != GP_COMPLEX) return afail(a, GP_ERR_STATE, "real time needs a GP_COMPLEX field");
    for (int s = 0; s < nsteps; ++s) {
        if ((st = run_step(a, true)) != GP_OK) return st;
        a->step += 1;
        a->t += a->dt;
    }
    return GP_OK;
}

gp_status gp_axial_observables(gp_axial a, gp_obs *out) {
    gp_status st = enter(a);
    if (st != GP_OK) return st;
    if ((st = queue_sums(a, a->d_obs, nullptr)) != GP_OK) return st;
    double o[6];
    AX_CK(a, cudaMemcpyAsync(o, a->d_obs, sizeof(o), cudaMemcpyDeviceToHost, a->stream));
    AX_CK(a, cudaStreamSynchronize(a->stream));
    if (out) {
        out->norm = o[0];
        out->mu = o[1];
        out->energy = o[2];
        out->rms_x = o[3];
        out->rms_y = o[3];
        out->rms_z = o[4];
        out->step = a->step;
        out->t = a->t;
    }
    if (o[5] != 1.0) return afail(a, GP_ERR_NONFINITE, "psi holds NaN or Inf");
    return GP_OK;
}

gp_status gp_axial_run_imag_until(gp_axial a, double mu_tol, int check_every, int max_steps, int *steps_taken) {
    if (steps_taken) *steps_taken = 0;
    gp_status st = enter(a);
    if (st != GP_OK) return st;
    if (!(mu_tol > 0.0) || check_every < 1 || max_steps < 0) return afail(a, GP_ERR_ARG, "bad stop rule arguments");
    gp_obs o;
    if ((st = gp_axial_observables(a, &o)) != GP_OK) return st;
    double mu_prev = o.mu;
    int taken = 0;
    while (taken < max_steps) {
        const int n = std::min(check_every, max_steps - taken);
        if ((st = gp_axial_step_imag(a, n)) != GP_OK) return st;
        taken += n;
        if ((st = gp_axial_observables(a, &o)) != GP_OK) return st;
        if (steps_taken) *steps_taken = taken;
        if (std::fabs(o.mu - mu_prev) < mu_tol) return GP_OK;
        mu_prev = o.mu;
    }
    return GP_OK;
}

}  // extern "C"

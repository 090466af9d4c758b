// gp_host.cu -- host-side helpers shared by the handle types (see gp_host.h).
#include "gp_host.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>

namespace gpcn {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

namespace {

// FP64 Thomas coefficients of the CN matrix (-c, 1+2c, -c) on n interior
// nodes: den[0] = 1+2c, den[t] = 1+2c + c cp[t-1], ip = 1/den, cp = -c ip.
// The inverse pivot is returned as its deviation from one,
// ipm1 = ip - 1 = (1 - den) / den, which the kernels apply as u + u ipm1.
void thomas_coefficients(std::complex<double> c, int n, std::vector<std::complex<double>> &cp,
                         std::vector<std::complex<double>> &ipm1) {
    cp.assign(n, 0.0);
    ipm1.assign(n, 0.0);
    for (int t = 0; t < n; ++t) {
        const std::complex<double> excess = 2.0 * c + (t == 0 ? 0.0 : c * cp[t - 1]);  // den - 1
        const std::complex<double> den = 1.0 + excess;
        ipm1[t] = -excess / den;
        cp[t] = -c / den;
    }
}

void put_real(char *dst, double v, bool f32) {
    if (f32) {
        const float f = (float)v;
        std::memcpy(dst, &f, sizeof(f));
    } else {
        std::memcpy(dst, &v, sizeof(v));
    }
}

}  // namespace

void append_tables(const Geometry &G, bool f32, int modes, std::vector<char> &host, Tables &T) {
    const size_t rsz = f32 ? sizeof(float) : sizeof(double);
    const double eps = f32 ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
    size_t off = align_up(host.size(), 256);
    for (int mode = 0; mode < modes; ++mode) {
        for (int ax = 0; ax < 3; ++ax) {
            const size_t esz = (mode == 1 ? 2 : 1) * rsz;
            const size_t nint = G.n[ax] > 2 ? (size_t)(G.n[ax] - 2) : 0;  // an absent axis has none
            AxisTables &at = T.ax[mode][ax];
            at.off_cp = off;
            off = align_up(off + esz * nint, 256);
            at.off_ip = off;
            off = align_up(off + esz * nint, 256);
        }
    }
    for (int ax = 0; ax < 3; ++ax) {
        T.kick_off[ax] = off;
        off = align_up(off + rsz * G.n[ax], 256);
        T.phase_off[ax] = off;
        off = align_up(off + rsz * G.n[ax], 256);
        T.phase_half_off[ax] = off;
        off = align_up(off + rsz * G.n[ax], 256);
    }
    host.resize(off, 0);
    // exp(-dt w^2 a^2 / 2) - 1 per node of each axis: the trap part of the
    // imaginary-time kick factorises over the axes (stored as deviations
    // from one, which keeps their rounding from acting as a potential error
    // of u / dt); its phase dt w^2 a^2 / 2 is the trap part of the real-time
    // kick's angle, a sum over the axes.
    for (int ax = 0; ax < 3; ++ax)
        for (int i = 0; i < G.n[ax]; ++i) {
            const double a = (i - 0.5 * (G.n[ax] - 1)) * G.d[ax];
            const double dv = G.dt * 0.5 * G.w[ax] * G.w[ax] * a * a;
            put_real(host.data() + T.kick_off[ax] + i * rsz, std::expm1(-dv), f32);
            put_real(host.data() + T.phase_off[ax] + i * rsz, dv, f32);
            put_real(host.data() + T.phase_half_off[ax] + i * rsz, 0.5 * dv, f32);
        }
    for (int mode = 0; mode < modes; ++mode) {
        for (int ax = 0; ax < 3; ++ax) {
            const int n = G.n[ax] - 2;
            if (n < 1) continue;  // an absent axis (one node) has no line solve
            const double kap = G.dt / (4.0 * G.d[ax] * G.d[ax]);
            const std::complex<double> c = mode == 1 ? std::complex<double>(0.0, kap)
                                                     : std::complex<double>(kap, 0.0);
            std::vector<std::complex<double>> cp, ip;
            thomas_coefficients(c, n, cp, ip);
            AxisTables &at = T.ax[mode][ax];
            at.cp_max = 0.0;
            for (int t = 0; t < n - 1; ++t) at.cp_max = std::max(at.cp_max, std::abs(cp[t]));
            // the smallest window whose truncation, at most cp_max^(W+1) of the
            // line's largest value, stays within half the unit roundoff (below
            // the rounding of a single operation)
            at.min_window = 0;
            for (int w : {4, 8, 16}) {
                if (std::pow(at.cp_max, w + 1) <= eps / 2.0) {
                    at.min_window = w;
                    break;
                }
            }
            for (int t = 0; t < n; ++t) {
                for (int which = 0; which < 2; ++which) {
                    const std::complex<double> v = which == 0 ? cp[t] : ip[t];
                    char *dst = host.data() + (which == 0 ? at.off_cp : at.off_ip);
                    if (mode == 1) {
                        put_real(dst + t * 2 * rsz, v.real(), f32);
                        put_real(dst + t * 2 * rsz + rsz, v.imag(), f32);
                    } else {
                        put_real(dst + t * rsz, v.real(), f32);
                    }
                }
            }
            // the stored entries settle to the line's last ones (bit for bit)
            // a few nodes in; kernels read them once from there on
            const size_t esz = (mode == 1 ? 2 : 1) * rsz;
            const char *tc = host.data() + at.off_cp, *ti = host.data() + at.off_ip;
            at.t_const = n;
            while (at.t_const > 0 && std::memcmp(tc + (at.t_const - 1) * esz, tc + (n - 1) * esz, esz) == 0 &&
                   std::memcmp(ti + (at.t_const - 1) * esz, ti + (n - 1) * esz, esz) == 0)
                --at.t_const;
        }
    }
}

int default_window(const AxisTables &t, bool f32) {
    // FP64 on this part runs at a small fraction of its FP32 rate, so the FP64
    // forms are ALU-bound: the exact two-pass solve (fewer flops, twice the
    // bytes) is faster there.  FP32 is bandwidth-bound and takes the
    // windowed single-pass solve.
    return f32 ? t.min_window : 0;
}

long long axis_lines(const Geometry &G, int ax) {
    const long long nx = G.n[0], ny = G.n[1], nz = G.n[2];
    return ax == 0 ? ny * nz : ax == 1 ? nx * nz : nx * ny;
}

void choose_segments(const Geometry &G, int ax, int window, int lpt, int elem_bytes, bool contiguous_z,
                     int override_len, int *seg_len, int *n_seg) {
    const int n = G.n[ax] - 2;
    if (n < 1) {  // an absent axis (one node) has no line solve
        *seg_len = *n_seg = 0;
        return;
    }
    const int chunk = (elem_bytes * lpt >= 16) ? 8 : 16;
    int len = n;
    if (window > 0) {
        if (override_len > 0) {
            len = std::min(n, override_len);
        } else if (ax == 2 && contiguous_z) {
            len = n;  // warp-tiled stride-1 axis: whole lines (measured best)
        } else {
            // about 128 nodes per segment (measured best on the strided axes),
            // rounded to whole chunks
            const int want = std::max(1, (n + 127) / 128);
            len = (n + want - 1) / want;
            len = (len + chunk - 1) / chunk * chunk;
            len = std::min(len, n);
        }
    }
    *seg_len = std::max(1, len);
    *n_seg = (n + *seg_len - 1) / *seg_len;
}

SweepArgs sweep_args(const Geometry &G, int ax, bool realtime, const void *in, void *out,
                     const char *tables, const Tables &T, int seg_len, int n_seg, const double *scale,
                     double *partials, unsigned int *counter, double *norm_out, double *scale_out,
                     bool half_kick) {
    SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    const long long ny = G.n[1], nz = G.n[2];
    const int mode = realtime ? 1 : 0;
    a.psi = in;
    a.psi_out = out;
    a.cp = tables + T.ax[mode][ax].off_cp;
    a.ip = tables + T.ax[mode][ax].off_ip;
    a.n_lines = axis_lines(G, ax);
    if (ax == 0) {
        a.inner = ny * nz;
        a.outer_stride = 0;
        a.stride = ny * nz;
    } else if (ax == 1) {
        a.inner = nz;
        a.outer_stride = ny * nz;
        a.stride = nz;
    } else {
        a.inner = 1;
        a.outer_stride = nz;
        a.stride = 1;
    }
    a.N = G.n[ax];
    a.t_const = T.ax[mode][ax].t_const;
    a.seg_len = seg_len;
    a.n_seg = n_seg;
    a.kappa = G.dt / (4.0 * G.d[ax] * G.d[ax]);
    a.scale = scale;
    if (!realtime) {
        a.kick_ex = tables + T.kick_off[0];
        a.kick_ey = tables + T.kick_off[1];
        a.kick_ez = tables + T.kick_off[2];
    } else {
        const size_t *ph = half_kick ? T.phase_half_off : T.phase_off;
        a.phase_ex = tables + ph[0];
        a.phase_ey = tables + ph[1];
        a.phase_ez = tables + ph[2];
    }
    a.dt = (realtime && half_kick) ? 0.5 * G.dt : G.dt;  // the kick's step (dt g |psi|^2)
    a.g = G.g;
    for (int q = 0; q < 3; ++q) {
        a.half_w2[q] = 0.5 * G.w[q] * G.w[q];
        a.origin[q] = -0.5 * (G.n[q] - 1) * G.d[q];
        a.d[q] = G.d[q];
    }
    a.nz = (int)nz;
    a.ny = (int)ny;
    a.partials = partials;
    a.counter = counter;
    a.norm_out = norm_out;
    a.scale_out = scale_out;
    a.dV = G.d[0] * G.d[1] * G.d[2];
    a.want_scale = realtime ? 0 : 1;
    return a;
}

FieldArgs field_args(const Geometry &G, const void *psi, const double *scale, double *partials,
                     unsigned int *counter, double *out, double *scale_out, double *norm_out) {
    FieldArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = const_cast<void *>(psi);
    for (int ax = 0; ax < 3; ++ax) {
        a.n[ax] = G.n[ax];
        a.d[ax] = G.d[ax];
        a.origin[ax] = -0.5 * (G.n[ax] - 1) * G.d[ax];
        a.w[ax] = G.w[ax];
        a.half_w2[ax] = 0.5 * G.w[ax] * G.w[ax];
    }
    a.g = G.g;
    a.scale = scale;
    a.dV = G.d[0] * G.d[1] * G.d[2];
    a.partials = partials;
    a.counter = counter;
    a.out = out;
    a.scale_out = scale_out;
    a.norm_out = norm_out;
    a.sites = (long long)G.n[0] * G.n[1] * G.n[2];
    return a;
}

// ------------------------------------------------------------------ allocation hook
namespace {
std::atomic<int> g_fail_alloc{0};  // > 0: the g_fail_alloc-th next allocation fails
}

cudaError_t dev_malloc_bytes(void **p, size_t bytes) {
    int n = g_fail_alloc.load();
    while (n > 0) {
        if (g_fail_alloc.compare_exchange_weak(n, n - 1)) {
            if (n == 1) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

void set_fail_alloc(int n) { g_fail_alloc.store(n > 0 ? n : 0); }

// ------------------------------------------------------------------ TMA maps
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}
}  // namespace

// Boxes of 64 bytes of a row x 64 rows, 64-byte swizzle, zero fill outside
// the array (the layout gp_sweep_tma.cuh reads and writes).  Each box row
// promotes a 256-byte L2 fetch: the next three boxes of the row then come
// from L2 (measured 2-3 % faster than 128-byte promotion on the z sweep).
bool encode_z_map(CUtensorMap *map, const void *base, int N, long long n_lines, int elem_bytes) {
    if (elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8) return false;
    if (((long long)N * elem_bytes) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
    if (n_lines <= 0 || n_lines > 0x7fffffffLL || N <= 0) return false;
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)n_lines};
    const cuuint64_t strides[1] = {(cuuint64_t)N * (cuuint64_t)elem_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)(64 / elem_bytes), 64u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUtensorMapDataType dt = elem_bytes == 8   ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                   : elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                     : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    return enc(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool line_tma_fits(int elem_bytes, int lpt, int window, long long inner, long long stride, int N) {
    const int mv = elem_bytes * lpt;
    if (window <= 0 || N < 3 || (mv != 4 && mv != 8 && mv != 16)) return false;
    if (inner % lpt != 0 || inner * elem_bytes / 4 > 0xffffffffLL) return false;
    return (stride * elem_bytes) % 16 == 0;
}

// Words of 4 bytes: d0 = the elements of one node of an outer group, d1 =
// the n interior nodes (origin at node 1), d2 = the outer groups (1 for x,
// nx planes for y).  No swizzle: box row q (node) is 32 MemV contiguous in
// shared memory.  Zero fill outside the array.
bool encode_line_map(CUtensorMap *map, const void *psi, int axis, const int n[3], int elem_bytes, int lpt,
                     int box_nodes) {
    if (axis != 0 && axis != 1) return false;
    const long long plane = (long long)n[1] * n[2];
    const long long inner = axis == 0 ? plane : n[2];
    const long long stride = axis == 0 ? plane : n[2];
    const int N = n[axis];
    if (!line_tma_fits(elem_bytes, lpt, 1, inner, stride, N)) return false;
    const long long s1 = stride * elem_bytes;  // bytes between nodes of a line
    const long long s2 = axis == 0 ? s1 * n[0] : plane * elem_bytes;
    const unsigned char *node1 = static_cast<const unsigned char *>(psi) + s1;
    if ((reinterpret_cast<uintptr_t>(node1) & 15u) != 0 || s2 % 16 != 0) return false;
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)(inner * elem_bytes / 4), (cuuint64_t)(N - 2),
                                (cuuint64_t)(axis == 0 ? 1 : n[0])};
    const cuuint64_t strides[2] = {(cuuint64_t)s1, (cuuint64_t)s2};
    const cuuint32_t box[3] = {(cuuint32_t)(32 * lpt * elem_bytes / 4), (cuuint32_t)box_nodes, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<unsigned char *>(node1), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace gpcn

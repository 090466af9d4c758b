// gp_internal.h -- launch descriptors shared by the runtime (gp_api.cu) and
// the kernel translation units.  Host-visible plain structs only.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace gpcn {

enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2 };  // P_F16: FP16 storage, FP32 arithmetic (real fields, imaginary time)

// The three arithmetic forms of a sweep:
//  IMAG_REAL  imaginary time on a real field   (c real, coefficients real)
//  IMAG_CPLX  imaginary time on a complex field (c real, coefficients real)
//  REALTIME   real time on a complex field     (c = i kappa, coefficients complex)
enum Form { F_IMAG_REAL = 0, F_IMAG_CPLX = 1, F_REALTIME = 2 };

// Which sweep of the step: X carries the fused kick, Z the fused norm.
enum Kind { K_X = 0, K_Y = 1, K_Z = 2 };

// Arguments of one line-solve launch (all lines of one axis).
struct SweepArgs {
    const void *psi;       // input element array, layout z-fastest
    void *psi_out;         // output array (a different buffer: sweeps are out of place)
    const void *cp;        // Thomas multipliers cp[t], t = 0..N-3 (real or complex)
    const void *ip;        // inverse pivots ip[t]
    long long n_lines;     // lines of this axis
    long long inner;       // line L starts at (L / inner) * outer_stride + (L % inner)
    long long outer_stride;
    long long stride;      // element stride along the line
    int N;                 // nodes along the line (interior N - 2)
    int seg_len;           // interior nodes per segment (a multiple of the chunk length)
    int n_seg;             // segments per line (grid.y); one thread per (line, segment)
    int t_const;           // cp[t], ip[t] equal cp[N-3], ip[N-3] (stored bits) for t >= t_const
    double kappa;          // |c| = dt / (4 d^2)
    // kick (K_X): site (i, j, k) with i along the line, (j, k) = (L / nz, L % nz)
    const double *scale;   // pending renormalisation factor applied on load
    const void *kick_ex;   // imaginary time: exp(-dt V_x(i)) - 1 per x node (else null)
    const void *kick_ey;   //                 exp(-dt V_y(j)) - 1 per y node
    const void *kick_ez;   //                 exp(-dt V_z(k)) - 1 per z node
    const void *phase_ex;  // real time: dt V_x(i) per x node (else null)
    const void *phase_ey;  //            dt V_y(j) per y node
    const void *phase_ez;  //            dt V_z(k) per z node
    double dt, g;
    double half_w2[3];     // (gamma^2, nu^2, lambda^2) / 2
    double origin[3];      // coordinate of node 0 per axis
    double d[3];           // spacings
    int nz, ny;
    // norm (K_Z): block partials, last-block-done counter, outputs
    double *partials;
    unsigned int *counter;
    double *norm_out;      // dV * sum |psi|^2 of the result
    double *scale_out;     // 1 / sqrt(norm) when want_scale
    double dV;
    int want_scale;
    unsigned int *status;  // 1 is or-ed in by a sweep kernel whose bounded wait expired (may be null)
};

// Tensor maps of the z sweep's input and output arrays, each a 2D array of
// n_lines rows of N elements (see gp_sweep_tma.cuh).
struct TmaMaps {
    CUtensorMap in, out;
};

// Whether the TMA z sweep serves a line of N nodes of elem_bytes (4 or 8)
// at window W cut into n_seg segments: whole lines (one segment), rows that
// start on 16-byte boundaries, a register ring of (chunk + W) pair values
// within 256 bytes (chunk = 64 bytes of nodes), and at least one chunk plus
// the window plus two interior nodes.
inline bool tma_z_fits(int elem_bytes, int W, int N, int n_seg, long long n_lines) {
    if (elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8) return false;
    const int chunk = 64 / elem_bytes;
    return W > 0 && (chunk + W) * 2 * elem_bytes <= 256 && n_seg == 1 && N - 2 >= chunk + W + 2 &&
           ((long long)N * elem_bytes) % 16 == 0 && n_lines > 0 && n_lines <= 0x7fffffffLL;
}

// Tensor maps of a batched TMA z sweep: instance q of the launch (its
// position in the launch's argument array) reads rows through in[q] and
// writes them through out[q].  Passed by value as one kernel parameter
// block (16 KB at 64 instances, within the 32 KB parameter limit).
constexpr int kTmaBatch = 64;
constexpr int kTmaBlockRows = 256;  // z lines per block of the TMA z sweep
struct BatchTmaMaps {
    CUtensorMap in[kTmaBatch], out[kTmaBatch];
};

struct SweepLaunch {
    Prec prec;
    Form form;
    Kind kind;
    int window;            // 4, 8, 16, or 0 for the exact two-pass solve
    int threads;           // threads per block
    int lpt;               // lines per thread of the strided kernel (1, or 2 or 4 adjacent lines)
    int contiguous;        // 1: warp-tiled kernel for the stride-1 axis
    const TmaMaps *tma = nullptr;  // z sweep through TMA tiles where the grid allows it
    const TmaMaps *lmaps = nullptr;  // x or y sweep through TMA boxes (encode_line_map; windowed)
};

cudaError_t launch_sweep(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s);
// Highest window the templates provide.
constexpr int kMaxWindow = 16;

// Gaussian initial state (unnormalised) plus its norm partials.
struct FieldArgs {
    void *psi;
    int n[3];
    double d[3];
    double origin[3];
    double w[3];           // trap frequencies
    double half_w2[3];
    double g;
    const double *scale;   // factor applied to psi on read
    double dV;
    double *partials;
    unsigned int *counter;
    double *out;           // observables: 9 raw sums + 6 derived values
    double *scale_out;
    double *norm_out;
    long long sites;
    unsigned int *status;  // 2 is or-ed in by an observables kernel whose bounded wait expired (may be null)
};

cudaError_t launch_gaussian(Prec p, bool cplx, const FieldArgs &a, cudaStream_t s);
cudaError_t launch_norm(Prec p, bool cplx, const FieldArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_observables(Prec p, bool cplx, const FieldArgs &a, cudaStream_t s);
// Look up, once per device, the launch shapes the field kernels take from
// the device (call from the current device, outside any stream capture).
void prepare_field_launches();
cudaError_t launch_apply_scale(Prec p, bool cplx, const FieldArgs &a, void *dst, cudaStream_t s);
// Real-time kick exp(-i kdt (V + g |psi|^2)) of a complex field into dst.
cudaError_t launch_kick(Prec p, const FieldArgs &a, double kdt, void *dst, cudaStream_t s);

// Observables output layout in FieldArgs::out.
enum ObsSlot {
    O_RHO = 0, O_V, O_RHO2, O_X2, O_Y2, O_Z2, O_LX, O_LY, O_LZ,   // raw sums
    O_NORM = 9, O_MU, O_E, O_RMSX, O_RMSY, O_RMSZ, O_FINITE,      // derived
    O_COUNT = 16
};

// The most blocks (partials) any observables launch over this field uses.
int observables_blocks(const FieldArgs &a);
// Blocks of the per-(j, k) observables kernels over one condensate (also one
// condensate's share of the batched observables launch).
int observables_body_blocks(const FieldArgs &a);
cudaError_t launch_observables_batch(Prec p, bool cplx, const FieldArgs *args, const unsigned *first, int n,
                                     unsigned total_blocks, cudaStream_t s);

// Batched sweep launch: instance i owns blocks [first[i], first[i+1]) of a
// 1D grid of total_blocks, laid out as its own grid (gridx[i] blocks along x,
// then the segment).  args, first, gridx are device arrays.
struct BatchLaunch {
    const SweepArgs *args;
    const unsigned *first;
    const unsigned *gridx;
    int n;
    unsigned total_blocks;
    const BatchTmaMaps *tma = nullptr;  // z sweep through TMA (n <= kTmaBatch instances that fit)
};
cudaError_t launch_sweep_batch(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s);
// Threads per block of the batched kernels.
constexpr int kBatchLineThreads = 64;
void set_thread_error(const char *msg);
// Every device allocation of the library goes through dev_malloc, so that
// tests can make the n-th next one fail (gp_debug_fail_alloc).
cudaError_t dev_malloc_bytes(void **p, size_t bytes);
template <typename T> inline cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc_bytes(reinterpret_cast<void **>(p), bytes);
}
void set_fail_alloc(int n);
// Encode the tensor map of an array of n_lines rows of N elements of
// elem_bytes (4 or 8) for the TMA z sweep; false if the layout does not allow
// one (row pitch or base not 16-byte aligned) or the CUDA driver offers no encoder.
bool encode_z_map(CUtensorMap *map, const void *base, int N, long long n_lines, int elem_bytes);
// Whether the x or y sweep (stride `stride` elements along the line, `inner`
// lines per outer group) of elem_bytes elements, lpt lines per thread, can
// take the strided TMA form: a windowed solve, a line stride of whole
// 16-byte units, and MemV of 4, 8 or 16 bytes.
bool line_tma_fits(int elem_bytes, int lpt, int window, long long inner, long long stride, int N);
// Encode the tensor map of the strided TMA form over the array at `psi`
// for axis 0 (x) or 1 (y) of an (nx, ny, nz) grid, boxes of 32 * lpt
// elements x `box_nodes` nodes; false if the layout does not allow one.
bool encode_line_map(CUtensorMap *map, const void *psi, int axis, const int n[3], int elem_bytes, int lpt,
                     int box_nodes);
constexpr int kReduceThreads = 256;

}  // namespace gpcn

// gp_api.cu -- the C ABI of libgpcn (include/gp.h): handle lifetime, host-side
// argument checks, the FP64 precomputation of the CN recursion coefficients,
// and the per-step launch sequence (kick + x sweep, y sweep, z sweep + norm).
#include "gp.h"
#include "gp_host.h"
#include "gp_internal.h"
#include "gp_nn_internal.h"
#include "gp_output.h"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <tuple>
#include <new>
#include <string>
#include <vector>

namespace gpcn {
cudaError_t launch_sweep_f32_ir(const SweepLaunch &, const SweepArgs &, cudaStream_t);
cudaError_t launch_sweep_f32_ic(const SweepLaunch &, const SweepArgs &, cudaStream_t);
cudaError_t launch_sweep_f32_rt(const SweepLaunch &, const SweepArgs &, cudaStream_t);
cudaError_t launch_sweep_f64_ir(const SweepLaunch &, const SweepArgs &, cudaStream_t);
cudaError_t launch_sweep_f64_ic(const SweepLaunch &, const SweepArgs &, cudaStream_t);
cudaError_t launch_sweep_f64_rt(const SweepLaunch &, const SweepArgs &, cudaStream_t);
cudaError_t launch_sweep_f16_ir(const SweepLaunch &, const SweepArgs &, cudaStream_t);

cudaError_t launch_sweep_f32_ir_batch(const SweepLaunch &, const BatchLaunch &, cudaStream_t);
cudaError_t launch_sweep_f32_ic_batch(const SweepLaunch &, const BatchLaunch &, cudaStream_t);
cudaError_t launch_sweep_f32_rt_batch(const SweepLaunch &, const BatchLaunch &, cudaStream_t);
cudaError_t launch_sweep_f64_ir_batch(const SweepLaunch &, const BatchLaunch &, cudaStream_t);
cudaError_t launch_sweep_f64_ic_batch(const SweepLaunch &, const BatchLaunch &, cudaStream_t);
cudaError_t launch_sweep_f64_rt_batch(const SweepLaunch &, const BatchLaunch &, cudaStream_t);

cudaError_t launch_sweep_batch(const SweepLaunch &L, const BatchLaunch &b, cudaStream_t s) {
    if (L.prec == P_F32) {
        switch (L.form) {
        case F_IMAG_REAL: return launch_sweep_f32_ir_batch(L, b, s);
        case F_IMAG_CPLX: return launch_sweep_f32_ic_batch(L, b, s);
        case F_REALTIME: return launch_sweep_f32_rt_batch(L, b, s);
        }
    } else {
        switch (L.form) {
        case F_IMAG_REAL: return launch_sweep_f64_ir_batch(L, b, s);
        case F_IMAG_CPLX: return launch_sweep_f64_ic_batch(L, b, s);
        case F_REALTIME: return launch_sweep_f64_rt_batch(L, b, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep(const SweepLaunch &L, const SweepArgs &a, cudaStream_t s) {
    if (L.prec == P_F16) return L.form == F_IMAG_REAL ? launch_sweep_f16_ir(L, a, s) : cudaErrorInvalidValue;
    if (L.prec == P_F32) {
        switch (L.form) {
        case F_IMAG_REAL: return launch_sweep_f32_ir(L, a, s);
        case F_IMAG_CPLX: return launch_sweep_f32_ic(L, a, s);
        case F_REALTIME: return launch_sweep_f32_rt(L, a, s);
        }
    } else {
        switch (L.form) {
        case F_IMAG_REAL: return launch_sweep_f64_ir(L, a, s);
        case F_IMAG_CPLX: return launch_sweep_f64_ic(L, a, s);
        case F_REALTIME: return launch_sweep_f64_rt(L, a, s);
        }
    }
    return cudaErrorInvalidValue;
}
}  // namespace gpcn

using namespace gpcn;

namespace {

thread_local std::string g_create_error;

}  // namespace

// Error message of a failed call that has no handle (read by gp_last_error(NULL)).
void gpcn::set_thread_error(const char *msg) { g_create_error = msg ? msg : ""; }

namespace {

// Device scalars of a handle.
enum Scalar { S_SCALE = 0, S_ONE = 1, S_NORM_SWEEP = 2, S_NORM_INIT = 3, S_SAVE = 4, S_COUNT = 8 };

}  // namespace

struct gp_handle_s {
    int device = 0;
    int n[3] = {0, 0, 0};
    double d[3] = {0, 0, 0};
    double dt = 0, w[3] = {0, 0, 0}, g = 0;
    gp_precision prec = GP_F64;
    gp_field field = GP_COMPLEX;
    size_t elem = 0, sites = 0, bytes = 0;
    void *buf[2] = {nullptr, nullptr};  // ping-pong psi buffers (sweeps are out of place)
    int cur = 0;                        // buf[cur] holds the current psi
    bool own_buf0 = false;
    cudaStream_t stream = nullptr;
    char *d_coef = nullptr;
    size_t coef_bytes = 0;
    Tables tab;                         // offsets of the coefficient tables in d_coef
    int window[2][3] = {{0, 0, 0}, {0, 0, 0}};  // window in use per mode and axis
    int forced_window = -1;
    double *d_scal = nullptr;
    double *d_obs = nullptr;
    double *d_partials = nullptr;
    size_t partial_cap = 0;
    unsigned int *d_counter = nullptr;
    bool scale_pending = false;
    long long step = 0;
    double t = 0;
    int threads[3] = {64, 64, 64};
    bool contiguous_z = true;  // warp-tiled kernel for the stride-1 axis
    bool tma_z = true;         // ... through TMA tiles where the grid allows it
    int tma_lines = -1;        // axes (bit 0: x, bit 1: y) whose sweeps read through TMA boxes where the grid
                               // allows it; -1: x in imaginary time (measured faster), none in real time
    int stop_rule = 0;         // gp_run_imag_until: 0 |dmu| < tol; 1 |dmu| < tol and |dE| < tol; 2 rule 1 twice in a row
    int splitting = 1;         // real time: 1 Lie (kick, sweeps), 2 symmetric (half kick, sweeps, half kick)
    bool kick_pending = false; // symmetric splitting: buf[cur] still lacks its trailing half kick
    bool zmap_ok = false;      // zmap[b]: tensor map of buf[b] as n_lines rows of nz elements
    CUtensorMap zmap[2];
    unsigned int *d_status = nullptr;  // nonzero after a kernel's bounded wait expired
    bool psi_lost = false;             // an expired wait was reported: psi is undefined until set again
    int max_lpt[2] = {4, 4};   // most adjacent lines per thread on the x and y sweeps (1, 2 or 4)
    int seg_override[3] = {0, 0, 0};  // interior nodes per segment, 0 = automatic
    // observables history queued during stepping
    int track_every = 0, track_cap = 0, track_count = 0;
    double *d_track = nullptr;
    std::vector<long long> track_step;
    std::vector<double> track_t;
    // CUDA graphs of blocks of steps, replayed on the handle's stream
    int graph_block = 16;              // steps per graph (0: launch kernel by kernel)
    cudaStream_t cap_stream = nullptr; // private stream used only for capture
    struct Graph {
        cudaGraphExec_t exec;
        int cur;                // the state the block leaves behind
        bool scale_pending, kick_pending;
    };
    std::map<std::tuple<int, int, int, int, int, int>, Graph> graphs;
    double *d_obs_graph = nullptr;     // tracking record written inside a graph
    std::string err;
};

namespace {

gp_status fail(gp_handle h, gp_status st, const std::string &msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return st;
}

#define GP_CK(h, call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail((h), GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

gp_status check_args(gp_grid grid, double dt, double gamma, double nu, double lambda, double g,
                     gp_precision prec, gp_field field) {
    const int n[3] = {grid.nx, grid.ny, grid.nz};
    const double d[3] = {grid.dx, grid.dy, grid.dz};
    for (int a = 0; a < 3; ++a) {
        // a y or z axis of one node is absent (1D and 2D condensates)
        if (n[a] < 3 && !(a > 0 && n[a] == 1))
            return fail(nullptr, GP_ERR_ARG, "nx needs at least 3 nodes, ny and nz at least 3 or exactly 1");
        if (!finite_pos(d[a])) return fail(nullptr, GP_ERR_ARG, "spacings must be finite and > 0");
    }
    if ((long long)n[0] * n[1] * n[2] > (1LL << 40))
        return fail(nullptr, GP_ERR_ARG, "grid too large");
    if (!finite_pos(dt)) return fail(nullptr, GP_ERR_ARG, "dt must be finite and > 0");
    const double w[3] = {gamma, nu, lambda};
    for (double x : w)
        if (!std::isfinite(x) || x < 0.0)
            return fail(nullptr, GP_ERR_ARG, "trap frequencies must be finite and >= 0");
    if (!std::isfinite(g)) return fail(nullptr, GP_ERR_ARG, "g must be finite");
    if (prec != GP_F64 && prec != GP_F32 && prec != GP_F16) return fail(nullptr, GP_ERR_ARG, "unknown precision");
    if (field != GP_COMPLEX && field != GP_REAL) return fail(nullptr, GP_ERR_ARG, "unknown field");
    if (prec == GP_F16) {
        // FP16 storage: real fields (imaginary time), the TMA z sweep on whole
        // rows of 16-byte units with room for a chunk of 32 nodes and the widest
        // window, and line pairs on x and y
        if (field != GP_REAL) return fail(nullptr, GP_ERR_ARG, "FP16 storage is for real fields (imaginary time) only");
        if (n[2] % 8 != 0 || n[2] < 56) return fail(nullptr, GP_ERR_ARG, "FP16 storage needs nz a multiple of 8, at least 56");
    }
    return GP_OK;
}

int modes_of(gp_handle h) { return h->field == GP_COMPLEX ? 2 : 1; }

Prec prec_of(gp_handle h) { return h->prec == GP_F64 ? P_F64 : (h->prec == GP_F32 ? P_F32 : P_F16); }
bool fp16(gp_handle h) { return h->prec == GP_F16; }

Geometry geom(gp_handle h) {
    Geometry G;
    for (int q = 0; q < 3; ++q) {
        G.n[q] = h->n[q];
        G.d[q] = h->d[q];
        G.w[q] = h->w[q];
    }
    G.dt = h->dt;
    G.g = h->g;
    return G;
}

// Build and upload the coefficient tables of both modes and all axes, and
// pick the window of the windowed backward sweep for each.
gp_status build_coefficients(gp_handle h) {
    const bool f32 = h->prec != GP_F64;  // FP32 tables for FP32 arithmetic (FP32 and FP16 storage)
    std::vector<char> host;
    append_tables(geom(h), f32, modes_of(h), host, h->tab);
    const size_t off = host.size();
    for (int mode = 0; mode < modes_of(h); ++mode)
        for (int ax = 0; ax < 3; ++ax) {
            const AxisTables &at = h->tab.ax[mode][ax];
            int w = default_window(at, f32);
            if (h->forced_window == 0 ||
                (h->forced_window > 0 && at.min_window > 0 && h->forced_window >= at.min_window))
                w = h->forced_window;
            h->window[mode][ax] = w;
        }
    if (h->d_coef && h->coef_bytes < off) {
        cudaFree(h->d_coef);
        h->d_coef = nullptr;
    }
    if (!h->d_coef) {
        if (gpcn::dev_malloc(&h->d_coef, off) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, GP_ERR_NOMEM, "cudaMalloc of the coefficient tables failed");
        }
        h->coef_bytes = off;
    }
    GP_CK(h, cudaMemcpyAsync(h->d_coef, host.data(), off, cudaMemcpyHostToDevice, h->stream));
    GP_CK(h, cudaStreamSynchronize(h->stream));
    return GP_OK;
}

long long sweep_lines(gp_handle h, int ax) { return axis_lines(geom(h), ax); }

size_t blocks_for(long long items, int threads) { return (size_t)((items + threads - 1) / threads); }

FieldArgs handle_field_args(gp_handle h) {
    FieldArgs a = field_args(geom(h), h->buf[h->cur], h->d_scal + (h->scale_pending ? S_SCALE : S_ONE),
                             h->d_partials, h->d_counter, h->d_obs, h->d_scal + S_SCALE, h->d_scal + S_NORM_INIT);
    a.status = h->d_status;
    return a;
}

constexpr int kNormBlocks = 152 * 4;

gp_status alloc_scratch(gp_handle h) {
    prepare_field_launches();
    // z sweep: at most one block per 32 (line, segment) threads, segments of >= 1 node
    size_t cap = kNormBlocks;
    if (h->n[2] > 1) cap = std::max(cap, blocks_for(sweep_lines(h, 2), 32) * (size_t)(h->n[2] - 2));
    FieldArgs fa = handle_field_args(h);
    cap = std::max(cap, (size_t)observables_blocks(fa) * 9);
    if (gpcn::dev_malloc(&h->d_partials, cap * sizeof(double)) != cudaSuccess ||
        gpcn::dev_malloc(&h->d_scal, S_COUNT * sizeof(double)) != cudaSuccess ||
        gpcn::dev_malloc(&h->d_obs, O_COUNT * sizeof(double)) != cudaSuccess ||
        gpcn::dev_malloc(&h->d_counter, 2 * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, GP_ERR_NOMEM, "cudaMalloc of reduction scratch failed");
    }
    h->partial_cap = cap;
    h->d_status = h->d_counter + 1;
    double init[S_COUNT] = {1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    GP_CK(h, cudaMemcpyAsync(h->d_scal, init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
    GP_CK(h, cudaMemsetAsync(h->d_counter, 0, 2 * sizeof(unsigned int), h->stream));
    GP_CK(h, cudaStreamSynchronize(h->stream));
    return GP_OK;
}

void release(gp_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->own_buf0 && h->buf[0]) cudaFree(h->buf[0]);
    if (h->buf[1]) cudaFree(h->buf[1]);
    cudaFree(h->d_coef);
    cudaFree(h->d_scal);
    cudaFree(h->d_obs);
    cudaFree(h->d_partials);
    cudaFree(h->d_counter);
    cudaFree(h->d_track);
    cudaFree(h->d_obs_graph);
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaGetLastError();
    delete h;
}

gp_status create_common(gp_handle *out, gp_grid grid, double dt, double gamma, double nu,
                        double lambda, double g, gp_precision prec, gp_field field, void *stream,
                        void *dev_psi, size_t bytes) {
    if (!out) return fail(nullptr, GP_ERR_ARG, "out is NULL");
    *out = nullptr;
    gp_status st = check_args(grid, dt, gamma, nu, lambda, g, prec, field);
    if (st != GP_OK) return st;
    gp_handle h = new (std::nothrow) gp_handle_s();
    if (!h) return fail(nullptr, GP_ERR_NOMEM, "host allocation failed");
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, GP_ERR_CUDA, "no CUDA device");
    }
    h->n[0] = grid.nx;
    h->n[1] = grid.ny;
    h->n[2] = grid.nz;
    h->d[0] = grid.dx;
    h->d[1] = grid.ny > 1 ? grid.dy : 1.0;  // an absent axis adds no spacing to the cell measure
    h->d[2] = grid.nz > 1 ? grid.dz : 1.0;
    h->dt = dt;
    h->w[0] = gamma;
    h->w[1] = nu;
    h->w[2] = lambda;
    h->g = g;
    h->prec = prec;
    h->field = field;
    h->stream = static_cast<cudaStream_t>(stream);
    h->elem = (prec == GP_F64 ? 8 : (prec == GP_F32 ? 4 : 2)) * (field == GP_COMPLEX ? 2 : 1);
    h->sites = (size_t)grid.nx * grid.ny * grid.nz;
    h->bytes = h->sites * h->elem;
    if (dev_psi) {
        if (bytes < h->bytes || (reinterpret_cast<uintptr_t>(dev_psi) & 15u)) {
            delete h;
            return fail(nullptr, GP_ERR_ARG, "dev_psi too small or not 16-byte aligned");
        }
        h->buf[0] = dev_psi;
        h->own_buf0 = false;
    } else {
        if (gpcn::dev_malloc(&h->buf[0], h->bytes) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail(nullptr, GP_ERR_NOMEM, "cudaMalloc of psi failed");
        }
        h->own_buf0 = true;
        if (cudaMemsetAsync(h->buf[0], 0, h->bytes, h->stream) != cudaSuccess) {
            cudaGetLastError();
            release(h);
            return fail(nullptr, GP_ERR_CUDA, "cudaMemsetAsync of psi failed");
        }
    }
    if (gpcn::dev_malloc(&h->buf[1], h->bytes) != cudaSuccess) {
        cudaGetLastError();
        release(h);
        return fail(nullptr, GP_ERR_NOMEM, "cudaMalloc of the second psi buffer failed");
    }
    st = alloc_scratch(h);
    if (st == GP_OK) st = build_coefficients(h);
    {
        const long long rows = (long long)grid.nx * grid.ny;
        h->zmap_ok = encode_z_map(&h->zmap[0], h->buf[0], grid.nz, rows, (int)h->elem) &&
                     encode_z_map(&h->zmap[1], h->buf[1], grid.nz, rows, (int)h->elem);
    }
    if (st == GP_OK && prec == GP_F16) {
        // every FP16 sweep is windowed and its z sweep is the TMA form
        for (int ax = 0; ax < 3 && st == GP_OK; ++ax)
            if (h->n[ax] > 1 && h->tab.ax[0][ax].min_window == 0)
                st = fail(h, GP_ERR_ARG, "FP16 storage needs a windowed solve: dt too large for this spacing");
        if (st == GP_OK && !h->zmap_ok) st = fail(h, GP_ERR_ARG, "FP16 storage: no tensor map for the z sweep");
    }
    if (st != GP_OK) {
        g_create_error = h->err;
        release(h);
        return st;
    }
    *out = h;
    return GP_OK;
}

gp_status enter(gp_handle h) {
    if (!h) return fail(nullptr, GP_ERR_ARG, "NULL handle");
    if (cudaSetDevice(h->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
    }
    return GP_OK;
}

// enter() for the calls that read or advance psi: after an expired TMA wait
// psi is lost (the results of the launch are undefined, other blocks' lines
// included), and those calls fail until psi is set again.
gp_status enter_psi(gp_handle h) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    if (h->psi_lost)
        return fail(h, GP_ERR_STATE, "psi was lost to an expired TMA wait; set it again (gp_set_psi, "
                                     "gp_init_gaussian)");
    return GP_OK;
}

gp_status queue_observables(gp_handle h, double *dst);

// After a synchronisation: a kernel whose bounded wait expired left a flag.
gp_status check_status(gp_handle h) {
    unsigned int flag = 0;
    GP_CK(h, cudaMemcpy(&flag, h->d_status, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(h->d_status, 0, sizeof(flag));
        if (flag & 1u) {
            h->psi_lost = true;
            return fail(h, GP_ERR_TIMEOUT,
                        "a sweep kernel's wait for its TMA copies expired; psi is lost until set again");
        }
        return fail(h, GP_ERR_TIMEOUT,
                    "the observables kernel's wait for its bulk copies expired; these observables are invalid "
                    "(psi is unchanged)");
    }
    return GP_OK;
}

// Adjacent lines per thread on the strided axes, up to max_lpt[ax]: a group
// of g lines must be adjacent in memory and g-element aligned, i.e. the line
// count a multiple of g and, for y lines (i, k), nz a multiple of g.  Pairs
// for elements of 8 bytes or less; groups of four for FP32 real fields with
// a windowed solve (the form that has a four-line variant).
int lines_per_thread(gp_handle h, int ax, int window) {
    if (ax == 2 || h->elem > 8) return 1;
    auto fits = [&](int g) { return sweep_lines(h, ax) % g == 0 && (ax != 1 || h->n[2] % g == 0); };
    if (h->max_lpt[ax] >= 4 && (h->elem == 4 || h->elem == 2) && window > 0 && fits(4)) return 4;  // real fields
    if (h->max_lpt[ax] >= 2 && fits(2)) return 2;
    return 1;
}

// Segments of one axis (see choose_segments).
void segments(gp_handle h, int ax, int window, int *seg_len, int *n_seg) {
    choose_segments(geom(h), ax, window, lines_per_thread(h, ax, window), (int)h->elem, h->contiguous_z,
                    h->seg_override[ax], seg_len, n_seg);
}

// The stage of an absent axis (one node: a 1D or 2D condensate) solves no
// lines.  Its bookkeeping stays: in imaginary time the z stage's norm and
// renormalisation factor come from a reduction over the last sweep's output;
// in symmetric real time the trailing half kick becomes pending.
gp_status absent_stage(gp_handle h, int stage, bool realtime) {
    if (stage != 2) return GP_OK;
    if (!realtime) {
        FieldArgs a = field_args(geom(h), h->buf[h->cur], h->d_scal + S_ONE, h->d_partials, h->d_counter,
                                 h->d_obs, h->d_scal + S_SCALE, h->d_scal + S_NORM_SWEEP);
        GP_CK(h, launch_norm(prec_of(h), h->field == GP_COMPLEX, a, kNormBlocks, h->stream));
        h->scale_pending = true;
    } else if (h->splitting == 2) {
        h->kick_pending = true;
    }
    return GP_OK;
}

// Axes whose sweeps read through TMA boxes in a mode (0 imaginary, 1 real
// time): the mask set, or by default x for real fields (imaginary time).
// Measured inside full steps on 480x400x320: FP32 real x 0.1067 against
// 0.1076 ms, FP16 (640x480x400) 0.348 against 0.371; complex64 imaginary
// x 0.1746 against 0.1740 and real-time x 0.173 against 0.170 (slower).
int tma_line_axes(gp_handle h, int mode) {
    if (h->tma_lines >= 0) return h->tma_lines;
    return (mode == 0 && h->field == GP_REAL) ? 1 : 0;
}

// One stage of a step: 0 = kick + x sweep, 1 = y sweep, 2 = z sweep + norm.
gp_status run_stage(gp_handle h, int stage, bool realtime) {
    if (h->n[stage] == 1) return absent_stage(h, stage, realtime);
    SweepLaunch L;
    L.prec = prec_of(h);
    L.form = realtime ? F_REALTIME : (h->field == GP_REAL ? F_IMAG_REAL : F_IMAG_CPLX);
    L.kind = static_cast<Kind>(stage);
    const int mode = realtime ? 1 : 0;
    const int ax = stage;
    L.window = h->window[mode][ax];
    L.threads = h->threads[ax];
    L.lpt = lines_per_thread(h, ax, L.window);
    L.contiguous = (ax == 2 && h->contiguous_z && L.window > 0) ? 1 : 0;
    int seg_len = 0, n_seg = 0;
    segments(h, ax, L.window, &seg_len, &n_seg);
    // symmetric splitting: the first step after a settled state starts with a
    // half kick; later steps merge the previous trailing half kick with their
    // leading one (a real-time kick keeps |psi|, so two half kicks are one)
    const bool half = realtime && stage == 0 && h->splitting == 2 && !h->kick_pending;
    SweepArgs a = sweep_args(geom(h), ax, realtime, h->buf[h->cur], h->buf[h->cur ^ 1], h->d_coef,
                             h->tab, seg_len, n_seg,
                             h->d_scal + (h->scale_pending ? S_SCALE : S_ONE), h->d_partials,
                             h->d_counter, h->d_scal + S_NORM_SWEEP, h->d_scal + S_SCALE, half);
    a.status = h->d_status;
    TmaMaps maps;
    if (L.contiguous && h->tma_z && h->zmap_ok) {
        maps.in = h->zmap[h->cur];
        maps.out = h->zmap[h->cur ^ 1];
        L.tma = &maps;
    }
    TmaMaps lmaps;  // the strided TMA form reads through lmaps.in and stores lane by lane
    std::memset(&lmaps, 0, sizeof(lmaps));
    if (ax < 2 && (tma_line_axes(h, mode) >> ax & 1) && line_tma_fits((int)h->elem, L.lpt, L.window, a.inner, a.stride, a.N)) {
        const int box_nodes = h->elem * L.lpt >= 16 ? 8 : 16;  // the kernel's chunk of MemV nodes
        if (encode_line_map(&lmaps.in, h->buf[h->cur], ax, h->n, (int)h->elem, L.lpt, box_nodes))
            L.lmaps = &lmaps;
    }
    if (fp16(h) && (L.window == 0 || (ax < 2 && L.lpt < 2) ||
                    (ax == 2 && !(L.tma && tma_z_fits((int)h->elem, L.window, a.N, a.n_seg, a.n_lines)))))
        return fail(h, GP_ERR_STATE, "FP16 storage: no kernel for this axis under the current settings");
    const int zthreads = L.contiguous ? 32 : L.threads;
    if (stage == 2 && blocks_for(a.n_lines, zthreads) * (size_t)a.n_seg > h->partial_cap)
        return fail(h, GP_ERR_STATE, "z sweep grid exceeds the partials buffer");
    GP_CK(h, launch_sweep(L, a, h->stream));
    h->cur ^= 1;
    if (stage == 0) h->scale_pending = false;
    if (stage == 2 && !realtime) h->scale_pending = true;
    if (stage == 2 && realtime && h->splitting == 2) h->kick_pending = true;
    return GP_OK;
}

// Symmetric splitting: apply the trailing half kick that buf[cur] lacks, so
// that psi is the state after the last full step.
gp_status settle(gp_handle h) {
    if (!h->kick_pending) return GP_OK;
    FieldArgs a = handle_field_args(h);
    GP_CK(h, launch_kick(prec_of(h), a, 0.5 * h->dt, h->buf[h->cur ^ 1], h->stream));
    h->cur ^= 1;
    h->scale_pending = false;
    h->kick_pending = false;
    return GP_OK;
}

void drop_graphs(gp_handle h) {
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
    h->graphs.clear();
}

// One block of `g` steps as a CUDA graph (captured on first use, keyed by the
// state the captured launches depend on: step kind, block length, which
// buffer holds psi, whether a renormalisation factor is pending, and whether
// the block ends with a tracking record), then launched on the handle's
// stream.  Returns GP_STATE if capture is not possible, so the caller can
// launch the block kernel by kernel instead.
gp_status run_graph_block(gp_handle h, int g, bool realtime, bool with_obs) {
    const auto key = std::make_tuple(realtime ? h->splitting : 0, g, h->cur, h->scale_pending ? 1 : 0,
                                     h->kick_pending ? 1 : 0, with_obs ? 1 : 0);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return GP_ERR_STATE;
        }
        if (with_obs && !h->d_obs_graph && gpcn::dev_malloc(&h->d_obs_graph, O_COUNT * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return GP_ERR_STATE;
        }
        const int cur0 = h->cur;
        const bool pend0 = h->scale_pending, kick0 = h->kick_pending;
        cudaStream_t user = h->stream;
        if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return GP_ERR_STATE;
        }
        h->stream = h->cap_stream;
        gp_status st = GP_OK;
        for (int s = 0; s < g && st == GP_OK; ++s)
            for (int stage = 0; stage < 3 && st == GP_OK; ++stage) st = run_stage(h, stage, realtime);
        if (st == GP_OK && with_obs) st = settle(h);
        if (st == GP_OK && with_obs) st = queue_observables(h, h->d_obs_graph);
        const gp_handle_s::Graph end{nullptr, h->cur, h->scale_pending, h->kick_pending};
        h->stream = user;
        h->cur = cur0;
        h->scale_pending = pend0;
        h->kick_pending = kick0;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
        cudaGraphExec_t exec = nullptr;
        const bool ok = st == GP_OK && ec == cudaSuccess && graph &&
                        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            cudaGetLastError();
            return GP_ERR_STATE;
        }
        it = h->graphs.emplace(key, gp_handle_s::Graph{exec, end.cur, end.scale_pending, end.kick_pending}).first;
    }
    GP_CK(h, cudaGraphLaunch(it->second.exec, h->stream));
    h->cur = it->second.cur;
    h->scale_pending = it->second.scale_pending;
    h->kick_pending = it->second.kick_pending;
    return GP_OK;
}

// Steps launched kernel by kernel (with tracking records queued in between).
gp_status run_eager(gp_handle h, int nsteps, bool realtime) {
    for (int s = 0; s < nsteps; ++s) {
        for (int stage = 0; stage < 3; ++stage) {
            gp_status st = run_stage(h, stage, realtime);
            if (st != GP_OK) return st;
        }
        h->step += 1;
        h->t += h->dt;
        if (h->track_every > 0 && h->step % h->track_every == 0 && h->track_count < h->track_cap) {
            gp_status st = settle(h);
            if (st == GP_OK) st = queue_observables(h, h->d_track + (size_t)h->track_count * O_COUNT);
            if (st != GP_OK) return st;
            h->track_step.push_back(h->step);
            h->track_t.push_back(h->t);
            h->track_count += 1;
        }
    }
    return GP_OK;
}

gp_status run_steps(gp_handle h, int nsteps, bool realtime) {
    if (nsteps < 0) return fail(h, GP_ERR_ARG, "nsteps < 0");
    if (realtime && h->field != GP_COMPLEX)
        return fail(h, GP_ERR_STATE, "real-time steps need a GP_COMPLEX field");
    if (!realtime) {
        gp_status st = settle(h);
        if (st != GP_OK) return st;
    }
    // Whole blocks as graphs.  With tracking on, a block is track_every steps
    // ending on a tracking step (its record is copied out of the graph's
    // slot); steps up to the next tracking step go kernel by kernel.
    while (nsteps > 1 && h->graph_block > 1) {
        const bool tracking = h->track_every > 0 && h->track_count < h->track_cap;
        int g = std::min(nsteps, h->graph_block);
        if (tracking) {
            const int lead = (int)((h->track_every - h->step % h->track_every) % h->track_every);
            if (lead > 0) {
                const int n = std::min(lead, nsteps);
                gp_status st = run_eager(h, n, realtime);
                if (st != GP_OK) return st;
                nsteps -= n;
                continue;
            }
            if (h->track_every < 2 || h->track_every > h->graph_block || nsteps < h->track_every) break;
            g = h->track_every;
        }
        const gp_status st = run_graph_block(h, g, realtime, tracking);
        if (st == GP_ERR_STATE) break;  // not capturable here: launch kernel by kernel
        if (st != GP_OK) return st;
        h->step += g;
        for (int k = 0; k < g; ++k) h->t += h->dt;  // same rounding as step by step
        nsteps -= g;
        if (tracking) {
            GP_CK(h, cudaMemcpyAsync(h->d_track + (size_t)h->track_count * O_COUNT, h->d_obs_graph,
                                     O_COUNT * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
            h->track_step.push_back(h->step);
            h->track_t.push_back(h->t);
            h->track_count += 1;
        }
    }
    return run_eager(h, nsteps, realtime);
}

gp_status queue_observables(gp_handle h, double *dst) {
    FieldArgs a = handle_field_args(h);
    a.out = dst;
    if ((size_t)observables_blocks(a) * 9 > h->partial_cap)
        return fail(h, GP_ERR_STATE, "observables grid exceeds the partials buffer");
    GP_CK(h, launch_observables(prec_of(h), h->field == GP_COMPLEX, a,
                                h->stream));
    return GP_OK;
}

void fill_obs(const double *o, long long step, double t, gp_obs *out) {
    out->norm = o[O_NORM];
    out->mu = o[O_MU];
    out->energy = o[O_E];
    out->rms_x = o[O_RMSX];
    out->rms_y = o[O_RMSY];
    out->rms_z = o[O_RMSZ];
    out->step = step;
    out->t = t;
}

gp_status observables(gp_handle h, gp_obs *out) {
    gp_status st = settle(h);
    if (st != GP_OK) return st;
    st = queue_observables(h, h->d_obs);
    if (st != GP_OK) return st;
    double o[O_COUNT];
    GP_CK(h, cudaMemcpyAsync(o, h->d_obs, sizeof(o), cudaMemcpyDeviceToHost, h->stream));
    GP_CK(h, cudaStreamSynchronize(h->stream));
    if (out) fill_obs(o, h->step, h->t, out);
    st = check_status(h);
    if (st != GP_OK) return st;
    if (o[O_FINITE] != 1.0) return fail(h, GP_ERR_NONFINITE, "psi holds NaN or Inf");
    return GP_OK;
}

}  // namespace

extern "C" {

gp_status gp_create(gp_handle *out, gp_grid grid, double dt, double gamma, double nu,
                    double lambda, double g, gp_precision prec, gp_field field,
                    void *cuda_stream) {
    return create_common(out, grid, dt, gamma, nu, lambda, g, prec, field, cuda_stream, nullptr, 0);
}

gp_status gp_create_ext(gp_handle *out, gp_grid grid, double dt, double gamma, double nu,
                        double lambda, double g, gp_precision prec, gp_field field,
                        void *cuda_stream, void *dev_psi, size_t bytes) {
    if (!dev_psi) return fail(nullptr, GP_ERR_ARG, "dev_psi is NULL");
    return create_common(out, grid, dt, gamma, nu, lambda, g, prec, field, cuda_stream, dev_psi,
                         bytes);
}

void gp_destroy(gp_handle h) { release(h); }

gp_status gp_init_gaussian(gp_handle h) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    FieldArgs a = handle_field_args(h);
    const Prec p = prec_of(h);
    const bool cplx = h->field == GP_COMPLEX;
    GP_CK(h, launch_gaussian(p, cplx, a, h->stream));
    GP_CK(h, launch_norm(p, cplx, a, kNormBlocks, h->stream));
    h->scale_pending = true;
    h->kick_pending = false;
    h->psi_lost = false;
    h->step = 0;
    h->t = 0.0;
    return GP_OK;
}

gp_status gp_set_psi(gp_handle h, const void *psi, int on_device) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    if (!psi) return fail(h, GP_ERR_ARG, "psi is NULL");
    GP_CK(h, cudaMemcpyAsync(h->buf[h->cur], psi, h->bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             h->stream));
    if (!on_device) GP_CK(h, cudaStreamSynchronize(h->stream));
    h->scale_pending = false;
    h->kick_pending = false;
    h->psi_lost = false;
    h->step = 0;
    h->t = 0.0;
    return GP_OK;
}

gp_status gp_get_psi(gp_handle h, void *psi, int on_device) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if (!psi) return fail(h, GP_ERR_ARG, "psi is NULL");
    if ((st = settle(h)) != GP_OK) return st;
    FieldArgs a = handle_field_args(h);
    const Prec p = prec_of(h);
    const bool cplx = h->field == GP_COMPLEX;
    if (on_device) {
        GP_CK(h, launch_apply_scale(p, cplx, a, psi, h->stream));
        return GP_OK;
    }
    if (h->scale_pending) {  // fold the pending factor into psi (same rounding as the next kick)
        GP_CK(h, launch_apply_scale(p, cplx, a, h->buf[h->cur], h->stream));
        h->scale_pending = false;
    }
    GP_CK(h, cudaMemcpyAsync(psi, h->buf[h->cur], h->bytes, cudaMemcpyDeviceToHost, h->stream));
    GP_CK(h, cudaStreamSynchronize(h->stream));
    return GP_OK;
}

gp_status gp_set_g(gp_handle h, double g) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    if (!std::isfinite(g)) return fail(h, GP_ERR_ARG, "g must be finite");
    if ((st = settle(h)) != GP_OK) return st;  // the pending half kick belongs to the old g
    if (g != h->g) drop_graphs(h);
    h->g = g;
    return GP_OK;
}

gp_status gp_set_dt(gp_handle h, double dt) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    if (!finite_pos(dt)) return fail(h, GP_ERR_ARG, "dt must be finite and > 0");
    if ((st = settle(h)) != GP_OK) return st;  // the pending half kick belongs to the old dt
    drop_graphs(h);
    h->dt = dt;
    return build_coefficients(h);
}

gp_status gp_step_imag(gp_handle h, int nsteps) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    return run_steps(h, nsteps, false);
}

gp_status gp_step_real(gp_handle h, int nsteps) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    return run_steps(h, nsteps, true);
}

gp_status gp_run_imag_until(gp_handle h, double mu_tol, int check_every, int max_steps,
                            int *steps_taken) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if (!(mu_tol > 0.0) || check_every < 1 || max_steps < 0)
        return fail(h, GP_ERR_ARG, "need mu_tol > 0, check_every >= 1, max_steps >= 0");
    gp_obs o;
    st = observables(h, &o);
    if (st != GP_OK) return st;
    double mu_prev = o.mu, e_prev = o.energy;
    int taken = 0, streak = 0;
    const int need = h->stop_rule == 2 ? 2 : 1;  // consecutive checks that must pass
    while (taken < max_steps) {
        const int n = std::min(check_every, max_steps - taken);
        st = run_steps(h, n, false);
        if (st != GP_OK) break;
        taken += n;
        st = observables(h, &o);
        if (st != GP_OK) break;
        const bool pass = std::fabs(o.mu - mu_prev) < mu_tol &&
                          (h->stop_rule == 0 || std::fabs(o.energy - e_prev) < mu_tol);
        streak = pass ? streak + 1 : 0;
        if (streak >= need) break;
        mu_prev = o.mu;
        e_prev = o.energy;
    }
    if (steps_taken) *steps_taken = taken;
    return st;
}

gp_status gp_run_imag_schedule(gp_handle h, int levels, const double *dt_scale, const double *mu_tol,
                               int check_every, int max_steps, int *steps_taken) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if (levels < 1 || !dt_scale || !mu_tol) return fail(h, GP_ERR_ARG, "need levels >= 1 and both arrays");
    for (int l = 0; l < levels; ++l)
        if (!finite_pos(dt_scale[l])) return fail(h, GP_ERR_ARG, "dt scales must be finite and > 0");
    const double base = h->dt;
    int total = 0;
    for (int l = 0; l < levels && st == GP_OK; ++l) {
        int part = 0;
        if (dt_scale[l] * base != h->dt) st = gp_set_dt(h, base * dt_scale[l]);
        if (st == GP_OK) st = gp_run_imag_until(h, mu_tol[l], check_every, max_steps, &part);
        total += part;
    }
    if (h->dt != base) {
        const gp_status back = gp_set_dt(h, base);
        if (st == GP_OK) st = back;
    }
    if (steps_taken) *steps_taken = total;
    return st;
}

gp_status gp_set_stop_rule(gp_handle h, int rule) {
    if (!h) return fail(h, GP_ERR_ARG, "NULL handle");
    if (rule < 0 || rule > 2) return fail(h, GP_ERR_ARG, "rule must be 0, 1 or 2");
    h->stop_rule = rule;
    return GP_OK;
}

gp_status gp_observables(gp_handle h, gp_obs *out) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if (!out) return fail(h, GP_ERR_ARG, "out is NULL");
    return observables(h, out);
}

gp_status gp_density_profiles(gp_handle h, double *rho_x, double *rho_y, double *rho_z) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if (fp16(h)) return fail(h, GP_ERR_STATE, "not for FP16 storage");
    if (!rho_x && !rho_y && !rho_z) return GP_OK;
    FieldArgs a = handle_field_args(h);  // the pending scale enters as s^2; a pending half kick is a phase
    const size_t nd = profile_scratch_doubles(a);
    const int total = h->n[0] + h->n[1] + h->n[2];
    double *scratch = nullptr;
    if (gpcn::dev_malloc(&scratch, nd * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, GP_ERR_NOMEM, "cudaMalloc of the profile scratch failed");
    }
    double *out = scratch + (nd - (size_t)total);
    std::vector<double> host((size_t)total);
    cudaError_t e = launch_density_profiles(prec_of(h), h->field == GP_COMPLEX, a, scratch,
                                            out, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host.data(), out, (size_t)total * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, GP_ERR_CUDA, std::string("density profiles: ") + cudaGetErrorString(e));
    }
    if (rho_x) std::copy(host.begin(), host.begin() + h->n[0], rho_x);
    if (rho_y) std::copy(host.begin() + h->n[0], host.begin() + h->n[0] + h->n[1], rho_y);
    if (rho_z) std::copy(host.begin() + h->n[0] + h->n[1], host.end(), rho_z);
    return GP_OK;
}

gp_status gp_write_wavefunction(gp_handle h, const char *path, int what) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if (fp16(h)) return fail(h, GP_ERR_STATE, "not for FP16 storage (read psi with gp_get_psi)");
    if (!path) return fail(h, GP_ERR_ARG, "path is NULL");
    if (what != GP_OUT_PSI && what != GP_OUT_DENSITY) return fail(h, GP_ERR_ARG, "what must be GP_OUT_PSI or GP_OUT_DENSITY");
    const bool f32 = h->prec == GP_F32, cplx = h->field == GP_COMPLEX;
    std::vector<char> buf;
    try {
        buf.resize(h->bytes);
    } catch (const std::bad_alloc &) {
        return fail(h, GP_ERR_NOMEM, "host buffer for the wavefunction");
    }
    if ((st = gp_get_psi(h, buf.data(), 0)) != GP_OK) return st;
    const char *descr = nullptr;
    size_t out_bytes = h->bytes;
    if (what == GP_OUT_PSI) {
        descr = cplx ? (f32 ? "<c8" : "<c16") : (f32 ? "<f4" : "<f8");
    } else {
        // |psi|^2 in FP64 from the stored values (exact products), rounded once
        descr = f32 ? "<f4" : "<f8";
        const size_t n = h->sites;
        for (size_t s = 0; s < n; ++s) {
            double d2;
            if (f32) {
                const float *p = reinterpret_cast<const float *>(buf.data()) + (cplx ? 2 * s : s);
                d2 = cplx ? (double)p[0] * p[0] + (double)p[1] * p[1] : (double)p[0] * p[0];
                const float f = (float)d2;
                std::memcpy(buf.data() + s * sizeof(float), &f, sizeof(f));  // s * 4 <= read offset
            } else {
                const double *p = reinterpret_cast<const double *>(buf.data()) + (cplx ? 2 * s : s);
                // both squares rounded before the sum on every host (no fused multiply-add)
                volatile double re2 = p[0] * p[0], im2 = cplx ? p[1] * p[1] : 0.0;
                d2 = re2 + im2;
                std::memcpy(buf.data() + s * sizeof(double), &d2, sizeof(d2));
            }
        }
        out_bytes = n * (f32 ? sizeof(float) : sizeof(double));
    }
    // NPY 1.0: magic, version, little-endian header length, a Python dict
    // literal padded with spaces to a 64-byte boundary and ended by '\n'
    std::string hdr = std::string("{'descr': '") + descr + "', 'fortran_order': False, 'shape': (" +
                      std::to_string(h->n[0]) + ", " + std::to_string(h->n[1]) + ", " + std::to_string(h->n[2]) +
                      "), }";
    const size_t pre = 10;
    const size_t total = (pre + hdr.size() + 1 + 63) / 64 * 64;
    hdr.append(total - pre - hdr.size() - 1, ' ');
    hdr.push_back('\n');
    unsigned char head[10] = {0x93, 'N', 'U', 'M', 'P', 'Y', 1, 0, (unsigned char)(hdr.size() & 0xff),
                              (unsigned char)(hdr.size() >> 8)};
    std::FILE *f = std::fopen(path, "wb");
    if (!f) return fail(h, GP_ERR_IO, std::string("cannot open ") + path);
    const bool ok = std::fwrite(head, 1, sizeof(head), f) == sizeof(head) &&
                    std::fwrite(hdr.data(), 1, hdr.size(), f) == hdr.size() &&
                    std::fwrite(buf.data(), 1, out_bytes, f) == out_bytes;
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) {
        std::remove(path);
        return fail(h, GP_ERR_IO, std::string("cannot write ") + path);
    }
    return GP_OK;
}

gp_status gp_set_tracking(gp_handle h, int every, int capacity) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    if (every < 0 || capacity < 0 || (every > 0 && capacity < 1))
        return fail(h, GP_ERR_ARG, "need every >= 0 and capacity >= 1 when tracking");
    GP_CK(h, cudaStreamSynchronize(h->stream));
    if (h->d_track && capacity > h->track_cap) {
        cudaFree(h->d_track);
        h->d_track = nullptr;
        h->track_cap = 0;
    }
    if (every > 0 && !h->d_track) {
        if (gpcn::dev_malloc(&h->d_track, (size_t)capacity * O_COUNT * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, GP_ERR_NOMEM, "cudaMalloc of the tracking history failed");
        }
        h->track_cap = capacity;
    }
    h->track_every = every;
    h->track_count = 0;
    h->track_step.clear();
    h->track_t.clear();
    return GP_OK;
}

gp_status gp_get_tracking(gp_handle h, gp_obs *out, int max, int *count) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    if (max < 0 || (max > 0 && !out)) return fail(h, GP_ERR_ARG, "bad output buffer");
    const int n = std::min(max, h->track_count);
    std::vector<double> buf((size_t)std::max(n, 1) * O_COUNT);
    if (n > 0)
        GP_CK(h, cudaMemcpyAsync(buf.data(), h->d_track, (size_t)n * O_COUNT * sizeof(double),
                                 cudaMemcpyDeviceToHost, h->stream));
    GP_CK(h, cudaStreamSynchronize(h->stream));
    bool finite = true;
    for (int r = 0; r < n; ++r) {
        fill_obs(buf.data() + (size_t)r * O_COUNT, h->track_step[r], h->track_t[r], out + r);
        finite = finite && buf[(size_t)r * O_COUNT + O_FINITE] == 1.0;
    }
    if (count) *count = h->track_count;
    if (!finite) return fail(h, GP_ERR_NONFINITE, "a tracked record is non-finite");
    return GP_OK;
}

gp_status gp_step_stage(gp_handle h, int stage, int realtime) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if (stage < 0 || stage > 2) return fail(h, GP_ERR_ARG, "stage must be 0, 1 or 2");
    if (realtime && h->field != GP_COMPLEX)
        return fail(h, GP_ERR_STATE, "real-time stages need a GP_COMPLEX field");
    if ((st = settle(h)) != GP_OK) return st;
    const int split = h->splitting;  // single stages are the Lie form's
    h->splitting = 1;
    st = run_stage(h, stage, realtime != 0);
    h->splitting = split;
    return st;
}

gp_status gp_set_stream(gp_handle h, void *cuda_stream) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    GP_CK(h, cudaStreamSynchronize(h->stream));
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return GP_OK;
}

gp_status gp_sync(gp_handle h) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    GP_CK(h, cudaStreamSynchronize(h->stream));
    return check_status(h);
}

gp_status gp_get_window(gp_handle h, int mode, int window[3]) {
    if (!h || !window || mode < 0 || mode > 1) return fail(h, GP_ERR_ARG, "bad arguments");
    if (mode >= modes_of(h)) return fail(h, GP_ERR_STATE, "no real-time tables on a GP_REAL field");
    for (int ax = 0; ax < 3; ++ax) window[ax] = h->window[mode][ax];
    return GP_OK;
}

gp_status gp_set_window(gp_handle h, int window) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    if (window != -1 && window != 0 && window != 4 && window != 8 && window != 16)
        return fail(h, GP_ERR_ARG, "window must be -1 (automatic), 0, 4, 8 or 16");
    if (window == 0 && fp16(h)) return fail(h, GP_ERR_ARG, "FP16 storage needs a windowed solve");
    if (window > 0) {
        for (int mode = 0; mode < modes_of(h); ++mode)
            for (int ax = 0; ax < 3; ++ax) {
                const AxisTables &at = h->tab.ax[mode][ax];
                if (h->n[ax] > 1 && (at.min_window == 0 || window < at.min_window))
                    return fail(h, GP_ERR_ARG, "window too small for the accuracy of this dt");
            }
    }
    for (int mode = 0; mode < modes_of(h); ++mode)
        for (int ax = 0; ax < 3; ++ax)
            h->window[mode][ax] = window >= 0 ? window : default_window(h->tab.ax[mode][ax], h->prec != GP_F64);
    h->forced_window = window;
    drop_graphs(h);
    return GP_OK;
}

gp_status gp_set_axis_window(gp_handle h, int axis, int window) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    if (axis < 0 || axis > 2) return fail(h, GP_ERR_ARG, "bad axis");
    if (window != -1 && window != 0 && window != 4 && window != 8 && window != 16)
        return fail(h, GP_ERR_ARG, "window must be -1 (automatic), 0, 4, 8 or 16");
    if (window == 0 && fp16(h)) return fail(h, GP_ERR_ARG, "FP16 storage needs a windowed solve");
    for (int mode = 0; mode < modes_of(h); ++mode) {
        const AxisTables &at = h->tab.ax[mode][axis];
        if (h->n[axis] > 1 && window > 0 && (at.min_window == 0 || window < at.min_window))
            return fail(h, GP_ERR_ARG, "window too small for the accuracy of this dt");
    }
    for (int mode = 0; mode < modes_of(h); ++mode)
        h->window[mode][axis] = window >= 0 ? window : default_window(h->tab.ax[mode][axis], h->prec != GP_F64);
    drop_graphs(h);
    return GP_OK;
}

gp_status gp_set_pair_lines(gp_handle h, int on) {
    if (!h) return fail(h, GP_ERR_ARG, "NULL handle");
    if (!on && fp16(h)) return fail(h, GP_ERR_ARG, "FP16 storage moves two or four lines per thread");
    h->max_lpt[0] = h->max_lpt[1] = on ? 4 : 1;
    drop_graphs(h);
    return GP_OK;
}

gp_status gp_set_lines_per_thread(gp_handle h, int axis, int lines) {
    if (!h || axis < 0 || axis > 1) return fail(h, GP_ERR_ARG, "axis must be 0 (x) or 1 (y)");
    if (lines != 1 && lines != 2 && lines != 4) return fail(h, GP_ERR_ARG, "lines must be 1, 2 or 4");
    if (lines == 1 && fp16(h)) return fail(h, GP_ERR_ARG, "FP16 storage moves two or four lines per thread");
    h->max_lpt[axis] = lines;
    drop_graphs(h);
    return GP_OK;
}

gp_status gp_get_lines_per_thread(gp_handle h, int mode, int lines[3]) {
    if (!h || !lines || mode < 0 || mode > 1) return fail(h, GP_ERR_ARG, "bad arguments");
    if (mode >= modes_of(h)) return fail(h, GP_ERR_STATE, "no real-time tables on a GP_REAL field");
    for (int ax = 0; ax < 3; ++ax) lines[ax] = lines_per_thread(h, ax, h->window[mode][ax]);
    return GP_OK;
}

gp_status gp_set_splitting(gp_handle h, int order) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    if (order != 1 && order != 2) return fail(h, GP_ERR_ARG, "order must be 1 or 2");
    if ((st = settle(h)) != GP_OK) return st;
    if (order != h->splitting) drop_graphs(h);
    h->splitting = order;
    return GP_OK;
}

gp_status gp_set_tma(gp_handle h, int on) {
    if (!h) return fail(h, GP_ERR_ARG, "NULL handle");
    if (!on && fp16(h)) return fail(h, GP_ERR_ARG, "the FP16 z sweep is the TMA form");
    h->tma_z = on != 0;
    drop_graphs(h);
    return GP_OK;
}

gp_status gp_get_tma(gp_handle h, int *in_use) {
    if (!h || !in_use) return fail(h, GP_ERR_ARG, "bad arguments");
    // the z sweep of either mode takes the TMA form: enabled, maps encoded,
    // the contiguous windowed solve, and rows and window that fit it
    int used = 0;
    for (int mode = 0; mode < modes_of(h); ++mode) {
        const int w = h->window[mode][2];
        int seg_len = 0, n_seg = 0;
        segments(h, 2, w, &seg_len, &n_seg);
        used |= (h->tma_z && h->zmap_ok && h->contiguous_z && w > 0 &&
                 tma_z_fits((int)h->elem, w, h->n[2], n_seg, sweep_lines(h, 2))) ? 1 : 0;
    }
    *in_use = used;
    return GP_OK;
}

gp_status gp_set_tma_lines(gp_handle h, int axes) {
    if (!h) return fail(h, GP_ERR_ARG, "NULL handle");
    if (axes < -1 || axes > 3) return fail(h, GP_ERR_ARG, "axes must be -1 or a mask of bit 0 (x) and bit 1 (y)");
    h->tma_lines = axes;
    drop_graphs(h);
    return GP_OK;
}

gp_status gp_get_tma_lines(gp_handle h, int *axes) {
    if (!h || !axes) return fail(h, GP_ERR_ARG, "bad arguments");
    int used = 0;
    for (int mode = 0; mode < modes_of(h); ++mode) {
        for (int ax = 0; ax < 2; ++ax) {
            if (h->n[ax] == 1) continue;
            const int w = h->window[mode][ax];
            const long long plane = (long long)h->n[1] * h->n[2];
            const long long inner = ax == 0 ? plane : h->n[2];
            const int lpt = lines_per_thread(h, ax, w);
            CUtensorMap probe;  // the map the launch would encode (x and y: inner is the node stride)
            if ((tma_line_axes(h, mode) >> ax & 1) && line_tma_fits((int)h->elem, lpt, w, inner, inner, h->n[ax]) &&
                encode_line_map(&probe, h->buf[0], ax, h->n, (int)h->elem, lpt, h->elem * lpt >= 16 ? 8 : 16))
                used |= 1 << ax;
        }
    }
    *axes = used;
    return GP_OK;
}

gp_status gp_set_threads(gp_handle h, int axis, int threads) {
    if (!h || axis < 0 || axis > 2) return fail(h, GP_ERR_ARG, "bad axis");
    if (threads < 32 || threads > 256 || threads % 32)
        return fail(h, GP_ERR_ARG, "threads must be a multiple of 32 in [32, 256]");
    h->threads[axis] = threads;
    drop_graphs(h);
    return GP_OK;
}

gp_status gp_set_segments(gp_handle h, int axis, int seg_len) {
    if (!h || axis < 0 || axis > 2) return fail(h, GP_ERR_ARG, "bad axis");
    if (seg_len < 0) return fail(h, GP_ERR_ARG, "seg_len must be >= 0");
    h->seg_override[axis] = seg_len;
    drop_graphs(h);
    return GP_OK;
}

gp_status gp_get_segments(gp_handle h, int mode, int seg_len[3], int n_seg[3]) {
    if (!h || !seg_len || !n_seg || mode < 0 || mode > 1) return fail(h, GP_ERR_ARG, "bad arguments");
    if (mode >= modes_of(h)) return fail(h, GP_ERR_STATE, "no real-time tables on a GP_REAL field");
    for (int ax = 0; ax < 3; ++ax) segments(h, ax, h->window[mode][ax], &seg_len[ax], &n_seg[ax]);
    return GP_OK;
}

gp_status gp_psi_device_ptr(gp_handle h, void **ptr, int *pending_scale) {
    if (!h || !ptr) return fail(h, GP_ERR_ARG, "bad arguments");
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if ((st = settle(h)) != GP_OK) return st;
    *ptr = h->buf[h->cur];
    if (pending_scale) *pending_scale = h->scale_pending ? 1 : 0;
    return GP_OK;
}

gp_status gp_debug_raise_status(gp_handle h, unsigned int bits) {
    if (!h || bits == 0u || bits > 3u) return fail(h, GP_ERR_ARG, "status bits must be 1, 2 or 3");
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    const unsigned int flag = bits;
    GP_CK(h, cudaMemcpyAsync(h->d_status, &flag, sizeof(flag), cudaMemcpyHostToDevice, h->stream));
    GP_CK(h, cudaStreamSynchronize(h->stream));
    return GP_OK;
}

gp_status gp_pending_scale(gp_handle h, double *scale) {
    if (!h || !scale) return fail(h, GP_ERR_ARG, "bad arguments");
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if ((st = settle(h)) != GP_OK) return st;
    double v = 1.0;
    if (h->scale_pending) {
        GP_CK(h, cudaMemcpyAsync(&v, h->d_scal + S_SCALE, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
        GP_CK(h, cudaStreamSynchronize(h->stream));
    }
    *scale = v;
    return GP_OK;
}

// ---------------------------------------------------------------- autotuner
namespace {

struct TuneChoice {
    int threads, seg, lpt;  // lpt: most lines per thread (strided axes)
};

std::string tune_key(gp_handle h, int realtime, int ax) {
    std::ostringstream k;
    k << h->n[0] << "x" << h->n[1] << "x" << h->n[2] << (h->prec == GP_F32 ? "/f32" : (h->prec == GP_F16 ? "/f16" : "/f64"))
      << (h->field == GP_COMPLEX ? "/c" : "/r") << (realtime ? "/rt" : "/it") << "/w" << h->window[realtime][ax]
      << "/ax" << ax << "/v2";
    return k.str();
}

// Cache file: one "key threads seg lpt" line per tuned (grid, form, axis).
bool cache_lookup(const char *path, const std::string &key, TuneChoice *c) {
    if (!path || !*path) return false;
    std::ifstream f(path);
    std::string k;
    TuneChoice t;
    bool found = false;
    while (f >> k >> t.threads >> t.seg >> t.lpt)
        if (k == key) {
            *c = t;
            found = true;
        }
    return found;
}

void cache_store(const char *path, const std::string &key, const TuneChoice &c) {
    if (!path || !*path) return;
    std::ofstream f(path, std::ios::app);
    f << key << " " << c.threads << " " << c.seg << " " << c.lpt << "\n";
}

}  // namespace

}  // extern "C"

namespace {
gp_status autotune(gp_handle h, int realtime, int reps, const char *cache_path) {
    gp_status st = GP_OK;
    const char *path = cache_path ? cache_path : std::getenv("GP_AUTOTUNE_CACHE");
    const int mode = realtime ? 1 : 0;
    // A stage reads buf[cur] and writes only buf[cur ^ 1] (free between
    // steps), so trials started from cur0 leave psi intact; the z stage of
    // imaginary time also writes the pending renormalisation factor, which
    // is saved in a spare scalar slot and restored.
    const int cur0 = h->cur;
    const bool pend0 = h->scale_pending;
    GP_CK(h, cudaMemcpyAsync(h->d_scal + S_SAVE, h->d_scal, 4 * sizeof(double), cudaMemcpyDeviceToDevice,
                             h->stream));
    cudaEvent_t e0, e1;
    GP_CK(h, cudaEventCreate(&e0));
    GP_CK(h, cudaEventCreate(&e1));
    for (int ax = 0; ax < 3 && st == GP_OK; ++ax) {
        if (h->n[ax] == 1) continue;  // an absent axis has no sweep
        const std::string key = tune_key(h, realtime, ax);
        TuneChoice best{h->threads[ax], h->seg_override[ax], ax < 2 ? h->max_lpt[ax] : 1};
        if (cache_lookup(path, key, &best)) {
            h->threads[ax] = best.threads;
            h->seg_override[ax] = best.seg;
            if (ax < 2) h->max_lpt[ax] = best.lpt;
            continue;
        }
        const int n = h->n[ax] - 2;
        std::vector<TuneChoice> cands;
        const int segs[] = {0, 64, 128, 256, n};
        for (int th : {64, 128})
            for (int sg : segs)
                for (int lp : {4, 2, 1}) {
                    if (ax == 2 && lp != 1) continue;  // line groups apply to the strided axes only
                    if (ax < 2 && lp == 1 && fp16(h)) continue;  // FP16 storage moves two or four lines
                    if (h->window[mode][ax] == 0 && sg != 0) continue;  // the exact solve has no segments
                    // skip limits that select the same group size as a larger one
                    if (ax < 2 && lp < 4) {
                        const int keep = h->max_lpt[ax];
                        h->max_lpt[ax] = lp * 2;
                        const int wider = lines_per_thread(h, ax, h->window[mode][ax]);
                        h->max_lpt[ax] = lp;
                        const int mine = lines_per_thread(h, ax, h->window[mode][ax]);
                        h->max_lpt[ax] = keep;
                        if (wider == mine) continue;
                    }
                    cands.push_back({th, sg, lp});
                }
        float best_ms = 1e30f;
        for (const TuneChoice &c : cands) {
            h->threads[ax] = c.threads;
            h->seg_override[ax] = c.seg;
            if (ax < 2) h->max_lpt[ax] = c.lpt;
            float ms = 0.f;
            for (int r = 0; r <= reps && st == GP_OK; ++r) {  // r = 0 warms up
                h->cur = cur0;
                h->scale_pending = pend0;
                if (r == 1) GP_CK(h, cudaEventRecord(e0, h->stream));
                st = run_stage(h, ax, realtime);
            }
            if (st != GP_OK) break;
            GP_CK(h, cudaEventRecord(e1, h->stream));
            GP_CK(h, cudaEventSynchronize(e1));
            GP_CK(h, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        h->threads[ax] = best.threads;
        h->seg_override[ax] = best.seg;
        if (ax < 2) h->max_lpt[ax] = best.lpt;
        cache_store(path, key, best);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cur = cur0;
    h->scale_pending = pend0;
    GP_CK(h, cudaMemcpyAsync(h->d_scal, h->d_scal + S_SAVE, 4 * sizeof(double), cudaMemcpyDeviceToDevice,
                             h->stream));
    GP_CK(h, cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    return st;
}
}  // namespace

extern "C" {

gp_status gp_autotune(gp_handle h, int realtime, int reps, const char *cache_path) {
    gp_status st = enter_psi(h);
    if (st != GP_OK) return st;
    if (realtime && h->field != GP_COMPLEX) return fail(h, GP_ERR_STATE, "real time needs a GP_COMPLEX field");
    if (reps < 1) return fail(h, GP_ERR_ARG, "reps must be >= 1");
    if ((st = settle(h)) != GP_OK) return st;
    const int split = h->splitting;  // trials time the Lie form's stages
    h->splitting = 1;
    st = autotune(h, realtime, reps, cache_path);
    h->splitting = split;
    return st;
}


gp_status gp_nn_predict(gp_nn net, gp_handle h) {
    gp_status st = enter(h);
    if (st != GP_OK) return st;
    const NNParams *P = nn_params(net);
    if (!P) return fail(h, GP_ERR_ARG, "NULL network");
    if (fp16(h)) return fail(h, GP_ERR_STATE, "not for FP16 storage");
    const NNInstance I = make_nn_instance(h->n, h->d, h->w, h->g);
    GP_CK(h, nn_launch_predict(*P, I, h->buf[h->cur], h->prec == GP_F32, h->field == GP_COMPLEX, h->stream));
    FieldArgs a = handle_field_args(h);
    GP_CK(h, launch_norm(prec_of(h), h->field == GP_COMPLEX, a, kNormBlocks, h->stream));
    h->scale_pending = true;
    h->kick_pending = false;
    h->psi_lost = false;
    h->step = 0;
    h->t = 0.0;
    return GP_OK;
}

gp_status gp_set_graph_block(gp_handle h, int steps) {
    if (!h) return fail(h, GP_ERR_ARG, "NULL handle");
    if (steps < 0 || steps > 1024) return fail(h, GP_ERR_ARG, "steps must be in [0, 1024]");
    h->graph_block = steps;
    return GP_OK;
}

const char *gp_last_error(gp_handle h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

const char *gp_version(void) { return "gpcn 0.1 (sm_103a)"; }

}  // extern "C"

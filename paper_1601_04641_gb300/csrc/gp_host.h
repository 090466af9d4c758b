// gp_host.h -- host-side helpers shared by the single-condensate handle
// (gp_api.cu) and the batch handle (gp_batch.cu): FP64 precomputation of
// the CN recursion coefficients and trap factors, segment choice, and the
// argument blocks of the sweep and field kernels.
#pragma once

#include "gp_internal.h"

#include <string>
#include <vector>

namespace gpcn {

// One condensate's grid and physics.
struct Geometry {
    int n[3];
    double d[3];
    double dt, w[3], g;
};

// Byte offsets of one axis's tables inside a table buffer, and the smallest
// window that keeps the windowed back substitution exact to roundoff.
struct AxisTables {
    size_t off_cp = 0, off_ip = 0;
    int min_window = 0;   // 4, 8 or 16; 0 when none is admissible
    int t_const = 0;      // first index from which both stored tables are constant
    double cp_max = 0.0;
};

struct Tables {
    AxisTables ax[2][3];   // [mode: 0 imaginary, 1 real][axis]
    size_t kick_off[3] = {0, 0, 0};   // exp(-dt w^2 a^2 / 2) - 1 per node (imaginary time)
    size_t phase_off[3] = {0, 0, 0};  // dt w^2 a^2 / 2 per node (real time)
    size_t phase_half_off[3] = {0, 0, 0};  // the same for dt / 2 (symmetric splitting's half kick)
};

// Append the tables of G (modes = 1: imaginary time only, 2: both) to `host`
// (each table 256-byte aligned); offsets are relative to the start of host.
void append_tables(const Geometry &G, bool f32, int modes, std::vector<char> &host, Tables &T);

// Default window of an axis: the smallest admissible one in FP32 (bandwidth
// bound), the exact two-pass solve (0) in FP64 (ALU bound).
int default_window(const AxisTables &t, bool f32);

long long axis_lines(const Geometry &G, int ax);

// Interior nodes per segment and segment count of one axis.
void choose_segments(const Geometry &G, int ax, int window, int lpt, int elem_bytes, bool contiguous_z,
                     int override_len, int *seg_len, int *n_seg);

// Argument block of one sweep launch over G (ax = 0, 1, 2).
SweepArgs sweep_args(const Geometry &G, int ax, bool realtime, const void *in, void *out,
                     const char *tables, const Tables &T, int seg_len, int n_seg, const double *scale,
                     double *partials, unsigned int *counter, double *norm_out, double *scale_out,
                     bool half_kick = false);

// Argument block of the whole-field kernels over G.
FieldArgs field_args(const Geometry &G, const void *psi, const double *scale, double *partials,
                     unsigned int *counter, double *out, double *scale_out, double *norm_out);

size_t align_up(size_t x, size_t a);

}  // namespace gpcn

/*
 * gp.h -- C ABI of libgpcn: one GB300 GPU advancing the 3D Gross-Pitaevskii
 * (GP) equation in a fully anisotropic harmonic trap by split-step
 * Crank-Nicolson (CN) steps, in imaginary time (stationary states) or real
 * time (dynamics).
 *
 * What the calls compute.  The paper (arXiv:1601.04641, "New version program
 * summary", fields "Solution method" and "Method of solution" of program
 * summaries (i) imagtime3d and (ii) realtime3d) solves the time-dependent GP
 * equation by the split-step CN method, discretised in space and time and
 * propagated over small time steps.  Its "Summary of revisions" names the
 * stages of one step and the data layout; this library keeps both:
 *
 *   calcnu   potential + nonlinear step  psi <- exp(-dt (V + g|psi|^2)) psi
 *            (imaginary time) or exp(-i dt (V + g|psi|^2)) psi (real time),
 *            V = (gamma^2 x^2 + nu^2 y^2 + lambda^2 z^2) / 2;
 *   calclux, calcluy, calcluz
 *            CN line solves along x, y and z: for c = dt/(4 d^2) (imaginary
 *            time) or c = i dt/(4 d^2) (real time) every line solves
 *            -c phi[m-1] + (1+2c) phi[m] - c phi[m+1]
 *               = c psi[m-1] + (1-2c) psi[m] + c psi[m+1]
 *            on its interior nodes with psi = 0 on the two end nodes;
 *   renormalisation (imaginary time) psi <- psi / sqrt(dV sum |psi|^2);
 *   calcrms, calcmuen  rms radii, chemical potential mu and energy E.
 *
 * Layout (paper, "Summary of revisions"): psi is ONE array of nx*ny*nz
 * elements with z stride 1, y stride nz and x stride ny*nz.  An element is
 * a double or float (GP_REAL, imaginary time only) or an interleaved
 * (re, im) pair of doubles or floats (GP_COMPLEX).  Node (i, j, k) sits at
 * x = (i - (nx-1)/2) dx, y = (j - (ny-1)/2) dy, z = (k - (nz-1)/2) dz.
 *
 * Conventions.
 *  - Every call returns a gp_status; nothing throws across this boundary.
 *    On error, gp_last_error(h) (or gp_last_error(NULL) for a failed
 *    create) returns a message valid until the next call on that handle
 *    from the same thread.
 *  - Arguments are checked on the host: every n >= 3, spacings and dt > 0
 *    and finite, trap frequencies >= 0 and finite, g finite.  Otherwise
 *    GP_ERR_ARG and nothing is launched.
 *  - Work is queued on the handle's CUDA stream.  Calls that return values
 *    to the host (gp_observables, gp_get_psi to host memory,
 *    gp_run_imag_until) synchronise that stream; the step calls do not.
 *  - Line solves are out of place: the handle keeps psi in two device
 *    buffers and each sweep reads one and writes the other.  The first
 *    buffer is the caller's when the handle was made by gp_create_ext (the
 *    caller keeps it alive until gp_destroy); the second, and every other
 *    device buffer (CN coefficient tables, reduction partials, scalars),
 *    is owned by the handle.  gp_get_psi / gp_psi_device_ptr give the
 *    current psi whichever buffer holds it.
 *  - A handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef GPCN_GP_H
#define GPCN_GP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_handle_s *gp_handle; /* opaque, owned by the library */

typedef enum {
    GP_OK = 0,
    GP_ERR_ARG = 1,       /* invalid argument, nothing done */
    GP_ERR_CUDA = 2,      /* a CUDA call failed; the handle may be unusable */
    GP_ERR_NOMEM = 3,     /* a device or host allocation failed */
    GP_ERR_NONFINITE = 4, /* psi holds NaN or Inf at an observables check */
    GP_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    GP_ERR_STATE = 6,     /* call not valid in the handle's state (e.g. real
                             time on a GP_REAL field) */
    GP_ERR_IO = 7         /* a file could not be opened or written */
} gp_status;

typedef enum { GP_F64 = 0, GP_F32 = 1, GP_F16 = 2 } gp_precision; /* element precision of psi;
                                                                     reductions are always FP64 */
/* GP_F16: psi stored in IEEE half precision (2 bytes a site) with every
 * operation in FP32 -- the sweeps, the kick and the observables widen on
 * load and round to nearest on store; the norm that sets the
 * renormalisation is summed from the FP32 results before rounding.  A
 * precision variant of the imaginary-time path (the paper computes in FP64
 * throughout): GP_REAL fields only, nz a multiple of 8 and at least 56 (the
 * z sweep is the TMA form, a chunk of 32 nodes plus its window), windowed
 * solves with two or four lines per thread on x and y (calls that would
 * select another form return GP_ERR_ARG).  Each sweep rounds psi to 2^-11
 * relative: where a step changes psi by less than that (dt small against
 * 2^-11 / (gap of the low modes)) the evolution stalls short of the ground
 * state, and the fixed point sits far from FP32's -- on the 640x480x400
 * benchmark grid mu was 4.7 % high after 250 steps at dt = 0.1 d^2 and
 * 0.2 % at dt = d^2.  A coarse stage at a large dt before an FP32 or FP64
 * finish.  gp_density_profiles, gp_write_wavefunction, gp_nn_predict, the
 * batched form and gp_observables_noalloc do not take it. */
typedef enum { GP_COMPLEX = 0, GP_REAL = 1 } gp_field;

typedef struct {
    int nx, ny, nz;       /* nodes per axis: nx >= 3; ny, nz >= 3, or 1 for an
                             absent axis (see below) */
    double dx, dy, dz;    /* spacings, > 0 (ignored for an absent axis) */
} gp_grid;

/* Lower-dimensional condensates (the 1D and 2D programs of the paper's
 * predecessor package, on which the 3D programs build): a y or z axis of
 * one node is absent.  It has no line solve, no links and no boundary
 * nodes, its coordinate is 0 (its trap frequency does not enter), and it
 * adds no spacing to the cell measure dV, so the norm is the 1D or 2D
 * integral and g is the 1D or 2D coupling of the same equation in the
 * present coordinates.  1D: (nx, 1, 1); 2D: (nx, ny, 1) or (nx, 1, nz) --
 * the latter keeps the stride-1 axis present, which the z sweep's TMA form
 * needs.  With nz = 1 the z stage of imaginary time is a norm reduction
 * only.  The single-condensate calls take these grids; the batched form and
 * gp_observables_noalloc take 3D grids. */

/* Observables of the current psi (paper, "Summary of revisions": norm,
 * rms radii from calcrms, chemical potential and energy from calcmuen),
 * with rectangle sums and forward-difference links:
 *   norm  = dV sum |psi|^2
 *   K     = (1/2) dV sum_axes sum_links |psi[m+1]-psi[m]|^2 / d^2
 *   P     = dV sum V |psi|^2,  I = dV sum |psi|^4
 *   mu    = (K + P + g I) / norm,  energy = (K + P + g I / 2) / norm
 *   rms_a = sqrt(dV sum a^2 |psi|^2 / norm). */
typedef struct {
    double norm, mu, energy, rms_x, rms_y, rms_z;
    long long step; /* steps taken since create / the last gp_set_psi */
    double t;       /* imaginary or real time advanced, sum of dt */
} gp_obs;

/* Create a solver for one condensate.  grid: nodes and spacings; dt: time
 * step; gamma, nu, lambda: trap frequencies along x, y, z; g: nonlinearity.
 * prec / field select the element type of psi (GP_REAL allows imaginary
 * time only).  cuda_stream: a cudaStream_t to queue work on, or NULL for the
 * legacy default stream.  psi is allocated on the current CUDA device and
 * zero-filled.  On success *out holds the handle. */
gp_status gp_create(gp_handle *out, gp_grid grid, double dt, double gamma, double nu,
                    double lambda, double g, gp_precision prec, gp_field field,
                    void *cuda_stream);

/* As gp_create, but psi lives in the caller's device buffer dev_psi of
 * `bytes` bytes (at least nx*ny*nz elements, 16-byte aligned), which the
 * caller keeps alive until gp_destroy.  Its contents are kept as they are
 * (taken as psi with no pending scale). */
gp_status gp_create_ext(gp_handle *out, gp_grid grid, double dt, double gamma, double nu,
                        double lambda, double g, gp_precision prec, gp_field field,
                        void *cuda_stream, void *dev_psi, size_t bytes);

/* Free every buffer the handle owns (not a gp_create_ext psi).  NULL is a no-op. */
void gp_destroy(gp_handle h);

/* psi <- the product Gaussian prod_a (w_a/pi)^(1/4) exp(-w_a a^2/2), zero on
 * the boundary nodes, normalised so that dV sum |psi|^2 = 1 (the g = 0
 * ground state of the continuum problem); resets step and t. */
gp_status gp_init_gaussian(gp_handle h);

/* Copy psi in (host memory if on_device == 0, device memory otherwise) in
 * the handle's element type and layout; resets step and t.  The caller
 * keeps ownership of the source. */
gp_status gp_set_psi(gp_handle h, const void *psi, int on_device);

/* Copy the current psi out (any pending renormalisation applied). */
gp_status gp_get_psi(gp_handle h, void *psi, int on_device);

/* Change g (a quench); the CN coefficients do not depend on g. */
gp_status gp_set_g(gp_handle h, double g);

/* Change dt; rebuilds the CN coefficient tables. */
gp_status gp_set_dt(gp_handle h, double dt);

/* Queue nsteps imaginary-time steps: kick, x, y and z line solves, then
 * renormalisation (applied lazily by the next read of psi). */
gp_status gp_step_imag(gp_handle h, int nsteps);

/* Queue nsteps real-time steps (GP_COMPLEX only): kick, x, y, z line solves. */
gp_status gp_step_real(gp_handle h, int nsteps);

/* Splitting of the real-time step: 1 (default) the program summary's order,
 * kick then the x, y and z line solves (first order in dt); 2 the symmetric
 * form, half kick, line solves, half kick (second order, time-reversible).
 * With order 2 consecutive steps share their half kicks (a real-time kick
 * keeps |psi|, so two half kicks are one full kick), and the trailing half
 * kick of the last step is applied when psi is next read or changed
 * (gp_get_psi, gp_psi_device_ptr, gp_observables, tracking records,
 * gp_set_g, gp_set_dt, imaginary-time steps).  Imaginary time always uses
 * order 1.  gp_step_stage runs the order-1 stages. */
gp_status gp_set_splitting(gp_handle h, int order);

/* Imaginary-time propagation until |mu(n) - mu(n - check_every)| < mu_tol,
 * checking every check_every steps, or max_steps.  *steps_taken (may be
 * NULL) receives the number of steps.  Synchronises at every check. */
gp_status gp_run_imag_until(gp_handle h, double mu_tol, int check_every, int max_steps,
                            int *steps_taken);

/* Imaginary time through `levels` steps: level l sets dt to the current dt
 * times dt_scale[l] (coefficients rebuilt) and runs gp_run_imag_until with
 * mu_tol[l]; dt is restored afterwards.  CN is stable at any dt and each
 * dt's fixed point differs from the next by O(dt^2) in mu, so converging at a
 * coarse dt first and finishing at the target dt (last level scale 1) reaches
 * the target's fixed point in fewer steps than starting there.  max_steps
 * bounds each level; *steps_taken (may be NULL) is their sum. */
gp_status gp_run_imag_schedule(gp_handle h, int levels, const double *dt_scale, const double *mu_tol,
                               int check_every, int max_steps, int *steps_taken);

/* Stop rule of gp_run_imag_until: 0 (default) |mu(n) - mu(n-K)| < mu_tol,
 * the program summary's convergence test on the chemical potential; 1 also
 * requires |E(n) - E(n-K)| < mu_tol.  mu is not variational: from a start
 * close to the ground state it can turn around on its way in, and at the
 * turning point its change between checks drops below the tolerance long
 * before convergence.  E decreases monotonically in imaginary time, so rule 1
 * stops only where both have settled.  2 requires rule 1's condition at two
 * consecutive checks: after a change of dt (a schedule's next level) mu and
 * E approach their new values along several modes at once, and a single
 * check can fall between a sign change of their differences.  No effect on
 * the steps themselves; GP_ERR_ARG for another rule. */
gp_status gp_set_stop_rule(gp_handle h, int rule);

/* Compute the observables of the current psi into *out (synchronises).
 * GP_ERR_NONFINITE if any reduction is NaN or Inf.  GP_ERR_TIMEOUT if the
 * FP32 observables kernel gave up waiting for its bulk copies (each wait is
 * bounded to about a second): *out is then invalid, psi is unchanged and
 * usable; or if a sweep kernel's wait expired since the last check (see
 * gp_sync). */
gp_status gp_observables(gp_handle h, gp_obs *out);

/* Track observables during stepping: after every `every` steps of
 * gp_step_imag / gp_step_real (counted by the handle's step counter) the
 * observables reduction is queued on the stream, with no host
 * synchronisation, into a device history of `capacity` records (the norm
 * and energy drift of a real-time run).  every = 0 turns tracking off.
 * Resets the history. */
gp_status gp_set_tracking(gp_handle h, int every, int capacity);

/* Copy up to max tracked records (oldest first) into out[] and their count
 * into *count (synchronises).  GP_ERR_NONFINITE if a record is non-finite. */
gp_status gp_get_tracking(gp_handle h, gp_obs *out, int max, int *count);

/* Run one stage of a step by itself (stage 0: kick + x line solve; 1: y
 * line solve; 2: z line solve, whose imaginary-time form also sets the
 * pending renormalisation).  realtime selects the real-time forms.  Stages
 * 0, 1, 2 in order are exactly one step.  For tests of single stages. */
gp_status gp_step_stage(gp_handle h, int stage, int realtime);

/* Queue all work on a new stream (a cudaStream_t, NULL for the legacy
 * default stream). */
gp_status gp_set_stream(gp_handle h, void *cuda_stream);

/* Block until the handle's queued work is done.  Returns GP_ERR_TIMEOUT if a
 * sweep kernel gave up waiting for its TMA copies (each wait is bounded to
 * about a second); gp_observables reports the same.  psi is then undefined
 * -- lines of other blocks of that launch included, since a copy may land
 * after its block has exited -- and every call that reads or advances psi
 * returns GP_ERR_STATE until gp_set_psi, gp_init_gaussian or gp_nn_predict
 * sets it again. */
gp_status gp_sync(gp_handle h);

/* Window of the windowed back substitution per axis for imaginary (mode 0)
 * or real (mode 1) time; 0 means the exact two-pass solve is used.  By
 * default FP32 fields use the smallest admissible window and FP64 fields the
 * exact solve (FP64 arithmetic, not memory, bounds the FP64 forms). */
gp_status gp_get_window(gp_handle h, int mode, int window[3]);

/* Override the window of every axis and mode: -1 restores the automatic
 * choice, 0 forces the exact two-pass solve, 4 / 8 / 16 force that window
 * (GP_ERR_ARG if it is below the smallest window that keeps the truncation
 * within half the unit roundoff for this dt). */
gp_status gp_set_window(gp_handle h, int window);

/* Window of one axis in both modes (-1 automatic, 0 exact, 4 / 8 / 16 if
 * admissible for that axis). */
gp_status gp_set_axis_window(gp_handle h, int axis, int window);

/* Several adjacent lines per thread on the strided axes (1, the default:
 * the widest group the layout and form allow) or one line per thread (0).
 * A group of g lines needs the axis's line count, and for the y sweep nz, to
 * be a multiple of g.  Pairs serve elements of up to 8 bytes; groups of four
 * serve FP32 real fields with a windowed solve, so that each row a warp
 * moves is 512 contiguous bytes.  The arithmetic per line is the same. */
gp_status gp_set_pair_lines(gp_handle h, int on);

/* The most adjacent lines per thread on one strided axis (axis 0 = x,
 * 1 = y; lines 1, 2 or 4; default 4), within the rules of gp_set_pair_lines.
 * GP_ERR_ARG for another axis or count. */
gp_status gp_set_lines_per_thread(gp_handle h, int axis, int lines);

/* Lines per thread each axis's sweep uses in `mode` (0 imaginary, 1 real
 * time) under the current settings (the z sweep always reports 1). */
gp_status gp_get_lines_per_thread(gp_handle h, int mode, int lines[3]);

/* The z sweep (stride-1 axis) through tensor-memory-accelerator tiles: one
 * bulk tensor copy per 64 lines x 64 bytes, two lines per thread (1, the
 * default), or through per-thread asynchronous copies (0).  The TMA form is
 * taken where the rows allow it: 2-, 4- or 8-byte elements, nz * element
 * size a multiple of 16 bytes, a window > 0 with (chunk + window) pair
 * values in at most 256 bytes (chunk = 64 bytes of nodes: every window for
 * FP16 and FP32 real fields, windows 4 and 8 for 8-byte elements), whole
 * lines, and nz - 2 at least one chunk plus the window plus 2; elsewhere
 * the other form runs (GP_F16 handles take only the TMA form).
 * The arithmetic per line is the same in both.  gp_get_tma reports whether
 * the z sweep of imaginary time, or (complex fields) of real time, takes the
 * TMA form under the current settings: selected, tensor maps encoded for the
 * handle's buffers, and the conditions above met. */
gp_status gp_set_tma(gp_handle h, int on);
gp_status gp_get_tma(gp_handle h, int *in_use);

/* The x and y sweeps (strided axes) reading through tensor-memory-
 * accelerator boxes: `axes` is a mask, bit 0 for x and bit 1 for y, in both
 * modes; -1 (the default) takes x for real fields (imaginary time) and
 * neither axis for complex fields.  An axis outside the mask reads through
 * per-thread asynchronous copies.  A warp streams 32 adjacent line groups
 * (1, 2 or 4 lines each, as gp_set_lines_per_thread gives) in boxes of one
 * chunk of nodes x 32 groups, one bulk tensor copy each; the last warp of a
 * plane (x) or of a row of a plane (y) may be partial.  Results are stored by the threads in both
 * forms.  The TMA form is taken where a windowed solve runs (window > 0) and
 * a line's node stride is a multiple of 16 bytes (ny * nz * element size
 * for x, nz * element size for y); elsewhere the other form runs.  Both
 * forms do the same arithmetic in the same order, so their results are
 * identical.  Measured inside full steps: it shortens the x sweep of real
 * fields (FP32 on 480x400x320 0.1076 -> 0.1067 ms, FP16 on 640x480x400
 * 0.371 -> 0.348 ms), and lengthens the complex64 x sweeps (imaginary time
 * 0.1740 -> 0.1746, real time 0.170 -> 0.173 ms) and the y sweeps (FP32
 * real 0.082 -> 0.086 ms in isolation).  gp_get_tma_lines gives the axes
 * that take it in either mode under the current settings (bit 0: x, bit 1:
 * y); GP_ERR_ARG for a mask outside -1..3. */
gp_status gp_set_tma_lines(gp_handle h, int axes);
gp_status gp_get_tma_lines(gp_handle h, int *axes);

/* Threads per block of the line-solve kernel of one axis (multiple of 32,
 * 32..256). */
gp_status gp_set_threads(gp_handle h, int axis, int threads);

/* Interior nodes per segment of the line solves of one axis (0 = the
 * automatic choice).  Lines are cut into segments, one thread each, that
 * warm their forward sweep up over the W+1 nodes before the segment. */
gp_status gp_set_segments(gp_handle h, int axis, int seg_len);

/* Segment length and count per axis that the next imaginary- (mode 0) or
 * real-time (mode 1) step will use. */
gp_status gp_get_segments(gp_handle h, int mode, int seg_len[3], int n_seg[3]);

/* Autotuner: for each axis, time the line-solve kernel of the imaginary-
 * (realtime = 0) or real-time (1) step on this handle's grid under every
 * candidate launch setting -- threads per block (64, 128), segment length
 * (automatic, 64, 128, 256, whole line) and one or two lines per thread --
 * with CUDA events over `reps` launches after a warm-up, and keep the
 * fastest.  psi is left unchanged (the trials run on a copy).  Choices are
 * cached as text lines "key threads seg pair" in cache_path (NULL: the
 * GP_AUTOTUNE_CACHE environment variable; unset: no cache); a cached key is
 * applied without timing.  Synchronises. */
gp_status gp_autotune(gp_handle h, int realtime, int reps, const char *cache_path);

/* Steps per CUDA graph: gp_step_imag / gp_step_real capture blocks of this
 * many steps into a graph once and replay it (default 16; 0 or 1 launches
 * kernel by kernel).  With tracking on, blocks are track_every steps long.
 * Changing g, dt, the window, threads, segments or the splitting
 * re-captures. */
gp_status gp_set_graph_block(gp_handle h, int steps);

/* Device pointer of the buffer that holds the current psi, and whether a
 * renormalisation factor is still pending on it (the value is then psi
 * times that factor; gp_get_psi applies it).  A pending half kick of the
 * symmetric splitting is applied first (queued on the stream).  Valid until
 * the next call that queues work on the handle. */
gp_status gp_psi_device_ptr(gp_handle h, void **ptr, int *pending_scale);

/* The renormalisation factor pending on the buffer gp_psi_device_ptr gives
 * (1.0 when none is pending): psi is that buffer times *scale.  Synchronises
 * the handle's stream.  A caller that reads the buffer directly -- e.g.
 * gp_observables_noalloc after imaginary-time steps -- passes this factor as
 * the read scale. */
gp_status gp_pending_scale(gp_handle h, double *scale);

/* Density output.  The paper's programs write the condensate wavefunction
 * to files ("Special features": each MPI process writes its part, and the
 * parts concatenated give the whole wavefunction); on one GPU the whole
 * wavefunction is one array, and these two calls give it and its integrated
 * densities.
 *
 * Integrated 1D densities of the current psi:
 *   rho_x[i] = dy dz sum_{j,k} |psi_ijk|^2   (nx values)
 *   rho_y[j] = dx dz sum_{i,k} |psi_ijk|^2   (ny values)
 *   rho_z[k] = dx dy sum_{i,j} |psi_ijk|^2   (nz values)
 * so that sum_i rho_x[i] dx is the norm (gp_obs.norm).  A pending
 * renormalisation factor s enters as s^2; a pending half kick of the
 * symmetric splitting is a phase and does not change |psi|^2.  Host arrays,
 * caller-owned; any of them may be NULL (not computed).  Computed on the
 * GPU in FP64 with every sum in a fixed order (deterministic), using
 * (nx ny + nx nz + nx + ny + nz) doubles of device scratch allocated for the
 * call (GP_ERR_NOMEM if that fails); synchronises the handle's stream. */
gp_status gp_density_profiles(gp_handle h, double *rho_x, double *rho_y, double *rho_z);

typedef enum { GP_OUT_PSI = 0, GP_OUT_DENSITY = 1 } gp_output;

/* Write the current psi (GP_OUT_PSI: the element type of the handle) or its
 * density |psi|^2 (GP_OUT_DENSITY: float or double, computed in FP64 from
 * the stored values and rounded once to the handle's precision) to `path` as
 * a NumPy .npy file (format version 1.0, little-endian, C order, shape
 * (nx, ny, nz): the layout above).  Pending factors are applied as by
 * gp_get_psi.  Needs one host buffer of the array's size (GP_ERR_NOMEM if it
 * cannot be allocated); GP_ERR_IO if the file cannot be opened or fully
 * written (a partly written file is removed); synchronises the stream. */
gp_status gp_write_wavefunction(gp_handle h, const char *path, int what);

/* Observables of a caller-owned device psi, computed without allocating any
 * device memory.  No counterpart in the paper: it serves callers that cannot
 * call cudaMalloc -- a host framework that owns all device memory through its
 * own pool, or a latency-critical loop that must not pay cudaMalloc's
 * implicit device synchronisation.  (A handle cannot serve them: gp_create
 * allocates.)
 *   dev_psi  device array of nx*ny*nz elements in the layout above, of the
 *            type given by prec / field; read only; values are multiplied by
 *            `scale` as they are read.
 *   dev_out  device array of 16 doubles written by the kernel: [0..8] the raw
 *            sums (|psi|^2, V|psi|^2, |psi|^4, x^2|psi|^2, y^2|psi|^2,
 *            z^2|psi|^2, and the squared differences along x, y, z), [9..14]
 *            norm, mu, energy, rms_x, rms_y, rms_z as in gp_obs, [15] 1.0 if
 *            all of them are finite, else 0.0.
 *   cuda_stream  stream to queue on (NULL: legacy default stream); the call
 *            returns without synchronising.
 * The reduction's block partials and completion counter live in one
 * fixed-size static device array (about 576 KB, held by every GPU that loads
 * the library until the process exits), so ny*nz may be at most 2,097,152;
 * larger planes return GP_ERR_ARG with a message in gp_last_error(NULL).  The
 * first call on each device looks the array's device address up (make it
 * before any stream capture on that device).  All calls share the array:
 * calls whose work overlaps on the GPU race and give undefined results.
 * Other arguments are checked like gp_create's. */
gp_status gp_observables_noalloc(const void *dev_psi, gp_grid grid, gp_precision prec,
                                 gp_field field, double gamma, double nu, double lambda, double g,
                                 double scale, double *dev_out, void *cuda_stream);

/* ------------------------------------------------------------------ batch
 * Many independent condensates -- each with its own grid, spacings, dt,
 * trap and g (the paper's programs run one condensate each) -- advanced in
 * imaginary time together: each step is one launch per sweep and stream
 * group (gp_batch_set_streams) covering that group's active instances (two
 * on a strided axis at window 4 with complex64 fields: instances whose
 * lines pair up in memory advance line pairs; two on the z axis when some
 * instances' rows fit the TMA form of gp_set_tma and others do not), with
 * per-instance arguments, norm partials and counters; blocks of steps are
 * replayed from CUDA graphs, and gp_batch_run_imag_until drops converged
 * instances from the launches.  All
 * instances share one precision and field; each axis uses one window for the
 * whole batch (the largest of the instances' smallest admissible windows;
 * the exact solve in FP64).  psi of instance i has the layout above. */
typedef struct gp_batch_s *gp_batch;

gp_status gp_batch_create(gp_batch *out, int n, const gp_grid *grids, const double *dt,
                          const double *gamma, const double *nu, const double *lambda,
                          const double *g, gp_precision prec, gp_field field, void *cuda_stream);
void gp_batch_destroy(gp_batch b);
/* Every instance <- its normalised Gaussian (as gp_init_gaussian). */
gp_status gp_batch_init_gaussian(gp_batch b);
gp_status gp_batch_set_psi(gp_batch b, int i, const void *psi, int on_device);
gp_status gp_batch_get_psi(gp_batch b, int i, void *psi, int on_device);
/* nsteps imaginary-time steps of every instance. */
gp_status gp_batch_step_imag(gp_batch b, int nsteps);
/* Observables of every instance into out[0..n-1] (synchronises). */
gp_status gp_batch_observables(gp_batch b, gp_obs *out);
/* Imaginary time until |mu(n) - mu(n - check_every)| < mu_tol per instance
 * (checked every check_every steps; converged instances stop stepping), or
 * max_steps.  steps_taken[i] (may be NULL) receives each instance's steps. */
gp_status gp_batch_run_imag_until(gp_batch b, double mu_tol, int check_every, int max_steps,
                                  int *steps_taken);
/* Stop rule of gp_batch_run_imag_until, as gp_set_stop_rule. */
gp_status gp_batch_set_stop_rule(gp_batch b, int rule);
/* Every instance steps with its creation dt times `scale` (tables, windows
 * and segments rebuilt; psi kept). */
gp_status gp_batch_set_dt_scale(gp_batch b, double scale);
/* As gp_run_imag_schedule, for every instance (scales relative to the
 * current scale, which is restored afterwards); steps_taken[i] per instance. */
gp_status gp_batch_run_imag_schedule(gp_batch b, int levels, const double *dt_scale, const double *mu_tol,
                                     int check_every, int max_steps, int *steps_taken);
/* The window per axis used for the whole batch. */
gp_status gp_batch_get_window(gp_batch b, int window[3]);
/* Segment length and count per axis of instance i. */
gp_status gp_batch_get_segments(gp_batch b, int i, int seg_len[3], int n_seg[3]);
/* Interior nodes per segment on the strided axes (x, y) of every instance
 * (seg_len >= 1, at most the line; 0, the default: about 128, in whole
 * chunks), for windowed solves.  Shorter segments give more threads per line
 * at the cost of W + 1 warm-up nodes per segment; psi is the same to
 * roundoff.  GP_ERR_ARG for seg_len < 0. */
gp_status gp_batch_set_segments(gp_batch b, int seg_len);
/* Steps per CUDA graph (default 16; 0 or 1: launch by launch). */
gp_status gp_batch_set_graph_block(gp_batch b, int steps);
/* Stream groups of a batched step (1..16, default 2): the active instances
 * are split into groups balanced by sites, and each group's x, y and z
 * sweeps run as one chain of launches on a stream of its own, forked from
 * and joined back into the batch's stream (and captured into its graphs as
 * parallel branches), so launches of different groups overlap.  psi is the
 * same for every setting. */
gp_status gp_batch_set_streams(gp_batch b, int streams);
/* z sweep of the instances whose rows fit the TMA form (the rules of
 * gp_set_tma, at the batch's z window; at most 64 instances, the first ones
 * in creation order) through TMA tiles (1, the default) or every instance
 * through per-thread copies (0).  Each TMA instance gets its own tensor maps;
 * the arithmetic per line, and so psi, is the same either way; norms may
 * differ by rounding (the two forms group the norm's sums differently).
 * gp_batch_get_tma gives the number of instances on the TMA form. */
gp_status gp_batch_set_tma(gp_batch b, int on);
gp_status gp_batch_get_tma(gp_batch b, int *count);
/* Last error of the batch (NULL: as gp_last_error(NULL)). */
const char *gp_batch_last_error(gp_batch b);

/* ------------------------------------------------------------------ warm start
 * A learned initial state for imaginary time (no counterpart in the paper,
 * which starts from a Gaussian): a conditioned coordinate MLP maps a grid
 * node x of a condensate with trap (gamma, nu, lambda) and nonlinearity g to
 * an amplitude.  Features: min(w_a x_a^2, 16)/8 - 1 per axis (even in x_a,
 * so every prediction is even, as the ground state is); min(sum (x_a/R_a)^2, 4)/2 - 1
 * with the Thomas-Fermi radii R_a = sqrt(2 mu_TF)/w_a, mu_TF =
 * (15 g w_x w_y w_z / 4 pi)^(2/5)/2; min(sum w_a x_a^2, 16)/8 - 1;
 * (ln g - 3.1)/3.1; (w_a - 1.75)/1.25 (9 used, padded to 16).  Layers: three
 * 64-wide tanh layers, then softplus(h . w3 + b3).  Parameters, FP32 master,
 * in this order ([in][out] row-major): W0 16x64, b0, W1 64x64, b1, W2 64x64,
 * b2, w3 64, b3 (gp_nn_param_count() floats).  Forward, backward and the
 * Adam step run on the GPU; the matrix layers use BF16 tensor-core
 * operands with FP32 accumulation. */
typedef struct gp_nn_s *gp_nn;

int gp_nn_param_count(void);
/* Glorot-uniform weights from SplitMix64(seed), zero biases. */
gp_status gp_nn_create(gp_nn *out, unsigned long long seed, void *cuda_stream);
void gp_nn_destroy(gp_nn net);
/* Set / get the FP32 master parameters (host arrays of gp_nn_param_count()).
 * Setting resets the Adam state. */
gp_status gp_nn_set_params(gp_nn net, const float *params, int count);
gp_status gp_nn_get_params(gp_nn net, float *params, int count);
/* Training set: n condensates (grid, trap, g) whose target amplitudes are
 * float32 arrays in the psi layout inside the caller's device buffer
 * dev_data (kept alive by the caller), instance i at element offsets[i];
 * the target of a node is its amplitude divided by psi_max[i]. */
gp_status gp_nn_set_data(gp_nn net, int n, const gp_grid *grids, const double *gamma,
                         const double *nu, const double *lambda, const double *g,
                         const float *dev_data, const long long *offsets, const float *psi_max);
/* `steps` Adam steps (learning rate lr) on the mean squared error of
 * `points` nodes per step (a multiple of 128) drawn uniformly over the
 * instances and their nodes by SplitMix64 from seed; *loss (may be NULL)
 * receives the last step's loss. */
gp_status gp_nn_train(gp_nn net, int steps, int points, float lr, unsigned long long seed, float *loss);
/* Loss and gradient (host array of gp_nn_param_count()) on explicit samples
 * (instance index, node index), count a multiple of 128; no update. */
gp_status gp_nn_loss_grad(gp_nn net, int count, const int *instance, const long long *site,
                          float *loss, float *grad);
/* psi <- the network's prediction on the handle's grid (boundary nodes 0),
 * normalised; resets step and t. */
gp_status gp_nn_predict(gp_nn net, gp_handle h);
/* The same for every instance of a batch. */
gp_status gp_nn_predict_batch(gp_nn net, gp_batch b);
const char *gp_nn_last_error(gp_nn net);

/* Last error message for this handle (or for the calling thread's last
 * failed create, or failed gp_observables_noalloc, when h is NULL).  Never
 * NULL. */
const char *gp_last_error(gp_handle h);

/* ---- axially symmetric condensates ----
 * psi(rho, z) for a trap with gamma = nu: the (rho, z) program variant of
 * the predecessor package the paper's programs extend.  The equation is the
 * 3D one (i dpsi/dt = [-(1/2) lap + V + g |psi|^2] psi, V = (gamma^2 rho^2 +
 * lambda^2 z^2) / 2, int 2 pi rho |psi|^2 drho dz = 1) for states without
 * circulation.  Grid psi[i][k] (k, along z, has stride 1; a C array of
 * shape (nx, nz)): radial node i = 1..nx-2 at rho = (i - 1/2) drho, node 0 a
 * ghost (read as 0, written 0), node nx-1 the Dirichlet boundary; z nodes
 * z_k = (k - (nz-1)/2) dz with psi = 0 at k = 0 and nz-1.  The radial line
 * solve is the CN step of the finite-volume operator (1/rho) d/drho (rho
 * d/drho) with face radii rho_{i +- 1/2} (no flux through the axis); a step
 * is kick, radial solves, z solves, and in imaginary time the
 * renormalisation in the cylindrical measure 2 pi rho drho dz.  Observables
 * are the discrete Rayleigh quotient of this operator; gp_obs.rms_x and
 * rms_y are both sqrt(<rho^2> / 2).  FP64 or FP32 fields (arithmetic in
 * the field's precision, sums in FP64), real (imaginary time only) or
 * complex.  gp_axial_create: nx, nz >= 3; drho, dz, dt, gamma, lambda > 0,
 * g finite, prec GP_F64 or GP_F32; GP_ERR_ARG otherwise, GP_ERR_CUDA
 * without a CUDA device, GP_ERR_NOMEM if device memory runs out.  psi
 * buffers of set/get hold nx * nz elements (host or device, as on_device
 * says; the caller owns them).  gp_axial_run_imag_until: the stop rule
 * |mu(n) - mu(n - check_every)| < mu_tol, at most max_steps steps. */
typedef struct gp_axial_s *gp_axial;
gp_status gp_axial_create(gp_axial *out, int nx, int nz, double drho, double dz, double dt, double gamma,
                          double lambda, double g, gp_precision prec, gp_field field, void *cuda_stream);
void gp_axial_destroy(gp_axial a);
const char *gp_axial_last_error(gp_axial a);
gp_status gp_axial_init_gaussian(gp_axial a);
gp_status gp_axial_set_psi(gp_axial a, const void *psi, int on_device);
gp_status gp_axial_get_psi(gp_axial a, void *psi, int on_device);
gp_status gp_axial_step_imag(gp_axial a, int nsteps);
gp_status gp_axial_step_real(gp_axial a, int nsteps);
gp_status gp_axial_observables(gp_axial a, gp_obs *out);
gp_status gp_axial_run_imag_until(gp_axial a, double mu_tol, int check_every, int max_steps, int *steps_taken);

/* ---- failure-detection self-tests (no counterpart in the paper) ----
 * gp_selftest_bounded_wait launches one warp on the given stream that waits,
 * with the bounded mbarrier wait the TMA sweep uses, on an mbarrier whose
 * phase completes (*completed = 1 expected) and on one that nothing arrives
 * at, giving up after `cycles` clock cycles (*expired = 1 expected).  Nothing
 * is copied and the kernel ends within about 2 * cycles; synchronises.
 * gp_debug_fail_alloc(n) makes the n-th next device allocation of the library
 * fail as if the device were out of memory (n <= 0: no failure); every
 * creating call then returns GP_ERR_NOMEM and frees what it had allocated.
 * gp_debug_raise_status(h, bits) or-s `bits` into the handle's device status
 * word from the host, as a kernel does when a bounded wait expires (nothing
 * waits or faults on the device): 1 as a sweep kernel does, 2 as the
 * observables kernel does (3: both); GP_ERR_ARG for other bits.  The next
 * synchronising call reports GP_ERR_TIMEOUT; with bit 1, psi is lost until
 * set again (see gp_sync); with bit 2 alone, only the observables computed
 * since are invalid and psi stays usable. */
gp_status gp_selftest_bounded_wait(long long cycles, void *cuda_stream, int *completed, int *expired);
void gp_debug_fail_alloc(int n);
gp_status gp_debug_raise_status(gp_handle h, unsigned int bits);

/* Library version string. */
const char *gp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GPCN_GP_H */

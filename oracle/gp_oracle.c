/*
 * gp_oracle.c -- plain FP64 CPU oracle for the split-step Crank-Nicolson (CN)
 * propagation of the 3D Gross-Pitaevskii (GP) equation in a fully anisotropic
 * harmonic trap.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  It is the parity authority for the
 * CUDA path and shares no code, header, table or constant with it.  Only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg load it.
 * It is deliberately slow: every stage runs over the whole grid in the order
 * the method states, every line solve is the textbook Thomas algorithm with
 * its own per-line elimination, and complex numbers are C99 `double complex`.
 *
 * Source of the method.  The paper ("New version program summary", fields
 * "Solution method" and "Method of solution" of program summaries (i) and
 * (ii)) states that the time-dependent GP equation is discretised in space
 * and time and propagated over small time steps by the split-step CN method,
 * in imaginary time (stationary states) or real time (dynamics).  Its
 * "Summary of revisions" names the numerical stages: calcnu (potential and
 * nonlinear step), calclux / calcluy / calcluz (CN line solves along x, y and
 * z), renormalisation and norm, calcrms (rms radii) and calcmuen (chemical
 * potential and energy), and fixes the wavefunction layout: one 1D array in
 * which z has stride 1, y stride Nz and x stride Ny*Nz.  The paper prints no
 * equation; the readings of the method taken here, numbered as they are
 * cited elsewhere in this repository, are:
 *
 *   R1  i dpsi/dt = [-(1/2) lap + V + g |psi|^2] psi,
 *       V = (gamma^2 x^2 + nu^2 y^2 + lambda^2 z^2) / 2,  int |psi|^2 = 1,
 *       so that at g = 0 the ground-state chemical potential is
 *       (gamma + nu + lambda) / 2.
 *   R2  nodes x_i = (i - (N-1)/2) d, i = 0..N-1 (trap centred in the box).
 *   R3  Dirichlet boundary: psi = 0 on the outermost nodes of every axis;
 *       boundary values are never read by a line solve and are written 0.
 *   R4  observables are rectangle sums with forward-difference links
 *       (the exact discrete Rayleigh quotient of the CN Laplacian).
 *   R5  first-order (Lie) splitting: kick, then x, y, z sweeps, each with
 *       the full dt; imaginary time then renormalises.
 *   R20 lower-dimensional condensates (the 1D and 2D programs of the
 *       predecessor package): an axis with a single node is absent.  It
 *       has no line solve, no links and no boundary nodes, its coordinate
 *       is 0 (so it adds nothing to V), and the cell measure dV is the
 *       product of the present axes' spacings; g is then the 1D or 2D
 *       coupling of the same equation R1 in the present coordinates.
 *
 * Imaginary time uses t -> -i tau, so the kick is exp(-dt (V + g|psi|^2))
 * and each sweep is CN for dpsi/dtau = (1/2) d^2 psi / dx^2; real time uses
 * the kick exp(-i dt (V + g|psi|^2)) and CN for i dpsi/dt = -(1/2) d^2 psi/dx^2.
 * With c = dt / (4 d^2) (imaginary time) or c = i dt / (4 d^2) (real time),
 * the CN line equation at interior node m is
 *     -c phi[m-1] + (1 + 2c) phi[m] - c phi[m+1]
 *         = c psi[m-1] + (1 - 2c) psi[m] + c psi[m+1].
 *
 * Every entry point returns 0 on success, -1 on bad arguments, -2 when an
 * allocation fails, -3 on a zero pivot.  Arrays of complex values are passed
 * as interleaved (re, im) doubles.
 *
 * The kick's sites and the sweeps' lines are independent, so their loops
 * carry OpenMP work-sharing pragmas: a build with -fopenmp spreads them over
 * the host cores (each site and each line computed exactly as in the serial
 * build, so the two builds agree bit for bit); a build without it ignores
 * them.  Every sum (norm, observables) stays a serial loop in a fixed order.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

typedef double complex cplx;

#define ORACLE_OK 0
#define ORACLE_EARG (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_EPIVOT (-3)

/* Offset of node (i, j, k): z stride 1, y stride Nz, x stride Ny*Nz
 * (paper, "Summary of revisions", layout of the psi array). */
static size_t site(const int n[3], int i, int j, int k)
{
    return ((size_t)i * (size_t)n[1] + (size_t)j) * (size_t)n[2] + (size_t)k;
}

/* Node coordinate along one axis (reading R2). */
static double node_coord(int idx, int n, double d)
{
    return ((double)idx - 0.5 * (double)(n - 1)) * d;
}

static int valid_grid(const int n[3], const double d[3])
{
    int present = 0;
    for (int a = 0; a < 3; a++) {
        if ((n[a] < 3 && n[a] != 1) || !(d[a] > 0.0) || !isfinite(d[a]))
            return 0;
        present += n[a] > 1;
    }
    return present > 0;
}

/* Cell measure: the product of the present axes' spacings (reading R20). */
static double cell_volume(const int n[3], const double d[3])
{
    double v = 1.0;
    for (int a = 0; a < 3; a++)
        if (n[a] > 1)
            v *= d[a];
    return v;
}

/* Whether index idx is a boundary node of an axis of n nodes (R3); an
 * absent axis (n = 1, R20) has none. */
static int boundary(int idx, int n)
{
    return n > 1 && (idx == 0 || idx == n - 1);
}

static size_t n_sites(const int n[3])
{
    return (size_t)n[0] * (size_t)n[1] * (size_t)n[2];
}

/* Harmonic trap V = (gamma^2 x^2 + nu^2 y^2 + lambda^2 z^2) / 2 (reading R1). */
static double trap(const int n[3], const double d[3], const double omega[3],
                   int i, int j, int k)
{
    double x = node_coord(i, n[0], d[0]);
    double y = node_coord(j, n[1], d[1]);
    double z = node_coord(k, n[2], d[2]);
    return 0.5 * (omega[0] * omega[0] * x * x + omega[1] * omega[1] * y * y +
                  omega[2] * omega[2] * z * z);
}

/*
 * Textbook Thomas algorithm for a tridiagonal system
 *     sub[m] x[m-1] + diag[m] x[m] + sup[m] x[m+1] = rhs[m],  m = 0..len-1,
 * with x[-1] = x[len] = 0 (sub[0] and sup[len-1] are ignored).  Forward
 * elimination builds the modified super-diagonal cp and right-hand side dp;
 * back substitution recovers x.  No pivoting (the CN matrices here are
 * strictly diagonally dominant).
 */
static int thomas_solve(int len, const cplx *sub, const cplx *diag, const cplx *sup,
                        const cplx *rhs, cplx *x)
{
    if (len < 1)
        return ORACLE_EARG;
    cplx *cp = malloc((size_t)len * sizeof(cplx));
    cplx *dp = malloc((size_t)len * sizeof(cplx));
    if (!cp || !dp) {
        free(cp);
        free(dp);
        return ORACLE_ENOMEM;
    }
    int rc = ORACLE_OK;
    cplx den = diag[0];
    if (den == 0.0) {
        rc = ORACLE_EPIVOT;
        goto out;
    }
    cp[0] = (len > 1 ? sup[0] : 0.0) / den;
    dp[0] = rhs[0] / den;
    for (int m = 1; m < len; m++) {
        den = diag[m] - sub[m] * cp[m - 1];
        if (den == 0.0) {
            rc = ORACLE_EPIVOT;
            goto out;
        }
        cp[m] = (m < len - 1 ? sup[m] : 0.0) / den;
        dp[m] = (rhs[m] - sub[m] * dp[m - 1]) / den;
    }
    x[len - 1] = dp[len - 1];
    for (int m = len - 2; m >= 0; m--)
        x[m] = dp[m] - cp[m] * x[m + 1];
out:
    free(cp);
    free(dp);
    return rc;
}

int oracle_thomas(int len, const double *sub, const double *diag, const double *sup,
                  const double *rhs, double *x)
{
    if (!sub || !diag || !sup || !rhs || !x)
        return ORACLE_EARG;
    return thomas_solve(len, (const cplx *)sub, (const cplx *)diag, (const cplx *)sup,
                        (const cplx *)rhs, (cplx *)x);
}

/*
 * Initial state: the product Gaussian prod_a (omega_a/pi)^(1/4)
 * exp(-omega_a x_a^2 / 2), zero on the boundary nodes (R3), normalised so
 * that dV * sum |psi|^2 = 1.  This is the g = 0 continuum ground state of
 * the reading R1.
 */
int oracle_gaussian(const int n[3], const double d[3], const double omega[3], double *psi_ri)
{
    if (!n || !d || !omega || !psi_ri || !valid_grid(n, d))
        return ORACLE_EARG;
    cplx *psi = (cplx *)psi_ri;
    double sum = 0.0;
    for (int i = 0; i < n[0]; i++)
        for (int j = 0; j < n[1]; j++)
            for (int k = 0; k < n[2]; k++) {
                double v = 0.0;
                int edge = boundary(i, n[0]) || boundary(j, n[1]) || boundary(k, n[2]);
                if (!edge) {
                    double x = node_coord(i, n[0], d[0]);
                    double y = node_coord(j, n[1], d[1]);
                    double z = node_coord(k, n[2], d[2]);
                    /* an absent axis contributes no factor (R20) */
                    double fx = n[0] > 1 ? pow(omega[0] / M_PI, 0.25) * exp(-0.5 * omega[0] * x * x) : 1.0;
                    double fy = n[1] > 1 ? pow(omega[1] / M_PI, 0.25) * exp(-0.5 * omega[1] * y * y) : 1.0;
                    double fz = n[2] > 1 ? pow(omega[2] / M_PI, 0.25) * exp(-0.5 * omega[2] * z * z) : 1.0;
                    v = fx * fy * fz;
                }
                psi[site(n, i, j, k)] = v;
                sum += v * v;
            }
    double dv = cell_volume(n, d);
    double scale = 1.0 / sqrt(dv * sum);
    for (size_t s = 0; s < n_sites(n); s++)
        psi[s] *= scale;
    return ORACLE_OK;
}

/*
 * Potential-plus-nonlinear step (calcnu): at every node, with rho = |psi|^2
 * taken before the step,
 *   imaginary time: psi <- exp(-dt (V + g rho)) psi,
 *   real time:      psi <- exp(-i dt (V + g rho)) psi.
 */
int oracle_kick(const int n[3], const double d[3], double *psi_ri, double dt,
                const double omega[3], double g, int realtime)
{
    if (!n || !d || !omega || !psi_ri || !valid_grid(n, d) || !isfinite(dt))
        return ORACLE_EARG;
    cplx *psi = (cplx *)psi_ri;
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < n[0]; i++)
        for (int j = 0; j < n[1]; j++)
            for (int k = 0; k < n[2]; k++) {
                size_t s = site(n, i, j, k);
                double rho = creal(psi[s] * conj(psi[s]));
                double arg = dt * (trap(n, d, omega, i, j, k) + g * rho);
                if (realtime)
                    psi[s] *= cexp(-I * arg);
                else
                    psi[s] *= exp(-arg);
            }
    return ORACLE_OK;
}

/*
 * CN line solve along one axis (calclux, calcluy, calcluz): for every line
 * along `axis`, build the right-hand side c psi[m-1] + (1-2c) psi[m] +
 * c psi[m+1] at the interior nodes m = 1..N-2 (boundary nodes count as 0,
 * R3), solve the tridiagonal system (-c, 1+2c, -c) with the Thomas
 * algorithm, and write the solution back with zeros on the two boundary
 * nodes.
 */
int oracle_sweep(const int n[3], const double d[3], double *psi_ri, int axis, double dt,
                 int realtime)
{
    if (!n || !d || !psi_ri || !valid_grid(n, d) || axis < 0 || axis > 2 || !isfinite(dt))
        return ORACLE_EARG;
    cplx *psi = (cplx *)psi_ri;
    const int len = n[axis];
    const int m_int = len - 2;
    if (len == 1)
        return ORACLE_OK; /* an absent axis has no line solve (R20) */
    const cplx c = (realtime ? I : 1.0) * dt / (4.0 * d[axis] * d[axis]);

    /* The two axes that label the lines, and the strides of all three. */
    const size_t stride[3] = {(size_t)n[1] * (size_t)n[2], (size_t)n[2], 1};
    const int a1 = (axis == 0) ? 1 : 0;
    const int a2 = (axis == 2) ? 1 : 2;
    int rc = ORACLE_OK;
#pragma omp parallel
    {
        /* each thread's own line buffers and matrix */
        cplx *sub = malloc((size_t)m_int * sizeof(cplx));
        cplx *diag = malloc((size_t)m_int * sizeof(cplx));
        cplx *sup = malloc((size_t)m_int * sizeof(cplx));
        cplx *rhs = malloc((size_t)m_int * sizeof(cplx));
        cplx *sol = malloc((size_t)m_int * sizeof(cplx));
        cplx *line = malloc((size_t)len * sizeof(cplx));
        int my_rc = (sub && diag && sup && rhs && sol && line) ? ORACLE_OK : ORACLE_ENOMEM;
        for (int m = 0; m < m_int && my_rc == ORACLE_OK; m++) {
            sub[m] = -c;
            diag[m] = 1.0 + 2.0 * c;
            sup[m] = -c;
        }
#pragma omp for collapse(2) schedule(static)
        for (int p = 0; p < n[a1]; p++) {
            for (int q = 0; q < n[a2]; q++) {
                if (my_rc != ORACLE_OK)
                    continue;
                size_t base = (size_t)p * stride[a1] + (size_t)q * stride[a2];
                for (int m = 0; m < len; m++)
                    line[m] = psi[base + (size_t)m * stride[axis]];
                for (int m = 1; m <= len - 2; m++) {
                    cplx left = (m - 1 >= 1) ? line[m - 1] : 0.0;
                    cplx right = (m + 1 <= len - 2) ? line[m + 1] : 0.0;
                    rhs[m - 1] = c * left + (1.0 - 2.0 * c) * line[m] + c * right;
                }
                my_rc = thomas_solve(m_int, sub, diag, sup, rhs, sol);
                if (my_rc != ORACLE_OK)
                    continue;
                psi[base] = 0.0;
                psi[base + (size_t)(len - 1) * stride[axis]] = 0.0;
                for (int m = 1; m <= len - 2; m++)
                    psi[base + (size_t)m * stride[axis]] = sol[m - 1];
            }
        }
#pragma omp critical
        {
            if (my_rc != ORACLE_OK && rc == ORACLE_OK)
                rc = my_rc;
        }
        free(sub);
        free(diag);
        free(sup);
        free(rhs);
        free(sol);
        free(line);
    }
    return rc;
}

/* Norm dV * sum |psi|^2 (rectangle rule, R4). */
static double grid_norm(const int n[3], const double d[3], const cplx *psi)
{
    double sum = 0.0;
    for (size_t s = 0; s < n_sites(n); s++)
        sum += creal(psi[s] * conj(psi[s]));
    return cell_volume(n, d) * sum;
}

/* Imaginary-time renormalisation psi <- psi / sqrt(norm). */
int oracle_renormalize(const int n[3], const double d[3], double *psi_ri)
{
    if (!n || !d || !psi_ri || !valid_grid(n, d))
        return ORACLE_EARG;
    cplx *psi = (cplx *)psi_ri;
    double nrm = grid_norm(n, d, psi);
    if (!(nrm > 0.0) || !isfinite(nrm))
        return ORACLE_EARG;
    double scale = 1.0 / sqrt(nrm);
    for (size_t s = 0; s < n_sites(n); s++)
        psi[s] *= scale;
    return ORACLE_OK;
}

/*
 * `nsteps` full split-step CN steps (R5): kick, sweep x, sweep y, sweep z,
 * and in imaginary time the renormalisation.
 */
int oracle_step(const int n[3], const double d[3], double *psi_ri, double dt,
                const double omega[3], double g, int realtime, int nsteps)
{
    if (nsteps < 0)
        return ORACLE_EARG;
    for (int s = 0; s < nsteps; s++) {
        int rc = oracle_kick(n, d, psi_ri, dt, omega, g, realtime);
        for (int axis = 0; axis < 3 && rc == ORACLE_OK; axis++)
            rc = oracle_sweep(n, d, psi_ri, axis, dt, realtime);
        if (rc == ORACLE_OK && !realtime)
            rc = oracle_renormalize(n, d, psi_ri);
        if (rc != ORACLE_OK)
            return rc;
    }
    return ORACLE_OK;
}

/*
 * Symmetric (Strang) splitting in real time, reading R17: every step is a
 * half kick exp(-i (dt/2) (V + g|psi|^2)), the x, y and z line solves with the
 * full dt, and a second half kick, each step computed on its own (no merging
 * of the half kicks of consecutive steps).  Real time only.
 */
int oracle_step_strang(const int n[3], const double d[3], double *psi_ri, double dt,
                       const double omega[3], double g, int nsteps)
{
    if (nsteps < 0)
        return ORACLE_EARG;
    for (int s = 0; s < nsteps; s++) {
        int rc = oracle_kick(n, d, psi_ri, 0.5 * dt, omega, g, 1);
        for (int axis = 0; axis < 3 && rc == ORACLE_OK; axis++)
            rc = oracle_sweep(n, d, psi_ri, axis, dt, 1);
        if (rc == ORACLE_OK)
            rc = oracle_kick(n, d, psi_ri, 0.5 * dt, omega, g, 1);
        if (rc != ORACLE_OK)
            return rc;
    }
    return ORACLE_OK;
}

/*
 * Observables (calcrms, calcmuen, norm), reading R4:
 *   norm = dV sum |psi|^2
 *   K    = (1/2) dV sum_axes sum_links |psi[m+1] - psi[m]|^2 / d^2
 *          (all links m = 0..N-2 along each axis)
 *   P    = dV sum V |psi|^2,   I = dV sum |psi|^4
 *   mu   = (K + P + g I) / norm,   E = (K + P + g I / 2) / norm
 *   rms_a = sqrt(dV sum a^2 |psi|^2 / norm)   (no mean subtraction).
 * out = {norm, mu, energy, rms_x, rms_y, rms_z}.
 */
int oracle_observables(const int n[3], const double d[3], const double *psi_ri,
                       const double omega[3], double g, double out[6])
{
    if (!n || !d || !omega || !psi_ri || !out || !valid_grid(n, d))
        return ORACLE_EARG;
    const cplx *psi = (const cplx *)psi_ri;
    double s_rho = 0.0, s_v = 0.0, s_rho2 = 0.0, s_x2 = 0.0, s_y2 = 0.0, s_z2 = 0.0;
    double links[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n[0]; i++)
        for (int j = 0; j < n[1]; j++)
            for (int k = 0; k < n[2]; k++) {
                cplx p = psi[site(n, i, j, k)];
                double rho = creal(p * conj(p));
                double x = node_coord(i, n[0], d[0]);
                double y = node_coord(j, n[1], d[1]);
                double z = node_coord(k, n[2], d[2]);
                s_rho += rho;
                s_v += trap(n, d, omega, i, j, k) * rho;
                s_rho2 += rho * rho;
                s_x2 += x * x * rho;
                s_y2 += y * y * rho;
                s_z2 += z * z * rho;
                if (i + 1 < n[0]) {
                    cplx df = psi[site(n, i + 1, j, k)] - p;
                    links[0] += creal(df * conj(df));
                }
                if (j + 1 < n[1]) {
                    cplx df = psi[site(n, i, j + 1, k)] - p;
                    links[1] += creal(df * conj(df));
                }
                if (k + 1 < n[2]) {
                    cplx df = psi[site(n, i, j, k + 1)] - p;
                    links[2] += creal(df * conj(df));
                }
            }
    const double dv = cell_volume(n, d);
    double norm = dv * s_rho;
    if (!(norm > 0.0))
        return ORACLE_EARG;
    double kin = 0.5 * dv *
                 (links[0] / (d[0] * d[0]) + links[1] / (d[1] * d[1]) + links[2] / (d[2] * d[2]));
    double pot = dv * s_v;
    double inter = dv * s_rho2;
    out[0] = norm;
    out[1] = (kin + pot + g * inter) / norm;
    out[2] = (kin + pot + 0.5 * g * inter) / norm;
    out[3] = sqrt(dv * s_x2 / norm);
    out[4] = sqrt(dv * s_y2 / norm);
    out[5] = sqrt(dv * s_z2 / norm);
    return ORACLE_OK;
}

/* ====================================================================
 * Axially symmetric condensates (reading R21), the (rho, z) program variant
 * of the predecessor package.  With gamma = nu the trap is symmetric about
 * the z axis and the ground state (no circulation) depends on (rho, z) only:
 *     i dpsi/dt = [-(1/2)((1/rho) d/drho (rho d/drho) + d^2/dz^2) + V + g|psi|^2] psi,
 *     V = (gamma^2 rho^2 + lambda^2 z^2) / 2,   int 2 pi rho |psi|^2 drho dz = 1.
 * Grid: psi[i][k] (k stride 1), nx nodes along rho and nz along z.  Radial
 * node i = 1..nx-2 sits at rho_i = (i - 1/2) drho (cell centres, so no node
 * lies on the axis); node 0 is a ghost that nothing couples to and node
 * nx-1, at rho = (nx - 3/2) drho, is the Dirichlet boundary (psi = 0).  The
 * z nodes are those of R2/R3.  The radial operator is the finite-volume
 * (1/rho) d/drho (rho d/drho):
 *     L psi_i = [rho_{i+1/2} (psi_{i+1} - psi_i) - rho_{i-1/2} (psi_i - psi_{i-1})] / (rho_i drho^2),
 * rho_{i+-1/2} = rho_i +- drho/2, so rho_{1/2} = 0: the axis carries no flux
 * (the symmetry condition).  It is symmetric in the cylindrical inner product
 * sum 2 pi rho_i drho dz phi* psi, so the CN radial sweep conserves that
 * norm in real time.  With wl_i = rho_{i-1/2}/rho_i, wr_i = rho_{i+1/2}/rho_i
 * and c as in the header, the radial CN equation at node i is
 *     -c wl_i phi[i-1] + (1 + c (wl_i + wr_i)) phi[i] - c wr_i phi[i+1]
 *         = c wl_i psi[i-1] + (1 - c (wl_i + wr_i)) psi[i] + c wr_i psi[i+1].
 * A step is kick, radial sweep, z sweep, then (imaginary time) the
 * renormalisation in the cylindrical measure (R5).  Observables: the
 * measure w_i = 2 pi rho_i drho dz; radial links at rho_{i+1/2} weighted
 * 2 pi rho_{i+1/2} dz / drho, z links weighted 2 pi rho_i drho / dz (the
 * discrete Rayleigh quotient of this operator, R4); rms_x = rms_y =
 * sqrt(<rho^2> / 2).
 * ==================================================================== */

static int axial_grid_ok(int nx, int nz, double drho, double dz)
{
    return nx >= 3 && nz >= 3 && isfinite(drho) && drho > 0.0 && isfinite(dz) && dz > 0.0;
}

static double axial_rho(int i, double drho) { return (i - 0.5) * drho; }

/* Cylindrical weight 2 pi rho_i drho dz of interior radial node i. */
static double axial_w(int i, double drho, double dz) { return 2.0 * M_PI * axial_rho(i, drho) * drho * dz; }

static int axial_interior(int nx, int nz, int i, int k) { return i >= 1 && i <= nx - 2 && k >= 1 && k <= nz - 2; }

static double axial_norm(int nx, int nz, double drho, double dz, const cplx *psi)
{
    double sum = 0.0;
    for (int i = 1; i <= nx - 2; i++)
        for (int k = 0; k < nz; k++) {
            cplx p = psi[(size_t)i * nz + k];
            sum += axial_w(i, drho, dz) * creal(p * conj(p));
        }
    return sum;
}

/* The continuum g = 0 ground state (gamma/pi)^(1/2) (lambda/pi)^(1/4)
 * exp(-(gamma rho^2 + lambda z^2)/2) at the interior nodes, zero elsewhere,
 * normalised in the cylindrical measure. */
int oracle_axial_gaussian(int nx, int nz, double drho, double dz, double gamma, double lambda, double *psi_ri)
{
    if (!psi_ri || !axial_grid_ok(nx, nz, drho, dz) || !(gamma > 0.0) || !(lambda > 0.0))
        return ORACLE_EARG;
    cplx *psi = (cplx *)psi_ri;
    for (int i = 0; i < nx; i++)
        for (int k = 0; k < nz; k++) {
            double v = 0.0;
            if (axial_interior(nx, nz, i, k)) {
                double r = axial_rho(i, drho), z = node_coord(k, nz, dz);
                v = sqrt(gamma / M_PI) * pow(lambda / M_PI, 0.25) * exp(-0.5 * (gamma * r * r + lambda * z * z));
            }
            psi[(size_t)i * nz + k] = v;
        }
    double scale = 1.0 / sqrt(axial_norm(nx, nz, drho, dz, psi));
    for (size_t s = 0; s < (size_t)nx * nz; s++)
        psi[s] *= scale;
    return ORACLE_OK;
}

/* Kick at every interior node with rho = |psi|^2 before the step:
 * exp(-dt (V + g rho)) (imaginary time) or exp(-i dt (V + g rho)). */
int oracle_axial_kick(int nx, int nz, double drho, double dz, double *psi_ri, double dt, double gamma,
                      double lambda, double g, int realtime)
{
    if (!psi_ri || !axial_grid_ok(nx, nz, drho, dz) || !isfinite(dt))
        return ORACLE_EARG;
    cplx *psi = (cplx *)psi_ri;
    for (int i = 1; i <= nx - 2; i++)
        for (int k = 1; k <= nz - 2; k++) {
            size_t s = (size_t)i * nz + k;
            double r = axial_rho(i, drho), z = node_coord(k, nz, dz);
            double v = 0.5 * (gamma * gamma * r * r + lambda * lambda * z * z);
            double arg = dt * (v + g * creal(psi[s] * conj(psi[s])));
            psi[s] = psi[s] * (realtime ? cexp(-I * arg) : exp(-arg));
        }
    return ORACLE_OK;
}

/* CN line solves along rho (axis 0: the radial equation above, for every z
 * line k = 1..nz-2) or z (axis 1: the Cartesian equation of the header, for
 * every radial node i = 1..nx-2).  Boundary and ghost nodes are written 0. */
int oracle_axial_sweep(int nx, int nz, double drho, double dz, double *psi_ri, int axis, double dt, int realtime)
{
    if (!psi_ri || !axial_grid_ok(nx, nz, drho, dz) || (axis != 0 && axis != 1) || !isfinite(dt))
        return ORACLE_EARG;
    cplx *psi = (cplx *)psi_ri;
    const double h = axis == 0 ? drho : dz;
    const cplx c = realtime ? I * dt / (4.0 * h * h) : dt / (4.0 * h * h);
    const int len = (axis == 0 ? nx : nz) - 2, lines = axis == 0 ? nz : nx;
    cplx *sub = malloc((size_t)len * sizeof(cplx)), *diag = malloc((size_t)len * sizeof(cplx));
    cplx *sup = malloc((size_t)len * sizeof(cplx)), *rhs = malloc((size_t)len * sizeof(cplx));
    cplx *x = malloc((size_t)len * sizeof(cplx));
    int rc = (sub && diag && sup && rhs && x) ? ORACLE_OK : ORACLE_ENOMEM;
    for (int l = 1; l <= lines - 2 && rc == ORACLE_OK; l++) {
        /* node m (1..len) of this line */
        size_t base = axis == 0 ? (size_t)l : (size_t)l * nz;
        size_t stride = axis == 0 ? (size_t)nz : 1;
        for (int m = 1; m <= len; m++) {
            double wl = 1.0, wr = 1.0;
            if (axis == 0) {
                double r = axial_rho(m, drho);
                wl = (r - 0.5 * drho) / r;
                wr = (r + 0.5 * drho) / r;
            }
            cplx pm = m > 1 ? psi[base + (size_t)(m - 1) * stride] : 0.0;  /* ghost / boundary node: 0 */
            cplx p0 = psi[base + (size_t)m * stride];
            cplx pp = m < len ? psi[base + (size_t)(m + 1) * stride] : 0.0;
            sub[m - 1] = -c * wl;
            diag[m - 1] = 1.0 + c * (wl + wr);
            sup[m - 1] = -c * wr;
            rhs[m - 1] = c * wl * pm + (1.0 - c * (wl + wr)) * p0 + c * wr * pp;
        }
        rc = thomas_solve(len, sub, diag, sup, rhs, x);
        if (rc != ORACLE_OK)
            break;
        psi[base] = 0.0;
        for (int m = 1; m <= len; m++)
            psi[base + (size_t)m * stride] = x[m - 1];
        psi[base + (size_t)(len + 1) * stride] = 0.0;
    }
    free(sub);
    free(diag);
    free(sup);
    free(rhs);
    free(x);
    return rc;
}

int oracle_axial_step(int nx, int nz, double drho, double dz, double *psi_ri, double dt, double gamma,
                      double lambda, double g, int realtime, int nsteps)
{
    if (nsteps < 0)
        return ORACLE_EARG;
    for (int s = 0; s < nsteps; s++) {
        int rc = oracle_axial_kick(nx, nz, drho, dz, psi_ri, dt, gamma, lambda, g, realtime);
        for (int axis = 0; axis < 2 && rc == ORACLE_OK; axis++)
            rc = oracle_axial_sweep(nx, nz, drho, dz, psi_ri, axis, dt, realtime);
        if (rc == ORACLE_OK && !realtime) {
            cplx *psi = (cplx *)psi_ri;
            double nrm = axial_norm(nx, nz, drho, dz, psi);
            if (!(nrm > 0.0) || !isfinite(nrm))
                return ORACLE_EARG;
            for (size_t q = 0; q < (size_t)nx * nz; q++)
                psi[q] /= sqrt(nrm);
        }
        if (rc != ORACLE_OK)
            return rc;
    }
    return ORACLE_OK;
}

/* out = {norm, mu, energy, rms_x, rms_y, rms_z} (rms_x = rms_y). */
int oracle_axial_observables(int nx, int nz, double drho, double dz, const double *psi_ri, double gamma,
                             double lambda, double g, double out[6])
{
    if (!psi_ri || !out || !axial_grid_ok(nx, nz, drho, dz))
        return ORACLE_EARG;
    const cplx *psi = (const cplx *)psi_ri;
    double enorm = 0.0, epot = 0.0, eint = 0.0, r2 = 0.0, z2 = 0.0, ekin = 0.0;
    for (int i = 1; i <= nx - 2; i++)
        for (int k = 0; k < nz; k++) {
            cplx p = psi[(size_t)i * nz + k];
            double rho = creal(p * conj(p));
            double r = axial_rho(i, drho), z = node_coord(k, nz, dz), w = axial_w(i, drho, dz);
            enorm += w * rho;
            epot += w * 0.5 * (gamma * gamma * r * r + lambda * lambda * z * z) * rho;
            eint += w * rho * rho;
            r2 += w * r * r * rho;
            z2 += w * z * z * rho;
            /* radial link to node i+1 (the last one reaches the boundary node) */
            cplx dr = psi[(size_t)(i + 1) * nz + k] - p;
            ekin += 0.5 * 2.0 * M_PI * (r + 0.5 * drho) * dz / drho * creal(dr * conj(dr));
            if (k + 1 < nz) {
                cplx dzp = psi[(size_t)i * nz + k + 1] - p;
                ekin += 0.5 * 2.0 * M_PI * r * drho / dz * creal(dzp * conj(dzp));
            }
        }
    if (!(enorm > 0.0))
        return ORACLE_EARG;
    out[0] = enorm;
    out[1] = (ekin + epot + g * eint) / enorm;
    out[2] = (ekin + epot + 0.5 * g * eint) / enorm;
    out[3] = sqrt(0.5 * r2 / enorm);
    out[4] = out[3];
    out[5] = sqrt(z2 / enorm);
    return ORACLE_OK;
}

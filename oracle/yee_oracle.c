/*
 * yee_oracle.c -- plain FP64 CPU oracle for the Yee FDTD time loop.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this code.  It shares no source with
 * the CUDA library and is written to be read against the method, not to be
 * fast: every field lives in a full (nz+1)(ny+1)(nx+1) array, every edge has
 * its own coefficients, and the CPML auxiliaries exist everywhere (they stay
 * exactly zero outside the absorbing slabs).
 *
 * What it computes (Sawant et al., "Characterization of Transmission Lines in
 * Microelectronics Circuits using the ARTEMIS Solver", arXiv 2208.04371):
 *   - the Yee staggered-grid leapfrog (Sec. II-A cites Yee 1966): H from the
 *     curl of E, then E from the curl of H, with per-edge permittivity and
 *     conductivity (Sec. II-B and III: dielectrics, lossy metals);
 *   - PEC ground and conductors: tangential E held at zero (Sec. II-A);
 *   - an absorbing layer on the chosen faces (Sec. II-A cites Berenger's PML),
 *     written as the stretched-coordinate CPML recursion;
 *   - a soft source added to E_z on the excitation plane e (Eq. 3);
 *   - the port voltage (surface integral of E_z divided by the strip width)
 *     and the port current (closed loop integral of H around the strip), Eq. 4.
 *
 * Order of one step n (E^0 = 0, H^{-1/2} = 0 unless initial fields are given):
 *   1. H^{n+1/2} from H^{n-1/2} and curl E^n   (forward differences)
 *   2. E^{n+1}   from E^n and curl H^{n+1/2}   (backward differences)
 *   3. E_z on plane e += A * s((n+1) dt)        (soft source)
 *   4. record V(t_{n+1}) and I(t_{n+1/2})
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 *
 * Parity pins (tests/test_oracle_*.py): exact discrete cavity eigenmodes (the
 * Yee dispersion relation), the discrete energy invariant of a lossless PEC
 * cavity, the Courant limit, brute-force PML reflection against a long domain;
 * the conductor coefficients by a lossy-filled cavity mode against the exact
 * recurrence of the time-centred conduction term (a dielectric loss and a
 * metal whose E factor is negative); the port voltage by a field linear across
 * the strip, which the trapezoid sum integrates exactly; the loop current by
 * the discrete Ampere law (loop sum of H = enclosed eps dE_x/dt flux).
 * The PML profile constants, the interface-averaging rule and the choice of
 * the I-loop margin have no physics pin: parity unpinned beyond GPU-vs-oracle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#include <omp.h>

/* CODATA 2018 vacuum constants (SI). */
#define OR_C0   299792458.0
#define OR_MU0  1.25663706212e-6
#define OR_EPS0 8.8541878128e-12

enum { OR_BC_PEC = 0, OR_BC_PML = 1 };
enum { OR_WAVE_NONE = 0, OR_WAVE_DIFF_GAUSS = 1, OR_WAVE_GAUSS_SINE = 2, OR_WAVE_TABLE = 3 };

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, dt;
    /* per-cell material index, nz*ny*nx, x fastest */
    const uint8_t *ids;
    int nmat;
    const double *eps_r, *sigma, *mu_r;
    const uint8_t *is_pec;
    /* zero-thickness PEC sheets: nsheets x {normal_axis, index, lo0, hi0, lo1, hi1} */
    int nsheets;
    const int *sheets;
    /* faces -x,+x,-y,+y,-z,+z : OR_BC_PEC or OR_BC_PML */
    int bc[6];
    int pml_n, pml_order;
    double pml_sigma_scale, pml_kappa_max, pml_alpha_max;
    /* soft source on the plane x = src_plane: E_z edges j in [j0,j1], k in [k0,k1) */
    int src_kind;
    int src_plane, src_j0, src_j1, src_k0, src_k1;
    double src_amp, src_p0, src_p1, src_t0;
    const double *src_table;
    long src_table_len;
    /* ports: nports x {plane, dir, j0, j1, k0, k1, kb, kt, margin}; width[p] in m */
    int nports;
    const int *ports;
    const double *port_width;
} oracle_problem;

typedef struct {
    int nx, ny, nz;
    long n; /* points per array */
    double *ex, *ey, *ez, *hx, *hy, *hz;
    /* per-edge update coefficients */
    double *ca_x, *cb_x, *ca_y, *cb_y, *ca_z, *cb_z;
    uint8_t *pec_x, *pec_y, *pec_z;
    /* per-face H coefficient dt/mu */
    double *db_x, *db_y, *db_z;
    /* CPML auxiliaries, one per (component, derivative axis) */
    double *psi_exy, *psi_exz, *psi_eyz, *psi_eyx, *psi_ezx, *psi_ezy;
    double *psi_hxy, *psi_hxz, *psi_hyz, *psi_hyx, *psi_hzx, *psi_hzy;
    /* 1-D CPML profiles per axis: at integer nodes (e) and half nodes (h) */
    double *be[3], *ae[3], *ke[3], *bh[3], *ah[3], *kh[3];
} oracle_state;

#define IDX(s, i, j, k) (((long)(k) * ((s)->ny + 1) + (j)) * ((s)->nx + 1) + (i))

static int cell_id(const oracle_problem *p, int i, int j, int k)
{
    return p->ids[((long)k * p->ny + j) * p->nx + i];
}

/* Edge material: mean eps_r and sigma of the four cells sharing the edge;
 * PEC if any of them is PEC. */
static void edge_coeffs(const oracle_problem *p, const int cells[4][3],
                        double *ca, double *cb, uint8_t *pec)
{
    double er = 0.0, sg = 0.0;
    int any_pec = 0;
    for (int c = 0; c < 4; ++c) {
        int id = cell_id(p, cells[c][0], cells[c][1], cells[c][2]);
        er += p->eps_r[id];
        sg += p->sigma[id];
        if (p->is_pec[id]) any_pec = 1;
    }
    er = er / 4.0;
    sg = sg / 4.0;
    if (any_pec) {
        *ca = 0.0; *cb = 0.0; *pec = 1;
        return;
    }
    /* conductive medium, time-centred loss term:
     *   eps dE/dt + sigma E = curl H
     *   E^{n+1} = (1 - sigma dt / 2eps)/(1 + sigma dt / 2eps) E^n
     *           + (dt/eps)/(1 + sigma dt / 2eps) curl H                        */
    double eps = OR_EPS0 * er;
    double loss = sg * p->dt / (2.0 * eps);
    *ca = (1.0 - loss) / (1.0 + loss);
    *cb = (p->dt / eps) / (1.0 + loss);
    *pec = 0;
}

static double face_db(const oracle_problem *p, int ncell, const int cells[2][3])
{
    double mr = 0.0;
    for (int c = 0; c < ncell; ++c)
        mr += p->mu_r[cell_id(p, cells[c][0], cells[c][1], cells[c][2])];
    mr = mr / (double)ncell;
    return p->dt / (OR_MU0 * mr);
}

static void set_pec_x(oracle_state *s, int i, int j, int k)
{
    long q = IDX(s, i, j, k);
    s->pec_x[q] = 1; s->ca_x[q] = 0.0; s->cb_x[q] = 0.0;
}
static void set_pec_y(oracle_state *s, int i, int j, int k)
{
    long q = IDX(s, i, j, k);
    s->pec_y[q] = 1; s->ca_y[q] = 0.0; s->cb_y[q] = 0.0;
}
static void set_pec_z(oracle_state *s, int i, int j, int k)
{
    long q = IDX(s, i, j, k);
    s->pec_z[q] = 1; s->ca_z[q] = 0.0; s->cb_z[q] = 0.0;
}

static void build_materials(const oracle_problem *p, oracle_state *s)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    /* every E edge starts as PEC: the domain walls keep that value */
    for (long q = 0; q < s->n; ++q) {
        s->pec_x[q] = s->pec_y[q] = s->pec_z[q] = 1;
    }
    /* E_x(i+1/2, j, k), interior j in [1,ny-1], k in [1,nz-1] */
    for (int k = 1; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int cells[4][3] = {{i, j - 1, k - 1}, {i, j, k - 1}, {i, j - 1, k}, {i, j, k}};
                long q = IDX(s, i, j, k);
                edge_coeffs(p, cells, &s->ca_x[q], &s->cb_x[q], &s->pec_x[q]);
            }
    /* E_y(i, j+1/2, k), interior i in [1,nx-1], k in [1,nz-1] */
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                int cells[4][3] = {{i - 1, j, k - 1}, {i, j, k - 1}, {i - 1, j, k}, {i, j, k}};
                long q = IDX(s, i, j, k);
                edge_coeffs(p, cells, &s->ca_y[q], &s->cb_y[q], &s->pec_y[q]);
            }
    /* E_z(i, j, k+1/2), interior i in [1,nx-1], j in [1,ny-1] */
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                int cells[4][3] = {{i - 1, j - 1, k}, {i, j - 1, k}, {i - 1, j, k}, {i, j, k}};
                long q = IDX(s, i, j, k);
                edge_coeffs(p, cells, &s->ca_z[q], &s->cb_z[q], &s->pec_z[q]);
            }
    /* zero-thickness sheets: the in-plane E edges on the sheet are PEC */
    for (int t = 0; t < p->nsheets; ++t) {
        const int *sh = p->sheets + 6 * t;
        int ax = sh[0], idx = sh[1], lo0 = sh[2], hi0 = sh[3], lo1 = sh[4], hi1 = sh[5];
        if (ax == 2) {          /* plane z = idx, in-plane axes (x, y) */
            for (int j = lo1; j <= hi1; ++j)
                for (int i = lo0; i < hi0; ++i) set_pec_x(s, i, j, idx);
            for (int j = lo1; j < hi1; ++j)
                for (int i = lo0; i <= hi0; ++i) set_pec_y(s, i, j, idx);
        } else if (ax == 1) {   /* plane y = idx, in-plane axes (x, z) */
            for (int k = lo1; k <= hi1; ++k)
                for (int i = lo0; i < hi0; ++i) set_pec_x(s, i, idx, k);
            for (int k = lo1; k < hi1; ++k)
                for (int i = lo0; i <= hi0; ++i) set_pec_z(s, i, idx, k);
        } else {                /* plane x = idx, in-plane axes (y, z) */
            for (int k = lo1; k <= hi1; ++k)
                for (int j = lo0; j < hi0; ++j) set_pec_y(s, idx, j, k);
            for (int k = lo1; k < hi1; ++k)
                for (int j = lo0; j <= hi0; ++j) set_pec_z(s, idx, j, k);
        }
    }
    /* H coefficients: mean mu_r of the (one or two) cells sharing the face */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {     /* H_x(i, j+1/2, k+1/2) */
                int cells[2][3]; int nc = 0;
                if (i > 0) { cells[nc][0] = i - 1; cells[nc][1] = j; cells[nc][2] = k; ++nc; }
                if (i < nx) { cells[nc][0] = i; cells[nc][1] = j; cells[nc][2] = k; ++nc; }
                s->db_x[IDX(s, i, j, k)] = face_db(p, nc, cells);
            }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {      /* H_y(i+1/2, j, k+1/2) */
                int cells[2][3]; int nc = 0;
                if (j > 0) { cells[nc][0] = i; cells[nc][1] = j - 1; cells[nc][2] = k; ++nc; }
                if (j < ny) { cells[nc][0] = i; cells[nc][1] = j; cells[nc][2] = k; ++nc; }
                s->db_y[IDX(s, i, j, k)] = face_db(p, nc, cells);
            }
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {      /* H_z(i+1/2, j+1/2, k) */
                int cells[2][3]; int nc = 0;
                if (k > 0) { cells[nc][0] = i; cells[nc][1] = j; cells[nc][2] = k - 1; ++nc; }
                if (k < nz) { cells[nc][0] = i; cells[nc][1] = j; cells[nc][2] = k; ++nc; }
                s->db_z[IDX(s, i, j, k)] = face_db(p, nc, cells);
            }
}

/* CPML profile value at position pos (in cells) along an axis of ncell cells. */
static void pml_point(const oracle_problem *p, int axis, int ncell, double delta, double pos,
                      double *b, double *a, double *kap)
{
    double depth = 0.0; /* normalised depth into the layer, 0 outside */
    double L = (double)p->pml_n;
    if (p->pml_n > 0) {
        if (p->bc[2 * axis] == OR_BC_PML && pos < L) depth = (L - pos) / L;
        if (p->bc[2 * axis + 1] == OR_BC_PML && pos > ncell - L) depth = (pos - (ncell - L)) / L;
    }
    if (depth <= 0.0) {
        *b = 1.0; *a = 0.0; *kap = 1.0;
        return;
    }
    double m = (double)p->pml_order;
    double eta0 = sqrt(OR_MU0 / OR_EPS0);
    double sigma_max = p->pml_sigma_scale * 0.8 * (m + 1.0) / (eta0 * delta);
    double g = pow(depth, m);
    double sigma = sigma_max * g;
    double kappa = 1.0 + (p->pml_kappa_max - 1.0) * g;
    double alpha = p->pml_alpha_max * (1.0 - depth);
    *b = exp(-(sigma / kappa + alpha) * p->dt / OR_EPS0);
    *a = (sigma > 0.0) ? sigma / (sigma * kappa + kappa * kappa * alpha) * (*b - 1.0) : 0.0;
    *kap = kappa;
}

static void build_pml(const oracle_problem *p, oracle_state *s)
{
    int nn[3] = {p->nx, p->ny, p->nz};
    double dd[3] = {p->dx, p->dy, p->dz};
    for (int a = 0; a < 3; ++a) {
        int n = nn[a];
        s->be[a] = calloc(n + 1, sizeof(double)); s->ae[a] = calloc(n + 1, sizeof(double));
        s->ke[a] = calloc(n + 1, sizeof(double)); s->bh[a] = calloc(n + 1, sizeof(double));
        s->ah[a] = calloc(n + 1, sizeof(double)); s->kh[a] = calloc(n + 1, sizeof(double));
        for (int q = 0; q <= n; ++q)
            pml_point(p, a, n, dd[a], (double)q, &s->be[a][q], &s->ae[a][q], &s->ke[a][q]);
        for (int q = 0; q < n; ++q)
            pml_point(p, a, n, dd[a], (double)q + 0.5, &s->bh[a][q], &s->ah[a][q], &s->kh[a][q]);
    }
}

static double waveform(const oracle_problem *p, long n_plus_1)
{
    double t = (double)n_plus_1 * p->dt;
    switch (p->src_kind) {
    case OR_WAVE_DIFF_GAUSS: {          /* Eq. 3: -2 (t - t0)/sigma exp(-(t - t0)^2 / sigma^2) */
        double sg = p->src_p0, u = (t - p->src_t0) / sg;
        return -2.0 * u * exp(-u * u);
    }
    case OR_WAVE_GAUSS_SINE: {          /* sin(2 pi f0 (t - t0)) exp(-((t - t0)/tau)^2), tau = 2/(pi bw) */
        double f0 = p->src_p0, tau = 2.0 / (M_PI * p->src_p1), u = t - p->src_t0;
        return sin(2.0 * M_PI * f0 * u) * exp(-(u / tau) * (u / tau));
    }
    case OR_WAVE_TABLE:
        return (n_plus_1 - 1 < p->src_table_len) ? p->src_table[n_plus_1 - 1] : 0.0;
    default:
        return 0.0;
    }
}

static void update_h(const oracle_problem *p, oracle_state *s)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double rdx = 1.0 / p->dx, rdy = 1.0 / p->dy, rdz = 1.0 / p->dz;
    /* H_x(i, j+1/2, k+1/2) -= dt/mu [ dEz/dy - dEy/dz ] */
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                long q = IDX(s, i, j, k);
                double dezdy = (s->ez[IDX(s, i, j + 1, k)] - s->ez[q]) * rdy;
                double deydz = (s->ey[IDX(s, i, j, k + 1)] - s->ey[q]) * rdz;
                s->psi_hxy[q] = s->bh[1][j] * s->psi_hxy[q] + s->ah[1][j] * dezdy;
                s->psi_hxz[q] = s->bh[2][k] * s->psi_hxz[q] + s->ah[2][k] * deydz;
                double curl = (dezdy / s->kh[1][j] + s->psi_hxy[q]) - (deydz / s->kh[2][k] + s->psi_hxz[q]);
                s->hx[q] = s->hx[q] - s->db_x[q] * curl;
            }
    /* H_y(i+1/2, j, k+1/2) -= dt/mu [ dEx/dz - dEz/dx ] */
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long q = IDX(s, i, j, k);
                double dexdz = (s->ex[IDX(s, i, j, k + 1)] - s->ex[q]) * rdz;
                double dezdx = (s->ez[IDX(s, i + 1, j, k)] - s->ez[q]) * rdx;
                s->psi_hyz[q] = s->bh[2][k] * s->psi_hyz[q] + s->ah[2][k] * dexdz;
                s->psi_hyx[q] = s->bh[0][i] * s->psi_hyx[q] + s->ah[0][i] * dezdx;
                double curl = (dexdz / s->kh[2][k] + s->psi_hyz[q]) - (dezdx / s->kh[0][i] + s->psi_hyx[q]);
                s->hy[q] = s->hy[q] - s->db_y[q] * curl;
            }
    /* H_z(i+1/2, j+1/2, k) -= dt/mu [ dEy/dx - dEx/dy ] */
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long q = IDX(s, i, j, k);
                double deydx = (s->ey[IDX(s, i + 1, j, k)] - s->ey[q]) * rdx;
                double dexdy = (s->ex[IDX(s, i, j + 1, k)] - s->ex[q]) * rdy;
                s->psi_hzx[q] = s->bh[0][i] * s->psi_hzx[q] + s->ah[0][i] * deydx;
                s->psi_hzy[q] = s->bh[1][j] * s->psi_hzy[q] + s->ah[1][j] * dexdy;
                double curl = (deydx / s->kh[0][i] + s->psi_hzx[q]) - (dexdy / s->kh[1][j] + s->psi_hzy[q]);
                s->hz[q] = s->hz[q] - s->db_z[q] * curl;
            }
}

static void update_e(const oracle_problem *p, oracle_state *s)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double rdx = 1.0 / p->dx, rdy = 1.0 / p->dy, rdz = 1.0 / p->dz;
    /* E_x(i+1/2, j, k) = Ca E_x + Cb [ dHz/dy - dHy/dz ] */
    #pragma omp parallel for
    for (int k = 1; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long q = IDX(s, i, j, k);
                if (s->pec_x[q]) continue;
                double dhzdy = (s->hz[q] - s->hz[IDX(s, i, j - 1, k)]) * rdy;
                double dhydz = (s->hy[q] - s->hy[IDX(s, i, j, k - 1)]) * rdz;
                s->psi_exy[q] = s->be[1][j] * s->psi_exy[q] + s->ae[1][j] * dhzdy;
                s->psi_exz[q] = s->be[2][k] * s->psi_exz[q] + s->ae[2][k] * dhydz;
                double curl = (dhzdy / s->ke[1][j] + s->psi_exy[q]) - (dhydz / s->ke[2][k] + s->psi_exz[q]);
                s->ex[q] = s->ca_x[q] * s->ex[q] + s->cb_x[q] * curl;
            }
    /* E_y(i, j+1/2, k) = Ca E_y + Cb [ dHx/dz - dHz/dx ] */
    #pragma omp parallel for
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                long q = IDX(s, i, j, k);
                if (s->pec_y[q]) continue;
                double dhxdz = (s->hx[q] - s->hx[IDX(s, i, j, k - 1)]) * rdz;
                double dhzdx = (s->hz[q] - s->hz[IDX(s, i - 1, j, k)]) * rdx;
                s->psi_eyz[q] = s->be[2][k] * s->psi_eyz[q] + s->ae[2][k] * dhxdz;
                s->psi_eyx[q] = s->be[0][i] * s->psi_eyx[q] + s->ae[0][i] * dhzdx;
                double curl = (dhxdz / s->ke[2][k] + s->psi_eyz[q]) - (dhzdx / s->ke[0][i] + s->psi_eyx[q]);
                s->ey[q] = s->ca_y[q] * s->ey[q] + s->cb_y[q] * curl;
            }
    /* E_z(i, j, k+1/2) = Ca E_z + Cb [ dHy/dx - dHx/dy ] */
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 1; i < nx; ++i) {
                long q = IDX(s, i, j, k);
                if (s->pec_z[q]) continue;
                double dhydx = (s->hy[q] - s->hy[IDX(s, i - 1, j, k)]) * rdx;
                double dhxdy = (s->hx[q] - s->hx[IDX(s, i, j - 1, k)]) * rdy;
                s->psi_ezx[q] = s->be[0][i] * s->psi_ezx[q] + s->ae[0][i] * dhydx;
                s->psi_ezy[q] = s->be[1][j] * s->psi_ezy[q] + s->ae[1][j] * dhxdy;
                double curl = (dhydx / s->ke[0][i] + s->psi_ezx[q]) - (dhxdy / s->ke[1][j] + s->psi_ezy[q]);
                s->ez[q] = s->ca_z[q] * s->ez[q] + s->cb_z[q] * curl;
            }
}

/* Eq. 4, first line: V = (1/w) * surface integral of E_z over surface e.
 * Sign: V is the strip potential above ground, V = -(1/w) sum E_z dy dz. */
static double port_voltage(const oracle_problem *p, const oracle_state *s, int t)
{
    const int *d = p->ports + 9 * t;
    int plane = d[0], j0 = d[2], j1 = d[3], k0 = d[4], k1 = d[5];
    double sum = 0.0;
    for (int k = k0; k < k1; ++k)
        for (int j = j0; j <= j1; ++j) {
            double wj = (j == j0 || j == j1) ? 0.5 : 1.0;   /* trapezoid across the strip */
            sum += wj * s->ez[IDX(s, plane, j, k)];
        }
    return -sum * p->dy * p->dz / p->port_width[t];
}

/* Eq. 4, second line: closed loop integral of H around the strip at x = ih + 1/2,
 * one cell (margin m) outside the conductor, oriented by the right-hand rule
 * about +x:  bottom (+y) , right (+z), top (-y), left (-z). */
static double loop_current(const oracle_problem *p, const oracle_state *s, int t, int ih)
{
    const int *d = p->ports + 9 * t;
    int j0 = d[2], j1 = d[3], kb = d[6], kt = d[7], m = d[8];
    double sum = 0.0;
    for (int j = j0 - m + 1; j <= j1 + m - 1; ++j) {
        sum += s->hy[IDX(s, ih, j, kb - m)] * p->dy;          /* bottom, along +y */
        sum -= s->hy[IDX(s, ih, j, kt + m - 1)] * p->dy;      /* top, along -y */
    }
    for (int k = kb - m + 1; k <= kt + m - 1; ++k) {
        sum += s->hz[IDX(s, ih, j1 + m - 1, k)] * p->dz;      /* right side, along +z */
        sum -= s->hz[IDX(s, ih, j0 - m, k)] * p->dz;          /* left side, along -z */
    }
    return sum;
}

static double port_current(const oracle_problem *p, const oracle_state *s, int t)
{
    const int *d = p->ports + 9 * t;
    int plane = d[0], dir = d[1];
    /* mean of the loops at x = plane - 1/2 and plane + 1/2 (co-located with V) */
    double ix = 0.5 * (loop_current(p, s, t, plane - 1) + loop_current(p, s, t, plane));
    return (double)dir * ix;
}

/* Discrete energy W^n = sum eps E^n.E^n + sum mu H^{n-1/2}.H^{n+1/2} (cell volume
 * factored out).  Meaningful for lossless media only: there dt/Cb is exactly
 * the edge permittivity.  Needs H^{n-1/2}, so it is evaluated around the H
 * update. */
static double energy_e(const oracle_problem *p, const oracle_state *s)
{
    double w = 0.0;
    for (long q = 0; q < s->n; ++q) {
        if (!s->pec_x[q]) w += (p->dt / s->cb_x[q]) * s->ex[q] * s->ex[q];
        if (!s->pec_y[q]) w += (p->dt / s->cb_y[q]) * s->ey[q] * s->ey[q];
        if (!s->pec_z[q]) w += (p->dt / s->cb_z[q]) * s->ez[q] * s->ez[q];
    }
    return w;
}

static void free_state(oracle_state *s)
{
    double **d[] = {&s->ex, &s->ey, &s->ez, &s->hx, &s->hy, &s->hz, &s->ca_x, &s->cb_x, &s->ca_y,
                    &s->cb_y, &s->ca_z, &s->cb_z, &s->db_x, &s->db_y, &s->db_z, &s->psi_exy,
                    &s->psi_exz, &s->psi_eyz, &s->psi_eyx, &s->psi_ezx, &s->psi_ezy, &s->psi_hxy,
                    &s->psi_hxz, &s->psi_hyz, &s->psi_hyx, &s->psi_hzx, &s->psi_hzy};
    for (size_t t = 0; t < sizeof(d) / sizeof(d[0]); ++t) { free(*d[t]); *d[t] = NULL; }
    free(s->pec_x); free(s->pec_y); free(s->pec_z);
    for (int a = 0; a < 3; ++a) {
        free(s->be[a]); free(s->ae[a]); free(s->ke[a]);
        free(s->bh[a]); free(s->ah[a]); free(s->kh[a]);
    }
}

static void record_ports(const oracle_problem *p, const oracle_state *s, long n, long nsteps,
                         double *V, double *I)
{
    for (int t = 0; t < p->nports; ++t) {
        V[(long)t * nsteps + n] = port_voltage(p, s, t);
        I[(long)t * nsteps + n] = port_current(p, s, t);
    }
}

/* Allocate the state, derive the edge coefficients and CPML profiles, load the initial
 * fields.  Returns 0, or -1 on allocation failure (nothing left allocated). */
static int setup_state(const oracle_problem *p, const double *fields_in, oracle_state *s)
{
    memset(s, 0, sizeof(*s));
    s->nx = p->nx; s->ny = p->ny; s->nz = p->nz;
    s->n = (long)(p->nx + 1) * (p->ny + 1) * (p->nz + 1);
    double **d[] = {&s->ex, &s->ey, &s->ez, &s->hx, &s->hy, &s->hz, &s->ca_x, &s->cb_x, &s->ca_y,
                    &s->cb_y, &s->ca_z, &s->cb_z, &s->db_x, &s->db_y, &s->db_z, &s->psi_exy,
                    &s->psi_exz, &s->psi_eyz, &s->psi_eyx, &s->psi_ezx, &s->psi_ezy, &s->psi_hxy,
                    &s->psi_hxz, &s->psi_hyz, &s->psi_hyx, &s->psi_hzx, &s->psi_hzy};
    for (size_t t = 0; t < sizeof(d) / sizeof(d[0]); ++t) {
        *d[t] = calloc(s->n, sizeof(double));
        if (!*d[t]) { free_state(s); return -1; }
    }
    s->pec_x = calloc(s->n, 1); s->pec_y = calloc(s->n, 1); s->pec_z = calloc(s->n, 1);
    if (!s->pec_x || !s->pec_y || !s->pec_z) { free_state(s); return -1; }
    build_materials(p, s);
    build_pml(p, s);
    if (fields_in) {
        /* initial E^0 and H^{-1/2}; tangential E on PEC edges and entries outside each
         * component's index range are held at zero */
        double *f[6] = {s->ex, s->ey, s->ez, s->hx, s->hy, s->hz};
        const uint8_t *pec[3] = {s->pec_x, s->pec_y, s->pec_z};
        const double *db[3] = {s->db_x, s->db_y, s->db_z};
        for (int c = 0; c < 6; ++c)
            for (long q = 0; q < s->n; ++q) {
                int live = (c < 3) ? !pec[c][q] : (db[c - 3][q] > 0.0);
                f[c][q] = live ? fields_in[(long)c * s->n + q] : 0.0;
            }
    }
    return 0;
}

/* Steps n0 .. n0+nsteps-1 of the time loop (see the order at the top of this file); the
 * port samples of step n go to V, I at column n - n0 of rows of length nsteps. */
static int time_loop(const oracle_problem *p, oracle_state *s, long n0, long nsteps, double *V,
                     double *I, double *energy)
{
    double *hprev = NULL;
    if (energy) {
        hprev = malloc(3 * s->n * sizeof(double));
        if (!hprev) return -1;
    }
    for (long n = n0; n < n0 + nsteps; ++n) {
        double we = 0.0;
        if (energy) {
            we = energy_e(p, s);
            memcpy(hprev, s->hx, s->n * sizeof(double));
            memcpy(hprev + s->n, s->hy, s->n * sizeof(double));
            memcpy(hprev + 2 * s->n, s->hz, s->n * sizeof(double));
        }
        update_h(p, s);
        if (energy) {
            double wh = 0.0;
            for (long q = 0; q < s->n; ++q) {
                if (s->db_x[q] > 0.0) wh += (p->dt / s->db_x[q]) * hprev[q] * s->hx[q];
                if (s->db_y[q] > 0.0) wh += (p->dt / s->db_y[q]) * hprev[s->n + q] * s->hy[q];
                if (s->db_z[q] > 0.0) wh += (p->dt / s->db_z[q]) * hprev[2 * s->n + q] * s->hz[q];
            }
            energy[n - n0] = we + wh;
        }
        update_e(p, s);
        if (p->src_kind != OR_WAVE_NONE) {
            double a = p->src_amp * waveform(p, n + 1);
            for (int k = p->src_k0; k < p->src_k1; ++k)
                for (int j = p->src_j0; j <= p->src_j1; ++j) {
                    long q = IDX(s, p->src_plane, j, k);
                    if (!s->pec_z[q]) s->ez[q] += a;
                }
        }
        record_ports(p, s, n - n0, nsteps, V, I);
    }
    free(hprev);
    return 0;
}

static void copy_fields_out(const oracle_state *s, double *fields_out)
{
    const double *f[6] = {s->ex, s->ey, s->ez, s->hx, s->hy, s->hz};
    for (int c = 0; c < 6; ++c) memcpy(fields_out + (long)c * s->n, f[c], s->n * sizeof(double));
}

/*
 * Run nsteps of the time loop.
 *   V, I       : nports*nsteps outputs (port-major), may be NULL when nports == 0
 *   fields_in  : optional 6 arrays (ex,ey,ez,hx,hy,hz) of (nz+1)(ny+1)(nx+1): E^0, H^{-1/2}
 *   fields_out : optional 6 arrays of the same shape: E^N, H^{N-1/2}
 *   energy     : optional nsteps values of W^n, n = 0..nsteps-1
 * Returns 0 on success, -1 on allocation failure.
 */
int oracle_run(const oracle_problem *p, long nsteps, double *V, double *I,
               const double *fields_in, double *fields_out, double *energy)
{
    oracle_state st;
    if (setup_state(p, fields_in, &st) != 0) return -1;
    int rc = time_loop(p, &st, 0, nsteps, V, I, energy);
    if (rc == 0 && fields_out) copy_fields_out(&st, fields_out);
    free_state(&st);
    return rc;
}

/*
 * A run held open between calls, for timing the stepping alone:
 *   oracle_open    allocates the state and does the set-up (coefficients, CPML
 *                  profiles), fields at zero; NULL on allocation failure;
 *   oracle_advance runs the next nsteps steps (the source clock continues from the
 *                  steps already taken), port samples into V, I (nports rows of
 *                  nsteps), and puts the wall-clock seconds of those steps alone in
 *                  *seconds; returns 0, or -1 on allocation failure;
 *   oracle_close   frees the state.
 * The problem must outlive the handle.
 */
typedef struct {
    oracle_state st;
    long steps_done;
} oracle_handle;

oracle_handle *oracle_open(const oracle_problem *p)
{
    oracle_handle *h = calloc(1, sizeof(oracle_handle));
    if (!h) return NULL;
    if (setup_state(p, NULL, &h->st) != 0) { free(h); return NULL; }
    return h;
}

int oracle_advance(oracle_handle *h, const oracle_problem *p, long nsteps, double *V, double *I,
                   double *seconds)
{
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    int rc = time_loop(p, &h->st, h->steps_done, nsteps, V, I, NULL);
    clock_gettime(CLOCK_MONOTONIC, &t1);
    if (seconds)
        *seconds = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
    if (rc == 0) h->steps_done += nsteps;
    return rc;
}

void oracle_close(oracle_handle *h)
{
    if (!h) return;
    free_state(&h->st);
    free(h);
}

/* Threads of the OpenMP loops over k-planes for the following runs (the environment
 * variable is read once, when the OpenMP runtime starts). */
void oracle_set_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
}

/* The waveform as the oracle evaluates it, for the closed-form DFT pins. */
double oracle_waveform(const oracle_problem *p, long n_plus_1)
{
    return waveform(p, n_plus_1);
}

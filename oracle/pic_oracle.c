/*
 * pic_oracle.c -- plain, slow, FP64 CPU oracle of one explicit, fully
 * relativistic 3D3V particle-in-cell time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no source with the CUDA path.
 *
 * The paper (Zenker et al., "Performance-Portable Many-Core Plasma
 * Simulations: Porting PIConGPU to OpenPower and Beyond", Sec. 4) names the
 * algorithms of its PIC cycle but prints no formula for them: the Boris
 * pusher, the Esirkepov current solver, the Yee field solver, interpolation
 * of the fields to the particles as a product of 1D weights ("trilinear"),
 * and the quadratic-spline (TSC) particle shape of Hockney & Eastwood.  Each
 * function below writes out the textbook definition of the algorithm the
 * paper names, in FP64, with plain loops and periodic index wrapping.  No
 * blocking, fusion or reordering beyond the definition.
 *
 * Conventions (the paper is silent; these are the readings the tests use):
 *   - normalised units: c = 1, eps0 = mu0 = 1; Maxwell's equations are
 *     dB/dt = -curl E and dE/dt = curl B - J;  momentum u = gamma v.
 *   - particle positions are global coordinates in cell units, x in [0, N).
 *   - Yee staggering: Ex at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at
 *     (i, j, k+1/2); Bx at (i, j+1/2, k+1/2), By at (i+1/2, j, k+1/2), Bz at
 *     (i+1/2, j+1/2, k); J co-located with E; charge density at the nodes.
 *     Array element [i,j,k] of a half-staggered component holds the value at
 *     the position whose half-staggered coordinates are i+1/2 (etc.).
 *   - field arrays are component-major, x fastest: F[c][k][j][i].
 *   - step order (leapfrog with B split in two halves so that B exists at
 *     integer time for the push): gather E^n, B^n at x^n; Boris u^{n-1/2} ->
 *     u^{n+1/2}; move x^{n+1} = x^n + dt u/gamma; Esirkepov J^{n+1/2};
 *     B^{n+1/2} = B^n - dt/2 curl E^n; E^{n+1} = E^n + dt (curl B^{n+1/2} -
 *     J^{n+1/2}); B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}.
 *   - a macro-particle of weight w and charge q carries the charge density
 *     q w S(x - node) / V_cell.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_DISPLACEMENT 2

typedef struct {
    int64_t nx, ny, nz;
    double dx, dy, dz;
} orc_grid;

static inline int64_t wrap(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

static inline int64_t cell_index(const orc_grid* g, int64_t i, int64_t j, int64_t k)
{
    return (wrap(k, g->nz) * g->ny + wrap(j, g->ny)) * g->nx + wrap(i, g->nx);
}

static inline int64_t ncells(const orc_grid* g) { return g->nx * g->ny * g->nz; }

/*
 * 1D assignment functions of Hockney & Eastwood, which Sec. 4 names for the
 * particle shape: order 1 = cloud-in-cell (linear), order 2 = triangular-
 * shaped cloud (quadratic spline); beyond the paper, order 3 = piecewise
 * cubic spline (PCS) and order 0 = nearest grid point (used only by the
 * energy-conserving gather).  d is the distance from the particle to a grid
 * point, in cells.  The six-point windows of the gather and the deposit
 * below cover the support of every order up to 3 for moves below one cell.
 */
double orc_shape(int order, double d)
{
    double a = fabs(d);
    if (order == 0) /* nearest grid point; a point half-way goes to the upper neighbour */
        return (d >= -0.5 && d < 0.5) ? 1.0 : 0.0;
    if (order == 1)
        return a < 1.0 ? 1.0 - a : 0.0;
    if (order == 2) {
        if (a <= 0.5)
            return 0.75 - a * a;
        if (a < 1.5)
            return 0.5 * (1.5 - a) * (1.5 - a);
        return 0.0;
    }
    if (order == 3) { /* piecewise cubic spline (PCS, the cubic B-spline) */
        if (a < 1.0)
            return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
        if (a < 2.0)
            return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
        return 0.0;
    }
    return 0.0;
}

/* Offsets (in cells) of the Yee positions of each field component. */
static const double E_STAGGER[3][3] = {{0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5}};
static const double B_STAGGER[3][3] = {{0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};

/*
 * Field gather (Sec. 4, "trilinear interpolation in field gathering", with
 * the TSC shape): F(x_p) = sum over the grid points m of the component of
 * F[m] * S(x_p - m - s) in x, y and z, s being the component's staggering.
 * The window of six points per axis covers the support of every shape.
 * ec (energy-conserving variant, beyond the paper): along each axis on which
 * the component is staggered by half a cell the shape is one order lower
 * (TSC -> CIC, CIC -> nearest grid point), so that the gather is the
 * transpose of the Esirkepov current along that axis.
 */
static double gather_component(const double* F, const orc_grid* g, int order,
                               const double x[3], const double s[3], int ec)
{
    int64_t base[3];
    double wt[3][6];
    for (int d = 0; d < 3; ++d) {
        int od = (ec && s[d] == 0.5) ? order - 1 : order;
        base[d] = (int64_t)floor(x[d] - s[d]) - 2;
        for (int n = 0; n < 6; ++n)
            wt[d][n] = orc_shape(od, x[d] - s[d] - (double)(base[d] + n));
    }
    double sum = 0.0;
    for (int c = 0; c < 6; ++c)
        for (int b = 0; b < 6; ++b)
            for (int a = 0; a < 6; ++a) {
                double w = wt[0][a] * wt[1][b] * wt[2][c];
                if (w != 0.0)
                    sum += w * F[cell_index(g, base[0] + a, base[1] + b, base[2] + c)];
            }
    return sum;
}

void orc_gather(const orc_grid* g, int order, const double* E, const double* B,
                const double x[3], double Ep[3], double Bp[3], int ec)
{
    int64_t nc = ncells(g);
    for (int c = 0; c < 3; ++c) {
        Ep[c] = gather_component(E + c * nc, g, order, x, E_STAGGER[c], ec);
        Bp[c] = gather_component(B + c * nc, g, order, x, B_STAGGER[c], ec);
    }
}

/*
 * Relativistic Boris push (Boris 1970, named in Sec. 4): half electric kick,
 * magnetic rotation, half electric kick, on u = gamma v.  gamma for the
 * rotation is taken from the momentum after the first half kick.
 */
void orc_boris(double q, double m, double dt, const double E[3], const double B[3], double u[3])
{
    double eps = q * dt / (2.0 * m);
    double um[3], t[3], s[3], up[3], uq[3];
    for (int d = 0; d < 3; ++d)
        um[d] = u[d] + eps * E[d];
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int d = 0; d < 3; ++d)
        t[d] = eps * B[d] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int d = 0; d < 3; ++d)
        s[d] = 2.0 * t[d] / (1.0 + t2);
    /* u' = u- + u- x t */
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    /* u+ = u- + u' x s */
    uq[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
    uq[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
    uq[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
    for (int d = 0; d < 3; ++d)
        u[d] = uq[d] + eps * E[d];
}

/*
 * Esirkepov (2001) charge-conserving current deposition, named in Sec. 4.
 * From the 1D shape factors S0 (at x0) and S1 (at x1) on a common window of
 * integer nodes, DS = S1 - S0, the density decomposition
 *   Wx = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3)
 * (and cyclic for Wy, Wz) gives the current by a running sum along each axis:
 *   Jx(i+1/2) = Jx(i-1/2) - q w dx / (V dt) Wx(i),   zero below the window.
 * The window of six nodes starting two below floor(x0) is valid for any
 * displacement shorter than one cell per axis; longer ones are rejected.
 */
int orc_deposit_esirkepov(const orc_grid* g, int order, double qw, double dt,
                          const double x0[3], const double x1[3], double* J)
{
    int64_t base[3];
    double S0[3][6], S1[3][6], DS[3][6];
    for (int d = 0; d < 3; ++d) {
        if (!(fabs(x1[d] - x0[d]) < 1.0))
            return ORC_ERR_DISPLACEMENT;
        base[d] = (int64_t)floor(x0[d]) - 2;
        for (int n = 0; n < 6; ++n) {
            S0[d][n] = orc_shape(order, x0[d] - (double)(base[d] + n));
            S1[d][n] = orc_shape(order, x1[d] - (double)(base[d] + n));
            DS[d][n] = S1[d][n] - S0[d][n];
        }
    }
    int64_t nc = ncells(g);
    double V = g->dx * g->dy * g->dz;
    double h[3] = {g->dx, g->dy, g->dz};
    for (int d = 0; d < 3; ++d) {
        /* axis d carries the current; e and f are the two transverse axes */
        int e = (d + 1) % 3, f = (d + 2) % 3;
        double coef = -qw * h[d] / (V * dt);
        double* Jd = J + d * nc;
        for (int nf = 0; nf < 6; ++nf)
            for (int ne = 0; ne < 6; ++ne) {
                double acc = 0.0;
                for (int nd = 0; nd < 6; ++nd) {
                    double W = DS[d][nd] * (S0[e][ne] * S0[f][nf] + 0.5 * DS[e][ne] * S0[f][nf] +
                                            0.5 * S0[e][ne] * DS[f][nf] +
                                            DS[e][ne] * DS[f][nf] / 3.0);
                    acc += coef * W;
                    if (acc == 0.0)
                        continue;
                    int64_t idx[3];
                    idx[d] = base[d] + nd; /* half node nd + 1/2 along d */
                    idx[e] = base[e] + ne;
                    idx[f] = base[f] + nf;
                    Jd[cell_index(g, idx[0], idx[1], idx[2])] += acc;
                }
            }
    }
    return ORC_OK;
}

/*
 * One particle species through gather -> Boris -> move -> Esirkepov (the
 * particle half of the PIC cycle, Sec. 2.1 and Sec. 4).  x is n x 3 in cell
 * units and is wrapped back into [0, N) after the move; u is n x 3; w is n
 * (NULL = all weights 1).  J accumulates (the caller zeroes it).  open_y:
 * the y coordinate is not wrapped, so that the caller can remove the
 * particles that left through a y face (they have deposited their current,
 * folded periodically like every other deposit).  ec: the energy-conserving
 * gather (see gather_component).
 */
int orc_push_deposit(const orc_grid* g, double dt, int order, double q, double m,
                     const double* E, const double* B, double* J,
                     int64_t n, double* x, double* u, const double* w, int open_y, int ec)
{
    double h[3] = {g->dx, g->dy, g->dz};
    int64_t N[3] = {g->nx, g->ny, g->nz};
    for (int64_t p = 0; p < n; ++p) {
        double* xp = x + 3 * p;
        double* up = u + 3 * p;
        double Ep[3], Bp[3];
        orc_gather(g, order, E, B, xp, Ep, Bp, ec);
        orc_boris(q, m, dt, Ep, Bp, up);
        double gam = sqrt(1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
        double x1[3];
        for (int d = 0; d < 3; ++d)
            x1[d] = xp[d] + dt * up[d] / (gam * h[d]);
        double wp = w ? w[p] : 1.0;
        int rc = orc_deposit_esirkepov(g, order, q * wp, dt, xp, x1, J);
        if (rc != ORC_OK)
            return rc;
        for (int d = 0; d < 3; ++d) {
            double y = x1[d];
            if (d == 1 && open_y) { /* left for the caller to remove when outside [0, ny) */
                xp[d] = y;
                continue;
            }
            if (y >= (double)N[d])
                y -= (double)N[d];
            else if (y < 0.0)
                y += (double)N[d];
            if (y >= (double)N[d]) /* -tiny + N rounded up to N */
                y = 0.0;
            xp[d] = y;
        }
    }
    return ORC_OK;
}

/*
 * Yee (1966) half update of B, named in Sec. 4: B -= tau * curl E with the
 * centred differences of the staggered grid, e.g.
 *   (curl E)x(i, j+1/2, k+1/2) = (Ez[i,j+1,k] - Ez[i,j,k]) / dy
 *                              - (Ey[i,j,k+1] - Ey[i,j,k]) / dz.
 */
void orc_yee_b(const orc_grid* g, double tau, const double* E, double* B)
{
    int64_t nc = ncells(g);
    const double *Ex = E, *Ey = E + nc, *Ez = E + 2 * nc;
    double *Bx = B, *By = B + nc, *Bz = B + 2 * nc;
    for (int64_t k = 0; k < g->nz; ++k)
        for (int64_t j = 0; j < g->ny; ++j)
            for (int64_t i = 0; i < g->nx; ++i) {
                int64_t c = cell_index(g, i, j, k);
                double cx = (Ez[cell_index(g, i, j + 1, k)] - Ez[c]) / g->dy -
                            (Ey[cell_index(g, i, j, k + 1)] - Ey[c]) / g->dz;
                double cy = (Ex[cell_index(g, i, j, k + 1)] - Ex[c]) / g->dz -
                            (Ez[cell_index(g, i + 1, j, k)] - Ez[c]) / g->dx;
                double cz = (Ey[cell_index(g, i + 1, j, k)] - Ey[c]) / g->dx -
                            (Ex[cell_index(g, i, j + 1, k)] - Ex[c]) / g->dy;
                Bx[c] -= tau * cx;
                By[c] -= tau * cy;
                Bz[c] -= tau * cz;
            }
}

/*
 * Yee update of E: E += dt * (curl B - J), e.g.
 *   (curl B)x(i+1/2, j, k) = (Bz[i,j,k] - Bz[i,j-1,k]) / dy
 *                          - (By[i,j,k] - By[i,j,k-1]) / dz.
 */
void orc_yee_e(const orc_grid* g, double dt, double* E, const double* B, const double* J)
{
    int64_t nc = ncells(g);
    double *Ex = E, *Ey = E + nc, *Ez = E + 2 * nc;
    const double *Bx = B, *By = B + nc, *Bz = B + 2 * nc;
    for (int64_t k = 0; k < g->nz; ++k)
        for (int64_t j = 0; j < g->ny; ++j)
            for (int64_t i = 0; i < g->nx; ++i) {
                int64_t c = cell_index(g, i, j, k);
                double cx = (Bz[c] - Bz[cell_index(g, i, j - 1, k)]) / g->dy -
                            (By[c] - By[cell_index(g, i, j, k - 1)]) / g->dz;
                double cy = (Bx[c] - Bx[cell_index(g, i, j, k - 1)]) / g->dz -
                            (Bz[c] - Bz[cell_index(g, i - 1, j, k)]) / g->dx;
                double cz = (By[c] - By[cell_index(g, i - 1, j, k)]) / g->dx -
                            (Bx[c] - Bx[cell_index(g, i, j - 1, k)]) / g->dy;
                Ex[c] += dt * (cx - J[c]);
                Ey[c] += dt * (cy - J[nc + c]);
                Ez[c] += dt * (cz - J[2 * nc + c]);
            }
}

/* The field half of the cycle in the step order above. */
void orc_yee_step(const orc_grid* g, double dt, double* E, double* B, const double* J)
{
    orc_yee_b(g, 0.5 * dt, E, B);
    orc_yee_e(g, dt, E, B, J);
    orc_yee_b(g, 0.5 * dt, E, B);
}

/* Charge density at the nodes: rho[m] += q w S(x - m) / V for each particle. */
void orc_deposit_rho(const orc_grid* g, int order, double q, int64_t n, const double* x,
                     const double* w, double* rho)
{
    double V = g->dx * g->dy * g->dz;
    for (int64_t p = 0; p < n; ++p) {
        const double* xp = x + 3 * p;
        int64_t base[3];
        double wt[3][6];
        for (int d = 0; d < 3; ++d) {
            base[d] = (int64_t)floor(xp[d]) - 2;
            for (int nn = 0; nn < 6; ++nn)
                wt[d][nn] = orc_shape(order, xp[d] - (double)(base[d] + nn));
        }
        double qw = q * (w ? w[p] : 1.0) / V;
        for (int c = 0; c < 6; ++c)
            for (int b = 0; b < 6; ++b)
                for (int a = 0; a < 6; ++a) {
                    double s = wt[0][a] * wt[1][b] * wt[2][c];
                    if (s != 0.0)
                        rho[cell_index(g, base[0] + a, base[1] + b, base[2] + c)] += qw * s;
                }
    }
}

/* Divergence of E at the nodes: sum over d of (Ed[m] - Ed[m - e_d]) / dx_d. */
void orc_div_e(const orc_grid* g, const double* E, double* div)
{
    int64_t nc = ncells(g);
    const double *Ex = E, *Ey = E + nc, *Ez = E + 2 * nc;
    for (int64_t k = 0; k < g->nz; ++k)
        for (int64_t j = 0; j < g->ny; ++j)
            for (int64_t i = 0; i < g->nx; ++i) {
                int64_t c = cell_index(g, i, j, k);
                div[c] = (Ex[c] - Ex[cell_index(g, i - 1, j, k)]) / g->dx +
                         (Ey[c] - Ey[cell_index(g, i, j - 1, k)]) / g->dy +
                         (Ez[c] - Ez[cell_index(g, i, j, k - 1)]) / g->dz;
            }
}

/* Divergence of a co-located-with-E current J at the nodes (same stencil). */
void orc_div_j(const orc_grid* g, const double* J, double* div) { orc_div_e(g, J, div); }

/* Field energy: sum over cells of (E^2 + B^2) / 2 times the cell volume. */
double orc_field_energy(const orc_grid* g, const double* E, const double* B)
{
    int64_t nc = ncells(g);
    double s = 0.0;
    for (int64_t c = 0; c < 3 * nc; ++c)
        s += 0.5 * (E[c] * E[c] + B[c] * B[c]);
    return s * g->dx * g->dy * g->dz;
}

/* Kinetic energy of one species: sum of w m (gamma - 1). */
double orc_kinetic_energy(double m, int64_t n, const double* u, const double* w)
{
    double s = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        const double* up = u + 3 * p;
        double u2 = up[0] * up[0] + up[1] * up[1] + up[2] * up[2];
        double gm1 = u2 / (sqrt(1.0 + u2) + 1.0); /* gamma - 1 without cancellation */
        s += (w ? w[p] : 1.0) * m * gm1;
    }
    return s;
}

/*
 * ---------------------------------------------------------------- open y
 * Boundaries along y for the laser-plasma setups (the paper's own runs are
 * periodic and it names no boundary scheme; these are the readings the
 * tests and the CUDA path share):
 *
 * Absorber: damping layers of A cells at both y faces.  After each full
 * field step every E and B component is multiplied by exp(-sigma delta^2),
 * delta in [0, 1] being the depth of the component's staggered y position
 * inside the layer, from 0 at the layer's inner edge to 1 at the face:
 * delta = (A - y) / A for y < A, (y - (ny - A)) / A for y > ny - A.
 */
double orc_absorb_factor(double y, double ny, double A, double sigma)
{
    double depth = 0.0;
    if (A <= 0.0)
        return 1.0;
    if (y < A)
        depth = (A - y) / A;
    else if (y > ny - A)
        depth = (y - (ny - A)) / A;
    if (depth > 1.0)
        depth = 1.0;
    return exp(-sigma * depth * depth);
}

void orc_absorb_y(const orc_grid* g, double A, double sigma, double* E, double* B)
{
    int64_t nc = ncells(g);
    for (int c = 0; c < 3; ++c)
        for (int64_t k = 0; k < g->nz; ++k)
            for (int64_t j = 0; j < g->ny; ++j) {
                double fe = orc_absorb_factor((double)j + E_STAGGER[c][1], (double)g->ny, A, sigma);
                double fb = orc_absorb_factor((double)j + B_STAGGER[c][1], (double)g->ny, A, sigma);
                for (int64_t i = 0; i < g->nx; ++i) {
                    int64_t idx = c * nc + cell_index(g, i, j, k);
                    E[idx] *= fe;
                    B[idx] *= fb;
                }
            }
}

/*
 * Laser antenna: a sheet of current along x on the node plane j = ja (the
 * Ex positions (i+1/2, ja, k)), added to J at the time t of the current
 * (t = (n + 1/2) dt for the step from n to n+1):
 *   Jx += J0 G(x, z) T(t) cos(omega (t - t0)),
 *   G = exp(-((x - xc)^2 + (z - zc)^2) / w0^2),  T = exp(-((t - t0) / tau)^2),
 *   J0 = -2 E0 cos(kappa / 2) / dy,
 * kappa being the wavenumber (per cell along y) that the Yee dispersion
 * relation gives for omega: sin(kappa / 2) = (dy / dt) sin(omega dt / 2).
 * On the Yee grid a sheet of surface current K oscillating at omega radiates
 * Ex = -K / (2 cos(kappa / 2)) to either side, so the plane wave leaving the
 * sheet has amplitude E0.  w0 <= 0: no transverse envelope (a plane sheet);
 * tau <= 0: no temporal envelope.  Returns ORC_ERR_ARG when omega has no
 * propagating wave on the grid.
 */
int orc_antenna_j0(double E0, double omega, double dt, double dy, double* J0)
{
    double sk = (dy / dt) * sin(0.5 * omega * dt);
    if (!(fabs(sk) < 1.0))
        return ORC_ERR_ARG;
    double kappa = 2.0 * asin(sk);
    *J0 = -2.0 * E0 * cos(0.5 * kappa) / dy;
    return ORC_OK;
}

int orc_antenna(const orc_grid* g, int64_t ja, double E0, double omega, double w0, double xc,
                double zc, double tau, double t0, double dt, double t, double* J)
{
    double J0;
    if (orc_antenna_j0(E0, omega, dt, g->dy, &J0) != ORC_OK)
        return ORC_ERR_ARG;
    double T = tau > 0.0 ? exp(-((t - t0) / tau) * ((t - t0) / tau)) : 1.0;
    double amp = J0 * T * cos(omega * (t - t0));
    for (int64_t k = 0; k < g->nz; ++k)
        for (int64_t i = 0; i < g->nx; ++i) {
            double x = ((double)i + 0.5) * g->dx, z = (double)k * g->dz;
            double r2 = (x - xc) * (x - xc) + (z - zc) * (z - zc);
            double G = w0 > 0.0 ? exp(-r2 / (w0 * w0)) : 1.0;
            J[cell_index(g, i, ja, k)] += amp * G;
        }
    return ORC_OK;
}

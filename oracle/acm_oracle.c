/*
 * acm_oracle.c -- FP64 CPU oracle of the conservative Allen-Cahn multiphase
 * lattice Boltzmann method (Holzer, Bauer, Koestler, Ruede, arXiv 2012.06144).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this code.  It shares nothing with the
 * CUDA library (no headers, tables or helpers); the two agree only on the
 * documented interface conventions (cell index x + nx*(y + ny*z), the
 * direction numbering, structure-of-arrays population planes).
 *
 * Everything is written out plainly, one cell at a time, in the paper's
 * notation (Section 3.1 "LB model for interface tracking", Section 3.2 "LB model
 * for hydrodynamics"), with the time levels of Algorithm 2 made explicit:
 *
 *   phase step(k):  phi_k = sum_i h_i^k                       (eq:updatePhaseField)
 *                   n, theta from the stored field Phi^{k-1}  (eq:interfaceTracking)
 *                   h^eq = phi_k Gamma_i(u_{k-1})
 *                   h* = h - w_phi (h - h^eq) + (1 - w_phi/2) F^phi  (eq:lb_interface, SRT)
 *                   stream h*  ->  h^{k+1};  store Phi^k = phi_k
 *   hydro step(k):  everything from Phi^k                     (Section 3.2)
 *                   forces F_p, F_s, F_mu, F_b;  u_k            (eq:forceHydro, eq:updateVelocityField)
 *                   weighted-orthogonal MRT with moment-space forcing
 *                   (eq:improved_collision) -> stream g* -> g^{k+1}
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *  - phase collision is single-relaxation-time with rate w_phi = 1/(tau_phi + 1/2),
 *    tau_phi = M / c_s^2 (shifted convention, as for nu = tau c_s^2 and s_nu = 1/(tau+1/2));
 *  - normal n = G/|G|, and n = 0 when |G|^2 <= 1e-24;
 *  - theta uses Phi^{k-1} at the cell (flag: the local phi_k instead);
 *  - phase gradient with the phase lattice's weights, hydro gradient/Laplacian with the hydro
 *    lattice's weights;
 *  - viscous force from the non-equilibrium second moments built with the
 *    velocity u' that carries all forces except F_mu itself;
 *  - every second-order moment (trace included) relaxes with s_nu, all other
 *    moments with rate 1; the force enters the first moments only;
 *  - walls: half-way bounce-back for h and g, mirrored ghost values of Phi;
 *  - buoyancy F_b = (rho - rho_ref) g;
 *  - optional clamp of phi to [0,1] inside rho and tau only (flag, default off).
 *
 * Because the hydro collision relaxes all second-order moments at one rate and
 * every moment of degree >= 3 at rate 1 with zero equilibrium, the product
 * M^{-1} [m - S (m - m^eq + F_m/2) + F_m] of eq:improved_collision reduces,
 * in any basis that is orthogonal under the weights w_i and built in degree
 * order, to the Hermite form used in hydro_cell below.  The test-suite checks
 * that reduction against a literal Gram-Schmidt moment-matrix implementation.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Lattices.  Directions are numbered: rest; the six faces (+x,-x,+y,-y,+z,-z);
 * the twelve edges; the eight corners, each direction followed by its opposite.
 * D3Q19 is the first 19 of the D3Q27 list, D3Q15 is rest + faces + corners, and
 * D2Q9 (the two-dimensional pair of Section 5.1) is rest + the four x, y faces +
 * the four xy edges.                                                         */

static const int E27[27][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},
    {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},
    {1, 1, 1},   {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};

typedef struct {
    int q;
    int dim; /* 3, or 2 for D2Q9 (velocities in the xy plane) */
    int e[27][3];
    double w[27];
    int opp[27];
} lattice;

/* Textbook weights of the lattices, selected by |e|^2. */
static double lattice_weight(int q, int e2) {
    if (q == 9) {
        static const double w9[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
        return w9[e2];
    }
    if (q == 15) {
        static const double w15[4] = {2.0 / 9.0, 1.0 / 9.0, 0.0, 1.0 / 72.0};
        return w15[e2];
    }
    if (q == 19) {
        static const double w19[4] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0, 0.0};
        return w19[e2];
    }
    static const double w27[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    return w27[e2];
}

static int make_lattice(lattice *L, int q) {
    int src[27], n = 0;
    if (q == 15) {
        for (int i = 0; i < 7; ++i) src[n++] = i;
        for (int i = 19; i < 27; ++i) src[n++] = i;
    } else if (q == 19 || q == 27) {
        for (int i = 0; i < q; ++i) src[n++] = i;
    } else if (q == 9) {
        for (int i = 0; i < 5; ++i) src[n++] = i;
        for (int i = 7; i < 11; ++i) src[n++] = i;
    } else {
        return -1;
    }
    L->q = q;
    L->dim = q == 9 ? 2 : 3;
    for (int i = 0; i < q; ++i) {
        const int *v = E27[src[i]];
        L->e[i][0] = v[0];
        L->e[i][1] = v[1];
        L->e[i][2] = v[2];
        L->w[i] = lattice_weight(q, v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }
    for (int i = 0; i < q; ++i) {
        L->opp[i] = -1;
        for (int j = 0; j < q; ++j)
            if (L->e[j][0] == -L->e[i][0] && L->e[j][1] == -L->e[i][1] && L->e[j][2] == -L->e[i][2])
                L->opp[i] = j;
    }
    return 0;
}

/* Exported for the tests: velocities, weights and opposites of one lattice. */
int orc_lattice_table(int q, int *e, double *w, int *opp) {
    lattice L;
    if (make_lattice(&L, q)) return -1;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = L.e[i][a];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
    }
    return q;
}

/* ------------------------------------------------------------------------ */
/* Problem statement (Section 3) and the parameters derived from it.          */

typedef struct {
    int nx, ny, nz;
    int wall[3];      /* 0: periodic axis, 1: no-slip walls on both faces     */
    int q_hydro;      /* 19 or 27                                             */
    double rho_H, rho_L;
    double nu_H, nu_L; /* kinematic viscosities of heavy and light fluid      */
    double sigma, xi, mobility;
    double gravity[3];
    double rho_ref;   /* buoyancy reference density: F_b = (rho - rho_ref) g  */
    int theta_from_local_phi; /* reading flag, default 0                      */
    int clamp_phi;            /* reading flag, default 0                      */
    int phase_mrt;            /* 0: SRT phase collision (Section 5's D3Q15 SRT);
                                 1: MRT of Section 3.1 -- first-order moments
                                 relaxed with omega_phi, all others with 1, in a
                                 weighted-orthogonal moment basis              */
    int q_phase;              /* phase-field lattice: 15 (Section 5), 19 or 27 (the
                                 stencil pairs of Section 5.1); 0 reads as 15  */
} orc_problem;

static int phase_q(const orc_problem *P) { return P->q_phase ? P->q_phase : 15; }

typedef struct {
    double tau_H, tau_L;   /* nu = tau c_s^2 (Section 3.2)                    */
    double omega_phi;      /* 1/(tau_phi + 1/2), M = tau_phi c_s^2 (eq:mobility) */
    double beta, kappa;    /* beta = 12 sigma/xi, kappa = 3 sigma xi / 2      */
} derived;

static const double CS2 = 1.0 / 3.0;

static derived derive(const orc_problem *P) {
    derived d;
    d.tau_H = P->nu_H / CS2;
    d.tau_L = P->nu_L / CS2;
    double tau_phi = P->mobility / CS2;
    d.omega_phi = 1.0 / (tau_phi + 0.5);
    d.beta = 12.0 * P->sigma / P->xi;
    d.kappa = 1.5 * P->sigma * P->xi;
    return d;
}

/* Exported for the tests: tau_H, tau_L, omega_phi, beta, kappa. */
void orc_derived(const orc_problem *P, double out[5]) {
    derived d = derive(P);
    out[0] = d.tau_H;
    out[1] = d.tau_L;
    out[2] = d.omega_phi;
    out[3] = d.beta;
    out[4] = d.kappa;
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers.                                                          */

static long cell_index(const orc_problem *P, int x, int y, int z) {
    return (long)x + (long)P->nx * ((long)y + (long)P->ny * (long)z);
}

static long ncells(const orc_problem *P) { return (long)P->nx * P->ny * P->nz; }

/* Coordinate of a stencil neighbour: wrap on periodic axes, mirror (clamp) on
 * walled axes, i.e. the ghost value beyond a wall repeats the first interior
 * cell. */
static int stencil_coord(int c, int n, int walled) {
    if (walled) {
        if (c < 0) return 0;
        if (c >= n) return n - 1;
        return c;
    }
    return ((c % n) + n) % n;
}

/* The 3x3x3 neighbourhood of a scalar field around (x,y,z), indexed
 * (dz+1)*9 + (dy+1)*3 + (dx+1). */
static void gather_stencil(const orc_problem *P, const double *f, int x, int y, int z, double nb[27]) {
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int cx = stencil_coord(x + dx, P->nx, P->wall[0]);
                int cy = stencil_coord(y + dy, P->ny, P->wall[1]);
                int cz = stencil_coord(z + dz, P->nz, P->wall[2]);
                nb[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = f[cell_index(P, cx, cy, cz)];
            }
}

static double nb_at(const double nb[27], const int e[3]) {
    return nb[(e[2] + 1) * 9 + (e[1] + 1) * 3 + (e[0] + 1)];
}

/* eq:grad with Delta x = c = 1: grad phi = (1/c_s^2) sum_i e_i w_i phi(x + e_i). */
static void stencil_gradient(const lattice *L, const double nb[27], double grad[3]) {
    grad[0] = grad[1] = grad[2] = 0.0;
    for (int i = 0; i < L->q; ++i) {
        double v = nb_at(nb, L->e[i]);
        for (int a = 0; a < 3; ++a) grad[a] += L->e[i][a] * L->w[i] * v;
    }
    for (int a = 0; a < 3; ++a) grad[a] /= CS2;
}

/* eq:lap with Delta x = c = 1: lap phi = (2/c_s^2) sum_i w_i [phi(x + e_i) - phi(x)]. */
static double stencil_laplacian(const lattice *L, const double nb[27]) {
    double centre = nb[13], s = 0.0;
    for (int i = 0; i < L->q; ++i) s += L->w[i] * (nb_at(nb, L->e[i]) - centre);
    return 2.0 * s / CS2;
}

/* Exported for the tests: gradient and Laplacian of a whole field with the
 * weights of lattice q and the box's boundary handling. */
int orc_gradient_laplacian(const orc_problem *P, int q, const double *phi, double *grad, double *lap) {
    lattice L;
    if (make_lattice(&L, q)) return -1;
    long N = ncells(P);
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                double nb[27], g[3];
                gather_stencil(P, phi, x, y, z, nb);
                stencil_gradient(&L, nb, g);
                long c = cell_index(P, x, y, z);
                for (int a = 0; a < 3; ++a) grad[a * N + c] = g[a];
                lap[c] = stencil_laplacian(&L, nb);
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 3.1: one phase-field collision at one cell.
 *   h      : the q_phase pre-collision populations h_i^k(x)
 *   nbprev : 3x3x3 neighbourhood of the stored phase field Phi^{k-1}
 *   u      : velocity u_{k-1}(x) of the previous hydrodynamic step
 * Outputs the post-collision populations and phi_k = sum_i h_i.            */
void orc_phase_cell(const orc_problem *P, const double *h, const double *nbprev, const double *u,
                    double *hstar, double *phi_out) {
    lattice L;
    make_lattice(&L, phase_q(P));
    derived d = derive(P);
    const int Q = L.q;

    /* eq:updatePhaseField */
    double phi = 0.0;
    for (int i = 0; i < Q; ++i) phi += h[i];

    /* interface normal from the isotropic gradient (eq:grad, phase-lattice weights) */
    double G[3], n[3];
    stencil_gradient(&L, nbprev, G);
    double G2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    if (G2 <= 1e-24) {
        n[0] = n[1] = n[2] = 0.0;
    } else {
        double inv = 1.0 / sqrt(G2);
        for (int a = 0; a < 3; ++a) n[a] = G[a] * inv;
    }

    /* theta = (1 - 4 (phi - phi_0)^2) / xi, phi_0 = 1/2 (eq:allen_cahn) */
    const double phi0 = 0.5;
    double phi_theta = P->theta_from_local_phi ? phi : nbprev[13];
    double theta = (1.0 - 4.0 * (phi_theta - phi0) * (phi_theta - phi0)) / P->xi;

    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double heq[27], F[27];
    for (int i = 0; i < Q; ++i) {
        double eu = L.e[i][0] * u[0] + L.e[i][1] * u[1] + L.e[i][2] * u[2];
        double en = L.e[i][0] * n[0] + L.e[i][1] * n[1] + L.e[i][2] * n[2];
        /* Gamma_i (Section 3.1) and h^eq = phi Gamma_i */
        double Gamma = L.w[i] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
        heq[i] = phi * Gamma;
        /* eq:interfaceTracking */
        F[i] = theta * L.w[i] * en;
    }
    if (!P->phase_mrt) {
        /* eq:lb_interface with Omega = omega_phi * identity */
        for (int i = 0; i < Q; ++i) hstar[i] = h[i] + d.omega_phi * (heq[i] - h[i] - 0.5 * F[i]) + F[i];
    } else {
        /* eq:lb_interface with Omega = M^-1 S M.  In a moment basis orthogonal
         * under the weights w (sum_i w_i M_ki M_li = 0 for k != l), the part of a
         * vector y in the first-order moments is w_i e_i . (sum_j e_j y_j) / c_s^2;
         * S relaxes those with omega_phi and every other moment with 1, so
         * Omega y = y - (1 - omega_phi) w_i e_i . (sum_j e_j y_j) / c_s^2. */
        double y[27], J[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            y[i] = heq[i] - h[i] - 0.5 * F[i];
            for (int a = 0; a < 3; ++a) J[a] += L.e[i][a] * y[i];
        }
        for (int i = 0; i < Q; ++i) {
            double eJ = L.e[i][0] * J[0] + L.e[i][1] * J[1] + L.e[i][2] * J[2];
            double Oy = y[i] - (1.0 - d.omega_phi) * L.w[i] * eJ / CS2;
            hstar[i] = h[i] + Oy + F[i];
        }
    }
    *phi_out = phi;
}

/* ------------------------------------------------------------------------ */
/* Section 3.2: one hydrodynamic collision at one cell.
 *   g   : the q_hydro pre-collision populations g_i^k(x)
 *   nb  : 3x3x3 neighbourhood of Phi^k
 * Outputs the post-collision populations, the velocity u_k (eq:updateVelocityField)
 * and, for the tests, aux = {rho, p*, s_nu, tau, F_x, F_y, F_z, mu_phi,
 * Fmu_x, Fmu_y, Fmu_z}.                                                     */
void orc_hydro_cell(const orc_problem *P, const double *g, const double *nb, double *gstar, double *u_out,
                    double *aux) {
    lattice L;
    make_lattice(&L, P->q_hydro);
    derived d = derive(P);
    const int Q = L.q;
    const double phi_L = 0.0, phi_H = 1.0, phi0 = 0.5;

    double phi = nb[13];
    double grad_phi[3];
    stencil_gradient(&L, nb, grad_phi);
    double lap_phi = stencil_laplacian(&L, nb);

    double phi_m = phi; /* phi used inside rho and tau */
    if (P->clamp_phi) phi_m = phi_m < 0.0 ? 0.0 : (phi_m > 1.0 ? 1.0 : phi_m);

    /* eq:density and its gradient */
    double rho = P->rho_L + (phi_m - phi_L) * (P->rho_H - P->rho_L);
    double grad_rho[3];
    for (int a = 0; a < 3; ++a) grad_rho[a] = (P->rho_H - P->rho_L) * grad_phi[a];

    /* relaxation time interpolation and s_nu */
    double tau = d.tau_L + (phi_m - phi_L) * (d.tau_H - d.tau_L);
    double s_nu = 1.0 / (tau + 0.5);

    /* eq:chemPot and eq:surfaceTension */
    double mu_phi = 4.0 * d.beta * (phi - phi_L) * (phi - phi_H) * (phi - phi0) - d.kappa * lap_phi;
    double F_s[3];
    for (int a = 0; a < 3; ++a) F_s[a] = mu_phi * grad_phi[a];

    /* p* = sum g_i and eq:pressure_force */
    double pstar = 0.0;
    for (int i = 0; i < Q; ++i) pstar += g[i];
    double F_p[3];
    for (int a = 0; a < 3; ++a) F_p[a] = -pstar * CS2 * grad_rho[a];

    /* buoyancy */
    double F_b[3];
    for (int a = 0; a < 3; ++a) F_b[a] = (rho - P->rho_ref) * P->gravity[a];

    /* first and second moments of g */
    double j[3] = {0, 0, 0}, m2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a) {
            j[a] += g[i] * L.e[i][a];
            for (int b = 0; b < 3; ++b) m2[a][b] += g[i] * L.e[i][a] * L.e[i][b];
        }

    /* velocity without the viscous force, for its own non-equilibrium */
    double up[3];
    for (int a = 0; a < 3; ++a) up[a] = j[a] + (F_p[a] + F_s[a] + F_b[a]) / (2.0 * rho);

    /* eq:viscousForce: sum_i e_a e_b [Omega (g - g^eq)]_i = s_nu (m2 - m2^eq),
     * m2^eq = p* c_s^2 delta + u'u'  (second moment of g^eq) */
    double Pi_neq[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < L.dim; ++a)
        for (int b = 0; b < L.dim; ++b)
            Pi_neq[a][b] = m2[a][b] - (a == b ? pstar * CS2 : 0.0) - up[a] * up[b];
    double nu = tau * CS2;
    double F_mu[3];
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int b = 0; b < 3; ++b) s += s_nu * Pi_neq[a][b] * grad_rho[b];
        F_mu[a] = -(nu / CS2) * s;
    }

    /* eq:forceHydro and eq:updateVelocityField */
    double F[3], u[3];
    for (int a = 0; a < 3; ++a) {
        F[a] = F_p[a] + F_s[a] + F_mu[a] + F_b[a];
        u[a] = j[a] + F[a] / (2.0 * rho);
    }

    /* eq:improved_collision in Hermite form:
     *  zeroth moment   p*            (rate 1, equilibrium p*)
     *  first moments   u + F/(2 rho) (rate 1, equilibrium u, forcing F/rho)
     *  second (Hermite) a2* = (1 - s_nu) a2 + s_nu u u
     *  higher moments  0             (rate 1, equilibrium 0)
     * The Hermite tensors run over the lattice's own dimensions (x, y for D2Q9). */
    const int D = L.dim;
    double a2s[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            double a2 = m2[a][b] - (a == b ? pstar * CS2 : 0.0);
            a2s[a][b] = (1.0 - s_nu) * a2 + s_nu * u[a] * u[b];
        }
    double m1s[3];
    for (int a = 0; a < 3; ++a) m1s[a] = u[a] + F[a] / (2.0 * rho);
    for (int i = 0; i < Q; ++i) {
        double first = 0.0, second = 0.0;
        for (int a = 0; a < D; ++a) {
            first += L.e[i][a] * m1s[a];
            for (int b = 0; b < D; ++b)
                second += (L.e[i][a] * L.e[i][b] - (a == b ? CS2 : 0.0)) * a2s[a][b];
        }
        gstar[i] = L.w[i] * (pstar + first / CS2 + second / (2.0 * CS2 * CS2));
    }

    for (int a = 0; a < 3; ++a) u_out[a] = u[a];
    if (aux) {
        aux[0] = rho;
        aux[1] = pstar;
        aux[2] = s_nu;
        aux[3] = tau;
        aux[4] = F[0];
        aux[5] = F[1];
        aux[6] = F[2];
        aux[7] = mu_phi;
        aux[8] = F_mu[0];
        aux[9] = F_mu[1];
        aux[10] = F_mu[2];
    }
}

/* ------------------------------------------------------------------------ */
/* Streaming: h*_i(x) moves to x + e_i.  Periodic axes wrap; if x + e_i leaves
 * the box through a walled face, the population bounces back half-way and
 * becomes h_{opp(i)}(x) of the next step.                                     */
static void stream_push(const orc_problem *P, const lattice *L, const double *fstar, int x, int y, int z,
                        double *fnext) {
    long N = ncells(P);
    int n[3] = {P->nx, P->ny, P->nz};
    int c[3] = {x, y, z};
    for (int i = 0; i < L->q; ++i) {
        int dst[3], bounce = 0;
        for (int a = 0; a < 3; ++a) {
            int t = c[a] + L->e[i][a];
            if (t < 0 || t >= n[a]) {
                if (P->wall[a]) bounce = 1;
                t = ((t % n[a]) + n[a]) % n[a];
            }
            dst[a] = t;
        }
        if (bounce)
            fnext[(long)L->opp[i] * N + cell_index(P, x, y, z)] = fstar[i];
        else
            fnext[(long)i * N + cell_index(P, dst[0], dst[1], dst[2])] = fstar[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Whole-box steps (two grids, push streaming).                              */

/* Phase step(k): h -> h_next, stores Phi^k = sum h^k in phi_now. */
void orc_phase_step(const orc_problem *P, const double *h, const double *phi_prev, const double *u_prev,
                    double *h_next, double *phi_now) {
    lattice L;
    make_lattice(&L, phase_q(P));
    long N = ncells(P);
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long c = cell_index(P, x, y, z);
                double hl[27], hs[27], nb[27], u[3], phi;
                for (int i = 0; i < L.q; ++i) hl[i] = h[(long)i * N + c];
                gather_stencil(P, phi_prev, x, y, z, nb);
                for (int a = 0; a < 3; ++a) u[a] = u_prev[a * N + c];
                orc_phase_cell(P, hl, nb, u, hs, &phi);
                phi_now[c] = phi;
                stream_push(P, &L, hs, x, y, z, h_next);
            }
}

/* Hydro step(k): g -> g_next using Phi^k; stores u_k. */
void orc_hydro_step(const orc_problem *P, const double *g, const double *phi, double *g_next, double *u_now) {
    lattice L;
    make_lattice(&L, P->q_hydro);
    long N = ncells(P);
    const int Q = L.q;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long c = cell_index(P, x, y, z);
                double gl[27], gs[27], nb[27], u[3];
                for (int i = 0; i < Q; ++i) gl[i] = g[(long)i * N + c];
                gather_stencil(P, phi, x, y, z, nb);
                orc_hydro_cell(P, gl, nb, gs, u, NULL);
                for (int a = 0; a < 3; ++a) u_now[a * N + c] = u[a];
                stream_push(P, &L, gs, x, y, z, g_next);
            }
}

/* Macroscopic fields from (g^k, Phi^k): u_k by the hydro-step formulas and the
 * pressure p = p* rho c_s^2 (p* = p / (rho c_s^2), Section 3.2). */
void orc_fields(const orc_problem *P, const double *g, const double *phi, double *u, double *p) {
    lattice L;
    make_lattice(&L, P->q_hydro);
    long N = ncells(P);
    const int Q = L.q;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long c = cell_index(P, x, y, z);
                double gl[27], gs[27], nb[27], uc[3], aux[11];
                for (int i = 0; i < Q; ++i) gl[i] = g[(long)i * N + c];
                gather_stencil(P, phi, x, y, z, nb);
                orc_hydro_cell(P, gl, nb, gs, uc, aux);
                for (int a = 0; a < 3; ++a) u[a * N + c] = uc[a];
                p[c] = aux[1] * aux[0] * CS2;
            }
}

/* Initial state: h_i = phi0 w_i (= phi Gamma_i at u = 0), g_i = 0 (p* = 0,
 * u = 0), Phi^{-1} = phi0, u_{-1} = 0. */
void orc_init(const orc_problem *P, const double *phi0, double *h, double *g, double *phi_prev, double *u_prev) {
    lattice LP, LG;
    make_lattice(&LP, phase_q(P));
    make_lattice(&LG, P->q_hydro);
    long N = ncells(P);
    for (long c = 0; c < N; ++c) {
        for (int i = 0; i < LP.q; ++i) h[(long)i * N + c] = LP.w[i] * phi0[c];
        for (int i = 0; i < LG.q; ++i) g[(long)i * N + c] = 0.0;
        phi_prev[c] = phi0[c];
        for (int a = 0; a < 3; ++a) u_prev[a * N + c] = 0.0;
    }
}

/* Advances the state (h^k, g^k, Phi^{k-1}, u_{k-1}) by nsteps time steps of
 * Algorithm 2: phase step, then hydro step. */
int orc_run(const orc_problem *P, double *h, double *g, double *phi_prev, double *u_prev, long nsteps) {
    long N = ncells(P);
    int Q = P->q_hydro, QP = phase_q(P);
    double *h2 = malloc(sizeof(double) * QP * N);
    double *g2 = malloc(sizeof(double) * Q * N);
    double *phi_now = malloc(sizeof(double) * N);
    if (!h2 || !g2 || !phi_now) {
        free(h2);
        free(g2);
        free(phi_now);
        return -1;
    }
    for (long k = 0; k < nsteps; ++k) {
        orc_phase_step(P, h, phi_prev, u_prev, h2, phi_now);
        orc_hydro_step(P, g, phi_now, g2, u_prev);
        memcpy(h, h2, sizeof(double) * QP * N);
        memcpy(g, g2, sizeof(double) * Q * N);
        memcpy(phi_prev, phi_now, sizeof(double) * N);
    }
    free(h2);
    free(g2);
    free(phi_now);
    return 0;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

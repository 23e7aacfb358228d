/*
 * ORACLE for the lattice-Boltzmann discrete particle simulation (LB-DPS) of
 * Wang, Zhang, Wang, Ge and Li, "Lattice Boltzmann based discrete simulation
 * for gas-solid fluidization" (arXiv 1303.2653).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64 CPU
 * restatement of one coupled time step, used to check the CUDA library.  Only
 * the tests, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never calls it.  It shares no code,
 * tables or helpers with the CUDA library.  Compile with -ffp-contract=off so
 * that no multiply-add is fused.
 *
 * Units: lattice units throughout (h = 1, dt = 1, reference gas density 1).
 * The SI inputs are converted in ob_units() (Tables 1-2 give the conversion).
 *
 * One step (Fig. 4, steps 2-6, with the cell sort at the end of the step so
 * that it serves both the collision search and the next deposition):
 *   deposit   n_tot, v_s (Eq. 8), eps_2d (Eq. 10), eps_3d (Eq. 11), omega (Eq. 20)
 *   collide   u (Eq. 24), LES tau_t (Eq. 13-15), Eq. 23 with Omega^s (Eq. 7),
 *             gamma (Eq. 9), F_p->g (Eq. 25), node beta (Eq. 19, 21, 22)
 *   stream    Eq. 2 (push), half-way bounce-back walls, velocity inlet,
 *             pressure outlet, periodic faces
 *   contacts  soft spheres only (R25): spring-dashpot contact forces
 *   drag      bilinear interpolation (step 4), Eq. 26-28
 *   integrate Eq. 16 (symplectic Euler), specular walls, periodic wrap
 *   sort      by (cell, id)
 *   collide   hard spheres only: TDHS detection (contact + approach, §2.2)
 *             and Eq. 17-18
 *
 * Readings of passages that are silent, ambiguous or garbled (each is listed
 * with its reason in the design notes):
 *   R1  Eq. 4 diagonal velocities: the printed angle (i-5)pi/2 yields
 *       off-lattice vectors; the standard +pi/4 phase is used.
 *   R2  n_tot counts particles whose centre lies in the cell.
 *   R3  Eq. 10 area fraction is capped at 2D close packing pi/(2 sqrt 3).
 *   R4  gamma uses the 2D solid fraction; beta, omega, Re_p and Eq. 26 use
 *       eps_g = eps_3d (Eq. 11).  In 3D eps_s is the sphere volume fraction
 *       (capped at pi/(3 sqrt 2)) and eps_g = 1 - eps_s.
 *   R5  omega = 1 for eps_g <= 0.74 (Eq. 20 has no branch there).
 *   R6  Eq. 24 is solved in closed form (it is linear in u); a gas body force
 *       F_b enters with the usual half-force term.
 *   R7  Eq. 15 with the density kept: tau_t = (tau + sqrt(tau^2 + 18 Cs^2 Q/rho))/2.
 *   R8  Eq. 23 literally: gamma(eps_s, tau_t) in the relaxation term and
 *       gamma(eps_s, tau) in the solid term.  Body force by Guo's source term.
 *   R9  Walls: half-way bounce-back (moving-wall variant for closed-form
 *       tests).  Inlet: incoming populations at feq(1, u_in), u_in that of
 *       the receiving cell's own column of the inlet face.  Outlet: incoming
 *       populations at feq(1, u of the receiving cell).
 *   R10 Node fields (rho, u, beta) are the collision-time values of the same
 *       step; superficial -> actual velocity divides by eps_2d (flag).
 *   R11 Bilinear (trilinear) interpolation from cell-centre nodes, clamped at
 *       walls and wrapped at periodic faces.
 *   R12 Eq. 28 with |S| <= 1e-12 sum|F_pre| uses the scale 1.
 *   R13 Eq. 16 integrated by symplectic Euler with -V_p grad p (flag for the
 *       printed +); effective gravity (1 - rho_g/rho_s) g (§3).
 *   R14 Collision rule: each particle picks its approaching contact of
 *       smallest distance (ties to the smaller id); mutual picks collide by
 *       Eq. 17-18 on pre-collision velocities; wall contacts (the wall is an
 *       infinitely heavy particle at rest) apply to the rest.
 *   R15 A 2D cell is h x h x h: Eq. 25 carries h^2/dt = 1 in lattice units
 *       and a particle is a sphere, m_p = rho_s pi d^3 / 6.
 *   R16 The gas density in Eq. 19, 21 and 22 is the reference density (1 in
 *       lattice units), not the local rho.
 *   R17 Every lattice quantity is derived from the SI columns of Tables 1-2
 *       (two printed dimensionless entries are garbled).
 *   R18 Particles in a cell are ordered by id, which fixes every summation
 *       order (Eq. 8, 27).
 *   R19 The bed-mean voidage is that of the current positions (Eq. 10-11
 *       from a fresh count), not of the last deposition.
 *   R21 Solids loop of the circulating bed (§3.2): a particle that crosses
 *       the outlet re-enters through the inlet face at the same lateral
 *       position and velocity and is counted; the outlet makes no contact.
 *   R23 Bubble regions (§3.1): cells whose voidage exceeds the threshold,
 *       connected along the axes; a region reaching the top row is freeboard.
 *   R25 Soft spheres, the DEM option of §2.2 for dense beds: each pair closer
 *       than d and each face closer than r pushes with max(0, k_n delta -
 *       eta v_n) along the line of centres, eta = 2 zeta sqrt(m_eff k_n),
 *       zeta = -ln e / sqrt(pi^2 + ln^2 e), m_eff = m/2 (pair) or m (wall);
 *       forces from the state at the start of the step, added in Eq. 16.
 *   R26 Friction of soft spheres (the tangential contact force §2.2 credits
 *       DEM with): at the contact point (half way between two centres, or on
 *       the face) the tangential slip v_t meets -min(gamma_t |v_t|, mu F_n)
 *       v_t / |v_t|; its torque turns the particles (I = 2/5 m r^2, one spin
 *       component in 2D, three in 3D), with the spin updated from the
 *       start-of-step torques.
 *   R27 Optional sequential hard-sphere rule (test only): every pair in
 *       contact in (id_i, id_j) order, resolved from the velocities the
 *       earlier ones left if it approaches then; then the walls.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OB_MAXQ 19

enum { OB_WALL = 0, OB_PERIODIC = 1, OB_INLET = 2, OB_OUTLET = 3 };

/* ---- SI description of a bed (mirrors the workload generator's fields) ---- */
typedef struct {
    int dim;
    int n[3];
    int bc[6];
    double h, dt;
    const double *inlet_u;   /* (cells of the inlet face) * dim, m/s, or NULL */
    double wall_u[6][3];     /* wall velocity per face, m/s */
    int64_t np;
    double d_p, rho_s, e;
    const double *pos;       /* np * dim, m */
    const double *vel;       /* np * dim, m/s */
    double rho_g, mu_g;
    double g[3], body_accel[3], u0[3];
    double cs_smag;
    int superficial_mode;    /* 0: u / eps_2d, 1: u / eps_g, 2: no conversion */
    int pressure_plus;       /* 1: +V_p grad p as printed in Eq. 16 */
    int recirculate;         /* 1: outlet -> inlet re-injection of particles (reading R21) */
    int collision_model;     /* 0: time-driven hard spheres (§2.2); 1: soft spheres (R25) */
    double dem_kn;           /* soft-sphere normal stiffness, N/m */
    double dem_mu;           /* soft-sphere Coulomb friction coefficient (R26; 0 = none) */
    double dem_gamma_t;      /* soft-sphere tangential damping, kg/s (R26) */
    int collision_rule;      /* hard spheres: 0 mutual nearest (R14), 1 sequential (R27) */
} ob_setup;

/* ---- lattice-unit constants derived from an ob_setup ---- */
typedef struct {
    double tau, nu, mu;      /* relaxation time (Eq. 3), viscosity */
    double rho_s;            /* solid density / gas density */
    double d, r, vp, mp;     /* diameter, radius, sphere volume, mass */
    double e;
    double g_eff[3];         /* (1 - rho_g/rho_s) g, §3 */
    double fb[3];            /* gas body force density */
    double u0[3];
    double wall_u[6][3];
    double cs_smag;
    double kn, eta, eta_w;   /* soft spheres: stiffness, pair and wall damping */
    double mu_f, gamma_t;    /* soft spheres: friction coefficient, tangential damping */
    double inertia;          /* moment of inertia of a particle, 2/5 m r^2 */
} ob_consts;

typedef struct {
    int dim, nq;
    int n[3];
    int64_t ncell;
    int bc[6];
    ob_consts k;
    int superficial_mode, pressure_plus;
    int recirculate;         /* reading R21 */
    int64_t solids_out;      /* particles that left through the outlet so far */
    double uscale;           /* SI velocity -> lattice units: dt / h */
    int c[OB_MAXQ][3];
    double w[OB_MAXQ];
    int opp[OB_MAXQ];
    double *f, *fnew;        /* nq * ncell, pre-collision populations */
    double *inlet_u;         /* inlet face cells * 3 (lattice units) */
    int inlet_face;          /* face index, -1 if none */
    /* node fields of the last step */
    int64_t *ntot;
    double *vs, *eps_s, *eps_2d, *eps_g, *omega;      /* deposition */
    double *rho, *u, *uact, *beta, *fpg, *tau_t;      /* collision */
    double *gradp;
    double *sum_pre, *sum_abs_pre;                    /* Eq. 27 per cell */
    /* particles, kept sorted by (cell, id) */
    int64_t np;
    double *P, *v;           /* np * 3 */
    int64_t *id, *cell;
    int64_t *cell_start;     /* ncell + 1 */
    double *fpre, *fd;       /* np * 3, sorted order, last step */
    double *fc;              /* np * 3, sorted order: soft-sphere contact forces */
    double *spin;            /* np * 3, sorted order: angular velocity (R26; z only in 2D) */
    double *tq;              /* np * 3, sorted order: contact torques of the step */
    int model;               /* collision model (0 hard, 1 soft spheres) */
    int rule;                /* hard-sphere rule: 0 mutual nearest, 1 sequential */
    double *diag_fpre, *diag_fd;   /* np * 3, id order, last step */
    double *diag_fc;               /* np * 3, id order, last step */
    int64_t *best;           /* chosen partner (id) or -1 */
    int *wall_hit;           /* bitmask of faces contacted */
    int64_t *pairs;          /* approaching contact pairs (id_i < id_j) */
    int64_t npairs, pairs_cap;
    int64_t steps;
} ob_bed;

/* ------------------------------------------------------------------------ */
/* Velocity sets.                                                             */
/* D2Q9 (§2.1, Eq. 4): c_0 = 0; c_1..4 = cos/sin((i-1)pi/2); c_5..8 along the */
/* diagonals (reading R1); weights 4/9, 1/9, 1/36.                           */
/* D3Q19 (the 3D extension named in §4): rest, 6 axis and 12 edge-diagonal    */
/* velocities with weights 1/3, 1/18, 1/36.                                   */
/* ------------------------------------------------------------------------ */
static void set_lattice(ob_bed *b)
{
    static const int c2[9][2] = {
        {0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    static const int c3[19][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    if (b->dim == 2) {
        b->nq = 9;
        for (int i = 0; i < 9; ++i) {
            b->c[i][0] = c2[i][0];
            b->c[i][1] = c2[i][1];
            b->c[i][2] = 0;
            b->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    } else {
        b->nq = 19;
        for (int i = 0; i < 19; ++i) {
            for (int a = 0; a < 3; ++a) b->c[i][a] = c3[i][a];
            b->w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
        }
    }
    for (int i = 0; i < b->nq; ++i) {
        for (int j = 0; j < b->nq; ++j) {
            if (b->c[j][0] == -b->c[i][0] && b->c[j][1] == -b->c[i][1] &&
                b->c[j][2] == -b->c[i][2]) b->opp[i] = j;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Closed-form pieces of the model, one per equation.                          */
/* ------------------------------------------------------------------------ */

/* Eq. 9: weighting function of Noble and Torczynski. */
double ob_gamma(double eps_s, double tau)
{
    return eps_s * (tau - 0.5) / ((1.0 - eps_s) + (tau - 0.5));
}

/* Eq. 11: 3D porosity from the 2D one (Ouyang and Li). */
double ob_eps3d(double eps_2d)
{
    return 1.0 - sqrt(2.0) / sqrt(M_PI * sqrt(3.0)) * pow(1.0 - eps_2d, 1.5);
}

/* Eq. 20: EMMS drag correction omega(eps_g) (reading R5 below 0.74). */
double ob_omega(double eps_g)
{
    if (eps_g <= 0.74) return 1.0;
    if (eps_g <= 0.82) {
        double t = eps_g - 0.7463;
        return 0.0214 / (4.0 * t * t + 0.0044) - 0.5760;
    }
    if (eps_g <= 0.97) {
        double t = eps_g - 0.7789;
        return 0.0038 / (4.0 * t * t + 0.0040) - 0.0101;
    }
    return 32.8295 * eps_g - 31.8295;
}

/* Eq. 22: particle Reynolds number. */
double ob_reynolds(double eps_g, double rho_g, double slip, double d, double mu)
{
    return eps_g * rho_g * slip * d / mu;
}

/*
 * Eq. 19 with Eq. 21-22: EMMS / Ergun inter-phase coefficient beta.
 * The dilute branch multiplies C_d0 by |u - v| before dividing by Re_p, which
 * is the same product written so that Re_p = 0 is finite:
 *   C_d0 |u-v| = 24 mu (1 + 0.15 Re^0.687) / (eps rho d)   for Re < 1000.
 */
double ob_beta(double eps_g, double slip, double rho_g, double mu, double d)
{
    if (eps_g > 0.74) {
        double omega = ob_omega(eps_g);
        double re = ob_reynolds(eps_g, rho_g, slip, d, mu);
        double cd0_slip;
        if (re < 1000.0)
            cd0_slip = 24.0 * mu * (1.0 + 0.15 * pow(re, 0.687)) / (eps_g * rho_g * d);
        else
            cd0_slip = 0.44 * slip;
        return 0.75 * (1.0 - eps_g) * eps_g * rho_g * cd0_slip / d * omega;
    }
    return 150.0 * (1.0 - eps_g) * (1.0 - eps_g) * mu / (eps_g * d * d) +
           1.75 * (1.0 - eps_g) * rho_g * slip / d;
}

/* Eq. 4: equilibrium distribution, c_s^2 = 1/3. */
static double feq(const ob_bed *b, int i, double rho, const double *u)
{
    const double cs2 = 1.0 / 3.0;
    double cu = 0.0, uu = 0.0;
    for (int a = 0; a < b->dim; ++a) {
        cu += b->c[i][a] * u[a];
        uu += u[a] * u[a];
    }
    return b->w[i] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
}

/*
 * Eq. 17-18: post-collision velocities of a binary collision.  n = P1 - P2,
 * g = v1 - v2.  A wall is the m2 -> infinity, v2 = 0 limit.
 */
void ob_binary_collision(int dim, double m1, double m2, double e, const double *p1,
                         const double *p2, double *v1, double *v2)
{
    double nvec[3], gdotn = 0.0, nn = 0.0;
    for (int a = 0; a < dim; ++a) {
        nvec[a] = p1[a] - p2[a];
        gdotn += (v1[a] - v2[a]) * nvec[a];
        nn += nvec[a] * nvec[a];
    }
    double k1 = (1.0 + e) * m2 / (m1 + m2) * gdotn / nn;
    double k2 = (1.0 + e) * m1 / (m1 + m2) * gdotn / nn;
    for (int a = 0; a < dim; ++a) {
        double n_a = nvec[a];
        v1[a] = v1[a] - k1 * n_a;
        v2[a] = v2[a] + k2 * n_a;
    }
}

/* ------------------------------------------------------------------------ */
/* Unit conversion (h = dt = 1, gas density 1), checked against Tables 1-2.    */
/* ------------------------------------------------------------------------ */
void ob_units(const ob_setup *s, ob_consts *k)
{
    double nu_si = s->mu_g / s->rho_g;
    k->nu = nu_si * s->dt / (s->h * s->h);
    k->mu = k->nu;                        /* gas density is 1 in lattice units */
    k->tau = 3.0 * k->nu + 0.5;           /* Eq. 3 with dt = 1 */
    k->rho_s = s->rho_s / s->rho_g;
    k->d = s->d_p / s->h;
    k->r = 0.5 * k->d;
    k->vp = M_PI * k->d * k->d * k->d / 6.0;
    k->mp = k->rho_s * k->vp;
    k->e = s->e;
    double gscale = s->dt * s->dt / s->h;
    double uscale = s->dt / s->h;
    for (int a = 0; a < 3; ++a) {
        k->g_eff[a] = (1.0 - s->rho_g / s->rho_s) * s->g[a] * gscale;
        k->fb[a] = s->body_accel[a] * gscale;
        k->u0[a] = s->u0[a] * uscale;
    }
    for (int f = 0; f < 6; ++f)
        for (int a = 0; a < 3; ++a) k->wall_u[f][a] = s->wall_u[f][a] * uscale;
    k->cs_smag = s->cs_smag;
    /* soft spheres (R25): F = k_n delta - eta v_n; the damping that gives the
     * restitution e to a linear spring-dashpot pair of reduced mass m/2 (and
     * to a particle against a wall, reduced mass m) */
    k->kn = s->dem_kn * s->dt * s->dt / (s->rho_g * s->h * s->h * s->h);
    k->mu_f = s->dem_mu;
    k->gamma_t = s->dem_gamma_t * s->dt / (s->rho_g * s->h * s->h * s->h);
    k->inertia = 0.4 * k->mp * k->r * k->r;
    k->eta = k->eta_w = 0.0;
    if (s->e > 0.0 && s->e < 1.0 && k->kn > 0.0) {
        double le = log(s->e);
        double z = -le / sqrt(M_PI * M_PI + le * le);
        k->eta = 2.0 * z * sqrt(0.5 * k->mp * k->kn);
        k->eta_w = 2.0 * z * sqrt(k->mp * k->kn);
    }
}

/* ------------------------------------------------------------------------ */
/* Bed life cycle.                                                            */
/* ------------------------------------------------------------------------ */
static int64_t cell_of(const ob_bed *b, const double *p)
{
    int64_t idx[3] = {0, 0, 0};
    for (int a = 0; a < b->dim; ++a) {
        int64_t q = (int64_t)floor(p[a]);
        if (q < 0) q = 0;
        if (q >= b->n[a]) q = b->n[a] - 1;
        idx[a] = q;
    }
    return idx[0] + (int64_t)b->n[0] * (idx[1] + (int64_t)b->n[1] * idx[2]);
}

static void sort_particles(ob_bed *b);

void ob_destroy(ob_bed *b)
{
    if (!b) return;
    void *ptrs[] = {b->f, b->fnew, b->inlet_u, b->ntot, b->vs, b->eps_s, b->eps_2d,
                    b->eps_g, b->omega, b->rho, b->u, b->uact, b->beta, b->fpg,
                    b->tau_t, b->gradp, b->sum_pre, b->sum_abs_pre, b->P, b->v, b->id,
                    b->cell, b->cell_start, b->fpre, b->fd, b->best, b->wall_hit,
                    b->pairs, b->diag_fpre, b->diag_fd, b->fc, b->diag_fc, b->spin, b->tq};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(b);
}

static int alloc_particles(ob_bed *b, int64_t np)
{
    free(b->P); free(b->v); free(b->id); free(b->cell); free(b->fpre); free(b->fd);
    free(b->best); free(b->wall_hit); free(b->diag_fpre); free(b->diag_fd); free(b->fc);
    free(b->diag_fc); free(b->spin); free(b->tq);
    size_t m = (size_t)(np > 0 ? np : 1);
    b->np = np;
    b->P = calloc(m * 3, sizeof(double));
    b->v = calloc(m * 3, sizeof(double));
    b->id = calloc(m, sizeof(int64_t));
    b->cell = calloc(m, sizeof(int64_t));
    b->fpre = calloc(m * 3, sizeof(double));
    b->fd = calloc(m * 3, sizeof(double));
    b->best = calloc(m, sizeof(int64_t));
    b->wall_hit = calloc(m, sizeof(int));
    b->diag_fpre = calloc(m * 3, sizeof(double));
    b->diag_fd = calloc(m * 3, sizeof(double));
    b->fc = calloc(m * 3, sizeof(double));
    b->diag_fc = calloc(m * 3, sizeof(double));
    b->spin = calloc(m * 3, sizeof(double));
    b->tq = calloc(m * 3, sizeof(double));
    return (b->P && b->v && b->id && b->cell && b->fpre && b->fd && b->best && b->wall_hit &&
            b->diag_fpre && b->diag_fd && b->fc && b->diag_fc && b->spin && b->tq);
}

ob_bed *ob_create(const ob_setup *s)
{
    if (s->dim != 2 && s->dim != 3) return NULL;
    /* the 3^dim cell search needs periodic axes of at least 3 cells and
     * particles no wider than a cell */
    for (int a = 0; a < s->dim; ++a) {
        if (s->n[a] < 1) return NULL;
        if (s->bc[2 * a] == OB_PERIODIC && s->n[a] < 3) return NULL;
    }
    if (!(s->d_p <= s->h)) return NULL;
    /* soft spheres need a stiffness and 0 < e <= 1 (R25) */
    if (s->collision_model != 0 && s->collision_model != 1) return NULL;
    if (s->collision_model == 1 && !(s->dem_kn > 0.0 && s->e > 0.0 && s->e <= 1.0)) return NULL;
    if (!(s->dem_mu >= 0.0) || !(s->dem_gamma_t >= 0.0)) return NULL;
    if (s->collision_rule != 0 && s->collision_rule != 1) return NULL;
    /* recirculation needs the inlet below and the outlet above (reading R21) */
    if (s->recirculate && !(s->bc[2 * (s->dim - 1)] == OB_INLET && s->bc[2 * s->dim - 1] == OB_OUTLET))
        return NULL;
    ob_bed *b = calloc(1, sizeof(ob_bed));
    if (!b) return NULL;
    b->dim = s->dim;
    b->n[0] = s->n[0];
    b->n[1] = s->n[1];
    b->n[2] = (s->dim == 3) ? s->n[2] : 1;
    b->ncell = (int64_t)b->n[0] * b->n[1] * b->n[2];
    for (int f = 0; f < 6; ++f) b->bc[f] = s->bc[f];
    if (s->dim == 2) b->bc[4] = b->bc[5] = OB_PERIODIC;
    ob_units(s, &b->k);
    b->superficial_mode = s->superficial_mode;
    b->pressure_plus = s->pressure_plus;
    b->recirculate = s->recirculate;
    b->model = s->collision_model;
    b->rule = s->collision_rule;
    b->solids_out = 0;
    b->uscale = s->dt / s->h;
    set_lattice(b);

    size_t nc = (size_t)b->ncell;
    b->f = calloc((size_t)b->nq * nc, sizeof(double));
    b->fnew = calloc((size_t)b->nq * nc, sizeof(double));
    b->ntot = calloc(nc, sizeof(int64_t));
    b->vs = calloc(nc * 3, sizeof(double));
    b->eps_s = calloc(nc, sizeof(double));
    b->eps_2d = calloc(nc, sizeof(double));
    b->eps_g = calloc(nc, sizeof(double));
    b->omega = calloc(nc, sizeof(double));
    b->rho = calloc(nc, sizeof(double));
    b->u = calloc(nc * 3, sizeof(double));
    b->uact = calloc(nc * 3, sizeof(double));
    b->beta = calloc(nc, sizeof(double));
    b->fpg = calloc(nc * 3, sizeof(double));
    b->tau_t = calloc(nc, sizeof(double));
    b->gradp = calloc(nc * 3, sizeof(double));
    b->sum_pre = calloc(nc * 3, sizeof(double));
    b->sum_abs_pre = calloc(nc * 3, sizeof(double));
    b->cell_start = calloc(nc + 1, sizeof(int64_t));
    if (!b->f || !b->fnew || !b->ntot || !b->vs || !b->eps_s || !b->eps_2d || !b->eps_g ||
        !b->omega || !b->rho || !b->u || !b->uact || !b->beta || !b->fpg || !b->tau_t ||
        !b->gradp || !b->sum_pre || !b->sum_abs_pre || !b->cell_start) {
        ob_destroy(b);
        return NULL;
    }

    /* inlet face: on the vertical (last) axis only */
    b->inlet_face = -1;
    int vert = b->dim - 1;
    int64_t nface = b->ncell / b->n[vert];
    b->inlet_u = calloc((size_t)nface * 3, sizeof(double));
    for (int f = 2 * vert; f <= 2 * vert + 1; ++f)
        if (b->bc[f] == OB_INLET) b->inlet_face = f;
    if (s->inlet_u) {
        double uscale = s->dt / s->h;
        for (int64_t j = 0; j < nface; ++j)
            for (int a = 0; a < b->dim; ++a)
                b->inlet_u[j * 3 + a] = s->inlet_u[j * b->dim + a] * uscale;
    }

    /* gas initially at equilibrium with rho = 1 and u = u0 */
    for (int64_t x = 0; x < b->ncell; ++x)
        for (int i = 0; i < b->nq; ++i)
            b->f[(size_t)i * nc + x] = feq(b, i, 1.0, b->k.u0);

    if (!alloc_particles(b, s->np)) { ob_destroy(b); return NULL; }
    for (int64_t p = 0; p < s->np; ++p) {
        b->id[p] = p;
        for (int a = 0; a < b->dim; ++a) {
            b->P[p * 3 + a] = s->pos[p * b->dim + a] / s->h;
            b->v[p * 3 + a] = s->vel[p * b->dim + a] * (s->dt / s->h);
        }
    }
    sort_particles(b);
    return b;
}

/* ------------------------------------------------------------------------ */
/* Sort by (cell, id): the cell list of Fig. 1.                               */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t cell, id, src; } sort_key;

static int cmp_key(const void *x, const void *y)
{
    const sort_key *a = x, *b = y;
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

static void sort_particles(ob_bed *b)
{
    int64_t np = b->np;
    sort_key *keys = malloc(sizeof(sort_key) * (size_t)(np > 0 ? np : 1));
    double *P2 = malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    double *v2 = malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    double *w2 = malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    for (int64_t p = 0; p < np; ++p) {
        keys[p].cell = cell_of(b, &b->P[p * 3]);
        keys[p].id = b->id[p];
        keys[p].src = p;
    }
    qsort(keys, (size_t)np, sizeof(sort_key), cmp_key);
    for (int64_t p = 0; p < np; ++p) {
        int64_t s = keys[p].src;
        for (int a = 0; a < 3; ++a) {
            P2[p * 3 + a] = b->P[s * 3 + a];
            v2[p * 3 + a] = b->v[s * 3 + a];
            w2[p * 3 + a] = b->spin[s * 3 + a];
        }
    }
    memcpy(b->P, P2, sizeof(double) * 3 * (size_t)np);
    memcpy(b->v, v2, sizeof(double) * 3 * (size_t)np);
    memcpy(b->spin, w2, sizeof(double) * 3 * (size_t)np);
    for (int64_t p = 0; p < np; ++p) {
        b->id[p] = keys[p].id;
        b->cell[p] = keys[p].cell;
    }
    for (int64_t c = 0; c <= b->ncell; ++c) b->cell_start[c] = 0;
    for (int64_t p = 0; p < np; ++p) b->cell_start[b->cell[p] + 1] += 1;
    for (int64_t c = 0; c < b->ncell; ++c) b->cell_start[c + 1] += b->cell_start[c];
    free(keys);
    free(P2);
    free(v2);
    free(w2);
}

/* ------------------------------------------------------------------------ */
/* Step 2 of Fig. 4: deposition of momentum (Eq. 8) and voidage (Eq. 10-11). */
/* ------------------------------------------------------------------------ */
/* Solid fraction (Eq. 10, capped at close packing, reading R3) and gas
 * voidage (Eq. 11 in 2D) of a cell holding n particle centres. */
static double voidage_of_count(const ob_bed *b, int64_t n, double *eps_s, double *eps_2d)
{
    const double cap2d = M_PI / (2.0 * sqrt(3.0));   /* close-packed discs (R3) */
    const double cap3d = M_PI / (3.0 * sqrt(2.0));   /* close-packed spheres */
    double es;
    if (b->dim == 2) {
        es = (double)n * M_PI * b->k.r * b->k.r;      /* Eq. 10, h = 1 */
        if (es > cap2d) es = cap2d;
    } else {
        es = (double)n * b->k.vp;
        if (es > cap3d) es = cap3d;
    }
    *eps_s = es;
    *eps_2d = 1.0 - es;
    return b->dim == 2 ? ob_eps3d(1.0 - es) : 1.0 - es;  /* Eq. 11 */
}

static void deposit(ob_bed *b)
{
    for (int64_t x = 0; x < b->ncell; ++x) {
        int64_t s = b->cell_start[x], t = b->cell_start[x + 1];
        int64_t n = t - s;
        double sum[3] = {0.0, 0.0, 0.0};
        for (int64_t p = s; p < t; ++p)
            for (int a = 0; a < 3; ++a) sum[a] += b->v[p * 3 + a];
        b->ntot[x] = n;
        for (int a = 0; a < 3; ++a) b->vs[x * 3 + a] = (n > 0) ? sum[a] / (double)n : 0.0;
        b->eps_g[x] = voidage_of_count(b, n, &b->eps_s[x], &b->eps_2d[x]);
        b->omega[x] = ob_omega(b->eps_g[x]);                      /* Eq. 20 */
    }
}

/* ------------------------------------------------------------------------ */
/* Step 3 of Fig. 4: modified LBE collision (Eq. 23) and streaming (Eq. 2).   */
/* ------------------------------------------------------------------------ */
static void neighbour(const ob_bed *b, int64_t x, const int *dir, int sign, int64_t *out,
                      int *wall_axis, int *open_axis)
{
    /* cell reached from x by sign*dir; reports the first wall axis crossed and
     * the first inlet/outlet axis crossed (-1 if none) */
    int64_t idx[3];
    idx[0] = x % b->n[0];
    idx[1] = (x / b->n[0]) % b->n[1];
    idx[2] = x / ((int64_t)b->n[0] * b->n[1]);
    *wall_axis = -1;
    *open_axis = -1;
    for (int a = 0; a < b->dim; ++a) {
        int64_t q = idx[a] + sign * dir[a];
        if (q < 0 || q >= b->n[a]) {
            int face = 2 * a + (q < 0 ? 0 : 1);
            int bc = b->bc[face];
            if (bc == OB_PERIODIC) {
                q = (q + b->n[a]) % b->n[a];
            } else if (bc == OB_WALL) {
                if (*wall_axis < 0) *wall_axis = face;
            } else {
                if (*open_axis < 0) *open_axis = face;
            }
        }
        idx[a] = q;
    }
    *out = idx[0] + (int64_t)b->n[0] * (idx[1] + (int64_t)b->n[1] * idx[2]);
}

static void collide_and_stream(ob_bed *b)
{
    const int nq = b->nq, dim = b->dim;
    const size_t nc = (size_t)b->ncell;
    const double tau = b->k.tau, cs = b->k.cs_smag;
    double *fstar = malloc(sizeof(double) * nq * nc);

    for (int64_t x = 0; x < b->ncell; ++x) {
        double fi[OB_MAXQ];
        for (int i = 0; i < nq; ++i) fi[i] = b->f[(size_t)i * nc + x];

        /* Eq. 5 moments */
        double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < nq; ++i) {
            rho += fi[i];
            for (int a = 0; a < dim; ++a) m[a] += b->c[i][a] * fi[i];
        }
        const double *vs = &b->vs[x * 3];
        double g_tau = ob_gamma(b->eps_s[x], tau);                /* Eq. 9 */
        double og = b->omega[x] * g_tau;                          /* omega*gamma */

        /*
         * Eq. 24, rho u = sum_i c_i (f_i + og/2 Omega^s_i) (+ F_b/2), is
         * linear in u.  Eq. 7 gives sum_i c_i Omega^s_i = rho u + rho v_s - 2m,
         * so rho u (1 - og/2) = m (1 - og) + og/2 rho v_s + F_b/2 (reading R6).
         */
        double u[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < dim; ++a)
            u[a] = (m[a] * (1.0 - og) + 0.5 * og * rho * vs[a] + 0.5 * b->k.fb[a]) /
                   (rho * (1.0 - 0.5 * og));

        double fe[OB_MAXQ], fe_s[OB_MAXQ];
        for (int i = 0; i < nq; ++i) {
            fe[i] = feq(b, i, rho, u);
            fe_s[i] = feq(b, i, rho, vs);
        }

        /* Eq. 13-15: Smagorinsky relaxation time (reading R7) */
        double tau_t = tau;
        if (cs > 0.0) {
            double qsum = 0.0;
            for (int a = 0; a < dim; ++a) {
                for (int bb = 0; bb < dim; ++bb) {
                    double qab = 0.0;
                    for (int i = 0; i < nq; ++i)
                        qab += b->c[i][a] * b->c[i][bb] * (fi[i] - fe[i]);
                    qsum += qab * qab;
                }
            }
            double qn = sqrt(2.0 * qsum);
            tau_t = 0.5 * (tau + sqrt(tau * tau + 18.0 * cs * cs * qn / rho));
        }
        double g_taut = ob_gamma(b->eps_s[x], tau_t);

        /* Eq. 7 and Eq. 23, plus the body-force source term (reading R8) */
        double fpg[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < nq; ++i) {
            int io = b->opp[i];
            double omega_s = fi[io] - fi[i] + fe_s[i] - fe[io];
            double src = 0.0;
            if (b->k.fb[0] != 0.0 || b->k.fb[1] != 0.0 || b->k.fb[2] != 0.0) {
                double cu = 0.0;
                for (int a = 0; a < dim; ++a) cu += b->c[i][a] * u[a];
                for (int a = 0; a < dim; ++a)
                    src += (3.0 * (b->c[i][a] - u[a]) + 9.0 * cu * b->c[i][a]) * b->k.fb[a];
                src *= (1.0 - 0.5 / tau_t) * b->w[i];
            }
            fstar[(size_t)i * nc + x] = fi[i] - (1.0 / tau_t) * (1.0 - g_taut) * (fi[i] - fe[i]) +
                                       og * omega_s + src;
            for (int a = 0; a < dim; ++a) fpg[a] += omega_s * b->c[i][a];
        }
        /* Eq. 25 with h^2/dt = 1 */
        for (int a = 0; a < 3; ++a) b->fpg[x * 3 + a] = (a < dim) ? og * fpg[a] : 0.0;

        /* node fields (reading R10) */
        b->rho[x] = rho;
        b->tau_t[x] = tau_t;
        double div = 1.0;
        if (b->superficial_mode == 0) div = b->eps_2d[x];
        else if (b->superficial_mode == 1) div = b->eps_g[x];
        double slip2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            b->u[x * 3 + a] = (a < dim) ? u[a] : 0.0;
            b->uact[x * 3 + a] = (a < dim) ? u[a] / div : 0.0;
            double sl = b->uact[x * 3 + a] - vs[a];
            if (a < dim) slip2 += sl * sl;
        }
        b->beta[x] = ob_beta(b->eps_g[x], sqrt(slip2), 1.0, b->k.mu, b->k.d);
    }

    /* Eq. 2 as a push from each cell (reading R9 at the boundary) */
    for (int64_t x = 0; x < b->ncell; ++x) {
        for (int i = 0; i < nq; ++i) {
            double val = fstar[(size_t)i * nc + x];
            int64_t to;
            int wall, open;
            neighbour(b, x, b->c[i], +1, &to, &wall, &open);
            if (wall >= 0) {
                double cu = 0.0;
                for (int a = 0; a < dim; ++a) cu += b->c[i][a] * b->k.wall_u[wall][a];
                b->fnew[(size_t)b->opp[i] * nc + x] = val - 6.0 * b->w[i] * b->rho[x] * cu;
            } else if (open < 0) {
                b->fnew[(size_t)i * nc + to] = val;
            }
            /* a population leaving through an inlet/outlet face is dropped */
        }
        /* populations entering through an inlet or outlet face */
        for (int i = 0; i < nq; ++i) {
            int64_t from;
            int wall, open;
            neighbour(b, x, b->c[i], -1, &from, &wall, &open);
            if (wall < 0 && open >= 0) {
                double uin[3] = {0.0, 0.0, 0.0};
                if (b->bc[open] == OB_INLET) {
                    int vert = dim - 1;
                    int64_t j = (vert == 1) ? (x % b->n[0]) : (x % ((int64_t)b->n[0] * b->n[1]));
                    for (int a = 0; a < dim; ++a) uin[a] = b->inlet_u[j * 3 + a];
                } else {
                    for (int a = 0; a < dim; ++a) uin[a] = b->u[x * 3 + a];
                }
                b->fnew[(size_t)i * nc + x] = feq(b, i, 1.0, uin);
            }
        }
    }
    double *t = b->f;
    b->f = b->fnew;
    b->fnew = t;
    free(fstar);
}

/* ------------------------------------------------------------------------ */
/* Step 4 of Fig. 4: interpolation, Eq. 26-28.                                */
/* ------------------------------------------------------------------------ */
static void pressure_gradient(ob_bed *b)
{
    /* p = c_s^2 rho; central differences, one-sided at non-periodic faces */
    for (int64_t x = 0; x < b->ncell; ++x) {
        int64_t idx[3] = {x % b->n[0], (x / b->n[0]) % b->n[1], x / ((int64_t)b->n[0] * b->n[1])};
        for (int a = 0; a < 3; ++a) {
            double gp = 0.0;
            if (a < b->dim && b->n[a] > 1) {
                int64_t stride = (a == 0) ? 1 : (a == 1) ? b->n[0] : (int64_t)b->n[0] * b->n[1];
                int64_t lo = idx[a] - 1, hi = idx[a] + 1;
                int periodic = (b->bc[2 * a] == OB_PERIODIC);
                double span = 2.0;
                if (lo < 0) { if (periodic) lo += b->n[a]; else { lo = idx[a]; span = 1.0; } }
                if (hi >= b->n[a]) { if (periodic) hi -= b->n[a]; else { hi = idx[a]; span = 1.0; } }
                int64_t xl = x + (lo - idx[a]) * stride, xh = x + (hi - idx[a]) * stride;
                gp = (b->rho[xh] - b->rho[xl]) / 3.0 / span;
            }
            b->gradp[x * 3 + a] = gp;
        }
    }
}

/* Interpolation stencil of a point: 2^dim nodes and weights (reading R11). */
static int stencil(const ob_bed *b, const double *p, int64_t *nodes, double *wts)
{
    int64_t i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0};
    double w1[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < b->dim; ++a) {
        double t = p[a] - 0.5;
        double fl = floor(t);
        w1[a] = t - fl;
        int64_t lo = (int64_t)fl, hi = lo + 1;
        if (b->bc[2 * a] == OB_PERIODIC) {
            lo = (lo % b->n[a] + b->n[a]) % b->n[a];
            hi = (hi % b->n[a] + b->n[a]) % b->n[a];
        } else {
            if (lo < 0) lo = 0;
            if (lo >= b->n[a]) lo = b->n[a] - 1;
            if (hi < 0) hi = 0;
            if (hi >= b->n[a]) hi = b->n[a] - 1;
        }
        i0[a] = lo;
        i1[a] = hi;
    }
    int cnt = 1 << b->dim;
    for (int k = 0; k < cnt; ++k) {
        int64_t idx[3] = {0, 0, 0};
        double wt = 1.0;
        for (int a = 0; a < b->dim; ++a) {
            int bit = (k >> a) & 1;
            idx[a] = bit ? i1[a] : i0[a];
            wt *= bit ? w1[a] : (1.0 - w1[a]);
        }
        nodes[k] = idx[0] + (int64_t)b->n[0] * (idx[1] + (int64_t)b->n[1] * idx[2]);
        wts[k] = wt;
    }
    return cnt;
}

static void drag_and_integrate(ob_bed *b)
{
    const int dim = b->dim;
    const double vp = b->k.vp, mp = b->k.mp;
    for (int64_t p = 0; p < b->np; ++p) {
        int64_t nodes[8];
        double wts[8];
        int cnt = stencil(b, &b->P[p * 3], nodes, wts);
        double uk[3] = {0, 0, 0}, gk[3] = {0, 0, 0}, ek = 0.0, bk = 0.0;
        for (int k = 0; k < cnt; ++k) {
            int64_t x = nodes[k];
            for (int a = 0; a < dim; ++a) {
                uk[a] += wts[k] * b->uact[x * 3 + a];
                gk[a] += wts[k] * b->gradp[x * 3 + a];
            }
            ek += wts[k] * b->eps_g[x];
            bk += wts[k] * b->beta[x];
        }
        /* Eq. 26 */
        for (int a = 0; a < 3; ++a)
            b->fpre[p * 3 + a] = (a < dim) ? vp * bk / (1.0 - ek) * (uk[a] - b->v[p * 3 + a]) : 0.0;
        for (int a = 0; a < 3; ++a) b->fd[p * 3 + a] = gk[a];   /* stash grad p */
    }
    /* Eq. 27 per cell, summed in sorted order; Eq. 28 rescale (reading R12) */
    for (int64_t x = 0; x < b->ncell; ++x) {
        int64_t s = b->cell_start[x], t = b->cell_start[x + 1];
        double S[3] = {0, 0, 0}, A[3] = {0, 0, 0};
        for (int64_t p = s; p < t; ++p)
            for (int a = 0; a < 3; ++a) {
                S[a] += b->fpre[p * 3 + a];
                A[a] += fabs(b->fpre[p * 3 + a]);
            }
        for (int a = 0; a < 3; ++a) {
            b->sum_pre[x * 3 + a] = S[a];
            b->sum_abs_pre[x * 3 + a] = A[a];
        }
        for (int64_t p = s; p < t; ++p) {
            double gk[3] = {b->fd[p * 3 + 0], b->fd[p * 3 + 1], b->fd[p * 3 + 2]};
            for (int a = 0; a < 3; ++a) {
                double scale = 1.0;
                if (!(fabs(S[a]) <= 1e-12 * A[a])) scale = fabs(b->fpg[x * 3 + a]) / fabs(S[a]);
                b->fd[p * 3 + a] = (a < dim) ? scale * b->fpre[p * 3 + a] : 0.0;
            }
            /* Step 5: Eq. 16, symplectic Euler (reading R13) */
            double sgn = b->pressure_plus ? 1.0 : -1.0;
            for (int a = 0; a < dim; ++a) {
                double fa = b->fd[p * 3 + a] + sgn * vp * gk[a];
                if (b->model == 1) fa += b->fc[p * 3 + a];   /* soft-sphere contacts (R25) */
                double acc = b->k.g_eff[a] + fa / mp;
                b->v[p * 3 + a] += acc;
                b->P[p * 3 + a] += b->v[p * 3 + a];
            }
            /* specular walls and periodic wrap */
            for (int a = 0; a < dim; ++a) {
                double L = (double)b->n[a];
                double *pa = &b->P[p * 3 + a];
                if (b->bc[2 * a] == OB_PERIODIC) {
                    if (*pa >= L) *pa -= L;
                    else if (*pa < 0.0) {
                        *pa += L;
                        if (*pa >= L) *pa = 0.0;
                    }
                } else if (b->recirculate && a == dim - 1 && *pa >= L) {
                    /* reading R21: through the outlet, back in at the inlet */
                    *pa -= L;
                    b->solids_out += 1;
                } else {
                    if (*pa < 0.0) {
                        *pa = -*pa;
                        b->v[p * 3 + a] = -b->k.e * b->v[p * 3 + a];
                    } else if (*pa >= L) {
                        *pa = 2.0 * L - *pa;
                        b->v[p * 3 + a] = -b->k.e * b->v[p * 3 + a];
                    }
                    if (*pa < 0.0) *pa = 0.0;
                    if (*pa >= L) *pa = nextafter(L, 0.0);
                }
            }
        }
    }
    for (int64_t p = 0; p < b->np; ++p)
        for (int a = 0; a < 3; ++a) {
            b->diag_fpre[b->id[p] * 3 + a] = b->fpre[p * 3 + a];
            b->diag_fd[b->id[p] * 3 + a] = b->fd[p * 3 + a];
        }
}

/* ------------------------------------------------------------------------ */
/* Step 6 of Fig. 4: TDHS detection and resolution (§2.2, Eq. 17-18).         */
/* ------------------------------------------------------------------------ */
/* minimum-image separation P_i - P_j along axis a */
static double sep_axis(const ob_bed *b, int a, double pi, double pj)
{
    double d = pi - pj;
    if (b->bc[2 * a] == OB_PERIODIC) {
        double L = (double)b->n[a];
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

static void push_pair(ob_bed *b, int64_t i, int64_t j)
{
    if (b->npairs == b->pairs_cap) {
        int64_t cap = b->pairs_cap ? 2 * b->pairs_cap : 1024;
        b->pairs = realloc(b->pairs, sizeof(int64_t) * 2 * (size_t)cap);
        b->pairs_cap = cap;
    }
    b->pairs[2 * b->npairs] = i;
    b->pairs[2 * b->npairs + 1] = j;
    b->npairs++;
}

static int cmp_pair(const void *x, const void *y)
{
    const int64_t *a = x, *b = y;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}

static void detect_and_resolve(ob_bed *b)
{
    const int dim = b->dim;
    const double dd = b->k.d * b->k.d, r = b->k.r;
    int64_t np = b->np;
    double *bestd2 = malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    int64_t *bestp = malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1));  /* sorted index */
    int64_t *pos_of = malloc(sizeof(int64_t) * (size_t)(np > 0 ? np : 1)); /* id -> index */
    for (int64_t p = 0; p < np; ++p) {
        bestd2[p] = INFINITY;
        bestp[p] = -1;
        b->best[p] = -1;
        b->wall_hit[p] = 0;
        pos_of[b->id[p]] = p;
    }
    b->npairs = 0;
    /* every pair in contact, for the sequential rule (R27) */
    int64_t ncont = 0, capc = 0, *cont = NULL;

    for (int64_t p = 0; p < np; ++p) {
        int64_t x = b->cell[p];
        int64_t idx[3] = {x % b->n[0], (x / b->n[0]) % b->n[1], x / ((int64_t)b->n[0] * b->n[1])};
        int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) { lo[a] = -1; hi[a] = 1; }
        for (int64_t oz = lo[2]; oz <= hi[2]; ++oz)
        for (int64_t oy = lo[1]; oy <= hi[1]; ++oy)
        for (int64_t ox = lo[0]; ox <= hi[0]; ++ox) {
            int64_t q[3] = {idx[0] + ox, idx[1] + oy, idx[2] + oz};
            int skip = 0;
            for (int a = 0; a < dim; ++a) {
                if (q[a] < 0 || q[a] >= b->n[a]) {
                    if (b->bc[2 * a] == OB_PERIODIC) q[a] = (q[a] + b->n[a]) % b->n[a];
                    else skip = 1;
                }
            }
            if (skip) continue;
            int64_t y = q[0] + (int64_t)b->n[0] * (q[1] + (int64_t)b->n[1] * q[2]);
            for (int64_t j = b->cell_start[y]; j < b->cell_start[y + 1]; ++j) {
                if (j == p) continue;
                /* contact: |P_i - P_j|^2 < d^2, summed axis by axis */
                double dx[3] = {0, 0, 0}, d2 = 0.0;
                for (int a = 0; a < dim; ++a) {
                    dx[a] = sep_axis(b, a, b->P[p * 3 + a], b->P[j * 3 + a]);
                    d2 = d2 + dx[a] * dx[a];
                }
                if (!(d2 < dd)) continue;
                if (b->rule == 1 && b->id[p] < b->id[j]) {
                    if (ncont == capc) {
                        capc = capc ? 2 * capc : 64;
                        cont = realloc(cont, sizeof(int64_t) * 2 * (size_t)capc);
                    }
                    cont[2 * ncont] = b->id[p];
                    cont[2 * ncont + 1] = b->id[j];
                    ++ncont;
                }
                /* approach: (P_i - P_j) . (v_i - v_j) < 0 */
                double dot = 0.0;
                for (int a = 0; a < dim; ++a)
                    dot = dot + dx[a] * (b->v[p * 3 + a] - b->v[j * 3 + a]);
                if (!(dot < 0.0)) continue;
                if (b->id[p] < b->id[j]) push_pair(b, b->id[p], b->id[j]);
                /* partner choice (reading R14) */
                if (d2 < bestd2[p] || (d2 == bestd2[p] && b->id[j] < b->id[bestp[p]])) {
                    bestd2[p] = d2;
                    bestp[p] = j;
                }
            }
        }
        /* wall contacts: distance to the face below r and moving toward it */
        for (int a = 0; a < dim; ++a) {
            if (b->bc[2 * a] == OB_PERIODIC) continue;
            double pa = b->P[p * 3 + a], va = b->v[p * 3 + a];
            if (pa < r && va < 0.0) b->wall_hit[p] |= 1 << (2 * a);
            /* with the solids loop closed the outlet lets particles through (R21) */
            const int open_top = b->recirculate && a == dim - 1;
            if (!open_top && (double)b->n[a] - pa < r && va > 0.0) b->wall_hit[p] |= 1 << (2 * a + 1);
        }
    }
    qsort(b->pairs, (size_t)b->npairs, 2 * sizeof(int64_t), cmp_pair);

    for (int64_t p = 0; p < np; ++p) b->best[p] = (bestp[p] >= 0) ? b->id[bestp[p]] : -1;

    if (b->rule == 1) {
        /* R27: every pair in contact in canonical order (id_i, id_j),
         * resolved by Eq. 17-18 from the velocities left by the earlier ones
         * if it approaches then; then every wall contact whose particle
         * moves toward the face */
        if (ncont > 0) qsort(cont, (size_t)ncont, 2 * sizeof(int64_t), cmp_pair);
        for (int64_t k = 0; k < ncont; ++k) {
            int64_t p = pos_of[cont[2 * k]], j = pos_of[cont[2 * k + 1]];
            double pi[3] = {0, 0, 0}, pj[3] = {0, 0, 0}, vi[3] = {0, 0, 0}, vj[3] = {0, 0, 0};
            double dot = 0.0;
            for (int a = 0; a < dim; ++a) {
                pi[a] = sep_axis(b, a, b->P[p * 3 + a], b->P[j * 3 + a]);
                vi[a] = b->v[p * 3 + a];
                vj[a] = b->v[j * 3 + a];
                dot = dot + pi[a] * (vi[a] - vj[a]);
            }
            if (!(dot < 0.0)) continue;
            ob_binary_collision(dim, b->k.mp, b->k.mp, b->k.e, pi, pj, vi, vj);
            for (int a = 0; a < dim; ++a) {
                b->v[p * 3 + a] = vi[a];
                b->v[j * 3 + a] = vj[a];
            }
        }
        for (int64_t p = 0; p < np; ++p)
            for (int a = 0; a < dim; ++a) {
                double *va = &b->v[p * 3 + a];
                if (((b->wall_hit[p] >> (2 * a)) & 1) && *va < 0.0) *va = -b->k.e * *va;
                if (((b->wall_hit[p] >> (2 * a + 1)) & 1) && *va > 0.0) *va = -b->k.e * *va;
            }
        free(cont);
        free(bestd2);
        free(bestp);
        free(pos_of);
        return;
    }

    /* Eq. 17-18 on mutual choices, from the pre-collision velocities */
    double *vnew = malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    memcpy(vnew, b->v, sizeof(double) * 3 * (size_t)np);
    int *paired = calloc((size_t)(np > 0 ? np : 1), sizeof(int));
    for (int64_t p = 0; p < np; ++p) {
        int64_t j = bestp[p];
        if (j < 0 || bestp[j] != p) continue;
        paired[p] = 1;
        if (b->id[p] > b->id[j]) continue;           /* handle each pair once */
        double pi[3] = {0, 0, 0}, pj[3] = {0, 0, 0}, vi[3] = {0, 0, 0}, vj[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
            pi[a] = sep_axis(b, a, b->P[p * 3 + a], b->P[j * 3 + a]);  /* P_j at origin */
            vi[a] = b->v[p * 3 + a];
            vj[a] = b->v[j * 3 + a];
        }
        ob_binary_collision(dim, b->k.mp, b->k.mp, b->k.e, pi, pj, vi, vj);
        for (int a = 0; a < dim; ++a) {
            vnew[p * 3 + a] = vi[a];
            vnew[j * 3 + a] = vj[a];
        }
    }
    /* wall collisions for particles not in a pair: v_n -> -e v_n */
    for (int64_t p = 0; p < np; ++p) {
        if (paired[p] || !b->wall_hit[p]) continue;
        for (int a = 0; a < dim; ++a)
            if (b->wall_hit[p] & (3 << (2 * a))) vnew[p * 3 + a] = -b->k.e * vnew[p * 3 + a];
    }
    memcpy(b->v, vnew, sizeof(double) * 3 * (size_t)np);
    free(vnew);
    free(paired);
    free(cont);
    free(bestd2);
    free(bestp);
    free(pos_of);
}

/* ------------------------------------------------------------------------ */
/* One coupled step (Fig. 4, steps 2-6).                                       */
/* ------------------------------------------------------------------------ */
/* ------------------------------------------------------------------------ */
/* Soft-sphere contacts (reading R25, the paper's §2.2 outlook on DEM for     */
/* dense beds): every overlapping pair and every wall overlap pushes with a  */
/* linear spring-dashpot normal force F = k_n delta - eta (v_rel . n),       */
/* never pulling.  With friction (R26) the contact point's tangential slip   */
/* meets a viscous force -gamma_t v_t capped at mu F (Coulomb), which also   */
/* turns the particles.  Forces and torques from the positions and           */
/* velocities at the start of the step, sorted order.                        */
/* ------------------------------------------------------------------------ */
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* One contact seen from particle p: unit normal nrm pointing towards p, lever
 * arm l from p's centre to the contact point (at -l nrm), normal force fn
 * (already clipped at zero), relative velocity of the contact point vc
 * (p's minus the other body's).  Adds the force on p to F and its torque to T. */
static void contact_add(const ob_bed *b, const double *nrm, double l, double fn, const double *vc,
                        double *F, double *T)
{
    for (int a = 0; a < 3; ++a) F[a] += fn * nrm[a];
    if (!(b->k.mu_f > 0.0 && b->k.gamma_t > 0.0 && fn > 0.0)) return;
    double vcn = vc[0] * nrm[0] + vc[1] * nrm[1] + vc[2] * nrm[2];
    double vt[3], s2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        vt[a] = vc[a] - vcn * nrm[a];
        s2 += vt[a] * vt[a];
    }
    double st = sqrt(s2);
    if (!(st > 0.0)) return;
    double mag = b->k.gamma_t * st, cap = b->k.mu_f * fn;
    if (mag > cap) mag = cap;
    double Ft[3], arm[3], t[3];
    for (int a = 0; a < 3; ++a) {
        Ft[a] = -mag * vt[a] / st;
        F[a] += Ft[a];
        arm[a] = -l * nrm[a];
    }
    cross3(arm, Ft, t);
    for (int a = 0; a < 3; ++a) T[a] += t[a];
}

static void contact_forces(ob_bed *b)
{
    const int dim = b->dim;
    const double d = b->k.d, r = b->k.r, kn = b->k.kn;
    for (int64_t p = 0; p < b->np; ++p) {
        double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
        const double *vp = &b->v[p * 3], *wp = &b->spin[p * 3];
        int64_t x = b->cell[p];
        int64_t idx[3] = {x % b->n[0], (x / b->n[0]) % b->n[1], x / ((int64_t)b->n[0] * b->n[1])};
        int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) { lo[a] = -1; hi[a] = 1; }
        for (int64_t oz = lo[2]; oz <= hi[2]; ++oz)
        for (int64_t oy = lo[1]; oy <= hi[1]; ++oy)
        for (int64_t ox = lo[0]; ox <= hi[0]; ++ox) {
            int64_t q[3] = {idx[0] + ox, idx[1] + oy, idx[2] + oz};
            int skip = 0;
            for (int a = 0; a < dim; ++a)
                if (q[a] < 0 || q[a] >= b->n[a]) {
                    if (b->bc[2 * a] == OB_PERIODIC) q[a] = (q[a] + b->n[a]) % b->n[a];
                    else skip = 1;
                }
            if (skip) continue;
            int64_t y = q[0] + (int64_t)b->n[0] * (q[1] + (int64_t)b->n[1] * q[2]);
            for (int64_t j = b->cell_start[y]; j < b->cell_start[y + 1]; ++j) {
                if (j == p) continue;
                double dx[3] = {0, 0, 0}, d2 = 0.0;
                for (int a = 0; a < dim; ++a) {
                    dx[a] = sep_axis(b, a, b->P[p * 3 + a], b->P[j * 3 + a]);
                    d2 += dx[a] * dx[a];
                }
                if (!(d2 < d * d)) continue;
                double dist = sqrt(d2), nrm[3], vn = 0.0;
                for (int a = 0; a < 3; ++a) nrm[a] = dx[a] / dist;
                for (int a = 0; a < dim; ++a) vn += (vp[a] - b->v[j * 3 + a]) * nrm[a];
                double f = kn * (d - dist) - b->k.eta * vn;
                if (f < 0.0) f = 0.0;
                /* contact point half way between the centres: relative
                 * velocity (v_p - v_j) - l (w_p + w_j) x n with l = dist / 2 */
                double l = 0.5 * dist, ws[3], wxn[3], vc[3];
                for (int a = 0; a < 3; ++a) ws[a] = wp[a] + b->spin[j * 3 + a];
                cross3(ws, nrm, wxn);
                for (int a = 0; a < 3; ++a)
                    vc[a] = (a < dim ? vp[a] - b->v[j * 3 + a] : 0.0) - l * wxn[a];
                contact_add(b, nrm, l, f, vc, F, T);
            }
        }
        /* walls (an open outlet of a circulating bed is not one, R21): the
         * contact point lies on the face, at the centre's distance from it */
        for (int a = 0; a < dim; ++a) {
            if (b->bc[2 * a] == OB_PERIODIC) continue;
            double pa = b->P[p * 3 + a], va = vp[a];
            for (int side = 0; side < 2; ++side) {
                if (side == 1 && b->recirculate && a == dim - 1) continue;
                double l = side == 0 ? pa : (double)b->n[a] - pa;
                if (!(l < r)) continue;
                double nrm[3] = {0, 0, 0};
                nrm[a] = side == 0 ? 1.0 : -1.0;
                double f = kn * (r - l) - b->k.eta_w * (va * nrm[a]);
                if (f < 0.0) f = 0.0;
                double wxn[3], vc[3];
                cross3(wp, nrm, wxn);
                for (int c = 0; c < 3; ++c) vc[c] = (c < dim ? vp[c] : 0.0) - l * wxn[c];
                contact_add(b, nrm, l, f, vc, F, T);
            }
        }
        for (int a = 0; a < 3; ++a) {
            b->fc[p * 3 + a] = a < dim ? F[a] : 0.0;
            b->tq[p * 3 + a] = T[a];
            b->diag_fc[b->id[p] * 3 + a] = b->fc[p * 3 + a];
        }
    }
    /* spin: I dw = T dt, after every torque has been taken from the
     * start-of-step state (in 2D only the z component is non-zero) */
    for (int64_t p = 0; p < b->np; ++p)
        for (int a = 0; a < 3; ++a) b->spin[p * 3 + a] += b->tq[p * 3 + a] / b->k.inertia;
}

void ob_step(ob_bed *b)
{
    deposit(b);
    collide_and_stream(b);
    pressure_gradient(b);
    if (b->model == 1) contact_forces(b);
    drag_and_integrate(b);
    sort_particles(b);
    if (b->model == 0) detect_and_resolve(b);
    b->steps++;
}

/* The particle half of step 6 alone (sort, detection, Eq. 17-18) on the
 * current state, for tests of the hard-sphere model in isolation. */
void ob_collide_particles(ob_bed *b)
{
    sort_particles(b);
    detect_and_resolve(b);
}

void ob_run(ob_bed *b, int64_t nsteps)
{
    for (int64_t s = 0; s < nsteps; ++s) ob_step(b);
}

/* ------------------------------------------------------------------------ */
/* State access.                                                              */
/* ------------------------------------------------------------------------ */
int ob_dim(const ob_bed *b) { return b->dim; }
int ob_nq(const ob_bed *b) { return b->nq; }
int64_t ob_ncell(const ob_bed *b) { return b->ncell; }
int64_t ob_np(const ob_bed *b) { return b->np; }
int64_t ob_npairs(const ob_bed *b) { return b->npairs; }

void ob_constants(const ob_bed *b, double *out)
{
    /* tau nu mu rho_s d r vp mp e g_eff[3] fb[3] u0[3] cs kn eta eta_w mu_f
     * gamma_t inertia */
    const ob_consts *k = &b->k;
    double v[] = {k->tau, k->nu, k->mu, k->rho_s, k->d, k->r, k->vp, k->mp, k->e,
                  k->g_eff[0], k->g_eff[1], k->g_eff[2], k->fb[0], k->fb[1], k->fb[2],
                  k->u0[0], k->u0[1], k->u0[2], k->cs_smag, k->kn, k->eta, k->eta_w, k->mu_f,
                  k->gamma_t, k->inertia};
    memcpy(out, v, sizeof(v));
}

void ob_units_flat(const ob_setup *s, double *out)
{
    ob_consts k;
    ob_units(s, &k);
    double v[] = {k.tau, k.nu, k.mu, k.rho_s, k.d, k.r, k.vp, k.mp, k.e,
                  k.g_eff[0], k.g_eff[1], k.g_eff[2], k.fb[0], k.fb[1], k.fb[2],
                  k.u0[0], k.u0[1], k.u0[2], k.cs_smag, k.kn, k.eta, k.eta_w, k.mu_f,
                  k.gamma_t, k.inertia};
    memcpy(out, v, sizeof(v));
}

/* populations in [q][cell] layout */
void ob_get_populations(const ob_bed *b, double *out)
{
    memcpy(out, b->f, sizeof(double) * (size_t)b->nq * (size_t)b->ncell);
}

void ob_set_populations(ob_bed *b, const double *in)
{
    memcpy(b->f, in, sizeof(double) * (size_t)b->nq * (size_t)b->ncell);
}

/* particles in id order, lattice units, np * dim */
void ob_get_particles(const ob_bed *b, double *P, double *v)
{
    for (int64_t p = 0; p < b->np; ++p) {
        int64_t id = b->id[p];
        for (int a = 0; a < b->dim; ++a) {
            P[id * b->dim + a] = b->P[p * 3 + a];
            v[id * b->dim + a] = b->v[p * 3 + a];
        }
    }
}

int ob_set_particles(ob_bed *b, int64_t np, const double *P, const double *v)
{
    if (!alloc_particles(b, np)) return -1;
    for (int64_t p = 0; p < np; ++p) {
        b->id[p] = p;
        for (int a = 0; a < b->dim; ++a) {
            b->P[p * 3 + a] = P[p * b->dim + a];
            b->v[p * 3 + a] = v[p * b->dim + a];
        }
    }
    sort_particles(b);
    return 0;
}

/* angular velocities (R26) in id order: the z component per particle in 2D,
 * three components in 3D */
void ob_get_spin(const ob_bed *b, double *out)
{
    const int nc = b->dim == 2 ? 1 : 3;
    for (int64_t p = 0; p < b->np; ++p)
        for (int c = 0; c < nc; ++c) out[b->id[p] * nc + c] = b->spin[p * 3 + (b->dim == 2 ? 2 : c)];
}

void ob_set_spin(ob_bed *b, const double *in)
{
    const int nc = b->dim == 2 ? 1 : 3;
    for (int64_t p = 0; p < b->np; ++p)
        for (int c = 0; c < nc; ++c) b->spin[p * 3 + (b->dim == 2 ? 2 : c)] = in[b->id[p] * nc + c];
}

/* sorted order: ids and cell_start */
void ob_get_sorted(const ob_bed *b, int64_t *ids, int64_t *cell_start)
{
    if (ids) memcpy(ids, b->id, sizeof(int64_t) * (size_t)b->np);
    if (cell_start) memcpy(cell_start, b->cell_start, sizeof(int64_t) * (size_t)(b->ncell + 1));
}

enum {
    OB_F_RHO = 0, OB_F_U = 1, OB_F_UACT = 2, OB_F_VS = 3, OB_F_EPS_S = 4, OB_F_EPS_G = 5,
    OB_F_OMEGA = 6, OB_F_BETA = 7, OB_F_FPG = 8, OB_F_GRADP = 9, OB_F_TAU_T = 10,
    OB_F_NTOT = 11, OB_F_SUM_PRE = 12, OB_F_SUM_ABS_PRE = 13, OB_F_EPS_2D = 14
};

/* a node field: scalar fields give ncell values, vector fields ncell * dim */
int ob_get_field(const ob_bed *b, int which, double *out)
{
    const double *src = NULL;
    int vec = 0;
    switch (which) {
    case OB_F_RHO: src = b->rho; break;
    case OB_F_U: src = b->u; vec = 1; break;
    case OB_F_UACT: src = b->uact; vec = 1; break;
    case OB_F_VS: src = b->vs; vec = 1; break;
    case OB_F_EPS_S: src = b->eps_s; break;
    case OB_F_EPS_G: src = b->eps_g; break;
    case OB_F_OMEGA: src = b->omega; break;
    case OB_F_BETA: src = b->beta; break;
    case OB_F_FPG: src = b->fpg; vec = 1; break;
    case OB_F_GRADP: src = b->gradp; vec = 1; break;
    case OB_F_TAU_T: src = b->tau_t; break;
    case OB_F_SUM_PRE: src = b->sum_pre; vec = 1; break;
    case OB_F_SUM_ABS_PRE: src = b->sum_abs_pre; vec = 1; break;
    case OB_F_EPS_2D: src = b->eps_2d; break;
    case OB_F_NTOT:
        for (int64_t x = 0; x < b->ncell; ++x) out[x] = (double)b->ntot[x];
        return 0;
    default: return -1;
    }
    for (int64_t x = 0; x < b->ncell; ++x) {
        if (vec) for (int a = 0; a < b->dim; ++a) out[x * b->dim + a] = src[x * 3 + a];
        else out[x] = src[x];
    }
    return 0;
}

enum { OB_P_FPRE = 0, OB_P_FD = 1, OB_P_CELL = 2, OB_P_BEST = 3, OB_P_WALL = 4, OB_P_FC = 5 };

/* per-particle diagnostics of the last step, id order */
int ob_get_particle_diag(const ob_bed *b, int which, double *out)
{
    for (int64_t p = 0; p < b->np; ++p) {
        int64_t id = b->id[p];
        switch (which) {
        case OB_P_FPRE:
            for (int a = 0; a < b->dim; ++a) out[id * b->dim + a] = b->diag_fpre[id * 3 + a];
            break;
        case OB_P_FD:
            for (int a = 0; a < b->dim; ++a) out[id * b->dim + a] = b->diag_fd[id * 3 + a];
            break;
        case OB_P_CELL: out[id] = (double)b->cell[p]; break;
        case OB_P_BEST: out[id] = (double)b->best[p]; break;
        case OB_P_WALL: out[id] = (double)b->wall_hit[p]; break;
        case OB_P_FC:
            for (int a = 0; a < b->dim; ++a) out[id * b->dim + a] = b->diag_fc[id * 3 + a];
            break;
        default: return -1;
        }
    }
    return 0;
}

/* approaching contact pairs (id_i < id_j) of the last detection, sorted */
int64_t ob_get_pairs(const ob_bed *b, int64_t *out, int64_t cap)
{
    int64_t n = b->npairs < cap ? b->npairs : cap;
    memcpy(out, b->pairs, sizeof(int64_t) * 2 * (size_t)n);
    return b->npairs;
}

/*
 * Diagnostics: [0] gas mass, [1..3] gas momentum sum_i c_i f_i (state),
 * [4..6] particle momentum m_p v, [7] mean eps_g over cells, [8] particle-
 * weighted mean |u_act - v_s| over occupied cells.  Sums are compensated
 * (Neumaier) so that conservation can be checked near round-off.
 */
static void nsum(double *s, double *c, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
    else *c += (x - t) + *s;
    *s = t;
}

int64_t ob_solids_out(const ob_bed *b) { return b->solids_out; }

/* Replace the inlet velocities (SI, inlet-face cells x dim), e.g. at the end
 * of the jet pulse of §3.1. */
void ob_set_inlet(ob_bed *b, const double *inlet_si)
{
    int64_t nface = b->ncell / b->n[b->dim - 1];
    for (int64_t j = 0; j < nface; ++j)
        for (int a = 0; a < b->dim; ++a) b->inlet_u[j * 3 + a] = inlet_si[j * b->dim + a] * b->uscale;
}

/* Bubbles (§3.1): regions of cells whose voidage (eps_2d of Eq. 10 for
 * voidage = 0, eps_g of Eq. 11 for 1, from the current particle counts)
 * exceeds the threshold, neighbours along the axes
 * (periodic faces wrap), without the regions that reach the top row of the
 * vertical axis.  Breadth-first flood fill.  out: [0] cells of the largest
 * region, [1] regions, [2] cells in all regions. */
void ob_bubbles(const ob_bed *b, double threshold, int voidage, int64_t *out)
{
    int64_t nc = b->ncell;
    char *in = calloc((size_t)nc, 1);
    char *seen = calloc((size_t)nc, 1);
    int64_t *queue = malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    for (int64_t x = 0; x < nc; ++x) {
        double es, e2;
        double eg = voidage_of_count(b, b->cell_start[x + 1] - b->cell_start[x], &es, &e2);
        in[x] = (voidage == 0 ? e2 : eg) > threshold;
    }
    int64_t stride[3] = {1, b->n[0], (int64_t)b->n[0] * b->n[1]};
    int vert = b->dim - 1;
    out[0] = out[1] = out[2] = 0;
    for (int64_t s0 = 0; s0 < nc; ++s0) {
        if (!in[s0] || seen[s0]) continue;
        int64_t head = 0, tail = 0, size = 0;
        int top = 0;
        queue[tail++] = s0;
        seen[s0] = 1;
        while (head < tail) {
            int64_t x = queue[head++];
            ++size;
            int64_t q[3] = {x % b->n[0], (x / b->n[0]) % b->n[1], x / stride[2]};
            if (q[vert] == b->n[vert] - 1) top = 1;
            for (int a = 0; a < b->dim; ++a)
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    int64_t qa = q[a] + sgn;
                    if (qa < 0 || qa >= b->n[a]) {
                        if (b->bc[2 * a] != OB_PERIODIC) continue;
                        qa = (qa + b->n[a]) % b->n[a];
                    }
                    int64_t y = x + (qa - q[a]) * stride[a];
                    if (in[y] && !seen[y]) {
                        seen[y] = 1;
                        queue[tail++] = y;
                    }
                }
        }
        if (top) continue;
        if (size > out[0]) out[0] = size;
        out[1] += 1;
        out[2] += size;
    }
    free(in);
    free(seen);
    free(queue);
}

void ob_stats(const ob_bed *b, double *out)
{
    double s[7] = {0}, c[7] = {0};
    size_t nc = (size_t)b->ncell;
    for (int64_t x = 0; x < b->ncell; ++x)
        for (int i = 0; i < b->nq; ++i) {
            double fi = b->f[(size_t)i * nc + x];
            nsum(&s[0], &c[0], fi);
            for (int a = 0; a < b->dim; ++a) nsum(&s[1 + a], &c[1 + a], b->c[i][a] * fi);
        }
    for (int64_t p = 0; p < b->np; ++p)
        for (int a = 0; a < b->dim; ++a) nsum(&s[4 + a], &c[4 + a], b->k.mp * b->v[p * 3 + a]);
    for (int k = 0; k < 7; ++k) out[k] = s[k] + c[k];
    double se = 0.0, ss = 0.0, nw = 0.0;
    for (int64_t x = 0; x < b->ncell; ++x) {
        /* voidage of the current positions (the particles were re-sorted
         * after the move, so cell_start is up to date) */
        double es, e2;
        se += voidage_of_count(b, b->cell_start[x + 1] - b->cell_start[x], &es, &e2);
        if (b->ntot[x] > 0) {
            double sl = 0.0;
            for (int a = 0; a < b->dim; ++a) {
                double d = b->uact[x * 3 + a] - b->vs[x * 3 + a];
                sl += d * d;
            }
            ss += (double)b->ntot[x] * sqrt(sl);
            nw += (double)b->ntot[x];
        }
    }
    out[7] = se / (double)b->ncell;
    out[8] = nw > 0 ? ss / nw : 0.0;
}

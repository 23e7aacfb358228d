/*
 * lbdps.h — C ABI of the GB300 (sm_103a) library for the coupled time step of
 * the lattice-Boltzmann based discrete particle simulation of Wang, Zhang,
 * Wang, Ge and Li, "Lattice Boltzmann based discrete simulation for gas-solid
 * fluidization" (arXiv 1303.2653).
 *
 * One step (the paper's Fig. 4, steps 2-6) advances:
 *   - deposition of solid velocity and voidage on the lattice (Eq. 8, 10, 11),
 *   - the modified LBE collide-and-stream with partially saturated cells,
 *     EMMS correction and optional Smagorinsky LES (Eq. 2-7, 9, 12-15, 20,
 *     23-25),
 *   - the interpolated EMMS/Ergun drag rescaled by Newton's third law and the
 *     particle integration (Eq. 16, 19-22, 26-28),
 *   - the time-driven hard-sphere step: cell binning, contact detection and
 *     binary collisions (section 2.2, Eq. 17-18).
 *
 * Conventions
 *   - Every function returning int returns LBDPS_OK (0) or a negative
 *     LBDPS_ERR_* code; nothing else crosses the ABI.  lbdps_last_error()
 *     returns a message for the most recent failure on the calling thread.
 *   - All pointer arguments are plain host pointers unless stated otherwise.
 *     Inputs are copied; the caller keeps ownership of its arrays.
 *   - Device memory is owned by the handle.  It is obtained from params.alloc
 *     (for example a framework's caching allocator) or, when that is NULL,
 *     from cudaMalloc, and released at lbdps_destroy.  Every block params.alloc
 *     returns must be 256-byte aligned (the kernels use 16-byte vector
 *     accesses); a misaligned block makes lbdps_create fail with
 *     LBDPS_ERR_INVALID before any kernel runs.
 *   - Work is issued on params.stream (a cudaStream_t, NULL = a stream the
 *     handle creates).  lbdps_step is asynchronous; functions that return
 *     host data synchronise that stream first.
 *   - A handle is not thread safe: use one handle per thread.
 *   - Lattice units: cell size h = 1, time step dt = 1, reference gas
 *     density 1.  SI inputs are converted at create (the paper's Tables 1-2
 *     list both forms).
 *   - Axes: x, y (and z in 3D); the last axis is vertical.  Cells are stored
 *     x-fastest; a cell index is x + nx*(y + ny*z).
 */
#ifndef LBDPS_H
#define LBDPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define LBDPS_OK            0
#define LBDPS_ERR_INVALID  (-1)  /* bad argument or description           */
#define LBDPS_ERR_OOM      (-2)  /* allocation failed                      */
#define LBDPS_ERR_CAPACITY (-3)  /* a caller buffer or table is too small  */
#define LBDPS_ERR_DIVERGED (-4)  /* NaN/Inf, rho <= 0 or |u| > 0.3 seen    */
#define LBDPS_ERR_DOMAIN   (-5)  /* a particle left the domain             */
#define LBDPS_ERR_TIMEOUT  (-6)  /* a bounded device wait gave up          */
#define LBDPS_ERR_CUDA     (-7)  /* a CUDA runtime call failed             */

/* ---- face types (lbdps_lattice_desc.bc) ------------------------------ */
#define LBDPS_WALL      0  /* half-way bounce-back for the gas, specular wall for particles */
#define LBDPS_PERIODIC  1
#define LBDPS_INLET     2  /* velocity inlet, vertical axis only; particles reflect          */
#define LBDPS_OUTLET    3  /* pressure outlet (rho = 1), vertical axis only; particles reflect */

/* ---- population storage (lbdps_params.storage) ---------------------- */
#define LBDPS_STORE_F64   0  /* FP64 deviations f_i - w_i, FP64 arithmetic          */
#define LBDPS_STORE_F32   1  /* FP32 deviations f_i - w_i, FP32 arithmetic          */
#define LBDPS_STORE_F16   2  /* FP16 of (f_i - w_i) * 2^10, FP32 arithmetic         */
#define LBDPS_STORE_BF16  3  /* BF16 of (f_i - w_i), FP32 arithmetic                */

/* ---- units of exported data ----------------------------------------- */
#define LBDPS_UNITS_LATTICE 0
#define LBDPS_UNITS_SI      1

/* ---- node fields of the last step (lbdps_fields mask bits) ---------- */
/* always available */
#define LBDPS_FIELD_RHO    (1 << 0)  /* gas density, Eq. 5                          (1)   */
#define LBDPS_FIELD_FPG    (1 << 2)  /* force on the gas from particles, Eq. 25     (dim) */
#define LBDPS_FIELD_BETA   (1 << 3)  /* inter-phase coefficient, Eq. 19             (1)   */
#define LBDPS_FIELD_UACT   (1 << 7)  /* interstitial gas velocity u / eps, the velocity
                                        the drag interpolates (Eq. 26)              (dim) */
/* the following need params.diagnostics = 1 */
#define LBDPS_FIELD_U      (1 << 1)  /* superficial gas velocity, Eq. 24            (dim) */
#define LBDPS_FIELD_VS     (1 << 4)  /* mean solid velocity, Eq. 8                  (dim) */
#define LBDPS_FIELD_NTOT   (1 << 5)  /* particles per cell, Fig. 1                  (1)   */
#define LBDPS_FIELD_TAU_T  (1 << 6)  /* LES relaxation time, Eq. 15                 (1)   */
#define LBDPS_FIELD_EPS_G  (1 << 8)  /* gas voidage used by the drag, Eq. 11        (1)   */

/* ---- per-particle diagnostics (lbdps_particle_diag) ----------------- */
#define LBDPS_PDIAG_FPRE   0  /* pre-estimated drag, Eq. 26 (dim, needs diagnostics) */
#define LBDPS_PDIAG_FD     1  /* rescaled drag, Eq. 28 (dim, needs diagnostics)      */
#define LBDPS_PDIAG_BEST   2  /* chosen collision partner id, or -1 (1)             */
#define LBDPS_PDIAG_WALL   3  /* wall contacts: bit 2a low face, 2a+1 high face (1) */
#define LBDPS_PDIAG_CELL   4  /* cell index of the particle (1)                     */
#define LBDPS_PDIAG_ORDER  5  /* ids in cell-sorted order: entry k is the id held
                                 in sorted slot k (1)                               */
#define LBDPS_PDIAG_FC     6  /* soft-sphere contact force of the last step (dim,
                                 LBDPS_COLLIDE_SOFT, needs diagnostics)               */

typedef struct lbdps lbdps_t;

/* Lattice and boundaries: the paper's step 1 "size and geometry of the
 * simulation domain ... boundary conditions" (Fig. 4). */
typedef struct {
    int dim;              /* 2 (D2Q9) or 3 (D3Q19)                                 */
    int n[3];             /* cells per axis; n[2] ignored in 2D                     */
    int bc[6];            /* face types x-, x+, y-, y+, z-, z+ (LBDPS_WALL ...)     */
    double h;             /* cell size, m                                          */
    double dt;            /* time step, s                                          */
    const double *inlet_u;   /* inlet-face velocities, m/s, (cells of the inlet face) x dim,
                                face cells x-fastest; NULL = zero; copied          */
    double wall_u[6][3];  /* wall velocity per face, m/s (moving-wall bounce-back) */
} lbdps_lattice_desc;

/* Particles: "mass, radius, position and velocity" of section 2.2; one
 * diameter and density for all (monodisperse).  Particle k has id k. */
typedef struct {
    int64_t n;            /* number of particles                                  */
    double d_p;           /* diameter, m (must not exceed h)                      */
    double rho_s;         /* solid density, kg/m^3                                */
    double e;             /* restitution coefficient, Eq. 17-18                   */
    const double *pos;    /* n x dim centres, m, inside the domain, non-overlapping; copied */
    const double *vel;    /* n x dim velocities, m/s; copied                      */
    int recirculate;      /* 1: a particle leaving through the outlet face of the vertical
                             axis re-enters through the inlet face at the same lateral
                             position and velocity (the solids loop of a circulating
                             bed, §3.2 / Fig. 9); needs the inlet below and the outlet
                             above.  0: particles reflect at every non-periodic face */
    int collision_model;  /* LBDPS_COLLIDE_HARD (0): time-driven hard spheres of §2.2,
                             Eq. 17-18.  LBDPS_COLLIDE_SOFT (1): soft spheres, the DEM
                             alternative §2.2 names for dense beds: each pair closer than
                             d_p and each face closer than d_p/2 pushes with
                             max(0, k_n overlap - eta v_n) along the line of centres, eta
                             giving the restitution e (which must then be > 0); the force
                             joins the drag of Eq. 16.  Positions may then overlap */
    double dem_kn;        /* soft-sphere normal stiffness k_n, N/m (> 0 with
                             LBDPS_COLLIDE_SOFT; a pair contact must last at least
                             4 steps: pi sqrt(m_p / (2 k_n)) >= 4 dt) */
    double dem_mu;        /* soft-sphere friction, the tangential contact force §2.2
                             credits DEM with: Coulomb coefficient mu >= 0.  With mu > 0
                             and dem_gamma_t > 0 the contact point's tangential slip v_t
                             (spins included) meets -min(gamma_t |v_t|, mu F_n) v_t/|v_t|,
                             whose torque turns the particles (I = 2/5 m_p r^2; one spin
                             component in 2D, three in 3D).  0 = no friction */
    double dem_gamma_t;   /* tangential damping gamma_t, kg/s (>= 0; at most 0.25 m_p / dt,
                             above which the explicit update of a sliding pair is unstable) */
} lbdps_particle_desc;

#define LBDPS_COLLIDE_HARD 0
#define LBDPS_COLLIDE_SOFT 1

/* Gas and run parameters. */
typedef struct {
    double rho_g;         /* gas density, kg/m^3                                  */
    double mu_g;          /* gas viscosity, Pa s (tau = 3 nu + 1/2, Eq. 3)         */
    double g[3];          /* gravity, m/s^2 (particles feel (1 - rho_g/rho_s) g)  */
    double body_accel[3]; /* gas body acceleration, m/s^2 (Guo forcing)            */
    double u0[3];         /* initial gas velocity, m/s (equilibrium at rho = 1)    */
    double cs_smag;       /* Smagorinsky constant C_s of Eq. 12-15; 0 = off        */
    int superficial_mode; /* actual velocity = u / eps_2d (0), u / eps_g (1), u (2) */
    int pressure_plus;    /* 1: +V_p grad p as printed in Eq. 16; 0: -V_p grad p   */
    int storage;          /* LBDPS_STORE_*                                         */
    int check_every;      /* read the health word every k steps in lbdps_step (0 = never) */
    int diagnostics;      /* 1: keep the extra node and particle diagnostics       */
    int use_graph;        /* 1: replay lbdps_step through a captured CUDA graph    */
    void *stream;         /* cudaStream_t for all work; NULL = the handle's own    */
    void *(*alloc)(size_t bytes, void *ctx);  /* device allocator, or NULL       */
    void (*free)(void *ptr, void *ctx);       /* matching release, or NULL       */
    void *alloc_ctx;
} lbdps_params;

typedef struct {
    double mass;                 /* sum of gas populations                          */
    double gas_momentum[3];      /* sum_i c_i f_i over the lattice                  */
    double particle_momentum[3]; /* sum m_p v                                       */
    double mean_eps_g;           /* lattice-mean gas voidage eps_g (Eq. 10-11) of the
                                    current particle positions                        */
    double mean_slip;            /* particle-weighted mean |u_act - v_s| of the last
                                    step (needs diagnostics, else NaN)                */
    int64_t steps;               /* steps taken so far                              */
    int health;                  /* bitmask: 1 diverged, 2 domain, 4 capacity, 8 packed
                                    (a statistics reduction saw a cell holding more
                                    particle centres than can be there without overlaps,
                                    the close-packing count of the cell grown by d_p:
                                    hard spheres piled up, §2.2 limits them to low solid
                                    fractions; reported only, never an error)          */
    int64_t solids_out;          /* particles that left through the outlet since creation
                                    (recirculate = 1; the solids flux of §3.2 is
                                    solids_out m_p / (outlet area x time))            */
} lbdps_stats_t;

/* Create a bed (the paper's step 1, Fig. 4).  Validates the description:
 * tau > 1/2, |u| < 0.3 in lattice units, d_p <= h, periodic axes of at least
 * 3 cells, inlet/outlet only on the vertical axis, particles inside the
 * domain and (hard spheres) pairwise at least d_p apart, the last checked on
 * the device after the initial sort.  Returns LBDPS_ERR_INVALID, _OOM or
 * _CUDA on failure and leaves *out NULL. */
int lbdps_create(const lbdps_lattice_desc *lattice, const lbdps_particle_desc *particles,
                 const lbdps_params *params, lbdps_t **out);

/* Release the handle and all its device memory (waits for its stream). */
void lbdps_destroy(lbdps_t *h);

/* Advance nsteps coupled steps (Fig. 4 steps 2-6), asynchronously on the
 * handle's stream.  With check_every > 0 the health word is read every
 * check_every steps and LBDPS_ERR_DIVERGED / _DOMAIN is returned. */
int lbdps_step(lbdps_t *h, int64_t nsteps);

/* Advance nsteps coupled steps and take the FP64 statistics of lbdps_stats
 * after every one of them, without a host wait between steps: each step's
 * reduction writes its results straight into mapped pinned host memory and
 * the host waits once per 1,024 steps.  Without node diagnostics (and with
 * graphs) the collision of step s + 1 also sums the gas mass and momentum of
 * the state after step s, whose reduction then runs right after step s + 1
 * on the handle's stream, reading the health word and outlet count from a
 * snapshot taken at the end of step s; mean_slip is then NaN.  The records
 * equal lbdps_stats taken after each step.  out receives nsteps records (host
 * array, caller-owned), record k describing the state after step k + 1 of the
 * call.  With check_every > 0, LBDPS_ERR_DIVERGED / _DOMAIN as lbdps_step;
 * LBDPS_ERR_OOM if the pinned buffer cannot be had. */
int lbdps_step_monitored(lbdps_t *h, int64_t nsteps, lbdps_stats_t *out);

/* Advance nsteps steps launching each kernel separately with CUDA events
 * around it; kernel_ms[k] receives the summed milliseconds of kernel class k
 * (order: collide_stream, drag, sort, collide_particles), cap entries at
 * most.  Returns the number of classes in *nclass. */
int lbdps_step_profiled(lbdps_t *h, int64_t nsteps, double *kernel_ms, int cap, int *nclass);

/* Wait for the handle's stream. */
int lbdps_sync(lbdps_t *h);

/* Copy node fields of the last step (collision-time values, Eq. 5, 24, 25,
 * 19) into out: for each bit of mask in increasing order, ncell values (or
 * ncell x dim, cell-major) as double.  cap is the capacity of out in doubles;
 * LBDPS_ERR_CAPACITY if too small.  Bits other than RHO, FPG, BETA and UACT
 * need params.diagnostics = 1 (else LBDPS_ERR_INVALID).  units:
 * LBDPS_UNITS_LATTICE or _SI. */
int lbdps_fields(lbdps_t *h, int mask, int units, double *out, size_t cap);

/* which voidage lbdps_bubbles thresholds */
#define LBDPS_VOIDAGE_2D 0   /* eps_2d = 1 - eps_s of the cell, Eq. 10          */
#define LBDPS_VOIDAGE_G  1   /* eps_g, the 3D voidage of Eq. 11 (= eps_2d in 3D) */

/* Bubble regions of the current particle positions (§3.1): connected regions
 * (neighbours along the axes, wrapping across periodic faces) of cells whose
 * voidage (LBDPS_VOIDAGE_*, from the cell's particle count) exceeds
 * threshold (0.85 in §3.1), leaving out the regions that reach the top row of
 * the vertical axis (the freeboard above the bed).  out[0] = cells of the
 * largest region, out[1] = number of regions, out[2] = cells in all regions.
 * The equivalent bubble diameter of §3.1 (a circle of the same area) is
 * 2 h sqrt(out[0] / pi) in 2D.  Device scratch of three ints per cell is
 * allocated on the first call and kept.  LBDPS_ERR_INVALID for a threshold
 * outside [0, 1) or an unknown voidage. */
int lbdps_bubbles(lbdps_t *h, double threshold, int voidage, int64_t out[3]);

/* Replace the inlet velocities (m/s, inlet-face cells x dim, x-fastest, as
 * lbdps_lattice_desc.inlet_u), e.g. to end a jet pulse (§3.1: the injection
 * lasts 0.006 s).  Takes effect from the next step, graphs included.
 * LBDPS_ERR_INVALID if the bed has no inlet or |u| >= 0.3 in lattice units. */
int lbdps_set_inlet(lbdps_t *h, const double *inlet_u);

/* Self-check of the handle's device memory (not in the paper): every block
 * the handle allocated is followed by a 256-byte guard zone written with a
 * fixed pattern at creation; *damaged receives the number of blocks whose
 * guard no longer holds it (a kernel wrote past the end of a buffer).  For
 * tests; waits for the handle's stream. */
int lbdps_check_guards(lbdps_t *h, int *damaged);

/* Copy the particle state (section 2.2: P, v) in id order, n x dim each.
 * cap is the capacity of each array in particles. */
int lbdps_particles(lbdps_t *h, int units, double *pos, double *vel, int64_t cap);

/* Replace the particle state: n particles in id order, lattice units,
 * n x dim each; sorts them into cells; spins (friction) restart at zero.
 * Checks that the positions lie inside the domain (no overlap check). */
int lbdps_set_particles(lbdps_t *h, int64_t n, const double *pos, const double *vel);

/* Particle spins of soft spheres with friction (dem_mu, dem_gamma_t > 0), in id
 * order: one value per particle in 2D (about the axis normal to the plane,
 * counter-clockwise positive), three in 3D; rad per step (LBDPS_UNITS_LATTICE)
 * or rad/s (LBDPS_UNITS_SI).  cap counts doubles.  Zeros without friction. */
int lbdps_particle_spin(lbdps_t *h, int units, double *out, int64_t cap);

/* Replace the spins (lattice units, layout of lbdps_particle_spin, n particles);
 * LBDPS_ERR_INVALID without friction. */
int lbdps_set_particle_spin(lbdps_t *h, const double *in, int64_t n);

/* Copy the pre-collision populations f_i (full values, Eq. 2) as double,
 * layout [q][cell]; cap in doubles (>= q * ncell). */
int lbdps_populations(lbdps_t *h, double *f, size_t cap);

/* Replace the populations (full values, [q][cell]); each value is rounded
 * to the storage format as the deviation f_i - w_i. */
int lbdps_set_populations(lbdps_t *h, const double *f, size_t count);

/* Per-particle diagnostics of the last step in id order (LBDPS_PDIAG_*),
 * as double; cap in doubles. */
int lbdps_particle_diag(lbdps_t *h, int which, double *out, size_t cap);

/* The particle half of step 6 alone on the current state: sort into cells,
 * detect approaching contacts (section 2.2) and apply Eq. 17-18.  When pairs
 * is not NULL the approaching contact pairs (id_i < id_j) are written as
 * 2*count int64 in increasing (id_i, id_j) order, cap pairs at most;
 * *npairs receives the total (LBDPS_ERR_CAPACITY if it exceeds cap). */
int lbdps_collide_particles(lbdps_t *h, int64_t *pairs, int64_t cap, int64_t *npairs);

/* Deterministic FP64 reductions of the current state. */
int lbdps_stats(lbdps_t *h, lbdps_stats_t *out);

/* Health bitmask (1 diverged, 2 domain, 4 capacity, 8 packed) accumulated so far. */
int lbdps_health(lbdps_t *h, int *health);

/* Lattice-unit constants derived at create, in this order: tau, nu, mu,
 * rho_s/rho_g, d, r, V_p, m_p, e, g_eff[3], F_b[3], u0[3], C_s, then (as far
 * as cap allows) the soft-sphere k_n, eta (pair), eta (wall), mu, gamma_t
 * (0 with hard spheres) and the moment of inertia 2/5 m_p r^2. */
int lbdps_constants(lbdps_t *h, double *out, int cap);

/* Shape queries. */
int lbdps_shape(lbdps_t *h, int *dim, int *q, int64_t *ncell, int64_t *nparticles);

/* Checkpoint: raw populations, particle arrays, cell list and step count.
 * lbdps_save writes at most cap bytes into buf (NULL buf: only *used is
 * set to the size needed).  lbdps_load restores a checkpoint made by a
 * handle of the same shape and storage; the continuation is bit-identical. */
int lbdps_save(lbdps_t *h, void *buf, size_t cap, size_t *used);
int lbdps_load(lbdps_t *h, const void *buf, size_t size);

/* Exact device-memory footprint, in bytes, of the bed lbdps_create would
 * build from this description (all buffers, rounded to 256 B each).  No
 * device work; the same validation as create except the overlap test. */
int lbdps_memory_estimate(const lbdps_lattice_desc *lattice, const lbdps_particle_desc *particles,
                          const lbdps_params *params, size_t *bytes);

/* Record the CUDA event `event` (a cudaEvent_t) on the handle's stream,
 * after all work issued so far. */
int lbdps_record_event(lbdps_t *h, void *event);

/* ---- serving: continuous batching of independent beds ----------------
 * Not in the paper: a request loop for many independent beds of different
 * sizes.  Requests queue in FIFO order; the head is admitted when its exact
 * footprint (lbdps_memory_estimate) fits in the HBM budget and fewer than
 * max_active beds are resident.  Every resident bed keeps its populations
 * and particles on the device, on a stream of its own; each poll advances
 * every resident bed by one tick (steps_per_tick steps, each a replay of the
 * bed's captured step graph), so the beds' work overlaps on the GPU.  A bed
 * that reached its step count is harvested: its statistics and times are
 * reported and its memory is released (or kept for lbdps_server_take), which
 * admits the next requests.  A bed's results are identical to running it
 * alone.  Times are seconds on the host's steady clock since server
 * creation.  The server is not thread safe. */
typedef struct lbdps_server lbdps_server_t;

typedef struct {
    uint64_t id;          /* request id from lbdps_server_submit                     */
    int status;           /* LBDPS_OK, or the error that ended the request           */
    int64_t steps;        /* steps taken                                             */
    double cells;         /* lattice cells                                           */
    double t_submit, t_admit, t_done;   /* seconds                                  */
    lbdps_stats_t stats;  /* FP64 statistics at completion                           */
} lbdps_done_t;

int lbdps_server_create(size_t hbm_budget, int max_active, int steps_per_tick,
                        lbdps_server_t **out);
/* Queue a bed (descriptions and arrays are copied).  keep = 1 keeps the
 * finished handle for lbdps_server_take.  LBDPS_ERR_CAPACITY if the bed can
 * never fit the budget. */
int lbdps_server_submit(lbdps_server_t *s, const lbdps_lattice_desc *lattice,
                        const lbdps_particle_desc *particles, const lbdps_params *params,
                        int64_t nsteps, int keep, uint64_t *req_id);
/* Admit, advance one tick and harvest, repeating for up to wait_s seconds
 * until at least one request completes; completion records are written to
 * out (cap entries at most), their number to *ndone. */
int lbdps_server_poll(lbdps_server_t *s, double wait_s, lbdps_done_t *out, int cap, int *ndone);
/* Queue length, resident beds and bytes of the budget in use. */
int lbdps_server_load(lbdps_server_t *s, int *queued, int *active, size_t *used);
/* Hand over a finished kept bed; the caller then owns the handle (lbdps_destroy). */
int lbdps_server_take(lbdps_server_t *s, uint64_t req_id, lbdps_t **out);
/* Batched stepping (on by default).  Small beds of the batched kind (2D,
 * FP32 arithmetic, FP32 / FP16 / BF16 population storage, hard spheres, at
 * most max_cells cells and at most one particle per cell on average) advance
 * together: each kernel of a coupled step is one launch over all of them, a
 * device work table of (bed, tile) entries walked by persistent thread
 * blocks, and a tick of steps_per_tick steps is one replay of a captured
 * CUDA graph.  Each bed's arithmetic is that of the bed run alone.  Larger
 * or denser beds, and beds of other kinds, advance on streams of their own
 * by replays of their own step graphs.  on = 0: every bed on its own stream.
 * max_cells = 0 keeps the default (32768 cells).  Applies to beds admitted
 * afterwards; LBDPS_ERR_INVALID for max_cells < 0. */
int lbdps_server_set_batching(lbdps_server_t *s, int on, int64_t max_cells);
/* Counters of the batch: ticks launched, graph captures, current members. */
int lbdps_server_batch_info(lbdps_server_t *s, int64_t *ticks, int64_t *captures, int *members);
void lbdps_server_destroy(lbdps_server_t *s);

/* Cell binning without device allocation.  The paper has no counterpart:
 * this is a service for callers that must not allocate GPU memory while they
 * run (work being recorded into a CUDA graph, real-time loops that cannot
 * afford the implicit synchronisation of cudaMalloc/cudaFree, hosts that own
 * a fixed device-memory budget).
 *
 * Computes the same (cell, id) ordering and cell list as the handle-based
 * path, for np particles with ids 0..np-1:
 *   dim          2 or 3;  n: cells per axis (n[2] ignored in 2D)
 *   pos[a]       DEVICE array of np FP64 coordinates along axis a, lattice
 *                units; a coordinate below 0 (or NaN) counts in the first
 *                cell of its axis, one at or above n[a] in the last
 *   cell_start   DEVICE output, ncell + 1 ints: particles of cell c occupy
 *                sorted slots cell_start[c] .. cell_start[c+1]-1
 *   order        DEVICE output, np ints: the particle id in each sorted slot
 *   stream       cudaStream_t (NULL = legacy default stream); asynchronous
 * The order inside a cell comes from a stable radix sort of the cell keys
 * (at most three 8-bit passes), so the work is linear in np whatever the
 * occupancy of the cells.  np < 0 returns LBDPS_ERR_INVALID.
 * Temporaries live in one fixed device array of about 28 MB, created on each
 * GPU that loads the library and kept until the process exits; this function
 * calls no cudaMalloc, cudaFree or allocating library routine.  Limits:
 * ncell <= 1048576 and np <= 1048576, otherwise LBDPS_ERR_CAPACITY with no
 * work issued.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  Every call shares the one array, so calls
 * whose work overlaps on the GPU (other streams, other host threads) race and
 * give wrong results: serialise them. */
int lbdps_bin_sort_noalloc(int dim, const int n[3], int64_t np, const double *const pos[3],
                           int *cell_start, int *order, void *stream);

/* Message text of a status code, and of the last failure on this thread. */
const char *lbdps_strerror(int code);
const char *lbdps_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBDPS_H */

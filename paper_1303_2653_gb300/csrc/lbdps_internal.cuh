// Internal declarations of the sm_103a LB-DPS library: lattice velocity sets,
// kernel parameter blocks, storage conversions and kernel launchers.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbdpsk {

enum { BC_WALL = 0, BC_PERIODIC = 1, BC_INLET = 2, BC_OUTLET = 3 };
enum { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };
// HEALTH_PACKED: a cell held more particle centres than could be there
// without overlaps (time-driven hard spheres cannot hold a dense bed apart,
// §2.2); found by the statistics reduction, reported, not an error
enum : unsigned { HEALTH_DIVERGED = 1u, HEALTH_DOMAIN = 2u, HEALTH_CAPACITY = 4u, HEALTH_PACKED = 8u };

// ---------------------------------------------------------------------------
// Velocity sets.  D2Q9 in the paper's order (Eq. 4): rest, the four axis
// directions counter-clockwise from +x, the four diagonals counter-clockwise
// from (1,1).  D3Q19: rest, +-x, +-y, +-z, then the twelve edge diagonals in
// opposite pairs.  Written as constexpr selections so that unrolled loops
// fold every c_ia into an immediate.
// ---------------------------------------------------------------------------
struct D2Q9 {
    static constexpr int D = 2, Q = 9;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        return a == 0 ? ((i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0)
             : a == 1 ? ((i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0)
                      : 0;
    }
    __host__ __device__ static constexpr int opp(int i)
    {
        return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
    }
    // first member of the k-th opposite pair (k = 0..3): 1, 2, 5, 6
    __host__ __device__ static constexpr int pair_first(int k) { return k < 2 ? k + 1 : k + 3; }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

struct D3Q19 {
    static constexpr int D = 3, Q = 19;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        return a == 0 ? ((i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
                         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0)
             : a == 1 ? ((i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
                         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0)
                      : ((i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
                         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    // first member of the k-th opposite pair (k = 0..8): 1, 3, 5, ..., 17
    __host__ __device__ static constexpr int pair_first(int k) { return 2 * k + 1; }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// ---------------------------------------------------------------------------
// Storage of population deviations f_i - w_i.
// ---------------------------------------------------------------------------
template <class S> struct Store;
template <> struct Store<double> {
    using R = double;
    __device__ static double load(double v) { return v; }
    __device__ static double save(double v) { return v; }
};
template <> struct Store<float> {
    using R = float;
    __device__ static float load(float v) { return v; }
    __device__ static float save(float v) { return v; }
};
// FP16 keeps the deviation scaled by 2^10 so that small deviations stay
// normal numbers (FP16 subnormals start below 6.1e-5).
constexpr float kF16Scale = 1024.0f;
template <> struct Store<__half> {
    using R = float;
    __device__ static float load(__half v) { return __half2float(v) * (1.0f / kF16Scale); }
    __device__ static __half save(float v) { return __float2half_rn(v * kF16Scale); }
};
template <> struct Store<__nv_bfloat16> {
    using R = float;
    __device__ static float load(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 save(float v) { return __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------------------
// Per-particle-count tables (deposition, Eq. 9-11, 19-20), built in FP64.
// Index n = particles whose centre lies in the cell, clamped to ntab - 1
// (beyond that the solid fraction is at its close-packing cap).
// ---------------------------------------------------------------------------
template <class R> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

template <class Real> struct CountTables {
    // packed copies for the lattice kernel: pk0 = {og, gam, inv_div, beta_a},
    // pk1 = {beta_b, beta_c, re_k, branch}
    const typename Vec4<Real>::type *pk0;
    const typename Vec4<Real>::type *pk1;
    const Real *eps_s;    // solid fraction (Eq. 10, capped)
    const Real *eps_g;    // gas voidage for the drag (Eq. 11 in 2D)
    const Real *sol_g;    // 1 - eps_g, kept separately so 1 - eps_k needs no cancellation
    const Real *inv_div;  // 1 / divisor of the superficial -> actual velocity
    const Real *og;       // omega(eps_g) * gamma(eps_s, tau)  (Eq. 20, 9)
    const Real *gam;      // gamma(eps_s, tau)
    const Real *beta_a;   // beta = beta_a + beta_b |slip| (Ergun branch) or
    const Real *beta_b;   //        beta_a (1 + 0.15 Re^0.687)            (dilute, Re < 1000)
    const Real *beta_c;   //        beta_c |slip|                          (dilute, Re >= 1000)
    const Real *re_k;     // Re_p = re_k |slip| (Eq. 22)
    const int *branch;    // 0 Ergun, 1 dilute (decided in FP64 on eps_g > 0.74)
    int ntab;
};

// ---------------------------------------------------------------------------
// Parameter block shared by all step kernels (passed by value).
// ---------------------------------------------------------------------------
template <class Real> struct StepParams {
    int dim;
    int n[3];
    int ncell;
    int bc[6];
    int vert;                 // vertical axis (dim - 1)
    Real tau, inv_tau;
    Real les_k;               // 18 C_s^2 (0 = LES off)
    Real fb[3];               // gas body force density
    int has_fb;
    Real wall_u[6][3];
    Real mu, d, r, vp, mp, e;
    Real geff[3];
    Real psign;               // -1 or +1 for the pressure-gradient force
    double d2;                // d^2 in FP64 for the contact test
    double r64;
    double len[3];            // domain lengths as double
    double len_below[3];      // largest double below len
    CountTables<Real> tab;
    const Real *inlet_u;      // inlet face cells x dim
    int inlet_face;           // face index or -1
    unsigned *health;
    int recirculate;          // 1: outlet -> inlet re-injection of particles
    unsigned long long *solids_out;   // particles through the outlet so far
    // soft spheres: contact forces of the step in sorted slot order (null
    // with hard spheres), stiffness and pair / wall damping
    Real *fc[3];
    Real kn, eta, eta_w;
    // soft-sphere friction: Coulomb coefficient, tangential damping and 1 / I
    // (mu_f = 0: none); the new spins go to spin_out (sorted slot order)
    Real mu_f, gamma_t, inv_inertia;
    Real *spin_out[3];
    // with a monitored step: per-warp sums of the cell moments (mass
    // deviation and momentum, Q-population sums of the state the collision
    // reads) of the collision's warps, 4 FP64 values per warp (null: none)
    double *gas_partials;
};

// Sum over a warp in a fixed order (butterfly of shuffles): every lane holds
// the total.
template <class T> __device__ __forceinline__ T warp_total(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Layout of the population arrays: the lattice plus one ghost layer on every
// face (x = -1 and n0, y = -1 and n1, and in 3D z = -1 and n2), rows padded to
// a multiple of 32 slots with x = 0 at offset 32, so that the cells of a row
// start a 128-byte line in FP32.  Direction i occupies nce consecutive slots.
// The populations are stored after the collision and pulled by the next one:
// f_i(x) is read at x - c_i, which is a ghost slot for directions entering
// through a face.
struct PopLayout {
    static constexpr int pad = 32;
    int n[3];
    int s0, s1;        // row and plane strides of the extended lattice
    int zo;            // 1 in 3D (one ghost plane below z = 0), 0 in 2D
    long long nce;     // slots per direction
    // slots of one direction are indexed in 32 bits (nce < 2^31, checked at
    // creation)
    __host__ __device__ int ext(const int *q) const
    {
        return pad + q[0] + s0 * ((q[1] + 1) + s1 * (q[2] + zo));
    }
    template <class L> __host__ __device__ int off(int i) const
    {
        return L::c(i, 0) + L::c(i, 1) * s0 + L::c(i, 2) * s0 * s1;
    }
};

// Per-direction base pointers of the population arrays for one collision:
// direction i of the cell at extended slot xe is read at pull[i][xe]
// (pull[i] = fin + i nce - off_i, the slot of x - c_i) and the cell's own
// post-collision value is written at own[i][xe] (own[i] = fout + i nce).
template <class S> struct PopPtrs {
    const S *pull[19];
    S *own[19];
};

inline PopLayout make_layout(int dim, const int *n)
{
    PopLayout l;
    for (int a = 0; a < 3; ++a) l.n[a] = n[a];
    l.s0 = ((n[0] + 2 + 31) / 32) * 32;
    l.s1 = n[1] + 2;
    l.zo = dim == 3 ? 1 : 0;
    const long long s2 = dim == 3 ? n[2] + 2 : 1;
    l.nce = (long long)l.s0 * l.s1 * s2 + PopLayout::pad;
    return l;
}

// Solid fraction (Eq. 10, capped at close packing) and gas voidage eps_g
// (Eq. 11 in 2D, 1 - eps_s in 3D) of a cell holding n particle centres, in
// FP64 (lattice units: r the particle radius, vp its volume).
__host__ __device__ inline void cell_voidage(int dim, double r, double vp, int n, double *es_out,
                                             double *eg_out, double *sg_out)
{
    const double pi = 3.141592653589793238462643383;
    double es, sg;
    if (dim == 2) {
        const double cap = pi / (2.0 * sqrt(3.0));
        es = fmin((double)n * pi * r * r, cap);
        const double s = 1.0 - (1.0 - es);                        // 1 - eps_2d
        sg = sqrt(2.0) / sqrt(pi * sqrt(3.0)) * (s * sqrt(s));   // eps_3d = 1 - sg
    } else {
        const double cap = pi / (3.0 * sqrt(2.0));
        es = fmin((double)n * vp, cap);
        sg = es;
    }
    *es_out = es;
    *sg_out = sg;
    *eg_out = 1.0 - sg;
}

// Device buffers of one bed.
// node4 is the record the drag reads at each stencil node, one 16-byte (FP32)
// load: {u_act,x, u_act,y, 1 - eps, beta} in 2D and {u_act,x, u_act,y,
// u_act,z, beta} in 3D, where 1 - eps is in solg.
template <class Real> struct Fields {
    Real *rho, *fpg[3];                                 // node outputs of the collision
    typename Vec4<Real>::type *node4;
    Real *solg;                                         // 3D only (null in 2D)
    Real *vs[3], *tau_t, *u[3], *eps_g;                 // diagnostics (may be null)
    int *ntot;                                          // diagnostics (may be null)
};

// Particle arrays in cell-sorted order.  Besides the FP64 centre P and the
// velocity v, each particle carries its cell index and its offset inside the
// cell, off = P - floor(P) (in the arithmetic type), so that interpolation
// weights and the coarse contact test need no FP64 arithmetic.
template <class Real> struct Particles {
    double *P[3];
    Real *v[3];
    int *id;
    int *cell;
    Real *off[3];
    // angular velocity of soft spheres with friction (null otherwise): the
    // component normal to the plane in 2D (w[0]), three components in 3D
    Real *w[3];
};

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files, explicitly instantiated).
// ---------------------------------------------------------------------------
// Cell list after a sort: particles of cell c occupy sorted slots
// begin(c) .. begin(c + 1) - 1.  It is kept in two levels so that one kernel
// can produce it: an exclusive prefix of the per-cell counts inside each tile
// of 2^shift cells, and the exclusive prefix of the tile totals.  Tiles hold
// 4,096 cells, or 16,384 on lattices of at least 2^22 cells, where the last
// block of the scan would otherwise add up tens of thousands of tile totals
// one block-width at a time.
constexpr int kCellTileLog2 = 12;
constexpr int kCellTileLog2Large = 14;
constexpr int kLargeLatticeCells = 1 << 22;
inline int cell_tile_log2(int ncell) { return ncell >= kLargeLatticeCells ? kCellTileLog2Large : kCellTileLog2; }
inline int cell_tiles(int ncell)
{
    const int s = cell_tile_log2(ncell);
    return (ncell + 1 + (1 << s) - 1) >> s;
}
struct CellList {
    const int *local;   // ncell + 1 entries
    const int *base;    // cell_tiles(ncell) + 1 entries
    int shift;          // cell_tile_log2(ncell)
    __device__ __forceinline__ int begin(int c) const
    {
        return __ldg(local + c) + __ldg(base + (c >> shift));
    }
};
struct CellListOut {
    int *local, *base, *tile_total;
    unsigned *ticket;   // zero between launches
    int shift;
};

// Scratch of the bubble labelling (one int per cell for parent, size and
// top flags; three counters; the count limit; an error word).
struct BubbleScratch {
    int *parent, *size, *top, *nlim;
    unsigned long long *out;   // largest region, regions, cells in regions
    unsigned *err;
};

// Bubble regions of the current cell list (§3.1): cells whose voidage
// (voidage 0: eps_2d, Eq. 10; 1: eps_g, Eq. 11) exceeds threshold, connected
// along the axes (periodic faces wrap), without the regions that reach the
// top row of the vertical axis.  per_mask bit a: axis a is periodic.
void launch_bubbles(int dim, const int *n, int per_mask, double r, double vp, int ntab,
                    double threshold, int voidage, CellList cells, BubbleScratch s,
                    cudaStream_t st);


template <class L, class Real, class S>
void launch_collide_stream(const StepParams<Real> &p, const PopLayout &lay, const S *fin, S *fout,
                           CellList cells, Particles<Real> parts, Fields<Real> fld, cudaStream_t st);

template <class L, class Real, class S>
void launch_init_equilibrium(const PopLayout &lay, const Real *u0, S *f, cudaStream_t st);

// Warps of a collide_stream launch on a lattice of n cells per axis (the
// size of the gas_partials array in groups of 4 doubles).
long long collide_warps(int dim, const int *n);

// The cell moments of the state held in f (as the next collision pulls it),
// summed per warp of the collision's grid exactly as a collision with
// gas_partials does: 4 doubles per warp into partials.
template <class L, class Real, class S>
void launch_gas_moments(const PopLayout &lay, const S *f, const int *n, double *partials,
                        cudaStream_t st);

template <class L, class Real, class S>
void launch_export_populations(const PopLayout &lay, int ncell, const S *f, double *out,
                               cudaStream_t st);

template <class L, class Real, class S>
void launch_import_populations(const PopLayout &lay, int ncell, const double *in, S *f,
                               cudaStream_t st);

template <class Real>
void launch_build_tables(int dim, double tau, double r, double vp, double d, double mu,
                         int superficial_mode, int ntab, double *scratch, CountTables<Real> tab,
                         cudaStream_t st);

// Fig. 4 steps 4-5 in one launch: Eq. 26-28 and the integration of Eq. 16.
// `out` receives the integrated P, v and in-cell offset in the same slots.
template <int D, class Real>
void launch_drag_step(const StepParams<Real> &p, Particles<Real> parts, Particles<Real> out,
                      CellList cells, Fields<Real> fld, int *key, int *counts, Real *diag_fpre,
                      Real *diag_fd, int np, cudaStream_t st);

template <int D, class Real>
void launch_cell_keys(const int *n, Particles<Real> parts, int *key, int *counts, int np,
                      cudaStream_t st);

// The particle state in id order, interleaved (np x D), positions times ps
// and velocities times vs in FP64 (either output may be null).
template <int D, class Real>
void launch_particles_to_host_order(Particles<Real> parts, int np, double ps, double vs,
                                    double *pos, double *vel, cudaStream_t st);
// Interleaved id-order positions and velocities (np x D) into the SoA arrays
// of dst in lattice units (positions / pos_div, velocities * vel_mul, both
// correctly rounded in FP64), with ids 0..np-1 and spins (if any) at rest.
template <int D, class Real>
void launch_particles_from_host_order(const double *pos, const double *vel, int np, double pos_div,
                                      double vel_mul, Particles<Real> dst, cudaStream_t st);

// one-launch scan of counts[0..ncell] (counts[ncell] = 0) into a CellList
void launch_cell_scan(const int *counts, CellListOut out, int ncell, cudaStream_t st);

// slot placement and in-cell ordering by id: src (any order) -> dst (cell, id)
template <class Real>
void launch_place(int dim, const int *key, int *counts, CellList cells, int2 *slot, int *idslot,
                  Particles<Real> src, Particles<Real> dst, int np, cudaStream_t st);

template <int D, class Real>
void launch_detect(const StepParams<Real> &p, Particles<Real> parts, CellList cells, int *best,
                   int *wall, long long *pairs, unsigned long long *npairs, long long pair_cap,
                   int np, cudaStream_t st);

// three-kernel scan into a plain cell_start[ncell + 1] (used by the
// allocation-free binning entry point)
void launch_scan(const int *counts, int *cell_start, int *block_sums, int ncell, cudaStream_t st);
int scan_block_count(int ncell);

// pairs of particles closer than d (creation check of hard spheres): count
// and the smallest (id_i << 32 | id_j), i < j
template <int D, class Real>
void launch_overlaps(const StepParams<Real> &p, Particles<Real> parts, CellList cells,
                     unsigned long long *count, unsigned long long *first, int np, cudaStream_t st);

// soft-sphere contact forces of the step into p.fc (sorted slot order)
template <int D, class Real>
void launch_contacts(const StepParams<Real> &p, Particles<Real> parts, CellList cells,
                     Real *diag_fc, int np, cudaStream_t st);

template <int D, class Real>
void launch_resolve(const StepParams<Real> &p, Particles<Real> parts, const int *best,
                    const int *wall, int np, cudaStream_t st);

// Sizes of the statistics buffers: the reduction runs at most
// kStatMaxBlocks blocks, each writing kStatValues partials; out holds
// kStatValues values plus the health word and the outlet count.
constexpr int kStatValues = 11;
constexpr int kStatMaxBlocks = 152 * 4;   // four blocks of 512 threads per SM
constexpr int kStatPartials = kStatValues * kStatMaxBlocks;
constexpr int kStatOut = kStatValues + 2;

// copies the health word and the outlet count to out[0], out[1]
void launch_snapshot(const unsigned *health, const unsigned long long *solids_out,
                     unsigned long long *out, cudaStream_t st);

// All bed statistics in one launch (values listed in stats_kernels.cu); gas
// = ngas groups of 4 FP64 sums of the cell moments of the same state
// (launch_gas_moments, or a collision with gas_partials); parts = the
// particles of that state in sorted (cell) order; bed = the diagnostic
// fields or null; ticket must be zero on entry and is zero again on exit.
template <class L, class Real>
void launch_reduce_all(int ncell, const double *gas, long long ngas, Particles<Real> parts, double mp,
                       int np, const Real *eps_tab, int ntab, const Fields<Real> *bed,
                       double *partials, unsigned *ticket,
                       const unsigned *health, const unsigned long long *solids_out, double *out,
                       unsigned *health_live, int packed_limit, cudaStream_t st);

int reduce_block_count(int n);

// ---------------------------------------------------------------------------
// Batched stepping of many beds (the serving loop).  Every buffer and
// parameter one coupled step of a bed reads, for both buffer parities; the
// kernels of a batch read these records from device memory.  Beds of a batch
// are 2D with FP32 arithmetic and hard spheres; their populations may be
// stored in FP32, FP16 or BF16 (storage).
// ---------------------------------------------------------------------------
struct BatchBed {
    StepParams<float> sp;
    PopLayout lay;
    const void *f[2];              // population buffers in the bed's storage type
    int *cl_local[2], *cl_base[2];
    int cl_shift;                  // tile size of the cell list (cell_tile_log2)
    int *tile_total;
    unsigned *ticket;
    Particles<float> part[2], stage;
    Fields<float> fld;
    int *key, *counts, *idslot;
    int2 *slot;
    int *best, *wall;
    float *diag_fpre, *diag_fd;
    int np, ncell, storage;
    int parity0;                   // buffer parity at the start of the tick
    int nsteps;                    // steps this bed takes in the tick (<= the tick's length)
};

// Work tables of a batch: (bed, tile) per thread block of each kernel class.
// Cell tiles cover kBatchTile consecutive cells of a bed, scan tiles the
// tiles of the cell list, particle tiles kBatchTile
// consecutive sorted particles.  The entry counts live in device memory
// (count[0..2]: cell, scan, particle tiles), so a captured tick stays valid
// when the tables are rewritten for another set of beds.
constexpr int kBatchTile = 256;
struct BatchWork {
    const int2 *cell_tiles;
    const int2 *scan_tiles;
    const int2 *part_tiles;
    const int *count;   // device; null: launch nothing
};

// One coupled step of every bed of the batch whose nsteps exceeds `step`
// (step = 0 .. tick length - 1): the seven kernels of the single-bed step,
// each one launch over all beds (persistent blocks walking the work table).
// The first call of each launcher sizes its grid (call it outside stream
// capture; a null count launches nothing).
void launch_collide_stream_batched(const BatchBed *beds, BatchWork work, int step, cudaStream_t st);
void launch_particles_batched(const BatchBed *beds, BatchWork work, int step, cudaStream_t st);
// Blocks of `threads` threads of kernel `kern` that fit on the whole GPU at
// once (at least 1, at most nwork).
int resident_grid(const void *kern, int threads, int nwork);

}  // namespace lbdpsk

// Internal hooks of the handle API used by the serving loop.
struct lbdps;
namespace lbdpsk {
// Fills *out for a bed that can join a batch (2D, FP32 arithmetic, hard
// spheres), else returns LBDPS_ERR_INVALID.  parity0 / nsteps are left 0.
int batch_describe(struct lbdps *h, BatchBed *out);
// The bed's parity and step count after the batch advanced it nsteps steps.
void batch_advanced(struct lbdps *h, long long nsteps);
cudaStream_t bed_stream(struct lbdps *h);
int bed_parity(struct lbdps *h);
}  // namespace lbdpsk

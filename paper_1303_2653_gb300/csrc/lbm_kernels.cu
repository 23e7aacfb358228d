// Lattice kernels: fused deposition + modified-LBE collision + streaming
// (the paper's Fig. 4 steps 2-3), the FP64 per-count tables, and population
// import/export.
#include "lbdps_internal.cuh"

#include <algorithm>

namespace lbdpsk {

// ---------------------------------------------------------------------------
// Per-count tables.  For a cell holding n particle centres (Fig. 1) every
// deposition quantity is a function of n alone: the solid fraction (Eq. 10,
// capped at close packing), the gas voidage of Eq. 11, omega of Eq. 20,
// gamma of Eq. 9 and the n-dependent factors of beta (Eq. 19, 21, 22).  They
// are evaluated once in FP64 here, so every branch of Eq. 19-20 is decided in
// FP64, and the step kernel only indexes them.
// ---------------------------------------------------------------------------
template <class Real> struct TableOut {
    Real *eps_s, *eps_g, *inv_div, *og, *gam, *beta_a, *beta_b, *beta_c, *re_k, *sol_g;
    int *branch;
    typename Vec4<Real>::type *pk0, *pk1;
};

__device__ double emms_omega(double eg)
{
    // Eq. 20 (Yang et al. fit); 1 in the Ergun regime eps_g <= 0.74
    if (eg <= 0.74) return 1.0;
    if (eg <= 0.82) {
        double t = eg - 0.7463;
        return 0.0214 / (4.0 * t * t + 0.0044) - 0.5760;
    }
    if (eg <= 0.97) {
        double t = eg - 0.7789;
        return 0.0038 / (4.0 * t * t + 0.0040) - 0.0101;
    }
    return 32.8295 * eg - 31.8295;
}

template <class Real>
__global__ void k_build_tables(int dim, double tau, double r, double vp, double d, double mu,
                               int mode, int ntab, TableOut<Real> t)
{
    const double pi = 3.141592653589793238462643383;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < ntab; n += gridDim.x * blockDim.x) {
        double es, eg, sg;
        cell_voidage(dim, r, vp, n, &es, &eg, &sg);   // Eq. 10-11
        const double e2 = 1.0 - es;
        double div = (mode == 0) ? e2 : (mode == 1) ? eg : 1.0;
        double om = emms_omega(eg);
        double gm = es * (tau - 0.5) / ((1.0 - es) + (tau - 0.5));      // Eq. 9
        t.eps_s[n] = (Real)es;
        t.eps_g[n] = (Real)eg;
        t.sol_g[n] = (Real)sg;
        t.inv_div[n] = (Real)(1.0 / div);
        t.og[n] = (Real)(om * gm);
        t.gam[n] = (Real)gm;
        if (eg > 0.74) {
            // dilute branch of Eq. 19 with Eq. 21-22 (gas density 1):
            // beta = 3/4 (1-e) e C_d0 |s| / d * omega, C_d0 |s| = 24 mu (1 + 0.15 Re^0.687)/(e d)
            t.branch[n] = 1;
            t.beta_a[n] = (Real)(0.75 * (1.0 - eg) * eg * 24.0 * mu / (eg * d) / d * om);
            t.beta_b[n] = (Real)0.0;
            t.beta_c[n] = (Real)(0.75 * (1.0 - eg) * eg * 0.44 / d * om);
            t.re_k[n] = (Real)(eg * d / mu);
        } else {
            // Ergun branch of Eq. 19
            t.branch[n] = 0;
            t.beta_a[n] = (Real)(150.0 * (1.0 - eg) * (1.0 - eg) * mu / (eg * d * d));
            t.beta_b[n] = (Real)(1.75 * (1.0 - eg) / d);
            t.beta_c[n] = (Real)0.0;
            t.re_k[n] = (Real)0.0;
        }
        t.pk0[n] = {t.og[n], t.gam[n], t.inv_div[n], t.beta_a[n]};
        t.pk1[n] = {t.beta_b[n], t.beta_c[n], t.re_k[n], (Real)t.branch[n]};
    }
}

template <class Real>
void launch_build_tables(int dim, double tau, double r, double vp, double d, double mu,
                         int superficial_mode, int ntab, double *, CountTables<Real> tab,
                         cudaStream_t st)
{
    TableOut<Real> t{const_cast<Real *>(tab.eps_s), const_cast<Real *>(tab.eps_g),
                     const_cast<Real *>(tab.inv_div), const_cast<Real *>(tab.og),
                     const_cast<Real *>(tab.gam), const_cast<Real *>(tab.beta_a),
                     const_cast<Real *>(tab.beta_b), const_cast<Real *>(tab.beta_c),
                     const_cast<Real *>(tab.re_k), const_cast<Real *>(tab.sol_g),
                     const_cast<int *>(tab.branch),
                     const_cast<typename Vec4<Real>::type *>(tab.pk0),
                     const_cast<typename Vec4<Real>::type *>(tab.pk1)};
    int blocks = (ntab + 127) / 128;
    k_build_tables<Real><<<blocks, 128, 0, st>>>(dim, tau, r, vp, d, mu, superficial_mode, ntab, t);
}

// ---------------------------------------------------------------------------
// K2: one thread per cell.
//   deposition   n_tot and v_s from this cell's slice of the cell-sorted
//                particles (Eq. 8), table lookups for Eq. 9-11, 20
//   moments      rho and m = sum_i c_i f_i from the deviations
//   Eq. 24       u = [m (1 - wg) + wg/2 rho v_s + F_b/2] / (rho (1 - wg/2)),
//                wg = omega * gamma(eps_s, tau) (closed form of the implicit Eq. 24)
//   Eq. 13-15    tau_t = (tau + sqrt(tau^2 + 18 C_s^2 Q / rho)) / 2 if LES is on
//   Eq. 7, 23    f*_i = f_i - (1 - gamma(eps_s, tau_t))/tau_t (f_i - feq_i)
//                       + wg Omega^s_i + Guo source
//   Eq. 25       F_p->g = wg (rho u + rho v_s - 2 m)  (sum_i c_i Omega^s_i in closed form)
//   Eq. 19       node beta from |u/eps - v_s|
//   Eq. 2        push streaming; half-way bounce-back (moving wall) on walls,
//                inlet/outlet incoming populations at feq(1, u_in | u)
// All arithmetic on deviations f_i - w_i so that FP32 keeps the small
// velocity moments accurate.
// ---------------------------------------------------------------------------
template <class L, class Real>
__device__ __forceinline__ Real cdot(int i, const Real *u)
{
    Real s = Real(0);
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
        if (L::c(i, a) == 1) s += u[a];
        else if (L::c(i, a) == -1) s -= u[a];
    }
    return s;
}

// Re^0.687 of Eq. 21: the hardware exp2/log2 pair in FP32 (a few ulp), the
// correctly rounded pow in FP64.
__device__ __forceinline__ float re_pow(float re) { return re > 0.f ? __powf(re, 0.687f) : 0.f; }
__device__ __forceinline__ double re_pow(double re) { return pow(re, 0.687); }
// Reciprocal and square root: hardware approximations (a few ulp) in FP32,
// correctly rounded in FP64.
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_pos(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double sqrt_pos(double x) { return sqrt(x); }

// The collision runs blocks of kCollideThreads threads (a row of up to that
// many cells).  Blocks per SM requested from the register allocator: D2Q9 in
// FP32 fits in ~40 registers (12 blocks); D3Q19 in FP32 takes 56 (9 blocks,
// 36 warps per SM: against 8 blocks at 64 registers, the 16-bit storages
// run 8-9 % faster, FP32 the same); FP64 needs more.
constexpr int kCollideThreads = 128;
template <class L, class Real> struct K2Occupancy { static constexpr int value = 8; };
#ifndef LBDPS_K2_BLOCKS_D2Q9_F32
#define LBDPS_K2_BLOCKS_D2Q9_F32 12
#endif
#ifndef LBDPS_K2_BLOCKS_D3Q19_F32
#define LBDPS_K2_BLOCKS_D3Q19_F32 9
#endif
template <> struct K2Occupancy<D2Q9, float> { static constexpr int value = LBDPS_K2_BLOCKS_D2Q9_F32; };
template <> struct K2Occupancy<D3Q19, float> { static constexpr int value = LBDPS_K2_BLOCKS_D3Q19_F32; };
template <> struct K2Occupancy<D3Q19, double> { static constexpr int value = 4; };

// Streaming across the faces of the lattice (Eq. 2 with the boundary rules),
// run by the cells on a face after their own post-collision values are
// stored.  Populations are pulled: the next collision of cell x reads
// direction i at x - c_i of the extended lattice.  A slot of the ghost layer
// is written by the one rule that feeds its reader:
//   a direction leaving through a wall returns to this cell as -c_i
//   (half-way bounce-back, moving-wall term -6 w_i rho c_i.u_w of the first
//   wall crossed): written where this cell pulls -c_i from;
//   a direction leaving through periodic faces only re-enters at the image
//   cell: written where the image pulls it from;
//   a direction leaving through an inlet or outlet is dropped, and the
//   direction entering through it (no wall crossed) is set to
//   feq(1, u_in) or feq(1, u of this cell).
template <class L, class Real, class S>
__device__ __forceinline__ void face_streaming(const StepParams<Real> &p, const PopLayout &lay,
                                               const PopPtrs<S> &pp, int xe, const int *idx,
                                               Real rho, const Real *u)
{
    constexpr int D = L::D, Q = L::Q;
    int wall_faces = 0, open_faces = 0;
#pragma unroll
    for (int f6 = 0; f6 < 2 * D; ++f6) {
        if (p.bc[f6] == BC_WALL) wall_faces |= 1 << f6;
        else if (p.bc[f6] != BC_PERIODIC) open_faces |= 1 << f6;
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        int out = 0, in = 0;   // faces crossed by x + c_i and by x - c_i
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int c = L::c(i, a);
            const bool lo = idx[a] == 0, hi = idx[a] == p.n[a] - 1;
            if (c == 1) {
                if (hi) out |= 2 << (2 * a);
                if (lo) in |= 1 << (2 * a);
            } else if (c == -1) {
                if (lo) out |= 1 << (2 * a);
                if (hi) in |= 2 << (2 * a);
            }
        }
        const int off = lay.off<L>(i);
        if (out) {
            const Real post = Store<S>::load(pp.own[i][xe]);
            const int walls = out & wall_faces;
            if (walls) {
                const int face = __ffs(walls) - 1;   // first (lowest-axis) wall crossed
                const Real cw = Real(L::c(i, 0)) * p.wall_u[face][0] +
                                Real(L::c(i, 1)) * p.wall_u[face][1] +
                                Real(L::c(i, 2)) * p.wall_u[face][2];
                pp.own[L::opp(i)][xe + off] = Store<S>::save(post - Real(6) * Real(L::w(i)) * rho * cw);
            } else if (!(out & open_faces)) {
                int q[3] = {idx[0], idx[1], idx[2]};
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    q[a] += L::c(i, a);
                    if (q[a] < 0) q[a] += p.n[a];
                    else if (q[a] >= p.n[a]) q[a] -= p.n[a];
                }
                pp.own[i][lay.ext(q) - off] = Store<S>::save(post);
            }
        }
        if (in && !(in & wall_faces) && (in & open_faces)) {
            const int open = __ffs(in & open_faces) - 1;
            Real ub[3] = {Real(0), Real(0), Real(0)};
            if (p.bc[open] == BC_INLET) {
                const int j = (D == 2) ? idx[0] : idx[0] + p.n[0] * idx[1];
#pragma unroll
                for (int a = 0; a < D; ++a) ub[a] = p.inlet_u[j * D + a];
            } else {
#pragma unroll
                for (int a = 0; a < D; ++a) ub[a] = u[a];
            }
            Real cu = cdot<L>(i, ub), ubb = Real(0);
#pragma unroll
            for (int a = 0; a < D; ++a) ubb += ub[a] * ub[a];
            pp.own[i][xe - off] =
                Store<S>::save(Real(L::w(i)) * (Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * ubb));
        }
    }
}

// The same rules for a cell on an x face only (off every y and z face): just
// the directions that cross its x face, known at compile time per side, so
// that a warp holding one such cell pays a few stores instead of the
// general per-direction face test.
template <class L, class Real, class S, int SIDE>
__device__ __forceinline__ void face_streaming_x(const StepParams<Real> &p, const PopLayout &lay,
                                                 const PopPtrs<S> &pp, int xe, const int *idx,
                                                 Real rho, const Real *u)
{
    constexpr int D = L::D, Q = L::Q;
    constexpr int f6 = SIDE < 0 ? 0 : 1;   // the low or high x face
    const int bc = p.bc[f6];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::c(i, 0) != SIDE) continue;   // leaves through this face
        const int off = lay.off<L>(i);
        const Real post = Store<S>::load(pp.own[i][xe]);
        if (bc == BC_WALL) {
            const Real cw = Real(L::c(i, 0)) * p.wall_u[f6][0] + Real(L::c(i, 1)) * p.wall_u[f6][1] +
                            Real(L::c(i, 2)) * p.wall_u[f6][2];
            pp.own[L::opp(i)][xe + off] = Store<S>::save(post - Real(6) * Real(L::w(i)) * rho * cw);
        } else if (bc == BC_PERIODIC) {
            int q[3] = {idx[0] + L::c(i, 0) - SIDE * p.n[0], idx[1] + L::c(i, 1), idx[2] + L::c(i, 2)};
            pp.own[i][lay.ext(q) - off] = Store<S>::save(post);
        }
    }
    if (bc == BC_WALL || bc == BC_PERIODIC) return;
    // inlet or outlet on this face: the directions entering through it
    Real ub[3] = {Real(0), Real(0), Real(0)};
    if (bc == BC_INLET) {
        const int j = (D == 2) ? idx[0] : idx[0] + p.n[0] * idx[1];
#pragma unroll
        for (int a = 0; a < D; ++a) ub[a] = p.inlet_u[j * D + a];
    } else {
#pragma unroll
        for (int a = 0; a < D; ++a) ub[a] = u[a];
    }
    Real ubb = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) ubb += ub[a] * ub[a];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::c(i, 0) != -SIDE) continue;
        const Real cu = cdot<L>(i, ub);
        pp.own[i][xe - lay.off<L>(i)] =
            Store<S>::save(Real(L::w(i)) * (Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * ubb));
    }
}

// Mass deviation and momentum of a cell, sum_i f_i and sum_i c_i f_i of
// its deviations, added in direction order.  The collision and the
// statistics of a state use this one function, so both add the same values
// in the same order.
template <class L, class Real>
__device__ __forceinline__ void cell_moments(const Real *f, Real &drho, Real *m)
{
    constexpr int D = L::D, Q = L::Q;
    drho = Real(0);
    m[0] = m[1] = m[2] = Real(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += f[i];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (L::c(i, a) == 1) m[a] += f[i];
            else if (L::c(i, a) == -1) m[a] -= f[i];
        }
    }
}

// Per-warp sums of the cell moments for the statistics of a state: each warp
// adds its lanes' values in the arithmetic type (butterfly) and lane 0
// stores the four totals in FP64.  Every lane of the warp calls it (mom:
// zeros for a lane without a cell); nothing waits on other warps.
template <class Real>
__device__ __forceinline__ void warp_gas_partials(const Real *mom, double *out)
{
    Real t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) t[k] = warp_total<Real>(mom[k]);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = (double)t[k];
    }
}

// The populations of cell idx as its collision pulls them: direction i from
// x - c_i of the last step's stored values.
template <class L, class Real, class S>
__device__ __forceinline__ void pull_cell(const PopLayout &lay, const PopPtrs<S> &pp, const int *idx,
                                          Real *f)
{
    const int xe = lay.ext(idx);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[i] = Store<S>::load(__ldg(pp.pull[i] + xe));
}

__device__ __forceinline__ long long grid_block_index()
{
    return blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
}

// index of this warp in the collision's grid (blocks in launch order, warps
// of a block in order)
__device__ __forceinline__ long long grid_warp_index()
{
    return grid_block_index() * (blockDim.x >> 5) + (threadIdx.x >> 5);
}

// Nothing to do once a cell's moments are known (the plain step).
struct NoMomentsHook {
    template <class Real> __device__ __forceinline__ void operator()(Real, const Real *) const {}
};

// The work of one cell (idx: its coordinates) from its pulled populations
// fin (pull_cell): deposition, collision, node outputs and streaming.
// Shared by the single-bed kernel and the batched kernel of the serving
// loop, so that a bed's arithmetic does not depend on how its cells are
// mapped to threads.  hook(drho, m) receives the moments of fin once the
// node outputs are written: by then every load of the cell has been issued
// and the momentum is no longer needed.
template <class L, class Real, class S, bool LES, bool FB, class Hook = NoMomentsHook>
__device__ __forceinline__ void collide_stream_cell(const StepParams<Real> &p, const PopLayout &lay,
                                                    const PopPtrs<S> &pp, const CellList &cells,
                                                    const Particles<Real> &parts,
                                                    const Fields<Real> &fld, const int *idx,
                                                    const Real *fin, const Hook &hook = Hook())
{
    constexpr int D = L::D, Q = L::Q;
    const int x = idx[0] + p.n[0] * (idx[1] + p.n[1] * idx[2]);
    const int xe = lay.ext(idx);
    Real f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = fin[i];

    // ---- deposition (Eq. 8) ----
    const int s0 = cells.begin(x), s1 = cells.begin(x + 1);
    const int n = s1 - s0;
    Real vs[3] = {Real(0), Real(0), Real(0)};
    for (int k = s0; k < s1; ++k) {
#pragma unroll
        for (int a = 0; a < D; ++a) vs[a] += parts.v[a][k];
    }
    if (n > 1) {
        const Real inv_n = rcp(Real(n));
#pragma unroll
        for (int a = 0; a < D; ++a) vs[a] *= inv_n;
    }
    const int nn = n < p.tab.ntab ? n : p.tab.ntab - 1;
    const auto t0 = p.tab.pk0[nn];   // og, gam, inv_div, beta_a
    const auto t1 = p.tab.pk1[nn];   // beta_b, beta_c, re_k, branch
    // an empty cell has og = 0 and v_s = 0, so the solid term below vanishes
    const Real og = t0.x;

    // ---- moments ----
    Real drho, m[3];
    cell_moments<L, Real>(f, drho, m);
    const Real rho = Real(1) + drho;

    // ---- Eq. 24 in closed form ----
    const Real half_og = Real(0.5) * og;
    const Real inv_denom = rcp(rho * (Real(1) - half_og));
    Real u[3] = {Real(0), Real(0), Real(0)};
    Real uu = Real(0), vv = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = (m[a] * (Real(1) - og) + half_og * rho * vs[a] + Real(0.5) * p.fb[a]) * inv_denom;
        uu += u[a] * u[a];
        vv += vs[a] * vs[a];
    }
    // feq_i - w_i = w_i [(rho - 1) + rho (3 cu + 9/2 cu^2 - 3/2 uu)], Eq. 4
    const Real eq0 = drho - Real(1.5) * rho * uu;
    const Real es0 = drho - Real(1.5) * rho * vv;


    // ---- node outputs (Eq. 5, 24, 25, 19) ----
    // Written before the collision so that m and the drag tables are dead
    // while the populations are relaxed and streamed.  The drag
    // interpolation reads u_act, beta and 1 - eps of each stencil node from
    // these arrays alone (no cell-list or table lookups).
    const Real inv_div = t0.z;
    Real slip2 = Real(0), ua[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        fld.fpg[a][x] = og * (rho * u[a] + rho * vs[a] - Real(2) * m[a]);
        ua[a] = u[a] * inv_div;
        const Real sl = ua[a] - vs[a];
        slip2 += sl * sl;
    }
    fld.rho[x] = rho;
    const Real solg = p.tab.sol_g[nn];
    const Real slip = sqrt_pos(slip2);
    Real beta;
    if (t1.w == Real(0)) {
        beta = t0.w + t1.x * slip;                                   // Ergun
    } else {
        const Real re = t1.z * slip;                                 // Eq. 22
        beta = (re < Real(1000)) ? t0.w * (Real(1) + Real(0.15) * re_pow(re))   // Eq. 19, 21
                                 : t1.y * slip;
    }
    if (D == 2) {
        fld.node4[x] = {ua[0], ua[1], solg, beta};
    } else {
        fld.node4[x] = {ua[0], ua[1], ua[2], beta};
        fld.solg[x] = solg;
    }
    hook(drho, static_cast<const Real *>(m));

    // ---- LES (Eq. 13-15) ----
    Real inv_tau_t = p.inv_tau, gam_t = t0.y, tau_t = p.tau;
    if (LES) {
        Real qab[6] = {Real(0), Real(0), Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Real cu = cdot<L>(i, u);
            const Real neq = f[i] - Real(L::w(i)) * (eq0 + rho * (Real(3) * cu + Real(4.5) * cu * cu));
            int k = 0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
#pragma unroll
                for (int b = a; b < D; ++b, ++k) {
                    const int cc = L::c(i, a) * L::c(i, b);
                    if (cc == 1) qab[k] += neq;
                    else if (cc == -1) qab[k] -= neq;
                }
            }
        }
        Real qs = Real(0);
        int k = 0;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b, ++k) qs += (a == b ? Real(1) : Real(2)) * qab[k] * qab[k];
        const Real qn = sqrt(Real(2) * qs);
        tau_t = Real(0.5) * (p.tau + sqrt(p.tau * p.tau + p.les_k * qn / rho));
        inv_tau_t = Real(1) / tau_t;
        const Real es = p.tab.eps_s[nn];
        gam_t = es * (tau_t - Real(0.5)) / ((Real(1) - es) + (tau_t - Real(0.5)));
    }
    const Real relax = inv_tau_t * (Real(1) - gam_t);
    const Real pref = Real(1) - Real(0.5) * inv_tau_t;
    Real uF = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) uF += u[a] * p.fb[a];

    // ---- collision (Eq. 7, 23); each post-collision value is stored in this
    // cell's own slot of the extended lattice (aligned, no face logic) ----
    {
        // rest population: cu = cv = 0
        const Real w = Real(L::w(0));
        Real post = f[0] - relax * (f[0] - w * eq0) + og * w * (es0 - eq0);
        if (FB) post -= pref * w * Real(3) * uF;
        pp.own[0][xe] = Store<S>::save(post);
    }
    const Real r3 = Real(3) * rho, r45 = Real(4.5) * rho;
#pragma unroll
    for (int k = 0; k < (Q - 1) / 2; ++k) {
        const int i = L::pair_first(k), io = L::opp(i);
        const Real w = Real(L::w(i));
        const Real cu = cdot<L>(i, u);
        const Real cv = cdot<L>(i, vs);
        const Real Eu = w * (eq0 + r45 * cu * cu), Au = w * r3 * cu;
        const Real Es = w * (es0 + r45 * cv * cv), As = w * r3 * cv;
        const Real feu_i = Eu + Au, feu_o = Eu - Au;      // feq_i(u), feq_-i(u), minus w
        const Real fi = f[i], fo = f[io];
        Real post_i = fi - relax * (fi - feu_i) + og * (fo - fi + (Es + As) - feu_o);
        Real post_o = fo - relax * (fo - feu_o) + og * (fi - fo + (Es - As) - feu_i);
        if (FB) {
            const Real cF = cdot<L>(i, p.fb);
            const Real even = pref * w * (Real(9) * cu * cF - Real(3) * uF);
            const Real odd = pref * w * Real(3) * cF;
            post_i += even + odd;
            post_o += even - odd;
        }
        pp.own[i][xe] = Store<S>::save(post_i);
        pp.own[io][xe] = Store<S>::save(post_o);
    }

    if (fld.ntot) {
        fld.ntot[x] = n;
        fld.tau_t[x] = tau_t;
        fld.eps_g[x] = p.tab.eps_g[nn];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            fld.vs[a][x] = vs[a];
            fld.u[a][x] = u[a];
        }
    }
    if (!(rho > Real(0)) || !(uu < Real(0.09))) atomicOr(p.health, HEALTH_DIVERGED);

    // ---- streaming across the faces of the lattice ----
    bool yz_face = false;
#pragma unroll
    for (int a = 1; a < D; ++a) yz_face = yz_face || idx[a] == 0 || idx[a] == p.n[a] - 1;
    const bool xlo = idx[0] == 0, xhi = idx[0] == p.n[0] - 1;
    if (yz_face || (xlo && xhi)) face_streaming<L, Real, S>(p, lay, pp, xe, idx, rho, u);
    else if (xlo) face_streaming_x<L, Real, S, -1>(p, lay, pp, xe, idx, rho, u);
    else if (xhi) face_streaming_x<L, Real, S, 1>(p, lay, pp, xe, idx, rho, u);
}

// The moments of one cell as a row of the per-warp sums (zeros for a lane
// without a cell).
template <class L, class Real, class S>
__device__ __forceinline__ void lane_moments(bool active, const PopLayout &lay, const PopPtrs<S> &pp,
                                             const int *idx, Real *mom)
{
    mom[0] = mom[1] = mom[2] = mom[3] = Real(0);
    if (active) {
        Real f[L::Q], m[3];
        pull_cell<L, Real, S>(lay, pp, idx, f);
        cell_moments<L, Real>(f, mom[0], m);
#pragma unroll
        for (int a = 0; a < 3; ++a) mom[1 + a] = m[a];
    }
}

// The per-warp moment sums of a monitored step, taken inside the collision
// once its moments are known (every lane of the warp has a cell).
template <class Real> struct WarpMomentsHook {
    double *partials;
    __device__ __forceinline__ void operator()(Real drho, const Real *m) const
    {
        const Real mom[4] = {drho, m[0], m[1], m[2]};
        warp_gas_partials<Real>(mom, partials + 4 * grid_warp_index());
    }
};

// STATS: also the per-warp moment sums of the state it reads (a monitored
// step; see p.gas_partials).  A warp whose lanes all have a cell adds them
// inside the collision, after the deposition's loads (cell list, particles,
// tables) have gone out with the populations; a warp at the end of a row
// with lanes past the lattice adds them first, from loads of its own.
template <class L, class Real, class S, bool LES, bool FB, bool STATS>
__global__ void __launch_bounds__(kCollideThreads, K2Occupancy<L, Real>::value)
k_collide_stream(StepParams<Real> p, PopLayout lay, PopPtrs<S> pp, CellList cells,
                 Particles<Real> parts, Fields<Real> fld)
{
    constexpr int Q = L::Q;
    // grid: x along blockIdx.x/threadIdx.x, y = blockIdx.y, z = blockIdx.z
    int idx[3];
    idx[0] = blockIdx.x * blockDim.x + threadIdx.x;
    idx[1] = blockIdx.y;
    idx[2] = blockIdx.z;
    const bool active = idx[0] < p.n[0];
    if (!STATS) {
        if (!active) return;
        Real f[Q];
        pull_cell<L, Real, S>(lay, pp, idx, f);
        collide_stream_cell<L, Real, S, LES, FB>(p, lay, pp, cells, parts, fld, idx, f);
        return;
    }
    Real f[Q];
    if (__all_sync(0xffffffffu, active)) {
        pull_cell<L, Real, S>(lay, pp, idx, f);
        collide_stream_cell<L, Real, S, LES, FB>(p, lay, pp, cells, parts, fld, idx, f,
                                                 WarpMomentsHook<Real>{p.gas_partials});
        return;
    }
    Real mom[4];
    lane_moments<L, Real, S>(active, lay, pp, idx, mom);
    warp_gas_partials<Real>(mom, p.gas_partials + 4 * grid_warp_index());
    if (!active) return;
    pull_cell<L, Real, S>(lay, pp, idx, f);
    collide_stream_cell<L, Real, S, LES, FB>(p, lay, pp, cells, parts, fld, idx, f);
}

// The cell moments of a state without a collision, with the collision's
// grid, loads and per-warp sums (the statistics of the last state of a run,
// and of any state on demand).
template <class L, class Real, class S>
__global__ void __launch_bounds__(256)
k_gas_moments(PopLayout lay, PopPtrs<S> pp, int n0, double *partials)
{
    int idx[3];
    idx[0] = blockIdx.x * blockDim.x + threadIdx.x;
    idx[1] = blockIdx.y;
    idx[2] = blockIdx.z;
    Real mom[4];
    lane_moments<L, Real, S>(idx[0] < n0, lay, pp, idx, mom);
    warp_gas_partials<Real>(mom, partials + 4 * grid_warp_index());
}

// the collision's launch shape: blocks along each lattice row, up to 128
// threads along x
static inline int collide_tx(int n0)
{
    return n0 >= kCollideThreads ? kCollideThreads : ((n0 + 31) / 32) * 32;
}

long long collide_warps(int dim, const int *n)
{
    const int tx = collide_tx(n[0]);
    return (long long)((n[0] + tx - 1) / tx) * n[1] * (dim == 3 ? n[2] : 1) * (tx / 32);
}

template <class L, class Real, class S>
void launch_gas_moments(const PopLayout &lay, const S *f, const int *n, double *partials,
                        cudaStream_t st)
{
    PopPtrs<S> pp{};
    for (int i = 0; i < L::Q; ++i) {
        pp.pull[i] = f + (long long)i * lay.nce - lay.off<L>(i);
        pp.own[i] = nullptr;
    }
    const int tx = collide_tx(n[0]);
    const dim3 grid((n[0] + tx - 1) / tx, n[1], L::D == 3 ? n[2] : 1);
    k_gas_moments<L, Real, S><<<grid, tx, 0, st>>>(lay, pp, n[0], partials);
}

template <class L, class Real, class S>
void launch_collide_stream(const StepParams<Real> &p, const PopLayout &lay, const S *fin, S *fout,
                           CellList cells, Particles<Real> parts, Fields<Real> fld, cudaStream_t st)
{
    PopPtrs<S> pp{};
    for (int i = 0; i < L::Q; ++i) {
        pp.pull[i] = fin + (long long)i * lay.nce - lay.off<L>(i);
        pp.own[i] = fout + (long long)i * lay.nce;
    }
    // blocks along each lattice row, up to kCollideThreads threads along x
    const int tx = collide_tx(p.n[0]);
    const dim3 grid((p.n[0] + tx - 1) / tx, p.n[1], L::D == 3 ? p.n[2] : 1);
    const bool les = p.les_k > Real(0), fb = p.has_fb != 0;
    if (p.gas_partials) {
        if (les && fb)
            k_collide_stream<L, Real, S, true, true, true><<<grid, tx, 0, st>>>(p, lay, pp, cells, parts, fld);
        else if (les)
            k_collide_stream<L, Real, S, true, false, true><<<grid, tx, 0, st>>>(p, lay, pp, cells, parts, fld);
        else if (fb)
            k_collide_stream<L, Real, S, false, true, true><<<grid, tx, 0, st>>>(p, lay, pp, cells, parts, fld);
        else
            k_collide_stream<L, Real, S, false, false, true><<<grid, tx, 0, st>>>(p, lay, pp, cells, parts, fld);
        return;
    }
    if (les && fb)
        k_collide_stream<L, Real, S, true, true, false><<<grid, tx, 0, st>>>(p, lay, pp, cells, parts, fld);
    else if (les)
        k_collide_stream<L, Real, S, true, false, false><<<grid, tx, 0, st>>>(p, lay, pp, cells, parts, fld);
    else if (fb)
        k_collide_stream<L, Real, S, false, true, false><<<grid, tx, 0, st>>>(p, lay, pp, cells, parts, fld);
    else
        k_collide_stream<L, Real, S, false, false, false><<<grid, tx, 0, st>>>(p, lay, pp, cells, parts, fld);
}

// ---------------------------------------------------------------------------
// Batched collide-stream of the serving loop: persistent blocks walk the
// work table of (bed, tile) entries; each entry is kBatchTile consecutive
// cells of one bed (rows follow each other, so narrow lattices fill the
// block).  Each cell runs collide_stream_cell with its bed's parameters and
// the instantiation of its bed's storage type and LES / body-force flags.
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ void batched_cell(const BatchBed &b, int a, const int *idx)
{
    PopPtrs<S> pp;
    const S *fin = static_cast<const S *>(b.f[a]);
    S *fout = const_cast<S *>(static_cast<const S *>(b.f[1 - a]));
#pragma unroll
    for (int i = 0; i < D2Q9::Q; ++i) {
        pp.pull[i] = fin + (long long)i * b.lay.nce - b.lay.off<D2Q9>(i);
        pp.own[i] = fout + (long long)i * b.lay.nce;
    }
    const CellList cells{b.cl_local[a], b.cl_base[a], b.cl_shift};
    const bool les = b.sp.les_k > 0.0f, fb = b.sp.has_fb != 0;
    float f[D2Q9::Q];
    pull_cell<D2Q9, float, S>(b.lay, pp, idx, f);
    if (les && fb)
        collide_stream_cell<D2Q9, float, S, true, true>(b.sp, b.lay, pp, cells, b.part[a], b.fld, idx, f);
    else if (les)
        collide_stream_cell<D2Q9, float, S, true, false>(b.sp, b.lay, pp, cells, b.part[a], b.fld, idx, f);
    else if (fb)
        collide_stream_cell<D2Q9, float, S, false, true>(b.sp, b.lay, pp, cells, b.part[a], b.fld, idx, f);
    else
        collide_stream_cell<D2Q9, float, S, false, false>(b.sp, b.lay, pp, cells, b.part[a], b.fld, idx, f);
}

// two blocks per SM: the three storage types and four flag combinations
// inlined in one kernel need up to 128 registers without spilling
constexpr int kBatchCsBlocksPerSm = 2;

__global__ void __launch_bounds__(kBatchTile, kBatchCsBlocksPerSm)
k_collide_stream_batched(const BatchBed *__restrict__ beds, const int2 *__restrict__ work,
                         const int *__restrict__ count, int step)
{
    const int nwork = *count;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int2 e = work[w];
        const BatchBed &b = beds[e.x];
        if (step >= b.nsteps) continue;
        const int c = e.y * kBatchTile + threadIdx.x;
        if (c >= b.ncell) continue;
        const int idx[3] = {c % b.sp.n[0], c / b.sp.n[0], 0};
        const int a = (b.parity0 + step) & 1;
        if (b.storage == ST_F16) batched_cell<__half>(b, a, idx);
        else if (b.storage == ST_BF16) batched_cell<__nv_bfloat16>(b, a, idx);
        else batched_cell<float>(b, a, idx);
    }
}

int resident_grid(const void *kern, int threads, int nwork)
{
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        nsm = 1;
        per_sm = 1;
    }
    const long long slots = (long long)std::max(per_sm, 1) * std::max(nsm, 1);
    return (int)std::max(1LL, std::min<long long>(slots, nwork));
}

void launch_collide_stream_batched(const BatchBed *beds, BatchWork work, int step, cudaStream_t st)
{
    static const int grid = resident_grid((const void *)k_collide_stream_batched, kBatchTile, 1 << 30);
    if (!work.count) return;
    k_collide_stream_batched<<<grid, kBatchTile, 0, st>>>(beds, work.cell_tiles, work.count, step);
}

// ---------------------------------------------------------------------------
// Equilibrium initialisation and population import/export (full values in
// FP64, cell-major per direction: index i * ncell + x).  The stored slot of
// population i of cell x is ext(x) - c_i (the value the next collision
// pulls).
// ---------------------------------------------------------------------------
template <class L, class Real, class S>
__global__ void __launch_bounds__(256) k_init_equilibrium(long long nce, Real u0x, Real u0y,
                                                          Real u0z, S *f)
{
    // a uniform state: every slot of direction i holds the same deviation,
    // evaluated once per block in FP64 (slow on this part) and then stored
    __shared__ S dev[L::Q];
    if (threadIdx.x < L::Q) {
        const int i = threadIdx.x;
        const double u[3] = {(double)u0x, (double)u0y, (double)u0z};
        double uu = 0.0, cu = 0.0;
        for (int a = 0; a < L::D; ++a) uu += u[a] * u[a];
        for (int a = 0; a < L::D; ++a) cu += (double)L::c(i, a) * u[a];
        dev[i] = Store<S>::save((Real)(L::w(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu)));
    }
    __syncthreads();
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nce;
         k += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) f[(long long)i * nce + k] = dev[i];
    }
}

template <class L, class Real, class S>
void launch_init_equilibrium(const PopLayout &lay, const Real *u0, S *f, cudaStream_t st)
{
    const long long blocks = std::min<long long>((lay.nce + 255) / 256, 152LL * 16);
    k_init_equilibrium<L, Real, S><<<(unsigned)blocks, 256, 0, st>>>(lay.nce, u0[0], u0[1], u0[2], f);
}

template <class L>
__device__ __forceinline__ long long pop_slot(const PopLayout &lay, int i, int x)
{
    int q[3];
    q[0] = x % lay.n[0];
    q[1] = (x / lay.n[0]) % lay.n[1];
    q[2] = x / (lay.n[0] * lay.n[1]);
    return (long long)i * lay.nce + lay.ext(q) - lay.off<L>(i);
}

template <class L, class Real, class S>
__global__ void k_export_populations(PopLayout lay, int ncell, const S *f, double *out)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)L::Q * ncell) return;
    const int i = (int)(k / ncell), x = (int)(k % ncell);
    out[k] = L::w(i) + (double)Store<S>::load(f[pop_slot<L>(lay, i, x)]);
}

template <class L, class Real, class S>
void launch_export_populations(const PopLayout &lay, int ncell, const S *f, double *out,
                               cudaStream_t st)
{
    const long long total = (long long)L::Q * ncell;
    k_export_populations<L, Real, S><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(lay, ncell, f,
                                                                                       out);
}

template <class L, class Real, class S>
__global__ void k_import_populations(PopLayout lay, int ncell, const double *in, S *f)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)L::Q * ncell) return;
    const int i = (int)(k / ncell), x = (int)(k % ncell);
    f[pop_slot<L>(lay, i, x)] = Store<S>::save((Real)(in[k] - L::w(i)));
}

template <class L, class Real, class S>
void launch_import_populations(const PopLayout &lay, int ncell, const double *in, S *f,
                               cudaStream_t st)
{
    const long long total = (long long)L::Q * ncell;
    k_import_populations<L, Real, S><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(lay, ncell, in,
                                                                                       f);
}

// ---------------------------------------------------------------------------
// Explicit instantiations: (lattice, arithmetic, storage).
// ---------------------------------------------------------------------------
#define LBDPS_INST_LBM(L, R, S)                                                                    \
    template void launch_collide_stream<L, R, S>(const StepParams<R> &, const PopLayout &,         \
                                                 const S *, S *, CellList, Particles<R>, Fields<R>, \
                                                 cudaStream_t);                                     \
    template void launch_init_equilibrium<L, R, S>(const PopLayout &, const R *, S *,               \
                                                   cudaStream_t);                                   \
    template void launch_gas_moments<L, R, S>(const PopLayout &, const S *, const int *, double *,  \
                                              cudaStream_t);                                       \
    template void launch_export_populations<L, R, S>(const PopLayout &, int, const S *, double *,   \
                                                     cudaStream_t);                                 \
    template void launch_import_populations<L, R, S>(const PopLayout &, int, const double *, S *,   \
                                                     cudaStream_t);

LBDPS_INST_LBM(D2Q9, double, double)
LBDPS_INST_LBM(D2Q9, float, float)
LBDPS_INST_LBM(D2Q9, float, __half)
LBDPS_INST_LBM(D2Q9, float, __nv_bfloat16)
LBDPS_INST_LBM(D3Q19, double, double)
LBDPS_INST_LBM(D3Q19, float, float)
LBDPS_INST_LBM(D3Q19, float, __half)
LBDPS_INST_LBM(D3Q19, float, __nv_bfloat16)

template void launch_build_tables<double>(int, double, double, double, double, double, int, int,
                                          double *, CountTables<double>, cudaStream_t);
template void launch_build_tables<float>(int, double, double, double, double, double, int, int,
                                         double *, CountTables<float>, cudaStream_t);

}  // namespace lbdpsk

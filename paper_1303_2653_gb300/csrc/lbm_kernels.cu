// Lattice kernels: fused deposition + modified-LBE collision + streaming
// (the paper's Fig. 4 steps 2-3), the FP64 per-count tables, and population
// import/export.
#include "lbdps_internal.cuh"

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
        double es, e2, eg, sg;
        if (dim == 2) {
            const double cap = pi / (2.0 * sqrt(3.0));
            es = fmin((double)n * pi * r * r, cap);                 // Eq. 10 with h = 1
            e2 = 1.0 - es;
            double s = 1.0 - e2;
            sg = sqrt(2.0) / sqrt(pi * sqrt(3.0)) * (s * sqrt(s));  // Eq. 11: eps_3d = 1 - sg
            eg = 1.0 - sg;
        } else {
            const double cap = pi / (3.0 * sqrt(2.0));
            es = fmin((double)n * vp, cap);
            e2 = 1.0 - es;
            sg = es;
            eg = 1.0 - es;
        }
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

// Blocks per SM requested from the register allocator: D2Q9 in FP32 fits in
// ~40 registers (6 blocks of 256 threads), D3Q19 and FP64 need more.
template <class L, class Real> struct K2Occupancy { static constexpr int value = 4; };
#ifndef LBDPS_K2_BLOCKS_D2Q9_F32
#define LBDPS_K2_BLOCKS_D2Q9_F32 6
#endif
#ifndef LBDPS_K2_BLOCKS_D3Q19_F32
#define LBDPS_K2_BLOCKS_D3Q19_F32 4
#endif
template <> struct K2Occupancy<D2Q9, float> { static constexpr int value = LBDPS_K2_BLOCKS_D2Q9_F32; };
template <> struct K2Occupancy<D3Q19, float> { static constexpr int value = LBDPS_K2_BLOCKS_D3Q19_F32; };
template <> struct K2Occupancy<D3Q19, double> { static constexpr int value = 2; };

// Store one post-collision population of direction I: to the neighbour, or
// reflected into this cell's opposite slot by a wall (half-way bounce-back
// with the moving-wall term -6 w_i rho c_i.u_w of the first wall crossed), or
// dropped through an inlet/outlet face.
template <class L, class Real, class S>
__device__ __forceinline__ void emit_population(int I, const StepParams<Real> &p, S *__restrict__ fout,
                                                size_t nc, int x, Real post, Real rho, bool on_face,
                                                int wall_mask, int open_mask, int offp0, int offm0,
                                                int offp1, int offm1, int offp2, int offm2)
{
    const int cx = L::c(I, 0), cy = L::c(I, 1), cz = L::c(I, 2);
    const int off = (cx == 1 ? offp0 : cx == -1 ? offm0 : 0) + (cy == 1 ? offp1 : cy == -1 ? offm1 : 0) +
                    (cz == 1 ? offp2 : cz == -1 ? offm2 : 0);
    if (!on_face) {
        fout[(size_t)I * nc + (x + off)] = Store<S>::save(post);
        return;
    }
    // faces crossed by this direction, as bits of the masks
    const int crossed = (cx == 1 ? 2 : cx == -1 ? 1 : 0) | (cy == 1 ? 8 : cy == -1 ? 4 : 0) |
                            (cz == 1 ? 32 : cz == -1 ? 16 : 0);
    const int walls = wall_mask & crossed;
    if (walls) {
        const int face = __ffs(walls) - 1;   // first (lowest-axis) wall crossed
        const Real cw = Real(cx) * p.wall_u[face][0] + Real(cy) * p.wall_u[face][1] +
                        Real(cz) * p.wall_u[face][2];
        fout[(size_t)L::opp(I) * nc + x] = Store<S>::save(post - Real(6) * Real(L::w(I)) * rho * cw);
    } else if (!(open_mask & crossed)) {
        fout[(size_t)I * nc + (x + off)] = Store<S>::save(post);
    }
}

template <class L, class Real, class S, bool LES, bool FB>
__global__ void __launch_bounds__(256, K2Occupancy<L, Real>::value)
k_collide_stream(StepParams<Real> p, const S *__restrict__ fin, S *__restrict__ fout,
                 CellList cells, Particles<Real> parts, Fields<Real> fld)
{
    constexpr int D = L::D, Q = L::Q;
    // grid: x along blockIdx.x/threadIdx.x, y = blockIdx.y, z = blockIdx.z
    int idx[3];
    idx[0] = blockIdx.x * blockDim.x + threadIdx.x;
    idx[1] = blockIdx.y;
    idx[2] = blockIdx.z;
    if (idx[0] >= p.n[0]) return;
    const int x = idx[0] + p.n[0] * (idx[1] + p.n[1] * idx[2]);
    const size_t nc = (size_t)p.ncell;

    Real f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = Store<S>::load(fin[(size_t)i * nc + x]);

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
    Real drho = Real(0), m[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += f[i];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (L::c(i, a) == 1) m[a] += f[i];
            else if (L::c(i, a) == -1) m[a] -= f[i];
        }
    }
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
    Real slip2 = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        fld.fpg[a][x] = og * (rho * u[a] + rho * vs[a] - Real(2) * m[a]);
        const Real ua = u[a] * inv_div;
        fld.uact[a][x] = ua;
        const Real sl = ua - vs[a];
        slip2 += sl * sl;
    }
    fld.rho[x] = rho;
    fld.solg[x] = p.tab.sol_g[nn];
    const Real slip = sqrt_pos(slip2);
    Real beta;
    if (t1.w == Real(0)) {
        beta = t0.w + t1.x * slip;                                   // Ergun
    } else {
        const Real re = t1.z * slip;                                 // Eq. 22
        beta = (re < Real(1000)) ? t0.w * (Real(1) + Real(0.15) * re_pow(re))   // Eq. 19, 21
                                 : t1.y * slip;
    }
    fld.beta[x] = beta;

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

    // ---- streaming geometry of this cell (Eq. 2, push) ----
    // offp/offm: linear offset to the +/- neighbour along each axis with
    // periodic wrap folded in; bit 2a (2a+1) of wall_mask / open_mask: the
    // low (high) face of this cell along axis a is a wall / an inlet-outlet.
    int offp0 = 1, offm0 = -1, offp1 = p.n[0], offm1 = -p.n[0];
    int offp2 = p.n[0] * p.n[1], offm2 = -p.n[0] * p.n[1];
    int wall_mask = 0, open_mask = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int st = a == 0 ? 1 : (a == 1 ? p.n[0] : p.n[0] * p.n[1]);
        int op = st, om = -st;
        if (idx[a] == p.n[a] - 1) {
            const int bc = p.bc[2 * a + 1];
            if (bc == BC_PERIODIC) op = -(p.n[a] - 1) * st;
            else if (bc == BC_WALL) wall_mask |= 1 << (2 * a + 1);
            else open_mask |= 1 << (2 * a + 1);
        }
        if (idx[a] == 0) {
            const int bc = p.bc[2 * a];
            if (bc == BC_PERIODIC) om = (p.n[a] - 1) * st;
            else if (bc == BC_WALL) wall_mask |= 1 << (2 * a);
            else open_mask |= 1 << (2 * a);
        }
        if (a == 0) { offp0 = op; offm0 = om; }
        else if (a == 1) { offp1 = op; offm1 = om; }
        else { offp2 = op; offm2 = om; }
    }
    const bool on_face = (wall_mask | open_mask) != 0;
#define LBDPS_EMIT(I, POST)                                                                        \
    emit_population<L, Real, S>((I), p, fout, nc, x, (POST), rho, on_face, wall_mask, open_mask,  \
                                      offp0, offm0, offp1, offm1, offp2, offm2)
    {
        // rest population: cu = cv = 0
        const Real w = Real(L::w(0));
        Real post = f[0] - relax * (f[0] - w * eq0) + og * w * (es0 - eq0);
        if (FB) post -= pref * w * Real(3) * uF;
        LBDPS_EMIT(0, post);
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
        LBDPS_EMIT(i, post_i);
        LBDPS_EMIT(io, post_o);
    }

#undef LBDPS_EMIT

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

    // ---- populations entering through an inlet or outlet face ----
    if (open_mask == 0) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int wall = -1, open = -1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int q = idx[a] - L::c(i, a);
            if (q < 0 || q >= p.n[a]) {
                const int face = 2 * a + (q < 0 ? 0 : 1);
                const int bc = p.bc[face];
                if (bc == BC_WALL) { if (wall < 0) wall = face; }
                else if (bc != BC_PERIODIC) { if (open < 0) open = face; }
            }
        }
        if (wall < 0 && open >= 0) {
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
            fout[(size_t)i * nc + x] =
                Store<S>::save(Real(L::w(i)) * (Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * ubb));
        }
    }
}

template <class L, class Real, class S>
void launch_collide_stream(const StepParams<Real> &p, const S *fin, S *fout, CellList cells,
                           Particles<Real> parts, Fields<Real> fld, cudaStream_t st)
{
    // one block row per lattice row; up to 256 threads along x
    const int tx = p.n[0] >= 256 ? 256 : ((p.n[0] + 31) / 32) * 32;
    const dim3 grid((p.n[0] + tx - 1) / tx, p.n[1], L::D == 3 ? p.n[2] : 1);
    const bool les = p.les_k > Real(0), fb = p.has_fb != 0;
    if (les && fb)
        k_collide_stream<L, Real, S, true, true><<<grid, tx, 0, st>>>(p, fin, fout, cells, parts, fld);
    else if (les)
        k_collide_stream<L, Real, S, true, false><<<grid, tx, 0, st>>>(p, fin, fout, cells, parts, fld);
    else if (fb)
        k_collide_stream<L, Real, S, false, true><<<grid, tx, 0, st>>>(p, fin, fout, cells, parts, fld);
    else
        k_collide_stream<L, Real, S, false, false><<<grid, tx, 0, st>>>(p, fin, fout, cells, parts, fld);
}

// ---------------------------------------------------------------------------
// Equilibrium initialisation and population import/export (full values in FP64).
// ---------------------------------------------------------------------------
template <class L, class Real, class S>
__global__ void k_init_equilibrium(int ncell, Real u0x, Real u0y, Real u0z, S *f)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ncell) return;
    const double u[3] = {(double)u0x, (double)u0y, (double)u0z};
    double uu = 0.0;
    for (int a = 0; a < L::D; ++a) uu += u[a] * u[a];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        double cu = 0.0;
        for (int a = 0; a < L::D; ++a) cu += (double)L::c(i, a) * u[a];
        double dev = L::w(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        f[(size_t)i * ncell + x] = Store<S>::save((Real)dev);
    }
}

template <class L, class Real, class S>
void launch_init_equilibrium(int ncell, const Real *u0, S *f, cudaStream_t st)
{
    k_init_equilibrium<L, Real, S><<<(ncell + 255) / 256, 256, 0, st>>>(ncell, u0[0], u0[1], u0[2], f);
}

template <class L, class Real, class S>
__global__ void k_export_populations(int ncell, const S *f, double *out)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)L::Q * ncell) return;
    const int i = (int)(k / ncell);
    out[k] = L::w(i) + (double)Store<S>::load(f[k]);
}

template <class L, class Real, class S>
void launch_export_populations(int ncell, const S *f, double *out, cudaStream_t st)
{
    size_t total = (size_t)L::Q * ncell;
    k_export_populations<L, Real, S><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(ncell, f, out);
}

template <class L, class Real, class S>
__global__ void k_import_populations(int ncell, const double *in, S *f)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)L::Q * ncell) return;
    const int i = (int)(k / ncell);
    f[k] = Store<S>::save((Real)(in[k] - L::w(i)));
}

template <class L, class Real, class S>
void launch_import_populations(int ncell, const double *in, S *f, cudaStream_t st)
{
    size_t total = (size_t)L::Q * ncell;
    k_import_populations<L, Real, S><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(ncell, in, f);
}

// ---------------------------------------------------------------------------
// Explicit instantiations: (lattice, arithmetic, storage).
// ---------------------------------------------------------------------------
#define LBDPS_INST_LBM(L, R, S)                                                                    \
    template void launch_collide_stream<L, R, S>(const StepParams<R> &, const S *, S *,            \
                                                 CellList, Particles<R>, Fields<R>, cudaStream_t);  \
    template void launch_init_equilibrium<L, R, S>(int, const R *, S *, cudaStream_t);             \
    template void launch_export_populations<L, R, S>(int, const S *, double *, cudaStream_t);      \
    template void launch_import_populations<L, R, S>(int, const double *, S *, cudaStream_t);

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

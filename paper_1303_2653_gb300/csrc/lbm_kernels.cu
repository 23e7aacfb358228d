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
                     const_cast<int *>(tab.branch)};
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

template <class L, class Real, class S>
__global__ void __launch_bounds__(256)
k_collide_stream(StepParams<Real> p, const S *__restrict__ fin, S *__restrict__ fout,
                 const int *__restrict__ cell_start, Particles<Real> parts, Fields<Real> fld)
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
    const int s0 = cell_start[x], s1 = cell_start[x + 1];
    const int n = s1 - s0;
    Real vs[3] = {Real(0), Real(0), Real(0)};
    for (int k = s0; k < s1; ++k) {
#pragma unroll
        for (int a = 0; a < D; ++a) vs[a] += parts.v[a][k];
    }
    if (n > 1) {
        const Real inv_n = Real(1) / Real(n);
#pragma unroll
        for (int a = 0; a < D; ++a) vs[a] *= inv_n;
    }
    const int nn = n < p.tab.ntab ? n : p.tab.ntab - 1;
    const Real og = p.tab.og[nn];

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
    const Real inv_denom = Real(1) / (rho * (Real(1) - half_og));
    Real u[3] = {Real(0), Real(0), Real(0)};
    Real uu = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = (m[a] * (Real(1) - og) + half_og * rho * vs[a] + Real(0.5) * p.fb[a]) * inv_denom;
        uu += u[a] * u[a];
    }

    // equilibrium deviations feq_i - w_i = w_i [(rho-1) + rho (3cu + 9/2 cu^2 - 3/2 uu)]
    Real feu[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        Real cu = cdot<L>(i, u);
        feu[i] = Real(L::w(i)) * (drho + rho * (Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * uu));
    }

    // ---- LES (Eq. 13-15) ----
    Real inv_tau_t = p.inv_tau, gam_t = p.tab.gam[nn], tau_t = p.tau;
    if (p.les_k > Real(0)) {
        Real qs = Real(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
#pragma unroll
            for (int b = a; b < D; ++b) {
                Real qab = Real(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int cc = L::c(i, a) * L::c(i, b);
                    if (cc == 1) qab += f[i] - feu[i];
                    else if (cc == -1) qab -= f[i] - feu[i];
                }
                qs += (a == b ? Real(1) : Real(2)) * qab * qab;
            }
        }
        const Real qn = sqrt(Real(2) * qs);
        tau_t = Real(0.5) * (p.tau + sqrt(p.tau * p.tau + p.les_k * qn / rho));
        inv_tau_t = Real(1) / tau_t;
        const Real es = p.tab.eps_s[nn];
        gam_t = es * (tau_t - Real(0.5)) / ((Real(1) - es) + (tau_t - Real(0.5)));
    }
    const Real relax = inv_tau_t * (Real(1) - gam_t);

    // ---- collision (Eq. 7, 23) ----
    Real fpost[Q];
    if (n > 0) {
        Real vv = Real(0);
#pragma unroll
        for (int a = 0; a < D; ++a) vv += vs[a] * vs[a];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int io = L::opp(i);
            Real cv = cdot<L>(i, vs);
            Real fes = Real(L::w(i)) * (drho + rho * (Real(3) * cv + Real(4.5) * cv * cv - Real(1.5) * vv));
            Real omega_s = f[io] - f[i] + fes - feu[io];
            fpost[i] = f[i] - relax * (f[i] - feu[i]) + og * omega_s;
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) fpost[i] = f[i] - relax * (f[i] - feu[i]);
    }
    if (p.has_fb) {
        // Guo source w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F_b (1 - 1/(2 tau_t))
        const Real pref = Real(1) - Real(0.5) * inv_tau_t;
        Real uF = Real(0);
#pragma unroll
        for (int a = 0; a < D; ++a) uF += u[a] * p.fb[a];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Real cu = cdot<L>(i, u);
            const Real cF = cdot<L>(i, p.fb);
            const Real src = Real(3) * (cF - uF) + Real(9) * cu * cF;
            fpost[i] += pref * Real(L::w(i)) * src;
        }
    }

    // ---- node outputs (Eq. 5, 24, 25, 19) ----
    const Real inv_div = p.tab.inv_div[nn];
    Real slip2 = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        fld.u[a][x] = u[a];
        fld.fpg[a][x] = og * (rho * u[a] + rho * vs[a] - Real(2) * m[a]);
        Real sl = u[a] * inv_div - vs[a];
        slip2 += sl * sl;
    }
    fld.rho[x] = rho;
    const Real slip = sqrt(slip2);
    Real beta;
    if (p.tab.branch[nn] == 0) {
        beta = p.tab.beta_a[nn] + p.tab.beta_b[nn] * slip;
    } else {
        const Real re = p.tab.re_k[nn] * slip;
        beta = (re < Real(1000)) ? p.tab.beta_a[nn] * (Real(1) + Real(0.15) * re_pow(re))
                                 : p.tab.beta_c[nn] * slip;
    }
    fld.beta[x] = beta;
    if (fld.ntot) {
        fld.ntot[x] = n;
        fld.tau_t[x] = tau_t;
        fld.eps_g[x] = p.tab.eps_g[nn];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            fld.vs[a][x] = vs[a];
            fld.uact[a][x] = u[a] * inv_div;
        }
    }
    if (!(rho > Real(0)) || !(uu < Real(0.09))) atomicOr(p.health, HEALTH_DIVERGED);

    // ---- streaming (Eq. 2, push) ----
    bool interior = true;
#pragma unroll
    for (int a = 0; a < D; ++a)
        if (idx[a] == 0 || idx[a] == p.n[a] - 1) interior = false;
    const int stride[3] = {1, p.n[0], p.n[0] * p.n[1]};
    if (interior) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int off = 0;
#pragma unroll
            for (int a = 0; a < D; ++a) off += L::c(i, a) * stride[a];
            fout[(size_t)i * nc + (x + off)] = Store<S>::save(fpost[i]);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int wall = -1, open = -1, tgt = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            int q = idx[a] + L::c(i, a);
            if (q < 0 || q >= p.n[a]) {
                const int face = 2 * a + (q < 0 ? 0 : 1);
                const int bc = p.bc[face];
                if (bc == BC_PERIODIC) q = (q + p.n[a]) % p.n[a];
                else if (bc == BC_WALL) { if (wall < 0) wall = face; }
                else { if (open < 0) open = face; }
            }
            tgt += q * stride[a];
        }
        if (wall >= 0) {
            Real cw = Real(0);
#pragma unroll
            for (int a = 0; a < D; ++a) cw += Real(L::c(i, a)) * p.wall_u[wall][a];
            fout[(size_t)L::opp(i) * nc + x] =
                Store<S>::save(fpost[i] - Real(6) * Real(L::w(i)) * rho * cw);
        } else if (open < 0) {
            fout[(size_t)i * nc + tgt] = Store<S>::save(fpost[i]);
        }
    }
    // populations entering through an inlet or outlet face
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int wall = -1, open = -1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            int q = idx[a] - L::c(i, a);
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
void launch_collide_stream(const StepParams<Real> &p, const S *fin, S *fout, const int *cell_start,
                           Particles<Real> parts, Fields<Real> fld, cudaStream_t st)
{
    // one block row per lattice row; up to 256 threads along x
    const int tx = p.n[0] >= 256 ? 256 : ((p.n[0] + 31) / 32) * 32;
    const dim3 grid((p.n[0] + tx - 1) / tx, p.n[1], L::D == 3 ? p.n[2] : 1);
    k_collide_stream<L, Real, S><<<grid, tx, 0, st>>>(p, fin, fout, cell_start, parts, fld);
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
                                                 const int *, Particles<R>, Fields<R>,             \
                                                 cudaStream_t);                                    \
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

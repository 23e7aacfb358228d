// Soft-sphere contact forces, the discrete-element alternative to the
// time-driven hard spheres that §2.2 names for dense beds (normal contact
// only).  Each pair closer than d and each face closer than r pushes with
//
//     F = max(0, k_n delta - eta v_n)      along the line of centres,
//
// delta the overlap and v_n the approach speed; eta is set at creation so that
// a contact without the max() would return the restitution e of Eq. 17-18.
// The forces come from the positions and velocities at the start of the step
// (after the previous sort) and enter Eq. 16 beside the drag and the pressure
// force, in the drag kernel.
//
// With friction (mu > 0) the contact point's tangential slip meets a viscous
// force capped at mu times the normal force (Coulomb), whose torque changes
// the particle spins; the spins after the step are written for the sort to
// carry, those of the start of the step are read.
//
// One thread per particle in sorted order, walking the cells within reach
// (as the hard-sphere detection does).  The separation of a pair is formed in
// the arithmetic type from the cell indices and in-cell offsets; only a pair
// whose squared distance lies within a thin band around d^2 (wider than the
// rounding of the offsets) takes the exact FP64 test on the positions that
// the oracle uses, so that every contact decision is the exact one.  FP64 is
// slow on this part, and in FP32 this keeps it off all but a few pairs.  The
// overlap is taken as (d^2 - |dx|^2) / (d + |dx|), free of cancellation.
#include "particle_common.cuh"

namespace lbdpsk {

// blocks of 256 threads per SM the register allocation is held to
template <int D, class Real, bool FRIC> struct ContactOccupancy { static constexpr int value = 2; };
template <> struct ContactOccupancy<2, float, false> { static constexpr int value = 6; };
template <> struct ContactOccupancy<2, float, true> { static constexpr int value = 5; };

// Tangential (friction) part of one contact seen from particle i: unit normal
// n towards i, lever arm l from i's centre to the contact point (at -l n),
// clipped normal force fn > 0, relative velocity of the contact point vc
// (i's minus the other body's, three components, z only used in 3D).  The
// slip v_t = vc - (vc.n) n meets -min(gamma_t |v_t|, mu fn) v_t / |v_t|,
// added to F; its torque (-l n) x F_t is added to T (T[0] holds the
// component normal to the plane in 2D).
template <int D, class Real>
__device__ __forceinline__ void friction(const StepParams<Real> &p, const Real *n, Real l, Real fn,
                                         const Real *vc, Real *F, Real *T)
{
    Real vcn = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) vcn += vc[a] * n[a];
    Real vt[3] = {Real(0), Real(0), Real(0)}, s2 = Real(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        vt[a] = vc[a] - vcn * n[a];
        s2 += vt[a] * vt[a];
    }
    if (!(s2 > Real(0))) return;
    const Real st = sqrt(s2);
    Real mag = p.gamma_t * st;
    const Real cap = p.mu_f * fn;
    if (mag > cap) mag = cap;
    const Real k = -mag / st;
    Real Ft[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        Ft[a] = k * vt[a];
        F[a] += Ft[a];
    }
    if (D == 2) {
        T[0] -= l * (n[0] * Ft[1] - n[1] * Ft[0]);
    } else {
        T[0] -= l * (n[1] * Ft[2] - n[2] * Ft[1]);
        T[1] -= l * (n[2] * Ft[0] - n[0] * Ft[2]);
        T[2] -= l * (n[0] * Ft[1] - n[1] * Ft[0]);
    }
}

// w x n for the spin w (one component normal to the plane in 2D) and an
// in-plane (2D) or 3D vector n
template <int D, class Real>
__device__ __forceinline__ void spin_cross(const Real *w, const Real *n, Real *out)
{
    if (D == 2) {
        out[0] = -w[0] * n[1];
        out[1] = w[0] * n[0];
        out[2] = Real(0);
    } else {
        out[0] = w[1] * n[2] - w[2] * n[1];
        out[1] = w[2] * n[0] - w[0] * n[2];
        out[2] = w[0] * n[1] - w[1] * n[0];
    }
}

// FRIC: soft spheres with friction (spins read from parts.w, the new spins
// written to p.spin_out)
template <int D, class Real, bool FRIC>
__global__ void __launch_bounds__(256, ContactOccupancy<D, Real, FRIC>::value)
k_contacts(StepParams<Real> p, Particles<Real> parts, CellList cells, Real *diag_fc, int np)
{
    constexpr int NW = D == 2 ? 1 : 3;   // spin components
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int idx[3];
    cell_coords(D, p.n, __ldg(parts.cell + i), idx);
    float oi[3] = {0.f, 0.f, 0.f};
    Real vi[3] = {Real(0), Real(0), Real(0)}, wi[3] = {Real(0), Real(0), Real(0)};
    bool per[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        per[a] = (a < D) && (p.bc[2 * a] == BC_PERIODIC);
        if (a < D) {
            oi[a] = (float)__ldg(parts.off[a] + i);
            vi[a] = __ldg(parts.v[a] + i);
        }
    }
    if (FRIC) {
#pragma unroll
        for (int c = 0; c < NW; ++c) wi[c] = __ldg(parts.w[c] + i);
    }
    const float cut = (float)p.d + 1e-4f;   // reach of the walk
    // squared distances beyond d2_hi cannot be contacts, those below d2_lo
    // are; the band between covers the rounding of the offsets (about 1e-7
    // in FP32 on a separation of at most 2)
    const Real band = sizeof(Real) == 4 ? Real(4e-6) : Real(1e-12);
    const Real dd = (Real)p.d2;
    const Real d2_lo = dd - band, d2_hi = dd + band;
    Real oR[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) oR[a] = __ldg(parts.off[a] + i);
    Real F[3] = {Real(0), Real(0), Real(0)}, T[3] = {Real(0), Real(0), Real(0)};

    auto pair = [&](int j, int rowbase, float sy, float sz) {
        if (j == i) return;
        const Real shift[3] = {(Real)x_shift(p, parts, idx, per[0], j, rowbase), (Real)sy, (Real)sz};
        Real dx[3] = {Real(0), Real(0), Real(0)};
        Real d2 = Real(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            dx[a] = oR[a] - __ldg(parts.off[a] + j) - shift[a];
            d2 += dx[a] * dx[a];
        }
        if (d2 > d2_hi) return;
        if (!(d2 < d2_lo)) {
            // near the contact distance: the exact test of the oracle
            double e2 = 0.0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const double t = sep_axis(__ldg(parts.P[a] + i), __ldg(parts.P[a] + j), per[a], p.len[a]);
                e2 = __dadd_rn(e2, __dmul_rn(t, t));
            }
            if (!(e2 < p.d2)) return;
            if (d2 >= dd) d2 = dd;   // the overlap is then below the rounding: zero
        }
        const Real dist = sqrt(d2);
        const Real delta = (dd - d2) / ((Real)p.d + dist);
        Real nrm[3] = {Real(0), Real(0), Real(0)}, vr[3] = {Real(0), Real(0), Real(0)};
        Real vn = Real(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            nrm[a] = dx[a] / dist;
            vr[a] = vi[a] - __ldg(parts.v[a] + j);
            vn += vr[a] * nrm[a];
        }
        const Real f = p.kn * delta - p.eta * vn;
        if (f > Real(0)) {
#pragma unroll
            for (int a = 0; a < D; ++a) F[a] += f * nrm[a];
            if (FRIC) {
                // contact point half way: vc = v_rel - l (w_i + w_j) x n
                const Real l = Real(0.5) * dist;
                Real ws[3] = {Real(0), Real(0), Real(0)}, wxn[3], vc[3];
#pragma unroll
                for (int c = 0; c < NW; ++c) ws[c] = wi[c] + __ldg(parts.w[c] + j);
                spin_cross<D, Real>(ws, nrm, wxn);
#pragma unroll
                for (int a = 0; a < 3; ++a) vc[a] = vr[a] - l * wxn[a];
                friction<D, Real>(p, nrm, l, f, vc, F, T);
            }
        }
    };
    visit_neighbours<D, Real>(p, cells, idx, per, oi, cut, pair);

    // faces: only the first and last cell of an axis can be within r < 1/2
    // of one; the open outlet of a circulating bed makes no contact.  The
    // contact point lies on the face, at the centre's distance from it.
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (per[a]) continue;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            if (side == 0 ? idx[a] != 0 : (idx[a] != p.n[a] - 1 || (p.recirculate && a == D - 1)))
                continue;
            const double Pa = __ldg(parts.P[a] + i);
            const double gap = side == 0 ? Pa : __dsub_rn(p.len[a], Pa);
            if (!(gap < p.r64)) continue;
            const Real sg = side == 0 ? Real(1) : Real(-1);   // normal into the bed
            const Real f = p.kn * (Real)__dsub_rn(p.r64, gap) - p.eta_w * (sg * vi[a]);
            if (!(f > Real(0))) continue;
            F[a] += sg * f;
            if (FRIC) {
                Real nrm[3] = {Real(0), Real(0), Real(0)}, wxn[3], vc[3];
                nrm[a] = sg;
                const Real l = (Real)gap;
                spin_cross<D, Real>(wi, nrm, wxn);
#pragma unroll
                for (int c = 0; c < 3; ++c) vc[c] = vi[c] - l * wxn[c];
                friction<D, Real>(p, nrm, l, f, vc, F, T);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) p.fc[a][i] = F[a];
    if (FRIC) {
        // I dw = T dt from the start-of-step state
#pragma unroll
        for (int c = 0; c < NW; ++c) p.spin_out[c][i] = wi[c] + T[c] * p.inv_inertia;
    }
    if (diag_fc) {
        const int id = parts.id[i];
#pragma unroll
        for (int a = 0; a < D; ++a) diag_fc[(size_t)a * np + id] = F[a];
    }
}

template <int D, class Real>
void launch_contacts(const StepParams<Real> &p, Particles<Real> parts, CellList cells,
                     Real *diag_fc, int np, cudaStream_t st)
{
    if (np == 0) return;
    if (p.spin_out[0]) {
        const int b = wave_block(k_contacts<D, Real, true>, np);
        k_contacts<D, Real, true><<<(np + b - 1) / b, b, 0, st>>>(p, parts, cells, diag_fc, np);
    } else {
        const int b = wave_block(k_contacts<D, Real, false>, np);
        k_contacts<D, Real, false><<<(np + b - 1) / b, b, 0, st>>>(p, parts, cells, diag_fc, np);
    }
}

#define LBDPS_INST_C(D, R)                                                                          \
    template void launch_contacts<D, R>(const StepParams<R> &, Particles<R>, CellList, R *, int,    \
                                        cudaStream_t);
LBDPS_INST_C(2, double)
LBDPS_INST_C(2, float)
LBDPS_INST_C(3, double)
LBDPS_INST_C(3, float)

}  // namespace lbdpsk

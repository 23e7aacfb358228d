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

template <int D, class Real> struct ContactOccupancy { static constexpr int value = 2; };
template <> struct ContactOccupancy<2, float> { static constexpr int value = 6; };
template <> struct ContactOccupancy<3, float> { static constexpr int value = 2; };

template <int D, class Real>
__global__ void __launch_bounds__(256, ContactOccupancy<D, Real>::value)
k_contacts(StepParams<Real> p, Particles<Real> parts, CellList cells, Real *diag_fc, int np)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int idx[3];
    cell_coords(D, p.n, __ldg(parts.cell + i), idx);
    float oi[3] = {0.f, 0.f, 0.f};
    Real vi[3] = {Real(0), Real(0), Real(0)};
    bool per[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        per[a] = (a < D) && (p.bc[2 * a] == BC_PERIODIC);
        if (a < D) {
            oi[a] = (float)__ldg(parts.off[a] + i);
            vi[a] = __ldg(parts.v[a] + i);
        }
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
    Real F[3] = {Real(0), Real(0), Real(0)};

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
        Real vn = Real(0);
#pragma unroll
        for (int a = 0; a < D; ++a) vn += (vi[a] - __ldg(parts.v[a] + j)) * dx[a];
        vn /= dist;
        const Real f = p.kn * delta - p.eta * vn;
        if (f > Real(0)) {
            const Real s = f / dist;
#pragma unroll
            for (int a = 0; a < D; ++a) F[a] += s * dx[a];
        }
    };
    visit_neighbours<D, Real>(p, cells, idx, per, oi, cut, pair);

    // faces: only the first and last cell of an axis can be within r < 1/2
    // of one; the open outlet of a circulating bed makes no contact
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (per[a]) continue;
        if (idx[a] == 0) {
            const double Pa = __ldg(parts.P[a] + i);
            if (Pa < p.r64) {
                const Real f = p.kn * (Real)__dsub_rn(p.r64, Pa) - p.eta_w * vi[a];
                if (f > Real(0)) F[a] += f;
            }
        }
        if (idx[a] == p.n[a] - 1 && !(p.recirculate && a == D - 1)) {
            const double gap = __dsub_rn(p.len[a], __ldg(parts.P[a] + i));
            if (gap < p.r64) {
                const Real f = p.kn * (Real)__dsub_rn(p.r64, gap) + p.eta_w * vi[a];
                if (f > Real(0)) F[a] -= f;
            }
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) p.fc[a][i] = F[a];
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
    const int b = wave_block(k_contacts<D, Real>, np);
    k_contacts<D, Real><<<(np + b - 1) / b, b, 0, st>>>(p, parts, cells, diag_fc, np);
}

#define LBDPS_INST_C(D, R)                                                                          \
    template void launch_contacts<D, R>(const StepParams<R> &, Particles<R>, CellList, R *, int,    \
                                        cudaStream_t);
LBDPS_INST_C(2, double)
LBDPS_INST_C(2, float)
LBDPS_INST_C(3, double)
LBDPS_INST_C(3, float)

}  // namespace lbdpsk

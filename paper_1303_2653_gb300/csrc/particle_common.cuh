// Helpers shared by the particle kernels: block sizing, cell coordinates, the
// minimum-image separation and the walk over a particle's neighbourhood of
// cells in the cell list.
#pragma once

#include "lbdps_internal.cuh"

#include <climits>
#include <map>
#include <mutex>

namespace lbdpsk {

// Block size for a kernel with one thread per item: the candidate that covers
// n items in the fewest waves of co-resident blocks (the largest candidate on
// a tie).  A grid a little larger than one wave pays a whole second wave for
// its last blocks, which dominates short particle kernels.
template <class K>
int wave_block(K kern, long long n)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> fit;   // (kernel, block) -> blocks per SM
    static int nsm = 0;
    constexpr int cand[3] = {256, 128, 64};
    std::lock_guard<std::mutex> lock(mu);
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            nsm = 0;
            return 256;
        }
    }
    int best = 256;
    long long best_waves = LLONG_MAX;
    for (int b : cand) {
        const auto key = std::make_pair((const void *)kern, b);
        auto it = fit.find(key);
        if (it == fit.end()) {
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b, 0) != cudaSuccess) {
                cudaGetLastError();
                per_sm = 0;
            }
            it = fit.emplace(key, per_sm).first;
        }
        if (it->second <= 0) continue;
        const long long blocks = (n + b - 1) / b;
        const long long slots = (long long)it->second * nsm;
        const long long waves = (blocks + slots - 1) / slots;
        if (waves < best_waves) {
            best_waves = waves;
            best = b;
        }
    }
    return best;
}

__device__ __forceinline__ void cell_coords(int D, const int *n, int c, int *idx)
{
    idx[0] = c % n[0];
    idx[1] = (D == 3) ? (c / n[0]) % n[1] : c / n[0];
    idx[2] = (D == 3) ? c / (n[0] * n[1]) : 0;
}

// Minimum-image separation along one axis (periodic faces wrap), FP64 with
// explicit rounding so that no multiply-add is fused.
__device__ __forceinline__ double sep_axis(double pi, double pj, bool periodic, double L)
{
    double d = __dsub_rn(pi, pj);
    if (periodic) {
        if (d > 0.5 * L) d = __dsub_rn(d, L);
        else if (d < -0.5 * L) d = __dadd_rn(d, L);
    }
    return d;
}

// Calls visit(j, rowbase, sy, sz) for every sorted slot j in the cells that
// can hold a particle within cut of particle i (idx: its cell, oi: its
// in-cell offsets): along each axis the neighbouring cell below only when
// oi < cut and the one above only when oi > 1 - cut, since a particle there
// is at least that far away along the axis.  Each cell is visited once,
// periodic axes wrap, cells beyond a non-periodic face are skipped.  rowbase
// is the cell index of x = 0 in j's row, sy and sz the y and z cell offsets
// of j's row from idx.  cut must exceed the contact distance by more than
// the rounding of the FP32 offsets.
//
// The neighbourhood is visited one lattice row (along x) at a time: the cells
// of a row are consecutive in the cell list, so a row is one range of slots.
// The slot ranges of the rows of a plane are read together and walked as one
// loop, so that a warp iterates the maximum over its threads of the total
// rather than the sum of per-row maxima.  Where a periodic x face wraps, the
// cell across it is visited separately.
template <int D, class Real, class F>
__device__ __forceinline__ void visit_neighbours(const StepParams<Real> &p, const CellList &cells,
                                                 const int *idx, const bool *per, const float *oi,
                                                 float cut, F &&visit)
{
    const bool lo[3] = {oi[0] < cut, oi[1] < cut, D == 3 && oi[2] < cut};
    const bool hi[3] = {oi[0] > 1.f - cut, oi[1] > 1.f - cut, D == 3 && oi[2] > 1.f - cut};
    int x0 = lo[0] ? idx[0] - 1 : idx[0], x1 = hi[0] ? idx[0] + 1 : idx[0], xw = -1;
    if (x0 < 0) {
        x0 = 0;
        if (per[0]) xw = p.n[0] - 1;
    }
    if (x1 >= p.n[0]) {
        x1 = p.n[0] - 1;
        if (per[0]) xw = 0;
    }
    const int oz0 = lo[2] ? -1 : 0, oz1 = hi[2] ? 1 : 0;
#pragma unroll 1
    for (int oz = oz0; oz <= oz1; ++oz) {
        int qz = idx[2] + oz;
        if (D == 3 && (qz < 0 || qz >= p.n[2])) {
            if (!per[2]) continue;
            qz = qz < 0 ? qz + p.n[2] : qz - p.n[2];
        }
        int rb[3], j0[3], j1[3];
        unsigned rows_ok = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            int qy = idx[1] + r - 1;
            bool ok = (r == 1) || (r == 0 ? lo[1] : hi[1]);
            if (qy < 0 || qy >= p.n[1]) {
                ok = ok && per[1];
                qy = qy < 0 ? qy + p.n[1] : qy - p.n[1];
            }
            rows_ok |= ok ? 1u << r : 0u;
            rb[r] = p.n[0] * (qy + p.n[1] * qz);
            j0[r] = ok ? cells.begin(rb[r] + x0) : 0;
            j1[r] = ok ? cells.begin(rb[r] + x1 + 1) : 0;
        }
        const float sz = (float)oz;
        const int n0 = j1[0] - j0[0], n01 = n0 + (j1[1] - j0[1]);
        const int ntot = n01 + (j1[2] - j0[2]);
        for (int t = 0; t < ntot; ++t) {
            const int r = t < n0 ? 0 : (t < n01 ? 1 : 2);
            const int j = r == 0 ? j0[0] + t : (r == 1 ? j0[1] + (t - n0) : j0[2] + (t - n01));
            visit(j, r == 0 ? rb[0] : (r == 1 ? rb[1] : rb[2]), (float)(r - 1), sz);
        }
        if (xw >= 0) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                if (!((rows_ok >> r) & 1u)) continue;
                const int w0 = cells.begin(rb[r] + xw), w1 = cells.begin(rb[r] + xw + 1);
                for (int j = w0; j < w1; ++j) visit(j, rb[r], (float)(r - 1), sz);
            }
        }
    }
}

// x cell offset of slot j's cell from particle i's cell, unwrapped across a
// periodic x face: the visited cells lie within one cell of i's, so on a
// periodic axis (at least 3 cells) an offset beyond one is a wrap.  The y and
// z offsets come from the walk.
template <class Real>
__device__ __forceinline__ int x_shift(const StepParams<Real> &p, const Particles<Real> &parts,
                                       const int *idx, bool per_x, int j, int rowbase)
{
    int sx = __ldg(parts.cell + j) - rowbase - idx[0];
    if (per_x) {
        if (sx > 1) sx -= p.n[0];
        else if (sx < -1) sx += p.n[0];
    }
    return sx;
}

// Coarse contact test in FP32 from cell indices and in-cell offsets:
// P_i - P_j = (o_i - o_j) - (cell_j - cell_i) with the cell offsets already
// reduced to the minimum image, so that no intermediate is larger than 2.
// Returns |P_i - P_j|^2 in FP32; pairs beyond (d + 1e-4)^2 cannot be in
// contact (the margin is far above the FP32 rounding of offsets in [0, 1)).
template <int D, class Real>
__device__ __forceinline__ float coarse_d2(const StepParams<Real> &p, const Particles<Real> &parts,
                                           const int *idx, const float *oi, const bool *per,
                                           int j, int rowbase, float sy, float sz)
{
    const float shift[3] = {(float)x_shift(p, parts, idx, per[0], j, rowbase), sy, sz};
    float d2f = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float dx = oi[a] - (float)__ldg(parts.off[a] + j) - shift[a];
        d2f += dx * dx;
    }
    return d2f;
}

}  // namespace lbdpsk

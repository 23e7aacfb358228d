// Bed statistics in one launch: gas mass and momentum, particle momentum,
// lattice-mean voidage of the current positions, and (with diagnostics) the
// voidage and particle-weighted slip of the last collision.
//
// The gas mass and momentum come as per-warp FP64 sums of the cell moments
// (written by the collision of a monitored step, which reads exactly this
// state, or by k_gas_moments with the same grid and order); this kernel adds
// them in FP64.  The lattice sum of eps_g follows the occupied cells (the
// first particle of each, in sorted order, adds its cell's departure from
// the empty-cell value), so without diagnostics no per-cell array is read.
// The other values: each thread accumulates over a grid-stride range of
// particles, and of cells for the diagnostics (in FP64 in the FP64 engine; in
// FP32 with Kahan compensation otherwise, since FP64 arithmetic is slow on
// this part), each warp sums its lanes in the arithmetic type, each block
// adds its warp totals in FP64 in a fixed order, and the block that finishes
// last (ticket counter, nothing waits) adds the block partials in a fixed
// order.  The result does not depend on scheduling.
// `out` is mapped pinned host memory: the last block's stores are the only
// traffic to the host, so no copy has to follow the launch on the stream.
#include "lbdps_internal.cuh"

namespace lbdpsk {

constexpr int kRedThreads = 512;
constexpr int kRedMaxBlocks = kStatMaxBlocks;

template <class Real> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ void add(double x) { s += x; }
    __device__ double value() const { return s; }
};
// Kahan-compensated FP32 sum (Kahan 1965)
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ float value() const { return s - c; }
};

// Sum over a warp in a fixed order (butterfly of shuffles): every lane
// holds the total.
template <class T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out: [0] sum of deviations f_i - w_i, [1..3] sum c_i f_i, [4..6] m_p sum v,
// [7] sum of eps_g of the current counts, [8] sum of the diagnostic eps_g,
// [9] sum n |u_act - v_s|, [10] sum n (kStatValues = 11)

template <class L, class Real, bool BED>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_all(int ncell, const double *__restrict__ gas, long long ngas, Particles<Real> parts,
             double mp, int np, const Real *__restrict__ eps_tab, int ntab,
             Fields<Real> fld, double *partials, unsigned *ticket, const unsigned *health,
             const unsigned long long *solids_out, double *out, unsigned *health_live,
             int packed_limit)
{
    constexpr int D = L::D;
    Acc<Real> acc[kStatValues];
    double gacc[4] = {0.0, 0.0, 0.0, 0.0};   // gas mass deviation and momentum
    int packed = 0;   // a cell held more centres than can be there without overlaps
    const int stride = gridDim.x * blockDim.x;
    for (long long b = blockIdx.x * blockDim.x + threadIdx.x; b < ngas; b += stride) {
#pragma unroll
        for (int k = 0; k < 4; ++k) gacc[k] += __ldg(gas + 4 * b + k);
    }
    // particles (sorted by cell): momentum, and the lattice sum of eps_g of
    // the current counts.  Every cell adds eps_g(0) (added once, by the last
    // block) and an occupied cell the difference eps_g(n) - eps_g(0), found
    // at its first particle, which also flags an over-packed cell; first
    // particle and count come from the neighbouring entries of the cell
    // array, so no load waits on another.
    const Real e0 = eps_tab[0];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += stride) {
        const int c = parts.cell[k];
        const int cp = k > 0 ? parts.cell[k - 1] : -1;
        const int cn = k + 1 < np ? parts.cell[k + 1] : -1;
        Real v[3];
#pragma unroll
        for (int a = 0; a < D; ++a) v[a] = parts.v[a][k];
        if (cp != c) {
            int n = 1;
            if (cn == c)
                for (n = 2; k + n < np && parts.cell[k + n] == c; ++n) {}
            acc[7].add(eps_tab[n < ntab ? n : ntab - 1] - e0);
            if (n > packed_limit) packed = 1;
        }
#pragma unroll
        for (int a = 0; a < D; ++a) acc[4 + a].add(v[a]);
    }
    // diagnostics: the per-cell fields of the last collision
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; BED && x < ncell; x += stride) {
        acc[8].add(fld.eps_g[x]);
        const int nt = fld.ntot[x];
        if (nt > 0) {
            const auto r4 = fld.node4[x];
            const Real ua[3] = {r4.x, r4.y, D == 3 ? r4.z : Real(0)};
            Real s2 = Real(0);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const Real d = ua[a] - fld.vs[a][x];
                s2 += d * d;
            }
            acc[9].add(Real(nt) * sqrt(s2));
            acc[10].add(Real(nt));
        }
    }
    // block partials: warp sums in the arithmetic type, then the eight warp
    // totals of each value added in FP64 in warp order (one barrier)
    constexpr int kWarps = kRedThreads / 32;
    __shared__ double sh[kWarps][kStatValues];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kStatValues; ++k) {
        if (k < 4) {
            const double t = warp_sum<double>(gacc[k]);
            if (lane == 0) sh[warp][k] = t;
        } else {
            const Real t = warp_sum<Real>(acc[k].value());
            if (lane == 0) sh[warp][k] = (double)t;
        }
    }
    if (__syncthreads_or(packed) && threadIdx.x == 0) atomicOr(health_live, HEALTH_PACKED);
    if (threadIdx.x < kStatValues) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += sh[w][threadIdx.x];
        partials[blockIdx.x * kStatValues + threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block: warp w adds values w, w + 8, ...; its lane l adds the
    // partials of blocks l, l + 32, ... in that order (independent loads,
    // issued eight at a time), then the warp adds its lanes in a fixed order
    for (int k = warp; k < kStatValues; k += kWarps) {
        double u = 0.0;
#pragma unroll 8
        for (int b = lane; b < (int)gridDim.x; b += 32) u += __ldcg(partials + b * kStatValues + k);
        u = warp_sum<double>(u);
        if (lane == 0) out[k] = (k >= 4 && k < 7) ? mp * u : (k == 7 ? u + (double)ncell * (double)e0 : u);
    }
    if (threadIdx.x == 0) {
        // the health word and the outlet count travel with the values, so
        // that the host reads everything with one copy
        unsigned long long *raw = reinterpret_cast<unsigned long long *>(out);
        raw[kStatValues] = *health | (__ldcg(health_live) & HEALTH_PACKED);
        raw[kStatValues + 1] = *solids_out;
        *ticket = 0u;
    }
}

template <class L, class Real>
void launch_reduce_all(int ncell, const double *gas, long long ngas, Particles<Real> parts, double mp,
                       int np, const Real *eps_tab, int ntab,
                       const Fields<Real> *bed, double *partials, unsigned *ticket,
                       const unsigned *health, const unsigned long long *solids_out, double *out,
                       unsigned *health_live, int packed_limit, cudaStream_t st)
{
    // the cells are walked only for the diagnostics
    long long n = bed ? (ncell > np ? ncell : np) : np;
    n = n > ngas ? n : ngas;
    long long nb = (n + kRedThreads - 1) / kRedThreads;
    nb = nb < 1 ? 1 : (nb > kRedMaxBlocks ? kRedMaxBlocks : nb);
    if (bed)
        k_reduce_all<L, Real, true><<<(int)nb, kRedThreads, 0, st>>>(
            ncell, gas, ngas, parts, mp, np, eps_tab, ntab, *bed, partials, ticket, health,
            solids_out, out, health_live, packed_limit);
    else
        k_reduce_all<L, Real, false><<<(int)nb, kRedThreads, 0, st>>>(
            ncell, gas, ngas, parts, mp, np, eps_tab, ntab, Fields<Real>{}, partials, ticket,
            health, solids_out, out, health_live, packed_limit);
}

// The health word and the outlet count at the end of a step, for the
// reduction of that step's state, which runs after the next step.
__global__ void k_snapshot(const unsigned *health, const unsigned long long *solids_out,
                           unsigned long long *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        out[0] = *health;
        out[1] = *solids_out;
    }
}

void launch_snapshot(const unsigned *health, const unsigned long long *solids_out,
                     unsigned long long *out, cudaStream_t st)
{
    k_snapshot<<<1, 32, 0, st>>>(health, solids_out, out);
}

#define LBDPS_INST_RED(L, R)                                                                       \
    template void launch_reduce_all<L, R>(int, const double *, long long, Particles<R>, double,      \
                                          int, const R *, int, const Fields<R> *,                    \
                                          double *, unsigned *, const unsigned *,                    \
                                          const unsigned long long *, double *, unsigned *, int,     \
                                          cudaStream_t);
LBDPS_INST_RED(D2Q9, double)
LBDPS_INST_RED(D2Q9, float)
LBDPS_INST_RED(D3Q19, double)
LBDPS_INST_RED(D3Q19, float)

}  // namespace lbdpsk

// Bed statistics in one launch: gas mass and momentum, particle momentum,
// lattice-mean voidage of the current positions, and (with diagnostics) the
// voidage and particle-weighted slip of the last collision.
//
// Each thread accumulates over a grid-stride range of cells and particles (in
// FP64 in the FP64 engine; in FP32 with Kahan compensation otherwise, since
// FP64 arithmetic is slow on this part), each warp sums its lanes in the
// arithmetic type, each block adds its warp totals in FP64 in a fixed order,
// and the block that finishes last (ticket counter, nothing waits) adds the
// block partials in a fixed order.  The result does not depend on scheduling.
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

template <class L, class Real, class S, bool BED>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_all(PopLayout lay, int ncell, const S *__restrict__ f, Particles<Real> parts, double mp,
             int np, CellList cells, const Real *__restrict__ eps_tab, int ntab, Fields<Real> fld,
             double *partials, unsigned *ticket, const unsigned *health,
             const unsigned long long *solids_out, double *out, unsigned *health_live,
             int packed_limit)
{
    constexpr int D = L::D, Q = L::Q;
    Acc<Real> acc[kStatValues];
    int packed = 0;   // a cell held more centres than can be there without overlaps
    const int stride = gridDim.x * blockDim.x;
    // cells in batches of kB per thread (x, x + stride, ...): the loads of
    // a batch are all issued before any is used, so that each thread keeps
    // kB cells' worth of memory requests in flight
    constexpr int kB = Q <= 9 ? 2 : 1;
    for (int x0 = blockIdx.x * blockDim.x + threadIdx.x; x0 < ncell; x0 += kB * stride) {
        Real fv[kB][Q];
        int nn[kB];
#pragma unroll
        for (int b = 0; b < kB; ++b) {
            const int x = x0 + b * stride < ncell ? x0 + b * stride : x0;
            int q[3];
            q[0] = x % lay.n[0];
            q[1] = (x / lay.n[0]) % lay.n[1];
            q[2] = x / (lay.n[0] * lay.n[1]);
            const int xe = lay.ext(q);
#pragma unroll
            for (int i = 0; i < Q; ++i)   // population i as the next collision pulls it
                fv[b][i] = Store<S>::load(f[(long long)i * lay.nce + xe - lay.off<L>(i)]);
            nn[b] = cells.begin(x + 1) - cells.begin(x);
        }
        Real ev[kB];
#pragma unroll
        for (int b = 0; b < kB; ++b) {
            ev[b] = eps_tab[nn[b] < ntab ? nn[b] : ntab - 1];
            if (x0 + b * stride < ncell && nn[b] > packed_limit) packed = 1;
        }
#pragma unroll
        for (int b = 0; b < kB; ++b) {
            const int x = x0 + b * stride;
            if (x >= ncell) break;
            Real sm = Real(0), m[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                sm += fv[b][i];
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    if (L::c(i, a) == 1) m[a] += fv[b][i];
                    else if (L::c(i, a) == -1) m[a] -= fv[b][i];
                }
            }
            acc[0].add(sm);
#pragma unroll
            for (int a = 0; a < D; ++a) acc[1 + a].add(m[a]);
            acc[7].add(ev[b]);
            if (BED) {
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
        }
    }
    // particles in batches of two
    for (int k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < np; k0 += 2 * stride) {
        const int k1 = k0 + stride;
        Real v0[3], v1[3];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            v0[a] = parts.v[a][k0];
            v1[a] = k1 < np ? parts.v[a][k1] : Real(0);
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            acc[4 + a].add(v0[a]);
            if (k1 < np) acc[4 + a].add(v1[a]);
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
        const Real t = warp_sum<Real>(acc[k].value());
        if (lane == 0) sh[warp][k] = (double)t;
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
        if (lane == 0) out[k] = (k >= 4 && k < 7) ? mp * u : u;
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

template <class L, class Real, class S>
void launch_reduce_all(const PopLayout &lay, int ncell, const S *f, Particles<Real> parts, double mp,
                       int np, CellList cells, const Real *eps_tab, int ntab,
                       const Fields<Real> *bed, double *partials, unsigned *ticket,
                       const unsigned *health, const unsigned long long *solids_out, double *out,
                       unsigned *health_live, int packed_limit, cudaStream_t st)
{
    const int n = ncell > np ? ncell : np;
    int nb = (n + kRedThreads - 1) / kRedThreads;
    nb = nb < 1 ? 1 : (nb > kRedMaxBlocks ? kRedMaxBlocks : nb);
    if (bed)
        k_reduce_all<L, Real, S, true><<<nb, kRedThreads, 0, st>>>(
            lay, ncell, f, parts, mp, np, cells, eps_tab, ntab, *bed, partials, ticket, health,
            solids_out, out, health_live, packed_limit);
    else
        k_reduce_all<L, Real, S, false><<<nb, kRedThreads, 0, st>>>(
            lay, ncell, f, parts, mp, np, cells, eps_tab, ntab, Fields<Real>{}, partials, ticket,
            health, solids_out, out, health_live, packed_limit);
}

// The health word and the outlet count at the end of a step, for a
// reduction that runs beside the next step on another stream.
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

#define LBDPS_INST_RED(L, R, S)                                                                    \
    template void launch_reduce_all<L, R, S>(const PopLayout &, int, const S *, Particles<R>,       \
                                             double, int, CellList, const R *, int,                \
                                             const Fields<R> *, double *, unsigned *,               \
                                             const unsigned *, const unsigned long long *,          \
                                             double *, unsigned *, int, cudaStream_t);
LBDPS_INST_RED(D2Q9, double, double)
LBDPS_INST_RED(D2Q9, float, float)
LBDPS_INST_RED(D2Q9, float, __half)
LBDPS_INST_RED(D2Q9, float, __nv_bfloat16)
LBDPS_INST_RED(D3Q19, double, double)
LBDPS_INST_RED(D3Q19, float, float)
LBDPS_INST_RED(D3Q19, float, __half)
LBDPS_INST_RED(D3Q19, float, __nv_bfloat16)

}  // namespace lbdpsk

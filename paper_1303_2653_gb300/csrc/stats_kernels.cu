// Deterministic FP64 reductions of a bed: gas mass and momentum, particle
// momentum, lattice-mean voidage and particle-weighted slip.  A fixed grid
// with grid-stride loops, a fixed shared-memory tree per block, then one
// block summing the block partials in order: the result does not depend on
// scheduling.
#include "lbdps_internal.cuh"

namespace lbdpsk {

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 512;

int reduce_block_count(int n)
{
    int b = (n + kRedThreads * 4 - 1) / (kRedThreads * 4);
    return b < 1 ? 1 : (b > kRedMaxBlocks ? kRedMaxBlocks : b);
}

template <int NV>
__device__ void block_sum_write(double (&acc)[NV], double *partials)
{
    __shared__ double sh[kRedThreads];
    for (int k = 0; k < NV; ++k) {
        sh[threadIdx.x] = acc[k];
        __syncthreads();
        for (int s = kRedThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[blockIdx.x * NV + k] = sh[0];
        __syncthreads();
    }
}

__global__ void k_reduce_final(const double *partials, int nb, int nv, double *out)
{
    const int k = threadIdx.x;
    if (k >= nv) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partials[b * nv + k];
    out[k] = s;
}

// values: [0] sum of deviations f_i - w_i, [1..3] sum c_i f_i, [4..6] m_p sum v
template <class L, class Real, class S>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_state(PopLayout lay, int ncell, const S *f, Particles<Real> parts, double mp, int np,
               double *partials)
{
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const int stride = gridDim.x * blockDim.x;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < ncell; x += stride) {
        int q[3];
        q[0] = x % lay.n[0];
        q[1] = (x / lay.n[0]) % lay.n[1];
        q[2] = x / (lay.n[0] * lay.n[1]);
        const long long xe = lay.ext(q);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            // population i of cell x as the next collision pulls it
            const double fi =
                (double)Store<S>::load(f[(long long)i * lay.nce + xe - lay.off<L>(i)]);
            acc[0] += fi;
#pragma unroll
            for (int a = 0; a < L::D; ++a) acc[1 + a] += (double)L::c(i, a) * fi;
        }
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += stride) {
#pragma unroll
        for (int a = 0; a < L::D; ++a) acc[4 + a] += mp * (double)parts.v[a][k];
    }
    block_sum_write<7>(acc, partials);
}

template <class L, class Real, class S>
void launch_reduce_state(const PopLayout &lay, int ncell, const S *f, Particles<Real> parts,
                         double mp, int np, double *partials, double *out, cudaStream_t st)
{
    const int nb = reduce_block_count(ncell > np ? ncell : np);
    k_reduce_state<L, Real, S><<<nb, kRedThreads, 0, st>>>(lay, ncell, f, parts, mp, np, partials);
    k_reduce_final<<<1, 32, 0, st>>>(partials, nb, 7, out);
}

// values: [0] sum eps_g, [1] sum n |u_act - v_s|, [2] sum n
template <class Real>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_bed(int ncell, int dim, const Real *eps_g, const int *ntot, const Real *u0, const Real *u1,
             const Real *u2, const Real *v0, const Real *v1, const Real *v2, double *partials)
{
    double acc[3] = {0, 0, 0};
    const int stride = gridDim.x * blockDim.x;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < ncell; x += stride) {
        acc[0] += (double)eps_g[x];
        const int n = ntot[x];
        if (n > 0) {
            double s = 0.0, d;
            d = (double)u0[x] - (double)v0[x]; s += d * d;
            d = (double)u1[x] - (double)v1[x]; s += d * d;
            if (dim == 3) { d = (double)u2[x] - (double)v2[x]; s += d * d; }
            acc[1] += (double)n * sqrt(s);
            acc[2] += (double)n;
        }
    }
    block_sum_write<3>(acc, partials);
}

template <class Real>
void launch_reduce_bed(int ncell, int dim, const Real *eps_g, const int *ntot,
                       const Real *const *uact, const Real *const *vs, double *partials,
                       double *out, cudaStream_t st)
{
    const int nb = reduce_block_count(ncell);
    k_reduce_bed<Real><<<nb, kRedThreads, 0, st>>>(ncell, dim, eps_g, ntot, uact[0], uact[1],
                                                   dim == 3 ? uact[2] : uact[1], vs[0], vs[1],
                                                   dim == 3 ? vs[2] : vs[1], partials);
    k_reduce_final<<<1, 32, 0, st>>>(partials, nb, 3, out);
}

// lattice mean of eps_g for the current particle positions: [0] sum over cells
template <class Real>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_voidage(int ncell, CellList cells, const Real *eps_g_tab, int ntab, double *partials)
{
    double acc[1] = {0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < ncell; x += stride) {
        const int n = cells.begin(x + 1) - cells.begin(x);
        acc[0] += (double)eps_g_tab[n < ntab ? n : ntab - 1];
    }
    block_sum_write<1>(acc, partials);
}

template <class Real>
void launch_reduce_voidage(int ncell, CellList cells, const Real *eps_g_tab, int ntab,
                           double *partials, double *out, cudaStream_t st)
{
    const int nb = reduce_block_count(ncell);
    k_reduce_voidage<Real><<<nb, kRedThreads, 0, st>>>(ncell, cells, eps_g_tab, ntab, partials);
    k_reduce_final<<<1, 32, 0, st>>>(partials, nb, 1, out);
}
template void launch_reduce_voidage<double>(int, CellList, const double *, int, double *, double *,
                                            cudaStream_t);
template void launch_reduce_voidage<float>(int, CellList, const float *, int, double *, double *,
                                           cudaStream_t);

#define LBDPS_INST_RED(L, R, S)                                                                   \
    template void launch_reduce_state<L, R, S>(const PopLayout &, int, const S *, Particles<R>,    \
                                               double, int, double *, double *, cudaStream_t);
LBDPS_INST_RED(D2Q9, double, double)
LBDPS_INST_RED(D2Q9, float, float)
LBDPS_INST_RED(D2Q9, float, __half)
LBDPS_INST_RED(D2Q9, float, __nv_bfloat16)
LBDPS_INST_RED(D3Q19, double, double)
LBDPS_INST_RED(D3Q19, float, float)
LBDPS_INST_RED(D3Q19, float, __half)
LBDPS_INST_RED(D3Q19, float, __nv_bfloat16)
template void launch_reduce_bed<double>(int, int, const double *, const int *,
                                        const double *const *, const double *const *, double *,
                                        double *, cudaStream_t);
template void launch_reduce_bed<float>(int, int, const float *, const int *,
                                       const float *const *, const float *const *, double *,
                                       double *, cudaStream_t);

}  // namespace lbdpsk

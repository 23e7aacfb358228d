// Bubble regions of a bed (§3.1): connected regions of cells whose voidage
// (eps_2d of Eq. 10 or eps_g of Eq. 11, from the particle counts of the
// current cell list) exceeds a threshold, leaving out the regions that reach the top of
// the bed (the freeboard above the particles).  The equivalent bubble
// diameter of §3.1 is that of a circle with the area of such a region.
//
// Connected-component labelling by a lock-free union-find over the cells:
// every in-region cell starts as its own root; each cell joins its forward
// neighbours along every axis (wrapping across periodic faces) by linking the
// larger root under the smaller with atomicMin, so parent indices only
// decrease and no cycle can form; a final pass points every cell at its
// root.  All loops are bounded by the cell count; a bound that is reached
// sets an error flag instead of spinning on.
#include "lbdps_internal.cuh"

namespace lbdpsk {

// the largest count n whose voidage exceeds the threshold (the voidage
// decreases with n): eps_2d = 1 - eps_s (Eq. 10) for voidage = 0, eps_g
// (Eq. 11) for voidage = 1; -1 when even an empty cell is not above it
__global__ void k_bubble_count_limit(int dim, double r, double vp, int ntab, double threshold,
                                     int voidage, int *nlim)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int lim = -1;
    for (int n = 0; n < ntab; ++n) {
        double es, eg, sg;
        cell_voidage(dim, r, vp, n, &es, &eg, &sg);
        const double e = voidage == 0 ? 1.0 - es : eg;
        if (e > threshold) lim = n;
        else break;
    }
    *nlim = lim;
}

__global__ void k_bubble_init(int ncell, CellList cells, const int *__restrict__ nlim,
                              int *__restrict__ parent)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ncell) return;
    const int n = cells.begin(x + 1) - cells.begin(x);
    parent[x] = (n <= *nlim) ? x : -1;
}

__device__ __forceinline__ int bubble_find(volatile int *parent, int x, int bound, unsigned *err)
{
    for (int it = 0; it < bound; ++it) {
        const int p = parent[x];
        if (p == x) return x;
        x = p;
    }
    atomicOr(err, 1u);
    return x;
}

__device__ __forceinline__ void bubble_union(int *parent, int a, int b, int bound, unsigned *err)
{
    volatile int *vp = parent;
    for (int it = 0; it < bound; ++it) {
        a = bubble_find(vp, a, bound, err);
        b = bubble_find(vp, b, bound, err);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(parent + a, b);
        if (old == a) return;   // a was a root and now hangs under b
        a = old;                // a had been linked meanwhile: retry from there
    }
    atomicOr(err, 2u);
}

__global__ void k_bubble_union(int dim, int n0, int n1, int n2, int per_mask, int *parent,
                               unsigned *err)
{
    const int ncell = n0 * n1 * n2;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ncell || parent[x] < 0) return;
    const int q[3] = {x % n0, (x / n0) % n1, x / (n0 * n1)};
    const int n[3] = {n0, n1, n2};
    const int stride[3] = {1, n0, n0 * n1};
    for (int a = 0; a < dim; ++a) {
        int y;
        if (q[a] + 1 < n[a]) y = x + stride[a];
        else if ((per_mask >> a) & 1) y = x - (n[a] - 1) * stride[a];
        else continue;
        if (y != x && parent[y] >= 0) bubble_union(parent, x, y, ncell + 16, err);
    }
}

__global__ void k_bubble_sizes(int dim, int n0, int n1, int n2, int *parent, int *size, int *top,
                               unsigned *err)
{
    const int ncell = n0 * n1 * n2;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ncell || parent[x] < 0) return;
    const int root = bubble_find(parent, x, ncell + 16, err);
    atomicAdd(size + root, 1);
    const int vert = dim == 2 ? x / n0 : x / (n0 * n1);
    const int nv = dim == 2 ? n1 : n2;
    if (vert == nv - 1) top[root] = 1;
}

__global__ void k_bubble_reduce(int ncell, const int *parent, const int *size, const int *top,
                                unsigned long long *out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ncell || parent[x] != x || top[x]) return;
    atomicMax(out + 0, (unsigned long long)size[x]);
    atomicAdd(out + 1, 1ull);
    atomicAdd(out + 2, (unsigned long long)size[x]);
}

void launch_bubbles(int dim, const int *n, int per_mask, double r, double vp, int ntab,
                    double threshold, int voidage, CellList cells, BubbleScratch s,
                    cudaStream_t st)
{
    const int ncell = n[0] * n[1] * n[2];
    const int nb = (ncell + 255) / 256;
    cudaMemsetAsync(s.size, 0, sizeof(int) * ncell, st);
    cudaMemsetAsync(s.top, 0, sizeof(int) * ncell, st);
    cudaMemsetAsync(s.out, 0, sizeof(unsigned long long) * 3, st);
    cudaMemsetAsync(s.err, 0, sizeof(unsigned), st);
    k_bubble_count_limit<<<1, 32, 0, st>>>(dim, r, vp, ntab, threshold, voidage, s.nlim);
    k_bubble_init<<<nb, 256, 0, st>>>(ncell, cells, s.nlim, s.parent);
    k_bubble_union<<<nb, 256, 0, st>>>(dim, n[0], n[1], n[2], per_mask, s.parent, s.err);
    k_bubble_sizes<<<nb, 256, 0, st>>>(dim, n[0], n[1], n[2], s.parent, s.size, s.top, s.err);
    k_bubble_reduce<<<nb, 256, 0, st>>>(ncell, s.parent, s.size, s.top, s.out);
}

}  // namespace lbdpsk

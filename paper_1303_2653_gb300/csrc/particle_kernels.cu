// Particle kernels: interpolated EMMS drag with the Newton's-third-law rescale
// and the integration of Eq. 16 (Fig. 4 steps 4-5), the cell sort of
// Fig. 1, and the time-driven hard-sphere collisions (step 6, Eq. 17-18).
//
// FP64 is slow on this part, so per-particle FP64 work is limited to the
// position update and its floor; everything per pair or per stencil node uses
// the cell index and the in-cell offset carried with each particle, and the
// exact FP64 contact test runs only for pairs that an FP32 test with a safety
// margin cannot exclude.
#include "lbdps_internal.cuh"

#include <climits>

namespace lbdpsk {

__device__ __forceinline__ void cell_coords(int D, const int *n, int c, int *idx)
{
    idx[0] = c % n[0];
    idx[1] = (D == 3) ? (c / n[0]) % n[1] : c / n[0];
    idx[2] = (D == 3) ? c / (n[0] * n[1]) : 0;
}

// Cell of an FP64 position and the offset inside it (floor in FP64, clamped
// to the lattice; positions are kept inside [0, n) by the integrator).
template <class Real>
__device__ __forceinline__ int cell_and_offset(int D, const int *n, const double *P, Real *off)
{
    int q[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
        const double fl = floor(P[a]);
        int v = (int)fl;
        v = v < 0 ? 0 : (v >= n[a] ? n[a] - 1 : v);
        q[a] = v;
        off[a] = (Real)(P[a] - (double)v);
    }
    return q[0] + n[0] * (q[1] + n[1] * q[2]);
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

// ---------------------------------------------------------------------------
// K3a: pre-estimated drag of Eq. 26 per particle.  u, beta, eps and grad p
// are interpolated bilinearly (trilinearly in 3D) from the cell-centre nodes
// around the particle (Fig. 4 step 4); nodes outside a wall clamp to the
// nearest cell, periodic faces wrap.  grad p uses central differences of
// p = rho/3 (one-sided next to non-periodic faces).
// ---------------------------------------------------------------------------
template <int D, class Real>
__device__ __forceinline__ Real node_gradp(const StepParams<Real> &p, const Real *rho, const int *q,
                                           int a)
{
    if (p.n[a] == 1) return Real(0);
    const int stride = (a == 0) ? 1 : (a == 1) ? p.n[0] : p.n[0] * p.n[1];
    const int x = q[0] + p.n[0] * (q[1] + p.n[1] * q[2]);
    int lo = q[a] - 1, hi = q[a] + 1;
    Real scale = Real(1) / Real(6);        // (1/3) / 2: central difference of rho/3
    const bool per = (p.bc[2 * a] == BC_PERIODIC);
    if (lo < 0) { if (per) lo += p.n[a]; else { lo = q[a]; scale = Real(1) / Real(3); } }
    if (hi >= p.n[a]) { if (per) hi -= p.n[a]; else { hi = q[a]; scale = Real(1) / Real(3); } }
    const int xl = x + (lo - q[a]) * stride, xh = x + (hi - q[a]) * stride;
    return (rho[xh] - rho[xl]) * scale;
}

template <int D, class Real>
__global__ void __launch_bounds__(256)
k_drag_pre(StepParams<Real> p, Particles<Real> parts, const int *__restrict__ cell_start,
           Fields<Real> fld, Real *__restrict__ fpre, Real *__restrict__ gradp, int np)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    int idx[3];
    cell_coords(D, p.n, parts.cell[k], idx);
    int i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0};
    Real w1[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        // t = P - 1/2 = cell + off - 1/2; floor(t) and t - floor(t) from the offset
        const Real o = parts.off[a][k];
        int lo;
        if (o >= Real(0.5)) { lo = idx[a]; w1[a] = o - Real(0.5); }
        else { lo = idx[a] - 1; w1[a] = o + Real(0.5); }
        int hi = lo + 1;
        if (p.bc[2 * a] == BC_PERIODIC) {
            if (lo < 0) lo += p.n[a];
            if (hi >= p.n[a]) hi -= p.n[a];
        } else {
            lo = lo < 0 ? 0 : lo;
            hi = hi >= p.n[a] ? p.n[a] - 1 : hi;
        }
        i0[a] = lo;
        i1[a] = hi;
    }
    Real uk[3] = {Real(0), Real(0), Real(0)}, gk[3] = {Real(0), Real(0), Real(0)};
    Real sk = Real(0), bk = Real(0);     // interpolated 1 - eps and beta
#pragma unroll
    for (int corner = 0; corner < (1 << D); ++corner) {
        int q[3] = {0, 0, 0};
        Real wt = Real(1);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int bit = (corner >> a) & 1;
            q[a] = bit ? i1[a] : i0[a];
            wt *= bit ? w1[a] : (Real(1) - w1[a]);
        }
        const int node = q[0] + p.n[0] * (q[1] + p.n[1] * q[2]);
        const int cnt = cell_start[node + 1] - cell_start[node];
        const int nn = cnt < p.tab.ntab ? cnt : p.tab.ntab - 1;
        const Real inv_div = p.tab.inv_div[nn];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            uk[a] += wt * (fld.u[a][node] * inv_div);
            gk[a] += wt * node_gradp<D>(p, fld.rho, q, a);
        }
        sk += wt * p.tab.sol_g[nn];
        bk += wt * fld.beta[node];
    }
    const Real coef = p.vp * bk / sk;   // V_p beta_k / (1 - eps_k), Eq. 26
#pragma unroll
    for (int a = 0; a < D; ++a) {
        fpre[(size_t)a * np + k] = coef * (uk[a] - parts.v[a][k]);
        gradp[(size_t)a * np + k] = gk[a];
    }
}

template <int D, class Real>
void launch_drag_pre(const StepParams<Real> &p, Particles<Real> parts, const int *cell_start,
                     Fields<Real> fld, Real *fpre, Real *gradp, int np, cudaStream_t st)
{
    if (np == 0) return;
    k_drag_pre<D, Real><<<(np + 255) / 256, 256, 0, st>>>(p, parts, cell_start, fld, fpre, gradp, np);
}

// ---------------------------------------------------------------------------
// K3b: Eq. 27-28 and the step-5 integration of Eq. 16.
//   S^a(c) = sum of F_pre^a over the particles of cell c in sorted order
//   F_d^a  = |F_p->g^a(c)| / |S^a(c)| * F_pre^a   (scale 1 when |S| <= 1e-12 sum|F_pre|)
//   v     += (1 - rho_g/rho_s) g + (F_d -+ V_p grad p) / m_p
//   P     += v  (FP64), specular walls (v_n -> -e v_n), periodic wrap
// then the new cell key, the new in-cell offset and the key's count
// (histogram for the sort).
// ---------------------------------------------------------------------------
template <int D, class Real>
__global__ void __launch_bounds__(256)
k_drag_integrate(StepParams<Real> p, Particles<Real> parts, const int *__restrict__ cell_start,
                 Fields<Real> fld, const Real *__restrict__ fpre, const Real *__restrict__ gradp,
                 int *__restrict__ key, int *__restrict__ counts, Real *diag_fpre, Real *diag_fd,
                 int np)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int c = parts.cell[k];
    const int s0 = cell_start[c], s1 = cell_start[c + 1];
    Real S[3] = {Real(0), Real(0), Real(0)}, A[3] = {Real(0), Real(0), Real(0)};
    for (int j = s0; j < s1; ++j) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const Real fj = fpre[(size_t)a * np + j];
            S[a] += fj;
            A[a] += fabs(fj);
        }
    }
    const int id = parts.id[k];
    unsigned flags = 0;
    double P[3] = {0.0, 0.0, 0.0};
    Real v[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        P[a] = parts.P[a][k];
        v[a] = parts.v[a][k];
        Real scale = Real(1);
        if (!(fabs(S[a]) <= Real(1e-12) * A[a])) scale = fabs(fld.fpg[a][c]) / fabs(S[a]);
        const Real fp = fpre[(size_t)a * np + k];
        const Real fd = scale * fp;
        if (diag_fd) {
            diag_fd[(size_t)a * np + id] = fd;
            diag_fpre[(size_t)a * np + id] = fp;
        }
        const Real acc = p.geff[a] + (fd + p.psign * p.vp * gradp[(size_t)a * np + k]) / p.mp;
        v[a] += acc;
        P[a] += (double)v[a];
        const double L = p.len[a];
        if (p.bc[2 * a] == BC_PERIODIC) {
            if (P[a] >= L) P[a] -= L;
            else if (P[a] < 0.0) {
                P[a] += L;
                if (P[a] >= L) P[a] = 0.0;
            }
        } else {
            if (P[a] < 0.0) {
                P[a] = -P[a];
                v[a] = -p.e * v[a];
            } else if (P[a] >= L) {
                P[a] = 2.0 * L - P[a];
                v[a] = -p.e * v[a];
            }
            if (P[a] < 0.0) P[a] = 0.0;
            if (P[a] >= L) P[a] = p.len_below[a];
        }
        if (!(P[a] >= 0.0 && P[a] < L)) {   // NaN position: keep the state finite and report
            P[a] = 0.0;
            flags |= HEALTH_DOMAIN;
        }
    }
    if (flags) atomicOr(p.health, flags);
    Real off[3];
    const int nk = cell_and_offset<Real>(D, p.n, P, off);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        parts.P[a][k] = P[a];
        parts.v[a][k] = v[a];
        parts.off[a][k] = off[a];
    }
    key[k] = nk;
    atomicAdd(&counts[nk], 1);
}

template <int D, class Real>
void launch_drag_integrate(const StepParams<Real> &p, Particles<Real> parts, const int *cell_start,
                           Fields<Real> fld, const Real *fpre, const Real *gradp, int *key,
                           int *counts, Real *diag_fpre, Real *diag_fd, int np, cudaStream_t st)
{
    if (np == 0) return;
    k_drag_integrate<D, Real><<<(np + 255) / 256, 256, 0, st>>>(p, parts, cell_start, fld, fpre,
                                                                 gradp, key, counts, diag_fpre,
                                                                 diag_fd, np);
}

// Keys, offsets and counts of the current positions (used when a particle
// state is loaded).
template <int D, class Real>
__global__ void k_cell_keys(int n0, int n1, int n2, Particles<Real> parts, int *key, int *counts,
                            int np)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int n[3] = {n0, n1, n2};
    double P[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D; ++a) P[a] = parts.P[a][k];
    Real off[3];
    const int c = cell_and_offset<Real>(D, n, P, off);
    for (int a = 0; a < D; ++a) parts.off[a][k] = off[a];
    key[k] = c;
    atomicAdd(&counts[c], 1);
}

template <int D, class Real>
void launch_cell_keys(const int *n, Particles<Real> parts, int *key, int *counts, int np,
                      cudaStream_t st)
{
    if (np == 0) return;
    k_cell_keys<D, Real><<<(np + 255) / 256, 256, 0, st>>>(n[0], n[1], n[2], parts, key, counts, np);
}

// ---------------------------------------------------------------------------
// Exclusive scan of the per-cell counts into cell_start[0..ncell] in three
// passes: per-block scans (4096 cells per block) with block totals, a scan of
// the block totals in one block, and the addition of block offsets.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

int scan_block_count(int ncell) { return (ncell + kScanTile - 1) / kScanTile; }

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tot, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int wv = lane < nw ? warp_tot[lane] : 0;
        int wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) warp_tot[lane] = wi - wv;
        if (lane == nw - 1) *total = wi;
    }
    __syncthreads();
    return warp_tot[warp] + inc - v;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const int *__restrict__ counts, int *__restrict__ out, int *__restrict__ block_sums,
             int n)
{
    __shared__ int warp_tot[32];
    __shared__ int total;
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int vals[kScanItems];
    int sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int e = base + j;
        vals[j] = e < n ? counts[e] : 0;
        sum += vals[j];
    }
    int run = block_exclusive_scan(sum, warp_tot, &total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int e = base + j;
        if (e < n) out[e] = run;
        run += vals[j];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_block_sums(int *block_sums, int nb)
{
    __shared__ int warp_tot[32];
    __shared__ int total;
    int carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int e = base + threadIdx.x;
        const int v = e < nb ? block_sums[e] : 0;
        const int ex = block_exclusive_scan(v, warp_tot, &total);
        if (e < nb) block_sums[e] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[nb] = carry;
}

__global__ void k_scan_add(int *out, const int *block_sums, int n, int nb)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] += block_sums[e / kScanTile];
    if (e == n) out[n] = block_sums[nb];
}

void launch_scan(const int *counts, int *cell_start, int *block_sums, int ncell, cudaStream_t st)
{
    const int nb = scan_block_count(ncell);
    k_scan_tiles<<<nb, kScanThreads, 0, st>>>(counts, cell_start, block_sums, ncell);
    k_scan_block_sums<<<1, 1024, 0, st>>>(block_sums, nb);
    k_scan_add<<<(ncell + 1 + 255) / 256, 256, 0, st>>>(cell_start, block_sums, ncell, nb);
}

// ---------------------------------------------------------------------------
// Placement.  Each particle takes a slot in its cell's range by an atomic
// decrement of the cell count (which also returns the counts to zero for the
// next histogram).  The order inside a cell is then made canonical: each slot
// ranks its particle among the cell's members by id and the payload is
// gathered to cell_start + rank, giving the (cell, id) order.
// ---------------------------------------------------------------------------
__global__ void k_scatter(const int *__restrict__ key, int *__restrict__ counts,
                          const int *__restrict__ cell_start, int *__restrict__ tmp, int np)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int c = key[k];
    const int old = atomicSub(&counts[c], 1);
    tmp[cell_start[c] + old - 1] = k;
}

template <class Real>
__global__ void k_gather(int dim, const int *__restrict__ key, const int *__restrict__ cell_start,
                         const int *__restrict__ tmp, Particles<Real> src, Particles<Real> dst,
                         int np)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const int k = tmp[s];
    const int c = key[k];
    const int my = src.id[k];
    const int lo = cell_start[c], hi = cell_start[c + 1];
    int rank = 0;
    for (int q = lo; q < hi; ++q) rank += (src.id[tmp[q]] < my) ? 1 : 0;
    const int d = lo + rank;
    for (int a = 0; a < dim; ++a) {
        dst.P[a][d] = src.P[a][k];
        dst.v[a][d] = src.v[a][k];
        dst.off[a][d] = src.off[a][k];
    }
    dst.id[d] = my;
    dst.cell[d] = c;
}

template <class Real>
void launch_scatter_gather(int ncell, int dim, const int *key, int *counts, const int *cell_start,
                           int *tmp, Particles<Real> src, Particles<Real> dst, int np,
                           cudaStream_t st)
{
    (void)ncell;
    if (np == 0) return;
    k_scatter<<<(np + 255) / 256, 256, 0, st>>>(key, counts, cell_start, tmp, np);
    k_gather<Real><<<(np + 255) / 256, 256, 0, st>>>(dim, key, cell_start, tmp, src, dst, np);
}

// ---------------------------------------------------------------------------
// K4a: contact detection (section 2.2).  A pair collides when the centres are
// closer than d and (P_i - P_j).(v_i - v_j) < 0; both tests in FP64 with
// explicitly rounded multiplies and adds (no fused multiply-add) so that the
// decisions are reproducible.  A pair is first tested in FP32 from the cell
// indices and in-cell offsets; only pairs whose FP32 distance is within
// d + 1e-4 (far above the FP32 rounding of offsets in [0, 1)) reach the FP64
// test.  Each particle keeps its nearest approaching contact (ties to the
// smaller id) and its wall contacts (distance to the face below r while
// moving toward it).
// ---------------------------------------------------------------------------
template <int D, class Real>
__global__ void __launch_bounds__(256)
k_detect(StepParams<Real> p, Particles<Real> parts, const int *__restrict__ cell_start,
         int *__restrict__ best_out, int *__restrict__ wall_out, long long *pairs,
         unsigned long long *npairs, long long pair_cap, int np)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int idx[3];
    cell_coords(D, p.n, parts.cell[i], idx);
    float oi[3] = {0.f, 0.f, 0.f};
    bool per[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        per[a] = (a < D) && (p.bc[2 * a] == BC_PERIODIC);
        if (a < D) oi[a] = (float)parts.off[a][i];
    }
    const float cut = (float)p.d + 1e-4f;
    const float cut2 = cut * cut;
    const int idi = parts.id[i];

    int best = -1, best_id = INT_MAX;
    double best_d2 = __longlong_as_double(0x7ff0000000000000ll);
    double Pi[3] = {0.0, 0.0, 0.0}, vi[3] = {0.0, 0.0, 0.0};
    bool have_i = false;
    const int oz0 = (D == 3) ? -1 : 0, oz1 = (D == 3) ? 1 : 0;
    for (int oz = oz0; oz <= oz1; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
    for (int ox = -1; ox <= 1; ++ox) {
        const int off3[3] = {ox, oy, oz};
        int q[3];
        float shift[3];
        bool skip = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            q[a] = idx[a] + off3[a];
            shift[a] = (float)off3[a];
            if (a < D && (q[a] < 0 || q[a] >= p.n[a])) {
                if (per[a]) q[a] = (q[a] + p.n[a]) % p.n[a];
                else skip = true;
            }
        }
        if (skip) continue;
        const int cc = q[0] + p.n[0] * (q[1] + p.n[1] * q[2]);
        const int j0 = cell_start[cc], j1 = cell_start[cc + 1];
        for (int j = j0; j < j1; ++j) {
            if (j == i) continue;
            // coarse test: P_i - P_j = (o_i - o_j) - shift, minimum image on periodic axes
            float d2f = 0.f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                float dx = oi[a] - (float)parts.off[a][j] - shift[a];
                if (per[a]) {
                    const float L = (float)p.n[a];
                    if (dx > 0.5f * L) dx -= L;
                    else if (dx < -0.5f * L) dx += L;
                }
                d2f += dx * dx;
            }
            if (d2f > cut2) continue;
            // exact test in FP64, as written in section 2.2
            if (!have_i) {
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    Pi[a] = parts.P[a][i];
                    vi[a] = (double)parts.v[a][i];
                }
                have_i = true;
            }
            double dx[3] = {0.0, 0.0, 0.0};
            double d2 = 0.0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                dx[a] = sep_axis(Pi[a], parts.P[a][j], per[a], p.len[a]);
                d2 = __dadd_rn(d2, __dmul_rn(dx[a], dx[a]));
            }
            if (!(d2 < p.d2)) continue;
            double dot = 0.0;
#pragma unroll
            for (int a = 0; a < D; ++a)
                dot = __dadd_rn(dot, __dmul_rn(dx[a], __dsub_rn(vi[a], (double)parts.v[a][j])));
            if (!(dot < 0.0)) continue;
            const int idj = parts.id[j];
            if (pairs && idi < idj) {
                const unsigned long long slot = atomicAdd(npairs, 1ull);
                if ((long long)slot < pair_cap) {
                    pairs[2 * slot] = idi;
                    pairs[2 * slot + 1] = idj;
                }
            }
            if (d2 < best_d2 || (d2 == best_d2 && idj < best_id)) {
                best = j;
                best_id = idj;
                best_d2 = d2;
            }
        }
    }
    int bits = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (per[a]) continue;
        // only the first and last cell of an axis can touch a face (r < 1)
        if (idx[a] == 0) {
            const double Pa = parts.P[a][i];
            if (Pa < p.r64 && (double)parts.v[a][i] < 0.0) bits |= 1 << (2 * a);
        }
        if (idx[a] == p.n[a] - 1) {
            const double Pa = parts.P[a][i];
            if (__dsub_rn(p.len[a], Pa) < p.r64 && (double)parts.v[a][i] > 0.0)
                bits |= 1 << (2 * a + 1);
        }
    }
    best_out[i] = best;
    wall_out[i] = bits;
}

template <int D, class Real>
void launch_detect(const StepParams<Real> &p, Particles<Real> parts, const int *cell_start,
                   int *best, int *wall, long long *pairs, unsigned long long *npairs,
                   long long pair_cap, int np, cudaStream_t st)
{
    if (np == 0) return;
    k_detect<D, Real><<<(np + 255) / 256, 256, 0, st>>>(p, parts, cell_start, best, wall, pairs,
                                                        npairs, pair_cap, np);
}

// ---------------------------------------------------------------------------
// K4b: resolution.  A pair collides when each particle chose the other; the
// one with the smaller id applies Eq. 17-18 (equal masses) to both from the
// pre-collision velocities.  Particles without a mutual pair reflect off the
// walls they touch (Eq. 17 with an infinitely heavy wall at rest:
// v_n -> -e v_n).
// ---------------------------------------------------------------------------
template <int D, class Real>
__global__ void __launch_bounds__(256)
k_resolve(StepParams<Real> p, Particles<Real> parts, const int *__restrict__ best,
          const int *__restrict__ wall, int np)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int j = best[i];
    const bool mutual = (j >= 0) && (best[j] == i);
    if (mutual) {
        if (parts.id[i] > parts.id[j]) return;
        Real nv[3], g[3];
        Real gn = Real(0), nn = Real(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const bool per = (p.bc[2 * a] == BC_PERIODIC);
            nv[a] = (Real)sep_axis(parts.P[a][i], parts.P[a][j], per, p.len[a]);
            g[a] = parts.v[a][i] - parts.v[a][j];
            gn += g[a] * nv[a];
            nn += nv[a] * nv[a];
        }
        const Real kf = (Real(1) + p.e) * Real(0.5) * gn / nn;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const Real vi = parts.v[a][i], vj = parts.v[a][j];
            parts.v[a][i] = vi - kf * nv[a];
            parts.v[a][j] = vj + kf * nv[a];
        }
        return;
    }
    const int bits = wall[i];
    if (!bits) return;
#pragma unroll
    for (int a = 0; a < D; ++a)
        if (bits & (3 << (2 * a))) parts.v[a][i] = -p.e * parts.v[a][i];
}

template <int D, class Real>
void launch_resolve(const StepParams<Real> &p, Particles<Real> parts, const int *best,
                    const int *wall, int np, cudaStream_t st)
{
    if (np == 0) return;
    k_resolve<D, Real><<<(np + 255) / 256, 256, 0, st>>>(p, parts, best, wall, np);
}

// ---------------------------------------------------------------------------
#define LBDPS_INST_P(D, R)                                                                          \
    template void launch_drag_pre<D, R>(const StepParams<R> &, Particles<R>, const int *,         \
                                        Fields<R>, R *, R *, int, cudaStream_t);                   \
    template void launch_drag_integrate<D, R>(const StepParams<R> &, Particles<R>, const int *,   \
                                              Fields<R>, const R *, const R *, int *, int *, R *, \
                                              R *, int, cudaStream_t);                             \
    template void launch_detect<D, R>(const StepParams<R> &, Particles<R>, const int *, int *,     \
                                      int *, long long *, unsigned long long *, long long, int,    \
                                      cudaStream_t);                                               \
    template void launch_resolve<D, R>(const StepParams<R> &, Particles<R>, const int *,           \
                                       const int *, int, cudaStream_t);                            \
    template void launch_cell_keys<D, R>(const int *, Particles<R>, int *, int *, int,              \
                                         cudaStream_t);

LBDPS_INST_P(2, double)
LBDPS_INST_P(2, float)
LBDPS_INST_P(3, double)
LBDPS_INST_P(3, float)

template void launch_scatter_gather<double>(int, int, const int *, int *, const int *, int *,
                                            Particles<double>, Particles<double>, int,
                                            cudaStream_t);
template void launch_scatter_gather<float>(int, int, const int *, int *, const int *, int *,
                                           Particles<float>, Particles<float>, int, cudaStream_t);

}  // namespace lbdpsk

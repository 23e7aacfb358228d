// Particle kernels: interpolated EMMS drag with the Newton's-third-law rescale
// and the integration of Eq. 16 (Fig. 4 steps 4-5), the cell sort of
// Fig. 1, and the time-driven hard-sphere collisions (step 6, Eq. 17-18).
//
// FP64 is slow on this part, so per-particle FP64 work is limited to the
// position update (and its floor when the particle may leave its cell);
// everything per pair or per stencil node uses the cell index and the in-cell
// offset carried with each particle, and the exact FP64 contact test runs
// only for pairs that an FP32 test with a safety margin cannot exclude.
#include "particle_common.cuh"

#include <algorithm>

namespace lbdpsk {

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

// ---------------------------------------------------------------------------
// Pre-estimated drag of Eq. 26 for one particle.  u, beta, 1 - eps and grad p
// are interpolated bilinearly (trilinearly in 3D) from the cell-centre nodes
// around the particle (Fig. 4 step 4); nodes outside a wall clamp to the
// nearest cell, periodic faces wrap.  grad p uses central differences of
// p = rho/3 (one-sided next to non-periodic faces).  1 - eps is interpolated
// from the tabulated solid fraction so that it needs no cancellation.
// ---------------------------------------------------------------------------
template <int D, class Real>
__device__ __forceinline__ void drag_pre_one(const StepParams<Real> &p, const Particles<Real> &parts,
                                             const Fields<Real> &fld, const int *idx,
                                             const Real *ok, const Real *vk, Real *fp, Real *gp)
{
    int i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0};
    Real w1[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        // t = P - 1/2 = cell + off - 1/2; floor(t) and t - floor(t) from the offset
        const Real o = ok[a];
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
    constexpr int NC = 1 << D;
    int node[NC];
    Real wt[NC];
#pragma unroll
    for (int corner = 0; corner < NC; ++corner) {
        int q[3] = {0, 0, 0};
        Real w = Real(1);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int bit = (corner >> a) & 1;
            q[a] = bit ? i1[a] : i0[a];
            w *= bit ? w1[a] : (Real(1) - w1[a]);
        }
        wt[corner] = w;
        node[corner] = q[0] + p.n[0] * (q[1] + p.n[1] * q[2]);
        const auto r4 = fld.node4[node[corner]];   // u_act, 1 - eps, beta of the node
        uk[0] += w * r4.x;
        uk[1] += w * r4.y;
        if (D == 3) {
            uk[2] += w * r4.z;
            sk += w * __ldg(fld.solg + node[corner]);
        } else {
            sk += w * r4.z;
        }
        bk += w * r4.w;
    }
    // grad p at each node: central differences of rho/3 (one-sided next to a
    // non-periodic face).  Every neighbour is loaded, also where it is itself
    // a stencil node (an L1 hit): independent loads keep more gathers in
    // flight than selects between loaded and loading values (3D riser: 720
    // against 747 us per launch)
#pragma unroll
    for (int corner = 0; corner < NC; ++corner) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (p.n[a] == 1) continue;
            const int bit = (corner >> a) & 1;
            const int q = bit ? i1[a] : i0[a];
            const int stride = (a == 0) ? 1 : (a == 1) ? p.n[0] : p.n[0] * p.n[1];
            int lo = q - 1, hi = q + 1;
            Real scale = Real(1) / Real(6);    // (1/3) / 2: central difference of rho/3
            const bool per = (p.bc[2 * a] == BC_PERIODIC);
            if (lo < 0) { if (per) lo += p.n[a]; else { lo = q; scale = Real(1) / Real(3); } }
            if (hi >= p.n[a]) { if (per) hi -= p.n[a]; else { hi = q; scale = Real(1) / Real(3); } }
            const int x = node[corner];
            const Real rh = __ldg(fld.rho + x + (hi - q) * stride);
            const Real rl = __ldg(fld.rho + x + (lo - q) * stride);
            gk[a] += wt[corner] * ((rh - rl) * scale);
        }
    }
    const Real coef = p.vp * bk / sk;   // V_p beta_k / (1 - eps_k), Eq. 26
#pragma unroll
    for (int a = 0; a < D; ++a) {
        fp[a] = coef * (uk[a] - vk[a]);
        gp[a] = gk[a];
    }
}

// ---------------------------------------------------------------------------
// Drag and integration (Fig. 4 steps 4-5), one thread per particle.
//   F_pre of the thread's particle (Eq. 26);
//   S^a(c) = sum of F_pre^a over the particles of its cell in sorted order
//           (Eq. 27): members in the same block come from shared memory,
//           members in a neighbouring block are recomputed (bit-identical),
//           so every member of a cell adds the same values in the same order;
//   F_d^a  = |F_p->g^a(c)| / |S^a| F_pre^a (Eq. 28; scale 1 when
//           |S| <= 1e-12 sum |F_pre|);
//   v += (1 - rho_g/rho_s) g + (F_d -+ V_p grad p) / m_p, P += v in FP64
//   (Eq. 16, symplectic Euler), specular walls (v_n -> -e v_n), periodic
//   wrap, then the new cell key, in-cell offset and its count for the sort.
// A particle that stays well inside its cell (FP32 offset test with a 1e-3
// margin, far above the offset rounding) takes its new offset from one FP64
// subtraction; otherwise the full FP64 wall / wrap / floor path runs.  Both
// give bit-identical results.
// ---------------------------------------------------------------------------
// Register budgets of the drag and detection kernels, as blocks of 256
// threads per SM.  Detection fits 40 registers in 2D FP32 (6 blocks: 200,000
// particles in one wave, see wave_block); the drag spills below 48.
#ifndef LBDPS_DRAG_BLOCKS_2D_F32
#define LBDPS_DRAG_BLOCKS_2D_F32 5
#endif
#ifndef LBDPS_DRAG_BLOCKS_3D_F32
#define LBDPS_DRAG_BLOCKS_3D_F32 3
#endif
template <int D, class Real> struct DragOccupancy { static constexpr int value = 2; };
template <> struct DragOccupancy<2, float> { static constexpr int value = LBDPS_DRAG_BLOCKS_2D_F32; };
template <> struct DragOccupancy<3, float> { static constexpr int value = LBDPS_DRAG_BLOCKS_3D_F32; };
template <int D, class Real> struct DetectOccupancy { static constexpr int value = 2; };
template <> struct DetectOccupancy<2, float> { static constexpr int value = 6; };
template <> struct DetectOccupancy<3, float> { static constexpr int value = 5; };

// Members of cells that straddle a block boundary and lie in other blocks
// ("foreign" members) are taken into the Eq. 27 sums of this block's members.
// Up to kForeignPerThread of them, each member recomputes their pre-drags
// itself; beyond that the block computes each one once, in chunks of
// kForeignChunk in sorted order, into shared memory (crowded cells: a cell of
// n members spread over several blocks then costs O(n) pre-drags instead of
// O(n^2)).  Both give the same values in the same order.
constexpr int kForeignPerThread = 8;
constexpr int kForeignChunk = 256;

// Adds to S and A (Eq. 27) the pre-drags of the foreign members [lo, hi) of
// cell `cell`, computed once per block; `mine`: this thread's particle is a
// member of that cell.  Block-uniform (every thread calls it).
template <int D, class Real>
__device__ __forceinline__ void foreign_sums(const StepParams<Real> &p, const Particles<Real> &parts,
                                             const Fields<Real> &fld, int cell, int lo, int hi,
                                             bool mine, Real (*sfor)[kForeignChunk], Real *S, Real *A)
{
    int idx[3] = {0, 0, 0};
    cell_coords(D, p.n, cell, idx);
    for (int base = lo; base < hi; base += kForeignChunk) {
        const int cnt = min(kForeignChunk, hi - base);
        __syncthreads();   // the previous chunk has been read
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            Real val[3], g2[3], vj[3], oj[3];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                vj[a] = __ldg(parts.v[a] + base + t);
                oj[a] = __ldg(parts.off[a] + base + t);
            }
            drag_pre_one<D, Real>(p, parts, fld, idx, oj, vj, val, g2);
#pragma unroll
            for (int a = 0; a < D; ++a) sfor[a][t] = val[a];
        }
        __syncthreads();
        if (mine) {
            for (int t = 0; t < cnt; ++t) {
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    S[a] += sfor[a][t];
                    A[a] += fabs(sfor[a][t]);
                }
            }
        }
    }
}

// SOFT: add the soft-sphere contact force of the step (p.fc) in Eq. 16.
// The work of particle k in a thread block holding sorted slots
// [block_first, block_end) (at most 256, block_first < np), whose pre-drags
// it shares through sfp (sfor: room for foreign pre-drags); every thread of
// the block calls it (it synchronises the block).
template <int D, class Real, bool SOFT>
__device__ __forceinline__ void drag_step_particle(const StepParams<Real> &p,
                                                   const Particles<Real> &parts,
                                                   const Particles<Real> &out, const CellList &cells,
                                                   const Fields<Real> &fld, int *__restrict__ key,
                                                   int *__restrict__ counts, Real *diag_fpre,
                                                   Real *diag_fd, int np, int k, int block_first,
                                                   int block_end, Real (*sfp)[256],
                                                   Real (*sfor)[kForeignChunk])
{
    // the integrated state goes to `out` (same slots): other blocks may still
    // read this particle's pre-step state to complete their cell sums
    const bool active = k < np;
    int c = -1, s0 = 0, s1 = 0;
    int idx[3] = {0, 0, 0};
    Real fp[3] = {Real(0), Real(0), Real(0)}, gp[3] = {Real(0), Real(0), Real(0)};
    // the particle's own state is loaded before the first dependent load
    Real v0[3] = {Real(0), Real(0), Real(0)}, o0[3] = {Real(0), Real(0), Real(0)};
    Real fpg[3] = {Real(0), Real(0), Real(0)};
    double P[3] = {0.0, 0.0, 0.0};
    if (active) {
        c = __ldg(parts.cell + k);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            v0[a] = __ldg(parts.v[a] + k);
            o0[a] = __ldg(parts.off[a] + k);
            P[a] = __ldg(parts.P[a] + k);
        }
        s0 = cells.begin(c);
        s1 = cells.begin(c + 1);
#pragma unroll
        for (int a = 0; a < D; ++a) fpg[a] = __ldg(fld.fpg[a] + c);
        cell_coords(D, p.n, c, idx);
        drag_pre_one<D, Real>(p, parts, fld, idx, o0, v0, fp, gp);
#pragma unroll
        for (int a = 0; a < D; ++a) sfp[a][k - block_first] = fp[a];
    }
    // Eq. 27 in sorted order: members held by this block come from shared
    // memory, the others are recomputed (bit-identical).  The block shares
    // the foreign pre-drags when a member's cell has more than a few (only
    // the cells of the block's first and last particles can have any).
    const int last = min(block_end, np) - 1;   // the block's last particle
    const int own_foreign = active ? (s0 < block_first ? block_first - s0 : 0) +
                                         (s1 > last + 1 ? s1 - (last + 1) : 0)
                                   : 0;
    const bool shared_foreign = __syncthreads_or(own_foreign > kForeignPerThread) != 0;
    Real S[3] = {Real(0), Real(0), Real(0)}, A[3] = {Real(0), Real(0), Real(0)};
    if (shared_foreign) {
        const int ch = __ldg(parts.cell + block_first), ct = __ldg(parts.cell + last);
        const int h0 = cells.begin(ch), t1 = cells.begin(ct + 1);
        // head cell's foreign members (before the block), the block's own,
        // then the tail cell's (after it): the sorted order of every cell
        foreign_sums<D, Real>(p, parts, fld, ch, h0, block_first, active && c == ch, sfor, S, A);
        if (active) {
            const int lo = max(s0, block_first), hi = min(s1, last + 1);
            for (int j = lo; j < hi; ++j) {
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    S[a] += sfp[a][j - block_first];
                    A[a] += fabs(sfp[a][j - block_first]);
                }
            }
        }
        foreign_sums<D, Real>(p, parts, fld, ct, last + 1, t1, active && c == ct, sfor, S, A);
        if (!active) return;
    } else {
        if (!active) return;
        for (int j = s0; j < s1; ++j) {
            Real val[3];
            if (j >= block_first && j < block_end) {
#pragma unroll
                for (int a = 0; a < D; ++a) val[a] = sfp[a][j - block_first];
            } else {
                Real g2[3], vj[3], oj[3];
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    vj[a] = __ldg(parts.v[a] + j);
                    oj[a] = __ldg(parts.off[a] + j);
                }
                drag_pre_one<D, Real>(p, parts, fld, idx, oj, vj, val, g2);
            }
#pragma unroll
            for (int a = 0; a < D; ++a) {
                S[a] += val[a];
                A[a] += fabs(val[a]);
            }
        }
    }

    Real v[3] = {Real(0), Real(0), Real(0)}, off[3] = {Real(0), Real(0), Real(0)};
    int q[3] = {0, 0, 0};
    bool stays = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        Real scale = Real(1);
        if (!(fabs(S[a]) <= Real(1e-12) * A[a])) scale = fabs(fpg[a]) / fabs(S[a]);
        const Real fd = scale * fp[a];
        if (diag_fd) {
            const int id = parts.id[k];
            diag_fd[(size_t)a * np + id] = fd;
            diag_fpre[(size_t)a * np + id] = fp[a];
        }
        Real fa = fd + p.psign * p.vp * gp[a];
        if (SOFT) fa += p.fc[a][k];
        v[a] = v0[a] + (p.geff[a] + fa / p.mp);
        P[a] = P[a] + (double)v[a];
        const Real on = o0[a] + v[a];
        if (on > Real(1e-3) && on < Real(1) - Real(1e-3)) {
            q[a] = idx[a];
            off[a] = (Real)(P[a] - (double)idx[a]);
        } else {
            stays = false;
        }
    }
    if (!stays) {
        unsigned flags = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const double L = p.len[a];
            if (p.bc[2 * a] == BC_PERIODIC) {
                if (P[a] >= L) P[a] -= L;
                else if (P[a] < 0.0) {
                    P[a] += L;
                    if (P[a] >= L) P[a] = 0.0;
                }
            } else if (p.recirculate && a == D - 1 && P[a] >= L) {
                // through the outlet, back in at the inlet (solids loop)
                P[a] -= L;
                atomicAdd(p.solids_out, 1ull);
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
            if (!(P[a] >= 0.0 && P[a] < L)) {   // NaN position: keep it finite, report
                P[a] = 0.0;
                flags |= HEALTH_DOMAIN;
            }
            int vq = (int)floor(P[a]);
            vq = vq < 0 ? 0 : (vq >= p.n[a] ? p.n[a] - 1 : vq);
            q[a] = vq;
            off[a] = (Real)(P[a] - (double)vq);
        }
        if (flags) atomicOr(p.health, flags);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        out.P[a][k] = P[a];
        out.v[a][k] = v[a];
        out.off[a][k] = off[a];
    }
    const int nk = q[0] + p.n[0] * (q[1] + p.n[1] * q[2]);
    key[k] = nk;
    atomicAdd(&counts[nk], 1);
}

template <int D, class Real, bool SOFT>
__global__ void __launch_bounds__(256, DragOccupancy<D, Real>::value)
k_drag_step(StepParams<Real> p, Particles<Real> parts, Particles<Real> out, CellList cells,
            Fields<Real> fld, int *__restrict__ key, int *__restrict__ counts, Real *diag_fpre,
            Real *diag_fd, int np)
{
    __shared__ Real sfp[D][256];   // pre-drag of the block's particles (blockDim <= 256)
    __shared__ Real sfor[D][kForeignChunk];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int block_first = k - (int)threadIdx.x;
    drag_step_particle<D, Real, SOFT>(p, parts, out, cells, fld, key, counts, diag_fpre, diag_fd,
                                      np, k, block_first, block_first + (int)blockDim.x, sfp, sfor);
}

template <int D, class Real>
void launch_drag_step(const StepParams<Real> &p, Particles<Real> parts, Particles<Real> out,
                      CellList cells, Fields<Real> fld, int *key, int *counts, Real *diag_fpre,
                      Real *diag_fd, int np, cudaStream_t st)
{
    if (np == 0) return;
    if (p.fc[0]) {
        const int b = wave_block(k_drag_step<D, Real, true>, np);
        k_drag_step<D, Real, true><<<(np + b - 1) / b, b, 0, st>>>(p, parts, out, cells, fld, key,
                                                                   counts, diag_fpre, diag_fd, np);
    } else {
        const int b = wave_block(k_drag_step<D, Real, false>, np);
        k_drag_step<D, Real, false><<<(np + b - 1) / b, b, 0, st>>>(p, parts, out, cells, fld, key,
                                                                    counts, diag_fpre, diag_fd, np);
    }
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

// The particle state in id order for the host (interleaved, scaled to the
// caller's units), and back.
template <int D, class Real>
__global__ void k_particles_to_host_order(Particles<Real> parts, int np, double ps, double vs,
                                          double *pos, double *vel)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const size_t o = (size_t)parts.id[k] * D;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (pos) pos[o + a] = parts.P[a][k] * ps;
        if (vel) vel[o + a] = (double)parts.v[a][k] * vs;
    }
}

template <int D, class Real>
void launch_particles_to_host_order(Particles<Real> parts, int np, double ps, double vs,
                                    double *pos, double *vel, cudaStream_t st)
{
    if (np == 0) return;
    k_particles_to_host_order<D, Real><<<(np + 255) / 256, 256, 0, st>>>(parts, np, ps, vs, pos, vel);
}

template <int D, class Real>
__global__ void k_particles_from_host_order(const double *pos, const double *vel, int np,
                                            double pos_div, double vel_mul, Particles<Real> dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    constexpr int NW = D == 2 ? 1 : 3;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        // correctly rounded FP64 division and product, as on the host
        dst.P[a][i] = __ddiv_rn(pos[(size_t)i * D + a], pos_div);
        dst.v[a][i] = (Real)__dmul_rn(vel[(size_t)i * D + a], vel_mul);
    }
    dst.id[i] = i;
    if (dst.w[0])
#pragma unroll
        for (int c = 0; c < NW; ++c) dst.w[c][i] = Real(0);
}

template <int D, class Real>
void launch_particles_from_host_order(const double *pos, const double *vel, int np, double pos_div,
                                      double vel_mul, Particles<Real> dst, cudaStream_t st)
{
    if (np == 0) return;
    k_particles_from_host_order<D, Real><<<(np + 255) / 256, 256, 0, st>>>(pos, vel, np, pos_div,
                                                                           vel_mul, dst);
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan helper (warp shuffles, then the warp totals).
// ---------------------------------------------------------------------------
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

// ---------------------------------------------------------------------------
// One-launch scan of counts[0..ncell] into a two-level cell list.  Each block
// scans one tile of 4,096 (or 16,384) counts, ITEMS consecutive counts per
// thread in 16-byte loads and stores, and writes its total; the block that
// finishes last (ticket counter, nothing waits) scans the tile totals and
// resets the ticket for the next launch.
// ---------------------------------------------------------------------------
constexpr int kCellScanThreads = 1024;

// Tile `tile` of `nt` (one block of kCellScanThreads threads; every thread
// calls it); ITEMS = tile cells / kCellScanThreads.
template <int ITEMS>
__device__ __forceinline__ void cell_scan_tile(const int *__restrict__ counts, const CellListOut &out,
                                               int n, int tile, int nt, int *warp_tot, int &total,
                                               bool &last)
{
    constexpr int kCellScanItems = ITEMS;
    constexpr int kCellScanVec = ITEMS / 4;   // int4 loads per thread
    static_assert(ITEMS % 4 == 0, "whole int4 per thread");
    const int base = tile * (kCellScanThreads * ITEMS) + threadIdx.x * kCellScanItems;
    // all of the thread's loads are issued before any is used
    int4 c4[kCellScanVec];
    const bool whole = base + kCellScanItems <= n;
#pragma unroll
    for (int v = 0; v < kCellScanVec; ++v) {
        if (whole) {
            c4[v] = __ldg(reinterpret_cast<const int4 *>(counts + base) + v);
        } else {
            const int e = base + 4 * v;
            c4[v] = make_int4(e + 0 < n ? counts[e + 0] : 0, e + 1 < n ? counts[e + 1] : 0,
                              e + 2 < n ? counts[e + 2] : 0, e + 3 < n ? counts[e + 3] : 0);
        }
    }
    int sum = 0;
#pragma unroll
    for (int v = 0; v < kCellScanVec; ++v) sum += c4[v].x + c4[v].y + c4[v].z + c4[v].w;
    int run = block_exclusive_scan(sum, warp_tot, &total);
#pragma unroll
    for (int v = 0; v < kCellScanVec; ++v) {
        const int4 e4 = make_int4(run, run + c4[v].x, run + c4[v].x + c4[v].y,
                                  run + c4[v].x + c4[v].y + c4[v].z);
        run += c4[v].x + c4[v].y + c4[v].z + c4[v].w;
        if (whole) {
            reinterpret_cast<int4 *>(out.local + base)[v] = e4;
        } else {
            const int e = base + 4 * v;
            if (e + 0 < n) out.local[e + 0] = e4.x;
            if (e + 1 < n) out.local[e + 1] = e4.y;
            if (e + 2 < n) out.local[e + 2] = e4.z;
            if (e + 3 < n) out.local[e + 3] = e4.w;
        }
    }
    if (threadIdx.x == 0) {
        out.tile_total[tile] = total;
        __threadfence();
        const unsigned done = atomicAdd(out.ticket, 1u);
        last = (done == (unsigned)nt - 1u);
    }
    __syncthreads();
    if (!last) return;
    // the last block: exclusive scan of the tile totals into base[]
    __threadfence();
    int carry = 0;
    for (int b0 = 0; b0 < nt; b0 += blockDim.x) {
        const int e = b0 + threadIdx.x;
        const int v = e < nt ? __ldcg(out.tile_total + e) : 0;
        const int ex = block_exclusive_scan(v, warp_tot, &total);
        if (e < nt) out.base[e] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out.base[nt] = carry;
        *out.ticket = 0u;
    }
}

template <int ITEMS>
__global__ void __launch_bounds__(kCellScanThreads)
k_cell_scan(const int *__restrict__ counts, CellListOut out, int n)
{
    __shared__ int warp_tot[32];
    __shared__ int total;
    __shared__ bool last;
    cell_scan_tile<ITEMS>(counts, out, n, blockIdx.x, gridDim.x, warp_tot, total, last);
}

static_assert((kCellScanThreads << 2) == (1 << kCellTileLog2), "4 counts per thread in small tiles");
static_assert((kCellScanThreads << 4) == (1 << kCellTileLog2Large), "16 in large ones");

void launch_cell_scan(const int *counts, CellListOut out, int ncell, cudaStream_t st)
{
    const int n = ncell + 1;
    const int nt = cell_tiles(ncell);
    if (out.shift == kCellTileLog2Large)
        k_cell_scan<16><<<nt, kCellScanThreads, 0, st>>>(counts, out, n);
    else
        k_cell_scan<4><<<nt, kCellScanThreads, 0, st>>>(counts, out, n);
}

// ---------------------------------------------------------------------------
// Three-kernel scan into a plain cell_start array (per-block scans with block
// totals, a scan of the block totals in one block, the block offsets added).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

int scan_block_count(int ncell) { return (ncell + kScanTile - 1) / kScanTile; }

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
// next histogram) and records its id there.  The order inside a cell is then
// made canonical: each slot ranks its particle among the cell's members by id
// and the payload is gathered to begin(cell) + rank, the (cell, id) order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scatter_one(const int *__restrict__ key, const int *__restrict__ id,
                                            int *__restrict__ counts, const CellList &cells,
                                            int2 *__restrict__ slot, int *__restrict__ idslot, int k)
{
    const int c = key[k];
    const int old = atomicSub(&counts[c], 1);
    const int s = cells.begin(c) + old - 1;
    slot[s] = make_int2(k, c);
    idslot[s] = id[k];
}

__global__ void k_scatter(const int *__restrict__ key, const int *__restrict__ id,
                          int *__restrict__ counts, CellList cells, int2 *__restrict__ slot,
                          int *__restrict__ idslot, int np)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    scatter_one(key, id, counts, cells, slot, idslot, k);
}

// The payload of the particle in slot s is loaded before its rank is known
// (the loads do not wait on the rank loop), then stored at begin(c) + rank.
template <int D, class Real>
__device__ __forceinline__ void gather_one(const CellList &cells, const int2 *__restrict__ slot,
                                           const int *__restrict__ idslot, const Particles<Real> &src,
                                           const Particles<Real> &dst, int s)
{
    const int2 kc = slot[s];
    const int my = idslot[s];
    constexpr int NW = D == 2 ? 1 : 3;   // spin components
    const bool spin = src.w[0] != nullptr;
    double P[D];
    Real v[D], off[D], w[NW];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        P[a] = __ldg(src.P[a] + kc.x);
        v[a] = __ldg(src.v[a] + kc.x);
        off[a] = __ldg(src.off[a] + kc.x);
    }
    if (spin) {
#pragma unroll
        for (int c = 0; c < NW; ++c) w[c] = __ldg(src.w[c] + kc.x);
    }
    const int lo = cells.begin(kc.y), hi = cells.begin(kc.y + 1);
    int rank = 0;
    if (hi - lo > 1)
        for (int q = lo; q < hi; ++q) rank += (__ldg(idslot + q) < my) ? 1 : 0;
    const int d = lo + rank;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        dst.P[a][d] = P[a];
        dst.v[a][d] = v[a];
        dst.off[a][d] = off[a];
    }
    if (spin) {
#pragma unroll
        for (int c = 0; c < NW; ++c) dst.w[c][d] = w[c];
    }
    dst.id[d] = my;
    dst.cell[d] = kc.y;
}

template <int D, class Real>
__global__ void __launch_bounds__(256)
k_gather(CellList cells, const int2 *__restrict__ slot, const int *__restrict__ idslot,
         Particles<Real> src, Particles<Real> dst, int np)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    gather_one<D, Real>(cells, slot, idslot, src, dst, s);
}

template <class Real>
void launch_place(int dim, const int *key, int *counts, CellList cells, int2 *slot, int *idslot,
                  Particles<Real> src, Particles<Real> dst, int np, cudaStream_t st)
{
    if (np == 0) return;
    const int bs = wave_block(k_scatter, np);
    k_scatter<<<(np + bs - 1) / bs, bs, 0, st>>>(key, src.id, counts, cells, slot, idslot, np);
    if (dim == 2) {
        const int b = wave_block(k_gather<2, Real>, np);
        k_gather<2, Real><<<(np + b - 1) / b, b, 0, st>>>(cells, slot, idslot, src, dst, np);
    } else {
        const int b = wave_block(k_gather<3, Real>, np);
        k_gather<3, Real><<<(np + b - 1) / b, b, 0, st>>>(cells, slot, idslot, src, dst, np);
    }
}

// ---------------------------------------------------------------------------
// Contact detection (section 2.2).  A pair collides when the centres are
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
__device__ __forceinline__ void detect_one(const StepParams<Real> &p, const Particles<Real> &parts,
                                           const CellList &cells, int *__restrict__ best_out,
                                           int *__restrict__ wall_out, long long *pairs,
                                           unsigned long long *npairs, long long pair_cap, int i)
{
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
    // candidate j, whose cell lies in the row starting at cell index rowbase
    // and whose y (z) cell offset from particle i is sy (sz)
    auto test = [&](int j, int rowbase, float sy, float sz) {
        if (j == i) return;
        if (coarse_d2<D, Real>(p, parts, idx, oi, per, j, rowbase, sy, sz) > cut2) return;
        // exact test in FP64, as written in section 2.2
        double dx[3] = {0.0, 0.0, 0.0};
        double d2 = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            dx[a] = sep_axis(parts.P[a][i], parts.P[a][j], per[a], p.len[a]);
            d2 = __dadd_rn(d2, __dmul_rn(dx[a], dx[a]));
        }
        if (!(d2 < p.d2)) return;
        double dot = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a)
            dot = __dadd_rn(dot, __dmul_rn(dx[a], __dsub_rn((double)parts.v[a][i],
                                                             (double)parts.v[a][j])));
        if (!(dot < 0.0)) return;
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
    };
    visit_neighbours<D, Real>(p, cells, idx, per, oi, cut, test);
    int bits = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (per[a]) continue;
        // only the first and last cell of an axis can touch a face (r < 1)
        if (idx[a] == 0) {
            const double Pa = parts.P[a][i];
            if (Pa < p.r64 && (double)parts.v[a][i] < 0.0) bits |= 1 << (2 * a);
        }
        // with the solids loop closed the outlet lets particles through
        if (idx[a] == p.n[a] - 1 && !(p.recirculate && a == D - 1)) {
            const double Pa = parts.P[a][i];
            if (__dsub_rn(p.len[a], Pa) < p.r64 && (double)parts.v[a][i] > 0.0)
                bits |= 1 << (2 * a + 1);
        }
    }
    best_out[i] = best;
    wall_out[i] = bits;
}

template <int D, class Real>
__global__ void __launch_bounds__(256, DetectOccupancy<D, Real>::value)
k_detect(StepParams<Real> p, Particles<Real> parts, CellList cells, int *__restrict__ best_out,
         int *__restrict__ wall_out, long long *pairs, unsigned long long *npairs,
         long long pair_cap, int np)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    detect_one<D, Real>(p, parts, cells, best_out, wall_out, pairs, npairs, pair_cap, i);
}

template <int D, class Real>
void launch_detect(const StepParams<Real> &p, Particles<Real> parts, CellList cells, int *best,
                   int *wall, long long *pairs, unsigned long long *npairs, long long pair_cap,
                   int np, cudaStream_t st)
{
    if (np == 0) return;
    const int b = wave_block(k_detect<D, Real>, np);
    k_detect<D, Real><<<(np + b - 1) / b, b, 0, st>>>(p, parts, cells, best, wall, pairs, npairs,
                                                      pair_cap, np);
}

// ---------------------------------------------------------------------------
// Resolution.  A pair collides when each particle chose the other; the one
// with the smaller id applies Eq. 17-18 (equal masses) to both from the
// pre-collision velocities.  Particles without a mutual pair reflect off the
// walls they touch (Eq. 17 with an infinitely heavy wall at rest:
// v_n -> -e v_n).
// ---------------------------------------------------------------------------
template <int D, class Real>
__device__ __forceinline__ void resolve_one(const StepParams<Real> &p, const Particles<Real> &parts,
                                            const int *__restrict__ best,
                                            const int *__restrict__ wall, int i)
{
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
__global__ void __launch_bounds__(256)
k_resolve(StepParams<Real> p, Particles<Real> parts, const int *__restrict__ best,
          const int *__restrict__ wall, int np)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    resolve_one<D, Real>(p, parts, best, wall, i);
}

template <int D, class Real>
void launch_resolve(const StepParams<Real> &p, Particles<Real> parts, const int *best,
                    const int *wall, int np, cudaStream_t st)
{
    if (np == 0) return;
    const int b = wave_block(k_resolve<D, Real>, np);
    k_resolve<D, Real><<<(np + b - 1) / b, b, 0, st>>>(p, parts, best, wall, np);
}

// ---------------------------------------------------------------------------
// Creation check for hard spheres: pairs closer than d (the FP64 test of the
// detection, without the approach condition).  Counts them and keeps the
// smallest (id_i, id_j), i < j, as ((u64)id_i << 32) | id_j.
// ---------------------------------------------------------------------------
template <int D, class Real>
__global__ void __launch_bounds__(256)
k_overlaps(StepParams<Real> p, Particles<Real> parts, CellList cells,
           unsigned long long *count, unsigned long long *first, int np)
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
    auto test = [&](int j, int rowbase, float sy, float sz) {
        const int idj = parts.id[j];
        if (!(idi < idj)) return;
        if (coarse_d2<D, Real>(p, parts, idx, oi, per, j, rowbase, sy, sz) > cut2) return;
        double d2 = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const double dx = sep_axis(parts.P[a][i], parts.P[a][j], per[a], p.len[a]);
            d2 = __dadd_rn(d2, __dmul_rn(dx, dx));
        }
        if (!(d2 < p.d2)) return;
        atomicAdd(count, 1ull);
        atomicMin(first, ((unsigned long long)idi << 32) | (unsigned long long)idj);
    };
    visit_neighbours<D, Real>(p, cells, idx, per, oi, cut, test);
}

template <int D, class Real>
void launch_overlaps(const StepParams<Real> &p, Particles<Real> parts, CellList cells,
                     unsigned long long *count, unsigned long long *first, int np, cudaStream_t st)
{
    if (np == 0) return;
    k_overlaps<D, Real><<<(np + 255) / 256, 256, 0, st>>>(p, parts, cells, count, first, np);
}

// ---------------------------------------------------------------------------
// Batched particle kernels of the serving loop.  Persistent blocks walk a
// work table of (bed, tile) entries; a block takes the whole entry, so the
// block-wide steps (the drag's shared pre-drags, the scan's tile) see one
// bed only.  Each entry runs the per-particle (per-tile) work of the
// single-bed kernels with its bed's buffers for the parity of this step, so a
// bed's results do not depend on the other beds of the batch.
// ---------------------------------------------------------------------------
struct BatchEntry {
    const BatchBed *b;
    int a;       // parity of the step's input buffers
    int tile;
};

__device__ __forceinline__ bool batch_entry(const BatchBed *__restrict__ beds,
                                            const int2 *__restrict__ work, int w, int step,
                                            BatchEntry &out)
{
    const int2 e = work[w];
    const BatchBed &b = beds[e.x];
    if (step >= b.nsteps) return false;
    out.b = &b;
    out.a = (b.parity0 + step) & 1;
    out.tile = e.y;
    return true;
}

__global__ void __launch_bounds__(kBatchTile, DragOccupancy<2, float>::value)
k_drag_batched(const BatchBed *__restrict__ beds, const int2 *__restrict__ work,
               const int *__restrict__ count, int step)
{
    __shared__ float sfp[2][256];
    __shared__ float sfor[2][kForeignChunk];
    const int nwork = *count;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        BatchEntry e;
        if (!batch_entry(beds, work, w, step, e)) continue;   // the same for the whole block
        const BatchBed &b = *e.b;
        const int first = e.tile * kBatchTile;
        const CellList cells{b.cl_local[e.a], b.cl_base[e.a], b.cl_shift};
        __syncthreads();   // the previous entry's readers of sfp are done
        drag_step_particle<2, float, false>(b.sp, b.part[e.a], b.stage, cells, b.fld, b.key,
                                            b.counts, b.diag_fpre, b.diag_fd, b.np,
                                            first + (int)threadIdx.x, first, first + kBatchTile, sfp,
                                            sfor);
    }
}

__global__ void __launch_bounds__(kCellScanThreads)
k_cell_scan_batched(const BatchBed *__restrict__ beds, const int2 *__restrict__ work,
                    const int *__restrict__ count, int step)
{
    __shared__ int warp_tot[32];
    __shared__ int total;
    __shared__ bool last;
    const int nwork = *count;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        BatchEntry e;
        if (!batch_entry(beds, work, w, step, e)) continue;
        const BatchBed &b = *e.b;
        const int nb = 1 - e.a;
        const CellListOut out{b.cl_local[nb], b.cl_base[nb], b.tile_total, b.ticket, b.cl_shift};
        const int nt = (b.ncell + 1 + (1 << b.cl_shift) - 1) >> b.cl_shift;
        __syncthreads();   // the previous entry's users of the shared words are done
        if (b.cl_shift == kCellTileLog2Large)
            cell_scan_tile<16>(b.counts, out, b.ncell + 1, e.tile, nt, warp_tot, total, last);
        else
            cell_scan_tile<4>(b.counts, out, b.ncell + 1, e.tile, nt, warp_tot, total, last);
    }
}

__global__ void __launch_bounds__(kBatchTile)
k_scatter_batched(const BatchBed *__restrict__ beds, const int2 *__restrict__ work,
                  const int *__restrict__ count, int step)
{
    const int nwork = *count;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        BatchEntry e;
        if (!batch_entry(beds, work, w, step, e)) continue;
        const BatchBed &b = *e.b;
        const int k = e.tile * kBatchTile + (int)threadIdx.x;
        if (k >= b.np) continue;
        const int nb = 1 - e.a;
        scatter_one(b.key, b.part[e.a].id, b.counts, CellList{b.cl_local[nb], b.cl_base[nb], b.cl_shift}, b.slot,
                    b.idslot, k);
    }
}

__global__ void __launch_bounds__(kBatchTile)
k_gather_batched(const BatchBed *__restrict__ beds, const int2 *__restrict__ work,
                 const int *__restrict__ count, int step)
{
    const int nwork = *count;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        BatchEntry e;
        if (!batch_entry(beds, work, w, step, e)) continue;
        const BatchBed &b = *e.b;
        const int s = e.tile * kBatchTile + (int)threadIdx.x;
        if (s >= b.np) continue;
        const int nb = 1 - e.a;
        Particles<float> src = b.stage;
        src.id = b.part[e.a].id;
        gather_one<2, float>(CellList{b.cl_local[nb], b.cl_base[nb], b.cl_shift}, b.slot, b.idslot, src,
                             b.part[nb], s);
    }
}

__global__ void __launch_bounds__(kBatchTile, DetectOccupancy<2, float>::value)
k_detect_batched(const BatchBed *__restrict__ beds, const int2 *__restrict__ work,
                 const int *__restrict__ count, int step)
{
    const int nwork = *count;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        BatchEntry e;
        if (!batch_entry(beds, work, w, step, e)) continue;
        const BatchBed &b = *e.b;
        const int i = e.tile * kBatchTile + (int)threadIdx.x;
        if (i >= b.np) continue;
        const int nb = 1 - e.a;
        detect_one<2, float>(b.sp, b.part[nb], CellList{b.cl_local[nb], b.cl_base[nb], b.cl_shift}, b.best,
                             b.wall, nullptr, nullptr, 0, i);
    }
}

__global__ void __launch_bounds__(kBatchTile)
k_resolve_batched(const BatchBed *__restrict__ beds, const int2 *__restrict__ work,
                  const int *__restrict__ count, int step)
{
    const int nwork = *count;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        BatchEntry e;
        if (!batch_entry(beds, work, w, step, e)) continue;
        const BatchBed &b = *e.b;
        const int i = e.tile * kBatchTile + (int)threadIdx.x;
        if (i >= b.np) continue;
        resolve_one<2, float>(b.sp, b.part[1 - e.a], b.best, b.wall, i);
    }
}

void launch_particles_batched(const BatchBed *beds, BatchWork work, int step, cudaStream_t st)
{
    static const int g_drag = resident_grid((const void *)k_drag_batched, kBatchTile, 1 << 30);
    static const int g_scan = resident_grid((const void *)k_cell_scan_batched, kCellScanThreads, 1 << 30);
    static const int g_scat = resident_grid((const void *)k_scatter_batched, kBatchTile, 1 << 30);
    static const int g_gath = resident_grid((const void *)k_gather_batched, kBatchTile, 1 << 30);
    static const int g_det = resident_grid((const void *)k_detect_batched, kBatchTile, 1 << 30);
    static const int g_res = resident_grid((const void *)k_resolve_batched, kBatchTile, 1 << 30);
    if (!work.count) return;
    const int *n_scan = work.count + 1, *n_part = work.count + 2;
    k_drag_batched<<<g_drag, kBatchTile, 0, st>>>(beds, work.part_tiles, n_part, step);
    k_cell_scan_batched<<<g_scan, kCellScanThreads, 0, st>>>(beds, work.scan_tiles, n_scan, step);
    k_scatter_batched<<<g_scat, kBatchTile, 0, st>>>(beds, work.part_tiles, n_part, step);
    k_gather_batched<<<g_gath, kBatchTile, 0, st>>>(beds, work.part_tiles, n_part, step);
    k_detect_batched<<<g_det, kBatchTile, 0, st>>>(beds, work.part_tiles, n_part, step);
    k_resolve_batched<<<g_res, kBatchTile, 0, st>>>(beds, work.part_tiles, n_part, step);
}

// ---------------------------------------------------------------------------
#define LBDPS_INST_P(D, R)                                                                          \
    template void launch_drag_step<D, R>(const StepParams<R> &, Particles<R>, Particles<R>,        \
                                         CellList, Fields<R>, int *, int *, R *, R *, int,          \
                                         cudaStream_t);                                             \
    template void launch_detect<D, R>(const StepParams<R> &, Particles<R>, CellList, int *, int *,  \
                                      long long *, unsigned long long *, long long, int,           \
                                      cudaStream_t);                                               \
    template void launch_resolve<D, R>(const StepParams<R> &, Particles<R>, const int *,           \
                                       const int *, int, cudaStream_t);                            \
    template void launch_cell_keys<D, R>(const int *, Particles<R>, int *, int *, int,              \
                                         cudaStream_t);                                             \
    template void launch_particles_to_host_order<D, R>(Particles<R>, int, double, double, double *, \
                                                       double *, cudaStream_t);                    \
    template void launch_particles_from_host_order<D, R>(const double *, const double *, int,       \
                                                         double, double, Particles<R>,             \
                                                         cudaStream_t);                            \
    template void launch_overlaps<D, R>(const StepParams<R> &, Particles<R>, CellList,              \
                                        unsigned long long *, unsigned long long *, int,            \
                                        cudaStream_t);

LBDPS_INST_P(2, double)
LBDPS_INST_P(2, float)
LBDPS_INST_P(3, double)
LBDPS_INST_P(3, float)

template void launch_place<double>(int, const int *, int *, CellList, int2 *, int *,
                                   Particles<double>, Particles<double>, int, cudaStream_t);
template void launch_place<float>(int, const int *, int *, CellList, int2 *, int *,
                                  Particles<float>, Particles<float>, int, cudaStream_t);

}  // namespace lbdpsk

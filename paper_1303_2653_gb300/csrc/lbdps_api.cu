// Host side of the C ABI declared in include/lbdps.h: validation, unit
// conversion, device memory, the step sequence (optionally replayed from a
// captured CUDA graph), data transfer, reductions and checkpoints.
#include "lbdps.h"
#include "lbdps_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <mutex>
#include <climits>
#include <cstdint>
#include <type_traits>
#include <vector>

using namespace lbdpsk;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(LBDPS_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                        __FILE__, __LINE__);                                              \
    } while (0)

#define CHECK_LAUNCH()                                                                    \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            return fail(LBDPS_ERR_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

// Lattice-unit constants (h = 1, dt = 1, reference gas density 1).
// Profiling events of one step: the intervals between them are collide_stream,
// soft-sphere contacts, drag, sort and hard-sphere collisions; the classes
// reported are collide_stream (0), drag (1), sort (2) and particle-particle
// contacts of either model (3).
constexpr int kStepEvents = 6;
constexpr int kStepEventClass[kStepEvents - 1] = {0, 3, 1, 2, 3};

struct Derived {
    double nu, mu, tau, rho_s, d, r, vp, mp, e;
    double geff[3], fb[3], u0[3], wall_u[6][3];
    double cs;
    double kn, eta, eta_w;     // soft spheres: stiffness, pair and wall damping
    double mu_f, gamma_t;      // soft-sphere friction: Coulomb coefficient, tangential damping
    double inertia;            // 2/5 m_p r^2
};

constexpr double kPi = 3.141592653589793238462643383;

Derived derive(const lbdps_lattice_desc &L, const lbdps_particle_desc &Pd, const lbdps_params &P)
{
    Derived k{};
    const double nu_si = P.mu_g / P.rho_g;
    k.nu = nu_si * L.dt / (L.h * L.h);
    k.mu = k.nu;
    k.tau = 3.0 * k.nu + 0.5;                          // Eq. 3
    k.rho_s = Pd.rho_s / P.rho_g;
    k.d = Pd.d_p / L.h;
    k.r = 0.5 * k.d;
    k.vp = kPi * k.d * k.d * k.d / 6.0;
    k.mp = k.rho_s * k.vp;
    k.e = Pd.e;
    const double gscale = L.dt * L.dt / L.h, uscale = L.dt / L.h;
    for (int a = 0; a < 3; ++a) {
        k.geff[a] = (1.0 - P.rho_g / Pd.rho_s) * P.g[a] * gscale;   // effective gravity (section 3)
        k.fb[a] = P.body_accel[a] * gscale;
        k.u0[a] = P.u0[a] * uscale;
    }
    for (int f = 0; f < 6; ++f)
        for (int a = 0; a < 3; ++a) k.wall_u[f][a] = L.wall_u[f][a] * uscale;
    k.cs = P.cs_smag;
    // soft spheres: the damping that gives a linear spring-dashpot contact
    // the restitution e, for the reduced mass m_p / 2 of a pair and m_p
    // against a wall (an infinitely heavy body)
    k.kn = k.eta = k.eta_w = 0.0;
    if (Pd.collision_model == LBDPS_COLLIDE_SOFT) {
        k.kn = Pd.dem_kn * L.dt * L.dt / (P.rho_g * L.h * L.h * L.h);
        if (k.e > 0.0 && k.e < 1.0 && k.kn > 0.0) {
            const double le = std::log(k.e);
            const double z = -le / std::sqrt(kPi * kPi + le * le);
            k.eta = 2.0 * z * std::sqrt(0.5 * k.mp * k.kn);
            k.eta_w = 2.0 * z * std::sqrt(k.mp * k.kn);
        }
        k.mu_f = Pd.dem_mu;
        k.gamma_t = Pd.dem_gamma_t * L.dt / (P.rho_g * L.h * L.h * L.h);
    }
    k.inertia = 0.4 * k.mp * k.r * k.r;
    return k;
}

// ---------------------------------------------------------------------------
// Host loops over particle arrays, split over the host's cores: f(lo, hi) for
// consecutive chunks of [0, n).  Large beds hold millions of coordinates, and
// one core spends milliseconds checking them or taking the first touch of a
// fresh output array's pages.
// ---------------------------------------------------------------------------
template <class F> void host_parallel(size_t n, F &&f, size_t min_chunk = 1 << 16)
{
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nt = std::min<size_t>({(size_t)hw, (size_t)16, (n + min_chunk - 1) / min_chunk});
    if (nt <= 1) {
        f((size_t)0, n);
        return;
    }
    std::vector<std::thread> pool;
    pool.reserve(nt - 1);
    const size_t chunk = (n + nt - 1) / nt;
    for (size_t t = 1; t < nt; ++t) {
        const size_t lo = std::min(n, t * chunk), hi = std::min(n, lo + chunk);
        try {
            pool.emplace_back([&f, lo, hi] { f(lo, hi); });
        } catch (...) {   // no thread to be had: run the chunk here
            f(lo, hi);
        }
    }
    f((size_t)0, std::min(n, chunk));
    for (auto &th : pool) th.join();
}

// The first touch of every page of a caller's output array, on all host
// cores.  A fresh array costs a page fault per page, which a copy from the
// device would otherwise take one after the other; the stores go to memory
// that the copy overwrites.
void touch_pages(void *p, size_t bytes)
{
    if (!p || bytes == 0) return;
    constexpr size_t kPage = 4096;   // the smallest page size: every page is touched
    volatile char *c = static_cast<volatile char *>(p);
    host_parallel(
        (bytes + kPage - 1) / kPage,
        [&](size_t lo, size_t hi) {
            for (size_t k = lo; k < hi; ++k) c[k * kPage] = 0;
        },
        256);
}

// Every block carries a guard zone of kGuardBytes right after the bytes that
// were asked for, filled with kGuardByte at allocation; lbdps_check_guards
// reports blocks whose guard was overwritten (a kernel that wrote past the
// end of its buffer).
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;

struct DeviceAlloc {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *ctx = nullptr;
    std::vector<void *> owned;
    std::vector<std::pair<char *, size_t>> guards;   // guard start, bytes asked for
    bool count_only = false;     // only add up the sizes (memory estimate)
    bool misaligned = false;     // params.alloc returned a block off a 256-byte boundary
    size_t counted = 0;
    cudaStream_t stream = nullptr;   // the handle's stream: guards are written on it
    char *slab = nullptr;            // the block get() carves from (begin_slab), or null
    size_t slab_size = 0, slab_used = 0;

    // a block of `bytes` from params.alloc or cudaMalloc (null on failure)
    void *take(size_t bytes)
    {
        void *p = nullptr;
        if (alloc) {
            p = alloc(bytes, ctx);
            if (p && ((uintptr_t)p & 255u)) {
                owned.push_back(p);
                misaligned = true;
                return nullptr;
            }
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) owned.push_back(p);
        return p;
    }
    // Take all of a handle's buffers as one block of `total` bytes (what a
    // count_only pass of the same get() calls added up): get() then hands
    // out consecutive pieces of it, so creating a bed costs one allocator
    // call instead of one per buffer.
    bool begin_slab(size_t total)
    {
        slab = static_cast<char *>(take(total));
        slab_size = slab ? total : 0;
        slab_used = 0;
        return slab != nullptr;
    }
    // later get() calls (buffers a bed takes on first use) allocate again
    // (the block stays owned)
    void end_slab()
    {
        slab = nullptr;
        slab_size = slab_used = 0;
    }
    void *get(size_t asked)
    {
        size_t bytes = ((asked + kGuardBytes) + 255) & ~size_t(255);
        if (count_only) {
            counted += bytes;
            return (void *)(uintptr_t)256;   // never dereferenced
        }
        void *p = nullptr;
        if (slab) {
            if (slab_used + bytes <= slab_size) {
                p = slab + slab_used;
                slab_used += bytes;
            }
        } else {
            p = take(bytes);
        }
        if (p) {
            char *g = static_cast<char *>(p) + asked;
            if (cudaMemsetAsync(g, kGuardByte, kGuardBytes, stream) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            guards.emplace_back(g, asked);
        }
        return p;
    }
    // number of blocks whose guard zone no longer holds kGuardByte
    int damaged(cudaStream_t st, int *bad) const
    {
        std::vector<unsigned char> h(kGuardBytes);
        int n = 0;
        for (const auto &g : guards) {
            if (cudaMemcpyAsync(h.data(), g.first, kGuardBytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                cudaGetLastError();
                return -1;
            }
            for (unsigned char c : h)
                if (c != kGuardByte) {
                    ++n;
                    break;
                }
        }
        *bad = n;
        return 0;
    }
    // a block for the duration of one call (no guard zone); give it back
    // with put_temp once the stream no longer uses it
    void *get_temp(size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        void *p = nullptr;
        if (alloc) {
            p = alloc(bytes, ctx);
            if (p && ((uintptr_t)p & 255u)) {
                release(p, ctx);
                p = nullptr;
            }
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return p;
    }
    void put_temp(void *p)
    {
        if (!p) return;
        if (release) release(p, ctx);
        else cudaFree(p);
    }
    void release_all()
    {
        if (count_only) return;
        for (void *p : owned) {
            if (release) release(p, ctx);
            else cudaFree(p);
        }
        owned.clear();
        guards.clear();
        end_slab();
    }
};

// Interface of one (lattice, arithmetic, storage) instantiation.
struct Engine {
    virtual ~Engine() {}
    virtual int allocate(DeviceAlloc &A) = 0;
    // particles as the caller holds them (id order, interleaved), converted
    // on the device: positions / pos_div, velocities * vel_mul
    virtual int upload_initial(const double *pos, const double *vel, double pos_div, double vel_mul) = 0;
    // gas_stats: the collision also writes the per-warp moment sums of the
    // state it reads (parity `parity`) into that parity's gas partials
    virtual int enqueue_step(int parity, cudaEvent_t *ev, bool gas_stats = false) = 0;
    virtual int fields(int mask, int units, double *out, size_t cap) = 0;
    virtual int particles(int units, double *pos, double *vel, int64_t cap) = 0;
    virtual int set_particles(const double *pos, const double *vel, double pos_div = 1.0,
                              double vel_mul = 1.0) = 0;
    virtual int spin(int units, double *out, int64_t cap) = 0;
    virtual int set_spin(const double *in) = 0;
    virtual int populations(double *f, size_t cap) = 0;
    virtual int set_populations(const double *f, size_t count) = 0;
    virtual int particle_diag(int which, double *out, size_t cap) = 0;
    virtual int collide_particles(int64_t *pairs, int64_t cap, int64_t *npairs) = 0;
    // pairs of the current (sorted) particles closer than d: count and the
    // pair of smallest ids
    virtual int overlaps(unsigned long long *count, int *id_i, int *id_j) = 0;
    virtual int stats(lbdps_stats_t *out) = 0;
    // reductions of the current state, written by the kernel into mapped
    // pinned host memory `dst` (kStatOut doubles) on the stream, no wait
    virtual int enqueue_stats(double *dst) = 0;
    // the reductions of the state of parity q after the next step's collision
    // wrote its gas partials, with the health word and outlet count of
    // snapshot slot `slot` (written by enqueue_snapshot at the end of the
    // step that produced the state) instead of the live words
    virtual int enqueue_stats_of(double *dst, int q, int slot) = 0;
    virtual int enqueue_snapshot(int slot) = 0;
    virtual int health(unsigned *out) = 0;
    virtual int bubbles(double threshold, int voidage, int64_t *out) = 0;
    virtual int set_inlet(const double *inlet_lat) = 0;
    virtual size_t checkpoint_bytes() const = 0;
    virtual int save(char *buf) = 0;
    virtual int load(const char *buf) = 0;
    // the bed's buffers and parameters for a batch of the serving loop
    // (2D, FP32 arithmetic, hard spheres only)
    virtual int batch_describe(BatchBed *) { return LBDPS_ERR_INVALID; }
};

}  // namespace

struct lbdps {
    int dim = 0, q = 0;
    int n[3] = {1, 1, 1};
    int ncell = 0, np = 0;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    double h = 1.0, dt = 1.0;
    lbdps_params prm{};
    Derived k{};
    int ntab = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DeviceAlloc mem;
    std::unique_ptr<Engine> eng;
    int parity = 0;
    int64_t steps = 0;
    int64_t since_check = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // one step, per starting parity
    cudaGraphExec_t chunk[2] = {nullptr, nullptr};   // kChunkSteps steps, per starting parity
    int recirculate = 0;               // outlet -> inlet re-injection of particles
    bool soft = false;                 // soft-sphere contacts in place of hard spheres
    bool friction = false;             // soft spheres with friction (spins kept)
    unsigned *health_host = nullptr;   // pinned: the health word, then 16 doubles of statistics
    double *stats_host = nullptr;      // inside the same pinned block
    double *mon_host = nullptr;        // pinned: kMonSteps statistics records (lbdps_step_monitored)
    // monitored steps: graphs of one step whose collision also sums the
    // moments of its input state, plus the snapshot of the step's health word
    // and outlet count (per starting parity)
    cudaGraphExec_t mon_graph[2] = {nullptr, nullptr};
    std::vector<double> inlet_lat;     // face cells x dim
};

namespace {

void decode_stats(lbdps *h, const double *v, bool bed, int64_t steps, lbdps_stats_t *out);

// ---------------------------------------------------------------------------
// Engine for one instantiation.
// ---------------------------------------------------------------------------
template <class L, class Real, class S> struct EngineT : Engine {
    static constexpr int D = L::D, Q = L::Q;
    static constexpr int NW = D == 2 ? 1 : 3;   // spin components
    lbdps *H;
    S *f[2] = {nullptr, nullptr};
    Fields<Real> fld{};
    Particles<Real> part[2]{};
    Particles<Real> stage{};   // integrated state of the step, before placement
    int *cl_local[2] = {nullptr, nullptr}, *cl_base[2] = {nullptr, nullptr};
    int *tile_total = nullptr;
    unsigned *ticket = nullptr;
    int *key = nullptr, *counts = nullptr, *idslot = nullptr;
    int2 *slot = nullptr;     // (source index, cell) of each sorted slot
    Real *diag_fpre = nullptr, *diag_fd = nullptr;
    int *best = nullptr, *wall = nullptr;
    Real *fc[3] = {nullptr, nullptr, nullptr};   // soft-sphere contact forces (sorted slots)
    Real *diag_fc = nullptr;                     // the same in id order (diagnostics)
    Real *tabs[10] = {};
    int *tab_branch = nullptr;
    typename Vec4<Real>::type *tab_pk[2] = {nullptr, nullptr};
    Real *inlet_dev = nullptr;
    unsigned *health_dev = nullptr;
    double *red_partials = nullptr;
    unsigned *red_ticket = nullptr;
    unsigned long long *solids_out = nullptr;   // particles through the outlet so far
    BubbleScratch bub{};                         // allocated on the first lbdps_bubbles
    unsigned long long *npairs_dev = nullptr;
    unsigned long long *ovl_dev = nullptr;      // overlap check: count, smallest pair
    unsigned long long *snap_dev = nullptr;     // 2 slots x (health word, outlet count)
    double *gas_part[2] = {nullptr, nullptr};   // per parity: moment sums of the collision's warps
    long long gas_warps = 0;   // groups of 4 doubles in each gas_part buffer
    StepParams<Real> sp{};
    PopLayout lay{};          // extended lattice of the population arrays
    int packed_limit = 0;     // more particle centres per cell cannot all be apart

    explicit EngineT(lbdps *h) : H(h) {}
    size_t pop_slots() const { return (size_t)Q * (size_t)lay.nce; }

    int allocate(DeviceAlloc &A) override
    {
        const size_t nc = (size_t)H->ncell, np = (size_t)std::max(H->np, 1);
        auto get = [&](size_t bytes) { return A.get(bytes); };
        lay = make_layout(D, H->n);
        if (lay.nce >= (1ll << 31))
            return fail(LBDPS_ERR_CAPACITY, "lattice too large: %lld slots per direction (limit 2^31)",
                        lay.nce);
        for (int b = 0; b < 2; ++b) {
            f[b] = (S *)get(sizeof(S) * pop_slots());
            cl_local[b] = (int *)get(sizeof(int) * (nc + 1));
            cl_base[b] = (int *)get(sizeof(int) * (cell_tiles(H->ncell) + 1));
            for (int a = 0; a < D; ++a) {
                part[b].P[a] = (double *)get(sizeof(double) * np);
                part[b].v[a] = (Real *)get(sizeof(Real) * np);
                part[b].off[a] = (Real *)get(sizeof(Real) * np);
            }
            part[b].id = (int *)get(sizeof(int) * np);
            part[b].cell = (int *)get(sizeof(int) * np);
        }
        for (int a = 0; a < D; ++a) {
            stage.P[a] = (double *)get(sizeof(double) * np);
            stage.v[a] = (Real *)get(sizeof(Real) * np);
            stage.off[a] = (Real *)get(sizeof(Real) * np);
            if (!stage.P[a] || !stage.v[a] || !stage.off[a])
                return fail(LBDPS_ERR_OOM, "device allocation failed");
        }
        fld.rho = (Real *)get(sizeof(Real) * nc);
        fld.node4 = (typename Vec4<Real>::type *)get(sizeof(typename Vec4<Real>::type) * nc);
        fld.solg = D == 3 ? (Real *)get(sizeof(Real) * nc) : nullptr;
        for (int a = 0; a < D; ++a) fld.fpg[a] = (Real *)get(sizeof(Real) * nc);
        if (H->prm.diagnostics) {
            fld.tau_t = (Real *)get(sizeof(Real) * nc);
            fld.eps_g = (Real *)get(sizeof(Real) * nc);
            fld.ntot = (int *)get(sizeof(int) * nc);
            for (int a = 0; a < D; ++a) {
                fld.vs[a] = (Real *)get(sizeof(Real) * nc);
                fld.u[a] = (Real *)get(sizeof(Real) * nc);
            }
            diag_fpre = (Real *)get(sizeof(Real) * D * np);
            diag_fd = (Real *)get(sizeof(Real) * D * np);
        }
        if (H->soft) {
            for (int a = 0; a < D; ++a) {
                fc[a] = (Real *)get(sizeof(Real) * np);
                if (!fc[a]) return fail(LBDPS_ERR_OOM, "device allocation failed");
            }
            if (H->friction)
                for (int c = 0; c < NW; ++c) {
                    part[0].w[c] = (Real *)get(sizeof(Real) * np);
                    part[1].w[c] = (Real *)get(sizeof(Real) * np);
                    stage.w[c] = (Real *)get(sizeof(Real) * np);
                    if (!part[0].w[c] || !part[1].w[c] || !stage.w[c])
                        return fail(LBDPS_ERR_OOM, "device allocation failed");
                }
            if (H->prm.diagnostics) {
                diag_fc = (Real *)get(sizeof(Real) * D * np);
                if (!diag_fc) return fail(LBDPS_ERR_OOM, "device allocation failed");
            }
        }
        key = (int *)get(sizeof(int) * np);
        counts = (int *)get(sizeof(int) * (nc + 1));
        slot = (int2 *)get(sizeof(int2) * np);
        idslot = (int *)get(sizeof(int) * np);
        tile_total = (int *)get(sizeof(int) * cell_tiles(H->ncell));
        ticket = (unsigned *)get(sizeof(unsigned));
        best = (int *)get(sizeof(int) * np);
        wall = (int *)get(sizeof(int) * np);
        for (int t = 0; t < 10; ++t) tabs[t] = (Real *)get(sizeof(Real) * H->ntab);
        tab_branch = (int *)get(sizeof(int) * H->ntab);
        for (int t = 0; t < 2; ++t)
            tab_pk[t] = (typename Vec4<Real>::type *)get(sizeof(typename Vec4<Real>::type) * H->ntab);
        const int nface = (int)(H->inlet_lat.size() / D);
        inlet_dev = (Real *)get(sizeof(Real) * D * std::max(nface, 1));
        health_dev = (unsigned *)get(sizeof(unsigned));
        red_partials = (double *)get(sizeof(double) * kStatPartials);
        red_ticket = (unsigned *)get(sizeof(unsigned));
        solids_out = (unsigned long long *)get(sizeof(unsigned long long));
        npairs_dev = (unsigned long long *)get(sizeof(unsigned long long));
        ovl_dev = (unsigned long long *)get(2 * sizeof(unsigned long long));
        snap_dev = (unsigned long long *)get(4 * sizeof(unsigned long long));
        gas_warps = collide_warps(D, H->n);
        for (int b = 0; b < 2; ++b) {
            gas_part[b] = (double *)get(sizeof(double) * 4 * (size_t)gas_warps);
            if (!gas_part[b]) return fail(LBDPS_ERR_OOM, "device allocation failed");
        }
        void *must[] = {f[0], f[1], cl_local[0], cl_local[1], cl_base[0], cl_base[1], fld.rho,
                        fld.node4, key, counts, slot, idslot, tile_total, ticket,
                        best, wall, tab_branch, inlet_dev, health_dev,
                        red_partials, red_ticket, solids_out, npairs_dev, ovl_dev, snap_dev, part[0].id, part[1].id,
                        part[0].cell, part[1].cell};
        for (void *p : must)
            if (!p) return fail(LBDPS_ERR_OOM, "device allocation failed");
        for (int a = 0; a < D; ++a)
            if (!fld.fpg[a] || !part[0].P[a] || !part[1].P[a] || !part[0].v[a] ||
                !part[1].v[a] || !part[0].off[a] || !part[1].off[a])
                return fail(LBDPS_ERR_OOM, "device allocation failed");
        if (D == 3 && !fld.solg) return fail(LBDPS_ERR_OOM, "device allocation failed");
        for (int t = 0; t < 10; ++t)
            if (!tabs[t]) return fail(LBDPS_ERR_OOM, "device allocation failed");
        if (!tab_pk[0] || !tab_pk[1]) return fail(LBDPS_ERR_OOM, "device allocation failed");
        if (H->prm.diagnostics && (!fld.tau_t || !fld.eps_g || !fld.ntot || !diag_fpre || !diag_fd ||
                                   !fld.vs[0] || !fld.u[0] || !fld.vs[D - 1] || !fld.u[D - 1]))
            return fail(LBDPS_ERR_OOM, "device allocation failed");
        fill_params();
        return LBDPS_OK;
    }

    CellList cells(int b) const { return CellList{cl_local[b], cl_base[b], cell_tile_log2(H->ncell)}; }
    CellListOut cells_out(int b)
    {
        return CellListOut{cl_local[b], cl_base[b], tile_total, ticket, cell_tile_log2(H->ncell)};
    }

    int clear_cells(int b)
    {
        CU(cudaMemsetAsync(cl_local[b], 0, sizeof(int) * (H->ncell + 1), H->stream));
        CU(cudaMemsetAsync(cl_base[b], 0, sizeof(int) * (cell_tiles(H->ncell) + 1), H->stream));
        return LBDPS_OK;
    }

    void fill_params()
    {
        const Derived &k = H->k;
        StepParams<Real> &p = sp;
        p.dim = D;
        for (int a = 0; a < 3; ++a) p.n[a] = H->n[a];
        p.ncell = H->ncell;
        for (int f6 = 0; f6 < 6; ++f6) p.bc[f6] = H->bc[f6];
        p.vert = D - 1;
        p.tau = (Real)k.tau;
        p.inv_tau = (Real)(1.0 / k.tau);
        p.les_k = (Real)(18.0 * k.cs * k.cs);
        p.has_fb = 0;
        for (int a = 0; a < 3; ++a) {
            p.fb[a] = (Real)k.fb[a];
            if (k.fb[a] != 0.0) p.has_fb = 1;
            p.geff[a] = (Real)k.geff[a];
        }
        for (int f6 = 0; f6 < 6; ++f6)
            for (int a = 0; a < 3; ++a) p.wall_u[f6][a] = (Real)k.wall_u[f6][a];
        p.mu = (Real)k.mu;
        p.d = (Real)k.d;
        p.r = (Real)k.r;
        p.vp = (Real)k.vp;
        p.mp = (Real)k.mp;
        p.e = (Real)k.e;
        p.psign = H->prm.pressure_plus ? Real(1) : Real(-1);
        p.d2 = k.d * k.d;
        p.r64 = k.r;
        for (int a = 0; a < 3; ++a) {
            p.len[a] = (double)H->n[a];
            p.len_below[a] = std::nextafter((double)H->n[a], 0.0);
        }
        CountTables<Real> &t = p.tab;
        t.eps_s = tabs[0];
        t.eps_g = tabs[1];
        t.inv_div = tabs[2];
        t.og = tabs[3];
        t.gam = tabs[4];
        t.beta_a = tabs[5];
        t.beta_b = tabs[6];
        t.beta_c = tabs[7];
        t.re_k = tabs[8];
        t.sol_g = tabs[9];
        t.pk0 = tab_pk[0];
        t.pk1 = tab_pk[1];
        t.branch = tab_branch;
        t.ntab = H->ntab;
        p.inlet_u = inlet_dev;
        p.inlet_face = -1;
        for (int f6 = 0; f6 < 6; ++f6)
            if (H->bc[f6] == BC_INLET) p.inlet_face = f6;
        p.health = health_dev;
        p.recirculate = H->recirculate;
        p.solids_out = solids_out;
        for (int a = 0; a < 3; ++a) p.fc[a] = a < D ? fc[a] : nullptr;
        p.kn = (Real)k.kn;
        p.eta = (Real)k.eta;
        p.eta_w = (Real)k.eta_w;
        p.mu_f = (Real)k.mu_f;
        p.gamma_t = (Real)k.gamma_t;
        p.inv_inertia = (Real)(1.0 / k.inertia);
        {
            // spheres centred in a cell lie in the cell grown by d: at close
            // packing that box holds at most this many (lattice units)
            const double unit = D == 2 ? kPi * k.r * k.r : k.vp;
            const double cap = D == 2 ? kPi / (2.0 * std::sqrt(3.0)) : kPi / (3.0 * std::sqrt(2.0));
            packed_limit = (int)std::ceil(cap * std::pow(1.0 + k.d, D) / unit);
        }
        for (int c = 0; c < 3; ++c) p.spin_out[c] = H->friction && c < NW ? stage.w[c] : nullptr;
        p.gas_partials = nullptr;
    }

    int upload_initial(const double *pos, const double *vel, double pos_div, double vel_mul) override
    {
        cudaStream_t st = H->stream;
        const Derived &k = H->k;
        launch_build_tables<Real>(D, k.tau, k.r, k.vp, k.d, k.mu, H->prm.superficial_mode, H->ntab,
                                  nullptr, sp.tab, st);
        CHECK_LAUNCH();
        Real u0[3] = {(Real)k.u0[0], (Real)k.u0[1], (Real)k.u0[2]};
        launch_init_equilibrium<L, Real, S>(lay, u0, f[0], st);
        CHECK_LAUNCH();
        if (!H->inlet_lat.empty()) {
            std::vector<Real> tmpu(H->inlet_lat.begin(), H->inlet_lat.end());
            CU(cudaMemcpyAsync(inlet_dev, tmpu.data(), sizeof(Real) * tmpu.size(),
                               cudaMemcpyHostToDevice, st));
            CU(cudaStreamSynchronize(st));
        }
        CU(cudaMemsetAsync(health_dev, 0, sizeof(unsigned), st));
        CU(cudaMemsetAsync(counts, 0, sizeof(int) * (H->ncell + 1), st));
        CU(cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
        CU(cudaMemsetAsync(red_ticket, 0, sizeof(unsigned), st));
        CU(cudaMemsetAsync(solids_out, 0, sizeof(unsigned long long), st));
        if (H->np == 0) {
            int rc = clear_cells(0);
            if (rc == LBDPS_OK) rc = clear_cells(1);
            return rc;
        }
        return set_particles(pos, vel, pos_div, vel_mul);
    }

    // Load particles (id order; lattice units once positions are divided by
    // pos_div and velocities multiplied by vel_mul) into the current buffers
    // and sort them.
    int set_particles(const double *pos, const double *vel, double pos_div, double vel_mul) override
    {
        cudaStream_t st = H->stream;
        const int np = H->np;
        const int cur = H->parity, nxt = 1 - cur;
        if (np == 0) return LBDPS_OK;
        // one copy per array from the caller's memory, split per axis on the
        // device (ids in order, spins at rest), then sorted into the current
        // buffers
        const size_t bytes = sizeof(double) * (size_t)np * D;
        double *dp = (double *)H->mem.get_temp(bytes);
        double *dv = dp ? (double *)H->mem.get_temp(bytes) : nullptr;
        if (dp && dv) {
            cudaError_t e = cudaMemcpyAsync(dp, pos, bytes, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dv, vel, bytes, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) {
                launch_particles_from_host_order<D, Real>(dp, dv, np, pos_div, vel_mul, part[nxt], st);
                e = cudaGetLastError();
            }
            const cudaError_t e2 = cudaStreamSynchronize(st);
            H->mem.put_temp(dp);
            H->mem.put_temp(dv);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                cudaGetLastError();
                return fail(LBDPS_ERR_CUDA, "particle upload: %s",
                            cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            return sort_from(nxt, cur);
        }
        // no room for the staging arrays: split per axis on the host
        H->mem.put_temp(dp);
        H->mem.put_temp(dv);
        std::vector<double> Pa((size_t)np);
        std::vector<Real> va((size_t)np);
        std::vector<int> ids((size_t)np);
        for (int i = 0; i < np; ++i) ids[i] = i;
        // stage into the next buffers, then sort into the current ones
        for (int a = 0; a < D; ++a) {
            for (int i = 0; i < np; ++i) {
                Pa[i] = pos[(size_t)i * D + a] / pos_div;
                va[i] = (Real)(vel[(size_t)i * D + a] * vel_mul);
            }
            CU(cudaMemcpyAsync(part[nxt].P[a], Pa.data(), sizeof(double) * np,
                               cudaMemcpyHostToDevice, st));
            CU(cudaMemcpyAsync(part[nxt].v[a], va.data(), sizeof(Real) * np,
                               cudaMemcpyHostToDevice, st));
            CU(cudaStreamSynchronize(st));
        }
        CU(cudaMemcpyAsync(part[nxt].id, ids.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
        for (int c = 0; c < NW && H->friction; ++c)
            CU(cudaMemsetAsync(part[nxt].w[c], 0, sizeof(Real) * np, st));   // particles start without spin
        CU(cudaStreamSynchronize(st));
        return sort_from(nxt, cur);
    }

    // Sort particles held in buffer `src` (any order) into buffer `dst` by (cell, id).
    int sort_from(int src, int dst)
    {
        cudaStream_t st = H->stream;
        CU(cudaMemsetAsync(counts, 0, sizeof(int) * (H->ncell + 1), st));
        launch_cell_keys<D, Real>(H->n, part[src], key, counts, H->np, st);
        CHECK_LAUNCH();
        launch_cell_scan(counts, cells_out(dst), H->ncell, st);
        CHECK_LAUNCH();
        launch_place<Real>(D, key, counts, cells(dst), slot, idslot, part[src], part[dst], H->np, st);
        CHECK_LAUNCH();
        return LBDPS_OK;
    }

    // One coupled step from buffers `parity` into buffers `1 - parity`.
    // ev (optional, kStepEvents events) brackets the kernels for profiling:
    // collide_stream, soft-sphere contacts, drag, sort, hard-sphere
    // collisions (kStepEventClass maps each interval to its class).
    int enqueue_step(int parity, cudaEvent_t *ev, bool gas_stats) override
    {
        cudaStream_t st = H->stream;
        const int a = parity, b = 1 - parity;
        const int np = H->np;
        if (ev) CU(cudaEventRecord(ev[0], st));
        StepParams<Real> spc = sp;
        if (gas_stats) spc.gas_partials = gas_part[a];
        launch_collide_stream<L, Real, S>(spc, lay, f[a], f[b], cells(a), part[a], fld, st);
        CHECK_LAUNCH();
        if (ev) CU(cudaEventRecord(ev[1], st));
        if (H->soft) {
            // contact forces of the start-of-step state, used by the drag kernel
            launch_contacts<D, Real>(sp, part[a], cells(a), diag_fc, np, st);
            CHECK_LAUNCH();
        }
        if (ev) CU(cudaEventRecord(ev[2], st));
        launch_drag_step<D, Real>(sp, part[a], stage, cells(a), fld, key, counts, diag_fpre,
                                  diag_fd, np, st);
        CHECK_LAUNCH();
        if (ev) CU(cudaEventRecord(ev[3], st));
        if (np > 0) {
            launch_cell_scan(counts, cells_out(b), H->ncell, st);
            CHECK_LAUNCH();
            Particles<Real> src = stage;
            src.id = part[a].id;
            launch_place<Real>(D, key, counts, cells(b), slot, idslot, src, part[b], np, st);
            CHECK_LAUNCH();
        } else {
            int rc = clear_cells(b);
            if (rc) return rc;
        }
        if (ev) CU(cudaEventRecord(ev[4], st));
        if (!H->soft) {
            launch_detect<D, Real>(sp, part[b], cells(b), best, wall, nullptr, nullptr, 0, np, st);
            CHECK_LAUNCH();
            launch_resolve<D, Real>(sp, part[b], best, wall, np, st);
            CHECK_LAUNCH();
        }
        if (ev) CU(cudaEventRecord(ev[5], st));
        return LBDPS_OK;
    }

    int collide_particles(int64_t *pairs_out, int64_t cap, int64_t *npairs) override
    {
        cudaStream_t st = H->stream;
        const int cur = H->parity, oth = 1 - cur;
        const int np = H->np;
        if (np == 0) {
            if (npairs) *npairs = 0;
            return LBDPS_OK;
        }
        // re-sort the current particles (positions may have been replaced)
        int rc = copy_particles(cur, oth);
        if (rc) return rc;
        rc = sort_from(oth, cur);
        if (rc) return rc;
        long long *pairs_dev = nullptr;
        long long pcap = 0;
        std::vector<long long> hp;
        if (pairs_out) {
            pcap = std::max<int64_t>(cap, 1);
            if (cudaMalloc(&pairs_dev, sizeof(long long) * 2 * pcap) != cudaSuccess) {
                cudaGetLastError();
                return fail(LBDPS_ERR_OOM, "pair buffer allocation failed");
            }
        }
        CU(cudaMemsetAsync(npairs_dev, 0, sizeof(unsigned long long), st));
        launch_detect<D, Real>(sp, part[cur], cells(cur), best, wall, pairs_dev, npairs_dev,
                               pcap, np, st);
        CHECK_LAUNCH();
        launch_resolve<D, Real>(sp, part[cur], best, wall, np, st);
        CHECK_LAUNCH();
        unsigned long long total = 0;
        CU(cudaMemcpyAsync(&total, npairs_dev, sizeof(total), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        int result = LBDPS_OK;
        if (pairs_out) {
            const int64_t got = std::min<int64_t>((int64_t)total, cap);
            hp.resize((size_t)std::max<int64_t>(got, 1) * 2);
            if (got > 0) {
                cudaError_t e = cudaMemcpy(hp.data(), pairs_dev, sizeof(long long) * 2 * got,
                                           cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) result = fail(LBDPS_ERR_CUDA, "pair copy: %s", cudaGetErrorString(e));
            }
            std::vector<std::pair<long long, long long>> pr((size_t)got);
            for (int64_t i = 0; i < got; ++i) pr[i] = {hp[2 * i], hp[2 * i + 1]};
            std::sort(pr.begin(), pr.end());
            for (int64_t i = 0; i < got; ++i) {
                pairs_out[2 * i] = pr[i].first;
                pairs_out[2 * i + 1] = pr[i].second;
            }
            cudaFree(pairs_dev);
            if (result == LBDPS_OK && (int64_t)total > cap)
                result = fail(LBDPS_ERR_CAPACITY, "%llu pairs exceed capacity %lld", total, (long long)cap);
        }
        if (npairs) *npairs = (int64_t)total;
        return result;
    }

    int overlaps(unsigned long long *count, int *id_i, int *id_j) override
    {
        cudaStream_t st = H->stream;
        const int cur = H->parity;
        const unsigned long long init[2] = {0ull, ~0ull};
        CU(cudaMemcpyAsync(ovl_dev, init, sizeof(init), cudaMemcpyHostToDevice, st));
        launch_overlaps<D, Real>(sp, part[cur], cells(cur), ovl_dev, ovl_dev + 1, H->np, st);
        CHECK_LAUNCH();
        unsigned long long res[2] = {0ull, 0ull};
        CU(cudaMemcpyAsync(res, ovl_dev, sizeof(res), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        *count = res[0];
        *id_i = (int)(res[1] >> 32);
        *id_j = (int)(res[1] & 0xffffffffull);
        return LBDPS_OK;
    }

    int copy_particles(int from, int to)
    {
        cudaStream_t st = H->stream;
        const size_t np = (size_t)H->np;
        for (int a = 0; a < D; ++a) {
            CU(cudaMemcpyAsync(part[to].P[a], part[from].P[a], sizeof(double) * np,
                               cudaMemcpyDeviceToDevice, st));
            CU(cudaMemcpyAsync(part[to].v[a], part[from].v[a], sizeof(Real) * np,
                               cudaMemcpyDeviceToDevice, st));
        }
        CU(cudaMemcpyAsync(part[to].id, part[from].id, sizeof(int) * np, cudaMemcpyDeviceToDevice, st));
        for (int c = 0; c < NW && H->friction; ++c)
            CU(cudaMemcpyAsync(part[to].w[c], part[from].w[c], sizeof(Real) * np,
                               cudaMemcpyDeviceToDevice, st));
        return LBDPS_OK;
    }

    template <class T> int d2h(std::vector<T> &dst, const T *src, size_t n)
    {
        dst.resize(std::max<size_t>(n, 1));
        CU(cudaMemcpyAsync(dst.data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost, H->stream));
        CU(cudaStreamSynchronize(H->stream));
        return LBDPS_OK;
    }

    int fields(int mask, int units, double *out, size_t cap) override
    {
        const size_t nc = (size_t)H->ncell;
        size_t need = 0;
        const int vec_bits = LBDPS_FIELD_U | LBDPS_FIELD_FPG | LBDPS_FIELD_VS | LBDPS_FIELD_UACT;
        for (int bit = 0; bit < 9; ++bit)
            if (mask & (1 << bit)) need += nc * (((1 << bit) & vec_bits) ? D : 1);
        if (mask & ~((1 << 9) - 1)) return fail(LBDPS_ERR_INVALID, "unknown field bits");
        if (need > cap) return fail(LBDPS_ERR_CAPACITY, "fields need %zu doubles", need);
        const int plain = LBDPS_FIELD_RHO | LBDPS_FIELD_FPG | LBDPS_FIELD_BETA | LBDPS_FIELD_UACT;
        if ((mask & ~plain) && !H->prm.diagnostics)
            return fail(LBDPS_ERR_INVALID, "diagnostic fields need params.diagnostics = 1");
        const double us = units == LBDPS_UNITS_SI ? H->h / H->dt : 1.0;
        const double rs = units == LBDPS_UNITS_SI ? H->prm.rho_g : 1.0;
        // force per cell: rho h^3 (h/dt) / dt in SI
        const double fs = units == LBDPS_UNITS_SI ? H->prm.rho_g * H->h * H->h * H->h * H->h / (H->dt * H->dt) : 1.0;
        const double bs = units == LBDPS_UNITS_SI ? H->prm.rho_g / H->dt : 1.0;
        const double ts = units == LBDPS_UNITS_SI ? H->dt : 1.0;
        std::vector<Real> hb;
        std::vector<int> hi;
        size_t o = 0;
        auto put_scalar = [&](const Real *src, double scale) -> int {
            int rc = d2h(hb, src, nc);
            if (rc) return rc;
            for (size_t x = 0; x < nc; ++x) out[o + x] = (double)hb[x] * scale;
            o += nc;
            return LBDPS_OK;
        };
        auto put_vec = [&](Real *const *src, double scale) -> int {
            for (int a = 0; a < D; ++a) {
                int rc = d2h(hb, src[a], nc);
                if (rc) return rc;
                for (size_t x = 0; x < nc; ++x) out[o + x * D + a] = (double)hb[x] * scale;
            }
            o += nc * D;
            return LBDPS_OK;
        };
        // components of the node record: beta is .w, u_act is .x, .y (, .z)
        using V4 = typename Vec4<Real>::type;
        std::vector<V4> h4;
        auto put_node = [&](int first, int count, double scale) -> int {
            if (h4.empty()) {
                h4.resize(nc);
                CU(cudaMemcpyAsync(h4.data(), fld.node4, sizeof(V4) * nc, cudaMemcpyDeviceToHost,
                                   H->stream));
                CU(cudaStreamSynchronize(H->stream));
            }
            for (size_t x = 0; x < nc; ++x) {
                const Real c4[4] = {h4[x].x, h4[x].y, h4[x].z, h4[x].w};
                for (int a = 0; a < count; ++a) out[o + x * count + a] = (double)c4[first + a] * scale;
            }
            o += nc * count;
            return LBDPS_OK;
        };
        int rc = LBDPS_OK;
        if (mask & LBDPS_FIELD_RHO) if ((rc = put_scalar(fld.rho, rs))) return rc;
        if (mask & LBDPS_FIELD_U) if ((rc = put_vec(fld.u, us))) return rc;
        if (mask & LBDPS_FIELD_FPG) if ((rc = put_vec(fld.fpg, fs))) return rc;
        if (mask & LBDPS_FIELD_BETA) if ((rc = put_node(3, 1, bs))) return rc;
        if (mask & LBDPS_FIELD_VS) if ((rc = put_vec(fld.vs, us))) return rc;
        if (mask & LBDPS_FIELD_NTOT) {
            if ((rc = d2h(hi, fld.ntot, nc))) return rc;
            for (size_t x = 0; x < nc; ++x) out[o + x] = (double)hi[x];
            o += nc;
        }
        if (mask & LBDPS_FIELD_TAU_T) if ((rc = put_scalar(fld.tau_t, ts))) return rc;
        if (mask & LBDPS_FIELD_UACT) if ((rc = put_node(0, D, us))) return rc;
        if (mask & LBDPS_FIELD_EPS_G) if ((rc = put_scalar(fld.eps_g, 1.0))) return rc;
        return LBDPS_OK;
    }

    int particles(int units, double *pos, double *vel, int64_t cap) override
    {
        const int np = H->np, cur = H->parity;
        if (cap < np) return fail(LBDPS_ERR_CAPACITY, "need room for %d particles", np);
        if (np == 0) return LBDPS_OK;
        const double ps = units == LBDPS_UNITS_SI ? H->h : 1.0;
        const double vs = units == LBDPS_UNITS_SI ? H->h / H->dt : 1.0;
        // on the device: id order, interleaved, scaled; one copy per array
        // into the caller's memory
        const size_t bytes = sizeof(double) * (size_t)np * D;
        double *dp = pos ? (double *)H->mem.get_temp(bytes) : nullptr;
        double *dv = vel ? (double *)H->mem.get_temp(bytes) : nullptr;
        if ((!pos || dp) && (!vel || dv)) {
            cudaStream_t st = H->stream;
            launch_particles_to_host_order<D, Real>(part[cur], np, ps, vs, dp, dv, st);
            cudaError_t e = cudaGetLastError();
            // while the kernel runs
            touch_pages(pos, bytes);
            touch_pages(vel, bytes);
            if (e == cudaSuccess && pos) e = cudaMemcpyAsync(pos, dp, bytes, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && vel) e = cudaMemcpyAsync(vel, dv, bytes, cudaMemcpyDeviceToHost, st);
            const cudaError_t e2 = cudaStreamSynchronize(st);
            H->mem.put_temp(dp);
            H->mem.put_temp(dv);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                cudaGetLastError();
                return fail(LBDPS_ERR_CUDA, "particle read-back: %s",
                            cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            return LBDPS_OK;
        }
        // no room for the staging arrays: copy per axis and order on the host
        H->mem.put_temp(dp);
        H->mem.put_temp(dv);
        std::vector<int> ids;
        std::vector<double> Pd;
        std::vector<Real> vd;
        int rc = d2h(ids, part[cur].id, np);
        if (rc) return rc;
        for (int a = 0; a < D; ++a) {
            if ((rc = d2h(Pd, part[cur].P[a], np))) return rc;
            if ((rc = d2h(vd, part[cur].v[a], np))) return rc;
            for (int k = 0; k < np; ++k) {
                const size_t o = (size_t)ids[k] * D + a;
                if (pos) pos[o] = Pd[k] * ps;
                if (vel) vel[o] = (double)vd[k] * vs;
            }
        }
        return LBDPS_OK;
    }

    // spins in id order: NW values per particle, rad per step (lattice) or rad / s
    int spin(int units, double *out, int64_t cap) override
    {
        const int np = H->np, cur = H->parity;
        if (cap < (int64_t)np * NW) return fail(LBDPS_ERR_CAPACITY, "need %lld doubles", (long long)np * NW);
        if (!H->friction) {
            std::fill(out, out + (size_t)np * NW, 0.0);
            return LBDPS_OK;
        }
        if (np == 0) return LBDPS_OK;
        std::vector<int> ids;
        std::vector<Real> wd;
        int rc = d2h(ids, part[cur].id, np);
        if (rc) return rc;
        const double ws = units == LBDPS_UNITS_SI ? 1.0 / H->dt : 1.0;
        for (int c = 0; c < NW; ++c) {
            if ((rc = d2h(wd, part[cur].w[c], np))) return rc;
            for (int k = 0; k < np; ++k) out[(size_t)ids[k] * NW + c] = (double)wd[k] * ws;
        }
        return LBDPS_OK;
    }

    int set_spin(const double *in) override
    {
        const int np = H->np, cur = H->parity;
        if (!H->friction) return fail(LBDPS_ERR_INVALID, "spins need soft spheres with friction");
        if (np == 0) return LBDPS_OK;
        std::vector<int> ids;
        int rc = d2h(ids, part[cur].id, np);
        if (rc) return rc;
        std::vector<Real> wd((size_t)np);
        for (int c = 0; c < NW; ++c) {
            for (int k = 0; k < np; ++k) wd[k] = (Real)in[(size_t)ids[k] * NW + c];
            CU(cudaMemcpyAsync(part[cur].w[c], wd.data(), sizeof(Real) * np, cudaMemcpyHostToDevice,
                               H->stream));
            CU(cudaStreamSynchronize(H->stream));
        }
        return LBDPS_OK;
    }

    int populations(double *out, size_t cap) override
    {
        const size_t total = (size_t)Q * H->ncell;
        if (cap < total) return fail(LBDPS_ERR_CAPACITY, "need %zu doubles", total);
        double *dev = nullptr;
        CU(cudaMalloc(&dev, sizeof(double) * total));
        launch_export_populations<L, Real, S>(lay, H->ncell, f[H->parity], dev, H->stream);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, dev, sizeof(double) * total, cudaMemcpyDeviceToHost, H->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(H->stream);
        cudaFree(dev);
        if (e != cudaSuccess) return fail(LBDPS_ERR_CUDA, "populations: %s", cudaGetErrorString(e));
        return LBDPS_OK;
    }

    int set_populations(const double *in, size_t count) override
    {
        const size_t total = (size_t)Q * H->ncell;
        if (count != total) return fail(LBDPS_ERR_INVALID, "expected %zu values", total);
        double *dev = nullptr;
        CU(cudaMalloc(&dev, sizeof(double) * total));
        cudaError_t e = cudaMemcpyAsync(dev, in, sizeof(double) * total, cudaMemcpyHostToDevice, H->stream);
        if (e == cudaSuccess) {
            launch_import_populations<L, Real, S>(lay, H->ncell, dev, f[H->parity], H->stream);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(H->stream);
        cudaFree(dev);
        if (e != cudaSuccess) return fail(LBDPS_ERR_CUDA, "set_populations: %s", cudaGetErrorString(e));
        return LBDPS_OK;
    }

    int particle_diag(int which, double *out, size_t cap) override
    {
        const int np = H->np, cur = H->parity;
        const bool vec = (which == LBDPS_PDIAG_FPRE || which == LBDPS_PDIAG_FD ||
                          which == LBDPS_PDIAG_FC);
        const size_t need = (size_t)np * (vec ? D : 1);
        if (cap < need) return fail(LBDPS_ERR_CAPACITY, "need %zu doubles", need);
        if (np == 0) return LBDPS_OK;
        int rc;
        if (vec) {
            if (!H->prm.diagnostics) return fail(LBDPS_ERR_INVALID, "needs params.diagnostics = 1");
            if (which == LBDPS_PDIAG_FC && !H->soft)
                return fail(LBDPS_ERR_INVALID, "contact forces need collision_model = LBDPS_COLLIDE_SOFT");
            std::vector<Real> hb;
            const Real *src = which == LBDPS_PDIAG_FPRE ? diag_fpre
                              : which == LBDPS_PDIAG_FD ? diag_fd : diag_fc;
            if ((rc = d2h(hb, src, (size_t)D * np))) return rc;
            for (int a = 0; a < D; ++a)
                for (int i = 0; i < np; ++i) out[(size_t)i * D + a] = (double)hb[(size_t)a * np + i];
            return LBDPS_OK;
        }
        std::vector<int> ids, vals;
        if ((rc = d2h(ids, part[cur].id, np))) return rc;
        if (which == LBDPS_PDIAG_BEST) {
            if ((rc = d2h(vals, best, np))) return rc;
            for (int k = 0; k < np; ++k) out[ids[k]] = vals[k] >= 0 ? (double)ids[vals[k]] : -1.0;
        } else if (which == LBDPS_PDIAG_WALL) {
            if ((rc = d2h(vals, wall, np))) return rc;
            for (int k = 0; k < np; ++k) out[ids[k]] = (double)vals[k];
        } else if (which == LBDPS_PDIAG_ORDER) {
            for (int k = 0; k < np; ++k) out[k] = (double)ids[k];
        } else if (which == LBDPS_PDIAG_CELL) {
            std::vector<int> loc, bas;
            if ((rc = d2h(loc, cl_local[cur], (size_t)H->ncell + 1))) return rc;
            if ((rc = d2h(bas, cl_base[cur], (size_t)cell_tiles(H->ncell) + 1))) return rc;
            const int shift = cell_tile_log2(H->ncell);
            auto begin = [&](int c) { return loc[c] + bas[c >> shift]; };
            for (int c = 0; c < H->ncell; ++c)
                for (int k = begin(c); k < begin(c + 1); ++k) out[ids[k]] = (double)c;
        } else {
            return fail(LBDPS_ERR_INVALID, "unknown diagnostic %d", which);
        }
        return LBDPS_OK;
    }

    // All reductions of the statistics in one launch whose last block stores
    // the results in mapped pinned host memory; stats() then waits once.
    int enqueue_stats(double *dst) override
    {
        const int cur = H->parity;
        const bool bed = H->prm.diagnostics && H->steps > 0;
        // the last block of the reduction stores the results over the
        // host link itself: no copy node follows the kernel on the stream
        double *dev = nullptr;
        CU(cudaHostGetDevicePointer((void **)&dev, dst, 0));
        launch_gas_moments<L, Real, S>(lay, f[cur], H->n, gas_part[cur], H->stream);
        CHECK_LAUNCH();
        launch_reduce_all<L, Real>(H->ncell, gas_part[cur], gas_warps, part[cur], H->k.mp, H->np,
                                   sp.tab.eps_g, H->ntab, bed ? &fld : nullptr,
                                   red_partials, red_ticket, health_dev, solids_out, dev, health_dev,
                                   packed_limit, H->stream);
        CHECK_LAUNCH();
        return LBDPS_OK;
    }

    int enqueue_stats_of(double *dst, int q, int slot) override
    {
        double *dev = nullptr;
        CU(cudaHostGetDevicePointer((void **)&dev, dst, 0));
        const unsigned long long *sn = snap_dev + 2 * slot;
        // no node diagnostics: the next step has rewritten those arrays
        launch_reduce_all<L, Real>(H->ncell, gas_part[q], gas_warps, part[q], H->k.mp, H->np,
                                   sp.tab.eps_g, H->ntab, nullptr, red_partials, red_ticket,
                                   reinterpret_cast<const unsigned *>(sn), sn + 1, dev, health_dev,
                                   packed_limit, H->stream);
        CHECK_LAUNCH();
        return LBDPS_OK;
    }

    int enqueue_snapshot(int slot) override
    {
        launch_snapshot(health_dev, solids_out, snap_dev + 2 * slot, H->stream);
        CHECK_LAUNCH();
        return LBDPS_OK;
    }

    int stats(lbdps_stats_t *out) override
    {
        int rc = enqueue_stats(H->stats_host);
        if (rc) return rc;
        CU(cudaStreamSynchronize(H->stream));
        decode_stats(H, H->stats_host, H->prm.diagnostics && H->steps > 0, H->steps, out);
        return LBDPS_OK;
    }

    int bubbles(double threshold, int voidage, int64_t *out) override
    {
        const int nc = H->ncell;
        if (!bub.parent) {
            BubbleScratch b{};
            b.parent = (int *)H->mem.get(sizeof(int) * nc);
            b.size = (int *)H->mem.get(sizeof(int) * nc);
            b.top = (int *)H->mem.get(sizeof(int) * nc);
            b.nlim = (int *)H->mem.get(sizeof(int));
            b.out = (unsigned long long *)H->mem.get(sizeof(unsigned long long) * 3);
            b.err = (unsigned *)H->mem.get(sizeof(unsigned));
            if (!b.parent || !b.size || !b.top || !b.nlim || !b.out || !b.err)
                return fail(LBDPS_ERR_OOM, "device allocation failed");
            bub = b;
        }
        int per_mask = 0;
        for (int a = 0; a < D; ++a)
            if (H->bc[2 * a] == BC_PERIODIC) per_mask |= 1 << a;
        launch_bubbles(D, H->n, per_mask, H->k.r, H->k.vp, H->ntab, threshold, voidage,
                       cells(H->parity), bub, H->stream);
        CHECK_LAUNCH();
        unsigned long long res[3] = {0, 0, 0};
        unsigned err = 0;
        CU(cudaMemcpyAsync(res, bub.out, sizeof(res), cudaMemcpyDeviceToHost, H->stream));
        CU(cudaMemcpyAsync(&err, bub.err, sizeof(err), cudaMemcpyDeviceToHost, H->stream));
        CU(cudaStreamSynchronize(H->stream));
        if (err) return fail(LBDPS_ERR_TIMEOUT, "bubble labelling exceeded its iteration bound");
        for (int k = 0; k < 3; ++k) out[k] = (int64_t)res[k];
        return LBDPS_OK;
    }

    int set_inlet(const double *inlet_lat) override
    {
        const size_t n = H->inlet_lat.size();
        std::vector<Real> tmp(n);
        for (size_t i = 0; i < n; ++i) tmp[i] = (Real)inlet_lat[i];
        CU(cudaMemcpyAsync(inlet_dev, tmp.data(), sizeof(Real) * n, cudaMemcpyHostToDevice, H->stream));
        CU(cudaStreamSynchronize(H->stream));
        H->inlet_lat.assign(inlet_lat, inlet_lat + n);
        return LBDPS_OK;
    }

    int health(unsigned *out) override
    {
        CU(cudaMemcpyAsync(H->health_host, health_word(), sizeof(unsigned), cudaMemcpyDeviceToHost,
                           H->stream));
        CU(cudaStreamSynchronize(H->stream));
        *out = *H->health_host;
        return LBDPS_OK;
    }
    unsigned *health_word() { return this->health_dev; }

    // checkpoint payload: populations, particles (P, v, id), cell list
    size_t checkpoint_bytes() const override
    {
        const size_t nc = (size_t)H->ncell, np = (size_t)H->np;
        return sizeof(S) * pop_slots() + (sizeof(double) + 2 * sizeof(Real)) * D * np +
               2 * sizeof(int) * np + sizeof(int) * (nc + 1) +
               sizeof(int) * (cell_tiles(H->ncell) + 1) + sizeof(unsigned long long) +
               (H->friction ? sizeof(Real) * NW * np : 0);
    }

    int save(char *buf) override
    {
        cudaStream_t st = H->stream;
        const size_t nc = (size_t)H->ncell, np = (size_t)H->np;
        const int cur = H->parity;
        size_t o = 0;
        CU(cudaMemcpyAsync(buf + o, f[cur], sizeof(S) * pop_slots(), cudaMemcpyDeviceToHost, st));
        o += sizeof(S) * pop_slots();
        for (int a = 0; a < D; ++a) {
            CU(cudaMemcpyAsync(buf + o, part[cur].P[a], sizeof(double) * np, cudaMemcpyDeviceToHost, st));
            o += sizeof(double) * np;
            CU(cudaMemcpyAsync(buf + o, part[cur].v[a], sizeof(Real) * np, cudaMemcpyDeviceToHost, st));
            o += sizeof(Real) * np;
            CU(cudaMemcpyAsync(buf + o, part[cur].off[a], sizeof(Real) * np, cudaMemcpyDeviceToHost, st));
            o += sizeof(Real) * np;
        }
        CU(cudaMemcpyAsync(buf + o, part[cur].id, sizeof(int) * np, cudaMemcpyDeviceToHost, st));
        o += sizeof(int) * np;
        CU(cudaMemcpyAsync(buf + o, part[cur].cell, sizeof(int) * np, cudaMemcpyDeviceToHost, st));
        o += sizeof(int) * np;
        CU(cudaMemcpyAsync(buf + o, cl_local[cur], sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost, st));
        o += sizeof(int) * (nc + 1);
        CU(cudaMemcpyAsync(buf + o, cl_base[cur], sizeof(int) * (cell_tiles(H->ncell) + 1),
                           cudaMemcpyDeviceToHost, st));
        o += sizeof(int) * (cell_tiles(H->ncell) + 1);
        CU(cudaMemcpyAsync(buf + o, solids_out, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        o += sizeof(unsigned long long);
        for (int c = 0; c < NW && H->friction; ++c) {
            CU(cudaMemcpyAsync(buf + o, part[cur].w[c], sizeof(Real) * np, cudaMemcpyDeviceToHost, st));
            o += sizeof(Real) * np;
        }
        CU(cudaStreamSynchronize(st));
        return LBDPS_OK;
    }

    int load(const char *buf) override
    {
        cudaStream_t st = H->stream;
        const size_t nc = (size_t)H->ncell, np = (size_t)H->np;
        const int cur = H->parity;
        size_t o = 0;
        CU(cudaMemcpyAsync(f[cur], buf + o, sizeof(S) * pop_slots(), cudaMemcpyHostToDevice, st));
        o += sizeof(S) * pop_slots();
        for (int a = 0; a < D; ++a) {
            CU(cudaMemcpyAsync(part[cur].P[a], buf + o, sizeof(double) * np, cudaMemcpyHostToDevice, st));
            o += sizeof(double) * np;
            CU(cudaMemcpyAsync(part[cur].v[a], buf + o, sizeof(Real) * np, cudaMemcpyHostToDevice, st));
            o += sizeof(Real) * np;
            CU(cudaMemcpyAsync(part[cur].off[a], buf + o, sizeof(Real) * np, cudaMemcpyHostToDevice, st));
            o += sizeof(Real) * np;
        }
        CU(cudaMemcpyAsync(part[cur].id, buf + o, sizeof(int) * np, cudaMemcpyHostToDevice, st));
        o += sizeof(int) * np;
        CU(cudaMemcpyAsync(part[cur].cell, buf + o, sizeof(int) * np, cudaMemcpyHostToDevice, st));
        o += sizeof(int) * np;
        CU(cudaMemcpyAsync(cl_local[cur], buf + o, sizeof(int) * (nc + 1), cudaMemcpyHostToDevice, st));
        o += sizeof(int) * (nc + 1);
        CU(cudaMemcpyAsync(cl_base[cur], buf + o, sizeof(int) * (cell_tiles(H->ncell) + 1),
                           cudaMemcpyHostToDevice, st));
        o += sizeof(int) * (cell_tiles(H->ncell) + 1);
        CU(cudaMemcpyAsync(solids_out, buf + o, sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
        o += sizeof(unsigned long long);
        for (int c = 0; c < NW && H->friction; ++c) {
            CU(cudaMemcpyAsync(part[cur].w[c], buf + o, sizeof(Real) * np, cudaMemcpyHostToDevice, st));
            o += sizeof(Real) * np;
        }
        CU(cudaMemsetAsync(counts, 0, sizeof(int) * (nc + 1), st));
        CU(cudaStreamSynchronize(st));
        return LBDPS_OK;
    }

    int batch_describe(BatchBed *out) override
    {
        if constexpr (D == 2 && std::is_same<Real, float>::value) {
            if (H->soft) return LBDPS_ERR_INVALID;
            BatchBed b{};
            b.sp = sp;
            b.lay = lay;
            for (int p = 0; p < 2; ++p) {
                b.f[p] = f[p];
                b.cl_local[p] = cl_local[p];
                b.cl_base[p] = cl_base[p];
                b.cl_shift = cell_tile_log2(H->ncell);
                b.part[p] = part[p];
            }
            b.tile_total = tile_total;
            b.ticket = ticket;
            b.stage = stage;
            b.fld = fld;
            b.key = key;
            b.counts = counts;
            b.idslot = idslot;
            b.slot = slot;
            b.best = best;
            b.wall = wall;
            b.diag_fpre = diag_fpre;
            b.diag_fd = diag_fd;
            b.np = H->np;
            b.ncell = H->ncell;
            b.storage = std::is_same<S, __half>::value ? ST_F16
                        : std::is_same<S, __nv_bfloat16>::value ? ST_BF16 : ST_F32;
            *out = b;
            return LBDPS_OK;
        } else {
            (void)out;
            return LBDPS_ERR_INVALID;
        }
    }
};

template <class L>
Engine *make_engine_l(lbdps *h)
{
    switch (h->prm.storage) {
    case ST_F64: return new (std::nothrow) EngineT<L, double, double>(h);
    case ST_F32: return new (std::nothrow) EngineT<L, float, float>(h);
    case ST_F16: return new (std::nothrow) EngineT<L, float, __half>(h);
    case ST_BF16: return new (std::nothrow) EngineT<L, float, __nv_bfloat16>(h);
    }
    return nullptr;
}

// ---------------------------------------------------------------------------
// Validation helpers.
// ---------------------------------------------------------------------------
// positions of the caller (id order, interleaved) inside the lattice once
// divided by pos_div (the cell size for SI positions, 1 for lattice units)
int validate_positions(const lbdps *h, const double *pos, double pos_div)
{
    const int D = h->dim, np = h->np;
    // below safe[a] = (n_a - 1) pos_div a coordinate is inside without the
    // division: x < fl((n - 1) h) gives fl(x / h) <= (n - 1)(1 + 2^-52)^2 < n
    double safe[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D; ++a) safe[a] = (double)(h->n[a] - 1) * pos_div;
    // the first particle (smallest index) outside the domain, as one loop
    // in index order would find it
    std::mutex mu;
    size_t first = SIZE_MAX;
    host_parallel((size_t)np, [&](size_t lo, size_t hi) {
        for (size_t i = lo; i < hi; ++i) {
            for (int a = 0; a < D; ++a) {
                const double x = pos[i * D + a];
                if (x >= 0.0 && x < safe[a]) continue;
                const double p = x / pos_div;
                if (!(p >= 0.0 && p < (double)h->n[a])) {
                    std::lock_guard<std::mutex> lock(mu);
                    first = std::min(first, i * D + a);
                    return;
                }
            }
        }
    });
    if (first != SIZE_MAX)
        return fail(LBDPS_ERR_INVALID, "particle %d lies outside the domain on axis %d",
                    (int)(first / D), (int)(first % D));
    return LBDPS_OK;
}

// Steps replayed by one launch of a chunk graph when a call asks for at least
// as many (an even count, so a chunk ends on the parity it started from).
constexpr int kChunkSteps = 16;

int capture_steps(lbdps *h, int nsteps, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = LBDPS_OK;
    for (int s = 0; s < nsteps && rc == LBDPS_OK; ++s) rc = h->eng->enqueue_step((h->parity + s) & 1, nullptr);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(LBDPS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(LBDPS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return LBDPS_OK;
}

// one step from parity h->parity followed by the snapshot into slot parity
int capture_monitored_step(lbdps *h, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = h->eng->enqueue_step(h->parity, nullptr, true);
    if (rc == LBDPS_OK) rc = h->eng->enqueue_snapshot(h->parity);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(LBDPS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(LBDPS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return LBDPS_OK;
}

int check_health(lbdps *h)
{
    int hw = 0;
    int rc = lbdps_health(h, &hw);
    if (rc) return rc;
    if (hw & HEALTH_DIVERGED) return fail(LBDPS_ERR_DIVERGED, "gas state diverged by step %lld", (long long)h->steps);
    if (hw & HEALTH_DOMAIN) return fail(LBDPS_ERR_DOMAIN, "a particle left the domain by step %lld", (long long)h->steps);
    return LBDPS_OK;
}

int run_steps(lbdps *h, int64_t nsteps)
{
    const int ce = h->prm.check_every;
    for (int64_t s = 0; s < nsteps;) {
        // a chunk when the call and the next health check leave room for one
        const bool chunk = h->prm.use_graph && nsteps - s >= kChunkSteps &&
                           (ce <= 0 || ce - h->since_check >= kChunkSteps);
        if (chunk) {
            if (!h->chunk[h->parity]) {
                int rc = capture_steps(h, kChunkSteps, &h->chunk[h->parity]);
                if (rc) return rc;
            }
            CU(cudaGraphLaunch(h->chunk[h->parity], h->stream));
            s += kChunkSteps;
            h->steps += kChunkSteps;
            if (ce > 0) h->since_check += kChunkSteps;
        } else {
            if (h->prm.use_graph) {
                if (!h->graph[h->parity]) {
                    int rc = capture_steps(h, 1, &h->graph[h->parity]);
                    if (rc) return rc;
                }
                CU(cudaGraphLaunch(h->graph[h->parity], h->stream));
            } else {
                int rc = h->eng->enqueue_step(h->parity, nullptr);
                if (rc) return rc;
            }
            h->parity ^= 1;
            s += 1;
            h->steps++;
            if (ce > 0) h->since_check += 1;
        }
        if (ce > 0 && h->since_check >= ce) {
            h->since_check = 0;
            int rc = check_health(h);
            if (rc) return rc;
        }
    }
    return LBDPS_OK;
}

// One statistics record from the kStatOut doubles of the reduction: the
// health word and the outlet count travel as raw 64-bit words at the end.
void decode_stats(lbdps *h, const double *v, bool bed, int64_t steps, lbdps_stats_t *out)
{
    const int D = h->dim;
    unsigned long long raw[2] = {0, 0};
    std::memcpy(raw, v + kStatValues, sizeof(raw));
    *h->health_host = (unsigned)raw[0];
    out->solids_out = (int64_t)raw[1];
    out->mass = v[0] + (double)h->ncell;
    for (int a = 0; a < 3; ++a) {
        out->gas_momentum[a] = a < D ? v[1 + a] : 0.0;
        out->particle_momentum[a] = a < D ? v[4 + a] : 0.0;
    }
    out->mean_eps_g = v[7] / (double)h->ncell;
    out->mean_slip = bed ? (v[10] > 0 ? v[9] / v[10] : 0.0) : NAN;
    out->steps = steps;
    out->health = (int)raw[0];
}

// Records of the pinned ring used by lbdps_step_monitored: the host waits
// once per kMonSteps steps.
constexpr int kMonSteps = 1024;

// Monitored steps with the statistics fused into the next collision.  The
// statistics of the state after step s need the gas mass and momentum of
// that state, which the collision of step s + 1 reads anyway: its graph
// (capture_monitored_step) has the collision write the per-warp moment
// sums of its input state into that parity's gas partials.  The reduction of
// the state after step s then runs right after step s + 1 on the same
// stream; it reads only those partials, the cell list and the particles of
// that state (step s + 1 writes the other buffers) and the health word and
// outlet count that the graph of step s snapshotted at its end.  The state
// after the last step gets its gas partials from one k_gas_moments pass.
int run_monitored_fused(lbdps *h, int64_t nsteps, lbdps_stats_t *out)
{
    int64_t done = 0;   // records written to out
    while (done < nsteps) {
        const int k = (int)std::min<int64_t>(kMonSteps, nsteps - done);
        // states after steps done + 1 .. done + k; the first step of the
        // batch also writes the partials of the state before it (unused)
        int prev = -1;   // parity of the state whose reduction is due
        for (int t = 0; t < k; ++t) {
            const int p = h->parity;
            if (!h->mon_graph[p]) {
                int rc = capture_monitored_step(h, &h->mon_graph[p]);
                if (rc) return rc;
            }
            CU(cudaGraphLaunch(h->mon_graph[p], h->stream));
            if (prev >= 0) {
                // the state before this step (parity p), made by the step
                // whose graph snapshotted into slot 1 - p
                int rc = h->eng->enqueue_stats_of(h->mon_host + (size_t)(t - 1) * kStatOut, p, 1 - p);
                if (rc) return rc;
            }
            h->parity ^= 1;
            h->steps++;
            prev = h->parity;
        }
        // the state after the batch's last step: its own moment pass
        int rc = h->eng->enqueue_stats(h->mon_host + (size_t)(k - 1) * kStatOut);
        if (rc) return rc;
        CU(cudaStreamSynchronize(h->stream));
        for (int t = 0; t < k; ++t)
            decode_stats(h, h->mon_host + (size_t)t * kStatOut, false, h->steps - k + 1 + t, out + done + t);
        done += k;
        // the health word of the last record, as lbdps_step checks it
        if (h->prm.check_every > 0) {
            const int hw = out[done - 1].health;
            if (hw & HEALTH_DIVERGED)
                return fail(LBDPS_ERR_DIVERGED, "gas state diverged by step %lld", (long long)h->steps);
            if (hw & HEALTH_DOMAIN)
                return fail(LBDPS_ERR_DOMAIN, "a particle left the domain by step %lld", (long long)h->steps);
        }
    }
    return LBDPS_OK;
}

int run_monitored(lbdps *h, int64_t nsteps, lbdps_stats_t *out)
{
    if (!h->mon_host) {
        if (cudaHostAlloc(&h->mon_host, sizeof(double) * kStatOut * kMonSteps, cudaHostAllocMapped) !=
            cudaSuccess) {
            cudaGetLastError();
            h->mon_host = nullptr;
            return fail(LBDPS_ERR_OOM, "pinned host allocation failed");
        }
    }
    // node diagnostics are rewritten by every step: with them, each
    // reduction runs before the next step on the handle's stream
    if (h->prm.use_graph && !h->prm.diagnostics) return run_monitored_fused(h, nsteps, out);
    for (int64_t s = 0; s < nsteps;) {
        const int k = (int)std::min<int64_t>(kMonSteps, nsteps - s);
        for (int t = 0; t < k; ++t) {
            int rc = run_steps(h, 1);
            if (rc) return rc;
            rc = h->eng->enqueue_stats(h->mon_host + (size_t)t * kStatOut);
            if (rc) return rc;
        }
        CU(cudaStreamSynchronize(h->stream));
        const bool bed = h->prm.diagnostics;
        for (int t = 0; t < k; ++t)
            decode_stats(h, h->mon_host + (size_t)t * kStatOut, bed, h->steps - k + 1 + t, out + s + t);
        s += k;
    }
    return LBDPS_OK;
}

void free_graphs(lbdps *h)
{
    for (int p = 0; p < 2; ++p) {
        if (h->mon_graph[p]) {
            cudaGraphExecDestroy(h->mon_graph[p]);
            h->mon_graph[p] = nullptr;
        }
        if (h->graph[p]) {
            cudaGraphExecDestroy(h->graph[p]);
            h->graph[p] = nullptr;
        }
        if (h->chunk[p]) {
            cudaGraphExecDestroy(h->chunk[p]);
            h->chunk[p] = nullptr;
        }
    }
}

}  // namespace

// Lets other translation units of the library report a failure through
// lbdps_last_error().
namespace lbdpsk {
void set_last_error(const char *msg) { g_last_error = msg; }

int batch_describe(lbdps *h, BatchBed *out)
{
    if (!h || !h->eng || !out) return LBDPS_ERR_INVALID;
    return h->eng->batch_describe(out);
}

void batch_advanced(lbdps *h, long long nsteps)
{
    h->parity ^= (int)(nsteps & 1);
    h->steps += nsteps;
}

cudaStream_t bed_stream(lbdps *h) { return h->stream; }
int bed_parity(lbdps *h) { return h->parity; }
}  // namespace lbdpsk

namespace {

struct CkptHeader {
    char magic[8];
    int dim, q, storage, n[3], np, ncell;
    long long steps;
    unsigned long long payload;
};

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

}  // extern "C"

// Validation and derived constants of a description, the particles checked
// in place (no device work; the conversion to lattice units happens on the
// device as they are loaded).  Shared by lbdps_create and
// lbdps_memory_estimate.
static int prepare_bed(const lbdps_lattice_desc *lat, const lbdps_particle_desc *par,
                       const lbdps_params *prm, std::unique_ptr<lbdps> &hout)
{
    if (!lat || !par || !prm) return fail(LBDPS_ERR_INVALID, "NULL description");
    const int D = lat->dim;
    if (D != 2 && D != 3) return fail(LBDPS_ERR_INVALID, "dim must be 2 or 3");
    long long ncell = 1;
    int n[3] = {1, 1, 1};
    for (int a = 0; a < D; ++a) {
        if (lat->n[a] < 1) return fail(LBDPS_ERR_INVALID, "n[%d] must be positive", a);
        n[a] = lat->n[a];
        ncell *= n[a];
    }
    const int Q = D == 2 ? 9 : 19;
    if (ncell >= (1ll << 31) - 1 || ncell * Q >= (1ll << 40))
        return fail(LBDPS_ERR_INVALID, "lattice too large");
    int bc[6];
    for (int f6 = 0; f6 < 6; ++f6) bc[f6] = lat->bc[f6];
    if (D == 2) bc[4] = bc[5] = BC_PERIODIC;
    for (int a = 0; a < D; ++a) {
        for (int s = 0; s < 2; ++s)
            if (bc[2 * a + s] < 0 || bc[2 * a + s] > 3)
                return fail(LBDPS_ERR_INVALID, "unknown face type on face %d", 2 * a + s);
        if ((bc[2 * a] == BC_PERIODIC) != (bc[2 * a + 1] == BC_PERIODIC))
            return fail(LBDPS_ERR_INVALID, "axis %d: periodic faces must come in pairs", a);
        if (bc[2 * a] == BC_PERIODIC && n[a] < 3)
            return fail(LBDPS_ERR_INVALID, "axis %d: periodic axes need at least 3 cells", a);
        const bool open = bc[2 * a] >= BC_INLET || bc[2 * a + 1] >= BC_INLET;
        if (open && a != D - 1)
            return fail(LBDPS_ERR_INVALID, "inlet/outlet faces only on the vertical axis");
    }
    if (bc[2 * (D - 1)] == BC_INLET && bc[2 * (D - 1) + 1] == BC_INLET)
        return fail(LBDPS_ERR_INVALID, "at most one inlet face");
    if (!(lat->h > 0) || !(lat->dt > 0)) return fail(LBDPS_ERR_INVALID, "h and dt must be positive");
    if (par->n < 0 || par->n >= (1ll << 31) - 1) return fail(LBDPS_ERR_INVALID, "bad particle count");
    if (par->n > 0 && (!par->pos || !par->vel)) return fail(LBDPS_ERR_INVALID, "NULL particle arrays");
    if (!(par->d_p > 0) || !(par->rho_s > 0) || !(par->e >= 0 && par->e <= 1))
        return fail(LBDPS_ERR_INVALID, "bad particle properties");
    if (!(par->d_p <= lat->h)) return fail(LBDPS_ERR_INVALID, "d_p must not exceed h");
    if (par->recirculate != 0 && par->recirculate != 1) return fail(LBDPS_ERR_INVALID, "bad recirculate");
    if (par->collision_model != LBDPS_COLLIDE_HARD && par->collision_model != LBDPS_COLLIDE_SOFT)
        return fail(LBDPS_ERR_INVALID, "bad collision_model");
    const bool soft = par->collision_model == LBDPS_COLLIDE_SOFT;
    if (soft && !(par->dem_kn > 0 && std::isfinite(par->dem_kn)))
        return fail(LBDPS_ERR_INVALID, "soft spheres need dem_kn > 0");
    if (soft && !(par->e > 0)) return fail(LBDPS_ERR_INVALID, "soft spheres need e > 0");
    if (!(par->dem_mu >= 0 && std::isfinite(par->dem_mu)) ||
        !(par->dem_gamma_t >= 0 && std::isfinite(par->dem_gamma_t)))
        return fail(LBDPS_ERR_INVALID, "dem_mu and dem_gamma_t must be finite and >= 0");
    const bool friction = par->dem_mu > 0 && par->dem_gamma_t > 0;
    if (friction && !soft) return fail(LBDPS_ERR_INVALID, "friction needs soft spheres");
    if (par->recirculate && !(bc[2 * (D - 1)] == BC_INLET && bc[2 * (D - 1) + 1] == BC_OUTLET))
        return fail(LBDPS_ERR_INVALID, "recirculate needs the inlet below and the outlet above");
    if (!(prm->rho_g > 0) || !(prm->mu_g > 0)) return fail(LBDPS_ERR_INVALID, "bad gas properties");
    if (prm->storage < 0 || prm->storage > 3) return fail(LBDPS_ERR_INVALID, "bad storage");
    if (!(prm->cs_smag >= 0)) return fail(LBDPS_ERR_INVALID, "bad Smagorinsky constant");
    if (prm->superficial_mode < 0 || prm->superficial_mode > 2)
        return fail(LBDPS_ERR_INVALID, "bad superficial_mode");

    std::unique_ptr<lbdps> h(new (std::nothrow) lbdps());
    if (!h) return fail(LBDPS_ERR_OOM, "host allocation failed");
    h->dim = D;
    h->q = Q;
    for (int a = 0; a < 3; ++a) h->n[a] = n[a];
    h->ncell = (int)ncell;
    h->np = (int)par->n;
    for (int f6 = 0; f6 < 6; ++f6) h->bc[f6] = bc[f6];
    h->h = lat->h;
    h->dt = lat->dt;
    h->recirculate = par->recirculate;
    h->soft = soft;
    h->friction = friction;
    h->prm = *prm;
    h->k = derive(*lat, *par, *prm);
    const Derived &k = h->k;
    if (!(k.tau > 0.5) || !std::isfinite(k.tau)) return fail(LBDPS_ERR_INVALID, "tau must exceed 1/2");
    // a pair contact (half a period of the undamped spring with the reduced
    // mass m_p / 2) must span a few steps for the explicit update to hold it
    if (soft && !(kPi * std::sqrt(0.5 * k.mp / k.kn) >= 4.0))
        return fail(LBDPS_ERR_INVALID, "dem_kn too stiff: a pair contact lasts %.3g steps (at least 4)",
                    kPi * std::sqrt(0.5 * k.mp / k.kn));
    // the viscous friction of a sliding pair damps the slip by gamma_t
    // (2 / m_p + 2 r^2 / I) = 7 gamma_t / m_p per step: explicit updates need
    // it well below 2
    if (friction && !(k.gamma_t <= 0.25 * k.mp))
        return fail(LBDPS_ERR_INVALID, "dem_gamma_t too large: %.3g m_p per step (at most 0.25)",
                    k.gamma_t / k.mp);
    double u0s = 0;
    for (int a = 0; a < D; ++a) u0s += k.u0[a] * k.u0[a];
    if (!(u0s < 0.09)) return fail(LBDPS_ERR_INVALID, "|u0| must be below 0.3 in lattice units");
    // count tables reach the close-packing cap
    const double unit = D == 2 ? kPi * k.r * k.r : k.vp;
    const double cap = D == 2 ? kPi / (2.0 * std::sqrt(3.0)) : kPi / (3.0 * std::sqrt(2.0));
    const double ncap = std::ceil(cap / unit);
    if (!(ncap < 4000)) return fail(LBDPS_ERR_INVALID, "particles too small for the cell (d_p/h)");
    h->ntab = (int)ncap + 2;
    // inlet velocities
    int inlet_face = -1;
    for (int f6 = 0; f6 < 6; ++f6)
        if (bc[f6] == BC_INLET) inlet_face = f6;
    if (inlet_face >= 0) {
        const int nface = (int)(ncell / n[D - 1]);
        h->inlet_lat.assign((size_t)nface * D, 0.0);
        if (lat->inlet_u) {
            const double us = lat->dt / lat->h;
            for (int j = 0; j < nface; ++j) {
                double s = 0;
                for (int a = 0; a < D; ++a) {
                    const double u = lat->inlet_u[(size_t)j * D + a] * us;
                    h->inlet_lat[(size_t)j * D + a] = u;
                    s += u * u;
                }
                if (!(s < 0.09)) return fail(LBDPS_ERR_INVALID, "inlet |u| must be below 0.3 in lattice units");
            }
        }
    }
    // particles inside the lattice (positions in lattice units are pos / h)
    int rc = validate_positions(h.get(), par->pos, lat->h);
    if (rc) return rc;
    hout = std::move(h);
    return LBDPS_OK;
}

extern "C" {

int lbdps_memory_estimate(const lbdps_lattice_desc *lat, const lbdps_particle_desc *par,
                          const lbdps_params *prm, size_t *bytes)
{
    if (!bytes) return fail(LBDPS_ERR_INVALID, "bytes is NULL");
    std::unique_ptr<lbdps> h;
    int rc = prepare_bed(lat, par, prm, h);
    if (rc) return rc;
    h->mem.count_only = true;
    h->eng.reset(h->dim == 2 ? make_engine_l<D2Q9>(h.get()) : make_engine_l<D3Q19>(h.get()));
    if (!h->eng) return fail(LBDPS_ERR_OOM, "engine allocation failed");
    rc = h->eng->allocate(h->mem);
    if (rc) return rc;
    *bytes = h->mem.counted;
    return LBDPS_OK;
}

int lbdps_create(const lbdps_lattice_desc *lat, const lbdps_particle_desc *par,
                 const lbdps_params *prm, lbdps_t **out)
{
    if (!out) return fail(LBDPS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    std::unique_ptr<lbdps> h;
    // the pairwise overlap test of hard spheres runs on the device once the
    // particles are sorted (below); the host checks the domain only
    int rc = prepare_bed(lat, par, prm, h);
    if (rc) return rc;
    const int D = h->dim;

    if (prm->stream) {
        h->stream = (cudaStream_t)prm->stream;
    } else {
        CU(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    h->mem.alloc = prm->alloc;
    h->mem.release = prm->free;
    h->mem.ctx = prm->alloc_ctx;
    h->mem.stream = h->stream;
    h->eng.reset(D == 2 ? make_engine_l<D2Q9>(h.get()) : make_engine_l<D3Q19>(h.get()));
    if (!h->eng) return fail(LBDPS_ERR_OOM, "engine allocation failed");
    auto cleanup = [&](int code) {
        if (h->stream) cudaStreamSynchronize(h->stream);
        h->mem.release_all();
        if (h->own_stream) cudaStreamDestroy(h->stream);
        return code;
    };
    // one block for all of the bed's buffers, sized by a counting pass of
    // the same allocation
    h->mem.count_only = true;
    rc = h->eng->allocate(h->mem);
    h->mem.count_only = false;
    if (rc) return cleanup(rc);
    if (!h->mem.begin_slab(h->mem.counted)) {
        if (h->mem.misaligned)
            return cleanup(fail(LBDPS_ERR_INVALID, "params.alloc returned a block that is not 256-byte aligned"));
        return cleanup(fail(LBDPS_ERR_OOM, "device allocation of %zu bytes failed", h->mem.counted));
    }
    rc = h->eng->allocate(h->mem);
    h->mem.end_slab();
    if (rc) return cleanup(rc);
    // mapped: the statistics reduction writes its results here directly
    if (cudaHostAlloc(&h->health_host, 256, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(LBDPS_ERR_OOM, "pinned allocation failed"));
    }
    static_assert(sizeof(double) * kStatOut <= 128, "statistics fit the pinned block");
    h->stats_host = reinterpret_cast<double *>(reinterpret_cast<char *>(h->health_host) + 128);
    if ((rc = h->eng->upload_initial(par->pos, par->vel, lat->h, lat->dt / lat->h))) {
        cudaFreeHost(h->health_host);
        return cleanup(rc);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaFreeHost(h->health_host);
        return cleanup(fail(LBDPS_ERR_CUDA, "create: %s", cudaGetErrorString(cudaGetLastError())));
    }
    if (!h->soft && h->np > 1) {
        unsigned long long novl = 0;
        int oi = 0, oj = 0;
        if ((rc = h->eng->overlaps(&novl, &oi, &oj))) {
            cudaFreeHost(h->health_host);
            return cleanup(rc);
        }
        if (novl > 0) {
            cudaFreeHost(h->health_host);
            return cleanup(fail(LBDPS_ERR_INVALID, "particles %d and %d overlap (%llu overlapping pairs)",
                                oi, oj, novl));
        }
    }
    *out = h.release();
    return LBDPS_OK;
}

void lbdps_destroy(lbdps_t *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_graphs(h);
    h->eng.reset();
    h->mem.release_all();
    if (h->health_host) cudaFreeHost(h->health_host);
    if (h->mon_host) cudaFreeHost(h->mon_host);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int lbdps_step(lbdps_t *h, int64_t nsteps)
{
    if (!h || nsteps < 0) return fail(LBDPS_ERR_INVALID, "bad arguments");
    return run_steps(h, nsteps);
}

int lbdps_step_monitored(lbdps_t *h, int64_t nsteps, lbdps_stats_t *out)
{
    if (!h || nsteps < 0 || (nsteps > 0 && !out)) return fail(LBDPS_ERR_INVALID, "bad arguments");
    return run_monitored(h, nsteps, out);
}

int lbdps_step_profiled(lbdps_t *h, int64_t nsteps, double *kernel_ms, int cap, int *nclass)
{
    if (!h || nsteps < 0 || (!kernel_ms && cap > 0)) return fail(LBDPS_ERR_INVALID, "bad arguments");
    constexpr int kClasses = 4;
    if (nclass) *nclass = kClasses;
    cudaEvent_t ev[kStepEvents];
    for (int e = 0; e < kStepEvents; ++e) CU(cudaEventCreate(&ev[e]));
    double acc[kClasses] = {0, 0, 0, 0};
    int rc = LBDPS_OK;
    for (int64_t s = 0; s < nsteps && rc == LBDPS_OK; ++s) {
        rc = h->eng->enqueue_step(h->parity, ev);
        if (rc) break;
        if (cudaEventSynchronize(ev[kStepEvents - 1]) != cudaSuccess) {
            rc = fail(LBDPS_ERR_CUDA, "profiling: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        for (int c = 0; c + 1 < kStepEvents; ++c) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[c], ev[c + 1]);
            acc[kStepEventClass[c]] += ms;
        }
        h->parity ^= 1;
        h->steps++;
    }
    for (int e = 0; e < kStepEvents; ++e) cudaEventDestroy(ev[e]);
    for (int c = 0; c < kClasses && c < cap; ++c) kernel_ms[c] = acc[c];
    return rc;
}

int lbdps_record_event(lbdps_t *h, void *event)
{
    if (!h || !event) return fail(LBDPS_ERR_INVALID, "bad arguments");
    CU(cudaEventRecord((cudaEvent_t)event, h->stream));
    return LBDPS_OK;
}

int lbdps_sync(lbdps_t *h)
{
    if (!h) return fail(LBDPS_ERR_INVALID, "NULL handle");
    CU(cudaStreamSynchronize(h->stream));
    return LBDPS_OK;
}

int lbdps_fields(lbdps_t *h, int mask, int units, double *out, size_t cap)
{
    if (!h || !out) return fail(LBDPS_ERR_INVALID, "bad arguments");
    CU(cudaStreamSynchronize(h->stream));
    return h->eng->fields(mask, units, out, cap);
}

int lbdps_particles(lbdps_t *h, int units, double *pos, double *vel, int64_t cap)
{
    if (!h) return fail(LBDPS_ERR_INVALID, "NULL handle");
    CU(cudaStreamSynchronize(h->stream));
    return h->eng->particles(units, pos, vel, cap);
}

int lbdps_set_particles(lbdps_t *h, int64_t n, const double *pos, const double *vel)
{
    if (!h || (n > 0 && (!pos || !vel))) return fail(LBDPS_ERR_INVALID, "bad arguments");
    if (n != h->np) return fail(LBDPS_ERR_INVALID, "particle count must stay %d", h->np);
    int rc = validate_positions(h, pos, 1.0);
    if (rc) return rc;
    CU(cudaStreamSynchronize(h->stream));
    rc = h->eng->set_particles(pos, vel);
    if (rc) return rc;
    CU(cudaStreamSynchronize(h->stream));
    return LBDPS_OK;
}

int lbdps_particle_spin(lbdps_t *h, int units, double *out, int64_t cap)
{
    if (!h || !out) return fail(LBDPS_ERR_INVALID, "bad arguments");
    CU(cudaStreamSynchronize(h->stream));
    return h->eng->spin(units, out, cap);
}

int lbdps_set_particle_spin(lbdps_t *h, const double *in, int64_t n)
{
    if (!h || (n > 0 && !in)) return fail(LBDPS_ERR_INVALID, "bad arguments");
    if (n != h->np) return fail(LBDPS_ERR_INVALID, "particle count must stay %d", h->np);
    CU(cudaStreamSynchronize(h->stream));
    return h->eng->set_spin(in);
}

int lbdps_populations(lbdps_t *h, double *f, size_t cap)
{
    if (!h || !f) return fail(LBDPS_ERR_INVALID, "bad arguments");
    CU(cudaStreamSynchronize(h->stream));
    return h->eng->populations(f, cap);
}

int lbdps_set_populations(lbdps_t *h, const double *f, size_t count)
{
    if (!h || !f) return fail(LBDPS_ERR_INVALID, "bad arguments");
    CU(cudaStreamSynchronize(h->stream));
    return h->eng->set_populations(f, count);
}

int lbdps_particle_diag(lbdps_t *h, int which, double *out, size_t cap)
{
    if (!h || !out) return fail(LBDPS_ERR_INVALID, "bad arguments");
    CU(cudaStreamSynchronize(h->stream));
    return h->eng->particle_diag(which, out, cap);
}

int lbdps_collide_particles(lbdps_t *h, int64_t *pairs, int64_t cap, int64_t *npairs)
{
    if (!h || cap < 0) return fail(LBDPS_ERR_INVALID, "bad arguments");
    CU(cudaStreamSynchronize(h->stream));
    return h->eng->collide_particles(pairs, cap, npairs);
}

int lbdps_stats(lbdps_t *h, lbdps_stats_t *out)
{
    if (!h || !out) return fail(LBDPS_ERR_INVALID, "bad arguments");
    return h->eng->stats(out);
}

int lbdps_health(lbdps_t *h, int *health)
{
    if (!h || !health) return fail(LBDPS_ERR_INVALID, "bad arguments");
    unsigned hw = 0;
    int rc = h->eng->health(&hw);
    if (rc) return rc;
    *health = (int)hw;
    return LBDPS_OK;
}

int lbdps_check_guards(lbdps_t *h, int *damaged)
{
    if (!h || !damaged) return fail(LBDPS_ERR_INVALID, "bad arguments");
    if (h->mem.damaged(h->stream, damaged)) return fail(LBDPS_ERR_CUDA, "guard read-back failed");
    return LBDPS_OK;
}

int lbdps_bubbles(lbdps_t *h, double threshold, int voidage, int64_t *out)
{
    if (!h || !out) return fail(LBDPS_ERR_INVALID, "bad arguments");
    if (!(threshold >= 0.0 && threshold < 1.0)) return fail(LBDPS_ERR_INVALID, "threshold must be in [0, 1)");
    if (voidage != LBDPS_VOIDAGE_2D && voidage != LBDPS_VOIDAGE_G)
        return fail(LBDPS_ERR_INVALID, "unknown voidage");
    return h->eng->bubbles(threshold, voidage, out);
}

int lbdps_set_inlet(lbdps_t *h, const double *inlet_u)
{
    if (!h || !inlet_u) return fail(LBDPS_ERR_INVALID, "bad arguments");
    if (h->inlet_lat.empty()) return fail(LBDPS_ERR_INVALID, "the bed has no inlet face");
    const int D = h->dim;
    const size_t nface = h->inlet_lat.size() / D;
    const double us = h->dt / h->h;
    std::vector<double> lat(h->inlet_lat.size());
    for (size_t j = 0; j < nface; ++j) {
        double s = 0.0;
        for (int a = 0; a < D; ++a) {
            const double u = inlet_u[j * D + a] * us;
            lat[j * D + a] = u;
            s += u * u;
        }
        if (!(s < 0.09)) return fail(LBDPS_ERR_INVALID, "inlet |u| must be below 0.3 in lattice units");
    }
    return h->eng->set_inlet(lat.data());
}

int lbdps_constants(lbdps_t *h, double *out, int cap)
{
    if (!h || !out) return fail(LBDPS_ERR_INVALID, "bad arguments");
    const Derived &k = h->k;
    const double v[25] = {k.tau, k.nu, k.mu, k.rho_s, k.d, k.r, k.vp, k.mp, k.e,
                          k.geff[0], k.geff[1], k.geff[2], k.fb[0], k.fb[1], k.fb[2],
                          k.u0[0], k.u0[1], k.u0[2], k.cs, k.kn, k.eta, k.eta_w, k.mu_f,
                          k.gamma_t, k.inertia};
    // the first 19 are always there; the soft-sphere constants follow when
    // there is room
    if (cap < 19) return fail(LBDPS_ERR_CAPACITY, "need 19 doubles");
    std::memcpy(out, v, sizeof(double) * (size_t)std::min(cap, 25));
    return LBDPS_OK;
}

int lbdps_shape(lbdps_t *h, int *dim, int *q, int64_t *ncell, int64_t *nparticles)
{
    if (!h) return fail(LBDPS_ERR_INVALID, "NULL handle");
    if (dim) *dim = h->dim;
    if (q) *q = h->q;
    if (ncell) *ncell = h->ncell;
    if (nparticles) *nparticles = h->np;
    return LBDPS_OK;
}

int lbdps_save(lbdps_t *h, void *buf, size_t cap, size_t *used)
{
    if (!h) return fail(LBDPS_ERR_INVALID, "NULL handle");
    const size_t need = sizeof(CkptHeader) + h->eng->checkpoint_bytes();
    if (used) *used = need;
    if (!buf) return LBDPS_OK;
    if (cap < need) return fail(LBDPS_ERR_CAPACITY, "checkpoint needs %zu bytes", need);
    CU(cudaStreamSynchronize(h->stream));
    CkptHeader hd{};
    std::memcpy(hd.magic, "LBDPSCK1", 8);
    hd.dim = h->dim;
    hd.q = h->q;
    hd.storage = h->prm.storage;
    for (int a = 0; a < 3; ++a) hd.n[a] = h->n[a];
    hd.np = h->np;
    hd.ncell = h->ncell;
    hd.steps = h->steps;
    hd.payload = h->eng->checkpoint_bytes();
    std::memcpy(buf, &hd, sizeof(hd));
    return h->eng->save((char *)buf + sizeof(hd));
}

int lbdps_load(lbdps_t *h, const void *buf, size_t size)
{
    if (!h || !buf || size < sizeof(CkptHeader)) return fail(LBDPS_ERR_INVALID, "bad arguments");
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, "LBDPSCK1", 8) != 0) return fail(LBDPS_ERR_INVALID, "not a checkpoint");
    if (hd.dim != h->dim || hd.q != h->q || hd.storage != h->prm.storage || hd.np != h->np ||
        hd.ncell != h->ncell || hd.n[0] != h->n[0] || hd.n[1] != h->n[1] || hd.n[2] != h->n[2])
        return fail(LBDPS_ERR_INVALID, "checkpoint shape differs from the handle");
    if (hd.payload != h->eng->checkpoint_bytes() || size < sizeof(hd) + hd.payload)
        return fail(LBDPS_ERR_INVALID, "checkpoint truncated");
    CU(cudaStreamSynchronize(h->stream));
    int rc = h->eng->load((const char *)buf + sizeof(hd));
    if (rc) return rc;
    h->steps = hd.steps;
    return LBDPS_OK;
}

const char *lbdps_strerror(int code)
{
    switch (code) {
    case LBDPS_OK: return "ok";
    case LBDPS_ERR_INVALID: return "invalid argument or description";
    case LBDPS_ERR_OOM: return "out of memory";
    case LBDPS_ERR_CAPACITY: return "capacity exceeded";
    case LBDPS_ERR_DIVERGED: return "gas state diverged";
    case LBDPS_ERR_DOMAIN: return "particle left the domain";
    case LBDPS_ERR_TIMEOUT: return "device wait timed out";
    case LBDPS_ERR_CUDA: return "CUDA runtime error";
    }
    return "unknown status";
}

const char *lbdps_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

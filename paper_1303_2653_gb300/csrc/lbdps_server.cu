// Continuous batching of independent beds (the serving loop).
//
// Requests (a bed description and a step count K) arrive at any time.  The
// server keeps a FIFO queue, admits the head request as soon as its exact
// device-memory footprint (lbdps_memory_estimate) fits in the HBM budget and
// an active slot is free, and keeps every admitted bed resident on the
// device.  A bed that has reached K steps is harvested: its FP64 statistics
// and completion time are recorded, its memory is released (or kept for the
// caller, see lbdps_server_take), and the freed budget admits the next
// requests.  Each bed's arithmetic is the same as when it runs alone.
//
// Small beds of the batched kind (2D, FP32 arithmetic with FP32, FP16 or
// BF16 population storage, hard spheres) advance together: one tick is a
// captured CUDA graph of steps_per_tick coupled steps in which each of the
// seven kernels of a step is one launch over all of them, persistent thread
// blocks walking a device work table of (bed, tile) entries.  The tables and
// their entry counts live in device memory, so the graph is captured once
// (again only when the tables outgrow their capacity); between ticks the
// beds' records (buffer parity at the start of the tick, steps to take in
// it) are uploaded, and when the set of batched beds changes, the tables.  A
// bed with fewer steps left than a tick takes only those; the kernels skip it
// for the rest of the tick.  Every other bed keeps a stream of its own and
// advances by replays of its own step graphs, overlapping with the batch.
#include "lbdps.h"
#include "lbdps_internal.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <climits>
#include <vector>

namespace lbdpsk {
void set_last_error(const char *msg);
}

namespace {

double now_s()
{
    using clock = std::chrono::steady_clock;
    static const clock::time_point t0 = clock::now();
    return std::chrono::duration<double>(clock::now() - t0).count();
}

struct Request {
    uint64_t id = 0;
    lbdps_lattice_desc lat{};
    lbdps_particle_desc par{};
    lbdps_params prm{};
    std::vector<double> pos, vel, inlet;
    int64_t steps = 0;
    size_t bytes = 0;
    int keep = 0;
    double t_submit = 0.0;
};

struct Active {
    Request req;
    lbdps_t *h = nullptr;
    int64_t issued = 0;
    double t_admit = 0.0;
    cudaEvent_t last = nullptr;   // recorded after the final step
    cudaEvent_t tick = nullptr;   // recorded after each tick
    bool tick_pending = false;
    bool batched = false;         // advanced by the batch (desc is its record)
    lbdpsk::BatchBed desc{};
    int64_t last_tick = 0;        // the batch tick that took its last steps so far
};

// The batched beds: their stream, the device copies of their records and
// work tables, and the captured tick.
struct Batch {
    bool ready = false;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;        // recorded after each tick
    bool pending = false;              // a tick is in flight
    lbdpsk::BatchBed *descs_dev = nullptr;
    lbdpsk::BatchBed *descs_host = nullptr;   // pinned staging of the records
    int2 *work_dev = nullptr;          // three sections of work_cap entries: cell, scan, particle tiles
    int2 *work_host = nullptr;         // pinned staging of the tables, then the counts
    int *count_dev = nullptr;          // entries of each section
    size_t work_cap = 0;
    cudaGraphExec_t graph = nullptr;   // captured once per table capacity
    bool dirty = true;                 // members changed: rewrite the tables
    std::vector<Active *> members;     // record k of descs_dev is members[k]
    lbdpsk::BatchWork work{};
    int64_t ticks = 0, captures = 0;
    int64_t done_ticks = 0;            // ticks known to have completed
};

// Beds up to this many cells may join the batch.  The batched kernels load
// each bed's parameters from device memory and cost 1.3-1.9x the single-bed
// kernels per bed-step, so batching pays where a bed's own launches are
// dominated by launch and dependent-load latency: on a GB300 the crossover
// measured on the mixed serving stream lies between 32,768 and 131,072 cells.
constexpr int kBatchMaxCells = 1 << 15;

int sfail(int code, const char *msg)
{
    lbdpsk::set_last_error(msg);
    return code;
}

}  // namespace

struct lbdps_server {
    size_t budget = 0, used = 0;
    int max_active = 0;
    int steps_per_tick = 1;
    uint64_t next_id = 1;
    std::deque<Request> queue;
    std::vector<std::unique_ptr<Active>> active;
    std::vector<lbdps_done_t> done;
    std::map<uint64_t, std::pair<lbdps_t *, size_t>> kept;
    double t0 = 0.0;
    bool batching = true;
    int batch_max_cells = kBatchMaxCells;
    Batch batch;
};

namespace {

// Stream, event and the device / pinned record arrays of the batch, on the
// first batched admission.
int batch_init(lbdps_server *s)
{
    Batch &b = s->batch;
    if (b.ready) return LBDPS_OK;
    const size_t bytes = sizeof(lbdpsk::BatchBed) * (size_t)s->max_active;
    if (cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc((void **)&b.descs_dev, bytes) != cudaSuccess ||
        cudaHostAlloc((void **)&b.descs_host, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return sfail(LBDPS_ERR_CUDA, "server: batch set-up failed");
    }
    // the launchers size their persistent grids on their first call: make
    // that call here, outside any capture (a null count launches nothing)
    lbdpsk::launch_collide_stream_batched(b.descs_dev, lbdpsk::BatchWork{}, 0, b.st);
    lbdpsk::launch_particles_batched(b.descs_dev, lbdpsk::BatchWork{}, 0, b.st);
    b.ready = true;
    return LBDPS_OK;
}

void batch_release(Batch &b)
{
    if (b.st) cudaStreamSynchronize(b.st);
    if (b.graph) cudaGraphExecDestroy(b.graph);
    if (b.work_dev) cudaFree(b.work_dev);
    if (b.work_host) cudaFreeHost(b.work_host);
    if (b.count_dev) cudaFree(b.count_dev);
    if (b.descs_dev) cudaFree(b.descs_dev);
    if (b.descs_host) cudaFreeHost(b.descs_host);
    if (b.done) cudaEventDestroy(b.done);
    if (b.st) cudaStreamDestroy(b.st);
    b = Batch{};
}

// Work tables of the current members, uploaded through pinned staging on the
// batch stream (no tick is in flight).  The tick's graph reads the tables
// and their entry counts from device memory, so it is captured again only
// when the tables outgrow their capacity.
int batch_rebuild(lbdps_server *s)
{
    Batch &b = s->batch;
    size_t n[3] = {0, 0, 0};
    for (Active *a : b.members) {
        const lbdpsk::BatchBed &d = a->desc;
        n[0] += (d.ncell + lbdpsk::kBatchTile - 1) / lbdpsk::kBatchTile;
        n[1] += lbdpsk::cell_tiles(d.ncell);
        n[2] += (d.np + lbdpsk::kBatchTile - 1) / lbdpsk::kBatchTile;
    }
    const size_t need = std::max({n[0], n[1], n[2], (size_t)1});
    if (need > b.work_cap) {
        size_t cap = std::max<size_t>(b.work_cap * 2, 1 << 14);
        while (cap < need) cap *= 2;
        if (b.work_dev) cudaFree(b.work_dev);
        if (b.work_host) cudaFreeHost(b.work_host);
        b.work_dev = nullptr;
        b.work_host = nullptr;
        b.work_cap = 0;
        if (!b.count_dev && cudaMalloc((void **)&b.count_dev, 4 * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return sfail(LBDPS_ERR_OOM, "server: batch work table allocation failed");
        }
        // three table sections, and two more entries of staging for the counts
        if (cudaMalloc((void **)&b.work_dev, sizeof(int2) * 3 * cap) != cudaSuccess ||
            cudaHostAlloc((void **)&b.work_host, sizeof(int2) * (3 * cap + 2), cudaHostAllocDefault) !=
                cudaSuccess) {
            cudaGetLastError();
            return sfail(LBDPS_ERR_OOM, "server: batch work table allocation failed");
        }
        b.work_cap = cap;
        if (b.graph) {
            cudaGraphExecDestroy(b.graph);
            b.graph = nullptr;
        }
    }
    int2 *sec[3] = {b.work_host, b.work_host + b.work_cap, b.work_host + 2 * b.work_cap};
    size_t m[3] = {0, 0, 0};
    for (size_t k = 0; k < b.members.size(); ++k) {
        const lbdpsk::BatchBed &d = b.members[k]->desc;
        const int bed = (int)k;
        for (int t = 0; t < (d.ncell + lbdpsk::kBatchTile - 1) / lbdpsk::kBatchTile; ++t)
            sec[0][m[0]++] = make_int2(bed, t);
        for (int t = 0; t < lbdpsk::cell_tiles(d.ncell); ++t) sec[1][m[1]++] = make_int2(bed, t);
        for (int t = 0; t < (d.np + lbdpsk::kBatchTile - 1) / lbdpsk::kBatchTile; ++t)
            sec[2][m[2]++] = make_int2(bed, t);
    }
    int *cnt = reinterpret_cast<int *>(b.work_host + 3 * b.work_cap);
    for (int k = 0; k < 3; ++k) cnt[k] = (int)m[k];
    bool ok = cudaMemcpyAsync(b.count_dev, cnt, 3 * sizeof(int), cudaMemcpyHostToDevice, b.st) ==
              cudaSuccess;
    for (int k = 0; k < 3 && ok; ++k)
        if (m[k])
            ok = cudaMemcpyAsync(b.work_dev + k * b.work_cap, sec[k], sizeof(int2) * m[k],
                                 cudaMemcpyHostToDevice, b.st) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return sfail(LBDPS_ERR_CUDA, "server: batch work table upload failed");
    }
    b.work.cell_tiles = b.work_dev;
    b.work.scan_tiles = b.work_dev + b.work_cap;
    b.work.part_tiles = b.work_dev + 2 * b.work_cap;
    b.work.count = b.count_dev;
    b.dirty = false;
    if (b.graph) return LBDPS_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return sfail(LBDPS_ERR_CUDA, "server: batch capture failed");
    }
    for (int step = 0; step < s->steps_per_tick; ++step) {
        lbdpsk::launch_collide_stream_batched(b.descs_dev, b.work, step, b.st);
        lbdpsk::launch_particles_batched(b.descs_dev, b.work, step, b.st);
    }
    cudaError_t e = cudaStreamEndCapture(b.st, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b.graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.graph = nullptr;
        b.dirty = true;
        return sfail(LBDPS_ERR_CUDA, "server: batch graph capture failed");
    }
    ++b.captures;
    return LBDPS_OK;
}

// Issue the next tick of the batch when none is in flight.
int batch_tick(lbdps_server *s)
{
    Batch &b = s->batch;
    if (!b.ready) return LBDPS_OK;
    if (b.pending) {
        const cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) return LBDPS_OK;
        if (q != cudaSuccess) return sfail(LBDPS_ERR_CUDA, "server: batch tick failed");
        b.pending = false;
        b.done_ticks = b.ticks;
    }
    std::vector<Active *> want;
    for (auto &a : s->active)
        if (a->batched && a->issued < a->req.steps) want.push_back(a.get());
    if (want.empty()) return LBDPS_OK;
    if (want != b.members) {
        b.members = want;
        b.dirty = true;
    }
    if (b.dirty) {
        int rc = batch_rebuild(s);
        if (rc) return rc;
    }
    for (size_t k = 0; k < b.members.size(); ++k) {
        Active &a = *b.members[k];
        lbdpsk::BatchBed d = a.desc;
        d.parity0 = lbdpsk::bed_parity(a.h);
        d.nsteps = (int)std::min<int64_t>(s->steps_per_tick, a.req.steps - a.issued);
        b.descs_host[k] = d;
    }
    if (cudaMemcpyAsync(b.descs_dev, b.descs_host, sizeof(lbdpsk::BatchBed) * b.members.size(),
                        cudaMemcpyHostToDevice, b.st) != cudaSuccess ||
        cudaGraphLaunch(b.graph, b.st) != cudaSuccess || cudaEventRecord(b.done, b.st) != cudaSuccess) {
        cudaGetLastError();
        return sfail(LBDPS_ERR_CUDA, "server: batch tick launch failed");
    }
    b.pending = true;
    ++b.ticks;
    for (size_t k = 0; k < b.members.size(); ++k) {
        Active &a = *b.members[k];
        const int n = b.descs_host[k].nsteps;
        a.issued += n;
        a.last_tick = b.ticks;
        lbdpsk::batch_advanced(a.h, n);
    }
    return LBDPS_OK;
}

int admit(lbdps_server *s)
{
    while (!s->queue.empty() && (int)s->active.size() < s->max_active &&
           s->used + s->queue.front().bytes <= s->budget) {
        Request &r = s->queue.front();
        std::unique_ptr<Active> a(new (std::nothrow) Active());
        if (!a) return sfail(LBDPS_ERR_OOM, "server: host allocation failed");
        a->req = std::move(r);
        s->queue.pop_front();
        Request &q = a->req;
        q.lat.inlet_u = q.inlet.empty() ? nullptr : q.inlet.data();
        q.par.pos = q.pos.data();
        q.par.vel = q.vel.data();
        q.prm.stream = nullptr;       // a stream of its own
        q.prm.use_graph = 1;
        lbdps_t *h = nullptr;
        int rc = lbdps_create(&q.lat, &q.par, &q.prm, &h);
        if (rc == LBDPS_ERR_OOM && !s->active.empty()) {
            // the allocator refused: retry when resident beds free memory
            s->queue.push_front(std::move(a->req));
            return LBDPS_OK;
        }
        if (rc != LBDPS_OK) {
            lbdps_done_t d{};
            d.id = q.id;
            d.status = rc;
            d.t_submit = q.t_submit - s->t0;
            d.t_done = now_s() - s->t0;
            s->done.push_back(d);
            continue;
        }
        if (cudaEventCreateWithFlags(&a->last, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&a->tick, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (a->last) cudaEventDestroy(a->last);
            lbdps_destroy(h);
            return sfail(LBDPS_ERR_CUDA, "server: event creation failed");
        }
        a->h = h;
        a->t_admit = now_s();
        // A bed joins the batch when it is small (see kBatchMaxCells) and not
        // dense (at most as many particle centres as cells): the batch
        // advances in lockstep, and the per-step cost of hard spheres grows
        // with the square of a cell's occupancy, so a dense bed would hold
        // every other bed of the batch at its pace.
        if (s->batching && lbdpsk::batch_describe(h, &a->desc) == LBDPS_OK &&
            a->desc.ncell <= s->batch_max_cells && a->desc.np <= a->desc.ncell &&
            batch_init(s) == LBDPS_OK) {
            // the batch stream starts on the bed after the work of its creation
            cudaEvent_t made = nullptr;
            if (cudaEventCreateWithFlags(&made, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventRecord(made, lbdpsk::bed_stream(h)) == cudaSuccess &&
                cudaStreamWaitEvent(s->batch.st, made, 0) == cudaSuccess) {
                a->batched = true;
                s->batch.dirty = true;
            }
            cudaGetLastError();
            if (made) cudaEventDestroy(made);
        }
        s->used += q.bytes;
        s->active.push_back(std::move(a));
    }
    return LBDPS_OK;
}

// Issue the next tick of a bed (at most one tick in flight per bed).
int launch_tick(lbdps_server *s, Active &a)
{
    if (a.issued >= a.req.steps) return LBDPS_OK;
    if (a.tick_pending) {
        const cudaError_t q = cudaEventQuery(a.tick);
        if (q == cudaErrorNotReady) return LBDPS_OK;      // one tick in flight per bed
        if (q != cudaSuccess) return sfail(LBDPS_ERR_CUDA, "server: tick failed");
        a.tick_pending = false;
    }
    const int64_t m = std::min<int64_t>(s->steps_per_tick, a.req.steps - a.issued);
    int rc = lbdps_step(a.h, m);
    if (rc) return rc;
    a.issued += m;
    rc = lbdps_record_event(a.h, a.issued >= a.req.steps ? a.last : a.tick);
    if (rc) return rc;
    if (a.issued < a.req.steps) a.tick_pending = true;
    return LBDPS_OK;
}

}  // namespace

extern "C" {

int lbdps_server_create(size_t hbm_budget, int max_active, int steps_per_tick,
                        lbdps_server_t **out)
{
    if (!out || hbm_budget == 0 || max_active < 1 || steps_per_tick < 1)
        return sfail(LBDPS_ERR_INVALID, "server: bad arguments");
    *out = nullptr;
    lbdps_server *s = new (std::nothrow) lbdps_server();
    if (!s) return sfail(LBDPS_ERR_OOM, "server: host allocation failed");
    s->budget = hbm_budget;
    s->max_active = max_active;
    s->steps_per_tick = steps_per_tick;
    s->t0 = now_s();
    *out = s;
    return LBDPS_OK;
}

int lbdps_server_submit(lbdps_server_t *s, const lbdps_lattice_desc *lat,
                        const lbdps_particle_desc *par, const lbdps_params *prm, int64_t nsteps,
                        int keep, uint64_t *req_id)
{
    if (!s || !lat || !par || !prm || nsteps < 0) return sfail(LBDPS_ERR_INVALID, "server: bad arguments");
    size_t bytes = 0;
    int rc = lbdps_memory_estimate(lat, par, prm, &bytes);
    if (rc) return rc;
    if (bytes > s->budget) return sfail(LBDPS_ERR_CAPACITY, "server: request exceeds the HBM budget");
    Request r;
    r.id = s->next_id++;
    r.lat = *lat;
    r.par = *par;
    r.prm = *prm;
    r.steps = nsteps;
    r.bytes = bytes;
    r.keep = keep;
    r.t_submit = now_s();
    const int D = lat->dim;
    r.pos.assign(par->pos, par->pos + (size_t)par->n * D);
    r.vel.assign(par->vel, par->vel + (size_t)par->n * D);
    if (lat->inlet_u) {
        const int vert = D - 1;
        size_t nface = 1;
        for (int a = 0; a < D; ++a)
            if (a != vert) nface *= (size_t)lat->n[a];
        r.inlet.assign(lat->inlet_u, lat->inlet_u + nface * D);
    }
    if (req_id) *req_id = r.id;
    s->queue.push_back(std::move(r));
    return admit(s);
}

int lbdps_server_poll(lbdps_server_t *s, double wait_s, lbdps_done_t *out, int cap, int *ndone)
{
    if (!s || (cap > 0 && !out) || !ndone) return sfail(LBDPS_ERR_INVALID, "server: bad arguments");
    *ndone = 0;
    const double deadline = now_s() + (wait_s > 0 ? wait_s : 0.0);
    for (;;) {
        int rc = admit(s);
        if (rc) return rc;
        for (auto &a : s->active) {
            if (a->batched) continue;
            rc = launch_tick(s, *a);
            if (rc) return rc;
        }
        rc = batch_tick(s);
        if (rc) return rc;
        // harvest beds whose last step has completed
        for (size_t i = 0; i < s->active.size();) {
            Active &a = *s->active[i];
            bool finished = false;
            if (a.issued >= a.req.steps) {
                if (a.batched) {
                    // the tick that took its last steps has completed
                    finished = a.last_tick <= s->batch.done_ticks;
                } else {
                    const cudaError_t q = cudaEventQuery(a.last);
                    if (q == cudaSuccess) finished = true;
                    else if (q != cudaErrorNotReady) return sfail(LBDPS_ERR_CUDA, "server: bed failed");
                }
            }
            if (!finished) {
                ++i;
                continue;
            }
            lbdps_done_t d{};
            d.id = a.req.id;
            d.steps = a.req.steps;
            d.cells = 1;
            for (int k = 0; k < a.req.lat.dim; ++k) d.cells *= a.req.lat.n[k];
            d.t_submit = a.req.t_submit - s->t0;
            d.t_admit = a.t_admit - s->t0;
            d.t_done = now_s() - s->t0;
            d.status = lbdps_stats(a.h, &d.stats);
            // a packed cell (health bit 8) is reported in the record, not a failure
            if (d.status == LBDPS_OK && (d.stats.health & 3)) d.status = LBDPS_ERR_DIVERGED;
            s->done.push_back(d);
            cudaEventDestroy(a.last);
            cudaEventDestroy(a.tick);
            if (a.req.keep) {
                s->kept[a.req.id] = {a.h, a.req.bytes};
            } else {
                lbdps_destroy(a.h);
                s->used -= a.req.bytes;
            }
            if (a.batched) {
                auto &m = s->batch.members;
                m.erase(std::remove(m.begin(), m.end(), &a), m.end());
                s->batch.dirty = true;
            }
            s->active.erase(s->active.begin() + i);
        }
        rc = admit(s);
        if (rc) return rc;
        if (!s->done.empty() || now_s() >= deadline || (s->active.empty() && s->queue.empty()))
            break;
    }
    const int n = (int)std::min<size_t>(s->done.size(), (size_t)(cap > 0 ? cap : 0));
    for (int i = 0; i < n; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + n);
    *ndone = n;
    return LBDPS_OK;
}

int lbdps_server_load(lbdps_server_t *s, int *queued, int *active, size_t *used)
{
    if (!s) return sfail(LBDPS_ERR_INVALID, "server: NULL handle");
    if (queued) *queued = (int)s->queue.size();
    if (active) *active = (int)s->active.size();
    if (used) *used = s->used;
    return LBDPS_OK;
}

int lbdps_server_take(lbdps_server_t *s, uint64_t req_id, lbdps_t **out)
{
    if (!s || !out) return sfail(LBDPS_ERR_INVALID, "server: bad arguments");
    *out = nullptr;
    auto it = s->kept.find(req_id);
    if (it == s->kept.end()) return sfail(LBDPS_ERR_INVALID, "server: no kept result with that id");
    *out = it->second.first;
    s->used -= it->second.second;
    s->kept.erase(it);
    return LBDPS_OK;
}

int lbdps_server_set_batching(lbdps_server_t *s, int on, int64_t max_cells)
{
    if (!s || max_cells < 0) return sfail(LBDPS_ERR_INVALID, "server: bad arguments");
    s->batching = on != 0;
    s->batch_max_cells = max_cells > 0 ? (int)std::min<int64_t>(max_cells, INT32_MAX) : kBatchMaxCells;
    return LBDPS_OK;
}

int lbdps_server_batch_info(lbdps_server_t *s, int64_t *ticks, int64_t *captures, int *members)
{
    if (!s) return sfail(LBDPS_ERR_INVALID, "server: NULL handle");
    if (ticks) *ticks = s->batch.ticks;
    if (captures) *captures = s->batch.captures;
    if (members) *members = (int)s->batch.members.size();
    return LBDPS_OK;
}

void lbdps_server_destroy(lbdps_server_t *s)
{
    if (!s) return;
    batch_release(s->batch);
    for (auto &a : s->active) {
        lbdps_destroy(a->h);
        cudaEventDestroy(a->last);
        cudaEventDestroy(a->tick);
    }
    for (auto &k : s->kept) lbdps_destroy(k.second.first);
    delete s;
}

}  // extern "C"

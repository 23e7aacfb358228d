// Continuous batching of independent beds (the serving loop).
//
// Requests (a bed description and a step count K) arrive at any time.  The
// server keeps a FIFO queue, admits the head request as soon as its exact
// device-memory footprint (lbdps_memory_estimate) fits in the HBM budget and
// an active slot is free, and keeps every admitted bed resident on the device
// on a stream of its own.  Each poll advances every active bed by one tick
// (a fixed number of steps, each a replay of the bed's captured step graph);
// ticks of different beds are independent stream work and overlap on the
// GPU.  A bed that has reached K steps is harvested: its FP64 statistics and
// completion time are recorded, its memory is released (or kept for the
// caller, see lbdps_server_take), and the freed budget admits the next
// requests.  Each bed's arithmetic is the same as when it runs alone.
#include "lbdps.h"

#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
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
};

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
};

namespace {

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
            rc = launch_tick(s, *a);
            if (rc) return rc;
        }
        // harvest beds whose last step has completed
        for (size_t i = 0; i < s->active.size();) {
            Active &a = *s->active[i];
            bool finished = false;
            if (a.issued >= a.req.steps) {
                const cudaError_t q = cudaEventQuery(a.last);
                if (q == cudaSuccess) finished = true;
                else if (q != cudaErrorNotReady) return sfail(LBDPS_ERR_CUDA, "server: bed failed");
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

void lbdps_server_destroy(lbdps_server_t *s)
{
    if (!s) return;
    for (auto &a : s->active) {
        lbdps_destroy(a->h);
        cudaEventDestroy(a->last);
        cudaEventDestroy(a->tick);
    }
    for (auto &k : s->kept) lbdps_destroy(k.second.first);
    delete s;
}

}  // extern "C"

// sx_server.cu -- the serving form: a request loop with continuous batching
// of backward-Euler steps (§3 Eqs. 2-3) over device-resident scenes.
//
// Built only on the public C ABI of include/sx.h. Requests are split by tet
// count into size-class lanes; each lane has its own context, CUDA stream
// (smaller classes at higher stream priority) and worker thread. Every tick
// of a lane admits that lane's waiting requests while they fit the shared
// memory budget and runs one sx_newton_step_batch over all of its resident
// scenes, so requests that arrive while others are on the GPU join at the
// lane's next tick, their work overlaps with the others' inside the same
// launches, and small scenes do not wait for the PCG of large ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/sx.h"

// 1: lanes of larger scenes leave room on the SMs for the lanes below them
// (measured: p50 step latency -5%, p99 +14% on the 48-request sample; off)
#ifndef SX_SERVER_SHARE
#define SX_SERVER_SHARE 0
#endif

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    std::vector<double> X, young, poisson;
    std::vector<int32_t> tets, pinned;
    double density = 0.0, gravity[3] = {0, 0, 0}, dt = 0.0;
    int n_steps = 0, lane = 0;
    int64_t n_nodes = 0, n_tets = 0, footprint = 0;
    double t_submit = 0, t_admit = -1, t_eligible = 0, t_done = 0;
    int steps_done = 0, status = SX_OK;
    sx_scene* scene = nullptr;
    double step_sum = 0.0;
    std::vector<double> x_final, v_final;
    std::string error;
};

double pct(std::vector<double> v, double p)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    double r = p * (double)(v.size() - 1);
    size_t i = (size_t)r;
    double f = r - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct Lane {
    int index = 0;
    sx_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::vector<Request*> active;
    bool ticking = false;
};

struct sx_server {
    int device = 0;
    int64_t budget = 0;
    sx_newton_opts opts{};
    std::mutex mu;
    std::condition_variable cv, idle_cv;
    std::deque<Request*> pending;
    std::vector<Lane*> lanes;
    std::vector<int64_t> bounds;   // lane i takes n_tets < bounds[i]; the last lane the rest
    int lane_cap = 0;              // most scenes resident in one lane (0: no limit)
    std::deque<sx_completion> completions;
    std::unordered_map<int64_t, Request*> finished;
    bool stop = false;
    int64_t next_id = 1, in_use = 0, peak = 0;
    int64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, element_steps = 0;
    int ticks = 0;
    double busy_ms = 0.0;
    std::vector<double> step_lat, req_lat;
    Clock::time_point t0;

    double now() const
    {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
};

namespace {

int64_t footprint(const Request& r)
{
    sx_scene_desc d{};
    d.n_nodes = r.n_nodes;
    d.n_tets = r.n_tets;
    int64_t b = 0;
    sx_scene_footprint(&d, &b);   // includes the projection scratch share
    return b;
}

// registration on the device; returns the status
int admit(Lane* L, Request* r)
{
    sx_scene* sc = nullptr;
    int rc = sx_scene_create(L->ctx, r->n_nodes, r->X.data(), 3, L->stream, &sc);
    if (rc == SX_OK)
        rc = sx_add_snh_tet4(sc, r->tets.data(), r->n_tets, r->young.data(), r->poisson.data(),
                             r->density, 0, L->stream, nullptr);
    if (rc == SX_OK && !r->pinned.empty())
        rc = sx_set_pinned(sc, r->pinned.data(), (int64_t)r->pinned.size(), L->stream);
    if (rc == SX_OK) rc = sx_set_gravity(sc, r->gravity);
    if (rc == SX_OK) rc = sx_finalize(sc, L->stream);
    if (rc != SX_OK) {
        if (sc) sx_scene_destroy(sc);
        return rc;
    }
    r->scene = sc;
    // host copies are no longer needed once the scene is resident
    std::vector<double>().swap(r->young);
    std::vector<double>().swap(r->poisson);
    std::vector<int32_t>().swap(r->tets);
    std::vector<int32_t>().swap(r->pinned);
    return SX_OK;
}

void retire(sx_server* S, Lane* L, Request* r, double t)
{
    if (r->scene) {
        r->x_final.resize(3 * r->n_nodes);
        r->v_final.resize(3 * r->n_nodes);
        sx_get_state(r->scene, r->x_final.data(), r->v_final.data(), L->stream);
        cudaStreamSynchronize(L->stream);
        sx_scene_destroy(r->scene);
        r->scene = nullptr;
    }
    std::vector<double>().swap(r->X);
    r->t_done = t;
    sx_completion c{};
    c.req_id = r->id;
    c.status = r->status;
    c.steps = r->steps_done;
    c.n_tets = r->n_tets;
    c.submit_ms = r->t_submit;
    c.admit_ms = r->t_admit;
    c.done_ms = r->t_done;
    c.mean_step_ms = r->steps_done ? r->step_sum / r->steps_done : 0.0;
    std::strncpy(c.error, r->error.c_str(), sizeof(c.error) - 1);
    c.error[sizeof(c.error) - 1] = 0;
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use -= r->footprint;
    S->completions.push_back(c);
    S->finished[r->id] = r;
    S->completed++;
    S->req_lat.push_back(r->t_done - r->t_submit);
    S->cv.notify_all();   // memory was released: other lanes may admit
}

// the lane's first waiting request (FIFO within a lane), or null
Request* first_pending(sx_server* S, const Lane* L)
{
    for (Request* r : S->pending)
        if (r->lane == L->index) return r;
    return nullptr;
}

bool all_idle(sx_server* S)
{
    if (!S->pending.empty()) return false;
    for (Lane* L : S->lanes)
        if (L->ticking || !L->active.empty()) return false;
    return true;
}

void lane_loop(sx_server* S, Lane* L)
{
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request*> to_admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] {
                if (S->stop || !L->active.empty()) return true;
                Request* f = first_pending(S, L);
                return f != nullptr && S->in_use + f->footprint <= S->budget;
            });
            if (S->stop) break;
            for (auto it = S->pending.begin(); it != S->pending.end();) {
                Request* r = *it;
                if (r->lane != L->index) {
                    ++it;
                    continue;
                }
                if (S->lane_cap > 0 &&
                    (int)(L->active.size() + to_admit.size()) >= S->lane_cap)
                    break;
                if (S->in_use + r->footprint > S->budget) break;
                S->in_use += r->footprint;
                S->peak = std::max(S->peak, S->in_use);
                to_admit.push_back(r);
                it = S->pending.erase(it);
            }
            L->ticking = true;
        }
        for (Request* r : to_admit) {
            int rc = admit(L, r);
            r->t_admit = r->t_eligible = S->now();
            if (rc != SX_OK) {
                r->status = rc;
                r->error = std::string("admission: ") + sx_last_error(L->ctx);
                retire(S, L, r, S->now());
                continue;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            S->admitted++;
            L->active.push_back(r);
        }
        std::vector<Request*> act = L->active;
        if (!act.empty()) {
            // one batched step per group of equal dt
            std::map<double, std::vector<Request*>> groups;
            for (Request* r : act) groups[r->dt].push_back(r);
            const double ts = S->now();
            for (auto& g : groups) {
                std::vector<sx_scene*> sc;
                for (Request* r : g.second) sc.push_back(r->scene);
                std::vector<sx_step_report> rep(sc.size());
                sx_newton_step_batch(L->ctx, sc.data(), (int)sc.size(), g.first, &S->opts,
                                     rep.data(), L->stream);
                const double te = S->now();
                for (size_t i = 0; i < g.second.size(); ++i) {
                    Request* r = g.second[i];
                    const double lat = te - r->t_eligible;
                    r->step_sum += lat;
                    r->steps_done++;
                    r->t_eligible = te;
                    if (rep[i].status != SX_OK && r->status == SX_OK) {
                        r->status = rep[i].status;
                        r->error = std::string("step ") + std::to_string(r->steps_done) +
                                   ": " + sx_last_error(L->ctx);
                    }
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->step_lat.push_back(lat);
                    S->element_steps += r->n_tets;
                }
            }
            const double te = S->now();
            std::vector<Request*> keep, fin;
            for (Request* r : act) {
                if (r->steps_done >= r->n_steps || r->status != SX_OK) fin.push_back(r);
                else keep.push_back(r);
            }
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->busy_ms += te - ts;
                S->ticks++;
                L->active = keep;
            }
            for (Request* r : fin) retire(S, L, r, te);
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            L->ticking = false;
            if (all_idle(S)) S->idle_cv.notify_all();
        }
    }
}

void stop_lanes(sx_server* S)
{
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (Lane* L : S->lanes)
        if (L->worker.joinable()) L->worker.join();
    for (Lane* L : S->lanes) {
        for (Request* r : L->active) {
            if (r->scene) sx_scene_destroy(r->scene);
            delete r;
        }
        if (L->ctx) sx_destroy(L->ctx);
        if (L->stream) cudaStreamDestroy(L->stream);
        delete L;
    }
    S->lanes.clear();
    S->stop = false;
}

// one lane per size class; lane 0 (the smallest scenes) gets the highest
// stream priority
int start_lanes(sx_server* S, const std::vector<int64_t>& bounds)
{
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    S->bounds = bounds;
    const int n = (int)bounds.size() + 1;
    for (int i = 0; i < n; ++i) {
        auto* L = new Lane();
        L->index = i;
        S->lanes.push_back(L);
        sx_options o{};
        o.device = S->device;
        // every lane but the one of the smallest scenes leaves room on the
        // SMs for the lanes below it
        o.share_sms = (SX_SERVER_SHARE && i > 0) ? 1 : 0;
        const int prio = std::min(least, greatest + i);
        if (sx_create(&L->ctx, &o) != SX_OK ||
            cudaStreamCreateWithPriority(&L->stream, cudaStreamNonBlocking, prio) != cudaSuccess) {
            stop_lanes(S);
            return SX_ECUDA;
        }
    }
    for (Lane* L : S->lanes) L->worker = std::thread(lane_loop, S, L);
    return SX_OK;
}

}  // namespace

extern "C" {

int sx_server_create(sx_ctx* ctx, int64_t budget, const sx_newton_opts* opts, sx_server** out)
{
    if (!ctx || !out || budget <= 0) return SX_EINVAL;
    auto* S = new sx_server();
    S->budget = budget;
    if (opts) S->opts = *opts;
    else sx_newton_opts_default(&S->opts);
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return SX_ECUDA;
    }
    S->t0 = Clock::now();
    const int rc = start_lanes(S, {20000, 120000});
    if (rc != SX_OK) {
        delete S;
        return rc;
    }
    *out = S;
    return SX_OK;
}

int sx_server_set_lane_cap(sx_server* S, int max_resident)
{
    if (!S || max_resident < 0) return SX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    S->lane_cap = max_resident;
    S->cv.notify_all();
    return SX_OK;
}

int sx_server_set_lanes(sx_server* S, int n_lanes, const int64_t* bounds)
{
    if (!S || n_lanes < 1 || n_lanes > SX_SERVER_MAX_LANES || (n_lanes > 1 && !bounds))
        return SX_EINVAL;
    std::vector<int64_t> b;
    for (int i = 0; i + 1 < n_lanes; ++i) {
        if (bounds[i] <= 0 || (i > 0 && bounds[i] <= bounds[i - 1])) return SX_EINVAL;
        b.push_back(bounds[i]);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->submitted > 0) return SX_EORDER;
    }
    stop_lanes(S);
    return start_lanes(S, b);
}

int sx_server_submit(sx_server* S, const sx_snh_scene_spec* spec, int n_steps, double dt,
                     int64_t* req_id)
{
    if (!S || !spec || n_steps <= 0 || !(dt > 0.0) || spec->n_nodes <= 0 || spec->n_tets <= 0 ||
        !spec->X || !spec->tets || !spec->young || !spec->poisson)
        return SX_EINVAL;
    auto* r = new Request();
    r->n_nodes = spec->n_nodes;
    r->n_tets = spec->n_tets;
    r->X.assign(spec->X, spec->X + 3 * spec->n_nodes);
    r->tets.assign(spec->tets, spec->tets + 4 * spec->n_tets);
    r->young.assign(spec->young, spec->young + spec->n_tets);
    r->poisson.assign(spec->poisson, spec->poisson + spec->n_tets);
    if (spec->pinned && spec->n_pinned > 0)
        r->pinned.assign(spec->pinned, spec->pinned + spec->n_pinned);
    r->density = spec->density;
    for (int i = 0; i < 3; ++i) r->gravity[i] = spec->gravity[i];
    r->n_steps = n_steps;
    r->dt = dt;
    r->footprint = footprint(*r);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->lane = (int)S->bounds.size();
        for (size_t i = 0; i < S->bounds.size(); ++i)
            if (r->n_tets < S->bounds[i]) {
                r->lane = (int)i;
                break;
            }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->submitted++;
    if (r->footprint > S->budget) {
        S->rejected++;
        delete r;
        return SX_EBUDGET;
    }
    r->id = S->next_id++;
    r->t_submit = S->now();
    if (req_id) *req_id = r->id;
    S->pending.push_back(r);
    S->cv.notify_all();
    return SX_OK;
}

int sx_server_poll(sx_server* S, sx_completion* out, int max, int* n)
{
    if (!S || !n || (max > 0 && !out)) return SX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    int k = 0;
    while (k < max && !S->completions.empty()) {
        out[k++] = S->completions.front();
        S->completions.pop_front();
    }
    *n = k;
    return SX_OK;
}

int sx_server_result(sx_server* S, int64_t req_id, double* x, double* v)
{
    if (!S) return SX_EINVAL;
    Request* r = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->finished.find(req_id);
        if (it == S->finished.end()) return SX_EINVAL;
        r = it->second;
        S->finished.erase(it);
    }
    if (x && !r->x_final.empty()) std::memcpy(x, r->x_final.data(), r->x_final.size() * sizeof(double));
    if (v && !r->v_final.empty()) std::memcpy(v, r->v_final.data(), r->v_final.size() * sizeof(double));
    delete r;
    return SX_OK;
}

int sx_server_drain(sx_server* S, double timeout_ms)
{
    if (!S) return SX_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    bool ok = S->idle_cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                  [&] { return all_idle(S); });
    return ok ? SX_OK : SX_ENOTCONV;
}

int sx_server_stats(sx_server* S, sx_serve_stats* st)
{
    if (!S || !st) return SX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    st->submitted = S->submitted;
    st->admitted = S->admitted;
    st->completed = S->completed;
    st->rejected = S->rejected;
    st->element_steps = S->element_steps;
    st->wall_ms = S->now();
    st->busy_ms = S->busy_ms;
    st->step_p50_ms = pct(S->step_lat, 0.50);
    st->step_p99_ms = pct(S->step_lat, 0.99);
    st->request_p50_ms = pct(S->req_lat, 0.50);
    st->request_p99_ms = pct(S->req_lat, 0.99);
    st->bytes_in_use = S->in_use;
    st->peak_bytes = S->peak;
    int act = 0;
    for (Lane* L : S->lanes) act += (int)L->active.size();
    st->active = act;
    st->pending = (int)S->pending.size();
    st->ticks = S->ticks;
    return SX_OK;
}

int sx_server_destroy(sx_server* S)
{
    if (!S) return SX_EINVAL;
    stop_lanes(S);
    for (Request* r : S->pending) delete r;
    for (auto& kv : S->finished) delete kv.second;
    delete S;
    return SX_OK;
}

}  // extern "C"

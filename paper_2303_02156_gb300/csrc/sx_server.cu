// sx_server.cu -- the serving form: a request loop with continuous batching
// of backward-Euler steps (§3 Eqs. 2-3) over device-resident scenes.
//
// Built only on the public C ABI of include/sx.h: each request becomes a
// scene of the server's context at admission; every tick runs one
// sx_newton_step_batch over all resident scenes, so requests that arrive
// while others are on the GPU join at the next tick and their work overlaps
// with the others' inside the same launches.
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

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    std::vector<double> X, young, poisson;
    std::vector<int32_t> tets, pinned;
    double density = 0.0, gravity[3] = {0, 0, 0}, dt = 0.0;
    int n_steps = 0;
    int64_t n_nodes = 0, n_tets = 0, footprint = 0;
    double t_submit = 0, t_admit = -1, t_eligible = 0, t_done = 0;
    int steps_done = 0, status = SX_OK;
    sx_scene* scene = nullptr;
    double step_sum = 0.0;
    std::vector<double> x_final, v_final;
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

struct sx_server {
    sx_ctx* ctx = nullptr;
    int device = 0;
    int64_t budget = 0;
    sx_newton_opts opts{};
    std::mutex mu;
    std::condition_variable cv, idle_cv;
    std::deque<Request*> pending;
    std::vector<Request*> active;
    std::deque<sx_completion> completions;
    std::unordered_map<int64_t, Request*> finished;
    std::thread worker;
    bool stop = false;
    bool ticking = false;
    int64_t next_id = 1, in_use = 0, peak = 0;
    int64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, element_steps = 0;
    int ticks = 0;
    double busy_ms = 0.0;
    std::vector<double> step_lat, req_lat;
    Clock::time_point t0;
    cudaStream_t stream = nullptr;

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
    sx_scene_footprint(&d, &b);
    return b + r.n_tets * 45 * 8;   // share of the context's projection queue
}

// registration on the device; returns the status
int admit(sx_server* S, Request* r)
{
    sx_scene* sc = nullptr;
    int rc = sx_scene_create(S->ctx, r->n_nodes, r->X.data(), 3, S->stream, &sc);
    if (rc == SX_OK)
        rc = sx_add_snh_tet4(sc, r->tets.data(), r->n_tets, r->young.data(), r->poisson.data(),
                             r->density, 0, S->stream, nullptr);
    if (rc == SX_OK && !r->pinned.empty())
        rc = sx_set_pinned(sc, r->pinned.data(), (int64_t)r->pinned.size(), S->stream);
    if (rc == SX_OK) rc = sx_set_gravity(sc, r->gravity);
    if (rc == SX_OK) rc = sx_finalize(sc, S->stream);
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

void retire(sx_server* S, Request* r, double t)
{
    if (r->scene) {
        r->x_final.resize(3 * r->n_nodes);
        r->v_final.resize(3 * r->n_nodes);
        sx_get_state(r->scene, r->x_final.data(), r->v_final.data(), S->stream);
        cudaStreamSynchronize(S->stream);
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
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use -= r->footprint;
    S->completions.push_back(c);
    S->finished[r->id] = r;
    S->completed++;
    S->req_lat.push_back(r->t_done - r->t_submit);
}

void worker_loop(sx_server* S)
{
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request*> to_admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->pending.empty() || !S->active.empty(); });
            if (S->stop) break;
            while (!S->pending.empty() && S->in_use + S->pending.front()->footprint <= S->budget) {
                Request* r = S->pending.front();
                S->pending.pop_front();
                S->in_use += r->footprint;
                S->peak = std::max(S->peak, S->in_use);
                to_admit.push_back(r);
            }
            S->ticking = true;
        }
        for (Request* r : to_admit) {
            int rc = admit(S, r);
            r->t_admit = r->t_eligible = S->now();
            if (rc != SX_OK) {
                r->status = rc;
                retire(S, r, S->now());
                continue;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            S->admitted++;
            S->active.push_back(r);
        }
        std::vector<Request*> act;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            act = S->active;
        }
        if (!act.empty()) {
            // one batched step per group of equal dt
            std::map<double, std::vector<Request*>> groups;
            for (Request* r : act) groups[r->dt].push_back(r);
            const double ts = S->now();
            for (auto& g : groups) {
                std::vector<sx_scene*> sc;
                for (Request* r : g.second) sc.push_back(r->scene);
                std::vector<sx_step_report> rep(sc.size());
                sx_newton_step_batch(S->ctx, sc.data(), (int)sc.size(), g.first, &S->opts, rep.data(),
                                     S->stream);
                const double te = S->now();
                for (size_t i = 0; i < g.second.size(); ++i) {
                    Request* r = g.second[i];
                    const double lat = te - r->t_eligible;
                    r->step_sum += lat;
                    r->steps_done++;
                    r->t_eligible = te;
                    if (rep[i].status != SX_OK) r->status = rep[i].status;
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
                // requests admitted during this tick were appended after act
                std::vector<Request*> rest(S->active.begin() + act.size(), S->active.end());
                S->active = keep;
                S->active.insert(S->active.end(), rest.begin(), rest.end());
            }
            for (Request* r : fin) retire(S, r, te);
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->ticking = false;
            if (S->pending.empty() && S->active.empty()) S->idle_cv.notify_all();
        }
    }
}

}  // namespace

extern "C" {

int sx_server_create(sx_ctx* ctx, int64_t budget, const sx_newton_opts* opts, sx_server** out)
{
    if (!ctx || !out || budget <= 0) return SX_EINVAL;
    auto* S = new sx_server();
    S->ctx = ctx;
    S->budget = budget;
    if (opts) S->opts = *opts;
    else sx_newton_opts_default(&S->opts);
    if (cudaGetDevice(&S->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return SX_ECUDA;
    }
    S->t0 = Clock::now();
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return SX_OK;
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
    S->cv.notify_one();
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
    bool ok = S->idle_cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), [&] {
        return S->pending.empty() && S->active.empty() && !S->ticking;
    });
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
    st->active = (int)S->active.size();
    st->pending = (int)S->pending.size();
    st->ticks = S->ticks;
    return SX_OK;
}

int sx_server_destroy(sx_server* S)
{
    if (!S) return SX_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Request* r : S->active)
        if (r->scene) sx_scene_destroy(r->scene);
    for (Request* r : S->active) delete r;
    for (Request* r : S->pending) delete r;
    for (auto& kv : S->finished) delete kv.second;
    cudaStreamDestroy(S->stream);
    delete S;
    return SX_OK;
}

}  // extern "C"

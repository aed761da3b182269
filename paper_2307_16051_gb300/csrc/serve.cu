// serve.cu — a request loop for H-equation solves (Section 3, eq. (3.2)) of
// different N and c arriving over time.
//
// Admission is by device-memory footprint: a request needs one solver handle
// for its N (J32, J16, the GMRES basis, vectors and workspaces; the double
// Jacobian too in FP64 mode), and the server holds handles up to a byte
// budget.  A finished request leaves its handle idle in a cache; a later
// request of the same N reuses it without allocating, and idle handles of
// other sizes are released (least recently used first) when a new size does
// not fit.  Among the requests that have arrived, the smallest N goes first
// (or the earliest, with the arrival-order policy); one that does not fit may
// be passed by others that do; once the oldest waiting request has waited
// for the starvation bound, it goes first and nothing passes it.
//
// Every admitted request runs on its own worker thread and CUDA stream (a
// high-priority stream for small N, whose short latency-bound kernels then
// start ahead of the large factorisations' tiles when SMs free up): its
// iterate, factors and Krylov state stay on the device across its Newton
// steps, and the kernels of the requests in flight overlap on the GPU.  A
// request admitted while others run joins them at once (continuous
// admission), and the result of a request does not depend on what else runs:
// each solve is the deterministic single-instance solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nl {

struct SReq {
    int64_t id = 0;
    int N = 0;
    double c = 0.0;
    double t_arrive = 0.0, t_admit = 0.0, t_done = 0.0;
    int status = -1;
    int reused = 0;
    std::vector<double> x;
    nl_stats_t st;
};

struct SHandle {
    nl_solver* h = nullptr;
    int N = 0;
    int64_t bytes = 0;
    bool busy = false;
    uint64_t last_use = 0;
};

}  // namespace nl

using namespace nl;

struct nl_server {
    nl_server_config cfg;
    int dev = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::shared_ptr<SReq>> reqs;  // index = id
    std::vector<int64_t> waiting;             // ids, ordered by arrival time
    std::list<SHandle> handles;
    int64_t bytes_held = 0, bytes_peak = 0;
    int inflight = 0, inflight_peak = 0;
    int created = 0, evicted = 0;
    int64_t completed = 0, failed = 0;
    uint64_t use_clock = 0;
    bool started = false, stop = false;
    std::chrono::steady_clock::time_point t0;
    std::vector<std::thread> workers;

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

static void worker_main(nl_server* S)
{
    cudaSetDevice(S->dev);
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);  // numerically lower = higher priority
    cudaStream_t st_lo = nullptr, st_hi = nullptr;
    cudaStreamCreateWithPriority(&st_lo, cudaStreamNonBlocking, lo);
    cudaStreamCreateWithPriority(&st_hi, cudaStreamNonBlocking, hi);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        if (!S->started) {
            S->cv.wait(lk);
            continue;
        }
        const double now = S->now();
        int pick = -1;
        std::list<SHandle>::iterator hit = S->handles.end();
        bool need_alloc = false;
        int64_t need = 0;
        std::vector<std::list<SHandle>::iterator> victims;
        double next_arrival = -1.0;
        // candidates: the arrived requests in arrival order, or, with the
        // smallest-first policy, by N (ties by arrival) unless the oldest has
        // waited past the starvation bound
        std::vector<size_t> cand;
        for (size_t k = 0; k < S->waiting.size(); ++k) {
            if (S->reqs[S->waiting[k]]->t_arrive > now) {
                next_arrival = S->reqs[S->waiting[k]]->t_arrive;
                break;  // later entries arrive later still
            }
            cand.push_back(k);
        }
        if (S->cfg.policy == 1 && !cand.empty() &&
            (now - S->reqs[S->waiting[cand[0]]]->t_arrive) * 1e3 <= S->cfg.starve_ms)
            std::stable_sort(cand.begin(), cand.end(),
                             [&](size_t a, size_t b) { return S->reqs[S->waiting[a]]->N < S->reqs[S->waiting[b]]->N; });
        for (size_t ci = 0; ci < cand.size(); ++ci) {
            const size_t k = cand[ci];
            SReq& r = *S->reqs[S->waiting[k]];
            for (auto it = S->handles.begin(); it != S->handles.end(); ++it)
                if (!it->busy && it->h && it->N == r.N) {
                    hit = it;
                    break;
                }
            if (hit != S->handles.end()) {
                pick = (int)k;
                break;
            }
            need = nl_footprint_bytes(r.N, (nl_mode)S->cfg.mode, &S->cfg.solver);
            if (S->bytes_held + need <= S->cfg.hbm_budget_bytes) {
                pick = (int)k;
                need_alloc = true;
                break;
            }
            // room after releasing idle handles, least recently used first
            std::vector<std::list<SHandle>::iterator> idle;
            int64_t idle_bytes = 0;
            for (auto it = S->handles.begin(); it != S->handles.end(); ++it)
                if (!it->busy && it->h) {
                    idle.push_back(it);
                    idle_bytes += it->bytes;
                }
            if (S->bytes_held - idle_bytes + need <= S->cfg.hbm_budget_bytes) {
                std::sort(idle.begin(), idle.end(), [](auto a, auto b) { return a->last_use < b->last_use; });
                int64_t held = S->bytes_held;
                for (auto it : idle) {
                    if (held + need <= S->cfg.hbm_budget_bytes) break;
                    victims.push_back(it);
                    held -= it->bytes;
                }
                pick = (int)k;
                need_alloc = true;
                break;
            }
            // it does not fit yet: later requests may pass it unless it has waited too long
            if (ci == 0 && (now - r.t_arrive) * 1e3 > S->cfg.starve_ms) break;
        }
        if (pick < 0) {
            if (next_arrival >= 0.0)
                S->cv.wait_for(lk, std::chrono::duration<double>(std::max(0.0, next_arrival - now)));
            else
                S->cv.wait(lk);
            continue;
        }
        std::shared_ptr<SReq> r = S->reqs[S->waiting[pick]];
        S->waiting.erase(S->waiting.begin() + pick);
        r->t_admit = now;
        S->inflight += 1;
        S->inflight_peak = std::max(S->inflight_peak, S->inflight);
        std::vector<nl_solver*> doomed;
        for (auto it : victims) {
            doomed.push_back(it->h);
            S->bytes_held -= it->bytes;
            S->evicted += 1;
            S->handles.erase(it);
        }
        if (need_alloc) {
            SHandle h;
            h.N = r->N;
            h.bytes = need;
            h.busy = true;
            S->handles.push_back(h);
            hit = std::prev(S->handles.end());
            S->bytes_held += need;
            S->bytes_peak = std::max(S->bytes_peak, S->bytes_held);
            S->created += 1;
        } else {
            hit->busy = true;
            r->reused = 1;
        }
        lk.unlock();
        for (nl_solver* d : doomed) nl_destroy(d);
        nl_status status = NL_OK;
        nl_solver* h = hit->h;
        if (!h) {
            status = nl_create(r->N, r->c, &S->cfg.solver, &h);
            if (status != NL_OK) h = nullptr;
        } else {
            status = nl_set_c(h, r->c);
        }
        if (status == NL_OK) {
            nl_set_stream(h, r->N <= S->cfg.priority_n ? st_hi : st_lo);
            r->x.assign(r->N, 0.0);
            status = nl_solve(h, nullptr, S->cfg.tol, (nl_mode)S->cfg.mode, r->x.data());
            nl_stats(h, &r->st);
            nl_set_stream(h, nullptr);  // the stream belongs to this worker; an idle handle keeps none
        }
        lk.lock();
        r->status = status;
        r->t_done = S->now();
        if (h) {
            hit->h = h;
            hit->busy = false;
            hit->last_use = ++S->use_clock;
        } else {
            S->bytes_held -= hit->bytes;
            S->handles.erase(hit);
        }
        S->inflight -= 1;
        if (status == NL_OK) S->completed += 1;
        else S->failed += 1;
        S->cv.notify_all();
    }
    lk.unlock();
    cudaStreamDestroy(st_lo);
    cudaStreamDestroy(st_hi);
}

extern "C" {

nl_status nl_server_config_default(nl_server_config* cfg)
{
    if (!cfg) {
        set_error("nl_server_config_default: cfg is NULL");
        return NL_EINVAL;
    }
    memset(cfg, 0, sizeof(*cfg));
    cfg->hbm_budget_bytes = (int64_t)64 << 30;
    cfg->max_inflight = 8;
    cfg->mode = NL_IR16_GMRES;
    cfg->tol = 1e-10;
    cfg->starve_ms = 250;
    cfg->priority_n = 1024;
    cfg->policy = 1;
    nl_config_default(&cfg->solver);
    return NL_OK;
}

nl_status nl_server_create(const nl_server_config* cfg, nl_server** out)
{
    set_error("");
    nl_server_config d;
    nl_server_config_default(&d);
    if (cfg) d = *cfg;
    if (!out || d.max_inflight < 1 || d.max_inflight > 256 || d.hbm_budget_bytes <= 0 || !(d.tol >= 0.0) ||
        !(d.mode >= NL_FP64LU && d.mode <= NL_IR16_GMRES) || d.starve_ms < 0 || d.policy < 0 || d.policy > 1) {
        set_error("nl_server_create: invalid configuration");
        return NL_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_error("nl_server_create: no CUDA device");
        return NL_ECUDA;
    }
    // one small solve on this thread initialises every kernel the workers use
    {
        nl_solver* w = nullptr;
        NL_TRY(nl_create(64, 0.5, &d.solver, &w));
        std::vector<double> x(64);
        nl_status s = nl_solve(w, nullptr, d.tol, (nl_mode)d.mode, x.data());
        nl_destroy(w);
        if (s != NL_OK) return s;
    }
    nl_server* S = new nl_server();
    S->cfg = d;
    cudaGetDevice(&S->dev);
    S->t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < d.max_inflight; ++k) S->workers.emplace_back(worker_main, S);
    *out = S;
    return NL_OK;
}

nl_status nl_server_submit(nl_server* S, int64_t N, double c, double arrival_s, int64_t* id)
{
    if (!S || !id || N < 1 || N > 32768 || !(c >= 0.0 && c < 1.0)) {
        set_error("nl_server_submit: need a server, id, N in [1, 32768] and 0 <= c < 1");
        return NL_EINVAL;
    }
    if (nl_footprint_bytes(N, (nl_mode)S->cfg.mode, &S->cfg.solver) > S->cfg.hbm_budget_bytes) {
        set_error("nl_server_submit: a handle for N = %lld needs more than the server's memory budget", (long long)N);
        return NL_EINVAL;
    }
    auto r = std::make_shared<SReq>();
    memset(&r->st, 0, sizeof(r->st));
    r->N = (int)N;
    r->c = c;
    std::lock_guard<std::mutex> lk(S->mu);
    r->t_arrive = (arrival_s < 0.0) ? (S->started ? S->now() : 0.0) : arrival_s;
    r->id = (int64_t)S->reqs.size();
    S->reqs.push_back(r);
    auto pos = std::upper_bound(S->waiting.begin(), S->waiting.end(), r->t_arrive,
                                [&](double t, int64_t k) { return t < S->reqs[k]->t_arrive; });
    S->waiting.insert(pos, r->id);
    *id = r->id;
    S->cv.notify_all();
    return NL_OK;
}

nl_status nl_server_start(nl_server* S)
{
    if (!S) {
        set_error("nl_server_start: NULL server");
        return NL_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->started) {
        S->t0 = std::chrono::steady_clock::now();
        S->started = true;
    }
    S->cv.notify_all();
    return NL_OK;
}

nl_status nl_server_result(nl_server* S, int64_t id, int wait, double* x_out, nl_stats_t* stats,
                           nl_request_info_t* info)
{
    if (!S) {
        set_error("nl_server_result: NULL server");
        return NL_EINVAL;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    if (id < 0 || id >= (int64_t)S->reqs.size()) {
        set_error("nl_server_result: unknown request %lld", (long long)id);
        return NL_EINVAL;
    }
    std::shared_ptr<SReq> r = S->reqs[id];
    if (wait)
        while (r->status < 0 && !S->stop) S->cv.wait(lk);
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = r->status;
        info->N = r->N;
        info->c = r->c;
        info->t_arrive_s = r->t_arrive;
        info->t_admit_s = r->t_admit;
        info->t_done_s = r->t_done;
        info->latency_ms = r->status >= 0 ? (r->t_done - r->t_arrive) * 1e3 : 0.0;
        info->newton_iters = r->st.newton_iters;
        info->handle_reused = r->reused;
    }
    if (r->status >= 0) {
        if (x_out && !r->x.empty()) memcpy(x_out, r->x.data(), sizeof(double) * r->x.size());
        if (stats) *stats = r->st;
    }
    return NL_OK;
}

nl_status nl_server_drain(nl_server* S, double timeout_s)
{
    if (!S) {
        set_error("nl_server_drain: NULL server");
        return NL_EINVAL;
    }
    auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop && (S->completed + S->failed) < (int64_t)S->reqs.size()) {
        if (S->cv.wait_until(lk, until) == std::cv_status::timeout &&
            (S->completed + S->failed) < (int64_t)S->reqs.size()) {
            set_error("nl_server_drain: %lld requests still pending",
                      (long long)((int64_t)S->reqs.size() - S->completed - S->failed));
            return NL_ETIMEOUT;
        }
    }
    return NL_OK;
}

nl_status nl_server_info(nl_server* S, nl_server_info_t* out)
{
    if (!S || !out) {
        set_error("nl_server_info: NULL argument");
        return NL_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = (int64_t)S->reqs.size();
    out->completed = S->completed;
    out->failed = S->failed;
    out->bytes_held = S->bytes_held;
    out->bytes_peak = S->bytes_peak;
    out->inflight_peak = S->inflight_peak;
    out->handles_created = S->created;
    out->handles_evicted = S->evicted;
    std::vector<double> lat;
    double first = 1e300, last = 0.0, sum = 0.0;
    for (auto& r : S->reqs)
        if (r->status == NL_OK) {
            const double l = (r->t_done - r->t_arrive) * 1e3;
            lat.push_back(l);
            sum += l;
            first = std::min(first, r->t_arrive);
            last = std::max(last, r->t_done);
        }
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double q) {
            size_t k = (size_t)std::ceil(q * (double)lat.size());
            return lat[std::min(lat.size() - 1, k > 0 ? k - 1 : 0)];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->mean_ms = sum / (double)lat.size();
        out->span_s = last - first;
        out->solves_per_s = out->span_s > 0 ? (double)lat.size() / out->span_s : 0.0;
    }
    return NL_OK;
}

void nl_server_destroy(nl_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    for (auto& t : S->workers) t.join();
    for (auto& h : S->handles)
        if (h.h) nl_destroy(h.h);
    delete S;
}

}  // extern "C"

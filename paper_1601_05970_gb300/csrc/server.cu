// Continuous-batching request loop for RVE increments (not in the paper; it
// serves the FE^2 use case of Section 1, where a macro solver issues one
// strain increment per Gauss point and per load step).
//
// A server owns one batch handle of `slots` cells of one grid size, one
// CUDA stream and one worker thread. Each request names a session (an RVE
// with its own microstructure and history) and a strain increment. The
// worker admits requests into free cells between Newton iterations, so
// requests that arrive while others are on the GPU join the running batch
// instead of waiting for it to drain; every cell keeps its own Newton and CG
// iteration and leaves the batch when it has converged. The number of slots
// is what the HBM budget allows (fftg_workspace_size_batch per slot); when
// all slots are taken, an idle resident session is evicted to host memory
// (its committed state) and restored when it is requested again.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fftg.h"
#include "driver.h"

using namespace fftg_detail;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    long long id = 0;
    long long session = 0;
    double dE[6] = {0, 0, 0, 0, 0, 0};
    double t_submit = 0.0;
};

struct Session {
    int slot = -1;                 // resident cell, or -1
    bool busy = false;             // a request of this session is in flight
    std::vector<uint8_t> phase;    // microstructure (kept for restores)
    std::vector<double> state;     // committed state while evicted (empty = fresh)
    double last_used = 0.0;
};

struct Inflight {
    bool on = false;
    Request req;
    double normE = 0.0;
    int it = 0;
    double t_start = 0.0;
};

}  // namespace

struct fftg_server {
    fftg_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    int N = 0;
    int slots = 0;
    double tol_newton = 1e-5, tol_cg = 1e-8, tol_inner = 1e-6;
    std::vector<long long> slot_session;  // session id of each slot, -1 = free
    std::unordered_map<long long, Session> sessions;
    std::deque<Request> incoming;          // submitted, not yet seen by the worker
    std::deque<Request> pending;           // seen, waiting for admission
    std::deque<fftg_result> done;
    std::vector<Inflight> inflight;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::thread worker;
    int error = FFTG_OK;
    long long n_evictions = 0, n_restores = 0, n_completed = 0;
    int max_concurrent = 0;
    double busy_rounds = 0.0;  // Newton rounds run
    double cells_in_rounds = 0.0;
};

namespace {

// Put a session into a cell: restore its state or start it fresh.
int make_resident(fftg_server* s, long long sid, Session& ss, int slot) {
    int rc = upload_cell(s->h, slot, ss.phase.data(), ss.state.empty() ? nullptr : ss.state.data());
    if (rc) return rc;
    if (!ss.state.empty()) ++s->n_restores;
    ss.state.clear();
    ss.state.shrink_to_fit();
    ss.slot = slot;
    s->slot_session[slot] = sid;
    return FFTG_OK;
}

// A cell for session sid: its own, a free one, or the least recently used
// idle one (evicted to host). -1 if every cell is busy.
int find_slot(fftg_server* s, long long sid, Session& ss) {
    if (ss.slot >= 0) return ss.slot;
    for (int k = 0; k < s->slots; ++k)
        if (s->slot_session[k] < 0) {
            if (make_resident(s, sid, ss, k)) return -2;
            return k;
        }
    int victim = -1;
    double oldest = 1e300;
    for (int k = 0; k < s->slots; ++k) {
        Session& o = s->sessions[s->slot_session[k]];
        if (!o.busy && o.last_used < oldest) {
            oldest = o.last_used;
            victim = k;
        }
    }
    if (victim < 0) return -1;
    Session& o = s->sessions[s->slot_session[victim]];
    o.state.resize((size_t)(6 + 13 * voxels(s->h)));
    if (download_cell(s->h, victim, o.state.data())) return -2;
    o.slot = -1;
    ++s->n_evictions;
    if (make_resident(s, sid, ss, victim)) return -2;
    return victim;
}

double frob6(const double* v) {
    return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + 2.0 * (v[3] * v[3] + v[4] * v[4] + v[5] * v[5]));
}

void worker_loop(fftg_server* s) {
    cudaStream_t st = s->stream;
    (void)st;
    const int S = s->slots;
    std::vector<int> run(S, 0), fin(S, 0), code(S, 0);
    std::vector<RoundOut> ro(S);
    std::vector<double> sig(6 * S, 0.0);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            bool any_inflight = false;
            for (int k = 0; k < S; ++k) any_inflight = any_inflight || s->inflight[k].on;
            if (!any_inflight && s->incoming.empty() && s->pending.empty())
                s->cv.wait(lk, [&] { return s->stop || !s->incoming.empty(); });
            if (s->stop && s->incoming.empty() && s->pending.empty() && !any_inflight) return;
            while (!s->incoming.empty()) {
                s->pending.push_back(s->incoming.front());
                s->incoming.pop_front();
            }
            // Admission between Newton iterations, in arrival order, under the
            // lock (submitters may add sessions meanwhile); a session with a
            // request in flight keeps its later requests waiting.
            for (auto it = s->pending.begin(); it != s->pending.end();) {
                Session& ss = s->sessions[it->session];
                if (ss.busy) {
                    ++it;
                    continue;
                }
                const int k = find_slot(s, it->session, ss);
                if (k == -2) {
                    s->error = FFTG_ECUDA;
                    s->cv.notify_all();
                    return;
                }
                if (k < 0) {  // every cell busy: this request waits, resident ones may go
                    ++it;
                    continue;
                }
                Inflight& f = s->inflight[k];
                f.on = true;
                f.req = *it;
                f.it = 0;
                f.t_start = now_s();
                double Et[6];
                const double* E = committed_E(s->h, k);
                for (int c = 0; c < 6; ++c) Et[c] = E[c] + it->dE[c];
                f.normE = std::sqrt((double)voxels(s->h)) * frob6(Et);
                reset_stats(s->h, k);
                if (set_trial_strain(s->h, k, Et, true)) {
                    s->error = FFTG_ECUDA;
                    s->cv.notify_all();
                    return;
                }
                ss.busy = true;
                it = s->pending.erase(it);
            }
        }
        int n_on = 0;
        for (int k = 0; k < S; ++k) {
            run[k] = s->inflight[k].on ? 1 : 0;
            n_on += run[k];
        }
        if (n_on == 0) continue;
        s->max_concurrent = std::max(s->max_concurrent, n_on);
        s->busy_rounds += 1.0;
        s->cells_in_rounds += n_on;
        if (newton_round(s->h, run.data(), s->tol_inner, ro.data())) {
            s->error = FFTG_ECUDA;
            return;
        }
        bool any_fin = false;
        for (int k = 0; k < S; ++k) {
            fin[k] = 0;
            code[k] = FFTG_OK;
            if (!run[k]) continue;
            Inflight& f = s->inflight[k];
            const int d = newton_decide(s->h, k, ro[k], f.normE, s->tol_newton, &f.it);
            if (d == 1) {
                fin[k] = 1;
                any_fin = true;
            } else if (d < 0) {
                set_status(s->h, k, d);
                code[k] = d;  // failed: reported, not committed
            }
        }
        if (any_fin && finish_cells(s->h, fin.data(), sig.data())) {
            s->error = FFTG_ECUDA;
            std::lock_guard<std::mutex> lk(s->mu);
            s->cv.notify_all();
            return;
        }
        const double t = now_s();
        std::lock_guard<std::mutex> lk(s->mu);
        for (int k = 0; k < S; ++k) {
            if (!run[k] || (fin[k] == 0 && code[k] == FFTG_OK)) continue;
            Inflight& f = s->inflight[k];
            fftg_result r{};
            r.request_id = f.req.id;
            r.session_id = f.req.session;
            r.status = fin[k] == 1 ? FFTG_OK : code[k];
            r.newton_iters = f.it;
            fftg_stats stt;
            fftg_select_cell(s->h, k);
            fftg_last_stats(s->h, &stt);
            r.cg_iters = stt.cg_iters;
            if (fin[k] == 1)
                for (int c = 0; c < 6; ++c) r.sigma[c] = sig[6 * k + c];
            r.t_submit = f.req.t_submit;
            r.t_start = f.t_start;
            r.t_done = t;
            s->done.push_back(r);
            Session& ss = s->sessions[f.req.session];
            ss.busy = false;
            ss.last_used = t;
            f.on = false;
            ++s->n_completed;
        }
        s->cv.notify_all();
    }
}

}  // namespace

extern "C" {

double fftg_server_clock(void) { return now_s(); }

int fftg_server_start(fftg_server** out, int N, int slots, int nphase, const fftg_phase* mats,
                      const fftg_options* opt, double tol_newton, double tol_cg) {
    if (!out || slots < 1 || !mats || nphase < 1 || !(tol_newton > 0) || !(tol_cg > 0)) return FFTG_EINVAL;
    *out = nullptr;
    fftg_server* s = new (std::nothrow) fftg_server();
    if (!s) return FFTG_ENOMEM;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return FFTG_ECUDA;
    }
    fftg_options o;
    if (opt) o = *opt; else fftg_default_options(&o);
    o.stream = s->stream;
    o.workspace = nullptr;  // the server owns its memory
    o.workspace_bytes = 0;
    o.nrhs_tangent = 0;
    std::vector<uint8_t> zero((size_t)N * N * N * slots, 0);
    int rc = fftg_create_batch(&s->h, N, slots, zero.data(), nphase, mats, &o);
    if (rc) {
        cudaStreamDestroy(s->stream);
        delete s;
        return rc;
    }
    s->N = N;
    s->slots = slots;
    s->tol_newton = tol_newton;
    s->tol_cg = tol_cg;
    s->tol_inner = is_mixed(s->h) ? std::max(tol_cg, o.cg_inner_floor) : tol_cg;
    s->slot_session.assign(slots, -1);
    s->inflight.assign(slots, Inflight{});
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return FFTG_OK;
}

int fftg_server_submit(fftg_server* s, long long request_id, long long session_id, const uint8_t* phase,
                       const double dE[6]) {
    if (!s || !dE) return FFTG_EINVAL;
    for (int c = 0; c < 6; ++c)
        if (!std::isfinite(dE[c])) return FFTG_ENAN;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return s->error;
    auto it = s->sessions.find(session_id);
    if (it == s->sessions.end()) {
        if (!phase) return FFTG_EINVAL;  // a new session needs its microstructure
        Session ss;
        const size_t V = (size_t)s->N * s->N * s->N;
        ss.phase.assign(phase, phase + V);
        s->sessions.emplace(session_id, std::move(ss));
    }
    Request r;
    r.id = request_id;
    r.session = session_id;
    std::memcpy(r.dE, dE, sizeof(r.dE));
    r.t_submit = now_s();
    s->incoming.push_back(r);
    s->cv.notify_all();
    return FFTG_OK;
}

int fftg_server_poll(fftg_server* s, fftg_result* out, int max, int* n, double wait_s) {
    if (!s || !out || !n || max < 1) return FFTG_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_s > 0)
        s->cv.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return !s->done.empty() || s->error; });
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n = k;
    return s->error;
}

int fftg_server_cancel_pending(fftg_server* s, long long* cancelled) {
    if (!s) return FFTG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const long long n = (long long)(s->incoming.size() + s->pending.size());
    s->incoming.clear();
    s->pending.clear();
    if (cancelled) *cancelled = n;
    return s->error;
}

int fftg_server_info(fftg_server* s, long long* completed, long long* evictions, long long* restores,
                     int* max_concurrent, double* mean_batch) {
    if (!s) return FFTG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->n_completed;
    if (evictions) *evictions = s->n_evictions;
    if (restores) *restores = s->n_restores;
    if (max_concurrent) *max_concurrent = s->max_concurrent;
    if (mean_batch) *mean_batch = s->busy_rounds > 0 ? s->cells_in_rounds / s->busy_rounds : 0.0;
    return s->error;
}

int fftg_server_stop(fftg_server* s) {
    if (!s) return FFTG_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    const int err = s->error;
    fftg_destroy(s->h);
    cudaStreamDestroy(s->stream);
    delete s;
    return err;
}

}  // extern "C"

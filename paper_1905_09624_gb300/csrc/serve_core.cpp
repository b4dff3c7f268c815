// Continuous-batching serve scheduler (device-independent part of the serve loop).
//
// One scheduler thread owns the backend's slots.  Requests wait in a FIFO until
// the score-buffer budget and a free slot admit them; everything admitted since
// the last launch forms the next wave (one batched launch sequence).  Waves on
// different slots overlap on the device.  A wave's completion is polled, never
// waited for; its results go to per-ticket entries and its budget is returned.
// Every wait is bounded by wait_timeout_ms: a wave that does not finish in time
// fails its tickets with COBS_ERR_TIMEOUT and its slot stays out of use until
// the backend reports it finished.  A cancelled ticket is dropped from the
// queue or, if already on the device, its result is discarded when the wave
// finishes (the budget it holds returns then).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "serve_core.h"

using namespace cobs;
using namespace cobs::serve;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Slot {
    bool busy = false;
    bool timed_out = false;  // its tickets already failed; the backend still runs the wave
    double t_launch = 0;
    uint64_t cost = 0;
    std::vector<Request> reqs;
};

}  // namespace

struct cobs_server {
    std::unique_ptr<Backend> be;
    cobs_serve_cfg cfg{};
    std::thread sched;
    std::mutex mu;
    std::condition_variable cv;
    bool stopping = false;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> done;
    std::unordered_set<uint64_t> waiting;    // submitted, not finished, not cancelled
    std::unordered_set<uint64_t> cancelled;  // cancelled while queued or on the device
    uint64_t next_ticket = 1;
    uint64_t budget_used = 0;
    std::vector<Slot> slots;
    std::vector<double> lat_ms;
    uint64_t completed = 0, waves = 0, rejected = 0, n_cancelled = 0, failed = 0;
    double wave_ms_sum = 0, wave_ms_max = 0;
    uint64_t wave_queries = 0;
    double t_first = -1, t_last = 0;
};

namespace {

// Results of a finished wave (lock held on entry and exit; released while the
// backend copies the results out).
void collect_wave(cobs_server *S, uint32_t si, std::unique_lock<std::mutex> &lk) {
    Slot &sl = S->slots[si];
    std::vector<Result> res;
    lk.unlock();
    cobs_status st = S->be->collect(si, res);
    lk.lock();
    if (st == COBS_OK && res.size() != sl.reqs.size())
        st = set_error(COBS_ERR_ARG, "backend returned %zu results for %zu requests", res.size(), sl.reqs.size());
    const double t = now_s();
    for (size_t i = 0; i < sl.reqs.size(); i++) {
        const Request &r = sl.reqs[i];
        if (S->cancelled.erase(r.ticket)) continue;  // its entry already says CANCELLED (or was released)
        Result d;
        if (st == COBS_OK) d = std::move(res[i]);
        else d.status = st;
        if (d.status != COBS_OK) S->failed++;
        S->done[r.ticket] = std::move(d);
        S->waiting.erase(r.ticket);
        S->lat_ms.push_back((t - r.t_submit) * 1e3);
        S->completed++;
    }
    S->t_last = t;
    const double wave_ms = (t - sl.t_launch) * 1e3;
    S->wave_ms_sum += wave_ms;
    S->wave_ms_max = std::max(S->wave_ms_max, wave_ms);
    S->wave_queries += sl.reqs.size();
    S->budget_used -= sl.cost;
    sl.cost = 0;
    sl.reqs.clear();
    sl.busy = false;
    S->cv.notify_all();
}

// Fail every ticket of a wave with `st` and return its budget.
void fail_wave(cobs_server *S, Slot &sl, cobs_status st) {
    for (const Request &r : sl.reqs) {
        if (S->cancelled.erase(r.ticket)) continue;
        Result d;
        d.status = st;
        S->done[r.ticket] = std::move(d);
        S->waiting.erase(r.ticket);
        S->failed++;
    }
    S->budget_used -= sl.cost;
    sl.cost = 0;
    sl.reqs.clear();
    S->cv.notify_all();
}

void scheduler(cobs_server *S) {
    S->be->thread_init();
    std::unique_lock<std::mutex> lk(S->mu);
    const double timeout_s = S->cfg.wait_timeout_ms / 1e3;
    for (;;) {
        bool any_busy = false;
        // 1. completions
        for (uint32_t si = 0; si < S->slots.size(); si++) {
            Slot &sl = S->slots[si];
            if (!sl.busy) continue;
            const int q = S->be->poll(si);
            if (sl.timed_out) {
                if (q != 0) sl.busy = sl.timed_out = false;  // the late wave is over: the slot is usable again
                continue;
            }
            if (q == 1) {
                collect_wave(S, si, lk);
            } else if (q < 0) {
                sl.busy = false;
                fail_wave(S, sl, (cobs_status)q);
            } else if (now_s() - sl.t_launch > timeout_s) {
                // device work cannot be cancelled: the slot stays busy until it ends
                set_error(COBS_ERR_TIMEOUT, "wave did not finish within %u ms", S->cfg.wait_timeout_ms);
                fail_wave(S, sl, COBS_ERR_TIMEOUT);
                sl.timed_out = true;
            } else {
                any_busy = true;
            }
        }
        // 2. admission: everything that fits the budget, into the next free slot
        for (uint32_t si = 0; si < S->slots.size(); si++) {
            Slot &sl = S->slots[si];
            if (sl.busy || S->queue.empty()) continue;
            while (!S->queue.empty() && sl.reqs.size() < S->cfg.max_wave_queries) {
                Request &f = S->queue.front();
                if (S->cancelled.count(f.ticket)) {  // cancelled while queued: never launched
                    S->cancelled.erase(f.ticket);
                    S->queue.pop_front();
                    continue;
                }
                if (S->budget_used + f.cost > S->cfg.score_budget_bytes) break;
                S->budget_used += f.cost;
                sl.cost += f.cost;
                sl.reqs.push_back(std::move(f));
                S->queue.pop_front();
            }
            if (sl.reqs.empty()) break;  // budget exhausted: wait for a completion
            lk.unlock();
            cobs_status st = S->be->launch(si, sl.reqs);
            lk.lock();
            if (st != COBS_OK) {
                fail_wave(S, sl, st);
            } else {
                sl.busy = true;
                sl.t_launch = now_s();
                S->waves++;
                any_busy = true;
            }
        }
        if (S->stopping && S->queue.empty() && !any_busy) break;
        // 3. idle: short bounded wait for new requests or a completion
        S->cv.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 500));
    }
}

}  // namespace

namespace cobs {

cobs_status serve_create(std::unique_ptr<Backend> backend, const cobs_serve_cfg *cfg, cobs_server **out) {
    if (!backend || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    cobs_server *S = new cobs_server();
    S->be = std::move(backend);
    if (cfg) S->cfg = *cfg;
    if (!S->cfg.score_budget_bytes) S->cfg.score_budget_bytes = 4ULL << 30;
    if (!S->cfg.max_wave_queries) S->cfg.max_wave_queries = 4096;
    if (!S->cfg.wait_timeout_ms) S->cfg.wait_timeout_ms = 10000;
    S->cfg.max_inflight_waves = S->be->n_slots();
    S->slots.resize(S->be->n_slots());
    S->sched = std::thread(scheduler, S);
    *out = S;
    return COBS_OK;
}

}  // namespace cobs

extern "C" cobs_status cobs_serve_submit(cobs_server *S, const uint8_t *q, uint64_t len, uint16_t thr_permille,
                                         uint64_t *ticket) {
    if (!S || !ticket || (len && !q)) return set_error(COBS_ERR_ARG, "NULL argument");
    if (thr_permille == 0 || thr_permille > 1000) return set_error(COBS_ERR_ARG, "threshold must be 1..1000 permille");
    cobs_status st = S->be->check_request(len);
    if (st != COBS_OK) return st;
    Request r;
    r.cost = S->be->request_cost(len);
    std::lock_guard<std::mutex> lk(S->mu);
    if (r.cost > S->cfg.score_budget_bytes) {
        S->rejected++;
        return set_error(COBS_ERR_BUDGET, "query needs %llu bytes, budget is %llu", (unsigned long long)r.cost,
                         (unsigned long long)S->cfg.score_budget_bytes);
    }
    if (S->stopping) return set_error(COBS_ERR_ARG, "server is stopping");
    r.ticket = S->next_ticket++;
    r.q.assign(q, q + len);
    r.thr = thr_permille;
    r.t_submit = now_s();
    if (S->t_first < 0) S->t_first = r.t_submit;
    S->waiting.insert(r.ticket);
    *ticket = r.ticket;
    S->queue.push_back(std::move(r));
    S->cv.notify_all();
    return COBS_OK;
}

extern "C" cobs_status cobs_serve_poll(cobs_server *S, uint64_t ticket, cobs_hits *out) {
    if (!S || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
        if (S->waiting.count(ticket)) return COBS_PENDING;
        return set_error(COBS_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    }
    const Result &d = it->second;
    if (d.status != COBS_OK) return set_error(d.status, "request failed (%d)", (int)d.status);
    out->n_terms = d.n_terms;
    out->min_score = d.min_score;
    out->n_hits = (uint32_t)d.ids.size();
    out->_pad = 0;
    out->doc_ids = d.ids.data();
    out->scores = d.scores.data();
    return COBS_OK;
}

extern "C" cobs_status cobs_serve_cancel(cobs_server *S, uint64_t ticket) {
    if (!S) return set_error(COBS_ERR_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    const bool is_waiting = S->waiting.count(ticket) != 0;
    if (it == S->done.end() && !is_waiting)
        return set_error(COBS_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (it != S->done.end() && it->second.status == COBS_ERR_CANCELLED) return COBS_OK;  // already cancelled
    if (is_waiting) {  // queued or on the device: its result, if any, is dropped when the wave ends
        S->waiting.erase(ticket);
        S->cancelled.insert(ticket);
    }
    Result d;
    d.status = COBS_ERR_CANCELLED;
    S->done[ticket] = std::move(d);
    S->n_cancelled++;
    S->cv.notify_all();
    return COBS_OK;
}

extern "C" void cobs_hits_release(cobs_server *S, uint64_t ticket) {
    if (!S) return;
    std::lock_guard<std::mutex> lk(S->mu);
    S->done.erase(ticket);
}

extern "C" cobs_status cobs_serve_stop(cobs_server *S, cobs_serve_stats *out) {
    if (!S) return set_error(COBS_ERR_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv.notify_all();
    }
    if (S->sched.joinable()) S->sched.join();
    if (out) {
        memset(out, 0, sizeof *out);
        std::vector<double> l = S->lat_ms;
        std::sort(l.begin(), l.end());
        out->completed = S->completed;
        out->waves = S->waves;
        out->rejected = S->rejected;
        if (!l.empty()) {
            out->p50_ms = l[(l.size() - 1) / 2];
            out->p99_ms = l[std::min(l.size() - 1, (size_t)((l.size() - 1) * 0.99 + 0.5))];
            out->max_ms = l.back();
        }
        out->seconds = S->t_first >= 0 ? S->t_last - S->t_first : 0.0;
        out->qps = out->seconds > 0 ? S->completed / out->seconds : 0.0;
        const double nw = (double)(S->waves ? S->waves : 1);
        out->mean_wave_queries = (double)S->wave_queries / nw;
        out->mean_wave_ms = S->wave_ms_sum / nw;
        out->max_wave_ms = S->wave_ms_max;
        out->cancelled = S->n_cancelled;
        out->failed = S->failed;
    }
    // bounded wait for work still on the device (a timed-out wave), then teardown
    for (uint32_t si = 0; si < S->slots.size(); si++)
        if (S->slots[si].busy) S->be->drain(si, S->cfg.wait_timeout_ms / 1e3);
    delete S;
    return COBS_OK;
}

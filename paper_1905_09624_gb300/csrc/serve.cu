// Continuous-batching serve loop over a resident index.
//
// One scheduler thread owns `max_inflight_waves` slots, each an engine on its
// own stream.  Requests wait in a FIFO until the score-buffer budget and a free
// slot admit them; everything admitted since the last launch forms the next wave
// (batched kernel, one launch sequence).  Waves on different slots overlap on the
// device.  A wave's completion is observed with cudaEventQuery (never a blocking
// wait), its hits are copied into per-ticket results and its budget is returned.
// Every wait is bounded by wait_timeout_ms; a wave that does not finish in time
// fails its tickets with COBS_ERR_TIMEOUT.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host_internal.h"

using namespace cobs;

namespace {

using clk = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(clk::now().time_since_epoch()).count(); }

struct Req {
    uint64_t ticket;
    std::vector<uint8_t> q;
    uint16_t thr;
    double t_submit;
    uint64_t cost;
};

struct Done {
    cobs_status status = COBS_OK;
    uint32_t n_terms = 0, min_score = 0;
    std::vector<uint32_t> ids, scores;
};

struct Slot {
    cobs_engine *eng = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool timed_out = false;  // its tickets already failed; the device work is still running
    double t_launch = 0;
    uint64_t cost = 0;
    std::vector<Req> reqs;
    PinBuf pin;
    DevBuf dbytes, doff, dthr;
    std::vector<uint64_t> hoff;
};

}  // namespace

struct cobs_server {
    cobs_device_index *dix = nullptr;
    cobs_serve_cfg cfg{};
    std::thread sched;
    std::mutex mu;
    std::condition_variable cv;
    bool stopping = false;
    std::deque<Req> queue;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_map<uint64_t, bool> inflight;  // ticket -> admitted
    uint64_t next_ticket = 1;
    uint64_t budget_used = 0;
    std::vector<std::unique_ptr<Slot>> slots;
    std::vector<double> lat_ms;
    uint64_t completed = 0, waves = 0, rejected = 0;
    double wave_ms_sum = 0, wave_ms_max = 0;
    uint64_t wave_queries = 0;
    double t_first = -1, t_last = 0;
    cobs_status fatal = COBS_OK;
};

namespace {

// Device memory a request occupies while in flight: a full score vector at the
// index's score width (the budget unit of the plain form) plus its term arrays
// and distinct-term set.
uint64_t request_cost(const cobs_device_index *dix, uint64_t len) {
    const uint64_t k = dix->params.q;
    const uint64_t np = len >= k ? len - k + 1 : 0;
    const uint64_t region = (np + TERM_ALIGN - 1) / TERM_ALIGN * TERM_ALIGN;
    return dix->n_docs * (dix->params.score_bits / 8) + region * dix->blocks.size() * dix->params.num_hashes * 4 +
           set_slots(np) * 8 + 64;
}

cobs_status launch_wave(cobs_server *S, Slot &sl) {
    const uint64_t n = sl.reqs.size();
    uint64_t total = 0;
    for (const Req &r : sl.reqs) total += r.q.size();
    const uint64_t o1 = (total + 15) / 16 * 16, o2 = o1 + (n + 1) * 8;
    if (sl.pin.ensure(o2 + n * 2 + 16) != cudaSuccess || sl.dbytes.ensure(total) != cudaSuccess ||
        sl.doff.ensure((n + 1) * 8) != cudaSuccess || sl.dthr.ensure(n * 2) != cudaSuccess)
        return set_error(COBS_ERR_OOM, "serve staging buffers");
    uint8_t *pin = sl.pin.as<uint8_t>();
    sl.hoff.assign(n + 1, 0);
    uint64_t pos = 0;
    for (uint64_t i = 0; i < n; i++) {
        memcpy(pin + pos, sl.reqs[i].q.data(), sl.reqs[i].q.size());
        pos += sl.reqs[i].q.size();
        sl.hoff[i + 1] = pos;
        reinterpret_cast<uint16_t *>(pin + o2)[i] = sl.reqs[i].thr;
    }
    memcpy(pin + o1, sl.hoff.data(), (n + 1) * 8);
    if (total && cudaMemcpyAsync(sl.dbytes.p, pin, total, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
        return set_error(COBS_ERR_CUDA, "serve H2D");
    if (cudaMemcpyAsync(sl.doff.p, pin + o1, (n + 1) * 8, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess ||
        cudaMemcpyAsync(sl.dthr.p, pin + o2, n * 2, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
        return set_error(COBS_ERR_CUDA, "serve H2D");
    cobs_status st = engine_query(sl.eng, sl.dbytes.as<uint8_t>(), sl.doff.as<uint64_t>(), sl.hoff.data(),
                                  sl.dthr.as<uint16_t>(), n, COBS_BATCHED);
    if (st != COBS_OK) return st;
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return set_error(COBS_ERR_CUDA, "serve event");
    sl.busy = true;
    sl.t_launch = now_s();
    return COBS_OK;
}

// Collect a finished wave (its event has completed).
void collect_wave(cobs_server *S, Slot &sl, std::unique_lock<std::mutex> &lk) {
    cobs_result *res = nullptr;
    lk.unlock();
    cobs_status st = cobs_engine_download(sl.eng, &res);
    lk.lock();
    double t = now_s();
    for (uint64_t i = 0; i < sl.reqs.size(); i++) {
        const Req &r = sl.reqs[i];
        Done d;
        d.status = st;
        if (st == COBS_OK) {
            const cobs_hits &h = res->hits[i];
            d.n_terms = h.n_terms;
            d.min_score = h.min_score;
            d.ids.assign(h.doc_ids, h.doc_ids + h.n_hits);
            d.scores.assign(h.scores, h.scores + h.n_hits);
        }
        S->done[r.ticket] = std::move(d);
        S->inflight.erase(r.ticket);
        S->lat_ms.push_back((t - r.t_submit) * 1e3);
        S->completed++;
    }
    S->t_last = t;
    const double wave_ms = (t - sl.t_launch) * 1e3;
    S->wave_ms_sum += wave_ms;
    S->wave_ms_max = std::max(S->wave_ms_max, wave_ms);
    S->wave_queries += sl.reqs.size();
    if (res) cobs_result_free(res);
    S->budget_used -= sl.cost;
    sl.cost = 0;
    sl.reqs.clear();
    sl.busy = false;
    S->cv.notify_all();
}

void fail_wave(cobs_server *S, Slot &sl, cobs_status st) {
    for (const Req &r : sl.reqs) {
        Done d;
        d.status = st;
        S->done[r.ticket] = std::move(d);
        S->inflight.erase(r.ticket);
    }
    S->budget_used -= sl.cost;
    sl.cost = 0;
    sl.reqs.clear();
    S->cv.notify_all();
}

void scheduler(cobs_server *S) {
    cudaSetDevice(S->dix->device);
    std::unique_lock<std::mutex> lk(S->mu);
    const double timeout_s = S->cfg.wait_timeout_ms / 1e3;
    for (;;) {
        bool any_busy = false;
        // 1. completions
        for (auto &sp : S->slots) {
            Slot &sl = *sp;
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (sl.timed_out) {
                if (q != cudaErrorNotReady) sl.busy = sl.timed_out = false;
                continue;
            }
            if (q == cudaSuccess) {
                collect_wave(S, sl, lk);
            } else if (q != cudaErrorNotReady) {
                sl.busy = false;
                fail_wave(S, sl, set_error(COBS_ERR_CUDA, "wave failed: %s", cudaGetErrorString(q)));
            } else if (now_s() - sl.t_launch > timeout_s) {
                // The device work cannot be cancelled; the slot stays unusable.
                set_error(COBS_ERR_TIMEOUT, "wave did not finish within %u ms", S->cfg.wait_timeout_ms);
                fail_wave(S, sl, COBS_ERR_TIMEOUT);
                sl.timed_out = true;
            } else {
                any_busy = true;
            }
        }
        // 2. admission: everything that fits the budget, into the next free slot
        for (auto &sp : S->slots) {
            Slot &sl = *sp;
            if (sl.busy || S->queue.empty()) continue;
            while (!S->queue.empty() && sl.reqs.size() < S->cfg.max_wave_queries &&
                   S->budget_used + S->queue.front().cost <= S->cfg.score_budget_bytes) {
                S->budget_used += S->queue.front().cost;
                sl.cost += S->queue.front().cost;
                S->inflight[S->queue.front().ticket] = true;
                sl.reqs.push_back(std::move(S->queue.front()));
                S->queue.pop_front();
            }
            if (sl.reqs.empty()) break;  // budget exhausted: wait for a completion
            lk.unlock();
            cobs_status st = launch_wave(S, sl);
            lk.lock();
            if (st != COBS_OK) fail_wave(S, sl, st);
            else {
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

extern "C" cobs_status cobs_serve_start(cobs_device_index *dix, const cobs_serve_cfg *cfg, cobs_server **out) {
    if (!dix || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    if (cudaSetDevice(dix->device) != cudaSuccess) return set_error(COBS_ERR_CUDA, "cudaSetDevice");
    cobs_server *S = new cobs_server();
    S->dix = dix;
    if (cfg) S->cfg = *cfg;
    if (!S->cfg.score_budget_bytes) S->cfg.score_budget_bytes = 4ULL << 30;
    if (!S->cfg.max_inflight_waves) S->cfg.max_inflight_waves = 2;
    if (!S->cfg.max_wave_queries) S->cfg.max_wave_queries = 4096;
    if (!S->cfg.wait_timeout_ms) S->cfg.wait_timeout_ms = 10000;
    for (uint32_t i = 0; i < S->cfg.max_inflight_waves; i++) S->slots.emplace_back(new Slot());
    for (auto &sp : S->slots) {
        Slot &sl = *sp;
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        cobs_engine_cfg ec{};
        cobs_status st = cobs_engine_create(dix, &ec, sl.stream, &sl.eng);
        if (st != COBS_OK) {
            cobs_serve_stop(S, nullptr);
            return st;
        }
    }
    S->sched = std::thread(scheduler, S);
    *out = S;
    return COBS_OK;
}

extern "C" cobs_status cobs_serve_submit(cobs_server *S, const uint8_t *q, uint64_t len, uint16_t thr_permille,
                                         uint64_t *ticket) {
    if (!S || !ticket || (len && !q)) return set_error(COBS_ERR_ARG, "NULL argument");
    if (thr_permille == 0 || thr_permille > 1000) return set_error(COBS_ERR_ARG, "threshold must be 1..1000 permille");
    const cobs_params &P = S->dix->params;
    const uint64_t np = len >= P.q ? len - P.q + 1 : 0;
    if (np > (P.score_bits == 16 ? 0xFFFFULL : 0xFFFFFFFFULL))
        return set_error(COBS_ERR_OVERFLOW, "query has more windows than the score width counts");
    Req r;
    r.cost = request_cost(S->dix, len);
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
    S->inflight[r.ticket] = false;
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
        if (S->inflight.count(ticket)) return COBS_PENDING;
        return set_error(COBS_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    }
    const Done &d = it->second;
    if (d.status != COBS_OK) return set_error(d.status, "request failed (%d)", (int)d.status);
    out->n_terms = d.n_terms;
    out->min_score = d.min_score;
    out->n_hits = (uint32_t)d.ids.size();
    out->_pad = 0;
    out->doc_ids = d.ids.data();
    out->scores = d.scores.data();
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
    }
    for (auto &sp : S->slots) {
        Slot &sl = *sp;
        // bounded wait for work still on the device (a timed-out wave)
        double t0 = now_s();
        while (sl.done && cudaEventQuery(sl.done) == cudaErrorNotReady && now_s() - t0 < S->cfg.wait_timeout_ms / 1e3)
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        if (sl.eng) cobs_engine_free(sl.eng);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete S;
    return COBS_OK;
}

// Test backend for the serve scheduler (paper_1905_09624_gb300/csrc/serve_core.cpp):
// waves run on no device, so admission, budget back-pressure, cancellation,
// wave failures, launch failures and timeouts are exercised on the host alone.
// Built by the tests with g++ together with serve_core.cpp and status.cpp; the
// library proper never contains it.
//
// A wave finishes `wave_us` microseconds after its launch.  Wave number
// `fail_launch_wave` fails at launch (as an allocation failure would), wave
// `fail_wave` reports a failure when polled, wave `hang_wave` never finishes
// until mock_release_hang().  The result of a request is a function of its bytes
// that the tests recompute: n_terms = max(0, len - q + 1), min_score =
// ceil(thr * n_terms / 1000), hits = {(fnv1a(bytes) % 1000, n_terms),
// (fnv1a(bytes) % 1000 + 1, min_score)}.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "serve_core.h"

using namespace cobs;

extern "C" {
typedef struct mock_cfg {
    uint32_t n_slots;
    uint32_t q;
    uint32_t wave_us;
    int32_t fail_launch_wave;
    int32_t fail_wave;
    int32_t hang_wave;
    uint64_t cost_base;
    uint64_t cost_per_byte;
    uint64_t max_windows;  // submit refuses longer queries with COBS_ERR_OVERFLOW (0 = no limit)
} mock_cfg;

typedef struct mock_stats {
    uint64_t launched_waves;
    uint64_t launched_requests;
    uint64_t finished_waves;     // polled as finished (or failed)
    uint64_t inflight_cost;      // cost of launched requests whose wave has not finished
    uint64_t max_inflight_cost;  // its maximum
    uint64_t max_wave_requests;
    uint64_t launch_order_ok;    // 1 while every wave's tickets were launched in submission order
} mock_stats;
}

namespace {

double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

uint32_t fnv1a(const std::vector<uint8_t> &b) {
    uint32_t h = 2166136261u;
    for (uint8_t c : b) h = (h ^ c) * 16777619u;
    return h;
}

class MockBackend;
std::mutex g_mu;
MockBackend *g_last = nullptr;  // the most recent live mock (owned by its server)

struct MockWave {
    int64_t number = -1;
    double t_launch = 0;
    uint64_t cost = 0;
    bool finished = true;
    std::vector<serve::Result> results;
};

class MockBackend final : public serve::Backend {
public:
    explicit MockBackend(const mock_cfg &c) : c_(c), slots_(c.n_slots ? c.n_slots : 2) {
        memset(&st_, 0, sizeof st_);
        st_.launch_order_ok = 1;
    }
    ~MockBackend() override {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_last == this) g_last = nullptr;
    }
    uint32_t n_slots() const override { return (uint32_t)slots_.size(); }
    uint64_t request_cost(uint64_t len) const override { return c_.cost_base + c_.cost_per_byte * len; }
    cobs_status check_request(uint64_t len) const override {
        const uint64_t np = len >= c_.q ? len - c_.q + 1 : 0;
        if (c_.max_windows && np > c_.max_windows) return set_error(COBS_ERR_OVERFLOW, "mock: too many windows");
        return COBS_OK;
    }
    cobs_status launch(uint32_t slot, const std::vector<serve::Request> &reqs) override {
        std::lock_guard<std::mutex> lk(mu_);
        const int64_t number = next_wave_++;
        if (number == c_.fail_launch_wave) return set_error(COBS_ERR_OOM, "mock: injected launch failure");
        MockWave &w = slots_[slot];
        w.number = number;
        w.t_launch = now_us();
        w.finished = false;
        w.cost = 0;
        w.results.clear();
        for (const serve::Request &r : reqs) {
            if (r.ticket <= last_ticket_) st_.launch_order_ok = 0;
            last_ticket_ = r.ticket;
            w.cost += request_cost(r.q.size());
            serve::Result d;
            const uint64_t len = r.q.size();
            d.n_terms = (uint32_t)(len >= c_.q ? len - c_.q + 1 : 0);
            d.min_score = (uint32_t)(((uint64_t)r.thr * d.n_terms + 999) / 1000);
            const uint32_t id = fnv1a(r.q) % 1000u;
            d.ids = {id, id + 1};
            d.scores = {d.n_terms, d.min_score};
            w.results.push_back(std::move(d));
        }
        st_.launched_waves++;
        st_.launched_requests += reqs.size();
        st_.max_wave_requests = std::max<uint64_t>(st_.max_wave_requests, reqs.size());
        st_.inflight_cost += w.cost;
        st_.max_inflight_cost = std::max(st_.max_inflight_cost, st_.inflight_cost);
        return COBS_OK;
    }
    int poll(uint32_t slot) override {
        std::lock_guard<std::mutex> lk(mu_);
        MockWave &w = slots_[slot];
        if (w.finished) return 1;
        int r = 0;
        if (w.number == c_.fail_wave) r = (int)set_error(COBS_ERR_CUDA, "mock: injected wave failure");
        else if (w.number == c_.hang_wave && !hang_released_) r = 0;
        else if (now_us() - w.t_launch >= c_.wave_us) r = 1;
        if (r != 0) {
            w.finished = true;
            st_.finished_waves++;
            st_.inflight_cost -= w.cost;
        }
        return r;
    }
    cobs_status collect(uint32_t slot, std::vector<serve::Result> &out) override {
        std::lock_guard<std::mutex> lk(mu_);
        out = std::move(slots_[slot].results);
        slots_[slot].results.clear();
        return COBS_OK;
    }
    void drain(uint32_t, double) override {}

    void stats(mock_stats *out) {
        std::lock_guard<std::mutex> lk(mu_);
        *out = st_;
    }
    void release_hang() {
        std::lock_guard<std::mutex> lk(mu_);
        hang_released_ = true;
    }

private:
    mock_cfg c_;
    std::mutex mu_;
    std::vector<MockWave> slots_;
    int64_t next_wave_ = 0;
    uint64_t last_ticket_ = 0;
    bool hang_released_ = false;
    mock_stats st_;
};

}  // namespace

extern "C" cobs_status mock_serve_start(const cobs_serve_cfg *cfg, const mock_cfg *mc, cobs_server **out) {
    if (!mc) return set_error(COBS_ERR_ARG, "NULL mock config");
    std::unique_ptr<MockBackend> be(new MockBackend(*mc));
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_last = be.get();
    }
    return serve_create(std::move(be), cfg, out);
}

// Counters of the most recent mock that is still alive (zeros once its server stopped).
extern "C" void mock_get_stats(mock_stats *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    memset(out, 0, sizeof *out);
    if (g_last) g_last->stats(out);
}

extern "C" void mock_release_hang(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_last) g_last->release_hang();
}

// Several client threads submit, poll and cancel concurrently against the serve
// scheduler on the mock backend (serve_mock.cpp).  The tests build it with
// -fsanitize=thread (data races) and with -fsanitize=address,undefined (memory
// errors) and expect exit status 0 and no sanitizer report.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <thread>
#include <vector>

#include "cobs_gpu.h"

extern "C" {
typedef struct mock_cfg {
    uint32_t n_slots, q, wave_us;
    int32_t fail_launch_wave, fail_wave, hang_wave;
    uint64_t cost_base, cost_per_byte, max_windows;
} mock_cfg;
cobs_status mock_serve_start(const cobs_serve_cfg *cfg, const mock_cfg *mc, cobs_server **out);
}

static uint32_t fnv1a(const std::vector<uint8_t> &b) {
    uint32_t h = 2166136261u;
    for (uint8_t c : b) h = (h ^ c) * 16777619u;
    return h;
}

int main() {
    const uint32_t Q = 4;
    mock_cfg mc = {3, Q, 300, -1, 5, -1, 100, 1, 0};  // wave 5 fails when polled
    cobs_serve_cfg cfg = {4000, 0, 16, 5000, 0};       // budget for a handful of requests
    cobs_server *srv = nullptr;
    if (mock_serve_start(&cfg, &mc, &srv) != COBS_OK) return 2;
    std::atomic<int> errors{0}, ok{0}, cancelled{0}, failed{0};
    auto client = [&](uint32_t seed) {
        uint64_t x = seed * 0x9E3779B97F4A7C15ULL + 1;
        auto rnd = [&]() { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return x; };
        struct T { uint64_t ticket; std::vector<uint8_t> q; uint16_t thr; bool cancel; };
        std::vector<T> mine;
        for (int i = 0; i < 200; i++) {
            T t;
            t.q.resize(rnd() % 300);
            for (auto &c : t.q) c = (uint8_t)("ACGT"[rnd() & 3]);
            t.thr = (uint16_t)(1 + rnd() % 1000);
            t.cancel = rnd() % 5 == 0;
            cobs_status st = cobs_serve_submit(srv, t.q.data(), t.q.size(), t.thr, &t.ticket);
            if (st != COBS_OK) { errors++; continue; }
            if (t.cancel && cobs_serve_cancel(srv, t.ticket) != COBS_OK) errors++;
            mine.push_back(std::move(t));
        }
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(20);
        for (const T &t : mine) {
            cobs_hits h;
            cobs_status st;
            while ((st = cobs_serve_poll(srv, t.ticket, &h)) == COBS_PENDING) {
                if (std::chrono::steady_clock::now() > deadline) { errors++; return; }
                std::this_thread::sleep_for(std::chrono::microseconds(50));
            }
            if (t.cancel) {
                if (st != COBS_ERR_CANCELLED) errors++;
                cancelled++;
            } else if (st == COBS_ERR_CUDA) {
                failed++;
            } else if (st == COBS_OK) {
                const uint32_t nt = t.q.size() >= Q ? (uint32_t)(t.q.size() - Q + 1) : 0;
                const uint32_t mn = (uint32_t)(((uint64_t)t.thr * nt + 999) / 1000);
                if (h.n_terms != nt || h.min_score != mn || h.n_hits != 2 || h.doc_ids[0] != fnv1a(t.q) % 1000u ||
                    h.scores[0] != nt || h.scores[1] != mn)
                    errors++;
                ok++;
            } else {
                errors++;
            }
            cobs_hits_release(srv, t.ticket);
            if (cobs_serve_poll(srv, t.ticket, &h) != COBS_ERR_NOT_FOUND) errors++;
        }
    };
    std::vector<std::thread> th;
    for (uint32_t i = 0; i < 4; i++) th.emplace_back(client, i + 1);
    for (auto &t : th) t.join();
    cobs_serve_stats st;
    if (cobs_serve_stop(srv, &st) != COBS_OK) errors++;
    if (st.cancelled != (uint64_t)cancelled.load()) errors++;
    if (st.completed < (uint64_t)ok.load()) errors++;
    std::printf("ok %d cancelled %d failed %d errors %d waves %llu\n", ok.load(), cancelled.load(), failed.load(),
                errors.load(), (unsigned long long)st.waves);
    return errors.load() == 0 && failed.load() > 0 ? 0 : 1;
}

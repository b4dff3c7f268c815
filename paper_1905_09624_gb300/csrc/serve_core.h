// Continuous-batching serve scheduler, independent of the device.
//
// The scheduler (serve_core.cpp) owns the request queue, the score-buffer
// budget, the tickets and the latency statistics; a Backend runs the waves.
// The library's backend (serve.cu) gives every slot a query engine on its own
// stream; a test backend can stand in for the device to exercise admission,
// cancellation, failures and timeouts on the host alone.  This header needs no
// CUDA headers.
#pragma once
#include <cstdint>
#include <memory>
#include <vector>

#include "status.h"

namespace cobs {
namespace serve {

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> q;  // the query bytes (copied at submit)
    uint16_t thr = 0;        // threshold, permille
    double t_submit = 0;     // seconds, steady clock
    uint64_t cost = 0;       // budget units held while admitted
};

struct Result {
    cobs_status status = COBS_OK;
    uint32_t n_terms = 0, min_score = 0;
    std::vector<uint32_t> ids, scores;
};

// One wave in flight per slot.  Called from the scheduler thread only, except
// check_request and request_cost (any thread).
class Backend {
public:
    virtual ~Backend() = default;
    virtual uint32_t n_slots() const = 0;
    // Called once on the scheduler thread before anything else (device binding).
    virtual void thread_init() {}
    // Budget units a query of `len` bytes holds while admitted.
    virtual uint64_t request_cost(uint64_t len) const = 0;
    // COBS_OK or the status that refuses the query at submit (e.g. overflow).
    virtual cobs_status check_request(uint64_t len) const = 0;
    // Start a wave of requests on a free slot; returns without waiting.
    virtual cobs_status launch(uint32_t slot, const std::vector<Request> &reqs) = 0;
    // 1 = the slot's wave has finished, 0 = still running, < 0 = it failed (status).
    virtual int poll(uint32_t slot) = 0;
    // Results of a finished wave, one per request in launch order.
    virtual cobs_status collect(uint32_t slot, std::vector<Result> &out) = 0;
    // Bounded wait (seconds) for work a slot still has in flight, before teardown.
    virtual void drain(uint32_t slot, double timeout_s) = 0;
};

}  // namespace serve

// Start the scheduler thread over a backend (takes ownership).  cfg may be NULL.
cobs_status serve_create(std::unique_ptr<serve::Backend> backend, const cobs_serve_cfg *cfg, cobs_server **out);

}  // namespace cobs

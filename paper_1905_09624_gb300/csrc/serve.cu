// The serve loop's device backend: every slot is a query engine on its own
// stream; a wave is one batched launch sequence of the engine, its completion an
// event polled with cudaEventQuery (never a blocking wait).  The scheduler
// itself (queue, budget, tickets, timeouts) is serve_core.cpp.
#include <chrono>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "host_internal.h"
#include "serve_core.h"

using namespace cobs;

namespace {

struct CudaSlot {
    cobs_engine *eng = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint64_t n = 0;
    PinBuf pin;
    DevBuf dbytes, doff, dthr;
    std::vector<uint64_t> hoff;
};

class CudaBackend final : public serve::Backend {
public:
    CudaBackend(cobs_device_index *dix, uint32_t flags) : dix_(dix), flags_(flags) {}

    ~CudaBackend() override {
        for (auto &sp : slots_) {
            if (sp->eng) cobs_engine_free(sp->eng);
            if (sp->done) cudaEventDestroy(sp->done);
            if (sp->stream) cudaStreamDestroy(sp->stream);
        }
    }

    cobs_status init(uint32_t n_slots) {
        for (uint32_t i = 0; i < n_slots; i++) {
            slots_.emplace_back(new CudaSlot());
            CudaSlot &sl = *slots_.back();
            if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
                return set_error(COBS_ERR_CUDA, "serve slot stream / event");
            cobs_engine_cfg ec{};
            cobs_status st = cobs_engine_create(dix_, &ec, sl.stream, &sl.eng);
            if (st != COBS_OK) return st;
        }
        return COBS_OK;
    }

    uint32_t n_slots() const override { return (uint32_t)slots_.size(); }

    void thread_init() override { cudaSetDevice(dix_->device); }

    // Device memory a request occupies while in flight: a full score vector at
    // the index's score width (the budget unit of the plain form) plus its term
    // arrays and distinct-term set.
    uint64_t request_cost(uint64_t len) const override {
        const uint64_t k = dix_->params.q;
        const uint64_t np = len >= k ? len - k + 1 : 0;
        const uint64_t region = (np + TERM_ALIGN - 1) / TERM_ALIGN * TERM_ALIGN;
        return dix_->n_docs * (dix_->params.score_bits / 8) +
               region * dix_->blocks.size() * dix_->params.num_hashes * 4 + set_slots(np) * 8 + 64;
    }

    cobs_status check_request(uint64_t len) const override {
        const cobs_params &P = dix_->params;
        const uint64_t np = len >= P.q ? len - P.q + 1 : 0;
        if (np > (P.score_bits == 16 ? 0xFFFFULL : 0xFFFFFFFFULL))
            return set_error(COBS_ERR_OVERFLOW, "query has more windows than the score width counts");
        return COBS_OK;
    }

    cobs_status launch(uint32_t slot, const std::vector<serve::Request> &reqs) override {
        TraceRange tr("cobs.serve.launch");
        CudaSlot &sl = *slots_[slot];
        const uint64_t n = reqs.size();
        uint64_t total = 0;
        for (const serve::Request &r : reqs) total += r.q.size();
        const uint64_t o1 = (total + 15) / 16 * 16, o2 = o1 + (n + 1) * 8;
        if (sl.pin.ensure(o2 + n * 2 + 16) != cudaSuccess || sl.dbytes.ensure(total) != cudaSuccess ||
            sl.doff.ensure((n + 1) * 8) != cudaSuccess || sl.dthr.ensure(n * 2) != cudaSuccess)
            return set_error(COBS_ERR_OOM, "serve staging buffers");
        uint8_t *pin = sl.pin.as<uint8_t>();
        sl.hoff.assign(n + 1, 0);
        uint64_t pos = 0;
        for (uint64_t i = 0; i < n; i++) {
            memcpy(pin + pos, reqs[i].q.data(), reqs[i].q.size());
            pos += reqs[i].q.size();
            sl.hoff[i + 1] = pos;
            reinterpret_cast<uint16_t *>(pin + o2)[i] = reqs[i].thr;
        }
        memcpy(pin + o1, sl.hoff.data(), (n + 1) * 8);
        if (total && cudaMemcpyAsync(sl.dbytes.p, pin, total, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            return set_error(COBS_ERR_CUDA, "serve H2D");
        if (cudaMemcpyAsync(sl.doff.p, pin + o1, (n + 1) * 8, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess ||
            cudaMemcpyAsync(sl.dthr.p, pin + o2, n * 2, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            return set_error(COBS_ERR_CUDA, "serve H2D");
        cobs_status st = engine_query(sl.eng, sl.dbytes.as<uint8_t>(), sl.doff.as<uint64_t>(), sl.hoff.data(),
                                      sl.dthr.as<uint16_t>(), n, flags_);
        if (st != COBS_OK) return st;
        if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return set_error(COBS_ERR_CUDA, "serve event");
        sl.n = n;
        return COBS_OK;
    }

    int poll(uint32_t slot) override {
        const cudaError_t q = cudaEventQuery(slots_[slot]->done);
        if (q == cudaSuccess) return 1;
        if (q == cudaErrorNotReady) return 0;
        return (int)set_error(COBS_ERR_CUDA, "wave failed: %s", cudaGetErrorString(q));
    }

    cobs_status collect(uint32_t slot, std::vector<serve::Result> &out) override {
        TraceRange tr("cobs.serve.collect");
        CudaSlot &sl = *slots_[slot];
        cobs_result *res = nullptr;
        const cobs_status st = cobs_engine_download(sl.eng, &res);
        if (st != COBS_OK) return st;
        out.resize(sl.n);
        for (uint64_t i = 0; i < sl.n; i++) {
            const cobs_hits &h = res->hits[i];
            serve::Result &d = out[i];
            d.n_terms = h.n_terms;
            d.min_score = h.min_score;
            d.ids.assign(h.doc_ids, h.doc_ids + h.n_hits);
            d.scores.assign(h.scores, h.scores + h.n_hits);
        }
        cobs_result_free(res);
        return COBS_OK;
    }

    void drain(uint32_t slot, double timeout_s) override {
        const auto t0 = std::chrono::steady_clock::now();
        while (cudaEventQuery(slots_[slot]->done) == cudaErrorNotReady &&
               std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() < timeout_s)
            std::this_thread::sleep_for(std::chrono::microseconds(100));
    }

private:
    cobs_device_index *dix_;
    uint32_t flags_;  // COBS_BATCHED or COBS_PLAIN
    std::vector<std::unique_ptr<CudaSlot>> slots_;
};

}  // namespace

extern "C" cobs_status cobs_serve_start(cobs_device_index *dix, const cobs_serve_cfg *cfg, cobs_server **out) {
    if (!dix || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    if (cudaSetDevice(dix->device) != cudaSuccess) return set_error(COBS_ERR_CUDA, "cudaSetDevice");
    const uint32_t form = cfg ? cfg->form : 0u;
    if (form != 0u && form != COBS_BATCHED && form != COBS_PLAIN)
        return set_error(COBS_ERR_ARG, "serve form must be 0, COBS_BATCHED or COBS_PLAIN");
    if (form == COBS_PLAIN && dix->streamed) return set_error(COBS_ERR_ARG, "the plain form needs a resident index");
    std::unique_ptr<CudaBackend> be(new CudaBackend(dix, form == COBS_PLAIN ? COBS_PLAIN : COBS_BATCHED));
    const uint32_t n_slots = cfg && cfg->max_inflight_waves ? cfg->max_inflight_waves : 2;
    cobs_status st = be->init(n_slots);
    if (st != COBS_OK) return st;
    return serve_create(std::move(be), cfg, out);
}

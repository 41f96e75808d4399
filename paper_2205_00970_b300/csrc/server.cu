// Continuous-batching server over a device-resident index: the CUDA executor
// of the scheduler in server_core.h and the lider_server_* entry points.
//
// Each execution slot owns a CUDA stream, an event, pinned host staging for
// max_batch queries and max_batch x max_k results, and device buffers of the
// same sizes.  A batch gathers its requests' queries into the slot's pinned
// buffer, copies them to the device, runs lider_search's kernels (scratch from
// the index's stream-ordered pool) and copies the results back, all on the
// slot's stream (queries already in pinned host memory are copied directly);
// finishing waits on the slot's event and scatters the rows to the requests'
// host buffers.
#include <cstring>
#include <memory>
#include <string>

#include "lider_internal.cuh"
#include "server_core.h"

namespace lider {

int search_entry(const lider_index*, const float*, int64_t, int, int, int64_t*, float*, const lider_trace*,
                 lider_search_stats*, void*);
int search_scratch_entry(const lider_index*, int64_t, int, int, size_t*);
const char* g_last_error_ptr();

namespace {

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    float* q_host = nullptr;
    int64_t* ids_host = nullptr;
    float* scores_host = nullptr;
    float* q_dev = nullptr;
    int64_t* ids_dev = nullptr;
    float* scores_dev = nullptr;
};

class CudaExecutor final : public serve::Executor {
  public:
    CudaExecutor(const lider_index* ix, int c, int slots, int64_t max_batch, int32_t max_k)
        : ix_(ix), c_(c), max_batch_(max_batch), max_k_(max_k), slots_(slots) {}

    int init(std::string* why) {
        cudaError_t e = cudaSetDevice(ix_->device);
        const size_t qb = (size_t)max_batch_ * ix_->g.d * 4, rb = (size_t)max_batch_ * max_k_;
        for (Slot& s : slots_) {
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMallocHost((void**)&s.q_host, qb);
            if (e == cudaSuccess) e = cudaMallocHost((void**)&s.ids_host, rb * 8);
            if (e == cudaSuccess) e = cudaMallocHost((void**)&s.scores_host, rb * 4);
            if (e == cudaSuccess) e = cudaMalloc((void**)&s.q_dev, qb);
            if (e == cudaSuccess) e = cudaMalloc((void**)&s.ids_dev, rb * 8);
            if (e == cudaSuccess) e = cudaMalloc((void**)&s.scores_dev, rb * 4);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            *why = std::string("server buffers: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? LIDER_ENOMEM : LIDER_ECUDA;
        }
        return LIDER_OK;
    }

    ~CudaExecutor() override {
        cudaSetDevice(ix_->device);
        for (Slot& s : slots_) {
            if (s.stream) cudaStreamSynchronize(s.stream);
            cudaFreeHost(s.q_host);
            cudaFreeHost(s.ids_host);
            cudaFreeHost(s.scores_host);
            cudaFree(s.q_dev);
            cudaFree(s.ids_dev);
            cudaFree(s.scores_dev);
            if (s.done) cudaEventDestroy(s.done);
            if (s.stream) cudaStreamDestroy(s.stream);
        }
    }

    size_t bytes(int64_t nq, int32_t k) override {
        size_t b = 0;
        return search_scratch_entry(ix_, nq, k, c_, &b) == LIDER_OK ? b : 0;
    }

    int launch(serve::Batch& b) override {
        if (b.nq > max_batch_ || b.k > max_k_) return fail_batch(b, LIDER_ELIMIT, "batch exceeds slot buffers");
        cudaError_t e = cudaSetDevice(ix_->device);
        if (e != cudaSuccess) return cuda_batch(b, e, "cudaSetDevice");
        Slot& s = slots_[b.slot];
        const int64_t d = ix_->g.d;
        // a failed batch returns its slot at once: drain what it enqueued first
        auto drained = [&](int rc) {
            cudaStreamSynchronize(s.stream);
            cudaGetLastError();
            return rc;
        };
        // Queries in pinned host memory are copied to the device directly;
        // the others are gathered into the slot's pinned staging first, each
        // run of consecutive such requests in one copy.
        int64_t off = 0, run = 0;            // the pending staged run: rows [off - run, off)
        auto flush = [&]() -> cudaError_t {
            if (run == 0) return cudaSuccess;
            const size_t r0 = (size_t)(off - run) * d;
            const cudaError_t ce = cudaMemcpyAsync(s.q_dev + r0, s.q_host + r0, (size_t)run * d * 4,
                                                   cudaMemcpyHostToDevice, s.stream);
            run = 0;
            return ce;
        };
        for (const serve::Request& r : b.reqs) {
            const size_t bytes = (size_t)r.nq * d * 4;
            if (pinned(r.queries)) {
                if ((e = flush()) == cudaSuccess)
                    e = cudaMemcpyAsync(s.q_dev + (size_t)off * d, r.queries, bytes, cudaMemcpyHostToDevice, s.stream);
                if (e != cudaSuccess) return drained(cuda_batch(b, e, "cudaMemcpyAsync(queries)"));
            } else {
                std::memcpy(s.q_host + (size_t)off * d, r.queries, bytes);
                run += r.nq;
            }
            off += r.nq;
        }
        if ((e = flush())) return drained(cuda_batch(b, e, "cudaMemcpyAsync(queries)"));
        const int rc = search_entry(ix_, s.q_dev, b.nq, b.k, c_, s.ids_dev, s.scores_dev, nullptr, nullptr,
                                    s.stream);
        if (rc != LIDER_OK) return drained(fail_batch(b, rc, g_last_error_ptr()));
        const size_t rn = (size_t)b.nq * b.k;
        if ((e = cudaMemcpyAsync(s.ids_host, s.ids_dev, rn * 8, cudaMemcpyDeviceToHost, s.stream)))
            return drained(cuda_batch(b, e, "cudaMemcpyAsync(ids)"));
        if ((e = cudaMemcpyAsync(s.scores_host, s.scores_dev, rn * 4, cudaMemcpyDeviceToHost, s.stream)))
            return drained(cuda_batch(b, e, "cudaMemcpyAsync(scores)"));
        if ((e = cudaEventRecord(s.done, s.stream))) return drained(cuda_batch(b, e, "cudaEventRecord"));
        return LIDER_OK;
    }

    int finish(serve::Batch& b) override {
        Slot& s = slots_[b.slot];
        cudaError_t e = cudaEventSynchronize(s.done);
        if (e != cudaSuccess) return cuda_batch(b, e, "cudaEventSynchronize");
        const int64_t k = b.k;
        const int64_t* ids = s.ids_host;
        const float* sc = s.scores_host;
        for (const serve::Request& r : b.reqs) {
            std::memcpy(r.ids, ids, (size_t)r.nq * k * 8);
            std::memcpy(r.scores, sc, (size_t)r.nq * k * 4);
            ids += r.nq * k;
            sc += r.nq * k;
        }
        return LIDER_OK;
    }

  private:
    // Whether p points into page-locked host memory (copies from it are DMA).
    static bool pinned(const void* p) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeHost;
    }
    static int fail_batch(serve::Batch& b, int code, const std::string& msg) {
        b.error = msg;
        return code;
    }
    static int cuda_batch(serve::Batch& b, cudaError_t e, const char* what) {
        cudaGetLastError();
        b.error = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? LIDER_ENOMEM : LIDER_ECUDA;
    }

    const lider_index* ix_;
    int c_;
    int64_t max_batch_;
    int32_t max_k_;
    std::vector<Slot> slots_;
};

}  // namespace
}  // namespace lider

struct lider_server {
    std::unique_ptr<lider::CudaExecutor> ex;
    std::unique_ptr<lider::serve::Scheduler> sched;
};

namespace lider {

int server_create_entry(const lider_index* ix, const lider_server_params* p, lider_server** out) {
    if (!out) return fail(LIDER_EINVAL, "lider_server_create: out is NULL");
    *out = nullptr;
    if (!ix || !p) return fail(LIDER_EINVAL, "lider_server_create: NULL argument");
    if (p->c < 1 || p->c > ix->g.ncl) return fail(LIDER_EINVAL, "lider_server_create: c must be in [1, n_clusters]");
    if (p->c > LIDER_MAX_C) return fail(LIDER_ELIMIT, "lider_server_create: c exceeds LIDER_MAX_C");
    if (p->slots < 1 || p->slots > 16) return fail(LIDER_EINVAL, "lider_server_create: slots must be in [1, 16]");
    if (p->max_batch < 1) return fail(LIDER_EINVAL, "lider_server_create: max_batch must be >= 1");
    if (p->max_k < 1 || p->max_k > LIDER_MAX_K)
        return fail(LIDER_EINVAL, "lider_server_create: max_k must be in [1, LIDER_MAX_K]");
    if (p->mem_budget < 1) return fail(LIDER_EINVAL, "lider_server_create: mem_budget must be >= 1");
    if (!(p->max_wait_us >= 0)) return fail(LIDER_EINVAL, "lider_server_create: max_wait_us must be >= 0");
    size_t probe = 0;
    int rc = search_scratch_entry(ix, p->max_batch, p->max_k, p->c, &probe);
    if (rc) return fail(rc, std::string("lider_server_create: a full batch of max_k is not searchable: ") +
                                g_last_error_ptr());
    auto s = std::make_unique<lider_server>();
    s->ex = std::make_unique<CudaExecutor>(ix, p->c, p->slots, p->max_batch, p->max_k);
    std::string why;
    if ((rc = s->ex->init(&why))) return fail(rc, "lider_server_create: " + why);
    serve::Config cfg;
    cfg.slots = p->slots;
    cfg.max_batch = p->max_batch;
    cfg.max_k = p->max_k;
    cfg.mem_budget = (size_t)p->mem_budget;
    cfg.max_wait_s = p->max_wait_us * 1e-6;
    s->sched = std::make_unique<serve::Scheduler>(s->ex.get(), cfg);
    *out = s.release();
    return LIDER_OK;
}

int server_submit_entry(lider_server* s, const float* q, int64_t nq, int32_t k, int64_t* ids, float* scores,
                        int64_t* ticket) {
    if (!s) return fail(LIDER_EINVAL, "lider_server_submit: server is NULL");
    std::string why;
    const int rc = s->sched->submit(q, nq, k, ids, scores, ticket, &why);
    return rc ? fail(rc, "lider_server_submit: " + why) : LIDER_OK;
}

int server_wait_entry(lider_server* s, int64_t ticket, double timeout_s) {
    if (!s) return fail(LIDER_EINVAL, "lider_server_wait: server is NULL");
    const int rc = s->sched->wait(ticket, timeout_s);
    if (rc == LIDER_EINVAL) return fail(rc, "lider_server_wait: unknown or already waited ticket");
    if (rc == LIDER_ETIMEDOUT) return fail(rc, "lider_server_wait: request still running");
    if (rc) return fail(rc, "lider_server_wait: batch failed: " + s->sched->last_error());
    return LIDER_OK;
}

int server_stats_entry(lider_server* s, lider_server_counters* st) {
    if (!s || !st) return fail(LIDER_EINVAL, "lider_server_stats: NULL argument");
    const serve::Counters c = s->sched->counters();
    *st = lider_server_counters{};
    st->requests = c.requests;
    st->queries = c.queries;
    st->batches = c.batches;
    st->refused = c.refused;
    st->failed = c.failed;
    st->max_inflight_batches = c.max_inflight_batches;
    st->max_inflight_bytes = (int64_t)c.max_inflight_bytes;
    st->launch_s = c.launch_s;
    st->finish_s = c.finish_s;
    return LIDER_OK;
}

int server_latencies_entry(lider_server* s, double* out_ms, int64_t cap, int32_t clear, int64_t* total) {
    if (!s || !total || cap < 0 || (cap > 0 && !out_ms))
        return fail(LIDER_EINVAL, "lider_server_latencies: bad argument");
    *total = s->sched->latencies(out_ms, cap, clear != 0);
    return LIDER_OK;
}

void server_destroy_entry(lider_server* s) {
    if (!s) return;
    s->sched->stop();
    s->sched.reset();
    s->ex.reset();
    delete s;
}

}  // namespace lider

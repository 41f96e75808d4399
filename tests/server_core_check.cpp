// Host-only checks of the continuous-batching scheduler (server_core.h) with
// a fake executor: no CUDA.  Built and run by test_serving.py; prints one
// line per failed check and exits non-zero if any failed.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <random>
#include <set>

#include "server_core.h"

using namespace lider::serve;

static int g_fail = 0;
#define CHECK(cond, ...)                                \
    do {                                                \
        if (!(cond)) {                                  \
            std::printf("FAIL %s:%d ", __FILE__, __LINE__); \
            std::printf(__VA_ARGS__);                   \
            std::printf("\n");                          \
            ++g_fail;                                   \
        }                                               \
    } while (0)

constexpr int D = 4;

// Per-query stand-in for a search: depends on the query's own row only.
static int64_t row_key(const float* q) {
    double s = 0;
    for (int j = 0; j < D; ++j) s += std::fabs(q[j]);
    return (int64_t)std::floor(s * 1000.0);
}

struct FakeExecutor : Executor {
    double delay_s = 0.002;
    std::function<bool(const Batch&)> fail_launch;
    std::mutex mu;
    std::set<int> active;
    int max_active = 0, reuse = 0, mixed_k = 0, oversize = 0;
    std::vector<std::pair<int64_t, int32_t>> batches;
    std::vector<Clock::time_point> ready;
    int64_t max_batch = 1 << 30;

    FakeExecutor() : ready(16) {}

    size_t bytes(int64_t nq, int32_t k) override { return 1000 + (size_t)nq * k * 10; }

    int launch(Batch& b) override {
        std::lock_guard<std::mutex> lk(mu);
        if (active.count(b.slot)) ++reuse;
        active.insert(b.slot);
        max_active = std::max(max_active, (int)active.size());
        batches.emplace_back(b.nq, b.k);
        for (const Request& r : b.reqs) mixed_k += r.k != b.k;
        if (b.nq > max_batch) ++oversize;
        if (fail_launch && fail_launch(b)) {
            active.erase(b.slot);
            b.error = "fake launch failure";
            return LIDER_ECUDA;
        }
        ready[b.slot] = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(delay_s));
        return LIDER_OK;
    }

    int finish(Batch& b) override {
        std::this_thread::sleep_until(ready[b.slot]);
        for (const Request& r : b.reqs)
            for (int64_t i = 0; i < r.nq; ++i) {
                const int64_t h = row_key(r.queries + i * D);
                for (int j = 0; j < b.k; ++j) {
                    r.ids[i * b.k + j] = h + j;
                    r.scores[i * b.k + j] = -(float)(h + j);
                }
            }
        std::lock_guard<std::mutex> lk(mu);
        active.erase(b.slot);
        return LIDER_OK;
    }
};

struct Req {
    std::vector<float> q;
    int32_t k;
    std::vector<int64_t> ids;
    std::vector<float> sc;
    int64_t ticket = -1;
    int rc = 0;
};

static Req make_req(std::mt19937& g, int max_nq, int32_t k) {
    Req r;
    const int nq = 1 + (int)(g() % max_nq);
    std::normal_distribution<float> nd;
    r.q.resize((size_t)nq * D);
    for (float& v : r.q) v = nd(g);
    r.k = k;
    r.ids.assign((size_t)nq * k, -7);
    r.sc.assign((size_t)nq * k, 0.f);
    return r;
}

static bool results_ok(const Req& r) {
    const int64_t nq = (int64_t)r.q.size() / D;
    for (int64_t i = 0; i < nq; ++i) {
        const int64_t h = row_key(r.q.data() + i * D);
        for (int j = 0; j < r.k; ++j)
            if (r.ids[i * r.k + j] != h + j || r.sc[i * r.k + j] != -(float)(h + j)) return false;
    }
    return true;
}

static int submit(Scheduler& s, Req& r) {
    std::string why;
    return s.submit(r.q.data(), (int64_t)r.q.size() / D, r.k, r.ids.data(), r.sc.data(), &r.ticket, &why);
}

static void test_routing_and_batching() {
    FakeExecutor ex;
    ex.max_batch = 64;
    Config cfg;
    cfg.slots = 3;
    cfg.max_batch = 64;
    cfg.max_k = 10;
    cfg.mem_budget = size_t(1) << 30;
    Scheduler s(&ex, cfg);
    std::mt19937 g(1);
    std::vector<Req> reqs;
    for (int i = 0; i < 300; ++i) reqs.push_back(make_req(g, 20, (i % 3) ? 5 : 10));
    for (Req& r : reqs) CHECK(submit(s, r) == LIDER_OK, "submit");
    for (Req& r : reqs) CHECK(s.wait(r.ticket, 10.0) == LIDER_OK, "wait");
    for (Req& r : reqs) CHECK(results_ok(r), "results of ticket %lld", (long long)r.ticket);
    CHECK(s.wait(reqs[0].ticket, 0.0) == LIDER_EINVAL, "second wait on a ticket");
    CHECK(s.wait(123456, 0.0) == LIDER_EINVAL, "unknown ticket");
    s.stop();
    const Counters c = s.counters();
    CHECK(c.requests == 300, "requests %lld", (long long)c.requests);
    CHECK(c.batches < 300, "no batching happened (%lld batches)", (long long)c.batches);
    CHECK(ex.reuse == 0, "slot reused while active");
    CHECK(ex.max_active <= 3, "more active slots than configured");
    CHECK(ex.mixed_k == 0, "a batch mixed k");
    CHECK(ex.oversize == 0, "a batch exceeded max_batch");
    CHECK(s.latencies(nullptr, 0, false) == 300, "latency count");
}

static void test_memory_budget() {
    FakeExecutor ex;
    ex.delay_s = 0.003;
    Config cfg;
    cfg.slots = 4;
    cfg.max_batch = 40;
    cfg.max_k = 10;
    cfg.mem_budget = ex.bytes(40, 10) + ex.bytes(10, 10);
    Scheduler s(&ex, cfg);
    std::mt19937 g(3);
    std::vector<Req> reqs;
    for (int i = 0; i < 80; ++i) reqs.push_back(make_req(g, 39, 10));
    for (Req& r : reqs) CHECK(submit(s, r) == LIDER_OK, "submit");
    for (Req& r : reqs) CHECK(s.wait(r.ticket, 20.0) == LIDER_OK, "wait");
    s.stop();
    const Counters c = s.counters();
    CHECK(c.max_inflight_bytes > 0 && c.max_inflight_bytes <= cfg.mem_budget, "in-flight bytes %zu > budget %zu",
          c.max_inflight_bytes, cfg.mem_budget);
    for (Req& r : reqs) CHECK(results_ok(r), "results");
}

static void test_refusals() {
    FakeExecutor ex;
    Config cfg;
    cfg.slots = 2;
    cfg.max_batch = 16;
    cfg.max_k = 100;
    cfg.mem_budget = ex.bytes(16, 10);
    Scheduler s(&ex, cfg);
    std::mt19937 g(4);
    Req big = make_req(g, 1, 10);
    big.q.assign(17 * D, 1.f);
    big.ids.resize(17 * 10);
    big.sc.resize(17 * 10);
    CHECK(submit(s, big) == LIDER_ELIMIT, "more queries than max_batch");
    Req mem = make_req(g, 1, 100);
    mem.q.assign(16 * D, 1.f);
    mem.ids.resize(16 * 100);
    mem.sc.resize(16 * 100);
    CHECK(submit(s, mem) == LIDER_ELIMIT, "scratch above the budget");
    Req kbig = make_req(g, 1, 101);
    CHECK(submit(s, kbig) == LIDER_ELIMIT, "k above max_k");
    Req ok = make_req(g, 16, 10);
    CHECK(submit(s, ok) == LIDER_OK && s.wait(ok.ticket, 5.0) == LIDER_OK && results_ok(ok), "admissible request");
    Req empty;
    empty.k = 3;
    std::string why;
    CHECK(s.submit(nullptr, 0, 3, nullptr, nullptr, &empty.ticket, &why) == LIDER_OK &&
              s.wait(empty.ticket, 0.0) == LIDER_OK,
          "empty request");
    CHECK(s.submit(nullptr, 2, 3, nullptr, nullptr, &empty.ticket, &why) == LIDER_EINVAL, "NULL buffers");
    s.stop();
    CHECK(s.counters().refused == 3, "refused %lld", (long long)s.counters().refused);
    CHECK(submit(s, ok) == LIDER_EINVAL, "submit after stop");
}

static void test_failure_propagates() {
    FakeExecutor ex;
    ex.fail_launch = [](const Batch& b) { return b.k == 3; };
    Config cfg;
    cfg.slots = 2;
    cfg.max_batch = 8;
    cfg.max_k = 10;
    Scheduler s(&ex, cfg);
    std::mt19937 g(5);
    Req bad = make_req(g, 2, 3);
    CHECK(submit(s, bad) == LIDER_OK, "submit");
    CHECK(s.wait(bad.ticket, 5.0) == LIDER_ECUDA, "failed batch status");
    CHECK(s.last_error() == "fake launch failure", "error message");
    Req good = make_req(g, 2, 5);
    CHECK(submit(s, good) == LIDER_OK && s.wait(good.ticket, 5.0) == LIDER_OK && results_ok(good),
          "server continues after a failed batch");
    s.stop();
    CHECK(s.counters().failed >= 1, "failed counter");
}

static void test_timeout_and_stop_drains() {
    FakeExecutor ex;
    ex.delay_s = 0.05;
    Config cfg;
    cfg.slots = 1;
    cfg.max_batch = 4;
    cfg.max_k = 2;
    Scheduler s(&ex, cfg);
    std::vector<Req> reqs;
    for (int i = 0; i < 10; ++i) {
        Req r;
        r.q.assign(3 * D, (float)i);
        r.k = 2;
        r.ids.assign(6, -7);
        r.sc.assign(6, 0.f);
        reqs.push_back(r);
    }
    for (Req& r : reqs) CHECK(submit(s, r) == LIDER_OK, "submit");
    CHECK(s.wait(reqs.back().ticket, 0.001) == LIDER_ETIMEDOUT, "wait times out while running");
    s.stop();                                   // drains all ten
    for (Req& r : reqs) CHECK(results_ok(r), "drained results");
    CHECK(s.counters().requests == 10, "all requests completed");
    for (Req& r : reqs) CHECK(s.wait(r.ticket, 0.0) == LIDER_OK, "wait after stop");
}

static void test_concurrent_clients() {
    FakeExecutor ex;
    ex.delay_s = 0.001;
    Config cfg;
    cfg.slots = 3;
    cfg.max_batch = 128;
    cfg.max_k = 20;
    Scheduler s(&ex, cfg);
    std::atomic<int> bad{0};
    std::vector<std::thread> th;
    for (int t = 0; t < 4; ++t)
        th.emplace_back([&, t] {
            std::mt19937 g(100 + t);
            std::vector<Req> reqs;
            for (int i = 0; i < 200; ++i) reqs.push_back(make_req(g, 16, (i % 2) ? 10 : 20));
            for (Req& r : reqs)
                if (submit(s, r) != LIDER_OK) ++bad;
            for (Req& r : reqs)
                if (s.wait(r.ticket, 20.0) != LIDER_OK || !results_ok(r)) ++bad;
        });
    for (auto& x : th) x.join();
    s.stop();
    CHECK(bad == 0, "%d bad requests across client threads", bad.load());
    CHECK(s.counters().requests == 800, "requests");
    CHECK(ex.reuse == 0 && ex.mixed_k == 0, "slot reuse or mixed k");
}

int main() {
    test_routing_and_batching();
    test_memory_budget();
    test_refusals();
    test_failure_propagates();
    test_timeout_and_stop_drains();
    test_concurrent_clients();
    if (g_fail) std::printf("%d checks failed\n", g_fail);
    else std::printf("all checks passed\n");
    return g_fail ? 1 : 0;
}

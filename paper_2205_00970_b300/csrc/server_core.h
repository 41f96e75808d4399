// Continuous-batching scheduler for k-NN requests (host only, no CUDA).
//
// Requests (a block of queries on the host, a k, and host buffers for the
// results) arrive at any time from any thread.  One scheduler thread packs
// pending requests of equal k, oldest first, into batches of at most
// max_batch queries.  A batch is admitted only when one of `slots` execution
// slots is free and the memory it needs (Executor::bytes) fits in the budget
// next to the batches already in flight; the scheduler then hands it to the
// executor (gather + asynchronous launch).  One completion thread finishes
// batches in launch order (wait + scatter into each request's buffers),
// records each request's latency from submission to results and wakes the
// waiters.  While batches are in flight the scheduler waits up to
// max_wait_s for more requests before launching a partly filled batch.
//
// k is equal within a batch because the expansion length R = r0 * k sets the
// candidate set of every query; a query's result does not depend on the other
// queries of its batch, so a request gets the same results alone or in any
// mix.  The executor is an interface so this logic is testable without a GPU.
#pragma once

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "lider.h"

namespace lider {
namespace serve {

using Clock = std::chrono::steady_clock;

struct Request {
    const float* queries;   // host, nq x d; valid until the request completes
    int64_t nq;
    int32_t k;
    int64_t* ids;           // host, nq x k
    float* scores;          // host, nq x k
    int64_t ticket;
    Clock::time_point t_arrival;
};

struct Batch {
    std::vector<Request> reqs;
    int32_t k = 0;
    int64_t nq = 0;
    size_t bytes = 0;
    int slot = -1;
    int status = LIDER_OK;   // result of Executor::launch
    std::string error;       // message of a failed launch or finish
};

// The device side of a batch.  launch() and finish() of one slot never run
// at the same time; a slot is reused only after finish() returned.
struct Executor {
    virtual ~Executor() = default;
    virtual size_t bytes(int64_t nq, int32_t k) = 0;   // device memory a batch needs (0 on error)
    virtual int launch(Batch& b) = 0;                  // gather queries, enqueue the search
    virtual int finish(Batch& b) = 0;                  // wait, scatter results to the requests
};

struct Config {
    int slots = 3;
    int64_t max_batch = 4096;
    int32_t max_k = 100;
    size_t mem_budget = size_t(8) << 30;
    double max_wait_s = 0.0005;
};

struct Counters {
    int64_t requests = 0, queries = 0, batches = 0, refused = 0, failed = 0;
    int32_t max_inflight_batches = 0;
    size_t max_inflight_bytes = 0;
    double launch_s = 0, finish_s = 0;
};

class Scheduler {
  public:
    Scheduler(Executor* ex, const Config& cfg) : ex_(ex), cfg_(cfg) {
        for (int s = 0; s < cfg_.slots; ++s) free_slots_.push_back(cfg_.slots - 1 - s);
        sched_ = std::thread([this] { schedule_loop(); });
        compl_ = std::thread([this] { complete_loop(); });
    }
    ~Scheduler() { stop(); }
    Scheduler(const Scheduler&) = delete;
    Scheduler& operator=(const Scheduler&) = delete;

    // Enqueue a request.  LIDER_ELIMIT if it can never be admitted (more than
    // max_batch queries, k above max_k, or more memory than the budget);
    // LIDER_EINVAL after stop() or for bad arguments.
    int submit(const float* q, int64_t nq, int32_t k, int64_t* ids, float* scores, int64_t* ticket,
               std::string* why) {
        if (!ticket || nq < 0 || k < 1 || (nq > 0 && (!q || !ids || !scores))) {
            *why = "bad request arguments";
            return LIDER_EINVAL;
        }
        if (nq > cfg_.max_batch || k > cfg_.max_k) {
            std::lock_guard<std::mutex> lk(m_);
            ++cnt_.refused;
            *why = "request has more queries than max_batch or k above max_k";
            return LIDER_ELIMIT;
        }
        const size_t need = nq ? ex_->bytes(nq, k) : 0;
        if (nq && (need == 0 || need > cfg_.mem_budget)) {
            std::lock_guard<std::mutex> lk(m_);
            ++cnt_.refused;
            *why = "request needs more device memory than the budget";
            return LIDER_ELIMIT;
        }
        std::lock_guard<std::mutex> lk(m_);
        if (stopping_) {
            *why = "server is stopping";
            return LIDER_EINVAL;
        }
        const int64_t t = next_ticket_++;
        *ticket = t;
        if (nq == 0) {                   // nothing to do: complete at once
            done_[t] = LIDER_OK;
            ++cnt_.requests;
            return LIDER_OK;
        }
        pending_.push_back(Request{q, nq, k, ids, scores, t, Clock::now()});
        pending_nq_ += nq;
        outstanding_.insert(t);
        cv_sched_.notify_one();
        return LIDER_OK;
    }

    // Wait for a request.  Its status (LIDER_OK or the batch's error) once it
    // completed; LIDER_ETIMEDOUT if still running after timeout_s (< 0: no
    // limit); LIDER_EINVAL for a ticket that is unknown or already waited.
    int wait(int64_t ticket, double timeout_s) {
        std::unique_lock<std::mutex> lk(m_);
        auto ready = [&] { return done_.count(ticket) != 0; };
        if (!ready()) {
            if (!outstanding_.count(ticket)) return LIDER_EINVAL;
            if (timeout_s < 0)
                cv_done_.wait(lk, ready);
            else if (!cv_done_.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
                return LIDER_ETIMEDOUT;
        }
        const int st = done_[ticket];
        done_.erase(ticket);
        return st;
    }

    // Finish every request already submitted, then join the threads.
    void stop() {
        {
            std::lock_guard<std::mutex> lk(m_);
            if (joined_) return;
            stopping_ = true;
        }
        cv_sched_.notify_all();
        cv_done_.notify_all();
        if (sched_.joinable()) sched_.join();
        if (compl_.joinable()) compl_.join();
        std::lock_guard<std::mutex> lk(m_);
        joined_ = true;
    }

    Counters counters() {
        std::lock_guard<std::mutex> lk(m_);
        return cnt_;
    }

    std::string last_error() {
        std::lock_guard<std::mutex> lk(m_);
        return last_error_;
    }

    // Copy up to cap latencies (ms, in completion order); clear: drop all.
    int64_t latencies(double* out, int64_t cap, bool clear) {
        std::lock_guard<std::mutex> lk(m_);
        const int64_t n = std::min<int64_t>(cap, (int64_t)lat_ms_.size());
        if (out) std::copy(lat_ms_.begin(), lat_ms_.begin() + n, out);
        const int64_t total = (int64_t)lat_ms_.size();
        if (clear) lat_ms_.clear();
        return total;
    }

  private:
    // Oldest request and every later one of the same k that still fits.
    Batch take_batch() {
        Batch b;
        b.k = pending_.front().k;
        std::deque<Request> keep;
        while (!pending_.empty()) {
            Request r = pending_.front();
            pending_.pop_front();
            if (r.k == b.k && b.nq + r.nq <= cfg_.max_batch) {
                b.nq += r.nq;
                b.reqs.push_back(r);
            } else {
                keep.push_back(r);
            }
        }
        pending_.swap(keep);
        return b;
    }

    void schedule_loop() {
        std::unique_lock<std::mutex> lk(m_);
        for (;;) {
            cv_sched_.wait(lk, [&] { return stopping_ || !pending_.empty(); });
            if (pending_.empty()) break;               // stopping and drained
            if (!inflight_.empty() && cfg_.max_wait_s > 0 && !stopping_ && pending_nq_ < cfg_.max_batch) {
                const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                                      std::chrono::duration<double>(cfg_.max_wait_s));
                cv_sched_.wait_until(lk, until, [&] { return stopping_ || pending_nq_ >= cfg_.max_batch; });
            }
            const Request& first = pending_.front();
            const size_t need_first = ex_->bytes(first.nq, first.k);
            cv_done_.wait(lk, [&] {
                return !free_slots_.empty() && inflight_bytes_ + need_first <= cfg_.mem_budget;
            });
            Batch b = take_batch();
            b.bytes = ex_->bytes(b.nq, b.k);
            while (inflight_bytes_ + b.bytes > cfg_.mem_budget && b.reqs.size() > 1) {
                pending_.push_front(b.reqs.back());     // give back the newest until it fits
                b.nq -= b.reqs.back().nq;
                b.reqs.pop_back();
                b.bytes = ex_->bytes(b.nq, b.k);
            }
            pending_nq_ -= b.nq;
            b.slot = free_slots_.back();
            free_slots_.pop_back();
            inflight_bytes_ += b.bytes;
            ++launching_;
            cnt_.max_inflight_bytes = std::max(cnt_.max_inflight_bytes, inflight_bytes_);
            lk.unlock();
            const auto t0 = Clock::now();
            b.status = ex_->launch(b);
            const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
            lk.lock();
            cnt_.launch_s += dt;
            --launching_;
            inflight_.push_back(std::move(b));
            cnt_.max_inflight_batches = std::max(cnt_.max_inflight_batches, (int32_t)inflight_.size());
            cv_compl_.notify_one();
        }
        sched_done_ = true;
        cv_compl_.notify_all();
    }

    void complete_loop() {
        std::unique_lock<std::mutex> lk(m_);
        for (;;) {
            cv_compl_.wait(lk, [&] { return !inflight_.empty() || (sched_done_ && launching_ == 0); });
            if (inflight_.empty()) break;
            Batch b = std::move(inflight_.front());
            inflight_.pop_front();
            lk.unlock();
            const auto t0 = Clock::now();
            int st = b.status;
            if (st == LIDER_OK) st = ex_->finish(b);
            const auto t1 = Clock::now();
            lk.lock();
            cnt_.finish_s += std::chrono::duration<double>(t1 - t0).count();
            for (const Request& r : b.reqs) {
                done_[r.ticket] = st;
                outstanding_.erase(r.ticket);
                lat_ms_.push_back(std::chrono::duration<double, std::milli>(t1 - r.t_arrival).count());
            }
            cnt_.requests += (int64_t)b.reqs.size();
            cnt_.queries += b.nq;
            cnt_.batches += 1;
            if (st != LIDER_OK) {
                cnt_.failed += (int64_t)b.reqs.size();
                last_error_ = b.error;
            }
            inflight_bytes_ -= b.bytes;
            free_slots_.push_back(b.slot);
            cv_done_.notify_all();
        }
    }

    Executor* ex_;
    Config cfg_;
    std::mutex m_;
    std::condition_variable cv_sched_, cv_compl_, cv_done_;
    std::deque<Request> pending_;
    int64_t pending_nq_ = 0;
    std::deque<Batch> inflight_;
    std::vector<int> free_slots_;
    size_t inflight_bytes_ = 0;
    int launching_ = 0;
    int64_t next_ticket_ = 0;
    std::unordered_map<int64_t, int> done_;
    std::unordered_set<int64_t> outstanding_;
    std::vector<double> lat_ms_;
    std::string last_error_;
    Counters cnt_;
    bool stopping_ = false, sched_done_ = false, joined_ = false;
    std::thread sched_, compl_;
};

}  // namespace serve
}  // namespace lider

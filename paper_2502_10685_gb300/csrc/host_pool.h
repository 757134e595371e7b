// host_pool.h -- one process-wide pool of host worker threads for the
// planner's independent jobs (instruction streams of a plan, staging copies):
// started once, so a circuit load does not pay for creating threads.
#pragma once

#include <condition_variable>
#include <deque>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace stab {

class HostPool {
public:
    // Runs every job; the calling thread takes jobs too.  Returns when all are
    // done.  Jobs must not throw.  Several callers may use the pool at once.
    static void run(std::vector<std::function<void()>> &jobs) {
        if (jobs.size() <= 1) {
            for (auto &j : jobs) j();
            return;
        }
        HostPool &p = get();
        Batch b;
        b.left = jobs.size();
        {
            std::lock_guard<std::mutex> g(p.mu_);
            for (size_t k = 1; k < jobs.size(); ++k) p.q_.push_back({&jobs[k], &b});
        }
        p.cv_.notify_all();
        jobs[0]();
        p.finish(&b);
        // help with queued jobs (of any caller) until this batch is done
        for (;;) {
            Item it{};
            {
                std::unique_lock<std::mutex> g(p.mu_);
                if (b.left == 0) return;
                if (p.q_.empty()) {
                    b.cv.wait(g, [&b] { return b.left == 0; });
                    return;
                }
                it = p.q_.front();
                p.q_.pop_front();
            }
            (*it.job)();
            p.finish(it.batch);
        }
    }

private:
    struct Batch {
        size_t left = 0;
        std::condition_variable cv;
    };
    struct Item {
        std::function<void()> *job;
        Batch *batch;
    };

    static HostPool &get() {
        static HostPool pool;
        return pool;
    }

    HostPool() {
        unsigned n = std::thread::hardware_concurrency();
        n = n < 2 ? 2 : (n > 8 ? 8 : n);
        for (unsigned i = 0; i + 1 < n; ++i) th_.emplace_back([this] { loop(); });
    }
    ~HostPool() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (std::thread &t : th_) t.join();
    }

    void finish(Batch *b) {
        std::lock_guard<std::mutex> g(mu_);
        if (--b->left == 0) b->cv.notify_all();
    }

    void loop() {
        for (;;) {
            Item it{};
            {
                std::unique_lock<std::mutex> g(mu_);
                cv_.wait(g, [this] { return stop_ || !q_.empty(); });
                if (stop_ && q_.empty()) return;
                it = q_.front();
                q_.pop_front();
            }
            (*it.job)();
            finish(it.batch);
        }
    }

    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<Item> q_;
    std::vector<std::thread> th_;
    bool stop_ = false;
};

}  // namespace stab

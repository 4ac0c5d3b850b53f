// copy_pool.cuh -- host threads for step a2, the copy of pageable rasters into
// the pinned ring before their upload.  One thread copies pageable memory at
// a small fraction of the host link's rate, so a chunk's copy is cut into
// pieces that several threads copy at once.
#pragma once

#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace cpt {

// A fixed set of worker threads that run the pieces of one job at a time.
// The submitting thread works on the job too and returns once every piece
// has finished, so the job's data may live on its stack.  Jobs come from one
// thread at a time (a context is used from one thread).
class CopyPool {
public:
    // Throws std::system_error when a thread cannot be started (the threads
    // already started are stopped and joined first).
    explicit CopyPool(int workers) {
        try {
            for (int i = 0; i < workers; ++i) threads_.emplace_back([this] { loop(); });
        } catch (...) {
            stop_all();
            throw;
        }
    }

    ~CopyPool() { stop_all(); }

    CopyPool(const CopyPool &) = delete;
    CopyPool &operator=(const CopyPool &) = delete;

    // Threads that copy, the caller included.
    int width() const { return (int)threads_.size() + 1; }

    // Runs piece(0), ..., piece(n - 1) on the workers and the caller.
    void run(int n, const std::function<void(int)> &piece) {
        if (n <= 0) return;
        {
            std::lock_guard<std::mutex> lock(mu_);
            job_ = &piece;
            next_ = 0;
            total_ = n;
            done_ = 0;
            ++generation_;
        }
        wake_.notify_all();
        work();
        std::unique_lock<std::mutex> lock(mu_);
        finished_.wait(lock, [this] { return done_ == total_; });
        job_ = nullptr;
    }

private:
    void stop_all() {
        {
            std::lock_guard<std::mutex> lock(mu_);
            stop_ = true;
        }
        wake_.notify_all();
        for (std::thread &t : threads_)
            if (t.joinable()) t.join();
        threads_.clear();
    }

    // Takes pieces of the current job until none is left.
    void work() {
        for (;;) {
            const std::function<void(int)> *job;
            int i;
            {
                std::lock_guard<std::mutex> lock(mu_);
                if (!job_ || next_ >= total_) return;
                job = job_;
                i = next_++;
            }
            (*job)(i);
            std::lock_guard<std::mutex> lock(mu_);
            if (++done_ == total_) finished_.notify_all();
        }
    }

    void loop() {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lock(mu_);
                wake_.wait(lock, [&] { return stop_ || (generation_ != seen && job_ && next_ < total_); });
                if (stop_) return;
                seen = generation_;
            }
            work();
        }
    }

    std::vector<std::thread> threads_;
    std::mutex mu_;
    std::condition_variable wake_, finished_;
    const std::function<void(int)> *job_ = nullptr;
    int next_ = 0, total_ = 0, done_ = 0;
    uint64_t generation_ = 0;
    bool stop_ = false;
};

}  // namespace cpt

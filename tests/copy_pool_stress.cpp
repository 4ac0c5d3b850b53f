// Stress test of the ingest copy pool (paper_2104_14667_gb300/csrc/copy_pool.cuh),
// built and run by tests/test_copy_pool_cpu.py: many jobs of uneven sizes on
// pools of several widths; every piece of every job must run exactly once,
// and run() must return only after all of them.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <vector>

#include "copy_pool.cuh"

int main() {
    int failures = 0;
    for (int workers : {0, 1, 3, 7, 15}) {
        cpt::CopyPool pool(workers);
        if (pool.width() != workers + 1) ++failures;
        for (int job = 0; job < 2000; ++job) {
            const int n = 1 + (job * 37) % 97;
            std::vector<std::atomic<int>> hits(n);
            for (auto &h : hits) h.store(0);
            pool.run(n, [&](int i) { hits[i].fetch_add(1); });
            for (int i = 0; i < n; ++i)
                if (hits[i].load() != 1) ++failures;
        }
        // a real copy cut into pieces
        std::vector<unsigned char> src(1 << 20), dst(1 << 20, 0);
        for (size_t i = 0; i < src.size(); ++i) src[i] = (unsigned char)(i * 131 + 7);
        pool.run(64, [&](int p) {
            const size_t piece = src.size() / 64;
            std::memcpy(dst.data() + p * piece, src.data() + p * piece, piece);
        });
        if (std::memcmp(src.data(), dst.data(), src.size()) != 0) ++failures;
        pool.run(0, [&](int) { ++failures; });
    }
    std::printf("failures %d\n", failures);
    return failures == 0 ? 0 : 1;
}

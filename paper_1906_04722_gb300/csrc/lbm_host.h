// lbm_host.h -- host-side helpers of the CUDA library (not part of the ABI).
#pragma once

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

namespace lbmk {

// f(t) for t in [0, n) on the host cores.  Returns false if an iteration threw
// (host allocation failure); f must not call set_error (its text is per thread).
template <class F>
bool host_parallel_for(int n, F&& f) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = std::max(1, std::min(n, (int)std::min(32u, hw)));
    std::atomic<int> next{0};
    std::atomic<bool> ok{true};
    auto work = [&]() {
        for (int t; (t = next.fetch_add(1)) < n;) {
            try {
                f(t);
            } catch (...) {
                ok = false;
            }
        }
    };
    std::vector<std::thread> pool;
    pool.reserve((size_t)nt - 1);
    for (int i = 0; i + 1 < nt; ++i) pool.emplace_back(work);
    work();
    for (std::thread& th : pool) th.join();
    return ok;
}

}  // namespace lbmk

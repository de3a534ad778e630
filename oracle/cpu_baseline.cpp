// Timed CPU baseline for the synchronization phase -- test/bench
// infrastructure only, not the oracle and not the product.
//
// What the GPU's validation and apply compute (Sec. IV-C), written the way a
// multicore host would: the log is cut into one slice per thread; pass 1
// flags every tuple whose granule is in RS_bmp (count summed over threads)
// and raises TS[addr] to the tuple's timestamp with a compare-and-swap loop;
// pass 2, after all threads joined, writes the value of the tuple holding
// TS[addr] into W and S.  The oracle (hetm_oracle.cpp) is the single-thread
// definition this is checked against; this file exists to be timed.
#include <cstdint>
#include <thread>
#include <vector>

namespace {

struct Entry {
    uint32_t addr;
    int32_t value;
    uint32_t ts;
};

void raise_ts(uint32_t *ts, uint32_t v) {
    uint32_t cur = __atomic_load_n(ts, __ATOMIC_RELAXED);
    while (cur < v && !__atomic_compare_exchange_n(ts, &cur, v, true, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
    }
}

}  // namespace

extern "C" int64_t hetm_cpu_validate_apply_mt(const void *log_v, uint64_t n, const uint32_t *rs,
                                              uint32_t gshift, uint64_t n_words, int32_t *W, int32_t *S,
                                              uint32_t *TS, uint8_t *flags, int threads) {
    const Entry *log = static_cast<const Entry *>(log_v);
    if (threads < 1) threads = 1;
    std::vector<int64_t> hits(threads, 0);
    std::vector<int> bad(threads, 0);
    auto slice = [&](int t, uint64_t *lo, uint64_t *hi) {
        *lo = n * (uint64_t)t / threads;
        *hi = n * (uint64_t)(t + 1) / threads;
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&, t] {
            uint64_t lo, hi;
            slice(t, &lo, &hi);
            int64_t h = 0;
            for (uint64_t i = lo; i < hi; ++i) {
                const uint32_t a = log[i].addr;
                if (a >= n_words) {
                    bad[t] = 1;
                    continue;
                }
                const uint64_t g = a >> gshift;
                const uint8_t f = (rs[g >> 5] >> (g & 31)) & 1u;
                if (flags) flags[i] = f;
                h += f;
                raise_ts(TS + a, log[i].ts);
            }
            hits[t] = h;
        });
    for (auto &th : pool) th.join();
    pool.clear();
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&, t] {
            uint64_t lo, hi;
            slice(t, &lo, &hi);
            for (uint64_t i = lo; i < hi; ++i) {
                const uint32_t a = log[i].addr;
                if (a < n_words && TS[a] == log[i].ts) {
                    W[a] = log[i].value;
                    S[a] = log[i].value;
                }
            }
        });
    for (auto &th : pool) th.join();
    int64_t total = 0;
    for (int t = 0; t < threads; ++t) {
        if (bad[t]) return -1;
        total += hits[t];
    }
    return total;
}

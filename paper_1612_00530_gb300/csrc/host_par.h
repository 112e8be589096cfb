// Host-side helpers shared by the generators and the format builders: a
// parallel loop over index ranges on plain std::threads, and an
// open-addressing table keyed by a double's 64-bit pattern (value tables
// count every stored value, so this is their inner loop).
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace spmvc {

inline uint64_t value_bits(double v) {
    uint64_t b;
    std::memcpy(&b, &v, 8);
    return b;
}

// Threads the host passes use: the hardware's count, at most 32.
inline unsigned host_threads() { return std::max(1u, std::min(32u, std::thread::hardware_concurrency())); }

// f(begin, end, part) over `parts` consecutive ranges covering [0, n); one
// thread a range.  Fewer parts for small n (each at least `grain` items);
// a single part runs on the calling thread.
template <class F>
void parallel_ranges(int64_t n, int64_t grain, F&& f) {
    int64_t parts = std::min<int64_t>(host_threads(), std::max<int64_t>(1, n / std::max<int64_t>(1, grain)));
    if (parts <= 1) {
        f(int64_t(0), n, 0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(parts);
    for (int64_t t = 0; t < parts; ++t) {
        const int64_t a = n * t / parts, b = n * (t + 1) / parts;
        th.emplace_back([&f, a, b, t] { f(a, b, int(t)); });
    }
    for (auto& x : th) x.join();
}

inline int parallel_parts(int64_t n, int64_t grain) {
    return int(std::min<int64_t>(host_threads(), std::max<int64_t>(1, n / std::max<int64_t>(1, grain))));
}

// 64-bit keys to int64 values, linear probing, Fibonacci hashing (Knuth's
// multiplicative method with 2^64 / golden ratio), doubled at half load.
class BitsTable {
public:
    explicit BitsTable(int log2cap = 10) { reset(log2cap); }

    void reset(int log2cap = 10) {
        shift_ = 64 - log2cap;
        keys_.assign(size_t(1) << log2cap, 0);
        vals_.assign(size_t(1) << log2cap, 0);
        used_.assign(size_t(1) << log2cap, 0);
        size_ = 0;
    }
    size_t size() const { return size_; }
    // empty, with room for n keys without growing
    void reserve_empty(size_t n) {
        int lg = 10;
        while ((size_t(1) << lg) < 2 * n + 2) ++lg;
        reset(lg);
    }

    // the value of `key`, inserted as 0 when absent
    int64_t& at(uint64_t key) {
        size_t i = slot(key);
        while (used_[i]) {
            if (keys_[i] == key) return vals_[i];
            i = (i + 1) & (keys_.size() - 1);
        }
        if (2 * (size_ + 1) > keys_.size()) {
            grow();
            return at(key);
        }
        used_[i] = 1;
        keys_[i] = key;
        vals_[i] = 0;
        ++size_;
        return vals_[i];
    }
    // the value of `key`, or `absent`
    int64_t get(uint64_t key, int64_t absent) const {
        size_t i = slot(key);
        while (used_[i]) {
            if (keys_[i] == key) return vals_[i];
            i = (i + 1) & (keys_.size() - 1);
        }
        return absent;
    }
    template <class F>
    void for_each(F&& f) const {
        for (size_t i = 0; i < keys_.size(); ++i)
            if (used_[i]) f(keys_[i], vals_[i]);
    }

private:
    size_t slot(uint64_t key) const { return size_t((key * 0x9E3779B97F4A7C15ull) >> shift_); }
    void grow() {
        std::vector<uint64_t> k = std::move(keys_);
        std::vector<int64_t> v = std::move(vals_);
        std::vector<uint8_t> u = std::move(used_);
        reset(64 - shift_ + 1);
        for (size_t i = 0; i < k.size(); ++i)
            if (u[i]) at(k[i]) = v[i];
    }
    int shift_ = 54;
    size_t size_ = 0;
    std::vector<uint64_t> keys_;
    std::vector<int64_t> vals_;
    std::vector<uint8_t> used_;
};

// How often each bit pattern occurs in val, counted in parallel.  With
// limit > 0 the count stops once more than `limit` distinct patterns are
// seen (then *over is set and *out is incomplete).  *nan is set when a NaN
// occurs.
inline void count_values(const std::vector<double>& val, size_t limit, BitsTable* out, bool* over, bool* nan) {
    const int64_t n = int64_t(val.size());
    const int parts = parallel_parts(n, 1 << 20);
    std::vector<BitsTable> part(parts);
    std::atomic<bool> stop{false}, any_nan{false};
    parallel_ranges(n, 1 << 20, [&](int64_t a, int64_t b, int t) {
        BitsTable& tab = part[t];
        uint64_t last = 0;
        int64_t* lastv = nullptr;
        for (int64_t k = a; k < b; ++k) {
            const double v = val[k];
            if (v != v) { any_nan = true; stop = true; return; }
            const uint64_t key = value_bits(v);
            if (lastv && key == last) { ++*lastv; continue; }
            lastv = &tab.at(key);
            ++*lastv;
            last = key;
            if (limit && tab.size() > limit) { stop = true; return; }
            if (((k - a) & 0xFFFF) == 0 && stop.load(std::memory_order_relaxed)) return;
        }
    });
    *nan = any_nan;
    *over = stop && !any_nan;
    // sized up front: keys taken from a table come in its slot order, which
    // would pile up into long probe runs in a smaller table
    size_t total = 0;
    for (const auto& p : part) total += p.size();
    out->reserve_empty(total);
    for (int t = 0; t < parts && !*over && !*nan; ++t) {
        part[t].for_each([&](uint64_t k, int64_t c) { out->at(k) += c; });
        if (limit && out->size() > limit) *over = true;
    }
}

}  // namespace spmvc
